// Adjoint shape gradients (placeholder until the adjoint kernels land).
#include "batch.h"

namespace pfq4 {

pf_status shape_gradient(Batch& b, int obj, int lo, int hi, double U, double tol, double* dev_dJdX, double* dJdc,
                         double* J) {
  (void)b; (void)obj; (void)lo; (void)hi; (void)U; (void)tol; (void)dev_dJdX; (void)dJdc; (void)J;
  throw Error{PF_EINVAL, "pf_grad: not available in this build"};
}

}  // namespace pfq4
