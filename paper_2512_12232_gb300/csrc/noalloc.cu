// Allocation-free form of the operator apply (pf_apply_noalloc).
//
// Some callers cannot allocate device memory at the moment they need the operator:
// code that runs inside a framework owning all device memory through its own arena
// or caching allocator, or a latency-critical loop that must not call cudaMalloc /
// cudaFree (they synchronise the device and can fail under memory pressure).  This
// entry point allocates nothing.  It reads the caller's logical input vector and
// writes the caller's logical output vector directly, and keeps its only scratch -
// the collapsed body rows - in a file-scope device array of fixed size that every
// GPU loading this library holds until the process exits.
//
// The scratch array is shared by every call on a device and keeps the last call's
// contents; each call overwrites every slot it reads back, so nothing needs clearing
// between calls.  Calls whose work overlaps on the GPU (for example on two streams at
// once) race on that array.  The call runs on the stream it is given and never touches
// the handle's own state, so a const handle stays unchanged.
#include <mutex>

#include "batch.h"

namespace pfq4 {

constexpr int NOALLOC_MAX_BODIES = PF_NOALLOC_MAX_BODIES;

// Collapsed body rows of the last pf_apply_noalloc call on this device.
static __device__ __align__(256) double g_apply_noalloc_scratch[NOALLOC_MAX_BODIES];

namespace {

std::mutex g_setup_mutex;
constexpr int MAX_DEVICES = 64;
double* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array for the current device, looked up on the first
// call made with that device current and kept for the life of the process (a
// cudaDeviceReset reloads the module, so the library is not used across one).
double* scratch_for_current_device() {
  int dev = -1;
  PF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) throw Error{PF_EINVAL, "device ordinal out of range"};
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_apply_noalloc_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error{PF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)};
    }
    g_scratch_ptr[dev] = (double*)p;
  }
  return g_scratch_ptr[dev];
}

__device__ __forceinline__ long long logical_base(const DevVariant* var, int v) {
  long long s = 0;
  for (int u = 0; u < v; ++u) s += (long long)(var[u].nx + 1) * (var[u].ny + 1);
  return s;
}

// One tile per CTA: y = A p with p read from, and y written to, logical arrays.
template <typename T>
__global__ void __launch_bounds__(NT) k_apply_logical(MeshDev m, const int* tile_var, const int2* tile_ij,
                                                      const double* __restrict__ p, double* __restrict__ y) {
  __shared__ T ps[TY + 2][SW];
  __shared__ uint8_t ts[TY + 2][SW];
  __shared__ long long s_lb;
  const long long t = blockIdx.x;
  const int v = tile_var[t];
  const DevVariant& V = m.var[v];
  const int tid = linear_tid();
  if (tid == 0) s_lb = logical_base(m.var, v);
  __syncthreads();
  const long long lb = s_lb;
  const long long row = V.nx + 1;
  const int2 ij = tile_ij[t];
  const int i = ij.x + threadIdx.x, j = ij.y + threadIdx.y;
  const bool in = (i <= V.nx) && (j <= V.ny);
  const long long n = V.base + (long long)j * V.P + i;
  const uint8_t tg = in ? m.tag[n] : K_INACT;
  ps[threadIdx.y + 1][threadIdx.x + 1] = in ? (T)p[lb + j * row + i] : T(0);
  ts[threadIdx.y + 1][threadIdx.x + 1] = tg;
  if (tid < NHALO) {
    int li, lj;
    halo_pos(tid, li, lj);
    const int hi = ij.x - 1 + li, hj = ij.y - 1 + lj;
    uint8_t ht = K_INACT;
    T hp = T(0);
    if (hi >= 0 && hj >= 0 && hi <= V.nx && hj <= V.ny) {
      ht = m.tag[V.base + (long long)hj * V.P + hi];
      hp = (T)p[lb + hj * row + hi];
    }
    ps[lj][li] = hp;
    ts[lj][li] = ht;
  }
  __syncthreads();
  if (!in) return;
  const int kind = tg & KIND_MASK;
  T out = T(0);
  if (kind == K_FREE || kind == K_BODY) {
    const T* K = sizeof(T) == 8 ? (const T*)m.K64 : (const T*)m.K32;
    const T* kr = sizeof(T) == 8 ? (const T*)V.kr64 : (const T*)V.kr32;
    out = q4_row<T>(ps, ts, threadIdx.x + 1, threadIdx.y + 1, n, V.P, K, m.Vtot, kr);
  }
  y[lb + j * row + i] = (double)out;
}

// Collapsed body rows: one CTA per global body, fixed-order sum of y (logical) over
// the body's nodes, written to the scratch array.
__global__ void __launch_bounds__(NT) k_body_rows_logical(MeshDev m, const int* body_var, const double* y,
                                                          double* sums) {
  __shared__ double scratch[NT / 32 + 1];
  __shared__ long long s_lb;
  const int gb = blockIdx.x;
  const int v = body_var[gb];
  const DevVariant& V = m.var[v];
  if (linear_tid() == 0) s_lb = logical_base(m.var, v);
  __syncthreads();
  const long long lb = s_lb;
  double s = 0.0;
  const int e1 = m.body_ptr[gb + 1];
  for (int e = m.body_ptr[gb] + linear_tid(); e < e1; e += NT) {
    const long long rem = m.body_nodes[e] - V.base;
    const long long i = rem % V.P, j = rem / V.P;
    s += y[lb + j * (V.nx + 1) + i];
  }
  s = block_sum(s, scratch);
  if (linear_tid() == 0) sums[gb] = s;
}

}  // namespace

// Same operator and outputs as apply_operator, without any device allocation, on
// stream s; reads the handle only.
void apply_operator_noalloc(const Batch& b, int precision, const double* dev_p, double* dev_y, double* body_sums,
                            cudaStream_t s) {
  if (b.B > NOALLOC_MAX_BODIES)
    throw Error{PF_EINVAL, "pf_apply_noalloc: the handle has " + std::to_string(b.B) +
                               " bodies; the allocation-free scratch holds at most " +
                               std::to_string(NOALLOC_MAX_BODIES)};
  double* sums = scratch_for_current_device();
  MeshDev m;
  m.var = b.d_var;
  m.tag = b.tag;
  m.bid = b.bid;
  m.body_ptr = b.body_ptr;
  m.body_nodes = b.body_nodes;
  m.K64 = b.K64;
  m.K32 = b.K32;
  m.Vtot = b.Vtot;
  const dim3 blk(TX, TY);
  if (precision == PF_FP64)
    k_apply_logical<double><<<(unsigned)b.T, blk, 0, s>>>(m, b.tile_var, b.tile_ij, dev_p, dev_y);
  else
    k_apply_logical<float><<<(unsigned)b.T, blk, 0, s>>>(m, b.tile_var, b.tile_ij, dev_p, dev_y);
  PF_CUDA(cudaGetLastError());
  if (b.B > 0) {
    k_body_rows_logical<<<b.B, blk, 0, s>>>(m, b.d_body_var, dev_y, sums);
    PF_CUDA(cudaGetLastError());
    if (body_sums) PF_CUDA(cudaMemcpyAsync(body_sums, sums, b.B * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  PF_CUDA(cudaStreamSynchronize(s));
}

}  // namespace pfq4

using namespace pfq4;

extern "C" pf_status pf_apply_noalloc(const pf_batch* h, int precision, const double* dev_p, double* dev_y,
                                      double* body_sums, void* stream) {
  try {
    const Batch* b = (const Batch*)h;
    if (!b) throw Error{PF_EINVAL, "NULL handle"};
    int dev = -1;
    PF_CUDA(cudaGetDevice(&dev));
    if (dev != b->device) throw Error{PF_EINVAL, "call made with another device current than the handle's"};
    if (!dev_p || !dev_y) throw Error{PF_EINVAL, "NULL vector"};
    if (precision != PF_FP64 && precision != PF_MIXED) throw Error{PF_EINVAL, "invalid precision"};
    // the call ends by synchronising its stream, which a capturing stream does not allow
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    PF_CUDA(cudaStreamIsCapturing((cudaStream_t)stream, &cap));
    if (cap != cudaStreamCaptureStatusNone) throw Error{PF_EINVAL, "the stream is capturing"};
    apply_operator_noalloc(*b, precision, dev_p, dev_y, body_sums, (cudaStream_t)stream);
    return PF_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return PF_EINVAL;
  }
}
