"""GB300-native matrix-free Q4 stream-function solver (multi-body potential flow).

C-ABI CUDA library (include/pfq4.h, csrc/) with a thin Python binding (api.py).
`workloads` holds the seeded synthetic geometry shared by tests and benchmarks."""
from . import workloads  # noqa: F401


def __getattr__(name):
    # the binding imports torch and loads the CUDA library lazily
    if name in ("api", "autograd"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    from . import api
    if hasattr(api, name):
        return getattr(api, name)
    raise AttributeError(name)
