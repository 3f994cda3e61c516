"""B300-native TPC track finding and refit (arXiv:1811.11481 hot path).

The compute path is libtpc.so (CUDA, sm_103a) behind the C ABI in
include/tpc.h; ``binding`` marshals arguments to it with ctypes and uses
torch only for device memory and streams. ``autograd`` exposes the refit and
its adjoint as a torch.autograd.Function.
"""
from .config import DEFAULT_PARAMS, default_params  # noqa: F401


def __getattr__(name):
    if name in ("Tracker", "load_library", "TpcError", "declared_functions"):
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)
