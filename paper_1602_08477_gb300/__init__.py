"""GB300-native FP64 GEMM library on the grid / block / thread / element work
division of Alpaka (arXiv 1602.08477).

The computation lives in libgbgemm.so (hand-written CUDA for sm_103a, C ABI in
include/gb_gemm.h); this package only builds it and marshals torch tensors and
streams into its calls.  Importing the package does not load the library;
the first call does, and raises if it is not built.
"""
from ._lib import GbError, Workdiv, load  # noqa: F401
from .gemm import (  # noqa: F401
    Device,
    Queue,
    alloc_workspace,
    default_queue,
    dgemm,
    dgemm_host,
    emulated_layout,
    host_schedule,
    host_workspace_size,
    emulated_crt_steps,
    emulated_steps,
    workdiv_suggest,
    workspace_size,
)


def build(verbose: bool = False) -> str:
    from .compile_lib import build as _build
    return _build(verbose=verbose)


from .grouped import (  # noqa: E402,F401
    GroupedPlan,
    dgemm_grouped,
    tune_get,
    tune_lookup,
    tune_lookup_emulated,
    tune_lookup_slices,
    tune_set,
)
from .serve import Server, fill_uniform  # noqa: E402,F401
from .execute import daxpy, enqueue, kernel_handle  # noqa: E402,F401
from .mem import Buffer, OwnedQueue, copy, dgemm_buffers  # noqa: E402,F401
