"""Compressed-matrix control step on GB300 (sm_103a).

A thin binding over the C ABI of ``libwhff.so`` (declared in include/whff.h):
every step of the path runs in the library's CUDA kernels; this package only
marshals arguments.  PyTorch supplies device memory and streams.  If the
library is missing it is built from ``csrc/`` with nvcc; if that is not
possible the import fails loudly -- there is no CPU fallback.
"""
from .whff import (  # noqa: F401
    Batch,
    Fields,
    FMT_BF16,
    FMT_FIXED_ACC,
    FMT_FIXED_BFP,
    FMT_FIXED_LIFT,
    FMT_FP8E4M3,
    FMT_FP16,
    FMT_FP32,
    FMT_ZFP,
    Graph,
    Handle,
    Server,
    WhffError,
    compressed_size,
    library,
    whff_compress,
    whff_compress_accuracy,
    whff_compress_accuracy_bands,
    whff_compress_bands,
    whff_create,
    whff_decompress,
    whff_destroy,
    whff_graph_create,
    whff_graph_create_host,
    whff_graph_create_rows,
    whff_read_probe,
    whff_step,
    whff_step_host,
    whff_step_noalloc,
    whff_step_rows,
)
