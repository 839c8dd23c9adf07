"""libpartition: in-place parallel partition (Smoothed Striding, Strided and
Blocked-Prefix-Sum variants), quicksort, batched and served partitions on one
GB300 GPU (sm_103a).  Kuszmaul & Westover, arXiv 2004.12532.

The compute path is the CUDA library libpartition.so behind the C ABI in
include/libpartition.h; `paper_2004_12532_gb300.binding` is a thin ctypes
binding with the same names.  Importing this package does not load the
library; the first call into the binding does, and fails loudly if it is
missing.
"""
__all__ = ["binding", "inputs"]
