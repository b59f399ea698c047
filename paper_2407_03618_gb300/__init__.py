"""GB300-native eager sparse BM25 scoring (BM25S, arXiv 2407.03618).

The index build and batched top-k retrieval run as hand-written sm_103a CUDA
kernels in libbm25gpu.so behind the C ABI of include/bm25.h; ``bm25`` is its
Python binding and ``synth`` the seeded synthetic corpora used by the tests
and the benchmark.
"""
from . import build_ext, synth  # noqa: F401
from .bm25 import (ACC_AUTO, ACC_L2_DENSE, ACC_SMEM_TILED, MAX_K, VARIANTS, BM25Error,  # noqa: F401
                   Index, Plan, Workspace, launch_count, load)

__all__ = ["Index", "Plan", "Workspace", "BM25Error", "VARIANTS", "MAX_K", "ACC_AUTO", "ACC_SMEM_TILED",
           "ACC_L2_DENSE", "load", "launch_count", "synth", "build_ext"]
