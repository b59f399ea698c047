"""GB300-native eager sparse BM25 scoring (BM25S, arXiv 2407.03618).

The index build and batched top-k retrieval run as hand-written sm_103a CUDA
kernels in libbm25gpu.so behind the C ABI of include/bm25.h; ``bm25`` is its
Python binding and ``synth`` the seeded synthetic corpora used by the tests
and the benchmark.
"""
from . import build_ext, synth  # noqa: F401
from .bm25 import (ACC_AUTO, ACC_L2_DENSE, ACC_SMEM_TILED, ACC_UNSET, MAX_K, VARIANTS,  # noqa: F401
                   BM25Error, Index, Plan, Server, Workspace, launch_count, load)

__all__ = ["Index", "Plan", "Server", "Workspace", "ACC_UNSET", "BM25Error", "VARIANTS", "MAX_K", "ACC_AUTO", "ACC_SMEM_TILED",
           "ACC_L2_DENSE", "load", "launch_count", "synth", "build_ext"]
