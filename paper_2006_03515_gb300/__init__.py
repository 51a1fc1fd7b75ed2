"""GB300 kernel-independent FMM for the Zheleznyak integral photoionization model.

The computation lives in libkifmm.so (CUDA, sm_103a) behind the C-ABI of
include/kifmm.h; ``kifmm`` is its thin Python binding and ``workloads`` the
seeded synthetic inputs. Importing the package does not load the library;
the first call that needs it does, and fails loudly if it is missing.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "kifmm", "build"]
