"""GB300-native (sm_103a) hot path of Dynamics-Aware Gaussian Splatting Streaming (arXiv 2411.14847).

The compute lives in the C-ABI CUDA library ``libdass.so`` (see include/dass.h); the
modules here only marshal arguments (`dass`), build the library (`build`) and draw
seeded synthetic inputs (`synth`). Nothing is loaded at import time: the library is
opened on first use and a missing library is an error, never a CPU fallback.
"""
__all__ = ["synth"]
