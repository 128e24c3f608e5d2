"""GB300-native tensor-train finite-volume shallow-water stage.

The hot path (arXiv 2408.03483, Sec. 4) runs in libttfv.so (hand-written
sm_103a CUDA behind the C ABI of include/tt_fv.h); ``api`` marshals PyTorch
device memory and streams to it.
"""
__all__ = ["api", "capi", "build"]
