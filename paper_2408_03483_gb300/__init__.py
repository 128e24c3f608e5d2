"""GB300-native tensor-train finite-volume shallow-water stage.

The hot path (arXiv 2408.03483, Sec. 4) runs in libttfv.so (hand-written
sm_103a CUDA behind the C ABI of include/tt_fv.h); ``api`` marshals PyTorch
device memory and streams to it.
"""
__all__ = ["api", "capi", "build"]

import os as _os

# The solver's stage graph runs up to 16 CUDA streams at once; CUDA's default
# of 8 hardware work queues would make kernels of unrelated streams wait for
# each other.  CUDA reads the variable when the process creates its context,
# so this takes effect only if the package is imported before the device is
# first used (bench.py and the tests set it themselves).
_os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
