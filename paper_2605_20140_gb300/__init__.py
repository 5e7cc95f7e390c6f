"""GB300 (sm_103a) implementation of the SIPF-W particle-field step.

The compute path is libsipf.so (CUDA kernels behind the C ABI in
include/sipf.h); ``paper_2605_20140_gb300.sipf`` is its ctypes binding.
"""

from . import sipf  # noqa: F401  (binding only; the library loads on first use)

__all__ = ["sipf"]
