"""GB300-native genome scan of TorchGWAS (arXiv 2604.21095): Python binding of libtg.so.

The scan itself (panel preparation, genotype decode, projection, the tensor-core or FP32
contraction and the statistics epilogue) runs in the library's sm_103a CUDA kernels behind
the C ABI declared in include/tg.h; this package only marshals arguments (see _binding.py)
and builds the library (build.py).
"""
from ._binding import *  # noqa: F401,F403
from ._binding import TgError, exported_symbols, hits_to_numpy, load, make_outputs  # noqa: F401
from .build import build  # noqa: F401
