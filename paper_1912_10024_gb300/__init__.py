"""GB300-native electron scattering self-energy (Eq. 3 of arXiv:1912.10024).

``binding`` exposes the C-ABI library libsse (include/sse.h) through ctypes
and the ``SigmaFunction`` autograd wrapper; ``inputs`` holds the seeded
synthetic input generators. Importing the package loads nothing: the CUDA
library is built/loaded on first use of ``binding``.
"""

__all__ = ["binding", "inputs", "build"]
