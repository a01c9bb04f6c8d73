"""GB300-native FFT pressure-projection path of FluTAS (arXiv 2204.08834, Sec. 3.3).

The compute path is libflups.so (include/flups.h), hand-written CUDA for sm_103a;
`flups` is its ctypes binding and `synth` the seeded synthetic-input generators.
"""

from . import synth  # noqa: F401
