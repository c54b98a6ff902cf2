"""B300-native line radiative-transfer march (arXiv 2509.03623, RadJAX hot path).

The compute path is the CUDA library `librt_b300.so` (C ABI in `include/rt.h`); this
package holds its ctypes binding and the seeded input generators.
"""

from . import synth  # noqa: F401
from ._rt import DeviceDisk, RTError, rt_count_gas_samples, rt_render, version  # noqa: F401
