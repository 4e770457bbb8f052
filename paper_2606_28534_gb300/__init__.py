"""GB300-native (sm_103a) 1D3V electrostatic PIC Monte Carlo step (BIT1 cycle, arXiv 2606.28534).

The compute path is the CUDA library ``libpicgb.so`` behind the C ABI of ``include/pic.h``;
``pic`` is its thin ctypes binding (the library is loaded on first use) and ``workloads`` holds
the seeded synthetic configurations.
"""
from . import pic, workloads  # noqa: F401
from .pic import Simulation, philox, poisson  # noqa: F401
