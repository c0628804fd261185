"""B300-native (sm_103a) weighted-upwind vector kinetic lattice Boltzmann method.

The compute path is the CUDA library ``libvklb.so`` (C ABI declared in
``include/vklb.h``); ``paper_2608_04283_b300.vklb`` is its thin ctypes binding.
Importing this package loads nothing; ``paper_2608_04283_b300.vklb`` raises if the
library has not been built.
"""
__all__ = ["vklb", "inputs"]
