"""GB300 (sm_103a) implementation of the 3D central-moment lattice Boltzmann
method with forcing (Premnath & Banerjee): the fused collide-and-stream step
on D3Q27 and D3Q15 behind the C ABI of include/lbm.h, built into
``liblbm.so`` by ``build.build()``; ``lbm`` is its Python binding."""
from .build import build  # noqa: F401
