"""GB300 (sm_103a) implementation of the cylindrical (m=0) laser-envelope PIC timestep of
Massimo et al., arXiv:1912.04674, behind the C ABI of ``include/lpic.h``."""
from .lpic import (Grid, Laser, LpicError, Plasma, Simulation, lib)  # noqa: F401
