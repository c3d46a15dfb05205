"""GB300 (sm_103a) implementation of the fragment kinetic Monte Carlo hot path
of H. Nakata, arXiv:2004.09081: windowed, checkerboard-coloured spatial
fragments each running rejection-free BKL (Sec. II), for O-vacancy and H-
diffusion on the perovskite O sublattice.  The compute path is the CUDA
library behind the C ABI in include/fkmc.h; this package is its binding."""
from .fkmc import (FKMC_H, FKMC_MIXED, FKMC_O, FKMC_PLAIN, FKMC_V, Batch, KmcError,  # noqa: F401
                   load)

__all__ = ["Batch", "KmcError", "load", "FKMC_O", "FKMC_H", "FKMC_V", "FKMC_PLAIN", "FKMC_MIXED"]
