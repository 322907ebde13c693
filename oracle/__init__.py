"""FP64 CPU oracle for the rank-2 Galerkin ROM leapfrog.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; nothing in the package may import,
call or link it.  Written from the paper (Eq. (shwave_rom_ode_tensor), the
leapfrog of Sec. 3.1, the Ricker point source of Sec. 2.2/3.2, receiver rows
of Sec. 4.5.2) and independent of the CUDA path.

Pins (tests/test_oracle_*.py): discrete-energy invariance, closed form by
eigendecomposition of the amplification matrix, the K = 1 textbook
oscillator, superposition, exact zeros, time reversal, spectral radius vs.
numpy's 2-norm, adjoint vs. finite differences and brute-force Jacobians,
ensemble statistics vs. numpy's quantile and hand-computed order statistics.
"""
from .oracle import (adjoint, build, energy, forward, inverse, max_threads,
                     problem_forward, ricker, spectral_radius, trace_stats, wavelet)

__all__ = ["adjoint", "build", "energy", "forward", "inverse", "max_threads",
           "problem_forward", "ricker", "spectral_radius", "trace_stats", "wavelet"]
