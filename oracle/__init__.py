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
The full-order model (fom_oracle.c, Sec. 3): exact fixed points of the
stencils (rigid rotation, hoop stress), exact discrete-energy invariance
under the weights that make the flux-form operator skew-adjoint, the
radial travel time at the shear speed, superposition.
"""
from .oracle import (FOM_APP_A, adjoint, build, energy, fom_dims, fom_forward, forward,
                     inverse, max_threads, problem_forward, ricker, spectral_radius,
                     trace_stats, wavelet)

__all__ = ["FOM_APP_A", "adjoint", "build", "energy", "fom_dims", "fom_forward", "forward",
           "inverse", "max_threads", "problem_forward", "ricker", "spectral_radius",
           "trace_stats", "wavelet"]
