"""Seeded synthetic inputs for the rank-2 Galerkin ROM leapfrog.

This module only *draws* inputs.  It holds none of the method's arithmetic:
no leapfrog step, no forcing evaluation, no operator products.  Both the
CUDA path and the FP64 oracle consume what it returns, so that the two sides
always see identical bytes.

Workload recipe (stands in for the random-operator ROM study of Sec. 4.2,
where the reduced operators are filled with random data, and for the
many-query Ricker-forcing study of Sec. 4.5):

* ``Asv`` (Ks x Kv) has i.i.d. N(0, 1/Kv) entries, drawn in row-major order.
* ``Avs = -Asv^T`` (the velocity/stress operators of Eq. (shwave_rom_ode_tensor)
  are negative transposes of each other for a skew-coupled wave system).
* ``g`` (Kv) is N(0,1), normalised to unit 2-norm: the row of the velocity
  basis at a point source (Sec. 2.2, sparse forcing; Sec. 3.2 source placement).
* ``C`` (R x Kv) has i.i.d. N(0, 1/Kv) entries: receiver rows of the basis
  (seismograms, Sec. 4.5.2).
* ``u_m ~ U[30, 60)`` and ``T_m = u_m * dt`` are the Ricker periods in time units,
  so one period spans 30..60 steps.
* ``dt = 0.5 / ||Asv||_2``; for the skew case this makes dt times the spectral
  radius of the coupled operator [[0, Avs], [Asv, 0]] equal to 0.5.

Draw order: Asv, g, C, u from ``numpy.random.default_rng(seed)`` (PCG64).
Every array, dt and T are rounded to float32 so that the FP32 GPU paths and
the FP64 oracle start from exactly the same values.

Array conventions: all 2-D arrays here are *logical* numpy arrays
(``A[i, k]`` is row i, column k).  The C ABI takes column-major buffers; the
binding converts.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "RomProblem",
    "make_problem",
    "random_state",
    "workload",
    "batched_problems",
    "WORKLOADS",
]


@dataclass
class RomProblem:
    """One reduced model plus its realization parameters (all float32-exact)."""

    Avs: np.ndarray  # (Kv, Ks) float32
    Asv: np.ndarray  # (Ks, Kv) float32
    g: np.ndarray  # (Kv,) float32
    C: np.ndarray  # (R, Kv) float32
    dt: float  # float32-exact python float
    T: np.ndarray  # (M,) float32 periods in time units
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def Kv(self) -> int:
        return int(self.Avs.shape[0])

    @property
    def Ks(self) -> int:
        return int(self.Avs.shape[1])

    @property
    def R(self) -> int:
        return int(self.C.shape[0])

    @property
    def M(self) -> int:
        return int(self.T.shape[0])


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def make_problem(Kv: int, Ks: int | None = None, M: int = 1, R: int = 0,
                 seed: int = 0, dt: float | None = None,
                 period_range: tuple = (30.0, 60.0)) -> RomProblem:
    """Draw one problem with the recipe in the module docstring (periods
    T_m = u_m dt with u_m uniform on `period_range`, in steps)."""
    if Ks is None:
        Ks = Kv
    rng = np.random.default_rng(seed)
    Asv = _f32(rng.standard_normal((Ks, Kv)) / np.sqrt(Kv))
    g = rng.standard_normal(Kv)
    g = _f32(g / np.linalg.norm(g))
    C = _f32(rng.standard_normal((R, Kv)) / np.sqrt(Kv))
    u = rng.uniform(period_range[0], period_range[1], M)
    Avs = np.ascontiguousarray(-Asv.T)
    if dt is None:
        dt = 0.5 / np.linalg.norm(Asv.astype(np.float64), 2)
    dt = float(np.float32(dt))
    T = _f32(u * dt)
    return RomProblem(Avs=Avs, Asv=Asv, g=g, C=C, dt=dt, T=T, seed=seed,
                      meta={"Kv": Kv, "Ks": Ks, "M": M, "R": R})


def random_state(K: int, M: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """A seeded non-zero (K, M) float32 state, for tests that need X0 != 0."""
    rng = np.random.default_rng(seed)
    return _f32(scale * rng.standard_normal((K, M)))


# The single-problem workloads 0-5 (3 is a batch).  ``steps`` and ``r``
# (trace interval) are part of the workload, not of the drawn arrays.
WORKLOADS = {
    0: dict(name="rank2-fp64-K128-M16-N1000", K=128, M=16, R=0, steps=1000,
            r=0, seed=0, prec="fp64"),
    1: dict(name="rank2-fp32-K512-M256-N10000-R64-r10", K=512, M=256, R=64,
            steps=10000, r=10, seed=0, prec="fp32"),
    2: dict(name="rank2-split-K1024-M1024-N20000-R64-r10", K=1024, M=1024, R=64,
            steps=20000, r=10, seed=0, prec="tf32x3"),
    3: dict(name="batched-64roms-K64..768-M4..256-N5000", steps=5000, r=0,
            prec="fp32", nroms=64),
    4: dict(name="adjoint-K512-M128-N4000-R64-r1-c64", K=512, M=128, R=64,
            steps=4000, r=1, seed=0, prec="fp32", ckpt=64, tstar_scale=1.05),
    # many-query UQ run shaped like the Monte Carlo study of Sec. 4.5.2:
    # K_v = 436, K_s = 417, 512 realizations of T ~ U(31, 69) (in steps),
    # 20000 steps, receiver traces every 10 steps, ensemble mean and
    # 5-95 % bands per receiver
    5: dict(name="uq-Kv436-Ks417-M512-N20000-R64-r10", Kv=436, Ks=417, M=512, R=64,
            steps=20000, r=10, seed=0, prec="fp32", period_range=(31.0, 69.0),
            probs=(0.05, 0.5, 0.95)),
}


def workload(i: int) -> RomProblem:
    """The problem of workload i (0, 1, 2, 4 or 5)."""
    c = WORKLOADS[i]
    if i == 3:
        raise ValueError("workload 3 is a batch; use batched_problems()")
    if i == 5:
        p = make_problem(c["Kv"], c["Ks"], c["M"], c["R"], seed=c["seed"],
                         period_range=c["period_range"])
        p.meta.update(c)
        return p
    p = make_problem(c["K"], c["K"], c["M"], c["R"], seed=c["seed"])
    p.meta.update(c)
    return p


def batched_sizes(nroms: int = 64, seed: int = 0, pow2_m: bool = False):
    """(K_i, M_i) of the batched workload: K_i uniform on {64, 128, ..., 768},
    M_i uniform on the integers [4, 256] (or on powers of two 4..256)."""
    rng = np.random.default_rng(seed)
    K = 64 * rng.integers(1, 13, nroms)
    if pow2_m:
        M = 2 ** rng.integers(2, 9, nroms)
    else:
        M = rng.integers(4, 257, nroms)
    return [(int(k), int(m)) for k, m in zip(K, M)]


def rank3_problems(nops: int, Kv: int, Ks: int, M: int, R: int = 0, seed: int = 0):
    """nops operators (seeds seed .. seed + nops - 1) that share one time step:
    the smallest of their own stable steps, so that every one of them is
    stable.  Each keeps its own g, C and periods."""
    first = [make_problem(Kv, Ks, M, R, seed=seed + i) for i in range(nops)]
    dt = min(p.dt for p in first)
    return [make_problem(Kv, Ks, M, R, seed=seed + i, dt=dt) for i in range(nops)]


def batched_problems(nroms: int = 64, seed: int = 0, pow2_m: bool = False):
    """The batched workload: ROM i is drawn with seed i + 1."""
    out = []
    for i, (K, M) in enumerate(batched_sizes(nroms, seed, pow2_m)):
        p = make_problem(K, K, M, 0, seed=i + 1)
        p.meta.update(name=f"rom{i}", steps=WORKLOADS[3]["steps"])
        out.append(p)
    return out
