"""Python front end of the FP64 oracle (``rom_oracle.c``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It is independent
of the CUDA library: it neither imports the package's binding nor links any
of its code.

All arrays are logical numpy arrays: ``Avs`` (Kv, Ks), ``Asv`` (Ks, Kv),
``C`` (R, Kv), states ``V`` (Kv, M) and ``S`` (Ks, M), forcing tables
(nsteps, M), trace records (nrec, R, M).  They are widened to float64 and
handed to C in column-major order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rom_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "fom_oracle.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP over realizations,
    no FMA contraction so every product and sum rounds on its own)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", *_SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_forward.restype = ctypes.c_int
            lib.orc_forward.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_long,
                                        ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp]
            lib.orc_inverse.restype = ctypes.c_int
            lib.orc_inverse.argtypes = [_dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, _dp, _dp, _dp, _dp, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_long, ctypes.c_int, ctypes.c_int,
                                        _dp, _dp]
            lib.orc_energy.restype = ctypes.c_double
            lib.orc_energy.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       _dp, _dp, ctypes.c_int]
            lib.orc_spectral_radius.restype = ctypes.c_int
            lib.orc_spectral_radius.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_double, _dp]
            lib.orc_adjoint.restype = ctypes.c_int
            lib.orc_adjoint.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_double, _dp, _dp, _dp,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_long, _dp,
                                        _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                        _dp, _dp]
            lib.orc_ricker.restype = None
            lib.orc_ricker.argtypes = [_dp, _dp, ctypes.c_int, _dp, _dp]
            lib.orc_wavelet.restype = None
            lib.orc_wavelet.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, _dp]
            lib.orc_max_threads.restype = ctypes.c_int
            _ip = ctypes.POINTER(ctypes.c_int)
            lib.orc_fom_dims.restype = None
            lib.orc_fom_dims.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _ip, _ip]
            lib.orc_fom_forward.restype = ctypes.c_int
            lib.orc_fom_forward.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, _dp, _dp, _dp, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_long, ctypes.c_int, _dp, _dp,
                                            ctypes.c_int, ctypes.c_int, _ip, ctypes.c_int, _dp,
                                            ctypes.c_int]
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().orc_max_threads())


def _cm(a) -> np.ndarray:
    """float64 column-major copy (Fortran order) of a logical 2-D array."""
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _check(rc: int, what: str):
    if rc < 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def wavelet(kind, t, T):
    """Source signal of `kind` (0 Ricker, 1 first derivative of a Gaussian,
    Sec. 3.2) and its T-derivative, elementwise (float64)."""
    t = np.asarray(t, np.float64)
    T = np.asarray(T, np.float64)
    shape = np.broadcast(t, T).shape
    tb = np.ascontiguousarray(np.broadcast_to(t, shape)).ravel()
    Tb = np.ascontiguousarray(np.broadcast_to(T, shape)).ravel()
    f = np.empty_like(tb)
    d = np.empty_like(tb)
    _load().orc_wavelet(int(kind), _ptr(tb), _ptr(Tb), tb.size, _ptr(f), _ptr(d))
    return f.reshape(shape), d.reshape(shape)


def ricker(t, T):
    """Ricker wavelet f(t; T) and its T-derivative, elementwise (float64)."""
    t = np.asarray(t, np.float64)
    T = np.asarray(T, np.float64)
    shape = np.broadcast(t, T).shape
    tb = np.ascontiguousarray(np.broadcast_to(t, shape)).ravel()
    Tb = np.ascontiguousarray(np.broadcast_to(T, shape)).ravel()
    f = np.empty_like(tb)
    d = np.empty_like(tb)
    _load().orc_ricker(_ptr(tb), _ptr(Tb), tb.size, _ptr(f), _ptr(d))
    return f.reshape(shape), d.reshape(shape)


def _xref(xref, Kv, Ks, M):
    """The reduced reference state (Eq. (rom_ode_tensor)) as two column-major
    FP64 blocks (Kv x M, Ks x M); None drops the term."""
    if xref is None:
        return None, None
    Xv, Xs = xref
    Xv = None if Xv is None else _cm(Xv)
    Xs = None if Xs is None else _cm(Xs)
    assert Xv is None or Xv.shape == (Kv, M)
    assert Xs is None or Xs.shape == (Ks, M)
    return Xv, Xs


def forward(Avs, Asv, g, C, dt, V0, S0, nsteps, T=None, ftab=None, n0=0, r=0,
            threads=0, wavelet=0, xref=None):
    """Leapfrog forward run.  Returns (V, S, traces) as float64 arrays;
    traces is (nsteps // r, R, M) or None when r == 0 or C has no rows.
    `wavelet` selects the source signal of the periods T (0 Ricker, 1 first
    derivative of a Gaussian).  `xref` = (Xv, Xs) adds the reduced reference
    state (Kv x M, Ks x M; either may be None) to the two halves of every
    step."""
    Avs = _cm(Avs)
    Asv = _cm(Asv)
    Kv, Ks = Avs.shape
    g = np.ascontiguousarray(np.asarray(g, np.float64))
    Cm = _cm(C) if C is not None else np.zeros((0, Kv), order="F")
    R = Cm.shape[0]
    V = _cm(V0).copy(order="F")
    S = _cm(S0).copy(order="F")
    M = V.shape[1]
    assert V.shape == (Kv, M) and S.shape == (Ks, M)
    Tc = None if T is None else np.ascontiguousarray(np.asarray(T, np.float64))
    Fc = None if ftab is None else np.ascontiguousarray(np.asarray(ftab, np.float64))
    if Fc is not None:
        assert Fc.shape == (nsteps, M)
    nrec = nsteps // r if (r > 0 and R > 0) else 0
    Xv, Xs = _xref(xref, Kv, Ks, M)
    # records are [rec][m][j] in C: allocate (nrec, M, R) C-order
    tr = np.zeros((nrec, M, R), np.float64) if nrec > 0 else None
    rc = _load().orc_forward(_ptr(Avs), _ptr(Asv), _ptr(g), _ptr(Cm) if R > 0 else None,
                             Kv, Ks, R, float(dt), _ptr(V), _ptr(S), _ptr(Tc), _ptr(Fc),
                             M, int(nsteps), int(n0), int(r) if nrec > 0 else 0,
                             _ptr(tr), int(threads), int(wavelet), _ptr(Xv), _ptr(Xs))
    _check(rc, "forward")
    traces = None if tr is None else np.ascontiguousarray(tr.transpose(0, 2, 1))
    return np.ascontiguousarray(V), np.ascontiguousarray(S), traces


def inverse(Avs, Asv, g, dt, V, S, nsteps, T=None, ftab=None, n0=0, threads=0, wavelet=0,
            xref=None):
    """Undo ``nsteps`` leapfrog steps (time reversal).  Returns (V0, S0)."""
    Avs = _cm(Avs)
    Asv = _cm(Asv)
    Kv, Ks = Avs.shape
    g = np.ascontiguousarray(np.asarray(g, np.float64))
    V = _cm(V).copy(order="F")
    S = _cm(S).copy(order="F")
    M = V.shape[1]
    Tc = None if T is None else np.ascontiguousarray(np.asarray(T, np.float64))
    Fc = None if ftab is None else np.ascontiguousarray(np.asarray(ftab, np.float64))
    Xv, Xs = _xref(xref, Kv, Ks, M)
    rc = _load().orc_inverse(_ptr(Avs), _ptr(Asv), _ptr(g), Kv, Ks, float(dt), _ptr(V),
                             _ptr(S), _ptr(Tc), _ptr(Fc), M, int(nsteps), int(n0),
                             int(threads), int(wavelet), _ptr(Xv), _ptr(Xs))
    _check(rc, "inverse")
    return np.ascontiguousarray(V), np.ascontiguousarray(S)


def energy(Asv, dt, V, S) -> float:
    """Discrete leapfrog energy ||V||^2 + ||S||^2 - dt <S, Asv V> (skew case)."""
    Asv = _cm(Asv)
    Ks, Kv = Asv.shape
    V = _cm(V)
    S = _cm(S)
    return float(_load().orc_energy(_ptr(Asv), Kv, Ks, float(dt), _ptr(V), _ptr(S),
                                    V.shape[1]))


def spectral_radius(Avs, Asv, max_iter=5000, tol=1e-13):
    """rho([[0, Avs], [Asv, 0]]) by FP64 power iteration on Avs Asv.
    Returns (rho, iterations)."""
    Avs = _cm(Avs)
    Asv = _cm(Asv)
    Kv, Ks = Avs.shape
    out = ctypes.c_double(0.0)
    it = _load().orc_spectral_radius(_ptr(Avs), _ptr(Asv), Kv, Ks, int(max_iter),
                                     float(tol), ctypes.byref(out))
    _check(it, "spectral_radius")
    return float(out.value), int(it)


def adjoint(Avs, Asv, g, C, dt, V0, S0, T, nsteps, ystar, n0=0, threads=0, wavelet=0,
            xref=None):
    """Loss and gradients of sum_n sum_m ||C V_m^n - ystar_m^n||^2.
    ystar is (nsteps, R, M).  Returns (loss, gV0, gS0, gT).  `xref` as in
    forward (it shifts the forward sweep only)."""
    Avs = _cm(Avs)
    Asv = _cm(Asv)
    Kv, Ks = Avs.shape
    g = np.ascontiguousarray(np.asarray(g, np.float64))
    Cm = _cm(C)
    R = Cm.shape[0]
    V0 = _cm(V0)
    S0 = _cm(S0)
    M = V0.shape[1]
    Tc = np.ascontiguousarray(np.asarray(T, np.float64))
    ys = np.ascontiguousarray(np.asarray(ystar, np.float64).transpose(0, 2, 1))  # (n, M, R)
    assert ys.shape == (nsteps, M, R)
    gV = np.zeros((Kv, M), order="F")
    gS = np.zeros((Ks, M), order="F")
    gT = np.zeros(M)
    loss = ctypes.c_double(0.0)
    Xv, Xs = _xref(xref, Kv, Ks, M)
    rc = _load().orc_adjoint(_ptr(Avs), _ptr(Asv), _ptr(g), _ptr(Cm), Kv, Ks, R,
                             float(dt), _ptr(V0), _ptr(S0), _ptr(Tc), M, int(nsteps),
                             int(n0), _ptr(ys), _ptr(gV), _ptr(gS), _ptr(gT),
                             ctypes.byref(loss), int(threads), int(wavelet),
                             _ptr(Xv), _ptr(Xs))
    _check(rc, "adjoint")
    return float(loss.value), np.ascontiguousarray(gV), np.ascontiguousarray(gS), gT


def problem_forward(p, V0=None, S0=None, nsteps=None, r=None, n0=0, T=None,
                    threads=0, columns=None, wavelet=0):
    """Convenience: run a ``RomProblem``-like object (fields Avs, Asv, g, C, dt, T).
    ``columns`` restricts the run to a subset of realizations (columns are
    independent, so a subset gives exactly those columns of the full run)."""
    Kv, Ks = p.Avs.shape
    Tm = np.asarray(p.T if T is None else T, np.float64)
    M = Tm.shape[0]
    if V0 is None:
        V0 = np.zeros((Kv, M))
    if S0 is None:
        S0 = np.zeros((Ks, M))
    V0 = np.asarray(V0, np.float64)
    S0 = np.asarray(S0, np.float64)
    if columns is not None:
        columns = np.asarray(columns)
        Tm = Tm[columns]
        V0 = V0[:, columns]
        S0 = S0[:, columns]
    steps = p.meta.get("steps") if nsteps is None else nsteps
    rr = p.meta.get("r", 0) if r is None else r
    return forward(p.Avs, p.Asv, p.g, p.C if p.C.shape[0] > 0 else None, p.dt, V0, S0,
                   steps, T=Tm, n0=n0, r=rr, threads=threads, wavelet=wavelet)


def trace_stats(traces, probs):
    """Ensemble statistics of receiver traces (Sec. 4.5.2: mean and
    percentile bands of the seismograms over the realizations).
    traces: (nrec, M, R) array (record, realization, receiver).  Returns
    (mean (nrec, R), q (len(probs), nrec, R)) in float64: the mean over the
    realizations, and for each p the quantile by linear interpolation between
    order statistics (Hyndman-Fan type 7): h = (M - 1) p, i = floor(h),
    t = h - i, q = x(i) + t (x(i+1) - x(i)), written as b - (1 - t)(b - a)
    for t >= 1/2 (a = x(i), b = x(i+1))."""
    x = np.asarray(traces, np.float64)
    nrec, M, R = x.shape
    mean = x.mean(axis=1)
    xs = np.sort(x, axis=1)
    q = np.zeros((len(probs), nrec, R))
    for n, p in enumerate(probs):
        h = (M - 1) * float(p)
        i = min(int(np.floor(h)), M - 1)
        t = h - i
        a = xs[:, i, :]
        b = xs[:, min(i + 1, M - 1), :]
        d = b - a
        q[n] = b - d * (1.0 - t) if t >= 0.5 else a + d * t
    return mean, q


# ------------------------------------------------------------------ FOM --
# The full-order shear-wave model of Sec. 3 (fom_oracle.c): staggered grid of
# Nr x Nt intervals on r_cmb <= r <= r_earth, 0 <= theta <= pi.

FOM_APP_A = {"rho": 2500.0, "vs": 5000.0, "r_cmb": 3480e3, "r_earth": 6371e3,
             "dt": 0.05, "src_depth": 640e3}
"""The homogeneous single-layer setup of App. A in SI units (rho in kg/m^3:
the paper's "g/cm^3" is read as a unit slip), dt in s, lengths in m."""


def fom_dims(Nr, Nt):
    """(nv, n1, n2): velocity, sigma_rp and sigma_tp unknowns of the grid."""
    a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _load().orc_fom_dims(int(Nr), int(Nt), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


def fom_forward(Nr, Nt, V0, S10, S20, nsteps, src=-1, T=None, ftab=None, wavelet=1, n0=0,
                recv=None, r=0, rho=2500.0, vs=5000.0, dt=0.05, r_cmb=3480e3,
                r_earth=6371e3, threads=0):
    """Leapfrog run of the FOM, one realization at a time.  V0 (nv, M),
    S10 (n1, M), S20 (n2, M); src: velocity unknown of the point source (-1:
    none); T (M) periods or ftab (nsteps, M); recv: velocity unknowns
    recorded every r steps.  Returns (V, S1, S2, traces (nrec, nrecv, M) or None)."""
    nv, n1, n2 = fom_dims(Nr, Nt)
    V = _cm(V0).copy(order="F")
    S1 = _cm(S10).copy(order="F")
    S2 = _cm(S20).copy(order="F")
    M = V.shape[1]
    assert V.shape == (nv, M) and S1.shape == (n1, M) and S2.shape == (n2, M)
    Tc = None if T is None else np.ascontiguousarray(np.asarray(T, np.float64))
    Fc = None if ftab is None else np.ascontiguousarray(np.asarray(ftab, np.float64))
    rc = None if recv is None else np.ascontiguousarray(np.asarray(recv, np.int32))
    nrecv = 0 if rc is None else rc.size
    nrec = nsteps // r if (r > 0 and nrecv > 0) else 0
    tr = np.zeros((nrec, M, nrecv), np.float64) if nrec > 0 else None
    ip = None if rc is None else rc.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    ret = _load().orc_fom_forward(int(Nr), int(Nt), float(r_cmb), float(r_earth), float(rho),
                                  float(vs), float(dt), _ptr(V), _ptr(S1), _ptr(S2), M,
                                  int(nsteps), int(n0), int(src), _ptr(Tc), _ptr(Fc),
                                  int(wavelet), nrecv, ip, int(r) if nrec > 0 else 0, _ptr(tr),
                                  int(threads))
    _check(ret, "fom_forward")
    traces = None if tr is None else np.ascontiguousarray(tr.transpose(0, 2, 1))
    return np.ascontiguousarray(V), np.ascontiguousarray(S1), np.ascontiguousarray(S2), traces
