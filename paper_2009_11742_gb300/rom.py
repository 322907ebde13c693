"""ctypes binding of librom.so (C ABI in include/rom.h).

Argument marshalling only: every step of the integration runs in the CUDA
library.  If the library has not been built, every call raises; there is no
CPU fallback.

The low-level functions keep the C names (``rom_create``, ``rom_run_rank2``,
...) and take raw pointers.  ``Rom`` wraps a handle and accepts torch tensors
(device or host) or numpy arrays, checking shapes, dtypes and the
column-major layout the ABI wants:

* states are logical (K, M) tensors stored column-major, i.e. the transpose of
  a contiguous (M, K) tensor -- ``Rom.new_state`` makes one;
* trace buffers are contiguous (nrec, M, R) tensors (record k is R x M
  column-major); ``Rom.trace_view`` gives the logical (nrec, R, M) view.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librom.so")

ROM_OK, ROM_E_INVAL, ROM_E_NOMEM, ROM_E_CUDA, ROM_E_UNSTABLE, ROM_E_TIMEOUT, \
    ROM_E_NONFINITE, ROM_E_UNSUPPORTED, ROM_E_NOCONV = range(9)
ROM_FP64, ROM_FP32, ROM_TF32X3, ROM_BF16X3, ROM_BF16, ROM_BF16S, ROM_AUTO = range(7)
ROM_IN_F64, ROM_IN_F32 = 0, 1
ROM_KERNEL_AUTO, ROM_KERNEL_ONE_BLOCK, ROM_KERNEL_TWO_BLOCK, ROM_KERNEL_DATAFLOW = 0, 1, 2, 3
ROM_WAVELET_RICKER, ROM_WAVELET_GAUSS1 = 0, 1
PRECISIONS = {"fp64": ROM_FP64, "fp32": ROM_FP32, "tf32x3": ROM_TF32X3,
              "bf16x3": ROM_BF16X3, "bf16": ROM_BF16, "bf16s": ROM_BF16S, "auto": ROM_AUTO}

EXPORTED = ["rom_create", "rom_destroy", "rom_spectral_radius", "rom_sync_status",
            "rom_get_dims", "rom_set_kernel", "rom_get_plan", "rom_set_tc_columns", "rom_set_wavelet", "rom_set_reference", "rom_autotune", "rom_autotune_batched", "rom_set_batched_form", "rom_set_wait_limit",
            "rom_debug_inject_stall", "rom_run_rank2", "rom_run_rank2_ex", "rom_run_rank1",
            "rom_run_rank1_ensemble", "rom_run_batched", "rom_run_rank3", "rom_adjoint",
            "rom_adjoint_workspace_size", "rom_rel_l2", "rom_spectral_radius_noalloc",
            "rom_measure_peak", "rom_set_companion", "rom_get_companion",
            "rom_trace_stats", "rom_fom_create", "rom_fom_destroy", "rom_fom_dims", "rom_fom_run",
            "rom_fom_set_passes",
            "rom_status_string", "rom_last_error", "rom_version"]

_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_l = ctypes.c_long
_d = ctypes.c_double


class RomError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({last_error()})")


def _signatures(lib):
    sig = {
        "rom_create": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _d, _i, ctypes.POINTER(_vp),
                            ctypes.POINTER(_d)]),
        "rom_destroy": (_i, [_vp]),
        "rom_spectral_radius": (_i, [_vp, ctypes.POINTER(_d)]),
        "rom_sync_status": (_i, [_vp, ctypes.POINTER(_i)]),
        "rom_get_dims": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                              ctypes.POINTER(_d)]),
        "rom_set_kernel": (_i, [_vp, _i]),
        "rom_set_wait_limit": (_i, [_vp, ctypes.c_longlong]),
        "rom_set_tc_columns": (_i, [_vp, _i]),
        "rom_set_wavelet": (_i, [_vp, _i]),
        "rom_set_reference": (_i, [_vp, _vp, _vp, _i, _i]),
        "rom_autotune": (_i, [_vp, _i, _i, _i, ctypes.POINTER(_d), _vp]),
        "rom_autotune_batched": (_i, [_vp, _i, _i, _i, ctypes.POINTER(_d), _vp]),
        "rom_set_batched_form": (_i, [_vp, _i, _i, _i, _i]),
        "rom_debug_inject_stall": (_i, [_vp, _i]),
        "rom_get_plan": (_i, [_vp, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i),
                              ctypes.POINTER(_i), ctypes.POINTER(_i)]),
        "rom_run_rank2": (_i, [_vp, _vp, _vp, _vp, _i, _i, _l, _i, _vp, _i, _vp]),
        "rom_run_rank2_ex": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _l, _i, _vp, _i,
                                  _vp]),
        "rom_run_rank1": (_i, [_vp, _vp, _vp, _d, _i, _l, _i, _vp, _i, _vp]),
        "rom_run_rank1_ensemble": (_i, [_vp, _vp, _vp, _vp, _i, _i, _l, _i, _vp, _i, _vp]),
        "rom_run_batched": (_i, [ctypes.c_void_p, _i, _i, _i, _i, _vp]),
        "rom_run_rank3": (_i, [ctypes.c_void_p, _i, _vp, _vp, _vp, _i, _i, _i, _vp, _i, _vp]),
        "rom_adjoint": (_i, [_vp, _vp, _vp, _vp, _i, _i, _vp, _i, _vp, _vp, _vp,
                             ctypes.POINTER(_d), _vp, ctypes.c_size_t, _i, _vp]),
        "rom_adjoint_workspace_size": (ctypes.c_size_t, [_vp, _i, _i, _i, _i]),
        "rom_rel_l2": (_i, [_vp, _i, _vp, _i, ctypes.c_size_t, ctypes.POINTER(_d), _vp]),
        "rom_spectral_radius_noalloc": (_i, [_vp, _vp, _i, _i, ctypes.POINTER(_d), _vp]),
        "rom_measure_peak": (_i, [_i, ctypes.POINTER(_d), ctypes.POINTER(_d), _vp]),
        "rom_set_companion": (_i, [_vp, _i, _i]),
        "rom_get_companion": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
        "rom_trace_stats": (_i, [_vp, _i, _i, _i, ctypes.POINTER(_d), _i, _vp, _vp, _vp]),
        "rom_fom_create": (_i, [_i, _i, _d, _d, _d, _d, _d, ctypes.POINTER(_vp)]),
        "rom_fom_destroy": (_i, [_vp]),
        "rom_fom_set_passes": (_i, [_vp, _i]),
        "rom_fom_dims": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
        "rom_fom_run": (_i, [_vp, _vp, _vp, _vp, _i, _i, ctypes.c_long, _i, _vp, _i, _vp, _i, _i,
                             _vp, _i, _vp]),
        "rom_status_string": (ctypes.c_char_p, [_i]),
        "rom_last_error": (ctypes.c_char_p, []),
        "rom_version": (_i, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


def load(path: str | None = None):
    """Load librom.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    f"librom.so not found at {p}: build it with "
                    "`python -m paper_2009_11742_gb300.build` (no CPU fallback exists)")
            lib = ctypes.CDLL(p)
            _signatures(lib)
            _lib = lib
    return _lib


def status_string(s: int) -> str:
    return load().rom_status_string(int(s)).decode()


def last_error() -> str:
    return load().rom_last_error().decode()


def _chk(st: int, what: str):
    if st != ROM_OK:
        raise RomError(st, what)


# ------------------------------------------------------------ raw C calls --
def rom_create(Avs, Asv, g, C, Kv, Ks, R, dt, in_dtype):
    h = _vp()
    rho = _d(0.0)
    st = load().rom_create(Avs, Asv, g, C, Kv, Ks, R, dt, in_dtype, ctypes.byref(h),
                           ctypes.byref(rho))
    return st, h.value, rho.value


def rom_destroy(h):
    return load().rom_destroy(h)


def rom_spectral_radius(h):
    rho = _d(0.0)
    st = load().rom_spectral_radius(h, ctypes.byref(rho))
    return st, rho.value


def rom_sync_status(h):
    s = _i(0)
    st = load().rom_sync_status(h, ctypes.byref(s))
    return st, s.value


def rom_get_dims(h):
    Kv, Ks, R, dt = _i(0), _i(0), _i(0), _d(0.0)
    st = load().rom_get_dims(h, ctypes.byref(Kv), ctypes.byref(Ks), ctypes.byref(R),
                             ctypes.byref(dt))
    return st, Kv.value, Ks.value, R.value, dt.value


def rom_set_kernel(h, kernel):
    return load().rom_set_kernel(h, kernel)


def rom_set_tc_columns(h, cols):
    return load().rom_set_tc_columns(h, int(cols))


def rom_set_wavelet(h, wavelet):
    return load().rom_set_wavelet(h, int(wavelet))


def rom_set_reference(h, Xv, Xs, M, in_dtype):
    """Raw call: Xv, Xs are addresses (or None), column-major."""
    return load().rom_set_reference(h, Xv, Xs, int(M), int(in_dtype))


def rom_autotune(h, prec, M, probe_steps, stream=None):
    """Returns (status, probe microseconds per step of the chosen plan)."""
    us = _d(0.0)
    st = load().rom_autotune(h, int(prec), int(M), int(probe_steps), ctypes.byref(us), stream)
    return st, us.value


def rom_set_wait_limit(h, cycles):
    return load().rom_set_wait_limit(h, int(cycles))


def rom_debug_inject_stall(h, on):
    return load().rom_debug_inject_stall(h, 1 if on else 0)


def rom_get_plan(h, prec, M):
    v, cs, w, nc = _i(0), _i(0), _i(0), _i(0)
    st = load().rom_get_plan(h, prec, M, ctypes.byref(v), ctypes.byref(cs), ctypes.byref(w),
                             ctypes.byref(nc))
    return st, v.value, cs.value, w.value, nc.value


def rom_set_companion(h, cluster_size, columns):
    return load().rom_set_companion(h, int(cluster_size), int(columns))


def rom_get_companion(h, M):
    cs, nc, cols = _i(0), _i(0), _i(0)
    st = load().rom_get_companion(h, int(M), ctypes.byref(cs), ctypes.byref(nc), ctypes.byref(cols))
    return st, cs.value, nc.value, cols.value


def rom_status_string(s):
    return load().rom_status_string(int(s))


def rom_last_error():
    return load().rom_last_error()


def rom_version():
    return load().rom_version()


def rom_run_rank2(h, V, S, T, M, nsteps, n0, r, traces, prec, stream):
    return load().rom_run_rank2(h, V, S, T, M, nsteps, n0, r, traces, prec, stream)


def rom_run_rank2_ex(h, V, S, T, ftab, compV, compS, M, nsteps, n0, r, traces, prec, stream):
    return load().rom_run_rank2_ex(h, V, S, T, ftab, compV, compS, M, nsteps, n0, r, traces,
                                   prec, stream)


def rom_run_rank1(h, v, s, T, nsteps, n0, r, trace, prec, stream):
    return load().rom_run_rank1(h, v, s, T, nsteps, n0, r, trace, prec, stream)


def rom_run_rank1_ensemble(h, V, S, T, M, nsteps, n0, r, traces, prec, stream):
    return load().rom_run_rank1_ensemble(h, V, S, T, M, nsteps, n0, r, traces, prec, stream)


class rom_job(ctypes.Structure):
    _fields_ = [("h", _vp), ("V", _vp), ("S", _vp), ("T", _vp), ("M", _i), ("traces", _vp)]


def rom_run_batched(jobs, njobs, nsteps, r, prec, stream):
    """jobs: a ctypes array of rom_job."""
    return load().rom_run_batched(ctypes.cast(jobs, ctypes.c_void_p), njobs, nsteps, r, prec,
                                  stream)


def rom_run_rank3(handles, nops, V, S, T, M, nsteps, r, traces, prec, stream):
    """Raw call: handles is a ctypes array of nops handle pointers."""
    return load().rom_run_rank3(ctypes.cast(handles, ctypes.c_void_p), int(nops), V, S, T, int(M),
                                int(nsteps), int(r), traces, int(prec), stream)


def run_rank3(roms, V, S, T, nsteps, r=0, traces=None, prec="fp32", stream=None):
    """Rank-3 run: len(roms) operators (sharing Kv, Ks, R, dt) times M forcings
    in one launch.  V (Kv, M * nops) and S (Ks, M * nops) column-major device
    tensors, operator i owning columns [i M, (i + 1) M); T (M * nops) periods
    or None; traces (optional) floor(nsteps / r) records of R x (M nops)."""
    p = PRECISIONS.get(prec, prec)
    dt = Rom.dtype_of(p)
    nops = len(roms)
    h0 = roms[0]
    Mt = V.shape[1]
    if Mt % nops:
        raise ValueError("V must have M * len(roms) columns")
    M = Mt // nops
    _check_colmajor(V, h0.Kv, Mt, "V", dt)
    _check_colmajor(S, h0.Ks, Mt, "S", dt)
    if T is not None:
        _check_vec(T, Mt, "T", dt)
    if traces is not None:
        _check_vec(traces, (nsteps // r) * Mt * h0.R, "traces", dt)
    arr = (ctypes.c_void_p * nops)(*[h.h for h in roms])
    st = rom_run_rank3(arr, nops, _ptr(V), _ptr(S), _ptr(T), M, nsteps, r, _ptr(traces), p,
                       _stream_handle(stream))
    _chk(st, "rom_run_rank3")


def run_batched(items, nsteps, r=0, prec="fp32", stream=None):
    """items: list of (Rom, V, S, T, traces or None) with column-major device
    states as for Rom.run_rank2.  One graph launch for all of them."""
    p = PRECISIONS.get(prec, prec)
    dt = Rom.dtype_of(p)
    arr = (rom_job * len(items))()
    for i, (h, V, S, T, tr) in enumerate(items):
        M = V.shape[1]
        _check_colmajor(V, h.Kv, M, "V", dt)
        _check_colmajor(S, h.Ks, M, "S", dt)
        if T is not None:
            _check_vec(T, M, "T", dt)
        if tr is not None:
            if r <= 0:
                raise ValueError("traces need r > 0")
            _check_vec(tr, (nsteps // r) * M * h.R, "traces", dt)
        arr[i] = rom_job(h.h, _ptr(V), _ptr(S), _ptr(T), M, _ptr(tr))
    st = rom_run_batched(arr, len(items), int(nsteps), int(r), p, _stream_handle(stream))
    _chk(st, "rom_run_batched")


def rom_autotune_batched(jobs, njobs, prec, probe_steps, stream=None):
    """Returns (status, probe microseconds per step of the chosen schedule)."""
    us = _d(0.0)
    st = load().rom_autotune_batched(jobs, int(njobs), int(prec), int(probe_steps), ctypes.byref(us), stream)
    return st, us.value


def rom_set_batched_form(jobs, njobs, prec, cluster_size, width_cap):
    return load().rom_set_batched_form(jobs, int(njobs), int(prec), int(cluster_size), int(width_cap))


def set_batched_form(items, cluster_size, width_cap=32, prec="fp32"):
    """Pin how run_batched runs `items` (as for run_batched; FP32): the
    work-list launch with clusters of 2, 4 or 8 CTAs and at most width_cap
    columns per item, or cluster_size 0 for one launch per job."""
    p = PRECISIONS.get(prec, prec)
    arr = (rom_job * len(items))()
    for i, (h, V, S, T, tr) in enumerate(items):
        arr[i] = rom_job(h.h, _ptr(V), _ptr(S), _ptr(T), V.shape[1], None)
    _chk(rom_set_batched_form(arr, len(items), p, cluster_size, width_cap), "rom_set_batched_form")


def autotune_batched(items, prec="fp32", probe_steps=200, stream=None):
    """Time the batching schedule of `items` (as for run_batched) at four
    cluster-budget scales on scratch state and keep the fastest for later
    run_batched calls on the same handles and widths.  Returns the chosen
    schedule's probe time per step in microseconds."""
    p = PRECISIONS.get(prec, prec)
    arr = (rom_job * len(items))()
    for i, (h, V, S, T, tr) in enumerate(items):
        arr[i] = rom_job(h.h, _ptr(V), _ptr(S), _ptr(T), V.shape[1], None)
    st, us = rom_autotune_batched(arr, len(items), p, probe_steps, _stream_handle(stream))
    _chk(st, "rom_autotune_batched")
    return us


def rom_adjoint(h, V0, S0, T, M, nsteps, ystar, ckpt_every, gV0, gS0, gT, workspace, ws_bytes,
                prec, stream):
    loss = _d(0.0)
    st = load().rom_adjoint(h, V0, S0, T, M, nsteps, ystar, ckpt_every, gV0, gS0, gT,
                            ctypes.byref(loss), workspace, ws_bytes, prec, stream)
    return st, loss.value


def rom_adjoint_workspace_size(h, M, nsteps, ckpt_every, prec):
    return load().rom_adjoint_workspace_size(h, M, nsteps, ckpt_every, prec)


def rom_rel_l2(x, x_dtype, ref, ref_dtype, n, stream=None):
    out = _d(0.0)
    st = load().rom_rel_l2(x, x_dtype, ref, ref_dtype, n, ctypes.byref(out), stream)
    return st, out.value


def rom_spectral_radius_noalloc(Avs, Asv, Kv, Ks, stream=None):
    """Allocation-free power iteration on caller-owned device operators
    (column-major FP64).  Returns (status, rho)."""
    out = _d(0.0)
    st = load().rom_spectral_radius_noalloc(Avs, Asv, Kv, Ks, ctypes.byref(out), stream)
    return st, out.value


ROM_PEAK_FP32, ROM_PEAK_FP64, ROM_PEAK_TF32, ROM_PEAK_BF16, ROM_PEAK_L2 = range(5)
PEAK_KINDS = {"fp32": ROM_PEAK_FP32, "fp64": ROM_PEAK_FP64, "tf32": ROM_PEAK_TF32,
              "bf16": ROM_PEAK_BF16, "l2": ROM_PEAK_L2}


def rom_measure_peak(kind, stream=None):
    """Measured peak of one pipe (TFLOP/s) or of L2 reads (GB/s) on the
    current device.  Returns (status, value, ms)."""
    v, ms = _d(0.0), _d(0.0)
    st = load().rom_measure_peak(int(kind), ctypes.byref(v), ctypes.byref(ms), stream)
    return st, v.value, ms.value


def measure_peak(kind):
    """rom_measure_peak by name ("fp32", "fp64", "tf32", "bf16", "l2");
    raises RomError on failure."""
    st, v, ms = rom_measure_peak(PEAK_KINDS[kind])
    _chk(st, "rom_measure_peak")
    return v, ms


# ------------------------------------------------------------ tensor glue --
def rom_trace_stats(traces, nrec, R, M, probs, nprobs, mean_out, q_out, stream=None):
    pr = (_d * max(1, nprobs))(*[float(x) for x in probs])
    return load().rom_trace_stats(traces, nrec, R, M, pr, nprobs, mean_out, q_out, stream)


def trace_stats(traces, probs=(0.05, 0.5, 0.95), stream=None):
    """Mean and quantile bands over the realizations of a (nrec, M, R) device
    float32 trace buffer (the layout run_rank2 writes).  Returns device
    float64 tensors mean (nrec, R) and q (len(probs), nrec, R)."""
    torch = _torch()
    nrec, M, R = traces.shape
    mean = torch.empty((nrec, R), dtype=torch.float64, device=traces.device)
    q = torch.empty((len(probs), nrec, R), dtype=torch.float64, device=traces.device)
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _chk(rom_trace_stats(traces.data_ptr(), nrec, R, M, list(probs), len(probs), mean.data_ptr(),
                         q.data_ptr(), st), "rom_trace_stats")
    return mean, q


def _torch():
    import torch
    return torch


def _ptr(x):
    """Address of a torch tensor / numpy array (None passes through)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_handle(stream):
    if stream is None:
        torch = _torch()
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check_colmajor(x, K, M, name, dtype):
    torch = _torch()
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or x.shape != (K, M) or not x.flags["F_CONTIGUOUS"]:
            raise ValueError(f"{name}: need a Fortran-ordered {dtype} array of shape {(K, M)}")
        return
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    if x.dtype != tdt or tuple(x.shape) != (K, M):
        raise ValueError(f"{name}: need {tdt} of shape {(K, M)}, got {x.dtype} {tuple(x.shape)}")
    if M > 1 and K > 1 and tuple(x.stride()) != (1, K):
        raise ValueError(f"{name}: must be column-major (strides (1, {K})); use Rom.new_state")


def _check_vec(x, n, name, dtype):
    torch = _torch()
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or x.size != n or not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name}: need a contiguous {dtype} array with {n} elements")
        return
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    if x.dtype != tdt or x.numel() != n or not x.is_contiguous():
        raise ValueError(f"{name}: need a contiguous {tdt} tensor with {n} elements")


class Rom:
    """A reduced model resident on the current CUDA device."""

    def __init__(self, Avs, Asv, g, C=None, dt=None):
        Avs = np.asfortranarray(np.asarray(Avs, dtype=np.float64))
        Asv = np.asfortranarray(np.asarray(Asv, dtype=np.float64))
        g = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
        self.Kv, self.Ks = Avs.shape
        if Asv.shape != (self.Ks, self.Kv) or g.shape != (self.Kv,):
            raise ValueError("shape mismatch: Avs (Kv,Ks), Asv (Ks,Kv), g (Kv,)")
        if C is None or np.asarray(C).size == 0:
            Cm, self.R = None, 0
        else:
            Cm = np.asfortranarray(np.asarray(C, dtype=np.float64))
            self.R = Cm.shape[0]
            if Cm.shape[1] != self.Kv:
                raise ValueError("C must be (R, Kv)")
        if dt is None:
            raise ValueError("dt is required")
        self.dt = float(dt)
        st, h, rho = rom_create(_ptr(Avs), _ptr(Asv), _ptr(g), _ptr(Cm), self.Kv, self.Ks,
                                self.R, self.dt, ROM_IN_F64)
        self.rho = rho
        _chk(st, "rom_create")
        self.h = h

    @classmethod
    def from_problem(cls, p):
        return cls(p.Avs, p.Asv, p.g, p.C if p.C.shape[0] else None, p.dt)

    def close(self):
        if getattr(self, "h", None):
            rom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ helpers
    @staticmethod
    def dtype_of(prec):
        return np.float64 if PRECISIONS.get(prec, prec) == ROM_FP64 else np.float32

    @staticmethod
    def new_state(K, M, prec="fp32", device="cuda", fill=None):
        """A column-major (K, M) state tensor (transpose of a contiguous (M, K))."""
        torch = _torch()
        dt = torch.float64 if Rom.dtype_of(prec) == np.float64 else torch.float32
        x = torch.zeros((M, K), dtype=dt, device=device)
        if fill is not None:
            x.copy_(torch.as_tensor(np.asarray(fill).T, dtype=dt))
        return x.t()

    @staticmethod
    def trace_view(traces):
        """Logical (nrec, R, M) view of a (nrec, M, R) trace buffer."""
        return traces.transpose(1, 2) if hasattr(traces, "transpose") and not isinstance(
            traces, np.ndarray) else np.transpose(traces, (0, 2, 1))

    def spectral_radius(self):
        st, rho = rom_spectral_radius(self.h)
        _chk(st, "rom_spectral_radius")
        return rho

    def set_kernel(self, kernel):
        _chk(rom_set_kernel(self.h, int(kernel)), "rom_set_kernel")

    def autotune(self, M, prec="fp32", probe_steps=200, stream=None):
        """Time every candidate plan for M realizations and keep the fastest;
        returns the chosen plan's probe time per step in microseconds."""
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        s, us = rom_autotune(self.h, PRECISIONS.get(prec, prec), M, probe_steps, st)
        _chk(s, "rom_autotune")
        return us

    def set_wavelet(self, wavelet):
        """Source signal of the periods: "ricker" (default) or "gauss1" (first
        derivative of a Gaussian), or the ROM_WAVELET_* code."""
        w = {"ricker": ROM_WAVELET_RICKER, "gauss1": ROM_WAVELET_GAUSS1}.get(wavelet, wavelet)
        _chk(rom_set_wavelet(self.h, int(w)), "rom_set_wavelet")

    def set_reference(self, Xv=None, Xs=None):
        """Reduced reference state of Eq. (rom_ode_tensor): Xv (Kv, M) and Xs
        (Ks, M), numpy arrays or torch tensors (host or device), either may
        be None; both None clears it.  Later runs add it to the two halves of
        every step.  The values are passed as float64 (the library keeps its
        own FP64 and FP32 copies)."""
        if Xv is None and Xs is None:
            _chk(rom_set_reference(self.h, None, None, 0, ROM_IN_F64), "rom_set_reference")
            return
        parts, M = [], None
        for X, K in ((Xv, self.Kv), (Xs, self.Ks)):
            if X is None:
                parts.append(None)
                continue
            if isinstance(X, np.ndarray):
                X = np.asfortranarray(X, dtype=np.float64)
            else:
                X = X.double().t().contiguous().t()  # column-major storage
            if X.ndim != 2 or X.shape[0] != K or (M is not None and X.shape[1] != M):
                raise ValueError("reference state parts must be (Kv, M) and (Ks, M)")
            M = X.shape[1]
            parts.append(X)
        _chk(rom_set_reference(self.h, _ptr(parts[0]), _ptr(parts[1]), M, ROM_IN_F64),
             "rom_set_reference")

    def plan(self, M, prec="fp32"):
        st, v, cs, w, nc = rom_get_plan(self.h, PRECISIONS.get(prec, prec), int(M))
        _chk(st, "rom_get_plan")
        out = {"variant": v, "cluster_size": cs, "cols_per_block": w, "nclusters": nc}
        if v == 4:
            st, ccs, cn, ccols = rom_get_companion(self.h, int(M))
            _chk(st, "rom_get_companion")
            out["companion"] = {"cluster_size": ccs, "nclusters": cn, "columns": ccols}
        return out

    def set_companion(self, cluster_size=0, columns=0):
        """Streaming companion of the FP32 two-block kernel: 0 lets the
        planner decide, -1 turns it off, 2 or 4 pins clusters of that size
        with `columns` columns."""
        _chk(rom_set_companion(self.h, cluster_size, columns), "rom_set_companion")

    def sync_status(self):
        st, dev = rom_sync_status(self.h)
        _chk(st, "rom_sync_status")
        return dev

    # ------------------------------------------------------------ integrate
    def run_rank2(self, V, S, T, nsteps, n0=0, r=0, traces=None, prec="fp32", stream=None,
                  ftab=None, compV=None, compS=None):
        p = PRECISIONS.get(prec, prec)
        dt = self.dtype_of(p)
        M = V.shape[1]
        _check_colmajor(V, self.Kv, M, "V", dt)
        _check_colmajor(S, self.Ks, M, "S", dt)
        if T is not None:
            _check_vec(T, M, "T", dt)
        if ftab is not None:
            _check_vec(ftab, nsteps * M, "ftab", dt)
        if traces is not None:
            nrec = nsteps // r if r > 0 else 0
            _check_vec(traces, nrec * M * self.R, "traces", dt)
        if compV is not None:
            _check_colmajor(compV, self.Kv, M, "compV", np.float32)
            _check_colmajor(compS, self.Ks, M, "compS", np.float32)
        sh = _stream_handle(stream)
        if ftab is None and compV is None:
            st = rom_run_rank2(self.h, _ptr(V), _ptr(S), _ptr(T), M, int(nsteps), int(n0),
                               int(r), _ptr(traces), p, sh)
        else:
            st = rom_run_rank2_ex(self.h, _ptr(V), _ptr(S), _ptr(T), _ptr(ftab), _ptr(compV),
                                  _ptr(compS), M, int(nsteps), int(n0), int(r), _ptr(traces),
                                  p, sh)
        _chk(st, "rom_run_rank2")

    def run_rank1(self, v, s, T, nsteps, n0=0, r=0, trace=None, prec="fp32", stream=None):
        p = PRECISIONS.get(prec, prec)
        dt = self.dtype_of(p)
        _check_vec(v, self.Kv, "v", dt)
        _check_vec(s, self.Ks, "s", dt)
        if trace is not None:
            _check_vec(trace, (nsteps // r) * self.R, "trace", dt)
        st = rom_run_rank1(self.h, _ptr(v), _ptr(s), float(T), int(nsteps), int(n0), int(r),
                           _ptr(trace), p, _stream_handle(stream))
        _chk(st, "rom_run_rank1")

    def run_rank1_ensemble(self, V, S, T, nsteps, n0=0, r=0, traces=None, prec="fp32",
                           stream=None):
        p = PRECISIONS.get(prec, prec)
        dt = self.dtype_of(p)
        M = V.shape[1]
        _check_colmajor(V, self.Kv, M, "V", dt)
        _check_colmajor(S, self.Ks, M, "S", dt)
        _check_vec(T, M, "T", dt)
        if traces is not None:
            _check_vec(traces, (nsteps // r) * M * self.R, "traces", dt)
        st = rom_run_rank1_ensemble(self.h, _ptr(V), _ptr(S), _ptr(T), M, int(nsteps), int(n0),
                                    int(r), _ptr(traces), p, _stream_handle(stream))
        _chk(st, "rom_run_rank1_ensemble")


def adjoint(h, V0, S0, T, ystar, nsteps, ckpt_every=0, stream=None):
    """Loss and gradients of sum_n ||C V^n - ystar^n||^2 (device tensors).
    V0 (Kv, M) and S0 (Ks, M) column-major; ystar a contiguous (nsteps, M, R)
    tensor (record n-1 = ystar^n).  float32 inputs run the FP32 path, float64
    inputs the FP64 one (Kv, Ks <= 512).  Returns (loss, gV0, gS0, gT) in the
    inputs' type."""
    torch = _torch()
    M = V0.shape[1]
    f64 = V0.dtype == torch.float64
    dt = np.float64 if f64 else np.float32
    _check_colmajor(V0, h.Kv, M, "V0", dt)
    _check_colmajor(S0, h.Ks, M, "S0", dt)
    _check_vec(T, M, "T", dt)
    _check_vec(ystar, nsteps * M * h.R, "ystar", dt)
    name = "fp64" if f64 else "fp32"
    gV = Rom.new_state(h.Kv, M, name, device=V0.device)
    gS = Rom.new_state(h.Ks, M, name, device=V0.device)
    gT = torch.zeros(M, dtype=V0.dtype, device=V0.device)
    st, loss = rom_adjoint(h.h, _ptr(V0), _ptr(S0), _ptr(T), M, int(nsteps), _ptr(ystar),
                           int(ckpt_every), _ptr(gV), _ptr(gS), _ptr(gT), None, 0,
                           ROM_FP64 if f64 else ROM_FP32, _stream_handle(stream))
    _chk(st, "rom_adjoint")
    return loss, gV, gS, gT


def _adjoint_function():
    torch = _torch()

    class RomAdjointFn(torch.autograd.Function):
        """loss = sum_n ||C V^n - ystar^n||^2 as a differentiable function of
        (V0, S0, T); the backward pass returns the reverse-leapfrog gradients
        computed together with the loss."""

        @staticmethod
        def forward(ctx, V0, S0, T, h, ystar, nsteps, ckpt_every):
            loss, gV, gS, gT = adjoint(h, V0.detach(), S0.detach(), T.detach(), ystar, nsteps,
                                       ckpt_every)
            ctx.save_for_backward(gV, gS, gT)
            return torch.tensor(loss, dtype=torch.float64, device=V0.device)

        @staticmethod
        def backward(ctx, gout):
            gV, gS, gT = ctx.saved_tensors
            s = gout.to(gV.dtype)
            return s * gV, s * gS, s * gT, None, None, None, None

    return RomAdjointFn


_RomAdjointFn = None


def rom_loss(h, V0, S0, T, ystar, nsteps, ckpt_every=0):
    """Differentiable misfit (torch.autograd): call .backward() for dL/dV0,
    dL/dS0, dL/dT."""
    global _RomAdjointFn
    if _RomAdjointFn is None:
        _RomAdjointFn = _adjoint_function()
    return _RomAdjointFn.apply(V0, S0, T, h, ystar, nsteps, ckpt_every)


def rel_l2(x, ref, stream=None) -> float:
    """FP64 relative L2 error of two device tensors, computed on the GPU."""
    torch = _torch()
    dmap = {torch.float64: ROM_IN_F64, torch.float32: ROM_IN_F32}
    if x.numel() != ref.numel():
        raise ValueError("size mismatch")
    xc = x.contiguous()
    rc = ref.contiguous()
    st, v = rom_rel_l2(xc.data_ptr(), dmap[xc.dtype], rc.data_ptr(), dmap[rc.dtype],
                       xc.numel(), _stream_handle(stream))
    _chk(st, "rom_rel_l2")
    return v


# ------------------------------------------------------------------ FOM --

def rom_fom_create(Nr, Ntheta, r_cmb, r_earth, rho, vs, dt):
    """Raw call.  Returns (status, handle)."""
    h = _vp()
    st = load().rom_fom_create(int(Nr), int(Ntheta), float(r_cmb), float(r_earth), float(rho),
                               float(vs), float(dt), ctypes.byref(h))
    return st, h.value


def rom_fom_destroy(h):
    return load().rom_fom_destroy(h)


def rom_fom_set_passes(h, passes):
    return load().rom_fom_set_passes(h, int(passes))


def rom_fom_dims(h):
    """Returns (status, nv, n1, n2)."""
    a, b, c = _i(0), _i(0), _i(0)
    st = load().rom_fom_dims(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return st, a.value, b.value, c.value


def rom_fom_run(h, V, S1, S2, M, nsteps, n0, src, T, wavelet, recv, nrecv, r, traces, prec, stream):
    return load().rom_fom_run(h, V, S1, S2, int(M), int(nsteps), int(n0), int(src), T, int(wavelet),
                              recv, int(nrecv), int(r), traces, int(prec), stream)


class Fom:
    """The rank-2 full-order shear-wave model of Sec. 3 (rom_fom_* of the C
    ABI).  Defaults: the homogeneous layer of App. A (rho 2500 kg/m^3, vs
    5000 m/s, dt 0.05 s) on the mantle shell 3480-6371 km.  States are
    unknown-major (n, M) contiguous device tensors, M realizations per row."""

    def __init__(self, Nr, Ntheta, r_cmb=3480e3, r_earth=6371e3, rho=2500.0, vs=5000.0, dt=0.05):
        st, h = rom_fom_create(Nr, Ntheta, r_cmb, r_earth, rho, vs, dt)
        _chk(st, "rom_fom_create")
        self.h = h
        self.Nr, self.Ntheta = int(Nr), int(Ntheta)
        self.r_cmb, self.r_earth, self.rho, self.vs, self.dt = r_cmb, r_earth, rho, vs, dt
        st, self.nv, self.n1, self.n2 = rom_fom_dims(h)
        _chk(st, "rom_fom_dims")

    def __del__(self):
        if getattr(self, "h", None):
            rom_fom_destroy(self.h)
            self.h = None

    def set_passes(self, passes):
        """1: fused single pass (default, 8 B per unknown and realization
        in FP32); 2: velocity pass then stress pass (12 B)."""
        _chk(rom_fom_set_passes(self.h, passes), "rom_fom_set_passes")

    def vindex(self, i, j):
        """Velocity unknown of grid point (r_{i+1/2}, theta_j)."""
        return int(i) * (self.Ntheta - 1) + (int(j) - 1)

    def source_index(self, depth, j=1):
        """Velocity unknown in the radial cell at `depth` below r_earth, on
        polar line j (default: next to the symmetry axis)."""
        dr = (self.r_earth - self.r_cmb) / self.Nr
        i = int((self.r_earth - depth - self.r_cmb) / dr)
        return self.vindex(min(max(i, 0), self.Nr - 1), j)

    def new_state(self, M, prec="fp32", device="cuda"):
        torch = _torch()
        dt = torch.float64 if prec == "fp64" else torch.float32
        return tuple(torch.zeros((n, M), dtype=dt, device=device) for n in (self.nv, self.n1, self.n2))

    def run(self, V, S1, S2, nsteps, src=-1, T=None, wavelet=ROM_WAVELET_GAUSS1, recv=None, r=0,
            traces=None, prec="fp32", n0=0, stream=None):
        p = PRECISIONS.get(prec, prec)
        M = V.shape[1]
        for x, n, name in ((V, self.nv, "V"), (S1, self.n1, "S1"), (S2, self.n2, "S2")):
            if tuple(x.shape) != (n, M) or not x.is_contiguous():
                raise ValueError(f"{name}: need a contiguous ({n}, {M}) tensor")
        nrecv = 0 if recv is None else recv.numel()
        st = rom_fom_run(self.h, _ptr(V), _ptr(S1), _ptr(S2), M, nsteps, n0, src, _ptr(T), wavelet,
                         _ptr(recv), nrecv, r, _ptr(traces), p, _stream_handle(stream))
        _chk(st, "rom_fom_run")
