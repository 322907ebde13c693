"""GPU parity with the paper's second source signal, the first derivative of
a Gaussian (Sec. 3.2), on every path that evaluates the forcing from the
periods: the three FP32 kernels, FP64, the tensor-core schemes, both rank-1
baselines and the adjoint's period gradient."""
import numpy as np
import pytest

import oracle
from paper_2009_11742_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rom():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_11742_gb300 import build
    build.build()
    from paper_2009_11742_gb300 import rom as R
    return R


def colmax_rel(a, b):
    """Largest per-realization relative L2 error (Eq. (errors), Sec. 4.4):
    the last axis indexes the realizations (columns), every other axis is
    one realization's values.  One bad column cannot hide among good ones."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    a = a.reshape(-1, a.shape[-1])
    b = b.reshape(-1, b.shape[-1])
    num = np.linalg.norm(a - b, axis=0)
    den = np.maximum(np.linalg.norm(b, axis=0), 1e-300)
    return float(np.max(num / den))


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run(R, h, p, N, prec, kernel=0, r=5, n0=3):
    h.set_kernel(kernel)
    dt = torch.float64 if prec == "fp64" else torch.float32
    V = R.Rom.new_state(p.Kv, p.M, prec)
    S = R.Rom.new_state(p.Ks, p.M, prec)
    T = torch.as_tensor(p.T, dtype=dt, device="cuda")
    tr = torch.zeros((N // r, p.M, p.R), dtype=dt, device="cuda")
    h.run_rank2(V, S, T, N, n0=n0, r=r, traces=tr, prec=prec)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    return V.cpu().numpy(), S.cpu().numpy(), tr.transpose(1, 2).cpu().numpy()


@pytest.mark.parametrize("prec,kernel,tol", [("fp32", 1, 1e-4), ("fp32", 2, 1e-4), ("fp32", 3, 1e-4),
                                              ("fp64", 0, 1e-12), ("tf32x3", 0, 1e-4), ("bf16s", 0, 1e-5)])
def test_gaussian_source_rank2(rom, prec, kernel, tol):
    p = inputs.make_problem(256, 200, 40, 8, seed=31)
    h = rom.Rom.from_problem(p)
    h.set_wavelet("gauss1")
    N = 300
    V, S, tr = run(rom, h, p, N, prec, kernel)
    Z1, Z2 = np.zeros((256, 40)), np.zeros((200, 40))
    Vo, So, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z1, Z2, N, T=p.T, n0=3, r=5, wavelet=1)
    errs = (rel(V, Vo), rel(S, So), rel(tr, tro))
    assert max(errs) <= tol, errs
    # the Ricker result is different, so the setting reached the kernel
    Vr, _, _ = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z1, Z2, N, T=p.T, n0=3, r=5)
    assert rel(V, Vr) > 1e-2


def test_gaussian_source_rank1(rom):
    p = inputs.make_problem(128, 128, 6, 4, seed=32)
    h = rom.Rom.from_problem(p)
    h.set_wavelet("gauss1")
    N = 200
    Z = np.zeros((128, 6))
    Vo, So, _ = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, N, T=p.T, wavelet=1)
    v = torch.zeros(128, device="cuda")
    s = torch.zeros(128, device="cuda")
    h.run_rank1(v, s, float(p.T[2]), N, prec="fp32")
    Ve = rom.Rom.new_state(128, 6, "fp32")
    Se = rom.Rom.new_state(128, 6, "fp32")
    h.run_rank1_ensemble(Ve, Se, torch.as_tensor(p.T, device="cuda"), N, prec="fp32")
    torch.cuda.synchronize()
    assert rel(v.cpu().numpy(), Vo[:, 2]) <= 1e-4
    assert colmax_rel(Ve.cpu().numpy(), Vo) <= 1e-4 and colmax_rel(Se.cpu().numpy(), So) <= 1e-4


def test_gaussian_source_adjoint_period_gradient(rom):
    p = inputs.make_problem(64, 64, 5, 3, seed=33)
    h = rom.Rom.from_problem(p)
    h.set_wavelet("gauss1")
    N = 60
    Z = np.zeros((64, 5))
    _, _, ys = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, N, T=1.05 * p.T.astype(np.float64),
                              r=1, wavelet=1)
    ys = ys.astype(np.float32)
    V0 = rom.Rom.new_state(64, 5, "fp32")
    S0 = rom.Rom.new_state(64, 5, "fp32")
    T = torch.as_tensor(p.T, device="cuda")
    yst = torch.as_tensor(np.ascontiguousarray(np.transpose(ys, (0, 2, 1))), device="cuda")
    loss, gV, gS, gT = rom.adjoint(h, V0, S0, T, yst, N, ckpt_every=16)
    torch.cuda.synchronize()
    Lo, gVo, gSo, gTo = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, p.T, N, ys, wavelet=1)
    assert abs(loss - Lo) <= 1e-4 * abs(Lo)
    assert rel(gT.cpu().numpy(), gTo) <= 1e-4 and rel(gV.cpu().numpy(), gVo) <= 1e-4


def test_wavelet_setting_is_checked(rom):
    p = inputs.make_problem(64, 64, 2, 0, seed=1)
    h = rom.Rom.from_problem(p)
    assert rom.rom_set_wavelet(h.h, 2) == rom.ROM_E_INVAL
    assert rom.rom_set_wavelet(h.h, -1) == rom.ROM_E_INVAL
    assert rom.rom_set_wavelet(h.h, rom.ROM_WAVELET_GAUSS1) == rom.ROM_OK
    assert rom.rom_set_wavelet(h.h, rom.ROM_WAVELET_RICKER) == rom.ROM_OK
