"""GPU parity of the reduced reference state (rom_set_reference; Eq. (rom_ode),
Eq. (rom_ode_tensor)) on every path against the FP64 oracle run with the same
term.  Tolerances: relative L2 (Eq. (errors), Sec. 4.4) of 1e-12 for FP64 and
1e-4 for FP32 and the tensor-core paths (TF32x3, which is reported rather than
accepted over long horizons, on a short run)."""
import numpy as np
import pytest

import oracle
from paper_2009_11742_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-4, "bf16s": 1e-4, "tf32x3": 1e-4}


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


@pytest.fixture(scope="module")
def rom():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_11742_gb300 import build
    build.build()
    from paper_2009_11742_gb300 import rom as R
    return R


def tdt(prec):
    return torch.float64 if prec == "fp64" else torch.float32


def case(Kv, Ks, M, R, seed, scale=0.05):
    p = inputs.make_problem(Kv, Ks, M, R, seed=seed)
    rng = np.random.default_rng(seed + 7)
    Xv = scale * rng.standard_normal((Kv, M))
    Xs = scale * rng.standard_normal((Ks, M))
    V0 = inputs.random_state(Kv, M, seed=seed + 1, scale=0.1)
    S0 = inputs.random_state(Ks, M, seed=seed + 2, scale=0.1)
    return p, Xv, Xs, V0, S0


def run(rom, h, p, V0, S0, N, prec, r=0):
    Kv, M = V0.shape
    Ks = S0.shape[0]
    V = rom.Rom.new_state(Kv, M, prec, fill=V0)
    S = rom.Rom.new_state(Ks, M, prec, fill=S0)
    T = torch.as_tensor(p.T, dtype=tdt(prec), device="cuda")
    tr = torch.zeros((N // r, M, p.C.shape[0]), dtype=tdt(prec), device="cuda") if r else None
    h.run_rank2(V, S, T, N, r=r, traces=tr, prec=prec)
    assert h.sync_status() == rom.ROM_OK
    trn = None if tr is None else tr.cpu().numpy().transpose(0, 2, 1)
    return V.cpu().numpy(), S.cpu().numpy(), trn


@pytest.mark.parametrize("prec,kernel,Kv,Ks,M,N", [
    ("fp64", 0, 192, 160, 11, 300),
    ("fp32", 0, 512, 512, 64, 400),     # two-block split kernel
    ("fp32", 1, 320, 300, 23, 300),     # one-block kernel
    ("fp32", 3, 256, 256, 40, 300),     # dataflow kernel
    ("bf16s", 0, 1024, 1000, 100, 200),
    ("bf16s", 0, 384, 384, 40, 300),
    ("tf32x3", 0, 512, 500, 70, 40),
])
def test_reference_state_vs_oracle(rom, prec, kernel, Kv, Ks, M, N):
    p, Xv, Xs, V0, S0 = case(Kv, Ks, M, 6, seed=Kv + M)
    h = rom.Rom.from_problem(p)
    if kernel:
        h.set_kernel(kernel)
    h.set_reference(Xv, Xs)
    r = 5
    V, S, tr = run(rom, h, p, V0, S0, N, prec, r=r)
    Vo, So, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, N, T=p.T, r=r,
                                 xref=(Xv, Xs))
    tol = TOL[prec]
    assert colmax_rel(V, Vo) <= tol and colmax_rel(S, So) <= tol and colmax_rel(tr, tro) <= tol
    # the term is not negligible in this case
    Vn, _, _ = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, N, T=p.T)
    assert rel(Vn, Vo) > 100 * tol


def test_reference_state_fixed_point_fp64(rom):
    """Xv = -Avs S*, Xs = -Asv V* hold (V*, S*) still (unforced)."""
    Kv, Ks, M = 256, 224, 9
    p = inputs.make_problem(Kv, Ks, M, 0, seed=88)
    rng = np.random.default_rng(3)
    Vs = rng.standard_normal((Kv, M))
    Ss = rng.standard_normal((Ks, M))
    h = rom.Rom.from_problem(p)
    h.set_reference(-p.Avs.astype(np.float64) @ Ss, -p.Asv.astype(np.float64) @ Vs)
    V = rom.Rom.new_state(Kv, M, "fp64", fill=Vs)
    S = rom.Rom.new_state(Ks, M, "fp64", fill=Ss)
    h.run_rank2(V, S, None, 500, prec="fp64")
    assert h.sync_status() == rom.ROM_OK
    assert rel(V.cpu().numpy(), Vs) < 1e-12 and rel(S.cpu().numpy(), Ss) < 1e-12


def test_reference_state_one_part_and_clear(rom):
    """Only Xs given; then cleared, the run equals a handle that never had one
    (bitwise)."""
    Kv, Ks, M, N = 256, 256, 30, 200
    p, _, Xs, V0, S0 = case(Kv, Ks, M, 4, seed=5)
    h = rom.Rom.from_problem(p)
    h.set_reference(None, Xs)
    V, S, _ = run(rom, h, p, V0, S0, N, "fp32")
    Vo, So, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, V0, S0, N, T=p.T, xref=(None, Xs))
    assert colmax_rel(V, Vo) <= 1e-4 and colmax_rel(S, So) <= 1e-4
    h.set_reference(None, None)
    V1, S1, _ = run(rom, h, p, V0, S0, N, "fp32")
    h2 = rom.Rom.from_problem(p)
    V2, S2, _ = run(rom, h2, p, V0, S0, N, "fp32")
    assert np.array_equal(V1, V2) and np.array_equal(S1, S2)


def test_reference_state_other_width_is_rejected(rom):
    Kv, Ks, M = 128, 128, 8
    p, Xv, Xs, V0, S0 = case(Kv, Ks, M, 2, seed=6)
    h = rom.Rom.from_problem(p)
    h.set_reference(Xv, Xs)
    V = rom.Rom.new_state(Kv, M + 1, "fp32")
    S = rom.Rom.new_state(Ks, M + 1, "fp32")
    T = torch.ones(M + 1, device="cuda") * float(p.T[0])
    with pytest.raises(RuntimeError):
        h.run_rank2(V, S, T, 10, prec="fp32")


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_reference_state_rank1_paths(rom, prec):
    """The rank-1 run (M = 1) and the rank-1 ensemble carry the term too."""
    Kv, Ks, M, N = 192, 160, 12, 250
    p, Xv, Xs, V0, S0 = case(Kv, Ks, M, 4, seed=9)
    Vo, So, _ = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, N, T=p.T, xref=(Xv, Xs))
    h = rom.Rom.from_problem(p)
    h.set_reference(Xv, Xs)
    V = rom.Rom.new_state(Kv, M, prec, fill=V0)
    S = rom.Rom.new_state(Ks, M, prec, fill=S0)
    T = torch.as_tensor(p.T, dtype=tdt(prec), device="cuda")
    h.run_rank1_ensemble(V, S, T, N, prec=prec)
    assert h.sync_status() == rom.ROM_OK
    tol = TOL[prec]
    assert colmax_rel(V.cpu().numpy(), Vo) <= tol and colmax_rel(S.cpu().numpy(), So) <= tol
    m = 4
    h1 = rom.Rom.from_problem(p)
    h1.set_reference(Xv[:, m:m + 1], Xs[:, m:m + 1])
    v = torch.as_tensor(V0[:, m], dtype=tdt(prec), device="cuda").clone()
    s = torch.as_tensor(S0[:, m], dtype=tdt(prec), device="cuda").clone()
    h1.run_rank1(v, s, float(p.T[m]), N, prec=prec)
    assert h1.sync_status() == rom.ROM_OK
    assert rel(v.cpu().numpy(), Vo[:, m]) <= tol and rel(s.cpu().numpy(), So[:, m]) <= tol


def test_reference_state_batched(rom):
    """Two ROMs in one batched launch, each with its own reference state."""
    N = 150
    items, refs = [], []
    for seed, (Kv, Ks, M) in enumerate([(256, 256, 20), (384, 320, 9)]):
        p, Xv, Xs, V0, S0 = case(Kv, Ks, M, 0, seed=30 + seed)
        h = rom.Rom.from_problem(p)
        h.set_reference(Xv, Xs)
        V = rom.Rom.new_state(Kv, M, "fp32", fill=V0)
        S = rom.Rom.new_state(Ks, M, "fp32", fill=S0)
        T = torch.as_tensor(p.T, device="cuda")
        items.append((h, V, S, T, None))
        refs.append((p, Xv, Xs, V0, S0))
    rom.run_batched(items, N, prec="fp32")
    torch.cuda.synchronize()
    for (h, V, S, _, _), (p, Xv, Xs, V0, S0) in zip(items, refs):
        assert h.sync_status() == rom.ROM_OK
        Vo, So, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, V0, S0, N, T=p.T,
                                   xref=(Xv, Xs))
        assert rel(V.cpu().numpy(), Vo) <= 1e-4 and rel(S.cpu().numpy(), So) <= 1e-4


def test_reference_state_adjoint(rom):
    """The adjoint's forward and recomputed sweeps carry the term; gradients
    against the oracle adjoint run with the same term."""
    Kv, Ks, M, R, N = 128, 128, 6, 3, 60
    p, Xv, Xs, V0, S0 = case(Kv, Ks, M, R, seed=12, scale=0.02)
    Z1, Z2 = np.zeros((Kv, M)), np.zeros((Ks, M))
    _, _, ystar = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z1, Z2, N,
                                 T=1.05 * p.T.astype(np.float64), r=1)
    ystar = ystar.astype(np.float32)
    h = rom.Rom.from_problem(p)
    h.set_reference(Xv, Xs)
    V0t = rom.Rom.new_state(Kv, M, "fp32", fill=V0)
    S0t = rom.Rom.new_state(Ks, M, "fp32", fill=S0)
    T = torch.as_tensor(p.T, device="cuda")
    ys = torch.as_tensor(np.ascontiguousarray(np.transpose(ystar, (0, 2, 1))), device="cuda")
    loss, gV, gS, gT = rom.adjoint(h, V0t, S0t, T, ys, N, ckpt_every=16)
    torch.cuda.synchronize()
    assert h.sync_status() == rom.ROM_OK
    Lo, gVo, gSo, gTo = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, p.T, N, ystar,
                                       xref=(Xv, Xs))
    assert abs(loss - Lo) <= 1e-4 * abs(Lo)
    assert rel(gV.cpu().numpy(), gVo) <= 1e-4 and rel(gS.cpu().numpy(), gSo) <= 1e-4
    assert rel(gT.cpu().numpy(), gTo) <= 1e-4
