"""GPU parity of the rank-3 launch (rom_run_rank3, the rank-3 outlook of
Sec. 5): nops operators times M forcings in one persistent launch, each
operator's slab against the FP64 oracle run one column at a time, and
bitwise against that operator's own rank-2 run on the same kernel."""
import numpy as np
import pytest

import oracle
from paper_2009_11742_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-4}


def colmax_rel(a, b):
    """Largest per-column relative L2 error (columns are realizations)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    num = np.linalg.norm(a - b, axis=0)
    return float(np.max(num / np.maximum(np.linalg.norm(b, axis=0), 1e-300)))


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


def operators(nops, Kv, Ks, M, R, seed):
    return inputs.rank3_problems(nops, Kv, Ks, M, R, seed=seed)


def rank3_run(rom, probs, V0, S0, N, prec, r):
    roms = [rom.Rom.from_problem(p) for p in probs]
    Kv, Mt = V0.shape
    Ks = S0.shape[0]
    R = probs[0].C.shape[0]
    V = rom.Rom.new_state(Kv, Mt, prec, fill=V0)
    S = rom.Rom.new_state(Ks, Mt, prec, fill=S0)
    T = torch.as_tensor(np.concatenate([p.T for p in probs]), dtype=tdt(prec), device="cuda")
    tr = torch.zeros((N // r, Mt, R), dtype=tdt(prec), device="cuda") if r else None
    rom.run_rank3(roms, V, S, T, N, r=r, traces=tr, prec=prec)
    assert roms[0].sync_status() == rom.ROM_OK
    return roms, V.cpu().numpy(), S.cpu().numpy(), None if tr is None else tr.cpu().numpy()


@pytest.mark.parametrize("prec,nops,Kv,Ks,M,N", [
    ("fp32", 3, 512, 512, 40, 200),   # split kernel, one wave
    ("fp32", 9, 512, 448, 8, 120),    # more operators than co-resident clusters
    ("fp32", 2, 640, 600, 24, 100),   # one-block kernel (K > 512)
    # enough columns for the planner to take clusters of 4 (22 row tiles
    # dealt 6, 6, 5, 5), 32 clusters per operator in two waves
    ("fp32", 2, 704, 680, 256, 40),
    ("fp64", 4, 192, 160, 10, 200),   # FP64 one-block kernel
    ("fp32", 1, 256, 256, 10, 100),   # one operator: the rank-2 run
])
def test_rank3_vs_oracle(rom, prec, nops, Kv, Ks, M, N):
    R, r = 5, 4
    probs = operators(nops, Kv, Ks, M, R, seed=50 + nops)
    V0 = inputs.random_state(Kv, M * nops, seed=1, scale=0.1)
    S0 = inputs.random_state(Ks, M * nops, seed=2, scale=0.1)
    _, V, S, tr = rank3_run(rom, probs, V0, S0, N, prec, r)
    tol = TOL[prec]
    for i, p in enumerate(probs):
        sl = slice(i * M, (i + 1) * M)
        Vo, So, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0[:, sl], S0[:, sl], N,
                                     T=p.T, r=r)
        assert colmax_rel(V[:, sl], Vo) <= tol and colmax_rel(S[:, sl], So) <= tol, i
        trg = tr[:, sl, :].transpose(0, 2, 1)  # records x receivers x columns
        assert colmax_rel(trg.reshape(-1, M), np.asarray(tro).reshape(-1, M)) <= tol, i


@pytest.mark.parametrize("prec,kernel", [("fp32", 2), ("fp64", 0)])
def test_rank3_equals_rank2_per_operator_bitwise(rom, prec, kernel):
    """Each operator's slab is computed exactly as that handle's own rank-2
    run over the same columns (same kernel): a column's arithmetic does not
    depend on its place in a block or on the operator's neighbours."""
    nops, Kv, Ks, M, N, R, r = 3, 256, 256, 20, 150, 4, 5
    probs = operators(nops, Kv, Ks, M, R, seed=70)
    V0 = inputs.random_state(Kv, M * nops, seed=3, scale=0.1)
    S0 = inputs.random_state(Ks, M * nops, seed=4, scale=0.1)
    roms, V, S, tr = rank3_run(rom, probs, V0, S0, N, prec, r)
    for i, (h, p) in enumerate(zip(roms, probs)):
        if kernel:
            h.set_kernel(kernel)
        sl = slice(i * M, (i + 1) * M)
        Vi = rom.Rom.new_state(Kv, M, prec, fill=V0[:, sl])
        Si = rom.Rom.new_state(Ks, M, prec, fill=S0[:, sl])
        Ti = torch.as_tensor(p.T, dtype=tdt(prec), device="cuda")
        tri = torch.zeros((N // r, M, R), dtype=tdt(prec), device="cuda")
        h.run_rank2(Vi, Si, Ti, N, r=r, traces=tri, prec=prec)
        assert h.sync_status() == rom.ROM_OK
        assert np.array_equal(Vi.cpu().numpy(), V[:, sl]), i
        assert np.array_equal(Si.cpu().numpy(), S[:, sl]), i
        assert np.array_equal(tri.cpu().numpy(), tr[:, sl, :]), i


def test_rank3_rejects_mismatched_operators(rom):
    p1 = inputs.make_problem(128, 128, 4, 2, seed=1)
    p2 = inputs.make_problem(128, 128, 4, 2, seed=2)  # another dt
    h1, h2 = rom.Rom.from_problem(p1), rom.Rom.from_problem(p2)
    V = rom.Rom.new_state(128, 8, "fp32")
    S = rom.Rom.new_state(128, 8, "fp32")
    with pytest.raises(RuntimeError):
        rom.run_rank3([h1, h2], V, S, None, 10)
    p3 = inputs.make_problem(128, 128, 4, 2, seed=3, dt=p1.dt)
    h3 = rom.Rom.from_problem(p3)
    h3.set_reference(np.ones((128, 4)), None)
    with pytest.raises(RuntimeError):
        rom.run_rank3([h1, h3], V, S, None, 10)
    with pytest.raises(RuntimeError):
        rom.run_rank3([h1, h1], V, S, None, 10, prec="bf16s")
