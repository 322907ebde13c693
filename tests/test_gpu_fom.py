"""GPU parity of the rank-2 full-order model (rom_fom_*; Sec. 3, Eq.
(fom_asym), App. A material) against the FP64 oracle (oracle/fom_oracle.c),
run one realization at a time."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = oracle.FOM_APP_A


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


def stable_dt(Nr, Nt):
    """dt = 0.5 / rho(L) of the probed oracle operators (L = [[0, A], [B, 0]])."""
    nv, n1, n2 = oracle.fom_dims(Nr, Nt)
    ns = n1 + n2
    V, _, _, _ = oracle.fom_forward(Nr, Nt, np.zeros((nv, ns)), np.eye(ns)[:n1], np.eye(ns)[n1:], 1, dt=1.0)
    _, S1, S2, _ = oracle.fom_forward(Nr, Nt, np.eye(nv), np.zeros((n1, nv)), np.zeros((n2, nv)), 1, dt=1.0)
    AB = V @ np.vstack([S1, S2])
    return 0.5 / np.sqrt(np.max(np.abs(np.linalg.eigvals(AB))))


def case(Nr, Nt, M, seed):
    nv, n1, n2 = oracle.fom_dims(Nr, Nt)
    rng = np.random.default_rng(seed)
    mu = P["rho"] * P["vs"] ** 2
    return (0.01 * rng.standard_normal((nv, M)), 0.01 * mu / P["vs"] * rng.standard_normal((n1, M)),
            0.01 * mu / P["vs"] * rng.standard_normal((n2, M)))


def gpu_run(rom, f, X0, N, prec, src=-1, T=None, recv=None, r=0, n0=0, wavelet=1):
    dt = torch.float64 if prec == "fp64" else torch.float32
    V, S1, S2 = (torch.as_tensor(np.ascontiguousarray(x), dtype=dt, device="cuda") for x in X0)
    Tt = None if T is None else torch.as_tensor(np.asarray(T), dtype=dt, device="cuda")
    rc = None if recv is None else torch.as_tensor(np.asarray(recv, np.int32), device="cuda")
    tr = None
    if recv is not None:
        tr = torch.zeros((N // r, len(recv), V.shape[1]), dtype=dt, device="cuda")
    f.run(V, S1, S2, N, src=src, T=Tt, wavelet=wavelet, recv=rc, r=r, traces=tr, prec=prec, n0=n0)
    torch.cuda.synchronize()
    return (V.cpu().numpy(), S1.cpu().numpy(), S2.cpu().numpy(),
            None if tr is None else tr.cpu().numpy())


@pytest.mark.parametrize("prec,tol,passes", [("fp64", 1e-12, 1), ("fp32", 1e-4, 1),
                                             ("fp64", 1e-12, 2), ("fp32", 1e-4, 2)])
def test_fom_vs_oracle(rom, prec, tol, passes):
    Nr, Nt, M, N, r = 24, 40, 5, 300, 7
    dt = stable_dt(Nr, Nt)
    f = rom.Fom(Nr, Nt, dt=dt)
    f.set_passes(passes)
    X0 = case(Nr, Nt, M, seed=1)
    T = np.linspace(60.0, 80.0, M)
    src = f.source_index(P["src_depth"], j=Nt // 3)
    recv = [f.vindex(Nr - 1, j) for j in (1, Nt // 3, Nt // 2, Nt - 1)]
    V, S1, S2, tr = gpu_run(rom, f, X0, N, prec, src=src, T=T, recv=recv, r=r)
    Vo, S1o, S2o, tro = oracle.fom_forward(Nr, Nt, *X0, N, src=src, T=T, wavelet=1, recv=recv, r=r, dt=dt)
    errs = [rel(V, Vo), rel(S1, S1o), rel(S2, S2o), rel(tr, tro)]
    print(prec, passes, "rel errors V/S1/S2/traces", errs)
    assert max(errs) <= tol, errs
    assert rel(Vo, X0[0]) > 0.1  # the run moved the state


@pytest.mark.parametrize("passes", [1, 2])
def test_fom_smallest_grid(rom, passes):
    """Nr = 2, Ntheta = 3: one sigma_rp face, one sigma_tp column, both
    velocity columns next to the axis."""
    Nr, Nt, M, N = 2, 3, 3, 200
    dt = stable_dt(Nr, Nt)
    f = rom.Fom(Nr, Nt, dt=dt)
    f.set_passes(passes)
    X0 = case(Nr, Nt, M, seed=5)
    T = np.array([60.0, 70.0, 80.0])
    V, S1, S2, _ = gpu_run(rom, f, X0, N, "fp64", src=1, T=T)
    Vo, S1o, S2o, _ = oracle.fom_forward(Nr, Nt, *X0, N, src=1, T=T, wavelet=1, dt=dt)
    assert rel(V, Vo) <= 1e-12 and rel(S1, S1o) <= 1e-12 and rel(S2, S2o) <= 1e-12


def test_fom_app_a_setup(rom):
    """The App. A setup on a 64 x 256 grid: rho 2500, vs 5000, dt 0.05 s,
    a source 640 km deep next to the axis, the first derivative of a
    Gaussian with periods in (60, 80) s and delay 1.5 T, 1000 FP32 steps from
    rest starting at t = 60 s (the pulse falls inside the run), receivers
    around the source; the fused pass against the oracle."""
    Nr, Nt, M, N, r, n0 = 64, 256, 4, 1000, 10, 1200
    f = rom.Fom(Nr, Nt)
    src = f.source_index(P["src_depth"], j=1)
    i_s = src // (Nt - 1)
    recv = [f.vindex(i, j) for i in (i_s - 3, i_s, i_s + 3) for j in (1, 4, 12)]
    T = np.random.default_rng(6).uniform(60.0, 80.0, M)
    nv, n1, n2 = f.nv, f.n1, f.n2
    X0 = (np.zeros((nv, M)), np.zeros((n1, M)), np.zeros((n2, M)))
    V, S1, S2, tr = gpu_run(rom, f, X0, N, "fp32", src=src, T=T, recv=recv, r=r, n0=n0)
    Vo, S1o, S2o, tro = oracle.fom_forward(Nr, Nt, *X0, N, src=src, T=T, wavelet=1, recv=recv, r=r,
                                           n0=n0, dt=P["dt"])
    errs = [rel(V, Vo), rel(S1, S1o), rel(S2, S2o), rel(tr, tro)]
    print("App. A setup rel errors V/S1/S2/traces", errs)
    assert max(errs) <= 1e-4, errs
    assert np.abs(Vo).max() > 0


def test_fom_rank2_equals_rank1_bitwise(rom):
    """Each realization's arithmetic does not depend on M: column m of a
    rank-2 run equals the single-realization run bitwise."""
    Nr, Nt, M, N = 16, 28, 4, 150
    f = rom.Fom(Nr, Nt, dt=stable_dt(Nr, Nt))
    X0 = case(Nr, Nt, M, seed=2)
    T = np.array([61.0, 65.0, 72.0, 79.0])
    src = f.source_index(P["src_depth"], j=3)
    V, S1, S2, _ = gpu_run(rom, f, X0, N, "fp32", src=src, T=T)
    for m in (0, 3):
        Xm = tuple(x[:, m:m + 1] for x in X0)
        v, s1, s2, _ = gpu_run(rom, f, Xm, N, "fp32", src=src, T=T[m:m + 1])
        assert np.array_equal(v[:, 0], V[:, m]) and np.array_equal(s1[:, 0], S1[:, m])
        assert np.array_equal(s2[:, 0], S2[:, m])


@pytest.mark.parametrize("passes", [1, 2])
def test_fom_chunked_equals_one_run_and_zero(rom, passes):
    """n0 continues the forcing clock: 71 + 129 steps equal 200 steps
    bitwise (the 64-step graph is replayed with steps past the end idle; an
    odd count ends in the fused pass's second buffer set and is copied
    back); zero state without forcing stays exactly zero."""
    Nr, Nt, M = 12, 20, 3
    f = rom.Fom(Nr, Nt, dt=stable_dt(Nr, Nt))
    f.set_passes(passes)
    X0 = case(Nr, Nt, M, seed=3)
    T = np.array([60.0, 70.0, 80.0])
    src = f.source_index(P["src_depth"], j=2)
    full = gpu_run(rom, f, X0, 200, "fp64", src=src, T=T)
    a = gpu_run(rom, f, X0, 71, "fp64", src=src, T=T)
    b = gpu_run(rom, f, a[:3], 129, "fp64", src=src, T=T, n0=71)
    for k in range(3):
        assert np.array_equal(full[k], b[k])
    nv, n1, n2 = f.nv, f.n1, f.n2
    z = gpu_run(rom, f, (np.zeros((nv, M)), np.zeros((n1, M)), np.zeros((n2, M))), 100, "fp32")
    assert not any(x.any() for x in z[:3])


def test_fom_fused_equals_two_passes(rom):
    """The fused pass computes the two passes' arithmetic (its halo values
    are recomputed by the same expressions): equal to FP32 rounding, on a
    grid with ragged strips and segments and the source in a halo column."""
    Nr, Nt, M, N = 45, 70, 32, 120
    f = rom.Fom(Nr, Nt, dt=stable_dt(20, 30) * 0.25)
    X0 = case(Nr, Nt, M, seed=4)
    T = np.linspace(60.0, 80.0, M)
    src = f.vindex(31, 32)  # halo column of strip 0 and recomputed row of segment 1
    outs = []
    for passes in (1, 2):
        f.set_passes(passes)
        outs.append(gpu_run(rom, f, X0, N, "fp32", src=src, T=T, recv=[src, f.vindex(Nr - 1, 5)], r=3))
    for k in range(4):
        assert rel(outs[0][k], outs[1][k]) <= 1e-6, k


def test_fom_rejects_bad_arguments(rom):
    f = rom.Fom(8, 12)
    V, S1, S2 = f.new_state(2)
    with pytest.raises(RuntimeError):
        f.run(V, S1, S2, 10, prec="bf16s")
    with pytest.raises(RuntimeError):
        f.run(V, S1, S2, 10, src=f.nv, T=torch.ones(2, device="cuda"))
    Vh, S1h, S2h = (x.cpu() for x in (V, S1, S2))
    with pytest.raises(RuntimeError):
        f.run(Vh, S1h, S2h, 10)
    with pytest.raises(RuntimeError):
        rom.Fom(1, 12)
    with pytest.raises(RuntimeError):
        f.set_passes(3)


def test_fom_full_size_sampled(rom):
    """The benchmark's grid and launch (512 x 2048, 3.14 M unknowns, M = 32,
    FP32 fused pass, the source 640 km deep next to the axis, 64 surface
    receivers every 10 steps), from a random state with the forcing clock at
    the pulse (n0 = 1700 steps = 85 s): realizations 0 and 31 against the
    oracle over 300 steps."""
    Nr, Nt, M, N, r, n0 = 512, 2048, 32, 300, 10, 1700
    f = rom.Fom(Nr, Nt)
    src = f.source_index(P["src_depth"], j=1)
    recv = [f.vindex(Nr - 1, int(j)) for j in np.linspace(1, Nt - 1, 64).astype(int)]
    X0 = case(Nr, Nt, M, seed=8)
    T = np.random.default_rng(9).uniform(60.0, 80.0, M)
    V, S1, S2, tr = gpu_run(rom, f, X0, N, "fp32", src=src, T=T, recv=recv, r=r, n0=n0)
    cols = [0, M - 1]
    Vo, S1o, S2o, tro = oracle.fom_forward(Nr, Nt, *(x[:, cols] for x in X0), N, src=src, T=T[cols],
                                           wavelet=1, recv=recv, r=r, n0=n0, dt=P["dt"])
    errs = [rel(V[:, cols], Vo), rel(S1[:, cols], S1o), rel(S2[:, cols], S2o), rel(tr[:, :, cols], tro)]
    print("full-size FOM rel errors V/S1/S2/traces", errs)
    assert max(errs) <= 1e-4, errs
    assert rel(Vo, X0[0][:, cols]) > 1e-3  # the run moved the state
