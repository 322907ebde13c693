"""GPU parity of the streaming companion of the FP32 two-block kernel
(rom_set_companion): the last columns of a run integrated by clusters of 2 or
4 CTAs that stream their operator rows from L2, beside the two-block kernel.
Against the FP64 oracle (relative L2, Eq. (errors), Sec. 4.4; per column,
<= 1e-4, the FP32 bar); bitwise equal to the two-block kernel alone (the
companion does the same arithmetic in the same order); bitwise across chunked
runs with Kahan carries; and with the automatic plan of the benchmark's
workload."""
import numpy as np
import pytest

import oracle
from paper_2009_11742_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def colmax_rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    a = a.reshape(-1, a.shape[-1])
    b = b.reshape(-1, b.shape[-1])
    num = np.linalg.norm(a - b, axis=0)
    return float(np.max(num / np.maximum(np.linalg.norm(b, axis=0), 1e-300)))


@pytest.fixture(scope="module")
def rom():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_11742_gb300 import build
    build.build()
    from paper_2009_11742_gb300 import rom as R
    return R


def run(R, h, p, V0, S0, N, r=0, n0=0, ftab=None):
    M = V0.shape[1]
    V = R.Rom.new_state(p.Kv, M, "fp32", fill=V0)
    S = R.Rom.new_state(p.Ks, M, "fp32", fill=S0)
    T = torch.as_tensor(p.T, dtype=torch.float32, device="cuda") if ftab is None else None
    ft = None if ftab is None else torch.as_tensor(ftab, dtype=torch.float32, device="cuda").contiguous()
    nrec = N // r if (r and p.R) else 0
    tr = torch.zeros((nrec, M, p.R), dtype=torch.float32, device="cuda") if nrec else None
    h.run_rank2(V, S, T, N, n0=n0, r=r if nrec else 0, traces=tr, prec="fp32", ftab=ft)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    return V.cpu().numpy(), S.cpu().numpy(), (None if tr is None else tr.transpose(1, 2).cpu().numpy())


@pytest.mark.parametrize("csz", [2, 4])
@pytest.mark.parametrize("Kv,Ks,M,R,N,r,cols", [
    (512, 512, 19, 16, 120, 8, 5),     # K = 512: two 16-CTA clusters and 2 companion clusters
    (200, 180, 37, 6, 150, 7, 9),      # ragged rows (Kp = 256), 3 companion clusters
    (256, 256, 6, 3, 200, 10, 6),      # every column on the companion, one 64-row pass per CTA
    (512, 500, 40, 64, 90, 3, 13),     # Ks < Kv, ragged last companion cluster, many receivers
    # partial last 64-row pass: Kp = 448 owns 224 / 112 rows per CTA (3.5 /
    # 1.75 passes), Kp = 192 owns 96 / 48 (1.5 passes / one partial pass)
    (436, 417, 33, 8, 80, 4, 11),
    (192, 170, 21, 5, 100, 5, 9),
])
def test_companion_vs_oracle(rom, csz, Kv, Ks, M, R, N, r, cols):
    p = inputs.make_problem(Kv, Ks, M, R, seed=Kv + M + csz)
    h = rom.Rom.from_problem(p)
    h.set_companion(csz, cols)
    plan = h.plan(M)
    assert plan["variant"] == 4 and plan["companion"]["columns"] == cols
    assert plan["companion"]["cluster_size"] == csz
    V0 = inputs.random_state(Kv, M, seed=1, scale=0.1)
    S0 = inputs.random_state(Ks, M, seed=2, scale=0.1)
    V, S, tr = run(rom, h, p, V0, S0, N, r=r, n0=4)
    Vo, So, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, N, T=p.T, n0=4, r=r)
    assert colmax_rel(V, Vo) <= 1e-4 and colmax_rel(S, So) <= 1e-4
    assert colmax_rel(tr, tro) <= 1e-4


@pytest.mark.parametrize("csz", [2, 4])
@pytest.mark.parametrize("Kv", [512, 448])
def test_companion_bitwise_equals_two_block_kernel(rom, csz, Kv):
    """The companion's columns (state and traces) are bit for bit what the
    two-block kernel alone computes for them (Kp = 448: a partial last
    pass per CTA)."""
    M, N, r = 40, 150, 5
    p = inputs.make_problem(Kv, Kv, M, 64, seed=31)
    V0 = inputs.random_state(Kv, M, seed=1, scale=0.1)
    S0 = inputs.random_state(Kv, M, seed=2, scale=0.1)
    h = rom.Rom.from_problem(p)
    h.set_companion(-1, 0)
    Va, Sa, tra = run(rom, h, p, V0, S0, N, r=r, n0=3)
    h.set_companion(csz, 13)
    assert h.plan(M)["variant"] == 4
    Vb, Sb, trb = run(rom, h, p, V0, S0, N, r=r, n0=3)
    assert np.array_equal(Va, Vb) and np.array_equal(Sa, Sb) and np.array_equal(tra, trb)


def test_companion_forcing_table_and_zeros(rom):
    """Tabulated forcing (the dense mode of Sec. 2.2) on the companion's
    columns; zero forcing and zero state stay exactly zero."""
    Kv, M, N = 256, 12, 80
    p = inputs.make_problem(Kv, Kv, M, 4, seed=5)
    h = rom.Rom.from_problem(p)
    h.set_companion(2, 7)
    rng = np.random.default_rng(3)
    ft = rng.standard_normal((N, M)).astype(np.float32)
    Z = np.zeros((Kv, M), np.float32)
    V, S, tr = run(rom, h, p, Z, Z, N, r=5, ftab=ft)
    Vo, So, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, N, ftab=ft, r=5)
    assert colmax_rel(V, Vo) <= 1e-4 and colmax_rel(S, So) <= 1e-4 and colmax_rel(tr, tro) <= 1e-4
    V, S, tr = run(rom, h, p, Z, Z, N, r=5, ftab=np.zeros((N, M), np.float32))
    assert not V.any() and not S.any() and not tr.any()


@pytest.mark.parametrize("csz", [2, 4])
def test_companion_chunked_is_bitwise_equal(rom, csz):
    """n0 and the Kahan carries make a run split into chunks bit-identical to
    one run, on the companion's columns as on the main kernel's."""
    Kv, M = 512, 24
    p = inputs.make_problem(Kv, Kv, M, 4, seed=9)
    h = rom.Rom.from_problem(p)
    h.set_companion(csz, 8)
    T = torch.as_tensor(p.T, device="cuda")

    def st():
        return [rom.Rom.new_state(Kv, M, "fp32") for _ in range(4)]
    V, S, cV, cS = st()
    h.run_rank2(V, S, T, 100, prec="fp32", compV=cV, compS=cS)
    V2, S2, cV2, cS2 = st()
    h.run_rank2(V2, S2, T, 30, n0=0, prec="fp32", compV=cV2, compS=cS2)
    h.run_rank2(V2, S2, T, 70, n0=30, prec="fp32", compV=cV2, compS=cS2)
    torch.cuda.synchronize()
    assert torch.equal(V, V2) and torch.equal(S, S2)


def test_companion_with_reference_state_falls_back(rom):
    """With a reduced reference state the two-block kernel runs alone (the
    companion does not carry the term): results still meet the bar."""
    Kv, M, N = 512, 20, 100
    p = inputs.make_problem(Kv, Kv, M, 0, seed=11)
    rng = np.random.default_rng(4)
    Xv, Xs = 0.05 * rng.standard_normal((Kv, M)), 0.05 * rng.standard_normal((Kv, M))
    h = rom.Rom.from_problem(p)
    h.set_companion(2, 6)
    h.set_reference(Xv, Xs)
    V0 = inputs.random_state(Kv, M, seed=1, scale=0.1)
    V, S, _ = run(rom, h, p, V0, V0, N)
    Vo, So, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, V0, V0, N, T=p.T, xref=(Xv, Xs))
    assert colmax_rel(V, Vo) <= 1e-4 and colmax_rel(S, So) <= 1e-4


def test_companion_headline_workload_sampled(rom):
    """The benchmark's workload (K = 512, M = 256, 10000 steps, R = 64,
    r = 10) in the automatic plan; 24 sampled columns, among them every
    column the companion owns when the plan has one, each held to the bar."""
    p = inputs.workload(1)
    h = rom.Rom.from_problem(p)
    plan = h.plan(256)
    Z = np.zeros((512, 256), np.float32)
    V, S, tr = run(rom, h, p, Z, Z, 10000, r=10)
    comp = plan.get("companion", {}).get("columns", 0)
    rng = np.random.default_rng(6)
    cols = np.unique(np.concatenate([np.arange(256 - min(comp, 16), 256), [0, 100, 200],
                                     rng.choice(256, 8, replace=False)]))
    Vo, So, tro = oracle.problem_forward(p, nsteps=10000, r=10, columns=cols)
    assert colmax_rel(V[:, cols], Vo) <= 1e-4
    assert colmax_rel(S[:, cols], So) <= 1e-4
    assert colmax_rel(tr[:, :, cols], tro) <= 1e-4


def test_set_companion_rejects_bad_arguments(rom):
    p = inputs.make_problem(64, 64, 4, 0, seed=1)
    h = rom.Rom.from_problem(p)
    assert rom.rom_set_companion(h.h, 3, 4) == rom.ROM_E_INVAL
    assert rom.rom_set_companion(h.h, 2, 0) == rom.ROM_E_INVAL
    assert rom.rom_set_companion(h.h, -1, 0) == rom.ROM_OK
    assert h.plan(4)["variant"] != 4
