"""GPU parity of the tensor-core (tcgen05) rank-2 path against the FP64 oracle.

Accepted (held to the FP32 bar, relative L2 <= 1e-4, Eq. (errors), Sec. 4.4,
over the full horizon): the exact sliced-integer BF16 scheme (bf16s), which
rounds nowhere inside the tensor core.  It is held to 1e-5 on short runs and
to 1e-4 over workload 2's 20000 steps.

Reported, not accepted: TF32x3, BF16x3 and plain BF16.  Their term splits
are accurate enough in exact arithmetic (a numpy emulation of the TF32x3 and
BF16x3 splits with exact sums stays within 5e-7 and 8e-6 of the oracle over
200 steps), but the tensor core's FP32 accumulation truncates, which biases
every product toward zero; over workload 2's 20000 steps TF32x3 then ends
about 1e-3 from the oracle.  Here they get short-run checks only: TF32x3
still meets 1e-4 on short runs; BF16x3 and BF16 get sanity bounds, as a
reported path does.
"""
import numpy as np
import pytest

import oracle
from paper_2009_11742_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# bars against the FP64 oracle on short runs: bf16s (accepted) and tf32x3;
# sanity bounds for the reported-only bf16x3 and bf16
TOL = {"tf32x3": 1e-4, "bf16x3": 1e-3, "bf16": 5e-2, "bf16s": 1e-5}


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


def run_tc(R, h, p, V0, S0, N, prec, r=0, n0=0, ftab=None, comp=None):
    M = V0.shape[1]
    V = R.Rom.new_state(p.Kv, M, "fp32", fill=V0)
    S = R.Rom.new_state(p.Ks, M, "fp32", fill=S0)
    T = torch.as_tensor(p.T, dtype=torch.float32, device="cuda") if ftab is None else None
    ft = None if ftab is None else torch.as_tensor(ftab, dtype=torch.float32, device="cuda").contiguous()
    nrec = N // r if (r and p.R) else 0
    tr = torch.zeros((nrec, M, p.R), dtype=torch.float32, device="cuda") if nrec else None
    h.run_rank2(V, S, T, N, n0=n0, r=r if nrec else 0, traces=tr, prec=prec, ftab=ft)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    return V.cpu().numpy(), S.cpu().numpy(), (None if tr is None else tr.transpose(1, 2).cpu().numpy())


SMALL_CASES = [(128, 128, 64, 4, 200, 10),   # one-CTA cluster
               (200, 180, 100, 8, 150, 6),   # ragged rows, 2 blocks
               (64, 64, 5, 2, 120, 4),       # K < 128, M < 64
               (384, 384, 70, 16, 100, 5)]   # 3-CTA cluster


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "bf16", "bf16s"])
@pytest.mark.parametrize("Kv,Ks,M,R,N,r", SMALL_CASES)
def test_tc_small_vs_oracle(rom, prec, Kv, Ks, M, R, N, r):
    p = inputs.make_problem(Kv, Ks, M, R, seed=Kv + M + 1)
    h = rom.Rom.from_problem(p)
    V0 = inputs.random_state(Kv, M, seed=3, scale=0.1)
    S0 = inputs.random_state(Ks, M, seed=4, scale=0.1)
    V, S, tr = run_tc(rom, h, p, V0, S0, N, prec, r=r, n0=2)
    Vo, So, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, N, T=p.T, n0=2, r=r)
    errs = (rel(V, Vo), rel(S, So), rel(tr, tro))
    assert max(errs) <= TOL[prec], errs


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "bf16", "bf16s"])
@pytest.mark.parametrize("Kv,Ks,M,R,N,r", [(1, 1, 1, 1, 100, 1),       # K = 1, M = 1: one padded tile, one column
                                           (256, 130, 33, 0, 90, 0),   # no receivers, Ks < Kv
                                           (130, 256, 129, 3, 60, 60),  # Kv < Ks, one column past two blocks, one record
                                           (256, 256, 48, 100, 40, 5)])  # R > 64: traces from global V
def test_tc_edge_shapes_vs_oracle(rom, prec, Kv, Ks, M, R, N, r):
    p = inputs.make_problem(Kv, Ks, M, R, seed=Kv + 2 * M + 5)
    h = rom.Rom.from_problem(p)
    V0 = inputs.random_state(Kv, M, seed=5, scale=0.1)
    S0 = inputs.random_state(Ks, M, seed=6, scale=0.1)
    V, S, tr = run_tc(rom, h, p, V0, S0, N, prec, r=r)
    Vo, So, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C if R else None, p.dt, V0, S0, N, T=p.T, r=r)
    errs = [rel(V, Vo), rel(S, So)]
    if R:
        errs.append(rel(tr, tro))
    else:
        assert tr is None and tro is None
    tol = TOL[prec]
    if prec == "bf16" and Kv == 1:
        # plain BF16 is reported, not held to a bar: with a 1 x 1 operator no
        # sum over K averages the 2^-9 rounding of the single entry, which
        # shifts the oscillator's frequency by up to 0.2 % (about 0.1 rad of
        # phase over 100 steps of 0.5 rad).  Checked instead against the
        # scheme's own arithmetic: operator and multiplied state rounded to
        # BF16, everything else in FP64.
        tol = 0.5
        bf = lambda x: torch.as_tensor(np.float32(x)).to(torch.bfloat16).double().numpy()
        a, b, g0 = bf(p.Asv[0, 0]), bf(p.Avs[0, 0]), float(p.g[0])
        v, sv = V0[0].astype(np.float64), S0[0].astype(np.float64)
        for n in range(N):
            f = oracle.ricker(np.full(M, n * p.dt), p.T)[0]
            v = v + p.dt * (b * bf(sv) + g0 * f)
            sv = sv + p.dt * (a * bf(v))
        assert rel(V[0], v) <= 1e-4 and rel(S[0], sv) <= 1e-4
    assert max(errs) <= tol, errs


@pytest.mark.parametrize("cols", [64, 128])
def test_tc_k1024_tf32x3(rom, cols):
    """K = 1024 (8-CTA clusters, the workload-2 operator size) over a short run,
    for each block width."""
    p = inputs.make_problem(1024, 1024, 96, 16, seed=7)
    h = rom.Rom.from_problem(p)
    assert rom.rom_set_tc_columns(h.h, cols) == rom.ROM_OK
    Z = np.zeros((1024, 96))
    V, S, tr = run_tc(rom, h, p, Z, Z, 120, "tf32x3", r=10)
    Vo, So, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, 120, T=p.T, r=10)
    assert colmax_rel(V, Vo) <= 1e-4 and colmax_rel(S, So) <= 1e-4 and colmax_rel(tr, tro) <= 1e-4


def test_tc_zero_in_zero_out(rom):
    p = inputs.make_problem(256, 256, 64, 4, seed=8)
    h = rom.Rom.from_problem(p)
    Z = np.zeros((256, 64))
    for prec in ("tf32x3", "bf16x3", "bf16", "bf16s"):
        V, S, tr = run_tc(rom, h, p, Z, Z, 50, prec, r=5, ftab=np.zeros((50, 64)))
        assert not V.any() and not S.any() and not tr.any()


@pytest.mark.parametrize("prec", ["tf32x3", "bf16s"])
def test_tc_chunked_is_bitwise_equal(rom, prec):
    """n0 plus the Kahan carries make chunked tensor-core runs bit-identical
    (for bf16s the column scales depend only on the state, so a restart
    slices the state exactly as the uninterrupted run does)."""
    p = inputs.make_problem(256, 256, 64, 4, seed=9)
    h = rom.Rom.from_problem(p)
    T = torch.as_tensor(p.T, device="cuda")

    def st():
        return [rom.Rom.new_state(256, 64, "fp32") for _ in range(4)]
    V, S, cV, cS = st()
    h.run_rank2(V, S, T, 100, prec=prec, compV=cV, compS=cS)
    V2, S2, cV2, cS2 = st()
    h.run_rank2(V2, S2, T, 40, n0=0, prec=prec, compV=cV2, compS=cS2)
    h.run_rank2(V2, S2, T, 60, n0=40, prec=prec, compV=cV2, compS=cS2)
    torch.cuda.synchronize()
    assert torch.equal(V, V2) and torch.equal(S, S2)


@pytest.mark.parametrize("cols", [32, 48, 64, 80])
def test_bf16s_k1024_every_width(rom, cols):
    """K = 1024 (8-CTA clusters, the split T1 accumulators) for every block
    width of the sliced scheme, with a ragged last block and random state."""
    p = inputs.make_problem(1024, 1000, 150, 16, seed=17)
    h = rom.Rom.from_problem(p)
    assert rom.rom_set_tc_columns(h.h, cols) == rom.ROM_OK
    V0 = inputs.random_state(1024, 150, seed=5, scale=0.3)
    S0 = inputs.random_state(1000, 150, seed=6, scale=0.3)
    V, S, tr = run_tc(rom, h, p, V0, S0, 150, "bf16s", r=10, n0=7)
    Vo, So, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, 150, T=p.T, n0=7, r=10)
    errs = (rel(V, Vo), rel(S, So), rel(tr, tro))
    assert max(errs) <= 1e-5, errs


def test_bf16s_scales_span_many_binades(rom):
    """Columns whose magnitudes differ by 2^40 keep their own column scale:
    each column is as accurate as if it ran alone."""
    p = inputs.make_problem(256, 256, 48, 4, seed=21)
    h = rom.Rom.from_problem(p)
    colscale = 2.0 ** np.linspace(-20, 20, 48)
    V0 = inputs.random_state(256, 48, seed=8, scale=1.0) * colscale
    S0 = inputs.random_state(256, 48, seed=9, scale=1.0) * colscale
    ft = np.zeros((80, 48))
    V, S, _ = run_tc(rom, h, p, V0.astype(np.float32), S0.astype(np.float32), 80, "bf16s", ftab=ft)
    Vo, So, _ = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0.astype(np.float32), S0.astype(np.float32),
                               80, ftab=ft)
    for m in (0, 24, 47):
        assert rel(V[:, m], Vo[:, m]) <= 1e-5 and rel(S[:, m], So[:, m]) <= 1e-5


def test_bf16s_config2_full_size_sampled(rom):
    """Workload 2 at full size with the exact sliced-integer scheme: the
    FP32 bar (relative L2 <= 1e-4) over all 20000 steps."""
    p = inputs.workload(2)
    h = rom.Rom.from_problem(p)
    Z = np.zeros((1024, 1024))
    V, S, tr = run_tc(rom, h, p, Z, Z, 20000, "bf16s", r=10)
    # block edges of the planner's 80-column blocks, the ragged tail and a
    # seeded draw; every column is held to the bar on its own
    rng = np.random.default_rng(2)
    cols = np.unique(np.concatenate([[0, 79, 80, 511, 959, 960, 1000, 1023],
                                     rng.choice(1024, 8, replace=False)]))
    Vo, So, tro = oracle.problem_forward(p, nsteps=20000, r=10, columns=cols)
    errs = (colmax_rel(V[:, cols], Vo), colmax_rel(S[:, cols], So), colmax_rel(tr[:, :, cols], tro))
    assert max(errs) <= 1e-4, errs
    assert np.all(np.isfinite(V))
