"""GPU parity of the batched many-ensemble launch (rom_run_batched) against
the FP64 oracle and against one-at-a-time rank-2 runs."""
import numpy as np
import pytest

import oracle
from paper_2009_11742_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def colmax_rel(a, b):
    """Largest per-column relative L2 error (columns are realizations)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
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


def make_jobs(R, sizes, with_traces, seed0=100):
    jobs, probs = [], []
    for i, (K, M, Rr) in enumerate(sizes):
        p = inputs.make_problem(K, K, M, Rr, seed=seed0 + i)
        h = R.Rom.from_problem(p)
        V = R.Rom.new_state(K, M, "fp32")
        S = R.Rom.new_state(K, M, "fp32")
        T = torch.as_tensor(p.T, device="cuda")
        tr = None
        if with_traces and Rr:
            tr = torch.zeros((with_traces, M, Rr), device="cuda")
        jobs.append((h, V, S, T, tr))
        probs.append(p)
    return jobs, probs


SIZES = [(64, 4, 2), (128, 17, 3), (200, 33, 0), (512, 64, 8), (576, 100, 4), (768, 5, 2),
         (320, 250, 0), (64, 256, 1)]


def test_batched_vs_oracle_and_individual(rom):
    N, r = 120, 10
    jobs, probs = make_jobs(rom, SIZES, with_traces=N // r)
    rom.run_batched(jobs, N, r=r, prec="fp32")
    torch.cuda.synchronize()
    for (h, V, S, T, tr), p in zip(jobs, probs):
        assert h.sync_status() == 0
        Z = np.zeros((p.Kv, p.M))
        Vo, So, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C if p.R else None, p.dt, Z, Z, N,
                                     T=p.T, r=r if p.R else 0)
        assert colmax_rel(V.cpu().numpy(), Vo) <= 1e-4 and colmax_rel(S.cpu().numpy(), So) <= 1e-4
        if tr is not None:
            # per realization m: every record of every receiver (oracle: nrec x R x M)
            trg = tr.transpose(1, 2).cpu().numpy().reshape(-1, p.M)
            assert colmax_rel(trg, np.asarray(tro).reshape(-1, p.M)) <= 1e-4
        # the same job alone through rom_run_rank2: the work-list kernel sums
        # in another order (32 k lanes, 4 rows a thread), so the two FP32
        # results agree to rounding, column by column
        V1 = rom.Rom.new_state(p.Kv, p.M, "fp32")
        S1 = rom.Rom.new_state(p.Ks, p.M, "fp32")
        h.run_rank2(V1, S1, T, N, prec="fp32")
        torch.cuda.synchronize()
        assert colmax_rel(V.cpu().numpy(), V1.cpu().numpy()) <= 2e-5
        assert colmax_rel(S.cpu().numpy(), S1.cpu().numpy()) <= 2e-5


@pytest.mark.parametrize("form", [None, (4, 16), (8, 64), (2, 8), (0, 0)])
def test_batched_worklist_edge_cases(rom, form):
    """The work-list launch on the cases its layout branches on, in the
    default form (clusters of 2, width cap 32) and pinned ones:
    - a one-column job at Kp = 1024, and ragged K (1000 -> Kp = 1024);
    - receiver rows too many to stage in shared memory (K = 640, R = 48:
      24 rows of C per CTA of a pair, 61 KB, read from L2);
    - Kp = 576 (18 row tiles: 5, 5, 4, 4 over a cluster of 4, and 3 or 2
      over one of 8), Kp = 320 (10 tiles: 3, 3, 2, 2 over 4);
    - Kp = 64 (2 tiles: over a cluster of 4 or 8 most CTAs own none);
    - (0, 0): one launch per job.
    Every column of state and traces is held to the FP64 oracle."""
    sizes = [(1024, 1, 3), (1000, 9, 40), (640, 20, 48), (576, 13, 5), (320, 30, 6), (64, 3, 0)]
    N, r = 40, 4
    jobs, probs = make_jobs(rom, sizes, with_traces=N // r, seed0=400)
    if form is not None:
        rom.set_batched_form(jobs, *form)
    rom.run_batched(jobs, N, r=r, prec="fp32")
    torch.cuda.synchronize()
    for (h, V, S, T, tr), p in zip(jobs, probs):
        assert h.sync_status() == 0
        Z = np.zeros((p.Kv, p.M))
        Vo, So, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C if p.R else None, p.dt, Z, Z, N,
                                     T=p.T, r=r if p.R else 0)
        assert colmax_rel(V.cpu().numpy(), Vo) <= 1e-4 and colmax_rel(S.cpu().numpy(), So) <= 1e-4
        if tr is not None:
            trg = tr.transpose(1, 2).cpu().numpy().reshape(-1, p.M)
            assert colmax_rel(trg, np.asarray(tro).reshape(-1, p.M)) <= 1e-4


@pytest.mark.parametrize("form", [None, (0, 0)])
def test_batched_nonfinite_job_flags_its_own_handle(rom, form):
    """A job whose state holds a NaN ends non-finite and its handle reports
    ROM_E_NONFINITE; the other jobs of the same launch (work list or one
    launch per job) are untouched and meet the oracle."""
    sizes = [(192, 24, 0), (640, 16, 0), (320, 40, 0)]
    jobs, probs = make_jobs(rom, sizes, with_traces=0, seed0=500)
    jobs[1][1][5, 3] = float("nan")
    if form is not None:
        rom.set_batched_form(jobs, *form)
    N = 30
    rom.run_batched(jobs, N, prec="fp32")
    torch.cuda.synchronize()
    for k, ((h, V, S, T, _), p) in enumerate(zip(jobs, probs)):
        if k == 1:
            assert h.sync_status() == rom.ROM_E_NONFINITE
            continue
        assert h.sync_status() == 0
        Z = np.zeros((p.Kv, p.M))
        Vo, So, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, Z, Z, N, T=p.T)
        assert colmax_rel(V.cpu().numpy(), Vo) <= 1e-4 and colmax_rel(S.cpu().numpy(), So) <= 1e-4


def test_batched_graph_replay(rom):
    """The second call replays the cached graph: the state advances by
    another nsteps (forcing restarts at t = 0 for every call)."""
    sizes = [(96, 10, 0), (256, 40, 0), (640, 12, 0)]
    jobs, probs = make_jobs(rom, sizes, with_traces=0, seed0=200)
    N = 80
    rom.run_batched(jobs, N, prec="fp32")
    rom.run_batched(jobs, N, prec="fp32")
    torch.cuda.synchronize()
    for (h, V, S, T, _), p in zip(jobs, probs):
        Z = np.zeros((p.Kv, p.M))
        V1, S1, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, Z, Z, N, T=p.T)
        V2, S2, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, V1, S1, N, T=p.T)
        assert colmax_rel(V.cpu().numpy(), V2) <= 1e-4 and colmax_rel(S.cpu().numpy(), S2) <= 1e-4


def test_batched_rejects_bad_jobs(rom):
    jobs, _ = make_jobs(rom, [(64, 4, 0), (64, 4, 0)], with_traces=0, seed0=300)
    dup = [jobs[0], jobs[0]]
    with pytest.raises(rom.RomError):
        rom.run_batched(dup, 10, prec="fp32")
    for bad in [(3, 32), (2, 12), (2, 0), (4, 264), (16, 32), (-2, 32)]:
        with pytest.raises(rom.RomError):
            rom.set_batched_form(jobs, *bad)
    with pytest.raises(rom.RomError):
        rom.set_batched_form(jobs, 2, 32, prec="fp64")


def test_batched_workload3_full_size_sampled(rom):
    """Workload 3: 64 ROMs, K_i in {64..768}, M_i in [4, 256], 5000 steps, one
    graph launch; the oracle recomputes the first, middle and last column of
    every fourth ROM, each column held to the bar on its own."""
    probs = inputs.batched_problems()
    jobs = []
    for p in probs:
        h = rom.Rom.from_problem(p)
        jobs.append((h, rom.Rom.new_state(p.Kv, p.M, "fp32"), rom.Rom.new_state(p.Ks, p.M, "fp32"),
                     torch.as_tensor(p.T, device="cuda"), None))
    rom.run_batched(jobs, 5000, prec="fp32")
    torch.cuda.synchronize()
    for i in range(0, 64, 4):
        h, V, S, T, _ = jobs[i]
        p = probs[i]
        cols = np.unique([0, p.M // 2, p.M - 1])
        Vo, So, _ = oracle.problem_forward(p, nsteps=5000, r=0, columns=cols)
        assert colmax_rel(V.cpu().numpy()[:, cols], Vo) <= 1e-4
        assert colmax_rel(S.cpu().numpy()[:, cols], So) <= 1e-4


def test_autotune_batched_keeps_results(rom):
    """The measured schedule changes only how the SMs are shared: every job's
    result stays within FP32 rounding of the untuned schedule."""
    probs = inputs.batched_problems()[:12]
    items = []
    for p in probs:
        h = rom.Rom.from_problem(p)
        items.append((h, rom.Rom.new_state(p.Kv, p.M, "fp32"), rom.Rom.new_state(p.Ks, p.M, "fp32"),
                      torch.as_tensor(p.T, device="cuda"), None))
    rom.run_batched(items, 300)
    torch.cuda.synchronize()
    ref = [(V.cpu().numpy(), S.cpu().numpy()) for (_, V, S, _, _) in items]
    us = rom.autotune_batched(items, probe_steps=50)
    assert us > 0
    for (_, V, S, _, _) in items:
        V.zero_()
        S.zero_()
    rom.run_batched(items, 300)
    torch.cuda.synchronize()
    for (Vr, Sr), (_, V, S, _, _) in zip(ref, items):
        v = V.cpu().numpy()
        assert np.linalg.norm(v - Vr) <= 1e-5 * np.linalg.norm(Vr)


def test_autotune_single_handle(rom):
    p = inputs.make_problem(512, 512, 256, 8, seed=2)
    h = rom.Rom.from_problem(p)
    T = torch.as_tensor(p.T, device="cuda")
    V1, S1 = rom.Rom.new_state(512, 256, "fp32"), rom.Rom.new_state(512, 256, "fp32")
    h.run_rank2(V1, S1, T, 200, prec="fp32")
    us = h.autotune(256, "fp32", probe_steps=100)
    assert us > 0
    V2, S2 = rom.Rom.new_state(512, 256, "fp32"), rom.Rom.new_state(512, 256, "fp32")
    h.run_rank2(V2, S2, T, 200, prec="fp32")
    torch.cuda.synchronize()
    a, b = V1.cpu().numpy(), V2.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(a)
    us_tc = h.autotune(256, "bf16s", probe_steps=50)
    assert us_tc > 0
    V3, S3 = rom.Rom.new_state(512, 256, "fp32"), rom.Rom.new_state(512, 256, "fp32")
    h.run_rank2(V3, S3, T, 200, prec="bf16s")
    torch.cuda.synchronize()
    assert np.linalg.norm(V3.cpu().numpy() - a) <= 1e-4 * np.linalg.norm(a)


def test_autotune_single_handle_above_512(rom):
    """K = 768: the planner picks clusters of 4 or 2 for the streamed
    operators; the tuner, which also times that plan, keeps one of the
    one-block cluster sizes, and its result holds the sampled columns to the
    oracle."""
    K, M, N = 768, 256, 120
    p = inputs.make_problem(K, K, M, 8, seed=21)
    h = rom.Rom.from_problem(p)
    T = torch.as_tensor(p.T, device="cuda")
    planned = h.plan(M)
    us = h.autotune(M, "fp32", probe_steps=100)
    assert us > 0
    tuned = h.plan(M)
    assert tuned["cluster_size"] in (2, 4, K // 64)
    V, S = rom.Rom.new_state(K, M, "fp32"), rom.Rom.new_state(K, M, "fp32")
    h.run_rank2(V, S, T, N, prec="fp32")
    torch.cuda.synchronize()
    cols = np.array([0, 100, 255])
    Vo, So, _ = oracle.problem_forward(p, nsteps=N, r=0, columns=cols)
    assert colmax_rel(V.cpu().numpy()[:, cols], Vo) <= 1e-4
    assert colmax_rel(S.cpu().numpy()[:, cols], So) <= 1e-4
    assert planned["cluster_size"] in (2, 4)  # the model's choice at this size


def test_batched_auto_precision(rom):
    """prec="auto": jobs with max(Kv, Ks) >= 256 take the exact-slice BF16
    tensor-core path, the others FP32; every result meets the FP32 bar
    against the oracle and equals the job run alone at its chosen precision
    bitwise.  After the threshold is tuned the results still meet the bar."""
    N, r = 120, 10
    jobs, probs = make_jobs(rom, SIZES, with_traces=N // r, seed0=400)
    rom.run_batched(jobs, N, r=r, prec="auto")
    torch.cuda.synchronize()
    chosen = set()
    for (h, V, S, T, tr), p in zip(jobs, probs):
        assert h.sync_status() == 0
        Z = np.zeros((p.Kv, p.M))
        Vo, So, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C if p.R else None, p.dt, Z, Z, N,
                                     T=p.T, r=r if p.R else 0)
        assert colmax_rel(V.cpu().numpy(), Vo) <= 1e-4 and colmax_rel(S.cpu().numpy(), So) <= 1e-4
        if tr is not None:
            assert colmax_rel(tr.transpose(1, 2).cpu().numpy(), tro) <= 1e-4
        prec = "bf16s" if max(p.Kv, p.Ks) >= 256 else "fp32"
        chosen.add(prec)
        V1 = rom.Rom.new_state(p.Kv, p.M, "fp32")
        S1 = rom.Rom.new_state(p.Ks, p.M, "fp32")
        h.run_rank2(V1, S1, T, N, prec=prec)
        torch.cuda.synchronize()
        assert torch.equal(V1, V) and torch.equal(S1, S), prec
    assert chosen == {"fp32", "bf16s"}
    us = rom.autotune_batched(jobs, prec="auto", probe_steps=50)
    assert us > 0
    for (_, V, S, _, _) in jobs:
        V.zero_()
        S.zero_()
    rom.run_batched([(h, V, S, T, None) for (h, V, S, T, _) in jobs], N, prec="auto")
    torch.cuda.synchronize()
    for (h, V, S, T, _), p in zip(jobs, probs):
        Z = np.zeros((p.Kv, p.M))
        Vo, So, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, Z, Z, N, T=p.T)
        assert colmax_rel(V.cpu().numpy(), Vo) <= 1e-4 and colmax_rel(S.cpu().numpy(), So) <= 1e-4


def test_destroyed_handles_leave_no_tuned_schedule(rom):
    """rom_destroy forgets the graphs and the tuned schedules of every job
    list that names the handle: a new list (whose handles may reuse the
    freed addresses) plans afresh and meets the bar."""
    sizes = [(128, 20, 0), (320, 40, 0), (512, 16, 0)]
    jobs, _ = make_jobs(rom, sizes, with_traces=0, seed0=500)
    rom.autotune_batched(jobs, prec="auto", probe_steps=20)
    rom.run_batched(jobs, 30, prec="auto")
    torch.cuda.synchronize()
    for (h, _, _, _, _) in jobs:
        h.close()
    del jobs
    jobs2, probs2 = make_jobs(rom, sizes, with_traces=0, seed0=510)
    N = 60
    rom.run_batched(jobs2, N, prec="auto")
    torch.cuda.synchronize()
    for (h, V, S, T, _), p in zip(jobs2, probs2):
        Z = np.zeros((p.Kv, p.M))
        Vo, So, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, Z, Z, N, T=p.T)
        assert colmax_rel(V.cpu().numpy(), Vo) <= 1e-4 and colmax_rel(S.cpu().numpy(), So) <= 1e-4
