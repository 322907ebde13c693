"""GPU parity of rom_trace_stats (ensemble mean and quantile bands of the
receiver traces, Sec. 4.5.2) against the oracle's plain definition.  The
quantiles are bit-exact (a sort is exact and both sides interpolate with
the same FP64 operations); the FP64 means agree to summation-order rounding."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PS = [0.05, 0.5, 0.95, 0.0, 1.0, 0.3]


@pytest.fixture(scope="module")
def rom():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_11742_gb300 import build
    build.build()
    from paper_2009_11742_gb300 import rom as R
    return R


def check(R, x):
    t = torch.as_tensor(x, device="cuda")
    mean, q = R.trace_stats(t, PS)
    torch.cuda.synchronize()
    mo, qo = oracle.trace_stats(x, PS)
    np.testing.assert_array_equal(q.cpu().numpy(), qo)
    scale = np.abs(x.astype(np.float64)).mean(axis=1) + 1e-300
    assert np.all(np.abs(mean.cpu().numpy() - mo) <= 1e-13 * scale)


@pytest.mark.parametrize("nrec,M,R", [(3, 1, 2), (5, 2, 3), (7, 37, 5), (2, 512, 64), (4, 1000, 3),
                                      (1, 4096, 2)])
def test_stats_vs_oracle(rom, nrec, M, R):
    rng = np.random.default_rng(nrec * 1000 + M)
    check(rom, rng.standard_normal((nrec, M, R)).astype(np.float32))


def test_stats_with_ties_and_signed_zeros(rom):
    rng = np.random.default_rng(11)
    x = np.round(rng.standard_normal((6, 300, 4)) * 2).astype(np.float32) / 2
    x[:, ::7, :] = -0.0
    check(rom, x)


def test_stats_of_simulated_traces(rom):
    """Traces from a rank-2 run (the intended use)."""
    from paper_2009_11742_gb300 import inputs
    p = inputs.make_problem(96, 80, 200, 6, seed=3)
    h = rom.Rom.from_problem(p)
    V = rom.Rom.new_state(96, 200, "fp32")
    S = rom.Rom.new_state(80, 200, "fp32")
    T = torch.as_tensor(p.T, device="cuda")
    tr = torch.zeros((30, 200, 6), device="cuda")
    h.run_rank2(V, S, T, 300, r=10, traces=tr, prec="fp32")
    torch.cuda.synchronize()
    check(rom, tr.cpu().numpy())


def test_stats_argument_errors(rom):
    x = torch.zeros((2, 4, 3), device="cuda")
    mean = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    q = torch.zeros((1, 2, 3), dtype=torch.float64, device="cuda")
    E = rom.ROM_E_INVAL
    assert rom.rom_trace_stats(x.data_ptr(), 2, 3, 4097, [0.5], 1, mean.data_ptr(), q.data_ptr()) == E
    assert rom.rom_trace_stats(x.data_ptr(), 2, 3, 4, [1.5], 1, mean.data_ptr(), q.data_ptr()) == E
    assert rom.rom_trace_stats(x.data_ptr(), 0, 3, 4, [0.5], 1, mean.data_ptr(), q.data_ptr()) == E
    host = np.zeros(24, np.float32)
    assert rom.rom_trace_stats(host.ctypes.data, 2, 3, 4, [0.5], 1, mean.data_ptr(), q.data_ptr()) == E
    assert rom.rom_trace_stats(x.data_ptr(), 2, 3, 4, [0.5], 1, mean.data_ptr(), q.data_ptr()) == rom.ROM_OK
