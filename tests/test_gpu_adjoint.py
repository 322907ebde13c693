"""GPU parity of the reverse-time adjoint (rom_adjoint) against the FP64
oracle adjoint, finite differences, and itself with / without checkpoints."""
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


@pytest.fixture(scope="module")
def rom():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_11742_gb300 import build
    build.build()
    from paper_2009_11742_gb300 import rom as R
    return R


def case(Kv, Ks, M, R, N, seed, x0=0.2):
    p = inputs.make_problem(Kv, Ks, M, R, seed=seed)
    Z1, Z2 = np.zeros((Kv, M)), np.zeros((Ks, M))
    _, _, ystar = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z1, Z2, N,
                                 T=1.05 * p.T.astype(np.float64), r=1)
    V0 = inputs.random_state(Kv, M, seed=seed + 1, scale=x0)
    S0 = inputs.random_state(Ks, M, seed=seed + 2, scale=x0)
    return p, V0, S0, ystar.astype(np.float32)


def gpu_adjoint(R, h, p, V0, S0, ystar, N, ckpt):
    M = V0.shape[1]
    V0t = R.Rom.new_state(p.Kv, M, "fp32", fill=V0)
    S0t = R.Rom.new_state(p.Ks, M, "fp32", fill=S0)
    T = torch.as_tensor(p.T, device="cuda")
    ys = torch.as_tensor(np.ascontiguousarray(np.transpose(ystar, (0, 2, 1))), device="cuda")
    loss, gV, gS, gT = R.adjoint(h, V0t, S0t, T, ys, N, ckpt_every=ckpt)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    return loss, gV.cpu().numpy(), gS.cpu().numpy(), gT.cpu().numpy()


@pytest.mark.parametrize("Kv,Ks,M,R,N,ckpt", [(64, 64, 7, 3, 60, 0), (64, 64, 7, 3, 60, 16),
                                               (200, 180, 20, 5, 100, 32), (512, 512, 9, 8, 40, 7)])
def test_adjoint_vs_oracle(rom, Kv, Ks, M, R, N, ckpt):
    p, V0, S0, ystar = case(Kv, Ks, M, R, N, seed=Kv + M)
    h = rom.Rom.from_problem(p)
    loss, gV, gS, gT = gpu_adjoint(rom, h, p, V0, S0, ystar, N, ckpt)
    Lo, gVo, gSo, gTo = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, p.T, N, ystar)
    assert abs(loss - Lo) <= 1e-4 * abs(Lo)
    assert rel(gV, gVo) <= 1e-4 and rel(gS, gSo) <= 1e-4 and rel(gT, gTo) <= 1e-4


def test_checkpointed_equals_stored_traces_bitwise(rom):
    """Recomputed segments reproduce the forward sweep bit for bit, so the
    gradients do not depend on the checkpoint interval.  The FP64 misfit is
    summed per segment with atomic adds, so only its last bits may differ."""
    p, V0, S0, ystar = case(128, 128, 16, 4, 90, seed=5)
    h = rom.Rom.from_problem(p)
    a = gpu_adjoint(rom, h, p, V0, S0, ystar, 90, 0)
    b = gpu_adjoint(rom, h, p, V0, S0, ystar, 90, 20)
    assert abs(a[0] - b[0]) <= 1e-13 * abs(a[0])
    for x, y in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(x, y)


def test_autograd_function(rom):
    p, V0, S0, ystar = case(64, 64, 5, 2, 40, seed=9)
    h = rom.Rom.from_problem(p)
    V0t = rom.Rom.new_state(64, 5, "fp32", fill=V0).requires_grad_(True)
    S0t = rom.Rom.new_state(64, 5, "fp32", fill=S0).requires_grad_(True)
    T = torch.as_tensor(p.T, device="cuda").requires_grad_(True)
    ys = torch.as_tensor(np.ascontiguousarray(np.transpose(ystar, (0, 2, 1))), device="cuda")
    L = rom.rom_loss(h, V0t, S0t, T, ys, 40)
    (3.0 * L).backward()
    loss, gV, gS, gT = gpu_adjoint(rom, h, p, V0, S0, ystar, 40, 0)
    assert abs(L.item() - loss) <= 1e-12 * abs(loss)
    np.testing.assert_allclose(V0t.grad.cpu().numpy(), 3.0 * gV, rtol=1e-6)
    np.testing.assert_allclose(S0t.grad.cpu().numpy(), 3.0 * gS, rtol=1e-6)
    np.testing.assert_allclose(T.grad.cpu().numpy(), 3.0 * gT, rtol=1e-6)


def test_period_gradient_vs_gpu_finite_difference(rom):
    """dL/dT_m against central differences (h = 1e-3) of the GPU misfit."""
    p, V0, S0, ystar = case(96, 96, 4, 4, 150, seed=13, x0=0.0)
    h = rom.Rom.from_problem(p)
    _, _, _, gT = gpu_adjoint(rom, h, p, V0, S0, ystar, 150, 0)
    step = 1e-3
    for m in (0, 3):
        Tp = p.T.astype(np.float64).copy()
        Tm = Tp.copy()
        Tp[m] += step
        Tm[m] -= step
        Lp = gpu_adjoint(rom, h, _with_T(p, Tp), V0, S0, ystar, 150, 0)[0]
        Lm = gpu_adjoint(rom, h, _with_T(p, Tm), V0, S0, ystar, 150, 0)[0]
        fd = (Lp - Lm) / (2 * step)
        assert abs(fd - gT[m]) <= 2e-3 * abs(gT[m]), (fd, gT[m])


def _with_T(p, T):
    import copy
    q = copy.copy(p)
    q.T = np.asarray(T, np.float32)
    return q


def test_adjoint_workload4_full_size_sampled(rom):
    """Workload 4: K = 512, M = 128, 4000 steps, R = 64, checkpoints every 64
    steps.  Targets come from the oracle at T* = 1.05 T for a sample of
    columns (zero elsewhere; the misfit is a sum over columns, so each
    column's gradient depends on its own target only)."""
    p = inputs.config(4)
    N = 4000
    cols = np.array([0, 77, 127])
    Z = np.zeros((512, len(cols)))
    T_s = p.T.astype(np.float64)[cols]
    _, _, ys_s = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, N, T=1.05 * T_s, r=1)
    ystar = np.zeros((N, 64, 128), np.float32)
    ystar[:, :, cols] = ys_s
    h = rom.Rom.from_problem(p)
    V0 = np.zeros((512, 128), np.float32)
    loss, gV, gS, gT = gpu_adjoint(rom, h, p, V0, V0, ystar, N, 64)
    Lo, gVo, gSo, gTo = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, T_s, N,
                                       ys_s.astype(np.float32))
    assert rel(gV[:, cols], gVo) <= 1e-4
    assert rel(gS[:, cols], gSo) <= 1e-4
    assert rel(gT[cols], gTo) <= 1e-4
