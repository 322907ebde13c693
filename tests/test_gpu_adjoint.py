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
                                               (200, 180, 20, 5, 100, 32), (512, 512, 9, 8, 40, 7),
                                               # one receiver, more receivers than rows per CTA, and
                                               # more than K (the source term in chunks of 64)
                                               (128, 96, 5, 1, 30, 0), (256, 256, 10, 100, 30, 8),
                                               (128, 128, 6, 300, 20, 0),
                                               # above K = 512: two 32-row tiles per CTA, the
                                               # transposed operators read from L2
                                               (640, 600, 11, 5, 36, 0), (1024, 1000, 6, 8, 40, 16),
                                               (1000, 1024, 17, 3, 25, 9),
                                               # enough columns for the planner to take clusters
                                               # of 4: 22 row tiles dealt 6, 6, 5, 5
                                               (704, 680, 256, 8, 20, 0)])
def test_adjoint_vs_oracle(rom, Kv, Ks, M, R, N, ckpt):
    p, V0, S0, ystar = case(Kv, Ks, M, R, N, seed=Kv + M)
    h = rom.Rom.from_problem(p)
    loss, gV, gS, gT = gpu_adjoint(rom, h, p, V0, S0, ystar, N, ckpt)
    Lo, gVo, gSo, gTo = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, p.T, N, ystar)
    assert abs(loss - Lo) <= 1e-4 * abs(Lo)
    assert colmax_rel(gV, gVo) <= 1e-4 and colmax_rel(gS, gSo) <= 1e-4 and rel(gT, gTo) <= 1e-4


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


def test_source_ranges_do_not_change_the_gradients(rom):
    """K = 1024, M = 300: the precomputed source term of one launch range is
    capped at 64 MB, so every trace kept (c = 0) runs ranges of 54, 54 and 12
    steps while c = 40 runs ranges of 40; the gradients are bitwise equal."""
    Kv = Ks = 1024
    M, R, N = 300, 8, 120
    p = inputs.make_problem(Kv, Ks, M, R, seed=13)
    V0 = inputs.random_state(Kv, M, seed=14, scale=0.2)
    S0 = inputs.random_state(Ks, M, seed=15, scale=0.2)
    ystar = inputs.random_state(N * R, M, seed=16, scale=0.1).reshape(N, R, M)
    h = rom.Rom.from_problem(p)
    a = gpu_adjoint(rom, h, p, V0, S0, ystar, N, 0)
    b = gpu_adjoint(rom, h, p, V0, S0, ystar, N, 40)
    assert np.isfinite(a[0]) and a[0] > 0
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


def test_gradients_vs_fp64_finite_differences_workload4_shape(rom):
    """Workload-4 shapes (K = 512, R = 64, a record every step, checkpoints
    every 64 steps) on four sampled realizations over 300 steps, from a seeded
    nonzero start.  The GPU adjoint's dL/dT_m and its gradients w.r.t. V0 and
    S0, projected on seeded random directions, are held to 1e-4 relative of
    central differences (h = 1e-3) of the misfit that the FP64 oracle's
    forward run gives.  The misfit is quadratic in (V0, S0), so those
    differences are exact up to rounding; for T the difference quotient's own
    error is O(h^2), far below the bar."""
    p = inputs.workload(4)
    N, K = 300, 512
    cols = np.array([0, 41, 77, 127])
    M = len(cols)
    T = p.T.astype(np.float64)[cols]
    Z = np.zeros((K, M))
    _, _, ys = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, N, T=1.05 * T, r=1)
    ystar = ys.astype(np.float32)
    ys64 = ystar.astype(np.float64)
    V0 = inputs.random_state(K, M, seed=41, scale=0.05).astype(np.float32).astype(np.float64)
    S0 = inputs.random_state(K, M, seed=42, scale=0.05).astype(np.float32).astype(np.float64)
    h = rom.Rom.from_problem(p)
    loss, gV, gS, gT = gpu_adjoint(rom, h, _with_T(p, T), V0, S0, ystar, N, 64)

    def misfit(V0_, S0_, T_):
        _, _, tr = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0_, S0_, N, T=T_, r=1)
        return float(np.sum((tr - ys64) ** 2))

    L0 = misfit(V0, S0, T)
    assert abs(loss - L0) <= 1e-4 * L0
    step = 1e-3
    for m in range(M):
        Tp, Tm = T.copy(), T.copy()
        Tp[m] += step
        Tm[m] -= step
        fd = (misfit(V0, S0, Tp) - misfit(V0, S0, Tm)) / (2 * step)
        assert abs(gT[m] - fd) <= 1e-4 * abs(fd), (m, gT[m], fd)
    rng = np.random.default_rng(7)
    for _ in range(2):
        D = rng.standard_normal((K, M))
        fdV = (misfit(V0 + step * D, S0, T) - misfit(V0 - step * D, S0, T)) / (2 * step)
        fdS = (misfit(V0, S0 + step * D, T) - misfit(V0, S0 - step * D, T)) / (2 * step)
        assert abs(float(np.sum(gV * D)) - fdV) <= 1e-4 * abs(fdV), (np.sum(gV * D), fdV)
        assert abs(float(np.sum(gS * D)) - fdS) <= 1e-4 * abs(fdS), (np.sum(gS * D), fdS)


def test_gradients_vs_fp64_finite_differences_k1024(rom):
    """K = 1024 (the largest size rom_create takes): dL/dT_m and the V0, S0
    gradients along a random direction against central differences of the
    FP64 oracle's misfit, at 1e-4 relative."""
    Kv = Ks = 1024
    M, R, N = 3, 8, 60
    p = inputs.make_problem(Kv, Ks, M, R, seed=77)
    T = p.T.astype(np.float64)
    Z = np.zeros((Kv, M))
    _, _, ys = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, N, T=1.05 * T, r=1)
    ystar = ys.astype(np.float32)
    ys64 = ystar.astype(np.float64)
    V0 = inputs.random_state(Kv, M, seed=5, scale=0.05).astype(np.float32).astype(np.float64)
    S0 = inputs.random_state(Ks, M, seed=6, scale=0.05).astype(np.float32).astype(np.float64)
    h = rom.Rom.from_problem(p)
    loss, gV, gS, gT = gpu_adjoint(rom, h, p, V0, S0, ystar, N, 16)

    def misfit(V0_, S0_, T_):
        _, _, tr = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0_, S0_, N, T=T_, r=1)
        return float(np.sum((tr - ys64) ** 2))

    step = 1e-3
    for m in range(M):
        Tp, Tm = T.copy(), T.copy()
        Tp[m] += step
        Tm[m] -= step
        fd = (misfit(V0, S0, Tp) - misfit(V0, S0, Tm)) / (2 * step)
        assert abs(gT[m] - fd) <= 1e-4 * abs(fd), (m, gT[m], fd)
    D = np.random.default_rng(8).standard_normal((Kv, M))
    fdV = (misfit(V0 + step * D, S0, T) - misfit(V0 - step * D, S0, T)) / (2 * step)
    fdS = (misfit(V0, S0 + step * D, T) - misfit(V0, S0 - step * D, T)) / (2 * step)
    assert abs(float(np.sum(gV * D)) - fdV) <= 1e-4 * abs(fdV)
    assert abs(float(np.sum(gS * D)) - fdS) <= 1e-4 * abs(fdS)


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
    p = inputs.workload(4)
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
    assert colmax_rel(gV[:, cols], gVo) <= 1e-4
    assert colmax_rel(gS[:, cols], gSo) <= 1e-4
    assert np.max(np.abs(gT[cols] - gTo) / np.abs(gTo)) <= 1e-4


# ---------------------------------------------------------------- FP64 path

def gpu_adjoint64(R, h, p, V0, S0, ystar, N, ckpt, T=None):
    M = V0.shape[1]
    V0t = R.Rom.new_state(p.Kv, M, "fp64", fill=V0)
    S0t = R.Rom.new_state(p.Ks, M, "fp64", fill=S0)
    Tt = torch.as_tensor(np.asarray(p.T if T is None else T, np.float64), device="cuda")
    ys = torch.as_tensor(np.ascontiguousarray(np.transpose(ystar, (0, 2, 1))), dtype=torch.float64,
                         device="cuda")
    loss, gV, gS, gT = R.adjoint(h, V0t, S0t, Tt, ys, N, ckpt_every=ckpt)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    assert gV.dtype == torch.float64 and gT.dtype == torch.float64
    return loss, gV.cpu().numpy(), gS.cpu().numpy(), gT.cpu().numpy()


@pytest.mark.parametrize("Kv,Ks,M,R,N,ckpt", [(64, 64, 7, 3, 60, 0), (200, 180, 20, 5, 100, 32),
                                               # Kp = 320 and 512: the FP64 kernel reads the
                                               # transposed operators from L2 every half-step
                                               (320, 300, 9, 4, 50, 16), (512, 512, 9, 8, 40, 7)])
def test_adjoint_fp64_vs_oracle(rom, Kv, Ks, M, R, N, ckpt):
    """The FP64 reverse sweep against the FP64 oracle adjoint: the two differ
    only in summation order, so they agree to 1e-10 relative."""
    p, V0, S0, ystar = case(Kv, Ks, M, R, N, seed=Kv + M + 1)
    V0 = V0.astype(np.float64)
    S0 = S0.astype(np.float64)
    ys64 = ystar.astype(np.float64)
    h = rom.Rom.from_problem(p)
    T = p.T.astype(np.float64)
    loss, gV, gS, gT = gpu_adjoint64(rom, h, p, V0, S0, ys64, N, ckpt, T=T)
    Lo, gVo, gSo, gTo = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, T, N, ys64)
    assert abs(loss - Lo) <= 1e-10 * abs(Lo)
    assert colmax_rel(gV, gVo) <= 1e-10 and colmax_rel(gS, gSo) <= 1e-10
    assert np.max(np.abs(gT - gTo) / np.abs(gTo)) <= 1e-10


def test_adjoint_fp64_vs_finite_differences(rom):
    """dL/dT_m and the V0, S0 gradients along random directions of the FP64
    path against central differences of the FP64 oracle's misfit, at 1e-6
    relative.  The state differences are exact up to rounding (the misfit is
    quadratic in V0, S0); the period differences' own error is O(h^2)."""
    Kv, Ks, M, R, N = 256, 240, 4, 6, 200
    p = inputs.make_problem(Kv, Ks, M, R, seed=91)
    T = p.T.astype(np.float64)
    _, _, ys = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, np.zeros((Kv, M)), np.zeros((Ks, M)), N,
                              T=1.05 * T, r=1)
    V0 = inputs.random_state(Kv, M, seed=92, scale=0.05).astype(np.float64)
    S0 = inputs.random_state(Ks, M, seed=93, scale=0.05).astype(np.float64)
    h = rom.Rom.from_problem(p)
    loss, gV, gS, gT = gpu_adjoint64(rom, h, p, V0, S0, ys, N, 32, T=T)

    def misfit(V0_, S0_, T_):
        _, _, tr = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0_, S0_, N, T=T_, r=1)
        return float(np.sum((tr - ys) ** 2))

    assert abs(loss - misfit(V0, S0, T)) <= 1e-12 * loss
    step = 1e-3
    for m in range(M):
        Tp, Tm = T.copy(), T.copy()
        Tp[m] += step
        Tm[m] -= step
        fd = (misfit(V0, S0, Tp) - misfit(V0, S0, Tm)) / (2 * step)
        assert abs(gT[m] - fd) <= 1e-6 * abs(fd), (m, gT[m], fd)
    rng = np.random.default_rng(94)
    for _ in range(2):
        DV = rng.standard_normal((Kv, M))
        DS = rng.standard_normal((Ks, M))
        fdV = (misfit(V0 + step * DV, S0, T) - misfit(V0 - step * DV, S0, T)) / (2 * step)
        fdS = (misfit(V0, S0 + step * DS, T) - misfit(V0, S0 - step * DS, T)) / (2 * step)
        assert abs(float(np.sum(gV * DV)) - fdV) <= 1e-6 * abs(fdV), (np.sum(gV * DV), fdV)
        assert abs(float(np.sum(gS * DS)) - fdS) <= 1e-6 * abs(fdS), (np.sum(gS * DS), fdS)


def test_adjoint_fp64_checkpoints_and_autograd(rom):
    """FP64: the gradients do not depend on the checkpoint interval (the
    recomputed segments repeat the forward sweep bit for bit), and the
    autograd function returns them for float64 leaves."""
    p, V0, S0, ystar = case(128, 128, 6, 4, 70, seed=17)
    V0 = V0.astype(np.float64)
    S0 = S0.astype(np.float64)
    ys64 = ystar.astype(np.float64)
    h = rom.Rom.from_problem(p)
    T = p.T.astype(np.float64)
    a = gpu_adjoint64(rom, h, p, V0, S0, ys64, 70, 0, T=T)
    b = gpu_adjoint64(rom, h, p, V0, S0, ys64, 70, 15, T=T)
    assert abs(a[0] - b[0]) <= 1e-13 * abs(a[0])
    for x, y in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(x, y)
    V0t = rom.Rom.new_state(128, 6, "fp64", fill=V0).requires_grad_(True)
    S0t = rom.Rom.new_state(128, 6, "fp64", fill=S0).requires_grad_(True)
    Tt = torch.as_tensor(T, device="cuda").requires_grad_(True)
    ys = torch.as_tensor(np.ascontiguousarray(np.transpose(ys64, (0, 2, 1))), device="cuda")
    L = rom.rom_loss(h, V0t, S0t, Tt, ys, 70)
    L.backward()
    np.testing.assert_array_equal(V0t.grad.cpu().numpy(), a[1])
    np.testing.assert_array_equal(S0t.grad.cpu().numpy(), a[2])
    np.testing.assert_array_equal(Tt.grad.cpu().numpy(), a[3])


@pytest.mark.parametrize("dtype", ["fp32", "fp64"])
def test_adjoint_caller_workspace(rom, dtype):
    """A caller-owned workspace of exactly rom_adjoint_workspace_size bytes
    (checkpoints, traces and one launch range's source term) gives the same
    gradients, bit for bit, as the library's own allocation (the loss to its
    last bits); one byte less is refused with ROM_E_INVAL."""
    Kv, Ks, M, R, N, ckpt = 192, 160, 9, 5, 150, 40
    p, V0, S0, ystar = case(Kv, Ks, M, R, N, seed=61)
    h = rom.Rom.from_problem(p)
    f64 = dtype == "fp64"
    tdt = torch.float64 if f64 else torch.float32
    ndt = np.float64 if f64 else np.float32
    V0t = rom.Rom.new_state(Kv, M, dtype, fill=V0.astype(ndt))
    S0t = rom.Rom.new_state(Ks, M, dtype, fill=S0.astype(ndt))
    T = torch.as_tensor(p.T.astype(ndt), device="cuda")
    ys = torch.as_tensor(np.ascontiguousarray(np.transpose(ystar.astype(ndt), (0, 2, 1))), device="cuda")
    ref = rom.adjoint(h, V0t, S0t, T, ys, N, ckpt_every=ckpt)
    prec = rom.ROM_FP64 if f64 else rom.ROM_FP32
    need = rom.rom_adjoint_workspace_size(h.h, M, N, ckpt, prec)
    assert need > 0
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    gV = rom.Rom.new_state(Kv, M, dtype)
    gS = rom.Rom.new_state(Ks, M, dtype)
    gT = torch.zeros(M, dtype=tdt, device="cuda")
    args = (h.h, V0t.data_ptr(), S0t.data_ptr(), T.data_ptr(), M, N, ys.data_ptr(), ckpt, gV.data_ptr(),
            gS.data_ptr(), gT.data_ptr())
    st, loss = rom.rom_adjoint(*args, ws.data_ptr(), need, prec, None)
    torch.cuda.synchronize()
    assert st == rom.ROM_OK and h.sync_status() == 0
    assert abs(loss - ref[0]) <= 1e-13 * abs(ref[0])  # the misfit's atomic sums
    for x, y in zip((gV, gS, gT), ref[1:]):
        np.testing.assert_array_equal(x.cpu().numpy(), y.cpu().numpy())
    st, _ = rom.rom_adjoint(*args, ws.data_ptr(), need - 1, prec, None)
    assert st == rom.ROM_E_INVAL


def test_adjoint_fp64_refuses_above_512(rom):
    p, V0, S0, ystar = case(576, 576, 2, 2, 5, seed=3)
    h = rom.Rom.from_problem(p)
    with pytest.raises(rom.RomError):
        gpu_adjoint64(rom, h, p, V0.astype(np.float64), S0.astype(np.float64),
                      ystar.astype(np.float64), 5, 0, T=p.T.astype(np.float64))


def test_adjoint_allocation_failure_is_reported(rom):
    """A workspace the GPU cannot hold (every trace of 10^7 steps kept:
    10^7 x 64 x 256 x 4 B = 655 GB) is refused with ROM_E_NOMEM before any
    kernel runs, and the next call on the same handle succeeds."""
    K, M, R = 64, 256, 64
    p, V0, S0, ystar = case(K, K, M, R, 10, seed=31)
    h = rom.Rom.from_problem(p)
    need = rom.rom_adjoint_workspace_size(h.h, M, 10 ** 7, 0, rom.ROM_FP32)
    assert need > 600 * 10 ** 9
    V0t = rom.Rom.new_state(K, M, "fp32", fill=V0)
    S0t = rom.Rom.new_state(K, M, "fp32", fill=S0)
    T = torch.as_tensor(p.T, device="cuda")
    ys = torch.zeros((10, M, R), device="cuda")  # never read: the allocation fails first
    gV = rom.Rom.new_state(K, M, "fp32")
    gS = rom.Rom.new_state(K, M, "fp32")
    gT = torch.zeros(M, device="cuda")
    st, _ = rom.rom_adjoint(h.h, V0t.data_ptr(), S0t.data_ptr(), T.data_ptr(), M, 10 ** 7,
                            ys.data_ptr(), 0, gV.data_ptr(), gS.data_ptr(), gT.data_ptr(), None, 0,
                            rom.ROM_FP32, None)
    assert st == rom.ROM_E_NOMEM
    loss, gV2, gS2, gT2 = gpu_adjoint(rom, h, p, V0, S0, ystar, 10, 0)
    Lo, gVo, _, _ = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, p.T, 10, ystar)
    assert abs(loss - Lo) <= 1e-4 * abs(Lo) and rel(gV2, gVo) <= 1e-4
