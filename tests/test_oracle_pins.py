"""Pins for the FP64 oracle: each test checks it against something the
mathematics fixes, not against a re-typed copy of its own formulas.

Paper passages: leapfrog, velocity first then stress (Sec. 3.1); reduced
model Eq. (shwave_rom_ode_tensor); rank-2 == M rank-1 runs (Sec. 2.4, 4.4);
LTI superposition (Sec. 1, 2); zero initial state (Sec. 3.1); symplectic,
time-reversible integrator (Sec. 3.1); stable dt (Sec. 4.4, App. A).
"""
import numpy as np
import pytest

import oracle
from paper_2009_11742_gb300 import inputs


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ---------------------------------------------------------------- Ricker --
def test_ricker_special_points():
    """Ricker wavelet (Sec. 3.2) at points fixed by its shape:
    f = 1 at the peak t = t0 = 1.5 T; f = 0 where u = pi^2 tau^2/T^2 = 1/2;
    the side lobes reach -2 e^{-3/2} at u = 3/2; f is even in tau."""
    T = np.array([7.0, 13.25, 30.0])
    t0 = 1.5 * T
    f, _ = oracle.ricker(t0, T)
    assert np.all(f == 1.0)
    tau0 = T / (np.pi * np.sqrt(2.0))
    f0p, _ = oracle.ricker(t0 + tau0, T)
    f0m, _ = oracle.ricker(t0 - tau0, T)
    assert np.max(np.abs(f0p)) < 1e-15 and np.max(np.abs(f0m)) < 1e-15
    tau1 = T * np.sqrt(1.5) / np.pi
    fm, _ = oracle.ricker(t0 + tau1, T)
    np.testing.assert_allclose(fm, -2.0 * np.exp(-1.5), rtol=1e-14)
    # it is the minimum: neighbours are larger
    fa, _ = oracle.ricker(t0 + tau1 * (1 + 1e-3), T)
    fb, _ = oracle.ricker(t0 + tau1 * (1 - 1e-3), T)
    assert np.all(fa > fm) and np.all(fb > fm)
    x = np.linspace(-3, 3, 41)
    fp, _ = oracle.ricker(t0[1] + x, T[1])
    fn, _ = oracle.ricker(t0[1] - x, T[1])
    np.testing.assert_array_equal(fp, fn)


def test_ricker_dT_matches_finite_difference():
    """df/dT (used by the adjoint) against a central difference of f."""
    rng = np.random.default_rng(3)
    T = rng.uniform(5, 20, 200)
    t = rng.uniform(0, 60, 200)
    _, d = oracle.ricker(t, T)
    h = 1e-5
    fp, _ = oracle.ricker(t, T + h)
    fm, _ = oracle.ricker(t, T - h)
    fd = (fp - fm) / (2 * h)
    np.testing.assert_allclose(d, fd, rtol=1e-6, atol=1e-9)


# -------------------------------------------------------- closed forms --
def amplification(Avs, Asv, g, dt):
    """One leapfrog step as X^{n+1} = G X^n + b f_n with X = [V; S]:
    G = [[I, dt Avs], [dt Asv, I + dt^2 Asv Avs]], b = [dt g; dt^2 Asv g]."""
    Avs = Avs.astype(np.float64)
    Asv = Asv.astype(np.float64)
    Kv, Ks = Avs.shape
    G = np.block([[np.eye(Kv), dt * Avs],
                  [dt * Asv, np.eye(Ks) + dt * dt * Asv @ Avs]])
    b = np.concatenate([dt * g, dt * dt * Asv @ g]).astype(np.float64)
    return G, b


def eig_solution(G, b, X0, ftab):
    """X^N = G^N X0 + sum_{n<N} G^{N-1-n} b f_n via G = P diag(lam) P^{-1}."""
    lam, P = np.linalg.eig(G)
    Pinv = np.linalg.inv(P)
    N = ftab.shape[0]
    Y0 = Pinv @ X0.astype(np.complex128)
    bb = Pinv @ b.astype(np.complex128)
    powN = lam[:, None] ** N
    out = powN * Y0
    # sum_n lam^{N-1-n} f_n  per eigenvalue and column
    e = np.arange(N)[::-1]
    W = lam[:, None] ** e[None, :]  # (2K, N)
    out = out + bb[:, None] * (W @ ftab)
    return (P @ out).real


@pytest.mark.parametrize("K,M,N,skew", [(1, 2, 300, True), (4, 3, 400, True),
                                        (8, 5, 500, True), (6, 2, 300, False),
                                        (3, 4, 200, False)])
def test_closed_form_eig(K, M, N, skew):
    """Oracle vs. the diagonalised amplification matrix (forced, nonzero X0)."""
    rng = np.random.default_rng(100 + K)
    p = inputs.make_problem(K, K, M, 0, seed=K)
    Avs, Asv = p.Avs.astype(np.float64), p.Asv.astype(np.float64)
    if not skew:
        # an independent Avs, scaled so the scheme stays stable
        Avs = -0.5 * (Asv.T + 0.3 * rng.standard_normal((K, K)) / np.sqrt(K))
    dt = p.dt
    V0 = rng.standard_normal((K, M))
    S0 = rng.standard_normal((K, M))
    ftab = rng.standard_normal((N, M))
    V, S, _ = oracle.forward(Avs, Asv, p.g, None, dt, V0, S0, N, ftab=ftab)
    G, b = amplification(Avs, Asv, p.g.astype(np.float64), dt)
    assert np.max(np.abs(np.linalg.eigvals(G))) < 1 + 1e-9 or not skew
    X = eig_solution(G, b, np.vstack([V0, S0]), ftab)
    assert rel(np.vstack([V, S]), X) < 1e-10


def _xref_case(Kv, Ks, M, seed):
    rng = np.random.default_rng(seed)
    p = inputs.make_problem(Kv, Ks, M, 0, seed=seed)
    Xv = rng.standard_normal((Kv, M))
    Xs = rng.standard_normal((Ks, M))
    return p, rng, Xv, Xs


@pytest.mark.parametrize("Kv,Ks,M,N", [(1, 1, 2, 300), (5, 4, 3, 250), (8, 8, 2, 400)])
def test_reference_state_closed_form(Kv, Ks, M, N):
    """Reduced reference state (Eq. (rom_ode_tensor)): a constant term per
    column in both halves.  With it one step is X^{n+1} = G X^n + b f_n + h,
    h = [dt Xv; dt^2 Asv Xv + dt Xs], so X^N = G^N X0 + sum_n G^{N-1-n} b f_n
    + (sum_{i<N} G^i) h.  The last sum is taken per eigenvalue of G."""
    p, rng, Xv, Xs = _xref_case(Kv, Ks, M, 60 + Kv)
    Avs, Asv, dt = p.Avs.astype(np.float64), p.Asv.astype(np.float64), p.dt
    V0 = rng.standard_normal((Kv, M))
    S0 = rng.standard_normal((Ks, M))
    ftab = rng.standard_normal((N, M))
    V, S, _ = oracle.forward(Avs, Asv, p.g, None, dt, V0, S0, N, ftab=ftab, xref=(Xv, Xs))
    G, b = amplification(Avs, Asv, p.g.astype(np.float64), dt)
    X = eig_solution(G, b, np.vstack([V0, S0]), ftab)
    H = np.vstack([dt * Xv, dt * dt * Asv @ Xv + dt * Xs])
    lam, P = np.linalg.eig(G)
    geo = (lam[:, None] ** np.arange(N)[None, :]).sum(axis=1)  # sum_{i<N} lam^i
    X = X + (P @ (geo[:, None] * (np.linalg.inv(P) @ H.astype(np.complex128)))).real
    assert rel(np.vstack([V, S]), X) < 1e-10


def test_reference_state_fixed_point():
    """With Xv = -Avs S* and Xs = -Asv V*, (V*, S*) is a fixed point of the
    unforced step: the state must not move (to FP64 rounding)."""
    Kv, Ks, M = 40, 32, 3
    p, rng, _, _ = _xref_case(Kv, Ks, M, 71)
    Vs = rng.standard_normal((Kv, M))
    Ss = rng.standard_normal((Ks, M))
    Xv = -p.Avs.astype(np.float64) @ Ss
    Xs = -p.Asv.astype(np.float64) @ Vs
    V, S, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, Vs, Ss, 500, xref=(Xv, Xs))
    assert rel(V, Vs) < 1e-13 and rel(S, Ss) < 1e-13
    # one of the two terms alone moves it
    V1, S1, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, Vs, Ss, 5, xref=(Xv, None))
    assert rel(np.vstack([V1, S1]), np.vstack([Vs, Ss])) > 1e-6


def test_reference_state_time_reversal_and_superposition():
    """The step with the constant term stays reversible, and the response is
    linear: Run(X0, f, Xref) = Run(X0, f, 0) + Run(0, 0, Xref)."""
    Kv, Ks, M, N = 24, 20, 3, 300
    p, rng, Xv, Xs = _xref_case(Kv, Ks, M, 72)
    V0 = rng.standard_normal((Kv, M))
    S0 = rng.standard_normal((Ks, M))
    T = p.T.astype(np.float64)
    V, S, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, V0, S0, N, T=T, xref=(Xv, Xs))
    Vb, Sb = oracle.inverse(p.Avs, p.Asv, p.g, p.dt, V, S, N, T=T, xref=(Xv, Xs))
    assert rel(Vb, V0) < 1e-10 and rel(Sb, S0) < 1e-10
    Va, Sa, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, V0, S0, N, T=T)
    Vr, Sr, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, np.zeros((Kv, M)),
                               np.zeros((Ks, M)), N, xref=(Xv, Xs))
    assert rel(V, Va + Vr) < 1e-12 and rel(S, Sa + Sr) < 1e-12


def test_k1_textbook_oscillator():
    """K = 1 with Avs = -a/dt, Asv = a/dt: the step matrix is
    G = [[1, -a], [a, 1 - a^2]] (det 1, cos theta = 1 - a^2/2) and
    G^n = sin(n th)/sin(th) G - sin((n-1) th)/sin(th) I (Cayley-Hamilton)."""
    dt = 0.1
    for a in (0.05, 0.7, 1.9):
        Avs = np.array([[-a / dt]])
        Asv = np.array([[a / dt]])
        th = np.arccos(1 - a * a / 2)
        G = np.array([[1.0, -a], [a, 1 - a * a]])
        x0 = np.array([1.0, 0.3])
        for n in (1, 2, 17, 1000):
            Gn = np.sin(n * th) / np.sin(th) * G - np.sin((n - 1) * th) / np.sin(th) * np.eye(2)
            V, S, _ = oracle.forward(Avs, Asv, np.zeros(1), None, dt,
                                     x0[:1, None], x0[1:, None], n)
            np.testing.assert_allclose([V[0, 0], S[0, 0]], Gn @ x0, rtol=1e-11, atol=1e-11)


def svd_chebyshev_solution(Asv, dt, V0, S0, N):
    """Skew case Avs = -Asv^T: with Asv = U diag(s) W^T, p = W^T V and
    q = U^T S decouple into scalar oscillators with a_j = dt s_j."""
    U, s, Wt = np.linalg.svd(Asv.astype(np.float64))
    p = Wt @ V0
    q = U.T @ S0
    a = dt * s
    th = np.arccos(1 - a * a / 2)
    c1 = np.sin(N * th) / np.sin(th)
    c0 = np.sin((N - 1) * th) / np.sin(th)
    pN = (c1 - c0)[:, None] * p + (-a * c1)[:, None] * q
    qN = (a * c1)[:, None] * p + (c1 * (1 - a * a) - c0)[:, None] * q
    return Wt.T @ pN, U @ qN


def test_closed_form_svd_k32():
    """Unforced skew system at K = 32 against the SVD/Chebyshev solution."""
    p = inputs.make_problem(32, 32, 4, 0, seed=5)
    rng = np.random.default_rng(9)
    V0 = rng.standard_normal((32, 4))
    S0 = rng.standard_normal((32, 4))
    N = 700
    V, S, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, V0, S0, N)
    Ve, Se = svd_chebyshev_solution(p.Asv, p.dt, V0, S0, N)
    assert rel(V, Ve) < 1e-10 and rel(S, Se) < 1e-10


# ----------------------------------------------------------- invariants --
def test_energy_exactly_conserved():
    """Unforced skew leapfrog conserves ||V||^2 + ||S||^2 - dt <S, Asv V>
    to roundoff over 1000 steps at K = 128 (workload-0 operator)."""
    p = inputs.workload(0)
    V0 = inputs.random_state(128, 4, seed=1).astype(np.float64)
    S0 = inputs.random_state(128, 4, seed=2).astype(np.float64)
    E0 = oracle.energy(p.Asv, p.dt, V0, S0)
    V, S, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, V0, S0, 1000)
    E1 = oracle.energy(p.Asv, p.dt, V, S)
    assert abs(E1 - E0) / E0 <= 1e-12
    # and it is not trivially conserved: the plain norm moves
    n0 = np.sum(V0 ** 2) + np.sum(S0 ** 2)
    n1 = np.sum(V ** 2) + np.sum(S ** 2)
    assert abs(n1 - n0) / n0 > 1e-6


def test_zero_in_zero_out():
    """Zero initial state with zero forcing stays exactly zero (Sec. 3.1)."""
    p = inputs.make_problem(16, 12, 5, 3, seed=4)
    Z = np.zeros((16, 5)), np.zeros((12, 5))
    V, S, tr = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z[0], Z[1], 50,
                              ftab=np.zeros((50, 5)), r=5)
    assert not V.any() and not S.any() and not tr.any()


def test_superposition():
    """LTI: Run(X0, f1 + f2) = Run(X0, f1) + Run(0, f2), and linear in g."""
    p = inputs.make_problem(24, 20, 3, 4, seed=6)
    rng = np.random.default_rng(11)
    V0 = rng.standard_normal((24, 3))
    S0 = rng.standard_normal((20, 3))
    f1 = rng.standard_normal((120, 3))
    f2 = rng.standard_normal((120, 3))
    Va, Sa, ta = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, 120, ftab=f1 + f2, r=7)
    Vb, Sb, tb = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, 120, ftab=f1, r=7)
    Vc, Sc, tc = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, 0 * V0, 0 * S0, 120, ftab=f2, r=7)
    assert rel(Va, Vb + Vc) < 1e-13 and rel(Sa, Sb + Sc) < 1e-13 and rel(ta, tb + tc) < 1e-13
    g2 = rng.standard_normal(24)
    Z = np.zeros((24, 3)), np.zeros((20, 3))
    V1, S1, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, *Z, 80, T=p.T)
    V2, S2, _ = oracle.forward(p.Avs, p.Asv, g2, None, p.dt, *Z, 80, T=p.T)
    V3, S3, _ = oracle.forward(p.Avs, p.Asv, p.g + g2, None, p.dt, *Z, 80, T=p.T)
    assert rel(V3, V1 + V2) < 1e-13 and rel(S3, S1 + S2) < 1e-13


def test_time_reversal():
    """Leapfrog is time reversible (Sec. 3.1): N steps back recover X0."""
    p = inputs.make_problem(64, 48, 4, 0, seed=7)
    rng = np.random.default_rng(12)
    V0 = rng.standard_normal((64, 4))
    S0 = rng.standard_normal((48, 4))
    V, S, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, V0, S0, 500, T=p.T, n0=3)
    Vb, Sb = oracle.inverse(p.Avs, p.Asv, p.g, p.dt, V, S, 500, T=p.T, n0=3)
    assert rel(Vb, V0) < 1e-12 and rel(Sb, S0) < 1e-12


def test_forcing_modes_and_chunking_agree():
    """T-mode forcing equals a table of f(t_n; T_m) with t_n = (n0 + n) dt, and
    a run split in chunks (n0 carried over) equals one long run bit for bit."""
    p = inputs.make_problem(20, 20, 4, 3, seed=8)
    Z = np.zeros((20, 4))
    N = 150
    tn = (5 + np.arange(N))[:, None] * p.dt
    ftab, _ = oracle.ricker(np.broadcast_to(tn, (N, 4)), np.broadcast_to(p.T.astype(np.float64), (N, 4)))
    ftab = ftab.reshape(N, 4)
    Va, Sa, ta = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, N, T=p.T, n0=5, r=10)
    Vb, Sb, tb = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, N, ftab=ftab, r=10)
    np.testing.assert_array_equal(Va, Vb)
    np.testing.assert_array_equal(ta, tb)
    V1, S1, t1 = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, 60, T=p.T, n0=5, r=10)
    V2, S2, t2 = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V1, S1, 90, T=p.T, n0=65, r=10)
    np.testing.assert_array_equal(V2, Va)
    np.testing.assert_array_equal(S2, Sa)
    np.testing.assert_array_equal(np.concatenate([t1, t2]), ta)


def test_traces_are_receiver_rows():
    """Trace record k is C V^{(k+1) r} (taken after the step, V^0 excluded)."""
    p = inputs.make_problem(16, 16, 3, 5, seed=9)
    Z = np.zeros((16, 3))
    _, _, tr = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, 40, T=p.T, r=8)
    assert tr.shape == (5, 5, 3)
    for k in range(5):
        Vk, _, _ = oracle.forward(p.Avs, p.Asv, p.g, None, p.dt, Z, Z, (k + 1) * 8, T=p.T)
        np.testing.assert_allclose(tr[k], p.C.astype(np.float64) @ Vk, rtol=1e-13, atol=1e-15)


def test_columns_independent_of_threads_and_batch():
    """Rank-2 column m equals rank-1 run m (Sec. 2.4, 4.4), for any thread count."""
    p = inputs.make_problem(32, 32, 6, 2, seed=10)
    Z = np.zeros((32, 6))
    Va, Sa, ta = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, 100, T=p.T, r=10, threads=1)
    Vb, Sb, tb = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z, Z, 100, T=p.T, r=10, threads=3)
    np.testing.assert_array_equal(Va, Vb)
    for m in range(6):
        Vm, Sm, tm = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, Z[:, :1], Z[:, :1], 100,
                                    T=p.T[m:m + 1], r=10)
        np.testing.assert_array_equal(Vm[:, 0], Va[:, m])
        np.testing.assert_array_equal(tm[:, :, 0], ta[:, :, m])


# ------------------------------------------------------- spectral radius --
@pytest.mark.parametrize("K", [8, 128, 300])
def test_spectral_radius_skew(K):
    """Power iteration vs. numpy's 2-norm: for Avs = -Asv^T the coupled
    operator [[0, Avs], [Asv, 0]] has spectral radius sigma_max(Asv)."""
    p = inputs.make_problem(K, K, 1, 0, seed=K)
    rho, it = oracle.spectral_radius(p.Avs, p.Asv, max_iter=20000, tol=1e-15)
    ref = np.linalg.norm(p.Asv.astype(np.float64), 2)
    assert abs(rho - ref) / ref < 1e-10, (rho, ref, it)
    # the generator's dt puts dt * rho at 0.5 (up to the float32 rounding of dt)
    assert abs(p.dt * rho - 0.5) < 1e-6


def test_spectral_radius_nonsymmetric():
    """A non-skew pair with a real dominant eigenvalue of Avs Asv."""
    rng = np.random.default_rng(21)
    K = 40
    Q, _ = np.linalg.qr(rng.standard_normal((K, K)))
    d = np.linspace(0.2, 3.0, K)
    Asv = Q @ np.diag(d) @ Q.T
    Avs = -np.diag(np.linspace(1.0, 2.0, K))
    lam = np.linalg.eigvals(Avs @ Asv)
    ref = np.sqrt(np.max(np.abs(lam)))
    rho, _ = oracle.spectral_radius(Avs, Asv, max_iter=20000, tol=1e-15)
    assert abs(rho - ref) / ref < 1e-8


# --------------------------------------------------------------- adjoint --
def _loss(p, V0, S0, T, N, ystar):
    V, S = V0.copy(), S0.copy()
    _, _, tr = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, N, T=T, r=1)
    return float(np.sum((tr - ystar) ** 2))


def _adjoint_case(K=6, M=3, N=200, R=2, seed=31):
    p = inputs.make_problem(K, K, M, R, seed=seed)
    rng = np.random.default_rng(seed + 1)
    _, _, ystar = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, np.zeros((K, M)),
                                 np.zeros((K, M)), N, T=1.05 * p.T.astype(np.float64), r=1)
    V0 = 0.3 * rng.standard_normal((K, M))
    S0 = 0.3 * rng.standard_normal((K, M))
    return p, V0, S0, ystar


def test_adjoint_vs_central_difference():
    """Adjoint gradients vs. central differences of the trace misfit.  The
    loss is quadratic in (V0, S0), so that difference is exact up to roundoff;
    in T it is a smooth function, differenced with h = 1e-3."""
    p, V0, S0, ystar = _adjoint_case()
    N = ystar.shape[0]
    T = p.T.astype(np.float64)
    L, gV, gS, gT = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, T, N, ystar)
    assert abs(L - _loss(p, V0, S0, T, N, ystar)) <= 1e-12 * L
    rng = np.random.default_rng(5)
    dV = rng.standard_normal(V0.shape)
    dS = rng.standard_normal(S0.shape)
    h = 1e-3
    fd = (_loss(p, V0 + h * dV, S0 + h * dS, T, N, ystar)
          - _loss(p, V0 - h * dV, S0 - h * dS, T, N, ystar)) / (2 * h)
    an = float(np.sum(gV * dV) + np.sum(gS * dS))
    assert abs(fd - an) <= 1e-8 * abs(an)
    for m in range(T.size):
        e = np.zeros_like(T)
        e[m] = 1e-3
        fdT = (_loss(p, V0, S0, T + e, N, ystar) - _loss(p, V0, S0, T - e, N, ystar)) / 2e-3
        assert abs(fdT - gT[m]) <= 1e-4 * max(abs(gT[m]), 1e-12) + 1e-9


def test_adjoint_with_reference_state_vs_central_difference():
    """The reference-state term shifts the forward sweep; the adjoint's
    gradients with respect to (V0, S0) and T must still match central
    differences of the misfit of runs that carry the same term."""
    p, V0, S0, ystar = _adjoint_case(K=5, M=2, N=150, R=2, seed=37)
    N = ystar.shape[0]
    T = p.T.astype(np.float64)
    rng = np.random.default_rng(9)
    xref = (0.05 * rng.standard_normal(V0.shape), 0.05 * rng.standard_normal(S0.shape))

    def loss(V0_, S0_, T_):
        _, _, tr = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0_, S0_, N, T=T_, r=1,
                                  xref=xref)
        return float(np.sum((tr - ystar) ** 2))

    L, gV, gS, gT = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, T, N, ystar, xref=xref)
    assert abs(L - loss(V0, S0, T)) <= 1e-12 * L
    L0, gV0, _, _ = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, T, N, ystar)
    assert abs(L - L0) > 1e-6 * L0 and rel(gV, gV0) > 1e-6  # the term matters here
    dV = rng.standard_normal(V0.shape)
    dS = rng.standard_normal(S0.shape)
    h = 1e-3
    fd = (loss(V0 + h * dV, S0 + h * dS, T) - loss(V0 - h * dV, S0 - h * dS, T)) / (2 * h)
    an = float(np.sum(gV * dV) + np.sum(gS * dS))
    assert abs(fd - an) <= 1e-8 * abs(an)
    for m in range(T.size):
        e = np.zeros_like(T)
        e[m] = 1e-3
        fdT = (loss(V0, S0, T + e) - loss(V0, S0, T - e)) / 2e-3
        assert abs(fdT - gT[m]) <= 1e-4 * max(abs(gT[m]), 1e-12) + 1e-9


def test_adjoint_vs_bruteforce_jacobian():
    """Tiny case: gradient = 2 J^T r with J the full Jacobian of all trace
    records with respect to (V0, S0), built column by column from unit runs."""
    K, M, N, R = 3, 1, 15, 2
    p, V0, S0, ystar = _adjoint_case(K, M, N, R, seed=41)
    T = p.T.astype(np.float64)
    _, gV, gS, _ = oracle.adjoint(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, T, N, ystar)
    _, _, base = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, V0, S0, N, T=T, r=1)
    res = (base - ystar).ravel()
    J = np.zeros((res.size, 2 * K))
    for j in range(2 * K):
        e = np.zeros((2 * K, 1))
        e[j] = 1.0
        _, _, tj = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, e[:K], e[K:], N, r=1)
        J[:, j] = tj.ravel()
    grad = 2 * J.T @ res
    np.testing.assert_allclose(np.concatenate([gV[:, 0], gS[:, 0]]), grad, rtol=1e-10, atol=1e-12)


def test_golden_small_forward_regression():
    """The oracle still reproduces its stored small-case output (written by
    tests/golden/make_golden.py from the oracle only)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_small_forward.json")
    gold = json.load(open(path))
    pr = gold["problem"]
    p = inputs.make_problem(pr["Kv"], pr["Ks"], pr["M"], pr["R"], seed=pr["seed"])
    assert p.dt == gold["dt"]
    V, S, tr = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, np.zeros((pr["Kv"], pr["M"])),
                              np.zeros((pr["Ks"], pr["M"])), pr["steps"], T=p.T, r=pr["r"])
    np.testing.assert_allclose(V, np.array(gold["V"]), rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(S, np.array(gold["S"]), rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(tr, np.array(gold["traces"]), rtol=1e-13, atol=1e-16)
