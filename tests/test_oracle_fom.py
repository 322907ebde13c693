"""Pins of the FP64 full-order-model oracle (oracle/fom_oracle.c; the
axisymmetric shear-wave system of Sec. 3, Eq. (fom_asym)) against what the
mathematics and physics fix: exact null vectors of the two stencils (rigid
rotation, hoop stress), the weighted skew-adjointness that makes the
flux-form operator energy-conserving, the paper's sparsity (at most four
and two non-zeros per row), discrete-energy invariance of the leapfrog,
superposition, and the radial travel time at the shear speed (App. A
material)."""
import numpy as np
import pytest

import oracle

P = oracle.FOM_APP_A
RHO, VS = P["rho"], P["vs"]
MU = RHO * VS * VS
RC, RE = P["r_cmb"], P["r_earth"]


def grid(Nr, Nt):
    dr, dth = (RE - RC) / Nr, np.pi / Nt
    i = np.arange(Nr)
    j = np.arange(1, Nt)
    # velocity (i + 1/2, j), sigma_rp (i, j) for i >= 1, sigma_tp (i + 1/2, j + 1/2) off the axis
    rv = np.repeat(RC + (i + 0.5) * dr, Nt - 1)
    tv = np.tile(j * dth, Nr)
    r1 = np.repeat(RC + np.arange(1, Nr) * dr, Nt - 1)
    t1 = np.tile(j * dth, Nr - 1)
    r2 = np.repeat(RC + (i + 0.5) * dr, Nt - 2)
    t2 = np.tile((np.arange(1, Nt - 1) + 0.5) * dth, Nr)
    return rv, tv, r1, t1, r2, t2


def zeros(Nr, Nt, M):
    nv, n1, n2 = oracle.fom_dims(Nr, Nt)
    return np.zeros((nv, M)), np.zeros((n1, M)), np.zeros((n2, M))


def operators(Nr, Nt, dt):
    """A (velocity rows, stress columns) and B (stress rows, velocity
    columns) of the leapfrog, probed from one-step oracle runs:
    v' = v + dt A s with v = 0, and s' = dt B v with s = 0."""
    nv, n1, n2 = oracle.fom_dims(Nr, Nt)
    ns = n1 + n2
    Vz, S1z, S2z = zeros(Nr, Nt, ns)
    E = np.eye(ns)
    V, _, _, _ = oracle.fom_forward(Nr, Nt, Vz, E[:n1], E[n1:], 1, dt=dt)
    A = V / dt
    _, S1, S2, _ = oracle.fom_forward(Nr, Nt, np.eye(nv), *zeros(Nr, Nt, nv)[1:], 1, dt=dt)
    B = np.vstack([S1, S2]) / dt
    return A, B


def weights(Nr, Nt):
    rv, tv, r1, t1, r2, t2 = grid(Nr, Nt)
    return RHO * rv ** 2 * np.sin(tv), np.concatenate([r1 ** 2 * np.sin(t1) / MU,
                                                       r2 ** 2 * np.sin(t2) / MU])


def test_dims_and_sparsity():
    """Unknown counts of the staggered grid, and at most four non-zeros per
    velocity row and two per stress row (Sec. 3)."""
    Nr, Nt = 5, 9
    nv, n1, n2 = oracle.fom_dims(Nr, Nt)
    assert (nv, n1, n2) == (Nr * (Nt - 1), (Nr - 1) * (Nt - 1), Nr * (Nt - 2))
    A, B = operators(Nr, Nt, 0.05)
    assert np.count_nonzero(A, axis=1).max() == 4
    assert np.count_nonzero(B, axis=1).max() == 2
    assert np.count_nonzero(A, axis=1).min() >= 2 and np.count_nonzero(B, axis=1).min() >= 1


def test_weighted_skew_adjointness():
    """W_v A = -(W_s B)^T with W_v = rho r^2 sin(theta) and W_s = r^2
    sin(theta) / mu at each unknown's own point: the discrete counterpart of
    integrating by parts against the volume element r^2 sin(theta)."""
    Nr, Nt = 6, 11
    A, B = operators(Nr, Nt, 0.05)
    Wv, Ws = weights(Nr, Nt)
    lhs = Wv[:, None] * A
    rhs = -(Ws[:, None] * B).T
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(lhs)


def test_energy_invariant_near_stability_limit():
    """Unforced leapfrog at dt = 0.5 / rho(L), L = [[0, A], [B, 0]]: the
    discrete energy ||V||^2_Wv + ||S||^2_Ws - dt <S, B V>_Ws is conserved."""
    Nr, Nt = 6, 11
    A, B = operators(Nr, Nt, 1.0)
    rho_L = np.sqrt(np.max(np.abs(np.linalg.eigvals(A @ B))))
    dt = 0.5 / rho_L
    Wv, Ws = weights(Nr, Nt)
    nv, n1, n2 = oracle.fom_dims(Nr, Nt)
    rng = np.random.default_rng(0)
    V0 = rng.standard_normal((nv, 2))
    S0 = rng.standard_normal((n1 + n2, 2)) * np.sqrt(RHO * MU)  # comparable energy shares

    def energy(V, S):
        BV = B @ V
        return float(np.sum(Wv[:, None] * V * V) + np.sum(Ws[:, None] * S * S)
                     - dt * np.sum(Ws[:, None] * S * BV))

    V, S1, S2, _ = oracle.fom_forward(Nr, Nt, V0, S0[:n1], S0[n1:], 3000, dt=dt)
    e0, e1 = energy(V0, S0), energy(V, np.vstack([S1, S2]))
    assert abs(e1 - e0) <= 1e-11 * abs(e0)
    assert np.linalg.norm(V - V0) > 0.1 * np.linalg.norm(V0)  # the state did move


def test_rigid_rotation_is_static():
    """v = r sin(theta) (rotation about the axis) has no strain: both
    stress stencils vanish on it, so the state must not move."""
    Nr, Nt = 16, 24
    rv, tv, *_ = grid(Nr, Nt)
    V0 = (rv * np.sin(tv))[:, None]
    _, S10, S20 = zeros(Nr, Nt, 1)
    V, S1, S2, _ = oracle.fom_forward(Nr, Nt, V0, S10, S20, 300)
    assert np.linalg.norm(V - V0) <= 1e-12 * np.linalg.norm(V0)
    # a strain of relative size 1e-12 would leave |S| ~ mu dt N 1e-12 |v| / r
    assert np.abs(S1).max() + np.abs(S2).max() <= 1e-9 * MU * 0.05 * 300 * np.abs(V0).max() / RC
    # a field with strain does move
    V2, _, _, _ = oracle.fom_forward(Nr, Nt, (rv ** 2 * np.sin(tv))[:, None] / RE, S10, S20, 300)
    assert np.linalg.norm(V2 - (rv ** 2 * np.sin(tv))[:, None] / RE) > 1e-6 * np.linalg.norm(V2)


def test_null_vectors_of_the_stencils():
    """Fields the flux form annihilates exactly: B kills rigid rotation
    v = r sin(theta) on every stress row; A kills sigma_tp = g(r) /
    sin^2(theta) on every velocity row whose two polar neighbours are off
    the axis, and sigma_rp = h(theta) / r^3 on every velocity row whose two
    radial neighbours are inside the shell."""
    Nr, Nt = 7, 12
    A, B = operators(Nr, Nt, 0.05)
    rv, tv, r1, t1, r2, t2 = grid(Nr, Nt)
    nv, n1, n2 = oracle.fom_dims(Nr, Nt)
    rot = rv * np.sin(tv)
    assert np.abs(B @ rot).max() <= 1e-12 * np.abs(B).max() * np.abs(rot).max()
    rng = np.random.default_rng(1)
    g = np.repeat(rng.standard_normal(Nr), Nt - 2)
    hoop = np.concatenate([np.zeros(n1), g / np.sin(t2) ** 2])
    jv = np.tile(np.arange(1, Nt), Nr)
    inner_t = (jv >= 2) & (jv <= Nt - 2)
    y = A @ hoop
    assert np.abs(y[inner_t]).max() <= 1e-12 * np.abs(A).max() * np.abs(hoop).max()
    assert np.abs(y[~inner_t]).max() > 1e-6 * np.abs(A).max() * np.abs(hoop).max()
    h = np.tile(rng.standard_normal(Nt - 1), Nr - 1)
    rad = np.concatenate([h / r1 ** 3, np.zeros(n2)])
    iv = np.repeat(np.arange(Nr), Nt - 1)
    inner_r = (iv >= 1) & (iv <= Nr - 2)
    y = A @ rad
    assert np.abs(y[inner_r]).max() <= 1e-12 * np.abs(A).max() * np.abs(rad).max()


def test_superposition_and_zero():
    Nr, Nt, N = 8, 12, 200
    nv, n1, n2 = oracle.fom_dims(Nr, Nt)
    rng = np.random.default_rng(2)
    V0, S10, S20 = rng.standard_normal((nv, 2)), rng.standard_normal((n1, 2)), rng.standard_normal((n2, 2))
    f = rng.standard_normal((N, 2))
    Z = zeros(Nr, Nt, 2)
    a = oracle.fom_forward(Nr, Nt, V0, S10, S20, N, src=7, ftab=f)
    b = oracle.fom_forward(Nr, Nt, V0, S10, S20, N)
    c = oracle.fom_forward(Nr, Nt, *Z, N, src=7, ftab=f)
    for k in range(3):
        assert np.linalg.norm(a[k] - b[k] - c[k]) <= 1e-12 * np.linalg.norm(a[k])
    z = oracle.fom_forward(Nr, Nt, *Z, N, src=7, ftab=np.zeros((N, 2)))
    assert not any(x.any() for x in z[:3])


def test_radial_travel_time_at_shear_speed():
    """A pulse from a point source 640 km deep (App. A) on the equator
    reaches the surface receiver straight above after d / vs."""
    Nr, Nt = 96, 192
    dr = (RE - RC) / Nr
    i_s = int((RE - P["src_depth"] - RC) / dr)
    j = Nt // 2
    src = i_s * (Nt - 1) + (j - 1)
    recv = (Nr - 1) * (Nt - 1) + (j - 1)
    d = (RC + (Nr - 0.5) * dr) - (RC + (i_s + 0.5) * dr)
    dt, t0, w = 0.5, 30.0, 6.0
    N = int((t0 + d / VS + 60.0) / dt)
    t = np.arange(N) * dt
    ftab = np.exp(-((t - t0) / w) ** 2)[:, None]
    V0, S10, S20 = zeros(Nr, Nt, 1)
    _, _, _, tr = oracle.fom_forward(Nr, Nt, V0, S10, S20, N, src=src, ftab=ftab, recv=[recv],
                                     r=1, dt=dt)
    v = tr[:, 0, 0]
    t_peak = (np.argmax(np.abs(v)) + 1) * dt
    assert abs(t_peak - (t0 + d / VS)) <= 0.06 * d / VS, (t_peak, t0 + d / VS)
