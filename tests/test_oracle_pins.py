"""Pins for the CPU oracle against facts fixed by mechanics and mathematics.

None of these compares the oracle with a re-typed copy of its own formula:
forces are pinned by symbolic differentiation of the softened potential
(sympy, exact), by Newton's third law, by equivariance, by F = -grad U through
the oracle's independent pair-potential loop, by the Newtonian limit; the
integrator by the Kepler closed form, the O(dt^2) order of leapfrog, time
reversibility and exact momentum / angular-momentum conservation; the
reductions by Plummer-model closed forms; the adjoint by symbolic and
finite-difference derivatives.
"""

import math

import numpy as np
import pytest

import oracle
from paper_2511_02655_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


# --------------------------------------------------------------------------------------
# forces


def _sympy_three_body(eps_val, G_val):
    """Exact forces/potentials/VJP for a fixed 3-body case by differentiating U symbolically."""
    sp = pytest.importorskip("sympy")
    X = sp.Matrix(3, 3, lambda i, c: sp.Symbol(f"x{i}{c}"))
    M = sp.symbols("m0:3")
    G, eps = sp.Rational(G_val), sp.Rational(eps_val)
    U = 0
    for i in range(3):
        for j in range(i + 1, 3):
            r2 = sum((X[j, c] - X[i, c]) ** 2 for c in range(3))
            U += -G * M[i] * M[j] / sp.sqrt(r2 + eps ** 2)
    # a_i = -(1/m_i) dU/dx_i ;  phi_i = dU/dm_i (U is bilinear in the masses)
    acc = [[-sp.diff(U, X[i, c]) / M[i] for c in range(3)] for i in range(3)]
    phi = [sp.diff(U, M[i]) for i in range(3)]
    xs = [[sp.Rational(1, 3), sp.Rational(-1, 2), sp.Rational(1, 5)],
          [sp.Rational(-2, 7), sp.Rational(3, 4), sp.Rational(0)],
          [sp.Rational(5, 6), sp.Rational(1, 8), sp.Rational(-3, 5)]]
    ms = [sp.Rational(1, 2), sp.Rational(1, 3), sp.Rational(1, 6)]
    W = [[sp.Rational(1, 2), sp.Rational(-1, 3), sp.Rational(2, 5)],
         [sp.Rational(-1, 4), sp.Rational(1, 7), sp.Rational(3, 8)],
         [sp.Rational(2, 3), sp.Rational(1, 9), sp.Rational(-1, 2)]]
    subs = {X[i, c]: xs[i][c] for i in range(3) for c in range(3)}
    subs.update({M[i]: ms[i] for i in range(3)})
    wa = sum(W[i][c] * acc[i][c] for i in range(3) for c in range(3))
    gx = [[sp.diff(wa, X[i, c]) for c in range(3)] for i in range(3)]
    gm = [sp.diff(wa, M[i]) for i in range(3)]
    ev = lambda e: float(sp.N(e.subs(subs), 30))
    return (np.array(xs, dtype=float), np.array(ms, dtype=float), np.array(W, dtype=float),
            np.array([[ev(acc[i][c]) for c in range(3)] for i in range(3)]),
            np.array([ev(p) for p in phi]),
            np.array([[ev(gx[i][c]) for c in range(3)] for i in range(3)]),
            np.array([ev(g) for g in gm]))


@pytest.mark.parametrize("eps,G", [("1/10", "1"), ("0", "3/2")])
def test_forces_match_symbolic_gradient_of_softened_potential(eps, G):
    x, m, w, a_ex, phi_ex, gx_ex, gm_ex = _sympy_three_body(eps, G)
    e, g = float(eval(eps)), float(eval(G))
    a, phi = oracle.forces(x, m, G=g, eps=e, threads=1)
    np.testing.assert_allclose(a, a_ex, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(phi, phi_ex, rtol=1e-13, atol=1e-15)
    gx, gm = oracle.force_vjp(x, m, w, G=g, eps=e, threads=1)
    np.testing.assert_allclose(gx, gx_ex, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(gm, gm_ex, rtol=1e-12, atol=1e-14)


def test_newton_limit_two_bodies():
    # eps -> 0: |a_0| = G m_1 / r^2 toward body 1 (Newton's law of gravitation)
    x = np.array([[0.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    m = np.array([3.0, 5.0])
    a, phi = oracle.forces(x, m, G=0.7, eps=0.0)
    np.testing.assert_allclose(a[0], [0.0, 0.7 * 5.0 / 4.0, 0.0], rtol=1e-15)
    np.testing.assert_allclose(a[1], [0.0, -0.7 * 3.0 / 4.0, 0.0], rtol=1e-15)
    np.testing.assert_allclose(phi, [-0.7 * 5.0 / 2.0, -0.7 * 3.0 / 2.0], rtol=1e-15)


def test_coincident_bodies_softened():
    x = np.zeros((2, 3))
    m = np.array([0.25, 0.75])
    a, phi = oracle.forces(x, m, G=1.0, eps=0.01)
    assert np.all(a == 0.0)
    np.testing.assert_allclose(phi, [-0.75 / 0.01, -0.25 / 0.01], rtol=1e-15)
    E = oracle.energy(x, np.zeros((2, 3)), m, G=1.0, eps=0.01)
    np.testing.assert_allclose(E[2], -0.25 * 0.75 / 0.01, rtol=1e-15)


def test_degenerate_sizes():
    a, phi = oracle.forces(np.zeros((1, 3)), np.ones(1), eps=0.1)
    assert np.all(a == 0) and np.all(phi == 0)
    a, phi = oracle.forces(np.zeros((0, 3)), np.zeros(0), eps=0.1)
    assert a.shape == (0, 3)


def test_newton_third_law_zero_net_force():
    x, v, m = inputs.plummer(512, seed=7)
    m = m * np.exp(0.3 * np.random.default_rng(1).standard_normal(512))
    a, _ = oracle.forces(x, m, G=1.0, eps=0.01)
    net = (m[:, None] * a).sum(0)
    scale = (m[:, None] * np.abs(a)).sum()
    assert np.abs(net).max() <= 1e-14 * scale


def test_translation_rotation_equivariance():
    x, _, m = inputs.plummer(256, seed=3)
    a, phi = oracle.forces(x, m, eps=0.02)
    q, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((3, 3)))
    shift = np.array([0.3, -1.2, 2.5])
    a2, phi2 = oracle.forces(x @ q.T + shift, m, eps=0.02)
    np.testing.assert_allclose(a2, a @ q.T, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(phi2, phi, rtol=1e-12)


def test_force_is_minus_gradient_of_pair_potential():
    # m_k a_k = -dU/dx_k with U from the independent pair loop in oracle.energy
    x, v, m = inputs.plummer(24, seed=11)
    eps, h = 0.05, 1e-5
    a, phi = oracle.forces(x, m, eps=eps)
    for k in (0, 5, 17):
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            dU = (oracle.energy(xp, v, m, eps=eps)[2] - oracle.energy(xm, v, m, eps=eps)[2]) / (2 * h)
            assert abs(-dU - m[k] * a[k, c]) <= 1e-7 * np.abs(m[k] * a[k]).max()
    # U = 1/2 sum m_i phi_i
    U = oracle.energy(x, v, m, eps=eps)[2]
    assert abs(U - 0.5 * (m * phi).sum()) <= 1e-13 * abs(U)


def test_forces_at_equals_rows_of_forces():
    x, _, m = inputs.plummer(300, seed=5)
    a, phi = oracle.forces(x, m, eps=0.01)
    idx = np.array([0, 7, 299, 150])
    a2, phi2 = oracle.forces_at(x, m, idx, eps=0.01)
    np.testing.assert_array_equal(a2, a[idx])
    np.testing.assert_array_equal(phi2, phi[idx])


# --------------------------------------------------------------------------------------
# KDK leapfrog


def _kepler_solution(t, m1, m2, a_sm, e, G=1.0):
    """Relative position of body 2 w.r.t. body 1 at time t from pericentre (Kepler's equation)."""
    M = m1 + m2
    n = math.sqrt(G * M / a_sm ** 3)
    Mean = n * t
    E = Mean if e < 0.8 else math.pi
    for _ in range(100):
        E -= (E - e * math.sin(E) - Mean) / (1 - e * math.cos(E))
    return np.array([a_sm * (math.cos(E) - e), a_sm * math.sqrt(1 - e * e) * math.sin(E), 0.0])


@pytest.mark.parametrize("e", [0.0, 0.5])
def test_kepler_orbit_second_order(e):
    m1, m2, a_sm = 0.6, 0.4, 1.0
    x0, v0, m, period = inputs.kepler_pair(m1, m2, a_sm, e)
    errs = []
    for nsteps in (2000, 4000):
        dt = period / nsteps
        x, v, _, _ = oracle.kdk(x0, v0, m, 1.0, 0.0, dt, nsteps // 2, threads=1)  # half an orbit
        t = dt * (nsteps // 2)
        rel_pos = x[1] - x[0]
        errs.append(np.linalg.norm(rel_pos - _kepler_solution(t, m1, m2, a_sm, e)))
        # centre of mass stays at rest at the origin
        assert np.abs((m[:, None] * x).sum(0)).max() < 1e-13
    assert errs[0] < 5e-4
    ratio = errs[0] / errs[1]
    assert 3.5 < ratio < 4.5, ratio


def test_energy_drift_is_second_order():
    x0, v0, m, period = inputs.kepler_pair(0.5, 0.5, 1.0, 0.6)
    drifts = []
    for nsteps in (1000, 2000):
        dt = period / nsteps
        _, _, _, log = oracle.kdk(x0, v0, m, 1.0, 0.0, dt, nsteps, energy_every=1, threads=1)
        E0 = oracle.energy(x0, v0, m, eps=0.0)[0]
        drifts.append(np.abs(log[:, 0] - E0).max() / abs(E0))
    ratio = drifts[0] / drifts[1]
    assert 3.6 < ratio < 4.4, ratio


def test_time_reversibility_and_conservation():
    x0, v0, m = inputs.plummer(64, seed=2)
    m = m * np.exp(0.2 * np.random.default_rng(9).standard_normal(64))
    G, eps, dt, n = 1.0, 0.05, 1e-3, 50
    x1, v1, a1, log = oracle.kdk(x0, v0, m, G, eps, dt, n, energy_every=10)
    # run back with negated velocities: returns to the start (leapfrog is time-symmetric)
    x2, v2, _, _ = oracle.kdk(x1, -v1, m, G, eps, dt, n, a=a1)
    assert np.abs(x2 - x0).max() < 1e-12
    assert np.abs(-v2 - v0).max() < 1e-11
    E0 = oracle.energy(x0, v0, m, G, eps)
    # momentum and angular momentum: exactly conserved by KDK with central pair forces
    assert np.abs(log[:, 3:6] - E0[3:6]).max() < 1e-14
    assert np.abs(log[:, 6:9] - E0[6:9]).max() < 1e-13
    assert np.abs(log[:, 0] - E0[0]).max() < 1e-4 * abs(E0[0])


def test_kdk_accepts_precomputed_force_and_zero_steps():
    x0, v0, m = inputs.plummer(32, seed=4)
    x1, v1, a1, _ = oracle.kdk(x0, v0, m, 1.0, 0.01, 1e-3, 0)
    np.testing.assert_array_equal(x1, x0)
    np.testing.assert_array_equal(a1, oracle.forces(x0, m, eps=0.01)[0])
    xa, va, aa, _ = oracle.kdk(x0, v0, m, 1.0, 0.01, 1e-3, 3)
    xb, vb, ab, _ = oracle.kdk(x0, v0, m, 1.0, 0.01, 1e-3, 3, a=a1)
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(aa, ab)


# --------------------------------------------------------------------------------------
# reductions and inputs (Plummer closed forms)


def test_plummer_energy_and_virial():
    # Plummer model, G = M = a = 1: U = -3 pi / 32, and virial equilibrium 2K + U = 0.
    Us, Ks = [], []
    for seed in (21, 22):
        x, v, m = inputs.plummer(6000, seed=seed)
        out = oracle.energy(x, v, m, G=1.0, eps=1e-4)
        Us.append(out[2]), Ks.append(out[1])
        np.testing.assert_allclose(out[3:6], 0.0, atol=1e-14)
    U, K = np.mean(Us), np.mean(Ks)
    assert abs(U / (-3 * math.pi / 32) - 1) < 0.03, U
    assert abs(2 * K / -U - 1) < 0.05, (K, U)


def test_plummer_radial_cdf():
    scipy_stats = pytest.importorskip("scipy.stats")
    x, _, m = inputs.plummer(20000, seed=8)
    r = np.linalg.norm(x, axis=1)  # COM shift is tiny at this N
    cdf_max = 20.0 ** 3 / (1 + 20.0 ** 2) ** 1.5
    res = scipy_stats.kstest(r, lambda s: np.minimum(s ** 3 / (1 + s * s) ** 1.5 / cdf_max, 1.0))
    assert res.pvalue > 1e-3
    assert abs(m.sum() - 1) < 1e-12


def test_two_spheres_layout():
    x, v, m = inputs.two_spheres(4096, seed=3)
    assert abs(m.sum() - 1) < 1e-12
    np.testing.assert_allclose((m[:, None] * x).sum(0), 0.0, atol=1e-12)
    np.testing.assert_allclose((m[:, None] * v).sum(0), 0.0, atol=1e-12)
    ca, cb = np.median(x[:2048], axis=0), np.median(x[2048:], axis=0)
    assert abs((cb - ca)[0] - 10.0) < 0.3
    va, vb = v[:2048].mean(0), v[2048:].mean(0)
    assert abs((va - vb)[0] - 0.5) < 0.05
    assert np.std(np.log(m)) == pytest.approx(0.5, rel=0.05)


def test_ensemble_sizes_log_uniform():
    s = inputs.ensemble_sizes(4096, seed=1)
    assert s.min() >= 64 and s.max() <= 16384
    u = (np.log(s) - math.log(64)) / (math.log(16384) - math.log(64))
    assert abs(u.mean() - 0.5) < 0.02
    ens = inputs.ensemble(5, seed=2)
    assert ens.offsets[0] == 0 and ens.offsets[-1] == ens.x.shape[0] == ens.m.shape[0]


# --------------------------------------------------------------------------------------
# virial diagnostics


def test_virial_equals_potential_when_unsoftened_and_matches_per_body_form():
    x, v, m = inputs.plummer(300, seed=2)
    m = m * np.exp(0.2 * np.random.default_rng(2).standard_normal(300))
    K, W, Q = oracle.virial(x, v, m, G=1.7, eps=0.0)
    E = oracle.energy(x, v, m, G=1.7, eps=0.0)
    # eps = 0: each pair gives -G m m r^2 / r^3 = -G m m / r, so W = U (Euler's theorem, degree -1)
    assert abs(W - E[2]) <= 1e-13 * abs(E[2]) and abs(K - E[1]) <= 1e-14 * E[1]
    assert Q == -2 * K / W
    # softened: the pair form equals sum_i m_i x_i . a_i of the force sum, for any origin
    for shift in (0.0, 3.0):
        xs = x + shift
        a, _ = oracle.forces(xs, m, G=1.7, eps=0.03)
        assert abs(oracle.virial(xs, v, m, G=1.7, eps=0.03)[1] - (m[:, None] * xs * a).sum()) <= 1e-12 * abs(W)


def test_virial_lennard_jones_pair_and_body_forms():
    # one pair: W = r F(r) = -r dV/dr, zero at the minimum r = 2^(1/6) sigma
    sig, el = 0.9, 1.3
    for r, expect_zero in ((2 ** (1 / 6) * sig, True), (0.95 * sig, False), (1.7 * sig, False)):
        x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
        v, m = np.zeros((2, 3)), np.ones(2)
        W = oracle.virial(x, v, m, law=1, eps_lj=el, sigma=sig)[1]
        h = 1e-6 * r
        U = lambda rr: oracle.lj_energy(np.array([[0.0, 0, 0], [rr, 0, 0]]), v, m, eps_lj=el, sigma=sig)[2]
        dV = (U(r + h) - U(r - h)) / (2 * h)
        assert abs(W - (-r * dV)) <= 1e-7 * max(1.0, abs(W))
        if expect_zero:
            assert abs(W) <= 1e-12
    x, v, m, box = inputs.lj_gas(200, seed=3)
    a, _ = oracle.lj_forces(x, m, eps_lj=el, sigma=sig)
    W = oracle.virial(x, v, m, law=1, eps_lj=el, sigma=sig)[1]
    assert abs(W - (m[:, None] * x * a).sum()) <= 1e-11 * abs(W)


def test_plummer_is_in_virial_equilibrium():
    # the Plummer model is a self-consistent equilibrium: -2K/W -> 1 (statistical, ~1/sqrt(N))
    x, v, m = inputs.plummer(4096, seed=11)
    K, W, Q = oracle.virial(x, v, m, G=1.0, eps=0.0)
    assert abs(Q - 1.0) <= 0.05, Q


# --------------------------------------------------------------------------------------
# adjoint


def test_force_vjp_matches_finite_differences():
    x, _, m = inputs.plummer(16, seed=6)
    w = np.random.default_rng(3).standard_normal((16, 3))
    eps, h = 0.03, 1e-6
    gx, gm = oracle.force_vjp(x, m, w, eps=eps)
    f = lambda xx, mm: float((w * oracle.forces(xx, mm, eps=eps)[0]).sum())
    for k, c in ((0, 0), (3, 2), (15, 1)):
        xp, xm = x.copy(), x.copy()
        xp[k, c] += h
        xm[k, c] -= h
        fd = (f(xp, m) - f(xm, m)) / (2 * h)
        assert abs(fd - gx[k, c]) <= 1e-6 * np.abs(gx).max()
    for k in (1, 9):
        mp, mm_ = m.copy(), m.copy()
        mp[k] += h * m[k]
        mm_[k] -= h * m[k]
        fd = (f(x, mp) - f(x, mm_)) / (2 * h * m[k])
        assert abs(fd - gm[k]) <= 1e-6 * np.abs(gm).max()


def test_adjoint_matches_finite_differences():
    # N=8, 20 KDK steps: oracle reverse sweep vs central differences of the loss.
    x0, v0, m = inputs.plummer(8, seed=12)
    m = m * np.exp(0.3 * np.random.default_rng(4).standard_normal(8))
    t = inputs.targets(8, seed=13)
    G, eps, dt, n = 1.0, 0.05, 1e-2, 20
    xT, vT, _, _ = oracle.kdk(x0, v0, m, G, eps, dt, n)
    gx, gv, gm = oracle.adjoint(x0, v0, m, G, eps, dt, n, 2 * (xT - t), np.zeros_like(vT))
    L = lambda xx, vv, mm: oracle.trajectory_loss(xx, vv, mm, G, eps, dt, n, t, threads=1)
    # h = 1e-4: the O(h^2) truncation (~1e-9 relative here) stays well below the bound,
    # while h = 1e-6 would leave ~1e-16 * L / h of rounding noise (L ~ 70).
    h = 1e-4
    for k, c in ((0, 0), (2, 1), (7, 2), (5, 0)):
        xp, xm = x0.copy(), x0.copy()
        xp[k, c] += h
        xm[k, c] -= h
        fd = (L(xp, v0, m) - L(xm, v0, m)) / (2 * h)
        assert abs(fd - gx[k, c]) <= 1e-7 * max(abs(fd), np.abs(gx).max() * 1e-2), (k, c, fd, gx[k, c])
        vp, vm = v0.copy(), v0.copy()
        vp[k, c] += h
        vm[k, c] -= h
        fd = (L(x0, vp, m) - L(x0, vm, m)) / (2 * h)
        assert abs(fd - gv[k, c]) <= 1e-7 * max(abs(fd), np.abs(gv).max() * 1e-2), (k, c, fd, gv[k, c])
    for k in (0, 3, 6):
        mp, mm_ = m.copy(), m.copy()
        mp[k] += h
        mm_[k] -= h
        fd = (L(x0, v0, mp) - L(x0, v0, mm_)) / (2 * h)
        assert abs(fd - gm[k]) <= 1e-7 * max(abs(fd), np.abs(gm).max() * 1e-2), (k, fd, gm[k])


def test_param_vjp_matches_finite_differences():
    # w . da/dG and w . da/deps of the force map against central differences of w . a.
    x, _, m = inputs.plummer(16, seed=7)
    w = np.random.default_rng(5).standard_normal((16, 3))
    G, eps = 1.7, 0.04
    pG, pe = oracle.param_vjp(x, m, w, G=G, eps=eps)
    f = lambda g, e: float((w * oracle.forces(x, m, G=g, eps=e)[0]).sum())
    h = 1e-6
    assert abs((f(G + h, eps) - f(G - h, eps)) / (2 * h) - pG) <= 1e-7 * abs(pG)
    assert abs((f(G, eps + h) - f(G, eps - h)) / (2 * h) - pe) <= 1e-6 * abs(pe)
    # a is linear in G: w . a = G (w . da/dG) exactly (up to rounding)
    assert abs(f(G, eps) - G * pG) <= 1e-12 * abs(f(G, eps))


def _param_case():
    x0, v0, m = inputs.plummer(8, seed=14)
    m = m * np.exp(0.3 * np.random.default_rng(6).standard_normal(8))
    t = inputs.targets(8, seed=15)
    G, eps, dt, n = 1.3, 0.05, 1e-2, 20
    xT, vT, _, _ = oracle.kdk(x0, v0, m, G, eps, dt, n)
    grads = oracle.adjoint_params(x0, v0, m, G, eps, dt, n, 2 * (xT - t), np.zeros_like(vT))
    return x0, v0, m, t, G, eps, dt, n, xT, grads


def test_adjoint_params_match_finite_differences():
    # dL/dG and dL/deps of the 20-step loss against central differences (h = 1e-4 relative:
    # truncation ~1e-8, rounding ~1e-16 L / h).
    x0, v0, m, t, G, eps, dt, n, xT, (gx, gv, gm, (gG, ge)) = _param_case()
    L = lambda g, e: oracle.trajectory_loss(x0, v0, m, g, e, dt, n, t, threads=1)
    hG, he = 1e-4 * G, 1e-4 * eps
    fdG = (L(G + hG, eps) - L(G - hG, eps)) / (2 * hG)
    fde = (L(G, eps + he) - L(G, eps - he)) / (2 * he)
    assert abs(fdG - gG) <= 1e-6 * abs(fdG), (fdG, gG)
    assert abs(fde - ge) <= 1e-5 * abs(fde), (fde, ge)
    # the parameter sweep leaves the other gradients unchanged
    gx0, gv0, gm0 = oracle.adjoint(x0, v0, m, G, eps, dt, n, 2 * (xT - t), np.zeros_like(xT))
    assert np.array_equal(gx, gx0) and np.array_equal(gv, gv0) and np.array_equal(gm, gm0)


def test_adjoint_params_scaling_identities():
    # Two exact symmetries of softened gravity under KDK pin dL/dG and dL/deps to the
    # (separately pinned) gradients in x0, v0, m:
    #  * G enters only as the product G m_j, so G dL/dG = sum_j m_j dL/dm_j;
    #  * (x, v, m, eps, targets) -> (s x, s v, s^3 m, s eps, s t) maps every KDK step to
    #    s times itself (a scales by s), so L scales by s^2 and, at s = 1,
    #    2 L = x0.g_x0 + v0.g_v0 + 3 m.g_m + eps dL/deps - 2 (x_T - t).t .
    x0, v0, m, t, G, eps, dt, n, xT, (gx, gv, gm, (gG, ge)) = _param_case()
    assert abs(G * gG - (m * gm).sum()) <= 1e-12 * abs(G * gG)
    L = float(((xT - t) ** 2).sum())
    rhs = 2 * L - (gx * x0).sum() - (gv * v0).sum() - 3 * (m * gm).sum() + 2 * ((xT - t) * t).sum()
    assert abs(eps * ge - rhs) <= 1e-9 * L, (eps * ge, rhs)


# --------------------------------------------------------------------------------------
# Lennard-Jones gas (the paper's pair law, Eq. 1)


def test_lj_forces_match_symbolic_gradient():
    sp = pytest.importorskip("sympy")
    X = sp.Matrix(3, 3, lambda i, c: sp.Symbol(f"x{i}{c}"))
    eps_lj, sig = sp.Rational(3, 2), sp.Rational(4, 5)
    U = 0
    for i in range(3):
        for j in range(i + 1, 3):
            r2 = sum((X[j, c] - X[i, c]) ** 2 for c in range(3))
            U += 4 * eps_lj * ((sig ** 2 / r2) ** 6 - (sig ** 2 / r2) ** 3)
    xs = [[sp.Rational(1, 3), sp.Rational(-1, 2), sp.Rational(1, 5)],
          [sp.Rational(-2, 7), sp.Rational(3, 4), sp.Rational(0)],
          [sp.Rational(5, 6), sp.Rational(1, 8), sp.Rational(-3, 5)]]
    ms = [2.0, 0.5, 1.25]
    subs = {X[i, c]: xs[i][c] for i in range(3) for c in range(3)}
    F = np.array([[float(sp.N(-sp.diff(U, X[i, c]).subs(subs), 30)) for c in range(3)] for i in range(3)])
    Uv = float(sp.N(U.subs(subs), 30))
    x = np.array(xs, dtype=float)
    a, phi = oracle.lj_forces(x, ms, eps_lj=1.5, sigma=0.8, threads=1)
    np.testing.assert_allclose(a * np.array(ms)[:, None], F, rtol=1e-12, atol=1e-12 * np.abs(F).max())
    assert abs(0.5 * (np.array(ms) * phi).sum() - Uv) <= 1e-12 * abs(Uv)
    E = oracle.lj_energy(x, np.zeros((3, 3)), ms, eps_lj=1.5, sigma=0.8)
    assert abs(E[2] - Uv) <= 1e-12 * abs(Uv)


def test_lj_pair_minimum_and_zero_crossing():
    # V has its minimum -eps at r = 2^{1/6} sigma (zero force) and crosses zero at r = sigma
    sig, e = 1.3, 0.7
    for r, V, sign in ((2 ** (1 / 6) * sig, -e, 0), (sig, 0.0, +1), (1.5 * sig, None, -1)):
        x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
        a, phi = oracle.lj_forces(x, [1.0, 1.0], eps_lj=e, sigma=sig)
        if V is not None:
            assert abs(phi[0] - V) <= 1e-14
        if sign == 0:
            assert np.abs(a).max() <= 1e-12
        else:  # repulsive inside the minimum (body 0 pushed to -x), attractive outside
            assert np.sign(-a[0, 0]) == sign


def test_lj_newton_third_law_and_energy_drift_order():
    x, v, m, box = inputs.lj_gas(64, seed=3, density=0.2, temperature=1.0)
    m = m * np.exp(0.2 * np.random.default_rng(2).standard_normal(64))
    a, _ = oracle.lj_forces(x, m)
    assert np.abs((m[:, None] * a).sum(0)).max() <= 1e-12 * (m[:, None] * np.abs(a)).sum()
    E0 = oracle.lj_energy(x, v, m)[0]
    drifts = []
    for dt in (2e-3, 1e-3):
        n = int(round(0.2 / dt))
        _, _, _, log = oracle.lj_kdk(x, v, m, 1.0, 1.0, 0.0, 0.0, dt, n, energy_every=1)
        drifts.append(np.abs(log[:, 0] - E0).max() / abs(E0))
    assert 3.0 < drifts[0] / drifts[1] < 5.0, drifts


def test_lj_reflecting_walls_free_particle():
    # two far-apart, effectively free particles bouncing in a box: triangle-wave closed form
    box, dt, n = 10.0, 1e-3, 7000
    x = np.array([[1.0, 2.0, 3.0], [9.0, 8.0, 7.0]])
    v = np.array([[3.0, -1.7, 0.9], [-2.2, 0.5, 4.1]])
    xf, vf, _, _ = oracle.lj_kdk(x, v, [1.0, 1.0], 1e-30, 1.0, 0.0, box, dt, n)
    t = dt * n
    u = np.mod(x + v * t, 2 * box)
    xe = np.where(u > box, 2 * box - u, u)
    ve = np.where(u > box, -v, v)
    np.testing.assert_allclose(xf, xe, atol=1e-9)
    np.testing.assert_allclose(vf, ve, atol=1e-12)


def test_lj_gas_generator():
    x, v, m, box = inputs.lj_gas(1000, seed=1, density=0.05, temperature=2.0)
    assert abs(box - (1000 / 0.05) ** (1 / 3)) < 1e-12
    assert x.min() > 0 and x.max() < box
    np.testing.assert_allclose(v.mean(0), 0.0, atol=1e-12)
    assert abs((v ** 2).mean() - 2.0) < 0.15
    d = np.linalg.norm(x[:, None, :] - x[None, :, :], axis=-1) + np.eye(1000) * 1e9
    assert d.min() > 0.5  # no overlapping pairs at the start


def test_lj_forces_at_equals_rows_of_lj_forces():
    x, v, m, box = inputs.lj_gas(300, seed=4, density=0.2)
    m = m * np.exp(0.2 * np.random.default_rng(8).standard_normal(300))
    a, phi = oracle.lj_forces(x, m, eps_lj=1.1, sigma=0.9)
    idx = np.array([0, 17, 299, 150, 17])
    ai, phii = oracle.lj_forces_at(x, m, idx, eps_lj=1.1, sigma=0.9)
    assert np.array_equal(ai, a[idx]) and np.array_equal(phii, phi[idx])


@pytest.mark.parametrize("gen", ["plummer", "two_spheres", "lj_gas", "targets"])
def test_generators_are_deterministic_by_seed(gen):
    f = getattr(inputs, gen)
    a1, a2, b = f(64, seed=3), f(64, seed=3), f(64, seed=4)
    flat = lambda r: np.concatenate([np.ravel(np.asarray(t, dtype=float)) for t in (r if isinstance(r, tuple) else (r,))])
    assert np.array_equal(flat(a1), flat(a2))
    assert not np.array_equal(flat(a1), flat(b))
