"""Pins of the FP64 CPU oracle against what arXiv 1510.03816 and the mathematics fix.

None of these tests re-types the oracle's formulas: each one checks a
property that a dropped term, a wrong sign, index or coefficient would break
(finite differences of H, conservation laws, exact special cases, closed
forms, and the Hamiltonian values the paper prints).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad, solve_ivp

from oracle import oracle as o
from paper_1510_03816_gb300 import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KERNELS = [(o.GAUSS, 0.3), (o.TENT, 0.45), (o.EXPCONE, 0.4)]


def _cloud(n, dim, seed, spread=1.0, pscale=0.3, min_gap=0.05, sigma=None, kernel=None):
    """Random positions with all pair distances away from 0 and, for the tent, from its
    kink at r = sigma."""
    if kernel is not None and kernel != o.TENT:
        sigma = None
    rng = np.random.default_rng(seed)
    for _ in range(1000):
        q = rng.uniform(0, spread, size=(n, dim))
        d = np.linalg.norm(q[:, None] - q[None], axis=-1)[np.triu_indices(n, 1)]
        if d.min() < min_gap:
            continue
        if sigma is not None and np.min(np.abs(d - sigma)) < min_gap:
            continue
        return q, rng.normal(0, pscale, size=(n, dim))
    raise RuntimeError("no admissible cloud")


# --------------------------------------------------------------------------- kernel functors
@pytest.mark.parametrize("kernel,sigma", KERNELS)
def test_functors_closed_forms_and_derivatives(kernel, sigma):
    # closed-form values
    assert o.G(kernel, sigma, 0.0) == 1.0
    if kernel == o.GAUSS:
        assert math.isclose(o.G(kernel, sigma, sigma), math.exp(-0.5), rel_tol=1e-15)
    elif kernel == o.TENT:
        assert o.G(kernel, sigma, 0.5 * sigma) == 0.5
        assert o.G(kernel, sigma, sigma) == 0.0 and o.G(kernel, sigma, 2 * sigma) == 0.0
        assert o.phi(kernel, sigma, 1.5 * sigma) == 0.0 and o.psi(kernel, sigma, 1.5 * sigma) == 0.0
    else:
        assert math.isclose(o.G(kernel, sigma, sigma), math.exp(-1.0), rel_tol=1e-15)
    # phi = G'/r and psi = phi'/r against central differences of G and phi
    for r in np.linspace(0.1, 0.9, 7) * sigma:
        h = 1e-6 * sigma
        dG = (o.G(kernel, sigma, r + h) - o.G(kernel, sigma, r - h)) / (2 * h)
        dphi = (o.phi(kernel, sigma, r + h) - o.phi(kernel, sigma, r - h)) / (2 * h)
        assert math.isclose(o.phi(kernel, sigma, r), dG / r, rel_tol=1e-7)
        assert math.isclose(o.psi(kernel, sigma, r), dphi / r, rel_tol=1e-6)


# --------------------------------------------------------------------------- right-hand side
@pytest.mark.parametrize("kernel,sigma", KERNELS)
@pytest.mark.parametrize("dim", [2, 3])
def test_rhs_is_symplectic_gradient_of_H(kernel, sigma, dim):
    """Eq. N-particle is Hamiltonian (Eq. charsham): dq = dH/dp, dp = -dH/dq (FD of Eq. H)."""
    q, p = _cloud(7, dim, seed=10 + dim + 3 * kernel, spread=0.6, sigma=sigma, kernel=kernel)
    dq, dp = o.rhs(q, p, kernel, sigma)
    h = 1e-6
    for i in range(q.shape[0]):
        for c in range(dim):
            e = np.zeros_like(q)
            e[i, c] = h
            dHdp = (o.hamiltonian(q, p + e, kernel, sigma) - o.hamiltonian(q, p - e, kernel, sigma)) / (2 * h)
            dHdq = (o.hamiltonian(q + e, p, kernel, sigma) - o.hamiltonian(q - e, p, kernel, sigma)) / (2 * h)
            assert abs(dq[i, c] - dHdp) < 1e-8 * (1 + abs(dHdp))
            assert abs(dp[i, c] + dHdq) < 1e-8 * (1 + abs(dHdq))


@pytest.mark.parametrize("kernel,sigma", KERNELS)
@pytest.mark.parametrize("dim", [2, 3])
def test_rhs_momentum_and_angular_momentum_rates_vanish(kernel, sigma, dim):
    q, p = _cloud(40, dim, seed=3, spread=1.0, min_gap=1e-3)
    dq, dp = o.rhs(q, p, kernel, sigma)
    scale = np.abs(dp).max() + np.abs(dq).max()
    assert np.all(np.abs(dp.sum(0)) < 1e-13 * q.shape[0] * scale)
    if dim == 2:
        lrate = np.sum(q[:, 0] * dp[:, 1] - q[:, 1] * dp[:, 0] + dq[:, 0] * p[:, 1] - dq[:, 1] * p[:, 0])
        assert abs(lrate) < 1e-12 * q.shape[0] * scale
    else:
        lrate = np.sum(np.cross(q, dp) + np.cross(dq, p), axis=0)
        assert np.all(np.abs(lrate) < 1e-12 * q.shape[0] * scale)


def test_rhs_self_term_and_isolated_particles():
    """dq includes j = i with G(0) = 1, dp excludes it (Eq. N-particle)."""
    q = np.array([[0.1, 0.2], [5.0, 5.0]])
    p = np.array([[0.3, -0.7], [1.0, 2.0]])
    dq, dp = o.rhs(q, p, o.TENT, 0.5)
    np.testing.assert_array_equal(dq, p)
    np.testing.assert_array_equal(dp, np.zeros_like(p))
    # coincident distinct particles: tent/expcone take phi = 0 at r = 0
    qc = np.array([[0.1, 0.2], [0.1, 0.2]])
    for k in (o.TENT, o.EXPCONE, o.GAUSS):
        dq, dp = o.rhs(qc, p, k, 0.5)
        np.testing.assert_allclose(dq, np.array([p.sum(0), p.sum(0)]), rtol=0, atol=1e-15)
        np.testing.assert_array_equal(dp, np.zeros_like(p))


def test_rhs_two_particles_by_hand():
    """Two particles, Gaussian: the sums of Eq. N-particle have two terms each."""
    s = 0.7
    q = np.array([[0.0, 0.0], [0.3, 0.4]])  # r = 0.5
    p = np.array([[1.0, 2.0], [-0.5, 0.25]])
    g = math.exp(-0.25 / (2 * s * s))
    dq, dp = o.rhs(q, p, o.GAUSS, s)
    np.testing.assert_allclose(dq[0], p[0] + g * p[1], rtol=1e-15)
    # dp_0 = -(p0.p1) G'(r) (q0 - q1)/r with G'(r) = -r/s^2 G
    pp = p[0] @ p[1]
    np.testing.assert_allclose(dp[0], -pp * (-0.5 / s**2 * g) * (q[0] - q[1]) / 0.5, rtol=1e-14)
    np.testing.assert_allclose(dp[1], -dp[0], rtol=1e-15)


# --------------------------------------------------------------------------- RK4 shoot
def _richardson(kernel, sigma, dim=2):
    q, p = _cloud(8, dim, seed=21, spread=0.5, pscale=0.2, min_gap=0.02)
    ref, _ = o.shoot(q, p, kernel, sigma, steps=512)
    errs = [np.abs(o.shoot(q, p, kernel, sigma, steps=s)[0] - ref).max() for s in (8, 16, 32)]
    return errs


@pytest.mark.parametrize("kernel,sigma", [(o.GAUSS, 0.3), (o.EXPCONE, 0.4)])
def test_rk4_is_fourth_order(kernel, sigma):
    e8, e16, e32 = _richardson(kernel, sigma)
    assert 12.0 < e8 / e16 < 20.0
    assert 12.0 < e16 / e32 < 20.0


def test_conservation_over_a_shoot():
    """Sum p is conserved to rounding (linear invariant, preserved by RK4); H and
    2-D angular momentum are conserved to O(dt^4)."""
    q, p = _cloud(30, 2, seed=5, spread=0.8, pscale=0.1, min_gap=0.01)
    k, s = o.GAUSS, 0.25
    H0 = o.hamiltonian(q, p, k, s)
    L0 = np.sum(q[:, 0] * p[:, 1] - q[:, 1] * p[:, 0])
    errH, errL = [], []
    for steps in (20, 40):
        q1, p1 = o.shoot(q, p, k, s, steps)
        np.testing.assert_allclose(p1.sum(0), p.sum(0), rtol=0, atol=1e-14)
        errH.append(abs(o.hamiltonian(q1, p1, k, s) - H0))
        errL.append(abs(np.sum(q1[:, 0] * p1[:, 1] - q1[:, 1] * p1[:, 0]) - L0))
    assert errH[1] < 1e-6 * abs(H0) and errH[0] / errH[1] > 10
    assert errL[1] < 1e-6 and errL[0] / max(errL[1], 1e-300) > 10


def test_time_reversal():
    q, p = _cloud(12, 2, seed=6, spread=0.6, pscale=0.2, min_gap=0.02)
    for steps in (20, 40):
        q1, p1 = o.shoot(q, p, o.GAUSS, 0.3, steps, t1=1.0)
        qb, pb = o.shoot(q1, p1, o.GAUSS, 0.3, steps, t1=-1.0)
        err = max(np.abs(qb - q).max(), np.abs(pb - p).max())
        if steps == 20:
            e20 = err
    assert err < 1e-7 and e20 / err > 10


def test_momentum_scaling_law():
    """F(q, s p) = (s F_q, s^2 F_p), so RK4 with momentum s p0 over [0, 1] equals RK4
    with p0 over [0, s] with the same number of steps (pins the t^2 law of the
    Hamiltonian series of Sec. 7, Example 1)."""
    q, p = _cloud(10, 2, seed=8, spread=0.6, pscale=0.2, min_gap=0.02)
    for sc in (0.25, 0.6):
        qa, pa = o.shoot(q, sc * p, o.EXPCONE, 0.5, 30, t1=1.0)
        qb, pb = o.shoot(q, p, o.EXPCONE, 0.5, 30, t1=sc)
        np.testing.assert_allclose(qa, qb, rtol=0, atol=1e-13)
        np.testing.assert_allclose(pa, sc * pb, rtol=0, atol=1e-13)
        assert math.isclose(o.hamiltonian(q, sc * p, o.EXPCONE, 0.5),
                            sc * sc * o.hamiltonian(q, p, o.EXPCONE, 0.5), rel_tol=1e-14)


def test_single_particle_and_far_apart_tent_particles_move_straight():
    X = np.array([[0.2, 0.3]])
    p0 = np.array([[0.05, -0.02]])
    q1, p1 = o.shoot(X, p0, o.GAUSS, 0.1, 7)
    np.testing.assert_allclose(q1, X + p0, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(p1, p0)
    # tent: pairs always farther apart than sigma do not interact
    Xf = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    pf = np.array([[0.1, 0.0], [0.0, 0.1], [-0.1, 0.0]])
    q1, p1 = o.shoot(Xf, pf, o.TENT, 0.5, 9)
    np.testing.assert_allclose(q1, Xf + pf, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(p1, pf)


def test_concentric_shoot_matches_one_dof_reduction():
    """Radial momenta on N equispaced points keep the ring a circle; with P_R = N P the
    reduced Hamiltonian is P_R^2 S(R) / (2N), S(R) = sum_k cos(2 pi k/N) G(2R |sin(pi k/N)|)."""
    N, R0, P = 16, 1.0, 0.05
    X, _ = w.concentric_circles(N, R0, R0)
    p0 = P * X / R0
    k = np.arange(N)
    sig = 0.8

    def S(R):
        return np.sum(np.cos(2 * np.pi * k / N) * np.exp(-(2 * R * np.abs(np.sin(np.pi * k / N))) ** 2 / (2 * sig**2)))

    def dS(R, h=1e-6):
        return (S(R + h) - S(R - h)) / (2 * h)

    def f(t, y):
        R, PR = y
        return [PR * S(R) / N, -PR * PR * dS(R) / (2 * N)]

    sol = solve_ivp(f, (0, 1), [R0, N * P], rtol=1e-12, atol=1e-14)
    q1, p1 = o.shoot(X, p0, o.GAUSS, sig, 100)
    radii = np.linalg.norm(q1, axis=1)
    np.testing.assert_allclose(radii, sol.y[0, -1], rtol=1e-8)
    np.testing.assert_allclose(np.sum(p1 * q1 / radii[:, None], axis=1), sol.y[1, -1] / N, rtol=1e-6)


# --------------------------------------------------------------------------- Algorithm 1
def _closed_form_H(N, R0, R1, G):
    k = np.arange(N)

    def S(R):
        return np.sum(np.cos(2 * np.pi * k / N) * G(2 * R * np.abs(np.sin(np.pi * k / N))))

    I = quad(lambda R: 1.0 / np.sqrt(S(R)), R0, R1, epsabs=1e-14, epsrel=1e-13)[0]
    return 0.5 * N * I * I


def test_match_concentric_circles_closed_form_and_paper_values():
    """Sec. 9, Fig. H_distance (b),(c): circle r=2 -> r=1 and r=2 -> r=3, N=64, G = e^{-r}.
    The converged H equals the 1-DOF quadrature (N/2)(int dR / sqrt(S(R)))^2, and the
    paper's printed numbers equal E = 2H (Eq. E=2H) to the paper's eps = 1e-3."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_fig8_hamiltonian.json")))
    N = gold["n"]
    for case in gold["cases"]:
        X, Y = w.concentric_circles(N, gold["reference_radius"], case["target_radius"])
        p, st, it, res, hist = o.match(X, Y, o.EXPCONE, 1.0, 50, eps=1e-11, maxit=2000)
        assert st == o.OK and res < 1e-11
        H = o.hamiltonian(X, p, o.EXPCONE, 1.0)
        Hc = _closed_form_H(N, gold["reference_radius"], case["target_radius"], lambda r: np.exp(-r))
        assert math.isclose(H, Hc, rel_tol=1e-7)
        assert math.isclose(2 * H, case["printed_H"], rel_tol=gold["rel_tol"])
        # the residual history decreases monotonically for this contraction
        assert np.all(np.diff(hist) < 0)


def test_match_single_particle_unit_gain_converges_in_one_update():
    X = np.array([[0.5, 0.5]])
    Y = np.array([[0.53, 0.48]])
    p, st, it, res, hist = o.match(X, Y, o.TENT, 0.25, 10, h=1.0, eps=1e-12)
    assert st == o.OK and it == 1
    np.testing.assert_allclose(p, Y - X, rtol=0, atol=1e-16)
    assert hist[0] == pytest.approx(0.03)


def test_match_update_rule_first_iterate():
    """With p0 = 0 the first shoot leaves X in place, so p1 = h (Y - X) exactly."""
    pr = w.circle_to_ellipse(16)
    h = 0.05
    p, st, it, res, hist = o.match(pr.X, pr.Y, pr.kernel, pr.sigma, 5, h=h, eps=0.0, maxit=1)
    assert st == o.ENOTCONVERGED and it == 1
    np.testing.assert_allclose(p, h * (pr.Y - pr.X), rtol=0, atol=1e-17)
    assert hist[0] == pytest.approx(np.abs(pr.Y - pr.X).max(), rel=1e-15)


def test_default_gain_closed_forms():
    """The default gain (the Gershgorin bound h = 1 / max_i sum_j G_ij on the largest
    eigenvalue of G(X), the momentum rule's stability limit h lambda_max < 2 with margin)
    on configurations whose row sums are known by hand: a lone particle (G(0) = 1, so
    h = 1), two particles at distance r (both rows 1 + G(r)), three collinear tent
    particles whose three row sums differ (so the max, the diagonal and the reciprocal
    each matter), and a 3-4-5 right triangle in 3-D whose right-angle vertex holds the
    largest row."""
    for kernel, sigma in KERNELS:
        assert o.default_gain(np.array([[0.3, 0.7]]), kernel, sigma) == 1.0
        assert o.default_gain(np.array([[0.3, 0.7, 0.1]]), kernel, sigma) == 1.0
    r = 0.13
    two = np.array([[0.2, 0.4], [0.2 + r * 0.6, 0.4 + r * 0.8]])
    closed = {o.GAUSS: math.exp(-r * r / (2 * 0.3 * 0.3)), o.TENT: 1.0 - r / 0.45, o.EXPCONE: math.exp(-r / 0.4)}
    for kernel, sigma in KERNELS:
        assert o.default_gain(two, kernel, sigma) == pytest.approx(1.0 / (1.0 + closed[kernel]), rel=1e-14)
    # tent sigma = 0.2 at x = 0, 0.1, 0.25: G = 0.5 (0-1), 0.25 (1-2), 0 (0-2, beyond sigma)
    # row sums 1.5, 1.75, 1.25 -> h = 1 / 1.75
    line = np.array([[0.0, 0.3], [0.1, 0.3], [0.25, 0.3]])
    assert o.default_gain(line, o.TENT, 0.2) == pytest.approx(1.0 / 1.75, rel=1e-14)
    assert o.default_gain(line[::-1].copy(), o.TENT, 0.2) == pytest.approx(1.0 / 1.75, rel=1e-14)
    # right triangle, legs 0.06 and 0.08, hypotenuse 0.1 (Gaussian sigma = 0.05)
    tri = np.array([[0.5, 0.5, 0.5], [0.56, 0.5, 0.5], [0.5, 0.58, 0.5]])
    g = lambda d: math.exp(-d * d / (2 * 0.05 * 0.05))  # noqa: E731
    rows = [1 + g(0.06) + g(0.08), 1 + g(0.06) + g(0.1), 1 + g(0.08) + g(0.1)]
    assert o.default_gain(tri, o.GAUSS, 0.05) == pytest.approx(1.0 / max(rows), rel=1e-14)
    # the bound: 1/h >= lambda_max(G(X)) for a random cloud (Gram matrix from the closed form)
    q, _ = _cloud(20, 2, seed=41)
    d = np.linalg.norm(q[:, None] - q[None], axis=-1)
    lam = np.linalg.eigvalsh(np.exp(-d * d / (2 * 0.3 * 0.3))).max()
    h = o.default_gain(q, o.GAUSS, 0.3)
    assert 1.0 / h >= lam * (1 - 1e-12)
    assert h * lam < 2.0  # the momentum rule's linear stability at the default gain


def test_match_reports_divergence():
    """Too large a gain blows up (Table 2, h > 1: NaN); the oracle reports it as a status."""
    pr = w.circle_to_ellipse(32)
    p, st, it, res, hist = o.match(pr.X, pr.Y, o.GAUSS, 0.1, 10, h=50.0, eps=1e-6, maxit=200)
    assert st in (o.EDIVERGED, o.ENOTCONVERGED)
    assert st == o.EDIVERGED or hist[-1] > 1e3 * hist[0]


def test_iso_invariance_of_H():
    """Table 4: H is invariant under rotation, translation and reflection of both templates,
    and p0 transforms covariantly (rotated/reflected with the landmarks)."""
    pr = w.circle_to_ellipse(24)
    k, s = o.EXPCONE, 0.1
    p, st, it, res, _ = o.match(pr.X, pr.Y, k, s, 10, h=0.5, eps=1e-12, maxit=3000)
    assert st == o.OK
    H = o.hamiltonian(pr.X, p, k, s)
    th = math.pi / 3
    Rm = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    Fm = np.array([[1.0, 0.0], [0.0, -1.0]])
    for A, b in ((Rm, 0.0), (np.eye(2), np.array([0.5, 0.5])), (Fm, 0.0)):
        Xg, Yg = pr.X @ A.T + b, pr.Y @ A.T + b
        pg, st, it, res, _ = o.match(Xg, Yg, k, s, 10, h=0.5, eps=1e-12, maxit=3000)
        assert st == o.OK
        assert abs(o.hamiltonian(Xg, pg, k, s) - H) < 1e-9 * H
        np.testing.assert_allclose(pg, p @ A.T, rtol=0, atol=1e-9)


# --------------------------------------------------------------------------- HVP and adjoint
@pytest.mark.parametrize("kernel,sigma", KERNELS)
@pytest.mark.parametrize("dim", [2, 3])
def test_hvp_matches_fd_of_gradient(kernel, sigma, dim):
    """d2H v against central differences of grad H = (-dp, dq) (from the RHS)."""
    q, p = _cloud(6, dim, seed=31 + dim, spread=0.6, sigma=sigma, kernel=kernel)
    rng = np.random.default_rng(2)
    vq, vp = rng.normal(size=q.shape), rng.normal(size=q.shape)
    hq, hp = o.hvp(q, p, vq, vp, kernel, sigma)
    h = 1e-6
    dqa, dpa = o.rhs(q + h * vq, p + h * vp, kernel, sigma)
    dqb, dpb = o.rhs(q - h * vq, p - h * vp, kernel, sigma)
    np.testing.assert_allclose(hq, -(dpa - dpb) / (2 * h), rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(hp, (dqa - dqb) / (2 * h), rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("kernel,sigma", KERNELS)
@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_gradient_matches_central_fd(kernel, sigma, dim):
    """dE/dp0 for E = 1/2 p0^T G(X) p0 + lam/2 ||Q(1) - Y||^2 (Eq. inexact-E) against
    central differences with step 1e-4 in FP64."""
    X, p0 = _cloud(6, dim, seed=41 + dim, spread=0.5, pscale=0.05, sigma=sigma, kernel=kernel)
    rng = np.random.default_rng(4)
    Y = X + rng.normal(0, 0.05, size=X.shape)
    steps, lam = 6, 10.0
    E, g = o.adjoint(X, p0, Y, kernel, sigma, steps, lam)
    assert math.isclose(E, o.energy(X, p0, Y, kernel, sigma, steps, lam), rel_tol=1e-13)
    h = 1e-4
    fd = np.zeros_like(p0)
    for i in range(p0.shape[0]):
        for c in range(dim):
            e = np.zeros_like(p0)
            e[i, c] = h
            fd[i, c] = (o.energy(X, p0 + e, Y, kernel, sigma, steps, lam) -
                        o.energy(X, p0 - e, Y, kernel, sigma, steps, lam)) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())


# --------------------------------------------------------------------------- cell-list predicate
@pytest.mark.parametrize("dim", [2, 3])
def test_cell_neighbor_predicate_agrees_with_fp64_distance(dim):
    rng = np.random.default_rng(9)
    n = 700 if dim == 2 else 900
    q = rng.uniform(0, 1, size=(n, dim))
    sigma = 0.07 if dim == 2 else 0.15
    cnt, hsh, tot = o.cell_neighbors(q, sigma)
    d = np.linalg.norm(q[:, None] - q[None], axis=-1)
    inside = d < sigma * (1 - 1e-5)
    maybe = d < sigma * (1 + 1e-5)
    cnt_lo = inside.sum(1)
    cnt_hi = maybe.sum(1)
    assert np.all(cnt >= cnt_lo) and np.all(cnt <= cnt_hi)
    assert tot == int(cnt.sum())
    # exact agreement away from the boundary band, via the set fingerprint
    ok = cnt_lo == cnt_hi
    idx = np.arange(1, n + 1, dtype=np.uint64) * np.uint64(2654435761)
    fp = np.array([np.sum(idx[inside[i]], dtype=np.uint64) for i in range(n)], dtype=np.uint64)
    assert np.all(hsh[ok] == fp[ok])
    assert ok.mean() > 0.99


def test_row_sampled_variants_equal_the_full_sums():
    """The row-sampled RHS and neighbour sets are the full functions restricted to rows."""
    rng = np.random.default_rng(12)
    q = rng.uniform(0, 1, size=(500, 2))
    p = rng.normal(0, 0.1, size=(500, 2))
    rows = np.array([0, 17, 250, 499])
    for k, s in KERNELS:
        dq, dp = o.rhs(q, p, k, s)
        rq, rp = o.rhs_rows(q, p, rows, k, s)
        np.testing.assert_array_equal(rq, dq[rows])
        np.testing.assert_array_equal(rp, dp[rows])
    cnt, hsh, _ = o.cell_neighbors(q, 0.06)
    rc, rh = o.cell_neighbors_rows(q, rows, 0.06)
    np.testing.assert_array_equal(rc, cnt[rows])
    np.testing.assert_array_equal(rh, hsh[rows])


# --------------------------------------------------------------------------- velocity field and flow (Eq. u)


@pytest.mark.parametrize("kernel,sigma", KERNELS)
@pytest.mark.parametrize("dim", [2, 3])
def test_velocity_is_the_probe_momentum_gradient_of_H(kernel, sigma, dim):
    """Eq. u is dH/dv for a zero-momentum probe particle at x: with the probe's momentum v,
    H = H(q, p) + sum_j (v . p_j) G(|x - q_j|) + |v|^2 G(0) / 2, whose central difference
    in v at v = 0 is u(x) exactly (the quadratic term cancels)."""
    q, p = _cloud(9, dim, seed=40 + dim + kernel, spread=0.8, pscale=0.3, min_gap=0.05, sigma=sigma, kernel=kernel)
    x = np.random.default_rng(41).uniform(0, 0.8, size=(4, dim))
    u = o.velocity(q, p, x, kernel, sigma)
    eps = 1e-3
    for k in range(x.shape[0]):
        qa = np.vstack([q, x[k]])
        for c in range(dim):
            v = np.zeros((1, dim))
            v[0, c] = eps
            hp = o.hamiltonian(qa, np.vstack([p, v]), kernel, sigma)
            hm = o.hamiltonian(qa, np.vstack([p, -v]), kernel, sigma)
            assert abs((hp - hm) / (2 * eps) - u[k, c]) < 1e-10 * max(1.0, abs(u[k, c]))


def test_velocity_at_the_particles_is_dq():
    """Eq. u evaluated at q_i is the position rate of Eq. N-particle (self term included)."""
    for kernel, sigma in KERNELS:
        q, p = _cloud(14, 2, seed=43, spread=0.8, pscale=0.3, min_gap=0.02, sigma=sigma, kernel=kernel)
        dq, _ = o.rhs(q, p, kernel, sigma)
        np.testing.assert_allclose(o.velocity(q, p, q, kernel, sigma), dq, rtol=0, atol=1e-15)


def test_flow_tracers_started_on_particles_follow_them():
    """A point started at a particle obeys the same ODE as that particle's position, so
    RK4 carries it exactly along: x1 = Q(1) of the plain shoot."""
    for kernel, sigma in KERNELS:
        q, p = _cloud(11, 2, seed=44, spread=0.7, pscale=0.2, min_gap=0.02, sigma=sigma, kernel=kernel)
        x0 = q[[0, 3, 7]]
        q1, p1, x1 = o.flow(q, p, x0, kernel, sigma, 13)
        qs, ps = o.shoot(q, p, kernel, sigma, 13)
        np.testing.assert_allclose(q1, qs, rtol=0, atol=1e-15)
        np.testing.assert_allclose(p1, ps, rtol=0, atol=1e-15)
        np.testing.assert_allclose(x1, qs[[0, 3, 7]], rtol=0, atol=1e-14)


def test_flow_without_momentum_is_the_identity_and_reverses_in_time():
    q, p = _cloud(10, 2, seed=45, spread=0.7, pscale=0.2, min_gap=0.02)
    x0 = np.random.default_rng(46).uniform(0, 0.7, size=(25, 2))
    _, _, x1 = o.flow(q, np.zeros_like(p), x0, o.GAUSS, 0.3, 5)
    np.testing.assert_array_equal(x1, x0)
    errs = []
    for steps in (20, 40):
        q1, p1, x1 = o.flow(q, p, x0, o.GAUSS, 0.3, steps, t1=1.0)
        _, _, xb = o.flow(q1, p1, x1, o.GAUSS, 0.3, steps, t1=-1.0)
        errs.append(np.abs(xb - x0).max())
    assert errs[1] < 1e-8 and errs[0] / errs[1] > 10


def test_flow_of_one_particle_matches_an_ode_solver_and_is_fourth_order():
    """One Gaussian particle moves straight (q = q0 + p0 t, p = p0); points follow
    dx/dt = G(|x - q(t)|) p0, solved here by an adaptive high-order integrator."""
    sigma = 0.2
    q0 = np.array([[0.3, 0.4]])
    p0 = np.array([[0.15, 0.05]])
    x0 = np.array([[0.35, 0.42], [0.1, 0.6], [0.5, 0.3]])

    def f(t, y):
        x = y.reshape(-1, 2)
        qt = q0[0] + p0[0] * t
        g = np.exp(-np.sum((x - qt) ** 2, axis=1) / (2 * sigma ** 2))
        return (g[:, None] * p0[0]).ravel()

    ref = solve_ivp(f, (0.0, 1.0), x0.ravel(), method="DOP853", rtol=1e-13, atol=1e-14).y[:, -1].reshape(-1, 2)
    errs = []
    for steps in (8, 16, 32):
        _, _, x1 = o.flow(q0, p0, x0, o.GAUSS, sigma, steps)
        errs.append(np.abs(x1 - ref).max())
    assert errs[2] < 1e-8
    assert 12.0 < errs[0] / errs[1] < 20.0 and 12.0 < errs[1] / errs[2] < 20.0


# --------------------------------------------------------------------------- the inexact system (Sec. 6)


@pytest.mark.parametrize("kernel,sigma", KERNELS)
@pytest.mark.parametrize("dim", [2, 3])
def test_inexact_rhs_is_the_symplectic_gradient_of_the_augmented_H(kernel, sigma, dim):
    """Eq. N-particle-inexact is Hamiltonian with H + (s2 / 2) sum_i |p_i|^2: dq = dH/dp,
    dp = -dH/dq, checked by central differences of the plain double sum of Eq. H."""
    s2 = 0.37
    q, p = _cloud(7, dim, seed=50 + dim + kernel, spread=0.8, pscale=0.3, min_gap=0.05, sigma=sigma, kernel=kernel)
    dq, dp = o.rhs_inexact(q, p, kernel, sigma, s2)

    def Ha(qq, pp):
        return o.hamiltonian(qq, pp, kernel, sigma) + 0.5 * s2 * np.sum(pp * pp)

    eps = 1e-6
    for i in range(q.shape[0]):
        for c in range(dim):
            e = np.zeros_like(q)
            e[i, c] = eps
            fdp = (Ha(q, p + e) - Ha(q, p - e)) / (2 * eps)
            fdq = (Ha(q + e, p) - Ha(q - e, p)) / (2 * eps)
            assert abs(fdp - dq[i, c]) < 1e-8 * max(1.0, abs(dq[i, c]))
            assert abs(-fdq - dp[i, c]) < 1e-7 * max(1.0, abs(dp[i, c]))


def test_inexact_shoot_reduces_to_the_exact_one_and_moves_one_particle_straight():
    q, p = _cloud(9, 2, seed=52, spread=0.7, pscale=0.2, min_gap=0.02)
    qa, pa = o.shoot_inexact(q, p, o.GAUSS, 0.3, 0.0, 11)
    qb, pb = o.shoot(q, p, o.GAUSS, 0.3, 11)
    np.testing.assert_array_equal(qa, qb)
    np.testing.assert_array_equal(pa, pb)
    # one particle: p constant, q(t) = q0 + (G(0) + s2) p0 t
    X, p0 = np.array([[0.2, 0.3]]), np.array([[0.05, -0.02]])
    q1, p1 = o.shoot_inexact(X, p0, o.TENT, 0.2, 0.3, 7)
    np.testing.assert_allclose(q1, X + 1.3 * p0, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(p1, p0)


def test_inexact_match_stops_on_the_momentum_difference():
    """One particle: Q(1) = X + (1 + s2) p, so p_k = c (1 - (1 - h (1 + s2))^k) with
    c = (Y - X) / (1 + s2), and the update at iterate k is h (1 + s2) (c - p_k); the loop
    stops after the first update smaller than eps."""
    s2, h, eps = 0.5, 0.3, 1e-6
    X, Y = np.array([[0.2, 0.3]]), np.array([[0.26, 0.27]])
    c = (Y - X) / (1 + s2)
    a = 1 - h * (1 + s2)
    k = 0
    while True:
        upd = np.abs(h * (1 + s2) * c * a ** k).max()
        k += 1
        if upd < eps:
            break
    p, st, it, res, hist = o.match_inexact(X, Y, o.GAUSS, 0.1, s2, 3, h=h, eps=eps, maxit=500)
    assert st == o.OK and it == k
    np.testing.assert_allclose(p, c * (1 - a ** k), rtol=0, atol=1e-15)
    assert len(hist) == k and abs(hist[0] - np.abs(Y - X).max()) < 1e-15
    # the default gain is 1 / (max row sum + s2)
    p, st, it, res, hist = o.match_inexact(X, Y, o.GAUSS, 0.1, s2, 3, eps=eps, maxit=500)
    np.testing.assert_allclose(p, c, rtol=0, atol=1e-15)  # h = 1 / (1 + s2): exact after one update
    assert st == o.OK and it == 2


# --------------------------------------------------------------------------- tangent-linear shoot and the Newton gain (Sec. 5)


@pytest.mark.parametrize("kernel,sigma", KERNELS)
@pytest.mark.parametrize("dim", [2, 3])
def test_tangent_shoot_matches_central_differences(kernel, sigma, dim):
    q, p = _cloud(8, dim, seed=60 + dim + kernel, spread=0.8, pscale=0.2, min_gap=0.05, sigma=sigma, kernel=kernel)
    rng = np.random.default_rng(61)
    vq, vp = rng.normal(size=q.shape), rng.normal(size=q.shape)
    steps, eps = 6, 1e-6
    q1, p1, dq1, dp1 = o.shoot_tangent(q, p, vq, vp, kernel, sigma, steps)
    qa, pa = o.shoot(q + eps * vq, p + eps * vp, kernel, sigma, steps)
    qb, pb = o.shoot(q - eps * vq, p - eps * vp, kernel, sigma, steps)
    scale = max(1.0, np.abs(dq1).max(), np.abs(dp1).max())
    assert np.abs((qa - qb) / (2 * eps) - dq1).max() < 1e-7 * scale
    assert np.abs((pa - pb) / (2 * eps) - dp1).max() < 1e-7 * scale
    # the primal part is the plain shoot, bit for bit
    qs, ps = o.shoot(q, p, kernel, sigma, steps)
    np.testing.assert_array_equal(q1, qs)
    np.testing.assert_array_equal(p1, ps)


def test_tangent_shoot_is_linear_in_the_direction():
    q, p = _cloud(10, 2, seed=62, spread=0.7, pscale=0.2, min_gap=0.02)
    rng = np.random.default_rng(63)
    v1, v2 = rng.normal(size=q.shape), rng.normal(size=q.shape)
    z = np.zeros_like(q)
    a = o.shoot_tangent(q, p, z, v1, o.GAUSS, 0.3, 7)[2]
    b = o.shoot_tangent(q, p, z, v2, o.GAUSS, 0.3, 7)[2]
    c = o.shoot_tangent(q, p, z, 2.0 * v1 - 3.0 * v2, o.GAUSS, 0.3, 7)[2]
    np.testing.assert_allclose(c, 2.0 * a - 3.0 * b, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(o.shoot_tangent(q, p, z, z, o.GAUSS, 0.3, 7)[2], 0.0)


def test_newton_gain_one_particle_and_quadratic_convergence():
    # one Gaussian particle: Q(1) = X + p0, D phi = I, so one full Newton step lands exactly
    X, Y = np.array([[0.3, 0.4]]), np.array([[0.35, 0.42]])
    p, st, it, res, hist = o.match_newton(X, Y, o.GAUSS, 0.2, 5, h=1.0, eps=1e-13)
    assert st == o.OK and it == 1 and res < 1e-15
    np.testing.assert_allclose(p, Y - X, rtol=0, atol=1e-16)
    # a 12-landmark circle -> ellipse (Gaussian sigma = 0.1, D phi well conditioned): the
    # residual squares from one iterate to the next
    pr = w.circle_to_ellipse(12, sigma=0.1, kernel=o.GAUSS, steps=10)
    p, st, it, res, hist = o.match_newton(pr.X, pr.Y, o.GAUSS, 0.1, 10, h=1.0, eps=1e-12, maxit=20)
    assert st == o.OK and it <= 6
    r = np.array(hist)
    assert np.all(r[1:] < r[:-1])
    assert np.all(r[2:] < 50.0 * r[1:-1] ** 2)


# --------------------------------------------------------------------------- velocity update rule (Algorithm 1 steps 3-4)


def test_gram_matrix_is_the_velocity_at_the_landmarks():
    # Eq. u at t = 0 and at the landmarks themselves: u(X) = G(X) p
    q, p = _cloud(9, 2, seed=70, spread=0.8, min_gap=0.03, sigma=0.45, kernel=o.TENT)
    for kernel, sigma in KERNELS:
        GX = o.gram(q, kernel, sigma)
        np.testing.assert_array_equal(GX, GX.T)
        np.testing.assert_array_equal(np.diag(GX), 1.0)
        np.testing.assert_allclose(GX @ p, o.velocity(q, p, q, kernel, sigma), rtol=0, atol=1e-14)


@pytest.mark.parametrize("kernel,sigma", [(o.TENT, 0.45), (o.EXPCONE, 0.4), (o.GAUSS, 0.15)])
def test_velocity_rule_inverts_the_linearised_shoot(kernel, sigma):
    # For a small displacement Y = X + e V the shoot is Q(1) = X + G(X) p0 + O(|p0|^2), so one
    # velocity-rule update from p0 = 0 with h = 1 leaves an O(e^2) residual: the ratio of the
    # two residuals falls in proportion to e.  The momentum rule only damps it by a constant.
    rng = np.random.default_rng(71)
    X = rng.uniform(0, 1, (10, 2))
    V = rng.normal(size=X.shape)
    ratios = []
    for e in (1e-3, 1e-4):
        hist = o.match_velocity(X, X + e * V, kernel, sigma, 8, h=1.0, eps=0.0, maxit=1)[4]
        ratios.append(hist[1] / hist[0])
        hm = o.match(X, X + e * V, kernel, sigma, 8, h=0.0, eps=0.0, maxit=1)[4]
        assert hm[1] / hm[0] > 0.5
    assert ratios[0] < 0.05
    assert 0.08 < ratios[1] / ratios[0] < 0.12


def test_velocity_rule_equals_momentum_rule_when_the_gram_matrix_is_identity():
    # landmarks farther apart than the tent's support: G(X) = I and the two rules coincide
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.2]])
    Y = X + np.array([[0.1, -0.05], [0.02, 0.08], [-0.06, 0.03], [0.04, 0.04]])
    np.testing.assert_array_equal(o.gram(X, o.TENT, 0.5), np.eye(4))
    a = o.match_velocity(X, Y, o.TENT, 0.5, 6, h=0.6, eps=1e-12, maxit=40)
    b = o.match(X, Y, o.TENT, 0.5, 6, h=0.6, eps=1e-12, maxit=40)
    assert a[1] == b[1] and a[2] == b[2]
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[4], b[4])


def test_velocity_rule_converges_on_a_noise_free_tent_problem():
    # circle -> ellipse with the tent (noise-free target): with h = 1/2 the velocity rule
    # contracts the residual at a steady linear rate near 1 - h (G(X)^-1 D phi is near I)
    pr = w.circle_to_ellipse(16, sigma=0.45, kernel=o.TENT, steps=20)
    p, st, it, res, hist = o.match_velocity(pr.X, pr.Y, o.TENT, 0.45, 20, h=0.5, eps=1e-8, maxit=80)
    assert st == o.OK and it < 60
    r = np.array(hist)
    assert np.all(r[-5:] / r[-6:-1] < 0.7)


def test_newton_step_solves_the_linearised_shooting_equation():
    # From a momentum large enough that D phi is far from symmetric (|J - J^T| ~ 0.9 |J|),
    # the Newton step delta must solve the linearised equation D phi delta = r, checked
    # with the plain shoot alone: (Q(1; p + t delta) - Q(1; p - t delta)) / 2t = r + O(t^2)
    pr = w.circle_to_ellipse(12, sigma=0.15, kernel=o.GAUSS, steps=10)
    pbar = 0.3 * np.random.default_rng(5).normal(size=pr.X.shape)
    p1 = o.match_newton(pr.X, pr.Y, o.GAUSS, 0.15, 10, h=1.0, eps=0.0, maxit=1, p0=pbar)[0]
    d = p1 - pbar
    r = pr.Y - o.shoot(pr.X, pbar, o.GAUSS, 0.15, 10)[0]
    errs = []
    for t in (1e-3, 1e-4):
        qa = o.shoot(pr.X, pbar + t * d, o.GAUSS, 0.15, 10)[0]
        qb = o.shoot(pr.X, pbar - t * d, o.GAUSS, 0.15, 10)[0]
        errs.append(np.abs((qa - qb) / (2 * t) - r).max() / np.abs(r).max())
    assert errs[1] < 1e-7
    assert errs[1] < 0.05 * errs[0]  # second order in t
