"""The tangent-linear shoot and the solved update rules of Algorithm 1 (Sec. 5: the
Newton-type gain M = h (D phi)^-1; Algorithm 1 steps 3-4: the velocity update
p0 += h G(X)^-1 r) on the GPU against the FP64 oracle through the C ABI.

Both sides are FP64; they differ in summation order (the GPU sums a row over CTA
lanes) and, for the rules, in the linear solve (GPU: restarted GMRES to a 1e-12
relative residual; oracle: a dense LU).  Uniform clouds of 300 points hold pairs
a few 1e-3 apart, where the expcone's 1/r and the tangent's 1/r^3 terms amplify the
rounding of the 300-term sums: the shoot agrees to 1e-11 of its scale and the
tangent to 1e-10 (the adjoint's bar, which runs through the same Hessian terms);
converged momenta to 1e-8 of theirs, with equal iteration counts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as o  # noqa: E402
from paper_1510_03816_gb300 import ep, workloads as w  # noqa: E402

KSIG = [(ep.GAUSS, 0.2), (ep.TENT, 0.3), (ep.EXPCONE, 0.2)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_03816_gb300 import build

    build.build()
    o.build()
    ep.load()


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def host(a):
    return a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)


def cloud(n, dim, seed, sigma=None, band=1e-9):
    """Positions in [0.2, 0.8]^dim with no pair distance within band of the tent's kink."""
    rng = np.random.default_rng(seed)
    for _ in range(200):
        q = rng.uniform(0.2, 0.8, size=(n, dim))
        if sigma is not None and n > 1:
            d = np.linalg.norm(q[:, None] - q[None], axis=-1)[np.triu_indices(n, 1)]
            if np.min(np.abs(d - sigma)) < band:
                continue
        return q, rng.normal(0, 0.1, size=(n, dim))
    raise RuntimeError("no admissible cloud")


@pytest.mark.parametrize("kernel,sigma", KSIG)
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n", [1, 37, 300])
def test_tangent_shoot_parity(kernel, sigma, dim, n):
    # 37: fewer particles than CTAs; 300: several rows per CTA (ragged split)
    q, p = cloud(n, dim, seed=80 + 7 * dim + kernel + n, sigma=sigma if kernel == ep.TENT else None)
    rng = np.random.default_rng(81 + n)
    vq, vp = rng.normal(size=q.shape), rng.normal(size=q.shape)
    steps = 5
    prm = ep.params(dim=dim, kernel=kernel, sigma=sigma, steps=steps, precision=ep.FP64, neigh=ep.ALLPAIRS)
    q1, p1, vq1, vp1 = ep.shoot_tangent(cuda(q), cuda(p), cuda(vq), cuda(vp), prm)
    rq, rp, rvq, rvp = o.shoot_tangent(q, p, vq, vp, kernel, sigma, steps)
    assert rel(q1, rq) < 1e-11 and rel(p1, rp) < 1e-11
    assert rel(vq1, rvq) < 1e-10
    assert rel(vp1, rvp) < 1e-10


def test_tangent_shoot_host_arrays_and_linearity():
    q, p = cloud(64, 2, seed=90)
    rng = np.random.default_rng(91)
    v1, v2 = rng.normal(size=q.shape), rng.normal(size=q.shape)
    z = np.zeros_like(q)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.2, steps=4, precision=ep.FP64, neigh=ep.ALLPAIRS)
    a = ep.shoot_tangent(q, p, z, v1, prm)[2]
    b = ep.shoot_tangent(q, p, z, v2, prm)[2]
    c = ep.shoot_tangent(q, p, z, 2.0 * v1 - 3.0 * v2, prm)[2]
    assert np.abs(c - (2.0 * a - 3.0 * b)).max() < 1e-12 * np.abs(c).max()
    assert np.all(ep.shoot_tangent(q, p, z, z, prm)[2] == 0.0)


def _match(X, Y, prm, rule, **kw):
    return ep.match(cuda(X), cuda(Y), prm, rule=rule, **kw)


def test_newton_rule_parity():
    pr = w.circle_to_ellipse(12, sigma=0.1, kernel=ep.GAUSS, steps=10)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=10, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(pr.X, pr.Y, prm, ep.RULE_NEWTON, h=1.0, eps=1e-12, maxit=20)
    rp, st, it, r, hist = o.match_newton(pr.X, pr.Y, o.GAUSS, 0.1, 10, h=1.0, eps=1e-12, maxit=20)
    assert res.status == st == ep.OK
    assert res.iters == it
    assert rel(res.p0, rp) < 1e-8
    # the residual history agrees while it is far above the solve's accuracy
    big = hist > 1e-6
    np.testing.assert_allclose(res.hist[big], hist[big], rtol=1e-6)
    assert res.H == pytest.approx(o.hamiltonian(pr.X, rp, o.GAUSS, 0.1), rel=1e-9)


@pytest.mark.parametrize("kernel,sigma", [(ep.TENT, 0.45), (ep.EXPCONE, 0.3)])
def test_newton_rule_parity_damped(kernel, sigma):
    pr = w.circle_to_ellipse(16, sigma=sigma, kernel=kernel, steps=12)
    prm = ep.params(dim=2, kernel=kernel, sigma=sigma, steps=12, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(pr.X, pr.Y, prm, ep.RULE_NEWTON, h=0.8, eps=1e-10, maxit=40)
    rp, st, it, r, hist = o.match_newton(pr.X, pr.Y, kernel, sigma, 12, h=0.8, eps=1e-10, maxit=40)
    assert res.status == st == ep.OK
    assert abs(res.iters - it) <= 1
    assert rel(res.p0, rp) < 1e-7


@pytest.mark.parametrize("kernel,sigma,h", [(ep.TENT, 0.45, 0.5), (ep.EXPCONE, 0.3, 0.7), (ep.GAUSS, 0.12, 0.6)])
def test_velocity_rule_parity(kernel, sigma, h):
    pr = w.circle_to_ellipse(16, sigma=sigma, kernel=kernel, steps=20)
    prm = ep.params(dim=2, kernel=kernel, sigma=sigma, steps=20, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(pr.X, pr.Y, prm, ep.RULE_VELOCITY, h=h, eps=1e-8, maxit=100)
    rp, st, it, r, hist = o.match_velocity(pr.X, pr.Y, kernel, sigma, 20, h=h, eps=1e-8, maxit=100)
    assert res.status == st
    assert abs(res.iters - it) <= 1
    k = min(len(res.hist), len(hist))
    np.testing.assert_allclose(res.hist[:k], hist[:k], rtol=1e-6, atol=1e-12)
    if res.iters == it:
        assert rel(res.p0, rp) < 1e-8


def test_velocity_rule_fixed_iterations_3d():
    # a fixed number of updates compared iterate by iterate (no convergence test involved)
    X, p = cloud(40, 3, seed=95)
    Y = X + 0.05 * np.random.default_rng(96).normal(size=X.shape)
    prm = ep.params(dim=3, kernel=ep.EXPCONE, sigma=0.15, steps=8, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(X, Y, prm, ep.RULE_VELOCITY, h=0.5, eps=0.0, maxit=6)
    rp, st, it, r, hist = o.match_velocity(X, Y, ep.EXPCONE, 0.15, 8, h=0.5, eps=0.0, maxit=6)
    assert res.status == st == ep.ENOTCONVERGED and res.iters == it == 6
    assert rel(res.p0, rp) < 1e-9
    np.testing.assert_allclose(res.hist, hist, rtol=1e-9)
    assert res.products >= 6


def test_velocity_rule_ragged_rows_2d():
    # 300 landmarks: two rows on most CTAs, one on the rest (the MINRES sums span every CTA)
    # (tent sigma = 0.03 against a mean spacing of 0.035: cond G(X) = 31)
    X, _ = cloud(300, 2, seed=98, sigma=0.03)
    Y = X + 0.005 * np.random.default_rng(99).normal(size=X.shape)
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=0.03, steps=4, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(X, Y, prm, ep.RULE_VELOCITY, h=0.5, eps=0.0, maxit=3)
    rp, st, it, r, hist = o.match_velocity(X, Y, ep.TENT, 0.03, 4, h=0.5, eps=0.0, maxit=3)
    assert res.iters == it == 3
    assert rel(res.p0, rp) < 1e-9
    np.testing.assert_allclose(res.hist, hist, rtol=1e-9)


def test_rule_refusals():
    X, _ = cloud(20, 2, seed=97)
    Y = X + 0.01
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.2, steps=4, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    # the mixed-precision Newton gain forms the whole Jacobian (n dim <= 384), the mixed
    # velocity update factors G(X) (n <= 512)
    Xb, _ = cloud(200, 2, seed=96)
    with pytest.raises(ep.EPError):
        _match(Xb, Xb + 0.01, prm, ep.RULE_NEWTON, maxit=3)
    Xc = np.random.default_rng(95).uniform(0, 1, size=(600, 2))
    with pytest.raises(ep.EPError):
        _match(Xc, Xc + 0.01, prm, ep.RULE_VELOCITY, maxit=3)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.2, steps=4, precision=ep.FP64, neigh=ep.ALLPAIRS, inexact=0.1)
    with pytest.raises(ep.EPError):
        _match(X, Y, prm, ep.RULE_NEWTON, maxit=3)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.2, steps=4, precision=ep.FP64, neigh=ep.ALLPAIRS)
    with pytest.raises(ep.EPError):
        _match(X, Y, prm, 7, maxit=3)
    with pytest.raises(ep.EPError):
        ep.shoot_tangent(X, X, X, X, ep.params(dim=2, kernel=ep.GAUSS, sigma=0.2, steps=4, precision=ep.MIXED,
                                               neigh=ep.ALLPAIRS))


def test_newton_rule_krylov_path_parity():
    # n dim = 420 > 384: the Newton update runs restarted GMRES over tangent shoots instead
    # of the dense Jacobian; two updates compared iterate by iterate (cond D phi ~ 3)
    X = np.stack(np.meshgrid(np.arange(14), np.arange(15)), -1).reshape(-1, 2) * 0.04 + 0.2
    Y = X + 0.002 * np.random.default_rng(42).normal(size=X.shape)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.02, steps=4, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(X, Y, prm, ep.RULE_NEWTON, h=1.0, eps=0.0, maxit=2)
    rp, st, it, r, hist = o.match_newton(X, Y, ep.GAUSS, 0.02, 4, h=1.0, eps=0.0, maxit=2)
    assert res.status == st == ep.ENOTCONVERGED and res.iters == it == 2
    assert rel(res.p0, rp) < 1e-8
    np.testing.assert_allclose(res.hist, hist, rtol=1e-6)
    assert res.products > 2 * 10  # Krylov products, not dense columns (2 x 420)
    assert res.products != 2 * X.size


def test_newton_rule_dense_path_counts_columns():
    # n dim = 24 <= 384: each update forms the whole Jacobian, n dim tangent shoots
    pr = w.circle_to_ellipse(12, sigma=0.1, kernel=ep.GAUSS, steps=10)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=10, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(pr.X, pr.Y, prm, ep.RULE_NEWTON, h=1.0, eps=0.0, maxit=3)
    rp, st, it, r, hist = o.match_newton(pr.X, pr.Y, o.GAUSS, 0.1, 10, h=1.0, eps=0.0, maxit=3)
    assert res.iters == it == 3 and res.products == 3 * 24
    assert rel(res.p0, rp) < 1e-9
    big = hist > 1e-6
    np.testing.assert_allclose(res.hist[big], hist[big], rtol=1e-6)


# --------------------------------------------------------------------------- the benchmark's configurations


def test_newton_bench_workload():
    # the bench row: circle -> ellipse, 64 landmarks, tent sigma = 0.25, 50 steps, h = 1, eps = 1e-6
    c = w.circle_to_ellipse()
    prm = ep.params(dim=2, kernel=c.kernel, sigma=c.sigma, steps=c.steps, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(c.X, c.Y, prm, ep.RULE_NEWTON, h=1.0, eps=c.eps, maxit=c.maxit)
    rp, st, it, r, hist = o.match_newton(c.X, c.Y, c.kernel, c.sigma, c.steps, h=1.0, eps=c.eps, maxit=c.maxit)
    assert res.status == st == ep.OK and res.iters == it
    assert rel(res.p0, rp) < 1e-7
    big = hist > 1e-6
    np.testing.assert_allclose(res.hist[big], hist[big], rtol=1e-6)


def test_velocity_rule_bench_workload():
    # the bench row: the same workload with the velocity update, h = 0.5
    c = w.circle_to_ellipse()
    prm = ep.params(dim=2, kernel=c.kernel, sigma=c.sigma, steps=c.steps, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(c.X, c.Y, prm, ep.RULE_VELOCITY, h=0.5, eps=c.eps, maxit=c.maxit)
    rp, st, it, r, hist = o.match_velocity(c.X, c.Y, c.kernel, c.sigma, c.steps, h=0.5, eps=c.eps, maxit=c.maxit)
    assert res.status == st == ep.OK
    assert abs(res.iters - it) <= 1
    k = min(len(res.hist), len(hist))
    np.testing.assert_allclose(res.hist[:k], hist[:k], rtol=1e-6, atol=1e-12)


def test_tangent_shoot_bench_workload():
    # the bench row: N = 1024 Fourier curve, Gaussian sigma = 0.1, 50 steps, direction (0, v)
    f = w.fourier_curve_warp(n=1024, steps=50)
    p0 = 0.002 * (f.Y - f.X)
    v = np.random.default_rng(3).normal(size=f.X.shape)
    z = np.zeros_like(f.X)
    prm = ep.params(dim=2, kernel=f.kernel, sigma=f.sigma, steps=50, precision=ep.FP64, neigh=ep.ALLPAIRS)
    q1, p1, vq1, vp1 = ep.shoot_tangent(cuda(f.X), cuda(p0), cuda(z), cuda(v), prm)
    rq, rp, rvq, rvp = o.shoot_tangent(f.X, p0, z, v, f.kernel, f.sigma, 50)
    assert rel(q1, rq) < 1e-12 and rel(p1, rp) < 1e-11
    assert rel(vq1, rvq) < 1e-10 and rel(vp1, rvp) < 1e-10


def test_velocity_rule_minres_path():
    # n = 624 > 512: G(X) is not factored and every update runs MINRES inside the launch
    # (tent sigma = 0.03 on a 0.025 grid: cond G(X) ~ 5); two updates, iterate by iterate
    X = np.stack(np.meshgrid(np.arange(26), np.arange(24)), -1).reshape(-1, 2) * 0.025 + 0.2
    Y = X + 0.002 * np.random.default_rng(7).normal(size=X.shape)
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=0.03, steps=4, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(X, Y, prm, ep.RULE_VELOCITY, h=0.5, eps=0.0, maxit=2)
    rp, st, it, r, hist = o.match_velocity(X, Y, ep.TENT, 0.03, 4, h=0.5, eps=0.0, maxit=2)
    assert res.iters == it == 2
    assert res.products > 2 * 2  # MINRES Gram products, not one solve per component and update
    assert rel(res.p0, rp) < 1e-9
    np.testing.assert_allclose(res.hist, hist, rtol=1e-9)


# --------------------------------------------------------------------------- degenerate cases


@pytest.mark.parametrize("rule", [ep.RULE_NEWTON, ep.RULE_VELOCITY])
def test_rules_one_particle_land_in_one_step(rule):
    # one Gaussian particle: Q(1) = X + p0, so D phi = I and G(X) = [1]: a full step lands
    X, Y = np.array([[0.3, 0.4]]), np.array([[0.35, 0.42]])
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.2, steps=5, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(X, Y, prm, rule, h=1.0, eps=1e-13, maxit=5)
    assert res.status == ep.OK and res.iters == 1 and res.resid < 1e-15
    np.testing.assert_allclose(host(res.p0), Y - X, rtol=0, atol=1e-16)


@pytest.mark.parametrize("rule", [ep.RULE_NEWTON, ep.RULE_VELOCITY])
def test_rules_no_update_and_converged_start(rule):
    pr = w.circle_to_ellipse(12, sigma=0.1, kernel=ep.GAUSS, steps=10)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=10, precision=ep.FP64, neigh=ep.ALLPAIRS)
    # maxit = 0: one shoot, no update, the residual of p0 = 0 is max |Y - X|
    res = _match(pr.X, pr.Y, prm, rule, h=1.0, eps=0.0, maxit=0)
    assert res.status == ep.ENOTCONVERGED and res.iters == 0 and res.products == 0
    assert res.resid == pytest.approx(np.abs(pr.Y - pr.X).max(), rel=1e-15)
    np.testing.assert_array_equal(host(res.p0), 0.0)
    # Y = X: converged before any update
    res = _match(pr.X, pr.X, prm, rule, h=1.0, eps=1e-12, maxit=5)
    assert res.status == ep.OK and res.iters == 0 and res.resid == 0.0


# --------------------------------------------------------------------------- both sides of each solver switch


def _grid(nx, ny, h, extra):
    X = np.stack(np.meshgrid(np.arange(nx), np.arange(ny)), -1).reshape(-1, 2) * h + 0.2
    return np.vstack([X, [[0.97, 0.97]]]) if extra else X  # one far point crosses the threshold


@pytest.mark.parametrize("extra", [0, 1])
def test_velocity_rule_at_the_factoring_threshold(extra):
    # 512 landmarks: G(X) factored; 513: MINRES (tent sigma = 0.03 on a 0.025 grid)
    X = _grid(32, 16, 0.025, extra)
    Y = X + 0.002 * np.random.default_rng(11).normal(size=X.shape)
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=0.03, steps=4, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(X, Y, prm, ep.RULE_VELOCITY, h=0.5, eps=0.0, maxit=1)
    rp, st, it, r, hist = o.match_velocity(X, Y, ep.TENT, 0.03, 4, h=0.5, eps=0.0, maxit=1)
    assert res.iters == it == 1
    assert (res.products == 2) == (X.shape[0] <= 512)  # one solve per component when factored
    assert rel(res.p0, rp) < 1e-9
    np.testing.assert_allclose(res.hist, hist, rtol=1e-9)


@pytest.mark.parametrize("extra", [0, 1])
def test_newton_rule_at_the_dense_threshold(extra):
    # 192 landmarks (n dim = 384): dense Jacobian; 193 (386): Krylov (Gaussian sigma = 0.02, 0.04 grid)
    X = _grid(16, 12, 0.04, extra)
    Y = X + 0.002 * np.random.default_rng(12).normal(size=X.shape)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.02, steps=4, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(X, Y, prm, ep.RULE_NEWTON, h=1.0, eps=0.0, maxit=1)
    rp, st, it, r, hist = o.match_newton(X, Y, ep.GAUSS, 0.02, 4, h=1.0, eps=0.0, maxit=1)
    assert res.iters == it == 1
    assert (res.products == X.size) == (X.size <= 384)  # the Jacobian's columns when dense
    assert rel(res.p0, rp) < 1e-8
    np.testing.assert_allclose(res.hist, hist, rtol=1e-8)


@pytest.mark.parametrize("extra", [0, 1])
def test_newton_rule_at_the_shared_memory_lu_threshold(extra):
    # 80 landmarks (n dim = 160): the LU runs on a shared-memory copy of D phi (the
    # largest, ~206 KB); 81 (162): in global memory.  Two Newton updates on each side.
    X = _grid(10, 8, 0.04, extra)
    Y = X + 0.002 * np.random.default_rng(13).normal(size=X.shape)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.03, steps=4, precision=ep.FP64, neigh=ep.ALLPAIRS)
    res = _match(X, Y, prm, ep.RULE_NEWTON, h=1.0, eps=0.0, maxit=2)
    rp, st, it, r, hist = o.match_newton(X, Y, ep.GAUSS, 0.03, 4, h=1.0, eps=0.0, maxit=2)
    assert X.size == (162 if extra else 160)
    assert res.iters == it == 2
    assert res.products == 2 * X.size
    assert rel(res.p0, rp) < 1e-8
    np.testing.assert_allclose(res.hist, hist, rtol=1e-8)


@pytest.mark.parametrize("n,prec", [(2, ep.FP64), (82, ep.FP64), (2, ep.MIXED)])
def test_newton_singular_jacobian_keeps_the_last_iterate(n, prec):
    # Two coincident landmarks: at p0 = 0 the shoot is Q(1) = X + G(X) p0 to first order,
    # so D phi has two equal rows and columns and the elimination meets an exact zero
    # pivot.  The match returns EP_EDIVERGED with p0 left at the iterate it was shot
    # from (the initial guess), no update counted, and that shoot's finite residual.
    # n dim = 4 factors in shared memory, 164 in global memory.
    X = _grid(9, 9, 0.05, 0)[: n - 1] if n > 2 else np.array([[0.4, 0.5]])
    X = np.vstack([X, X[-1:]])
    Y = X + 0.01 * np.random.default_rng(14).normal(size=X.shape)
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=0.12, steps=5, precision=prec, neigh=ep.ALLPAIRS)
    res = _match(X, Y, prm, ep.RULE_NEWTON, h=1.0, eps=1e-9, maxit=5)
    assert res.status == ep.EDIVERGED
    assert res.iters == 0
    assert np.all(host(res.p0) == 0.0)
    assert np.isfinite(res.resid) and res.resid == pytest.approx(np.abs(Y - X).max(), rel=1e-6)
    assert "singular" in ep.last_error()


# --------------------------------------------------------------------------- mixed precision (Newton)


@pytest.mark.parametrize("kernel,sigma,n,h", [(ep.GAUSS, 0.1, 12, 1.0), (ep.TENT, 0.45, 16, 0.8),
                                              (ep.EXPCONE, 0.3, 16, 0.8)])
def test_newton_rule_mixed_precision(kernel, sigma, n, h):
    # FP32 Jacobian (an inexact Newton method), FP64 residual, solve and update: the
    # iteration converges to the mixed shooting map's root, which agrees with the FP64
    # oracle's to the mixed-precision bound.  The mixed shoot's endpoint carries FP32
    # rounding noise of ~1e-8 (the residual cannot fall below it), so eps = 1e-7.
    pr = w.circle_to_ellipse(n, sigma=sigma, kernel=kernel, steps=12)
    prm = ep.params(dim=2, kernel=kernel, sigma=sigma, steps=12, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    res = _match(pr.X, pr.Y, prm, ep.RULE_NEWTON, h=h, eps=1e-7, maxit=40)
    rp, st, it, r, hist = o.match_newton(pr.X, pr.Y, kernel, sigma, 12, h=h, eps=1e-7, maxit=40)
    assert res.status == st == ep.OK
    assert it <= res.iters <= it + 3
    assert rel(res.p0, rp) < 1e-4
    assert res.products == res.iters * pr.X.size
    # early iterates follow the exact Newton iteration closely
    np.testing.assert_allclose(res.hist[:2], hist[:2], rtol=1e-4)


def test_newton_rule_mixed_3d():
    X, _ = cloud(30, 3, seed=93)
    Y = X + 0.01 * np.random.default_rng(94).normal(size=X.shape)
    prm = ep.params(dim=3, kernel=ep.GAUSS, sigma=0.15, steps=6, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    res = _match(X, Y, prm, ep.RULE_NEWTON, h=1.0, eps=1e-7, maxit=20)
    rp, st, it, r, hist = o.match_newton(X, Y, ep.GAUSS, 0.15, 6, h=1.0, eps=1e-7, maxit=20)
    assert res.status == st == ep.OK and it <= res.iters <= it + 3
    assert rel(res.p0, rp) < 1e-4


# --------------------------------------------------------------------------- the C ABI: host arrays, device history, initial guess


@pytest.mark.parametrize("rule", [ep.RULE_NEWTON, ep.RULE_VELOCITY])
def test_rules_host_arrays_and_initial_guess(rule):
    pr = w.circle_to_ellipse(12, sigma=0.1, kernel=ep.GAUSS, steps=10)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=10, precision=ep.FP64, neigh=ep.ALLPAIRS)
    h = 1.0 if rule == ep.RULE_NEWTON else 0.5
    f = o.match_newton if rule == ep.RULE_NEWTON else o.match_velocity
    # numpy in, numpy out
    res = ep.match(pr.X, pr.Y, prm, h=h, eps=0.0, maxit=2, rule=rule)
    assert isinstance(res.p0, np.ndarray)
    rp = f(pr.X, pr.Y, o.GAUSS, 0.1, 10, h=h, eps=0.0, maxit=2)[0]
    assert rel(res.p0, rp) < 1e-9
    # a non-zero initial guess: two more updates from there equal four from zero
    res2 = ep.match(pr.X, pr.Y, prm, h=h, eps=0.0, maxit=2, rule=rule, p0=res.p0)
    rp4 = f(pr.X, pr.Y, o.GAUSS, 0.1, 10, h=h, eps=0.0, maxit=4)[0]
    assert rel(res2.p0, rp4) < 1e-8


@pytest.mark.parametrize("rule", [ep.RULE_NEWTON, ep.RULE_VELOCITY])
def test_rules_history_in_device_memory(rule):
    import ctypes
    pr = w.circle_to_ellipse(12, sigma=0.1, kernel=ep.GAUSS, steps=10)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=10, precision=ep.FP64, neigh=ep.ALLPAIRS)
    X, Y = cuda(pr.X), cuda(pr.Y)
    p = torch.zeros_like(X)
    hist = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    info = ep.MatchInfo(0.5, 0.0, 3, 0, 0.0, 0.0, hist.data_ptr(), int(rule), 0)
    lib = ep.load()
    st = lib.ep_match(ctypes.byref(ep._with_dim(prm, 2)), 12, X.data_ptr(), Y.data_ptr(), p.data_ptr(),
                      ctypes.byref(info), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st == ep.ENOTCONVERGED and info.iters == 3
    f = o.match_newton if rule == ep.RULE_NEWTON else o.match_velocity
    rp, _, _, _, rh = f(pr.X, pr.Y, o.GAUSS, 0.1, 10, h=0.5, eps=0.0, maxit=3)
    np.testing.assert_allclose(hist.cpu().numpy(), rh, rtol=1e-9)
    assert rel(p, rp) < 1e-9
    assert info.resid_inf == pytest.approx(rh[-1], rel=1e-9)


# --------------------------------------------------------------------------- mixed precision (velocity update)


@pytest.mark.parametrize("kernel,sigma,h", [(ep.TENT, 0.45, 0.5), (ep.EXPCONE, 0.3, 0.7), (ep.GAUSS, 0.12, 0.6)])
def test_velocity_rule_mixed_precision(kernel, sigma, h):
    # mixed shoots, G(X) in FP64 factored once: the iterates follow the FP64 oracle's to the
    # mixed-precision bound (eps above the mixed shoot's ~1e-8 endpoint noise)
    pr = w.circle_to_ellipse(16, sigma=sigma, kernel=kernel, steps=20)
    prm = ep.params(dim=2, kernel=kernel, sigma=sigma, steps=20, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    res = _match(pr.X, pr.Y, prm, ep.RULE_VELOCITY, h=h, eps=1e-7, maxit=100)
    rp, st, it, r, hist = o.match_velocity(pr.X, pr.Y, kernel, sigma, 20, h=h, eps=1e-7, maxit=100)
    assert res.status == st == ep.OK
    assert abs(res.iters - it) <= 1
    k = min(len(res.hist), len(hist))
    # residuals differ by the mixed shoot's endpoint error (~2e-8 here; the mixed bound is
    # 1e-4 of the positions)
    np.testing.assert_allclose(res.hist[:k], hist[:k], rtol=1e-4, atol=1e-6)
    assert rel(res.p0, rp) < 1e-4


def test_velocity_rule_mixed_bench_workload():
    c = w.circle_to_ellipse()
    prm = ep.params(dim=2, kernel=c.kernel, sigma=c.sigma, steps=c.steps, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    res = _match(c.X, c.Y, prm, ep.RULE_VELOCITY, h=0.5, eps=c.eps, maxit=c.maxit)
    rp, st, it, r, hist = o.match_velocity(c.X, c.Y, c.kernel, c.sigma, c.steps, h=0.5, eps=c.eps, maxit=c.maxit)
    assert res.status == st == ep.OK and abs(res.iters - it) <= 1
    assert rel(res.p0, rp) < 1e-4


@pytest.mark.parametrize("dim,n", [(3, 24), (2, 400)])
def test_velocity_rule_mixed_host_loop(dim, n):
    # beyond the one-launch solver (3-D, or planar n > 384): mixed persistent shoots and
    # one warp's substitutions with the factored G(X) per update, on the host loop
    sigma = 0.08 if dim == 3 else 0.03
    X, _ = cloud(n, dim, seed=31 + dim, sigma=sigma, band=1e-4)
    Y = X + 0.002 * np.random.default_rng(32).normal(size=X.shape)
    prm = ep.params(dim=dim, kernel=ep.TENT, sigma=sigma, steps=6, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    res = _match(X, Y, prm, ep.RULE_VELOCITY, h=0.5, eps=0.0, maxit=3)
    rp, st, it, r, hist = o.match_velocity(X, Y, ep.TENT, sigma, 6, h=0.5, eps=0.0, maxit=3)
    assert res.iters == it == 3 and res.products == 3 * dim
    assert rel(res.p0, rp) < 1e-4
    np.testing.assert_allclose(res.hist, hist, rtol=1e-4)
