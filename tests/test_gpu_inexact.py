"""The inexact particle system (Sec. 6, Eq. N-particle-inexact: dq_i gains
sigma_n^2 p_i) on the GPU against the FP64 oracle through the C ABI: right-hand
side, shoot, and Algorithm 1 with the momentum-difference stop.  Tolerances as for
the exact system (mixed: RHS 1e-5, endpoints and momenta 1e-4; FP64 1e-12)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as o  # noqa: E402
from paper_1510_03816_gb300 import ep, workloads as w  # noqa: E402

KSIG = [(ep.GAUSS, 0.1), (ep.TENT, 0.15), (ep.EXPCONE, 0.08)]
S2 = 0.3


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


def cloud(n, dim, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.2, 0.8, size=(n, dim)), rng.normal(0, 0.05, size=(n, dim))


def tent_boundary_rows(q, sigma, band=1e-5):
    d = np.linalg.norm(q[:, None, :] - q[None, :, :], axis=-1)
    return np.any(np.abs(d - sigma) < band * sigma, axis=1)


@pytest.mark.parametrize("prec", [ep.MIXED, ep.FP64])
@pytest.mark.parametrize("kernel,sigma", KSIG)
@pytest.mark.parametrize("dim", [2, 3])
def test_rhs_parity(prec, kernel, sigma, dim):
    q, p = cloud(300, dim, seed=20 + dim + kernel)
    prm = ep.params(dim=dim, kernel=kernel, sigma=sigma, precision=prec, neigh=ep.ALLPAIRS, inexact=S2)
    dq, dp = ep.rhs(cuda(q), cuda(p), prm)
    rq, rp = o.rhs_inexact(q, p, kernel, sigma, S2)
    tol = 1e-12 if prec == ep.FP64 else 1e-5
    assert rel(dq, rq) < tol
    keep = ~tent_boundary_rows(q, sigma) if kernel == ep.TENT else np.ones(len(q), bool)
    assert rel(dp.cpu().numpy()[keep], rp[keep]) < tol


@pytest.mark.parametrize("prec", [ep.MIXED, ep.FP64])
@pytest.mark.parametrize("kernel,sigma", KSIG)
@pytest.mark.parametrize("dim", [2, 3])
def test_shoot_parity(prec, kernel, sigma, dim):
    q, p = cloud(200, dim, seed=30 + dim + kernel)
    prm = ep.params(dim=dim, kernel=kernel, sigma=sigma, steps=6, precision=prec, neigh=ep.ALLPAIRS, inexact=S2)
    q1, p1 = ep.shoot(cuda(q), cuda(p), prm)
    rq, rp = o.shoot_inexact(q, p, kernel, sigma, S2, 6)
    tol = 1e-12 if prec == ep.FP64 else 1e-4
    assert rel(q1, rq) < tol and rel(p1, rp) < tol


@pytest.mark.parametrize("n", [1000, 5000])
def test_persistent_2d_gaussian_shoot(n):
    """The owner-computes / stream-K persistent kernels carry the inexact term too."""
    pr = w.fourier_curve_warp(n=n)
    p0 = 0.002 * (pr.Y - pr.X)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=5, precision=ep.MIXED, neigh=ep.ALLPAIRS, inexact=0.05)
    q1, p1 = ep.shoot(cuda(pr.X), cuda(p0), prm)
    rq, rp = o.shoot_inexact(pr.X, p0, ep.GAUSS, 0.1, 0.05, 5)
    assert rel(q1, rq) < 1e-4 and rel(p1, rp) < 1e-4
    assert np.abs(q1.cpu().numpy() - rq).max() < 1e-6


@pytest.mark.parametrize("prec", [ep.FP64, ep.MIXED])
def test_match_momentum_difference_stop(prec):
    pr = w.circle_to_ellipse(64)
    prm = ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, steps=20, precision=prec, neigh=ep.ALLPAIRS,
                    inexact=0.05)
    r = ep.match(cuda(pr.X), cuda(pr.Y), prm, h=0.0, eps=2e-4, maxit=300)
    p, st, it, res, hist = o.match_inexact(pr.X, pr.Y, pr.kernel, pr.sigma, 0.05, 20, h=0.0, eps=2e-4, maxit=300)
    assert st == ep.OK and r.status == st and r.iters == it
    tol = 1e-12 if prec == ep.FP64 else 1e-4
    # default gain 1 / (max row sum + sigma_n^2); mixed precision sums G in FP32
    assert abs(r.h - 1.0 / (1.0 / o.default_gain(pr.X, pr.kernel, pr.sigma) + 0.05)) < (
        1e-12 if prec == ep.FP64 else 1e-6) * r.h
    assert rel(r.p0, p) < tol
    assert len(r.hist) == len(hist) == it
    np.testing.assert_allclose(r.hist, hist, rtol=tol)


def test_paths_without_the_inexact_system_refuse_it():
    q, p = cloud(40, 2, seed=1)
    bad = ep.params(dim=2, kernel=ep.TENT, sigma=0.1, steps=3, neigh=ep.CELLLIST, inexact=0.1)
    with pytest.raises(ep.EPError):
        ep.rhs(cuda(q), cuda(p), bad)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=3, neigh=ep.ALLPAIRS, inexact=0.1)
    with pytest.raises(ep.EPError):
        ep.adjoint(cuda(q), cuda(p), cuda(q), prm, 10.0, 1)
    with pytest.raises(ep.EPError):
        ep.match_batched([q], [q], [prm], maxit=1)
    with pytest.raises(ep.EPError):
        ep.flow(cuda(q), cuda(p), cuda(q), prm)
    with pytest.raises(ep.EPError):
        ep.rhs(cuda(q), cuda(p), ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, inexact=-1.0))
