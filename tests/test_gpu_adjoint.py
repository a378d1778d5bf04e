"""GPU parity of the Hessian-vector product (ep_hvp) and of the discrete RK4 adjoint
(ep_adjoint) against the FP64 CPU oracle, through the C ABI.

Tolerances: FP64 mode <= 1e-10 (relative max-norm); mixed precision (FP32 pair
terms, FP64 sums): HVP <= 1e-5 (the RHS bound; measured <= 1.4e-6), gradient
<= 1e-4 (the shot-endpoint bound; measured <= 2e-7, and 9.5e-7 against the FP64
gradient at N = 16384 3-D), energy <= 1e-5.  The mixed gradient at the full 3-D
size is also checked by a directional finite difference of the energy, a property
that holds at any size.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as o  # noqa: E402
from paper_1510_03816_gb300 import ep, workloads as w  # noqa: E402

KSIG = [(ep.GAUSS, 0.15), (ep.TENT, 0.2), (ep.EXPCONE, 0.1)]


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


def tent_safe(q, sigma, band=1e-3):
    d = np.linalg.norm(q[:, None] - q[None], axis=-1)
    return not np.any(np.abs(d - sigma) < band * sigma)


def cloud(n, dim, seed, kernel, sigma):
    rng = np.random.default_rng(seed)
    for _ in range(200):
        q = rng.uniform(0.3, 0.7, size=(n, dim))
        if kernel != ep.TENT or tent_safe(q, sigma):
            break
    p = rng.normal(0, 0.02, size=(n, dim))
    return q, p


@pytest.mark.parametrize("prec", [ep.FP64, ep.MIXED])
@pytest.mark.parametrize("kernel,sigma", KSIG)
@pytest.mark.parametrize("dim", [2, 3])
def test_hvp_parity(prec, kernel, sigma, dim):
    n = 150
    q, p = cloud(n, dim, 3 + dim + kernel, kernel, sigma)
    rng = np.random.default_rng(7)
    vq, vp = rng.normal(size=q.shape), rng.normal(size=q.shape)
    prm = ep.params(dim=dim, kernel=kernel, sigma=sigma, precision=prec, neigh=ep.ALLPAIRS)
    hq, hp = ep.hvp(cuda(q), cuda(p), cuda(vq), cuda(vp), prm)
    rq, rp = o.hvp(q, p, vq, vp, kernel, sigma)
    tol = 1e-10 if prec == ep.FP64 else 1e-5
    assert rel(hq, rq) < tol
    assert rel(hp, rp) < tol


@pytest.mark.parametrize("prec", [ep.FP64, ep.MIXED])
@pytest.mark.parametrize("kernel,sigma", KSIG)
@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_parity(prec, kernel, sigma, dim):
    """Gradient and energy of E = 1/2 p0^T G p0 + lam/2 |Q(1)-Y|^2 with 8 RK4 steps
    checkpointed every 3 (segments of 3, 3, 2)."""
    n = 130
    X, p0 = cloud(n, dim, 11 + dim + kernel, kernel, sigma)
    rng = np.random.default_rng(8)
    Y = X + rng.normal(0, 0.02, size=X.shape)
    lam, steps = 50.0, 8
    prm = ep.params(dim=dim, kernel=kernel, sigma=sigma, steps=steps, precision=prec, neigh=ep.ALLPAIRS)
    E, g = ep.adjoint(cuda(X), cuda(p0), cuda(Y), prm, lam, ckpt_every=3)
    Er, gr = o.adjoint(X, p0, Y, kernel, sigma, steps, lam)
    if prec == ep.FP64:
        assert rel(g, gr) < 1e-10 and abs(E - Er) < 1e-10 * abs(Er)
    else:
        assert rel(g, gr) < 1e-4 and abs(E - Er) < 1e-5 * abs(Er)


def test_adjoint_checkpoint_interval_does_not_change_the_result():
    X, p0 = cloud(100, 2, 5, ep.GAUSS, 0.15)
    Y = X + 0.01
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.15, steps=10, precision=ep.FP64)
    g = [ep.adjoint(cuda(X), cuda(p0), cuda(Y), prm, 20.0, ckpt_every=c)[1] for c in (1, 4, 10, 50)]
    for gk in g[1:]:
        assert rel(gk, g[0].cpu().numpy()) < 1e-13


def test_adjoint_host_arrays_and_autograd():
    from paper_1510_03816_gb300 import autograd

    X, p0 = cloud(80, 2, 9, ep.EXPCONE, 0.1)
    Y = X + 0.02
    prm = ep.params(dim=2, kernel=ep.EXPCONE, sigma=0.1, steps=6, precision=ep.FP64)
    E, g = ep.adjoint(X, p0, Y, prm, 10.0, ckpt_every=2)  # numpy in/out
    Er, gr = o.adjoint(X, p0, Y, ep.EXPCONE, 0.1, 6, 10.0)
    assert rel(g, gr) < 1e-10 and abs(E - Er) < 1e-10 * abs(Er)
    p = cuda(p0).requires_grad_(True)
    e = autograd.inexact_energy(cuda(X), p, cuda(Y), prm, 10.0, ckpt_every=2)
    e.backward()
    assert abs(e.item() - Er) < 1e-10 * abs(Er)
    assert rel(p.grad, gr) < 1e-10


def test_adjoint_full_size_star_surface_directional_fd():
    """N = 16384 3-D, Gaussian sigma = 0.05, lambda = 100, 100 steps, checkpoints every 10
    (the configuration the adjoint is measured on): <grad, v> against a central
    difference of the mixed-precision energy along a random direction v."""
    pr = w.star_surface_3d()
    X, Y, p0 = cuda(pr.X), cuda(pr.Y), cuda(pr.p0)
    prm = ep.params(dim=3, kernel=pr.kernel, sigma=pr.sigma, steps=pr.steps, precision=ep.MIXED)
    E, g = ep.adjoint(X, p0, Y, prm, pr.lam, ckpt_every=10)
    v = cuda(np.random.default_rng(3).normal(size=pr.p0.shape))
    v = v / v.norm() * p0.norm()
    h = 1e-2
    Ep = ep.adjoint(X, p0 + h * v, Y, prm, pr.lam, ckpt_every=10)[0]
    Em = ep.adjoint(X, p0 - h * v, Y, prm, pr.lam, ckpt_every=10)[0]
    fd = (Ep - Em) / (2 * h)
    dd = float((g * v).sum())
    assert abs(fd - dd) < 2e-3 * abs(dd)


def test_adjoint_full_size_star_surface_fp64_central_differences():
    """The gradient check of the inexact-matching energy at its stated size (Sec. 6,
    Eq. inexact-E): N = 16384 3-D, Gaussian sigma = 0.05, lambda = 100, 100 RK4 steps,
    checkpoints every 10, FP64.  <dE/dp0, v> from the discrete adjoint against the
    central difference (E(p0 + h v) - E(p0 - h v)) / 2h with h = 1e-4, every energy in
    FP64 (1/2 p0^T G(X) p0 = H(X, p0) of Eq. H, plus lambda/2 |Q(1) - Y|^2 from the plain
    FP64 shoot); the O(h^2) truncation leaves ~1e-8 of the derivative.  The mixed-
    precision gradient agrees with the FP64 one to the adjoint's mixed bound."""
    pr = w.star_surface_3d()
    X, Y, p0 = cuda(pr.X), cuda(pr.Y), cuda(pr.p0)
    prm = ep.params(dim=3, kernel=pr.kernel, sigma=pr.sigma, steps=pr.steps, precision=ep.FP64)
    E, g = ep.adjoint(X, p0, Y, prm, pr.lam, ckpt_every=10)

    def energy(p):
        q1, _ = ep.shoot(X, p, prm)
        return ep.hamiltonian(X, p, prm) + 0.5 * pr.lam * float(((q1 - Y) ** 2).sum())

    assert abs(energy(p0) - E) < 1e-11 * abs(E)
    v = cuda(np.random.default_rng(17).normal(size=pr.p0.shape))
    v = v / v.norm() * p0.norm()
    h = 1e-4
    fd = (energy(p0 + h * v) - energy(p0 - h * v)) / (2 * h)
    dd = float((g * v).sum())
    assert abs(fd - dd) < 1e-6 * abs(dd)
    prm_m = ep.params(dim=3, kernel=pr.kernel, sigma=pr.sigma, steps=pr.steps, precision=ep.MIXED)
    Em, gm = ep.adjoint(X, p0, Y, prm_m, pr.lam, ckpt_every=10)
    assert rel(gm, g.cpu().numpy()) < 1e-4
    assert abs(Em - E) < 1e-4 * abs(E)
