"""ep_velocity (Eq. u at arbitrary points) and ep_flow (points carried by the flow
of a shoot) against the FP64 oracle through the C ABI.

Tolerances: FP64 mode <= 1e-12 relative; mixed precision (FP32 pair terms and
FP32 per-stage sums, as the particles' own mixed shoot): velocities <= 1e-5
relative (the RHS bound), transported points <= 1e-4 of the largest displacement
(the shoot's endpoint bound: the points follow the recorded stages of the mixed
shoot, whose 2-D Gaussian runs the factored pair form, ~4e-5 of the displacement
when points move half the domain), <= 2e-6 absolute where displacements are
O(0.05)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as o  # noqa: E402
from paper_1510_03816_gb300 import ep, workloads as w  # noqa: E402

KSIG = [(ep.GAUSS, 0.1), (ep.TENT, 0.15), (ep.EXPCONE, 0.08)]


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


def cloud(n, dim, seed, pscale=0.05):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.2, 0.8, size=(n, dim)), rng.normal(0, pscale, size=(n, dim))


@pytest.mark.parametrize("prec", [ep.MIXED, ep.FP64])
@pytest.mark.parametrize("kernel,sigma", KSIG)
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n,m", [(1, 1), (300, 777), (2049, 513)])
def test_velocity_parity(prec, kernel, sigma, dim, n, m):
    q, p = cloud(n, dim, seed=n + m + dim + kernel)
    x = np.random.default_rng(m).uniform(0.1, 0.9, size=(m, dim))
    prm = ep.params(dim=dim, kernel=kernel, sigma=sigma, precision=prec, neigh=ep.ALLPAIRS)
    u = ep.velocity(cuda(q), cuda(p), cuda(x), prm)
    ref = o.velocity(q, p, x, kernel, sigma)
    assert rel(u, ref) < (1e-12 if prec == ep.FP64 else 1e-5)


@pytest.mark.parametrize("prec", [ep.MIXED, ep.FP64])
def test_velocity_at_particles_equals_rhs_dq(prec):
    q, p = cloud(500, 2, seed=1)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, precision=prec, neigh=ep.ALLPAIRS)
    u = ep.velocity(cuda(q), cuda(p), cuda(q), prm)
    dq, _ = ep.rhs(cuda(q), cuda(p), prm)
    assert rel(u, dq.cpu().numpy()) < (1e-13 if prec == ep.FP64 else 1e-5)


@pytest.mark.parametrize("prec", [ep.MIXED, ep.FP64])
@pytest.mark.parametrize("kernel,sigma", KSIG)
@pytest.mark.parametrize("dim", [2, 3])
def test_flow_parity(prec, kernel, sigma, dim):
    q, p = cloud(200, dim, seed=7 + dim + kernel, pscale=0.1)
    x0 = np.random.default_rng(8).uniform(0.1, 0.9, size=(300, dim))
    prm = ep.params(dim=dim, kernel=kernel, sigma=sigma, steps=8, precision=prec, neigh=ep.ALLPAIRS)
    x1 = ep.flow(cuda(q), cuda(p), cuda(x0), prm)
    _, _, ref = o.flow(q, p, x0, kernel, sigma, 8)
    if prec == ep.FP64:
        assert rel(x1, ref) < 1e-12
    else:
        # mixed: relative to the displacement (these momenta move points by up to ~0.5)
        assert np.abs(x1.cpu().numpy() - ref).max() < 1e-4 * np.abs(ref - x0).max()


@pytest.mark.parametrize("prec", [ep.MIXED, ep.FP64])
def test_flow_tracers_on_particles_follow_the_shoot(prec):
    pr = w.fourier_curve_warp(n=1000)
    p0 = 0.002 * (pr.Y - pr.X)
    prm = ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, steps=12, precision=prec, neigh=ep.ALLPAIRS)
    X, P = cuda(pr.X), cuda(p0)
    x1 = ep.flow(X, P, X[::7], prm)
    q1, _ = ep.shoot(X, P, prm)
    err = np.abs(x1.cpu().numpy() - q1.cpu().numpy()[::7]).max()
    assert err < (1e-12 if prec == ep.FP64 else 2e-6)


def test_flow_full_size_sampled():
    """The N = 4096 Fourier-curve shoot (mixed) carrying a 64 x 64 grid; the oracle
    transports 48 sampled grid points (20 RK4 steps to keep the oracle short)."""
    pr = w.fourier_curve_warp()
    p0 = 0.002 * (pr.Y - pr.X)
    g = np.stack(np.meshgrid(np.linspace(0.1, 0.9, 64), np.linspace(0.1, 0.9, 64)), -1).reshape(-1, 2)
    prm = ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, steps=20, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    x1 = ep.flow(cuda(pr.X), cuda(p0), cuda(g), prm).cpu().numpy()
    rows = np.random.default_rng(3).choice(g.shape[0], 48, replace=False)
    _, _, ref = o.flow(pr.X, p0, g[rows], pr.kernel, pr.sigma, 20)
    assert np.abs(x1[rows] - ref).max() < 2e-6
    assert np.abs(x1 - g).max() > 1e-3  # the grid does move


def test_flow_and_velocity_edge_cases():
    q, p = cloud(50, 2, seed=9)
    x = np.random.default_rng(10).uniform(0.1, 0.9, size=(40, 2))
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=5, precision=ep.FP64, neigh=ep.ALLPAIRS)
    # host arrays in and out
    u = ep.velocity(q, p, x, prm)
    assert isinstance(u, np.ndarray) and rel(u, o.velocity(q, p, x, ep.GAUSS, 0.1)) < 1e-12
    x1 = ep.flow(q, p, x, prm)
    assert rel(x1, o.flow(q, p, x, ep.GAUSS, 0.1, 5)[2]) < 1e-12
    # no targets; no particles (zero velocity, identity flow); in-place flow
    assert ep.flow(q, p, np.zeros((0, 2)), prm).shape == (0, 2)
    np.testing.assert_array_equal(ep.velocity(np.zeros((0, 2)), np.zeros((0, 2)), x, prm), 0.0)
    np.testing.assert_array_equal(ep.flow(np.zeros((0, 2)), np.zeros((0, 2)), x, prm), x)
    xt, qt, pt = cuda(x), cuda(q), cuda(p)  # keep the tensors alive across the raw call
    lib = ep.load()
    import ctypes
    st = lib.ep_flow(ctypes.byref(ep._with_dim(prm, 2)), 50, qt.data_ptr(), pt.data_ptr(), 40,
                     xt.data_ptr(), xt.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == ep.OK
    assert rel(xt, o.flow(q, p, x, ep.GAUSS, 0.1, 5)[2]) < 1e-12
    with pytest.raises(ep.EPError):
        ep.flow(q, p, x, ep.params(dim=2, kernel=ep.TENT, sigma=0.1, steps=5, neigh=ep.CELLLIST))
