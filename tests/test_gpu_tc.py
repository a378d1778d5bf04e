"""The tensor-core (tcgen05) path of the 2-D Gaussian in mixed precision: parity
with the FP64 oracle on ragged sizes, on multi-block segments and on tiles that
take the CUDA-core difference form (|q_i|^2 beyond the factoring bound), and
agreement with the CUDA-core path (the default; EP_TC=1 selects the tensor
cores) through the C ABI.

Tolerances as for the mixed path: RHS <= 1e-5, shot endpoints <= 1e-4 relative
(max-norm of the difference over the max-norm of the oracle's block).  The
factored form sums G_ij p_j and G_ij q_j (x) p_j about a common tile centre, so
dp carries an absolute floor of a few FP32 roundings of |q_i - c| |p|^2 / sigma^2
(the self term cancels only to that level): where the exact dp nearly cancels
(two distant particles) the dp bound adds 1e-6 |p|_max^2 R / sigma^2, R = half
the diagonal of the particles' bounding box."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as o  # noqa: E402
from paper_1510_03816_gb300 import ep, workloads as w  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_03816_gb300 import build

    build.build()
    o.build()
    ep.load()
    old = os.environ.get("EP_TC")
    os.environ["EP_TC"] = "1"  # the tensor-core path is opt-in
    yield
    if old is None:
        del os.environ["EP_TC"]
    else:
        os.environ["EP_TC"] = old


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def dp_floor_scale(q, sigma):
    """R / sigma^2 with R = half the diagonal of the bounding box of q."""
    return 0.5 * np.linalg.norm(q.max(0) - q.min(0)) / sigma ** 2


def prm(sigma=0.1, steps=1):
    return ep.params(dim=2, kernel=ep.GAUSS, sigma=sigma, steps=steps, precision=ep.MIXED, neigh=ep.ALLPAIRS)


class cuda_core_path:
    """EP_TC=0 for the duration (the library reads it on every call)."""

    def __enter__(self):
        self.old = os.environ.get("EP_TC")
        os.environ["EP_TC"] = "0"

    def __exit__(self, *a):
        if self.old is None:
            del os.environ["EP_TC"]
        else:
            os.environ["EP_TC"] = self.old


@pytest.mark.parametrize("n", [1, 2, 3, 63, 64, 65, 127, 128, 129, 1000, 3001])
def test_rhs_ragged_sizes_cloud(n):
    """Uniform cloud in [0.2, 0.8]^2 (every pair interacts: dp is well conditioned)."""
    rng = np.random.default_rng(100 + n)
    q = rng.uniform(0.2, 0.8, size=(n, 2))
    p = rng.normal(0, 0.05, size=(n, 2))
    dq, dp = ep.rhs(cuda(q), cuda(p), prm())
    rq, rp = o.rhs(q, p, ep.GAUSS, 0.1)
    assert rel(dq, rq) < 1e-5
    floor = 1e-6 * np.abs(p).max() ** 2 * dp_floor_scale(q, 0.1)
    assert np.abs(dp.cpu().numpy() - rp).max() <= 1e-5 * np.abs(rp).max() + floor


@pytest.mark.parametrize("n", [63, 64, 65, 127, 128, 129, 1000, 3001])
def test_rhs_ragged_sizes_curve(n):
    pr = w.fourier_curve_warp(n=n)
    p = 0.01 * (pr.Y - pr.X)
    dq, dp = ep.rhs(cuda(pr.X), cuda(p), prm())
    rq, rp = o.rhs(pr.X, p, ep.GAUSS, 0.1)
    assert rel(dq, rq) < 1e-5
    assert rel(dp, rp) < 1e-5


def test_rhs_difference_form_tiles():
    """A compact curve (factored tiles) followed by particles spread over a box 40
    sigma wide (|q_i|^2 far beyond the bound: the CUDA-core difference form), in
    one call; also a tile mixing both."""
    rng = np.random.default_rng(5)
    t = np.linspace(0, 2 * np.pi, 700, endpoint=False)
    curve = np.stack([0.5 + 0.05 * np.cos(t), 0.5 + 0.05 * np.sin(t)], 1)
    box = rng.uniform(0.0, 0.8, size=(600, 2))
    q = np.concatenate([curve, box])
    p = rng.normal(0, 0.05, size=q.shape)
    sigma = 0.02
    dq, dp = ep.rhs(cuda(q), cuda(p), prm(sigma))
    rq, rp = o.rhs(q, p, ep.GAUSS, sigma)
    assert rel(dq, rq) < 1e-5
    assert rel(dp, rp) < 1e-5


def test_rhs_multi_block_segments_sampled_rows():
    """N = 16384: every segment spans many shared-memory blocks of sources."""
    pr = w.fourier_curve_warp(n=16384)
    p = 0.01 * (pr.Y - pr.X)
    dq, dp = ep.rhs(cuda(pr.X), cuda(p), prm())
    rows = np.random.default_rng(2).choice(pr.n, 600, replace=False)
    rq, rp = o.rhs_rows(pr.X, p, rows, ep.GAUSS, 0.1)
    assert rel(dq.cpu().numpy()[rows], rq) < 1e-5
    assert rel(dp.cpu().numpy()[rows], rp) < 1e-5


@pytest.mark.parametrize("n", [65, 300, 2049])
def test_shoot_ragged_sizes(n):
    pr = w.fourier_curve_warp(n=n)
    p0 = 0.002 * (pr.Y - pr.X)
    q1, p1 = ep.shoot(cuda(pr.X), cuda(p0), prm(steps=6))
    rq, rp = o.shoot(pr.X, p0, ep.GAUSS, 0.1, 6)
    assert rel(q1, rq) < 1e-4 and rel(p1, rp) < 1e-4


def test_agrees_with_cuda_core_path():
    pr = w.fourier_curve_warp(n=4096)
    p0 = 0.002 * (pr.Y - pr.X)
    X, P = cuda(pr.X), cuda(p0)
    q_tc, p_tc = ep.shoot(X, P, prm(steps=10))
    dq_tc, dp_tc = ep.rhs(X, P, prm())
    with cuda_core_path():
        q_cc, p_cc = ep.shoot(X, P, prm(steps=10))
        dq_cc, dp_cc = ep.rhs(X, P, prm())
    rq, rp = o.shoot(pr.X, p0, ep.GAUSS, 0.1, 10)
    e_tc = np.abs(q_tc.cpu().numpy() - rq).max()
    e_cc = np.abs(q_cc.cpu().numpy() - rq).max()
    assert e_tc < 1e-6 and e_cc < 1e-6, (e_tc, e_cc)
    a = dq_cc.cpu().numpy()
    assert rel(dq_tc, a) < 1e-5 and rel(dp_tc, dp_cc.cpu().numpy()) < 1e-5


def test_deterministic():
    pr = w.fourier_curve_warp(n=3000)
    p0 = 0.002 * (pr.Y - pr.X)
    a = ep.shoot(cuda(pr.X), cuda(p0), prm(steps=3))[0]
    b = ep.shoot(cuda(pr.X), cuda(p0), prm(steps=3))[0]
    assert torch.equal(a, b)
