"""GPU cell list (tent kernel, 2-D): neighbour sets bit-exact against the oracle's
brute force of the same predicate, and RHS / shoot / match parity with the FP64
oracle (mixed precision: RHS <= 1e-5 away from the tent's jump at r = sigma,
endpoints <= 1e-4), through the C ABI.  At the full 512 x 512 jittered-grid size
the oracle checks a sample of rows."""
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


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def grid_problem(side, seed_stream=3):
    pr = w.jittered_grid(side=side, stream=seed_stream)
    p = 0.01 * (pr.Y - pr.X)
    return pr, p


def boundary_rows(q, sigma, rows=None, band=1e-4):
    """Particles with a neighbour within band*sigma of distance sigma (the tent's dp
    weight jumps there, so FP32 and FP64 may legitimately disagree)."""
    idx = np.arange(q.shape[0]) if rows is None else rows
    out = np.zeros(idx.size, dtype=bool)
    for k, i in enumerate(idx):
        d = np.linalg.norm(q - q[i], axis=1)
        out[k] = np.any(np.abs(d - sigma) < band * sigma)
    return out


@pytest.mark.parametrize("side,seed", [(24, 1), (64, 2)])
def test_neighbor_sets_bit_exact(side, seed):
    pr, _ = grid_problem(side, seed)
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=pr.sigma, precision=ep.MIXED, neigh=ep.CELLLIST)
    cnt, hsh, tot = ep.cell_neighbors(cuda(pr.X), prm)
    rc, rh, rt = o.cell_neighbors(pr.X, pr.sigma)
    np.testing.assert_array_equal(cnt.cpu().numpy(), rc)
    np.testing.assert_array_equal(hsh.cpu().numpy().view(np.uint64), rh)
    assert tot == rt


def test_neighbor_sets_random_cloud_and_clamped_outliers():
    rng = np.random.default_rng(4)
    q = rng.uniform(0, 1, size=(3000, 2))
    q[:5] += 3.0  # far outliers stretch the grid: many empty cells
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=0.03, neigh=ep.CELLLIST)
    cnt, hsh, tot = ep.cell_neighbors(q, prm)  # host arrays
    rc, rh, rt = o.cell_neighbors(q, 0.03)
    np.testing.assert_array_equal(cnt, rc)
    np.testing.assert_array_equal(hsh, rh)


def test_neighbor_sets_full_size_sampled_rows():
    pr = w.jittered_grid()
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=pr.sigma, neigh=ep.CELLLIST)
    cnt, hsh, tot = ep.cell_neighbors(cuda(pr.X), prm)
    rows = np.random.default_rng(0).choice(pr.n, 2000, replace=False)
    rc, rh = o.cell_neighbors_rows(pr.X, rows, pr.sigma)
    np.testing.assert_array_equal(cnt.cpu().numpy()[rows], rc)
    np.testing.assert_array_equal(hsh.cpu().numpy().view(np.uint64)[rows], rh)
    assert 25 < tot / pr.n < 40  # about 32 neighbours + self per particle


def test_rhs_parity_and_against_all_pairs():
    pr, p = grid_problem(64)
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=pr.sigma, precision=ep.MIXED, neigh=ep.CELLLIST)
    dq, dp = ep.rhs(cuda(pr.X), cuda(p), prm)
    rq, rp = o.rhs(pr.X, p, ep.TENT, pr.sigma)
    keep = ~boundary_rows(pr.X, pr.sigma)
    assert rel(dq, rq) < 1e-5
    assert rel(dp.cpu().numpy()[keep], rp[keep]) < 1e-5
    prm_ap = ep.params(dim=2, kernel=ep.TENT, sigma=pr.sigma, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    aq, apv = ep.rhs(cuda(pr.X), cuda(p), prm_ap)
    assert rel(dq, aq.cpu().numpy()) < 1e-5


def test_rhs_full_size_sampled_rows():
    pr = w.jittered_grid()
    p = 0.01 * (pr.Y - pr.X)
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=pr.sigma, neigh=ep.CELLLIST)
    dq, dp = ep.rhs(cuda(pr.X), cuda(p), prm)
    rows = np.random.default_rng(1).choice(pr.n, 1500, replace=False)
    rq, rp = o.rhs_rows(pr.X, p, rows, ep.TENT, pr.sigma)
    keep = ~boundary_rows(pr.X, pr.sigma, rows)
    assert rel(dq.cpu().numpy()[rows], rq) < 1e-5
    assert rel(dp.cpu().numpy()[rows][keep], rp[keep]) < 1e-5


def test_shoot_and_match_parity():
    pr, p = grid_problem(40)
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=pr.sigma, steps=6, precision=ep.MIXED, neigh=ep.CELLLIST)
    q1, p1 = ep.shoot(cuda(pr.X), cuda(p), prm)
    rq, rp = o.shoot(pr.X, p, ep.TENT, pr.sigma, 6)
    assert rel(q1, rq) < 1e-4 and rel(p1, rp) < 1e-4
    assert np.abs(q1.cpu().numpy() - rq).max() < 1e-6
    r = ep.match(cuda(pr.X), cuda(pr.Y), prm, h=0.02, eps=1e-9, maxit=4)
    pm, st, it, res, hist = o.match(pr.X, pr.Y, ep.TENT, pr.sigma, 6, h=0.02, eps=1e-9, maxit=4)
    assert r.iters == it
    assert rel(r.p0, pm) < 1e-4
    np.testing.assert_allclose(r.hist, hist, rtol=1e-4)


def test_cell_list_is_deterministic():
    pr, p = grid_problem(48)
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=pr.sigma, steps=3, neigh=ep.CELLLIST)
    a = ep.shoot(cuda(pr.X), cuda(p), prm)[0]
    b = ep.shoot(cuda(pr.X), cuda(p), prm)[0]
    assert torch.equal(a, b)


def test_shoot_with_large_motion():
    # momenta large enough to carry particles more than a cell edge: particles change
    # cells many times along the shoot (and some leave the starting grid's interior)
    pr, p = grid_problem(40)
    p = 80.0 * p
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=pr.sigma, steps=20, precision=ep.MIXED, neigh=ep.CELLLIST)
    q1, p1 = ep.shoot(cuda(pr.X), cuda(p), prm)
    rq, rp = o.shoot(pr.X, p, ep.TENT, pr.sigma, 20)
    assert np.abs(rq - pr.X).max() > 1.2 * pr.sigma
    assert rel(q1, rq) < 1e-4 and rel(p1, rp) < 1e-4


def test_dense_cluster_beyond_the_staging_capacity():
    # 2500 particles within 0.6 sigma of each other, in a few cells: more records than
    # a sweep block stages in shared memory, so the sweep reads them from global memory
    rng = np.random.default_rng(5)
    sigma = 0.05
    ang, rad = rng.uniform(0, 2 * np.pi, 2500), 0.3 * sigma * np.sqrt(rng.uniform(0, 1, 2500))
    X = 0.5 + np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    p = rng.normal(0, 1e-4, size=X.shape)
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=sigma, steps=4, precision=ep.MIXED, neigh=ep.CELLLIST)
    q1, p1 = ep.shoot(cuda(X), cuda(p), prm)
    rq, rp = o.shoot(X, p, ep.TENT, sigma, 4)
    assert rel(q1, rq) < 1e-4 and rel(p1, rp) < 1e-4


def _converging_ring():
    """A 40 x 40 jittered grid (tent sigma = 0.05, about 11 particles per cell, so the
    cell grid's slots fit) with a ring of 60 particles moving in on its centre: the ring
    piles more than 32 particles into one cell after the first step and spreads out again
    later, so a shoot switches from the slot layout to the scanned one and back."""
    sig = 0.05
    g = np.linspace(0.2, 0.8, 40)
    rng = np.random.default_rng(7)
    B = np.stack(np.meshgrid(g, g), -1).reshape(-1, 2) + rng.uniform(-0.003, 0.003, (1600, 2))
    th = np.linspace(0, 2 * np.pi, 60, endpoint=False)
    ring = 0.5 + 0.12 * np.stack([np.cos(th), np.sin(th)], 1)
    X = np.vstack([B, ring])
    p = np.zeros_like(X)
    p[1600:] = -(ring - 0.5)
    return X, p, sig


def test_slot_and_scanned_layouts_agree_through_overflow():
    import os

    X, p, sig = _converging_ring()
    # the oracle's trajectory: some cell of the sweep grid (edge sigma (1 + 2^-8), origin
    # min - 2 h) holds more than 32 particles mid-shoot but not at the first step
    h = sig * 1.00390625
    lo = X.min(0) - 2 * h
    q, pp, most = X.copy(), p.copy(), []
    for _ in range(20):
        q, pp = o.shoot(q, pp, ep.TENT, sig, 1, 0.05)
        c = np.floor((q - lo) / h).astype(int)
        most.append(np.unique(c[:, 1] * 4096 + c[:, 0], return_counts=True)[1].max())
    assert most[0] <= 32 and max(most) > 40
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=sig, steps=20, precision=ep.MIXED, neigh=ep.CELLLIST)
    q1, p1 = ep.shoot(cuda(X), cuda(p), prm)
    old = os.environ.get("EP_CELL_SLOTS")
    try:
        os.environ["EP_CELL_SLOTS"] = "0"
        q2, p2 = ep.shoot(cuda(X), cuda(p), prm)
    finally:
        if old is None:
            os.environ.pop("EP_CELL_SLOTS", None)
        else:
            os.environ["EP_CELL_SLOTS"] = old
    assert torch.equal(q1, q2) and torch.equal(p1, p2)  # both layouts sum cells in particle-index order
    rq, rp = o.shoot(X, p, ep.TENT, sig, 20)
    assert rel(q1, rq) < 1e-4 and rel(p1, rp) < 1e-4
