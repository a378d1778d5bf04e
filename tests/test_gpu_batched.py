"""ep_match_batched: many independent matchings of uneven size in one persistent
launch, checked per problem against the FP64 oracle (and the single-problem
GPU path) through the C ABI.  Mixed precision: momenta <= 1e-4 relative for
both kernels."""
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


def problems(sizes, steps):
    out = []
    for b, n in enumerate(sizes):
        if b % 2 == 0:
            pr = w.circle_to_ellipse(int(n), stream=2000 + b, sigma=0.2, kernel=ep.TENT, steps=steps)
        else:
            pr = w.circle_to_ellipse(int(n), stream=2000 + b, sigma=0.1, kernel=ep.GAUSS, steps=steps)
        out.append(pr)
    return out


def run_batched(prs, h, eps, maxit, cuda=True):
    Xs = [torch.tensor(p.X, device="cuda") if cuda else p.X for p in prs]
    Ys = [torch.tensor(p.Y, device="cuda") if cuda else p.Y for p in prs]
    prms = [ep.params(dim=2, kernel=p.kernel, sigma=p.sigma, steps=p.steps, precision=ep.MIXED, neigh=ep.ALLPAIRS)
            for p in prs]
    return ep.match_batched(Xs, Ys, prms, h=h, eps=eps, maxit=maxit)


def test_batched_per_problem_parity_with_oracle():
    """Solo problems (n < 2048, one CTA each) and team problems (n >= 2048, a whole
    cluster of CTAs with distributed shared memory) against the oracle."""
    sizes = [32, 33, 97, 256, 500, 1023, 1500, 2047, 2048, 2600]
    prs = problems(sizes, steps=4)
    res = run_batched(prs, 0.0, eps=1e-12, maxit=3)  # default gain per problem
    for pr, r in zip(prs, res):
        assert abs(r.h - o.default_gain(pr.X, pr.kernel, pr.sigma)) < 1e-6 * r.h
        p, st, it, resid, hist = o.match(pr.X, pr.Y, pr.kernel, pr.sigma, pr.steps, h=r.h, eps=1e-12, maxit=3)
        assert r.iters == it == 3
        tol = 1e-4  # both kernels (tent measured <= 3e-7)
        assert rel(r.p0, p) < tol, (pr.n, pr.kernel, rel(r.p0, p))
        assert abs(r.resid - resid) < tol * resid
        assert abs(r.H - o.hamiltonian(pr.X, p, pr.kernel, pr.sigma)) < 10 * tol * abs(r.H)


def test_batched_default_gain_convergence_and_host_arrays():
    sizes = [40, 64, 64, 300]
    prs = problems(sizes, steps=5)
    res = run_batched(prs, 0.0, eps=5e-3, maxit=60, cuda=False)
    for pr, r in zip(prs, res):
        assert abs(r.h - o.default_gain(pr.X, pr.kernel, pr.sigma)) < 1e-6 * r.h
        p, st, it, resid, hist = o.match(pr.X, pr.Y, pr.kernel, pr.sigma, pr.steps, h=r.h, eps=5e-3, maxit=60)
        assert r.status == st and r.iters == it
        assert rel(r.p0, p) < 1e-4


def test_batched_matches_single_problem_path():
    prs = problems([700, 2100], steps=6)
    res = run_batched(prs, 0.002, eps=1e-12, maxit=2)
    for pr, r in zip(prs, res):
        prm = ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, steps=pr.steps, precision=ep.MIXED,
                        neigh=ep.ALLPAIRS)
        s = ep.match(torch.tensor(pr.X, device="cuda"), torch.tensor(pr.Y, device="cuda"), prm, h=0.002, eps=1e-12,
                     maxit=2)
        assert s.iters == r.iters
        assert rel(r.p0, s.p0.cpu().numpy()) < 1e-4


def test_batched_full_workload_sampled():
    """The 512-problem workload (n log-uniform in [32, 8192]) with 2 feedback updates;
    a sample of problems checked against the oracle."""
    prs = w.batched_curves()
    res = run_batched(prs, 0.0, eps=1e-12, maxit=2)
    assert len(res) == 512 and all(r.iters == 2 for r in res)
    sizes = np.array([p.n for p in prs])
    under = np.where(sizes < 3000)[0]
    picks = [int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]), int(under[np.argmax(sizes[under])])]
    for b in picks:
        pr = prs[b]
        p, st, it, resid, hist = o.match(pr.X, pr.Y, pr.kernel, pr.sigma, pr.steps, h=res[b].h, eps=1e-12,
                                         maxit=2)
        tol = 1e-4  # both kernels (tent measured <= 3e-7)
        assert rel(res[b].p0, p) < tol


def test_batched_invalid_sizes():
    X = [np.zeros((9000, 2))]
    with pytest.raises(ep.EPError):
        ep.match_batched(X, X, [ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=2)], maxit=1)
    assert ep.match_batched([], [], []) == []


def test_batched_per_problem_status_through_the_c_abi():
    """ep_match_batched reports each problem's own status in infos[b].status (Algorithm 1
    steps 2-3, decided on the device): one problem converges, one stops at the cap, one
    diverges under too large a gain; the oracle agrees on each."""
    import ctypes

    prs = problems([48, 64, 80], steps=5)
    hs = [0.0, 0.002, 60.0]  # default gain; a gain too small to converge in maxit; divergence
    eps, maxit = 2e-2, 40
    offs = np.zeros(len(prs) + 1, dtype=np.int64)
    for b, pr in enumerate(prs):
        offs[b + 1] = offs[b] + pr.n
    X = torch.tensor(np.concatenate([p.X for p in prs]), device="cuda")
    Y = torch.tensor(np.concatenate([p.Y for p in prs]), device="cuda")
    p0 = torch.zeros_like(X)
    P = (ep.Params * 3)(*[ep.params(dim=2, kernel=p.kernel, sigma=p.sigma, steps=p.steps, precision=ep.MIXED,
                                     neigh=ep.ALLPAIRS) for p in prs])
    infos = (ep.MatchInfo * 3)(*[ep.MatchInfo(hs[b], eps, maxit, 0, 0.0, 0.0, None) for b in range(3)])
    for b in range(3):
        infos[b].status = -1
    lib = ep.load()
    st = lib.ep_match_batched(P, 3, offs.ctypes.data, X.data_ptr(), Y.data_ptr(), p0.data_ptr(), infos,
                              torch.cuda.current_stream().cuda_stream)
    statuses = [infos[b].status for b in range(3)]
    ref = []
    for b, pr in enumerate(prs):
        h = infos[b].h
        _, s_ref, it, _, _ = o.match(pr.X, pr.Y, pr.kernel, pr.sigma, pr.steps, h=h, eps=eps, maxit=maxit)
        ref.append(s_ref)
        if s_ref != ep.EDIVERGED:
            assert infos[b].iters == it
    assert statuses == ref == [ep.OK, ep.ENOTCONVERGED, ep.EDIVERGED]
    assert st == ep.ENOTCONVERGED  # the first non-OK status in problem order
    res = ep.match_batched([torch.tensor(p.X, device="cuda") for p in prs],
                           [torch.tensor(p.Y, device="cuda") for p in prs],
                           [ep.params(dim=2, kernel=p.kernel, sigma=p.sigma, steps=p.steps, precision=ep.MIXED)
                            for p in prs], h=hs, eps=eps, maxit=maxit)
    assert [r.status for r in res] == statuses


def test_batched_autotuned_shape_matches_the_default_shape():
    """The launch shape (cluster size, team threshold, lanes per particle) is chosen by the
    library's autotuner; whatever it picks, the matchings agree with the default shape's
    (EP_AUTOTUNE=0) to FP32 summation-order level, and the shape is reported."""
    import os

    prs = problems([40, 300, 1100, 2100, 2500, 5000], steps=3)
    old = os.environ.get("EP_AUTOTUNE")
    try:
        os.environ["EP_AUTOTUNE"] = "0"
        ref = run_batched(prs, 0.0, eps=1e-12, maxit=2)
        os.environ["EP_AUTOTUNE"] = "1"
        run_batched(prs, 0.0, eps=1e-12, maxit=0)  # tunes
        ep.set_launch_timing(True)
        res = run_batched(prs, 0.0, eps=1e-12, maxit=2)
        ms, shape = ep.last_launch()
    finally:
        ep.set_launch_timing(False)
        if old is None:
            os.environ.pop("EP_AUTOTUNE", None)
        else:
            os.environ["EP_AUTOTUNE"] = old
    assert shape.startswith("k_batched (cluster ") and ms > 0
    for r, s in zip(res, ref):
        assert r.iters == s.iters == 2
        assert rel(r.p0, s.p0.cpu().numpy()) < 1e-5
