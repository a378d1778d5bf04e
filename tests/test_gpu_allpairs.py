"""GPU parity of the all-pairs path (ep_rhs, ep_shoot, ep_match, ep_hamiltonian)
against the FP64 CPU oracle, through the C ABI.

Tolerances: mixed precision (FP32 pair terms, FP64 sums): RHS <= 1e-5 and
shot endpoints <= 1e-4 relative (max-norm of the difference over the max-norm
of the oracle's block); FP64 mode <= 1e-12.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as o  # noqa: E402
from paper_1510_03816_gb300 import ep, workloads as w  # noqa: E402

TOL = {ep.MIXED: {"rhs": 1e-5, "shoot": 1e-4}, ep.FP64: {"rhs": 1e-12, "shoot": 1e-12}}
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


def tent_boundary_rows(q, sigma, band=1e-5):
    """Particles with a pair distance within band*sigma of sigma: the tent's
    momentum weight jumps there, so FP32 and FP64 may legitimately disagree."""
    d = np.linalg.norm(q[:, None, :] - q[None, :, :], axis=-1)
    return np.any(np.abs(d - sigma) < band * sigma, axis=1)


def cloud(n, dim, seed):
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.2, 0.8, size=(n, dim))
    p = rng.normal(0, 0.05, size=(n, dim))
    return q, p


@pytest.mark.parametrize("prec", [ep.MIXED, ep.FP64])
@pytest.mark.parametrize("kernel,sigma", KSIG)
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("n", [1, 63, 1000])
def test_rhs_parity(prec, kernel, sigma, dim, n):
    q, p = cloud(n, dim, seed=n + 7 * dim + kernel)
    prm = ep.params(dim=dim, kernel=kernel, sigma=sigma, precision=prec, neigh=ep.ALLPAIRS)
    dq, dp = ep.rhs(cuda(q), cuda(p), prm)
    rq, rp = o.rhs(q, p, kernel, sigma)
    assert rel(dq, rq) < TOL[prec]["rhs"]
    if kernel == ep.TENT:
        keep = ~tent_boundary_rows(q, sigma)
        assert rel(dp.cpu().numpy()[keep], rp[keep]) < TOL[prec]["rhs"]
    else:
        assert rel(dp, rp) < TOL[prec]["rhs"]


@pytest.mark.parametrize("prec", [ep.MIXED, ep.FP64])
def test_rhs_full_size_fourier_curve(prec):
    """N = 4096 Gaussian sigma = 0.1 (the benchmark's launch configuration), every row."""
    pr = w.fourier_curve_warp()
    p = 0.01 * (pr.Y - pr.X)
    prm = ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, precision=prec, neigh=ep.ALLPAIRS)
    dq, dp = ep.rhs(cuda(pr.X), cuda(p), prm)
    rq, rp = o.rhs(pr.X, p, pr.kernel, pr.sigma)
    assert rel(dq, rq) < TOL[prec]["rhs"]
    assert rel(dp, rp) < TOL[prec]["rhs"]


@pytest.mark.parametrize("prec", [ep.MIXED, ep.FP64])
@pytest.mark.parametrize("kernel,sigma", KSIG)
@pytest.mark.parametrize("dim", [2, 3])
def test_shoot_parity(prec, kernel, sigma, dim):
    n = 300
    q, p = cloud(n, dim, seed=11 + dim + kernel)
    p *= 0.5
    prm = ep.params(dim=dim, kernel=kernel, sigma=sigma, steps=8, precision=prec, neigh=ep.ALLPAIRS)
    q1, p1 = ep.shoot(cuda(q), cuda(p), prm)
    rq, rp = o.shoot(q, p, kernel, sigma, 8)
    # the tent's momentum weight jumps at r = sigma; the mixed shoot still meets the
    # endpoint bound (measured <= 6e-7: a stage evaluation would have to land within
    # FP32 rounding of the kink for FP32 and FP64 to take different sides)
    tol = TOL[prec]["shoot"]
    assert rel(q1, rq) < tol
    assert rel(p1, rp) < tol


def test_shoot_full_size_fourier_curve_mixed():
    """N = 4096 in the benchmark's launch configuration (10 RK4 steps): endpoints within
    1e-4 relative and 1e-6 absolute of the oracle."""
    pr = w.fourier_curve_warp()
    p0 = 0.002 * (pr.Y - pr.X)
    prm = ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, steps=10, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    q1, p1 = ep.shoot(cuda(pr.X), cuda(p0), prm)
    rq, rp = o.shoot(pr.X, p0, pr.kernel, pr.sigma, 10)
    assert rel(q1, rq) < 1e-4 and rel(p1, rp) < 1e-4
    assert np.abs(q1.cpu().numpy() - rq).max() < 1e-6


def test_benchmark_match_per_iterate_parity():
    """The benchmarked call itself: ep_match of the N = 4096 Fourier-curve workload
    (Gaussian sigma = 0.1, 100 RK4 steps, mixed precision, all pairs, the default
    gain, p0 = 0), i.e. the persistent all-pairs shoot with the FP64 residual and
    momentum update of Algorithm 1, stopped after 2 updates.  The residual of each
    of the 3 shoots and the momenta after the last update agree with the oracle's
    Algorithm 1 element by element within the shot-endpoint bound 1e-4."""
    pr = w.fourier_curve_warp()
    maxit = 2
    prm = ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, steps=pr.steps, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    r = ep.match(cuda(pr.X), cuda(pr.Y), prm, h=0.0, eps=pr.eps, maxit=maxit)
    h_ref = o.default_gain(pr.X, pr.kernel, pr.sigma)
    assert abs(r.h - h_ref) < 1e-6 * h_ref
    p, st, it, res, hist = o.match(pr.X, pr.Y, pr.kernel, pr.sigma, pr.steps, h=h_ref, eps=pr.eps, maxit=maxit)
    assert r.status == st == ep.ENOTCONVERGED and r.iters == it == maxit
    assert len(r.hist) == len(hist) == maxit + 1
    np.testing.assert_allclose(r.hist, hist, rtol=1e-4)
    assert rel(r.p0, p) < 1e-4
    assert np.abs(r.p0.cpu().numpy() - p).max() < 1e-4 * np.abs(p).max()


def test_shoot_aliasing_and_host_pointers():
    q, p = cloud(100, 2, seed=3)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=5, precision=ep.FP64)
    q1h, p1h = ep.shoot(q, p, prm)  # numpy in, numpy out (host staging)
    rq, rp = o.shoot(q, p, ep.GAUSS, 0.1, 5)
    assert rel(q1h, rq) < 1e-12 and rel(p1h, rp) < 1e-12
    tq, tp = cuda(q), cuda(p)
    lib = ep.load()
    import ctypes
    prm2 = ep._with_dim(prm, 2)
    st = lib.ep_shoot(ctypes.byref(prm2), 100, tq.data_ptr(), tp.data_ptr(), tq.data_ptr(), tp.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
    assert st == ep.OK
    assert rel(tq, rq) < 1e-12 and rel(tp, rp) < 1e-12


@pytest.mark.parametrize("prec", [ep.FP64, ep.MIXED])
def test_match_per_iterate_parity_circle_to_ellipse(prec):
    """Algorithm 1 on the N = 64 circle -> ellipse (tent sigma = 0.25): the residual
    history and the momenta after 25 updates agree with the oracle."""
    pr = w.circle_to_ellipse(64)
    steps, h, maxit = 20, 0.1, 25
    prm = ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, steps=steps, precision=prec, neigh=ep.ALLPAIRS)
    r = ep.match(cuda(pr.X), cuda(pr.Y), prm, h=h, eps=1e-6, maxit=maxit)
    p, st, it, res, hist = o.match(pr.X, pr.Y, pr.kernel, pr.sigma, steps, h=h, eps=1e-6, maxit=maxit)
    assert r.status == st and r.iters == it
    tol = 1e-12 if prec == ep.FP64 else 1e-4
    assert rel(r.p0, p) < tol
    np.testing.assert_allclose(r.hist, hist, rtol=tol)
    assert abs(r.H - o.hamiltonian(pr.X, p, pr.kernel, pr.sigma)) < 10 * tol * abs(r.H)


def test_match_default_gain_and_convergence():
    pr = w.circle_to_ellipse(32)
    X, Y = pr.X, pr.Y
    prm = ep.params(dim=2, kernel=ep.EXPCONE, sigma=0.1, steps=10, precision=ep.FP64)
    r = ep.match(cuda(X), cuda(Y), prm, h=0.0, eps=1e-9, maxit=2000)
    h_ref = o.default_gain(X, ep.EXPCONE, 0.1)
    assert abs(r.h - h_ref) < 1e-13 * h_ref
    p, st, it, res, hist = o.match(X, Y, ep.EXPCONE, 0.1, 10, h=0.0, eps=1e-9, maxit=2000)
    assert st == ep.OK and r.status == ep.OK and r.iters == it
    assert rel(r.p0, p) < 1e-10


def test_match_reports_divergence_and_cap():
    pr = w.circle_to_ellipse(32)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=10, precision=ep.FP64)
    r = ep.match(cuda(pr.X), cuda(pr.Y), prm, h=50.0, eps=1e-6, maxit=200)
    p, st, it, res, hist = o.match(pr.X, pr.Y, ep.GAUSS, 0.1, 10, h=50.0, eps=1e-6, maxit=200)
    assert r.status == st and r.iters == it
    r = ep.match(cuda(pr.X), cuda(pr.Y), prm, h=0.05, eps=0.0, maxit=3)
    assert r.status == ep.ENOTCONVERGED and r.iters == 3 and len(r.hist) == 4


@pytest.mark.parametrize("prec", [ep.FP64, ep.MIXED])
def test_hamiltonian(prec):
    q, p = cloud(500, 3, seed=5)
    prm = ep.params(dim=3, kernel=ep.GAUSS, sigma=0.2, precision=prec)
    H = ep.hamiltonian(cuda(q), cuda(p), prm)
    Hr = o.hamiltonian(q, p, ep.GAUSS, 0.2)
    assert abs(H - Hr) < (1e-12 if prec == ep.FP64 else 1e-5) * abs(Hr)


def test_empty_and_invalid_inputs():
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1)
    dq, dp = ep.rhs(cuda(np.zeros((0, 2))), cuda(np.zeros((0, 2))), prm)
    assert dq.shape == (0, 2)
    with pytest.raises(ep.EPError) as e:
        ep.rhs(cuda(np.zeros((4, 2))), cuda(np.zeros((4, 2))), ep.params(dim=2, kernel=ep.GAUSS, sigma=-1.0))
    assert e.value.status == ep.EINVAL
    with pytest.raises(ep.EPError):
        ep.shoot(cuda(np.zeros((4, 2))), cuda(np.zeros((4, 2))), ep.params(dim=2, steps=0))
    with pytest.raises(ep.EPError):
        ep.rhs(cuda(np.zeros((4, 2))), cuda(np.zeros((4, 2))), ep.params(dim=2, kernel=ep.GAUSS, neigh=ep.CELLLIST))


@pytest.mark.parametrize("n", [3700, 4096, 1000, 301])
def test_owner_kernel_default_forms_parity(n, monkeypatch):
    """The persistent 2-D Gaussian shoot in its default configuration (EP_AUTOTUNE=0):
    the 512-thread form with 8 rows per lane for n >= 24 rows per SM (3700: ragged rows
    per CTA), the 1024-thread form with 8-row sub-tiles below; endpoints against the
    oracle within 1e-4, and the form the launch used is the owner kernel."""
    monkeypatch.setenv("EP_AUTOTUNE", "0")
    pr = w.fourier_curve_warp(n=n)
    p0 = 0.004 * (pr.Y - pr.X)
    prm = ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, steps=6, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    ep.set_launch_timing(True)
    try:
        q1, p1 = ep.shoot(cuda(pr.X), cuda(p0), prm)
        _, kname = ep.last_launch()
    finally:
        ep.set_launch_timing(False)
    assert kname.startswith("k_shoot_owner<512,8>" if n >= 3648 else "k_shoot_owner<1024,16>"), kname
    rq, rp = o.shoot(pr.X, p0, pr.kernel, pr.sigma, 6)
    assert rel(q1, rq) < 1e-4 and rel(p1, rp) < 1e-4


def _device_loop_case(name):
    if name == "benchmark_cap":
        pr = w.fourier_curve_warp()
        return pr.X, pr.Y, ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, steps=pr.steps, precision=ep.MIXED,
                                     neigh=ep.ALLPAIRS), dict(h=0.0, eps=pr.eps, maxit=3)
    if name == "ragged_converges":
        pr = w.circle_to_ellipse(n=3700, kernel=ep.GAUSS, sigma=0.1, steps=20)
        return pr.X, pr.Y, ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=20, precision=ep.MIXED,
                                     neigh=ep.ALLPAIRS), dict(h=0.0, eps=2e-2, maxit=60)
    if name == "1024_thread_form":
        pr = w.circle_to_ellipse(n=1000, kernel=ep.GAUSS, sigma=0.1, steps=20)
        return pr.X, pr.Y, ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=20, precision=ep.MIXED,
                                     neigh=ep.ALLPAIRS), dict(h=0.0, eps=1e-6, maxit=4)
    if name == "inexact_stop":
        pr = w.circle_to_ellipse(n=1000, kernel=ep.GAUSS, sigma=0.1, steps=20)
        return pr.X, pr.Y, ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=20, precision=ep.MIXED,
                                     neigh=ep.ALLPAIRS, inexact=0.05), dict(h=0.0, eps=2e-3, maxit=200)
    pr = w.circle_to_ellipse(n=500, kernel=ep.GAUSS, sigma=0.1, steps=10)  # diverges
    return pr.X, pr.Y, ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=10, precision=ep.MIXED,
                                 neigh=ep.ALLPAIRS), dict(h=60.0, eps=1e-6, maxit=40)


@pytest.mark.parametrize("case", ["benchmark_cap", "ragged_converges", "1024_thread_form", "inexact_stop",
                                  "diverges"])
def test_device_matching_loop_equals_host_loop(case, monkeypatch):
    """Algorithm 1 as one CUDA graph (a while-loop node over the load, the owner-computes
    shoot and k_match_step: FP64 residual, stop tests and momentum update on the device)
    against the host loop of ep_match over the same shoot kernel (EP_DEVICE_MATCH=0):
    the same momenta, residual history, update count and status, bit for bit, in the
    default launch configurations (EP_AUTOTUNE=0)."""
    monkeypatch.setenv("EP_AUTOTUNE", "0")
    X, Y, prm, kw = _device_loop_case(case)
    ep.set_launch_timing(True)
    try:
        rd = ep.match(cuda(X), cuda(Y), prm, **kw)
        _, kname = ep.last_launch()
    finally:
        ep.set_launch_timing(False)
    assert kname.startswith("matching graph: k_shoot_owner<"), kname
    monkeypatch.setenv("EP_DEVICE_MATCH", "0")
    rh = ep.match(cuda(X), cuda(Y), prm, **kw)
    assert (rd.status, rd.iters) == (rh.status, rh.iters)
    assert rd.h == rh.h
    assert rd.H == rh.H or (np.isnan(rd.H) and np.isnan(rh.H))
    assert np.array_equal(rd.p0.cpu().numpy(), rh.p0.cpu().numpy())
    assert np.array_equal(np.asarray(rd.hist), np.asarray(rh.hist), equal_nan=True)
    expect = {"benchmark_cap": ep.ENOTCONVERGED, "ragged_converges": ep.OK, "1024_thread_form": ep.ENOTCONVERGED,
              "inexact_stop": ep.OK, "diverges": ep.EDIVERGED}[case]
    assert rd.status == expect, (case, rd.status, rd.iters, rd.hist[-3:])


@pytest.mark.parametrize("kernel,sigma,dim", [(ep.TENT, 0.1, 2), (ep.EXPCONE, 0.05, 2), (ep.GAUSS, 0.15, 3),
                                              (ep.TENT, 0.2, 3)])
def test_rhs_parity_packed_generic_multi_chunk(kernel, sigma, dim):
    """The packed 512-thread pair stage of the tent, the exp-cone and 3-D (sources staged
    in pairs, an odd count padded with a far, momentum-free source) over several staged
    chunks with an odd tail: n = 4099, every row against the oracle within the RHS bound."""
    n = 4099
    q, p = cloud(n, dim, seed=11 + kernel + 3 * dim)
    prm = ep.params(dim=dim, kernel=kernel, sigma=sigma, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    dq, dp = ep.rhs(cuda(q), cuda(p), prm)
    rq, rp = o.rhs(q, p, kernel, sigma)
    assert rel(dq, rq) < TOL[ep.MIXED]["rhs"]
    keep = ~tent_boundary_rows(q, sigma) if kernel == ep.TENT else np.ones(n, bool)
    assert rel(dp.cpu().numpy()[keep], rp[keep]) < TOL[ep.MIXED]["rhs"]


@pytest.mark.parametrize("variant", ["maxit0", "no_hist", "host_arrays"])
def test_device_matching_loop_edge_calls(variant, monkeypatch):
    """The matching graph at its edges: a single shoot (maxit = 0), no residual history
    requested, and host (numpy) arrays staged through the C ABI; momenta, status and
    update count equal the host loop's bit for bit."""
    monkeypatch.setenv("EP_AUTOTUNE", "0")
    pr = w.circle_to_ellipse(n=1000, kernel=ep.GAUSS, sigma=0.1, steps=10)
    prm = ep.params(dim=2, kernel=ep.GAUSS, sigma=0.1, steps=10, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    kw = dict(h=0.0, eps=1e-6, maxit=0 if variant == "maxit0" else 3, hist=variant != "no_hist")

    def run():
        if variant == "host_arrays":
            r = ep.match(np.asarray(pr.X), np.asarray(pr.Y), prm, **kw)
            return r, np.asarray(r.p0)
        r = ep.match(cuda(pr.X), cuda(pr.Y), prm, **kw)
        return r, r.p0.cpu().numpy()

    ep.set_launch_timing(True)
    try:
        rd, pd = run()
        _, kname = ep.last_launch()
    finally:
        ep.set_launch_timing(False)
    assert kname.startswith("matching graph: k_shoot_owner<"), kname
    monkeypatch.setenv("EP_DEVICE_MATCH", "0")
    rh, ph = run()
    assert (rd.status, rd.iters, rd.resid) == (rh.status, rh.iters, rh.resid)
    assert rd.status == ep.ENOTCONVERGED and rd.iters == kw["maxit"]
    assert np.array_equal(pd, ph)
    if kw["hist"]:
        assert np.array_equal(np.asarray(rd.hist), np.asarray(rh.hist)) and len(rd.hist) == kw["maxit"] + 1
    else:
        assert rd.hist is None and rh.hist is None
