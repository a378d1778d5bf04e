"""ep_rhs_noalloc, the right-hand side for callers that may not allocate.

Some callers cannot let the library call cudaMalloc while they evaluate the
right-hand side (a real-time loop that must not synchronise the device, or a
framework whose own memory pool owns the GPU).  ep_rhs_noalloc takes its
scratch from a fixed array compiled into libep.so instead.  These tests call it
through the C ABI and check it against ep_rhs, the allocating entry point, on
two calls in a row (the second with a different size, so a stale accumulator
left in the shared array by the first call would show).  The file name makes
pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1510_03816_gb300 import ep  # noqa: E402

TOL = {ep.MIXED: 1e-5, ep.FP64: 1e-12}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1510_03816_gb300 import build

    build.build()
    return ep.load()


def _inputs(n, dim, seed):
    rng = np.random.default_rng(seed)
    q = torch.tensor(rng.uniform(0.2, 0.8, size=(n, dim)), device="cuda")
    p = torch.tensor(rng.normal(0.0, 0.05, size=(n, dim)), device="cuda")
    return q, p


def _noalloc(lib, q, p, prm):
    n, dim = q.shape
    dq = torch.empty_like(q)
    dp = torch.empty_like(q)
    P = ep._with_dim(prm, dim)
    st = lib.ep_rhs_noalloc(ctypes.byref(P), n, q.data_ptr(), p.data_ptr(), dq.data_ptr(), dp.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    assert st == ep.OK, ep.last_error()
    return dq, dp


def _rel(a, b):
    den = b.abs().max().item()
    return (a - b).abs().max().item() / (den if den > 0 else 1.0)


@pytest.mark.parametrize("prec", [ep.MIXED, ep.FP64])
@pytest.mark.parametrize("dim", [2, 3])
def test_noalloc_matches_rhs_on_consecutive_calls(lib, prec, dim):
    prm = ep.params(dim=dim, kernel=ep.GAUSS, sigma=0.1, precision=prec, neigh=ep.ALLPAIRS)
    for n, seed in ((1000, 1), (700, 2)):
        q, p = _inputs(n, dim, seed)
        dq, dp = _noalloc(lib, q, p, prm)
        rq, rp = ep.rhs(q, p, prm)
        torch.cuda.synchronize()
        assert _rel(dq, rq) < TOL[prec]
        assert _rel(dp, rp) < TOL[prec]


def test_noalloc_largest_size_and_limits(lib):
    prm = ep.params(dim=3, kernel=ep.TENT, sigma=0.2, precision=ep.FP64, neigh=ep.ALLPAIRS)
    n = 8192  # EP_NOALLOC_MAX_N, the size of the fixed scratch array
    q, p = _inputs(n, 3, 5)
    dq, dp = _noalloc(lib, q, p, prm)
    rq, rp = ep.rhs(q, p, prm)
    torch.cuda.synchronize()
    assert _rel(dq, rq) < TOL[ep.FP64] and _rel(dp, rp) < TOL[ep.FP64]
    # one particle more than the array holds is refused, not truncated
    q2, p2 = _inputs(n + 1, 3, 6)
    P = ep._with_dim(prm, 3)
    out = torch.empty_like(q2)
    st = lib.ep_rhs_noalloc(ctypes.byref(P), n + 1, q2.data_ptr(), p2.data_ptr(), out.data_ptr(),
                            out.data_ptr(), 0)
    assert st == ep.EINVAL and "8192" in ep.last_error()
    # host arrays would need staging memory: refused
    qh = np.zeros((4, 3))
    st = lib.ep_rhs_noalloc(ctypes.byref(P), 4, qh.ctypes.data, qh.ctypes.data, qh.ctypes.data, qh.ctypes.data, 0)
    assert st == ep.EINVAL
