"""Python binding of libep.so (include/ep.h): argument marshalling only.

Every function has the name of the C entry point it calls (without the ``ep_``
prefix).  Arrays are torch tensors (CUDA or CPU) or numpy arrays of float64
with shape (n, dim); outputs are allocated like the first input (same device /
library).  CUDA tensors are passed by device pointer on torch's current
stream; CPU tensors and numpy arrays are passed as host pointers and staged by
the library.  Nothing here computes any part of the method: if libep.so is
missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

try:  # torch is only plumbing (device memory, streams)
    import torch
except Exception:  # pragma: no cover
    torch = None

GAUSS, TENT, EXPCONE = 0, 1, 2
FP64, MIXED = 0, 1
AUTO, ALLPAIRS, CELLLIST = 0, 1, 2
OK, EINVAL, ENOMEM, ECUDA, ENOTCONVERGED, EDIVERGED, ETIMEOUT = range(7)
STATUS_NAMES = {0: "EP_OK", 1: "EP_EINVAL", 2: "EP_ENOMEM", 3: "EP_ECUDA", 4: "EP_ENOTCONVERGED",
                5: "EP_EDIVERGED", 6: "EP_ETIMEOUT"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libep.so")

# Every symbol include/ep.h declares (checked by the ABI test).
EXPORTS = ("ep_rhs", "ep_shoot", "ep_match", "ep_adjoint", "ep_match_batched", "ep_hamiltonian",
           "ep_hvp", "ep_cell_neighbors", "ep_release_workspace", "ep_last_error", "ep_version",
           "ep_launch_count", "ep_rhs_noalloc", "ep_set_launch_timing", "ep_last_launch_ms",
           "ep_last_launch_kernel", "ep_velocity", "ep_flow", "ep_shoot_tangent")


class EPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("kernel", ctypes.c_int), ("sigma", ctypes.c_double),
                ("steps", ctypes.c_int), ("t1", ctypes.c_double), ("precision", ctypes.c_int),
                ("neigh", ctypes.c_int), ("inexact", ctypes.c_double)]


class MatchInfo(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("eps", ctypes.c_double), ("maxit", ctypes.c_int),
                ("iters", ctypes.c_int), ("resid_inf", ctypes.c_double), ("H", ctypes.c_double),
                ("hist", ctypes.c_void_p), ("rule", ctypes.c_int), ("krylov", ctypes.c_int),
                ("products", ctypes.c_int), ("status", ctypes.c_int)]


# ep_rule: the update of Algorithm 1 step 3 (p0 += h r, h G(X)^-1 r, h (D phi)^-1 r)
RULE_MOMENTUM, RULE_VELOCITY, RULE_NEWTON = 0, 1, 2


@dataclass
class MatchResult:
    p0: object
    status: int
    iters: int
    resid: float
    H: float
    h: float
    hist: object | None
    products: int = 0


_lib = None


def load():
    """Load libep.so; raise if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libep.so not found at {LIB_PATH}; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER(Params)
    I64, VP, D = ctypes.c_int64, ctypes.c_void_p, ctypes.c_double
    sig = {
        "ep_rhs": [P, I64, VP, VP, VP, VP, VP],
        "ep_rhs_noalloc": [P, I64, VP, VP, VP, VP, VP],
        "ep_shoot": [P, I64, VP, VP, VP, VP, VP],
        "ep_match": [P, I64, VP, VP, VP, ctypes.POINTER(MatchInfo), VP],
        "ep_adjoint": [P, I64, VP, VP, VP, D, ctypes.c_int, VP, VP, VP],
        "ep_match_batched": [P, ctypes.c_int, VP, VP, VP, VP, ctypes.POINTER(MatchInfo), VP],
        "ep_hamiltonian": [P, I64, VP, VP, VP, VP],
        "ep_hvp": [P, I64, VP, VP, VP, VP, VP, VP, VP],
        "ep_shoot_tangent": [P, I64, VP, VP, VP, VP, VP, VP, VP, VP, VP],
        "ep_cell_neighbors": [P, I64, VP, VP, VP, VP, VP],
        "ep_release_workspace": [],
        "ep_velocity": [P, I64, VP, VP, I64, VP, VP, VP],
        "ep_flow": [P, I64, VP, VP, I64, VP, VP, VP],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.ep_last_error.restype = ctypes.c_char_p
    lib.ep_last_error.argtypes = []
    lib.ep_version.restype = ctypes.c_int
    lib.ep_version.argtypes = []
    lib.ep_launch_count.restype = ctypes.c_int64
    lib.ep_launch_count.argtypes = []
    lib.ep_set_launch_timing.restype = None
    lib.ep_set_launch_timing.argtypes = [ctypes.c_int]
    lib.ep_last_launch_ms.restype = ctypes.c_double
    lib.ep_last_launch_ms.argtypes = []
    lib.ep_last_launch_kernel.restype = ctypes.c_char_p
    lib.ep_last_launch_kernel.argtypes = []
    _lib = lib
    return lib


def last_error() -> str:
    return load().ep_last_error().decode()


def version() -> int:
    return int(load().ep_version())


def launch_count() -> int:
    """Kernels libep.so has launched in this process (ep_launch_count)."""
    return int(load().ep_launch_count())


def set_launch_timing(on: bool) -> None:
    """Record CUDA events around each persistent shoot launch (ep_set_launch_timing)."""
    load().ep_set_launch_timing(1 if on else 0)


def last_launch() -> tuple[float, str]:
    """(duration in ms, kernel name) of the last timed persistent shoot launch."""
    lib = load()
    return float(lib.ep_last_launch_ms()), lib.ep_last_launch_kernel().decode()


def release_workspace() -> None:
    _check(load().ep_release_workspace())


def _check(status: int, allowed=(OK,)) -> int:
    if status not in allowed:
        raise EPError(status, last_error())
    return status


def params(dim: int = 2, kernel: int = GAUSS, sigma: float = 0.1, steps: int = 100, t1: float = 1.0,
           precision: int = MIXED, neigh: int = AUTO, inexact: float = 0.0) -> Params:
    """ep_params; inexact = sigma_n^2 of the inexact particle system (0: exact)."""
    return Params(int(dim), int(kernel), float(sigma), int(steps), float(t1), int(precision), int(neigh),
                  float(inexact))


# ------------------------------------------------------------------ array marshalling
def _is_torch(a) -> bool:
    return torch is not None and isinstance(a, torch.Tensor)


def _prep(a, name: str):
    """Return (array, pointer) for a float64 C-contiguous input."""
    if _is_torch(a):
        if a.dtype != torch.float64:
            raise TypeError(f"{name}: expected float64, got {a.dtype}")
        a = a.contiguous()
        return a, a.data_ptr()
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data


def _empty_like(a, shape=None, dtype=None):
    if _is_torch(a):
        pin = (not a.is_cuda) and a.is_pinned()
        return torch.empty(shape if shape is not None else a.shape,
                           dtype=dtype if dtype is not None else torch.float64, device=a.device,
                           pin_memory=pin)
    return np.empty(shape if shape is not None else a.shape, dtype=dtype if dtype is not None else np.float64)


def _ptr(a) -> int:
    return a.data_ptr() if _is_torch(a) else a.ctypes.data


def _stream_for(a) -> int:
    if _is_torch(a) and a.is_cuda:
        return torch.cuda.current_stream(a.device).cuda_stream
    return 0


def _shape(q):
    if q.ndim != 2 or q.shape[1] not in (2, 3):
        raise ValueError(f"expected an (n, 2) or (n, 3) array, got {tuple(q.shape)}")
    return int(q.shape[0]), int(q.shape[1])


def _with_dim(prm: Params, dim: int) -> Params:
    p = Params.from_buffer_copy(prm)
    p.dim = dim
    return p


# ------------------------------------------------------------------ entry points
def rhs(q, p, prm: Params):
    """ep_rhs: right-hand side of Eq. N-particle -> (dq, dp)."""
    q, qp = _prep(q, "q")
    p, pp = _prep(p, "p")
    n, dim = _shape(q)
    dq, dp = _empty_like(q), _empty_like(q)
    _check(load().ep_rhs(ctypes.byref(_with_dim(prm, dim)), n, qp, pp, _ptr(dq), _ptr(dp), _stream_for(q)))
    return dq, dp


def rhs_noalloc(q, p, prm: Params, dq=None, dp=None):
    """ep_rhs_noalloc: ep_rhs without any allocation inside the library (device arrays,
    n <= 8192).  Pass preallocated dq, dp to keep the call free of allocations here too."""
    q, qp = _prep(q, "q")
    p, pp = _prep(p, "p")
    n, dim = _shape(q)
    dq = _empty_like(q) if dq is None else dq
    dp = _empty_like(q) if dp is None else dp
    _check(load().ep_rhs_noalloc(ctypes.byref(_with_dim(prm, dim)), n, qp, pp, _ptr(dq), _ptr(dp),
                                 _stream_for(q)))
    return dq, dp


def shoot(q0, p0, prm: Params):
    """ep_shoot: RK4 flow from (q0, p0) over [0, t1] -> (q1, p1)."""
    q0, qp = _prep(q0, "q0")
    p0, pp = _prep(p0, "p0")
    n, dim = _shape(q0)
    q1, p1 = _empty_like(q0), _empty_like(q0)
    _check(load().ep_shoot(ctypes.byref(_with_dim(prm, dim)), n, qp, pp, _ptr(q1), _ptr(p1), _stream_for(q0)))
    return q1, p1


def shoot_tangent(q0, p0, vq0, vp0, prm: Params):
    """ep_shoot_tangent: the RK4 shoot and its derivative along (vq0, vp0) -> (q1, p1, vq1, vp1)."""
    q0, qp = _prep(q0, "q0")
    p0, pp = _prep(p0, "p0")
    vq0, vqp = _prep(vq0, "vq0")
    vp0, vpp = _prep(vp0, "vp0")
    n, dim = _shape(q0)
    q1, p1, vq1, vp1 = (_empty_like(q0) for _ in range(4))
    _check(load().ep_shoot_tangent(ctypes.byref(_with_dim(prm, dim)), n, qp, pp, vqp, vpp, _ptr(q1), _ptr(p1),
                                   _ptr(vq1), _ptr(vp1), _stream_for(q0)))
    return q1, p1, vq1, vp1


def velocity(q, p, x, prm: Params):
    """ep_velocity: u(x_k) = sum_j G(|x_k - q_j|) p_j at the points x (Eq. u)."""
    q, qp = _prep(q, "q")
    p, pp = _prep(p, "p")
    x, xp = _prep(x, "x")
    n, dim = _shape(q)
    m, xdim = _shape(x)
    if xdim != dim:
        raise ValueError(f"x has dimension {xdim}, the particles {dim}")
    u = _empty_like(x)
    _check(load().ep_velocity(ctypes.byref(_with_dim(prm, dim)), n, qp, pp, m, xp, _ptr(u), _stream_for(x)))
    return u


def flow(q0, p0, x0, prm: Params):
    """ep_flow: the points x0 carried by the flow of the shoot from (q0, p0) -> x1."""
    q0, qp = _prep(q0, "q0")
    p0, pp = _prep(p0, "p0")
    x0, xp = _prep(x0, "x0")
    n, dim = _shape(q0)
    m, xdim = _shape(x0)
    if xdim != dim:
        raise ValueError(f"x0 has dimension {xdim}, the particles {dim}")
    x1 = _empty_like(x0)
    _check(load().ep_flow(ctypes.byref(_with_dim(prm, dim)), n, qp, pp, m, xp, _ptr(x1), _stream_for(x0)))
    return x1


def hamiltonian(q, p, prm: Params) -> float:
    """ep_hamiltonian: H of Eq. H (host result)."""
    q, qp = _prep(q, "q")
    p, pp = _prep(p, "p")
    n, dim = _shape(q)
    out = ctypes.c_double(0.0)
    _check(load().ep_hamiltonian(ctypes.byref(_with_dim(prm, dim)), n, qp, pp, ctypes.addressof(out),
                                 _stream_for(q)))
    return out.value


def _shoots(prm: Params, info: MatchInfo, status: int) -> int:
    """Shoots of a matching: iters + 1, except that the inexact system's loop (Sec. 6)
    ends on an update when it converges."""
    return info.iters if (prm.inexact != 0.0 and status == OK) else info.iters + 1


def match(X, Y, prm: Params, h: float = 0.0, eps: float = 1e-6, maxit: int = 200, p0=None,
          hist: bool = True, rule: int = RULE_MOMENTUM, krylov: int = 0) -> MatchResult:
    """ep_match: Algorithm 1 with the update ``rule`` (RULE_MOMENTUM: M = h I on the
    momenta; RULE_VELOCITY: p0 += h G(X)^-1 r; RULE_NEWTON: p0 += h (D phi)^-1 r).
    p0=None starts from zero."""
    X, xp = _prep(X, "X")
    Y, yp = _prep(Y, "Y")
    n, dim = _shape(X)
    if p0 is None:
        p = _empty_like(X)
        if _is_torch(p):
            p.zero_()
        else:
            p[...] = 0.0
    else:
        src, _ = _prep(p0, "p0")
        p = _empty_like(src)
        if _is_torch(p):
            p.copy_(src)
        else:
            p[...] = src
    hbuf = np.full(maxit + 1, np.nan) if hist else None
    info = MatchInfo(float(h), float(eps), int(maxit), 0, 0.0, 0.0, hbuf.ctypes.data if hist else None,
                     int(rule), int(krylov))
    st = load().ep_match(ctypes.byref(_with_dim(prm, dim)), n, xp, yp, _ptr(p), ctypes.byref(info),
                         _stream_for(X))
    _check(st, allowed=(OK, ENOTCONVERGED, EDIVERGED))
    return MatchResult(p, st, info.iters, info.resid_inf, info.H, info.h,
                       hbuf[: _shoots(prm, info, st)] if hist else None, info.products)


def hvp(q, p, vq, vp, prm: Params):
    """ep_hvp: Hessian of H applied to (vq, vp) -> (hq, hp)."""
    q, qp = _prep(q, "q")
    p, pp = _prep(p, "p")
    vq, vqp = _prep(vq, "vq")
    vp, vpp = _prep(vp, "vp")
    n, dim = _shape(q)
    hq, hp = _empty_like(q), _empty_like(q)
    _check(load().ep_hvp(ctypes.byref(_with_dim(prm, dim)), n, qp, pp, vqp, vpp, _ptr(hq), _ptr(hp),
                         _stream_for(q)))
    return hq, hp


def adjoint(X, p0, Y, prm: Params, lam: float, ckpt_every: int = 10):
    """ep_adjoint: (E, dE/dp0) for E = 1/2 p0^T G(X) p0 + lam/2 ||Q(1) - Y||^2."""
    X, xp = _prep(X, "X")
    p0, pp = _prep(p0, "p0")
    Y, yp = _prep(Y, "Y")
    n, dim = _shape(X)
    g = _empty_like(X)
    e = ctypes.c_double(0.0)
    _check(load().ep_adjoint(ctypes.byref(_with_dim(prm, dim)), n, xp, pp, yp, float(lam), int(ckpt_every),
                             _ptr(g), ctypes.addressof(e), _stream_for(X)))
    return e.value, g


def match_batched(Xs, Ys, prms, h=0.0, eps: float = 1e-6, maxit: int = 200):
    """ep_match_batched on a list of problems (X_b, Y_b, params_b); returns a list of MatchResult.

    h may be one value for all problems or a sequence (<= 0: default gain)."""
    if not Xs:
        return []
    t = _is_torch(Xs[0])
    offs = np.zeros(len(Xs) + 1, dtype=np.int64)
    for b, X in enumerate(Xs):
        offs[b + 1] = offs[b] + X.shape[0]
    if t:
        X = torch.cat([x.to(torch.float64) for x in Xs]).contiguous()
        Y = torch.cat([y.to(torch.float64) for y in Ys]).contiguous()
        p = torch.zeros_like(X)
    else:
        X = np.ascontiguousarray(np.concatenate(Xs), dtype=np.float64)
        Y = np.ascontiguousarray(np.concatenate(Ys), dtype=np.float64)
        p = np.zeros_like(X)
    dim = int(X.shape[1])
    nprob = len(Xs)
    P = (Params * nprob)(*[_with_dim(pr, dim) for pr in prms])
    hs = list(h) if hasattr(h, "__len__") else [h] * nprob
    infos = (MatchInfo * nprob)(*[MatchInfo(float(hs[b]), float(eps), int(maxit), 0, 0.0, 0.0, None)
                                  for b in range(nprob)])
    st = load().ep_match_batched(P, nprob, offs.ctypes.data, _ptr(X), _ptr(Y), _ptr(p), infos, _stream_for(X))
    _check(st, allowed=(OK, ENOTCONVERGED, EDIVERGED))
    out = []
    for b in range(nprob):
        sl = slice(int(offs[b]), int(offs[b + 1]))
        inf = infos[b]
        out.append(MatchResult(p[sl], int(inf.status), inf.iters, inf.resid_inf, inf.H, inf.h, None))
    return out


def cell_neighbors(q, prm: Params):
    """ep_cell_neighbors: (count[n] int64, hash[n] uint64, total) of the cell-list predicate."""
    q, qp = _prep(q, "q")
    n, dim = _shape(q)
    if _is_torch(q):
        cnt = torch.empty(n, dtype=torch.int64, device=q.device)
        hsh = torch.empty(n, dtype=torch.int64, device=q.device)  # uint64 bits
    else:
        cnt = np.empty(n, dtype=np.int64)
        hsh = np.empty(n, dtype=np.uint64)
    tot = ctypes.c_int64(0)
    _check(load().ep_cell_neighbors(ctypes.byref(_with_dim(prm, dim)), n, qp, _ptr(cnt), _ptr(hsh),
                                    ctypes.addressof(tot), _stream_for(q)))
    return cnt, hsh, tot.value
