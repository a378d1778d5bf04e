"""ctypes front end of the FP64 CPU oracle (``ep_oracle.c``).

TEST INFRASTRUCTURE ONLY: the independent reference that the CUDA library is
checked against.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module; the library itself never
does, and this module imports nothing from the library.

Each function marshals numpy float64 arrays of shape (n, dim) into the C
routine of the same name and documents the passage of arXiv 1510.03816 it
follows (see the C file for the formulas).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

GAUSS, TENT, EXPCONE = 0, 1, 2
OK, EINVAL, ENOTCONVERGED, EDIVERGED = 0, 1, 4, 5

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ep_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libep_oracle.so")
# A prebuilt variant of the oracle (used only by the mutation test, which plants
# mistakes in a copy of ep_oracle.c and checks that the pins reject it).
_VARIANT = os.environ.get("EP_ORACLE_VARIANT_LIB")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``ep_oracle.c`` into ``libep_oracle.so`` next to it (gcc, OpenMP).

    ``-ffp-contract=off`` keeps every FP64 expression rounded as written.  No
    ``-march`` flag: the same source builds on x86-64 and aarch64.
    """
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-std=c11", "-shared", "-fPIC",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if _VARIANT:
            lib = ctypes.CDLL(_VARIANT)
        else:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
        d, i, l, p = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
        lib.orc_G.restype = d
        lib.orc_G.argtypes = [i, d, d]
        lib.orc_phi.restype = d
        lib.orc_phi.argtypes = [i, d, d]
        lib.orc_psi.restype = d
        lib.orc_psi.argtypes = [i, d, d]
        lib.orc_rhs.restype = None
        lib.orc_rhs.argtypes = [i, i, d, l, p, p, p, p]
        lib.orc_hamiltonian.restype = d
        lib.orc_hamiltonian.argtypes = [i, i, d, l, p, p]
        lib.orc_shoot.restype = i
        lib.orc_shoot.argtypes = [i, i, d, i, d, l, p, p, p, p]
        lib.orc_default_gain.restype = d
        lib.orc_default_gain.argtypes = [i, i, d, l, p]
        lib.orc_match.restype = i
        lib.orc_match.argtypes = [i, i, d, i, d, l, p, p, d, d, i, p, p, p, p]
        lib.orc_hvp.restype = None
        lib.orc_hvp.argtypes = [i, i, d, l, p, p, p, p, p, p]
        lib.orc_adjoint.restype = d
        lib.orc_adjoint.argtypes = [i, i, d, i, d, l, p, p, p, d, p]
        lib.orc_cell_grid.restype = None
        lib.orc_cell_grid.argtypes = [i, d, l, p, p, p, p]
        lib.orc_cell_neighbors.restype = l
        lib.orc_cell_neighbors.argtypes = [i, d, l, p, p, p]
        lib.orc_rhs_rows.restype = None
        lib.orc_rhs_rows.argtypes = [i, i, d, l, p, p, p, l, p, p]
        lib.orc_cell_neighbors_rows.restype = None
        lib.orc_cell_neighbors_rows.argtypes = [i, d, l, p, p, l, p, p]
        lib.orc_velocity.restype = None
        lib.orc_velocity.argtypes = [i, i, d, l, p, p, l, p, p]
        lib.orc_flow.restype = i
        lib.orc_flow.argtypes = [i, i, d, i, d, l, p, p, l, p, p, p, p]
        lib.orc_rhs_inexact.restype = None
        lib.orc_rhs_inexact.argtypes = [i, i, d, d, l, p, p, p, p]
        lib.orc_shoot_inexact.restype = i
        lib.orc_shoot_inexact.argtypes = [i, i, d, d, i, d, l, p, p, p, p]
        lib.orc_match_inexact.restype = i
        lib.orc_match_inexact.argtypes = [i, i, d, d, i, d, l, p, p, d, d, i, p, p, p, p]
        lib.orc_shoot_tangent.restype = i
        lib.orc_shoot_tangent.argtypes = [i, i, d, i, d, l, p, p, p, p, p, p, p, p]
        lib.orc_set_threads.restype = None
        lib.orc_set_threads.argtypes = [i]
        lib.orc_max_threads.restype = i
        lib.orc_max_threads.argtypes = []
        _lib = lib
        return lib


def _arr(a, dim=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if dim is not None and (a.ndim != 2 or a.shape[1] != dim):
        raise ValueError(f"expected an (n, {dim}) array, got {a.shape}")
    return a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def G(kernel: int, sigma: float, r: float) -> float:
    """Kernel value (Sec. 3, Eq. Green-nD family; Gaussian, tent, expcone)."""
    return _load().orc_G(kernel, sigma, r)


def phi(kernel: int, sigma: float, r: float) -> float:
    """G'(r)/r, the radial factor of the momentum equation of Eq. N-particle."""
    return _load().orc_phi(kernel, sigma, r)


def psi(kernel: int, sigma: float, r: float) -> float:
    """phi'(r)/r, needed by the Hessian of H."""
    return _load().orc_psi(kernel, sigma, r)


def rhs(q, p, kernel: int, sigma: float):
    """Right-hand side of Eq. N-particle: returns (dq/dt, dp/dt)."""
    q = _arr(q)
    dim = q.shape[1]
    p = _arr(p, dim)
    dq = np.empty_like(q)
    dp = np.empty_like(q)
    _load().orc_rhs(dim, kernel, sigma, q.shape[0], _ptr(q), _ptr(p), _ptr(dq), _ptr(dp))
    return dq, dp


def hamiltonian(q, p, kernel: int, sigma: float) -> float:
    """Discrete Hamiltonian of Eq. H (E = 2H is the kinetic energy, Eq. E=2H)."""
    q = _arr(q)
    p = _arr(p, q.shape[1])
    return _load().orc_hamiltonian(q.shape[1], kernel, sigma, q.shape[0], _ptr(q), _ptr(p))


def shoot(q0, p0, kernel: int, sigma: float, steps: int, t1: float = 1.0):
    """Classical RK4 flow of Eq. N-particle from (q0, p0) to t1: returns (q1, p1)."""
    q0 = _arr(q0)
    p0 = _arr(p0, q0.shape[1])
    q1 = np.empty_like(q0)
    p1 = np.empty_like(q0)
    st = _load().orc_shoot(q0.shape[1], kernel, sigma, steps, t1, q0.shape[0], _ptr(q0), _ptr(p0),
                           _ptr(q1), _ptr(p1))
    if st != OK:
        raise ValueError(f"orc_shoot status {st}")
    return q1, p1


def default_gain(X, kernel: int, sigma: float) -> float:
    """h = 1 / max_i sum_j |G(|X_i - X_j|)| (Gershgorin bound on lambda_max of G(X))."""
    X = _arr(X)
    return _load().orc_default_gain(X.shape[1], kernel, sigma, X.shape[0], _ptr(X))


def match(X, Y, kernel: int, sigma: float, steps: int, h: float = 0.0, eps: float = 1e-6,
          maxit: int = 200, p0=None, t1: float = 1.0):
    """Algorithm 1 with gain M = h I on the momenta (p0 += h (Y - Q(1))).

    Returns (p0, status, iters, resid, hist) where hist[k] is the max-norm
    residual of shoot k (iters + 1 shoots).
    """
    X = _arr(X)
    dim = X.shape[1]
    Y = _arr(Y, dim)
    p = np.zeros_like(X) if p0 is None else _arr(p0, dim).copy()
    iters = ctypes.c_int(0)
    resid = ctypes.c_double(0.0)
    hist = np.full(maxit + 1, np.nan)
    st = _load().orc_match(dim, kernel, sigma, steps, t1, X.shape[0], _ptr(X), _ptr(Y), h, eps, maxit,
                           _ptr(p), ctypes.byref(iters), ctypes.byref(resid), _ptr(hist))
    if st == EINVAL:
        raise ValueError("orc_match: invalid arguments")
    return p, st, iters.value, resid.value, hist[: iters.value + 1]


def hvp(q, p, vq, vp, kernel: int, sigma: float):
    """Hessian of H (Eq. H) applied to (vq, vp): returns (Hv_q, Hv_p)."""
    q = _arr(q)
    dim = q.shape[1]
    p, vq, vp = _arr(p, dim), _arr(vq, dim), _arr(vp, dim)
    hq = np.empty_like(q)
    hp = np.empty_like(q)
    _load().orc_hvp(dim, kernel, sigma, q.shape[0], _ptr(q), _ptr(p), _ptr(vq), _ptr(vp), _ptr(hq),
                    _ptr(hp))
    return hq, hp


def adjoint(X, p0, Y, kernel: int, sigma: float, steps: int, lam: float, t1: float = 1.0):
    """Energy E = H(X, p0) + lam/2 ||Q(1) - Y||^2 (Eq. inexact-E) and dE/dp0 by the
    exact discrete adjoint of the RK4 shoot.  Returns (E, grad)."""
    X = _arr(X)
    dim = X.shape[1]
    p0, Y = _arr(p0, dim), _arr(Y, dim)
    grad = np.empty_like(X)
    e = _load().orc_adjoint(dim, kernel, sigma, steps, t1, X.shape[0], _ptr(X), _ptr(p0), _ptr(Y), lam,
                            _ptr(grad))
    return e, grad


def energy(X, p0, Y, kernel: int, sigma: float, steps: int, lam: float, t1: float = 1.0) -> float:
    """E(p0) = H(X, p0) + lam/2 ||Q(1) - Y||^2 by a forward shoot (no gradient)."""
    q1, _ = shoot(X, p0, kernel, sigma, steps, t1)
    return hamiltonian(X, p0, kernel, sigma) + 0.5 * lam * float(np.sum((q1 - _arr(Y)) ** 2))


def cell_grid(q, sigma: float):
    """Grid of the cell-list acceptance test (lo, cell edge, cell count per axis)."""
    q = _arr(q)
    dim = q.shape[1]
    lo = np.zeros(3)
    hc = np.zeros(3)
    nc = np.zeros(3, dtype=np.int64)
    _load().orc_cell_grid(dim, sigma, q.shape[0], _ptr(q), _ptr(lo), _ptr(hc),
                          nc.ctypes.data_as(ctypes.c_void_p))
    return lo[:dim], hc[:dim], nc[:dim]


def cell_neighbors(q, sigma: float):
    """Brute-force neighbour sets of the cell-list predicate.

    Returns (count[n] int64, hash[n] uint64, total accepted pairs)."""
    q = _arr(q)
    n, dim = q.shape
    cnt = np.zeros(n, dtype=np.int64)
    hsh = np.zeros(n, dtype=np.uint64)
    tot = _load().orc_cell_neighbors(dim, sigma, n, _ptr(q), cnt.ctypes.data_as(ctypes.c_void_p),
                                     hsh.ctypes.data_as(ctypes.c_void_p))
    return cnt, hsh, int(tot)


def rhs_rows(q, p, rows, kernel: int, sigma: float):
    """Eq. N-particle for the particles in ``rows`` only (sums over all j)."""
    q = _arr(q)
    dim = q.shape[1]
    p = _arr(p, dim)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    dq = np.empty((rows.size, dim))
    dp = np.empty((rows.size, dim))
    _load().orc_rhs_rows(dim, kernel, sigma, q.shape[0], _ptr(q), _ptr(p), rows.ctypes.data_as(ctypes.c_void_p),
                         rows.size, _ptr(dq), _ptr(dp))
    return dq, dp


def cell_neighbors_rows(q, rows, sigma: float):
    """Brute-force neighbour sets of the cell-list predicate for the particles in ``rows``."""
    q = _arr(q)
    n, dim = q.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cnt = np.zeros(rows.size, dtype=np.int64)
    hsh = np.zeros(rows.size, dtype=np.uint64)
    _load().orc_cell_neighbors_rows(dim, sigma, n, _ptr(q), rows.ctypes.data_as(ctypes.c_void_p), rows.size,
                                    cnt.ctypes.data_as(ctypes.c_void_p), hsh.ctypes.data_as(ctypes.c_void_p))
    return cnt, hsh


def velocity(q, p, x, kernel: int, sigma: float):
    """Eq. u: u(x_k) = sum_j G(|x_k - q_j|) p_j at the points x (m, dim)."""
    q = _arr(q)
    dim = q.shape[1]
    p = _arr(p, dim)
    x = _arr(x, dim)
    u = np.empty_like(x)
    _load().orc_velocity(dim, kernel, sigma, q.shape[0], _ptr(q), _ptr(p), x.shape[0], _ptr(x), _ptr(u))
    return u


def flow(q0, p0, x0, kernel: int, sigma: float, steps: int, t1: float = 1.0):
    """Points x0 transported by the flow of the shoot from (q0, p0): returns (Q1, P1, X1)."""
    q0 = _arr(q0)
    dim = q0.shape[1]
    p0 = _arr(p0, dim)
    x0 = _arr(x0, dim)
    q1, p1, x1 = np.empty_like(q0), np.empty_like(p0), np.empty_like(x0)
    st = _load().orc_flow(dim, kernel, sigma, steps, t1, q0.shape[0], _ptr(q0), _ptr(p0), x0.shape[0], _ptr(x0),
                          _ptr(q1), _ptr(p1), _ptr(x1))
    if st != 0:
        raise ValueError("orc_flow: invalid arguments")
    return q1, p1, x1


def rhs_inexact(q, p, kernel: int, sigma: float, s2: float):
    """Eq. N-particle-inexact: dq gains s2 p_i (s2 = sigma_n^2)."""
    q = _arr(q)
    dim = q.shape[1]
    p = _arr(p, dim)
    dq, dp = np.empty_like(q), np.empty_like(q)
    _load().orc_rhs_inexact(dim, kernel, sigma, s2, q.shape[0], _ptr(q), _ptr(p), _ptr(dq), _ptr(dp))
    return dq, dp


def shoot_inexact(q0, p0, kernel: int, sigma: float, s2: float, steps: int, t1: float = 1.0):
    q0 = _arr(q0)
    dim = q0.shape[1]
    p0 = _arr(p0, dim)
    q1, p1 = np.empty_like(q0), np.empty_like(p0)
    if _load().orc_shoot_inexact(dim, kernel, sigma, s2, steps, t1, q0.shape[0], _ptr(q0), _ptr(p0), _ptr(q1),
                                 _ptr(p1)) != 0:
        raise ValueError("orc_shoot_inexact: invalid arguments")
    return q1, p1


def match_inexact(X, Y, kernel: int, sigma: float, s2: float, steps: int, h: float = 0.0, eps: float = 1e-6,
                  maxit: int = 200, p0=None, t1: float = 1.0):
    """Algorithm 1 on the inexact system with the momentum-difference stop:
    returns (p0, status, iters, resid, hist)."""
    X = _arr(X)
    dim = X.shape[1]
    Y = _arr(Y, dim)
    p = np.zeros_like(X) if p0 is None else _arr(p0, dim).copy()
    it, res = ctypes.c_int(0), ctypes.c_double(0.0)
    hist = np.full(maxit + 1, np.nan)
    st = _load().orc_match_inexact(dim, kernel, sigma, s2, steps, t1, X.shape[0], _ptr(X), _ptr(Y), h, eps, maxit,
                                   _ptr(p), ctypes.byref(it), ctypes.byref(res), _ptr(hist))
    if st == EINVAL:
        raise ValueError("orc_match_inexact: invalid arguments")
    shoots = it.value if st == OK else it.value + 1  # a converged loop ends on an update
    return p, st, it.value, res.value, hist[:shoots]


def shoot_tangent(q0, p0, vq0, vp0, kernel: int, sigma: float, steps: int, t1: float = 1.0):
    """Derivative of the RK4 shoot at (q0, p0) along (vq0, vp0): returns (Q1, P1, dQ1, dP1)."""
    q0 = _arr(q0)
    dim = q0.shape[1]
    p0, vq0, vp0 = _arr(p0, dim), _arr(vq0, dim), _arr(vp0, dim)
    q1, p1, vq1, vp1 = (np.empty_like(q0) for _ in range(4))
    if _load().orc_shoot_tangent(dim, kernel, sigma, steps, t1, q0.shape[0], _ptr(q0), _ptr(p0), _ptr(vq0),
                                 _ptr(vp0), _ptr(q1), _ptr(p1), _ptr(vq1), _ptr(vp1)) != 0:
        raise ValueError("orc_shoot_tangent: invalid arguments")
    return q1, p1, vq1, vp1


def shooting_jacobian(X, p0, kernel: int, sigma: float, steps: int, t1: float = 1.0):
    """D phi = dQ(1)/dp0 (n d x n d, row-major flattening), one tangent shoot per column."""
    X = _arr(X)
    n, dim = X.shape
    p0 = _arr(p0, dim)
    J = np.empty((n * dim, n * dim))
    zero = np.zeros_like(X)
    for a in range(n * dim):
        e = np.zeros(n * dim)
        e[a] = 1.0
        J[:, a] = shoot_tangent(X, p0, zero, e.reshape(n, dim), kernel, sigma, steps, t1)[2].ravel()
    return J


def match_newton(X, Y, kernel: int, sigma: float, steps: int, h: float = 1.0, eps: float = 1e-6,
                 maxit: int = 50, p0=None, t1: float = 1.0):
    """Algorithm 1 with the Newton-type gain of Sec. 5: p0 <- p0 + h (D phi)^-1 (Y - Q(1)),
    D phi from tangent shoots and solved directly (a library LU).  Stopping as Algorithm 1;
    returns (p0, status, iters, resid, hist)."""
    X = _arr(X)
    n, dim = X.shape
    Y = _arr(Y, dim)
    p = np.zeros_like(X) if p0 is None else _arr(p0, dim).copy()
    hist = []
    k = 0
    while True:
        q1, _ = shoot(X, p, kernel, sigma, steps, t1)
        r = Y - q1
        res = float(np.abs(r).max()) if np.all(np.isfinite(r)) else float("nan")
        hist.append(res)
        if not np.isfinite(res):
            return p, EDIVERGED, k, res, np.array(hist)
        if res < eps:
            return p, OK, k, res, np.array(hist)
        if k == maxit:
            return p, ENOTCONVERGED, k, res, np.array(hist)
        J = shooting_jacobian(X, p, kernel, sigma, steps, t1)
        p = p + h * np.linalg.solve(J, r.ravel()).reshape(n, dim)
        k += 1


def gram(X, kernel: int, sigma: float):
    """G(X): the n x n matrix of kernel values G(|X_i - X_j|) (Eq. u at t = 0 is u = G(X) p)."""
    X = _arr(X)
    n = X.shape[0]
    K = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            K[i, j] = G(kernel, sigma, float(np.sqrt(np.sum((X[i] - X[j]) ** 2))))
    return K


def match_velocity(X, Y, kernel: int, sigma: float, steps: int, h: float = 1.0, eps: float = 1e-6,
                   maxit: int = 200, p0=None, t1: float = 1.0):
    """Algorithm 1 with the update applied to the velocity (steps 3 and 4): u0 = G(X) p0 is
    corrected by u0 += h (Y - Q(1)) and the momenta recovered from it, p0 = G(X)^-1 u0, i.e.
    p0 <- p0 + h G(X)^-1 (Y - Q(1)) (a library LU per component).  Stopping as Algorithm 1;
    returns (p0, status, iters, resid, hist)."""
    X = _arr(X)
    n, dim = X.shape
    Y = _arr(Y, dim)
    p = np.zeros_like(X) if p0 is None else _arr(p0, dim).copy()
    GX = gram(X, kernel, sigma)
    hist = []
    k = 0
    while True:
        q1, _ = shoot(X, p, kernel, sigma, steps, t1)
        r = Y - q1
        res = float(np.abs(r).max()) if np.all(np.isfinite(r)) else float("nan")
        hist.append(res)
        if not np.isfinite(res):
            return p, EDIVERGED, k, res, np.array(hist)
        if res < eps:
            return p, OK, k, res, np.array(hist)
        if k == maxit:
            return p, ENOTCONVERGED, k, res, np.array(hist)
        p = p + h * np.linalg.solve(GX, r)
        k += 1
