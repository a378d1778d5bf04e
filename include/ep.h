/*
 * ep.h -- C ABI of libep.so: GPU (sm_103a) geodesic landmark shooting with the
 * N-particle Euler-Poincare system of Camassa, Kuang & Lee (arXiv 1510.03816).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Arrays are row-major (n, dim) float64 with dim in {2, 3}: particle i's
 *    coordinates are a[i*dim + 0 .. i*dim + dim-1].
 *  - Array pointers may be CUDA device memory or host memory (pageable or
 *    pinned); the library detects which with cudaPointerGetAttributes and
 *    stages host arrays through its own device workspace.  The caller owns
 *    every array; the library never frees or retains them past the call.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    stream-ordered and asynchronous when all arrays are device memory, except
 *    where an entry point says it synchronises.  When any array is host
 *    memory the call synchronises the stream before returning.
 *  - The library allocates its workspace itself (cached per device and
 *    stream, grown on demand, released by ep_release_workspace).
 *  - Every entry point returns an ep_status and never throws.  On an error the
 *    outputs are unspecified unless stated; ep_last_error() describes it.
 *  - Not thread-safe for concurrent calls on the same stream.
 */
#ifndef EP_H
#define EP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EP_OK = 0,
    EP_EINVAL = 1,        /* bad argument (size, pointer, parameter) */
    EP_ENOMEM = 2,        /* workspace allocation failed */
    EP_ECUDA = 3,         /* a CUDA runtime call or kernel failed */
    EP_ENOTCONVERGED = 4, /* ep_match: iteration cap reached; p0 holds the last iterate */
    EP_EDIVERGED = 5,     /* ep_match: residual became NaN/Inf; p0 holds the last finite iterate */
    EP_ETIMEOUT = 6       /* a device-side bounded wait gave up (kernel returned early) */
} ep_status;

/* Kernels G(r) of the N-particle system (Sec. 3 of the paper).
 *  EP_GAUSS   G = exp(-r^2 / (2 sigma^2))   smooth kernel of the metric H^inf (Sec. 6)
 *  EP_TENT    G = max(1 - r/sigma, 0)       compactly supported cone; enables the cell list
 *  EP_EXPCONE G = exp(-r / sigma)           the paper's "conon" (Eq. nu=3/2, alpha = sigma) */
typedef enum { EP_GAUSS = 0, EP_TENT = 1, EP_EXPCONE = 2 } ep_kernel;

/* EP_FP64: every operation in FP64 (the plain comparison path).
 * EP_MIXED: pair terms in FP32; each per-particle sum of the all-pairs right-hand
 *           side (and of the adjoint's Hessian products) is formed in FP32 over
 *           blocks of at most 256 sources per warp, and the blocks are accumulated
 *           in compensated double-FP32 (TwoSum) arithmetic and, across thread
 *           blocks, in FP64, so the sums carry FP64-level accumulation error
 *           whatever n is; the batched solver folds FP32 runs of 512 sources into
 *           FP64; the cell list sums each particle's at most nine neighbour cells
 *           in FP32 (a bounded block).  The RK4 stage combination is FP32 on the
 *           sums rounded once; the step state, the feedback residual and the
 *           momentum update are FP64. */
typedef enum { EP_FP64 = 0, EP_MIXED = 1 } ep_precision;

/* EP_AUTO picks the cell list for EP_TENT when it pays off, else all-pairs. */
typedef enum { EP_AUTO = 0, EP_ALLPAIRS = 1, EP_CELLLIST = 2 } ep_neigh;

/* Update rule of ep_match (Algorithm 1 steps 3-4 and Sec. 5), r = Y - Q(1):
 *  EP_RULE_MOMENTUM  p0 += h r              M = h I applied to the momenta (default)
 *  EP_RULE_VELOCITY  p0 += h G(X)^-1 r      the velocity u = G(X) p0 (Eq. u at t = 0) is
 *                                           updated by u += h r and p0 recovered from u
 *                                           (Algorithm 1 step 4)
 *  EP_RULE_NEWTON    p0 += h (D phi)^-1 r   the gain M = h (D phi)^-1 of Theorem 1,
 *                                           D phi = dQ(1)/dp0 of the RK4 shoot
 * The solved rules (velocity, Newton) run on the all-pairs path of the exact system
 * (EP_EINVAL otherwise); their residual, solve and update are FP64.
 *  - Velocity, FP64: inside the device-resident matching launch.  For n <= 512 G(X)
 *    is factored once (LU with partial pivoting); otherwise, or when a pivot
 *    vanishes, every update runs MINRES on the symmetric G(X) (the tent's need not
 *    be positive definite), one all-pairs Gram product per iteration.
 *  - Velocity, mixed precision (n <= 512): mixed shoots, G(X) in FP64 factored once.
 *  - Newton, n dim <= 384: D phi formed whole on the device, one tangent-linear shoot
 *    per column, all in one launch (FP64; FP32 in mixed precision, an inexact
 *    Newton method), solved by Gaussian elimination with partial pivoting (a
 *    singular D phi returns EP_EDIVERGED).
 *  - Newton, FP64, larger: restarted GMRES on the host (ep_match_info.krylov vectors)
 *    whose products are tangent-linear shoots along (0, v) (ep_shoot_tangent). */
typedef enum { EP_RULE_MOMENTUM = 0, EP_RULE_VELOCITY = 1, EP_RULE_NEWTON = 2 } ep_rule;

typedef struct {
    int dim;        /* 2 or 3 */
    int kernel;     /* ep_kernel */
    double sigma;   /* kernel width, > 0 */
    int steps;      /* RK4 steps S >= 1 on [0, t1] */
    double t1;      /* end time; 1.0 for the matching problem (Eq. exact-matching) */
    int precision;  /* ep_precision */
    int neigh;      /* ep_neigh */
    double inexact; /* sigma_n^2 >= 0 of the inexact particle system (Sec. 6, Eq.
                       N-particle-inexact): dq_i gains inexact * p_i.  0 = the exact
                       system.  With inexact > 0, ep_match stops when two consecutive
                       initial momenta differ by less than eps (Sec. 6) and its default
                       gain is 1 / (max_i sum_j G_ij + inexact).  Supported on the
                       all-pairs paths of ep_rhs, ep_shoot, ep_match and ep_rhs_noalloc;
                       the cell list, ep_match_batched, ep_hvp, ep_adjoint, ep_velocity
                       and ep_flow return EP_EINVAL for inexact != 0. */
} ep_params;

typedef struct {
    double h;        /* in: gain of M = h I (<= 0: h = 1 / max_i sum_j G_ij); out: gain used */
    double eps;      /* in: stop when max_i,c |Y - Q(1)| < eps */
    int maxit;       /* in: maximum number of momentum updates (>= 0) */
    int iters;       /* out: number of updates performed (shoots = iters + 1; iters when an
                        inexact matching converges, since it ends on an update) */
    double resid_inf;/* out: max-norm residual of the last shoot */
    double H;        /* out: Hamiltonian H(X, p0) of Eq. H for the returned p0 */
    double* hist;    /* in, optional: maxit + 1 doubles (host or device) that receive the
                        residual of every shoot; NULL for none */
    int rule;        /* in: ep_rule (0 = EP_RULE_MOMENTUM).  For the solved rules h <= 0
                        means h = 1; ep_match_batched requires EP_RULE_MOMENTUM */
    int krylov;      /* in: Krylov size of the solved rules (0 = min(n dim, 200)): the GMRES
                        restart length (Newton); the inner solve (GMRES or MINRES) stops at
                        relative residual 1e-12 or after 4 krylov products */
    int products;    /* out: matrix-vector products of the solved rules over the whole
                        matching: tangent shoots (Jacobian columns or Krylov products) for
                        Newton; MINRES Gram products, or one solve per component and
                        update with the factored G(X), for the velocity rule; 0 for the
                        momentum rule */
    int status;      /* out: ep_status of this matching (Algorithm 1 steps 2-3: EP_OK when
                        max|Y - Q(1)| < eps was reached, EP_ENOTCONVERGED at the iteration
                        cap, EP_EDIVERGED on a non-finite residual or a singular solve).
                        ep_match sets it to its return value; ep_match_batched sets it per
                        problem (its return value is the first non-OK one) */
} ep_match_info;

/* Right-hand side of the N-particle system (Sec. 3.1, Eq. N-particle):
 *   dq_i =  sum_j G(|q_i - q_j|) p_j                    (j = i included, G(0) = 1)
 *   dp_i = -sum_{j != i} (p_i . p_j) G'(r_ij) (q_i - q_j) / r_ij
 * Tent and expcone take the dp term of a coincident pair (r = 0) as zero; the tent's
 * dp term vanishes for r >= sigma.  q, p: inputs (n, dim); dq, dp: outputs (n, dim).
 * n = 0 is a no-op.  Errors: EP_EINVAL for a bad params/n/pointer. */
ep_status ep_rhs(const ep_params* params, int64_t n, const double* q, const double* p,
                 double* dq, double* dp, void* stream);

/* Geodesic shoot (Sec. 4, Algorithm 1 step 1): classical RK4 (Note 1 item 5) with
 * params->steps uniform steps from (q0, p0) at t = 0 to t = params->t1.  Outputs
 * q1, p1 (n, dim); they may alias q0, p0. */
ep_status ep_shoot(const ep_params* params, int64_t n, const double* q0, const double* p0,
                   double* q1, double* p1, void* stream);

/* Feedback-control matching (Sec. 4, Algorithm 1 with the constant gain M = h I of
 * Sec. 5, applied to the momenta): repeat { Q(1) = shoot(X, p0); r = Y - Q(1);
 * stop if max|r| < eps; p0 += h r } at most info->maxit updates.  p0: in = initial
 * guess (zeros for the paper's default, Note 1 item 4), out = last iterate.  The
 * residual and the update are FP64 in both precisions.  Synchronises the stream.
 * Where the loop runs: FP64 on the all-pairs path, one cooperative launch; small 2-D
 * mixed-precision problems (n <= 384), one CTA of the batched solver; the 2-D Gaussian
 * in mixed precision with the owner-computes shoot (n <= 4096), one CUDA graph per
 * matching (a while-loop node over the shoot and a one-CTA kernel for the residual,
 * the stopping test and the update; EP_DEVICE_MATCH=0 in the environment selects the
 * host loop instead, with the same results); otherwise a host loop that reads the
 * stopping test back each iteration.  Returns EP_OK, EP_ENOTCONVERGED or EP_EDIVERGED
 * (EP_ETIMEOUT if a grid-barrier wait of a persistent shoot gave up); info is filled
 * in the first three cases. */
ep_status ep_match(const ep_params* params, int64_t n, const double* X, const double* Y,
                   double* p0, ep_match_info* info, void* stream);

/* Tangent-linear shoot (Sec. 5, the derivative D phi of the shooting map): the RK4
 * shoot of ep_shoot from (q0, p0) differentiated along (vq0, vp0); each stage
 * applies the Jacobian of Eq. N-particle's right-hand side, (d2H v)_p and -(d2H v)_q
 * of Eq. H, at the recorded stage state.  Outputs q1, p1 (the shoot, may be NULL) and
 * vq1, vp1 = d(Q(1), P(1)) along (vq0, vp0), all (n, dim).  FP64, all-pairs, exact
 * system (EP_EINVAL otherwise).  Synchronises the stream. */
ep_status ep_shoot_tangent(const ep_params* params, int64_t n, const double* q0, const double* p0,
                           const double* vq0, const double* vp0, double* q1, double* p1, double* vq1,
                           double* vp1, void* stream);

/* Gradient of the inexact-matching energy (Sec. 6, Eq. inexact-E, written with
 * Eq. E=2H):  E(p0) = 1/2 p0^T G(X) p0 + lambda/2 ||Q(1) - Y||^2  with respect to
 * p0, by the exact discrete adjoint of the RK4 shoot.  Step states are
 * checkpointed every ckpt_every steps (>= 1) and recomputed in reverse.
 * grad_p0: output (n, dim).  energy: output, one double (host or device), may be
 * NULL. */
ep_status ep_adjoint(const ep_params* params, int64_t n, const double* X, const double* p0,
                     const double* Y, double lambda, int ckpt_every, double* grad_p0,
                     double* energy, void* stream);

/* nprob independent matchings in one persistent launch.  Problem b has
 * n_b = offsets[b+1] - offsets[b] particles stored at rows offsets[b] .. of X, Y and
 * p0 (all (offsets[nprob], dim)); p0 holds the initial guesses on entry and the last
 * iterates on return.  params[b] and infos[b] are its parameters and result (host
 * arrays; infos[b].hist is ignored).  Limits: dim = 2, EP_MIXED, n_b <= 8192.  offsets: host array of nprob+1
 * int64 with offsets[0] = 0, non-decreasing.  All problems must share dim.
 * Synchronises the stream.  Returns EP_OK when every problem converged, else
 * the first non-OK status in problem order; infos[b].status holds problem b's own
 * status (set by the solver on the device). */
ep_status ep_match_batched(const ep_params* params, int nprob, const int64_t* offsets,
                           const double* X, const double* Y, double* p0, ep_match_info* infos,
                           void* stream);

/* Discrete Hamiltonian (Sec. 3.1, Eq. H): H = 1/2 sum_i sum_j (p_i . p_j) G(|q_i - q_j|)
 * (the kinetic energy of Eq. E=2H is 2H).  H_out: one double (host or device). */
ep_status ep_hamiltonian(const ep_params* params, int64_t n, const double* q, const double* p,
                         double* H_out, void* stream);

/* Hessian of H applied to v = (vq, vp): (hq, hp) = d2H(q, p) . (vq, vp).  This is the
 * pair kernel of the adjoint (the transposed stage Jacobian is J^T w = d2H . (-w_p, w_q)).
 * All arrays (n, dim). */
ep_status ep_hvp(const ep_params* params, int64_t n, const double* q, const double* p,
                 const double* vq, const double* vp, double* hq, double* hp, void* stream);

/* Neighbour sets of the cell-list path (EP_TENT only) at positions q (n, dim), for
 * validation: count[i] = number of accepted j (self included) and
 * hash[i] = sum over accepted j of (j + 1) * 2654435761 mod 2^64.  The grid and the
 * FP32 acceptance test are the ones the cell-list RHS uses: cell edge
 * h = sigma (1 + 2^-8) per axis (wider when more than 2048 (2-D) / 256 (3-D) cells
 * would be needed), origin min(q) - 2h, local FP32 offsets in units of sigma, and
 * accept iff fmaf(d0, d0, d1*d1 [+ d2*d2]) < 1.0f.  count, hash: outputs (n) int64
 * and uint64; total: output, one int64 (host or device), may be NULL. */
ep_status ep_cell_neighbors(const ep_params* params, int64_t n, const double* q, int64_t* count,
                            uint64_t* hash, int64_t* total, void* stream);

/* ep_rhs for callers that may not allocate device memory during the call.  The
 * paper has no counterpart: this is a library-interface variant of ep_rhs.
 * Some callers cannot call cudaMalloc at that point, for example a real-time or
 * callback context where cudaMalloc's implicit synchronisation is not allowed, or
 * a host framework whose memory pool owns the device.  This call takes all its
 * scratch from a fixed array compiled into the library (about 1.25 MiB on every
 * device that loads libep.so, held until the process exits) and never allocates.
 * Limits and rules:
 *  - n <= EP_NOALLOC_MAX_N; larger n returns EP_EINVAL.
 *  - all-pairs path only (params->neigh == EP_CELLLIST returns EP_EINVAL);
 *  - q, p, dq, dp must be device memory (host arrays return EP_EINVAL);
 *  - the first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.  The address is kept per device and context:
 *    after cudaDeviceReset the next call looks it up again (so it too should
 *    come before any capture);
 *  - every call shares the one array; calls whose GPU work overlaps (for
 *    example on two unordered streams) race and give wrong results.
 * Results are those of ep_rhs (same kernels). */
#define EP_NOALLOC_MAX_N 8192
ep_status ep_rhs_noalloc(const ep_params* params, int64_t n, const double* q, const double* p,
                         double* dq, double* dp, void* stream);

/* Velocity field of the particles' momenta at m points (Sec. 3.1, Eq. u):
 *   u(x_k) = sum_{j=1..n} G(|x_k - q_j|) p_j.
 * q, p: (n, dim); x, u: (m, dim); row-major FP64, device or host memory (host
 * arrays are staged and the call then synchronises).  All pairs over the n
 * particles in params->precision (EP_MIXED: FP32 pair terms, FP32 sums, FP64
 * result); params->neigh must not be EP_CELLLIST.  x and u may alias.  Errors:
 * EP_EINVAL for bad sizes, NULL arrays or parameters. */
ep_status ep_velocity(const ep_params* params, int64_t n, const double* q, const double* p, int64_t m,
                      const double* x, double* u, void* stream);

/* Transport of m points by the flow of the shoot from (q0, p0): Eq. u integrated
 * together with Eq. N-particle by the shoot's RK4 (params->steps steps on
 * [0, params->t1]), so x1 = phi_t1(x0) -- the deformation the momenta define, of
 * a grid or of any point set.  Arrays and rules as ep_velocity; x1 may alias x0.
 * The particles' own endpoint is ep_shoot's.  Memory: the particle state of
 * every RK4 stage is recorded, (4 steps + 1) x n x (16 B mixed 2-D, 32 B mixed
 * 3-D, 16 dim B FP64). */
ep_status ep_flow(const ep_params* params, int64_t n, const double* q0, const double* p0, int64_t m,
                  const double* x0, double* x1, void* stream);

/* Free the cached device workspaces of every stream (synchronises the device). */
ep_status ep_release_workspace(void);

/* Message describing the last error on the calling host thread ("" if none). */
const char* ep_last_error(void);

/* Number of CUDA kernels this library has launched in this process (all
 * devices and streams); a monotone counter for instrumentation. */
int64_t ep_launch_count(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int ep_version(void);

/* Launch timing of the persistent all-pairs shoot (the fused RK4 integration of
 * Sec. 4; one cooperative launch per ep_shoot and per feedback iterate of
 * ep_match) and of the persistent batched launch of ep_match_batched.  With timing
 * on, CUDA events are recorded on the caller's stream around that launch:
 * ep_last_launch_ms() returns the duration of the last timed launch in
 * milliseconds (-1 if none) and ep_last_launch_kernel() the name of its kernel and
 * launch shape ("" if none; for the batched launch the autotuned cluster size,
 * team threshold and lanes per particle).  Off by default; process-wide. */
void ep_set_launch_timing(int on);
double ep_last_launch_ms(void);
const char* ep_last_launch_kernel(void);

#ifdef __cplusplus
}
#endif

#endif /* EP_H */
