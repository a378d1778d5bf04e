// ep_batched.cu -- many independent matchings (Algorithm 1 of the paper, gain
// M = h I on the momenta) in one persistent launch.
//
// Work distribution.  Problems are ordered by decreasing cost (n^2, longest
// processing time first) and handed out through two global counters.  The
// launch is a grid of thread-block clusters of C CTAs, sized to what can
// be resident at once, so no CTA ever waits for one that is not running:
//   - "team" problems (n >= team_min): all CTAs of a cluster solve one problem
//     together.  CTA r owns the particle slice [r n / C, (r+1) n / C); every
//     CTA keeps the whole problem's FP32 stage records in its shared memory, and
//     after each RK4 stage each CTA writes its slice's new records into the
//     shared memory of every CTA of the cluster (distributed shared memory),
//     separated by hardware cluster barriers;
//   - "solo" problems: each CTA solves one problem alone, independently of the
//     others in its cluster.
// Each solve runs the whole feedback loop on the GPU: the shoot (RK4 stages
// with the pair sums over all sources in shared memory, FP32 pair terms,
// per-particle sums over runs of kFold sources added in FP64 when there are several), the FP64 max-norm
// residual, the FP64 momentum update, and finally H(X, p0) (Eq. H).
//
// Launch shape.  The cluster size, the team threshold team_min and the most lanes
// sharing one particle's source loop are chosen per batch by an autotuner that
// times a short trial of the batch itself with each valid shape (batched_tune) and
// caches the fastest for the batch's size signature.
//
// Scaled coordinates as in the all-pairs path: q' = s (q - c0), c0 the centre of
// the bounding box of X, s and the momentum factor dp_scale from the kernel.
#include <cooperative_groups.h>
#include <math.h>

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "ep_allpairs.cuh"
#include "ep_features.cuh"

namespace cg = cooperative_groups;

namespace ep {

namespace {

constexpr int kCluster = 4;          // default cluster size (the autotuner may pick another)
constexpr int kThreads = 1024;
constexpr int kMaxN = 8192;          // particles per problem (shared-memory records)
constexpr int kMaxPerThread = 2;     // particles i per thread and CTA slice
constexpr int kFold = 512;           // FP32 partial sums folded into FP64 every kFold sources

struct BProb {
    long long off;   // first row in X, Y, p0
    int n;
    int kernel;
    int steps;
    int maxit;
    double sigma;
    double t1;
    double h;
    double eps;
    double s;        // coordinate scale
    double dp_scale;
    double* hist;    // optional device array (maxit + 1): residual of every shoot
    const double* ginv;  // G(X)^-1 (n x n, row-major, FP64): velocity update (solo problems); null: momentum rule
};

struct BOut {
    int iters;
    int status;      // ep_status of this problem
    double resid;
    double H;
    double h;
};

struct BArgs {
    const BProb* probs;
    BOut* outs;
    const int* order;   // team problems first, each group by decreasing cost
    int nteam;
    int nprob;
    int* ctr;           // [0] team counter, [1] solo counter
    const double* X;
    const double* Y;
    double* p0;
    double* xs;         // FP64 step state, 4 doubles per particle: (qx, qy, px, py)
    float* acc;         // FP32 RK4 accumulator, 4 floats per particle
    int lmax;           // most lanes that share one particle's source loop (a power of two <= 32)
};

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// G and the momentum weight w of one pair at scaled squared distance r2.
template <int KER>
__device__ __forceinline__ void kfun(float r2, float& G, float& w)
{
    if constexpr (KER == EP_GAUSS) {
        G = ex2_approx(-r2);
        w = G;
    } else if constexpr (KER == EP_TENT) {
        const float rs = rsqrt_approx(fmaxf(r2, 1e-30f));
        const bool in = r2 < 1.0f;
        G = in ? fmaf(-r2, rs, 1.0f) : 0.0f;
        w = in ? rs : 0.0f;
    } else {
        const float rs = rsqrt_approx(fmaxf(r2, 1e-30f));
        G = ex2_approx(-r2 * rs);
        w = G * rs;
    }
}

// Stage records in pairs: sources 2p and 2p+1 share the float4 slots 2p (positions
// x_2p, x_2p+1, y_2p, y_2p+1) and 2p+1 (momenta px_2p, px_2p+1, py_2p, py_2p+1), so
// one shared-memory load gives the packed f32x2 operands of two sources.  An odd n
// has a padding source at index n, far away and without momentum: its terms are
// exactly zero for every kernel.
constexpr float kPadCoord = 1.0e18f;

__device__ __forceinline__ int rec_pairs(int n) { return (n + 1) >> 1; }

__device__ __forceinline__ void rec_put_local(float4* rec, int i, float4 v)
{
    float* a = reinterpret_cast<float*>(rec + 2 * (i >> 1));
    const int h = i & 1;
    a[h] = v.x;
    a[2 + h] = v.y;
    a[4 + h] = v.z;
    a[6 + h] = v.w;
}

__device__ __forceinline__ float4 rec_get(const float4* rec, int i)
{
    const float* a = reinterpret_cast<const float*>(rec + 2 * (i >> 1));
    const int h = i & 1;
    return make_float4(a[h], a[2 + h], a[4 + h], a[6 + h]);
}

// The padding source of an odd n (every CTA that loads the records writes it).
__device__ __forceinline__ void rec_pad(float4* rec, int n)
{
    if ((n & 1) && threadIdx.x == 0) rec_put_local(rec, n, make_float4(kPadCoord, kPadCoord, 0.0f, 0.0f));
}

// The pair terms of Eq. N-particle for two sources at once (the halves of the record
// pair A = positions, B = momenta) added to the packed FP32 sums s = (dq_x, dq_y,
// -m_x, -m_y) of one particle, given as broadcast pairs (-x_i, -y_i, px_i, py_i).  The
// differences are taken as q_j - q_i (exactly the negated q_i - q_j), so the momentum
// sums come out negated; the halves are added when the sums are folded.
template <int KER>
__device__ __forceinline__ void pair_term2(const float2 nx, const float2 ny, const float2 ipx, const float2 ipy,
                                           const float4& A, const float4& B, float2 (&s)[4])
{
    const float2 dx = __fadd2_rn(make_float2(A.x, A.y), nx);
    const float2 dy = __fadd2_rn(make_float2(A.z, A.w), ny);
    const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
    float2 G, w;
    kfun<KER>(r2.x, G.x, w.x);
    kfun<KER>(r2.y, G.y, w.y);
    const float2 px = make_float2(B.x, B.y), py = make_float2(B.z, B.w);
    s[0] = __ffma2_rn(G, px, s[0]);
    s[1] = __ffma2_rn(G, py, s[1]);
    const float2 c = __fmul2_rn(w, __ffma2_rn(ipx, px, __fmul2_rn(ipy, py)));
    s[2] = __ffma2_rn(c, dx, s[2]);
    s[3] = __ffma2_rn(c, dy, s[3]);
}

// Broadcast operand pairs of particle record r.
struct PairOps {
    float2 nx, ny, px, py;
};
__device__ __forceinline__ PairOps pair_ops(const float4& r)
{
    return PairOps{make_float2(-r.x, -r.x), make_float2(-r.y, -r.y), make_float2(r.z, r.z), make_float2(r.w, r.w)};
}

// Team context: the CTAs that solve one problem together.
struct Team {
    int rank, size;
    bool cluster;
};

__device__ __forceinline__ void team_sync(const Team& t)
{
    if (t.cluster) cg::this_cluster().sync();
    else __syncthreads();
}

// Sum (or max) of one double per CTA over the team; every thread gets the result.
__device__ double team_reduce(const Team& t, double v, bool take_max, double* s_red, double* s_slot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_xor_sync(0xffffffffu, v, o);
        v = take_max ? fmax(v, u) : v + u;
    }
    if (lane == 0) s_red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = take_max ? -INFINITY : 0.0;
        for (int k = 0; k < kThreads / 32; ++k) a = take_max ? fmax(a, s_red[k]) : a + s_red[k];
        *s_slot = a;
    }
    team_sync(t);
    double r = take_max ? -INFINITY : 0.0;
    if (t.cluster) {
        cg::cluster_group cl = cg::this_cluster();
        for (int k = 0; k < t.size; ++k) {
            const double u = *cl.map_shared_rank(s_slot, k);
            r = take_max ? fmax(r, u) : r + u;
        }
    } else {
        r = *s_slot;
    }
    team_sync(t);
    return r;
}

// Particle of slot r of this thread: L lanes (a power of two dividing 32) share one
// particle when the slice is small, each summing every L-th source.
__device__ __forceinline__ int slot_particle(int lo, int L, int r)
{
    return lo + (int)threadIdx.x / L + r * (kThreads / L);
}

// Pair sums over all n sources in shared memory for the thread's particles
// (slot r: particle slot_particle(lo, L, r) if < hi); k = (dq, dp) per particle,
// complete in every lane of the particle's lane group.  The sources are taken in
// record pairs (packed f32x2 arithmetic, the two halves summed apart), each
// particle's pairs in increasing order: FP32 partial sums per run of kFold sources,
// added in FP64 when there are several (FP64 costs ~60 FP32 issue slots per warp
// here).  A thread that holds two particles (L = 1 and a slice of more than kThreads)
// sums them one after the other: two passes over the records keep fewer registers
// live than one pass holding both (the kernel has 64 per thread), and measured 17 %
// faster on the 512-problem batch.
template <int KER>
__device__ void pair_sums_k(const float4* rec, int n, int lo, int hi, int L, float dp_scale,
                            float (&kq)[kMaxPerThread][2], float (&kp)[kMaxPerThread][2])
{
    const int sub = (int)threadIdx.x % L;
    const int np = rec_pairs(n);
    constexpr int kFoldPairs = kFold / 2;
    const bool multi = np > kFoldPairs;
#pragma unroll
    for (int r = 0; r < kMaxPerThread; ++r) kq[r][0] = kq[r][1] = kp[r][0] = kp[r][1] = 0.f;
    if (L == 1 && hi - lo > kThreads) {
#pragma unroll 1
        for (int r = 0; r < kMaxPerThread; ++r) {
            const int i = slot_particle(lo, 1, r);
            if (i >= hi) break;
            const PairOps o = pair_ops(rec_get(rec, i));
            float2 s2[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) s2[c] = make_float2(0.f, 0.f);
            double acc[4] = {0, 0, 0, 0};
            for (int q0 = 0; q0 < np; q0 += kFoldPairs) {
                const int q1 = min(np, q0 + kFoldPairs);
#pragma unroll 4
                for (int q = q0; q < q1; ++q) pair_term2<KER>(o.nx, o.ny, o.px, o.py, rec[2 * q], rec[2 * q + 1], s2);
                if (multi) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        acc[c] += (double)s2[c].x;
                        acc[c] += (double)s2[c].y;
                        s2[c] = make_float2(0.f, 0.f);
                    }
                }
            }
            float f[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) f[c] = multi ? (float)acc[c] : s2[c].x + s2[c].y;
            kq[r][0] = f[0]; kq[r][1] = f[1]; kp[r][0] = -dp_scale * f[2]; kp[r][1] = -dp_scale * f[3];
        }
        return;
    }
    // one particle per lane group (slot 0); lane sub takes every L-th record pair
    const int i = slot_particle(lo, L, 0);
    float sm[4] = {0.f, 0.f, 0.f, 0.f};
    if (i < hi) {
        const PairOps o = pair_ops(rec_get(rec, i));
        float2 s2[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) s2[c] = make_float2(0.f, 0.f);
        double acc[4] = {0, 0, 0, 0};
        for (int q0 = 0; q0 < np; q0 += kFoldPairs) {
            const int q1 = min(np, q0 + kFoldPairs);
#pragma unroll 4
            for (int q = q0 + sub; q < q1; q += L) pair_term2<KER>(o.nx, o.ny, o.px, o.py, rec[2 * q], rec[2 * q + 1], s2);
            if (multi) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    acc[c] += (double)s2[c].x;
                    acc[c] += (double)s2[c].y;
                    s2[c] = make_float2(0.f, 0.f);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) sm[c] = multi ? (float)acc[c] : s2[c].x + s2[c].y;
    }
    // combine the lane group in FP32 (whole groups are active or inactive together)
    for (int o = L >> 1; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 4; ++c) sm[c] += __shfl_xor_sync(0xffffffffu, sm[c], o);
    kq[0][0] = sm[0];
    kq[0][1] = sm[1];
    kp[0][0] = -dp_scale * sm[2];
    kp[0][1] = -dp_scale * sm[3];
}

__device__ __forceinline__ void pair_sums(const float4* rec, int n, int lo, int hi, int L, int ker, float dp_scale,
                                          float (&kq)[kMaxPerThread][2], float (&kp)[kMaxPerThread][2])
{
    if (ker == EP_GAUSS) pair_sums_k<EP_GAUSS>(rec, n, lo, hi, L, dp_scale, kq, kp);
    else if (ker == EP_TENT) pair_sums_k<EP_TENT>(rec, n, lo, hi, L, dp_scale, kq, kp);
    else pair_sums_k<EP_EXPCONE>(rec, n, lo, hi, L, dp_scale, kq, kp);
}

// Write one record into the shared memory of every CTA of the team.
__device__ __forceinline__ void put_record(const Team& t, float4* rec, int i, float4 v)
{
    if (t.cluster) {
        cg::cluster_group cl = cg::this_cluster();
        for (int k = 0; k < t.size; ++k) rec_put_local(cl.map_shared_rank(rec, k), i, v);
    } else {
        rec_put_local(rec, i, v);
    }
}

// One complete matching of problem b by the team.
__device__ void solve(const BArgs& a, int b, const Team& t, float4* rec, double* s_red, double* s_slot)
{
    const BProb P = a.probs[b];
    const int n = P.n;
    const int lo = (int)((long long)t.rank * n / t.size), hi = (int)((long long)(t.rank + 1) * n / t.size);
    const double* X = a.X + 2 * P.off;
    const double* Y = a.Y + 2 * P.off;
    double* p0 = a.p0 + 2 * P.off;
    // a solo problem keeps its step state and RK4 accumulator in shared memory after
    // the records (n <= 2047: 16 + 16 + 32 bytes per particle fit the 128 KB region)
    double* xs = a.xs + 4 * P.off;
    float* acc = a.acc + 4 * P.off;
    if (!t.cluster && n <= kThreads * kMaxPerThread) {
        acc = reinterpret_cast<float*>(rec + 2 * rec_pairs(n));
        xs = reinterpret_cast<double*>(acc + 4 * (size_t)n);
    }
    const float s_f = (float)P.s, dps = (float)P.dp_scale;
    int L = 1;
    while (L < a.lmax && (hi - lo) * 2 * L <= kThreads) L *= 2;
    const bool lead = ((int)threadIdx.x % L) == 0;  // the lane that finishes its particle

    // centre of the bounding box of X (every CTA computes it)
    double c0x, c0y;
    {
        double mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
        for (int i = threadIdx.x; i < n; i += kThreads) {
            mnx = fmin(mnx, X[2 * i]); mny = fmin(mny, X[2 * i + 1]);
            mxx = fmax(mxx, X[2 * i]); mxy = fmax(mxy, X[2 * i + 1]);
        }
        const Team solo{0, 1, false};
        mnx = -team_reduce(solo, -mnx, true, s_red, s_slot);
        mny = -team_reduce(solo, -mny, true, s_red, s_slot);
        mxx = team_reduce(solo, mxx, true, s_red, s_slot);
        mxy = team_reduce(solo, mxy, true, s_red, s_slot);
        c0x = 0.5 * (mnx + mxx);
        c0y = 0.5 * (mny + mxy);
    }
    float kq[kMaxPerThread][2], kp[kMaxPerThread][2];

    // default gain h = 1 / max_i sum_j G_ij (pair sums at unit momenta (1, 0))
    double h = P.h;
    if (!(h > 0.0)) {
        for (int i = threadIdx.x; i < n; i += kThreads)
            rec_put_local(rec, i, make_float4((float)((X[2 * i] - c0x) * P.s), (float)((X[2 * i + 1] - c0y) * P.s),
                                              1.0f, 0.0f));
        rec_pad(rec, n);
        __syncthreads();
        pair_sums(rec, n, lo, hi, L, P.kernel, dps, kq, kp);
        double mx = 0.0;
#pragma unroll
        for (int r = 0; r < kMaxPerThread; ++r)
            if (slot_particle(lo, L, r) < hi) mx = fmax(mx, fabs((double)kq[r][0]));
        mx = team_reduce(t, mx, true, s_red, s_slot);
        h = mx > 0.0 ? 1.0 / mx : 1.0;
    }
    team_sync(t);

    const double dt = P.t1 / P.steps;
    const float dt_f = (float)dt;
    int status = EP_ENOTCONVERGED, k = 0;
    double res = 0.0;
    for (;;) {
        // shoot from (X, p0): every CTA loads all records itself from global memory
        for (int i = threadIdx.x; i < n; i += kThreads)
            rec_put_local(rec, i, make_float4((float)((X[2 * i] - c0x) * P.s), (float)((X[2 * i + 1] - c0y) * P.s),
                                              (float)__ldcg(p0 + 2 * i), (float)__ldcg(p0 + 2 * i + 1)));
        rec_pad(rec, n);
        for (int i = lo + threadIdx.x; i < hi; i += kThreads) {
            xs[4 * i] = X[2 * i];
            xs[4 * i + 1] = X[2 * i + 1];
            xs[4 * i + 2] = p0[2 * i];
            xs[4 * i + 3] = p0[2 * i + 1];
        }
        __syncthreads();
        float4 xr[kMaxPerThread];  // the thread's particles at the start of the step (scaled)
#pragma unroll
        for (int r = 0; r < kMaxPerThread; ++r) {
            const int i = slot_particle(lo, L, r);
            xr[r] = i < hi ? rec_get(rec, i) : make_float4(0, 0, 0, 0);
        }
        for (int step = 0; step < P.steps; ++step) {
            for (int stage = 0; stage < 4; ++stage) {
                pair_sums(rec, n, lo, hi, L, P.kernel, dps, kq, kp);
                team_sync(t);  // every CTA has finished reading the stage records
#pragma unroll
                for (int r = 0; r < kMaxPerThread; ++r) {
                    const int i = slot_particle(lo, L, r);
                    if (i >= hi || !lead || (r > 0 && L > 1)) continue;
                    float* A = acc + 4 * i;
                    float4 y;
                    if (stage < 3) {
                        const float cdt = (stage == 2 ? 1.0f : 0.5f) * dt_f;
                        const float bw = stage == 0 ? 1.0f : 2.0f;
                        y = make_float4(fmaf(cdt * s_f, kq[r][0], xr[r].x), fmaf(cdt * s_f, kq[r][1], xr[r].y),
                                        fmaf(cdt, kp[r][0], xr[r].z), fmaf(cdt, kp[r][1], xr[r].w));
                        if (stage == 0) {
                            A[0] = kq[r][0]; A[1] = kq[r][1]; A[2] = kp[r][0]; A[3] = kp[r][1];
                        } else {
                            A[0] = fmaf(bw, kq[r][0], A[0]); A[1] = fmaf(bw, kq[r][1], A[1]);
                            A[2] = fmaf(bw, kp[r][0], A[2]); A[3] = fmaf(bw, kp[r][1], A[3]);
                        }
                    } else {
                        const float f = dt_f * (1.0f / 6.0f);
                        double* x = xs + 4 * i;
                        const double q0 = x[0] + (double)(f * (A[0] + kq[r][0]));
                        const double q1 = x[1] + (double)(f * (A[1] + kq[r][1]));
                        const double v0 = x[2] + (double)(f * (A[2] + kp[r][0]));
                        const double v1 = x[3] + (double)(f * (A[3] + kp[r][1]));
                        x[0] = q0; x[1] = q1; x[2] = v0; x[3] = v1;
                        y = make_float4((float)((q0 - c0x) * P.s), (float)((q1 - c0y) * P.s), (float)v0, (float)v1);
                        xr[r] = y;
                    }
                    put_record(t, rec, i, y);
                }
                team_sync(t);  // new records visible in every CTA
            }
        }
        // FP64 max-norm residual of Y - Q(1)
        double mx = 0.0, bad = 0.0;
        for (int i = lo + threadIdx.x; i < hi; i += kThreads)
            for (int c = 0; c < 2; ++c) {
                const double r = Y[2 * i + c] - xs[4 * i + c];
                if (!isfinite(r)) bad = 1.0;
                mx = fmax(mx, fabs(r));
            }
        bad = team_reduce(t, bad, true, s_red, s_slot);
        mx = team_reduce(t, mx, true, s_red, s_slot);
        res = bad > 0.0 ? NAN : mx;
        if (P.hist && t.rank == 0 && threadIdx.x == 0) P.hist[k] = res;
        if (bad > 0.0) { status = EP_EDIVERGED; break; }
        if (res < P.eps) { status = EP_OK; break; }
        if (k == P.maxit) { status = EP_ENOTCONVERGED; break; }
        if (P.ginv) {
            // velocity update (Algorithm 1 steps 3-4): u0 = G(X) p0 gains h (Y - Q(1)) and
            // p0 = G(X)^-1 u0, i.e. p0 += h G(X)^-1 (Y - Q(1)); one thread per (row, component),
            // FP64 (a solo problem: this CTA holds every Q(1))
            for (int e = threadIdx.x; e < 2 * n; e += kThreads) {
                const int i = e >> 1, c = e & 1;
                const double* g = P.ginv + (size_t)i * n;
                double sdl = 0.0;
                for (int j = 0; j < n; ++j) sdl = fma(g[j], Y[2 * j + c] - xs[4 * j + c], sdl);
                p0[e] = fma(h, sdl, p0[e]);
            }
        } else {
            // p0 += h (Y - Q(1))   (FP64)
            for (int i = lo + threadIdx.x; i < hi; i += kThreads)
                for (int c = 0; c < 2; ++c) p0[2 * i + c] = fma(h, Y[2 * i + c] - xs[4 * i + c], p0[2 * i + c]);
        }
        ++k;
        team_sync(t);  // p0 of every slice written before the next shoot reads it
    }
    team_sync(t);
    // H(X, p0) = 1/2 sum_i p_i . (sum_j G_ij p_j)
    for (int i = threadIdx.x; i < n; i += kThreads)
        rec_put_local(rec, i, make_float4((float)((X[2 * i] - c0x) * P.s), (float)((X[2 * i + 1] - c0y) * P.s),
                                          (float)__ldcg(p0 + 2 * i), (float)__ldcg(p0 + 2 * i + 1)));
    rec_pad(rec, n);
    __syncthreads();
    pair_sums(rec, n, lo, hi, L, P.kernel, dps, kq, kp);
    double hs = 0.0;
#pragma unroll
    for (int r = 0; r < kMaxPerThread; ++r) {
        const int i = slot_particle(lo, L, r);
        if (i < hi && lead && !(r > 0 && L > 1))
            hs += 0.5 * (__ldcg(p0 + 2 * i) * (double)kq[r][0] + __ldcg(p0 + 2 * i + 1) * (double)kq[r][1]);
    }
    hs = team_reduce(t, hs, false, s_red, s_slot);
    if (t.rank == 0 && threadIdx.x == 0) {
        BOut o;
        o.iters = k;
        o.status = status;
        o.resid = res;
        o.H = hs;
        o.h = h;
        a.outs[b] = o;
    }
    team_sync(t);
}

__global__ void __launch_bounds__(kThreads, 1) k_batched(BArgs a)
{
    extern __shared__ float4 rec[];
    __shared__ double s_red[kThreads / 32];
    __shared__ double s_slot;
    __shared__ int s_item;
    cg::cluster_group cl = cg::this_cluster();
    const Team team{(int)cl.block_rank(), (int)cl.num_blocks(), true};
    // team problems: the whole cluster on one problem
    for (;;) {
        if (team.rank == 0 && threadIdx.x == 0) s_item = atomicAdd(a.ctr, 1);
        cl.sync();
        const int item = *cl.map_shared_rank(&s_item, 0);
        cl.sync();
        if (item >= a.nteam) break;
        solve(a, a.order[item], team, rec, s_red, &s_slot);
    }
    // solo problems: every CTA on its own
    const Team solo{0, 1, false};
    for (;;) {
        if (threadIdx.x == 0) s_item = a.nteam + atomicAdd(a.ctr + 1, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= a.nprob) break;
        solve(a, a.order[item], solo, rec, s_red, &s_slot);
    }
    cl.sync();
}

bool is_dev(const void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

ep_status batched_run(const ep_params* params, int nprob, const int64_t* offsets, const double* X, const double* Y,
                      double* p0, ep_match_info* infos, void* stream, double* const* hist_dev,
                      const double* const* ginv = nullptr);


ep_status batched_entry(const ep_params* params, int nprob, const int64_t* offsets, const double* X,
                        const double* Y, double* p0, ep_match_info* infos, void* stream)
{
    return batched_run(params, nprob, offsets, X, Y, p0, infos, stream, nullptr);
}

// ep_match of one small 2-D mixed-precision problem on one CTA (the batched solver).
ep_status match_small(const ep_params* params, int64_t n, const double* X, const double* Y, double* p0,
                      ep_match_info* info, void* stream, const double* ginv)
{
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t offsets[2] = {0, n};
    double* hdev = nullptr;
    bool hist_host = false;
    if (info->hist) {
        if (is_dev(info->hist)) {
            hdev = info->hist;
        } else {
            hist_host = true;
            EP_TRY_CUDA(cudaMallocAsync(&hdev, sizeof(double) * (info->maxit + 1), st));
        }
    }
    ep_status s = batched_run(params, 1, offsets, X, Y, p0, info, stream, &hdev, ginv ? &ginv : nullptr);
    if (hist_host) {
        EP_TRY_CUDA(cudaMemcpyAsync(info->hist, hdev, sizeof(double) * (info->iters + 1), cudaMemcpyDeviceToHost, st));
        EP_TRY_CUDA(cudaFreeAsync(hdev, st));
        EP_TRY_CUDA(cudaStreamSynchronize(st));
    }
    return s;
}


// ------------------------------------------------------------------ launch shapes and their autotuner
// The free parameters of the batched launch: the cluster size C (the CTAs that solve
// one team problem together, and the grid granularity), the size team_min from which
// a problem is a team problem, and the most lanes lmax that share one particle's
// source loop (a solo slice of m particles gets the largest L <= lmax with
// 2 m L <= kThreads).  A team problem's slice must fit one CTA (n / C <= 2048) and so
// must a solo problem (n < team_min <= 2048).
struct BTune {
    int cluster = kCluster;
    int team_min = 2048;
    int lmax = 32;
    bool operator==(const BTune& o) const
    {
        return cluster == o.cluster && team_min == o.team_min && lmax == o.lmax;
    }
};

bool tune_valid(const BTune& c, const std::vector<BProb>& probs)
{
    for (const BProb& q : probs) {
        if (q.ginv && q.n >= c.team_min) return false;  // the velocity update is solo only
        if (q.n >= c.team_min && (q.n + c.cluster - 1) / c.cluster > kThreads * kMaxPerThread) return false;
    }
    return c.team_min <= kThreads * kMaxPerThread + 1;
}

// Problem order for team_min: team problems, then solo problems, each by decreasing n^2
// (longest processing time first).  Returns the number of team problems.
int batch_order(const std::vector<BProb>& probs, int team_min, std::vector<int>* order)
{
    std::vector<int> team, solo;
    for (int b = 0; b < (int)probs.size(); ++b) (probs[b].n >= team_min ? team : solo).push_back(b);
    auto by_cost = [&](int x, int y) { return probs[x].n > probs[y].n || (probs[x].n == probs[y].n && x < y); };
    std::sort(team.begin(), team.end(), by_cost);
    std::sort(solo.begin(), solo.end(), by_cost);
    *order = team;
    order->insert(order->end(), solo.begin(), solo.end());
    return (int)team.size();
}

// One launch of the persistent kernel with shape c on stream st: the problems (probs)
// and the order are uploaded into dprobs / dorder, then the launch (counter reset +
// kernel) runs as a CUDA graph, captured on a library stream and replayed on st; it
// is rebuilt only when the arguments or the shape change.  Events e0 / e1, when
// given, bracket the graph launch.
ep_status batched_launch(const BTune& c, BArgs a, const std::vector<BProb>& probs, BProb* dprobs, int* dorder,
                         cudaStream_t st, cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr)
{
    static std::mutex mu;
    static std::map<std::pair<int, int>, int> resident;  // (device, cluster size) -> resident clusters
    DeviceInfo di{};
    EP_TRY(device_info(&di));
    std::vector<int> order;
    a.nteam = batch_order(probs, c.team_min, &order);
    a.lmax = c.lmax;
    a.probs = dprobs;
    a.order = dorder;
    const int nprob = (int)probs.size();
    EP_TRY_CUDA(cudaMemcpyAsync(dprobs, probs.data(), sizeof(BProb) * nprob, cudaMemcpyHostToDevice, st));
    EP_TRY_CUDA(cudaMemcpyAsync(dorder, order.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice, st));
    const size_t smem = sizeof(float4) * kMaxN;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attrs[1];
    attrs[0].id = cudaLaunchAttributeClusterDimension;
    attrs[0].val.clusterDim.x = (unsigned)c.cluster;
    attrs[0].val.clusterDim.y = 1;
    attrs[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attrs;
    cfg.numAttrs = 1;
    int nclusters = 0;
    std::lock_guard<std::mutex> lk(mu);
    {
        auto it = resident.find({di.device, c.cluster});
        if (it == resident.end()) {
            EP_TRY_CUDA(cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            if (c.cluster > 8)
                EP_TRY_CUDA(cudaFuncSetAttribute(k_batched, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            cfg.gridDim = dim3((unsigned)(di.sm_count / c.cluster * c.cluster));
            EP_TRY_CUDA(cudaOccupancyMaxActiveClusters(&nclusters, k_batched, &cfg));
            resident[{di.device, c.cluster}] = nclusters;
        } else {
            nclusters = it->second;
        }
    }
    if (nclusters < 1) return set_error("ep_match_batched: no cluster of %d CTAs fits", c.cluster), EP_ECUDA;
    cfg.gridDim = dim3((unsigned)(nclusters * c.cluster));
    struct GraphCache {
        cudaStream_t cap = nullptr;
        cudaGraphExec_t exec = nullptr;
        BArgs args{};
        unsigned grid = 0;
        int cluster = 0;
    };
    static std::map<std::pair<int, cudaStream_t>, GraphCache> graphs;
    GraphCache& gc = graphs[{di.device, st}];
    if (!gc.exec || memcmp(&gc.args, &a, sizeof a) != 0 || gc.grid != cfg.gridDim.x || gc.cluster != c.cluster) {
        if (gc.exec) {
            EP_TRY_CUDA(cudaStreamSynchronize(st));
            cudaGraphExecDestroy(gc.exec);
            gc.exec = nullptr;
        }
        if (!gc.cap) EP_TRY_CUDA(cudaStreamCreateWithFlags(&gc.cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        EP_TRY_CUDA(cudaStreamBeginCapture(gc.cap, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(a.ctr, 0, sizeof(int) * 4, gc.cap);
        cfg.stream = gc.cap;
        cudaLaunchKernelEx(&cfg, k_batched, a);
        EP_TRY_CUDA(cudaStreamEndCapture(gc.cap, &graph));
        cudaError_t e = cudaGraphInstantiate(&gc.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (batched launch)");
        gc.args = a;
        gc.grid = cfg.gridDim.x;
        gc.cluster = c.cluster;
    }
    count_launch();
    if (e0) EP_TRY_CUDA(cudaEventRecord(e0, st));
    EP_TRY_CUDA(cudaGraphLaunch(gc.exec, st));
    if (e1) EP_TRY_CUDA(cudaEventRecord(e1, st));
    return EP_OK;
}

// Key of a tuned shape: the batch's size signature on a device.
struct BTuneKey {
    int dev, nprob, nmax, ntent;
    long long n2;
    bool operator<(const BTuneKey& o) const
    {
        if (dev != o.dev) return dev < o.dev;
        if (nprob != o.nprob) return nprob < o.nprob;
        if (nmax != o.nmax) return nmax < o.nmax;
        if (ntent != o.ntent) return ntent < o.ntent;
        return n2 < o.n2;
    }
};
std::mutex g_btune_mu;
std::map<BTuneKey, BTune> g_btuned;

bool batched_autotune_enabled()
{
    const char* e = getenv("EP_AUTOTUNE");
    return !(e && e[0] == '0');
}

// The autotuner: each valid candidate shape runs a short trial of the same batch (one
// shoot per problem, at most kTuneSteps RK4 steps, momenta copied to scratch so the
// caller's are untouched), timed with CUDA events (best of two after one untimed
// run); the fastest shape is cached for the batch's size signature.
constexpr int kTuneSteps = 4;
ep_status batched_tune(const BArgs& a0, const std::vector<BProb>& probs, BProb* dprobs, int* dorder,
                       double* p_scratch, size_t m, cudaStream_t st, BTune* best)
{
    std::vector<BProb> trial(probs);
    for (BProb& q : trial) {
        q.maxit = 0;
        q.steps = std::min(q.steps, kTuneSteps);
        q.hist = nullptr;
    }
    BArgs a = a0;
    a.p0 = p_scratch;
    std::vector<BTune> cand;
    for (int C : {4, 8, 2})
        for (int tm : {2048, 1024})
            for (int lm : {32, 8}) {
                BTune c;
                c.cluster = C;
                c.team_min = tm;
                c.lmax = lm;
                if (tune_valid(c, probs)) cand.push_back(c);
            }
    cudaEvent_t e0, e1;
    EP_TRY_CUDA(cudaEventCreate(&e0));
    EP_TRY_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    ep_status out = EP_OK;
    for (const BTune& c : cand) {
        float ms = 1e30f;
        for (int rep = 0; rep < 3 && out == EP_OK; ++rep) {
            out = cudaMemcpyAsync(p_scratch, a0.p0, sizeof(double) * m, cudaMemcpyDeviceToDevice, st) == cudaSuccess
                      ? batched_launch(c, a, trial, dprobs, dorder, st, e0, e1)
                      : EP_ECUDA;
            if (out != EP_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) { out = EP_ECUDA; break; }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms = std::min(ms, t);
        }
        if (out != EP_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            *best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return out;
}

// The shape a batch runs with (tuned once per size signature; defaults with
// EP_AUTOTUNE=0 or for a single problem); the last choice is readable for reporting.
BTune g_last_btune;

ep_status batched_run(const ep_params* params, int nprob, const int64_t* offsets, const double* X, const double* Y,
                      double* p0, ep_match_info* infos, void* stream, double* const* hist_dev,
                      const double* const* ginv)
{
    if (nprob < 0) return set_error("ep_match_batched: nprob < 0"), EP_EINVAL;
    if (nprob == 0) return EP_OK;
    if (!params || !offsets || !infos) return set_error("ep_match_batched: NULL argument"), EP_EINVAL;
    if (offsets[0] != 0) return set_error("ep_match_batched: offsets[0] must be 0"), EP_EINVAL;
    std::vector<BProb> probs((size_t)nprob);
    for (int b = 0; b < nprob; ++b) {
        const ep_params& P = params[b];
        EP_TRY(check_params(&P));
        if (P.inexact != 0.0) return set_error("ep_match_batched solves the exact system"), EP_EINVAL;
        if (P.dim != 2) return set_error("ep_match_batched: problem %d: dim must be 2", b), EP_EINVAL;
        if (P.precision != EP_MIXED)
            return set_error("ep_match_batched: problem %d: the batched path runs in mixed precision", b), EP_EINVAL;
        const int64_t nb = offsets[b + 1] - offsets[b];
        if (nb < 0 || nb > kMaxN)
            return set_error("ep_match_batched: problem %d has n = %lld (allowed 0..%d)", b, (long long)nb, kMaxN),
                   EP_EINVAL;
        const ep_match_info& I = infos[b];
        if (I.maxit < 0 || !(I.eps >= 0.0)) return set_error("ep_match_batched: problem %d: bad maxit/eps", b), EP_EINVAL;
        const bool vel = ginv && ginv[b];
        if (I.rule != (vel ? EP_RULE_VELOCITY : EP_RULE_MOMENTUM))
            return set_error("ep_match_batched: problem %d: only the momentum update rule is batched", b), EP_EINVAL;
        if (vel && nb > kThreads * kMaxPerThread) return set_error("ep_match: internal size limit (velocity update)"), EP_EINVAL;
        const KernelScale ks = kernel_scale(P.kernel, P.sigma);
        BProb& q = probs[b];
        q.off = offsets[b];
        q.n = (int)nb;
        q.kernel = P.kernel;
        q.steps = P.steps;
        q.maxit = I.maxit;
        q.sigma = P.sigma;
        q.t1 = P.t1;
        q.h = I.h;
        q.eps = I.eps;
        q.s = ks.s;
        q.dp_scale = ks.dp_scale;
        q.hist = hist_dev ? hist_dev[b] : nullptr;
        q.ginv = vel ? ginv[b] : nullptr;
    }
    const int64_t ntot = offsets[nprob];
    cudaStream_t st = (cudaStream_t)stream;
    const size_t m = 2 * (size_t)ntot;
    Sizer z;
    z.add(sizeof(BProb) * nprob);
    z.add(sizeof(BOut) * nprob);
    z.add(sizeof(int) * nprob);
    z.add(sizeof(int) * 4);
    z.add(sizeof(double) * 4 * (size_t)ntot);
    z.add(sizeof(float) * 4 * (size_t)ntot);
    z.add(sizeof(double) * m * 4);
    Arena* ar = nullptr;
    EP_TRY(arena_acquire(st, z.total, &ar));
    BProb* dprobs = (BProb*)ar->carve(sizeof(BProb) * nprob);
    BOut* douts = (BOut*)ar->carve(sizeof(BOut) * nprob);
    int* dorder = (int*)ar->carve(sizeof(int) * nprob);
    int* dctr = (int*)ar->carve(sizeof(int) * 4);
    double* xs = (double*)ar->carve(sizeof(double) * 4 * (size_t)ntot + 8);
    float* acc = (float*)ar->carve(sizeof(float) * 4 * (size_t)ntot + 8);
    const double* dX = X;
    const double* dY = Y;
    double* dp0 = p0;
    const bool xh = !is_dev(X), yh = !is_dev(Y), ph = !is_dev(p0);
    if (xh) {
        double* t = (double*)ar->carve(sizeof(double) * m + 8);
        EP_TRY_CUDA(cudaMemcpyAsync(t, X, sizeof(double) * m, cudaMemcpyHostToDevice, st));
        dX = t;
    }
    if (yh) {
        double* t = (double*)ar->carve(sizeof(double) * m + 8);
        EP_TRY_CUDA(cudaMemcpyAsync(t, Y, sizeof(double) * m, cudaMemcpyHostToDevice, st));
        dY = t;
    }
    if (ph) {
        dp0 = (double*)ar->carve(sizeof(double) * m + 8);
        if (!dp0) return set_error("ep_match_batched: workspace too small"), EP_ENOMEM;
        EP_TRY_CUDA(cudaMemcpyAsync(dp0, p0, sizeof(double) * m, cudaMemcpyHostToDevice, st));
    }
    BArgs a{};
    a.outs = douts;
    a.nprob = nprob;
    a.ctr = dctr;
    a.X = dX;
    a.Y = dY;
    a.p0 = dp0;
    a.xs = xs;
    a.acc = acc;

    // the launch shape: tuned once per batch size signature (several problems), else defaults
    BTune shape;
    if (nprob > 1 && batched_autotune_enabled()) {
        DeviceInfo di{};
        EP_TRY(device_info(&di));
        BTuneKey key{di.device, nprob, 0, 0, 0};
        for (const BProb& q : probs) {
            key.nmax = std::max(key.nmax, q.n);
            key.ntent += q.kernel == EP_TENT ? 1 : 0;
            key.n2 += (long long)q.n * q.n;
        }
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(g_btune_mu);
            auto it = g_btuned.find(key);
            if (it != g_btuned.end()) shape = it->second, have = true;
        }
        if (!have) {
            double* scratch = (double*)ar->carve(sizeof(double) * m + 8);
            if (!scratch) return set_error("ep_match_batched: workspace too small"), EP_ENOMEM;
            EP_TRY(batched_tune(a, probs, dprobs, dorder, scratch, m, st, &shape));
            std::lock_guard<std::mutex> lk(g_btune_mu);
            g_btuned[key] = shape;
        }
    }
    if (!tune_valid(shape, probs)) return set_error("ep_match_batched: no valid launch shape"), EP_EINVAL;
    g_last_btune = shape;
    // with launch timing on (ep_set_launch_timing), CUDA events around the graph launch;
    // the reported name carries the launch shape
    cudaEvent_t te0 = nullptr, te1 = nullptr;
    if (launch_timing_enabled() && nprob > 1) {
        if (cudaEventCreate(&te0) != cudaSuccess || cudaEventCreate(&te1) != cudaSuccess) {
            if (te0) cudaEventDestroy(te0);
            te0 = te1 = nullptr;
        }
    }
    const ep_status ls = batched_launch(shape, a, probs, dprobs, dorder, st, te0, te1);
    if (te0 && ls == EP_OK && cudaEventSynchronize(te1) == cudaSuccess) {
        char name[96];
        snprintf(name, sizeof(name), "k_batched (cluster %d, team_min %d, lmax %d)", shape.cluster, shape.team_min,
                 shape.lmax);
        record_launch_time(te0, te1, name);
    }
    if (te0) {
        cudaEventDestroy(te0);
        cudaEventDestroy(te1);
    }
    EP_TRY(ls);

    std::vector<BOut> outs((size_t)nprob);
    EP_TRY_CUDA(cudaMemcpyAsync(outs.data(), douts, sizeof(BOut) * nprob, cudaMemcpyDeviceToHost, st));
    if (ph) EP_TRY_CUDA(cudaMemcpyAsync(p0, dp0, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    EP_TRY_CUDA(cudaGetLastError());
    ep_status first = EP_OK;
    for (int b = 0; b < nprob; ++b) {
        infos[b].status = outs[b].status;
        infos[b].iters = outs[b].iters;
        infos[b].resid_inf = outs[b].resid;
        infos[b].H = outs[b].H;
        infos[b].h = outs[b].h;
        if (first == EP_OK && outs[b].status != EP_OK) first = (ep_status)outs[b].status;
    }
    if (first != EP_OK) set_error("ep_match_batched: not every problem converged");
    return first;
}


}  // namespace ep
