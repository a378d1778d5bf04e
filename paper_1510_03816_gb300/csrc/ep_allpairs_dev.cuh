// ep_allpairs_dev.cuh -- device pieces shared by the all-pairs kernels: the
// stage arguments, pair-kernel functions, the RK4 stage epilogue (Sec. 4,
// Note 1 item 5) and the bounded grid-wide barrier of the persistent shoots.
#pragma once

#include "ep_allpairs.cuh"

namespace ep {
namespace {

struct StageArgs {
    long long U;
    int n;
    int G;
    int mode;
    int stage;
    float dt_f;
    double dt;
    float s_f;
    double s;
    double dp_scale;
    float dp_scale_f;
    double s2;          // sigma_n^2 of the inexact system (Sec. 6), 0 for the exact one
    float s2_f;
    const double* c0;
    const float4* S_in;
    float4* S_out;
    const float4* Sx;   // step-start stage copy (mixed)
    float4* Sx_w;       // written at stage 3 (mixed)
    float4* rec_out;    // if set, a second copy of the stage output (mixed; a recorded shoot)
    const double* D_in; // fp64 stage copies
    double* D_out;
    double* x;
    float* acc;
    double* dacc;
    double* K;
    int* counters;
    double* out_q;
    double* out_p;
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

// Kernel value G and momentum weight w of one pair from the scaled squared
// distance r2 = |d'|^2 (see ep_common.cuh for the scalings).
template <int KER>
__device__ __forceinline__ void kfun_f32(float r2, float& G, float& w)
{
    if constexpr (KER == EP_GAUSS) {
        G = ex2_approx(-r2);
        w = G;
    } else if constexpr (KER == EP_TENT) {
        // r2 = 0 (self or coincident pair): rs stays finite and d' = 0, so the
        // momentum term vanishes (phi = 0 at r = 0) while G(0) = 1.
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

// FP64 kernel value and phi = G'(r)/r (unscaled).  The reciprocals of sigma are
// loop invariants and 1/r comes from rsqrt, so a pair needs no division (FP64
// runs at 1/64 of the FP32 rate here); the tent keeps the correctly rounded
// r = sqrt(r2) for its support test r < sigma.
template <int KER>
__device__ __forceinline__ void kfun_f64(double r2, double sigma, double& G, double& phi)
{
    const double is = 1.0 / sigma;
    if constexpr (KER == EP_GAUSS) {
        G = exp(-0.5 * (r2 * (is * is)));
        phi = -G * (is * is);
    } else if constexpr (KER == EP_TENT) {
        const double r = sqrt(r2);
        const bool in = r < sigma;
        G = in ? 1.0 - r * is : 0.0;
        phi = (in && r2 > 0.0) ? -is * rsqrt(r2) : 0.0;
    } else {
        const double r = sqrt(r2);
        G = exp(-r * is);
        phi = r2 > 0.0 ? -G * is * rsqrt(r2) : 0.0;
    }
}

__device__ __forceinline__ int cta_of_unit(long long u, long long U, int G)
{
    return (int)(((u + 1) * (long long)G - 1) / U);
}

__device__ __forceinline__ int tile_contributors(int b, const StageArgs& a)
{
    const long long ub = (long long)b * a.n;
    return cta_of_unit(ub + a.n - 1, a.U, a.G) - cta_of_unit(ub, a.U, a.G) + 1;
}

// ------------------------------------------------------------------ mixed
// Epilogue of one particle i in tile order; k = (dq, dp) of the stage input.
// kk = the particle's pair sums: 2-D (dq_x, dq_y, M_xx, M_xy, M_yx, M_yy) with
// M_cd = sum_j G_ij (q'_i - q'_j)_c p_j,d; 3-D (dq, sum_j w_ij (p_i.p_j) d'_ij).
template <int DIM>
__device__ void epilogue_mixed_k(const StageArgs& a, int i, const double* kk)
{
    // momentum of the stage input (FP32 copy) for the 2-D contraction
    float pin[3];
    if constexpr (DIM == 2) {
        const float4 v = __ldcg(a.S_in + i);
        pin[0] = v.z;
        pin[1] = v.w;
    } else {
        const float4 v = __ldcg(a.S_in + 2 * (size_t)i + 1);
        pin[0] = v.x;
        pin[1] = v.y;
        pin[2] = v.z;
    }
    if (a.mode == MODE_RHS) {
        double kq[DIM], kp[DIM];
        if constexpr (DIM == 2) {
            kq[0] = kk[0] + a.s2 * (double)pin[0];
            kq[1] = kk[1] + a.s2 * (double)pin[1];
            kp[0] = a.dp_scale * (kk[2] * (double)pin[0] + kk[3] * (double)pin[1]);
            kp[1] = a.dp_scale * (kk[4] * (double)pin[0] + kk[5] * (double)pin[1]);
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                kq[c] = kk[c] + a.s2 * (double)pin[c];
                kp[c] = a.dp_scale * kk[3 + c];
            }
        }
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            a.out_q[(size_t)i * DIM + c] = kq[c];
            a.out_p[(size_t)i * DIM + c] = kp[c];
        }
        return;
    }
    float kq[DIM], kp[DIM];
    if constexpr (DIM == 2) {
        kq[0] = fmaf(a.s2_f, pin[0], (float)kk[0]);
        kq[1] = fmaf(a.s2_f, pin[1], (float)kk[1]);
        kp[0] = a.dp_scale_f * fmaf((float)kk[2], pin[0], (float)kk[3] * pin[1]);
        kp[1] = a.dp_scale_f * fmaf((float)kk[4], pin[0], (float)kk[5] * pin[1]);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            kq[c] = fmaf(a.s2_f, pin[c], (float)kk[c]);
            kp[c] = a.dp_scale_f * (float)kk[3 + c];
        }
    }
    float* A = a.acc + (size_t)i * 2 * DIM;
    if (a.stage < 3) {
        // y_{s+1} = x_n + c_{s+1} dt k_s, c = 1/2, 1/2, 1 (FP32, scaled positions)
        const float cdt = (a.stage == 2 ? 1.0f : 0.5f) * a.dt_f;
        const float bw = a.stage == 0 ? 1.0f : 2.0f;
        float xs[2 * DIM];
        if constexpr (DIM == 2) {
            const float4 v = a.Sx[i];
            xs[0] = v.x; xs[1] = v.y; xs[2] = v.z; xs[3] = v.w;
        } else {
            const float4 v0 = a.Sx[2 * (size_t)i], v1 = a.Sx[2 * (size_t)i + 1];
            xs[0] = v0.x; xs[1] = v0.y; xs[2] = v0.z; xs[3] = v1.x; xs[4] = v1.y; xs[5] = v1.z;
        }
        float y[2 * DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            y[c] = fmaf(cdt * a.s_f, kq[c], xs[c]);
            y[DIM + c] = fmaf(cdt, kp[c], xs[DIM + c]);
            if (a.stage == 0) {
                A[c] = kq[c];
                A[DIM + c] = kp[c];
            } else {
                A[c] = fmaf(bw, kq[c], A[c]);
                A[DIM + c] = fmaf(bw, kp[c], A[DIM + c]);
            }
        }
        if constexpr (DIM == 2) {
            a.S_out[i] = make_float4(y[0], y[1], y[2], y[3]);
            if (a.rec_out) a.rec_out[i] = make_float4(y[0], y[1], y[2], y[3]);
        } else {
            a.S_out[2 * (size_t)i] = make_float4(y[0], y[1], y[2], 0.0f);
            a.S_out[2 * (size_t)i + 1] = make_float4(y[3], y[4], y[5], 0.0f);
            if (a.rec_out) {
                a.rec_out[2 * (size_t)i] = make_float4(y[0], y[1], y[2], 0.0f);
                a.rec_out[2 * (size_t)i + 1] = make_float4(y[3], y[4], y[5], 0.0f);
            }
        }
    } else {
        // x_{n+1} = x_n + dt/6 (k1 + 2 k2 + 2 k3 + k4): the increment in FP32, the state in FP64
        const int n = a.n;
        double* xq = a.x + (size_t)i * DIM;
        double* xp = a.x + (size_t)n * DIM + (size_t)i * DIM;
        float y[2 * DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            const double nq = xq[c] + (double)(a.dt_f * (1.0f / 6.0f) * (A[c] + kq[c]));
            const double np = xp[c] + (double)(a.dt_f * (1.0f / 6.0f) * (A[DIM + c] + kp[c]));
            xq[c] = nq;
            xp[c] = np;
            y[c] = (float)((nq - a.c0[c]) * a.s);
            y[DIM + c] = (float)np;
        }
        if constexpr (DIM == 2) {
            a.Sx_w[i] = make_float4(y[0], y[1], y[2], y[3]);
            if (a.rec_out) a.rec_out[i] = make_float4(y[0], y[1], y[2], y[3]);
        } else {
            a.Sx_w[2 * (size_t)i] = make_float4(y[0], y[1], y[2], 0.0f);
            a.Sx_w[2 * (size_t)i + 1] = make_float4(y[3], y[4], y[5], 0.0f);
            if (a.rec_out) {
                a.rec_out[2 * (size_t)i] = make_float4(y[0], y[1], y[2], 0.0f);
                a.rec_out[2 * (size_t)i + 1] = make_float4(y[3], y[4], y[5], 0.0f);
            }
        }
    }
}

// The same, reading (and clearing) the particle's FP64 accumulator K.
template <int DIM>
__device__ void epilogue_mixed(const StageArgs& a, int i)
{
    double kk[kKWidth];
#pragma unroll
    for (int t = 0; t < kKWidth; ++t) {
        kk[t] = __ldcg(a.K + (size_t)i * kKWidth + t);
        a.K[(size_t)i * kKWidth + t] = 0.0;
    }
    epilogue_mixed_k<DIM>(a, i, kk);
}

// Sum of V <= 8 doubles over a CTA of THREADS threads, complete in every thread on
// return; sm holds (THREADS / 32 + 1) * 8 doubles.  An FP64 warp instruction holds
// its sub-partition's FP64 pipe for the same time whatever the number of active
// lanes, so the sum minimises FP64 instructions: a reduce-scatter butterfly over
// the lanes (each round halves the values a lane holds: 6 adds for 4 values, 9 for
// 8, against 5 per value for a plain butterfly), then one thread per value adds
// the warps' totals.  Fixed order: the same bits on every call and in every CTA.
template <int V, int THREADS>
__device__ __forceinline__ void cta_sum_f64(double (&v)[V], double* sm)
{
    static_assert(V >= 1 && V <= 8, "cta_sum_f64 takes 1 to 8 values");
    constexpr int W = THREADS / 32;
    constexpr int P = V == 1 ? 1 : V == 2 ? 2 : V <= 4 ? 4 : 8;  // padded to a power of two
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double u[P];
#pragma unroll
    for (int k = 0; k < P; ++k) u[k] = k < V ? v[k] : 0.0;
    int first = 0;  // the value index this lane ends up holding
    int cnt = P;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (cnt > 1) {
            const int h = cnt / 2;
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int k = 0; k < P / 2; ++k) {
                if (k < h) {
                    const double send = upper ? u[k] : u[k + h];
                    const double keep = upper ? u[k + h] : u[k];
                    u[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
            }
            if (upper) first += h;
            cnt = h;
        } else {
            u[0] += __shfl_xor_sync(0xffffffffu, u[0], o);
        }
    }
    if ((lane & (32 / P - 1)) == 0 && first < V) sm[warp * P + first] = u[0];
    __syncthreads();
    if (threadIdx.x < V) {
        double t = 0.0;
        for (int w = 0; w < W; ++w) t += sm[w * P + threadIdx.x];
        sm[W * P + threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = sm[W * P + k];
}

// Dense LU factorisation with partial pivoting by one CTA of THREADS threads:
// A (N x N, column-major, A[c N + r]) is overwritten by L (unit lower, below the
// diagonal) and U; piv[k] = the row swapped with row k at step k (the largest
// |pivot| in the column, the first on ties).  Returns false (in every thread) when a
// pivot is zero or no pivot is finite.  scratch: 2 * THREADS / 32 + 2 words of
// shared memory.
template <int THREADS>
__device__ bool cta_lu_factor(int N, double* A, int* piv, double* s_val, int* s_idx)
{
    constexpr int W = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool ok = true;
    for (int k = 0; k < N; ++k) {
        double best = -1.0;
        int bi = N;
        for (int r = k + (int)threadIdx.x; r < N; r += THREADS) {
            const double v = fabs(A[(size_t)k * N + r]);
            if (v > best || (v == best && r < bi)) { best = v; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double bv = s_val[0];
            int bix = s_idx[0];
            for (int w = 1; w < W; ++w)
                if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bix)) { bv = s_val[w]; bix = s_idx[w]; }
            s_idx[W] = bv > 0.0 ? bix : -1;
        }
        __syncthreads();
        const int pr = s_idx[W];
        if (pr < 0) { ok = false; break; }  // uniform: every thread read the same slot
        if (threadIdx.x == 0) piv[k] = pr;
        if (pr != k)
            for (int c = (int)threadIdx.x; c < N; c += THREADS) {
                const double t = A[(size_t)c * N + k];
                A[(size_t)c * N + k] = A[(size_t)c * N + pr];
                A[(size_t)c * N + pr] = t;
            }
        __syncthreads();
        const double d = A[(size_t)k * N + k];
        for (int r = k + 1 + (int)threadIdx.x; r < N; r += THREADS) A[(size_t)k * N + r] /= d;
        __syncthreads();
        const int rows = N - k - 1;
        for (int t = (int)threadIdx.x; t < rows * rows; t += THREADS) {
            const int r = k + 1 + t % rows, c = k + 1 + t / rows;
            A[(size_t)c * N + r] -= A[(size_t)k * N + r] * A[(size_t)c * N + k];
        }
        __syncthreads();
    }
    return ok;
}

// Solve A x = b with the factors of cta_lu_factor (b overwritten by x) by one warp:
// the row swaps, forward substitution with the unit L, back substitution with U,
// each step's dot product split over the lanes and summed by shuffles.
__device__ void warp_lu_solve(int N, const double* A, const int* piv, double* b)
{
    const int lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < N; ++k) {
            const int p = piv[k];
            if (p != k) { const double t = b[k]; b[k] = b[p]; b[p] = t; }
        }
    __syncwarp();
    for (int pass = 0; pass < 2; ++pass) {
        for (int s = 0; s < N; ++s) {
            const int k = pass == 0 ? s : N - 1 - s;
            double sum = 0.0;
            if (pass == 0)
                for (int c = lane; c < k; c += 32) sum += A[(size_t)c * N + k] * b[c];
            else
                for (int c = k + 1 + lane; c < N; c += 32) sum += A[(size_t)c * N + k] * b[c];
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == 0) b[k] = pass == 0 ? b[k] - sum : (b[k] - sum) / A[(size_t)k * N + k];
            __syncwarp();
        }
    }
}

// Grid-wide barrier of a cooperative launch (all CTAs resident).  The counter
// only grows: barrier number e completes when it reaches e * gridDim.x.  The
// wait is bounded; on giving up it raises the shared error flag, and every CTA
// that sees the flag returns false so the kernel ends instead of hanging.
constexpr long long kSpinLimit = 1LL << 22;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ bool grid_barrier(unsigned* bar, int* err, unsigned epoch)
{
    // bar[0..7]: arrival counters, CTA c arrives on bar[c % 8]; barrier e completes
    // when bar[k] reaches e * (CTAs on k).  (The eight words share one L2 sector:
    // counters on separate L2 lines, a release-ordered arrival without the fence, and
    // per-CTA completion flags polled by each warp for its own sources all measured no
    // faster in the persistent 2-D Gaussian shoot on GB300.)
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const unsigned G = gridDim.x;
        if (lane == 0) {
            __threadfence();
            atomicAdd(bar + (blockIdx.x & 7), 1u);
        }
        const unsigned mine = lane < 8 ? (G / 8 + ((unsigned)lane < (G & 7) ? 1u : 0u)) : 0u;
        const unsigned target = epoch * mine;
        int ok = 1;
        long long spins = 0;
        for (;;) {
            const unsigned v = lane < 8 ? ld_acquire_u32(bar + lane) : 0u;
            if (__all_sync(0xffffffffu, v >= target)) break;
            if ((++spins & 63) == 0 && *(volatile int*)err) { ok = 0; break; }
            if (spins > kSpinLimit) {
                if (lane == 0) atomicExch(err, 1);
                ok = 0;
                break;
            }
        }
        if (lane == 0) s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}


// Host: the stage arguments common to every launch of one problem.
StageArgs base_args(const ep_params& P, const AllPairsBufs& b, const APConfig& cfg)
{
    StageArgs a{};
    const int ntiles = (b.n + kTileI - 1) / kTileI;
    a.n = b.n;
    a.U = (long long)ntiles * b.n;
    a.G = (int)std::min<long long>(cfg.ctas, a.U);
    const KernelScale ks = kernel_scale(P.kernel, P.sigma);
    a.s = ks.s;
    a.s_f = (float)ks.s;
    a.dp_scale = ks.dp_scale;
    a.dp_scale_f = (float)ks.dp_scale;
    a.s2 = P.inexact;
    a.s2_f = (float)P.inexact;
    a.c0 = b.c0;
    a.x = b.x;
    a.acc = b.acc;
    a.dacc = b.dacc;
    a.K = b.K;
    a.counters = b.counters;
    return a;
}

}  // namespace
}  // namespace ep
