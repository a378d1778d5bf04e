// ep_allpairs.cu -- all-pairs right-hand side of the N-particle system
// (Sec. 3.1, Eq. N-particle) with the classical RK4 stage (Sec. 4, Note 1
// item 5) fused into the kernel.
//
// Work decomposition (stream-K over the pair matrix).  Particles i are grouped
// in tiles of 64 (32 lanes x 2 registers).  The pair matrix is the sequence of
// U = ntiles * n units (tile b, source j), cut into G equal contiguous ranges,
// one per CTA, G = (SM count) x (resident CTAs per SM).  A CTA's range covers
// one or a few tile segments [j0, j1).  For each segment the CTA stages the
// FP32 source data of [j0, j1) in shared memory, its warps split the j range,
// every lane accumulates its two particles' sums in registers (FP32), the
// warps' partials are summed in shared memory, and the CTA adds its partial
// into the FP64 accumulator K of the tile's particles (red.global.add.f64:
// the per-particle sums are accumulated in FP64).  The last CTA to arrive at
// a tile (per-tile counter) applies the RK4 stage to the tile's particles:
// it reads k = K, forms the next stage input, resets K and the counter.
//
// Precision modes: EP_MIXED evaluates pair terms in FP32 on scaled
// coordinates (see ep_common.cuh), keeps the step state x_n in FP64 and the
// RK4 stage combination in FP32; EP_FP64 does every operation in FP64.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "ep_allpairs.cuh"

namespace ep {

namespace {

constexpr int kChunk = 2048;  // sources staged per shared-memory fill (mixed)
constexpr int kChunk64 = 1024;

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
    const double* c0;
    const float4* S_in;
    float4* S_out;
    const float4* Sx;   // step-start stage copy (mixed)
    float4* Sx_w;       // written at stage 3 (mixed)
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

// Exact FP64 kernel value and phi = G'(r)/r (unscaled).
template <int KER>
__device__ __forceinline__ void kfun_f64(double r2, double sigma, double& G, double& phi)
{
    if constexpr (KER == EP_GAUSS) {
        G = exp(-r2 / (2.0 * sigma * sigma));
        phi = -G / (sigma * sigma);
    } else if constexpr (KER == EP_TENT) {
        const double r = sqrt(r2);
        const bool in = r < sigma;
        G = in ? 1.0 - r / sigma : 0.0;
        phi = (in && r > 0.0) ? -1.0 / (sigma * r) : 0.0;
    } else {
        const double r = sqrt(r2);
        G = exp(-r / sigma);
        phi = r > 0.0 ? -G / (sigma * r) : 0.0;
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
template <int DIM>
__device__ void epilogue_mixed(const StageArgs& a, int i)
{
    constexpr int V = DIM == 2 ? 1 : 2;
    double kk[kKWidth];
#pragma unroll
    for (int t = 0; t < kKWidth; ++t) {
        kk[t] = __ldcg(a.K + (size_t)i * kKWidth + t);
        a.K[(size_t)i * kKWidth + t] = 0.0;
    }
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
            kq[0] = kk[0];
            kq[1] = kk[1];
            kp[0] = a.dp_scale * (kk[2] * (double)pin[0] + kk[3] * (double)pin[1]);
            kp[1] = a.dp_scale * (kk[4] * (double)pin[0] + kk[5] * (double)pin[1]);
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                kq[c] = kk[c];
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
        kq[0] = (float)kk[0];
        kq[1] = (float)kk[1];
        kp[0] = a.dp_scale_f * fmaf((float)kk[2], pin[0], (float)kk[3] * pin[1]);
        kp[1] = a.dp_scale_f * fmaf((float)kk[4], pin[0], (float)kk[5] * pin[1]);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            kq[c] = (float)kk[c];
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
        } else {
            a.S_out[2 * (size_t)i] = make_float4(y[0], y[1], y[2], 0.0f);
            a.S_out[2 * (size_t)i + 1] = make_float4(y[3], y[4], y[5], 0.0f);
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
        } else {
            a.Sx_w[2 * (size_t)i] = make_float4(y[0], y[1], y[2], 0.0f);
            a.Sx_w[2 * (size_t)i + 1] = make_float4(y[3], y[4], y[5], 0.0f);
        }
    }
}

// The pair phase of one stage over this CTA's stream-K range: per tile segment,
// stage the sources in shared memory, sum in registers, reduce over warps and
// add into the FP64 accumulator K.  With LAST the last CTA to reach a tile also
// applies the RK4 stage to it (one launch per stage); without LAST the caller
// finishes the particles after a grid-wide barrier (persistent shoot).
template <int DIM, int KER, int THREADS, bool LAST>
__device__ __forceinline__ void stage_pairs(const StageArgs& a, float4* smem, int* s_last)
{
    constexpr int W = THREADS / 32;
    constexpr int V = DIM == 2 ? 1 : 2;  // float4 per particle
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int n = a.n;
    long long u0 = (long long)blockIdx.x * a.U / a.G;
    const long long u1 = (long long)(blockIdx.x + 1) * a.U / a.G;

    while (u0 < u1) {
        const int b = (int)(u0 / n);
        const int j0 = (int)(u0 - (long long)b * n);
        const int j1 = (int)min((long long)n, (long long)j0 + (u1 - u0));

        // the two particles of this lane (zeros beyond n contribute nothing used)
        float qi[2][DIM], pi[2][DIM];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int i = b * kTileI + lane + 32 * r;
            if (i < n) {
                if constexpr (DIM == 2) {
                    const float4 v = __ldcg(a.S_in + i);
                    qi[r][0] = v.x; qi[r][1] = v.y; pi[r][0] = v.z; pi[r][1] = v.w;
                } else {
                    const float4 v0 = __ldcg(a.S_in + 2 * (size_t)i), v1 = __ldcg(a.S_in + 2 * (size_t)i + 1);
                    qi[r][0] = v0.x; qi[r][1] = v0.y; qi[r][2] = v0.z;
                    pi[r][0] = v1.x; pi[r][1] = v1.y; pi[r][2] = v1.z;
                }
            } else {
#pragma unroll
                for (int c = 0; c < DIM; ++c) { qi[r][c] = 0.0f; pi[r][c] = 0.0f; }
            }
        }
        float acc[2][kKWidth];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int t = 0; t < kKWidth; ++t) acc[r][t] = 0.0f;

        for (int cj = j0; cj < j1; cj += kChunk) {
            const int L = min(kChunk, j1 - cj);
            __syncthreads();
            for (int t = threadIdx.x; t < L * V; t += THREADS) smem[t] = __ldcg(a.S_in + (size_t)cj * V + t);
            __syncthreads();
            const int ja = warp * L / W, jb = (warp + 1) * L / W;
#pragma unroll 4
            for (int j = ja; j < jb; ++j) {
                if constexpr (DIM == 2) {
                    const float4 v = smem[j];
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const float dx = qi[r][0] - v.x, dy = qi[r][1] - v.y;
                        const float r2 = fmaf(dx, dx, dy * dy);
                        float G, w;
                        kfun_f32<KER>(r2, G, w);
                        acc[r][0] = fmaf(G, v.z, acc[r][0]);
                        acc[r][1] = fmaf(G, v.w, acc[r][1]);
                        const float tx = w * dx, ty = w * dy;
                        acc[r][2] = fmaf(tx, v.z, acc[r][2]);
                        acc[r][3] = fmaf(tx, v.w, acc[r][3]);
                        acc[r][4] = fmaf(ty, v.z, acc[r][4]);
                        acc[r][5] = fmaf(ty, v.w, acc[r][5]);
                    }
                } else {
                    const float4 v0 = smem[2 * j], v1 = smem[2 * j + 1];
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const float dx = qi[r][0] - v0.x, dy = qi[r][1] - v0.y, dz = qi[r][2] - v0.z;
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        float G, w;
                        kfun_f32<KER>(r2, G, w);
                        acc[r][0] = fmaf(G, v1.x, acc[r][0]);
                        acc[r][1] = fmaf(G, v1.y, acc[r][1]);
                        acc[r][2] = fmaf(G, v1.z, acc[r][2]);
                        const float pp = fmaf(pi[r][0], v1.x, fmaf(pi[r][1], v1.y, pi[r][2] * v1.z));
                        const float c = w * pp;
                        acc[r][3] = fmaf(c, dx, acc[r][3]);
                        acc[r][4] = fmaf(c, dy, acc[r][4]);
                        acc[r][5] = fmaf(c, dz, acc[r][5]);
                    }
                }
            }
        }

        // warps' partials -> shared memory [W][6][64] -> FP64 accumulator
        __syncthreads();
        float* red = reinterpret_cast<float*>(smem);
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int t = 0; t < kKWidth; ++t) red[(warp * kKWidth + t) * kTileI + lane + 32 * r] = acc[r][t];
        __syncthreads();
        for (int t = threadIdx.x; t < kKWidth * kTileI; t += THREADS) {
            const int k = t / kTileI, il = t % kTileI;
            float s = 0.0f;
#pragma unroll 8
            for (int w2 = 0; w2 < W; ++w2) s += red[(w2 * kKWidth + k) * kTileI + il];
            const int i = b * kTileI + il;
            if (i < n) atomicAdd(a.K + (size_t)i * kKWidth + k, (double)s);
        }
        if constexpr (LAST) {
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                const int prev = atomicAdd(a.counters + b, 1);
                *s_last = (prev == tile_contributors(b, a) - 1);
            }
            __syncthreads();
            if (*s_last) {
                __threadfence();
                if (threadIdx.x < kTileI) {
                    const int i = b * kTileI + threadIdx.x;
                    if (i < n) epilogue_mixed<DIM>(a, i);
                }
                if (threadIdx.x == 0) a.counters[b] = 0;
            }
        }
        u0 += (j1 - j0);
    }
}

// ------------------------------------------------------------------ 2-D Gaussian, factored
// The pair phase of the 2-D Gaussian in tiles of kTileG = 128 particles (32 lanes
// x 4 registers), on coordinates centred on the tile's first particle,
// q'' = q' - q'_first.  With G = 2^-|q''_i - q''_j|^2 (scaled units),
//   G_ij = 2^-|q''_i|^2 * 2^t,   t = 2 q''_i . q''_j - |q''_j|^2  (<= |q''_i|^2),
//   dq_i = E_i sum_j g_ij p_j,   M_i = q''_i (x) dq_i - E_i sum_j g_ij (q''_j (x) p_j),
// with g = 2^t and E_i = 2^-|q''_i|^2, so a pair costs two FMAs for t, one ex2 and
// three packed f32x2 FMAs (six FP32 FMAs), against per-source records
// (2x, 2y, -|q''|^2, y px), (px, py, x px, x py), (y py) built once per staged chunk.  t never exceeds |q''_i|^2; a tile
// whose |q''_i|^2 could overflow (> kFactorMax) takes the difference form
// d = q''_i - q''_j instead (same records).
constexpr int kTileG = 128;
constexpr int kChunkG = 2048;
constexpr float kFactorMax = 60.0f;

template <int THREADS>
__device__ __forceinline__ void stage_pairs_gauss2(const StageArgs& a, float4* smem)
{
    constexpr int W = THREADS / 32;
    constexpr int RI = kTileG / 32;
    float4* recA = smem;                                         // [2 * kChunkG]
    float* recB = reinterpret_cast<float*>(smem + 2 * kChunkG);  // [kChunkG]
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int n = a.n;
    long long u0 = (long long)blockIdx.x * a.U / a.G;
    const long long u1 = (long long)(blockIdx.x + 1) * a.U / a.G;
    while (u0 < u1) {
        const int b = (int)(u0 / n);
        const int j0 = (int)(u0 - (long long)b * n);
        const int j1 = (int)min((long long)n, (long long)j0 + (u1 - u0));
        // issue every load of the segment start at once: the tile centre, the
        // lane's particles and the first chunk's sources (kChunkG / THREADS each)
        constexpr int PF = kChunkG / THREADS;
        const int L0 = min(kChunkG, j1 - j0);
        float4 pre[PF];
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            const int t = threadIdx.x + k * THREADS;
            pre[k] = t < L0 ? __ldcg(a.S_in + j0 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const float4 c4 = __ldcg(a.S_in + (size_t)b * kTileG);  // tile centre: its first particle
        float4 vi[RI];
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int i = b * kTileG + lane + 32 * r;
            vi[r] = i < n ? __ldcg(a.S_in + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float qx[RI], qy[RI];
        float mq = 0.0f;
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int i = b * kTileG + lane + 32 * r;
            const float4 v = i < n ? vi[r] : c4;
            qx[r] = v.x - c4.x;
            qy[r] = v.y - c4.y;
            mq = fmaxf(mq, fmaf(qx[r], qx[r], qy[r] * qy[r]));
        }
        const bool factored = !__syncthreads_or(mq > kFactorMax);
        // per particle: (sum g px, sum g py), (sum g x px, sum g x py), (sum g y px, sum g y py),
        // packed so every accumulation is one f32x2 FMA
        float2 sqv[RI], sbx[RI], sby[RI];
#pragma unroll
        for (int r = 0; r < RI; ++r) sqv[r] = sbx[r] = sby[r] = make_float2(0.0f, 0.0f);
        for (int cj = j0; cj < j1; cj += kChunkG) {
            const int L = min(kChunkG, j1 - cj);
            __syncthreads();
            for (int t = threadIdx.x; t < L; t += THREADS) {
                const float4 v = cj == j0 ? pre[t / THREADS] : __ldcg(a.S_in + cj + t);
                const float x = v.x - c4.x, y = v.y - c4.y;
                recA[2 * t] = make_float4(2.0f * x, 2.0f * y, -fmaf(x, x, y * y), y * v.z);
                recA[2 * t + 1] = make_float4(v.z, v.w, x * v.z, x * v.w);
                recB[t] = y * v.w;
            }
            __syncthreads();
            const int ja = warp * L / W, jb = (warp + 1) * L / W;
            if (factored) {
#pragma unroll 2
                for (int j = ja; j < jb; ++j) {
                    // A = (2x, 2y, -|q''|^2, y px), B = (px, py, x px, x py), byy = y py
                    const float4 A = recA[2 * j], B = recA[2 * j + 1];
                    const float byy = recB[j];
                    const float2 pxy = make_float2(B.x, B.y), xp = make_float2(B.z, B.w);
                    const float2 yp = make_float2(A.w, byy);
#pragma unroll
                    for (int r = 0; r < RI; ++r) {
                        const float g = ex2_approx(fmaf(qx[r], A.x, fmaf(qy[r], A.y, A.z)));
                        const float2 gg = make_float2(g, g);
                        sqv[r] = __ffma2_rn(gg, pxy, sqv[r]);
                        sbx[r] = __ffma2_rn(gg, xp, sbx[r]);
                        sby[r] = __ffma2_rn(gg, yp, sby[r]);
                    }
                }
            } else {
                // difference form: G = ex2(-|d|^2) with d = q''_i - q''_j, same sums
                for (int j = ja; j < jb; ++j) {
                    const float4 A = recA[2 * j], B = recA[2 * j + 1];
                    const float byy = recB[j];
                    const float2 pxy = make_float2(B.x, B.y), xp = make_float2(B.z, B.w);
                    const float2 yp = make_float2(A.w, byy);
#pragma unroll
                    for (int r = 0; r < RI; ++r) {
                        const float dx = fmaf(-0.5f, A.x, qx[r]), dy = fmaf(-0.5f, A.y, qy[r]);
                        const float G = ex2_approx(-fmaf(dx, dx, dy * dy));
                        const float2 gg = make_float2(G, G);
                        sqv[r] = __ffma2_rn(gg, pxy, sqv[r]);
                        sbx[r] = __ffma2_rn(gg, xp, sbx[r]);
                        sby[r] = __ffma2_rn(gg, yp, sby[r]);
                    }
                }
            }
        }
        // per particle: dq = E sq, M = q'' (x) dq - E sb  (E = 1 in the difference form)
        __syncthreads();
        float* red = reinterpret_cast<float*>(smem);  // [W][6][kTileG]
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const float E = factored ? ex2_approx(-fmaf(qx[r], qx[r], qy[r] * qy[r])) : 1.0f;
            const float d0 = E * sqv[r].x, d1 = E * sqv[r].y;
            float* o = red + (size_t)warp * kKWidth * kTileG + lane + 32 * r;
            o[0 * kTileG] = d0;
            o[1 * kTileG] = d1;
            o[2 * kTileG] = fmaf(qx[r], d0, -E * sbx[r].x);
            o[3 * kTileG] = fmaf(qx[r], d1, -E * sbx[r].y);
            o[4 * kTileG] = fmaf(qy[r], d0, -E * sby[r].x);
            o[5 * kTileG] = fmaf(qy[r], d1, -E * sby[r].y);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < kKWidth * kTileG; t += THREADS) {
            const int k = t / kTileG, il = t % kTileG;
            float sum = 0.0f;
#pragma unroll 8
            for (int w2 = 0; w2 < W; ++w2) sum += red[(w2 * kKWidth + k) * kTileG + il];
            const int i = b * kTileG + il;
            if (i < n) atomicAdd(a.K + (size_t)i * kKWidth + k, (double)sum);
        }
        u0 += (j1 - j0);
    }
}

template <int DIM, int KER, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) k_stage_mixed(StageArgs a)
{
    extern __shared__ float4 smem[];
    __shared__ int s_last;
    stage_pairs<DIM, KER, THREADS, true>(a, smem, &s_last);
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
    // bar[0..7]: arrival counters, CTA c arrives on bar[c % 8] (spreads the atomics
    // over eight L2 lines); barrier e completes when bar[k] reaches e * (CTAs on k)
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

// A whole shoot of `steps` RK4 steps in one cooperative launch: per stage, the
// pair phase, a barrier, the RK4 stage of the particles this CTA owns
// ([c n / G, (c+1) n / G)), and a barrier.
template <int DIM, int KER, int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
    k_shoot_mixed(StageArgs a, const float4* Sx, float4* Sa, float4* Sb, int steps, unsigned* bar, int* err)
{
    extern __shared__ float4 smem[];
    const int n = a.n;
    const int i0 = (int)((long long)blockIdx.x * n / gridDim.x), i1 = (int)((long long)(blockIdx.x + 1) * n / gridDim.x);
    unsigned epoch = 0;
    a.Sx = Sx;
    for (int s = 0; s < steps; ++s) {
        for (int stage = 0; stage < 4; ++stage) {
            a.stage = stage;
            a.S_in = stage == 0 ? Sx : (stage == 2 ? Sb : Sa);
            a.S_out = stage == 1 ? Sb : Sa;
            if constexpr (DIM == 2 && KER == EP_GAUSS) {
                stage_pairs_gauss2<THREADS>(a, smem);
            } else {
                stage_pairs<DIM, KER, THREADS, false>(a, smem, nullptr);
            }
            if (!grid_barrier(bar, err, ++epoch)) return;
            for (int i = i0 + threadIdx.x; i < i1; i += THREADS) epilogue_mixed<DIM>(a, i);
            if (!grid_barrier(bar, err, ++epoch)) return;
        }
    }
}

// ------------------------------------------------------------------ fp64
template <int DIM>
__device__ void epilogue_fp64(const StageArgs& a, int i, double sigma_unused)
{
    (void)sigma_unused;
    double kq[DIM], kp[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        kq[c] = __ldcg(a.K + (size_t)i * kKWidth + c);
        kp[c] = __ldcg(a.K + (size_t)i * kKWidth + 3 + c);
        a.K[(size_t)i * kKWidth + c] = 0.0;
        a.K[(size_t)i * kKWidth + 3 + c] = 0.0;
    }
    if (a.mode == MODE_RHS) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            a.out_q[(size_t)i * DIM + c] = kq[c];
            a.out_p[(size_t)i * DIM + c] = kp[c];
        }
        return;
    }
    const int n = a.n;
    double* xq = a.x + (size_t)i * DIM;
    double* xp = a.x + (size_t)n * DIM + (size_t)i * DIM;
    double* A = a.dacc + (size_t)i * 2 * DIM;
    if (a.stage < 3) {
        const double cdt = (a.stage == 2 ? 1.0 : 0.5) * a.dt;
        const double bw = a.stage == 0 ? 1.0 : 2.0;
        double* out = a.D_out + (size_t)i * 2 * DIM;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            out[c] = xq[c] + cdt * kq[c];
            out[DIM + c] = xp[c] + cdt * kp[c];
            A[c] = (a.stage == 0 ? 0.0 : A[c]) + bw * kq[c];
            A[DIM + c] = (a.stage == 0 ? 0.0 : A[DIM + c]) + bw * kp[c];
        }
    } else {
        double* out = a.D_out + (size_t)i * 2 * DIM;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            const double nq = xq[c] + a.dt / 6.0 * (A[c] + kq[c]);
            const double np = xp[c] + a.dt / 6.0 * (A[DIM + c] + kp[c]);
            xq[c] = nq;
            xp[c] = np;
            out[c] = nq;
            out[DIM + c] = np;
        }
    }
}

template <int DIM, int KER, int THREADS>
__global__ void __launch_bounds__(THREADS) k_stage_fp64(StageArgs a, double sigma)
{
    constexpr int W = THREADS / 32;
    constexpr int S = 2 * DIM;  // doubles per particle in the stage copy
    extern __shared__ double dsm[];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int n = a.n;
    long long u0 = (long long)blockIdx.x * a.U / a.G;
    const long long u1 = (long long)(blockIdx.x + 1) * a.U / a.G;
    while (u0 < u1) {
        const int b = (int)(u0 / n);
        const int j0 = (int)(u0 - (long long)b * n);
        const int j1 = (int)min((long long)n, (long long)j0 + (u1 - u0));
        double qi[2][DIM], pi[2][DIM];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int i = b * kTileI + lane + 32 * r;
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                qi[r][c] = i < n ? a.D_in[(size_t)i * S + c] : 0.0;
                pi[r][c] = i < n ? a.D_in[(size_t)i * S + DIM + c] : 0.0;
            }
        }
        double acc[2][2 * DIM];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int t = 0; t < 2 * DIM; ++t) acc[r][t] = 0.0;
        for (int cj = j0; cj < j1; cj += kChunk64) {
            const int L = min(kChunk64, j1 - cj);
            __syncthreads();
            for (int t = threadIdx.x; t < L * S; t += THREADS) dsm[t] = a.D_in[(size_t)cj * S + t];
            __syncthreads();
            const int ja = warp * L / W, jb = (warp + 1) * L / W;
            for (int j = ja; j < jb; ++j) {
                const double* v = dsm + (size_t)j * S;
                const int jg = cj + j;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    double d[DIM], r2 = 0.0, pp = 0.0;
#pragma unroll
                    for (int c = 0; c < DIM; ++c) {
                        d[c] = qi[r][c] - v[c];
                        r2 += d[c] * d[c];
                        pp += pi[r][c] * v[DIM + c];
                    }
                    double G, phi;
                    kfun_f64<KER>(r2, sigma, G, phi);
                    const int i = b * kTileI + lane + 32 * r;
                    const double wgt = (jg == i) ? 0.0 : -pp * phi;
#pragma unroll
                    for (int c = 0; c < DIM; ++c) {
                        acc[r][c] += G * v[DIM + c];
                        acc[r][DIM + c] += wgt * d[c];
                    }
                }
            }
        }
        __syncthreads();
        double* red = dsm;  // [W][2*DIM][64]
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int t = 0; t < 2 * DIM; ++t) red[(warp * 2 * DIM + t) * kTileI + lane + 32 * r] = acc[r][t];
        __syncthreads();
        for (int t = threadIdx.x; t < 2 * DIM * kTileI; t += THREADS) {
            const int k = t / kTileI, il = t % kTileI;
            double s = 0.0;
            for (int w2 = 0; w2 < W; ++w2) s += red[(w2 * 2 * DIM + k) * kTileI + il];
            const int i = b * kTileI + il;
            const int slot = k < DIM ? k : 3 + (k - DIM);
            if (i < n) atomicAdd(a.K + (size_t)i * kKWidth + slot, s);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const int prev = atomicAdd(a.counters + b, 1);
            s_last = (prev == tile_contributors(b, a) - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            if (threadIdx.x < kTileI) {
                const int i = b * kTileI + threadIdx.x;
                if (i < n) epilogue_fp64<DIM>(a, i, sigma);
            }
            if (threadIdx.x == 0) a.counters[b] = 0;
        }
        u0 += (j1 - j0);
    }
}

// ------------------------------------------------------------------ helpers
// c0 = centre of the bounding box of q (one CTA).
__global__ void k_bbox_center(const double* __restrict__ q, int n, int dim, double* c0)
{
    __shared__ double smin[3][32], smax[3][32];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int c = 0; c < dim; ++c) {
            const double v = q[(size_t)i * dim + c];
            mn[c] = fmin(mn[c], v);
            mx[c] = fmax(mx[c], v);
        }
    for (int c = 0; c < dim; ++c)
        for (int o = 16; o > 0; o >>= 1) {
            mn[c] = fmin(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = fmax(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int c = 0; c < dim; ++c) { smin[c][w] = mn[c]; smax[c][w] = mx[c]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int c = 0; c < 3; ++c) {
            double a = INFINITY, b2 = -INFINITY;
            if (c < dim)
                for (int k = 0; k < nw; ++k) { a = fmin(a, smin[c][k]); b2 = fmax(b2, smax[c][k]); }
            c0[c] = (c < dim && n > 0) ? 0.5 * (a + b2) : 0.0;
        }
    }
}

// x = [q | p] and the step-start stage copy.
__global__ void k_load_state(const double* __restrict__ q, const double* __restrict__ p, int n, int dim,
                             double* __restrict__ x, const double* __restrict__ c0, double s,
                             float4* __restrict__ Sx, double* __restrict__ Dx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double qq[3] = {0, 0, 0}, pp[3] = {0, 0, 0};
    for (int c = 0; c < dim; ++c) {
        qq[c] = q[(size_t)i * dim + c];
        pp[c] = p[(size_t)i * dim + c];
        x[(size_t)i * dim + c] = qq[c];
        x[(size_t)n * dim + (size_t)i * dim + c] = pp[c];
    }
    if (Sx) {
        float y[3];
        for (int c = 0; c < 3; ++c) y[c] = c < dim ? (float)((qq[c] - c0[c]) * s) : 0.0f;
        if (dim == 2) {
            Sx[i] = make_float4(y[0], y[1], (float)pp[0], (float)pp[1]);
        } else {
            Sx[2 * (size_t)i] = make_float4(y[0], y[1], y[2], 0.0f);
            Sx[2 * (size_t)i + 1] = make_float4((float)pp[0], (float)pp[1], (float)pp[2], 0.0f);
        }
    }
    if (Dx) {
        for (int c = 0; c < dim; ++c) {
            Dx[(size_t)i * 2 * dim + c] = qq[c];
            Dx[(size_t)i * 2 * dim + dim + c] = pp[c];
        }
    }
}

template <int DIM, int KER, int THREADS>
ep_status launch_mixed(const StageArgs& a, cudaStream_t st)
{
    constexpr int W = THREADS / 32;
    constexpr int V = DIM == 2 ? 1 : 2;
    const size_t smem = std::max((size_t)kChunk * V * sizeof(float4), (size_t)W * kKWidth * kTileI * sizeof(float));
    static bool attr = false;
    if (!attr) {
        EP_TRY_CUDA(cudaFuncSetAttribute(k_stage_mixed<DIM, KER, THREADS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    count_launch();
    k_stage_mixed<DIM, KER, THREADS><<<a.G, THREADS, smem, st>>>(a);
    return EP_OK;
}

template <int DIM, int KER>
ep_status launch_fp64(const StageArgs& a, double sigma, cudaStream_t st)
{
    constexpr int THREADS = 256;
    constexpr int W = THREADS / 32;
    const size_t smem = std::max((size_t)kChunk64 * 2 * DIM * sizeof(double),
                                 (size_t)W * 2 * DIM * kTileI * sizeof(double));
    static bool attr = false;
    if (!attr) {
        EP_TRY_CUDA(cudaFuncSetAttribute(k_stage_fp64<DIM, KER, THREADS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    count_launch();
    k_stage_fp64<DIM, KER, THREADS><<<a.G, THREADS, smem, st>>>(a, sigma);
    return EP_OK;
}

ep_status launch_stage(const ep_params& P, const StageArgs& a, int threads, cudaStream_t st)
{
#define EP_MIXED_CASE(D, K)                                                       \
    if (P.dim == D && P.kernel == K) {                                            \
        if (threads == 1024) return launch_mixed<D, K, 1024>(a, st);              \
        if (threads == 512) return launch_mixed<D, K, 512>(a, st);                \
        return launch_mixed<D, K, 256>(a, st);                                    \
    }
#define EP_FP64_CASE(D, K) \
    if (P.dim == D && P.kernel == K) return launch_fp64<D, K>(a, P.sigma, st);
    if (P.precision == EP_MIXED) {
        EP_MIXED_CASE(2, EP_GAUSS) EP_MIXED_CASE(2, EP_TENT) EP_MIXED_CASE(2, EP_EXPCONE)
        EP_MIXED_CASE(3, EP_GAUSS) EP_MIXED_CASE(3, EP_TENT) EP_MIXED_CASE(3, EP_EXPCONE)
    } else {
        EP_FP64_CASE(2, EP_GAUSS) EP_FP64_CASE(2, EP_TENT) EP_FP64_CASE(2, EP_EXPCONE)
        EP_FP64_CASE(3, EP_GAUSS) EP_FP64_CASE(3, EP_TENT) EP_FP64_CASE(3, EP_EXPCONE)
    }
#undef EP_MIXED_CASE
#undef EP_FP64_CASE
    set_error("no all-pairs kernel for dim=%d kernel=%d precision=%d", P.dim, P.kernel, P.precision);
    return EP_EINVAL;
}

// EP_PERSISTENT=0 in the environment selects one launch per RK4 stage instead of
// the persistent shoot (both compute the same result).
bool allpairs_persistent_enabled()
{
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("EP_PERSISTENT");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

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
    a.c0 = b.c0;
    a.x = b.x;
    a.acc = b.acc;
    a.dacc = b.dacc;
    a.K = b.K;
    a.counters = b.counters;
    return a;
}

}  // namespace

size_t allpairs_bytes(int n, int dim, int prec)
{
    Sizer z;
    const int ntiles = (n + kTileI - 1) / kTileI;
    z.add(sizeof(double) * 2 * dim * (size_t)n);   // x
    z.add(sizeof(double) * kKWidth * (size_t)n);   // K
    z.add(sizeof(int) * (size_t)ntiles);           // counters
    z.add(sizeof(double) * 4);                     // c0
    z.add(sizeof(unsigned) * 12);                  // barrier counters, error flag
    if (prec == EP_MIXED && dim == 2) {
        z.add(sizeof(double) * 2 * dim * (size_t)n);  // tuner backup of x
        z.add(sizeof(float4) * (size_t)n);            // tuner backup of the stage copy
    }
    if (prec == EP_MIXED) {
        const int V = dim == 2 ? 1 : 2;
        for (int k = 0; k < 3; ++k) z.add(sizeof(float4) * V * (size_t)n);
        z.add(sizeof(float) * 2 * dim * (size_t)n);
    } else {
        for (int k = 0; k < 3; ++k) z.add(sizeof(double) * 2 * dim * (size_t)n);
        z.add(sizeof(double) * 2 * dim * (size_t)n);
    }
    return z.total;
}

ep_status allpairs_carve(Arena* ar, int n, int dim, int prec, AllPairsBufs* b)
{
    const int ntiles = (n + kTileI - 1) / kTileI;
    b->n = n;
    b->dim = dim;
    b->prec = prec;
    b->x = (double*)ar->carve(sizeof(double) * 2 * dim * (size_t)n);
    b->K = (double*)ar->carve(sizeof(double) * kKWidth * (size_t)n);
    b->counters = (int*)ar->carve(sizeof(int) * (size_t)ntiles);
    b->c0 = (double*)ar->carve(sizeof(double) * 4);
    b->bar = (unsigned*)ar->carve(sizeof(unsigned) * 12);
    b->err = (int*)(b->bar ? b->bar + 8 : nullptr);
    if (prec == EP_MIXED && dim == 2) {
        b->x_bak = (double*)ar->carve(sizeof(double) * 2 * dim * (size_t)n);
        b->S_bak = (float4*)ar->carve(sizeof(float4) * (size_t)n);
    }
    if (prec == EP_MIXED) {
        const int V = dim == 2 ? 1 : 2;
        b->Sx = (float4*)ar->carve(sizeof(float4) * V * (size_t)n);
        b->Sa = (float4*)ar->carve(sizeof(float4) * V * (size_t)n);
        b->Sb = (float4*)ar->carve(sizeof(float4) * V * (size_t)n);
        b->acc = (float*)ar->carve(sizeof(float) * 2 * dim * (size_t)n);
        if (!b->acc) return set_error("workspace too small"), EP_ENOMEM;
    } else {
        b->Dx = (double*)ar->carve(sizeof(double) * 2 * dim * (size_t)n);
        b->Da = (double*)ar->carve(sizeof(double) * 2 * dim * (size_t)n);
        b->Db = (double*)ar->carve(sizeof(double) * 2 * dim * (size_t)n);
        b->dacc = (double*)ar->carve(sizeof(double) * 2 * dim * (size_t)n);
        if (!b->dacc) return set_error("workspace too small"), EP_ENOMEM;
    }
    if (!b->c0) return set_error("workspace too small"), EP_ENOMEM;
    return EP_OK;
}

APConfig allpairs_config(int n, int dim, int prec, int kernel)
{
    (void)kernel;
    APConfig c;
    DeviceInfo di{};
    if (device_info(&di) != EP_OK) di.sm_count = 1;
    if (prec == EP_MIXED) {
        // one CTA per SM
        c.threads = 1024;
        c.ctas = di.sm_count;
    } else {
        c.threads = 256;
        c.ctas = di.sm_count * 4;
    }
    // keep at least ~256 units (mixed) or ~16 units (FP64, whose pairs cost ~60x more)
    // per CTA for tiny problems
    const long long ntiles = (n + kTileI - 1) / kTileI;
    const long long U = ntiles * (long long)n;
    const long long maxc = std::max<long long>(1, U / (prec == EP_MIXED ? 256 : 16));
    c.ctas = (int)std::max<long long>(1, std::min<long long>(c.ctas, maxc));
    return c;
}

ep_status allpairs_load(const ep_params& P, const AllPairsBufs& b, const double* q, const double* p,
                        cudaStream_t st)
{
    const int n = b.n;
    const int ntiles = (n + kTileI - 1) / kTileI;
    EP_TRY_CUDA(cudaMemsetAsync(b.K, 0, sizeof(double) * kKWidth * (size_t)n, st));
    EP_TRY_CUDA(cudaMemsetAsync(b.counters, 0, sizeof(int) * (size_t)ntiles, st));
    count_launch();
    k_bbox_center<<<1, 1024, 0, st>>>(q, n, P.dim, b.c0);
    const KernelScale ks = kernel_scale(P.kernel, P.sigma);
    if (n > 0) {
        count_launch();
        k_load_state<<<(n + 255) / 256, 256, 0, st>>>(q, p, n, P.dim, b.x, b.c0, ks.s, b.Sx, b.Dx);
    }
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

ep_status allpairs_rhs(const ep_params& P, const AllPairsBufs& b, double* dq, double* dp, cudaStream_t st)
{
    if (b.n == 0) return EP_OK;
    const APConfig cfg = allpairs_config(b.n, P.dim, P.precision, P.kernel);
    StageArgs a = base_args(P, b, cfg);
    a.mode = MODE_RHS;
    a.stage = 0;
    a.S_in = b.Sx;
    a.D_in = b.Dx;
    a.out_q = dq;
    a.out_p = dp;
    EP_TRY(launch_stage(P, a, cfg.threads, st));
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

template <int DIM, int KER>
ep_status launch_shoot_mixed(const StageArgs& a0, const AllPairsBufs& b, int steps, cudaStream_t st, bool* done,
                             cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr)
{
    constexpr int THREADS = 1024;
    constexpr int W = THREADS / 32;
    constexpr int V = DIM == 2 ? 1 : 2;
    constexpr bool kFact = DIM == 2 && KER == EP_GAUSS;
    const size_t smem = kFact ? std::max((size_t)kChunkG * (2 * sizeof(float4) + sizeof(float)),
                                         (size_t)W * kKWidth * kTileG * sizeof(float))
                              : std::max((size_t)kChunk * V * sizeof(float4), (size_t)W * kKWidth * kTileI * sizeof(float));
    auto fn = k_shoot_mixed<DIM, KER, THREADS>;
    static int resident = -1;
    if (resident < 0) {
        EP_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        EP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, THREADS, smem));
        DeviceInfo di{};
        EP_TRY(device_info(&di));
        resident = per_sm * di.sm_count;
    }
    *done = false;
    if (a0.G > resident) return EP_OK;  // not all CTAs can be resident: per-stage launches instead
    StageArgs a = a0;
    if (kFact) {
        // tiles of kTileG particles: units and CTA count of that decomposition
        a.U = (long long)((b.n + kTileG - 1) / kTileG) * b.n;
        a.G = (int)std::min<long long>(a.G, a.U);
    }
    const float4* Sx = b.Sx;
    float4* Sa = b.Sa;
    float4* Sb = b.Sb;
    unsigned* bar = b.bar;
    int* err = b.err;
    EP_TRY_CUDA(cudaMemsetAsync(b.bar, 0, sizeof(unsigned) * 9, st));
    void* args[] = {&a, &Sx, &Sa, &Sb, &steps, &bar, &err};
    count_launch();
    if (ev0) EP_TRY_CUDA(cudaEventRecord(ev0, st));
    EP_TRY_CUDA(cudaLaunchCooperativeKernel((void*)fn, dim3(a.G), dim3(THREADS), args, smem, st));
    if (ev1) EP_TRY_CUDA(cudaEventRecord(ev1, st));
    int herr = 0;
    EP_TRY_CUDA(cudaMemcpyAsync(&herr, b.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    if (herr) {
        set_error("persistent shoot: a grid-barrier wait gave up (kernel ended early)");
        return EP_ETIMEOUT;
    }
    *done = true;
    return EP_OK;
}

ep_status launch_shoot(const ep_params& P, const StageArgs& a, const AllPairsBufs& b, int steps, cudaStream_t st,
                       bool* done, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr)
{
#define EP_SHOOT_CASE(D, K) \
    if (P.dim == D && P.kernel == K) return launch_shoot_mixed<D, K>(a, b, steps, st, done, ev0, ev1);
    EP_SHOOT_CASE(2, EP_GAUSS) EP_SHOOT_CASE(2, EP_TENT) EP_SHOOT_CASE(2, EP_EXPCONE)
    EP_SHOOT_CASE(3, EP_GAUSS) EP_SHOOT_CASE(3, EP_TENT) EP_SHOOT_CASE(3, EP_EXPCONE)
#undef EP_SHOOT_CASE
    *done = false;
    return EP_OK;
}

// ------------------------------------------------------------------ autotuner
// The persistent 2-D Gaussian shoot splits the pair matrix (tiles of kTileG x n)
// over G CTAs.  G = SM count balances the work exactly but lets some CTAs span two
// tiles (each segment start costs a round of loads and a reduction); a G that is a
// multiple of the tile count keeps every CTA inside one tile at the price of idle
// SMs.  The tuner times a one-step shoot for each candidate on the loaded state
// (restoring it afterwards) and caches the fastest per (n, dim, kernel).
// EP_AUTOTUNE=0 in the environment skips it (G = SM count).
struct TuneKey {
    int n, dim, kernel, dev;
    bool operator<(const TuneKey& o) const
    {
        return n != o.n ? n < o.n : dim != o.dim ? dim < o.dim : kernel != o.kernel ? kernel < o.kernel : dev < o.dev;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

bool autotune_enabled()
{
    const char* e = getenv("EP_AUTOTUNE");
    return !(e && e[0] == '0');
}

ep_status tune_persistent(const ep_params& P, const AllPairsBufs& b, StageArgs a, double dt, cudaStream_t st, int* best)
{
    DeviceInfo di{};
    EP_TRY(device_info(&di));
    const int sm = di.sm_count;
    const int ntiles = (b.n + kTileG - 1) / kTileG;
    // the default split, the full and 7/8 SM counts, the two largest tile-aligned counts
    std::vector<int> cand = {a.G, sm, sm - sm / 8};
    for (int k = sm / std::max(1, ntiles), c = 0; k >= 1 && c < 2; --k, ++c) cand.push_back(ntiles * k);
    for (int& g : cand) g = (int)std::min<long long>(g, a.U);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    const size_t m2 = 2 * (size_t)P.dim * b.n;
    EP_TRY_CUDA(cudaMemcpyAsync(b.x_bak, b.x, sizeof(double) * m2, cudaMemcpyDeviceToDevice, st));
    EP_TRY_CUDA(cudaMemcpyAsync(b.S_bak, b.Sx, sizeof(float4) * (size_t)b.n, cudaMemcpyDeviceToDevice, st));
    cudaEvent_t e0, e1;
    EP_TRY_CUDA(cudaEventCreate(&e0));
    EP_TRY_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    *best = sm;
    a.dt = dt;
    a.dt_f = (float)dt;
    for (int G : cand) {
        if (G < 1) continue;
        a.G = G;
        float ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            EP_TRY_CUDA(cudaMemcpyAsync(b.x, b.x_bak, sizeof(double) * m2, cudaMemcpyDeviceToDevice, st));
            EP_TRY_CUDA(cudaMemcpyAsync(b.Sx, b.S_bak, sizeof(float4) * (size_t)b.n, cudaMemcpyDeviceToDevice, st));
            bool done = false;
            ep_status s = launch_shoot(P, a, b, 1, st, &done, e0, e1);
            if (s != EP_OK || !done) break;
            float t = 0.f;
            EP_TRY_CUDA(cudaEventElapsedTime(&t, e0, e1));
            if (rep > 0) ms = std::min(ms, t);
        }
        if (ms < best_ms) {
            best_ms = ms;
            *best = G;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    EP_TRY_CUDA(cudaMemcpyAsync(b.x, b.x_bak, sizeof(double) * m2, cudaMemcpyDeviceToDevice, st));
    EP_TRY_CUDA(cudaMemcpyAsync(b.Sx, b.S_bak, sizeof(float4) * (size_t)b.n, cudaMemcpyDeviceToDevice, st));
    return EP_OK;
}

ep_status allpairs_steps(const ep_params& P, const AllPairsBufs& b, int steps, double dt, cudaStream_t st)
{
    if (b.n == 0 || steps == 0) return EP_OK;
    const APConfig cfg = allpairs_config(b.n, P.dim, P.precision, P.kernel);
    StageArgs a = base_args(P, b, cfg);
    a.mode = MODE_RK4;
    a.dt = dt;
    a.dt_f = (float)dt;
    if (P.precision == EP_MIXED && cfg.threads == 1024 && allpairs_persistent_enabled()) {
        a.Sx_w = b.Sx;
        if (P.dim == 2 && P.kernel == EP_GAUSS && b.x_bak && autotune_enabled()) {
            DeviceInfo di{};
            EP_TRY(device_info(&di));
            const TuneKey key{b.n, P.dim, P.kernel, di.device};
            int G = -1;
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                auto it = g_tuned.find(key);
                if (it != g_tuned.end()) G = it->second;
            }
            if (G < 0) {
                EP_TRY(tune_persistent(P, b, a, dt, st, &G));
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tuned[key] = G;
            }
            a.G = G;
        }
        bool done = false;
        EP_TRY(launch_shoot(P, a, b, steps, st, &done));
        if (done) return EP_OK;
    }
    a.Sx = b.Sx;
    a.Sx_w = b.Sx;
    for (int s = 0; s < steps; ++s) {
        for (int stage = 0; stage < 4; ++stage) {
            a.stage = stage;
            // stage inputs: Sx -> Sa -> Sb -> Sa, stage 3 writes the next Sx
            if (P.precision == EP_MIXED) {
                a.S_in = stage == 0 ? b.Sx : (stage == 2 ? b.Sb : b.Sa);
                a.S_out = stage == 1 ? b.Sb : b.Sa;
            } else {
                a.D_in = stage == 0 ? b.Dx : (stage == 2 ? b.Db : b.Da);
                a.D_out = stage == 3 ? b.Dx : (stage == 1 ? b.Db : b.Da);
            }
            EP_TRY(launch_stage(P, a, cfg.threads, st));
        }
    }
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

ep_status allpairs_steps_rec(const ep_params& P, const AllPairsBufs& b, int steps, double dt, float4* rec,
                             double* drec, cudaStream_t st)
{
    if (b.n == 0 || steps == 0) return EP_OK;
    const APConfig cfg = allpairs_config(b.n, P.dim, P.precision, P.kernel);
    StageArgs a = base_args(P, b, cfg);
    a.mode = MODE_RK4;
    a.dt = dt;
    a.dt_f = (float)dt;
    const size_t V = P.dim == 2 ? 1 : 2;
    const size_t cm = V * (size_t)b.n;               // float4 per stage copy
    const size_t cd = 2 * (size_t)P.dim * b.n;       // doubles per stage copy
    if (P.precision == EP_MIXED)
        EP_TRY_CUDA(cudaMemcpyAsync(rec, b.Sx, sizeof(float4) * cm, cudaMemcpyDeviceToDevice, st));
    else
        EP_TRY_CUDA(cudaMemcpyAsync(drec, b.Dx, sizeof(double) * cd, cudaMemcpyDeviceToDevice, st));
    for (int k = 0; k < steps; ++k) {
        for (int stage = 0; stage < 4; ++stage) {
            a.stage = stage;
            const size_t in = 4 * (size_t)k + stage;
            if (P.precision == EP_MIXED) {
                a.Sx = rec + 4 * (size_t)k * cm;
                a.Sx_w = rec + 4 * (size_t)(k + 1) * cm;
                a.S_in = rec + in * cm;
                a.S_out = rec + (in + 1) * cm;
            } else {
                a.D_in = drec + in * cd;
                a.D_out = drec + (in + 1) * cd;
            }
            EP_TRY(launch_stage(P, a, cfg.threads, st));
        }
    }
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

}  // namespace ep
