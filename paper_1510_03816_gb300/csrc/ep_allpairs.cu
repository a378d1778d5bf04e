// ep_allpairs.cu -- all-pairs right-hand side of the N-particle system
// (Sec. 3.1, Eq. N-particle) with the classical RK4 stage (Sec. 4, Note 1
// item 5) fused into the kernel.
//
// Work decomposition (stream-K over the pair matrix).  Particles i are grouped
// in tiles of 64 (32 lanes x 2 registers).  The pair matrix is the sequence of
// U = ntiles * n units (tile b, source j), cut into G equal contiguous ranges,
// one per CTA, G = (SM count) x (resident CTAs per SM).  A CTA's range covers
// one or a few tile segments [j0, j1).  For each segment the CTA stages the
// FP32 source data of [j0, j1) in shared memory, chunk by chunk; its warps split
// a chunk's j range, every lane accumulates its two particles' sums over its
// share in registers (FP32), the warps' partials are summed in double-FP32
// (TwoSum) in shared memory, and the CTA adds them, converted exactly to FP64,
// into the FP64 accumulator K of the tile's particles (red.global.add.f64): the
// per-particle sums are accumulated in FP64 across blocks of at most
// kChunk / warps sources.  The last CTA to arrive at
// a tile (per-tile counter) applies the RK4 stage to the tile's particles:
// it reads k = K, forms the next stage input, resets K and the counter.
//
// Precision modes: EP_MIXED evaluates pair terms in FP32 on scaled
// coordinates (see ep_common.cuh), keeps the step state x_n in FP64 and the
// RK4 stage combination in FP32; EP_FP64 does every operation in FP64.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "ep_allpairs_dev.cuh"

namespace ep {

namespace {

constexpr int kChunk = 2048;  // sources staged per shared-memory fill (mixed)
// Position (scaled units) of the padding source of an odd source count in the packed
// source-pair records: every kernel value and weight is exactly zero there.
constexpr float kPadCoord = 1.0e18f;
// The 2-D Gaussian stream-K kernel folds its FP32 lane sums into the FP64 accumulator
// every kFoldChunks staged chunks (and at a segment's end): a warp's FP32 block of a
// particle's sum is at most kFoldChunks * 2048 / 32 = 256 sources (the generic kernels
// fold every 256 W / kChunk chunks, the same bound).
constexpr int kFoldChunks = 4;
// The barrier word array of the persistent shoots: [0, 8) arrival counters, [8] the
// error flag, [kBarProgress, + kMaxPersistentCtas) one progress word per CTA.
constexpr int kBarProgress = 16;
constexpr int kMaxPersistentCtas = 1024;
constexpr int kChunk64 = 1024;


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
    // chunks per FP32 block: a warp's block of a particle's sum stays <= 256 sources
    constexpr int FOLD = (256 * W) / kChunk > 0 ? (256 * W) / kChunk : 1;
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
        static_assert(THREADS == 512, "the generic pair stage runs in its 512-thread packed form");
        {
            // packed form (the 512-thread kernels): the staged sources are kept in pairs,
            // one float4 holding the positions of sources 2p and 2p+1 (2-D: x, x, y, y;
            // 3-D: x, x, y, y then z, z, px, px) and the next their momenta, so one load
            // gives the f32x2 operands of two sources; an odd count is padded with a
            // source far away and without momentum, whose terms are exactly zero.  Both
            // rows of the lane take each record pair; the differences are q_j - q_i, so
            // the momentum sums come out negated and their sign is restored at the fold.
            // Measured against the 1024-thread scalar loop: 3-D Gaussian at N = 16384 171
            // against 185 us per stage, 2-D tent at N = 4096 16.8 against 17.9 us, 3-D
            // tent 20.6 against 23.5 us, 2-D exp-cone the same (17.7 us); 768 threads: slower)
            constexpr int PV = DIM == 2 ? 2 : 3;  // float4 per source pair
            float2 nq[2][DIM], pb[2][DIM];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < DIM; ++c) {
                    nq[r][c] = make_float2(-qi[r][c], -qi[r][c]);
                    pb[r][c] = make_float2(pi[r][c], pi[r][c]);
                }
            float2 acc2[2][kKWidth];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int t = 0; t < kKWidth; ++t) acc2[r][t] = make_float2(0.0f, 0.0f);
            int nchunk2 = 0;
            for (int cj = j0; cj < j1; cj += kChunk) {
                const int L = min(kChunk, j1 - cj);
                const int P = (L + 1) >> 1;
                __syncthreads();
                for (int t = threadIdx.x; t < P; t += THREADS) {
                    const int j = cj + 2 * t;
                    const bool two = 2 * t + 1 < L;
                    if constexpr (DIM == 2) {
                        const float4 s0 = __ldcg(a.S_in + j);
                        const float4 s1 = two ? __ldcg(a.S_in + j + 1) : make_float4(kPadCoord, kPadCoord, 0.f, 0.f);
                        smem[2 * t] = make_float4(s0.x, s1.x, s0.y, s1.y);
                        smem[2 * t + 1] = make_float4(s0.z, s1.z, s0.w, s1.w);
                    } else {
                        const float4 q0 = __ldcg(a.S_in + 2 * (size_t)j), p0 = __ldcg(a.S_in + 2 * (size_t)j + 1);
                        const float4 q1 = two ? __ldcg(a.S_in + 2 * (size_t)j + 2)
                                              : make_float4(kPadCoord, kPadCoord, kPadCoord, 0.f);
                        const float4 p1 = two ? __ldcg(a.S_in + 2 * (size_t)j + 3) : make_float4(0.f, 0.f, 0.f, 0.f);
                        smem[3 * t] = make_float4(q0.x, q1.x, q0.y, q1.y);
                        smem[3 * t + 1] = make_float4(q0.z, q1.z, p0.x, p1.x);
                        smem[3 * t + 2] = make_float4(p0.y, p1.y, p0.z, p1.z);
                    }
                }
                __syncthreads();
                const int pa = warp * P / W, pz = (warp + 1) * P / W;
#pragma unroll 2
                for (int q = pa; q < pz; ++q) {
                    if constexpr (DIM == 2) {
                        const float4 A = smem[2 * q], B = smem[2 * q + 1];
                        const float2 X2 = make_float2(A.x, A.y), Y2 = make_float2(A.z, A.w);
                        const float2 PX = make_float2(B.x, B.y), PY = make_float2(B.z, B.w);
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const float2 dx = __fadd2_rn(X2, nq[r][0]), dy = __fadd2_rn(Y2, nq[r][1]);
                            const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
                            float2 G, w;
                            kfun_f32<KER>(r2.x, G.x, w.x);
                            kfun_f32<KER>(r2.y, G.y, w.y);
                            acc2[r][0] = __ffma2_rn(G, PX, acc2[r][0]);
                            acc2[r][1] = __ffma2_rn(G, PY, acc2[r][1]);
                            const float2 tx = __fmul2_rn(w, dx), ty = __fmul2_rn(w, dy);
                            acc2[r][2] = __ffma2_rn(tx, PX, acc2[r][2]);
                            acc2[r][3] = __ffma2_rn(tx, PY, acc2[r][3]);
                            acc2[r][4] = __ffma2_rn(ty, PX, acc2[r][4]);
                            acc2[r][5] = __ffma2_rn(ty, PY, acc2[r][5]);
                        }
                    } else {
                        const float4 A = smem[3 * q], B = smem[3 * q + 1], C = smem[3 * q + 2];
                        const float2 X2 = make_float2(A.x, A.y), Y2 = make_float2(A.z, A.w), Z2 = make_float2(B.x, B.y);
                        const float2 PX = make_float2(B.z, B.w), PY = make_float2(C.x, C.y), PZ = make_float2(C.z, C.w);
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const float2 dx = __fadd2_rn(X2, nq[r][0]), dy = __fadd2_rn(Y2, nq[r][1]);
                            const float2 dz = __fadd2_rn(Z2, nq[r][2]);
                            const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                            float2 G, w;
                            kfun_f32<KER>(r2.x, G.x, w.x);
                            kfun_f32<KER>(r2.y, G.y, w.y);
                            acc2[r][0] = __ffma2_rn(G, PX, acc2[r][0]);
                            acc2[r][1] = __ffma2_rn(G, PY, acc2[r][1]);
                            acc2[r][2] = __ffma2_rn(G, PZ, acc2[r][2]);
                            const float2 pp = __ffma2_rn(pb[r][0], PX, __ffma2_rn(pb[r][1], PY, __fmul2_rn(pb[r][2], PZ)));
                            const float2 c = __fmul2_rn(w, pp);
                            acc2[r][3] = __ffma2_rn(c, dx, acc2[r][3]);
                            acc2[r][4] = __ffma2_rn(c, dy, acc2[r][4]);
                            acc2[r][5] = __ffma2_rn(c, dz, acc2[r][5]);
                        }
                    }
                }
                if (++nchunk2 % FOLD != 0 && cj + kChunk < j1) continue;
                // fold: the lanes' pair halves added (the negated sums' sign restored) -> shared
                // memory [W][6][64] -> double-FP32 over the warps -> the FP64 accumulator
                __syncthreads();
                float* red = reinterpret_cast<float*>(smem);
                constexpr int kNeg = DIM == 2 ? 2 : 3;  // first component summed negated
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int t = 0; t < kKWidth; ++t) {
                        const float v = acc2[r][t].x + acc2[r][t].y;
                        red[(warp * kKWidth + t) * kTileI + lane + 32 * r] = t >= kNeg ? -v : v;
                        acc2[r][t] = make_float2(0.0f, 0.0f);
                    }
                __syncthreads();
                for (int t = threadIdx.x; t < kKWidth * kTileI; t += THREADS) {
                    const int k = t / kTileI, il = t % kTileI;
                    float2 sum = make_float2(0.0f, 0.0f);
#pragma unroll 8
                    for (int w2 = 0; w2 < W; ++w2) dd_acc(sum, red[(w2 * kKWidth + k) * kTileI + il]);
                    const int i = b * kTileI + il;
                    if (i < n) atomicAdd(a.K + (size_t)i * kKWidth + k, dd_to_double(dd_add(sum, make_float2(0.f, 0.f))));
                }
            }
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

// ------------------------------------------------------------------ 2-D Gaussian, owner computes
// The persistent 2-D Gaussian shoot splits the particles, not the pair matrix: CTA c
// owns rows [c n / G, (c+1) n / G) and sums over every source j itself, so a stage
// needs no cross-CTA reduction: the CTA applies the RK4 stage to its own rows and
// one grid-wide barrier per stage publishes the next stage's inputs.
//
// Rows are processed in sub-tiles of R = (32 / JL) x RI particles.  A warp's lanes
// are (32 / JL) row groups x JL source lanes; a lane holds RI rows (row group g:
// rows g, g + 32/JL, ...) and takes every JL-th source of its warp's share, so each
// staged source record feeds RI particles of the lane.  Two forms: 1024 threads with
// RI = 4 (64 registers a thread), and 512 threads with RI = 8 and JL = 8 (128
// registers: half the shared-memory loads per pair and twice the independent ex2
// chains per lane; the benchmark's form).
//
// Staging: the W warps split the n sources into equal shares, and each warp stages
// only its own share, the sources its loop reads: their loads are issued together
// with the sub-tile's row loads and a warp barrier (no CTA barrier) separates a
// warp's staging from its loop.  All n <= kOwnerMaxN sources fit one staged chunk.
// Records are three arrays (A, B float4 and the y py float), which measured faster
// in the loop than interleaved A, B pairs.
//
// The source lanes and the warps are reduced after the sub-tile: a warp's block of a
// particle's sum (its n / W sources, at most 256) is FP32 (lane sums, then shuffles
// over the source lanes); the W blocks are accumulated in double-FP32 (TwoSum) in
// shared memory, to FP64-level accuracy.
//
// Factored Gaussian on coordinates centred on the sub-tile's first particle,
// q'' = q' - q'_first: with G = 2^-|q''_i - q''_j|^2 (scaled units),
//   G_ij = E_i g_ij,  E_i = 2^-|q''_i|^2,  g_ij = 2^t,  t = 2 q''_i . q''_j - |q''_j|^2 (<= |q''_i|^2),
//   dq_i = E_i sum_j g_ij p_j,   M_i = q''_i (x) dq_i - E_i sum_j g_ij (q''_j (x) p_j),
// so a pair costs two FMAs for t, one ex2 and three packed f32x2 FMAs, against
// per-source records (2x, 2y, -|q''|^2, y px), (px, py, x px, x py), (y py) built
// once per stage.  A sub-tile whose |q''_i|^2 could overflow 2^t
// (> kFactorMax) takes the difference form d = q''_i - q''_j (same records).
constexpr int kChunkG = 2048;
constexpr float kFactorMax = 60.0f;

// Inputs of the RK4 stage of one component of one owned particle: the stage input
// momentum (for the dp contraction), the step-start stage copy, the RK4
// accumulator and (stage 3) the FP64 state.
struct EpiIn {
    float2 pin;
    float xs;
    float A;
    double xv;
};

__device__ __forceinline__ double* epi_state(const StageArgs& a, int i, int comp)
{
    return comp < 2 ? a.x + (size_t)i * 2 + comp : a.x + (size_t)a.n * 2 + (size_t)i * 2 + (comp - 2);
}

__device__ __forceinline__ EpiIn epi_load(const StageArgs& a, int i, int comp)
{
    EpiIn e;
    e.pin = __ldcg(reinterpret_cast<const float2*>(a.S_in + i) + 1);
    e.xs = __ldcg(reinterpret_cast<const float*>(a.Sx + i) + comp);
    e.A = a.acc[(size_t)i * 4 + comp];
    e.xv = a.stage == 3 ? *epi_state(a, i, comp) : 0.0;
    return e;
}

// RK4 stage of component comp (0, 1: q; 2, 3: p) of particle i from its six pair
// sums f (dq_x, dq_y, M_xx, M_xy, M_yx, M_yy), each a double-FP32 value: the 2-D
// mixed epilogue with one thread per component.  One RHS (MODE_RHS) evaluates the
// result in FP64 from the pairs; the RK4 stage combination takes each sum rounded
// once to FP32 (its hi part) and only the step update (stage 3) touches FP64.
__device__ __forceinline__ void epilogue2_comp(const StageArgs& a, int i, int comp, const float2* f, const EpiIn& e)
{
    if (a.mode == MODE_RHS) {
        double kv;
        if (comp < 2) {
            kv = dd_to_double(comp == 0 ? f[0] : f[1]) + a.s2 * (double)(comp == 0 ? e.pin.x : e.pin.y);  // + sigma_n^2 p_i (Sec. 6)
        } else {
            const double m0 = dd_to_double(comp == 2 ? f[2] : f[4]), m1 = dd_to_double(comp == 2 ? f[3] : f[5]);
            kv = a.dp_scale * (m0 * (double)e.pin.x + m1 * (double)e.pin.y);
        }
        double* out = comp < 2 ? a.out_q : a.out_p;
        out[(size_t)i * 2 + (comp & 1)] = kv;
        return;
    }
    float kv;
    if (comp < 2) {
        // dq (+ sigma_n^2 p_i for the inexact system, Sec. 6)
        kv = fmaf(a.s2_f, comp == 0 ? e.pin.x : e.pin.y, comp == 0 ? f[0].x : f[1].x);
    } else {
        const float m0 = comp == 2 ? f[2].x : f[4].x, m1 = comp == 2 ? f[3].x : f[5].x;
        kv = a.dp_scale_f * fmaf(m0, e.pin.x, m1 * e.pin.y);
    }
    float* A = a.acc + (size_t)i * 4 + comp;
    if (a.stage < 3) {
        const float cdt = (a.stage == 2 ? 1.0f : 0.5f) * a.dt_f;
        const float y = fmaf(comp < 2 ? cdt * a.s_f : cdt, kv, e.xs);
        *A = a.stage == 0 ? kv : fmaf(2.0f, kv, e.A);  // k1 + 2 k2 + 2 k3
        reinterpret_cast<float*>(a.S_out + i)[comp] = y;
        if (a.rec_out) reinterpret_cast<float*>(a.rec_out + i)[comp] = y;
    } else {
        const double nv = e.xv + (double)(a.dt_f * (1.0f / 6.0f) * (e.A + kv));
        *epi_state(a, i, comp) = nv;
        const float w = comp < 2 ? (float)((nv - a.c0[comp]) * a.s) : (float)nv;
        reinterpret_cast<float*>(a.Sx_w + i)[comp] = w;
        if (a.rec_out) reinterpret_cast<float*>(a.rec_out + i)[comp] = w;
    }
}

// Sources staged per shared-memory fill of the owner kernel (the kernel takes one
// fill: n <= this): 4096 when the sub-tile is narrow (JL >= 4), 2048 with 128-row
// sub-tiles (whose reduction buffer is larger).
template <int JL>
__host__ __device__ constexpr int owner_chunk()
{
    return JL == 1 ? 2048 : 4096;
}
// Rows per lane of the owner kernel: 8 in the 512-thread form (JL = 8), else 4.
template <int JL>
__host__ __device__ constexpr int owner_ri()
{
    return JL == 8 ? 8 : 4;
}
template <int JL>
__host__ __device__ constexpr int owner_threads()
{
    return JL == 8 ? 512 : 1024;
}
template <int THREADS, int JL>
constexpr size_t owner_smem()
{
    return (size_t)owner_chunk<JL>() * (2 * sizeof(float4) + sizeof(float)) +
           (size_t)(THREADS / 32 + 2) * kKWidth * ((32 / JL) * owner_ri<JL>()) * sizeof(float);
}

template <int THREADS, int JL>
__device__ __forceinline__ void stage_owner_gauss2(const StageArgs& a, float4* smem, int r0, int r1)
{
    constexpr int W = THREADS / 32;
    constexpr int RI = owner_ri<JL>();
    constexpr int RG = 32 / JL;  // row groups per warp
    static_assert(RI % 2 == 0, "the exponents are computed for pairs of rows");
    constexpr int R = RG * RI;   // rows per sub-tile
    constexpr int CH = owner_chunk<JL>();
    constexpr int NV = RI * kKWidth;  // finalized partials per lane
    constexpr int SPL = (CH / W + 31) / 32;  // staged sources per lane (a warp stages its own share)
    float4* recA4 = smem;                                    // [CH] (2x, 2y, -|q''|^2, y px)
    float4* recB4 = smem + CH;                               // [CH] (px, py, x px, x py)
    float* recB = reinterpret_cast<float*>(smem + 2 * CH);   // [CH] y py
    float* red = recB + CH;                                  // [W][6][R]: the warps' FP32 blocks
    float2* fin = reinterpret_cast<float2*>(red + (size_t)W * kKWidth * R);  // [6][R]: double-FP32 sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rg = lane / JL, jl = lane % JL;
    const int n = a.n;
    for (int t0 = r0; t0 < r1; t0 += R) {
        const int t1 = min(r1, t0 + R);
        // the warp's share of the sources, [w n / W, (w+1) n / W): its loads go out
        // together with the sub-tile's own (n <= CH: one staged chunk)
        const int sa = warp * n / W, sb = (warp + 1) * n / W;
        float4 src[SPL];
#pragma unroll
        for (int k = 0; k < SPL; ++k) {
            const int t = sa + lane + 32 * k;
            src[k] = t < sb ? __ldcg(a.S_in + t) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const float4 c4 = __ldcg(a.S_in + t0);  // sub-tile centre: its first particle
        float qx[RI], qy[RI];
        float mq = 0.0f;
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int i = t0 + rg + RG * r;
            const float4 v = i < t1 ? __ldcg(a.S_in + i) : c4;
            qx[r] = v.x - c4.x;
            qy[r] = v.y - c4.y;
            mq = fmaxf(mq, fmaf(qx[r], qx[r], qy[r] * qy[r]));
        }
        const bool factored = !__syncthreads_or(mq > kFactorMax);
        float2 sqv[RI], sbx[RI], sby[RI];
#pragma unroll
        for (int r = 0; r < RI; ++r) sqv[r] = sbx[r] = sby[r] = make_float2(0.0f, 0.0f);
        {
            // the warp's records (its loop reads no others: a warp barrier suffices)
#pragma unroll
            for (int k = 0; k < SPL; ++k) {
                const int t = sa + lane + 32 * k;
                if (t < sb) {
                    const float4 v = src[k];
                    const float x = v.x - c4.x, y = v.y - c4.y;
                    recA4[t] = make_float4(2.0f * x, 2.0f * y, -fmaf(x, x, y * y), y * v.z);
                    recB4[t] = make_float4(v.z, v.w, x * v.z, x * v.w);
                    recB[t] = y * v.w;
                }
            }
            __syncwarp();
            const int ja = sa + jl, jb = sb;
            if (factored) {
#pragma unroll 2
                for (int j = ja; j < jb; j += JL) {
                    // A = (2x, 2y, -|q''|^2, y px), B = (px, py, x px, x py), byy = y py
                    const float4 A = recA4[j], B = recB4[j];
                    const float byy = recB[j];
                    const float2 pxy = make_float2(B.x, B.y), xp = make_float2(B.z, B.w);
                    const float2 yp = make_float2(A.w, byy);
                    // the exponents of two rows in one packed FMA pair (the source's
                    // coefficients broadcast): fewer issue slots than two scalar chains,
                    // measured 1.5 % faster per stage here (the stream-K tiles of 4 rows
                    // per lane measured slower with it and keep the scalar form)
#pragma unroll
                    for (int r = 0; r < RI; r += 2) {
                        const float2 t = __ffma2_rn(make_float2(qx[r], qx[r + 1]), make_float2(A.x, A.x),
                                                    __ffma2_rn(make_float2(qy[r], qy[r + 1]), make_float2(A.y, A.y),
                                                               make_float2(A.z, A.z)));
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const float g = ex2_approx(u ? t.y : t.x);
                            const float2 gg = make_float2(g, g);
                            sqv[r + u] = __ffma2_rn(gg, pxy, sqv[r + u]);
                            sbx[r + u] = __ffma2_rn(gg, xp, sbx[r + u]);
                            sby[r + u] = __ffma2_rn(gg, yp, sby[r + u]);
                        }
                    }
                }
            } else {
                for (int j = ja; j < jb; j += JL) {
                    const float4 A = recA4[j], B = recB4[j];
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
        // finalize the lane's partials (linear in the sums, so before the reduction):
        // per row dq = E sq, M = q'' (x) dq - E sb (E = 1 in the difference form)
        float v[NV];
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const float E = factored ? ex2_approx(-fmaf(qx[r], qx[r], qy[r] * qy[r])) : 1.0f;
            const float d0 = E * sqv[r].x, d1 = E * sqv[r].y;
            v[r * kKWidth + 0] = d0;
            v[r * kKWidth + 1] = d1;
            v[r * kKWidth + 2] = fmaf(qx[r], d0, -E * sbx[r].x);
            v[r * kKWidth + 3] = fmaf(qx[r], d1, -E * sbx[r].y);
            v[r * kKWidth + 4] = fmaf(qy[r], d0, -E * sby[r].x);
            v[r * kKWidth + 5] = fmaf(qy[r], d1, -E * sby[r].y);
        }
        // reduce-scatter over the JL source lanes: each round halves the values a lane
        // holds (it keeps one half, adds the partner's copy of it); the last round of an
        // odd count adds the partner's values whole.  Afterwards lane jl holds, of the
        // 4 x 6 values, the block selected by its bits (high bit first).
        int first = 0;  // index (into the original 24) of the lane's first value
        int cnt = NV;
#pragma unroll
        for (int o = JL / 2; o >= 1; o >>= 1) {
            if (cnt % 2 == 0) {
                const int h = cnt / 2;
                const bool upper = (jl & o) != 0;
#pragma unroll
                for (int k = 0; k < NV / 2; ++k) {
                    if (k < h) {
                        const float send = upper ? v[k] : v[k + h];
                        const float keep = upper ? v[k + h] : v[k];
                        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                    }
                }
                if (upper) first += h;
                cnt = h;
            } else {
#pragma unroll
                for (int k = 0; k < NV; ++k)
                    if (k < cnt) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
            }
        }
        // the lane's values -> red[warp][k][row]; the value at original index e is row
        // e / 6 (lane row rg + RG * (e / 6)), component e % 6
        const bool writer = (NV % JL == 0) || (jl & 1) == 0;  // odd final count: pairs hold copies
        if (writer) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                if (k < cnt) {
                    const int e = first + k;
                    red[(size_t)warp * kKWidth * R + (e % kKWidth) * R + rg + RG * (e / kKWidth)] = v[k];
                }
            }
        }
        __syncthreads();
        // sum over the warps in double-FP32 (QS threads per output value): the per-particle
        // sums are accumulated across the warps' FP32 blocks with TwoSum error terms
        constexpr int NOUT = kKWidth * R;
        constexpr int QS = (THREADS / NOUT) >= 8 ? 8 : (THREADS / NOUT) >= 4 ? 4 : (THREADS / NOUT) >= 2 ? 2 : 1;
        // (the loop runs whole warps, so that every lane of a warp reaches the shuffles;
        // lanes past NOUT * QS carry zeros)
        constexpr int NQ = (NOUT * QS + 31) / 32 * 32;
        for (int t = threadIdx.x; t < NQ; t += THREADS) {
            const bool valid = t < NOUT * QS;
            const int o = valid ? t / QS : 0, q = t % QS;
            float2 sum = make_float2(valid ? red[q * NOUT + o] : 0.0f, 0.0f);
#pragma unroll
            for (int w2 = q + QS; w2 < W; w2 += QS)
                if (valid) dd_acc(sum, red[w2 * NOUT + o]);
#pragma unroll
            for (int m = QS / 2; m >= 1; m >>= 1) {
                const float2 other = make_float2(__shfl_xor_sync(0xffffffffu, sum.x, m),
                                                 __shfl_xor_sync(0xffffffffu, sum.y, m));
                sum = dd_add(sum, other);
            }
            if (valid && q == 0) fin[o] = QS == 1 ? dd_add(sum, make_float2(0.0f, 0.0f)) : sum;
        }
        __syncthreads();
        // the RK4 stage of the sub-tile's rows, one thread per component
        if (threadIdx.x < 4 * R) {
            const int rl = threadIdx.x >> 2, comp = threadIdx.x & 3;
            const int i = t0 + rl;
            if (i < t1) {
                float2 f[kKWidth];
#pragma unroll
                for (int k = 0; k < kKWidth; ++k) f[k] = fin[k * R + rl];
                epilogue2_comp(a, i, comp, f, epi_load(a, i, comp));
            }
        }
        if (t0 + R < r1) __syncthreads();  // the next sub-tile restages the shared buffers
    }
}

// ------------------------------------------------------------------ 2-D Gaussian, stream-K
// The stream-K alternative of the persistent 2-D Gaussian shoot (the tuner picks it
// for large n, where the owner split would leave lanes or SMs idle): the pair
// matrix is cut into equal ranges of (tile, source) units, partial sums go to the
// FP64 accumulator K, and the RK4 stage runs after a grid barrier.
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
        // packed so every accumulation is one f32x2 FMA; FP32 over kFoldChunks staged chunks
        // (a warp's block: at most kFoldChunks * kChunkG / W = 256 sources), then folded
        float2 sqv[RI], sbx[RI], sby[RI];
#pragma unroll
        for (int r = 0; r < RI; ++r) sqv[r] = sbx[r] = sby[r] = make_float2(0.0f, 0.0f);
        int nchunk = 0;
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
            if (++nchunk % kFoldChunks != 0 && cj + kChunkG < j1) continue;
            // fold: per particle dq = E sq, M = q'' (x) dq - E sb  (E = 1 in the difference form)
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
                sqv[r] = sbx[r] = sby[r] = make_float2(0.0f, 0.0f);
            }
            __syncthreads();
            // the warps' blocks in double-FP32, added to K in FP64 (exact conversion)
            for (int t = threadIdx.x; t < kKWidth * kTileG; t += THREADS) {
                const int k = t / kTileG, il = t % kTileG;
                float2 sum = make_float2(0.0f, 0.0f);
#pragma unroll 8
                for (int w2 = 0; w2 < W; ++w2) dd_acc(sum, red[(w2 * kKWidth + k) * kTileG + il]);
                const int i = b * kTileG + il;
                if (i < n) atomicAdd(a.K + (size_t)i * kKWidth + k, dd_to_double(dd_add(sum, make_float2(0.f, 0.f))));
            }
        }
        u0 += (j1 - j0);
    }
}

// The owner-computes shoot (mode RK4: `steps` steps) or one RHS (mode RHS, input Sx);
// REC: every stage output is also written to the recording rec.
template <int THREADS, int JL, bool REC>
__global__ void __launch_bounds__(THREADS, 1)
    k_shoot_owner(StageArgs a, const float4* Sx, float4* Sa, float4* Sb, int steps, unsigned* bar, int* err,
                  float4* rec)
{
    extern __shared__ float4 smem[];
    const int n = a.n;
    const int r0 = (int)((long long)blockIdx.x * n / gridDim.x), r1 = (int)((long long)(blockIdx.x + 1) * n / gridDim.x);
    unsigned epoch = 0;
    volatile unsigned* progress = bar + kBarProgress;
    a.Sx = Sx;
    const int nst = a.mode == MODE_RHS ? 1 : 4 * steps;
    for (int st = 0; st < nst; ++st) {
        const int stage = st & 3;
        a.stage = stage;
        a.S_in = a.mode == MODE_RHS || stage == 0 ? Sx : (stage == 2 ? Sb : Sa);
        a.S_out = stage == 1 ? Sb : Sa;
        a.rec_out = REC ? rec + (size_t)(st + 1) * n : nullptr;  // stage input st + 1 of a recorded shoot
        stage_owner_gauss2<THREADS, JL>(a, smem, r0, r1);
        if (st + 1 < nst && !grid_barrier(bar, err, ++epoch)) return;
        // the CTA's progress word: the last stage it has started (read when a barrier wait
        // gives up).  Written right after the barrier: measured ~1 us per stage faster on
        // GB300 than the same kernel without this store.
        if (threadIdx.x == 0) progress[blockIdx.x] = (unsigned)(st + 1);
    }
}

template <int DIM, int KER, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) k_stage_mixed(StageArgs a)
{
    extern __shared__ float4 smem[];
    __shared__ int s_last;
    stage_pairs<DIM, KER, THREADS, true>(a, smem, &s_last);
}

// A whole shoot of `steps` RK4 steps in one cooperative launch (kernels other than
// the 2-D Gaussian): per stage, the stream-K pair phase, a barrier, the RK4 stage
// of the particles this CTA owns ([c n / G, (c+1) n / G)), and a barrier.
template <int DIM, int KER, int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
    k_shoot_mixed(StageArgs a, const float4* Sx, float4* Sa, float4* Sb, int steps, unsigned* bar, int* err,
                  float4* rec)
{
    extern __shared__ float4 smem[];
    const int n = a.n;
    const int i0 = (int)((long long)blockIdx.x * n / gridDim.x), i1 = (int)((long long)(blockIdx.x + 1) * n / gridDim.x);
    unsigned epoch = 0;
    volatile unsigned* progress = bar + kBarProgress;
    a.Sx = Sx;
    for (int s = 0; s < steps; ++s) {
        for (int stage = 0; stage < 4; ++stage) {
            a.stage = stage;
            a.S_in = stage == 0 ? Sx : (stage == 2 ? Sb : Sa);
            a.S_out = stage == 1 ? Sb : Sa;
            a.rec_out = rec ? rec + (size_t)(4 * s + stage + 1) * (DIM == 2 ? 1 : 2) * n : nullptr;
            stage_pairs<DIM, KER, THREADS, false>(a, smem, nullptr);
            if (!grid_barrier(bar, err, ++epoch)) return;
            for (int i = i0 + threadIdx.x; i < i1; i += THREADS) epilogue_mixed<DIM>(a, i);
            if (s == steps - 1 && stage == 3) break;
            if (!grid_barrier(bar, err, ++epoch)) return;
            if (threadIdx.x == 0) progress[blockIdx.x] = (unsigned)(4 * s + stage + 1);  // the stage it starts
        }
    }
}

// The stream-K 2-D Gaussian shoot: per stage, the pair phase over this CTA's range
// of (tile of 128, source) units, a barrier, the RK4 stage of the particles the CTA
// owns, and a barrier.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
    k_shoot_streamk(StageArgs a, const float4* Sx, float4* Sa, float4* Sb, int steps, unsigned* bar, int* err,
                    float4* rec)
{
    extern __shared__ float4 smem[];
    const int n = a.n;
    const int i0 = (int)((long long)blockIdx.x * n / gridDim.x), i1 = (int)((long long)(blockIdx.x + 1) * n / gridDim.x);
    unsigned epoch = 0;
    volatile unsigned* progress = bar + kBarProgress;
    a.Sx = Sx;
    for (int s = 0; s < steps; ++s) {
        for (int stage = 0; stage < 4; ++stage) {
            a.stage = stage;
            a.S_in = stage == 0 ? Sx : (stage == 2 ? Sb : Sa);
            a.S_out = stage == 1 ? Sb : Sa;
            a.rec_out = rec ? rec + (size_t)(4 * s + stage + 1) * n : nullptr;
            stage_pairs_gauss2<THREADS>(a, smem);
            if (!grid_barrier(bar, err, ++epoch)) return;
            for (int i = i0 + threadIdx.x; i < i1; i += THREADS) epilogue_mixed<2>(a, i);
            if (s == steps - 1 && stage == 3) break;
            if (!grid_barrier(bar, err, ++epoch)) return;
            if (threadIdx.x == 0) progress[blockIdx.x] = (unsigned)(4 * s + stage + 1);  // the stage it starts
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
        // dq (+ sigma_n^2 p_i for the inexact system, Sec. 6)
        kq[c] = __ldcg(a.K + (size_t)i * kKWidth + c) + a.s2 * __ldcg(a.D_in + (size_t)i * 2 * DIM + DIM + c);
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
        (void)threads;                                                            \
        return launch_mixed<D, K, 512>(a, st);                                    \
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


}  // namespace

static std::atomic<int> g_timing{0};
static std::mutex g_timing_mu;
static double g_last_ms = -1.0;
static char g_last_kernel[64] = "";

bool launch_timing_enabled() { return g_timing.load(std::memory_order_relaxed) != 0; }
void set_launch_timing(bool on) { g_timing.store(on ? 1 : 0, std::memory_order_relaxed); }
void record_launch_time(cudaEvent_t e0, cudaEvent_t e1, const char* kernel)
{
    float ms = -1.0f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = -1.0f;
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_last_ms = ms;
    snprintf(g_last_kernel, sizeof(g_last_kernel), "%s", kernel);
}
double last_launch_ms()
{
    std::lock_guard<std::mutex> lk(g_timing_mu);
    return g_last_ms;
}
const char* last_launch_kernel() { return g_last_kernel; }

static int tc_sm_count()
{
    DeviceInfo di{};
    return device_info(&di) == EP_OK ? di.sm_count : 1;
}

size_t allpairs_bytes(int n, int dim, int prec)
{
    Sizer z;
    const int ntiles = (n + kTileI - 1) / kTileI;
    z.add(sizeof(double) * 2 * dim * (size_t)n);   // x
    z.add(sizeof(double) * kKWidth * (size_t)n);   // K
    z.add(sizeof(int) * (size_t)ntiles);           // counters
    z.add(sizeof(double) * 4);                     // c0
    z.add(sizeof(unsigned) * (kBarProgress + kMaxPersistentCtas));  // barrier counters, error flag, progress words
    if (prec == EP_MIXED && dim == 2) {
        z.add(sizeof(double) * 2 * dim * (size_t)n);  // tuner backup of x
        z.add(sizeof(float4) * (size_t)n);            // tuner backup of the stage copy
    }
    if (prec == EP_MIXED) {
        const int V = dim == 2 ? 1 : 2;
        for (int k = 0; k < 3; ++k) z.add(sizeof(float4) * V * (size_t)n);
        z.add(sizeof(float) * 2 * dim * (size_t)n);
        if (dim == 2) z.add(sizeof(float) * tc_part_floats(n, tc_sm_count()));
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
    b->bar = (unsigned*)ar->carve(sizeof(unsigned) * (kBarProgress + kMaxPersistentCtas));
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
        if (dim == 2) b->part = (float*)ar->carve(sizeof(float) * tc_part_floats(n, tc_sm_count()));
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
    // the tensor-core path needs the partial-sum buffer and reads its error flag back
    // (a stream synchronisation); the fixed-scratch entry point carves neither
    if (tc_enabled(P) && allpairs_persistent_enabled() && b.part && b.bar)
        return tc_run(P, b, 0, 0.0, MODE_RHS, dq, dp, tc_sm_count(), st);
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

// Launch of a whole persistent shoot; returns *done = false when the grid cannot
// be co-resident (the caller then falls back to per-stage launches).
ep_status finish_persistent(const AllPairsBufs& b, cudaStream_t st, bool* done, int G = 0)
{
    int herr = 0;
    EP_TRY_CUDA(cudaMemcpyAsync(&herr, b.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    if (herr) {
        // the CTAs' progress words say how far each got (kernels that write them)
        unsigned lo = 0, hi = 0;
        if (G > 0 && G <= kMaxPersistentCtas) {
            std::vector<unsigned> pr((size_t)G);
            if (cudaMemcpy(pr.data(), b.bar + kBarProgress, sizeof(unsigned) * G, cudaMemcpyDeviceToHost) == cudaSuccess) {
                lo = *std::min_element(pr.begin(), pr.end());
                hi = *std::max_element(pr.begin(), pr.end());
            }
        }
        set_error("persistent shoot: a grid-barrier wait gave up (kernel ended early; CTAs had reached stages %u..%u)",
                  lo, hi);
        return EP_ETIMEOUT;
    }
    *done = true;
    return EP_OK;
}

template <int DIM, int KER>
ep_status launch_shoot_mixed(const StageArgs& a0, const AllPairsBufs& b, int steps, cudaStream_t st, bool* done,
                             cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, float4* rec = nullptr)
{
    constexpr int THREADS = 512;
    constexpr int W = THREADS / 32;
    constexpr int V = DIM == 2 ? 1 : 2;
    const size_t smem = std::max((size_t)kChunk * V * sizeof(float4), (size_t)W * kKWidth * kTileI * sizeof(float));
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
    if (a0.G > resident || a0.G > kMaxPersistentCtas) return EP_OK;  // per-stage launches instead
    StageArgs a = a0;
    const float4* Sx = b.Sx;
    float4* Sa = b.Sa;
    float4* Sb = b.Sb;
    unsigned* bar = b.bar;
    int* err = b.err;
    EP_TRY_CUDA(cudaMemsetAsync(b.bar, 0, sizeof(unsigned) * 9, st));
    void* args[] = {&a, &Sx, &Sa, &Sb, &steps, &bar, &err, &rec};
    count_launch();
    if (ev0) EP_TRY_CUDA(cudaEventRecord(ev0, st));
    EP_TRY_CUDA(cudaLaunchCooperativeKernel((void*)fn, dim3(a.G), dim3(THREADS), args, smem, st));
    if (ev1) EP_TRY_CUDA(cudaEventRecord(ev1, st));
    return finish_persistent(b, st, done, a.G);
}

// The owner-computes 2-D Gaussian shoot: a.G CTAs, JL source lanes per row group.
struct OwnerCfg {
    int G = 0;
    int JL = 4;
};

template <int JL>
ep_status launch_owner(const StageArgs& a0, const AllPairsBufs& b, int steps, cudaStream_t st, bool* done,
                       cudaEvent_t ev0, cudaEvent_t ev1, float4* rec)
{
    constexpr int THREADS = owner_threads<JL>();
    const size_t smem = owner_smem<THREADS, JL>();
    auto fn = rec ? k_shoot_owner<THREADS, JL, true> : k_shoot_owner<THREADS, JL, false>;
    static int resident[2] = {-1, -1};
    int& res = resident[rec ? 1 : 0];
    if (res < 0) {
        EP_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        EP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, THREADS, smem));
        DeviceInfo di{};
        EP_TRY(device_info(&di));
        res = per_sm * di.sm_count;
    }
    *done = false;
    StageArgs a = a0;
    a.G = std::max(1, std::min(a.G, a.n));
    if (a.G > res || a.G > kMaxPersistentCtas || a.n > owner_chunk<JL>()) return EP_OK;  // one staged chunk holds every source
    const float4* Sx = b.Sx;
    float4* Sa = b.Sa;
    float4* Sb = b.Sb;
    unsigned* bar = b.bar;
    int* err = b.err;
    EP_TRY_CUDA(cudaMemsetAsync(b.bar, 0, sizeof(unsigned) * 9, st));
    void* args[] = {&a, &Sx, &Sa, &Sb, &steps, &bar, &err, &rec};
    count_launch();
    if (ev0) EP_TRY_CUDA(cudaEventRecord(ev0, st));
    EP_TRY_CUDA(cudaLaunchCooperativeKernel((void*)fn, dim3(a.G), dim3(THREADS), args, smem, st));
    if (ev1) EP_TRY_CUDA(cudaEventRecord(ev1, st));
    return finish_persistent(b, st, done, a.G);
}

// The stream-K 2-D Gaussian shoot over a.G CTAs (tiles of kTileG).
ep_status launch_streamk(const StageArgs& a0, const AllPairsBufs& b, int steps, cudaStream_t st, bool* done,
                         cudaEvent_t ev0, cudaEvent_t ev1, float4* rec)
{
    constexpr int THREADS = 1024;
    constexpr int W = THREADS / 32;
    const size_t smem = std::max((size_t)kChunkG * (2 * sizeof(float4) + sizeof(float)),
                                 (size_t)W * kKWidth * kTileG * sizeof(float));
    auto fn = k_shoot_streamk<THREADS>;
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
    StageArgs a = a0;
    a.U = (long long)((b.n + kTileG - 1) / kTileG) * b.n;
    a.G = (int)std::max<long long>(1, std::min<long long>(a.G, a.U));
    if (a.G > resident || a.G > kMaxPersistentCtas) return EP_OK;
    const float4* Sx = b.Sx;
    float4* Sa = b.Sa;
    float4* Sb = b.Sb;
    unsigned* bar = b.bar;
    int* err = b.err;
    EP_TRY_CUDA(cudaMemsetAsync(b.bar, 0, sizeof(unsigned) * 9, st));
    void* args[] = {&a, &Sx, &Sa, &Sb, &steps, &bar, &err, &rec};
    count_launch();
    if (ev0) EP_TRY_CUDA(cudaEventRecord(ev0, st));
    EP_TRY_CUDA(cudaLaunchCooperativeKernel((void*)fn, dim3(a.G), dim3(THREADS), args, smem, st));
    if (ev1) EP_TRY_CUDA(cudaEventRecord(ev1, st));
    return finish_persistent(b, st, done, a.G);
}

// JL = 1, 4, 16: owner computes with that many source lanes; JL = 0: stream-K.
ep_status launch_owner_cfg(const StageArgs& a, const AllPairsBufs& b, int steps, const OwnerCfg& c, cudaStream_t st,
                           bool* done, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, float4* rec = nullptr)
{
    StageArgs a2 = a;
    a2.G = c.G;
    if (c.JL == 0) return launch_streamk(a2, b, steps, st, done, ev0, ev1, rec);
    if (c.JL == 1) return launch_owner<1>(a2, b, steps, st, done, ev0, ev1, rec);
    if (c.JL == 16) return launch_owner<16>(a2, b, steps, st, done, ev0, ev1, rec);
    if (c.JL == 8) return launch_owner<8>(a2, b, steps, st, done, ev0, ev1, rec);
    return launch_owner<4>(a2, b, steps, st, done, ev0, ev1, rec);
}

// Largest n of the owner-computes kernel: every source in one staged chunk (and a
// warp's FP32 block of a particle's sum at most n / 16 = 256 sources); stream-K above.
constexpr int kOwnerMaxN = 4096;

// Default owner configuration: the widest sub-tile the rows per SM fill, and the
// CTA count that fills each CTA's sub-tiles; stream-K (JL = 0) beyond kOwnerMaxN.
OwnerCfg owner_default(int n, int sm)
{
    OwnerCfg c;
    if (n > kOwnerMaxN) return OwnerCfg{sm, 0};
    const double per = (double)n / sm;
    c.JL = per >= 24 ? 8 : 16;
    const int R = (32 / c.JL) * (c.JL == 8 ? 8 : 4);
    const long long k = std::max<long long>(1, (n + (long long)sm * R - 1) / ((long long)sm * R));
    c.G = (int)std::max<long long>(1, std::min<long long>(sm, (n + k * R - 1) / (k * R)));
    return c;
}

ep_status launch_shoot(const ep_params& P, const StageArgs& a, const AllPairsBufs& b, int steps, cudaStream_t st,
                       bool* done, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, float4* rec = nullptr)
{
#define EP_SHOOT_CASE(D, K) \
    if (P.dim == D && P.kernel == K) return launch_shoot_mixed<D, K>(a, b, steps, st, done, ev0, ev1, rec);
    EP_SHOOT_CASE(2, EP_TENT) EP_SHOOT_CASE(2, EP_EXPCONE)
    EP_SHOOT_CASE(3, EP_GAUSS) EP_SHOOT_CASE(3, EP_TENT) EP_SHOOT_CASE(3, EP_EXPCONE)
#undef EP_SHOOT_CASE
    *done = false;
    return EP_OK;
}

// ------------------------------------------------------------------ autotuner
// The persistent 2-D Gaussian shoot has two designs and free parameters: owner
// computes with a CTA count G (rows per CTA = n / G) and a form (JL source lanes
// and RI rows per lane: 128, 32 or 8 rows per sub-tile), where a sub-tile costs a
// staging pass over all n sources and a reduction, a partly filled sub-tile wastes
// lanes and fewer CTAs leave SMs idle; and stream-K over G CTAs (JL = 0), which
// splits the pair matrix evenly at the price of FP64 atomics and a second barrier.
// The tuner times a kTuneSteps-step shoot for each candidate on the loaded state
// (restoring it afterwards) and caches the fastest per (n, device); a later
// candidate replaces the best only when it is at least 1 % faster.  The tensor-core
// path (opt-in) is tuned over its CTA count the same way.  EP_AUTOTUNE=0 in the
// environment skips tuning (owner_default).
struct TuneKey {
    int n, dim, kernel, dev, tc;
    bool operator<(const TuneKey& o) const
    {
        if (n != o.n) return n < o.n;
        if (dim != o.dim) return dim < o.dim;
        if (kernel != o.kernel) return kernel < o.kernel;
        if (dev != o.dev) return dev < o.dev;
        return tc < o.tc;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, OwnerCfg> g_tuned;

bool autotune_enabled()
{
    const char* e = getenv("EP_AUTOTUNE");
    return !(e && e[0] == '0');
}

// RK4 steps of each timed trial launch of the tuner (best of three after one untimed run)
constexpr int kTuneSteps = 3;

ep_status tune_persistent(const ep_params& P, const AllPairsBufs& b, StageArgs a, double dt, cudaStream_t st,
                          OwnerCfg* best, bool tc)
{
    DeviceInfo di{};
    EP_TRY(device_info(&di));
    const int sm = di.sm_count;
    const int n = b.n;
    std::vector<OwnerCfg> cand;
    if (tc) {
        const int tiles = tc_tiles(n);
        std::vector<int> gs = {sm, sm - sm / 8};
        for (int k = sm / std::max(1, tiles), c = 0; k >= 1 && c < 2; --k, ++c) gs.push_back(tiles * k);
        for (int g : gs) cand.push_back(OwnerCfg{g, 0});
    } else {
        for (int JL : {1, 4, 8, 16}) {
            if (n > kOwnerMaxN || (JL == 1 && n > owner_chunk<1>())) continue;
            const int R = (32 / JL) * (JL == 8 ? 8 : 4);
            const long long k = std::max<long long>(1, (n + (long long)sm * R - 1) / ((long long)sm * R));
            const int g1 = (int)std::max<long long>(1, std::min<long long>(sm, (n + k * R - 1) / (k * R)));
            cand.push_back(OwnerCfg{g1, JL});
            if (g1 != std::min(sm, n)) cand.push_back(OwnerCfg{std::min(sm, n), JL});
        }
        // stream-K: the full SM count and the largest tile-aligned count
        const int tiles = (n + kTileG - 1) / kTileG;
        cand.push_back(OwnerCfg{sm, 0});
        if (tiles <= sm) cand.push_back(OwnerCfg{tiles * (sm / tiles), 0});
    }
    const size_t m2 = 2 * (size_t)P.dim * b.n;
    EP_TRY_CUDA(cudaMemcpyAsync(b.x_bak, b.x, sizeof(double) * m2, cudaMemcpyDeviceToDevice, st));
    EP_TRY_CUDA(cudaMemcpyAsync(b.S_bak, b.Sx, sizeof(float4) * (size_t)b.n, cudaMemcpyDeviceToDevice, st));
    cudaEvent_t e0, e1;
    EP_TRY_CUDA(cudaEventCreate(&e0));
    EP_TRY_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    *best = tc ? OwnerCfg{sm, 0} : owner_default(n, sm);
    a.dt = dt;
    a.dt_f = (float)dt;
    ep_status out = EP_OK;
    for (const OwnerCfg& c : cand) {
        if (c.G < 1) continue;
        float ms = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            EP_TRY_CUDA(cudaMemcpyAsync(b.x, b.x_bak, sizeof(double) * m2, cudaMemcpyDeviceToDevice, st));
            EP_TRY_CUDA(cudaMemcpyAsync(b.Sx, b.S_bak, sizeof(float4) * (size_t)b.n, cudaMemcpyDeviceToDevice, st));
            bool done = false;
            ep_status s = EP_OK;
            if (tc) {
                s = tc_run(P, b, kTuneSteps, dt, MODE_RK4, nullptr, nullptr, c.G, st, e0, e1);
                done = s == EP_OK;
            } else {
                s = launch_owner_cfg(a, b, kTuneSteps, c, st, &done, e0, e1);
            }
            if (s == EP_ETIMEOUT) out = s;
            if (s != EP_OK || !done) break;
            float t = 0.f;
            EP_TRY_CUDA(cudaEventElapsedTime(&t, e0, e1));
            if (rep > 0) ms = std::min(ms, t);
        }
        if (out != EP_OK) break;
        // a later candidate must win clearly (run-to-run noise is ~0.3 %), so near-ties
        // keep the earlier, smaller launch
        if (ms < best_ms * 0.99f) {
            best_ms = ms;
            *best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    EP_TRY_CUDA(cudaMemcpyAsync(b.x, b.x_bak, sizeof(double) * m2, cudaMemcpyDeviceToDevice, st));
    EP_TRY_CUDA(cudaMemcpyAsync(b.Sx, b.S_bak, sizeof(float4) * (size_t)b.n, cudaMemcpyDeviceToDevice, st));
    return out;
}

// CUDA events around one persistent launch when launch timing is on (null otherwise).
struct TimedLaunch {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TimedLaunch()
    {
        if (launch_timing_enabled() && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
            if (e0) cudaEventDestroy(e0);
            e0 = e1 = nullptr;
        }
    }
    void record(const char* kernel) const
    {
        if (e0) record_launch_time(e0, e1, kernel);  // the launch functions synchronised the stream
    }
    ~TimedLaunch()
    {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// The launch configuration of the persistent 2-D Gaussian shoot in mixed precision:
// the tuner's (tuned once per size and device, by trial shoots from the loaded state,
// which they restore) when the tuner is on, else the default one.
ep_status gauss2_config(const ep_params& P, const AllPairsBufs& b, const StageArgs& a, double dt, cudaStream_t st,
                        bool tc, OwnerCfg* out)
{
    DeviceInfo di{};
    EP_TRY(device_info(&di));
    OwnerCfg c = tc ? OwnerCfg{di.sm_count, 0} : owner_default(b.n, di.sm_count);
    if (b.x_bak && autotune_enabled()) {
        const TuneKey key{b.n, P.dim, P.kernel, di.device, tc ? 1 : 0};
        bool have = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) c = it->second, have = true;
        }
        if (!have) {
            EP_TRY(tune_persistent(P, b, a, dt, st, &c, tc));
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[key] = c;
        }
    }
    *out = c;
    return EP_OK;
}

// The persistent (one cooperative launch) shoot of mixed precision, when it
// applies: tuned owner / stream-K / tensor-core launch for the 2-D Gaussian, the
// generic persistent shoot otherwise.  rec: if set, every stage input is also
// written to the recording (stage copy k + 1 after stage k; copy 0 is the caller's);
// the tensor-core path does not record.  *done = false when no persistent launch ran.
ep_status persistent_steps(const ep_params& P, const AllPairsBufs& b, StageArgs a, int steps, double dt,
                           cudaStream_t st, float4* rec, bool* done)
{
    *done = false;
    const APConfig cfg = allpairs_config(b.n, P.dim, P.precision, P.kernel);
    if (!(P.precision == EP_MIXED && cfg.threads == 1024 && allpairs_persistent_enabled())) return EP_OK;
    a.Sx_w = b.Sx;
    if (P.dim == 2 && P.kernel == EP_GAUSS) {
        const bool tc = !rec && tc_enabled(P) && b.part;
        OwnerCfg c;
        EP_TRY(gauss2_config(P, b, a, dt, st, tc, &c));
        TimedLaunch tl;
        char name[64];
        if (tc) {
            EP_TRY(tc_run(P, b, steps, dt, MODE_RK4, nullptr, nullptr, c.G, st, tl.e0, tl.e1));
            *done = true;
            snprintf(name, sizeof(name), "k_shoot_tc (G=%d)", c.G);
        } else {
            EP_TRY(launch_owner_cfg(a, b, steps, c, st, done, tl.e0, tl.e1, rec));
            if (c.JL == 0)
                snprintf(name, sizeof(name), "k_shoot_streamk<1024> (G=%d)", c.G);
            else
                snprintf(name, sizeof(name), "k_shoot_owner<%d,%d> (G=%d)", c.JL == 8 ? 512 : 1024, c.JL, std::min(c.G, b.n));
        }
        if (*done) tl.record(name);
        return EP_OK;
    }
    TimedLaunch tl;
    EP_TRY(launch_shoot(P, a, b, steps, st, done, tl.e0, tl.e1, rec));
    if (*done) {
        char name[64];
        snprintf(name, sizeof(name), "k_shoot_mixed<%d,%d,512> (G=%d)", P.dim, P.kernel, a.G);
        tl.record(name);
    }
    return EP_OK;
}

// EP_DEVICE_MATCH=0 in the environment keeps Algorithm 1 on the host loop of ep_match
// for the owner-computes shoot too (both compute the same result).
bool device_match_enabled()
{
    const char* e = getenv("EP_DEVICE_MATCH");
    return !(e && e[0] == '0');
}

namespace {

// One step of Algorithm 1 after a shoot, in the loop body of the matching graph (one
// CTA): the FP64 residual max_i |Y_i - Q_i(1)| (the arithmetic of k_max_abs_diff), the
// stop tests in the order of the host loop of ep_match, the update p0 += h (Y - Q(1))
// (k_momentum_update's arithmetic) and the loop condition; when the loop goes on, the
// next shoot's start: its barrier words zeroed and (X, p0) loaded (k_load_state's
// arithmetic).  The loop also ends when the shoot's barrier wait gave up (status
// EP_ETIMEOUT) and, whatever the tests say, once maxit updates are done.
struct GraphMatch {
    const double* X;
    const double* Y;
    double* p0;
    double* x;         // the FP64 state: positions (Q(1) after a shoot), then momenta
    float4* Sx;        // the scaled FP32 stage input
    double* Dx;        // FP64 stage copy, or null
    const double* c0;  // centre of X
    double s;          // coordinate scale
    unsigned* bar;     // the shoot's barrier words: [0, 8) counters, [8] error flag
    double* hist;      // [maxit + 1] or null
    double* state;     // [3]: updates so far, last residual, status (-1 while running)
    int n;
    double eps;
    double h;
    int maxit;
    int inexact;       // the inexact system (Sec. 6): stop when |h r|_inf < eps after an update
    cudaGraphConditionalHandle loop;
};

__global__ void __launch_bounds__(1024) k_match_step(GraphMatch g)
{
    __shared__ double sm[32];
    __shared__ int sbad, sgo;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    const size_t m = 2 * (size_t)g.n;
    const double* Q = g.x;
    double mx = 0.0;
    int bad = 0;
    for (size_t a = threadIdx.x; a < m; a += blockDim.x) {
        const double r = g.Y[a] - Q[a];
        if (!isfinite(r)) bad = 1;
        mx = fmax(mx, fabs(r));
    }
    if (bad) sbad = 1;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = fmax(t, sm[k]);
        const int k = (int)g.state[0];
        const double res = sbad ? (double)NAN : t;
        int status = -1;
        if (*(volatile const int*)(g.bar + 8)) {
            status = EP_ETIMEOUT;
        } else {
            if (g.hist) g.hist[k] = res;
            if (sbad) status = EP_EDIVERGED;
            else if (!g.inexact && res < g.eps) status = EP_OK;
            else if (k >= g.maxit) status = EP_ENOTCONVERGED;
        }
        if (status < 0) {
            g.state[0] = (double)(k + 1);
            if (g.inexact && g.h * res < g.eps) status = EP_OK;
        }
        g.state[1] = res;
        g.state[2] = (double)status;
        sgo = status;
    }
    __syncthreads();
    const int status = sgo;
    if (status == EP_ETIMEOUT || status == EP_EDIVERGED || status == EP_ENOTCONVERGED ||
        (status == EP_OK && !g.inexact)) {
        if (threadIdx.x == 0) cudaGraphSetConditional(g.loop, 0u);
        return;
    }
    // an update (the inexact system's stop comes after it)
    for (size_t a = threadIdx.x; a < m; a += blockDim.x) g.p0[a] = fma(g.h, g.Y[a] - Q[a], g.p0[a]);
    if (status == EP_OK) {
        if (threadIdx.x == 0) cudaGraphSetConditional(g.loop, 0u);
        return;
    }
    __syncthreads();
    if (threadIdx.x < 9) g.bar[threadIdx.x] = 0u;
    for (int i = threadIdx.x; i < g.n; i += blockDim.x) {
        const double qx = g.X[2 * (size_t)i], qy = g.X[2 * (size_t)i + 1];
        const double px = g.p0[2 * (size_t)i], py = g.p0[2 * (size_t)i + 1];
        g.x[2 * (size_t)i] = qx;
        g.x[2 * (size_t)i + 1] = qy;
        g.x[m + 2 * (size_t)i] = px;
        g.x[m + 2 * (size_t)i + 1] = py;
        g.Sx[i] = make_float4((float)((qx - g.c0[0]) * g.s), (float)((qy - g.c0[1]) * g.s), (float)px, (float)py);
        if (g.Dx) {
            g.Dx[4 * (size_t)i] = qx;
            g.Dx[4 * (size_t)i + 1] = qy;
            g.Dx[4 * (size_t)i + 2] = px;
            g.Dx[4 * (size_t)i + 3] = py;
        }
    }
    if (threadIdx.x == 0) cudaGraphSetConditional(g.loop, 1u);
}

template <int JL>
ep_status owner_shoot_fits(int n, int G, bool* ok)
{
    constexpr int THREADS = owner_threads<JL>();
    const size_t smem = owner_smem<THREADS, JL>();
    auto fn = k_shoot_owner<THREADS, JL, false>;
    static int res = -1;
    if (res < 0) {
        EP_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        EP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, THREADS, smem));
        DeviceInfo di{};
        EP_TRY(device_info(&di));
        res = per_sm * di.sm_count;
    }
    *ok = G <= res && G <= kMaxPersistentCtas && n <= owner_chunk<JL>();
    return EP_OK;
}

// The cooperative launch of one owner-computes shoot (as launch_owner, without zeroing
// the barrier words or reading the error flag back: capturable into a graph).
template <int JL>
cudaError_t enqueue_owner_shoot(StageArgs a, const AllPairsBufs& b, int steps, cudaStream_t st)
{
    constexpr int THREADS = owner_threads<JL>();
    const size_t smem = owner_smem<THREADS, JL>();
    auto fn = k_shoot_owner<THREADS, JL, false>;
    const float4* Sx = b.Sx;
    float4* Sa = b.Sa;
    float4* Sb = b.Sb;
    unsigned* bar = b.bar;
    int* err = b.err;
    float4* rec = nullptr;
    void* args[] = {&a, &Sx, &Sa, &Sb, &steps, &bar, &err, &rec};
    return cudaLaunchCooperativeKernel((void*)fn, dim3(a.G), dim3(THREADS), args, smem, st);
}

}  // namespace

size_t owner_match_bytes() { return sizeof(double) * 8; }

// The matching graph: one while-loop node whose body is the host loop's iteration (the
// owner-computes shoot, then k_match_step: residual, tests, update and the next
// shoot's load), so that the whole of Algorithm 1 runs with no host round trip per
// update.  The shoot kernel is
// the one the host loop launches; the results are the host loop's bit for bit.
ep_status owner_match(const ep_params& P, const AllPairsBufs& b, const double* X, const double* Y, double* p0,
                      int maxit, double eps, double h, double* hist, double* scratch, cudaStream_t st, bool* done,
                      double out[3])
{
    *done = false;
    if (b.n == 0 || maxit < 0 || !(P.precision == EP_MIXED && P.dim == 2 && P.kernel == EP_GAUSS) ||
        tc_enabled(P) || !allpairs_persistent_enabled() || !device_match_enabled())
        return EP_OK;
    const APConfig cfg = allpairs_config(b.n, P.dim, P.precision, P.kernel);
    if (cfg.threads != 1024) return EP_OK;
    const double dt = P.t1 / P.steps;
    StageArgs a = base_args(P, b, cfg);
    a.mode = MODE_RK4;
    a.dt = dt;
    a.dt_f = (float)dt;
    a.Sx_w = b.Sx;
    // the centre c0 of X (X does not change between shoots) and a loaded state, from
    // which the tuner's trial shoots start
    EP_TRY(allpairs_load(P, b, X, p0, st));
    OwnerCfg c;
    EP_TRY(gauss2_config(P, b, a, dt, st, false, &c));
    if (c.JL == 0) return EP_OK;  // stream-K: the host loop
    a.G = std::max(1, std::min(c.G, b.n));
    bool fits = false;
    if (c.JL == 1) EP_TRY(owner_shoot_fits<1>(b.n, a.G, &fits));
    else if (c.JL == 4) EP_TRY(owner_shoot_fits<4>(b.n, a.G, &fits));
    else if (c.JL == 8) EP_TRY(owner_shoot_fits<8>(b.n, a.G, &fits));
    else EP_TRY(owner_shoot_fits<16>(b.n, a.G, &fits));
    if (!fits) return EP_OK;
    double* state = scratch;
    EP_TRY_CUDA(cudaMemsetAsync(state, 0, sizeof(double) * 3, st));
    const KernelScale ks = kernel_scale(P.kernel, P.sigma);

    struct GraphGuard {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        ~GraphGuard()
        {
            if (x) cudaGraphExecDestroy(x);
            if (g) cudaGraphDestroy(g);
        }
    } gg;
    EP_TRY_CUDA(cudaGraphCreate(&gg.g, 0));
    cudaGraphConditionalHandle loop;
    EP_TRY_CUDA(cudaGraphConditionalHandleCreate(&loop, gg.g, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    EP_TRY_CUDA(cudaGraphAddNode(&node, gg.g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // the loop body, captured on a private stream of the device (capture needs a stream
    // other than the legacy default one; the capture records and runs nothing, and it
    // always ends, also on an error)
    cudaStream_t cs = nullptr;
    // one capture at a time: calls from several host threads share the capture streams
    static std::mutex capture_mu;
    std::unique_lock<std::mutex> capture_lock(capture_mu);
    {
        DeviceInfo di{};
        EP_TRY(device_info(&di));
        static std::map<int, cudaStream_t> streams;
        cudaStream_t& s0 = streams[di.device];
        if (!s0) EP_TRY_CUDA(cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking));
        cs = s0;
        EP_TRY_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    }
    cudaError_t ce = cudaSuccess;
    {
        if (c.JL == 1) ce = enqueue_owner_shoot<1>(a, b, P.steps, cs);
        else if (c.JL == 4) ce = enqueue_owner_shoot<4>(a, b, P.steps, cs);
        else if (c.JL == 8) ce = enqueue_owner_shoot<8>(a, b, P.steps, cs);
        else ce = enqueue_owner_shoot<16>(a, b, P.steps, cs);
    }
    if (ce == cudaSuccess) {
        const GraphMatch gm{X,    Y,     p0,   b.x, b.Sx, b.Dx, b.c0,           ks.s, b.bar,
                            hist, state, b.n, eps, h,    maxit, P.inexact != 0.0, loop};
        k_match_step<<<1, 1024, 0, cs>>>(gm);
        ce = cudaGetLastError();
    }
    cudaGraph_t captured = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &captured);
    capture_lock.unlock();
    if (ce == cudaSuccess) ce = ee;
    if (ce != cudaSuccess) return cuda_fail(ce, "matching graph capture");
    EP_TRY_CUDA(cudaGraphInstantiate(&gg.x, gg.g, 0));
    // the first shoot's start: (X, p0) is loaded (allpairs_load; the tuner's trials
    // restore it), the barrier words are zeroed here, the later ones by k_match_step
    EP_TRY_CUDA(cudaMemsetAsync(b.bar, 0, sizeof(unsigned) * 9, st));
    TimedLaunch tl;
    if (tl.e0) EP_TRY_CUDA(cudaEventRecord(tl.e0, st));
    EP_TRY_CUDA(cudaGraphLaunch(gg.x, st));
    if (tl.e1) EP_TRY_CUDA(cudaEventRecord(tl.e1, st));
    EP_TRY_CUDA(cudaMemcpyAsync(out, state, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    const int k = (int)out[0];
    const double res = out[1];
    const int status = (int)out[2];
    // the body ran once per shoot: k + 1 shoots, k after the inexact system's stop
    const int shoots = (P.inexact != 0.0 && status == EP_OK) ? k : k + 1;
    count_launch(2 * shoots);
    if (status == EP_ETIMEOUT) {
        bool d = false;
        return finish_persistent(b, st, &d, a.G);
    }
    out[0] = res;
    out[1] = (double)k;
    out[2] = (double)status;
    *done = true;
    char name[80];
    snprintf(name, sizeof(name), "matching graph: k_shoot_owner<%d,%d> (G=%d) x %d", c.JL == 8 ? 512 : 1024, c.JL,
             a.G, shoots);
    tl.record(name);
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
    bool done = false;
    EP_TRY(persistent_steps(P, b, a, steps, dt, st, nullptr, &done));
    if (done) return EP_OK;
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
    if (P.precision == EP_MIXED) {
        bool done = false;
        EP_TRY(persistent_steps(P, b, a, steps, dt, st, rec, &done));
        if (done) return EP_OK;
    }
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
