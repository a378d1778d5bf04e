// ep_adjoint.cu -- Hessian-vector product of H and the exact discrete adjoint
// of the RK4 shoot: the gradient of the inexact-matching energy
//   E(p0) = 1/2 p0^T G(X) p0 + lambda/2 || Q(1) - Y ||^2
// (Sec. 6, Eq. inexact-E written with Eq. E=2H).
//
// Hessian of H (Eq. H) along v = (vq, vp), with d = q_i - q_j, dv = vq_i - vq_j,
// phi = G'(r)/r, psi = phi'(r)/r:
//   (d2H v)_p_i = sum_j      [ G vp_j + phi (d.dv) p_j ]
//   (d2H v)_q_i = sum_{j!=i} [ (vp_i.p_j + p_i.vp_j) phi d + (p_i.p_j)(phi dv + psi (d.dv) d) ]
// The transposed RK4 stage Jacobian is J_F(y)^T w = d2H(y) . (-w_p, w_q).
//
// GPU structure.  The Hessian-vector product is one stream-K pair sweep with
// the same decomposition as the forward stage kernel (tiles of 64 particles,
// one range of (tile, source) units per CTA, FP32 pair terms on scaled
// coordinates, FP64 accumulation, last-arriving CTA per tile finishes the
// particles).  In the adjoint, that last CTA applies one reverse RK4 stage:
//   xb += ybar;  kb_{s-1} += c dt ybar;  next direction = (-kb_p, kb_q).
// Forward states are checkpointed every ckpt_every steps (FP64); each segment
// is recomputed once with every stage input recorded, then reversed.
//
// Scaled units (mixed precision): with q' = s q, the sums above become
//   (d2H v)_p = sum [G vp_j + phi' (d'.dv') p_j],
//   (d2H v)_q = s sum [a phi' d' + b (phi' dv' + psi' (d'.dv') d')],
// phi' = phi / s^2, psi' = psi / s^4 as functions of r' = s r:
//   Gaussian  G = ex2(-r'^2), phi' = -k G, psi' = k^2 G, k = 2 / log2(e)
//   tent      G = 1 - r',     phi' = -1/r', psi' = 1/r'^3          (0 < r' < 1)
//   expcone   G = ex2(-r'),   phi' = -G/(L r'), psi' = G (1/(L r')^2 + 1/(L r'^3)), L = log2(e)
#include <math.h>

#include <algorithm>

#include "ep_allpairs.cuh"
#include "ep_features.cuh"

namespace ep {

namespace {

constexpr int kHvpThreads = 512;
constexpr int kHvpChunk = 1024;
// A warp's FP32 block of a particle's HVP sums covers kHvpFoldChunks staged chunks
// (kHvpFoldChunks * kHvpChunk / 16 = 256 sources); the blocks are accumulated in
// double-FP32 across warps and blocks and in FP64 across CTAs.
constexpr int kHvpFoldChunks = 4;
constexpr float kLog2e = 1.4426950408889634f;

enum HvpMode { HVP_STAGE = 0, HVP_SINGLE = 1 };

struct HvpArgs {
    long long U;
    int n;
    int G;
    int mode;
    int rstage;  // reverse stage 4, 3, 2, 1
    double dt;
    double s;      // coordinate scale of the records (1 in FP64)
    float s_f;
    double sigma;
    const float4* Y;  // mixed: state records (q', p)
    const float4* Din;  // mixed: direction records (s vq, vp)
    float4* Dout;
    const double* YD;   // fp64: state records (q, p)
    const double* DinD; // fp64: direction records (vq, vp)
    double* DoutD;
    double* K;
    int* counters;
    double* xb;   // adjoint state [q | p], FP64
    double* kb1;
    double* kb2;
    double* kb3;
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

template <int KER>
__device__ __forceinline__ void hfun_f32(float r2, float& G, float& ph, float& ps)
{
    if constexpr (KER == EP_GAUSS) {
        const float k = 2.0f / kLog2e;
        G = ex2_approx(-r2);
        ph = -k * G;
        ps = k * k * G;
    } else if constexpr (KER == EP_TENT) {
        const float rs = rsqrt_approx(fmaxf(r2, 1e-20f));
        const bool in = r2 < 1.0f;
        const bool pos = in && r2 > 0.0f;
        G = in ? fmaf(-r2, rs, 1.0f) : 0.0f;
        ph = pos ? -rs : 0.0f;
        ps = pos ? rs * rs * rs : 0.0f;
    } else {
        const float rs = rsqrt_approx(fmaxf(r2, 1e-20f));
        G = ex2_approx(-r2 * rs);
        const bool pos = r2 > 0.0f;
        const float t = rs * (1.0f / kLog2e);
        // t = 1/(L r'): phi' = -G t, psi' = G (t^2 + t rs^2) = G t (t + rs^2)
        ph = pos ? -G * t : 0.0f;
        ps = pos ? G * t * (t + rs * rs) : 0.0f;
    }
}

template <int KER>
__device__ __forceinline__ void hfun_f64(double r2, double sigma, double& G, double& ph, double& ps)
{
    if constexpr (KER == EP_GAUSS) {
        G = exp(-r2 / (2.0 * sigma * sigma));
        ph = -G / (sigma * sigma);
        ps = G / (sigma * sigma * sigma * sigma);
    } else if constexpr (KER == EP_TENT) {
        const double r = sqrt(r2);
        const bool in = r < sigma, pos = in && r > 0.0;
        G = in ? 1.0 - r / sigma : 0.0;
        ph = pos ? -1.0 / (sigma * r) : 0.0;
        ps = pos ? 1.0 / (sigma * r * r * r) : 0.0;
    } else {
        const double r = sqrt(r2);
        G = exp(-r / sigma);
        ph = r > 0.0 ? -G / (sigma * r) : 0.0;
        ps = r > 0.0 ? G * (1.0 / (sigma * sigma * r * r) + 1.0 / (sigma * r * r * r)) : 0.0;
    }
}

__device__ __forceinline__ int cta_of_unit(long long u, long long U, int G)
{
    return (int)(((u + 1) * (long long)G - 1) / U);
}

// Finish particle i: ybar = d2H v (FP64), then the reverse stage or the output.
template <int DIM>
__device__ void hvp_epilogue(const HvpArgs& a, int i, bool mixed)
{
    double yq[DIM], yp[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        yq[c] = __ldcg(a.K + (size_t)i * kKWidth + c) * (mixed ? a.s : 1.0);
        yp[c] = __ldcg(a.K + (size_t)i * kKWidth + 3 + c);
        a.K[(size_t)i * kKWidth + c] = 0.0;
        a.K[(size_t)i * kKWidth + 3 + c] = 0.0;
    }
    if (a.mode == HVP_SINGLE) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            a.out_q[(size_t)i * DIM + c] = yq[c];
            a.out_p[(size_t)i * DIM + c] = yp[c];
        }
        return;
    }
    const size_t m = (size_t)a.n * DIM;
    double* xq = a.xb + (size_t)i * DIM;
    double* xp = a.xb + m + (size_t)i * DIM;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        xq[c] += yq[c];
        xp[c] += yp[c];
    }
    if (a.rstage == 1) return;
    double* kb = a.rstage == 4 ? a.kb3 : (a.rstage == 3 ? a.kb2 : a.kb1);
    const double cdt = (a.rstage == 4 ? 1.0 : 0.5) * a.dt;
    double kq[DIM], kp[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        kq[c] = kb[(size_t)i * DIM + c] + cdt * yq[c];
        kp[c] = kb[m + (size_t)i * DIM + c] + cdt * yp[c];
        kb[(size_t)i * DIM + c] = kq[c];
        kb[m + (size_t)i * DIM + c] = kp[c];
    }
    // next direction v = (-kb_p, kb_q)
    if (mixed) {
        if constexpr (DIM == 2) {
            a.Dout[i] = make_float4((float)(-a.s * kp[0]), (float)(-a.s * kp[1]), (float)kq[0], (float)kq[1]);
        } else {
            a.Dout[2 * (size_t)i] = make_float4((float)(-a.s * kp[0]), (float)(-a.s * kp[1]), (float)(-a.s * kp[2]), 0.f);
            a.Dout[2 * (size_t)i + 1] = make_float4((float)kq[0], (float)kq[1], (float)kq[2], 0.f);
        }
    } else {
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            a.DoutD[(size_t)i * 2 * DIM + c] = -kp[c];
            a.DoutD[(size_t)i * 2 * DIM + DIM + c] = kq[c];
        }
    }
}

// Per source j: state (q', p) and direction (vq', vp), FP32.
template <int DIM>
struct RecF32 {
    float q[DIM], p[DIM], vq[DIM], vp[DIM];
};

template <int DIM>
__device__ __forceinline__ void load_rec_f32(const float4* Y, const float4* D, int j, RecF32<DIM>& r)
{
    if constexpr (DIM == 2) {
        const float4 a = Y[j], b = D[j];
        r.q[0] = a.x; r.q[1] = a.y; r.p[0] = a.z; r.p[1] = a.w;
        r.vq[0] = b.x; r.vq[1] = b.y; r.vp[0] = b.z; r.vp[1] = b.w;
    } else {
        const float4 a0 = Y[2 * (size_t)j], a1 = Y[2 * (size_t)j + 1];
        const float4 b0 = D[2 * (size_t)j], b1 = D[2 * (size_t)j + 1];
        r.q[0] = a0.x; r.q[1] = a0.y; r.q[2] = a0.z; r.p[0] = a1.x; r.p[1] = a1.y; r.p[2] = a1.z;
        r.vq[0] = b0.x; r.vq[1] = b0.y; r.vq[2] = b0.z; r.vp[0] = b1.x; r.vp[1] = b1.y; r.vp[2] = b1.z;
    }
}

// The Hessian-vector pair loop keeps its staged sources in pairs: float4 k of pair t
// holds the components 2k and 2k+1 (in the order q, p, vq, vp) of sources 2t and
// 2t+1, so one load gives the f32x2 operands of two sources, and both rows of a lane
// take each record pair (measured 304 against 314 ms per N = 16384 3-D gradient for the
// scalar loop; one row per pass measured no faster).  The differences are taken as
// q_j - q_i and vq_j - vq_i, so the hq sums come out negated and their sign is
// restored when they are added up.  An odd count is padded with a source far away and
// without momentum or direction (position kPadCoord), whose terms are exactly zero.
constexpr float kPadCoord = 1.0e18f;

// The 4 DIM components (q, p, vq, vp) of source j, or of the padding source.
template <int DIM>
__device__ __forceinline__ void rec_comps(const float4* Y, const float4* D, int j, bool real, float (&c)[4 * DIM])
{
    RecF32<DIM> r;
    if (real) {
        load_rec_f32<DIM>(Y, D, j, r);
    } else {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            r.q[k] = kPadCoord;
            r.p[k] = r.vq[k] = r.vp[k] = 0.f;
        }
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        c[k] = r.q[k];
        c[DIM + k] = r.p[k];
        c[2 * DIM + k] = r.vq[k];
        c[3 * DIM + k] = r.vp[k];
    }
}

// Component c of both sources of a record pair.
template <int DIM>
__device__ __forceinline__ float2 pair_comp(const float4 (&S)[2 * DIM], int c)
{
    const float4& v = S[c >> 1];
    return (c & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
}

template <int DIM, int KER>
__global__ void __launch_bounds__(kHvpThreads, 1) k_hvp_mixed(HvpArgs a)
{
    constexpr int W = kHvpThreads / 32;
    constexpr int V = DIM == 2 ? 1 : 2;  // float4 per particle per record
    extern __shared__ float4 smem[];     // [chunk][state V | direction V]
    __shared__ int s_last;
    __shared__ float2 fin[2 * DIM * kTileI];  // double-FP32 sums of the tile's segment
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = a.n;
    long long u0 = (long long)blockIdx.x * a.U / a.G;
    const long long u1 = (long long)(blockIdx.x + 1) * a.U / a.G;
    while (u0 < u1) {
        const int b = (int)(u0 / n);
        const int j0 = (int)(u0 - (long long)b * n);
        const int j1 = (int)min((long long)n, (long long)j0 + (u1 - u0));
        RecF32<DIM> ri[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int i = b * kTileI + lane + 32 * r;
            if (i < n) {
                load_rec_f32<DIM>(a.Y, a.Din, i, ri[r]);
            } else {
#pragma unroll
                for (int c = 0; c < DIM; ++c) ri[r].q[c] = ri[r].p[c] = ri[r].vq[c] = ri[r].vp[c] = 0.f;
            }
        }
        float hq[2][DIM], hp[2][DIM];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < DIM; ++c) hq[r][c] = hp[r][c] = 0.f;
        int nchunk = 0;
        bool first = true;
        // broadcast operand pairs of the lane's two rows (differences taken as q_j - q_i)
        float2 nq[2][DIM], nv[2][DIM], bp[2][DIM], bv[2][DIM];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                nq[r][c] = make_float2(-ri[r].q[c], -ri[r].q[c]);
                nv[r][c] = make_float2(-ri[r].vq[c], -ri[r].vq[c]);
                bp[r][c] = make_float2(ri[r].p[c], ri[r].p[c]);
                bv[r][c] = make_float2(ri[r].vp[c], ri[r].vp[c]);
            }
        for (int cj = j0; cj < j1; cj += kHvpChunk) {
            const int L = min(kHvpChunk, j1 - cj);
            const int P = (L + 1) >> 1;
            __syncthreads();
            for (int t = threadIdx.x; t < P; t += kHvpThreads) {
                const int j = cj + 2 * t;
                float c0[4 * DIM], c1[4 * DIM];
                rec_comps<DIM>(a.Y, a.Din, j, true, c0);
                rec_comps<DIM>(a.Y, a.Din, j + 1, 2 * t + 1 < L, c1);
#pragma unroll
                for (int k = 0; k < 2 * DIM; ++k)
                    smem[(size_t)t * 2 * DIM + k] = make_float4(c0[2 * k], c1[2 * k], c0[2 * k + 1], c1[2 * k + 1]);
            }
            __syncthreads();
            const int pa = warp * P / W, pz = (warp + 1) * P / W;
            float2 aq[2][DIM], ap[2][DIM];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < DIM; ++c) aq[r][c] = ap[r][c] = make_float2(0.f, 0.f);
            for (int q = pa; q < pz; ++q) {
                float4 S[2 * DIM];
#pragma unroll
                for (int k = 0; k < 2 * DIM; ++k) S[k] = smem[(size_t)q * 2 * DIM + k];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    float2 d[DIM], dv[DIM];
                    float2 r2 = make_float2(0.f, 0.f), dd = r2, pa2 = r2, pb2 = r2;
#pragma unroll
                    for (int c = 0; c < DIM; ++c) {
                        d[c] = __fadd2_rn(pair_comp<DIM>(S, c), nq[r][c]);
                        dv[c] = __fadd2_rn(pair_comp<DIM>(S, 2 * DIM + c), nv[r][c]);
                        r2 = __ffma2_rn(d[c], d[c], r2);
                        dd = __ffma2_rn(d[c], dv[c], dd);
                        pa2 = __ffma2_rn(bv[r][c], pair_comp<DIM>(S, DIM + c),
                                         __ffma2_rn(bp[r][c], pair_comp<DIM>(S, 3 * DIM + c), pa2));
                        pb2 = __ffma2_rn(bp[r][c], pair_comp<DIM>(S, DIM + c), pb2);
                    }
                    float2 G, ph, ps;
                    hfun_f32<KER>(r2.x, G.x, ph.x, ps.x);
                    hfun_f32<KER>(r2.y, G.y, ph.y, ps.y);
                    const float2 t = __fmul2_rn(ph, dd);
                    const float2 cd = __ffma2_rn(pa2, ph, __fmul2_rn(__fmul2_rn(pb2, ps), dd));
                    const float2 cv = __fmul2_rn(pb2, ph);
#pragma unroll
                    for (int c = 0; c < DIM; ++c) {
                        ap[r][c] = __ffma2_rn(G, pair_comp<DIM>(S, 3 * DIM + c),
                                              __ffma2_rn(t, pair_comp<DIM>(S, DIM + c), ap[r][c]));
                        aq[r][c] = __ffma2_rn(cd, d[c], __ffma2_rn(cv, dv[c], aq[r][c]));
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < DIM; ++c) {
                    hq[r][c] -= aq[r][c].x + aq[r][c].y;
                    hp[r][c] += ap[r][c].x + ap[r][c].y;
                }
            // fold the lanes' FP32 blocks: every kHvpFoldChunks chunks and at the segment end
            if (++nchunk % kHvpFoldChunks != 0 && cj + kHvpChunk < j1) continue;
            __syncthreads();
            float* red = reinterpret_cast<float*>(smem);  // [W][2*DIM][64]
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < DIM; ++c) {
                    red[(warp * 2 * DIM + c) * kTileI + lane + 32 * r] = hq[r][c];
                    red[(warp * 2 * DIM + DIM + c) * kTileI + lane + 32 * r] = hp[r][c];
                    hq[r][c] = hp[r][c] = 0.f;
                }
            __syncthreads();
            for (int t = threadIdx.x; t < 2 * DIM * kTileI; t += kHvpThreads) {
                float2 sum = make_float2(red[t], 0.f);
                for (int w2 = 1; w2 < W; ++w2) dd_acc(sum, red[w2 * 2 * DIM * kTileI + t]);
                fin[t] = first ? dd_add(sum, make_float2(0.f, 0.f)) : dd_add(fin[t], sum);
            }
            first = false;
        }
        // the segment's sums into the FP64 accumulator (each fin entry is read by the
        // thread that wrote it)
        for (int t = threadIdx.x; t < 2 * DIM * kTileI; t += kHvpThreads) {
            const int k = t / kTileI, il = t % kTileI;
            const int i = b * kTileI + il;
            const int slot = k < DIM ? k : 3 + (k - DIM);
            if (i < n) atomicAdd(a.K + (size_t)i * kKWidth + slot, dd_to_double(fin[t]));
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const long long ub = (long long)b * n;
            const int cnt = cta_of_unit(ub + n - 1, a.U, a.G) - cta_of_unit(ub, a.U, a.G) + 1;
            s_last = (atomicAdd(a.counters + b, 1) == cnt - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            if (threadIdx.x < kTileI) {
                const int i = b * kTileI + threadIdx.x;
                if (i < n) hvp_epilogue<DIM>(a, i, true);
            }
            if (threadIdx.x == 0) a.counters[b] = 0;
        }
        u0 += (j1 - j0);
    }
}

template <int DIM, int KER>
__global__ void __launch_bounds__(256) k_hvp_fp64(HvpArgs a)
{
    constexpr int T = 256, W = T / 32, S = 4 * DIM;  // doubles per source: q p vq vp
    constexpr int CH = 512;
    extern __shared__ double dsm[];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = a.n;
    long long u0 = (long long)blockIdx.x * a.U / a.G;
    const long long u1 = (long long)(blockIdx.x + 1) * a.U / a.G;
    while (u0 < u1) {
        const int b = (int)(u0 / n);
        const int j0 = (int)(u0 - (long long)b * n);
        const int j1 = (int)min((long long)n, (long long)j0 + (u1 - u0));
        double qi[2][DIM], pi[2][DIM], vqi[2][DIM], vpi[2][DIM];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int i = b * kTileI + lane + 32 * r;
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                qi[r][c] = i < n ? a.YD[(size_t)i * 2 * DIM + c] : 0.0;
                pi[r][c] = i < n ? a.YD[(size_t)i * 2 * DIM + DIM + c] : 0.0;
                vqi[r][c] = i < n ? a.DinD[(size_t)i * 2 * DIM + c] : 0.0;
                vpi[r][c] = i < n ? a.DinD[(size_t)i * 2 * DIM + DIM + c] : 0.0;
            }
        }
        double hq[2][DIM], hp[2][DIM];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < DIM; ++c) hq[r][c] = hp[r][c] = 0.0;
        for (int cj = j0; cj < j1; cj += CH) {
            const int L = min(CH, j1 - cj);
            __syncthreads();
            for (int t = threadIdx.x; t < L * S; t += T) {
                const int jj = t / S, k = t % S;
                dsm[t] = k < 2 * DIM ? a.YD[(size_t)(cj + jj) * 2 * DIM + k]
                                     : a.DinD[(size_t)(cj + jj) * 2 * DIM + (k - 2 * DIM)];
            }
            __syncthreads();
            const int ja = warp * L / W, jb = (warp + 1) * L / W;
            for (int j = ja; j < jb; ++j) {
                const double* v = dsm + (size_t)j * S;
                const int jg = cj + j;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int i = b * kTileI + lane + 32 * r;
                    double d[DIM], dv[DIM], r2 = 0, dd = 0, pa = 0, pb = 0;
#pragma unroll
                    for (int c = 0; c < DIM; ++c) {
                        d[c] = qi[r][c] - v[c];
                        dv[c] = vqi[r][c] - v[2 * DIM + c];
                        r2 += d[c] * d[c];
                        dd += d[c] * dv[c];
                        pa += vpi[r][c] * v[DIM + c] + pi[r][c] * v[3 * DIM + c];
                        pb += pi[r][c] * v[DIM + c];
                    }
                    double G, ph, ps;
                    hfun_f64<KER>(r2, a.sigma, G, ph, ps);
                    const bool self = (jg == i);
#pragma unroll
                    for (int c = 0; c < DIM; ++c) {
                        hp[r][c] += G * v[3 * DIM + c] + ph * dd * v[DIM + c];
                        if (!self) hq[r][c] += pa * ph * d[c] + pb * (ph * dv[c] + ps * dd * d[c]);
                    }
                }
            }
        }
        __syncthreads();
        double* red = dsm;
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                red[(warp * 2 * DIM + c) * kTileI + lane + 32 * r] = hq[r][c];
                red[(warp * 2 * DIM + DIM + c) * kTileI + lane + 32 * r] = hp[r][c];
            }
        __syncthreads();
        for (int t = threadIdx.x; t < 2 * DIM * kTileI; t += T) {
            const int k = t / kTileI, il = t % kTileI;
            double sum = 0.0;
            for (int w2 = 0; w2 < W; ++w2) sum += red[(w2 * 2 * DIM + k) * kTileI + il];
            const int i = b * kTileI + il;
            const int slot = k < DIM ? k : 3 + (k - DIM);
            if (i < n) atomicAdd(a.K + (size_t)i * kKWidth + slot, sum);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const long long ub = (long long)b * n;
            const int cnt = cta_of_unit(ub + n - 1, a.U, a.G) - cta_of_unit(ub, a.U, a.G) + 1;
            s_last = (atomicAdd(a.counters + b, 1) == cnt - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            if (threadIdx.x < kTileI) {
                const int i = b * kTileI + threadIdx.x;
                if (i < n) hvp_epilogue<DIM>(a, i, false);
            }
            if (threadIdx.x == 0) a.counters[b] = 0;
        }
        u0 += (j1 - j0);
    }
}

// ------------------------------------------------------------------ small kernels
// FP32 / FP64 direction records from FP64 (vq, vp), and the mixed state records
// of an arbitrary (q, p) are built by allpairs_load.
__global__ void k_dir_records(const double* __restrict__ vq, const double* __restrict__ vp, int n, int dim,
                              double s, float4* __restrict__ D, double* __restrict__ DD)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    for (int c = 0; c < dim; ++c) {
        a[c] = vq[(size_t)i * dim + c];
        b[c] = vp[(size_t)i * dim + c];
    }
    if (D) {
        if (dim == 2) {
            D[i] = make_float4((float)(s * a[0]), (float)(s * a[1]), (float)b[0], (float)b[1]);
        } else {
            D[2 * (size_t)i] = make_float4((float)(s * a[0]), (float)(s * a[1]), (float)(s * a[2]), 0.f);
            D[2 * (size_t)i + 1] = make_float4((float)b[0], (float)b[1], (float)b[2], 0.f);
        }
    }
    if (DD)
        for (int c = 0; c < dim; ++c) {
            DD[(size_t)i * 2 * dim + c] = a[c];
            DD[(size_t)i * 2 * dim + dim + c] = b[c];
        }
}

// Start of a reverse step from abar = xb: kb3 = kb2 = dt/3 abar, kb1 = dt/6 abar and
// the stage-4 direction from kb4 = dt/6 abar: v = (-kb4_p, kb4_q).
__global__ void k_adj_begin(const double* __restrict__ xb, double* kb1, double* kb2, double* kb3, int n, int dim,
                            double dt, double s, float4* __restrict__ D, double* __restrict__ DD)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t m = (size_t)n * dim;
    double aq[3] = {0, 0, 0}, ap[3] = {0, 0, 0};
    for (int c = 0; c < dim; ++c) {
        aq[c] = xb[(size_t)i * dim + c];
        ap[c] = xb[m + (size_t)i * dim + c];
        kb3[(size_t)i * dim + c] = kb2[(size_t)i * dim + c] = dt / 3.0 * aq[c];
        kb3[m + (size_t)i * dim + c] = kb2[m + (size_t)i * dim + c] = dt / 3.0 * ap[c];
        kb1[(size_t)i * dim + c] = dt / 6.0 * aq[c];
        kb1[m + (size_t)i * dim + c] = dt / 6.0 * ap[c];
    }
    double vq[3], vp[3];
    for (int c = 0; c < 3; ++c) {
        vq[c] = -dt / 6.0 * ap[c];
        vp[c] = dt / 6.0 * aq[c];
    }
    if (D) {
        if (dim == 2) {
            D[i] = make_float4((float)(s * vq[0]), (float)(s * vq[1]), (float)vp[0], (float)vp[1]);
        } else {
            D[2 * (size_t)i] = make_float4((float)(s * vq[0]), (float)(s * vq[1]), (float)(s * vq[2]), 0.f);
            D[2 * (size_t)i + 1] = make_float4((float)vp[0], (float)vp[1], (float)vp[2], 0.f);
        }
    }
    if (DD)
        for (int c = 0; c < dim; ++c) {
            DD[(size_t)i * 2 * dim + c] = vq[c];
            DD[(size_t)i * 2 * dim + dim + c] = vp[c];
        }
}

// xb = (lambda (Q1 - Y), 0)
__global__ void k_adj_terminal(const double* __restrict__ Q1, const double* __restrict__ Y, size_t m,
                               double lambda, double* __restrict__ xb)
{
    const size_t a = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (a < m) {
        xb[a] = lambda * (Q1[a] - Y[a]);
        xb[m + a] = 0.0;
    }
}

// E = 1/2 p0 . (G(X) p0) + lambda/2 |Q1 - Y|^2 (one CTA, fixed order)
__global__ void k_energy(const double* __restrict__ p0, const double* __restrict__ gp, const double* __restrict__ Q1,
                         const double* __restrict__ Y, size_t m, double lambda, double* out)
{
    __shared__ double sm[32];
    double s = 0.0;
    for (size_t a = threadIdx.x; a < m; a += blockDim.x) {
        const double r = Q1[a] - Y[a];
        s += 0.5 * p0[a] * gp[a] + 0.5 * lambda * r * r;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sm[k];
        *out = t;
    }
}

// grad = G(X) p0 + xb_p
__global__ void k_adj_grad(const double* __restrict__ gp, const double* __restrict__ xb, size_t m,
                           double* __restrict__ grad)
{
    const size_t a = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (a < m) grad[a] = gp[a] + xb[m + a];
}

ep_status launch_hvp(const ep_params& P, const HvpArgs& a, cudaStream_t st)
{
    const bool mixed = P.precision == EP_MIXED;
#define EP_HVP_CASE(D, K)                                                                                   \
    if (P.dim == D && P.kernel == K) {                                                                      \
        if (mixed) {                                                                                        \
            const size_t smem = std::max((size_t)kHvpChunk * 2 * (D == 2 ? 1 : 2) * sizeof(float4),          \
                                         (size_t)(kHvpThreads / 32) * 2 * D * kTileI * sizeof(float));       \
            static bool attr = false;                                                                       \
            if (!attr) {                                                                                    \
                EP_TRY_CUDA(cudaFuncSetAttribute(k_hvp_mixed<D, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                                 (int)smem));                                               \
                attr = true;                                                                                \
            }                                                                                               \
            count_launch();                                                                                 \
            k_hvp_mixed<D, K><<<a.G, kHvpThreads, smem, st>>>(a);                                           \
        } else {                                                                                            \
            const size_t smem = std::max((size_t)512 * 4 * D * sizeof(double),                               \
                                         (size_t)8 * 2 * D * kTileI * sizeof(double));                       \
            static bool attr = false;                                                                       \
            if (!attr) {                                                                                    \
                EP_TRY_CUDA(cudaFuncSetAttribute(k_hvp_fp64<D, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                                 (int)smem));                                               \
                attr = true;                                                                                \
            }                                                                                               \
            count_launch();                                                                                 \
            k_hvp_fp64<D, K><<<a.G, 256, smem, st>>>(a);                                                    \
        }                                                                                                   \
        return EP_OK;                                                                                       \
    }
    EP_HVP_CASE(2, EP_GAUSS) EP_HVP_CASE(2, EP_TENT) EP_HVP_CASE(2, EP_EXPCONE)
    EP_HVP_CASE(3, EP_GAUSS) EP_HVP_CASE(3, EP_TENT) EP_HVP_CASE(3, EP_EXPCONE)
#undef EP_HVP_CASE
    set_error("no HVP kernel for dim=%d kernel=%d", P.dim, P.kernel);
    return EP_EINVAL;
}

HvpArgs hvp_base(const ep_params& P, const AllPairsBufs& b)
{
    HvpArgs a{};
    DeviceInfo di{};
    if (device_info(&di) != EP_OK) di.sm_count = 1;
    const int ntiles = (b.n + kTileI - 1) / kTileI;
    a.n = b.n;
    a.U = (long long)ntiles * b.n;
    const long long want = P.precision == EP_MIXED ? di.sm_count : 4LL * di.sm_count;
    a.G = (int)std::max<long long>(1, std::min<long long>(want, std::max<long long>(1, a.U / 256)));
    a.G = (int)std::min<long long>(a.G, a.U);
    a.s = P.precision == EP_MIXED ? kernel_scale(P.kernel, P.sigma).s : 1.0;
    a.s_f = (float)a.s;
    a.sigma = P.sigma;
    a.K = b.K;
    a.counters = b.counters;
    return a;
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

// Copy a caller array into device memory (carved from the arena) when it is host memory.
ep_status dev_in(Arena* ar, const double* p, size_t cnt, cudaStream_t st, const double** out)
{
    if (is_dev(p)) {
        *out = p;
        return EP_OK;
    }
    double* d = (double*)ar->carve(sizeof(double) * cnt);
    if (!d) return set_error("workspace too small"), EP_ENOMEM;
    EP_TRY_CUDA(cudaMemcpyAsync(d, p, sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
    *out = d;
    return EP_OK;
}

}  // namespace

ep_status hvp_entry(const ep_params* params, int64_t n, const double* q, const double* p, const double* vq,
                    const double* vp, double* hq, double* hp, void* stream)
{
    EP_TRY(check_params(params));
    if (params->inexact != 0.0) return set_error("the Hessian and the adjoint are built for the exact system"), EP_EINVAL;
    if (n < 0 || n > ((int64_t)1 << 26)) return set_error("ep_hvp: bad n"), EP_EINVAL;
    if (n == 0) return EP_OK;
    if (!q || !p || !vq || !vp || !hq || !hp) return set_error("ep_hvp: NULL array"), EP_EINVAL;
    const ep_params& P = *params;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t m = (size_t)n * P.dim;
    const bool mixed = P.precision == EP_MIXED;
    Sizer z;
    z.add(allpairs_bytes((int)n, P.dim, P.precision));
    z.add(sizeof(double) * m * 6);
    z.add(sizeof(double) * m * 2 * 2 + 64);
    Arena* ar = nullptr;
    EP_TRY(arena_acquire(st, z.total, &ar));
    AllPairsBufs b;
    EP_TRY(allpairs_carve(ar, (int)n, P.dim, P.precision, &b));
    const double *dq_ = nullptr, *dp_ = nullptr, *dvq = nullptr, *dvp = nullptr;
    EP_TRY(dev_in(ar, q, m, st, &dq_));
    EP_TRY(dev_in(ar, p, m, st, &dp_));
    EP_TRY(dev_in(ar, vq, m, st, &dvq));
    EP_TRY(dev_in(ar, vp, m, st, &dvp));
    const bool hq_host = !is_dev(hq), hp_host = !is_dev(hp);
    double* oq = hq_host ? (double*)ar->carve(sizeof(double) * m) : hq;
    double* op = hp_host ? (double*)ar->carve(sizeof(double) * m) : hp;
    // direction records in the Sa / Da buffer (unused by a single evaluation)
    EP_TRY(allpairs_load(P, b, dq_, dp_, st));
    HvpArgs a = hvp_base(P, b);
    a.mode = HVP_SINGLE;
    a.out_q = oq;
    a.out_p = op;
    count_launch();
    k_dir_records<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dvq, dvp, (int)n, P.dim, a.s,
                                                               mixed ? b.Sa : nullptr, mixed ? nullptr : b.Da);
    a.Y = b.Sx;
    a.Din = b.Sa;
    a.YD = b.Dx;
    a.DinD = b.Da;
    EP_TRY(launch_hvp(P, a, st));
    if (hq_host) EP_TRY_CUDA(cudaMemcpyAsync(hq, oq, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    if (hp_host) EP_TRY_CUDA(cudaMemcpyAsync(hp, op, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    if (hq_host || hp_host || !is_dev(q) || !is_dev(p) || !is_dev(vq) || !is_dev(vp))
        EP_TRY_CUDA(cudaStreamSynchronize(st));
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

ep_status adjoint_entry(const ep_params* params, int64_t n, const double* X, const double* p0,
                        const double* Y, double lambda, int ckpt_every, double* grad_p0, double* energy,
                        void* stream)
{
    EP_TRY(check_params(params));
    if (params->inexact != 0.0) return set_error("the Hessian and the adjoint are built for the exact system"), EP_EINVAL;
    if (n < 0 || n > ((int64_t)1 << 26)) return set_error("ep_adjoint: bad n"), EP_EINVAL;
    if (ckpt_every < 1) return set_error("ep_adjoint: ckpt_every must be >= 1"), EP_EINVAL;
    if (!isfinite(lambda)) return set_error("ep_adjoint: lambda must be finite"), EP_EINVAL;
    if (params->neigh == EP_CELLLIST)
        return set_error("ep_adjoint: the adjoint runs on the all-pairs path"), EP_EINVAL;
    const ep_params& P = *params;
    cudaStream_t st = (cudaStream_t)stream;
    const bool e_dev = energy && is_dev(energy);
    if (n == 0) {
        const double z0 = 0.0;
        if (energy) {
            if (e_dev) EP_TRY_CUDA(cudaMemcpyAsync(energy, &z0, sizeof z0, cudaMemcpyHostToDevice, st));
            else *energy = 0.0;
        }
        return EP_OK;
    }
    if (!X || !p0 || !Y || !grad_p0) return set_error("ep_adjoint: NULL array"), EP_EINVAL;
    const int S = P.steps;
    const int C = std::min(ckpt_every, S);
    const int nseg = (S + C - 1) / C;
    const size_t m = (size_t)n * P.dim;
    const bool mixed = P.precision == EP_MIXED;
    const size_t V = P.dim == 2 ? 1 : 2;
    const size_t rec_bytes = mixed ? sizeof(float4) * V * (size_t)n : sizeof(double) * 2 * m;
    Sizer z;
    z.add(allpairs_bytes((int)n, P.dim, P.precision));
    z.add(sizeof(double) * 2 * m * (nseg + 1));          // checkpoints
    z.add(rec_bytes * (4 * (size_t)C + 1));              // recorded stage inputs of one segment
    z.add(sizeof(double) * 2 * m * 4);                   // xb, kb1, kb2, kb3
    z.add(rec_bytes * 2);                                // direction ping-pong
    z.add(sizeof(double) * m * 2);                       // G(X) p0 and scratch
    z.add(sizeof(double) * m * 4 + 64);                  // staging + scalar
    Arena* ar = nullptr;
    EP_TRY(arena_acquire(st, z.total, &ar));
    AllPairsBufs b;
    EP_TRY(allpairs_carve(ar, (int)n, P.dim, P.precision, &b));
    double* ck = (double*)ar->carve(sizeof(double) * 2 * m * (nseg + 1));
    char* rec = (char*)ar->carve(rec_bytes * (4 * (size_t)C + 1));
    double* xb = (double*)ar->carve(sizeof(double) * 2 * m);
    double* kb1 = (double*)ar->carve(sizeof(double) * 2 * m);
    double* kb2 = (double*)ar->carve(sizeof(double) * 2 * m);
    double* kb3 = (double*)ar->carve(sizeof(double) * 2 * m);
    char* dirA = (char*)ar->carve(rec_bytes);
    char* dirB = (char*)ar->carve(rec_bytes);
    double* gp = (double*)ar->carve(sizeof(double) * m);
    double* scratch = (double*)ar->carve(sizeof(double) * m);
    const double *dX = nullptr, *dp0 = nullptr, *dY = nullptr;
    EP_TRY(dev_in(ar, X, m, st, &dX));
    EP_TRY(dev_in(ar, p0, m, st, &dp0));
    EP_TRY(dev_in(ar, Y, m, st, &dY));
    const bool g_host = !is_dev(grad_p0);
    double* dgrad = g_host ? (double*)ar->carve(sizeof(double) * m) : grad_p0;
    double* scal = (double*)ar->carve(64);
    if (!scal) return set_error("ep_adjoint: workspace too small"), EP_ENOMEM;
    const double dt = P.t1 / S;
    const unsigned gm = (unsigned)((m + 255) / 256), gn = (unsigned)((n + 255) / 256);

    // G(X) p0 = dq of the right-hand side at (X, p0)
    EP_TRY(allpairs_load(P, b, dX, dp0, st));
    EP_TRY(allpairs_rhs(P, b, gp, scratch, st));
    // forward with checkpoints every C steps
    EP_TRY(allpairs_load(P, b, dX, dp0, st));
    EP_TRY_CUDA(cudaMemcpyAsync(ck, b.x, sizeof(double) * 2 * m, cudaMemcpyDeviceToDevice, st));
    for (int sg = 0; sg < nseg; ++sg) {
        const int ns = std::min(C, S - sg * C);
        EP_TRY(allpairs_steps(P, b, ns, dt, st));
        EP_TRY_CUDA(cudaMemcpyAsync(ck + 2 * m * (sg + 1), b.x, sizeof(double) * 2 * m, cudaMemcpyDeviceToDevice, st));
    }
    const double* Q1 = ck + 2 * m * nseg;
    count_launch(2);
    k_energy<<<1, 1024, 0, st>>>(dp0, gp, Q1, dY, m, lambda, scal);
    k_adj_terminal<<<gm, 256, 0, st>>>(Q1, dY, m, lambda, xb);

    HvpArgs a = hvp_base(P, b);
    a.mode = HVP_STAGE;
    a.dt = dt;
    a.xb = xb;
    a.kb1 = kb1;
    a.kb2 = kb2;
    a.kb3 = kb3;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int ns = std::min(C, S - sg * C);
        const double* x0 = ck + 2 * m * sg;
        EP_TRY(allpairs_load(P, b, x0, x0 + m, st));
        EP_TRY(allpairs_steps_rec(P, b, ns, dt, mixed ? (float4*)rec : nullptr, mixed ? nullptr : (double*)rec, st));
        for (int k = ns - 1; k >= 0; --k) {
            count_launch();
            k_adj_begin<<<gn, 256, 0, st>>>(xb, kb1, kb2, kb3, (int)n, P.dim, dt, a.s,
                                            mixed ? (float4*)dirA : nullptr, mixed ? nullptr : (double*)dirA);
            for (int rs = 4; rs >= 1; --rs) {
                a.rstage = rs;
                const char* yin = rec + rec_bytes * (4 * (size_t)k + (rs - 1));
                const char* din = (rs == 4 || rs == 2) ? dirA : dirB;
                char* dout = (rs == 4 || rs == 2) ? dirB : dirA;
                a.Y = (const float4*)yin;
                a.YD = (const double*)yin;
                a.Din = (const float4*)din;
                a.DinD = (const double*)din;
                a.Dout = (float4*)dout;
                a.DoutD = (double*)dout;
                EP_TRY(launch_hvp(P, a, st));
            }
        }
    }
    count_launch();
    k_adj_grad<<<gm, 256, 0, st>>>(gp, xb, m, dgrad);
    if (g_host) EP_TRY_CUDA(cudaMemcpyAsync(grad_p0, dgrad, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    if (energy) {
        if (e_dev) EP_TRY_CUDA(cudaMemcpyAsync(energy, scal, sizeof(double), cudaMemcpyDeviceToDevice, st));
        else EP_TRY_CUDA(cudaMemcpyAsync(energy, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    if (g_host || (energy && !e_dev) || !is_dev(X) || !is_dev(p0) || !is_dev(Y))
        EP_TRY_CUDA(cudaStreamSynchronize(st));
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

}  // namespace ep
