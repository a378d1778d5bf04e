// ep_tc.cu -- tensor-core (tcgen05) pair phase of the 2-D Gaussian N-particle
// system (Sec. 3.1, Eq. N-particle) inside the persistent RK4 shoot (Sec. 4,
// Note 1 item 5), mixed precision.
//
// The pair sums of one stage are a dense contraction.  In scaled coordinates
// (G = 2^-|q'_i - q'_j|^2) centred on the tile of particles i, q = q' - c,
//   G_ij = E_i g_ij,  E_i = 2^-|q_i|^2,  g_ij = 2^t_ij,  t_ij = 2 q_i.q_j - |q_j|^2,
//   dq_i = E_i sum_j g_ij p_j,
//   M_i  = q_i (x) dq_i - E_i sum_j g_ij (q_j (x) p_j)      (M_cd = sum_j G_ij (q_i - q_j)_c p_j,d),
// so per tile of 128 particles the stage needs  T = Q R^T  (the exponents, a
// rank-3 product) and  S = g V  with V_j = (p_j, q_j (x) p_j) (six columns).
// Both products run on the tensor cores in TF32 with a hi/lo split of every
// operand (hi = TF32 rounding, lo = the rest), which keeps them at FP32-level
// accuracy:
//   MMA 1 (M=128, N=64, K=8):  A row i = (qx_h, qy_h, 1, qx_l, qy_l, qx_h, qy_h, 1)
//                              B row j = (X_h, Y_h, P_h, X_h, Y_h, X_l, Y_l, P_l)
//                              with X = 2x_j, Y = 2y_j, P = -|q_j|^2  ->  t_ij;
//   CUDA cores:                g = ex2(t), g_h = tf32(g), g_l = g - g_h  -> tensor memory;
//   MMA 2 (M=128, N=16, K=64): D = g_h [V_h | V_l | 0] + g_l [V_h | V_l | 0] per chunk,
//                              so D[:, c] + D[:, 6 + c] = sum over the chunk of g_ij V_jc;
//   CUDA cores:                the chunk sums are read back and added in FP32 registers
//                              (a chunk is 64 sources: no long accumulation on the tensor cores).
// A tile whose |q_i|^2 exceeds kTcFactorMax (2^t could overflow) takes the
// difference form on the CUDA cores instead.
//
// Status: opt-in (EP_TC=1), not the default.  On GB300 a kind::tf32 MMA with
// M = 128, K = 8 occupies the tensor pipe for about 96 cycles for every N up to
// 128 (only N = 256 reaches the pipe's peak), and the accumulation here has 12
// useful columns: MMA 2 costs 16 such instructions per 64 x 128 pairs, a ceiling
// of about 5 pairs per clock per SM, half of what the CUDA-core loop sustains.
//
// Work decomposition: the units (tile b of 128, source j) are cut into G equal
// ranges, one per CTA (one CTA per SM, cooperative launch); a CTA's range is one
// or two tile segments.  Per segment the CTA writes its six FP32 partial sums per
// particle into its own slot (CTA c, tile b -> slot c + b, unique); the last CTA
// to arrive at a tile sums the slots in CTA order in FP64 and applies the RK4
// stage to the tile, then every CTA meets at one grid barrier per stage.
//
// Roles in a CTA of 8 + 1 warps: warps 0..7 turn exponents into g (warp w owns
// TMEM lanes 32 (w % 4) .. + 31 and half w / 4 of each chunk's 64 columns); warp 8
// allocates tensor memory and one of its threads issues the MMAs.  Every thread
// stages the source records of a block of up to kTcLB sources in shared memory.
// Pipelines: E[2] (exponents), Gh[2], Gl[2] (the split g) and D[2] (chunk sums)
// double-buffered in tensor memory, with mbarriers E (MMA 1 done), G (g stored),
// F (MMA 2 done: g buffer free, chunk sums ready) per buffer and D (block's MMAs
// done).  Warps 0..3 read chunk k - 2's sums while preparing chunk k.  Every wait is bounded
// by a %globaltimer deadline; on expiry the CTA raises the error flag and runs
// to the end without issuing further tensor-core work.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "ep_allpairs_dev.cuh"

namespace ep {

namespace {

constexpr int kTcM = 128;       // particles per tile (MMA M)
constexpr int kTcNC = 64;       // sources per chunk (N of MMA 1, K of MMA 2)
constexpr int kTcLB = 1024;     // sources staged in shared memory per block
constexpr int kTcExpW = 8;      // exponent warps
constexpr int kTcThreads = kTcExpW * 32 + 32;
constexpr float kTcFactorMax = 60.0f;

// shared memory (dynamic): A1 | B1 | B2 | raw source records
constexpr int kOffA1 = 0;                          // 128 rows x 8 tf32, K-major
constexpr int kOffB1 = 4096;                       // kTcLB rows x 8 tf32, K-major
constexpr int kOffB2 = kOffB1 + kTcLB * 32;        // 16 columns x kTcLB tf32, K-major
constexpr int kOffRaw = kOffB2 + kTcLB * 64;       // kTcLB float4
constexpr int kTcSmem = kOffRaw + kTcLB * 16;

// tensor memory columns (512 allocated)
constexpr uint32_t kColE = 0;     // 2 x 64
constexpr uint32_t kColGh = 128;  // 2 x 64
constexpr uint32_t kColGl = 256;  // 2 x 64
constexpr uint32_t kColD = 384;   // 2 x 16: one chunk's sums per buffer

// mbarriers
constexpr int kBarE = 0, kBarG = 2, kBarF = 4, kBarD = 6, kBarFin = 7, kNumBars = 8;

// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t kIdesc1 = idesc_tf32(128, kTcNC);
constexpr uint32_t kIdesc2 = idesc_tf32(128, 16);

// Shared-memory matrix descriptor, no swizzle: core matrices of 8 rows x 16 bytes;
// lbo = byte stride between core matrices along K, sbo = along the rows (8-row groups).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(tf32_rna(x)); }
__device__ __forceinline__ float tf32_lo(float x) { return __uint_as_float(tf32_rna(x - tf32_hi(x))); }

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s: far beyond any legitimate wait

// Wait for phase `parity` of mbarrier b by one thread.  Gives up (false) when the
// CTA is already aborting or after kWaitNs, raising the abort and error flags.
__device__ bool mbar_wait_one(uint64_t* b, uint32_t parity, volatile int* abort, int* err)
{
    if (*abort) return false;
    uint64_t t0 = 0;
    for (unsigned it = 1;; ++it) {
        if (mbar_try(b, parity)) return true;
        if ((it & 255u) == 0) {
            if (*abort) return false;
            const uint64_t t = globaltimer();
            if (t0 == 0) {
                t0 = t;
            } else if (t - t0 > kWaitNs) {
                *abort = 1;
                atomicExch(err, 2);
                return false;
            }
        }
    }
}

// Warp-uniform wait: lane 0 polls, the warp shares the outcome.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* b, uint32_t parity, volatile int* abort, int* err)
{
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait_one(b, parity, abort, err) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p; }" ::"r"(d),
        "r"(a), "l"(b), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
                 : "memory");
}

// 32 lanes x 32 columns of 32 bits: thread t <-> lane (base lane + t), columns col .. col + 31
__device__ __forceinline__ void tm_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]),
        "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]),
        "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Column c of the MMA-2 operand [V_h | V_l | 0] for one source, V = (px, py, x px, x py, y px, y py).
__device__ __forceinline__ float v_col(int c, float px, float py, float x, float y)
{
    const int k = c < 6 ? c : c - 6;
    float v;
    switch (k) {
    case 0: v = px; break;
    case 1: v = py; break;
    case 2: v = x * px; break;
    case 3: v = x * py; break;
    case 4: v = y * px; break;
    default: v = y * py; break;
    }
    if (c >= 12) return 0.0f;
    return c < 6 ? tf32_hi(v) : tf32_lo(v);
}

struct TcState {
    uint64_t* bars;
    uint32_t tm;       // tensor-memory base address
    uint32_t kc;       // chunks issued so far (buffer = kc & 1, use = kc >> 1)
    uint32_t blk;      // blocks so far (phase of the D barrier)
    uint32_t seg0;     // first chunk of the current segment
    volatile int* abort;
    int* err;
};

// MMA issue for one block of nb chunks (one thread).
__device__ void tc_issue_block(TcState& S, uint32_t sA1, uint32_t sB1, uint32_t sB2, int nb, int Lp)
{
    const uint64_t dA = sdesc(sA1, 128, 256);
    const uint32_t sbo2 = (uint32_t)Lp * 32u;
    auto mma1 = [&](int c) {
        const uint32_t buf = (S.kc + c) & 1u;
        mma_ss(S.tm + kColE + 64u * buf, dA, sdesc(sB1 + (uint32_t)c * 2048u, 128, 256), kIdesc1, 0);
        mma_commit(&S.bars[kBarE + buf]);
    };
    mma1(0);
    if (nb > 1) mma1(1);
    for (int c = 0; c < nb; ++c) {
        const uint32_t k = S.kc + c, buf = k & 1u, u = k >> 1;
        if (!mbar_wait_one(&S.bars[kBarG + buf], u & 1u, S.abort, S.err)) return;
        tc_fence_after();
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const uint64_t dB = sdesc(sB2 + (uint32_t)(16 * c + 2 * s) * 128u, 128, sbo2);
            mma_ts(S.tm + kColD + 16u * buf, S.tm + kColGh + 64u * buf + 8u * s, dB, kIdesc2, s == 0 ? 0u : 1u);
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const uint64_t dB = sdesc(sB2 + (uint32_t)(16 * c + 2 * s) * 128u, 128, sbo2);
            mma_ts(S.tm + kColD + 16u * buf, S.tm + kColGl + 64u * buf + 8u * s, dB, kIdesc2, 1u);
        }
        mma_commit(&S.bars[kBarF + buf]);
        if (c + 2 < nb) mma1(c + 2);
    }
    mma_commit(&S.bars[kBarD]);
}

// Warps 0..3: add chunk k's sums (D buffer k & 1, rows = this warp's lanes) into acc.
__device__ __forceinline__ void tc_read_chunk(const TcState& S, uint32_t k, float (&acc)[6])
{
    const int warp = threadIdx.x >> 5;
    uint32_t d[16];
    tm_ld16(S.tm + ((uint32_t)(warp * 32) << 16) + kColD + 16u * (k & 1u), d);
    tm_wait_ld();
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += __uint_as_float(d[c]) + __uint_as_float(d[6 + c]);
}

// Exponent warps for one block: E -> (g_h, g_l) per chunk (warps 0..3 also fold
// chunk k - 2's sums into acc), then wait for the block's MMAs.
__device__ void tc_exp_block(TcState& S, int nb, float (&acc)[6])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t col = 32u * (uint32_t)(warp >> 2);
    for (int c = 0; c < nb; ++c) {
        const uint32_t k = S.kc + c, buf = k & 1u, u = k >> 1;
        if (!mbar_wait_warp(&S.bars[kBarE + buf], u & 1u, S.abort, S.err)) continue;
        // chunk k - 2 (same buffers) must be through MMA 2: its g buffers are free and its sums final
        if (u >= 1 && !mbar_wait_warp(&S.bars[kBarF + buf], (u - 1) & 1u, S.abort, S.err)) continue;
        tc_fence_after();
        if (warp < 4 && u >= 1 && k - 2 >= S.seg0) tc_read_chunk(S, k - 2, acc);
        uint32_t t[32];
        tm_ld32(S.tm + lanes + kColE + 64u * buf + col, t);
        tm_wait_ld();
        uint32_t gh[32], gl[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const float g = ex2_approx(__uint_as_float(t[q]));
            gh[q] = tf32_rna(g);
            gl[q] = __float_as_uint(g - __uint_as_float(gh[q]));
        }
        tm_st32(S.tm + lanes + kColGh + 64u * buf + col, gh);
        tm_st32(S.tm + lanes + kColGl + 64u * buf + col, gl);
        tm_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.bars[kBarG + buf]);
    }
    mbar_wait_warp(&S.bars[kBarD], S.blk & 1u, S.abort, S.err);
}

// Difference form on the CUDA cores (tiles whose |q_i|^2 may overflow 2^t):
// rows lane + 32 r of the tile, sources split over the 9 warps, warp partials
// reduced in shared memory.  q = tile-centred coordinates (cx, cy).
__device__ void tc_fallback_block(const float4* raw, int L, float cx, float cy, const float (&qx)[4],
                                  const float (&qy)[4], float (&acc)[4][6])
{
    constexpr int W = kTcThreads / 32;
    const int warp = threadIdx.x >> 5;
    const int ja = warp * L / W, jb = (warp + 1) * L / W;
    for (int j = ja; j < jb; ++j) {
        const float4 v = raw[j];
        const float x = v.x - cx, y = v.y - cy;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float dx = qx[r] - x, dy = qy[r] - y;
            const float G = ex2_approx(-fmaf(dx, dx, dy * dy));
            const float gx = G * dx, gy = G * dy;
            acc[r][0] = fmaf(G, v.z, acc[r][0]);
            acc[r][1] = fmaf(G, v.w, acc[r][1]);
            acc[r][2] = fmaf(gx, v.z, acc[r][2]);
            acc[r][3] = fmaf(gx, v.w, acc[r][3]);
            acc[r][4] = fmaf(gy, v.z, acc[r][4]);
            acc[r][5] = fmaf(gy, v.w, acc[r][5]);
        }
    }
}

// One tile segment [j0, j1) of tile b: writes the six FP32 partial sums of each
// of the tile's particles to slot[k * 128 + r].
__device__ void tc_segment(const StageArgs& a, int b, int j0, int j1, unsigned char* smem, TcState& S, float* slot,
                           float (*s_box)[4])
{
    constexpr int NT = kTcThreads;
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n;
    float4* raw = reinterpret_cast<float4*>(smem + kOffRaw);
    const uint32_t uA1 = smem_u32(smem + kOffA1), uB1 = smem_u32(smem + kOffB1), uB2 = smem_u32(smem + kOffB2);

    // tile rows (threads 0..127) and the centre of their bounding box
    float qx = 0.0f, qy = 0.0f;
    {
        float mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY;
        if (tid < kTcM) {
            const int i = b * kTcM + tid;
            const float4 v = __ldcg(a.S_in + (i < n ? i : b * kTcM));
            qx = v.x;
            qy = v.y;
            mnx = mxx = qx;
            mny = mxy = qy;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
            mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
            mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
            mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
        }
        if (lane == 0 && warp < 4) {
            s_box[warp][0] = mnx;
            s_box[warp][1] = mxx;
            s_box[warp][2] = mny;
            s_box[warp][3] = mxy;
        }
    }
    __syncthreads();
    const float cx = 0.5f * (fminf(fminf(s_box[0][0], s_box[1][0]), fminf(s_box[2][0], s_box[3][0])) +
                             fmaxf(fmaxf(s_box[0][1], s_box[1][1]), fmaxf(s_box[2][1], s_box[3][1])));
    const float cy = 0.5f * (fminf(fminf(s_box[0][2], s_box[1][2]), fminf(s_box[2][2], s_box[3][2])) +
                             fmaxf(fmaxf(s_box[0][3], s_box[1][3]), fmaxf(s_box[2][3], s_box[3][3])));
    qx -= cx;
    qy -= cy;
    const float mq = tid < kTcM ? fmaf(qx, qx, qy * qy) : 0.0f;
    const bool factored = !__syncthreads_or(mq > kTcFactorMax);

    if (!factored) {
        // difference form: every lane holds rows lane + 32 r
        float fx[4], fy[4], acc[4][6];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = b * kTcM + lane + 32 * r;
            const float4 v = __ldcg(a.S_in + (i < n ? i : b * kTcM));
            fx[r] = v.x - cx;
            fy[r] = v.y - cy;
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[r][k] = 0.0f;
        }
        for (int jb = j0; jb < j1; jb += kTcLB) {
            const int L = min(kTcLB, j1 - jb);
            __syncthreads();
            for (int t = tid; t < L; t += NT) raw[t] = __ldcg(a.S_in + jb + t);
            __syncthreads();
            tc_fallback_block(raw, L, cx, cy, fx, fy, acc);
        }
        __syncthreads();
        float* red = reinterpret_cast<float*>(smem + kOffB1);  // [NW][6][128]
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < 6; ++k) red[(warp * 6 + k) * kTcM + lane + 32 * r] = acc[r][k];
        __syncthreads();
        for (int t = tid; t < 6 * kTcM; t += NT) {
            float s = 0.0f;
            for (int w = 0; w < NW; ++w) s += red[w * 6 * kTcM + t];
            slot[t] = s;
        }
        return;
    }

    // A1 rows (tf32 hi/lo split of the tile-centred coordinates)
    if (tid < kTcM) {
        const float xh = tf32_hi(qx), yh = tf32_hi(qy), xl = tf32_lo(qx), yl = tf32_lo(qy);
        float* row0 = reinterpret_cast<float*>(smem + kOffA1 + (tid / 8) * 256 + (tid % 8) * 16);
        float* row1 = row0 + 32;  // + 128 bytes: K elements 4..7
        row0[0] = xh; row0[1] = yh; row0[2] = 1.0f; row0[3] = xl;
        row1[0] = yl; row1[1] = xh; row1[2] = yh; row1[3] = 1.0f;
    }
    float acc[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};  // warps 0..3: row tid's sums
    S.seg0 = S.kc;
    for (int jb = j0; jb < j1; jb += kTcLB) {
        const int L = min(kTcLB, j1 - jb);
        const int Lp = (L + kTcNC - 1) / kTcNC * kTcNC;
        const int nb = Lp / kTcNC;
        // raw records; the padding (q = centre, p = 0) contributes nothing
        for (int t = tid; t < Lp; t += NT)
            raw[t] = t < L ? __ldcg(a.S_in + jb + t) : make_float4(cx, cy, 0.0f, 0.0f);
        __syncthreads();
        // B1: a warp writes 16 sources x 2 K-halves = 512 contiguous bytes
        for (int base = warp * 16; base < Lp; base += NW * 16) {
            const int jl = base + (lane & 15), kh = lane >> 4;
            const float4 v = raw[jl];
            const float x = v.x - cx, y = v.y - cy;
            const float X = 2.0f * x, Y = 2.0f * y, P = -fmaf(x, x, y * y);
            const float4 o = kh == 0 ? make_float4(tf32_hi(X), tf32_hi(Y), tf32_hi(P), tf32_hi(X))
                                     : make_float4(tf32_hi(Y), tf32_lo(X), tf32_lo(Y), tf32_lo(P));
            *reinterpret_cast<float4*>(smem + kOffB1 + (jl / 8) * 256 + kh * 128 + (jl % 8) * 16) = o;
        }
        // B2: thread (source group g of 4, column n8) writes columns n8 and n8 + 8
        const int sbo2 = Lp * 32;
        for (int item = tid; item < (Lp / 4) * 8; item += NT) {
            const int n8 = item & 7, g = item >> 3;
            float c0[4], c1[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = raw[4 * g + q];
                const float x = v.x - cx, y = v.y - cy;
                c0[q] = v_col(n8, v.z, v.w, x, y);
                c1[q] = v_col(n8 + 8, v.z, v.w, x, y);
            }
            *reinterpret_cast<float4*>(smem + kOffB2 + g * 128 + n8 * 16) = make_float4(c0[0], c0[1], c0[2], c0[3]);
            *reinterpret_cast<float4*>(smem + kOffB2 + sbo2 + g * 128 + n8 * 16) =
                make_float4(c1[0], c1[1], c1[2], c1[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (warp == kTcExpW) {
            tc_fence_after();
            if (lane == 0 && !*S.abort) tc_issue_block(S, uA1, uB1, uB2, nb, Lp);
            __syncwarp();
        } else {
            tc_exp_block(S, nb, acc);
        }
        S.kc += (uint32_t)nb;
        S.blk += 1u;
        tc_fence_before();
        __syncthreads();
    }
    // the last one or two chunks' sums, then the partial sums (warps 0..3: row = tid)
    if (warp < 4) {
        tc_fence_after();
        if (!*S.abort) {
            for (uint32_t k = S.kc - min(S.kc - S.seg0, 2u); k < S.kc; ++k) tc_read_chunk(S, k, acc);
        }
        const float* s6 = acc;
        const float E = ex2_approx(-fmaf(qx, qx, qy * qy));
        const float d0 = E * s6[0], d1 = E * s6[1];
        slot[0 * kTcM + tid] = d0;
        slot[1 * kTcM + tid] = d1;
        slot[2 * kTcM + tid] = fmaf(qx, d0, -E * s6[2]);
        slot[3 * kTcM + tid] = fmaf(qx, d1, -E * s6[3]);
        slot[4 * kTcM + tid] = fmaf(qy, d0, -E * s6[4]);
        slot[5 * kTcM + tid] = fmaf(qy, d1, -E * s6[5]);
        tc_fence_before();
    }
}

// The persistent shoot (mode RK4: 4 * steps stages) or one RHS evaluation
// (mode RHS: one stage, input Sx).
__global__ void __launch_bounds__(kTcThreads, 1)
    k_shoot_tc(StageArgs a, const float4* Sx, float4* Sa, float4* Sb, int steps, unsigned* bar, int* err, float* part)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_bars[kNumBars];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    __shared__ int s_last;
    __shared__ float s_box[4][4];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int n = a.n;
    if (tid == 0) {
        for (int k = 0; k < kNumBars; ++k) mbar_init(&s_bars[k], (k == kBarG || k == kBarG + 1) ? kTcExpW : 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kTcExpW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    TcState S{s_bars, s_tmem, 0u, 0u, 0u, &s_abort, err};
    a.Sx = Sx;
    const int nst = a.mode == MODE_RHS ? 1 : 4 * steps;
    unsigned epoch = 0;
    for (int st = 0; st < nst; ++st) {
        const int stage = st & 3;
        a.stage = stage;
        if (a.mode == MODE_RHS) {
            a.S_in = Sx;
        } else {
            a.S_in = stage == 0 ? Sx : (stage == 2 ? Sb : Sa);
            a.S_out = stage == 1 ? Sb : Sa;
        }
        long long u0 = (long long)blockIdx.x * a.U / a.G;
        const long long u1 = (long long)(blockIdx.x + 1) * a.U / a.G;
        while (u0 < u1) {
            const int b = (int)(u0 / n);
            const int j0 = (int)(u0 - (long long)b * n);
            const int j1 = (int)min((long long)n, (long long)j0 + (u1 - u0));
            float* slot = part + (size_t)(blockIdx.x + b) * 6 * kTcM;
            __syncthreads();
            tc_segment(a, b, j0, j1, smem, S, slot, s_box);
            // arrival at tile b; the last CTA sums the slots (CTA order, FP64) and applies the stage
            __threadfence();
            __syncthreads();
            const long long ub = (long long)b * n;
            const int c0 = cta_of_unit(ub, a.U, a.G), c1 = cta_of_unit(ub + n - 1, a.U, a.G);
            if (tid == 0) {
                const int prev = atomicAdd(a.counters + b, 1);
                s_last = prev == c1 - c0;
            }
            __syncthreads();
            if (s_last) {
                __threadfence();
                if (tid < kTcM) {
                    const int i = b * kTcM + tid;
                    if (i < n) {
                        double kk[kKWidth];
#pragma unroll
                        for (int k = 0; k < kKWidth; ++k) kk[k] = 0.0;
                        for (int c = c0; c <= c1; ++c) {
                            const float* sl = part + (size_t)(c + b) * 6 * kTcM;
#pragma unroll
                            for (int k = 0; k < 6; ++k) kk[k] += (double)__ldcg(sl + k * kTcM + tid);
                        }
                        epilogue_mixed_k<2>(a, i, kk);
                    }
                }
                if (tid == 0) a.counters[b] = 0;
            }
            u0 += (j1 - j0);
        }
        if (st + 1 < nst && !grid_barrier(bar, err, ++epoch)) break;
    }
    // teardown: no tensor-core work may be in flight when the columns are freed
    __syncthreads();
    if (warp == kTcExpW) {
        if ((tid & 31) == 0) {
            mma_commit(&s_bars[kBarFin]);
            uint64_t t0 = globaltimer();
            while (!mbar_try(&s_bars[kBarFin], 0) && globaltimer() - t0 < kWaitNs) {
            }
        }
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(s_tmem) : "memory");
    }
}

}  // namespace

bool tc_enabled(const ep_params& P)
{
    if (!(P.dim == 2 && P.kernel == EP_GAUSS && P.precision == EP_MIXED)) return false;
    const char* e = getenv("EP_TC");  // opt-in, read per call: a process may switch paths
    return e && e[0] == '1';
}

size_t tc_part_floats(int n, int sm_count)
{
    const int tiles = (n + kTcM - 1) / kTcM;
    return (size_t)(sm_count + tiles) * 6 * kTcM;
}

int tc_tiles(int n) { return (n + kTcM - 1) / kTcM; }

ep_status tc_run(const ep_params& P, const AllPairsBufs& b, int steps, double dt, int mode, double* out_q,
                 double* out_p, int G, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1)
{
    if (b.n == 0) return EP_OK;
    if (!b.part) return set_error("tensor-core path: no partial-sum buffer"), EP_EINVAL;
    static int resident = -1;
    if (resident < 0) {
        EP_TRY_CUDA(cudaFuncSetAttribute(k_shoot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
        int per_sm = 0;
        EP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shoot_tc, kTcThreads, kTcSmem));
        DeviceInfo di{};
        EP_TRY(device_info(&di));
        resident = std::min(per_sm, 1) * di.sm_count;  // tensor memory: one CTA per SM
    }
    if (resident < 1) return set_error("tensor-core shoot: kernel does not fit on an SM"), EP_EINVAL;
    APConfig cfg;
    cfg.threads = kTcThreads;
    cfg.ctas = G;
    StageArgs a = base_args(P, b, cfg);
    a.U = (long long)tc_tiles(b.n) * b.n;
    a.G = (int)std::min<long long>(std::max(1, std::min(G, resident)), a.U);
    a.mode = mode;
    a.dt = dt;
    a.dt_f = (float)dt;
    a.out_q = out_q;
    a.out_p = out_p;
    a.Sx_w = b.Sx;
    const float4* Sx = b.Sx;
    float4* Sa = b.Sa;
    float4* Sb = b.Sb;
    unsigned* bar = b.bar;
    int* err = b.err;
    float* part = b.part;
    EP_TRY_CUDA(cudaMemsetAsync(b.bar, 0, sizeof(unsigned) * 9, st));
    void* args[] = {&a, &Sx, &Sa, &Sb, &steps, &bar, &err, &part};
    count_launch();
    if (ev0) EP_TRY_CUDA(cudaEventRecord(ev0, st));
    EP_TRY_CUDA(cudaLaunchCooperativeKernel((void*)k_shoot_tc, dim3(a.G), dim3(kTcThreads), args, kTcSmem, st));
    if (ev1) EP_TRY_CUDA(cudaEventRecord(ev1, st));
    int herr = 0;
    EP_TRY_CUDA(cudaMemcpyAsync(&herr, b.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    if (herr) {
        set_error(herr == 2 ? "tensor-core shoot: a pipeline wait gave up (kernel ended early)"
                            : "tensor-core shoot: a grid-barrier wait gave up (kernel ended early)");
        return EP_ETIMEOUT;
    }
    return EP_OK;
}

}  // namespace ep
