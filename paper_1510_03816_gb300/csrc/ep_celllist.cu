// ep_celllist.cu -- uniform-grid cell list for the compactly supported tent
// kernel G = max(1 - r/sigma, 0) (2-D): the sums of Eq. N-particle restricted
// to pairs closer than sigma, with the RK4 stage fused into the sweep.
//
// Grid (fixed for one call, from the call's starting positions q):
//   h = sigma (1 + 2^-8);  lo_c = min_c q - 2h;  nc_c = min(floor((max - min)/h) + 5, 2048)
//   (when capped, h_c = (max - min + 4h) / 2047); particles that later leave the
//   grid are clamped into its border cells, which keeps every pair closer than
//   sigma in adjacent cells.
// A particle is stored as its cell (cx, cy) and its FP32 offset from the cell's
// lower corner in units of sigma: o = (float)((q - lo - cell h) / sigma).  Offsets
// are small numbers, so the pair difference
//   d = (o_i - o_j) + (cell_i - cell_j) e,   e = (float)(h / sigma)
// is accurate to ~1e-7 sigma even for sigma ~ 6e-3, where FP32 absolute
// positions would only resolve ~1e-5 sigma.  A pair is accepted iff
// fmaf(d0, d0, d1 * d1) < 1.0f (the definition ep_cell_neighbors exposes).
//
// One stage = block-wise exclusive scan of the cell counts (the last block scans
// the block totals) -> scatter into cell order -> sweep: each CTA owns an 8 x 8
// block of cells, stages the records of its 10 x 10 halo in shared memory with
// each cell's records ordered by particle index (so sums do not depend on the
// order atomics gave), and every thread sums the 3 x 3 neighbour cells of
// kSweepRI particles of one cell in FP32, then applies the RK4 stage and bins
// each particle for the next stage (cell count by atomics).  (Measured on the
// 512 x 512 grid: one particle per thread is as fast as two to four sharing each
// record load; the sweep is bound by the CTAs' low warp occupancy.)  Stage positions inside a step are
// anchor + c dt k in FP32 on the offsets (re-celled by floor(o / e)); the step
// state x is FP64 and the anchor is re-derived from it in FP64 every step.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ep_features.cuh"

namespace ep {

namespace {

constexpr int kBlk = 8;                        // cells per sweep block side
constexpr int kHalo = kBlk + 2;
constexpr int kSweepThreads = 256;
constexpr int kSweepRI = 1;                    // particles of one cell per sweep thread
constexpr int kSweepCap = 2048;                // halo records staged in shared memory (~2x the mean halo)
constexpr int kScanBlock = 4096;               // cells per scan block (1024 threads x 4)
constexpr int kMaxCellsPerAxis2D = 2048;
// Slot layout: cell k's records at slots [k kSlotCap, k kSlotCap + count[k]), written by
// the binning itself, so a stage needs no scan and no scatter.  Used while the grid's
// slots fit kSlotFactor n and no cell holds more than kSlotCap particles; a cell that
// overflows raises a flag and the next stage takes the scanned layout instead.
constexpr int kSlotCap = 32;
constexpr int kSlotFactor = 8;

struct Grid {
    double lo[2], h[2], inv_h[2];
    int nc[2];
    long long ncell;
    float e[2];
    double inv_sigma;
};

// Remaining device buffers (carved from the arena after CellBufs::x).
struct Impl {
    int2* cellX;     // step-start cells (stage-0 input)
    float4* recX;    // step-start records (o.x, o.y, p.x, p.y)
    int2* cellA;
    float4* recA;
    int2* cellB;
    float4* recB;
    float* acc;      // FP32 RK4 accumulator (n x 4)
    int* key;
    int* rank;
    int* sidx;       // particle index of each sorted slot
    float4* srec;    // records in cell order
    int* count[3];   // per cell (rotating by stage: read, binned into, zeroed), then local exclusive scan
    float4* frec[2]; // slot layout of the records (by stage parity)
    int* fidx[2];    // slot layout of the particle indices
    int* ovf;        // [3] per count buffer: a cell's count exceeded kSlotCap
    int* bsum;       // per scan block total, then exclusive block offsets
    int* scan_ctr;   // arrival counter of the block scan
    double* bbox;    // keys (k_bbox2) of min x, min y, max x, max y
    Grid g;
    int cur;         // count buffer holding the next stage's bins
    int par;         // slot layout the next stage reads
    int slots;       // the grid's slots fit (kSlotCap ncell <= kSlotFactor n)
};

static_assert(sizeof(Impl) <= 1024, "Impl must fit the CellBufs host block");

struct Args {
    int n;
    int mode;   // 0 RK4 stage, 1 RHS, 2 neighbour count
    int stage;
    float dt_f;
    float dp_scale_f;
    double dp_scale;
    double sigma;
    Grid g;
    const int* count;   // local scan (scanned layout) or cell counts (slot layout)
    const int* boff;    // block offsets
    int* count_next;    // bins of the next stage
    int* count_zero;    // the count buffer of the stage after next, zeroed here
    int slots;          // slot layout available for this grid
    const int* ovf_in;  // a cell of this stage's bins overflowed: scanned layout
    int* ovf_out;       // raised when a next-stage bin overflows
    int* ovf_zero;      // the flag of the stage after next, cleared here
    const float4* frec_in;
    const int* fidx_in;
    float4* frec_out;
    int* fidx_out;
    int* key_out;
    int* rank_out;
    const int* sidx;
    const float4* srec;
    const int2* cellX;
    const float4* recX;
    int2* cellOut;
    float4* recOut;
    float* acc;
    double* x;
    double* out_q;
    double* out_p;
    long long* out_cnt;
    unsigned long long* out_hash;
};

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int cell_start(const int* count, const int* boff, long long c)
{
    return count[c] + boff[c / kScanBlock];
}

// (cell, offset) of an FP64 position, per the written definition (no contraction).
__device__ __forceinline__ void locate(double q, int axis, const Grid& g, int& cell, float& off)
{
    const double t = __dsub_rn(q, g.lo[axis]);
    double k = floor(__dmul_rn(t, g.inv_h[axis]));
    k = fmin(fmax(k, 0.0), (double)(g.nc[axis] - 1));
    cell = (int)k;
    off = (float)__dmul_rn(__dsub_rn(t, __dmul_rn(k, g.h[axis])), g.inv_sigma);
}

// ------------------------------------------------------------------ kernels
// Order-preserving map of a double to an unsigned key (negative values flipped
// whole, non-negative ones get the sign bit), so min / max become integer atomics.
__device__ __forceinline__ unsigned long long dkey(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
inline double dkey_value(unsigned long long k)
{
    const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    double v;
    memcpy(&v, &b, sizeof v);
    return v;
}

// Bounding box of the n positions q (2-D), NaN coordinates ignored: each CTA
// reduces a grid-strided share and merges it into out[0..3] (keys of min x, min y,
// max x, max y; initialised to the identities) by integer atomics.
__global__ void __launch_bounds__(256) k_bbox2(const double* __restrict__ q, int n, unsigned long long* out)
{
    __shared__ unsigned long long s[4][8];
    unsigned long long v[4] = {~0ull, ~0ull, 0ull, 0ull};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double a = q[2 * (size_t)i], b = q[2 * (size_t)i + 1];
        if (a == a) {
            const unsigned long long k = dkey(a);
            v[0] = min(v[0], k);
            v[2] = max(v[2], k);
        }
        if (b == b) {
            const unsigned long long k = dkey(b);
            v[1] = min(v[1], k);
            v[3] = max(v[3], k);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = min(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
        v[1] = min(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
        v[2] = max(v[2], __shfl_xor_sync(0xffffffffu, v[2], o));
        v[3] = max(v[3], __shfl_xor_sync(0xffffffffu, v[3], o));
    }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 4; ++k) s[k][threadIdx.x >> 5] = v[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        const int k = threadIdx.x;
        unsigned long long r = s[k][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = k < 2 ? min(r, s[k][w]) : max(r, s[k][w]);
        if (k < 2) atomicMin(out + k, r);
        else atomicMax(out + k, r);
    }
}

// x = (q, p) and the step-start cells / records from FP64.
__global__ void k_cell_anchor(const double* __restrict__ q, const double* __restrict__ p, int n, Grid g,
                              double* __restrict__ x, int2* __restrict__ cellX, float4* __restrict__ recX,
                              int* __restrict__ count, int* __restrict__ key, int* __restrict__ rank, int slots,
                              float4* __restrict__ frec, int* __restrict__ fidx, int* __restrict__ ovf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double qx = q[2 * (size_t)i], qy = q[2 * (size_t)i + 1];
    const double px = p[2 * (size_t)i], py = p[2 * (size_t)i + 1];
    if (x) {
        x[2 * (size_t)i] = qx;
        x[2 * (size_t)i + 1] = qy;
        x[2 * (size_t)n + 2 * (size_t)i] = px;
        x[2 * (size_t)n + 2 * (size_t)i + 1] = py;
    }
    int cx, cy;
    float ox, oy;
    locate(qx, 0, g, cx, ox);
    locate(qy, 1, g, cy, oy);
    cellX[i] = make_int2(cx, cy);
    const float4 r = make_float4(ox, oy, (float)px, (float)py);
    recX[i] = r;
    const int k = cy * g.nc[0] + cx;
    key[i] = k;
    const int rk = atomicAdd(count + k, 1);
    rank[i] = rk;
    if (slots) {
        if (rk < kSlotCap) {
            frec[(size_t)k * kSlotCap + rk] = r;
            fidx[(size_t)k * kSlotCap + rk] = i;
        } else {
            *ovf = 1;
        }
    }
}

// Exclusive scan of 4 x 1024 values in place (one CTA); returns nothing.
__device__ void cta_exclusive_scan4(int* __restrict__ v, long long count, int* sw, bool cg)
{
    const long long base = 4LL * threadIdx.x;
    int x[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        x[k] = (base + k < count) ? (cg ? __ldcg(v + base + k) : v[base + k]) : 0;
        s += x[k];
    }
    int incl = s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sw[w] = incl;
    __syncthreads();
    if (w == 0) {
        int t = sw[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        sw[lane] = t;
    }
    __syncthreads();
    int run = incl - s + (w > 0 ? sw[w - 1] : 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < count) v[base + k] = run;
        run += x[k];
    }
}

// Exclusive scan of the cell counts within blocks of kScanBlock cells; bsum[b] =
// block total.  The last block to finish scans the block totals into block
// offsets.  Only for the scanned layout: with the slot layout in use (slots and no
// overflow flag) the kernel returns at once.
__global__ void __launch_bounds__(1024) k_scan_local(int* __restrict__ count, long long ncell, int* __restrict__ bsum,
                                                     int* __restrict__ ctr, int nb, int slots, const int* __restrict__ ovf)
{
    __shared__ int sw[32];
    __shared__ int last;
    if (slots && *ovf == 0) return;
    int* blk = count + (long long)blockIdx.x * kScanBlock;
    const long long cnt = min((long long)kScanBlock, ncell - (long long)blockIdx.x * kScanBlock);
    // block total first (the scan overwrites the counts)
    int s = 0;
    for (int k = 0; k < 4; ++k) {
        const long long c = 4LL * threadIdx.x + k;
        if (c < cnt) s += blk[c];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int k = 0; k < 32; ++k) t += sw[k];
        bsum[blockIdx.x] = t;
    }
    __syncthreads();
    cta_exclusive_scan4(blk, cnt, sw, false);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(ctr, 1) == nb - 1);
    __syncthreads();
    if (last) {
        __threadfence();
        cta_exclusive_scan4(bsum, nb, sw, true);
        if (threadIdx.x == 0) *ctr = 0;
    }
}

__global__ void k_cell_scatter(const int* __restrict__ key, const int* __restrict__ rank, const int* __restrict__ count,
                               const int* __restrict__ boff, const float4* __restrict__ recIn, int n,
                               int* __restrict__ sidx, float4* __restrict__ srec, int slots, const int* __restrict__ ovf)
{
    if (slots && *ovf == 0) return;  // the slot layout is in use
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k = key[i];
        const int slot = cell_start(count, boff, k) + rank[i];
        sidx[slot] = i;
        srec[slot] = recIn[i];
    }
}

// Finish particle i: RHS output, or the RK4 stage plus the binning of the
// particle's next-stage cell (key, rank within the cell).
__device__ void epilogue(const Args& a, int i, float dqx, float dqy, float dpx, float dpy)
{
    if (a.mode == 1) {
        a.out_q[2 * (size_t)i] = (double)dqx;
        a.out_q[2 * (size_t)i + 1] = (double)dqy;
        a.out_p[2 * (size_t)i] = a.dp_scale * (double)dpx;
        a.out_p[2 * (size_t)i + 1] = a.dp_scale * (double)dpy;
        return;
    }
    const float kq0 = dqx, kq1 = dqy, kp0 = a.dp_scale_f * dpx, kp1 = a.dp_scale_f * dpy;
    float* A = a.acc + 4 * (size_t)i;
    int c0, c1;
    if (a.stage < 3) {
        const float cdt = (a.stage == 2 ? 1.0f : 0.5f) * a.dt_f;
        const float bw = a.stage == 0 ? 1.0f : 2.0f;
        const int2 ax = a.cellX[i];
        const float4 rx = a.recX[i];
        const float is = (float)a.g.inv_sigma;
        // stage position: anchor offset + c dt kq (units of sigma), re-celled
        float o0 = fmaf(cdt * is, kq0, rx.x), o1 = fmaf(cdt * is, kq1, rx.y);
        c0 = ax.x + (int)floorf(o0 / a.g.e[0]);
        c1 = ax.y + (int)floorf(o1 / a.g.e[1]);
        c0 = min(max(c0, 0), a.g.nc[0] - 1);
        c1 = min(max(c1, 0), a.g.nc[1] - 1);
        o0 -= (float)(c0 - ax.x) * a.g.e[0];
        o1 -= (float)(c1 - ax.y) * a.g.e[1];
        a.cellOut[i] = make_int2(c0, c1);
        a.recOut[i] = make_float4(o0, o1, fmaf(cdt, kp0, rx.z), fmaf(cdt, kp1, rx.w));
        if (a.stage == 0) {
            A[0] = kq0; A[1] = kq1; A[2] = kp0; A[3] = kp1;
        } else {
            A[0] = fmaf(bw, kq0, A[0]); A[1] = fmaf(bw, kq1, A[1]);
            A[2] = fmaf(bw, kp0, A[2]); A[3] = fmaf(bw, kp1, A[3]);
        }
    } else {
        const int n = a.n;
        double* xq = a.x + 2 * (size_t)i;
        double* xp = a.x + 2 * (size_t)n + 2 * (size_t)i;
        const float f = a.dt_f * (1.0f / 6.0f);
        const double q0 = xq[0] + (double)(f * (A[0] + kq0)), q1 = xq[1] + (double)(f * (A[1] + kq1));
        const double p0 = xp[0] + (double)(f * (A[2] + kp0)), p1 = xp[1] + (double)(f * (A[3] + kp1));
        xq[0] = q0; xq[1] = q1; xp[0] = p0; xp[1] = p1;
        float o0, o1;
        locate(q0, 0, a.g, c0, o0);
        locate(q1, 1, a.g, c1, o1);
        a.cellOut[i] = make_int2(c0, c1);
        a.recOut[i] = make_float4(o0, o1, (float)p0, (float)p1);
    }
    const int k = c1 * a.g.nc[0] + c0;
    a.key_out[i] = k;
    const int rk = atomicAdd(a.count_next + k, 1);
    a.rank_out[i] = rk;
    if (a.slots) {
        if (rk < kSlotCap) {
            a.frec_out[(size_t)k * kSlotCap + rk] = a.recOut[i];
            a.fidx_out[(size_t)k * kSlotCap + rk] = i;
        } else {
            *a.ovf_out = 1;
        }
    }
}

// Exclusive prefix sum of NV values (NV <= 4 x 32) by one warp: out[t] for t < NV,
// out[NV] = total.
template <int NV, typename F>
__device__ __forceinline__ void warp_exclusive_scan(F value, int* out)
{
    constexpr int PER = (NV + 31) / 32;
    const int lane = threadIdx.x & 31;
    int v[PER], s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int t = PER * lane + k;
        v[k] = t < NV ? value(t) : 0;
        s += v[k];
    }
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    int run = incl - s;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int t = PER * lane + k;
        if (t < NV) out[t] = run;
        run += v[k];
    }
    if (lane == 31) out[NV] = incl;
}

// Largest t in [0, n) with pre[t] <= u (pre non-decreasing, pre[0] <= u < pre[n]).
__device__ __forceinline__ int find_segment(const int* pre, int n, int u)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}

// One CTA per 8 x 8 block of cells.  Halo cell t = hy * 10 + hx covers grid cell
// (cx0 - 1 + hx, cy0 - 1 + hy).  The halo's records are staged in shared memory,
// each cell's records ordered by particle index (every staged record finds its
// rank among its cell's members), so the sums do not depend on the order the
// binning atomics gave.  A thread then takes RI particles of one own cell and sums
// their 3 x 3 neighbour cells, each loaded record serving the RI particles; the
// pair terms are predicated (a rejected pair adds exact zeros), in the order
// rows dy, cells dx, records by particle index.  MODE: 0 RK4 stage, 1 RHS,
// 2 neighbour count and hash.
template <int MODE, int RI>
__global__ void __launch_bounds__(kSweepThreads) k_cell_sweep(Args a)
{
    constexpr int NH = kHalo * kHalo;
    constexpr int NO = kBlk * kBlk;
    __shared__ float4 s_rec[kSweepCap];
    __shared__ int s_idx[kSweepCap];
    __shared__ int c_start[NH + 1];  // exclusive prefix of the halo cell lengths
    __shared__ int c_len[NH];
    __shared__ int c_gs[NH];         // global slot of each halo cell's first record
    __shared__ int t_pre[NO + 1];    // exclusive prefix of the tasks per own cell
    const int warp = threadIdx.x >> 5;
    const int ncx = a.g.nc[0], ncy = a.g.nc[1];
    const int cx0 = blockIdx.x * kBlk, cy0 = blockIdx.y * kBlk;
    // this stage's layout: slots (each cell at k kSlotCap, count[k] long) or scanned
    const bool use_slots = a.slots && *a.ovf_in == 0;
    for (int t = threadIdx.x; t < NH; t += kSweepThreads) {
        const int hx = t % kHalo, hy = t / kHalo;
        const int row = cy0 - 1 + hy, col = cx0 - 1 + hx;
        int gs = 0, len = 0;
        if (row >= 0 && row < ncy && col >= 0 && col < ncx) {
            const long long c = (long long)row * ncx + col;
            if (use_slots) {
                gs = (int)(c * kSlotCap);
                len = a.count[c];
            } else {
                gs = cell_start(a.count, a.boff, c);
                const int ge = (c + 1 < a.g.ncell) ? cell_start(a.count, a.boff, c + 1) : a.n;
                len = ge - gs;
            }
        }
        c_gs[t] = gs;
        c_len[t] = len;
    }
    // the bins of the stage after next start from zero: this CTA's own cells
    if (a.count_zero) {
        for (int t = threadIdx.x; t < kBlk * kBlk; t += kSweepThreads) {
            const int row = cy0 + t / kBlk, col = cx0 + t % kBlk;
            if (row < ncy && col < ncx) a.count_zero[(long long)row * ncx + col] = 0;
        }
        if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *a.ovf_zero = 0;
    }
    const int* gidx = use_slots ? a.fidx_in : a.sidx;
    const float4* grec = use_slots ? a.frec_in : a.srec;
    __syncthreads();
    if (warp == 0) warp_exclusive_scan<NH>([&](int t) { return c_len[t]; }, c_start);
    if (warp == 1)
        warp_exclusive_scan<NO>([&](int k) { return (c_len[((k / kBlk) + 1) * kHalo + (k % kBlk) + 1] + RI - 1) / RI; },
                                t_pre);
    __syncthreads();
    const bool sm = c_start[NH] <= kSweepCap;
    if (sm) {
        const int tot = c_start[NH];
        for (int u = threadIdx.x; u < tot; u += kSweepThreads) {
            const int t = find_segment(c_start, NH, u);
            const int g0 = c_gs[t], len = c_len[t];
            const int g = g0 + (u - c_start[t]);
            const int my = __ldg(gidx + g);
            int rank = 0;
            for (int v = 0; v < len; ++v) rank += __ldg(gidx + g0 + v) < my ? 1 : 0;
            s_idx[c_start[t] + rank] = my;
            s_rec[c_start[t] + rank] = __ldg(grec + g);
        }
        __syncthreads();
    }
    const float4* rec = sm ? s_rec : grec;
    const int* idx = sm ? s_idx : gidx;
    const int* cst = sm ? c_start : c_gs;
    const float e0 = a.g.e[0], e1 = a.g.e[1];
    const int ntask = t_pre[NO];
    for (int task = threadIdx.x; task < ntask; task += kSweepThreads) {
        const int kc = find_segment(t_pre, NO, task);
        const int h = ((kc / kBlk) + 1) * kHalo + (kc % kBlk) + 1;
        const int first = (task - t_pre[kc]) * RI;
        const int nact = min(RI, c_len[h] - first);
        float4 ri[RI];
        int ii[RI];
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int u = cst[h] + first + (r < nact ? r : 0);
            ri[r] = rec[u];
            ii[r] = idx[u];
        }
        float dqx[RI], dqy[RI], dpx[RI], dpy[RI];
        int cnt[RI];
        unsigned long long hs[RI];
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            dqx[r] = dqy[r] = dpx[r] = dpy[r] = 0.0f;
            cnt[r] = 0;
            hs[r] = 0ull;
        }
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int h2 = h + dy * kHalo + dx;
                const int len = c_len[h2], s0 = cst[h2];
                const float sx = __fmul_rn((float)(-dx), e0), sy = __fmul_rn((float)(-dy), e1);
#pragma unroll 2
                for (int v = 0; v < len; ++v) {
                    const float4 rj = rec[s0 + v];
                    int jj = 0;
                    if (MODE == 2) jj = idx[s0 + v];
#pragma unroll
                    for (int r = 0; r < RI; ++r) {
                        const float d0 = __fadd_rn(__fsub_rn(ri[r].x, rj.x), sx);
                        const float d1 = __fadd_rn(__fsub_rn(ri[r].y, rj.y), sy);
                        const float r2 = __fmaf_rn(d0, d0, __fmul_rn(d1, d1));
                        const bool in = r2 < 1.0f;
                        if (MODE == 2) {
                            cnt[r] += in ? 1 : 0;
                            hs[r] += in ? (unsigned long long)(jj + 1) * 2654435761ull : 0ull;
                        } else {
                            const float rs = rsqrt_approx(fmaxf(r2, 1e-30f));
                            const float G = in ? fmaf(-r2, rs, 1.0f) : 0.0f;
                            dqx[r] = fmaf(G, rj.z, dqx[r]);
                            dqy[r] = fmaf(G, rj.w, dqy[r]);
                            const float c2 = in ? rs * fmaf(ri[r].z, rj.z, ri[r].w * rj.w) : 0.0f;
                            dpx[r] = fmaf(c2, d0, dpx[r]);
                            dpy[r] = fmaf(c2, d1, dpy[r]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            if (r < nact) {
                if (MODE == 2) {
                    a.out_cnt[ii[r]] = (long long)cnt[r];
                    a.out_hash[ii[r]] = hs[r];
                } else {
                    epilogue(a, ii[r], dqx[r], dqy[r], dpx[r], dpy[r]);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ host
Impl* impl_of(const CellBufs& b) { return (Impl*)b.host; }

Grid make_grid(const double* bb, double sigma)
{
    Grid g{};
    const double h = sigma * 1.00390625;
    for (int c = 0; c < 2; ++c) {
        const double mn = bb[c], mx = bb[2 + c];
        g.lo[c] = mn - 2.0 * h;
        const double cells = floor((mx - mn) / h) + 5.0;
        if (cells > (double)kMaxCellsPerAxis2D) {
            g.nc[c] = kMaxCellsPerAxis2D;
            g.h[c] = (mx - mn + 4.0 * h) / (double)(kMaxCellsPerAxis2D - 1);
        } else {
            g.nc[c] = (int)cells;
            g.h[c] = h;
        }
        g.inv_h[c] = 1.0 / g.h[c];
    }
    g.inv_sigma = 1.0 / sigma;
    for (int c = 0; c < 2; ++c) g.e[c] = (float)(g.h[c] * g.inv_sigma);
    g.ncell = (long long)g.nc[0] * g.nc[1];
    return g;
}

size_t impl_bytes(int n)
{
    Sizer z;
    for (int k = 0; k < 3; ++k) {
        z.add(sizeof(int2) * (size_t)n);
        z.add(sizeof(float4) * (size_t)n);
    }
    z.add(sizeof(float) * 4 * (size_t)n);
    z.add(sizeof(int) * (size_t)n * 3);
    z.add(sizeof(float4) * (size_t)n);
    const size_t maxcell = (size_t)kMaxCellsPerAxis2D * kMaxCellsPerAxis2D;
    for (int k = 0; k < 3; ++k) z.add(sizeof(int) * maxcell);
    z.add(sizeof(int) * (maxcell / kScanBlock + 1));
    z.add(sizeof(int) * 4);
    z.add(sizeof(double) * 4);
    for (int k = 0; k < 2; ++k) {
        z.add(sizeof(float4) * (size_t)kSlotFactor * n);
        z.add(sizeof(int) * (size_t)kSlotFactor * n);
    }
    z.add(sizeof(int) * 4);
    return z.total;
}

// One stage on the current bins (im->cur): scan, scatter, sweep.  In RK4 mode the
// sweep bins the next stage into the other count buffer and the bins flip.
ep_status run_stage(const ep_params& P, const CellBufs& b, Args a, const float4* recIn, cudaStream_t st)
{
    Impl* im = impl_of(b);
    const Grid& g = im->g;
    const int n = b.n;
    // the scatter strides over the particles with a small grid (so that, with the slot
    // layout in use, its early return costs little)
    DeviceInfo di{};
    EP_TRY(device_info(&di));
    const unsigned gn = (unsigned)std::max(1, std::min((n + 255) / 256, 2 * di.sm_count));
    const int nb = (int)((g.ncell + kScanBlock - 1) / kScanBlock);
    const int cur = im->cur, nx = (cur + 1) % 3, nn = (cur + 2) % 3;
    int* cnt = im->count[cur];
    count_launch(2);
    // scan and scatter run only for the scanned layout (they return at once otherwise)
    k_scan_local<<<nb, 1024, 0, st>>>(cnt, g.ncell, im->bsum, im->scan_ctr, nb, im->slots, im->ovf + cur);
    k_cell_scatter<<<gn, 256, 0, st>>>(im->key, im->rank, cnt, im->bsum, recIn, n, im->sidx, im->srec, im->slots,
                                       im->ovf + cur);
    a.n = n;
    a.g = g;
    a.count = cnt;
    a.boff = im->bsum;
    a.count_next = im->count[nx];
    a.count_zero = a.mode == 0 ? im->count[nn] : nullptr;
    a.slots = im->slots;
    a.ovf_in = im->ovf + cur;
    a.ovf_out = im->ovf + nx;
    a.ovf_zero = im->ovf + nn;
    a.frec_in = im->frec[im->par];
    a.fidx_in = im->fidx[im->par];
    a.frec_out = im->frec[im->par ^ 1];
    a.fidx_out = im->fidx[im->par ^ 1];
    a.key_out = im->key;
    a.rank_out = im->rank;
    a.sidx = im->sidx;
    a.srec = im->srec;
    a.cellX = im->cellX;
    a.recX = im->recX;
    a.acc = im->acc;
    a.x = b.x;
    a.sigma = P.sigma;
    a.dp_scale = 1.0 / P.sigma;
    a.dp_scale_f = (float)(1.0 / P.sigma);
    dim3 grid((unsigned)((g.nc[0] + kBlk - 1) / kBlk), (unsigned)((g.nc[1] + kBlk - 1) / kBlk));
    count_launch();
    if (a.mode == 2)
        k_cell_sweep<2, kSweepRI><<<grid, kSweepThreads, 0, st>>>(a);
    else if (a.mode == 1)
        k_cell_sweep<1, kSweepRI><<<grid, kSweepThreads, 0, st>>>(a);
    else
        k_cell_sweep<0, kSweepRI><<<grid, kSweepThreads, 0, st>>>(a);
    EP_TRY_CUDA(cudaGetLastError());
    if (a.mode == 0) {
        im->cur = nx;
        im->par ^= 1;
    }
    return EP_OK;
}

ep_status check_cell_params(const ep_params& P)
{
    if (P.kernel != EP_TENT) return set_error("the cell list needs the tent kernel"), EP_EINVAL;
    if (P.dim != 2) return set_error("the cell list is built for dim = 2"), EP_EINVAL;
    if (P.precision != EP_MIXED) return set_error("the cell list runs in mixed precision"), EP_EINVAL;
    return EP_OK;
}

// Grid from the bounding box of q (one sync), then the step-start records.
ep_status load_anchor(const ep_params& P, CellBufs& b, const double* q, const double* p, cudaStream_t st,
                      bool write_x)
{
    Impl* im = impl_of(b);
    const int n = b.n;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(im->bbox);
    EP_TRY_CUDA(cudaMemsetAsync(keys, 0xFF, 2 * sizeof(unsigned long long), st));
    EP_TRY_CUDA(cudaMemsetAsync(keys + 2, 0, 2 * sizeof(unsigned long long), st));
    DeviceInfo di{};
    EP_TRY(device_info(&di));
    const int nbb = std::max(1, std::min((n + 255) / 256, 2 * di.sm_count));
    count_launch();
    k_bbox2<<<nbb, 256, 0, st>>>(q, n, keys);
    unsigned long long kb[4];
    EP_TRY_CUDA(cudaMemcpyAsync(kb, keys, sizeof kb, cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    double bb[4];
    for (int k = 0; k < 4; ++k) bb[k] = dkey_value(kb[k]);
    im->g = make_grid(bb, P.sigma);
    im->cur = 0;
    im->par = 0;
    // EP_CELL_SLOTS=0 in the environment keeps the scanned layout (same sums, bit for bit)
    const char* es = getenv("EP_CELL_SLOTS");
    im->slots = (im->g.ncell * kSlotCap <= (long long)kSlotFactor * n && !(es && es[0] == '0')) ? 1 : 0;
    EP_TRY_CUDA(cudaMemsetAsync(im->count[0], 0, sizeof(int) * (size_t)im->g.ncell, st));
    EP_TRY_CUDA(cudaMemsetAsync(im->count[1], 0, sizeof(int) * (size_t)im->g.ncell, st));
    EP_TRY_CUDA(cudaMemsetAsync(im->scan_ctr, 0, sizeof(int) * 4, st));
    EP_TRY_CUDA(cudaMemsetAsync(im->ovf, 0, sizeof(int) * 4, st));
    count_launch();
    k_cell_anchor<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(q, p, n, im->g, write_x ? b.x : nullptr, im->cellX,
                                                                im->recX, im->count[0], im->key, im->rank, im->slots,
                                                                im->frec[0], im->fidx[0], im->ovf);
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

}  // namespace

size_t cell_bytes(int n, int dim, int prec)
{
    (void)prec;
    Sizer z;
    z.add(sizeof(double) * 2 * dim * (size_t)n);
    z.add(impl_bytes(n));
    return z.total;
}

ep_status cell_carve(Arena* ar, int n, int dim, int prec, CellBufs* b)
{
    b->n = n;
    b->dim = dim;
    b->prec = prec;
    b->x = (double*)ar->carve(sizeof(double) * 2 * dim * (size_t)n);
    Impl* im = (Impl*)b->host;
    *im = Impl{};
    im->cellX = (int2*)ar->carve(sizeof(int2) * (size_t)n);
    im->recX = (float4*)ar->carve(sizeof(float4) * (size_t)n);
    im->cellA = (int2*)ar->carve(sizeof(int2) * (size_t)n);
    im->recA = (float4*)ar->carve(sizeof(float4) * (size_t)n);
    im->cellB = (int2*)ar->carve(sizeof(int2) * (size_t)n);
    im->recB = (float4*)ar->carve(sizeof(float4) * (size_t)n);
    im->acc = (float*)ar->carve(sizeof(float) * 4 * (size_t)n);
    im->key = (int*)ar->carve(sizeof(int) * (size_t)n);
    im->rank = (int*)ar->carve(sizeof(int) * (size_t)n);
    im->sidx = (int*)ar->carve(sizeof(int) * (size_t)n);
    im->srec = (float4*)ar->carve(sizeof(float4) * (size_t)n);
    const size_t maxcell = (size_t)kMaxCellsPerAxis2D * kMaxCellsPerAxis2D;
    for (int k = 0; k < 3; ++k) im->count[k] = (int*)ar->carve(sizeof(int) * maxcell);
    im->bsum = (int*)ar->carve(sizeof(int) * (maxcell / kScanBlock + 1));
    im->scan_ctr = (int*)ar->carve(sizeof(int) * 4);
    im->bbox = (double*)ar->carve(sizeof(double) * 4);
    for (int k = 0; k < 2; ++k) {
        im->frec[k] = (float4*)ar->carve(sizeof(float4) * (size_t)kSlotFactor * n);
        im->fidx[k] = (int*)ar->carve(sizeof(int) * (size_t)kSlotFactor * n);
    }
    im->ovf = (int*)ar->carve(sizeof(int) * 4);
    if (!im->ovf) return set_error("workspace too small for the cell list"), EP_ENOMEM;
    return EP_OK;
}

ep_status cell_load(const ep_params& P, CellBufs& b, const double* q, const double* p, cudaStream_t st)
{
    EP_TRY(check_cell_params(P));
    if (b.n == 0) return EP_OK;
    return load_anchor(P, b, q, p, st, true);
}

ep_status cell_rhs(const ep_params& P, const CellBufs& b, double* dq, double* dp, cudaStream_t st)
{
    if (b.n == 0) return EP_OK;
    Impl* im = impl_of(b);
    Args a{};
    a.mode = 1;
    a.out_q = dq;
    a.out_p = dp;
    return run_stage(P, b, a, im->recX, st);
}

ep_status cell_steps(const ep_params& P, const CellBufs& b, int steps, double dt, cudaStream_t st)
{
    if (b.n == 0) return EP_OK;
    Impl* im = impl_of(b);
    Args a{};
    a.mode = 0;
    a.dt_f = (float)dt;
    for (int s = 0; s < steps; ++s) {
        for (int stage = 0; stage < 4; ++stage) {
            a.stage = stage;
            const float4* rin = stage == 0 ? im->recX : (stage == 2 ? im->recB : im->recA);
            a.cellOut = stage == 3 ? im->cellX : (stage == 1 ? im->cellB : im->cellA);
            a.recOut = stage == 3 ? im->recX : (stage == 1 ? im->recB : im->recA);
            EP_TRY(run_stage(P, b, a, rin, st));
        }
    }
    return EP_OK;
}

ep_status cell_neighbors_entry(const ep_params* params, int64_t n, const double* q, int64_t* count,
                               uint64_t* hash, int64_t* total, void* stream)
{
    EP_TRY(check_params(params));
    ep_params P = *params;
    P.neigh = EP_CELLLIST;
    P.precision = EP_MIXED;
    EP_TRY(check_cell_params(P));
    if (n < 0 || n > ((int64_t)1 << 26)) return set_error("ep_cell_neighbors: bad n"), EP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) {
        if (total) *total = 0;
        return EP_OK;
    }
    if (!q || !count || !hash) return set_error("ep_cell_neighbors: NULL array"), EP_EINVAL;
    auto is_dev = [](const void* p) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    };
    const size_t m = (size_t)n * 2;
    Sizer z;
    z.add(cell_bytes((int)n, 2, EP_MIXED));
    z.add(sizeof(double) * m * 2);
    z.add(sizeof(int64_t) * (size_t)n * 2);
    Arena* ar = nullptr;
    EP_TRY(arena_acquire(st, z.total, &ar));
    CellBufs b;
    EP_TRY(cell_carve(ar, (int)n, 2, EP_MIXED, &b));
    const double* dq = q;
    if (!is_dev(q)) {
        double* t = (double*)ar->carve(sizeof(double) * m);
        EP_TRY_CUDA(cudaMemcpyAsync(t, q, sizeof(double) * m, cudaMemcpyHostToDevice, st));
        dq = t;
    }
    double* zeros = (double*)ar->carve(sizeof(double) * m);
    EP_TRY_CUDA(cudaMemsetAsync(zeros, 0, sizeof(double) * m, st));
    const bool cdev = is_dev(count), hdev = is_dev(hash);
    long long* dcnt = cdev ? (long long*)count : (long long*)ar->carve(sizeof(int64_t) * (size_t)n);
    unsigned long long* dhs = hdev ? (unsigned long long*)hash : (unsigned long long*)ar->carve(sizeof(int64_t) * (size_t)n);
    EP_TRY(load_anchor(P, b, dq, zeros, st, false));
    Impl* im = impl_of(b);
    Args a{};
    a.mode = 2;
    a.out_cnt = dcnt;
    a.out_hash = dhs;
    EP_TRY(run_stage(P, b, a, im->recX, st));
    if (!cdev) EP_TRY_CUDA(cudaMemcpyAsync(count, dcnt, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, st));
    if (!hdev) EP_TRY_CUDA(cudaMemcpyAsync(hash, dhs, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    if (total) {
        // total accepted pairs = sum of counts (host side after the copy)
        int64_t t = 0;
        if (!cdev) {
            for (int64_t i = 0; i < n; ++i) t += count[i];
        } else {
            std::vector<int64_t> h((size_t)n);
            EP_TRY_CUDA(cudaMemcpy(h.data(), count, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost));
            for (int64_t v : h) t += v;
        }
        if (is_dev(total)) EP_TRY_CUDA(cudaMemcpy(total, &t, sizeof t, cudaMemcpyHostToDevice));
        else *total = t;
    }
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

}  // namespace ep
