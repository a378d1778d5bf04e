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
// One stage = bin (cell key + rank by atomics) -> block-wise exclusive scan of the
// cell counts -> scatter into cell order -> sort each cell by particle index
// (deterministic sums) -> sweep: each CTA owns an 8 x 8 block of cells, stages the
// records of its 10 x 10 halo (contiguous row segments of the sorted array) in
// shared memory, and every thread sums its particles' 3 x 3 neighbour cells in
// FP32, then applies the RK4 stage.  Stage positions inside a step are
// anchor + c dt k in FP32 on the offsets (re-celled by floor(o / e)); the step
// state x is FP64 and the anchor is re-derived from it in FP64 every step.
#include <math.h>

#include <algorithm>
#include <vector>

#include "ep_features.cuh"

namespace ep {

namespace {

constexpr int kBlk = 8;                        // cells per sweep block side
constexpr int kHalo = kBlk + 2;
constexpr int kSweepThreads = 256;
constexpr int kSweepCap = 3072;                // halo records staged in shared memory
constexpr int kScanBlock = 4096;               // cells per scan block (1024 threads x 4)
constexpr int kMaxCellsPerAxis2D = 2048;

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
    int* count;      // per cell, then local exclusive scan
    int* bsum;       // per scan block total, then exclusive block offsets
    double* bbox;    // min x, min y, max x, max y
    Grid g;
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
    const int2* cellIn;
    const int* key;
    const int* count;   // local scan
    const int* boff;    // block offsets
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
__global__ void k_bbox2(const double* __restrict__ q, int n, double* out)
{
    __shared__ double s[4][32];
    double v[4] = {INFINITY, INFINITY, -INFINITY, -INFINITY};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double a = q[2 * (size_t)i], b = q[2 * (size_t)i + 1];
        v[0] = fmin(v[0], a); v[1] = fmin(v[1], b); v[2] = fmax(v[2], a); v[3] = fmax(v[3], b);
    }
    for (int o = 16; o > 0; o >>= 1) {
        v[0] = fmin(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
        v[1] = fmin(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
        v[2] = fmax(v[2], __shfl_xor_sync(0xffffffffu, v[2], o));
        v[3] = fmax(v[3], __shfl_xor_sync(0xffffffffu, v[3], o));
    }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 4; ++k) s[k][threadIdx.x >> 5] = v[k];
    __syncthreads();
    if (threadIdx.x < 4) {
        double r = threadIdx.x < 2 ? INFINITY : -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            r = threadIdx.x < 2 ? fmin(r, s[threadIdx.x][w]) : fmax(r, s[threadIdx.x][w]);
        out[threadIdx.x] = r;
    }
}

// x = (q, p) and the step-start cells / records from FP64.
__global__ void k_cell_anchor(const double* __restrict__ q, const double* __restrict__ p, int n, Grid g,
                              double* __restrict__ x, int2* __restrict__ cellX, float4* __restrict__ recX)
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
    recX[i] = make_float4(ox, oy, (float)px, (float)py);
}

__global__ void k_cell_bin(const int2* __restrict__ cellIn, int n, int ncx, int* __restrict__ count,
                           int* __restrict__ key, int* __restrict__ rank)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 c = cellIn[i];
    const int k = c.y * ncx + c.x;
    key[i] = k;
    rank[i] = atomicAdd(count + k, 1);
}

// Exclusive scan of count within blocks of kScanBlock cells; bsum[b] = block total.
__global__ void __launch_bounds__(1024) k_scan_local(int* __restrict__ count, long long ncell, int* __restrict__ bsum)
{
    __shared__ int sw[32];
    const long long base = (long long)blockIdx.x * kScanBlock + 4LL * threadIdx.x;
    int v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = (base + k < ncell) ? count[base + k] : 0;
        s += v[k];
    }
    // inclusive warp scan of the thread totals
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
        if (base + k < ncell) count[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 1023) bsum[blockIdx.x] = run;
}

// Exclusive scan of the block totals in place (one CTA; at most 1024 x 4 blocks).
__global__ void __launch_bounds__(1024) k_scan_top(int* __restrict__ bsum, int nb)
{
    __shared__ int sw[32];
    int v[4], s = 0;
    for (int k = 0; k < 4; ++k) {
        const int b = 4 * threadIdx.x + k;
        v[k] = b < nb ? bsum[b] : 0;
        s += v[k];
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
    for (int k = 0; k < 4; ++k) {
        const int b = 4 * threadIdx.x + k;
        if (b < nb) bsum[b] = run;
        run += v[k];
    }
}

__global__ void k_cell_scatter(const int* __restrict__ key, const int* __restrict__ rank, const int* __restrict__ count,
                               const int* __restrict__ boff, const float4* __restrict__ recIn, int n,
                               int* __restrict__ sidx, float4* __restrict__ srec)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = key[i];
    const int slot = cell_start(count, boff, k) + rank[i];
    sidx[slot] = i;
    srec[slot] = recIn[i];
}

// Sort each cell's slots by particle index (insertion sort; cells hold ~10 particles).
__global__ void k_cell_sort(const int* __restrict__ count, const int* __restrict__ boff, long long ncell, int n,
                            int* __restrict__ sidx, float4* __restrict__ srec)
{
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int a = cell_start(count, boff, c);
    const int b = (c + 1 < ncell) ? cell_start(count, boff, c + 1) : n;
    for (int u = a + 1; u < b; ++u) {
        const int ki = sidx[u];
        const float4 kr = srec[u];
        int v = u - 1;
        while (v >= a && sidx[v] > ki) {
            sidx[v + 1] = sidx[v];
            srec[v + 1] = srec[v];
            --v;
        }
        sidx[v + 1] = ki;
        srec[v + 1] = kr;
    }
}

__device__ void epilogue(const Args& a, int i, float dqx, float dqy, float dpx, float dpy, int cx, int cy)
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
    if (a.stage < 3) {
        const float cdt = (a.stage == 2 ? 1.0f : 0.5f) * a.dt_f;
        const float bw = a.stage == 0 ? 1.0f : 2.0f;
        const int2 ax = a.cellX[i];
        const float4 rx = a.recX[i];
        const float is = (float)a.g.inv_sigma;
        // stage position: anchor offset + c dt kq (units of sigma), re-celled
        float o0 = fmaf(cdt * is, kq0, rx.x), o1 = fmaf(cdt * is, kq1, rx.y);
        int c0 = ax.x + (int)floorf(o0 / a.g.e[0]), c1 = ax.y + (int)floorf(o1 / a.g.e[1]);
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
        int c0, c1;
        float o0, o1;
        locate(q0, 0, a.g, c0, o0);
        locate(q1, 1, a.g, c1, o1);
        a.cellOut[i] = make_int2(c0, c1);
        a.recOut[i] = make_float4(o0, o1, (float)p0, (float)p1);
    }
    (void)cx;
    (void)cy;
}

// One CTA per 8 x 8 block of cells.
__global__ void __launch_bounds__(kSweepThreads) k_cell_sweep(Args a)
{
    __shared__ float4 srec[kSweepCap];
    __shared__ int hoff[kHalo * kHalo + 1];   // halo cell -> first record (local or global)
    __shared__ int rowbase[kHalo];
    __shared__ int own_off[kBlk + 1];         // own particles: prefix over own rows
    __shared__ int use_smem;
    const int ncx = a.g.nc[0], ncy = a.g.nc[1];
    const int cx0 = blockIdx.x * kBlk, cy0 = blockIdx.y * kBlk;
    // halo: rows cy0-1 .. cy0+kBlk, cells cx0-1 .. cx0+kBlk (clipped to the grid)
    const int xa = max(cx0 - 1, 0), xb = min(cx0 + kBlk, ncx - 1);
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int hy = 0; hy < kHalo; ++hy) {
            const int row = cy0 - 1 + hy;
            rowbase[hy] = tot;
            if (row < 0 || row >= ncy) continue;
            const long long c_a = (long long)row * ncx + xa, c_b = (long long)row * ncx + xb;
            const int s0 = cell_start(a.count, a.boff, c_a);
            const int s1 = (c_b + 1 < a.g.ncell) ? cell_start(a.count, a.boff, c_b + 1) : a.n;
            tot += s1 - s0;
        }
        use_smem = tot <= kSweepCap;
        // own rows prefix
        int ot = 0;
        for (int ly = 0; ly < kBlk; ++ly) {
            own_off[ly] = ot;
            const int row = cy0 + ly;
            if (row >= ncy || cx0 >= ncx) continue;
            const long long c_a = (long long)row * ncx + cx0;
            const long long c_b = (long long)row * ncx + min(cx0 + kBlk - 1, ncx - 1);
            const int s0 = cell_start(a.count, a.boff, c_a);
            const int s1 = (c_b + 1 < a.g.ncell) ? cell_start(a.count, a.boff, c_b + 1) : a.n;
            ot += s1 - s0;
        }
        own_off[kBlk] = ot;
    }
    __syncthreads();
    const bool sm = use_smem != 0;
    // per halo cell: first record index (in shared memory, or the global slot)
    for (int t = threadIdx.x; t < kHalo * kHalo; t += kSweepThreads) {
        const int hx = t % kHalo, hy = t / kHalo;
        const int row = cy0 - 1 + hy, col = cx0 - 1 + hx;
        int v = -1;
        if (row >= 0 && row < ncy && col >= 0 && col < ncx) {
            const long long c = (long long)row * ncx + col;
            const int g0 = cell_start(a.count, a.boff, c);
            if (sm) {
                const int ra = cell_start(a.count, a.boff, (long long)row * ncx + xa);
                v = rowbase[hy] + (g0 - ra);
            } else {
                v = g0;
            }
        }
        hoff[t] = v;
    }
    // stage the halo records (contiguous row segments of the sorted array)
    if (sm) {
        for (int hy = 0; hy < kHalo; ++hy) {
            const int row = cy0 - 1 + hy;
            if (row < 0 || row >= ncy) continue;
            const long long c_a = (long long)row * ncx + xa, c_b = (long long)row * ncx + xb;
            const int s0 = cell_start(a.count, a.boff, c_a);
            const int s1 = (c_b + 1 < a.g.ncell) ? cell_start(a.count, a.boff, c_b + 1) : a.n;
            for (int u = s0 + threadIdx.x; u < s1; u += kSweepThreads) srec[rowbase[hy] + (u - s0)] = a.srec[u];
        }
    }
    __syncthreads();
    const float4* base = sm ? srec : a.srec;
    const float e0 = a.g.e[0], e1 = a.g.e[1];
    const int nown = own_off[kBlk];
    for (int k = threadIdx.x; k < nown; k += kSweepThreads) {
        // own particle k: row ly, its global slot and cell
        int ly = 0;
        while (own_off[ly + 1] <= k) ++ly;
        const int row = cy0 + ly;
        const int sa = cell_start(a.count, a.boff, (long long)row * ncx + cx0);
        const int slot = sa + (k - own_off[ly]);
        // find the column: largest col in the own range with start <= slot
        int col = cx0;
        const int colmax = min(cx0 + kBlk - 1, ncx - 1);
        while (col < colmax && cell_start(a.count, a.boff, (long long)row * ncx + col + 1) <= slot) ++col;
        const float4 ri = a.srec[slot];
        const int i = a.sidx[slot];
        float dqx = 0.f, dqy = 0.f, dpx = 0.f, dpy = 0.f;
        int cnt = 0;
        unsigned long long hs = 0ull;
        const int lx = col - cx0, lyy = row - cy0;
        for (int dy = -1; dy <= 1; ++dy) {
            for (int dx = -1; dx <= 1; ++dx) {
                const int hx = lx + 1 + dx, hy = lyy + 1 + dy;
                const int h0 = hoff[hy * kHalo + hx];
                if (h0 < 0) continue;
                // end of this cell: next cell's start in the same row, or the row/array end
                const int ccol = col + dx, crow = row + dy;
                const long long c = (long long)crow * ncx + ccol;
                const int gs = cell_start(a.count, a.boff, c);
                const int ge = (c + 1 < a.g.ncell) ? cell_start(a.count, a.boff, c + 1) : a.n;
                const int len = ge - gs;
                const float sx = __fmul_rn((float)(-dx), e0), sy = __fmul_rn((float)(-dy), e1);
                for (int v = 0; v < len; ++v) {
                    const float4 rj = base[h0 + v];
                    const float d0 = __fadd_rn(__fsub_rn(ri.x, rj.x), sx);
                    const float d1 = __fadd_rn(__fsub_rn(ri.y, rj.y), sy);
                    const float r2 = __fmaf_rn(d0, d0, __fmul_rn(d1, d1));
                    if (r2 < 1.0f) {
                        if (a.mode == 2) {
                            ++cnt;
                            const int j = a.sidx[gs + v];
                            hs += (unsigned long long)(j + 1) * 2654435761ull;
                        } else {
                            const float rs = rsqrt_approx(fmaxf(r2, 1e-30f));
                            const float G = fmaf(-r2, rs, 1.0f);
                            dqx = fmaf(G, rj.z, dqx);
                            dqy = fmaf(G, rj.w, dqy);
                            const float c2 = rs * fmaf(ri.z, rj.z, ri.w * rj.w);
                            dpx = fmaf(c2, d0, dpx);
                            dpy = fmaf(c2, d1, dpy);
                        }
                    }
                }
            }
        }
        if (a.mode == 2) {
            a.out_cnt[i] = (long long)cnt;
            a.out_hash[i] = hs;
        } else {
            epilogue(a, i, dqx, dqy, dpx, dpy, col, row);
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
    z.add(sizeof(int) * maxcell);
    z.add(sizeof(int) * (maxcell / kScanBlock + 1));
    z.add(sizeof(double) * 4);
    return z.total;
}

ep_status run_stage(const ep_params& P, const CellBufs& b, Args a, const int2* cellIn, const float4* recIn,
                    cudaStream_t st)
{
    Impl* im = impl_of(b);
    const Grid& g = im->g;
    const int n = b.n;
    const unsigned gn = (unsigned)((n + 255) / 256);
    const int nb = (int)((g.ncell + kScanBlock - 1) / kScanBlock);
    EP_TRY_CUDA(cudaMemsetAsync(im->count, 0, sizeof(int) * (size_t)g.ncell, st));
    count_launch(5);
    k_cell_bin<<<gn, 256, 0, st>>>(cellIn, n, g.nc[0], im->count, im->key, im->rank);
    k_scan_local<<<nb, 1024, 0, st>>>(im->count, g.ncell, im->bsum);
    k_scan_top<<<1, 1024, 0, st>>>(im->bsum, nb);
    k_cell_scatter<<<gn, 256, 0, st>>>(im->key, im->rank, im->count, im->bsum, recIn, n, im->sidx, im->srec);
    k_cell_sort<<<(unsigned)((g.ncell + 255) / 256), 256, 0, st>>>(im->count, im->bsum, g.ncell, n, im->sidx, im->srec);
    a.n = n;
    a.g = g;
    a.count = im->count;
    a.boff = im->bsum;
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
    k_cell_sweep<<<grid, kSweepThreads, 0, st>>>(a);
    EP_TRY_CUDA(cudaGetLastError());
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
    count_launch();
    k_bbox2<<<1, 1024, 0, st>>>(q, n, im->bbox);
    double bb[4];
    EP_TRY_CUDA(cudaMemcpyAsync(bb, im->bbox, sizeof bb, cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    im->g = make_grid(bb, P.sigma);
    count_launch();
    k_cell_anchor<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(q, p, n, im->g, write_x ? b.x : nullptr, im->cellX,
                                                                im->recX);
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
    im->count = (int*)ar->carve(sizeof(int) * maxcell);
    im->bsum = (int*)ar->carve(sizeof(int) * (maxcell / kScanBlock + 1));
    im->bbox = (double*)ar->carve(sizeof(double) * 4);
    if (!im->bbox) return set_error("workspace too small for the cell list"), EP_ENOMEM;
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
    return run_stage(P, b, a, im->cellX, im->recX, st);
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
            const int2* cin = stage == 0 ? im->cellX : (stage == 2 ? im->cellB : im->cellA);
            const float4* rin = stage == 0 ? im->recX : (stage == 2 ? im->recB : im->recA);
            a.cellOut = stage == 3 ? im->cellX : (stage == 1 ? im->cellB : im->cellA);
            a.recOut = stage == 3 ? im->recX : (stage == 1 ? im->recB : im->recA);
            EP_TRY(run_stage(P, b, a, cin, rin, st));
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
    EP_TRY(run_stage(P, b, a, im->cellX, im->recX, st));
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
