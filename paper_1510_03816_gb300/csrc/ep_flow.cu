// ep_flow.cu -- the velocity field of the particles' momenta at arbitrary points
// (Sec. 3.1, Eq. u) and the transport of points by the flow of a shoot (the
// deformation phi_t: d phi_t(x)/dt = u(phi_t(x), t)), all pairs.
//
// The particles are shot first with every RK4 stage input recorded (the same
// recording the adjoint uses), so the stage states the particles' RK4 visited
// are known; each target point then runs its own classical RK4 against them:
//   k1 = u(x_n; stage 1), y = x_n + dt/2 k1, k2 = u(y; stage 2), y = x_n + dt/2 k2,
//   k3 = u(y; stage 3), y = x_n + dt k3, k4 = u(y; stage 4),
//   x_{n+1} = x_n + dt/6 (k1 + 2 k2 + 2 k3 + k4),
// which is the joint RK4 of (q, p, x) because x never feeds back into (q, p).
// Targets are independent, so one launch covers the whole flow with no grid
// synchronisation: a CTA owns 64 targets and, stage by stage, streams the
// recorded particle copy through shared memory, its 8 warps splitting the
// particles.
//
// Mixed precision: the particle copies are the FP32 scaled records of the
// all-pairs path (q' = s (q - c0)); a target's stage position is formed in FP64
// and scaled the same way, pair terms are FP32 and each stage's velocity is
// accumulated in FP32, the target state in FP64.  FP64 mode does everything in
// FP64.  A velocity evaluation is the same kernel with one stage at copy 0.
#include <stdint.h>

#include <algorithm>

#include "ep_allpairs_dev.cuh"
#include "ep_features.cuh"

namespace ep {

namespace {

constexpr int kFlowThreads = 256;
constexpr int kFlowRT = 2;         // targets per lane
constexpr int kFlowTile = 32 * kFlowRT;  // targets per CTA
constexpr int kFlowChunk = 2048;   // particle records per shared-memory fill (mixed)
constexpr int kFlowChunk64 = 1024; // (FP64)

struct FlowArgs {
    int n, m, steps;               // steps = 0: one velocity evaluation at copy 0
    double dt;
    const float4* rec;             // mixed: (4 steps + 1) particle copies of V float4 each
    const double* drec;            // FP64: (4 steps + 1) copies of (q, p), 2 dim doubles each
    const double* c0;              // origin of the scaled coordinates (mixed)
    double s;                      // coordinate scale (mixed)
    double sigma;
    const double* x0;              // targets (m, dim)
    double* x1;                    // result: phi(x0), or u(x0) for a velocity evaluation
};

bool is_dev_array(const void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Copy a caller array into device memory (from the arena) when it is host memory.
ep_status to_device(Arena* ar, const double* p, size_t cnt, cudaStream_t st, const double** out)
{
    if (is_dev_array(p)) {
        *out = p;
        return EP_OK;
    }
    double* d = (double*)ar->carve(sizeof(double) * cnt);
    if (!d) return set_error("workspace too small"), EP_ENOMEM;
    EP_TRY_CUDA(cudaMemcpyAsync(d, p, sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
    *out = d;
    return EP_OK;
}

// RK4 stage bookkeeping of one target component: k = velocity of stage st.
struct Rk4 {
    double x, acc, y;
    __device__ __forceinline__ void stage(int st, double k, double dt)
    {
        if (st == 0) {
            acc = k;
            y = x + 0.5 * dt * k;
        } else if (st == 1) {
            acc += 2.0 * k;
            y = x + 0.5 * dt * k;
        } else if (st == 2) {
            acc += 2.0 * k;
            y = x + dt * k;
        } else {
            x += dt / 6.0 * (acc + k);
            y = x;
        }
    }
};

// Position (scaled units) of the padding particle of an odd particle count in the
// packed source-pair records: its kernel value is exactly zero at every target.
constexpr float kPadCoord = 1.0e18f;

// Component c (q then p) of both particles of a staged record pair.
template <int DIM>
__device__ __forceinline__ float2 flow_comp(const float4 (&S)[DIM], int c)
{
    const float4& v = S[c >> 1];
    return (c & 1) ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
}

// One CTA: kFlowTile targets (lane l of every warp holds targets l and l + 32);
// the 8 warps split each staged chunk of particles, their partial velocities are
// summed in shared memory, and warp 0 applies the RK4 stage and publishes the
// targets' next stage positions.
template <int DIM, int KER>
__global__ void __launch_bounds__(kFlowThreads) k_flow_mixed(FlowArgs a)
{
    constexpr int V = DIM == 2 ? 1 : 2;
    constexpr int W = kFlowThreads / 32;
    extern __shared__ float4 sm[];                                  // [V * kFlowChunk]
    __shared__ float s_y[kFlowTile][DIM];                           // targets' stage positions (scaled)
    __shared__ float s_red[W][kFlowTile][DIM];                      // warps' partial velocities
    const int n = a.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double c0[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) c0[c] = a.c0[c];
    int tgt[kFlowRT];
    Rk4 st[kFlowRT][DIM];  // meaningful in warp 0
#pragma unroll
    for (int r = 0; r < kFlowRT; ++r) {
        tgt[r] = blockIdx.x * kFlowTile + lane + 32 * r;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            const double v = tgt[r] < a.m ? a.x0[(size_t)tgt[r] * DIM + c] : 0.0;
            st[r][c].x = v;
            st[r][c].y = v;
            st[r][c].acc = 0.0;
            if (warp == 0) s_y[lane + 32 * r][c] = (float)((v - c0[c]) * a.s);
        }
    }
    const int nst = a.steps == 0 ? 1 : 4 * a.steps;
    for (int k = 0; k < nst; ++k) {
        const float4* copy = a.rec + (size_t)k * V * n;
        __syncthreads();
        float y[kFlowRT][DIM], u[kFlowRT][DIM];
#pragma unroll
        for (int r = 0; r < kFlowRT; ++r)
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                y[r][c] = s_y[lane + 32 * r][c];
                u[r][c] = 0.0f;
            }
        // the targets' negated positions as broadcast pairs; the particle records are
        // staged in source pairs (float4 k of a pair holds components 2k and 2k+1, in
        // the order q, p, of both sources), so one load gives the f32x2 operands of
        // two particles; an odd count is padded with a particle far away and without
        // momentum, whose terms are exactly zero
        constexpr int PV = DIM;  // float4 per source pair
        float2 ny[kFlowRT][DIM], u2[kFlowRT][DIM];
#pragma unroll
        for (int r = 0; r < kFlowRT; ++r)
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                ny[r][c] = make_float2(-y[r][c], -y[r][c]);
                u2[r][c] = make_float2(0.0f, 0.0f);
            }
        for (int cj = 0; cj < n; cj += kFlowChunk) {
            const int L = min(kFlowChunk, n - cj);
            const int P = (L + 1) >> 1;
            if (cj > 0) __syncthreads();
            for (int t = threadIdx.x; t < P; t += kFlowThreads) {
                const int j = cj + 2 * t;
                const bool two = 2 * t + 1 < L;
                float c0[2 * DIM], c1[2 * DIM];
                if constexpr (DIM == 2) {
                    const float4 v0 = __ldg(copy + j);
                    const float4 v1 = two ? __ldg(copy + j + 1) : make_float4(kPadCoord, kPadCoord, 0.f, 0.f);
                    c0[0] = v0.x; c0[1] = v0.y; c0[2] = v0.z; c0[3] = v0.w;
                    c1[0] = v1.x; c1[1] = v1.y; c1[2] = v1.z; c1[3] = v1.w;
                } else {
                    const float4 q0 = __ldg(copy + 2 * (size_t)j), p0 = __ldg(copy + 2 * (size_t)j + 1);
                    const float4 q1 = two ? __ldg(copy + 2 * (size_t)j + 2) : make_float4(kPadCoord, kPadCoord, kPadCoord, 0.f);
                    const float4 p1 = two ? __ldg(copy + 2 * (size_t)j + 3) : make_float4(0.f, 0.f, 0.f, 0.f);
                    c0[0] = q0.x; c0[1] = q0.y; c0[2] = q0.z; c0[3] = p0.x; c0[4] = p0.y; c0[5] = p0.z;
                    c1[0] = q1.x; c1[1] = q1.y; c1[2] = q1.z; c1[3] = p1.x; c1[4] = p1.y; c1[5] = p1.z;
                }
#pragma unroll
                for (int k = 0; k < PV; ++k)
                    sm[(size_t)t * PV + k] = make_float4(c0[2 * k], c1[2 * k], c0[2 * k + 1], c1[2 * k + 1]);
            }
            __syncthreads();
            const int pa = warp * P / W, pz = (warp + 1) * P / W;
#pragma unroll 2
            for (int q = pa; q < pz; ++q) {
                float4 S[PV];
#pragma unroll
                for (int k = 0; k < PV; ++k) S[k] = sm[(size_t)q * PV + k];
#pragma unroll
                for (int r = 0; r < kFlowRT; ++r) {
                    float2 r2 = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int c = 0; c < DIM; ++c) {
                        const float2 d = __fadd2_rn(flow_comp<DIM>(S, c), ny[r][c]);
                        r2 = __ffma2_rn(d, d, r2);
                    }
                    float2 G, w;
                    kfun_f32<KER>(r2.x, G.x, w.x);
                    kfun_f32<KER>(r2.y, G.y, w.y);
#pragma unroll
                    for (int c = 0; c < DIM; ++c) u2[r][c] = __ffma2_rn(G, flow_comp<DIM>(S, DIM + c), u2[r][c]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kFlowRT; ++r)
#pragma unroll
            for (int c = 0; c < DIM; ++c) u[r][c] = u2[r][c].x + u2[r][c].y;
#pragma unroll
        for (int r = 0; r < kFlowRT; ++r)
#pragma unroll
            for (int c = 0; c < DIM; ++c) s_red[warp][lane + 32 * r][c] = u[r][c];
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int r = 0; r < kFlowRT; ++r)
#pragma unroll
                for (int c = 0; c < DIM; ++c) {
                    float sum = 0.0f;
#pragma unroll
                    for (int w2 = 0; w2 < W; ++w2) sum += s_red[w2][lane + 32 * r][c];
                    if (a.steps == 0) {
                        st[r][c].x = (double)sum;
                    } else {
                        st[r][c].stage(k & 3, (double)sum, a.dt);
                        s_y[lane + 32 * r][c] = (float)((st[r][c].y - c0[c]) * a.s);
                    }
                }
        }
    }
    if (warp == 0)
#pragma unroll
        for (int r = 0; r < kFlowRT; ++r)
            if (tgt[r] < a.m)
#pragma unroll
                for (int c = 0; c < DIM; ++c) a.x1[(size_t)tgt[r] * DIM + c] = st[r][c].x;
}

template <int DIM, int KER>
__global__ void __launch_bounds__(kFlowThreads) k_flow_fp64(FlowArgs a)
{
    constexpr int S2 = 2 * DIM;
    constexpr int W = kFlowThreads / 32;
    extern __shared__ double dsm[];                                 // [S2 * kFlowChunk64]
    __shared__ double s_y[kFlowTile][DIM];
    __shared__ double s_red[W][kFlowTile][DIM];
    const int n = a.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int tgt[kFlowRT];
    Rk4 st[kFlowRT][DIM];  // meaningful in warp 0
#pragma unroll
    for (int r = 0; r < kFlowRT; ++r) {
        tgt[r] = blockIdx.x * kFlowTile + lane + 32 * r;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            const double v = tgt[r] < a.m ? a.x0[(size_t)tgt[r] * DIM + c] : 0.0;
            st[r][c].x = v;
            st[r][c].y = v;
            st[r][c].acc = 0.0;
            if (warp == 0) s_y[lane + 32 * r][c] = v;
        }
    }
    const int nst = a.steps == 0 ? 1 : 4 * a.steps;
    for (int k = 0; k < nst; ++k) {
        const double* copy = a.drec + (size_t)k * S2 * n;
        __syncthreads();
        double y[kFlowRT][DIM], u[kFlowRT][DIM];
#pragma unroll
        for (int r = 0; r < kFlowRT; ++r)
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                y[r][c] = s_y[lane + 32 * r][c];
                u[r][c] = 0.0;
            }
        for (int cj = 0; cj < n; cj += kFlowChunk64) {
            const int L = min(kFlowChunk64, n - cj);
            if (cj > 0) __syncthreads();
            for (int t = threadIdx.x; t < L * S2; t += kFlowThreads) dsm[t] = __ldg(copy + (size_t)cj * S2 + t);
            __syncthreads();
            const int ja = warp * L / W, jb = (warp + 1) * L / W;
            for (int j = ja; j < jb; ++j) {
                const double* v = dsm + (size_t)j * S2;
#pragma unroll
                for (int r = 0; r < kFlowRT; ++r) {
                    double r2 = 0.0;
#pragma unroll
                    for (int c = 0; c < DIM; ++c) {
                        const double d = y[r][c] - v[c];
                        r2 += d * d;
                    }
                    double G, phi;
                    kfun_f64<KER>(r2, a.sigma, G, phi);
#pragma unroll
                    for (int c = 0; c < DIM; ++c) u[r][c] += G * v[DIM + c];
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kFlowRT; ++r)
#pragma unroll
            for (int c = 0; c < DIM; ++c) s_red[warp][lane + 32 * r][c] = u[r][c];
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int r = 0; r < kFlowRT; ++r)
#pragma unroll
                for (int c = 0; c < DIM; ++c) {
                    double sum = 0.0;
#pragma unroll
                    for (int w2 = 0; w2 < W; ++w2) sum += s_red[w2][lane + 32 * r][c];
                    if (a.steps == 0) {
                        st[r][c].x = sum;
                    } else {
                        st[r][c].stage(k & 3, sum, a.dt);
                        s_y[lane + 32 * r][c] = st[r][c].y;
                    }
                }
        }
    }
    if (warp == 0)
#pragma unroll
        for (int r = 0; r < kFlowRT; ++r)
            if (tgt[r] < a.m)
#pragma unroll
                for (int c = 0; c < DIM; ++c) a.x1[(size_t)tgt[r] * DIM + c] = st[r][c].x;
}

template <int DIM, int KER>
ep_status launch_flow(const ep_params& P, FlowArgs& a, cudaStream_t st)
{
    const unsigned grid = (unsigned)((a.m + kFlowTile - 1) / kFlowTile);
    if (grid == 0) return EP_OK;
    count_launch();
    if (P.precision == EP_MIXED) {
        constexpr int V = DIM == 2 ? 1 : 2;
        const size_t smem = sizeof(float4) * V * kFlowChunk;
        static bool attr = false;
        if (!attr) {
            EP_TRY_CUDA(cudaFuncSetAttribute(k_flow_mixed<DIM, KER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            attr = true;
        }
        k_flow_mixed<DIM, KER><<<grid, kFlowThreads, smem, st>>>(a);
    } else {
        const size_t smem = sizeof(double) * 2 * DIM * kFlowChunk64;
        static bool attr = false;
        if (!attr) {
            EP_TRY_CUDA(cudaFuncSetAttribute(k_flow_fp64<DIM, KER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            attr = true;
        }
        k_flow_fp64<DIM, KER><<<grid, kFlowThreads, smem, st>>>(a);
    }
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

ep_status dispatch_flow(const ep_params& P, FlowArgs& a, cudaStream_t st)
{
#define EP_FLOW_CASE(D, K) \
    if (P.dim == D && P.kernel == K) return launch_flow<D, K>(P, a, st);
    EP_FLOW_CASE(2, EP_GAUSS) EP_FLOW_CASE(2, EP_TENT) EP_FLOW_CASE(2, EP_EXPCONE)
    EP_FLOW_CASE(3, EP_GAUSS) EP_FLOW_CASE(3, EP_TENT) EP_FLOW_CASE(3, EP_EXPCONE)
#undef EP_FLOW_CASE
    set_error("no flow kernel for dim=%d kernel=%d", P.dim, P.kernel);
    return EP_EINVAL;
}

// Shared body of ep_velocity (steps = 0) and ep_flow.
ep_status flow_common(const ep_params* params, int64_t n, const double* q, const double* p, int64_t m,
                      const double* x0, double* x1, bool velocity, void* stream, const char* name)
{
    EP_TRY(check_params(params));
    if (n < 0 || n > ((int64_t)1 << 26) || m < 0 || m > ((int64_t)1 << 30))
        return set_error("%s: bad n or m", name), EP_EINVAL;
    const ep_params& P = *params;
    if (P.neigh == EP_CELLLIST) return set_error("%s: runs on the all-pairs path", name), EP_EINVAL;
    if (P.inexact != 0.0) return set_error("%s: built for the exact system", name), EP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (m == 0) return EP_OK;
    if (!x0 || !x1 || (n > 0 && (!q || !p))) return set_error("%s: NULL array", name), EP_EINVAL;
    const size_t nd = (size_t)n * P.dim, md = (size_t)m * P.dim;
    const bool mixed = P.precision == EP_MIXED;
    const size_t V = P.dim == 2 ? 1 : 2;
    const int copies = velocity ? 1 : 4 * P.steps + 1;
    const size_t rec_bytes = mixed ? sizeof(float4) * V * (size_t)n : sizeof(double) * 2 * nd;
    Sizer z;
    z.add(allpairs_bytes((int)n, P.dim, P.precision));
    z.add(rec_bytes * (size_t)copies);
    z.add(sizeof(double) * (2 * nd + 2 * md));
    Arena* ar = nullptr;
    EP_TRY(arena_acquire(st, z.total, &ar));
    AllPairsBufs b;
    EP_TRY(allpairs_carve(ar, (int)n, P.dim, P.precision, &b));
    char* rec = (char*)ar->carve(rec_bytes * (size_t)copies);
    const double *dq = nullptr, *dp = nullptr, *dx0 = nullptr;
    if (n > 0) {
        EP_TRY(to_device(ar, q, nd, st, &dq));
        EP_TRY(to_device(ar, p, nd, st, &dp));
    }
    EP_TRY(to_device(ar, x0, md, st, &dx0));
    const bool out_host = !is_dev_array(x1);
    double* dx1 = out_host ? (double*)ar->carve(sizeof(double) * md) : x1;
    if (!dx1 || (n > 0 && !rec)) return set_error("%s: workspace too small", name), EP_ENOMEM;
    FlowArgs a{};
    a.n = (int)n;
    a.m = (int)m;
    a.steps = velocity ? 0 : P.steps;
    a.dt = P.t1 / P.steps;
    a.sigma = P.sigma;
    a.s = mixed ? kernel_scale(P.kernel, P.sigma).s : 1.0;
    a.x0 = dx0;
    a.x1 = dx1;
    if (n > 0) {
        EP_TRY(allpairs_load(P, b, dq, dp, st));
        if (velocity) {
            a.rec = mixed ? b.Sx : nullptr;
            a.drec = mixed ? nullptr : b.Dx;
        } else {
            EP_TRY(allpairs_steps_rec(P, b, P.steps, a.dt, mixed ? (float4*)rec : nullptr,
                                      mixed ? nullptr : (double*)rec, st));
            a.rec = mixed ? (const float4*)rec : nullptr;
            a.drec = mixed ? nullptr : (const double*)rec;
        }
        a.c0 = b.c0;
        EP_TRY(dispatch_flow(P, a, st));
    } else if (velocity) {
        EP_TRY_CUDA(cudaMemsetAsync(dx1, 0, sizeof(double) * md, st));  // no particles: u = 0
    } else if (dx1 != dx0) {
        EP_TRY_CUDA(cudaMemcpyAsync(dx1, dx0, sizeof(double) * md, cudaMemcpyDeviceToDevice, st));
    }
    if (out_host) {
        EP_TRY_CUDA(cudaMemcpyAsync(x1, dx1, sizeof(double) * md, cudaMemcpyDeviceToHost, st));
        EP_TRY_CUDA(cudaStreamSynchronize(st));
    }
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

}  // namespace

ep_status velocity_entry(const ep_params* params, int64_t n, const double* q, const double* p, int64_t m,
                         const double* x, double* u, void* stream)
{
    return flow_common(params, n, q, p, m, x, u, true, stream, "ep_velocity");
}

ep_status flow_entry(const ep_params* params, int64_t n, const double* q0, const double* p0, int64_t m,
                     const double* x0, double* x1, void* stream)
{
    return flow_common(params, n, q0, p0, m, x0, x1, false, stream, "ep_flow");
}

}  // namespace ep
