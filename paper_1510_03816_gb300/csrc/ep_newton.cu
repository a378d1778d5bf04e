// ep_newton.cu -- the tangent-linear RK4 shoot (the directional derivative of
// the shooting map p0 -> (Q(1), P(1))) and Algorithm 1 with the Newton-type gain
// M = h (D phi)^-1 of Sec. 5 (Theorem 1), plain FP64 method.
//
// Tangent-linear shoot.  The primal shoot is run once with every RK4 stage input
// recorded.  With F = (dH/dp, -dH/dq) of Eq. N-particle, a stage's derivative is
//   J_F(y) v = ( sum_j [G_ij dp_j + phi_ij (d_ij . dd_ij) p_j] ,
//               -sum_{j != i} [(dp_i . p_j + p_i . dp_j) phi_ij d_ij
//                              + (p_i . p_j)(phi_ij dd_ij + psi_ij (d_ij . dd_ij) d_ij)] )
// (the two blocks of the Hessian of Eq. H, d_ij = q_i - q_j, dd_ij = dq_i - dq_j),
// and the tangent follows the primal RK4 stage by stage:
//   dk_s = J_F(y_s) dy_s,  dy_{s+1} = dx_n + c_{s+1} dt dk_s,
//   dx_{n+1} = dx_n + dt/6 (dk_1 + 2 dk_2 + 2 dk_3 + dk_4).
// One cooperative launch covers the whole tangent shoot: every CTA owns the
// particles [c n / G, (c+1) n / G), sums their rows over all sources in FP64
// against the recorded stage state, and applies the tangent RK4 stage; one grid
// barrier per stage publishes the next tangent stage inputs.
//
// Newton gain.  Each iterate shoots (recording the stages), takes the max-norm
// residual r = Y - Q(1) and stops as Algorithm 1 does; otherwise it solves
// (D phi) delta = r by restarted GMRES whose matrix-vector products are tangent
// shoots along (0, v) (matrix-free: D phi = dQ(1)/dp0 is never formed), and
// updates p0 += h delta.  The Krylov basis lives on the host (n dim doubles per
// vector); each product is one launch.  Problems with n dim <= kDenseNewtonMax form
// D phi whole instead (one CTA per column, all columns in one launch) and solve it
// by Gaussian elimination with partial pivoting on one CTA; the residual and the
// update stay on the device.
#include <math.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ep_allpairs.cuh"
#include "ep_allpairs_dev.cuh"
#include "ep_features.cuh"

namespace ep {

namespace {

constexpr int kTanThreads = 256;
// relative residual at which the inner Krylov solve of a gained update stops
constexpr double kKrylovTol = 1e-12;

// FP64 kernel value, phi = G'(r)/r and psi = phi'(r)/r (unscaled): the
// derivatives the Hessian of Eq. H needs.  Reciprocals of sigma are hoisted and
// 1/r comes from rsqrt; the tent keeps r = sqrt(r2) for its support test.
template <int KER>
__device__ __forceinline__ void kfun3_f64(double r2, double sigma, double& G, double& phi, double& psi)
{
    const double is = 1.0 / sigma;
    if constexpr (KER == EP_GAUSS) {
        G = exp(-0.5 * (r2 * (is * is)));
        phi = -G * (is * is);
        psi = G * (is * is) * (is * is);
    } else if constexpr (KER == EP_TENT) {
        const double r = sqrt(r2);
        const bool in = r < sigma && r2 > 0.0;
        const double rs = r2 > 0.0 ? rsqrt(r2) : 0.0;
        G = r < sigma ? 1.0 - r * is : 0.0;
        phi = in ? -is * rs : 0.0;
        psi = in ? is * rs * rs * rs : 0.0;
    } else {
        const double r = sqrt(r2);
        const double rs = r2 > 0.0 ? rsqrt(r2) : 0.0;
        G = exp(-r * is);
        phi = r2 > 0.0 ? -G * is * rs : 0.0;
        psi = r2 > 0.0 ? G * (is * is * rs * rs + is * rs * rs * rs) : 0.0;
    }
}

struct TanArgs {
    int n, steps;
    double dt, sigma;
    const double* drec;  // (4 steps + 1) primal stage copies, (q, p) = 2 dim doubles per particle
    const double* v0;    // initial tangent [dq (n dim) | dp (n dim)]
    double* dx;          // tangent state at the step start (2 dim per particle, own rows)
    double* dacc;        // tangent RK4 accumulator dk1 + 2 dk2 + 2 dk3
    double* T[2];        // tangent stage inputs (2 dim per particle), ping-pong
    double* out;         // [dQ(1) (n dim) | dP(1) (n dim)]
    unsigned* bar;
    int* err;
};

template <int DIM, int KER>
__global__ void __launch_bounds__(kTanThreads) k_tangent_fp64(TanArgs a)
{
    constexpr int S2 = 2 * DIM;
    __shared__ double sm_d[(kTanThreads / 32 + 1) * 8];
    const int n = a.n;
    const int r0 = (int)((long long)blockIdx.x * n / gridDim.x), r1 = (int)((long long)(blockIdx.x + 1) * n / gridDim.x);
    const size_t nd = (size_t)n * DIM;
    unsigned epoch = 0;
    // dx = v0, first stage input T[0] = v0 (own particles)
    for (int t = threadIdx.x; t < (r1 - r0) * S2; t += kTanThreads) {
        const int i = r0 + t / S2, c = t % S2;
        const double v = c < DIM ? a.v0[(size_t)i * DIM + c] : a.v0[nd + (size_t)i * DIM + (c - DIM)];
        a.dx[(size_t)i * S2 + c] = v;
        a.T[0][(size_t)i * S2 + c] = v;
    }
    if (!grid_barrier(a.bar, a.err, ++epoch)) return;
    int cur = 0;
    for (int k = 0; k < a.steps; ++k) {
        for (int s = 0; s < 4; ++s) {
            const double* Y = a.drec + (size_t)(4 * k + s) * S2 * n;
            const double* Tin = a.T[cur];
            double* Tout = a.T[cur ^ 1];
            for (int i = r0; i < r1; ++i) {
                double qi[DIM], pi[DIM], vqi[DIM], vpi[DIM];
#pragma unroll
                for (int c = 0; c < DIM; ++c) {
                    qi[c] = __ldcg(Y + (size_t)i * S2 + c);
                    pi[c] = __ldcg(Y + (size_t)i * S2 + DIM + c);
                    vqi[c] = __ldcg(Tin + (size_t)i * S2 + c);
                    vpi[c] = __ldcg(Tin + (size_t)i * S2 + DIM + c);
                }
                // h[0..DIM): (d2H v)_p block; h[DIM..2 DIM): (d2H v)_q block
                double h[S2];
#pragma unroll
                for (int u = 0; u < S2; ++u) h[u] = 0.0;
                for (int j = threadIdx.x; j < n; j += kTanThreads) {
                    double d[DIM], dv[DIM], pj[DIM], vpj[DIM];
                    double r2 = 0.0, ddv = 0.0, pp = 0.0, a1 = 0.0;
#pragma unroll
                    for (int c = 0; c < DIM; ++c) {
                        d[c] = qi[c] - __ldcg(Y + (size_t)j * S2 + c);
                        dv[c] = vqi[c] - __ldcg(Tin + (size_t)j * S2 + c);
                        pj[c] = __ldcg(Y + (size_t)j * S2 + DIM + c);
                        vpj[c] = __ldcg(Tin + (size_t)j * S2 + DIM + c);
                        r2 += d[c] * d[c];
                        ddv += d[c] * dv[c];
                        pp += pi[c] * pj[c];
                        a1 += vpi[c] * pj[c] + pi[c] * vpj[c];
                    }
                    double G, phi, psi;
                    kfun3_f64<KER>(r2, a.sigma, G, phi, psi);
#pragma unroll
                    for (int c = 0; c < DIM; ++c) h[c] += G * vpj[c] + phi * ddv * pj[c];
                    if (j != i) {
#pragma unroll
                        for (int c = 0; c < DIM; ++c) h[DIM + c] += a1 * phi * d[c] + pp * (phi * dv[c] + psi * ddv * d[c]);
                    }
                }
                cta_sum_f64<S2, kTanThreads>(h, sm_d);
                // dk = (h_p, -h_q); the tangent RK4 stage, one thread per component
                if (threadIdx.x < S2) {
                    const int c = threadIdx.x;
                    double hc = h[0];
#pragma unroll
                    for (int u = 1; u < S2; ++u) hc = c == u ? h[u] : hc;
                    const double dk = c < DIM ? hc : -hc;
                    double* X = a.dx + (size_t)i * S2 + c;
                    double* A = a.dacc + (size_t)i * S2 + c;
                    if (s < 3) {
                        const double cdt = (s == 2 ? 1.0 : 0.5) * a.dt;
                        Tout[(size_t)i * S2 + c] = *X + cdt * dk;
                        *A = s == 0 ? dk : *A + 2.0 * dk;
                    } else {
                        const double nv = *X + a.dt / 6.0 * (*A + dk);
                        *X = nv;
                        Tout[(size_t)i * S2 + c] = nv;
                    }
                }
            }
            cur ^= 1;
            if (!grid_barrier(a.bar, a.err, ++epoch)) return;
        }
    }
    for (int t = threadIdx.x; t < (r1 - r0) * S2; t += kTanThreads) {
        const int i = r0 + t / S2, c = t % S2;
        const double v = a.dx[(size_t)i * S2 + c];
        if (c < DIM)
            a.out[(size_t)i * DIM + c] = v;
        else
            a.out[nd + (size_t)i * DIM + (c - DIM)] = v;
    }
}

// ------------------------------------------------------------------ dense Newton (small n)
// For n dim <= kDenseNewtonMax the Jacobian D phi = dQ(1)/dp0 is formed column by
// column in one launch: CTA c integrates the tangent shoot along (0, e_c) over all
// particles itself (its tangent state in shared memory, __syncthreads between
// stages, no grid-wide barrier), so the n dim directions run on that many SMs at
// once.  One CTA then solves (D phi) delta = r by Gaussian elimination with
// partial pivoting.
constexpr int kDenseNewtonMax = 384;
constexpr int kJacThreads = 256;       // FP64 columns: the FP64 pipe is the bound
constexpr int kJacMixedThreads = 512;  // FP32 columns: latency-bound, more warps per column

struct JacArgs {
    int n, steps;
    double dt, sigma;
    const double* drec;  // (4 steps + 1) primal stage copies, (q, p) = 2 dim doubles per particle
    double* J;           // n dim x n dim, column-major: J[c N + r] = d Q(1)_r / d p0_c
};

// Warp sum of V <= 8 doubles, reduce-scatter form; afterwards lane l holds the total
// of value first(l) and the lanes with (l & (32 / P - 1)) == 0 hold distinct values.
template <int V, typename T>
__device__ __forceinline__ T warp_sum_scatter(T (&v)[V], int& first)
{
    constexpr int P = V == 1 ? 1 : V == 2 ? 2 : V <= 4 ? 4 : 8;
    const int lane = threadIdx.x & 31;
    T u[P];
#pragma unroll
    for (int k = 0; k < P; ++k) u[k] = k < V ? v[k] : T(0);
    first = 0;
    int cnt = P;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (cnt > 1) {
            const int h = cnt / 2;
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int k = 0; k < P / 2; ++k) {
                if (k < h) {
                    const T send = upper ? u[k] : u[k + h];
                    const T keep = upper ? u[k + h] : u[k];
                    u[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
            }
            if (upper) first += h;
            cnt = h;
        } else {
            u[0] += __shfl_xor_sync(0xffffffffu, u[0], o);
        }
    }
    return u[0];
}

template <int DIM, int KER>
__global__ void __launch_bounds__(kJacThreads) k_jac_fp64(JacArgs a)
{
    constexpr int S2 = 2 * DIM;
    constexpr int P = S2 <= 4 ? 4 : 8;
    extern __shared__ double js[];
    const int n = a.n;
    const int N = n * DIM;
    const int c = blockIdx.x;  // direction (0, e_c)
    const size_t sn = (size_t)S2 * n;
    double* T0 = js;           // tangent stage inputs (ping-pong)
    double* T1 = js + sn;
    double* X0 = js + 2 * sn;  // tangent state at the step start
    double* A = js + 3 * sn;   // tangent RK4 accumulator
    for (int t = threadIdx.x; t < (int)sn; t += kJacThreads) {
        const int i = t / S2, k = t % S2;
        const double v = (k >= DIM && i * DIM + (k - DIM) == c) ? 1.0 : 0.0;
        T0[t] = v;
        X0[t] = v;
        A[t] = 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int W = kJacThreads / 32;
    double* Tin = T0;
    double* Tout = T1;
    for (int k = 0; k < a.steps; ++k) {
        for (int s = 0; s < 4; ++s) {
            const double* Y = a.drec + (size_t)(4 * k + s) * sn;
            for (int i = warp; i < n; i += W) {
                double qi[DIM], pi[DIM], vqi[DIM], vpi[DIM];
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    qi[d] = __ldg(Y + (size_t)i * S2 + d);
                    pi[d] = __ldg(Y + (size_t)i * S2 + DIM + d);
                    vqi[d] = Tin[i * S2 + d];
                    vpi[d] = Tin[i * S2 + DIM + d];
                }
                double h[S2];
#pragma unroll
                for (int u = 0; u < S2; ++u) h[u] = 0.0;
                for (int j = lane; j < n; j += 32) {
                    double dd[DIM], dv[DIM], pj[DIM], vpj[DIM];
                    double r2 = 0.0, ddv = 0.0, pp = 0.0, a1 = 0.0;
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        dd[d] = qi[d] - __ldg(Y + (size_t)j * S2 + d);
                        dv[d] = vqi[d] - Tin[j * S2 + d];
                        pj[d] = __ldg(Y + (size_t)j * S2 + DIM + d);
                        vpj[d] = Tin[j * S2 + DIM + d];
                        r2 += dd[d] * dd[d];
                        ddv += dd[d] * dv[d];
                        pp += pi[d] * pj[d];
                        a1 += vpi[d] * pj[d] + pi[d] * vpj[d];
                    }
                    double G, phi, psi;
                    kfun3_f64<KER>(r2, a.sigma, G, phi, psi);
#pragma unroll
                    for (int d = 0; d < DIM; ++d) h[d] += G * vpj[d] + phi * ddv * pj[d];
                    if (j != i) {
#pragma unroll
                        for (int d = 0; d < DIM; ++d) h[DIM + d] += a1 * phi * dd[d] + pp * (phi * dv[d] + psi * ddv * dd[d]);
                    }
                }
                int first;
                const double tot = warp_sum_scatter<S2, double>(h, first);
                // the tangent RK4 stage of component `first` of row i, dk = (h_p, -h_q)
                if ((lane & (32 / P - 1)) == 0 && first < S2) {
                    const int e = i * S2 + first;
                    const double dk = first < DIM ? tot : -tot;
                    if (s < 3) {
                        const double cdt = (s == 2 ? 1.0 : 0.5) * a.dt;
                        Tout[e] = X0[e] + cdt * dk;
                        A[e] = s == 0 ? dk : A[e] + 2.0 * dk;
                    } else {
                        const double nv = X0[e] + a.dt / 6.0 * (A[e] + dk);
                        X0[e] = nv;
                        Tout[e] = nv;
                    }
                }
            }
            __syncthreads();
            double* tmp = Tin;
            Tin = Tout;
            Tout = tmp;
        }
    }
    // column c of D phi: the position part of the tangent at t1
    for (int r = threadIdx.x; r < N; r += kJacThreads) a.J[(size_t)c * N + r] = X0[(r / DIM) * S2 + (r % DIM)];
}

// FP32 kernel value, phi and psi (unscaled), for the mixed-precision Jacobian.
template <int KER>
__device__ __forceinline__ void kfun3_f32(float r2, float sigma, float& G, float& phi, float& psi)
{
    const float is = 1.0f / sigma;
    if constexpr (KER == EP_GAUSS) {
        G = expf(-0.5f * (r2 * (is * is)));
        phi = -G * (is * is);
        psi = G * (is * is) * (is * is);
    } else if constexpr (KER == EP_TENT) {
        const float r = sqrtf(r2);
        const bool in = r < sigma && r2 > 0.0f;
        const float rs = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
        G = r < sigma ? 1.0f - r * is : 0.0f;
        phi = in ? -is * rs : 0.0f;
        psi = in ? is * rs * rs * rs : 0.0f;
    } else {
        const float r = sqrtf(r2);
        const float rs = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
        G = expf(-r * is);
        phi = r2 > 0.0f ? -G * is * rs : 0.0f;
        psi = r2 > 0.0f ? G * (is * is * rs * rs + is * rs * rs * rs) : 0.0f;
    }
}

// The mixed-precision Jacobian: as k_jac_fp64 with FP32 pair terms and FP32 tangent
// state, against the mixed shoot's recorded stages (scaled positions q' = s (q - c0)
// and momenta in float4 records; d = (q'_i - q'_j) / s).  Newton converges with this
// Jacobian as an inexact Newton method; the residual, the solve and the update stay FP64.
struct JacMArgs {
    int n, steps;
    float dt, sigma, inv_s;
    const float4* rec;  // (4 steps + 1) stage copies, (dim == 2 ? 1 : 2) float4 per particle
    double* J;
};

template <int DIM>
__device__ __forceinline__ void rec_load(const float4* Y, int i, float (&q)[DIM], float (&p)[DIM])
{
    if constexpr (DIM == 2) {
        const float4 v = __ldg(Y + i);
        q[0] = v.x; q[1] = v.y; p[0] = v.z; p[1] = v.w;
    } else {
        const float4 a = __ldg(Y + 2 * (size_t)i), b = __ldg(Y + 2 * (size_t)i + 1);
        q[0] = a.x; q[1] = a.y; q[2] = a.z; p[0] = b.x; p[1] = b.y; p[2] = b.z;
    }
}

template <int DIM, int KER>
__global__ void __launch_bounds__(kJacMixedThreads) k_jac_mixed(JacMArgs a)
{
    constexpr int S2 = 2 * DIM;
    constexpr int P = S2 <= 4 ? 4 : 8;
    constexpr int V = DIM == 2 ? 1 : 2;
    extern __shared__ float jf[];
    const int n = a.n;
    const int N = n * DIM;
    const int c = blockIdx.x;
    const size_t sn = (size_t)S2 * n;
    float* T0 = jf;
    float* T1 = jf + sn;
    float* X0 = jf + 2 * sn;
    float* A = jf + 3 * sn;
    for (int t = threadIdx.x; t < (int)sn; t += kJacMixedThreads) {
        const int i = t / S2, k = t % S2;
        const float v = (k >= DIM && i * DIM + (k - DIM) == c) ? 1.0f : 0.0f;
        T0[t] = v;
        X0[t] = v;
        A[t] = 0.0f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int W = kJacMixedThreads / 32;
    float* Tin = T0;
    float* Tout = T1;
    for (int k = 0; k < a.steps; ++k) {
        for (int s = 0; s < 4; ++s) {
            const float4* Y = a.rec + (size_t)(4 * k + s) * V * n;
            for (int i = warp; i < n; i += W) {
                float qi[DIM], pi[DIM], vqi[DIM], vpi[DIM];
                rec_load<DIM>(Y, i, qi, pi);
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    vqi[d] = Tin[i * S2 + d];
                    vpi[d] = Tin[i * S2 + DIM + d];
                }
                float h[S2];
#pragma unroll
                for (int u = 0; u < S2; ++u) h[u] = 0.0f;
                for (int j = lane; j < n; j += 32) {
                    float qj[DIM], pj[DIM];
                    rec_load<DIM>(Y, j, qj, pj);
                    float dd[DIM], dv[DIM], vpj[DIM];
                    float r2 = 0.0f, ddv = 0.0f, pp = 0.0f, a1 = 0.0f;
#pragma unroll
                    for (int d = 0; d < DIM; ++d) {
                        dd[d] = (qi[d] - qj[d]) * a.inv_s;
                        dv[d] = vqi[d] - Tin[j * S2 + d];
                        vpj[d] = Tin[j * S2 + DIM + d];
                        r2 += dd[d] * dd[d];
                        ddv += dd[d] * dv[d];
                        pp += pi[d] * pj[d];
                        a1 += vpi[d] * pj[d] + pi[d] * vpj[d];
                    }
                    float G, phi, psi;
                    kfun3_f32<KER>(r2, a.sigma, G, phi, psi);
#pragma unroll
                    for (int d = 0; d < DIM; ++d) h[d] += G * vpj[d] + phi * ddv * pj[d];
                    if (j != i) {
#pragma unroll
                        for (int d = 0; d < DIM; ++d) h[DIM + d] += a1 * phi * dd[d] + pp * (phi * dv[d] + psi * ddv * dd[d]);
                    }
                }
                int first;
                const float tot = warp_sum_scatter<S2, float>(h, first);
                if ((lane & (32 / P - 1)) == 0 && first < S2) {
                    const int e = i * S2 + first;
                    const float dk = first < DIM ? tot : -tot;
                    if (s < 3) {
                        const float cdt = (s == 2 ? 1.0f : 0.5f) * a.dt;
                        Tout[e] = X0[e] + cdt * dk;
                        A[e] = s == 0 ? dk : A[e] + 2.0f * dk;
                    } else {
                        const float nv = X0[e] + a.dt / 6.0f * (A[e] + dk);
                        X0[e] = nv;
                        Tout[e] = nv;
                    }
                }
            }
            __syncthreads();
            float* tmp = Tin;
            Tin = Tout;
            Tout = tmp;
        }
    }
    for (int r = threadIdx.x; r < N; r += kJacMixedThreads) a.J[(size_t)c * N + r] = (double)X0[(r / DIM) * S2 + (r % DIM)];
}

// r = Y - Q(1) (Q(1): the first m entries of the step state) and the max-norm of r
// by atomicMax on the IEEE bits (non-finite values rank above every finite one).
__global__ void k_residual(const double* __restrict__ Y, const double* __restrict__ Q1, int m, double* __restrict__ r,
                           unsigned long long* res_bits)
{
    unsigned long long mb = 0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
        const double v = Y[e] - Q1[e];
        r[e] = v;
        const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v));
        mb = b > mb ? b : mb;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = u > mb ? u : mb;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(res_bits, mb);
}

// p += h delta, unless *skip is set (skip may be NULL): a singular solve leaves
// delta unfinished, and p0 must stay the last iterate.
__global__ void k_axpy_update(double* __restrict__ p, const double* __restrict__ delta, double h, int m,
                              const int* __restrict__ skip)
{
    if (skip && *skip) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) p[e] += h * delta[e];
}

// Solve J x = b (J column-major N x N; b overwritten by x) by Gaussian elimination
// with partial pivoting (the largest |pivot| in the column, the first on ties), one
// CTA.  *singular = 1 when a pivot is zero; b is then left partly eliminated and
// must not be used.
// SMEM = false factors J in place (J holds its LU factors afterwards).  SMEM = true
// (N <= kLuSmemMaxN) copies J and b into shared memory, factors the copy and writes
// only x back: J keeps the unfactored matrix.  Callers use x alone and must not rely
// on J's contents after the call.  The arithmetic and its order are the same.
constexpr int kLuThreads = 512;
constexpr int kLuSmemMaxN = 160;  // N^2 + N doubles <= 206 KB of shared memory
template <bool SMEM>
__global__ void __launch_bounds__(kLuThreads) k_lu_solve(int N, double* __restrict__ Jg, double* __restrict__ bg,
                                                        int* singular)
{
    __shared__ double s_val[kLuThreads / 32];
    __shared__ int s_idx[kLuThreads / 32];
    __shared__ int s_piv;
    __shared__ double s_x;
    extern __shared__ double s_mat[];
    double* J = Jg;
    double* b = bg;
    if constexpr (SMEM) {
        J = s_mat;
        b = s_mat + (size_t)N * N;
        for (int t = threadIdx.x; t < N * N; t += kLuThreads) J[t] = Jg[t];
        for (int t = threadIdx.x; t < N; t += kLuThreads) b[t] = bg[t];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int W = kLuThreads / 32;
    auto at = [&](int r, int c) -> double& { return J[(size_t)c * N + r]; };
    for (int k = 0; k < N; ++k) {
        // pivot row: max |J(r, k)| over r >= k
        double best = -1.0;
        int bi = N;
        for (int r = k + threadIdx.x; r < N; r += kLuThreads) {
            const double v = fabs(at(r, k));
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
            s_piv = bix;
            if (!(bv > 0.0)) *singular = 1;
        }
        __syncthreads();
        const int pr = s_piv;
        if (pr >= N) return;  // no pivot at all (all entries NaN): the flag is raised, b is left as is
        // swap rows k and pr over columns k..N-1 and b
        if (pr != k) {
            for (int c = k + threadIdx.x; c <= N; c += kLuThreads) {
                double* x = c < N ? &at(k, c) : &b[k];
                double* y = c < N ? &at(pr, c) : &b[pr];
                const double t = *x;
                *x = *y;
                *y = t;
            }
        }
        __syncthreads();
        const double piv = at(k, k);
        if (piv == 0.0) continue;
        // multipliers, then the trailing update (column c, rows > k) and b
        for (int r = k + 1 + threadIdx.x; r < N; r += kLuThreads) at(r, k) /= piv;
        __syncthreads();
        const int rows = N - k - 1;
        for (int t = threadIdx.x; t < rows * (N - k); t += kLuThreads) {
            const int r = k + 1 + t % rows, c = k + 1 + t / rows;  // c == N: the right-hand side
            if (c < N) at(r, c) -= at(r, k) * at(k, c);
            else b[r] -= at(r, k) * b[k];
        }
        __syncthreads();
    }
    // back substitution
    for (int k = N - 1; k >= 0; --k) {
        double sum = 0.0;
        for (int c = k + 1 + threadIdx.x; c < N; c += kLuThreads) sum += at(k, c) * b[c];
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) s_val[warp] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tsum = 0.0;
            for (int w = 0; w < W; ++w) tsum += s_val[w];
            const double d = at(k, k);
            s_x = d != 0.0 ? (b[k] - tsum) / d : 0.0;
            b[k] = s_x;
        }
        __syncthreads();
    }
    if constexpr (SMEM)
        for (int t = threadIdx.x; t < N; t += kLuThreads) bg[t] = b[t];
}

// ------------------------------------------------------------------ velocity update, mixed precision
// G(X) (FP64 kernel values, all n^2 entries, row-major = column-major: symmetric).
template <int DIM, int KER>
__global__ void k_gram_fp64(const double* __restrict__ X, int n, double sigma, double* __restrict__ Gm)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    const int i = (int)(e / n), j = (int)(e % n);
    double r2 = 0.0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        const double d = X[(size_t)i * DIM + c] - X[(size_t)j * DIM + c];
        r2 += d * d;
    }
    double G, phi;
    kfun_f64<KER>(r2, sigma, G, phi);
    Gm[e] = G;
}

// LU factors of G(X) in place (one CTA); *ok = 1 on success.
__global__ void __launch_bounds__(kLuThreads) k_lu_factor(int n, double* Gm, int* piv, int* ok)
{
    __shared__ double s_v[kLuThreads / 32 + 1];
    __shared__ int s_i[kLuThreads / 32 + 1];
    const bool good = cta_lu_factor<kLuThreads>(n, Gm, piv, s_v, s_i);
    if (threadIdx.x == 0) *ok = good ? 1 : 0;
}

// delta = G(X)^-1 r per component (one warp; scratch: n doubles), r and delta (n, dim).
__global__ void k_gram_solve(int n, int dim, const double* Gm, const int* piv, const double* __restrict__ r,
                             double* __restrict__ delta, double* scratch)
{
    for (int c = 0; c < dim; ++c) {
        for (int i = threadIdx.x; i < n; i += 32) scratch[i] = r[(size_t)i * dim + c];
        __syncwarp();
        warp_lu_solve(n, Gm, piv, scratch);
        for (int i = threadIdx.x; i < n; i += 32) delta[(size_t)i * dim + c] = scratch[i];
        __syncwarp();
    }
}

// G(X)^-1 from its LU factors, one column per CTA (one warp: the substitutions of
// LU x = P e_c); Ginv row-major (n x n).  n <= kSmallMatchMaxN (shared scratch).
__global__ void k_lu_inverse(int n, const double* __restrict__ LU, const int* __restrict__ piv, double* __restrict__ Ginv)
{
    __shared__ double b[kSmallMatchMaxN];
    const int c = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += 32) b[i] = i == c ? 1.0 : 0.0;
    __syncwarp();
    warp_lu_solve(n, LU, piv, b);
    for (int i = threadIdx.x; i < n; i += 32) Ginv[(size_t)i * n + c] = b[i];
}

// Device buffers of one tangent-linear problem.
struct TanBufs {
    AllPairsBufs ap;
    double* drec = nullptr;  // FP64 recording
    float4* rec = nullptr;   // mixed recording (scaled positions, FP32)
    double* dx = nullptr;
    double* dacc = nullptr;
    double* T[2] = {nullptr, nullptr};
    double* v0 = nullptr;
    double* out = nullptr;
    unsigned* bar = nullptr;
    int* err = nullptr;
};

size_t tan_bytes(int64_t n, int dim, int steps, int prec = EP_FP64)
{
    Sizer z;
    const size_t m = (size_t)n * dim;
    z.add(allpairs_bytes((int)n, dim, prec));
    if (prec == EP_MIXED)
        z.add(sizeof(float4) * (dim == 2 ? 1 : 2) * (size_t)n * (4 * (size_t)steps + 1));  // recorded stages
    else
        z.add(sizeof(double) * 2 * m * (4 * (size_t)steps + 1));
    for (int k = 0; k < 4; ++k) z.add(sizeof(double) * 2 * m);  // dx, dacc, T[2]
    z.add(sizeof(double) * 2 * m * 2);                          // v0, out
    z.add(sizeof(unsigned) * 12);
    return z.total;
}

ep_status tan_carve(Arena* ar, int64_t n, int dim, int steps, TanBufs* t, int prec = EP_FP64)
{
    const size_t m = (size_t)n * dim;
    EP_TRY(allpairs_carve(ar, (int)n, dim, prec, &t->ap));
    if (prec == EP_MIXED)
        t->rec = (float4*)ar->carve(sizeof(float4) * (dim == 2 ? 1 : 2) * (size_t)n * (4 * (size_t)steps + 1));
    else
        t->drec = (double*)ar->carve(sizeof(double) * 2 * m * (4 * (size_t)steps + 1));
    t->dx = (double*)ar->carve(sizeof(double) * 2 * m);
    t->dacc = (double*)ar->carve(sizeof(double) * 2 * m);
    t->T[0] = (double*)ar->carve(sizeof(double) * 2 * m);
    t->T[1] = (double*)ar->carve(sizeof(double) * 2 * m);
    t->v0 = (double*)ar->carve(sizeof(double) * 2 * m);
    t->out = (double*)ar->carve(sizeof(double) * 2 * m);
    t->bar = (unsigned*)ar->carve(sizeof(unsigned) * 12);
    if (!t->bar) return set_error("workspace too small for the tangent shoot"), EP_ENOMEM;
    t->err = (int*)(t->bar + 8);
    return EP_OK;
}

// Primal shoot from (q0, p0) with every stage input recorded in t.drec (FP64) or
// t.rec (mixed).
ep_status tan_record(const ep_params& P, TanBufs& t, const double* q0, const double* p0, cudaStream_t st)
{
    EP_TRY(allpairs_load(P, t.ap, q0, p0, st));
    return allpairs_steps_rec(P, t.ap, P.steps, P.t1 / P.steps, t.rec, t.drec, st);
}

template <int DIM, int KER>
ep_status launch_tangent(TanArgs& a, cudaStream_t st)
{
    auto fn = k_tangent_fp64<DIM, KER>;
    static int resident = -1;
    if (resident < 0) {
        int per_sm = 0;
        EP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTanThreads, 0));
        DeviceInfo di{};
        EP_TRY(device_info(&di));
        resident = per_sm * di.sm_count;
    }
    DeviceInfo di{};
    EP_TRY(device_info(&di));
    const int G = std::max(1, std::min({a.n, di.sm_count, resident}));
    void* args[] = {&a};
    count_launch();
    EP_TRY_CUDA(cudaLaunchCooperativeKernel((void*)fn, dim3(G), dim3(kTanThreads), args, 0, st));
    return EP_OK;
}

// Tangent shoot along t.v0 at the recorded primal trajectory; result in t.out.
ep_status tan_apply(const ep_params& P, TanBufs& t, int64_t n, cudaStream_t st)
{
    TanArgs a{};
    a.n = (int)n;
    a.steps = P.steps;
    a.dt = P.t1 / P.steps;
    a.sigma = P.sigma;
    a.drec = t.drec;
    a.v0 = t.v0;
    a.dx = t.dx;
    a.dacc = t.dacc;
    a.T[0] = t.T[0];
    a.T[1] = t.T[1];
    a.out = t.out;
    a.bar = t.bar;
    a.err = t.err;
    EP_TRY_CUDA(cudaMemsetAsync(t.bar, 0, sizeof(unsigned) * 12, st));
    // optional CUDA events around the launch (ep_set_launch_timing)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (launch_timing_enabled() && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
        if (e0) cudaEventDestroy(e0);
        e0 = e1 = nullptr;
    }
    if (e0) cudaEventRecord(e0, st);
    ep_status s = EP_EINVAL;
#define EP_TAN_CASE(D, K) \
    if (P.dim == D && P.kernel == K) s = launch_tangent<D, K>(a, st);
    EP_TAN_CASE(2, EP_GAUSS) EP_TAN_CASE(2, EP_TENT) EP_TAN_CASE(2, EP_EXPCONE)
    EP_TAN_CASE(3, EP_GAUSS) EP_TAN_CASE(3, EP_TENT) EP_TAN_CASE(3, EP_EXPCONE)
#undef EP_TAN_CASE
    if (e0) cudaEventRecord(e1, st);
    int herr = 0;
    if (s == EP_OK) s = cudaMemcpyAsync(&herr, t.err, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess
                            ? EP_OK : cuda_fail(cudaGetLastError(), "tangent error flag");
    if (s == EP_OK) s = cudaStreamSynchronize(st) == cudaSuccess ? EP_OK : cuda_fail(cudaGetLastError(), "tangent sync");
    if (e0 && s == EP_OK) record_launch_time(e0, e1, "k_tangent_fp64");
    if (e0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (s != EP_OK) return s == EP_EINVAL ? (set_error("no tangent kernel for this kernel"), s) : s;
    if (herr) return set_error("tangent shoot: a grid-barrier wait gave up (kernel ended early)"), EP_ETIMEOUT;
    return EP_OK;
}

bool dev_ptr(const void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

ep_status copy_in(double* dst, const double* src, size_t cnt, cudaStream_t st)
{
    EP_TRY_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * cnt, cudaMemcpyDefault, st));
    return EP_OK;
}

// Restarted GMRES for (D phi) x = b with products y = (D phi) v computed by apply.
// Stops at |b - (D phi) x| <= tol |b|, after maxit products in total, or at
// breakdown.  Returns the number of products used.
template <typename Apply>
ep_status gmres(Apply apply, const std::vector<double>& b, std::vector<double>& x, int m, int maxit, double tol,
                int* used)
{
    const size_t N = b.size();
    x.assign(N, 0.0);
    double bn = 0.0;
    for (double v : b) bn += v * v;
    bn = sqrt(bn);
    *used = 0;
    if (bn == 0.0) return EP_OK;
    std::vector<std::vector<double>> V(m + 1, std::vector<double>(N));
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), w(N), y(m);
    std::vector<double> r(b);
    bool first = true;
    while (*used < maxit) {
        if (!first) {
            EP_TRY(apply(x, w));
            ++*used;
            for (size_t k = 0; k < N; ++k) r[k] = b[k] - w[k];
        }
        first = false;
        double beta = 0.0;
        for (double v : r) beta += v * v;
        beta = sqrt(beta);
        if (beta <= tol * bn) break;
        for (size_t k = 0; k < N; ++k) V[0][k] = r[k] / beta;
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jend = 0;
        bool converged = false;
        for (int j = 0; j < m && *used < maxit; ++j) {
            EP_TRY(apply(V[j], w));
            ++*used;
            for (int i = 0; i <= j; ++i) {  // modified Gram-Schmidt
                double hij = 0.0;
                for (size_t k = 0; k < N; ++k) hij += w[k] * V[i][k];
                H[(size_t)i * m + j] = hij;
                for (size_t k = 0; k < N; ++k) w[k] -= hij * V[i][k];
            }
            double hn = 0.0;
            for (double v : w) hn += v * v;
            hn = sqrt(hn);
            H[(size_t)(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {  // previous rotations
                const double a0 = H[(size_t)i * m + j], a1 = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a0 + sn[i] * a1;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a0 + cs[i] * a1;
            }
            const double a0 = H[(size_t)j * m + j], a1 = H[(size_t)(j + 1) * m + j];
            const double den = hypot(a0, a1);
            cs[j] = den > 0.0 ? a0 / den : 1.0;
            sn[j] = den > 0.0 ? a1 / den : 0.0;
            H[(size_t)j * m + j] = den;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            jend = j + 1;
            if (fabs(g[j + 1]) <= tol * bn || hn == 0.0) {
                converged = true;
                break;
            }
            for (size_t k = 0; k < N; ++k) V[j + 1][k] = w[k] / hn;
        }
        for (int i = jend - 1; i >= 0; --i) {  // back substitution
            double s = g[i];
            for (int k = i + 1; k < jend; ++k) s -= H[(size_t)i * m + k] * y[k];
            y[i] = H[(size_t)i * m + i] != 0.0 ? s / H[(size_t)i * m + i] : 0.0;
        }
        for (int i = 0; i < jend; ++i)
            for (size_t k = 0; k < N; ++k) x[k] += y[i] * V[i][k];
        // converged (or broke down) inside the cycle, else restart from the true residual
        if (jend == 0 || converged) break;
    }
    return EP_OK;
}

}  // namespace

ep_status tangent_entry(const ep_params* params, int64_t n, const double* q0, const double* p0, const double* vq0,
                        const double* vp0, double* q1, double* p1, double* vq1, double* vp1, void* stream)
{
    EP_TRY(check_params(params));
    const ep_params& P = *params;
    if (n < 0 || n > ((int64_t)1 << 26)) return set_error("ep_shoot_tangent: bad n"), EP_EINVAL;
    if (P.precision != EP_FP64) return set_error("ep_shoot_tangent runs in FP64"), EP_EINVAL;
    if (P.neigh == EP_CELLLIST) return set_error("ep_shoot_tangent runs on the all-pairs path"), EP_EINVAL;
    if (P.inexact != 0.0) return set_error("ep_shoot_tangent is built for the exact system"), EP_EINVAL;
    if (n == 0) return EP_OK;
    if (!q0 || !p0 || !vq0 || !vp0 || !vq1 || !vp1) return set_error("ep_shoot_tangent: NULL array"), EP_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t m = (size_t)n * P.dim;
    Sizer z;
    z.add(tan_bytes(n, P.dim, P.steps));
    z.add(sizeof(double) * m * 2);
    Arena* ar = nullptr;
    EP_TRY(arena_acquire(st, z.total, &ar));
    TanBufs t;
    EP_TRY(tan_carve(ar, n, P.dim, P.steps, &t));
    double* dq0 = (double*)ar->carve(sizeof(double) * m);
    double* dp0 = (double*)ar->carve(sizeof(double) * m);
    if (!dp0) return set_error("ep_shoot_tangent: workspace too small"), EP_ENOMEM;
    EP_TRY(copy_in(dq0, q0, m, st));
    EP_TRY(copy_in(dp0, p0, m, st));
    EP_TRY(copy_in(t.v0, vq0, m, st));
    EP_TRY(copy_in(t.v0 + m, vp0, m, st));
    EP_TRY(tan_record(P, t, dq0, dp0, st));
    EP_TRY(tan_apply(P, t, n, st));
    if (q1) EP_TRY_CUDA(cudaMemcpyAsync(q1, t.ap.x, sizeof(double) * m, cudaMemcpyDefault, st));
    if (p1) EP_TRY_CUDA(cudaMemcpyAsync(p1, t.ap.x + m, sizeof(double) * m, cudaMemcpyDefault, st));
    EP_TRY_CUDA(cudaMemcpyAsync(vq1, t.out, sizeof(double) * m, cudaMemcpyDefault, st));
    EP_TRY_CUDA(cudaMemcpyAsync(vp1, t.out + m, sizeof(double) * m, cudaMemcpyDefault, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    return EP_OK;
}

// Algorithm 1 with the Newton-type gain M = h (D phi)^-1 of Sec. 5 (Theorem 1):
// (D phi) delta = r solved by restarted GMRES (D phi is not symmetric) whose
// products are tangent shoots.
ep_status rule_match(const ep_params& P, int64_t n, const double* X, const double* Y, double* p0,
                     ep_match_info* info, cudaStream_t st)
{
    const size_t m0 = (size_t)n * P.dim;
    const bool mixed = P.precision == EP_MIXED;
    if (mixed && m0 > (size_t)kDenseNewtonMax)
        return set_error("ep_match: the mixed-precision Newton gain forms the whole Jacobian (n dim <= %d)",
                         kDenseNewtonMax), EP_EINVAL;
    if (P.neigh == EP_CELLLIST) return set_error("ep_match: the Newton gain runs on the all-pairs path"), EP_EINVAL;
    if (P.inexact != 0.0) return set_error("ep_match: the Newton gain is built for the exact system"), EP_EINVAL;
    if (info->krylov < 0) return set_error("ep_match: krylov must be >= 0"), EP_EINVAL;
    const size_t m = (size_t)n * P.dim;
    // small problems form D phi whole (one CTA per column) and solve it densely
    const bool dense = m <= (size_t)kDenseNewtonMax;
    Sizer z;
    z.add(tan_bytes(n, P.dim, P.steps, P.precision));
    z.add(sizeof(double) * m * 6);
    if (dense) {
        z.add(sizeof(double) * m * m);
        z.add(sizeof(double) * m * 2);
        z.add(64);
    }
    Arena* ar = nullptr;
    EP_TRY(arena_acquire(st, z.total, &ar));
    TanBufs t;
    EP_TRY(tan_carve(ar, n, P.dim, P.steps, &t, P.precision));
    double* dX = (double*)ar->carve(sizeof(double) * m);
    double* dp = (double*)ar->carve(sizeof(double) * m);
    double* dk = (double*)ar->carve(sizeof(double) * m);
    double* dd = (double*)ar->carve(sizeof(double) * m);
    if (!dd) return set_error("ep_match: workspace too small"), EP_ENOMEM;
    double *dJ = nullptr, *dY = nullptr, *dr = nullptr;
    unsigned long long* dres = nullptr;
    int* dsing = nullptr;
    if (dense) {
        dJ = (double*)ar->carve(sizeof(double) * m * m);
        dY = (double*)ar->carve(sizeof(double) * m);
        dr = (double*)ar->carve(sizeof(double) * m);
        dres = (unsigned long long*)ar->carve(64);
        if (!dres) return set_error("ep_match: workspace too small"), EP_ENOMEM;
        dsing = (int*)(dres + 4);
        EP_TRY(copy_in(dY, Y, m, st));
    }
    EP_TRY(copy_in(dX, X, m, st));
    EP_TRY(copy_in(dp, p0, m, st));
    std::vector<double> hY(m), hp(m), hq(m), r(m), delta;
    EP_TRY_CUDA(cudaMemcpyAsync(hY.data(), Y, sizeof(double) * m, cudaMemcpyDefault, st));
    EP_TRY_CUDA(cudaMemcpyAsync(hp.data(), dp, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    const double h = info->h > 0.0 ? info->h : 1.0;
    info->h = h;
    const int N = (int)std::min<size_t>(m, (size_t)1 << 30);
    const int krylov = info->krylov > 0 ? std::min(info->krylov, N) : std::min(N, 200);
    const int maxprod = 4 * krylov;
    const bool hist_dev = info->hist && dev_ptr(info->hist);
    // (D phi) v: a tangent shoot along (0, v) at the recorded trajectory
    auto apply = [&](const std::vector<double>& v, std::vector<double>& out) -> ep_status {
        EP_TRY_CUDA(cudaMemsetAsync(t.v0, 0, sizeof(double) * m, st));
        EP_TRY_CUDA(cudaMemcpyAsync(t.v0 + m, v.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
        EP_TRY(tan_apply(P, t, n, st));
        EP_TRY_CUDA(cudaMemcpyAsync(out.data(), t.out, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
        EP_TRY_CUDA(cudaStreamSynchronize(st));
        return EP_OK;
    };
    ep_status status = EP_ENOTCONVERGED;
    int k = 0;
    double res = 0.0;
    bool singular = false;
    for (;;) {
        // Q(1): the step state x of the all-pairs buffers after the recorded shoot
        EP_TRY(tan_record(P, t, dX, dp, st));
        bool finite = true;
        if (dense) {
            // r = Y - Q(1) and |r|_inf on the device
            unsigned long long rb = 0;
            EP_TRY_CUDA(cudaMemsetAsync(dres, 0, sizeof(unsigned long long), st));
            count_launch();
            k_residual<<<(unsigned)std::min<size_t>((m + 255) / 256, 1024), 256, 0, st>>>(dY, t.ap.x, (int)m, dr, dres);
            EP_TRY_CUDA(cudaGetLastError());
            EP_TRY_CUDA(cudaMemcpyAsync(&rb, dres, sizeof rb, cudaMemcpyDeviceToHost, st));
            EP_TRY_CUDA(cudaStreamSynchronize(st));
            finite = rb < 0x7FF0000000000000ull;
            memcpy(&res, &rb, sizeof res);
        } else {
            EP_TRY_CUDA(cudaMemcpyAsync(hq.data(), t.ap.x, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
            EP_TRY_CUDA(cudaStreamSynchronize(st));
            res = 0.0;
            for (size_t a = 0; a < m; ++a) {
                r[a] = hY[a] - hq[a];
                if (!std::isfinite(r[a])) finite = false;
                res = std::max(res, fabs(r[a]));
            }
        }
        if (!finite) res = NAN;
        if (info->hist) {
            if (hist_dev)
                EP_TRY_CUDA(cudaMemcpyAsync(info->hist + k, &res, sizeof(double), cudaMemcpyHostToDevice, st));
            else
                info->hist[k] = res;
        }
        if (!finite) {
            status = EP_EDIVERGED;
            break;
        }
        if (res < info->eps) {
            status = EP_OK;
            break;
        }
        if (k == info->maxit) {
            status = EP_ENOTCONVERGED;
            break;
        }
        if (dense) {
            // D phi by columns (one tangent shoot per CTA), then (D phi) delta = r, p0 += h delta
            JacArgs ja{};
            ja.n = (int)n;
            ja.steps = P.steps;
            ja.dt = P.t1 / P.steps;
            ja.sigma = P.sigma;
            ja.drec = t.drec;
            ja.J = dJ;
            ep_status ls = EP_EINVAL;
            if (mixed) {
                JacMArgs jm{};
                jm.n = (int)n;
                jm.steps = P.steps;
                jm.dt = (float)(P.t1 / P.steps);
                jm.sigma = (float)P.sigma;
                jm.inv_s = (float)(1.0 / kernel_scale(P.kernel, P.sigma).s);
                jm.rec = t.rec;
                jm.J = dJ;
                const size_t smem = sizeof(float) * 4 * 2 * (size_t)P.dim * n;
#define EP_JAC_CASE(D, K) \
    if (P.dim == D && P.kernel == K) { count_launch(); k_jac_mixed<D, K><<<(unsigned)m, kJacMixedThreads, smem, st>>>(jm); ls = EP_OK; }
                EP_JAC_CASE(2, EP_GAUSS) EP_JAC_CASE(2, EP_TENT) EP_JAC_CASE(2, EP_EXPCONE)
                EP_JAC_CASE(3, EP_GAUSS) EP_JAC_CASE(3, EP_TENT) EP_JAC_CASE(3, EP_EXPCONE)
#undef EP_JAC_CASE
            } else {
                const size_t smem = sizeof(double) * 4 * 2 * (size_t)P.dim * n;
#define EP_JAC_CASE(D, K) \
    if (P.dim == D && P.kernel == K) { count_launch(); k_jac_fp64<D, K><<<(unsigned)m, kJacThreads, smem, st>>>(ja); ls = EP_OK; }
                EP_JAC_CASE(2, EP_GAUSS) EP_JAC_CASE(2, EP_TENT) EP_JAC_CASE(2, EP_EXPCONE)
                EP_JAC_CASE(3, EP_GAUSS) EP_JAC_CASE(3, EP_TENT) EP_JAC_CASE(3, EP_EXPCONE)
#undef EP_JAC_CASE
            }
            if (ls != EP_OK) return set_error("ep_match: no Jacobian kernel for this kernel"), ls;
            EP_TRY_CUDA(cudaMemsetAsync(dsing, 0, sizeof(int), st));
            count_launch(2);
            if (m <= (size_t)kLuSmemMaxN) {
                const size_t lsm = sizeof(double) * (m * m + m);
                EP_TRY_CUDA(cudaFuncSetAttribute(k_lu_solve<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm));
                k_lu_solve<true><<<1, kLuThreads, lsm, st>>>((int)m, dJ, dr, dsing);
            } else {
                k_lu_solve<false><<<1, kLuThreads, 0, st>>>((int)m, dJ, dr, dsing);
            }
            k_axpy_update<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(dp, dr, h, (int)m, dsing);
            EP_TRY_CUDA(cudaGetLastError());
            int sing = 0;
            EP_TRY_CUDA(cudaMemcpyAsync(&sing, dsing, sizeof(int), cudaMemcpyDeviceToHost, st));
            EP_TRY_CUDA(cudaStreamSynchronize(st));
            info->products += (int)m;
            if (sing) {
                // no update was applied: p0 is the iterate of the last shoot
                set_error("ep_match: the shooting Jacobian is singular after %d updates", k);
                singular = true;
                status = EP_EDIVERGED;
                break;
            }
            ++k;
            continue;
        }
        int used = 0;
        EP_TRY(gmres(apply, r, delta, krylov, maxprod, kKrylovTol, &used));
        info->products += used;
        for (size_t a = 0; a < m; ++a) hp[a] += h * delta[a];
        EP_TRY_CUDA(cudaMemcpyAsync(dp, hp.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
        ++k;
    }
    info->iters = k;
    info->resid_inf = res;
    EP_TRY_CUDA(cudaMemcpyAsync(p0, dp, sizeof(double) * m, cudaMemcpyDefault, st));
    if (dense) EP_TRY_CUDA(cudaMemcpyAsync(hp.data(), dp, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    // H(X, p0) of Eq. H: 1/2 sum_i p_i . dq_i
    EP_TRY(allpairs_load(P, t.ap, dX, dp, st));
    EP_TRY(allpairs_rhs(P, t.ap, dk, dd, st));
    std::vector<double> hdq(m);
    EP_TRY_CUDA(cudaMemcpyAsync(hdq.data(), dk, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    double H = 0.0;
    for (size_t a = 0; a < m; ++a) H += 0.5 * hp[a] * hdq[a];
    info->H = H;
    if (status == EP_ENOTCONVERGED) set_error("ep_match: %d iterations, residual %.3e >= eps %.3e", k, res, info->eps);
    if (status == EP_EDIVERGED && !singular) set_error("ep_match: residual became non-finite after %d updates", k);
    return status;
}

// Algorithm 1 with the velocity update in mixed precision (n <= kGramLuMaxMixed):
// mixed shoots, FP64 residual, G(X) built in FP64 and factored once, each update a
// forward and a back substitution per component, FP64 update.
constexpr int64_t kGramLuMaxMixed = 512;

ep_status velocity_mixed_match(const ep_params& P, int64_t n, const double* X, const double* Y, double* p0,
                               ep_match_info* info, cudaStream_t st)
{
    if (n > kGramLuMaxMixed)
        return set_error("ep_match: the mixed-precision velocity update factors G(X) (n <= %lld)",
                         (long long)kGramLuMaxMixed), EP_EINVAL;
    if (P.neigh == EP_CELLLIST) return set_error("ep_match: the velocity update runs on the all-pairs path"), EP_EINVAL;
    if (P.inexact != 0.0) return set_error("ep_match: the velocity update is built for the exact system"), EP_EINVAL;
    const size_t m = (size_t)n * P.dim;
    Sizer z;
    z.add(allpairs_bytes((int)n, P.dim, EP_MIXED));
    z.add(sizeof(double) * (size_t)n * n);
    z.add(sizeof(int) * (size_t)n);
    for (int k = 0; k < 7; ++k) z.add(sizeof(double) * m);
    z.add(64);
    z.add(sizeof(double) * (size_t)n * n);  // G(X)^-1 (small planar problems)
    Arena* ar = nullptr;
    EP_TRY(arena_acquire(st, z.total, &ar));
    AllPairsBufs ap;
    EP_TRY(allpairs_carve(ar, (int)n, P.dim, EP_MIXED, &ap));
    double* Gm = (double*)ar->carve(sizeof(double) * (size_t)n * n);
    int* piv = (int*)ar->carve(sizeof(int) * (size_t)n);
    double* dX = (double*)ar->carve(sizeof(double) * m);
    double* dY = (double*)ar->carve(sizeof(double) * m);
    double* dp = (double*)ar->carve(sizeof(double) * m);
    double* dr = (double*)ar->carve(sizeof(double) * m);
    double* dl = (double*)ar->carve(sizeof(double) * m);
    double* dk = (double*)ar->carve(sizeof(double) * m);
    double* dd = (double*)ar->carve(sizeof(double) * m);
    unsigned long long* dres = (unsigned long long*)ar->carve(64);
    if (!dres) return set_error("ep_match: workspace too small"), EP_ENOMEM;
    int* dok = (int*)(dres + 4);
    EP_TRY(copy_in(dX, X, m, st));
    EP_TRY(copy_in(dY, Y, m, st));
    EP_TRY(copy_in(dp, p0, m, st));
    const double h = info->h > 0.0 ? info->h : 1.0;
    info->h = h;
    const bool hist_dev = info->hist && dev_ptr(info->hist);
    // G(X) and its LU factors, once
    const long long nn = (long long)n * n;
    ep_status ls = EP_EINVAL;
#define EP_GRAM_CASE(D, K) \
    if (P.dim == D && P.kernel == K) { count_launch(); k_gram_fp64<D, K><<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(dX, (int)n, P.sigma, Gm); ls = EP_OK; }
    EP_GRAM_CASE(2, EP_GAUSS) EP_GRAM_CASE(2, EP_TENT) EP_GRAM_CASE(2, EP_EXPCONE)
    EP_GRAM_CASE(3, EP_GAUSS) EP_GRAM_CASE(3, EP_TENT) EP_GRAM_CASE(3, EP_EXPCONE)
#undef EP_GRAM_CASE
    if (ls != EP_OK) return set_error("ep_match: no Gram kernel for this kernel"), ls;
    count_launch();
    k_lu_factor<<<1, kLuThreads, 0, st>>>((int)n, Gm, piv, dok);
    EP_TRY_CUDA(cudaGetLastError());
    int ok = 0;
    EP_TRY_CUDA(cudaMemcpyAsync(&ok, dok, sizeof(int), cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    if (!ok) return set_error("ep_match: G(X) is singular (the velocity update needs G(X)^-1)"), EP_EDIVERGED;
    if (P.dim == 2 && n <= kSmallMatchMaxN) {
        // small planar problems: G(X)^-1 formed once, then the whole feedback loop (mixed
        // shoots, FP64 residual, FP64 update p0 += h G(X)^-1 r) in one launch on one CTA
        double* Ginv = (double*)ar->carve(sizeof(double) * (size_t)n * n);
        if (!Ginv) return set_error("ep_match: workspace too small"), EP_ENOMEM;
        count_launch();
        k_lu_inverse<<<(unsigned)n, 32, 0, st>>>((int)n, Gm, piv, Ginv);
        EP_TRY_CUDA(cudaGetLastError());
        ep_params Pv = P;
        ep_match_info iv = *info;
        const ep_status s = match_small(&Pv, n, dX, dY, dp, &iv, st, Ginv);
        if (s != EP_OK && s != EP_ENOTCONVERGED && s != EP_EDIVERGED) return s;
        info->iters = iv.iters;
        info->resid_inf = iv.resid_inf;
        info->H = iv.H;
        info->products = P.dim * iv.iters;
        EP_TRY_CUDA(cudaMemcpyAsync(p0, dp, sizeof(double) * m, cudaMemcpyDefault, st));
        EP_TRY_CUDA(cudaStreamSynchronize(st));
        if (s == EP_ENOTCONVERGED)
            set_error("ep_match: %d iterations, residual %.3e >= eps %.3e", iv.iters, iv.resid_inf, info->eps);
        if (s == EP_EDIVERGED) set_error("ep_match: residual became non-finite after %d updates", iv.iters);
        return s;
    }
    ep_status status = EP_ENOTCONVERGED;
    int k = 0;
    double res = 0.0;
    const double dt = P.t1 / P.steps;
    for (;;) {
        EP_TRY(allpairs_load(P, ap, dX, dp, st));
        EP_TRY(allpairs_steps(P, ap, P.steps, dt, st));
        unsigned long long rb = 0;
        EP_TRY_CUDA(cudaMemsetAsync(dres, 0, sizeof(unsigned long long), st));
        count_launch();
        k_residual<<<(unsigned)std::min<size_t>((m + 255) / 256, 1024), 256, 0, st>>>(dY, ap.x, (int)m, dr, dres);
        EP_TRY_CUDA(cudaGetLastError());
        EP_TRY_CUDA(cudaMemcpyAsync(&rb, dres, sizeof rb, cudaMemcpyDeviceToHost, st));
        EP_TRY_CUDA(cudaStreamSynchronize(st));
        const bool finite = rb < 0x7FF0000000000000ull;
        memcpy(&res, &rb, sizeof res);
        if (!finite) res = NAN;
        if (info->hist) {
            if (hist_dev)
                EP_TRY_CUDA(cudaMemcpyAsync(info->hist + k, &res, sizeof(double), cudaMemcpyHostToDevice, st));
            else
                info->hist[k] = res;
        }
        if (!finite) { status = EP_EDIVERGED; break; }
        if (res < info->eps) { status = EP_OK; break; }
        if (k == info->maxit) { status = EP_ENOTCONVERGED; break; }
        count_launch(2);
        k_gram_solve<<<1, 32, 0, st>>>((int)n, P.dim, Gm, piv, dr, dl, dk);
        k_axpy_update<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(dp, dl, h, (int)m, nullptr);
        EP_TRY_CUDA(cudaGetLastError());
        info->products += P.dim;
        ++k;
    }
    info->iters = k;
    info->resid_inf = res;
    EP_TRY_CUDA(cudaMemcpyAsync(p0, dp, sizeof(double) * m, cudaMemcpyDefault, st));
    // H(X, p0) of Eq. H: 1/2 sum_i p_i . dq_i
    EP_TRY(allpairs_load(P, ap, dX, dp, st));
    EP_TRY(allpairs_rhs(P, ap, dk, dd, st));
    std::vector<double> hp(m), hdq(m);
    EP_TRY_CUDA(cudaMemcpyAsync(hp.data(), dp, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaMemcpyAsync(hdq.data(), dk, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    double H = 0.0;
    for (size_t a = 0; a < m; ++a) H += 0.5 * hp[a] * hdq[a];
    info->H = H;
    if (status == EP_ENOTCONVERGED) set_error("ep_match: %d iterations, residual %.3e >= eps %.3e", k, res, info->eps);
    if (status == EP_EDIVERGED) set_error("ep_match: residual became non-finite after %d updates", k);
    return status;
}

}  // namespace ep
