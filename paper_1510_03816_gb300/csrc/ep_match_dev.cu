// ep_match_dev.cu -- Algorithm 1 (the feedback-control shooting iteration,
// Sec. 3) run entirely on the device for the plain FP64 method: one cooperative
// launch per match, no host round trip per iterate or per RK4 stage.
//
// Every CTA owns the particles [c n / G, (c+1) n / G) and evaluates their rows of
// Eq. N-particle over all n sources in FP64, then applies the classical RK4 stage
// (Sec. 4) to them; one grid-wide barrier per stage publishes the next stage's
// inputs.  After a shoot the max-norm residual |Y - Q(1)|_inf is reduced across
// CTAs (each CTA's maximum joins a per-iterate slot by atomicMax on the IEEE bit
// pattern, which orders non-negative doubles and ranks inf and NaN above every
// finite value), and every CTA takes the same stop decision after the barrier:
// non-finite -> diverged, below eps -> converged, maxit updates -> not converged,
// else p0 += h (Y - Q(1)) on its own particles (the momentum rule).  The default
// gain h = 1 / max_i sum_j G_ij is computed the same way before the first shoot,
// and H(X, p0) of the returned momenta (Eq. H) after the last.
//
// The velocity rule (Algorithm 1 steps 3-4: u = G(X) p0 gains h (Y - Q(1)), then
// p0 = G(X)^-1 u) replaces the update by p0 += h delta with G(X) delta = Y - Q(1),
// solved in the same launch by MINRES (Paige and Saunders' minimum-residual
// Lanczos method: G(X) is symmetric but the tent's need not be positive definite
// in two or three dimensions).  Each MINRES iteration is one Gram product on the
// owned rows (G(X) v over all sources), two grid-wide sums (v . z and |z|^2, as
// per-CTA partials that every CTA adds in the same order, so all CTAs hold the same
// scalars) and the publication of the next Lanczos vector: three grid barriers.
// For n <= kGramLuMaxN, CTA 0 instead factors G(X) once (LU with partial pivoting,
// G(X) being symmetric and fixed for the whole matching) and each update is a
// forward and a back substitution per component by one warp; MINRES remains the
// solver when a pivot vanishes.
//
// FP64 on this GPU runs at 1/64 of the FP32 rate, so a small problem's FP64 pair
// work is spread over as many SMs as there are particles (up to the SM count);
// within a CTA the sources of a row are split across all warps, so every SM
// sub-partition's FP64 pipe works on it.
#include <stdint.h>

#include <algorithm>

#include "ep_allpairs_dev.cuh"
#include "ep_features.cuh"

namespace ep {

namespace {

constexpr int kMatchThreads = 256;
constexpr int kGramLuMaxN = 512;  // the velocity rule factors G(X) up to this many landmarks

struct MatchArgs {
    int n, steps, maxit;
    int rule;                  // EP_RULE_MOMENTUM or EP_RULE_VELOCITY
    int kmax;                  // MINRES iteration cap of one velocity-rule solve
    double ktol;               // MINRES stop: |G delta - r| <= ktol |r|
    double sigma, dt, eps, h;  // h <= 0: default gain, computed in the kernel
    double s2;                 // sigma_n^2 of the inexact system (Sec. 6), 0 for the exact one
    const double* X;
    const double* Y;
    double* p0;                // in: initial momenta, out: the last iterate
    double* x;                 // step state [q (n dim) | p (n dim)]
    double* D[3];              // stage copies (2 dim per particle): step start, ping, pong
    double* acc;               // RK4 accumulator k1 + 2 k2 + 2 k3 (2 dim per particle)
    double* hist;              // maxit + 1 residuals (device) or null
    unsigned long long* red;   // [0] max row sum (bits), [1 + k] residual of iterate k (bits)
    double* part;              // per-CTA partial sums (H; v . z and |z|^2 of MINRES), 3 slots of gridDim.x
    double* V[2];              // MINRES Lanczos vector, published (ping-pong), n dim each
    double* Vold;              // previous Lanczos vector (own rows)
    double* W[2];              // MINRES search directions w_{k-1}, w_{k-2} (own rows)
    double* Z;                 // G(X) v - beta v_old (own rows)
    double* Del;               // the MINRES iterate delta (own rows)
    double* Gm;                // G(X), n x n row-major (own rows written), or null: evaluate per pair
    int* piv;                  // pivots of the LU factors of G(X) (n <= kGramLuMaxN)
    int* lu_ok;                // 1 when CTA 0 factored G(X) (then the updates solve with the factors)
    double* out;               // h, residual, H, iterations, status, Gram products
    unsigned* bar;
    int* err;
};

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

template <int V>
__device__ __forceinline__ void cta_sum(double (&v)[V], double* sm)
{
    cta_sum_f64<V, kMatchThreads>(v, sm);
}

__device__ __forceinline__ unsigned long long cta_max_bits(unsigned long long v, unsigned long long* sm)
{
    constexpr int W = kMatchThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    unsigned long long m = 0;
    for (int w = 0; w < W; ++w) m = sm[w] > m ? sm[w] : m;
    return m;
}

// Row i of Eq. N-particle at the stage input D (FP64): s[0..DIM) = sum_j G_ij p_j,
// s[DIM..2 DIM) = -sum_{j != i} (p_i . p_j) phi_ij (q_i - q_j).  Sources are dealt
// to the threads in order (j -> thread j % 256), so warps run with all lanes
// active: an FP64 warp instruction occupies its sub-partition's FP64 pipe for the
// same time whatever the number of active lanes.  The sums are complete in every
// thread on return.
template <int DIM, int KER>
__device__ void row_sums(const double* D, int n, int i, double sigma, double (&s)[2 * DIM], double* sm)
{
    constexpr int S2 = 2 * DIM;
    double qi[DIM], pi[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        qi[c] = __ldcg(D + (size_t)i * S2 + c);
        pi[c] = __ldcg(D + (size_t)i * S2 + DIM + c);
    }
#pragma unroll
    for (int k = 0; k < S2; ++k) s[k] = 0.0;
    for (int j = threadIdx.x; j < n; j += kMatchThreads) {
        double d[DIM], r2 = 0.0, pp = 0.0, pj[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            d[c] = qi[c] - __ldcg(D + (size_t)j * S2 + c);
            pj[c] = __ldcg(D + (size_t)j * S2 + DIM + c);
            r2 += d[c] * d[c];
            pp += pi[c] * pj[c];
        }
        double G, phi;
        kfun_f64<KER>(r2, sigma, G, phi);
        const double wgt = (j == i) ? 0.0 : -pp * phi;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            s[c] += G * pj[c];
            s[DIM + c] += wgt * d[c];
        }
    }
    cta_sum<S2>(s, sm);
}

// Row i of the Gram product: s = sum_j G(|X_i - X_j|) v_j (Eq. u at t = 0 and at the
// landmarks), from the stored row Gm[i n ..] when the matrix is kept, else with the
// kernel evaluated per pair; complete in every thread on return.
template <int DIM, int KER>
__device__ void gram_row(const double* X, const double* Gm, const double* v, int n, int i, double sigma,
                         double (&s)[DIM], double* sm)
{
    double xi[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        xi[c] = X[(size_t)i * DIM + c];
        s[c] = 0.0;
    }
    for (int j = threadIdx.x; j < n; j += kMatchThreads) {
        double G;
        if (Gm) {
            G = __ldcg(Gm + (size_t)i * n + j);
        } else {
            double r2 = 0.0;
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                const double d = xi[c] - X[(size_t)j * DIM + c];
                r2 += d * d;
            }
            double phi;
            kfun_f64<KER>(r2, sigma, G, phi);
        }
#pragma unroll
        for (int c = 0; c < DIM; ++c) s[c] += G * __ldcg(v + (size_t)j * DIM + c);
    }
    cta_sum<DIM>(s, sm);
}

// Grid-wide sum of V per-CTA values: each CTA writes its partials to slots
// part[k * gridDim.x + cta] (k < V); after the barrier warp 0 of every CTA adds
// them (lane l takes CTAs l, l + 32, ..., then a butterfly over the lanes), the
// same operations in the same order in every CTA, so every CTA holds the same
// bits.  False when a barrier wait gave up.
template <int V>
__device__ bool grid_sum(double (&v)[V], double* part, unsigned* bar, int* err, unsigned& epoch, double* sm)
{
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < V; ++k) part[k * gridDim.x + blockIdx.x] = v[k];
    if (!grid_barrier(bar, err, ++epoch)) return false;
    if (threadIdx.x < 32) {
        const unsigned lane = threadIdx.x;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            double t = 0.0;
            for (unsigned c = lane; c < gridDim.x; c += 32) t += __ldcg(part + k * gridDim.x + c);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) sm[k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = sm[k];
    __syncthreads();
    return true;
}

// MINRES for G(X) delta = r with r = Y - Q(1) (x holds Q(1)); delta in a.Del (own
// rows).  Returns the number of Gram products, or -1 when a barrier wait gave up.
template <int DIM, int KER>
__device__ int minres_gram(const MatchArgs& a, int r0, int r1, double* sm, unsigned& epoch)
{
    const int n = a.n;
    const int e0 = r0 * DIM, e1 = r1 * DIM;
    // beta_1 = |r|, v_1 = r / beta_1; v_0 = w_0 = w_{-1} = delta = 0
    double b1[1] = {0.0};
    for (int e = e0 + (int)threadIdx.x; e < e1; e += kMatchThreads) {
        const double r = a.Y[e] - a.x[e];
        b1[0] += r * r;
    }
    cta_sum<1>(b1, sm);
    if (!grid_sum<1>(b1, a.part + 3 * gridDim.x, a.bar, a.err, epoch, sm)) return -1;
    const double beta1 = sqrt(b1[0]);
    for (int e = e0 + (int)threadIdx.x; e < e1; e += kMatchThreads) {
        a.Del[e] = 0.0;
        a.Vold[e] = 0.0;
        a.W[0][e] = 0.0;
        a.W[1][e] = 0.0;
        a.V[0][e] = beta1 > 0.0 ? (a.Y[e] - a.x[e]) / beta1 : 0.0;
    }
    if (beta1 == 0.0) return 0;
    if (!grid_barrier(a.bar, a.err, ++epoch)) return -1;
    double beta = beta1, eta = beta1;
    double c_old = 1.0, s_old = 0.0, c = 1.0, s = 0.0;
    int cur = 0, it = 0;
    while (it < a.kmax) {
        const double* v = a.V[cur];
        // z = G(X) v - beta v_old; alpha = v . z
        double al[1] = {0.0};
        for (int i = r0; i < r1; ++i) {
            double g[DIM];
            gram_row<DIM, KER>(a.X, a.Gm, v, n, i, a.sigma, g, sm);
            if (threadIdx.x < DIM) {
                const int e = i * DIM + (int)threadIdx.x;
                double gc = g[0];
#pragma unroll
                for (int u = 1; u < DIM; ++u) gc = (int)threadIdx.x == u ? g[u] : gc;
                a.Z[e] = gc - beta * a.Vold[e];
            }
        }
        __syncthreads();
        for (int e = e0 + (int)threadIdx.x; e < e1; e += kMatchThreads) al[0] += __ldcg(v + e) * a.Z[e];
        cta_sum<1>(al, sm);
        if (!grid_sum<1>(al, a.part, a.bar, a.err, epoch, sm)) return -1;
        const double alpha = al[0];
        // z -= alpha v; beta_new = |z|
        double zz[1] = {0.0};
        for (int e = e0 + (int)threadIdx.x; e < e1; e += kMatchThreads) {
            const double z = a.Z[e] - alpha * __ldcg(v + e);
            a.Z[e] = z;
            zz[0] += z * z;
        }
        cta_sum<1>(zz, sm);
        if (!grid_sum<1>(zz, a.part + gridDim.x, a.bar, a.err, epoch, sm)) return -1;
        const double beta_new = sqrt(zz[0]);
        ++it;
        // the previous two rotations applied to the new column (beta, alpha, beta_new) of
        // the Lanczos tridiagonal, then the rotation that annihilates beta_new
        const double eps_k = s_old * beta;
        const double dbar = c_old * beta;
        const double delta = c * dbar + s * alpha;
        const double gbar = -s * dbar + c * alpha;
        const double gamma = sqrt(gbar * gbar + beta_new * beta_new);
        if (gamma == 0.0) break;  // singular Lanczos matrix: keep the current iterate
        const double c_new = gbar / gamma, s_new = beta_new / gamma;
        const double tau = c_new * eta;
        eta = -s_new * eta;
        // w_k = (v_k - delta w_{k-1} - eps w_{k-2}) / gamma; delta += tau w_k;
        // v_{k+1} = z / beta_new (published for the next Gram product)
        double* Wm1 = a.W[it & 1];        // w_{k-1}
        double* Wm2 = a.W[(it & 1) ^ 1];  // w_{k-2}, overwritten by w_k
        double* vn = a.V[cur ^ 1];
        for (int e = e0 + (int)threadIdx.x; e < e1; e += kMatchThreads) {
            const double vk = __ldcg(v + e);
            const double w = (vk - delta * Wm1[e] - eps_k * Wm2[e]) / gamma;
            Wm2[e] = w;
            a.Del[e] += tau * w;
            a.Vold[e] = vk;
            vn[e] = beta_new > 0.0 ? a.Z[e] / beta_new : 0.0;
        }
        c_old = c;
        s_old = s;
        c = c_new;
        s = s_new;
        beta = beta_new;
        cur ^= 1;
        if (fabs(eta) <= a.ktol * beta1 || beta_new == 0.0) break;
        if (!grid_barrier(a.bar, a.err, ++epoch)) return -1;
    }
    return it;
}

template <int DIM, int KER>
__global__ void __launch_bounds__(kMatchThreads) k_match_fp64(MatchArgs a)
{
    constexpr int S2 = 2 * DIM;
    __shared__ double sm_d[(kMatchThreads / 32 + 1) * 8];
    __shared__ unsigned long long sm_u[kMatchThreads / 32];
    const int n = a.n;
    const int r0 = (int)((long long)blockIdx.x * n / gridDim.x), r1 = (int)((long long)(blockIdx.x + 1) * n / gridDim.x);
    const size_t nd = (size_t)n * DIM;
    unsigned epoch = 0;
    // default gain: h = 1 / max_i sum_j G(X_i, X_j)
    double h = a.h;
    if (!(h > 0.0) && a.rule == EP_RULE_VELOCITY) h = 1.0;
    // the velocity rule's G(X) is fixed for the whole matching: store its owned rows once
    if (a.rule == EP_RULE_VELOCITY && a.Gm) {
        for (int i = r0; i < r1; ++i)
            for (int j = threadIdx.x; j < n; j += kMatchThreads) {
                double r2 = 0.0;
#pragma unroll
                for (int c = 0; c < DIM; ++c) {
                    const double d = a.X[(size_t)i * DIM + c] - a.X[(size_t)j * DIM + c];
                    r2 += d * d;
                }
                double G, phi;
                kfun_f64<KER>(r2, a.sigma, G, phi);
                a.Gm[(size_t)i * n + j] = G;
            }
        if (a.piv) {
            // every row of G(X) written, then CTA 0 factors it (symmetric: the row-major
            // rows are the column-major columns); the other CTAs go on to the first shoot
            if (!grid_barrier(a.bar, a.err, ++epoch)) return;
            if (blockIdx.x == 0) {
                __shared__ double s_lv[kMatchThreads / 32 + 1];
                __shared__ int s_li[kMatchThreads / 32 + 1];
                const bool ok = cta_lu_factor<kMatchThreads>(n, a.Gm, a.piv, s_lv, s_li);
                if (threadIdx.x == 0) *a.lu_ok = ok ? 1 : 0;
            }
        }
    }
    if (!(h > 0.0)) {
        // the stage copy D[0] holds (X, 1) for the row sums
        for (int t = threadIdx.x; t < (r1 - r0) * DIM; t += kMatchThreads) {
            const int i = r0 + t / DIM, c = t % DIM;
            a.D[0][(size_t)i * S2 + c] = a.X[(size_t)i * DIM + c];
            a.D[0][(size_t)i * S2 + DIM + c] = 1.0;
        }
        if (!grid_barrier(a.bar, a.err, ++epoch)) return;
        unsigned long long mx = 0;
        for (int i = r0; i < r1; ++i) {
            double s[S2];
            row_sums<DIM, KER>(a.D[0], n, i, a.sigma, s, sm_d);
            const unsigned long long b = dbits(fabs(s[0]));
            mx = b > mx ? b : mx;
        }
        if (threadIdx.x == 0 && r1 > r0) atomicMax(a.red, mx);
        if (!grid_barrier(a.bar, a.err, ++epoch)) return;
        const double m = bitsd(ld_acquire_u64(a.red)) + a.s2;
        h = m > 0.0 ? 1.0 / m : 1.0;
    }
    int k = 0, status = EP_ENOTCONVERGED;
    long long products = 0;
    double res = 0.0;
    for (;; ++k) {
        // shoot from (X, p0): x = (X, p0), step-start copy D[0] = x (own particles)
        for (int t = threadIdx.x; t < (r1 - r0) * DIM; t += kMatchThreads) {
            const int i = r0 + t / DIM, c = t % DIM;
            const double q = a.X[(size_t)i * DIM + c], p = a.p0[(size_t)i * DIM + c];
            a.x[(size_t)i * DIM + c] = q;
            a.x[nd + (size_t)i * DIM + c] = p;
            a.D[0][(size_t)i * S2 + c] = q;
            a.D[0][(size_t)i * S2 + DIM + c] = p;
        }
        if (!grid_barrier(a.bar, a.err, ++epoch)) return;
        for (int s = 0; s < a.steps; ++s) {
            for (int stage = 0; stage < 4; ++stage) {
                const double* Din = a.D[stage == 0 ? 0 : (stage == 2 ? 2 : 1)];
                double* Dout = a.D[stage == 3 ? 0 : (stage == 1 ? 2 : 1)];
                for (int i = r0; i < r1; ++i) {
                    double kk[S2];
                    row_sums<DIM, KER>(Din, n, i, a.sigma, kk, sm_d);
                    // y = x_n + c dt k (c = 1/2, 1/2, 1), acc = k1 + 2 k2 + 2 k3;
                    // x_{n+1} = x_n + dt/6 (acc + k4): one thread per component
                    if (threadIdx.x < S2) {
                        const int c = threadIdx.x;
                        double kv = kk[0];
#pragma unroll
                        for (int u = 1; u < S2; ++u) kv = c == u ? kk[u] : kv;
                        // dq + sigma_n^2 p_i for the inexact system (Sec. 6)
                        if (c < DIM) kv += a.s2 * __ldcg(Din + (size_t)i * S2 + DIM + c);
                        double* xs = c < DIM ? a.x + (size_t)i * DIM + c : a.x + nd + (size_t)i * DIM + (c - DIM);
                        double* A = a.acc + (size_t)i * S2 + c;
                        if (stage < 3) {
                            const double cdt = (stage == 2 ? 1.0 : 0.5) * a.dt;
                            Dout[(size_t)i * S2 + c] = *xs + cdt * kv;
                            *A = stage == 0 ? kv : *A + 2.0 * kv;
                        } else {
                            const double nv = *xs + a.dt / 6.0 * (*A + kv);
                            *xs = nv;
                            Dout[(size_t)i * S2 + c] = nv;
                        }
                    }
                }
                if (!grid_barrier(a.bar, a.err, ++epoch)) return;
            }
        }
        // residual |Y - Q(1)|_inf over all particles and components
        unsigned long long mb = 0;
        for (int t = threadIdx.x; t < (r1 - r0) * DIM; t += kMatchThreads) {
            const size_t e = (size_t)r0 * DIM + t;
            const unsigned long long b = dbits(fabs(a.Y[e] - a.x[e]));
            mb = b > mb ? b : mb;
        }
        mb = cta_max_bits(mb, sm_u);
        if (threadIdx.x == 0 && r1 > r0) atomicMax(a.red + 1 + k, mb);
        if (!grid_barrier(a.bar, a.err, ++epoch)) return;
        const unsigned long long rb = ld_acquire_u64(a.red + 1 + k);
        const bool finite = rb < 0x7FF0000000000000ull;
        res = finite ? bitsd(rb) : __longlong_as_double(0x7FF8000000000000ll);
        if (a.hist && blockIdx.x == 0 && threadIdx.x == 0) a.hist[k] = res;
        if (!finite) { status = EP_EDIVERGED; break; }
        if (a.s2 == 0.0 && res < a.eps) { status = EP_OK; break; }
        if (k == a.maxit) { status = EP_ENOTCONVERGED; break; }
        if (a.rule == EP_RULE_VELOCITY && a.piv && __ldcg(a.lu_ok) == 1) {
            // G(X) delta = r with the factors: CTA 0, one warp, one component at a time
            if (blockIdx.x == 0 && threadIdx.x < 32) {
                for (int c = 0; c < DIM; ++c) {
                    double* bc = a.Z + (size_t)c * n;
                    for (int i = threadIdx.x; i < n; i += 32)
                        bc[i] = __ldcg(a.Y + (size_t)i * DIM + c) - __ldcg(a.x + (size_t)i * DIM + c);
                    __syncwarp();
                    warp_lu_solve(n, a.Gm, a.piv, bc);
                    for (int i = threadIdx.x; i < n; i += 32) a.Del[(size_t)i * DIM + c] = bc[i];
                    __syncwarp();
                }
            }
            products += DIM;
            if (!grid_barrier(a.bar, a.err, ++epoch)) return;
            for (int t = threadIdx.x; t < (r1 - r0) * DIM; t += kMatchThreads) {
                const size_t e = (size_t)r0 * DIM + t;
                a.p0[e] += h * __ldcg(a.Del + e);
            }
            continue;
        }
        if (a.rule == EP_RULE_VELOCITY) {
            const int used = minres_gram<DIM, KER>(a, r0, r1, sm_d, epoch);
            if (used < 0) return;
            products += used;
            for (int t = threadIdx.x; t < (r1 - r0) * DIM; t += kMatchThreads) {
                const size_t e = (size_t)r0 * DIM + t;
                a.p0[e] += h * a.Del[e];
            }
            continue;
        }
        for (int t = threadIdx.x; t < (r1 - r0) * DIM; t += kMatchThreads) {
            const size_t e = (size_t)r0 * DIM + t;
            a.p0[e] += h * (a.Y[e] - a.x[e]);
        }
        // the inexact system (Sec. 6) stops on the change of the momenta, |h (Y - Q(1))|_inf
        if (a.s2 != 0.0 && h * res < a.eps) { ++k; status = EP_OK; break; }
    }
    // H(X, p0) = 1/2 sum_i p_i . sum_j G_ij p_j (Eq. H) of the returned momenta
    for (int t = threadIdx.x; t < (r1 - r0) * DIM; t += kMatchThreads) {
        const int i = r0 + t / DIM, c = t % DIM;
        a.D[0][(size_t)i * S2 + c] = a.X[(size_t)i * DIM + c];
        a.D[0][(size_t)i * S2 + DIM + c] = a.p0[(size_t)i * DIM + c];
    }
    if (!grid_barrier(a.bar, a.err, ++epoch)) return;
    double hp = 0.0;
    for (int i = r0; i < r1; ++i) {
        double s[S2];
        row_sums<DIM, KER>(a.D[0], n, i, a.sigma, s, sm_d);
        double dot = 0.0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) dot += a.p0[(size_t)i * DIM + c] * s[c];
        hp += 0.5 * dot;
    }
    if (threadIdx.x == 0) a.part[blockIdx.x] = hp;
    if (!grid_barrier(a.bar, a.err, ++epoch)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double H = 0.0;
        for (unsigned c = 0; c < gridDim.x; ++c) H += __ldcg(a.part + c);
        a.out[0] = h;
        a.out[1] = res;
        a.out[2] = H;
        a.out[3] = (double)k;
        a.out[4] = (double)status;
        a.out[5] = (double)products;
    }
}

template <int DIM, int KER>
ep_status launch_match_fp64(MatchArgs& a, cudaStream_t st)
{
    auto fn = k_match_fp64<DIM, KER>;
    static int resident = -1;
    if (resident < 0) {
        int per_sm = 0;
        EP_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMatchThreads, 0));
        DeviceInfo di{};
        EP_TRY(device_info(&di));
        resident = per_sm * di.sm_count;
    }
    DeviceInfo di{};
    EP_TRY(device_info(&di));
    // at most 256 CTAs: the per-CTA partial sums use 4 slots of a 1024-double buffer
    const int G = std::max(1, std::min({a.n, di.sm_count, resident, 256}));
    void* args[] = {&a};
    count_launch();
    EP_TRY_CUDA(cudaLaunchCooperativeKernel((void*)fn, dim3(G), dim3(kMatchThreads), args, 0, st));
    return EP_OK;
}

}  // namespace

// the velocity rule keeps G(X) in memory up to this many landmarks (n^2 doubles, 512 MB)
constexpr int64_t kGramStoreMaxN = 8192;

size_t match_device_bytes(int64_t n, int dim, int maxit, int rule)
{
    Sizer z;
    const size_t m = (size_t)n * dim;
    z.add(sizeof(double) * 2 * m);          // x
    for (int k = 0; k < 3; ++k) z.add(sizeof(double) * 2 * m);  // stage copies
    z.add(sizeof(double) * 2 * m);          // acc
    z.add(sizeof(unsigned long long) * ((size_t)maxit + 2));
    z.add(sizeof(double) * 1024);           // per-CTA partials
    for (int k = 0; k < 7; ++k) z.add(sizeof(double) * m);  // MINRES vectors
    if (rule == EP_RULE_VELOCITY && n <= kGramStoreMaxN) z.add(sizeof(double) * (size_t)n * n);  // G(X)
    if (rule == EP_RULE_VELOCITY && n <= kGramLuMaxN) {
        z.add(sizeof(int) * (size_t)n);  // pivots
        z.add(sizeof(int) * 4);          // factorisation flag
    }
    z.add(sizeof(double) * 8);              // outputs
    z.add(sizeof(unsigned) * 12);           // barrier + error flag
    return z.total;
}

ep_status match_device_fp64(const ep_params& P, int64_t n, const double* X, const double* Y, double* p0,
                            ep_match_info* info, double* hist_dev, Arena* ar, cudaStream_t st, double out[6])
{
    const size_t m = (size_t)n * P.dim;
    MatchArgs a{};
    a.n = (int)n;
    a.steps = P.steps;
    a.maxit = info->maxit;
    a.sigma = P.sigma;
    a.dt = P.t1 / P.steps;
    a.eps = info->eps;
    a.h = info->h;
    a.s2 = P.inexact;
    a.X = X;
    a.Y = Y;
    a.p0 = p0;
    a.x = (double*)ar->carve(sizeof(double) * 2 * m);
    for (int k = 0; k < 3; ++k) a.D[k] = (double*)ar->carve(sizeof(double) * 2 * m);
    a.acc = (double*)ar->carve(sizeof(double) * 2 * m);
    a.red = (unsigned long long*)ar->carve(sizeof(unsigned long long) * ((size_t)a.maxit + 2));
    a.part = (double*)ar->carve(sizeof(double) * 1024);
    a.rule = info->rule;
    {
        const int N = (int)std::min<size_t>(m, (size_t)1 << 28);
        const int krylov = info->krylov > 0 ? std::min(info->krylov, N) : std::min(N, 200);
        a.kmax = 4 * krylov;
        a.ktol = 1e-12;
    }
    for (int k = 0; k < 2; ++k) a.V[k] = (double*)ar->carve(sizeof(double) * m);
    for (int k = 0; k < 2; ++k) a.W[k] = (double*)ar->carve(sizeof(double) * m);
    a.Vold = (double*)ar->carve(sizeof(double) * m);
    a.Z = (double*)ar->carve(sizeof(double) * m);
    a.Del = (double*)ar->carve(sizeof(double) * m);
    a.Gm = a.rule == EP_RULE_VELOCITY && n <= kGramStoreMaxN ? (double*)ar->carve(sizeof(double) * (size_t)n * n)
                                                               : nullptr;
    if (a.Gm && n <= kGramLuMaxN) {
        a.piv = (int*)ar->carve(sizeof(int) * (size_t)n);
        a.lu_ok = (int*)ar->carve(sizeof(int) * 4);
        if (!a.lu_ok) return set_error("ep_match: workspace too small"), EP_ENOMEM;
        EP_TRY_CUDA(cudaMemsetAsync(a.lu_ok, 0, sizeof(int) * 4, st));
    }
    a.out = (double*)ar->carve(sizeof(double) * 8);
    a.bar = (unsigned*)ar->carve(sizeof(unsigned) * 12);
    if (!a.bar) return set_error("ep_match: workspace too small"), EP_ENOMEM;
    a.err = (int*)(a.bar + 8);
    a.hist = hist_dev;
    EP_TRY_CUDA(cudaMemsetAsync(a.red, 0, sizeof(unsigned long long) * ((size_t)a.maxit + 2), st));
    EP_TRY_CUDA(cudaMemsetAsync(a.bar, 0, sizeof(unsigned) * 12, st));
    ep_status s = EP_EINVAL;
#define EP_MATCH_CASE(D, K) \
    if (P.dim == D && P.kernel == K) s = launch_match_fp64<D, K>(a, st);
    EP_MATCH_CASE(2, EP_GAUSS) EP_MATCH_CASE(2, EP_TENT) EP_MATCH_CASE(2, EP_EXPCONE)
    EP_MATCH_CASE(3, EP_GAUSS) EP_MATCH_CASE(3, EP_TENT) EP_MATCH_CASE(3, EP_EXPCONE)
#undef EP_MATCH_CASE
    if (s != EP_OK) return s == EP_EINVAL ? (set_error("ep_match: no device match for this kernel"), s) : s;
    int herr = 0;
    EP_TRY_CUDA(cudaMemcpyAsync(out, a.out, sizeof(double) * 6, cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaMemcpyAsync(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    if (herr) return set_error("ep_match: a grid-barrier wait gave up (kernel ended early)"), EP_ETIMEOUT;
    return EP_OK;
}

}  // namespace ep
