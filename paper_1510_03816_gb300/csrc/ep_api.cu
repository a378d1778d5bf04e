// ep_api.cu -- C ABI of libep.so: argument checks, host/device staging,
// workspace arenas and the host side of Algorithm 1 (Sec. 4 of the paper).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "ep_allpairs.cuh"
#include "ep_common.cuh"
#include "ep_features.cuh"

namespace ep {

// ------------------------------------------------------------------ launch counter
static std::atomic<long long> g_launches{0};

void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

ep_status cuda_fail(cudaError_t e, const char* what)
{
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return EP_ECUDA;
}

ep_status device_info(DeviceInfo* out)
{
    static std::mutex mu;
    static std::map<int, DeviceInfo> cache;
    int dev = 0;
    EP_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) {
        *out = it->second;
        return EP_OK;
    }
    DeviceInfo d{};
    d.device = dev;
    EP_TRY_CUDA(cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev));
    EP_TRY_CUDA(cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    EP_TRY_CUDA(cudaDeviceGetAttribute(&d.cc_major, cudaDevAttrComputeCapabilityMajor, dev));
    EP_TRY_CUDA(cudaDeviceGetAttribute(&d.cc_minor, cudaDevAttrComputeCapabilityMinor, dev));
    cache[dev] = d;
    *out = d;
    return EP_OK;
}

// ------------------------------------------------------------------ workspace
static std::mutex g_arena_mu;
static std::map<std::pair<int, cudaStream_t>, Arena> g_arenas;

ep_status arena_acquire(cudaStream_t stream, size_t bytes, Arena** out)
{
    int dev = 0;
    EP_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_arena_mu);
    Arena& a = g_arenas[{dev, stream}];
    if (a.cap < bytes) {
        if (a.base) {
            EP_TRY_CUDA(cudaStreamSynchronize(stream));
            EP_TRY_CUDA(cudaFree(a.base));
            a.base = nullptr;
            a.cap = 0;
        }
        const size_t want = std::max<size_t>(bytes + bytes / 4, 1 << 20);
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc of %zu bytes failed: %s", want, cudaGetErrorString(e));
            return EP_ENOMEM;
        }
        a.base = (char*)p;
        a.cap = want;
    }
    a.used = 0;
    *out = &a;
    return EP_OK;
}

ep_status release_all_arenas()
{
    std::lock_guard<std::mutex> lk(g_arena_mu);
    EP_TRY_CUDA(cudaDeviceSynchronize());
    for (auto& kv : g_arenas)
        if (kv.second.base) cudaFree(kv.second.base);
    g_arenas.clear();
    return EP_OK;
}

ep_status check_params(const ep_params* p)
{
    if (!p) return set_error("params is NULL"), EP_EINVAL;
    if (p->dim != 2 && p->dim != 3) return set_error("dim must be 2 or 3 (got %d)", p->dim), EP_EINVAL;
    if (p->kernel < EP_GAUSS || p->kernel > EP_EXPCONE)
        return set_error("unknown kernel %d", p->kernel), EP_EINVAL;
    if (!(p->sigma > 0.0) || !isfinite(p->sigma)) return set_error("sigma must be > 0"), EP_EINVAL;
    if (p->steps < 1) return set_error("steps must be >= 1 (got %d)", p->steps), EP_EINVAL;
    if (!isfinite(p->t1)) return set_error("t1 must be finite"), EP_EINVAL;
    if (p->precision != EP_FP64 && p->precision != EP_MIXED)
        return set_error("unknown precision %d", p->precision), EP_EINVAL;
    if (p->neigh < EP_AUTO || p->neigh > EP_CELLLIST) return set_error("unknown neigh %d", p->neigh), EP_EINVAL;
    if (p->neigh == EP_CELLLIST && p->kernel != EP_TENT)
        return set_error("the cell list needs the compactly supported tent kernel"), EP_EINVAL;
    if (!(p->inexact >= 0.0) || !isfinite(p->inexact))
        return set_error("inexact (sigma_n^2) must be finite and >= 0"), EP_EINVAL;
    if (p->inexact != 0.0 && p->neigh == EP_CELLLIST)
        return set_error("the inexact system runs on the all-pairs path"), EP_EINVAL;
    return EP_OK;
}

static ep_status check_n(int64_t n)
{
    if (n < 0) return set_error("n must be >= 0"), EP_EINVAL;
    if (n > (int64_t)1 << 26) return set_error("n = %lld exceeds the supported 2^26", (long long)n), EP_EINVAL;
    return EP_OK;
}

// A caller array on the device, staged through the arena when it is host memory.
struct Staged {
    const void* user = nullptr;
    double* dev = nullptr;
    size_t count = 0;
    bool host = false;
};

static bool is_device_ptr(const void* p)
{
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static void plan_stage(Sizer& z, const void* p, size_t count)
{
    if (p && !is_device_ptr(p)) z.add(sizeof(double) * count);
}

static ep_status stage_in(Arena* ar, const double* p, size_t count, cudaStream_t st, Staged* s)
{
    s->user = p;
    s->count = count;
    s->host = !is_device_ptr(p);
    if (!s->host) {
        s->dev = const_cast<double*>(p);
        return EP_OK;
    }
    s->dev = (double*)ar->carve(sizeof(double) * count);
    if (!s->dev) return set_error("workspace too small for staging"), EP_ENOMEM;
    if (count) EP_TRY_CUDA(cudaMemcpyAsync(s->dev, p, sizeof(double) * count, cudaMemcpyHostToDevice, st));
    return EP_OK;
}

static ep_status stage_out_alloc(Arena* ar, double* p, size_t count, Staged* s)
{
    s->user = p;
    s->count = count;
    s->host = !is_device_ptr(p);
    if (!s->host) {
        s->dev = p;
        return EP_OK;
    }
    s->dev = (double*)ar->carve(sizeof(double) * count);
    if (!s->dev) return set_error("workspace too small for staging"), EP_ENOMEM;
    return EP_OK;
}

static ep_status stage_out_finish(const Staged& s, cudaStream_t st)
{
    if (s.host && s.count)
        EP_TRY_CUDA(cudaMemcpyAsync(const_cast<void*>(s.user), s.dev, sizeof(double) * s.count,
                                    cudaMemcpyDeviceToHost, st));
    return EP_OK;
}

// ------------------------------------------------------------------ small FP64 kernels
// Deterministic single-CTA reductions (fixed order per thread, fixed tree).
__global__ void k_max_abs_diff(const double* __restrict__ Y, const double* __restrict__ Q, size_t m,
                               double* out /* [0] = max |Y - Q|, [1] = 1 if non-finite */)
{
    __shared__ double sm[32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    double mx = 0.0;
    int bad = 0;
    for (size_t a = threadIdx.x; a < m; a += blockDim.x) {
        const double r = Y[a] - Q[a];
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
        out[0] = t;
        out[1] = sbad ? 1.0 : 0.0;
    }
}

// p += h (Y - Q)   (Algorithm 1 steps 3-4 with M = h I on the momenta)
__global__ void k_momentum_update(double* __restrict__ p, const double* __restrict__ Y,
                                  const double* __restrict__ Q, size_t m, double h)
{
    const size_t a = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (a < m) p[a] = fma(h, Y[a] - Q[a], p[a]);
}

__global__ void k_half_dot(const double* __restrict__ p, const double* __restrict__ dq, size_t m,
                           double* out)
{
    __shared__ double sm[32];
    double s = 0.0;
    for (size_t a = threadIdx.x; a < m; a += blockDim.x) s = fma(p[a], dq[a], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sm[k];
        *out = 0.5 * t;
    }
}

// out = max_i v[i*dim] (first component), for the default gain
__global__ void k_max_first(const double* __restrict__ v, int n, int dim, double* out)
{
    __shared__ double sm[32];
    double mx = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(v[(size_t)i * dim]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = fmax(t, sm[k]);
        *out = t;
    }
}

__global__ void k_fill_unit_x(double* v, int n, int dim)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        for (int c = 0; c < dim; ++c) v[(size_t)i * dim + c] = c == 0 ? 1.0 : 0.0;
}

// ------------------------------------------------------------------ path selection
bool use_celllist(const ep_params& P, int64_t n)
{
    if (P.kernel != EP_TENT) return false;
    if (P.neigh == EP_CELLLIST) return true;
    if (P.neigh == EP_ALLPAIRS) return false;
    // EP_AUTO: the cell list (2-D, mixed precision) for large tent problems of the exact system
    return P.dim == 2 && P.precision == EP_MIXED && P.inexact == 0.0 && n >= 16384;
}

// Problem state of one forward pass, whichever neighbour path it uses.
struct Forward {
    bool cells = false;
    AllPairsBufs ap;
    CellBufs cl;
};

static size_t forward_bytes(const ep_params& P, int64_t n)
{
    return use_celllist(P, n) ? cell_bytes((int)n, P.dim, P.precision)
                              : allpairs_bytes((int)n, P.dim, P.precision);
}

static ep_status forward_carve(Arena* ar, const ep_params& P, int64_t n, Forward* f)
{
    f->cells = use_celllist(P, n);
    if (f->cells) return cell_carve(ar, (int)n, P.dim, P.precision, &f->cl);
    return allpairs_carve(ar, (int)n, P.dim, P.precision, &f->ap);
}

static ep_status forward_load(const ep_params& P, Forward& f, const double* q, const double* p,
                              cudaStream_t st)
{
    return f.cells ? cell_load(P, f.cl, q, p, st) : allpairs_load(P, f.ap, q, p, st);
}

static ep_status forward_rhs(const ep_params& P, const Forward& f, double* dq, double* dp, cudaStream_t st)
{
    return f.cells ? cell_rhs(P, f.cl, dq, dp, st) : allpairs_rhs(P, f.ap, dq, dp, st);
}

static ep_status forward_steps(const ep_params& P, const Forward& f, int steps, double dt, cudaStream_t st)
{
    return f.cells ? cell_steps(P, f.cl, steps, dt, st) : allpairs_steps(P, f.ap, steps, dt, st);
}

static double* forward_state(const Forward& f) { return f.cells ? f.cl.x : f.ap.x; }

// Default gain h = 1 / max_i sum_j G(|X_i - X_j|) (Gershgorin bound on the largest
// eigenvalue of G(X); all three kernels are non-negative so |G| = G).  Computed with
// the right-hand side at unit momenta (1, 0[, 0]): dq_i,x = sum_j G_ij.
static ep_status default_gain(const ep_params& P, Forward& f, int64_t n, const double* X, double* unit,
                              double* dq, double* dp, double* scal, cudaStream_t st, double* h_out)
{
    count_launch();
    k_fill_unit_x<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(unit, (int)n, P.dim);
    EP_TRY(forward_load(P, f, X, unit, st));
    EP_TRY(forward_rhs(P, f, dq, dp, st));
    count_launch();
    k_max_first<<<1, 1024, 0, st>>>(dq, (int)n, P.dim, scal);
    double mx = 0.0;
    EP_TRY_CUDA(cudaMemcpyAsync(&mx, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    *h_out = mx > 0.0 ? 1.0 / mx : 1.0;
    return EP_OK;
}

}  // namespace ep

using namespace ep;

static cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

extern "C" {

int ep_version(void) { return 10000; }

int64_t ep_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

void ep_set_launch_timing(int on) { set_launch_timing(on != 0); }

double ep_last_launch_ms(void) { return last_launch_ms(); }

const char* ep_last_launch_kernel(void) { return last_launch_kernel(); }

const char* ep_last_error(void) { return g_err; }

ep_status ep_release_workspace(void) { return release_all_arenas(); }

ep_status ep_velocity(const ep_params* params, int64_t n, const double* q, const double* p, int64_t m,
                      const double* x, double* u, void* stream)
{
    return velocity_entry(params, n, q, p, m, x, u, stream);
}

ep_status ep_flow(const ep_params* params, int64_t n, const double* q0, const double* p0, int64_t m,
                  const double* x0, double* x1, void* stream)
{
    return flow_entry(params, n, q0, p0, m, x0, x1, stream);
}

ep_status ep_rhs(const ep_params* params, int64_t n, const double* q, const double* p, double* dq,
                 double* dp, void* stream)
{
    EP_TRY(check_params(params));
    EP_TRY(check_n(n));
    if (n == 0) return EP_OK;
    if (!q || !p || !dq || !dp) return set_error("ep_rhs: NULL array"), EP_EINVAL;
    const ep_params& P = *params;
    cudaStream_t st = as_stream(stream);
    const size_t m = (size_t)n * P.dim;
    Sizer z;
    z.add(forward_bytes(P, n));
    plan_stage(z, q, m);
    plan_stage(z, p, m);
    plan_stage(z, dq, m);
    plan_stage(z, dp, m);
    Arena* ar = nullptr;
    EP_TRY(arena_acquire(st, z.total, &ar));
    Forward f;
    EP_TRY(forward_carve(ar, P, n, &f));
    Staged sq, sp, sdq, sdp;
    EP_TRY(stage_in(ar, q, m, st, &sq));
    EP_TRY(stage_in(ar, p, m, st, &sp));
    EP_TRY(stage_out_alloc(ar, dq, m, &sdq));
    EP_TRY(stage_out_alloc(ar, dp, m, &sdp));
    EP_TRY(forward_load(P, f, sq.dev, sp.dev, st));
    EP_TRY(forward_rhs(P, f, sdq.dev, sdp.dev, st));
    EP_TRY(stage_out_finish(sdq, st));
    EP_TRY(stage_out_finish(sdp, st));
    if (sq.host || sp.host || sdq.host || sdp.host) EP_TRY_CUDA(cudaStreamSynchronize(st));
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

ep_status ep_shoot(const ep_params* params, int64_t n, const double* q0, const double* p0, double* q1,
                   double* p1, void* stream)
{
    EP_TRY(check_params(params));
    EP_TRY(check_n(n));
    if (n == 0) return EP_OK;
    if (!q0 || !p0 || !q1 || !p1) return set_error("ep_shoot: NULL array"), EP_EINVAL;
    const ep_params& P = *params;
    cudaStream_t st = as_stream(stream);
    const size_t m = (size_t)n * P.dim;
    Sizer z;
    z.add(forward_bytes(P, n));
    plan_stage(z, q0, m);
    plan_stage(z, p0, m);
    plan_stage(z, q1, m);
    plan_stage(z, p1, m);
    Arena* ar = nullptr;
    EP_TRY(arena_acquire(st, z.total, &ar));
    Forward f;
    EP_TRY(forward_carve(ar, P, n, &f));
    Staged sq, sp, sq1, sp1;
    EP_TRY(stage_in(ar, q0, m, st, &sq));
    EP_TRY(stage_in(ar, p0, m, st, &sp));
    EP_TRY(stage_out_alloc(ar, q1, m, &sq1));
    EP_TRY(stage_out_alloc(ar, p1, m, &sp1));
    EP_TRY(forward_load(P, f, sq.dev, sp.dev, st));
    EP_TRY(forward_steps(P, f, P.steps, P.t1 / P.steps, st));
    double* x = forward_state(f);
    EP_TRY_CUDA(cudaMemcpyAsync(sq1.dev, x, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
    EP_TRY_CUDA(cudaMemcpyAsync(sp1.dev, x + m, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
    EP_TRY(stage_out_finish(sq1, st));
    EP_TRY(stage_out_finish(sp1, st));
    if (sq.host || sp.host || sq1.host || sp1.host) EP_TRY_CUDA(cudaStreamSynchronize(st));
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

ep_status ep_hamiltonian(const ep_params* params, int64_t n, const double* q, const double* p, double* H_out,
                         void* stream)
{
    EP_TRY(check_params(params));
    EP_TRY(check_n(n));
    if (!H_out) return set_error("ep_hamiltonian: NULL H_out"), EP_EINVAL;
    const ep_params& P = *params;
    cudaStream_t st = as_stream(stream);
    const bool hout_dev = is_device_ptr(H_out);
    if (n == 0) {
        const double zero = 0.0;
        if (hout_dev) EP_TRY_CUDA(cudaMemcpyAsync(H_out, &zero, sizeof zero, cudaMemcpyHostToDevice, st));
        else *H_out = 0.0;
        return EP_OK;
    }
    if (!q || !p) return set_error("ep_hamiltonian: NULL array"), EP_EINVAL;
    const size_t m = (size_t)n * P.dim;
    Sizer z;
    z.add(forward_bytes(P, n));
    plan_stage(z, q, m);
    plan_stage(z, p, m);
    z.add(sizeof(double) * 2 * m);
    z.add(64);
    Arena* ar = nullptr;
    EP_TRY(arena_acquire(st, z.total, &ar));
    Forward f;
    EP_TRY(forward_carve(ar, P, n, &f));
    Staged sq, sp;
    EP_TRY(stage_in(ar, q, m, st, &sq));
    EP_TRY(stage_in(ar, p, m, st, &sp));
    double* dq = (double*)ar->carve(sizeof(double) * m);
    double* dp = (double*)ar->carve(sizeof(double) * m);
    double* scal = (double*)ar->carve(64);
    EP_TRY(forward_load(P, f, sq.dev, sp.dev, st));
    EP_TRY(forward_rhs(P, f, dq, dp, st));
    count_launch();
    k_half_dot<<<1, 1024, 0, st>>>(sp.dev, dq, m, hout_dev ? H_out : scal);
    if (!hout_dev) {
        EP_TRY_CUDA(cudaMemcpyAsync(H_out, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
        EP_TRY_CUDA(cudaStreamSynchronize(st));
    } else if (sq.host || sp.host) {
        EP_TRY_CUDA(cudaStreamSynchronize(st));
    }
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}

static ep_status match_entry(const ep_params* params, int64_t n, const double* X, const double* Y, double* p0,
                             ep_match_info* info, void* stream)
{
    EP_TRY(check_params(params));
    EP_TRY(check_n(n));
    if (!info) return set_error("ep_match: NULL info"), EP_EINVAL;
    if (info->maxit < 0) return set_error("ep_match: maxit must be >= 0"), EP_EINVAL;
    if (!(info->eps >= 0.0)) return set_error("ep_match: eps must be >= 0"), EP_EINVAL;
    if (n > 0 && (!X || !Y || !p0)) return set_error("ep_match: NULL array"), EP_EINVAL;
    const ep_params& P = *params;
    cudaStream_t st = as_stream(stream);
    const size_t m = (size_t)n * P.dim;
    if (info->rule < EP_RULE_MOMENTUM || info->rule > EP_RULE_NEWTON)
        return set_error("ep_match: unknown update rule %d", info->rule), EP_EINVAL;
    info->iters = 0;
    info->resid_inf = 0.0;
    info->H = 0.0;
    info->products = 0;
    if (n == 0) {
        if (info->h <= 0.0) info->h = 1.0;
        return EP_OK;
    }
    // the plain FP64 all-pairs method runs the whole feedback loop on the device, with
    // the momentum rule or the velocity rule (G(X) factored in the launch, or MINRES)
    const bool device_loop = P.precision == EP_FP64 && !use_celllist(P, n) &&
                             ((info->rule == EP_RULE_MOMENTUM && n <= kDeviceMatchMaxN) ||
                              (info->rule == EP_RULE_VELOCITY && P.inexact == 0.0));
    // the velocity update in mixed precision: mixed shoots, G(X) factored once in FP64
    if (info->rule == EP_RULE_VELOCITY && P.precision == EP_MIXED) return velocity_mixed_match(P, n, X, Y, p0, info, st);
    if (info->rule == EP_RULE_VELOCITY && !device_loop)
        return set_error("ep_match: the velocity update runs on the all-pairs path of the exact system"), EP_EINVAL;
    // the Newton gain: the whole Jacobian and a dense solve for small problems, host
    // GMRES over tangent-linear shoots beyond (ep_newton.cu)
    if (info->rule == EP_RULE_NEWTON) return rule_match(P, n, X, Y, p0, info, st);
    // small 2-D mixed problems: the whole feedback loop on one CTA (no grid-wide sync per stage)
    if (P.precision == EP_MIXED && P.dim == 2 && !use_celllist(P, n) && n <= kSmallMatchMaxN && P.inexact == 0.0) {
        ep_status s = match_small(params, n, X, Y, p0, info, stream);
        if (s == EP_ENOTCONVERGED)
            set_error("ep_match: %d iterations, residual %.3e >= eps %.3e", info->iters, info->resid_inf, info->eps);
        if (s == EP_EDIVERGED) set_error("ep_match: residual became non-finite after %d updates", info->iters);
        return s;
    }
    const bool hist_dev = info->hist && is_device_ptr(info->hist);
    Sizer z;
    if (device_loop) z.add(match_device_bytes(n, P.dim, info->maxit, info->rule));
    else z.add(owner_match_bytes());
    z.add(sizeof(double) * ((size_t)info->maxit + 1));
    z.add(forward_bytes(P, n));
    plan_stage(z, X, m);
    plan_stage(z, Y, m);
    plan_stage(z, p0, m);
    for (int k = 0; k < 3; ++k) z.add(sizeof(double) * m);  // t0, t1, t2 (each carve is aligned)
    z.add(64);
    Arena* ar = nullptr;
    EP_TRY(arena_acquire(st, z.total, &ar));
    Forward f;
    EP_TRY(forward_carve(ar, P, n, &f));
    Staged sX, sY, sp;
    EP_TRY(stage_in(ar, X, m, st, &sX));
    EP_TRY(stage_in(ar, Y, m, st, &sY));
    EP_TRY(stage_in(ar, p0, m, st, &sp));
    if (device_loop) {
        double* hist_d = hist_dev ? info->hist : nullptr;
        if (info->hist && !hist_dev) hist_d = (double*)ar->carve(sizeof(double) * ((size_t)info->maxit + 1));
        double out[6];
        EP_TRY(match_device_fp64(P, n, sX.dev, sY.dev, sp.dev, info, hist_d, ar, st, out));
        info->products = (int)out[5];
        info->h = out[0];
        info->resid_inf = out[1];
        info->H = out[2];
        info->iters = (int)out[3];
        const ep_status status = (ep_status)(int)out[4];
        if (sp.host) EP_TRY_CUDA(cudaMemcpyAsync(p0, sp.dev, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
        if (info->hist && !hist_dev)
            EP_TRY_CUDA(cudaMemcpyAsync(info->hist, hist_d, sizeof(double) * ((size_t)info->iters + 1),
                                        cudaMemcpyDeviceToHost, st));
        EP_TRY_CUDA(cudaStreamSynchronize(st));
        if (status == EP_ENOTCONVERGED)
            set_error("ep_match: %d iterations, residual %.3e >= eps %.3e", info->iters, info->resid_inf, info->eps);
        if (status == EP_EDIVERGED) set_error("ep_match: residual became non-finite after %d updates", info->iters);
        return status;
    }
    double* t0 = (double*)ar->carve(sizeof(double) * m);
    double* t1 = (double*)ar->carve(sizeof(double) * m);
    double* t2 = (double*)ar->carve(sizeof(double) * m);
    double* scal = (double*)ar->carve(64);
    double h = info->h;
    if (!(h > 0.0)) EP_TRY(default_gain(P, f, n, sX.dev, t0, t1, t2, scal, st, &h));
    info->h = h;
    const double dt = P.t1 / P.steps;
    double* Q1 = forward_state(f);
    ep_status status = EP_ENOTCONVERGED;
    int k = 0;
    double res = 0.0;
    double host_res[2];
    // the owner-computes 2-D Gaussian shoot runs the whole loop in one launch
    bool on_device = false;
    if (!f.cells) {
        double* hist_d = hist_dev ? info->hist : nullptr;
        if (info->hist && !hist_dev) hist_d = (double*)ar->carve(sizeof(double) * ((size_t)info->maxit + 1));
        double* scratch = (double*)ar->carve(owner_match_bytes());
        if (!scratch || (info->hist && !hist_d)) return set_error("ep_match: workspace plan too small"), EP_ENOMEM;
        double out[3];
        EP_TRY(owner_match(P, f.ap, sX.dev, sY.dev, sp.dev, info->maxit, info->eps, h, hist_d, scratch, st,
                           &on_device, out));
        if (on_device) {
            res = out[0];
            k = (int)out[1];
            status = (ep_status)(int)out[2];
            // shoots: k + 1, except the inexact system's stop after an update
            const int shoots = (P.inexact != 0.0 && status == EP_OK) ? k : k + 1;
            if (info->hist && !hist_dev)
                EP_TRY_CUDA(cudaMemcpyAsync(info->hist, hist_d, sizeof(double) * (size_t)shoots,
                                            cudaMemcpyDeviceToHost, st));
        }
    }
    while (!on_device) {
        EP_TRY(forward_load(P, f, sX.dev, sp.dev, st));
        EP_TRY(forward_steps(P, f, P.steps, dt, st));
        count_launch();
        k_max_abs_diff<<<1, 1024, 0, st>>>(sY.dev, Q1, m, scal);
        EP_TRY_CUDA(cudaMemcpyAsync(host_res, scal, sizeof host_res, cudaMemcpyDeviceToHost, st));
        EP_TRY_CUDA(cudaStreamSynchronize(st));
        const bool finite = host_res[1] == 0.0;
        res = finite ? host_res[0] : NAN;
        if (info->hist) {
            if (hist_dev) EP_TRY_CUDA(cudaMemcpyAsync(info->hist + k, &res, sizeof(double), cudaMemcpyHostToDevice, st));
            else info->hist[k] = res;
        }
        if (!finite) { status = EP_EDIVERGED; break; }
        if (P.inexact == 0.0 && res < info->eps) { status = EP_OK; break; }
        if (k == info->maxit) { status = EP_ENOTCONVERGED; break; }
        count_launch();
        k_momentum_update<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(sp.dev, sY.dev, Q1, m, h);
        ++k;
        // the inexact system (Sec. 6) stops on the change of the momenta: |h (Y - Q(1))|_inf
        if (P.inexact != 0.0 && h * res < info->eps) { status = EP_OK; break; }
    }
    info->iters = k;
    info->resid_inf = res;
    // H(X, p0) of the returned momenta (Eq. H)
    EP_TRY(forward_load(P, f, sX.dev, sp.dev, st));
    EP_TRY(forward_rhs(P, f, t0, t1, st));
    count_launch();
    k_half_dot<<<1, 1024, 0, st>>>(sp.dev, t0, m, scal);
    EP_TRY_CUDA(cudaMemcpyAsync(&info->H, scal, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (sp.host) EP_TRY_CUDA(cudaMemcpyAsync(p0, sp.dev, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    EP_TRY_CUDA(cudaStreamSynchronize(st));
    EP_TRY_CUDA(cudaGetLastError());
    if (status == EP_ENOTCONVERGED) set_error("ep_match: %d iterations, residual %.3e >= eps %.3e", k, res, info->eps);
    if (status == EP_EDIVERGED) set_error("ep_match: residual became non-finite after %d updates", k);
    return status;
}

ep_status ep_shoot_tangent(const ep_params* params, int64_t n, const double* q0, const double* p0,
                           const double* vq0, const double* vp0, double* q1, double* p1, double* vq1, double* vp1,
                           void* stream)
{
    return tangent_entry(params, n, q0, p0, vq0, vp0, q1, p1, vq1, vp1, as_stream(stream));
}

ep_status ep_hvp(const ep_params* params, int64_t n, const double* q, const double* p, const double* vq,
                 const double* vp, double* hq, double* hp, void* stream)
{
    return hvp_entry(params, n, q, p, vq, vp, hq, hp, stream);
}

ep_status ep_adjoint(const ep_params* params, int64_t n, const double* X, const double* p0, const double* Y,
                     double lambda, int ckpt_every, double* grad_p0, double* energy, void* stream)
{
    return adjoint_entry(params, n, X, p0, Y, lambda, ckpt_every, grad_p0, energy, stream);
}

ep_status ep_match(const ep_params* params, int64_t n, const double* X, const double* Y, double* p0,
                   ep_match_info* info, void* stream)
{
    const ep_status s = match_entry(params, n, X, Y, p0, info, stream);
    if (info) info->status = (int)s;
    return s;
}

ep_status ep_match_batched(const ep_params* params, int nprob, const int64_t* offsets, const double* X,
                           const double* Y, double* p0, ep_match_info* infos, void* stream)
{
    return batched_entry(params, nprob, offsets, X, Y, p0, infos, stream);
}

ep_status ep_cell_neighbors(const ep_params* params, int64_t n, const double* q, int64_t* count,
                            uint64_t* hash, int64_t* total, void* stream)
{
    return cell_neighbors_entry(params, n, q, count, hash, total, stream);
}

}  // extern "C"
