// ep_common.cuh -- shared host/device definitions of libep.so (GB300, sm_103a).
//
// Scaled coordinates.  The FP32 pair kernels work on positions multiplied by a
// per-kernel scale s so that the kernel becomes a bare hardware function of the
// scaled distance r' = s r (Sec. 3 kernels; the factors fold back in below):
//   EP_GAUSS   s = sqrt(log2(e) / (2 sigma^2)):  G = ex2(-r'^2),   w = G
//   EP_TENT    s = 1 / sigma:                    G = 1 - r',       w = 1/r'  (r' < 1)
//   EP_EXPCONE s = log2(e) / sigma:              G = ex2(-r'),     w = G/r'
// and with d' = s (q_i - q_j) the momentum sum of Eq. N-particle is
//   dp_i = dp_scale * sum_j w_ij (p_i . p_j) d'_ij,
//   dp_scale = 1/(s sigma^2) (Gaussian), 1/sigma (tent, expcone).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ep.h"

namespace ep {

constexpr int kTileI = 64;     // particles i per tile: 32 lanes x 2 registers
constexpr int kKWidth = 6;     // FP64 words per particle in the k accumulator

struct KernelScale {
    double s;         // coordinate scale
    double dp_scale;  // factor of the momentum sum
};

inline KernelScale kernel_scale(int kernel, double sigma)
{
    const double log2e = 1.4426950408889634;
    KernelScale k{};
    switch (kernel) {
    case EP_GAUSS:
        k.s = sqrt(log2e / (2.0 * sigma * sigma));
        k.dp_scale = 1.0 / (k.s * sigma * sigma);
        break;
    case EP_TENT:
        k.s = 1.0 / sigma;
        k.dp_scale = 1.0 / sigma;
        break;
    default:
        k.s = log2e / sigma;
        k.dp_scale = 1.0 / sigma;
        break;
    }
    return k;
}

// ---------------------------------------------------------------- launch counter
// Incremented once per kernel launch (exported as ep_launch_count).
void count_launch(int k = 1);

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
ep_status cuda_fail(cudaError_t e, const char* what);

#define EP_TRY_CUDA(expr)                                         \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return ::ep::cuda_fail(_e, #expr); \
    } while (0)

#define EP_TRY(expr)                         \
    do {                                     \
        ep_status _s = (expr);               \
        if (_s != EP_OK) return _s;          \
    } while (0)

// ---------------------------------------------------------------- device info
struct DeviceInfo {
    int device;
    int sm_count;
    int max_smem_optin;
    int cc_major, cc_minor;
};
ep_status device_info(DeviceInfo* out);

// ---------------------------------------------------------------- workspace
// A grow-only device arena per (device, stream).  Allocation happens only when
// a call needs more bytes than the arena holds (cudaMalloc after a stream
// synchronise); the arena is reused by every later call on that stream.
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t used = 0;
    void* carve(size_t bytes)
    {
        size_t off = (used + 255) & ~size_t(255);
        if (off + bytes > cap) return nullptr;
        used = off + bytes;
        return base + off;
    }
};
ep_status arena_acquire(cudaStream_t stream, size_t bytes, Arena** out);

// Bytes a carve sequence needs (each carve rounded up to 256 bytes).
struct Sizer {
    size_t total = 0;
    void add(size_t bytes) { total += (bytes + 255) & ~size_t(255); }
};

// ---- compensated (double-FP32) accumulation of the per-particle sums
// A value is an unevaluated pair (hi, lo) of floats whose exact sum carries ~48
// significant bits; the intrinsics keep the compiler from contracting or
// reassociating the error terms.  The lane sums over one staged chunk are FP32;
// every sum across warps, chunks and CTAs goes through these, so a particle's
// sum is accumulated to FP64-level accuracy whatever n is.
//
// Error-free transformation of a sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float& e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// acc += b (cascaded: the rounding errors gather in acc.y; no renormalisation)
__device__ __forceinline__ void dd_acc(float2& acc, float b)
{
    float e;
    acc.x = two_sum(acc.x, b, e);
    acc.y = __fadd_rn(acc.y, e);
}

// a + b, renormalised so that hi is the float nearest to the pair's value
__device__ __forceinline__ float2 dd_add(float2 a, float2 b)
{
    float e;
    const float s = two_sum(a.x, b.x, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    const float h = __fadd_rn(s, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

// The pair's value in FP64 (exact for a renormalised pair, whose two parts span at
// most 48 bits).
__device__ __forceinline__ double dd_to_double(float2 a)
{
    return (double)a.x + (double)a.y;
}

// ---------------------------------------------------------------- validation
ep_status check_params(const ep_params* p);

}  // namespace ep
