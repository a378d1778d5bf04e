// ep_features.cuh -- entry points and buffers of the cell-list, adjoint and
// batched paths (declarations shared with ep_api.cu).
#pragma once

#include "ep_common.cuh"

namespace ep {

// ---------------------------------------------------------------- cell list (tent kernel)
struct CellBufs {
    int n = 0, dim = 2, prec = EP_MIXED;
    double* x = nullptr;  // FP64 step state [q (n*dim) | p (n*dim)]
    // device pointers and the grid of the current call, owned by ep_celllist.cu
    alignas(16) char host[1024];
};
size_t cell_bytes(int n, int dim, int prec);
ep_status cell_carve(Arena* ar, int n, int dim, int prec, CellBufs* b);
ep_status cell_load(const ep_params& P, CellBufs& b, const double* q, const double* p, cudaStream_t st);
ep_status cell_rhs(const ep_params& P, const CellBufs& b, double* dq, double* dp, cudaStream_t st);
ep_status cell_steps(const ep_params& P, const CellBufs& b, int steps, double dt, cudaStream_t st);

bool use_celllist(const ep_params& P, int64_t n);

// ---------------------------------------------------------------- entry points
ep_status cell_neighbors_entry(const ep_params* params, int64_t n, const double* q, int64_t* count,
                               uint64_t* hash, int64_t* total, void* stream);
ep_status hvp_entry(const ep_params* params, int64_t n, const double* q, const double* p, const double* vq,
                    const double* vp, double* hq, double* hp, void* stream);
ep_status adjoint_entry(const ep_params* params, int64_t n, const double* X, const double* p0,
                        const double* Y, double lambda, int ckpt_every, double* grad_p0, double* energy,
                        void* stream);
ep_status batched_entry(const ep_params* params, int nprob, const int64_t* offsets, const double* X,
                        const double* Y, double* p0, ep_match_info* infos, void* stream);
ep_status velocity_entry(const ep_params* params, int64_t n, const double* q, const double* p, int64_t m,
                         const double* x, double* u, void* stream);
ep_status flow_entry(const ep_params* params, int64_t n, const double* q0, const double* p0, int64_t m,
                     const double* x0, double* x1, void* stream);
// ep_match of one small 2-D mixed-precision problem, solved entirely on one CTA.
// ginv (device, n x n row-major, or null): G(X)^-1 for the velocity update
// p0 += h G(X)^-1 (Y - Q(1)); null runs the momentum rule.
ep_status match_small(const ep_params* params, int64_t n, const double* X, const double* Y, double* p0,
                      ep_match_info* info, void* stream, const double* ginv = nullptr);

// Algorithm 1 for the plain FP64 method in one cooperative launch (ep_match_dev.cu):
// X, Y, p0 device arrays (p0 in/out), hist_dev maxit + 1 doubles on the device or
// null; workspace from ar (match_device_bytes); out = h, residual, H, iterations,
// status, Gram products (the velocity rule's MINRES iterations).  Runs the momentum
// rule and the velocity rule (info->rule).
size_t match_device_bytes(int64_t n, int dim, int maxit, int rule);
ep_status match_device_fp64(const ep_params& P, int64_t n, const double* X, const double* Y, double* p0,
                            ep_match_info* info, double* hist_dev, Arena* ar, cudaStream_t st, double out[6]);
constexpr int64_t kDeviceMatchMaxN = 16384;

// Tangent-linear shoot and the solved update rules of ep_match (ep_newton.cu).
ep_status tangent_entry(const ep_params* params, int64_t n, const double* q0, const double* p0, const double* vq0,
                        const double* vp0, double* q1, double* p1, double* vq1, double* vp1, void* stream);
ep_status rule_match(const ep_params& P, int64_t n, const double* X, const double* Y, double* p0,
                     ep_match_info* info, cudaStream_t st);
ep_status velocity_mixed_match(const ep_params& P, int64_t n, const double* X, const double* Y, double* p0,
                               ep_match_info* info, cudaStream_t st);
constexpr int64_t kSmallMatchMaxN = 384;

}  // namespace ep
