// ep_allpairs.cuh -- all-pairs RHS / fused RK4 stage kernels (declarations).
#pragma once

#include "ep_common.cuh"

namespace ep {

enum StageMode { MODE_RK4 = 0, MODE_RHS = 1 };

// Device buffers of one all-pairs problem of n particles.  Mixed precision uses
// the float4 stage copies; FP64 mode uses the double stage copies.
struct AllPairsBufs {
    int n = 0, dim = 2, prec = EP_MIXED;
    double* x = nullptr;     // FP64 step state [q (n*dim) | p (n*dim)]
    double* K = nullptr;     // FP64 k accumulator, n * kKWidth, zero between launches
    int* counters = nullptr; // per-tile arrival counters, zero between launches
    double* c0 = nullptr;    // origin of the scaled coordinates (3 doubles)
    unsigned* bar = nullptr; // grid-barrier counter of the persistent shoot
    int* err = nullptr;      // error flag of the persistent shoot (1 = a barrier wait gave up)
    double* x_bak = nullptr; // autotuner backups of x and the stage copy (2-D mixed only)
    float4* S_bak = nullptr;
    // mixed
    float4* Sx = nullptr;    // step-start stage copy (stage-0 input)
    float4* Sa = nullptr;    // stage copies (ping-pong)
    float4* Sb = nullptr;
    float* acc = nullptr;    // FP32 RK4 accumulator, n * 2 * dim
    float* part = nullptr;   // per-(CTA, tile) partial sums of the tensor-core path (2-D mixed)
    // fp64
    double* Dx = nullptr;
    double* Da = nullptr;
    double* Db = nullptr;
    double* dacc = nullptr;  // FP64 RK4 accumulator
};

size_t allpairs_bytes(int n, int dim, int prec);
ep_status allpairs_carve(Arena* ar, int n, int dim, int prec, AllPairsBufs* b);

// Launch configuration (CTA count, threads) chosen by the tuner.
struct APConfig {
    int threads = 1024;
    int ctas = 0;
};
APConfig allpairs_config(int n, int dim, int prec, int kernel);

// x <- (q, p); stage copy Sx/Dx <- x; K, counters zeroed; c0 = bbox centre of q.
ep_status allpairs_load(const ep_params& P, const AllPairsBufs& b, const double* q,
                        const double* p, cudaStream_t st);
// One RHS evaluation at the state in x; writes dq, dp (device, n*dim each).
ep_status allpairs_rhs(const ep_params& P, const AllPairsBufs& b, double* dq, double* dp,
                       cudaStream_t st);
// steps RK4 steps of size dt from the state in x (x updated in place).
ep_status allpairs_steps(const ep_params& P, const AllPairsBufs& b, int steps, double dt,
                         cudaStream_t st);

// As allpairs_steps, recording every stage input: stage copy 4k + s (s = 0..3) of
// rec (mixed; float4 x (dim == 2 ? 1 : 2) per particle, scaled positions) or drec
// (FP64; 2*dim doubles per particle) holds the input of stage s of step k, and
// copy 4*steps the final state.  rec / drec hold 4*steps + 1 stage copies.
ep_status allpairs_steps_rec(const ep_params& P, const AllPairsBufs& b, int steps, double dt, float4* rec,
                             double* drec, cudaStream_t st);

// Algorithm 1 with M = h I on the momenta (Sec. 4) of a mixed-precision 2-D Gaussian
// problem in one cooperative launch, when the shoot's (tuned) configuration is an
// owner-computes kernel; *done = false otherwise, and the caller runs its host loop.
// X, Y, p0: device, n x 2 row-major; p0 is updated in place.  hist: maxit + 1 device
// doubles (the residual of every shoot) or null; scratch: owner_match_bytes() of device
// memory; out (host) = {final residual, updates, status}.  Same results as the host loop.
ep_status owner_match(const ep_params& P, const AllPairsBufs& b, const double* X, const double* Y, double* p0,
                      int maxit, double eps, double h, double* hist, double* scratch, cudaStream_t st, bool* done,
                      double out[3]);
size_t owner_match_bytes();

// Launch timing of the persistent shoot (ep_set_launch_timing): when on, the
// launch functions record CUDA events around the cooperative launch.
bool launch_timing_enabled();
void set_launch_timing(bool on);
void record_launch_time(cudaEvent_t e0, cudaEvent_t e1, const char* kernel);
double last_launch_ms();
const char* last_launch_kernel();

// Tensor-core (tcgen05) persistent path of the 2-D Gaussian in mixed precision
// (ep_tc.cu).  Opt-in: EP_TC=1 in the environment selects it (the CUDA-core path
// is faster for this contraction, see ep_tc.cu).
bool tc_enabled(const ep_params& P);
int tc_tiles(int n);
size_t tc_part_floats(int n, int sm_count);
// mode MODE_RK4: `steps` RK4 steps of size dt from the state in x (x, Sx updated);
// mode MODE_RHS: one RHS at Sx into out_q, out_p.  G = requested CTA count.
ep_status tc_run(const ep_params& P, const AllPairsBufs& b, int steps, double dt, int mode, double* out_q,
                 double* out_p, int G, cudaStream_t st, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);

}  // namespace ep
