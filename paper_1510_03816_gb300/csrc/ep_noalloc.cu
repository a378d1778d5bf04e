// ep_noalloc.cu -- ep_rhs_noalloc: the all-pairs right-hand side with its
// scratch memory in a fixed device array, so that the call never allocates.
//
// Who needs it: a caller that may not call cudaMalloc (or any allocating
// routine) at the moment it evaluates the right-hand side.  Examples are code
// running inside a host callback or a real-time loop where cudaMalloc's
// implicit device synchronisation is not acceptable, and plug-ins hosted by a
// framework whose memory pool owns the whole device and forbids allocations
// outside it.  ep_rhs would grow its workspace arena on the first call of a
// given size; this entry point takes every byte of scratch from one
// file-scope __device__ array instead.
//
// The array is part of the library image: every GPU that loads libep.so holds
// kNoAllocScratchBytes of it until the process exits.  It bounds the problem
// size to EP_NOALLOC_MAX_N particles.  All calls share the array, and each call
// leaves its contents behind; the parts that must start at zero (the FP64
// accumulator and the per-tile counters) are cleared by every call.  Calls
// whose GPU work overlaps (e.g. issued on two streams without ordering) race
// on the array and give wrong results.
#include <map>
#include <mutex>

#include "ep_allpairs.cuh"

namespace ep {

namespace {

// Scratch for n <= EP_NOALLOC_MAX_N in either precision and dimension: the FP64
// state x (n*2*dim doubles), the FP64 accumulator K (n*6 doubles), the per-tile
// counters, the origin c0 and one stage copy (FP32 float4 x (dim == 2 ? 1 : 2)
// per particle, or FP64 2*dim doubles per particle), each rounded up to 256 bytes.
constexpr size_t kNoAllocScratchBytes = 1280 * 1024;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
// (device, context id) -> device address of g_noalloc_scratch.  The context id
// is part of the key because cudaDeviceReset (or any destruction and re-creation
// of the primary context) loads the module again, possibly at another address.
std::map<std::pair<int, unsigned long long>, void*> g_addr;

// The current context's id (cuCtxGetId, unique for the life of the process), by
// way of the runtime's driver entry points so that the library needs no link
// against the driver library.  0 when the driver does not provide it.
unsigned long long current_context_id()
{
    typedef int (*ctx_get_current_t)(void**);
    typedef int (*ctx_get_id_t)(void*, unsigned long long*);
    static ctx_get_current_t get_current = nullptr;
    static ctx_get_id_t get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (ctx_get_current_t)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (ctx_get_id_t)f;
        cudaGetLastError();
    });
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
    return 0;
}

// Set-up, once per device (and per context on it), with that device current:
// look up the array's device address.  In host code the symbol is only a
// host-side stand-in.  Before the first runtime call on a thread no context may
// be current (id 0): the lookup then creates the primary context, and the entry
// is stored under the id of the context it was made in.
ep_status scratch_address(void** out)
{
    int dev = 0;
    EP_TRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long id = current_context_id();
    if (id != 0) {
        auto it = g_addr.find(std::make_pair(dev, id));
        if (it != g_addr.end()) {
            *out = it->second;
            return EP_OK;
        }
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_addr[std::make_pair(dev, current_context_id())] = p;
    *out = p;
    return EP_OK;
}

bool on_device(const void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Only the buffers one RHS evaluation touches.
ep_status carve_rhs(Arena* ar, int n, int dim, int prec, AllPairsBufs* b)
{
    const int ntiles = (n + kTileI - 1) / kTileI;
    b->n = n;
    b->dim = dim;
    b->prec = prec;
    b->x = (double*)ar->carve(sizeof(double) * 2 * dim * (size_t)n);
    b->K = (double*)ar->carve(sizeof(double) * kKWidth * (size_t)n);
    b->counters = (int*)ar->carve(sizeof(int) * (size_t)ntiles);
    b->c0 = (double*)ar->carve(sizeof(double) * 4);
    if (prec == EP_MIXED)
        b->Sx = (float4*)ar->carve(sizeof(float4) * (dim == 2 ? 1 : 2) * (size_t)n);
    else
        b->Dx = (double*)ar->carve(sizeof(double) * 2 * dim * (size_t)n);
    if (!b->c0 || !(prec == EP_MIXED ? (void*)b->Sx : (void*)b->Dx)) {
        set_error("ep_rhs_noalloc: scratch array too small for n = %d", n);
        return EP_EINVAL;
    }
    return EP_OK;
}

}  // namespace

}  // namespace ep

using namespace ep;

extern "C" ep_status ep_rhs_noalloc(const ep_params* params, int64_t n, const double* q, const double* p,
                                    double* dq, double* dp, void* stream)
{
    EP_TRY(check_params(params));
    if (n < 0 || n > EP_NOALLOC_MAX_N) {
        set_error("ep_rhs_noalloc: n = %lld outside [0, %d] (the fixed scratch array's limit)", (long long)n,
                  EP_NOALLOC_MAX_N);
        return EP_EINVAL;
    }
    if (params->neigh == EP_CELLLIST) {
        set_error("ep_rhs_noalloc: only the all-pairs path is available without allocation");
        return EP_EINVAL;
    }
    void* base = nullptr;
    EP_TRY(scratch_address(&base));
    if (n == 0) return EP_OK;
    if (!q || !p || !dq || !dp) return set_error("ep_rhs_noalloc: NULL array"), EP_EINVAL;
    if (!on_device(q) || !on_device(p) || !on_device(dq) || !on_device(dp)) {
        set_error("ep_rhs_noalloc: arrays must be device memory (host arrays would need staging memory)");
        return EP_EINVAL;
    }
    const ep_params& P = *params;
    cudaStream_t st = (cudaStream_t)stream;
    Arena ar;
    ar.base = (char*)base;
    ar.cap = kNoAllocScratchBytes;
    AllPairsBufs b;
    EP_TRY(carve_rhs(&ar, (int)n, P.dim, P.precision, &b));
    // allpairs_load clears K and the counters before the RHS kernel reads them
    EP_TRY(allpairs_load(P, b, q, p, st));
    EP_TRY(allpairs_rhs(P, b, dq, dp, st));
    EP_TRY_CUDA(cudaGetLastError());
    return EP_OK;
}
