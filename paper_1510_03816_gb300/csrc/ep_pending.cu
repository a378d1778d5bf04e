// ep_pending.cu -- entry points whose GPU paths are not built yet: they
// report EP_EINVAL with a message instead of computing anything.
#include "ep_features.cuh"

namespace ep {

static ep_status pending(const char* what)
{
    set_error("%s is not available in this build", what);
    return EP_EINVAL;
}

size_t cell_bytes(int, int, int) { return 0; }
ep_status cell_carve(Arena*, int, int, int, CellBufs*) { return pending("the cell list"); }
ep_status cell_load(const ep_params&, const CellBufs&, const double*, const double*, cudaStream_t) { return pending("the cell list"); }
ep_status cell_rhs(const ep_params&, const CellBufs&, double*, double*, cudaStream_t) { return pending("the cell list"); }
ep_status cell_steps(const ep_params&, const CellBufs&, int, double, cudaStream_t) { return pending("the cell list"); }
ep_status cell_neighbors_entry(const ep_params*, int64_t, const double*, int64_t*, uint64_t*, int64_t*, void*) { return pending("ep_cell_neighbors"); }
ep_status batched_entry(const ep_params*, int, const int64_t*, const double*, const double*, double*, ep_match_info*, void*) { return pending("ep_match_batched"); }

}  // namespace ep
