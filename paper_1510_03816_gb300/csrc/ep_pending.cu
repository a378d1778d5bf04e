// ep_pending.cu -- entry points whose GPU paths are not built yet: they
// report EP_EINVAL with a message instead of computing anything.
#include "ep_features.cuh"

namespace ep {

static ep_status pending(const char* what)
{
    set_error("%s is not available in this build", what);
    return EP_EINVAL;
}

ep_status batched_entry(const ep_params*, int, const int64_t*, const double*, const double*, double*, ep_match_info*, void*) { return pending("ep_match_batched"); }

}  // namespace ep
