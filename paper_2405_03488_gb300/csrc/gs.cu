// Colour sparsification and exact counting (filled in below the NS path).
#include "internal.h"

using namespace gpm;

extern "C" gpm_status gpm_exact_count(gpm_graph *, const gpm_pattern *, uint64_t *) {
    set_error("gpm_exact_count: not built yet");
    return GPM_ERR_UNSUPPORTED;
}

extern "C" gpm_status gpm_sparsify(gpm_graph *, uint32_t, uint64_t, uint32_t, uint32_t, uint64_t *, uint32_t *,
                                   uint64_t *) {
    set_error("gpm_sparsify: not built yet");
    return GPM_ERR_UNSUPPORTED;
}

extern "C" gpm_status gpm_estimate_batch(gpm_graph *, uint32_t, const gpm_pattern *, const double *, double,
                                         uint64_t, const gpm_config *, gpm_result *) {
    set_error("gpm_estimate_batch: not built yet");
    return GPM_ERR_UNSUPPORTED;
}
