// api.cu -- library-level entry points: status strings, version, workspace sizes.
#include "common.cuh"

namespace lsrvt {
size_t ccl_workspace(Dims d);
size_t saliency_workspace(Dims d);
size_t seed_workspace(Dims d, int32_t sb, int32_t max_comp, int64_t max_rec);
int64_t seed_default_strata(Dims d, int32_t sb, int32_t max_comp);
size_t cvt_workspace(Dims d, int32_t max_sites);
size_t aggregate_workspace(int32_t max_sites, int32_t m);
size_t merge_workspace(int32_t max_sites, int32_t max_comp, int32_t n_bands, int32_t m);
}  // namespace lsrvt

using namespace lsrvt;

extern "C" const char *lsrvt_status_string(lsrvt_status s) {
    switch (s) {
        case LSRVT_OK: return "ok";
        case LSRVT_ERR_INVALID_ARG: return "invalid argument";
        case LSRVT_ERR_NOT_SORTED: return "isovalues not strictly increasing";
        case LSRVT_ERR_CAPACITY: return "capacity exceeded";
        case LSRVT_ERR_NONFINITE: return "non-finite input value";
        case LSRVT_ERR_TIMEOUT: return "device loop limit reached";
        case LSRVT_ERR_OVERFLOW: return "geodesic distance overflow";
        case LSRVT_ERR_CUDA: return "CUDA launch failure";
        case LSRVT_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    }
    return "unknown status";
}

extern "C" int32_t lsrvt_version(void) { return 10000; }

// The seed step's workspace uses the default stratum capacity (strat_block 16); callers that
// pass another strat_block or max_strata size their workspace with the largest they use.
extern "C" size_t lsrvt_workspace_bytes(lsrvt_step step, lsrvt_dims dd, int32_t max_comp, int32_t max_sites,
                                        int32_t n_aux) {
    if (!dims_ok(dd) || max_comp < 0 || max_sites < 0 || n_aux < 0) return 0;
    Dims d{dd.nx, dd.ny, dd.nz};
    switch (step) {
        case LSRVT_STEP_CLASSIFY: return 0;
        case LSRVT_STEP_LABEL: return ccl_workspace(d);
        case LSRVT_STEP_SALIENCY: return saliency_workspace(d);
        case LSRVT_STEP_SEED: {
            size_t a = seed_workspace(d, 16, max_comp, seed_default_strata(d, 16, max_comp));
            size_t b = seed_workspace(d, 1, max_comp, seed_default_strata(d, 1, max_comp));
            return a > b ? a : b;
        }
        case LSRVT_STEP_CVT: return cvt_workspace(d, max_sites);
        case LSRVT_STEP_AGGREGATE: return aggregate_workspace(max_sites, n_aux);
        case LSRVT_STEP_MERGE: return merge_workspace(max_sites, max_comp, 255, n_aux);
    }
    return 0;
}
