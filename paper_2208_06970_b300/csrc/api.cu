// api.cu -- library-level entry points: status strings, version, workspace sizes.
#include <cudaTypedefs.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "tma.cuh"

namespace lsrvt {
size_t ccl_workspace(Dims d);
size_t saliency_workspace(Dims d);
size_t seed_workspace(Dims d, int32_t sb, int32_t max_comp, int64_t max_rec);
int64_t seed_default_strata(Dims d, int32_t sb, int32_t max_comp);
size_t cvt_workspace(Dims d, int32_t max_sites);
size_t cvt_anyangle_workspace(Dims d, int32_t max_sites, int32_t max_rounds);
size_t aggregate_workspace(Dims d, int32_t max_sites, int32_t m);
size_t merge_workspace(int32_t max_sites, int32_t max_comp, int32_t n_bands, int32_t m);
size_t layout_workspace(Dims d, int32_t max_sites);
size_t joint_workspace(int32_t max_ranges, int64_t n_positions, int32_t m);
size_t joint_merge_workspace(int32_t max_sites, int32_t max_comp, int32_t m);
size_t graph_workspace(Dims d);
}  // namespace lsrvt

namespace lsrvt {

namespace {
// the driver's encoder, looked up once through the runtime (no link-time libcuda dependency)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    return encode;
}
}  // namespace

bool encode_volume_map(CUtensorMap *map, const void *base, CUtensorMapDataType type, int elem_bytes, int nx, int ny,
                       int nz, int bx, int by, int bz) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode || !base || ((uintptr_t)base & 15) || ((int64_t)nx * elem_bytes) % 16) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * elem_bytes, (cuuint64_t)nx * ny * elem_bytes};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estride[3] = {1, 1, 1};
    return encode(map, type, 3, const_cast<void *>(base), dims, strides, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_stack_map(CUtensorMap *map, const void *base, CUtensorMapDataType type, int elem_bytes, int nx, int ny,
                      int nz, int m, int64_t vol_pitch, int bx, int by, int bz, int bw) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode || !base || ((uintptr_t)base & 15) || ((int64_t)nx * elem_bytes) % 16 || vol_pitch <= 0 ||
        vol_pitch % 16 || bw > 256)
        return false;
    const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)m};
    const cuuint64_t strides[3] = {(cuuint64_t)nx * elem_bytes, (cuuint64_t)nx * ny * elem_bytes,
                                   (cuuint64_t)vol_pitch};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, (cuuint32_t)bw};
    const cuuint32_t estride[4] = {1, 1, 1, 1};
    return encode(map, type, 4, const_cast<void *>(base), dims, strides, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {
std::mutex g_share_mu;
std::vector<std::pair<cudaStream_t, int>> g_share;  // stream -> percent of the SMs
}  // namespace

int stream_sms(cudaStream_t s) {
    static const int nsm = []() {
        int dev = 0, n = kSMs;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : kSMs;
    }();
    std::lock_guard<std::mutex> lk(g_share_mu);
    for (const auto &e : g_share)
        if (e.first == s) {
            const int k = (int)((int64_t)nsm * e.second / 100);
            return k > 0 ? k : 1;
        }
    return nsm;
}

}  // namespace lsrvt

using namespace lsrvt;

extern "C" lsrvt_status lsrvt_set_stream_share(void *stream, int32_t percent) {
    if (percent < 1 || percent > 100) return LSRVT_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    std::lock_guard<std::mutex> lk(g_share_mu);
    for (size_t i = 0; i < g_share.size(); ++i)
        if (g_share[i].first == s) {
            if (percent == 100) g_share.erase(g_share.begin() + (long)i);
            else g_share[i].second = percent;
            return LSRVT_OK;
        }
    if (percent < 100) g_share.emplace_back(s, percent);
    return LSRVT_OK;
}

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
        case LSRVT_STEP_AGGREGATE: return aggregate_workspace(d, max_sites, n_aux);
        case LSRVT_STEP_MERGE: return merge_workspace(max_sites, max_comp, 255, n_aux);
        case LSRVT_STEP_LAYOUT: return layout_workspace(d, max_sites > 0 ? max_sites : 1);
        case LSRVT_STEP_GRAPH: return graph_workspace(d);
        case LSRVT_STEP_CVT_ANYANGLE: return cvt_anyangle_workspace(d, max_sites, n_aux > 0 ? n_aux : 1);
        case LSRVT_STEP_JOINT: {
            // the moments over max_sites ranges of d.n() positions, and the merge of max_sites cell
            // records into max_comp components (n_aux = the variable count)
            const size_t a = joint_workspace(max_sites, d.n(), n_aux), b = joint_merge_workspace(max_sites, max_comp, n_aux);
            return a > b ? a : b;
        }
    }
    return 0;
}
