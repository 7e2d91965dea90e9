// Count Sketch update kernels for the prime msf::P61 (one translation unit per
// prime so that they compile in parallel).
#include "k_update_dispatch.cuh"

namespace msk {

cudaError_t launch_update_p61(const UpdateArgs& a, const u64* coef_host, const LaunchCfg& cfg,
                              cudaStream_t stream, int* specialized, int* occupancy) {
    return launch_update_for<msf::P61>(a, coef_host, cfg, stream, specialized, occupancy);
}

cudaError_t launch_point_query_p61_sd(const QueryArgs& a, const u64* coef_host,
                                      cudaStream_t stream) {
    const bool two = a.mode == CS_TWO_POLY, any = a.arb_r != 0;
    if (a.t == 5) {
        if (two) return any ? point_query_sd<5, 2, true>(a, coef_host, stream)
                            : point_query_sd<5, 2, false>(a, coef_host, stream);
        return any ? point_query_sd<5, 1, true>(a, coef_host, stream)
                   : point_query_sd<5, 1, false>(a, coef_host, stream);
    }
    if (two) return any ? point_query_sd<7, 2, true>(a, coef_host, stream)
                        : point_query_sd<7, 2, false>(a, coef_host, stream);
    return any ? point_query_sd<7, 1, true>(a, coef_host, stream)
               : point_query_sd<7, 1, false>(a, coef_host, stream);
}

cudaError_t launch_gtable_drain_p61(const UpdateArgs& a, const u64* coef_host,
                                    cudaStream_t stream) {
    return launch_gtable_drain_for<msf::P61>(a, coef_host, stream);
}

}  // namespace msk
