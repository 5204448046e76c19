// Weighted edge sampling (Algorithm 3).  Placeholder until the sampler lands.
#include "wtri_internal.cuh"

namespace wtri {

int sample_topk_device(const wtri_graph* g, int pcode, int32_t k, int64_t nsamples, uint64_t seed,
                       wtri_tri* d_tris, double* d_weight, int32_t* d_count, cudaStream_t stream,
                       int retry_scale) {
    (void)g; (void)pcode; (void)k; (void)nsamples; (void)seed; (void)d_tris; (void)d_weight;
    (void)d_count; (void)stream; (void)retry_scale;
    return set_error(WTRI_EUNSUPPORTED, "edge sampling is not built yet");
}

}  // namespace wtri
