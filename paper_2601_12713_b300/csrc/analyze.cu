// analyze.cu -- odp_analyze (placeholder until the analysis kernels land).
#include "common.cuh"

extern "C" int odp_analyze(const odp_event* events, uint64_t n, const odp_findings* out,
                           cudaStream_t stream) {
    (void)events; (void)n; (void)out; (void)stream;
    return ODP_ERR_UNSUPPORTED;
}
