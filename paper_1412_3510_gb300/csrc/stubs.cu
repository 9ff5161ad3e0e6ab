// Entry points declared in rpca.h whose kernels are not built yet.
#include "internal.cuh"

extern "C" size_t rpca_csr_workspace_size(int64_t, int64_t, int64_t, const rpca_opts *) { return 0; }
extern "C" int rpca_csr(int64_t, int64_t, int64_t, const int32_t *, const int32_t *, const float *,
                        const rpca_opts *, float *, int64_t, float *, float *, int64_t, void *, size_t,
                        rpca_stream_t) { return RPCA_ERR_UNSUPPORTED; }
