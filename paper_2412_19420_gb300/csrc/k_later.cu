// k_later.cu -- entry points whose kernels are not written yet.  Each returns
// FIM_E_INVAL so a caller can tell the feature is absent.
#include "fim_common.cuh"



extern "C" {
int fim_mine_batched(fim_ctx *, int, const fim_db_desc *, uint32_t) { return FIM_E_INVAL; }
int fim_fetch_batched(fim_ctx *, int, uint64_t *, uint64_t *, uint64_t *, uint32_t *, uint32_t *,
                      uint64_t, uint64_t, uint32_t) { return FIM_E_INVAL; }
int fim_sched_load_weights(fim_ctx *, const float *, size_t) { return FIM_E_INVAL; }
int fim_fetch_traces(fim_ctx *, uint64_t *, float *, float *, uint64_t) { return FIM_E_INVAL; }
int fim_mlp_forward(fim_ctx *, const float *, const float *, int64_t, float *, float *, int) { return FIM_E_INVAL; }
int fim_mlp_backward(fim_ctx *, const float *, const float *, const float *, const float *, const float *,
                     int64_t, float *, float *, int) { return FIM_E_INVAL; }
int fim_mlp_adam(fim_ctx *, float *, const float *, float *, float *, int, float, float, float, float) {
    return FIM_E_INVAL;
}
}
