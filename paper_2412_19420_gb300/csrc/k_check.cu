// k_check.cu -- opt-in runtime invariants (the "debug_checks" knob), the
// library's stand-in for a sanitizer on a pool where compute-sanitizer is
// closed.  Nothing here changes results; a violated invariant turns the call
// into FIM_E_CHECK.
//
// Guard words: the bit columns are padded from nw to nwp words, and the last
// word of a column holds only n mod 32 transactions; every pad bit and pad
// word must still be zero after the build (an out-of-range write there would
// show), and the popcounts of Eq. 3 rely on it.
//
// Output invariants of a mine (Eq. 3 and the canonical order): every set is
// non-empty, its items are strictly ascending and below n_items, its support
// passes the threshold, and consecutive sets are strictly increasing in
// (size, items) order -- so no set appears twice.
#include "fim_common.cuh"

namespace {

__global__ void check_pads_kernel(const uint32_t *__restrict__ bm, int32_t m, int64_t n, int64_t nw, int64_t nwp,
                                  int *__restrict__ bad) {
    const int64_t pad = nwp - nw + 1;  // the last data word (its high bits) and the pad words
    const int64_t total = (int64_t)m * pad;
    const uint32_t last_mask = (n % 32) ? ~((1u << (n % 32)) - 1u) : 0xFFFFFFFFu;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = i / pad, w = nw - 1 + i % pad;
        if (w < 0) continue;  // n == 0: no data word
        const uint32_t v = bm[j * nwp + w];
        const uint32_t must_be_zero = w == nw - 1 ? (n % 32 ? last_mask : 0u) : 0xFFFFFFFFu;
        if (v & must_be_zero) atomicExch(bad, 1);
    }
}

__global__ void check_output_kernel(const unsigned long long *__restrict__ off, const uint32_t *__restrict__ items,
                                    const uint32_t *__restrict__ sup, unsigned long long R, uint32_t n_items,
                                    uint32_t thr, int *__restrict__ bad) {
    for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < R;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long o = off[q], e = off[q + 1];
        bool ok = e > o && sup[q] >= thr;
        for (unsigned long long i = o; ok && i < e; i++) ok = items[i] < n_items && (i == o || items[i - 1] < items[i]);
        if (ok && q + 1 < R) {  // strictly before the next set in (size, items) order
            const unsigned long long o2 = off[q + 1], e2 = off[q + 2];
            const unsigned long long l1 = e - o, l2 = e2 - o2;
            if (l1 != l2) {
                ok = l1 < l2;
            } else {
                int c = 0;
                for (unsigned long long k = 0; k < l1 && c == 0; k++)
                    c = items[o + k] < items[o2 + k] ? -1 : (items[o + k] > items[o2 + k] ? 1 : 0);
                ok = c < 0;
            }
        }
        if (!ok) atomicExch(bad, 1);
    }
}

}  // namespace

int run_check_pads(fim_ctx *ctx) {
    if (ctx->m <= 0 || ctx->nwp <= 0) return FIM_OK;
    int *bad = ctx->dev_flag.as<int>() + 3;
    cudaStream_t st = ctx->stream;
    FIM_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    const unsigned grid = (unsigned)(ctx->num_sms > 0 ? ctx->num_sms : 1) * 4u;
    ctx->launches++;
    check_pads_kernel<<<grid, 256, 0, st>>>(ctx->bm.as<uint32_t>(), ctx->m, ctx->n, ctx->nw, ctx->nwp, bad);
    FIM_CUDA_TRY(cudaGetLastError());
    int h = 0;
    FIM_CUDA_TRY(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    FIM_CUDA_TRY(cudaStreamSynchronize(st));
    return h ? FIM_E_CHECK : FIM_OK;
}

int run_check_output(fim_ctx *ctx, uint32_t thr) {
    const unsigned long long R = ctx->out_sets;
    if (R == 0) return FIM_OK;
    int *bad = ctx->dev_flag.as<int>() + 3;
    cudaStream_t st = ctx->stream;
    FIM_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
    const unsigned grid = (unsigned)(ctx->num_sms > 0 ? ctx->num_sms : 1) * 4u;
    ctx->launches++;
    check_output_kernel<<<grid, 256, 0, st>>>(ctx->out_off.as<unsigned long long>(), ctx->out_items.as<uint32_t>(),
                                              ctx->out_sup.as<uint32_t>(), R, (uint32_t)ctx->m, thr, bad);
    FIM_CUDA_TRY(cudaGetLastError());
    int h = 0;
    FIM_CUDA_TRY(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    FIM_CUDA_TRY(cudaStreamSynchronize(st));
    return h ? FIM_E_CHECK : FIM_OK;
}
