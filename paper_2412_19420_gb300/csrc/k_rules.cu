// k_rules.cu -- association rules from the frequent itemsets: a post-pass over
// the canonical output of the extraction (Eq. 3), for the confidence and lift
// measures the paper names beside support.
//
// For every frequent Z with 2 <= |Z| <= FIM_RULES_MAX_LEN and every nonempty
// proper subset X of Z (Y = Z \ X), the rule X -> Y has
//     conf = S(Z) / S(X),     lift = S(Z) n / (S(X) S(Y)),
// and is kept when S(Z) * 10^6 >= min_conf_ppm * S(X) (exact integers).
// S(X) and S(Y) are looked up in the canonical output itself, which is sorted
// by (size, items): every subset of a frequent set is frequent (downward
// closure), so a binary search always finds it.
//
// One warp per Z: lane l takes the antecedent masks l + 1, l + 33, ... in
// rounds of 32, so each round's kept rules are compacted with one ballot and
// stay in mask order.  Pass 1 counts the kept rules of every Z, a scan gives
// each Z its slice, pass 2 writes (set index, mask, conf, lift).
#include "fim_common.cuh"

namespace {

constexpr int RMAX = FIM_RULES_MAX_LEN;
constexpr int RULE_WARPS = 8;  // warps (sets) per 256-thread CTA

// Index in the canonical order of the subset of z (|z| = L, items ascending)
// picked by the bits of mask, or -1 if it is not in the output.  The canonical
// order is (size, items lexicographic), so a binary search over the sets finds
// it; the subset's k-th item is z[k-th set bit of mask].
__device__ int64_t find_subset(const unsigned long long *__restrict__ off, const uint32_t *__restrict__ items,
                               int64_t R, const uint32_t *z, int L, uint32_t mask) {
    const int ls = __popc(mask);
    int64_t lo = 0, hi = R;  // first r with key(r) >= key(subset)
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const unsigned long long o = off[mid];
        const int lm = (int)(off[mid + 1] - o);
        int c = lm < ls ? -1 : (lm > ls ? 1 : 0);
        if (c == 0) {
            int k = 0;
            for (int i = 0; i < L; i++) {
                if (!((mask >> i) & 1u)) continue;
                const uint32_t a = items[o + k++], b = z[i];
                if (a != b) {
                    c = a < b ? -1 : 1;
                    break;
                }
            }
        }
        if (c < 0) lo = mid + 1;
        else hi = mid;
    }
    if (lo >= R) return -1;
    const unsigned long long o = off[lo];
    if ((int)(off[lo + 1] - o) != ls) return -1;
    int k = 0;
    for (int i = 0; i < L; i++)
        if (((mask >> i) & 1u) && items[o + k++] != z[i]) return -1;
    return lo;
}

// One warp per frequent set z.  WRITE = false: cnt[z] = kept rules of z.
// WRITE = true: the kept rules of z go to [base[z], base[z] + cnt[z]) in
// antecedent-mask order.
template <bool WRITE>
__global__ void __launch_bounds__(RULE_WARPS * 32)
rules_kernel(const unsigned long long *__restrict__ off, const uint32_t *__restrict__ items,
             const uint32_t *__restrict__ sup, int64_t R, uint64_t n, uint32_t ppm, int max_len,
             unsigned long long *__restrict__ cnt, const unsigned long long *__restrict__ base,
             unsigned long long *__restrict__ set_index, uint32_t *__restrict__ ante_mask,
             double *__restrict__ conf, double *__restrict__ lift, int *__restrict__ err) {
    __shared__ uint32_t zs[RULE_WARPS][RMAX];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t z = (int64_t)blockIdx.x * RULE_WARPS + wid;
    if (z >= R) return;
    const int L = (int)(off[z + 1] - off[z]);
    if (L < 2 || L > max_len) {
        if (!WRITE && lane == 0) cnt[z] = 0;
        return;
    }
    uint32_t *zi = zs[wid];
    if (lane < L) zi[lane] = items[off[z] + lane];
    __syncwarp();
    const uint64_t sz = sup[z];
    const uint32_t full = (1u << L) - 1u;  // antecedent masks 1 .. full - 1
    unsigned long long pos = WRITE ? base[z] : 0ull;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t m0 = 1; m0 < full; m0 += 32) {
        const uint32_t m = m0 + lane;
        bool keep = false;
        double c = 0.0, l = 0.0;
        if (m < full) {
            const int64_t rx = find_subset(off, items, R, zi, L, m);
            const int64_t ry = find_subset(off, items, R, zi, L, full & ~m);
            if (rx < 0 || ry < 0) {
                atomicExch(err, 1);  // a subset is missing: the sets are not downward closed
            } else {
                const uint64_t sx = sup[rx], sy = sup[ry];
                keep = sz * 1000000ull >= (uint64_t)ppm * sx;
                if (WRITE && keep) {
                    c = (double)sz / (double)sx;
                    l = (double)(sz * n) / (double)(sx * sy);
                }
            }
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, keep);
        if (WRITE && keep) {
            const unsigned long long at = pos + __popc(bal & lt);
            set_index[at] = (unsigned long long)z;
            ante_mask[at] = m;
            conf[at] = c;
            lift[at] = l;
        }
        pos += __popc(bal);
    }
    if (!WRITE && lane == 0) cnt[z] = pos;
}

// Exclusive scan of cnt[0..R) into base[0..R), total into base[R] (one CTA).
__global__ void __launch_bounds__(1024)
rules_scan_kernel(const unsigned long long *__restrict__ cnt, int64_t R, unsigned long long *__restrict__ base) {
    __shared__ unsigned long long s[1024];
    const int64_t seg = (R + 1023) / 1024;
    const int64_t b = (int64_t)threadIdx.x * seg, e = b + seg < R ? b + seg : R;
    unsigned long long sum = 0;
    for (int64_t i = b; i < e; i++) sum += cnt[i];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const unsigned long long v = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0ull;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = s[threadIdx.x] - sum;
    for (int64_t i = b; i < e; i++) {
        base[i] = run;
        run += cnt[i];
    }
    if (threadIdx.x == 1023) base[R] = s[1023];
}

}  // namespace

extern "C" {

int fim_rules(fim_ctx *ctx, uint32_t min_conf_ppm, int max_len, uint64_t *n_rules) {
    if (!ctx || !n_rules || min_conf_ppm > 1000000u) return FIM_E_INVAL;
    if (max_len == 0) max_len = RMAX;
    if (max_len < 2 || max_len > RMAX) return FIM_E_INVAL;
    *n_rules = 0;
    if (!ctx->mined) return FIM_E_STATE;
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FIM_E_CUDA;
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{dev_prev};
    cudaStream_t st = ctx->stream;
    const int64_t R = (int64_t)ctx->out_sets;
    ctx->rules_n = 0;
    ctx->rules_of = 0;
    if (R > 0) {
        FIM_TRY(fim_reserve(ctx, ctx->rule_cnt, sizeof(unsigned long long) * (size_t)(2 * R + 1)));
        unsigned long long *cnt = ctx->rule_cnt.as<unsigned long long>(), *base = cnt + R;
        int *err = ctx->dev_flag.as<int>() + 2;
        FIM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
        const unsigned blocks = (unsigned)ceil_div64(R, RULE_WARPS);
        const unsigned long long *off = ctx->out_off.as<unsigned long long>();
        const uint32_t *items = ctx->out_items.as<uint32_t>(), *sup = ctx->out_sup.as<uint32_t>();
        ctx->launches += 2;
        rules_kernel<false><<<blocks, RULE_WARPS * 32, 0, st>>>(off, items, sup, R, (uint64_t)ctx->n, min_conf_ppm,
                                                                max_len, cnt, nullptr, nullptr, nullptr, nullptr,
                                                                nullptr, err);
        rules_scan_kernel<<<1, 1024, 0, st>>>(cnt, R, base);
        FIM_CUDA_TRY(cudaGetLastError());
        unsigned long long total = 0;
        int bad = 0;
        FIM_CUDA_TRY(cudaMemcpyAsync(&total, base + R, sizeof(total), cudaMemcpyDeviceToHost, st));
        FIM_CUDA_TRY(cudaMemcpyAsync(&bad, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        FIM_CUDA_TRY(cudaStreamSynchronize(st));
        if (bad) return FIM_E_STATE;  // not the output of a mine
        if (total) {
            FIM_TRY(fim_reserve(ctx, ctx->rule_set, sizeof(unsigned long long) * (size_t)total));
            FIM_TRY(fim_reserve(ctx, ctx->rule_mask, sizeof(uint32_t) * (size_t)total));
            FIM_TRY(fim_reserve(ctx, ctx->rule_conf, sizeof(double) * (size_t)total));
            FIM_TRY(fim_reserve(ctx, ctx->rule_lift, sizeof(double) * (size_t)total));
            ctx->launches++;
            rules_kernel<true><<<blocks, RULE_WARPS * 32, 0, st>>>(
                off, items, sup, R, (uint64_t)ctx->n, min_conf_ppm, max_len, cnt, base,
                ctx->rule_set.as<unsigned long long>(), ctx->rule_mask.as<uint32_t>(), ctx->rule_conf.as<double>(),
                ctx->rule_lift.as<double>(), err);
            FIM_CUDA_TRY(cudaGetLastError());
            FIM_CUDA_TRY(cudaStreamSynchronize(st));
        }
        ctx->rules_n = total;
    }
    ctx->rules_of = ctx->mine_serial;
    if (ctx->bytes_held > ctx->stats.peak_device_bytes) ctx->stats.peak_device_bytes = ctx->bytes_held;
    *n_rules = ctx->rules_n;
    return FIM_OK;
}

int fim_fetch_rules(fim_ctx *ctx, uint64_t *n_rules, uint64_t *set_index, uint32_t *ante_mask, double *conf,
                    double *lift, uint64_t cap, uint32_t flags) {
    if (!ctx || !n_rules) return FIM_E_INVAL;
    if (!ctx->mined || ctx->rules_of != ctx->mine_serial) return FIM_E_STATE;
    *n_rules = ctx->rules_n;
    if (!set_index && !ante_mask && !conf && !lift) return FIM_OK;
    if (!set_index || !ante_mask || !conf || !lift) return FIM_E_INVAL;
    if (cap < ctx->rules_n) return FIM_E_TOO_SMALL;
    if (ctx->rules_n == 0) return FIM_OK;
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FIM_E_CUDA;
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{dev_prev};
    const cudaMemcpyKind k = (flags & FIM_OUTPUT_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaStream_t st = ctx->stream;
    const size_t nr = (size_t)ctx->rules_n;
    FIM_CUDA_TRY(cudaMemcpyAsync(set_index, ctx->rule_set.p, sizeof(uint64_t) * nr, k, st));
    FIM_CUDA_TRY(cudaMemcpyAsync(ante_mask, ctx->rule_mask.p, sizeof(uint32_t) * nr, k, st));
    FIM_CUDA_TRY(cudaMemcpyAsync(conf, ctx->rule_conf.p, sizeof(double) * nr, k, st));
    FIM_CUDA_TRY(cudaMemcpyAsync(lift, ctx->rule_lift.p, sizeof(double) * nr, k, st));
    FIM_CUDA_TRY(cudaStreamSynchronize(st));
    return FIM_OK;
}

}  // extern "C"
