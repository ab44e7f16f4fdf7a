// k_rules.cu -- association rules from the frequent itemsets: a post-pass over
// the canonical output of the extraction (Eq. 3), for the confidence and lift
// measures the paper names beside support (Section IV.A).
//
// For every frequent Z with 2 <= |Z| <= max_len and every nonempty proper
// subset X of Z (Y = Z \ X), the rule X -> Y has
//     conf = S(Z) / S(X),     lift = S(Z) n / (S(X) S(Y)),
// and is kept when S(Z) * 10^6 >= min_conf_ppm * S(X) (exact integers).
//
// Work layout.  The candidate rules of all sets form one flat space of
// E = sum_Z (2^|Z| - 2) evaluations in (set index, antecedent mask) order, so
// a set of 11 items spreads its 2,046 antecedents over 2,046 threads instead
// of serialising them in one warp.  Evaluation e belongs to the set z with
// ebase[z] <= e < ebase[z+1] (ebase = exclusive scan of the per-set counts)
// and has mask e - ebase[z] + 1.
//   1. size_bounds: first set index of every size (the output is ordered by
//      size, then lexicographically), so a subset lookup searches only the
//      sets of its own size;
//   2. scan of the per-set counts -> ebase, E;
//   3. keep: one thread per evaluation looks up S(X) and S(Y) by binary search
//      (every subset of a frequent set is frequent: downward closure), decides
//      the threshold, and one ballot per 32 evaluations stores a keep word;
//   4. scan of the keep words' popcounts -> each word's first output slot;
//   5. write: the kept evaluations write (set index, mask, conf, lift) at their
//      slot, so the output keeps evaluation order; the keep pass leaves them
//      their three set indices (12 bytes a candidate, up to 2^27 candidates;
//      beyond that the write pass repeats the lookups).
// The itemsets (offsets, items, supports) stay resident from the mine and the
// lookups hit L2 for outputs up to tens of MB: the kernels are bound by
// dependent-load latency, not by HBM bandwidth.
#include "fim_common.cuh"

namespace {

constexpr int RMAX = FIM_RULES_MAX_LEN;
constexpr int RT = 256;                    // threads per CTA of the evaluation kernels
constexpr int SCAN_T = 1024, SCAN_I = 8;   // scan: 1024 threads x 8 elements per CTA
constexpr int SCAN_CHUNK = SCAN_T * SCAN_I;
constexpr int NSIZE = 32;                  // size_start entries (sizes 0 .. 31)
constexpr unsigned long long kRuleSetsMax = 1ull << 27;  // candidates whose lookups are kept (1.5 GB)

struct SetsView {
    const unsigned long long *off;         // [R + 1]
    const uint32_t *items;
    const uint32_t *sup;                   // [R]
    const unsigned long long *size_start;  // [NSIZE]: first set with |set| >= l
    int64_t R;
};

// Set sizes do not decrease along the canonical order: size_start[l] is the
// first set index with size >= l (R if none).
__global__ void size_bounds_kernel(const unsigned long long *__restrict__ off, int64_t R,
                                   unsigned long long *__restrict__ size_start) {
    const int l = threadIdx.x;
    if (l >= NSIZE) return;
    int64_t lo = 0, hi = R;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)(off[mid + 1] - off[mid]) < l) lo = mid + 1;
        else hi = mid;
    }
    size_start[l] = (unsigned long long)lo;
}

// Compares a stored set of size |mask| with the subset of z picked by mask.
__device__ __forceinline__ int cmp_subset(const uint32_t *__restrict__ it, const uint32_t *__restrict__ zp,
                                          uint32_t mask) {
    int k = 0;
    for (uint32_t mm = mask; mm; mm &= mm - 1) {
        const uint32_t a = it[k++], b = __ldg(zp + (__ffs(mm) - 1));
        if (a != b) return a < b ? -1 : 1;
    }
    return 0;
}

// Index of the subset of z (items at zp, ascending) picked by mask, or -1.
__device__ __forceinline__ int64_t find_subset(const SetsView &v, const uint32_t *zp, uint32_t mask) {
    const int ls = __popc(mask);
    int64_t lo = (int64_t)v.size_start[ls], hi = (int64_t)v.size_start[ls + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int c = cmp_subset(v.items + v.off[mid], zp, mask);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1;
        else hi = mid;
    }
    return -1;
}

// The set of evaluation e < E = ebase[R]: the last z with ebase[z] <= e.
__device__ __forceinline__ int64_t set_of_eval(const unsigned long long *__restrict__ ebase, int64_t R,
                                               unsigned long long e) {
    int64_t lo = 0, hi = R;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (ebase[mid] <= e) lo = mid + 1;
        else hi = mid;
    }
    return lo - 1;
}

struct Eval {
    int64_t z, rx, ry;
    uint32_t mask;
    uint64_t sz, sx, sy;
    bool ok;  // both subsets found
};

// The three set indices of a kept candidate, carried from the keep pass to the
// write pass when the scratch fits (12 bytes per candidate).
struct RuleSets {
    uint32_t z, x, y;
};

__device__ __forceinline__ Eval evaluate(const SetsView &v, const unsigned long long *__restrict__ ebase,
                                         unsigned long long e) {
    Eval r;
    r.z = set_of_eval(ebase, v.R, e);
    const unsigned long long o = v.off[r.z];
    const int L = (int)(v.off[r.z + 1] - o);
    const uint32_t full = (1u << L) - 1u;
    r.mask = (uint32_t)(e - ebase[r.z]) + 1u;
    const uint32_t *zp = v.items + o;
    r.rx = find_subset(v, zp, r.mask);
    r.ry = find_subset(v, zp, full & ~r.mask);
    r.ok = r.rx >= 0 && r.ry >= 0;
    r.sz = v.sup[r.z];
    r.sx = r.ok ? v.sup[r.rx] : 1;
    r.sy = r.ok ? v.sup[r.ry] : 1;
    return r;
}

// Candidate rules of a set: 2^L - 2 for 2 <= L <= max_len, else none.
struct SetEvals {
    const unsigned long long *off;
    int max_len;
    __device__ __forceinline__ unsigned long long operator()(unsigned long long i) const {
        const int L = (int)(off[i + 1] - off[i]);
        return (L >= 2 && L <= max_len) ? (1ull << L) - 2ull : 0ull;
    }
};

struct WordPop {
    const uint32_t *bits;
    __device__ __forceinline__ unsigned long long operator()(unsigned long long i) const {
        return (unsigned long long)__popc(bits[i]);
    }
};

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive scan of src(0 .. n-1) into out[0 .. n], out[n] = total, in three
// launches: chunk sums, a scan of the chunk sums in one CTA, a rescan of every
// chunk from its base.
template <class Src>
__global__ void __launch_bounds__(SCAN_T)
scan_sum_kernel(Src src, unsigned long long n, unsigned long long *__restrict__ part) {
    __shared__ unsigned long long s[SCAN_T / 32];
    const unsigned long long b = (unsigned long long)blockIdx.x * SCAN_CHUNK + (unsigned long long)threadIdx.x * SCAN_I;
    unsigned long long v = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; i++)
        if (b + i < n) v += src(b + i);
    v = warp_sum_u64(v);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long t = s[threadIdx.x];
        t = warp_sum_u64(t);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024)
scan_part_kernel(unsigned long long *__restrict__ part, unsigned long long np) {
    __shared__ unsigned long long s[1024];
    const unsigned long long seg = (np + 1023) / 1024;
    const unsigned long long b = threadIdx.x * seg, e = b + seg < np ? b + seg : np;
    unsigned long long sum = 0;
    for (unsigned long long i = b; i < e; i++) sum += part[i];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const unsigned long long v = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0ull;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = s[threadIdx.x] - sum;
    for (unsigned long long i = b; i < e; i++) {
        const unsigned long long v = part[i];
        part[i] = run;
        run += v;
    }
    if (threadIdx.x == 1023) part[np] = s[1023];
}

template <class Src>
__global__ void __launch_bounds__(SCAN_T)
scan_out_kernel(Src src, unsigned long long n, const unsigned long long *__restrict__ part,
                unsigned long long *__restrict__ out) {
    __shared__ unsigned long long s[SCAN_T / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long b = (unsigned long long)blockIdx.x * SCAN_CHUNK + (unsigned long long)threadIdx.x * SCAN_I;
    unsigned long long v[SCAN_I], sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; i++) {
        v[i] = b + i < n ? src(b + i) : 0ull;
        sum += v[i];
    }
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long acc = part[blockIdx.x];
        for (int w = 0; w < SCAN_T / 32; w++) {
            const unsigned long long t = s[w];
            s[w] = acc;
            acc += t;
        }
    }
    __syncthreads();
    unsigned long long run = s[warp] + x - sum;
#pragma unroll
    for (int i = 0; i < SCAN_I; i++) {
        if (b + i < n) out[b + i] = run;
        run += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = part[gridDim.x];
}

// One thread per evaluation; warp w of the grid-stride loop owns evaluations
// [32w, 32w + 32) and stores their keep bits as one word.
__global__ void __launch_bounds__(RT)
rule_keep_kernel(SetsView v, const unsigned long long *__restrict__ ebase, unsigned long long E, uint32_t ppm,
                 uint32_t *__restrict__ keep_bits, RuleSets *__restrict__ sets, int *__restrict__ err) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = (E + 31) / 32;
    const unsigned long long tw = (unsigned long long)gridDim.x * (RT / 32);
    for (unsigned long long w = ((unsigned long long)blockIdx.x * RT + threadIdx.x) >> 5; w < nw; w += tw) {
        const unsigned long long e = w * 32 + lane;
        bool keep = false;
        if (e < E) {
            const Eval r = evaluate(v, ebase, e);
            if (!r.ok) atomicExch(err, 1);  // a subset is missing: not a mine's output
            else keep = r.sz * 1000000ull >= (uint64_t)ppm * r.sx;
            if (keep && sets) sets[e] = RuleSets{(uint32_t)r.z, (uint32_t)r.rx, (uint32_t)r.ry};
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) keep_bits[w] = bal;
    }
}

__global__ void __launch_bounds__(RT)
rule_write_kernel(SetsView v, const unsigned long long *__restrict__ ebase, unsigned long long E, uint64_t n,
                  const uint32_t *__restrict__ keep_bits, const unsigned long long *__restrict__ kbase,
                  const RuleSets *__restrict__ sets, unsigned long long *__restrict__ set_index,
                  uint32_t *__restrict__ ante_mask, double *__restrict__ conf, double *__restrict__ lift) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = (E + 31) / 32;
    const unsigned long long tw = (unsigned long long)gridDim.x * (RT / 32);
    const uint32_t lt = (1u << lane) - 1u;
    for (unsigned long long w = ((unsigned long long)blockIdx.x * RT + threadIdx.x) >> 5; w < nw; w += tw) {
        const uint32_t bits = keep_bits[w];
        if (!((bits >> lane) & 1u)) continue;
        const unsigned long long e = w * 32 + lane;
        int64_t z;
        uint32_t mask;
        uint64_t sz, sx, sy;
        if (sets) {  // the keep pass's lookups
            const RuleSets q = sets[e];
            z = q.z;
            mask = (uint32_t)(e - ebase[z]) + 1u;
            sz = v.sup[q.z];
            sx = v.sup[q.x];
            sy = v.sup[q.y];
        } else {
            const Eval r = evaluate(v, ebase, e);
            z = r.z;
            mask = r.mask;
            sz = r.sz;
            sx = r.sx;
            sy = r.sy;
        }
        const unsigned long long at = kbase[w] + __popc(bits & lt);
        set_index[at] = (unsigned long long)z;
        ante_mask[at] = mask;
        conf[at] = (double)sz / (double)sx;
        lift[at] = (double)(sz * n) / (double)(sx * sy);
    }
}

template <class Src>
int scan_into(fim_ctx *ctx, Src src, unsigned long long n, unsigned long long *out) {
    const unsigned long long np = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    FIM_TRY(fim_reserve(ctx, ctx->rule_part, sizeof(unsigned long long) * (size_t)(np + 1)));
    unsigned long long *part = ctx->rule_part.as<unsigned long long>();
    cudaStream_t st = ctx->stream;
    ctx->launches += 3;
    scan_sum_kernel<<<(unsigned)np, SCAN_T, 0, st>>>(src, n, part);
    scan_part_kernel<<<1, 1024, 0, st>>>(part, np);
    scan_out_kernel<<<(unsigned)np, SCAN_T, 0, st>>>(src, n, part, out);
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

}  // namespace

extern "C" {

int fim_rules(fim_ctx *ctx, uint32_t min_conf_ppm, int max_len, uint64_t *n_rules) {
    FIM_NVTX("fim_rules");
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
    ctx->rules_evaluated = 0;
    if (R > 0) {
        // ebase [R + 1], then size_start [NSIZE]
        FIM_TRY(fim_reserve(ctx, ctx->rule_base, sizeof(unsigned long long) * (size_t)(R + 1 + NSIZE)));
        unsigned long long *ebase = ctx->rule_base.as<unsigned long long>(), *size_start = ebase + R + 1;
        const SetsView v{ctx->out_off.as<unsigned long long>(), ctx->out_items.as<uint32_t>(),
                         ctx->out_sup.as<uint32_t>(), size_start, R};
        ctx->launches++;
        size_bounds_kernel<<<1, NSIZE, 0, st>>>(v.off, R, size_start);
        FIM_TRY(scan_into(ctx, SetEvals{v.off, max_len}, (unsigned long long)R, ebase));
        unsigned long long E = 0;
        FIM_CUDA_TRY(cudaMemcpyAsync(&E, ebase + R, sizeof(E), cudaMemcpyDeviceToHost, st));
        FIM_CUDA_TRY(cudaStreamSynchronize(st));
        ctx->rules_evaluated = E;
        if (E > 0) {
            const unsigned long long nw = (E + 31) / 32;
            FIM_TRY(fim_reserve(ctx, ctx->rule_bits, sizeof(uint32_t) * (size_t)nw));
            FIM_TRY(fim_reserve(ctx, ctx->rule_kbase, sizeof(unsigned long long) * (size_t)(nw + 1)));
            uint32_t *bits = ctx->rule_bits.as<uint32_t>();
            unsigned long long *kbase = ctx->rule_kbase.as<unsigned long long>();
            int *err = ctx->dev_flag.as<int>() + 2;
            FIM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
            RuleSets *sets = nullptr;
            if (E <= kRuleSetsMax && (unsigned long long)R <= 0xFFFFFFFFull) {
                FIM_TRY(fim_reserve(ctx, ctx->rule_sets, sizeof(RuleSets) * (size_t)E));
                sets = ctx->rule_sets.as<RuleSets>();
            }
            const unsigned long long want = (nw + RT / 32 - 1) / (RT / 32);
            const unsigned long long cap = (unsigned long long)(ctx->num_sms > 0 ? ctx->num_sms : 1) * 8ull;  // 2,048 threads per SM
            const unsigned grid = (unsigned)(want < cap ? want : cap);
            ctx->launches++;
            rule_keep_kernel<<<grid, RT, 0, st>>>(v, ebase, E, min_conf_ppm, bits, sets, err);
            FIM_CUDA_TRY(cudaGetLastError());
            FIM_TRY(scan_into(ctx, WordPop{bits}, nw, kbase));
            unsigned long long total = 0;
            int bad = 0;
            FIM_CUDA_TRY(cudaMemcpyAsync(&total, kbase + nw, sizeof(total), cudaMemcpyDeviceToHost, st));
            FIM_CUDA_TRY(cudaMemcpyAsync(&bad, err, sizeof(int), cudaMemcpyDeviceToHost, st));
            FIM_CUDA_TRY(cudaStreamSynchronize(st));
            if (bad) return FIM_E_STATE;  // the held sets are not downward closed
            if (total) {
                FIM_TRY(fim_reserve(ctx, ctx->rule_set, sizeof(unsigned long long) * (size_t)total));
                FIM_TRY(fim_reserve(ctx, ctx->rule_mask, sizeof(uint32_t) * (size_t)total));
                FIM_TRY(fim_reserve(ctx, ctx->rule_conf, sizeof(double) * (size_t)total));
                FIM_TRY(fim_reserve(ctx, ctx->rule_lift, sizeof(double) * (size_t)total));
                ctx->launches++;
                rule_write_kernel<<<grid, RT, 0, st>>>(v, ebase, E, (uint64_t)ctx->out_n, bits, kbase, sets,
                                                       ctx->rule_set.as<unsigned long long>(),
                                                       ctx->rule_mask.as<uint32_t>(), ctx->rule_conf.as<double>(),
                                                       ctx->rule_lift.as<double>());
                FIM_CUDA_TRY(cudaGetLastError());
                FIM_CUDA_TRY(cudaStreamSynchronize(st));
            }
            ctx->rules_n = total;
        }
    }
    ctx->rules_of = ctx->mine_serial;
    if (ctx->bytes_held > ctx->stats.peak_device_bytes) ctx->stats.peak_device_bytes = ctx->bytes_held;
    *n_rules = ctx->rules_n;
    return FIM_OK;
}

int fim_rules_evaluated(const fim_ctx *ctx, uint64_t *n_evaluated) {
    FIM_NVTX("fim_rules_evaluated");
    if (!ctx || !n_evaluated) return FIM_E_INVAL;
    if (!ctx->mined || ctx->rules_of != ctx->mine_serial) return FIM_E_STATE;
    *n_evaluated = ctx->rules_evaluated;
    return FIM_OK;
}

int fim_fetch_rules(fim_ctx *ctx, uint64_t *n_rules, uint64_t *set_index, uint32_t *ante_mask, double *conf,
                    double *lift, uint64_t cap, uint32_t flags) {
    FIM_NVTX("fim_fetch_rules");
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
