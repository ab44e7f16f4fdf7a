// k_shard.cu -- prefix-class sharding of one mine over several GPUs, and the
// merge of the shards' outputs.
//
// The decomposition: after the pair pass every frequent pair {a, b} (a < b,
// internal ids) roots an independent prefix class whose members are the
// frequent sets with smallest two items a, b; the classes partition the sets
// of size >= 3.  Shard s of N mines the classes it owns; shard 0 also emits
// the singletons and pairs.  The union of the N outputs is the full answer,
// with no set in two shards.
//
// Ownership must come out the same on every GPU without communication, so it
// is a function of integers every shard computes identically (the pair
// bitsets): the roots, numbered in (a, b) order, are dealt round-robin --
// root number P belongs to shard P mod N.  Contiguous ranges of equal
// estimated cost balanced the estimate but not the work: a planted pattern's
// heavy classes sit next to each other in (a, b) order, and on a 10^5 x 2,000
// planted workload one of 8 ranges held 94% of the sets of size >= 3.  No
// single class holds more than a few percent there, so dealing the roots out
// one by one spreads them: the largest of 8 shards then holds 13-16% of those
// sets (ideal 12.5%) on the Quest-style and planted workloads alike.
//
// The merge concatenates the shards' canonical lists (caller item ids) into
// the record pool and re-runs the compactor's sort with the identity item
// map, so the merged list is canonical again.
#include "fim_common.cuh"

namespace {

constexpr int SH_T = 256;

__device__ __forceinline__ bool pair_frequent(const uint32_t *__restrict__ pairbits, int mpw, int a, int b) {
    return (pairbits[(int64_t)a * mpw + (b >> 5)] >> (b & 31)) & 1u;
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long *red) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0;
    for (int w = 0; w < SH_T / 32; w++) t += red[w];
    __syncthreads();
    return t;
}

// One CTA per row a: rowcount[a] = number of roots (a, b), i.e. of frequent
// pairs in row a of the pair bitsets.
__global__ void __launch_bounds__(SH_T)
row_count_kernel(const uint32_t *__restrict__ pairbits, int mf, int mpw, unsigned long long *__restrict__ rowcount) {
    __shared__ unsigned long long red[SH_T / 32];
    const int a = blockIdx.x;
    unsigned long long v = 0;
    for (int w = threadIdx.x; w < mpw; w += SH_T) v += (unsigned long long)__popc(pairbits[(int64_t)a * mpw + w]);
    v = block_sum_u64(v, red);
    if (threadIdx.x == 0) rowcount[a] = v;
}

// Exclusive scan of rowcount[0 .. mf) into rowbase, rowbase[mf] = the number
// of roots (one CTA).
__global__ void __launch_bounds__(1024)
row_scan_kernel(const unsigned long long *__restrict__ rowcount, int mf, unsigned long long *__restrict__ rowbase) {
    __shared__ unsigned long long s[1024];
    const int seg = (mf + 1023) / 1024;
    const int b = threadIdx.x * seg, e = b + seg < mf ? b + seg : mf;
    unsigned long long sum = 0;
    for (int i = b; i < e; i++) sum += rowcount[i];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const unsigned long long v = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0ull;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = s[threadIdx.x] - sum;
    for (int i = b; i < e; i++) {
        rowbase[i] = run;
        run += rowcount[i];
    }
    if (threadIdx.x == 1023) rowbase[mf] = s[1023];
}

// One CTA per row a: walks b ascending in blocks of SH_T, numbers every root
// in (a, b) order, and appends the roots this shard owns (number mod N).
__global__ void __launch_bounds__(SH_T)
shard_roots_kernel(const uint32_t *__restrict__ pairbits, const int *__restrict__ pair_cnt, int mf, int mpw,
                   const unsigned long long *__restrict__ rowbase, int shard, int n_shards, MineCounters *ctr,
                   uint32_t *__restrict__ root_a, uint32_t *__restrict__ root_b, uint32_t *__restrict__ root_sup) {
    __shared__ unsigned long long wsum[SH_T / 32];
    const int a = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long run = rowbase[a];
    for (int b0 = a + 1; b0 < mf; b0 += SH_T) {
        const int b = b0 + threadIdx.x;
        const bool f = b < mf && pair_frequent(pairbits, mpw, a, b);
        const unsigned long long c = f ? 1ull : 0ull;
        // block exclusive scan of c in thread order (= b order)
        unsigned long long x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        unsigned long long before = 0, total = 0;
        for (int w = 0; w < SH_T / 32; w++) {
            if (w < warp) before += wsum[w];
            total += wsum[w];
        }
        __syncthreads();
        const unsigned long long P = run + before + x - c;  // the root's number in (a, b) order
        const bool own = f && P % (unsigned long long)n_shards == (unsigned long long)shard;
        const uint32_t bal = __ballot_sync(0xffffffffu, own);
        if (bal) {
            unsigned long long base = 0;
            if (lane == 0) {
                base = atomicAdd(&ctr->n_roots, (unsigned long long)__popc(bal));
                atomicAdd((unsigned long long *)&ctr->pending, (unsigned long long)__popc(bal));
            }
            base = __shfl_sync(0xffffffffu, base, 0);
            if (own) {
                const unsigned long long at = base + __popc(bal & ((1u << lane) - 1u));
                root_a[at] = (uint32_t)a;
                root_b[at] = (uint32_t)b;
                root_sup[at] = (uint32_t)pair_cnt[(int64_t)a * mf + b];
            }
        }
        run += total;
    }
}

// ---- merge ------------------------------------------------------------------

// Records of one part: rec_off = item_base + off[i], rec_len = off[i+1] - off[i];
// checks off[0] == 0, non-decreasing offsets, 1 <= len <= 255, off[n] == n_items.
__global__ void merge_records_kernel(const unsigned long long *__restrict__ off, unsigned long long n,
                                     unsigned long long n_items, unsigned long long set_base,
                                     unsigned long long item_base, unsigned long long *__restrict__ rec_off,
                                     uint32_t *__restrict__ rec_len, int *__restrict__ flag) {
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (off[0] != 0ull || off[n] != n_items)) atomicExch(flag, 1);
    if (i >= n) return;
    const unsigned long long o = off[i], e = off[i + 1];
    if (e <= o || e - o > 255ull || e > n_items) {
        atomicExch(flag, 1);
        return;
    }
    rec_off[set_base + i] = item_base + o;
    rec_len[set_base + i] = (uint32_t)(e - o);
    atomicMax(flag + 1, (int)(e - o));
}

__global__ void check_items_kernel(const uint32_t *__restrict__ items, unsigned long long n, uint32_t m,
                                   int *__restrict__ flag) {
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        if (items[i] >= m) atomicExch(flag, 1);
}

}  // namespace

int launch_shard_roots(fim_ctx *ctx, MineCounters *d_ctr, int shard, int n_shards) {
    const int mf = ctx->mfreq;
    if (mf < 2) return FIM_OK;
    const int mpw = (int)ceil_div64(mf, 32);
    const size_t npairs = (size_t)mf * (mf - 1) / 2;
    FIM_TRY(fim_reserve(ctx, ctx->shard_cost, sizeof(unsigned long long) * (size_t)(2 * mf + 1)));
    unsigned long long *rowcount = ctx->shard_cost.as<unsigned long long>(), *rowbase = rowcount + mf;
    uint32_t *roots = ctx->roots.as<uint32_t>();
    cudaStream_t st = ctx->stream;
    const uint32_t *pb = ctx->pairbits.as<uint32_t>();
    ctx->launches += 3;
    row_count_kernel<<<mf, SH_T, 0, st>>>(pb, mf, mpw, rowcount);
    row_scan_kernel<<<1, 1024, 0, st>>>(rowcount, mf, rowbase);
    shard_roots_kernel<<<mf, SH_T, 0, st>>>(pb, ctx->pair_cnt.as<int>(), mf, mpw, rowbase, shard, n_shards, d_ctr,
                                            roots, roots + npairs, roots + 2 * npairs);
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

extern "C" {

int fim_merge_results(fim_ctx *ctx, int64_t n_trans, int32_t n_items, int n_parts, const uint64_t *n_sets,
                      const uint64_t *n_items_total, const uint64_t *const *offsets, const uint32_t *const *items,
                      const uint32_t *const *supports, uint32_t flags) {
    FIM_NVTX("fim_merge_results");
    if (!ctx || n_parts < 1 || !n_sets || !n_items_total || !offsets || !items || !supports) return FIM_E_INVAL;
    FIM_TRY(fim_finish_phase_times(ctx));  // before the events are recorded again
    if (n_trans < 0 || n_trans > FIM_MAX_TRANS || n_items < 0 || n_items > FIM_MAX_ITEMS) return FIM_E_INVAL;
    unsigned long long R = 0, T = 0;
    for (int p = 0; p < n_parts; p++) {
        if (!offsets[p] || (n_sets[p] && (!supports[p] || !items[p]))) return FIM_E_INVAL;
        if (n_items_total[p] < n_sets[p]) return FIM_E_INVAL;  // every set has an item
        R += n_sets[p];
        T += n_items_total[p];
    }
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FIM_E_CUDA;
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{dev_prev};
    cudaStream_t st = ctx->stream;
    ctx->mined = false;
    const uint64_t launches0 = ctx->launches;
    const cudaMemcpyKind k = (flags & FIM_INPUT_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (R > ctx->rec_cap) ctx->rec_cap = R;
    if (T > ctx->rec_items_cap) ctx->rec_items_cap = T;
    if (ctx->rec_cap == 0) ctx->rec_cap = 1;
    if (ctx->rec_items_cap == 0) ctx->rec_items_cap = 1;
    FIM_TRY(fim_reserve(ctx, ctx->rec_off, sizeof(unsigned long long) * ctx->rec_cap));
    FIM_TRY(fim_reserve(ctx, ctx->rec_len, sizeof(uint32_t) * ctx->rec_cap));
    FIM_TRY(fim_reserve(ctx, ctx->rec_sup, sizeof(uint32_t) * ctx->rec_cap));
    FIM_TRY(fim_reserve(ctx, ctx->rec_items, sizeof(uint32_t) * ctx->rec_items_cap));
    FIM_TRY(fim_reserve(ctx, ctx->rec_db, sizeof(uint32_t) * ctx->rec_cap));
    FIM_TRY(fim_reserve(ctx, ctx->dev_flag, 4 * sizeof(int)));
    int *flag = ctx->dev_flag.as<int>();
    FIM_CUDA_TRY(cudaMemsetAsync(flag, 0, 2 * sizeof(int), st));
    unsigned long long sb = 0, ib = 0;
    for (int p = 0; p < n_parts; p++) {
        const unsigned long long np = n_sets[p], ni = n_items_total[p];
        const unsigned long long *d_off = reinterpret_cast<const unsigned long long *>(offsets[p]);
        if (!(flags & FIM_INPUT_DEVICE)) {  // stage host offsets
            FIM_TRY(fim_reserve(ctx, ctx->merge_off, sizeof(unsigned long long) * (size_t)(np + 1)));
            FIM_CUDA_TRY(cudaMemcpyAsync(ctx->merge_off.p, offsets[p], sizeof(uint64_t) * (np + 1), k, st));
            d_off = ctx->merge_off.as<unsigned long long>();
        }
        if (ni) FIM_CUDA_TRY(cudaMemcpyAsync(ctx->rec_items.as<uint32_t>() + ib, items[p], sizeof(uint32_t) * ni, k, st));
        if (np) FIM_CUDA_TRY(cudaMemcpyAsync(ctx->rec_sup.as<uint32_t>() + sb, supports[p], sizeof(uint32_t) * np, k, st));
        ctx->launches++;
        merge_records_kernel<<<(unsigned)ceil_div64((int64_t)(np ? np : 1), 256), 256, 0, st>>>(
            d_off, np, ni, sb, ib, ctx->rec_off.as<unsigned long long>(), ctx->rec_len.as<uint32_t>(), flag);
        FIM_CUDA_TRY(cudaGetLastError());
        if (!(flags & FIM_INPUT_DEVICE)) FIM_CUDA_TRY(cudaStreamSynchronize(st));  // staging is reused
        sb += np;
        ib += ni;
    }
    if (T) {
        ctx->launches++;
        const unsigned long long want = (T + 255) / 256;
        check_items_kernel<<<(unsigned)(want < 4096 ? want : 4096), 256, 0, st>>>(ctx->rec_items.as<uint32_t>(), T,
                                                                               (uint32_t)n_items, flag);
        FIM_CUDA_TRY(cudaGetLastError());
    }
    int h[2] = {0, 0};
    FIM_CUDA_TRY(cudaMemcpyAsync(h, flag, sizeof(h), cudaMemcpyDeviceToHost, st));
    FIM_CUDA_TRY(cudaStreamSynchronize(st));
    if (h[0]) return FIM_E_INVAL;
    // the single-database table the compactor reads (item map: identity)
    ctx->host_db = DbDesc{};
    ctx->host_db.n = n_trans;
    ctx->host_db.m = n_items;
    FIM_TRY(fim_reserve(ctx, ctx->dbdesc, sizeof(DbDesc)));
    ctx->up_desc.clear();  // the batched mine's table is overwritten
    FIM_CUDA_TRY(cudaMemcpyAsync(ctx->dbdesc.p, &ctx->host_db, sizeof(DbDesc), cudaMemcpyHostToDevice, st));
    ctx->host_ctr = MineCounters{};
    ctx->host_ctr.n_records = R;
    ctx->host_ctr.n_rec_items = T;
    ctx->host_ctr.max_len = h[1];
    cudaEventRecord(ctx->ev[3], st);
    FIM_TRY(launch_compact(ctx, R, R, 1, n_items > 0 ? n_items : 1, /*identity_items=*/true));
    cudaEventRecord(ctx->ev[4], st);
    FIM_CUDA_TRY(cudaStreamSynchronize(st));
    FIM_CUDA_TRY(cudaGetLastError());
    cudaEventElapsedTime(&ctx->stats.ms_compact, ctx->ev[3], ctx->ev[4]);
    ctx->stats.n_sets = R;
    ctx->stats.max_len = (uint64_t)h[1];
    ctx->stats.launches_mine = ctx->launches - launches0;
    if (ctx->bytes_held > ctx->stats.peak_device_bytes) ctx->stats.peak_device_bytes = ctx->bytes_held;
    ctx->out_n = n_trans;
    ctx->mined = true;
    ctx->mine_serial++;
    return FIM_OK;
}

}  // extern "C"
