// k_matrix.cu -- matrix construction (Eq. 1) and singleton support (Eq. 3).
//
// build_bitmaps_kernel: one CTA owns a block of WB words (32*WB transactions)
// and a range of IB items.  Each warp streams a 32-row group's elements
// (coalesced) and ORs every (transaction, item) pair into a shared-memory
// tile with atomicOr -- OR makes repeated items idempotent, which is the set
// membership of Eq. 1 -- and the tile goes out as WB-word (64-byte) runs of
// each item column with 16-byte stores.  A 64-byte run keeps the tile at
// 64 KB for 1,024 items, so several CTAs share an SM.  The CTA also validates
// its slice of the CSR (monotone indptr, items in [0, m)).  CMP: the CSR is
// compact (uint32 row offsets, uint16 item ids) instead of int64 / int32.
#include <type_traits>

#include "fim_common.cuh"

namespace {

constexpr int WB = 16;          // words per CTA tile row (64 bytes)
constexpr int BUILD_THREADS = 512;

template <bool CMP>
__global__ void __launch_bounds__(BUILD_THREADS)
build_bitmaps_kernel(const void *__restrict__ indptr_v, const void *__restrict__ indices_v,
                     int64_t n, int32_t m, int64_t nnz, int64_t nwp, int ib, int64_t blk0,
                     uint32_t *__restrict__ bm, int *__restrict__ flag, int *__restrict__ max_len) {
    using Off = typename std::conditional<CMP, uint32_t, int64_t>::type;
    using Id = typename std::conditional<CMP, unsigned short, int32_t>::type;
    const Off *const indptr = static_cast<const Off *>(indptr_v);
    const Id *const indices = static_cast<const Id *>(indices_v);
    // [WB][ib + 1], word-major and padded: the 32 rows of a warp's group share
    // their word, so their items' bits spread over the banks
    extern __shared__ __align__(16) uint32_t tile[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ms = ib + 1;
    const int64_t w0 = (blk0 + (int64_t)blockIdx.x) * WB;
    const int i0 = blockIdx.y * ib;
    const int icount = min(ib, m - i0);
    const int64_t t0 = w0 * 32;
    const int64_t t1 = min(n, t0 + WB * 32);
    int bad = 0, my_max = 0;
    if (nnz < 0) {  // device input: indptr[n] read here, and indptr[0] checked once
        nnz = (int64_t)indptr[n];
        if (nnz < 0) bad = 1;
        if (blockIdx.x == 0 && blockIdx.y == 0 && blk0 == 0 && threadIdx.x == 0 && indptr[0] != 0) bad = 1;
    }

    for (int k = threadIdx.x; k < WB * ms; k += blockDim.x) tile[k] = 0u;
    __syncthreads();
    // warp w takes 32-row groups: lane i holds the group's start of row i, the
    // warp streams the group's elements 32 at a time (coalesced) and each
    // element finds its row by a binary search over the lanes' starts
    for (int64_t rb = t0 + 32 * warp; rb < t1; rb += 32 * (int64_t)(blockDim.x >> 5)) {
        const int nr = (int)min64(32, t1 - rb);
        const int64_t off = (int64_t)indptr[rb + (lane < nr ? lane : nr)];
        const int64_t e_end = (int64_t)indptr[rb + nr];
        int64_t off_next = __shfl_down_sync(0xffffffffu, off, 1);
        if (lane == nr - 1) off_next = e_end;
        if (lane < nr) {
            if (off_next < off || off < 0 || off_next > nnz) bad = 1;
            else my_max = max(my_max, (int)min64(off_next - off, 1 << 30));
        }
        if (__any_sync(0xffffffffu, bad)) continue;  // malformed: flagged, not read
        const int64_t e_begin = __shfl_sync(0xffffffffu, off, 0);
        const uint32_t wl = (uint32_t)((rb - t0) >> 5);
        for (int64_t e0 = e_begin; e0 < e_end; e0 += 32) {
            const int64_t e = e0 + lane;
            const bool v = e < e_end;
            const int32_t it = v ? (int32_t)indices[e] : 0;
            int r = 0;  // largest r < nr with start(r) <= e
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int c = r + step;
                const int64_t oc = __shfl_sync(0xffffffffu, off, c < 32 ? c : 31);
                if (c < nr && oc <= e) r = c;
            }
            if (!v) continue;
            if (it < 0 || it >= m) { bad = 1; continue; }
            if (it < i0 || it >= i0 + icount) continue;
            atomicOr(&tile[wl * ms + (it - i0)], 1u << r);
        }
    }
    if (bad) atomicExch(flag, 1);
    if (blockIdx.y == 0 && my_max > 0) atomicMax(max_len, my_max);
    __syncthreads();
    // write-out: 16-byte stores, four consecutive threads per 64-byte row
    for (int k = threadIdx.x; k < icount * (WB / 4); k += blockDim.x) {
        const int r = k / (WB / 4), c = k % (WB / 4);
        const uint4 v = make_uint4(tile[(4 * c + 0) * ms + r], tile[(4 * c + 1) * ms + r],
                                   tile[(4 * c + 2) * ms + r], tile[(4 * c + 3) * ms + r]);
        *reinterpret_cast<uint4 *>(bm + (int64_t)(i0 + r) * nwp + w0 + 4 * c) = v;
    }
}

// S(I_j) = popcount of column j, split over segments of SEG words.
constexpr int SEG = 8192;
__global__ void __launch_bounds__(256)
item_support_kernel(const uint32_t *__restrict__ bm, int64_t nwp, uint32_t *__restrict__ sup) {
    const int j = blockIdx.x;
    const int64_t b = (int64_t)blockIdx.y * SEG;
    const int64_t e = min64(nwp, b + SEG);
    const uint32_t *col = bm + (int64_t)j * nwp;
    uint32_t c = 0;
    for (int64_t w = b + 4 * threadIdx.x; w < e; w += 4 * blockDim.x) {
        uint4 v = ldg_u4(col + w);
        c += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
    }
    c = warp_sum_u32(c);
    __shared__ uint32_t s[8];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += s[k];
        if (t) atomicAdd(&sup[j], t);
    }
}

// Internal ids: frequent items ordered by (support, id) ascending.  One warp
// per item counts the frequent items with a smaller key (ties impossible).
__global__ void rank_items_kernel(const uint32_t *__restrict__ sup, int32_t m, uint32_t thr,
                                  int32_t *__restrict__ perm, int32_t *__restrict__ rank,
                                  MineCounters *ctr) {
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= m) return;
    const uint32_t sj = sup[j];
    if (sj < thr) {
        if (lane == 0) rank[j] = -1;
        return;
    }
    uint32_t below = 0;
    for (int i = lane; i < m; i += 32) {
        uint32_t si = sup[i];
        below += (si >= thr) && (si < sj || (si == sj && i < j));
    }
    below = warp_sum_u32(below);
    if (lane == 0) {
        rank[j] = (int32_t)below;
        perm[below] = j;
        atomicAdd(&ctr->m_freq, 1);
    }
}

// Singletons are the first m' records: record r = {r} with support S(perm[r]).
__global__ void emit_singletons_kernel(const uint32_t *__restrict__ sup, const int32_t *__restrict__ perm,
                                       MineCounters *ctr, unsigned long long *rec_off,
                                       uint32_t *rec_len, uint32_t *rec_sup, uint32_t *rec_items,
                                       unsigned long long rec_cap, unsigned long long items_cap) {
    const int mf = ctr->m_freq;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) {
        ctr->n_records = (unsigned long long)mf;
        ctr->n_rec_items = (unsigned long long)mf;
        if ((unsigned long long)mf > rec_cap) atomicOr(&ctr->overflow, 1);
        if ((unsigned long long)mf > items_cap) atomicOr(&ctr->overflow, 2);
    }
    if (r < mf && (unsigned long long)r < rec_cap && (unsigned long long)r < items_cap) {
        rec_off[r] = (unsigned long long)r;
        rec_len[r] = 1;
        rec_sup[r] = sup[perm[r]];
        rec_items[r] = (uint32_t)r;
    }
}

}  // namespace

int launch_build_bitmaps(fim_ctx *ctx, const void *d_indptr, const void *d_indices, int64_t nnz,
                         const void *h_indptr, const void *h_indices, bool cmp) {
    auto kern = cmp ? build_bitmaps_kernel<true> : build_bitmaps_kernel<false>;
    const size_t ib_bytes = csr_id_bytes(cmp);
    const int64_t nblk = ctx->nwp / WB;
    int ib = ctx->m < 1024 ? ctx->m : 1024;
    if (ib < 1) ib = 1;
    const int niblk = (int)ceil_div64(ctx->m > 0 ? ctx->m : 1, ib);
    const size_t smem = (size_t)(ib + 1) * WB * sizeof(uint32_t);
    FIM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int *flag = ctx->dev_flag.as<int>();
    cudaStream_t st = ctx->stream;
    FIM_CUDA_TRY(cudaMemsetAsync(flag, 0, 2 * sizeof(int), st));
    if (nblk <= 0 || ctx->m <= 0) return FIM_OK;
    // device input (nnz < 0): the kernel reads indptr[n] itself
    // Host input: the indices go up in chunks of row blocks on side streams,
    // and each chunk's blocks are built as soon as its copy has landed, so the
    // upload overlaps the construction.  A chunk needs the elements
    // [indptr[t0], indptr[t1]) of its transactions; an indptr that is not
    // monotone there is flagged by the kernel, which then reads nothing.
    int chunks = h_indices ? ctx->upload_chunks : 1;
    if (chunks > nblk) chunks = (int)nblk;
    if (chunks < 1) chunks = 1;
    const int nstreams = h_indices ? ctx->upload_streams : 0;
    for (int s = 0; s < nstreams; s++) {
        if (!ctx->up_stream[s]) FIM_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->up_stream[s], cudaStreamNonBlocking));
        // the copies overwrite the staging buffer: after all earlier work on the ctx stream
        FIM_CUDA_TRY(cudaStreamWaitEvent(ctx->up_stream[s], ctx->ev[0], 0));
    }
    for (int c = 0; c < chunks && h_indices; c++)
        if (!ctx->up_ev[c]) FIM_CUDA_TRY(cudaEventCreateWithFlags(&ctx->up_ev[c], cudaEventDisableTiming));
    const int64_t per = ceil_div64(nblk, chunks);
    const int64_t tpb = (int64_t)WB * 32;  // transactions per row block
    for (int c = 0; c < chunks; c++) {
        const int64_t b0 = (int64_t)c * per, b1 = min64(nblk, b0 + per);
        if (b0 >= b1) break;
        if (h_indices) {
            const int64_t t0 = min64(ctx->n, b0 * tpb), t1 = min64(ctx->n, b1 * tpb);
            int64_t lo = csr_off(h_indptr, cmp, t0), hi = csr_off(h_indptr, cmp, t1);
            lo = lo < 0 ? 0 : (lo > nnz ? nnz : lo);
            hi = hi < lo ? lo : (hi > nnz ? nnz : hi);
            if (hi > lo) {
                cudaStream_t cs = ctx->up_stream[c % nstreams];
                FIM_CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(const_cast<void *>(d_indices)) + ib_bytes * (size_t)lo,
                                             static_cast<const char *>(h_indices) + ib_bytes * (size_t)lo,
                                             ib_bytes * (size_t)(hi - lo), cudaMemcpyHostToDevice, cs));
                FIM_CUDA_TRY(cudaEventRecord(ctx->up_ev[c], cs));
                FIM_CUDA_TRY(cudaStreamWaitEvent(st, ctx->up_ev[c], 0));
            }
        }
        dim3 grid((unsigned)(b1 - b0), (unsigned)niblk);
        ctx->launches++;
        kern<<<grid, BUILD_THREADS, smem, st>>>(d_indptr, d_indices, ctx->n, ctx->m, nnz, ctx->nwp, ib, b0,
                                                ctx->bm.as<uint32_t>(), flag, flag + 1);
        FIM_CUDA_TRY(cudaGetLastError());
    }
    return FIM_OK;
}

int launch_item_support(fim_ctx *ctx) {
    uint32_t *sup = ctx->item_sup.as<uint32_t>();
    FIM_CUDA_TRY(cudaMemsetAsync(sup, 0, sizeof(uint32_t) * (size_t)ctx->m, ctx->stream));
    if (ctx->m == 0 || ctx->nwp == 0) return FIM_OK;
    dim3 grid((unsigned)ctx->m, (unsigned)ceil_div64(ctx->nwp, SEG));
    ctx->launches++;
    item_support_kernel<<<grid, 256, 0, ctx->stream>>>(ctx->bm.as<uint32_t>(), ctx->nwp, sup);
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

int launch_rank_items(fim_ctx *ctx, uint32_t thr, MineCounters *d_ctr) {
    if (ctx->m == 0) return FIM_OK;
    const int threads = 256;
    const int blocks = (int)ceil_div64((int64_t)ctx->m * 32, threads);
    ctx->launches++;
    rank_items_kernel<<<blocks, threads, 0, ctx->stream>>>(
        ctx->item_sup.as<uint32_t>(), ctx->m, thr, ctx->perm.as<int32_t>(),
        ctx->rank.as<int32_t>(), d_ctr);
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

int launch_emit_singletons(fim_ctx *ctx, MineCounters *d_ctr) {
    const int threads = 256;
    const int blocks = (int)ceil_div64(ctx->m > 0 ? ctx->m : 1, threads);
    ctx->launches++;
    emit_singletons_kernel<<<blocks, threads, 0, ctx->stream>>>(
        ctx->item_sup.as<uint32_t>(), ctx->perm.as<int32_t>(), d_ctr,
        ctx->rec_off.as<unsigned long long>(), ctx->rec_len.as<uint32_t>(),
        ctx->rec_sup.as<uint32_t>(), ctx->rec_items.as<uint32_t>(), ctx->rec_cap,
        ctx->rec_items_cap);
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}
