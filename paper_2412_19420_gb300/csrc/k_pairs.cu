// k_pairs.cu -- pair supports S(I_a n I_b) = sum_i M[i,a] AND M[i,b] (Eq. 2)
// for all frequent items a < b, i.e. the upper triangle of C = A^T A where A
// is the n x m' 0/1 matrix of frequent columns, then the threshold (Eq. 3).
//
// pairs_popc_kernel: exact CUDA-core path.  A CTA owns a 64x64 tile of
// (a, b) and a slice of the words; operands are 32 words of 64 columns each,
// staged in shared memory, and every thread accumulates a 4x4 block of
// popc(a_word AND b_word).  Split-K partial sums meet in pair_cnt by atomicAdd.
// (The tensor-core path lives in k_pairs_tc.cu.)
//
// pairs_finalize_kernel: threshold every S(ab); set the pair bit, emit the
// frequent pair as a result record, and list it as a root prefix class.
#include "fim_common.cuh"

namespace {

constexpr int TI = 64;   // items per tile side
constexpr int KW = 32;   // words per k-step
constexpr int PT = 256;  // threads

__global__ void __launch_bounds__(PT)
pairs_popc_kernel(const uint32_t *__restrict__ bm, const int32_t *__restrict__ perm, int64_t nwp,
                  int64_t nw, int mf, int nt, int64_t words_per_split, int *__restrict__ pair_cnt) {
    __shared__ __align__(16) uint32_t As[KW][TI];
    __shared__ __align__(16) uint32_t Bs[KW][TI];
    // upper-triangle tile (ta <= tb) from the linear block index
    int idx = blockIdx.x, ta = 0;
    while (idx >= nt - ta) { idx -= nt - ta; ta++; }
    const int tb = ta + idx;
    const int64_t k0 = (int64_t)blockIdx.y * words_per_split;
    const int64_t k1 = min64(nw, k0 + words_per_split);
    if (k0 >= k1) return;

    const int t = threadIdx.x;
    const int lr = t & 63;           // loader: row within tile
    const int lc = (t >> 6) * 8;     // loader: 8 words starting here
    const int ra = ta * TI + lr, rb = tb * TI + lr;
    const uint32_t *pa = ra < mf ? bm + (int64_t)perm[ra] * nwp : nullptr;
    const uint32_t *pb = rb < mf ? bm + (int64_t)perm[rb] * nwp : nullptr;
    const int ty = t >> 4, tx = t & 15;
    uint32_t acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0;

    for (int64_t k = k0; k < k1; k += KW) {
        // columns are padded to a multiple of 128 words with zeros, so whole
        // 8-word runs past nw read zeros rather than out of bounds
        uint4 a0 = make_uint4(0, 0, 0, 0), a1 = a0, b0 = a0, b1 = a0;
        if (pa) { a0 = ldg_u4(pa + k + lc); a1 = ldg_u4(pa + k + lc + 4); }
        if (pb) { b0 = ldg_u4(pb + k + lc); b1 = ldg_u4(pb + k + lc + 4); }
        __syncthreads();
        As[lc + 0][lr] = a0.x; As[lc + 1][lr] = a0.y; As[lc + 2][lr] = a0.z; As[lc + 3][lr] = a0.w;
        As[lc + 4][lr] = a1.x; As[lc + 5][lr] = a1.y; As[lc + 6][lr] = a1.z; As[lc + 7][lr] = a1.w;
        Bs[lc + 0][lr] = b0.x; Bs[lc + 1][lr] = b0.y; Bs[lc + 2][lr] = b0.z; Bs[lc + 3][lr] = b0.w;
        Bs[lc + 4][lr] = b1.x; Bs[lc + 5][lr] = b1.y; Bs[lc + 6][lr] = b1.z; Bs[lc + 7][lr] = b1.w;
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < KW; kk++) {
            uint4 a = *reinterpret_cast<const uint4 *>(&As[kk][ty * 4]);
            uint4 b = *reinterpret_cast<const uint4 *>(&Bs[kk][tx * 4]);
            uint32_t av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] += __popc(av[i] & bv[j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int a = ta * TI + ty * 4 + i, b = tb * TI + tx * 4 + j;
            if (a < b && b < mf && acc[i][j]) atomicAdd(&pair_cnt[(int64_t)a * mf + b], (int)acc[i][j]);
        }
}

// One CTA per row a; warps sweep b in 32-wide words of the pair bitset.
__global__ void __launch_bounds__(256)
pairs_finalize_kernel(const int *__restrict__ pair_cnt, int mf, int mpw, uint32_t thr,
                      uint32_t *__restrict__ pairbits, MineCounters *ctr,
                      unsigned long long *rec_off, uint32_t *rec_len, uint32_t *rec_sup,
                      uint32_t *rec_items, unsigned long long rec_cap, unsigned long long items_cap,
                      uint32_t *root_a, uint32_t *root_b, uint32_t *root_sup, int emit, int emit_roots) {
    const int a = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int w = warp; w < mpw; w += nwarp) {
        const int b = w * 32 + lane;
        uint32_t s = 0;
        if (b > a && b < mf) s = (uint32_t)pair_cnt[(int64_t)a * mf + b];
        const bool f = b > a && b < mf && s >= thr;
        const uint32_t bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) pairbits[(int64_t)a * mpw + w] = bal;
        if (!emit || bal == 0) continue;
        const int cnt = __popc(bal);
        unsigned long long rbase = 0, ibase = 0, root = 0;
        if (lane == 0) {
            rbase = atomicAdd(&ctr->n_records, (unsigned long long)cnt);
            ibase = atomicAdd(&ctr->n_rec_items, 2ull * cnt);
            if (emit_roots) {
                root = atomicAdd(&ctr->n_roots, (unsigned long long)cnt);
                atomicAdd((unsigned long long *)&ctr->pending, (unsigned long long)cnt);
            }
        }
        rbase = __shfl_sync(0xffffffffu, rbase, 0);
        ibase = __shfl_sync(0xffffffffu, ibase, 0);
        root = __shfl_sync(0xffffffffu, root, 0);
        if (f) {
            const int pos = __popc(bal & ((1u << lane) - 1));
            const unsigned long long r = rbase + pos, it = ibase + 2ull * pos;
            if (r < rec_cap && it + 2 <= items_cap) {
                rec_off[r] = it;
                rec_len[r] = 2;
                rec_sup[r] = s;
                rec_items[it] = (uint32_t)a;
                rec_items[it + 1] = (uint32_t)b;
            } else {
                atomicOr(&ctr->overflow, r < rec_cap ? 2 : 1);
            }
            if (emit_roots) {
                root_a[root + pos] = (uint32_t)a;
                root_b[root + pos] = (uint32_t)b;
                root_sup[root + pos] = s;
            }
        }
    }
}

}  // namespace

int launch_pairs_popc(fim_ctx *ctx) {
    const int mf = ctx->mfreq;
    if (mf < 2) return FIM_OK;
    const int nt = (int)ceil_div64(mf, TI);
    const int tiles = nt * (nt + 1) / 2;
    const int64_t ksteps = ceil_div64(ctx->nw, KW);
    int64_t split = ceil_div64(4LL * ctx->num_sms, tiles);
    if (split > ksteps) split = ksteps;
    if (split < 1) split = 1;
    const int64_t wps = ceil_div64(ksteps, split) * KW;
    split = ceil_div64(ctx->nw, wps);
    FIM_CUDA_TRY(cudaMemsetAsync(ctx->pair_cnt.p, 0, sizeof(int) * (size_t)mf * mf, ctx->stream));
    if (split > 0) {
        dim3 grid((unsigned)tiles, (unsigned)split);
        ctx->launches++;
        pairs_popc_kernel<<<grid, PT, 0, ctx->stream>>>(ctx->bm.as<uint32_t>(), ctx->perm.as<int32_t>(),
                                                         ctx->nwp, ctx->nw, mf, nt, wps,
                                                         ctx->pair_cnt.as<int>());
        FIM_CUDA_TRY(cudaGetLastError());
    }
    return FIM_OK;
}

int launch_pairs_finalize(fim_ctx *ctx, uint32_t thr, MineCounters *d_ctr) {
    const int mf = ctx->mfreq;
    if (mf < 2) return FIM_OK;
    const int mpw = (int)ceil_div64(mf, 32);
    uint32_t *roots = ctx->roots.as<uint32_t>();
    const size_t npairs = (size_t)mf * (mf - 1) / 2;
    ctx->launches++;
    pairs_finalize_kernel<<<mf, 256, 0, ctx->stream>>>(
        ctx->pair_cnt.as<int>(), mf, mpw, thr, ctx->pairbits.as<uint32_t>(), d_ctr,
        ctx->rec_off.as<unsigned long long>(), ctx->rec_len.as<uint32_t>(),
        ctx->rec_sup.as<uint32_t>(), ctx->rec_items.as<uint32_t>(), ctx->rec_cap,
        ctx->rec_items_cap, roots, roots + npairs, roots + 2 * npairs,
        ctx->shard == 0 && ((ctx->mflags & FIM_MAXLEN(0xff)) == 0 || (ctx->mflags >> 24) >= 2),
        ctx->n_shards == 1);
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}
