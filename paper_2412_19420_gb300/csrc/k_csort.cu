// k_csort.cu -- the compactor's sort for small outputs in one launch: a
// thread-block cluster keeps every key in distributed shared memory.
//
// The LSD radix sort of the compactor (8-bit digits of the big-endian
// (size, items) key, least significant first, stable) normally runs as a
// histogram / scan / scatter launch triple per digit.  For outputs of up to a
// few tens of thousands of sets those launches, not the bytes, set the time.
// Here one cluster of CL CTAs (16 where the GPU allows it) holds the records:
// CTA c owns global positions [c * per, c * per + per).  Per digit:
//   1. each CTA counts the digit over its records (shared-memory histogram);
//   2. cluster barrier; every CTA reads the CL histograms through distributed
//      shared memory and derives, per digit value, where its records go: all
//      records with a smaller digit, plus the same digit in lower CTAs;
//   3. each CTA ranks its records stably in tiles of 1,024 (warp match for
//      the rank among equal digits, per-warp counts for the warps before) and
//      stores each record (key words + record index) straight into the
//      shared memory of the CTA that owns its new position;
//   4. cluster barrier; the two record buffers swap roles.
// After the last digit, CTA c writes the record indices of its positions.
// Every CTA runs the same digit loop, so the barriers are always matched.
#include <cooperative_groups.h>

#include <utility>
#include <vector>

#include "fim_common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int CT = 1024;        // threads per CTA
constexpr int CS_MAXKW = 4;     // key words the cluster path takes
constexpr int CS_MAXPASS = 32;  // digit passes (<= 8 per key word)

struct CsPasses {
    int n;
    signed char word[CS_MAXPASS];
    signed char shift[CS_MAXPASS];
};

// Dynamic shared memory: keys A [kw][cap], keys B [kw][cap], idx A [cap],
// idx B [cap], then the fixed part (histogram, bases, per-warp counts).
struct CsFixed {
    uint32_t hist[256];
    uint32_t base[256];
    uint32_t tot[256];
    uint8_t wc[CT / 32][256];
};

size_t cs_smem(int kw, int cap) {
    return (size_t)cap * (2 * 8 * (size_t)kw + 2 * 4) + sizeof(CsFixed);
}

__global__ void __launch_bounds__(CT, 1)
cluster_sort_kernel(const unsigned long long *__restrict__ keys, unsigned long long R, int kw, int cap, int per,
                    CsPasses passes, uint32_t *__restrict__ idx_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int c = (int)cluster.block_rank();
    const int ncl = (int)cluster.num_blocks();
    unsigned long long *const kA = reinterpret_cast<unsigned long long *>(smem);
    unsigned long long *const kB = kA + (size_t)kw * cap;
    uint32_t *const iA = reinterpret_cast<uint32_t *>(kB + (size_t)kw * cap);
    uint32_t *const iB = iA + cap;
    CsFixed &f = *reinterpret_cast<CsFixed *>(iB + cap);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    const long long my0 = (long long)c * per;
    long long rem = (long long)R - my0;
    const int myn = rem <= 0 ? 0 : (rem < per ? (int)rem : per);
    for (int i = tid; i < myn; i += CT) {
        for (int w = 0; w < kw; w++) kA[(size_t)w * cap + i] = keys[(size_t)w * R + (size_t)(my0 + i)];
        iA[i] = (uint32_t)(my0 + i);
    }
    int cur = 0;
    for (int p = 0; p < passes.n; p++) {
        const int w = passes.word[p], sh = passes.shift[p];
        unsigned long long *const kc = cur ? kB : kA, *const kn = cur ? kA : kB;
        uint32_t *const ic = cur ? iB : iA, *const in = cur ? iA : iB;
        const unsigned long long *kin = kc + (size_t)w * cap;
        // 1. local histogram (one shared atomic per distinct digit of a warp)
        if (tid < 256) f.hist[tid] = 0;
        __syncthreads();
        for (int i0 = 0; i0 < myn; i0 += CT) {
            const int i = i0 + tid;
            const uint32_t d = i < myn ? (uint32_t)((kin[i] >> sh) & 255u) : 256u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (d < 256u && lane == __ffs(peers) - 1) atomicAdd(&f.hist[d], (uint32_t)__popc(peers));
        }
        cluster.sync();
        // 2. destination base of every digit value for this CTA's records
        if (tid < 256) {  // all 16 remote reads in flight at once
            uint32_t h[16];
#pragma unroll
            for (int q = 0; q < 16; q++) h[q] = q < ncl ? cluster.map_shared_rank(f.hist, q)[tid] : 0u;
            uint32_t tot = 0, pre = 0;
#pragma unroll
            for (int q = 0; q < 16; q++) {
                tot += h[q];
                pre += q < c ? h[q] : 0u;
            }
            f.tot[tid] = tot;
            f.base[tid] = pre;
        }
        __syncthreads();
        if (tid < 32) {  // exclusive scan of the 256 totals, 8 per lane
            uint32_t v[8], s = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                v[j] = f.tot[tid * 8 + j];
                s += v[j];
            }
            uint32_t x = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            uint32_t run = x - s;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                f.base[tid * 8 + j] += run;
                run += v[j];
            }
        }
        __syncthreads();
        // 3. stable scatter into the owners' other buffers
        for (int i0 = 0; i0 < myn; i0 += CT) {
            const int i = i0 + tid;
            const bool valid = i < myn;
            const uint32_t d = valid ? (uint32_t)((kin[i] >> sh) & 255u) : 256u;
            for (int q = tid; q < (CT / 32) * 256; q += CT) (&f.wc[0][0])[q] = 0;
            __syncthreads();
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
            if (valid && rank == 0) f.wc[warp][d] = (uint8_t)__popc(peers);
            __syncthreads();
            if (valid) {
                uint32_t off = f.base[d] + rank;
                for (int q = 0; q < warp; q++) off += f.wc[q][d];
                const int dst = (int)(off / (uint32_t)per), slot = (int)(off % (uint32_t)per);
                unsigned long long *rk = cluster.map_shared_rank(kn, dst);
                uint32_t *ri = cluster.map_shared_rank(in, dst);
                for (int ww = 0; ww < kw; ww++) rk[(size_t)ww * cap + slot] = kc[(size_t)ww * cap + i];
                ri[slot] = ic[i];
            }
            __syncthreads();
            if (tid < 256) {
                uint32_t add = 0;
                for (int q = 0; q < CT / 32; q++) add += f.wc[q][tid];
                f.base[tid] += add;
            }
            __syncthreads();
        }
        cluster.sync();
        cur ^= 1;
    }
    const uint32_t *ifin = cur ? iB : iA;
    for (int i = tid; i < myn; i += CT) idx_out[my0 + i] = ifin[i];
}

}  // namespace

// Cluster shape and capacity on this GPU, found once per ctx: 16 CTAs where
// the GPU can co-schedule them with the shared memory a record buffer needs,
// else 8, else none.
static int cs_cluster(fim_ctx *ctx, int kw, int *cap_out) {
    if (kw > CS_MAXKW) return 0;
    int dev = 0;
    cudaGetDevice(&dev);
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int cap = (int)((smem_optin - (int)sizeof(CsFixed) - 64) / (2 * 8 * kw + 8));
    cap = cap / 32 * 32;
    if (cap > 8192) cap = 8192;
    if (cap < 1024) return 0;
    *cap_out = cap;
    if (ctx->csort_cl[kw] != 0) return ctx->csort_cl[kw] > 0 ? ctx->csort_cl[kw] : 0;
    const size_t smem = cs_smem(kw, cap);
    int result = -1;
    // the attribute is the kernel's for every key width: the opt-in maximum
    if (cudaFuncSetAttribute(cluster_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin) ==
            cudaSuccess &&
        cudaFuncSetAttribute(cluster_sort_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        for (int cl : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(cl, 1, 1);
            cfg.blockDim = dim3(CT, 1, 1);
            cfg.dynamicSmemBytes = smem;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = cl;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, cluster_sort_kernel, &cfg) == cudaSuccess && nclusters > 0) {
                result = cl;
                break;
            }
        }
    }
    cudaGetLastError();  // a refused attribute or query leaves no sticky error
    ctx->csort_cl[kw] = result;
    return result > 0 ? result : 0;
}

int cluster_sort_plan(fim_ctx *ctx, uint64_t R, int kw, int *cl_out, int *cap_out, int *per_out) {
    if (!ctx->compact_cluster || R == 0 || kw < 1) return 0;
    int cap = 0;
    const int cl = cs_cluster(ctx, kw, &cap);
    if (cl == 0) return 0;
    const uint64_t per = (R + (uint64_t)cl - 1) / (uint64_t)cl;
    if (per > (uint64_t)cap) return 0;
    *cl_out = cl;
    *cap_out = cap;
    *per_out = (int)per;
    return 1;
}

int launch_cluster_sort(fim_ctx *ctx, const unsigned long long *keys, uint64_t R, int kw,
                        const std::vector<std::pair<int, int>> &passes, int cl, int cap, int per, uint32_t *idx_out,
                        cudaStream_t st) {
    if ((int)passes.size() > CS_MAXPASS || kw > CS_MAXKW) return FIM_E_INVAL;
    CsPasses P{};
    P.n = (int)passes.size();
    for (int i = 0; i < P.n; i++) {
        P.word[i] = (signed char)passes[i].first;
        P.shift[i] = (signed char)passes[i].second;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl, 1, 1);
    cfg.blockDim = dim3(CT, 1, 1);
    cfg.dynamicSmemBytes = cs_smem(kw, cap);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FIM_CUDA_TRY(cudaLaunchKernelEx(&cfg, cluster_sort_kernel, keys, (unsigned long long)R, kw, cap, per, P, idx_out));
    return FIM_OK;
}
