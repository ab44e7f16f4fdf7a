// k_noalloc.cu -- pair supports of a small database without any allocation.
//
// Some callers cannot allocate device memory while they run this library:
// hosts that hand out every device byte through their own allocator and
// forbid others, and paths that must not block in cudaMalloc/cudaFree, which
// can synchronise the whole device.  fim_pair_supports_noalloc serves them:
// the caller passes the CSR and the output matrix, and the only other device
// memory it touches is the file-scope array below, which every GPU that loads
// the library holds until the process exits.  The call does wait for its own
// work: it reads the CSR's element count and the validation flag back to the
// host, each with a synchronisation of the caller's stream.
//
// It is a variant of the CUDA-core pair pass (k_pairs.cu): the bit columns it
// needs live in g_noalloc_bits instead of a ctx-owned buffer, all items are
// kept (no threshold), and the counts go straight to the caller's matrix.
#include <mutex>

#include "fim_common.cuh"

#define FIM_NOALLOC_WORDS (FIM_NOALLOC_MAX_BYTES / 4)

namespace {

static __device__ __align__(256) uint32_t g_noalloc_bits[FIM_NOALLOC_WORDS];
static __device__ __align__(256) int g_noalloc_flag[2];

constexpr int NA_WB = 32;  // words per build tile row
constexpr int NA_TI = 64;
constexpr int NA_KW = 32;

// Bit columns of a CSR slice (as build_bitmaps_kernel, into the static array).
__global__ void __launch_bounds__(256)
na_build_kernel(const int64_t *__restrict__ indptr, const int32_t *__restrict__ indices, int64_t n,
                int32_t m, int64_t nnz, int64_t nwp, int ib, uint32_t *__restrict__ bits, int *flag) {
    extern __shared__ uint32_t tile[];
    __shared__ int64_t s_ptr[NA_WB * 32 + 1];
    const int64_t w0 = (int64_t)blockIdx.x * NA_WB;
    const int i0 = blockIdx.y * ib;
    const int icount = min(ib, m - i0);
    const int64_t t0 = w0 * 32;
    const int64_t t1 = min64(n, t0 + NA_WB * 32);
    const int rows = t1 > t0 ? (int)(t1 - t0) : 0;
    for (int k = threadIdx.x; k < icount * NA_WB; k += blockDim.x) tile[k] = 0u;
    if (rows > 0)
        for (int k = threadIdx.x; k <= rows; k += blockDim.x) s_ptr[k] = indptr[t0 + k];
    __syncthreads();
    int bad = 0;
    if (rows > 0) {
        for (int k = threadIdx.x; k < rows; k += blockDim.x)
            if (s_ptr[k + 1] < s_ptr[k] || s_ptr[k] < 0 || s_ptr[k + 1] > nnz) bad = 1;
        const int64_t e0 = max64(0, s_ptr[0]), e1 = min64(nnz, s_ptr[rows]);
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const int32_t it = indices[e];
            if (it < 0 || it >= m) { bad = 1; continue; }
            if (it < i0 || it >= i0 + icount) continue;
            int lo = 0, hi = rows;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_ptr[mid] <= e) lo = mid; else hi = mid;
            }
            atomicOr(&tile[(it - i0) * NA_WB + (lo >> 5)], 1u << (lo & 31));
        }
    }
    if (bad) atomicExch(flag, 1);
    __syncthreads();
    for (int k = threadIdx.x; k < icount * NA_WB; k += blockDim.x)
        bits[(int64_t)(i0 + k / NA_WB) * nwp + w0 + k % NA_WB] = tile[k];
}

// S(I_a n I_b) for a <= b over all items (the diagonal is S(I_a)).
__global__ void __launch_bounds__(256)
na_pairs_kernel(const uint32_t *__restrict__ bits, int64_t nwp, int64_t nw, int m, int nt,
                int64_t words_per_split, uint32_t *__restrict__ out) {
    __shared__ __align__(16) uint32_t As[NA_KW][NA_TI];
    __shared__ __align__(16) uint32_t Bs[NA_KW][NA_TI];
    int idx = blockIdx.x, ta = 0;
    while (idx >= nt - ta) { idx -= nt - ta; ta++; }
    const int tb = ta + idx;
    const int64_t k0 = (int64_t)blockIdx.y * words_per_split;
    const int64_t k1 = min64(nw, k0 + words_per_split);
    if (k0 >= k1) return;
    const int t = threadIdx.x, lr = t & 63, lc = (t >> 6) * 8;
    const int ra = ta * NA_TI + lr, rb = tb * NA_TI + lr;
    const uint32_t *pa = ra < m ? bits + (int64_t)ra * nwp : nullptr;
    const uint32_t *pb = rb < m ? bits + (int64_t)rb * nwp : nullptr;
    const int ty = t >> 4, tx = t & 15;
    uint32_t acc[4][4] = {};
    for (int64_t k = k0; k < k1; k += NA_KW) {
        uint4 a0 = make_uint4(0, 0, 0, 0), a1 = a0, b0 = a0, b1 = a0;
        if (pa) { a0 = *reinterpret_cast<const uint4 *>(pa + k + lc); a1 = *reinterpret_cast<const uint4 *>(pa + k + lc + 4); }
        if (pb) { b0 = *reinterpret_cast<const uint4 *>(pb + k + lc); b1 = *reinterpret_cast<const uint4 *>(pb + k + lc + 4); }
        __syncthreads();
        const uint32_t av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const uint32_t bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int q = 0; q < 8; q++) { As[lc + q][lr] = av[q]; Bs[lc + q][lr] = bv[q]; }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < NA_KW; kk++) {
            const uint4 a = *reinterpret_cast<const uint4 *>(&As[kk][ty * 4]);
            const uint4 b = *reinterpret_cast<const uint4 *>(&Bs[kk][tx * 4]);
            const uint32_t x[4] = {a.x, a.y, a.z, a.w}, y[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] += __popc(x[i] & y[j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int a = ta * NA_TI + ty * 4 + i, b = tb * NA_TI + tx * 4 + j;
            if (a <= b && b < m && acc[i][j]) atomicAdd(&out[(int64_t)a * m + b], acc[i][j]);
        }
}

// Device address of the static scratch, looked up once per device.
struct NoallocSlot {
    uint32_t *bits = nullptr;
    int *flag = nullptr;
};
constexpr int kMaxDevices = 64;
NoallocSlot g_slots[kMaxDevices];
std::mutex g_slots_mu;

int noalloc_setup(int dev, NoallocSlot *out) {
    if (dev < 0 || dev >= kMaxDevices) return FIM_E_NODEV;
    std::lock_guard<std::mutex> lk(g_slots_mu);
    NoallocSlot &s = g_slots[dev];
    if (!s.bits) {
        void *pb = nullptr, *pf = nullptr;
        cudaError_t e1 = cudaGetSymbolAddress(&pb, g_noalloc_bits);
        cudaError_t e2 = cudaGetSymbolAddress(&pf, g_noalloc_flag);
        if (e1 != cudaSuccess || e2 != cudaSuccess || !pb || !pf) {
            fim_set_cuda_error(e1 != cudaSuccess ? e1 : e2, "cudaGetSymbolAddress", __FILE__, __LINE__);
            return FIM_E_CUDA;
        }
        s.bits = static_cast<uint32_t *>(pb);
        s.flag = static_cast<int *>(pf);
    }
    *out = s;
    return FIM_OK;
}

}  // namespace

extern "C" int fim_pair_supports_noalloc(const int64_t *d_indptr, const int32_t *d_indices, int64_t n_trans,
                                         int32_t n_items, uint32_t *d_pair_counts, void *cuda_stream) {
    FIM_NVTX("fim_pair_supports_noalloc");
    if (!d_indptr || !d_pair_counts || n_trans < 0 || n_items < 0 || n_items > FIM_MAX_ITEMS)
        return FIM_E_INVAL;
    const int64_t nw = ceil_div64(n_trans, 32);
    const int64_t nwp = round_up64(nw, NA_WB);
    if ((uint64_t)nwp * (uint64_t)(n_items > 0 ? n_items : 1) > (uint64_t)FIM_NOALLOC_WORDS) return FIM_E_INVAL;
    int dev = 0;
    FIM_CUDA_TRY(cudaGetDevice(&dev));
    NoallocSlot slot;
    FIM_TRY(noalloc_setup(dev, &slot));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int m = n_items;
    FIM_CUDA_TRY(cudaMemsetAsync(d_pair_counts, 0, sizeof(uint32_t) * (size_t)m * (size_t)m, st));
    FIM_CUDA_TRY(cudaMemsetAsync(slot.flag, 0, sizeof(int), st));
    if (m == 0 || nw == 0) {
        // nothing to count: the cleared matrix is the answer, complete on return
        FIM_CUDA_TRY(cudaStreamSynchronize(st));
        return FIM_OK;
    }
    int64_t nnz = 0;
    FIM_CUDA_TRY(cudaMemcpyAsync(&nnz, d_indptr + n_trans, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    FIM_CUDA_TRY(cudaStreamSynchronize(st));
    if (nnz < 0 || (nnz > 0 && !d_indices)) return FIM_E_INVAL;
    const int ib = m < 1024 ? m : 1024;
    const size_t smem = (size_t)ib * NA_WB * sizeof(uint32_t);
    FIM_CUDA_TRY(cudaFuncSetAttribute(na_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // every word of the m x nwp region is written, so stale contents of an
    // earlier call never leak into this one
    na_build_kernel<<<dim3((unsigned)(nwp / NA_WB), (unsigned)ceil_div64(m, ib)), 256, smem, st>>>(
        d_indptr, d_indices, n_trans, m, nnz, nwp, ib, slot.bits, slot.flag);
    FIM_CUDA_TRY(cudaGetLastError());
    const int nt = (int)ceil_div64(m, NA_TI);
    const int tiles = nt * (nt + 1) / 2;
    int64_t ksteps = ceil_div64(nw, NA_KW), split = ceil_div64(512, tiles);
    if (split > ksteps) split = ksteps;
    if (split < 1) split = 1;
    const int64_t wps = ceil_div64(ksteps, split) * NA_KW;
    split = ceil_div64(nw, wps);
    na_pairs_kernel<<<dim3((unsigned)tiles, (unsigned)split), 256, 0, st>>>(slot.bits, nwp, nw, m, nt, wps,
                                                                          d_pair_counts);
    FIM_CUDA_TRY(cudaGetLastError());
    int bad = 0;
    FIM_CUDA_TRY(cudaMemcpyAsync(&bad, slot.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    FIM_CUDA_TRY(cudaStreamSynchronize(st));
    return bad ? FIM_E_INVAL : FIM_OK;
}
