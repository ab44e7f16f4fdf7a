// k_pairs_tc.cu -- pair supports on the 5th-generation tensor cores.
//
// S(I_a n I_b) = sum_i M[i,a] M[i,b] (Eq. 2) for all frequent a < b is the
// upper triangle of C = A^T A, A the n x m' 0/1 matrix of frequent columns: a
// dense contraction over the transactions.  (sm_103a has no integer MMA, so
// the entries are fed as e4m3 values 0.0 / 2.0 to tcgen05.mma kind::f8f6f4
// with an f32 accumulator in tensor memory.)
//
// Exactness: every product is 0 or 4 and every partial sum is a multiple of
// 4.  The accumulator is drained into int32 registers every `kdrain` x 128
// transactions (8,192 by default) and restarted, so no f32 partial sum ever
// exceeds 4 x 131,072 = 2^19 even at the largest kdrain; the int32 totals
// (partial / 4) are exact for any n < 2^31.
//
// CTA (544 threads) = one 128 x 128 tile (items a in tile ta, b in tile tb,
// ta <= tb) x one slice of the transactions:
//   warps 0-7   producers, one operand row each (A rows, then B rows; a
//               diagonal tile has A = B): read the row's 128 bits per stage
//               from its item bit column, expand each bit to an e4m3 byte
//               (0x40 = 2.0) and store the 128 x 128-byte operand tiles in the
//               SWIZZLE_128B K-major layout the MMA descriptors name;
//   warp 16     one elected thread issues 4 MMAs (K = 32 each) per stage and
//               commits stage release / accumulator-ready to mbarriers;
//   warps 8-15  epilogue: tcgen05.ld the f32 accumulator (two TMEM buffers,
//               so draining one overlaps the MMAs into the other), convert to
//               int32 and keep running totals; finally atomicAdd into pair_cnt.
// Every mbarrier wait is bounded; on expiry the CTA records an error, lets
// its MMAs finish, frees its tensor memory and returns.
#include "fim_common.cuh"

namespace {

constexpr int TM = 128;              // tile rows (items a)
constexpr int TN = 128;              // tile cols (items b)
constexpr int KB = 128;              // K elements (transactions) per stage = 128 bytes per row
constexpr int STAGES = 4;
constexpr int NPROD = 256;           // producer threads (one operand row each: A then B)
constexpr int NEPI = 256;            // epilogue threads
constexpr int THREADS = NPROD + NEPI + 32;
constexpr int TILE_BYTES = TM * KB;  // 16 KB per operand per stage
constexpr uint32_t TMEM_COLS = 256;  // two 128-column f32 accumulators
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s: far above any legitimate wait

struct __align__(1024) TcSmem {
    uint8_t a[STAGES][TILE_BYTES];
    uint8_t b[STAGES][TILE_BYTES];
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t done;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and the CTA's abort flag set) when WAIT_NS of
// %globaltimer pass, or when another role of the CTA has already aborted.
__device__ __forceinline__ bool mbar_wait(TcSmem &s, uint64_t *b, uint32_t parity) {
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (uint32_t i = 1;; i++) {
        if (mbar_try(b, parity)) return true;
        if ((i & 63) == 0) {
            if (*(volatile int *)&s.abort) return false;
            if (globaltimer_ns() - t0 > WAIT_NS) {
                atomicExch(&s.abort, 1);
                return false;
            }
        }
    }
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, SWIZZLE_128B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4)  // start address
           | (1ull << 16)                        // leading byte offset (unused for swizzled K-major)
           | ((uint64_t)(1024 >> 4) << 32)       // stride byte offset
           | (1ull << 46)                        // descriptor version
           | (2ull << 61);                       // SWIZZLE_128B
}

// Instruction descriptor: kind::f8f6f4, A = B = E4M3, D = F32, K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f8(int M, int N) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 4 bits -> 4 bytes of e4m3 (0x40 = 2.0, 0x00 = 0.0), bit j -> byte j.
// x * 0x08102040 is x << 6 + x << 13 + x << 20 + x << 27: the four copies
// occupy bits 6-9, 13-16, 20-23, 27-30 (no carries), and bit j of the copy
// shifted by 6 + 7j lands on bit 8j + 6, the only set bit of 0x40 in byte j.
// A set bit is encoded as 2.0 (one bit, two instructions per 4 bytes); every
// product is then 4, so the epilogue divides the exact sums by 4.
__device__ __forceinline__ uint32_t nib_to_e4m3(uint32_t x) {
    return (x * 0x08102040u) & 0x40404040u;
}
__device__ __forceinline__ uint4 bits16_to_e4m3(uint32_t h) {
    return make_uint4(nib_to_e4m3(h & 15u), nib_to_e4m3((h >> 4) & 15u), nib_to_e4m3((h >> 8) & 15u),
                      nib_to_e4m3((h >> 12) & 15u));
}

// Row r of a 128 x 128-byte SWIZZLE_128B tile: 16-byte chunk c lives at
// (r / 8) * 1024 + (r % 8) * 128 + ((c ^ (r % 8)) * 16).
__device__ __forceinline__ void store_row(uint8_t *tile, int r, uint4 w) {
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
    uint8_t *row = tile + (r >> 3) * 1024 + (r & 7) * 128;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const uint32_t h = (words[c >> 1] >> ((c & 1) * 16)) & 0xFFFFu;
        *reinterpret_cast<uint4 *>(row + ((c ^ (r & 7)) << 4)) = bits16_to_e4m3(h);
    }
}

__global__ void __launch_bounds__(THREADS, 1)
pairs_tc_kernel(const uint32_t *__restrict__ bm, const int32_t *__restrict__ perm, int64_t nwp, int mf,
                int nt, int64_t stages_total, int64_t stages_per_split, int kdrain,
                int *__restrict__ pair_cnt, int *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    TcSmem &s = *reinterpret_cast<TcSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    int idx = blockIdx.x, ta = 0;
    while (idx >= nt - ta) { idx -= nt - ta; ta++; }
    const int tb = ta + idx;
    const bool diag = ta == tb;
    const int64_t st0 = (int64_t)blockIdx.y * stages_per_split;
    const int64_t st1 = min64(stages_total, st0 + stages_per_split);
    const int nst = (int)(st1 > st0 ? st1 - st0 : 0);
    const int nchunks = (nst + kdrain - 1) / kdrain;

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; i++) { mbar_init(&s.full[i], NPROD); mbar_init(&s.empty[i], 1); }
        for (int i = 0; i < 2; i++) { mbar_init(&s.acc_full[i], 1); mbar_init(&s.acc_empty[i], NEPI); }
        mbar_init(&s.done, 1);
        s.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&s.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s.tmem_base;

    if (warp < NPROD / 32) {
        // ---------------- producers: one operand row each ----------------
        const int r = threadIdx.x & (TM - 1);
        const bool is_b = threadIdx.x >= TM;   // threads 128..255 fill B (none on diagonal tiles)
        const int item = (is_b ? tb * TN : ta * TM) + r;
        const uint32_t *col = (item < mf && !(is_b && diag)) ? bm + (int64_t)perm[item] * nwp : nullptr;
        for (int it = 0; it < nst; it++) {
            const int slot = it % STAGES;
            const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
            const int64_t w = (st0 + it) * 4;  // 4 words = 128 transactions
            const uint4 v = col ? ldg_u4(col + w) : make_uint4(0, 0, 0, 0);
            if (!mbar_wait(s, &s.empty[slot], ph ^ 1u)) break;
            if (!(is_b && diag)) store_row(is_b ? s.b[slot] : s.a[slot], r, v);
            fence_proxy_async();
            mbar_arrive(&s.full[slot]);
        }
    } else if (warp < (NPROD + NEPI) / 32) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;          // TMEM lane quarter this warp may read
        const int half = (warp - NPROD / 32) >> 2;  // columns [64*half, 64*half + 64)
        int acc[64];
#pragma unroll
        for (int c = 0; c < 64; c++) acc[c] = 0;
        for (int j = 0; j < nchunks; j++) {
            const int buf = j & 1;
            if (!mbar_wait(s, &s.acc_full[buf], (uint32_t)(j >> 1) & 1u)) break;
            tc_fence_after();
#pragma unroll
            for (int x = 0; x < 4; x++) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * TN + half * 64 + x * 16);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int c = 0; c < 16; c++) acc[x * 16 + c] += __float2int_rn(__uint_as_float(v[c])) >> 2;
            }
            tc_fence_before();
            mbar_arrive(&s.acc_empty[buf]);
        }
        const int a = ta * TM + q * 32 + lane;
#pragma unroll
        for (int c = 0; c < 64; c++) {
            const int b = tb * TN + half * 64 + c;
            if (a < b && b < mf && acc[c]) atomicAdd(&pair_cnt[(int64_t)a * mf + b], acc[c]);
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t IDESC = idesc_f8(TM, TN);
        bool ok = true;
        for (int it = 0; it < nst && ok; it++) {
            const int slot = it % STAGES;
            const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
            const int j = it / kdrain;
            const int buf = j & 1;
            const bool first = (it % kdrain) == 0;
            const bool last = (it % kdrain) == kdrain - 1 || it == nst - 1;
            if (first) {
                if (!(ok = mbar_wait(s, &s.acc_empty[buf], ((uint32_t)(j >> 1) & 1u) ^ 1u))) break;
                tc_fence_after();
            }
            if (!(ok = mbar_wait(s, &s.full[slot], ph))) break;
            tc_fence_after();
            const uint32_t a0 = smem_addr(s.a[slot]);
            const uint32_t b0 = diag ? a0 : smem_addr(s.b[slot]);
#pragma unroll
            for (int kk = 0; kk < KB / 32; kk++)
                mma_f8(tmem + (uint32_t)(buf * TN), sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), IDESC,
                       (first && kk == 0) ? 0u : 1u);
            mma_commit(&s.empty[slot]);
            if (last) mma_commit(&s.acc_full[buf]);
        }
        // make sure no MMA is in flight before the tensor memory is freed
        mma_commit(&s.done);
        const unsigned long long t0 = globaltimer_ns();
        while (!mbar_try(&s.done, 0) && globaltimer_ns() - t0 < WAIT_NS) {
        }
    }
    tc_fence_before();
    __syncthreads();
    if (s.abort && threadIdx.x == 0) atomicExch(err, FIM_E_TIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

int launch_pairs_tc(fim_ctx *ctx) {
    const int mf = ctx->mfreq;
    if (mf < 2) return FIM_OK;
    const int nt = (int)ceil_div64(mf, TM);
    const int tiles = nt * (nt + 1) / 2;
    const int64_t stages = ceil_div64(ctx->nw, 4);  // 128 transactions per stage
    int64_t split = ctx->pairs_split > 0 ? ctx->pairs_split : ceil_div64(2LL * ctx->num_sms, tiles);
    if (split > stages) split = stages;
    if (split < 1) split = 1;
    const int64_t sps = ceil_div64(stages, split);
    split = ceil_div64(stages, sps);
    const int kdrain = ctx->pairs_kdrain > 0 ? ctx->pairs_kdrain : 64;  // 64 stages = 8192 transactions
    const size_t smem = sizeof(TcSmem) + 1024;
    FIM_CUDA_TRY(cudaFuncSetAttribute(pairs_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FIM_CUDA_TRY(cudaMemsetAsync(ctx->pair_cnt.p, 0, sizeof(int) * (size_t)mf * mf, ctx->stream));
    int *err = &ctx->counters.as<MineCounters>()->err;  // zeroed at the start of every mine
    if (stages > 0) {
        dim3 grid((unsigned)tiles, (unsigned)split);
        ctx->launches++;
        pairs_tc_kernel<<<grid, THREADS, smem, ctx->stream>>>(ctx->bm.as<uint32_t>(), ctx->perm.as<int32_t>(),
                                                               ctx->nwp, mf, nt, stages, sps, kdrain,
                                                               ctx->pair_cnt.as<int>(), err);
        FIM_CUDA_TRY(cudaGetLastError());
    }
    return FIM_OK;
}
