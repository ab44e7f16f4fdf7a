// k_pairs_tc.cu -- pair supports on the 5th-generation tensor cores.
//
// S(I_a n I_b) = sum_i M[i,a] M[i,b] (Eq. 2) for all frequent a < b is the
// upper triangle of C = A^T A, A the n x m' 0/1 matrix of frequent columns: a
// dense contraction over the transactions.  (sm_103a has no integer MMA, so
// the entries are fed as e4m3 values 0.0 / 2.0 to tcgen05.mma kind::f8f6f4
// with an f32 accumulator in tensor memory.)
//
// Exactness: every product is 0 or 4, so a partial sum over t transactions is
// 4 x an integer <= 4t.  One accumulator sums at most `kdrain` x 128
// transactions (at most 32,768 x 128 = 2^22) before it is drained, so every
// partial is an integer <= 2^24, exact in f32; the drained counts (partial / 4)
// meet in int32 by atomicAdd and are exact for any n < 2^31.
//
// Work: C is cut into 128 x 256 tiles (items a in A-block ta, b in B-block tb)
// that hold at least one pair a < b; each tile's reduction runs over
// ceil(nw / 4) stages of 128 transactions.  The (tile, stage) space is split
// into one contiguous range per CTA (one CTA per SM by default), so every SM
// gets the same number of MMA stages whatever the tile count; a range is
// processed as segments that never cross a tile or a multiple of kdrain stages.
//
// CTA (672 threads):
//   warps 0-3   A producers, one row each: copy the row's bits D stages
//               ahead into shared memory (cp.async), expand each bit to an e4m3 byte (0x40 = 2.0)
//               and write the 128-byte row straight into tensor memory
//               (tcgen05.st; the MMA reads A from TMEM, so A costs no
//               shared-memory bandwidth).  When the A-block lies inside the
//               B-block, A is read from B's shared-memory tile instead and
//               these warps only arrive;
//   warps 4-11  B producers, one row each: the same expansion into the
//               SWIZZLE_128B K-major shared-memory tile the B descriptor names;
//   warps 12-19 epilogue: per segment, tcgen05.ld the f32 accumulator,
//               convert to counts, transpose 32 x 16 blocks through shared
//               memory and add them into pair_cnt[a][b] with coalesced
//               atomics;
//   warp 20     one elected thread issues 4 MMAs (128 x 256 x 32) per stage
//               and commits stage release / accumulator-ready to mbarriers.
// Tensor memory: the 256-column accumulator at column 0, then one 32-column
// A slot per pipeline stage.  Shared-memory traffic per stage is the B tile
// written once and read once (64 KB for 8.4 MFLOP).
// Every mbarrier wait is bounded; on expiry the CTA records an error, lets
// its MMAs finish, frees its tensor memory and returns.
#include "fim_common.cuh"
#include "tc_util.cuh"

namespace {

constexpr int TM = 128;               // A rows (items a) per tile
constexpr int TN = 256;               // B rows (items b) per tile
constexpr int KB = 128;               // K elements (transactions) per stage = 128 bytes per row
constexpr int STAGES = 5;
constexpr int NPROD = TM + TN;        // producer threads, one operand row each
constexpr int NEPI = 256;             // epilogue threads
constexpr int THREADS = NPROD + NEPI + 32;
constexpr int A_BYTES = TM * KB;      // 16 KB: A inside B's tile starts this far in
constexpr int B_BYTES = TN * KB;      // 32 KB per stage
constexpr int D = 8;                  // stages a producer's raw bits are copied ahead (cp.async)
constexpr int G = 2;                  // stages a producer publishes per fence
constexpr uint32_t ACC_COL = 0;       // f32 accumulator: columns [0, 256)
constexpr uint32_t A_COL = TN;        // A slot s: columns [A_COL + 32 s, A_COL + 32 s + 32)
constexpr uint32_t A_SLOT_COLS = KB / 4;
constexpr uint32_t TMEM_COLS = 512;   // power of two >= A_COL + STAGES * A_SLOT_COLS
static_assert(A_COL + STAGES * A_SLOT_COLS <= TMEM_COLS, "tensor memory layout");
constexpr int KDRAIN_MAX = 32768;     // 2^22 transactions: partials stay <= 2^24
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s: far above any legitimate wait

struct __align__(1024) TcSmem {
    uint8_t b[STAGES][B_BYTES];
    uint4 stg[D][NPROD];              // raw bits: producer t's row, stage k at stg[k % D][t]
    int xp[NEPI / 32][16][34];        // per epilogue warp: 16 columns x 32 rows (+2 pad)
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t acc_full;
    uint64_t acc_empty;
    uint64_t done;
    uint32_t tmem_base;
    int abort;
};

static_assert(sizeof(TcSmem) + 1024 <= 232448, "shared memory per CTA");

using namespace fim_tc;

// Bounded wait on the CTA's abort flag: false (and the flag set) when WAIT_NS
// of %globaltimer pass, or when another role of the CTA has already aborted.
__device__ __forceinline__ bool mbar_wait(TcSmem &s, uint64_t *b, uint32_t parity) {
    return mbar_wait_bounded(b, parity, &s.abort, WAIT_NS);
}

// Tiles (ta, tb) with at least one pair a < b < mf, ta-major.  The first
// B-block that reaches past a = 128 ta is tb = ta / 2; the last A-block may
// hold only the last item, which pairs with nothing.
__host__ __device__ __forceinline__ int tiles_of_row(int ta, int mf, int ntb) {
    const int lo = ta >> 1;
    if (lo >= ntb) return 0;
    if (lo == ntb - 1 && !(mf - 1 > ta * TM)) return 0;
    return ntb - lo;
}
__device__ __forceinline__ void tile_coords(int t, int mf, int ntb, int &ta, int &tb) {
    for (ta = 0;; ta++) {
        const int c = tiles_of_row(ta, mf, ntb);
        if (t < c) { tb = (ta >> 1) + t; return; }
        t -= c;
    }
}

// Segment of a CTA's (tile, stage) range starting at flat index w: the run
// stays in one tile and ends at a multiple of kdrain stages.
struct Seg {
    int tile;
    int64_t st;   // first stage
    int len;      // stages
};
__device__ __forceinline__ Seg next_seg(int64_t w, int64_t w1, int64_t S, int kd) {
    Seg g;
    g.tile = (int)(w / S);
    g.st = w - (int64_t)g.tile * S;
    int64_t end = min64(w1 - (int64_t)g.tile * S, S);
    end = min64(end, (g.st / kd + 1) * kd);
    g.len = (int)(end - g.st);
    return g;
}

__global__ void __launch_bounds__(THREADS, 1)
pairs_tc_kernel(const uint32_t *__restrict__ bm, const int32_t *__restrict__ perm, int64_t nwp, int mf,
                int ntb, int64_t S, int64_t W, int kd, int *__restrict__ pair_cnt, int *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    TcSmem &s = *reinterpret_cast<TcSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * W / gridDim.x;
    const int64_t w1 = (int64_t)(blockIdx.x + 1) * W / gridDim.x;

    if (threadIdx.x == 0) {
        // one arrival per producer warp and stage
        for (int i = 0; i < STAGES; i++) { mbar_init(&s.full[i], NPROD / 32); mbar_init(&s.empty[i], 1); }
        mbar_init(&s.acc_full, 1);
        mbar_init(&s.acc_empty, NEPI);
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
        const bool is_a = threadIdx.x < TM;
        const int r = is_a ? threadIdx.x : threadIdx.x - TM;
        int it = 0;  // stages produced by this CTA (ring position)
        bool ok = true;
        for (int64_t w = w0; w < w1 && ok;) {
            const Seg g = next_seg(w, w1, S, kd);
            w += g.len;
            int ta, tb;
            tile_coords(g.tile, mf, ntb, ta, tb);
            const bool a_in_b = tb == (ta >> 1);  // A rows are rows 128*(ta&1).. of B's tile
            const bool store = !(is_a && a_in_b);
            const int item = is_a ? ta * TM + r : tb * TN + r;
            const uint32_t *col = (store && item < mf) ? bm + (int64_t)perm[item] * nwp : nullptr;
            // Raw bits are staged in shared memory D = 8 stages ahead, refilled
            // a quad of 4 stages at a time: the warp copies its 32 rows x 64
            // contiguous bytes (4 lanes per row, 16 B each), so DRAM sees
            // 64-byte runs however the rows are scattered.  Stage k of the
            // segment lives in stg[k % D]; one copy group per quad.
            uint4 *const my = &s.stg[0][threadIdx.x];
            const int row0 = threadIdx.x - lane;  // the warp's first producer thread
            auto refill = [&](int q0) {  // stages [q0, q0 + 4) of the segment
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int piece = i * 32 + lane, rw = piece >> 2, k = q0 + (piece & 3);
                    const uint32_t *c = reinterpret_cast<const uint32_t *>(
                        __shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(col), rw));
                    if (c && k < g.len)
                        cp_async16(smem_addr(&s.stg[k % D][row0 + rw]), c + (g.st + k) * 4);
                }
                cp_async_commit();
            };
            refill(0);
            refill(4);
            for (int q0 = 0; q0 < g.len && ok; q0 += 4) {
                cp_async_wait<1>();  // this lane's copies of quad q0 have landed ...
                __syncwarp();        // ... and so have the other lanes' (they filled my row)
                // stages go out in pairs: both slots are filled, then one fence
                // (proxy or tensor-memory) publishes both, so a producer pays
                // that round trip once per two stages
#pragma unroll
                for (int k0 = q0; k0 < q0 + 4; k0 += G) {
                    const int cnt = min(G, g.len - k0);
                    if (cnt <= 0 || !ok) break;
                    uint4 x[G];
#pragma unroll
                    for (int v = 0; v < G; v++)
                        x[v] = (col && v < cnt) ? my[((k0 + v) % D) * NPROD] : make_uint4(0, 0, 0, 0);
                    bool wok = true;  // lane 0 waits for the warp
                    if (lane == 0) {
#pragma unroll
                        for (int v = 0; v < G; v++)
                            if (v < cnt && wok) {
                                const int sl = (it + v) % STAGES;
                                wok = mbar_wait(s, &s.empty[sl], ((uint32_t)((it + v) / STAGES) & 1u) ^ 1u);
                            }
                    }
                    ok = __shfl_sync(0xffffffffu, wok, 0);
                    if (!ok) break;
                    if (is_a) {
                        if (store) {  // warp-uniform: a warp's 32 rows are all A or all B
                            tc_fence_after();  // after the MMAs that read these slots
#pragma unroll
                            for (int v = 0; v < G; v++)
                                if (v < cnt)
                                    store_row_tmem(tmem + ((uint32_t)(warp * 32) << 16) +
                                                       (A_COL + (uint32_t)((it + v) % STAGES) * A_SLOT_COLS),
                                                   x[v]);
                            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                            tc_fence_before();
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < G; v++)
                            if (v < cnt) store_row(s.b[(it + v) % STAGES], r, x[v]);
                        fence_proxy_async();
                    }
                    __syncwarp();  // the warp's stores are fenced: lane 0 arrives for it
#pragma unroll
                    for (int v = 0; v < G; v++)
                        if (v < cnt && lane == 0) mbar_arrive(&s.full[(it + v) % STAGES]);
                    it += cnt;
                }
                if (!ok) break;
                // every lane has consumed its row of quad q0 (the stores above
                // used the values), so the quad's slots can take stages q0 + 8
                __syncwarp();
                refill(q0 + D);
            }
            cp_async_wait<0>();  // the staging slots serve the next segment
        }
    } else if (warp < (NPROD + NEPI) / 32) {
        // ---------------- epilogue ----------------
        const int e = warp - NPROD / 32;
        const int q = warp & 3;          // TMEM lane quarter this warp may read
        const int half = e >> 2;         // accumulator columns [128*half, 128*half + 128)
        int (*xp)[34] = s.xp[e];
        int j = 0;
        for (int64_t w = w0; w < w1; j++) {
            const Seg g = next_seg(w, w1, S, kd);
            w += g.len;
            int ta, tb;
            tile_coords(g.tile, mf, ntb, ta, tb);
            // warp-uniform: tcgen05.ld below is a .sync.aligned warp instruction
            if (!__all_sync(0xffffffffu, mbar_wait(s, &s.acc_full, (uint32_t)j & 1u))) break;
            tc_fence_after();
#pragma unroll 1
            for (int x = 0; x < 8; x++) {
                uint32_t v[16];
                const uint32_t taddr =
                    tmem + ((uint32_t)(q * 32) << 16) + (ACC_COL + (uint32_t)(half * 128 + x * 16));
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // lane = row a; transpose so that a warp store covers 2 rows x 16 columns
#pragma unroll
                for (int c = 0; c < 16; c++) xp[c][lane] = __float2int_rn(__uint_as_float(v[c])) >> 2;
                __syncwarp();
                const int c = lane & 15;
                const int b = tb * TN + half * 128 + x * 16 + c;
#pragma unroll 4
                for (int i = 0; i < 16; i++) {
                    const int rr = 2 * i + (lane >> 4);
                    const int a = ta * TM + q * 32 + rr;
                    const int val = xp[c][rr];
                    if (a < b && b < mf && val) atomicAdd(&pair_cnt[(int64_t)a * mf + b], val);
                }
                __syncwarp();
            }
            tc_fence_before();
            mbar_arrive(&s.acc_empty);
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t IDESC = idesc_f8(TM, TN);
        bool ok = true;
        int it = 0, j = 0;
        for (int64_t w = w0; w < w1 && ok; j++) {
            const Seg g = next_seg(w, w1, S, kd);
            w += g.len;
            int ta, tb;
            tile_coords(g.tile, mf, ntb, ta, tb);
            const bool a_in_b = tb == (ta >> 1);
            // one accumulator: segment j starts once segment j - 1 is drained
            if (!(ok = mbar_wait(s, &s.acc_empty, ((uint32_t)j & 1u) ^ 1u))) break;
            tc_fence_after();
            for (int k = 0; k < g.len; k++, it++) {
                const int slot = it % STAGES;
                const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                if (!(ok = mbar_wait(s, &s.full[slot], ph))) break;
                tc_fence_after();
                const uint32_t b0 = smem_addr(s.b[slot]);
                if (a_in_b) {
                    const uint32_t a0 = b0 + (uint32_t)((ta & 1) * A_BYTES);
#pragma unroll
                    for (int kk = 0; kk < KB / 32; kk++)
                        mma_f8(tmem + ACC_COL, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), IDESC,
                               (k == 0 && kk == 0) ? 0u : 1u);
                } else {
                    const uint32_t a0 = tmem + A_COL + (uint32_t)slot * A_SLOT_COLS;
#pragma unroll
                    for (int kk = 0; kk < KB / 32; kk++)  // 32 fp8 elements = 8 columns per MMA
                        mma_f8_ts(tmem + ACC_COL, a0 + 8u * kk, sdesc(b0 + kk * 32), IDESC,
                                  (k == 0 && kk == 0) ? 0u : 1u);
                }
                mma_commit(&s.empty[slot]);
            }
            if (ok) mma_commit(&s.acc_full);
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
    const int nta = (int)ceil_div64(mf, TM), ntb = (int)ceil_div64(mf, TN);
    int64_t tiles = 0;
    for (int ta = 0; ta < nta; ta++) tiles += tiles_of_row(ta, mf, ntb);
    const int64_t S = ceil_div64(ctx->nw, 4);  // 128 transactions per stage
    const int64_t W = tiles * S;
    const int kd = ctx->pairs_kdrain > 0 ? ctx->pairs_kdrain : KDRAIN_MAX;
    int64_t grid = ctx->pairs_split > 0 ? ctx->pairs_split : ctx->num_sms;
    if (grid > W) grid = W;
    const size_t smem = sizeof(TcSmem) + 1024;
    FIM_CUDA_TRY(cudaFuncSetAttribute(pairs_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FIM_CUDA_TRY(cudaMemsetAsync(ctx->pair_cnt.p, 0, sizeof(int) * (size_t)mf * mf, ctx->stream));
    int *err = &ctx->counters.as<MineCounters>()->err;  // zeroed at the start of every mine
    if (grid > 0) {
        ctx->launches++;
        pairs_tc_kernel<<<(unsigned)grid, THREADS, smem, ctx->stream>>>(
            ctx->bm.as<uint32_t>(), ctx->perm.as<int32_t>(), ctx->nwp, mf, ntb, S, W, kd,
            ctx->pair_cnt.as<int>(), err);
        FIM_CUDA_TRY(cudaGetLastError());
    }
    return FIM_OK;
}
