// k_batch_pairs_tc.cu -- pair supports of every database of a batch on the
// 5th-generation tensor cores.
//
// For database d with m'_d frequent items, S(I_a n I_b) = sum_i M[i,a] M[i,b]
// (Eq. 2) for a < b < m'_d is the upper triangle of A_d^T A_d, A_d its n_d x m'_d
// 0/1 matrix of frequent columns.  The 0/1 entries are fed as e4m3 2.0 / 0.0 to
// tcgen05.mma kind::f8f6f4 with an f32 accumulator in tensor memory (every
// product is 4; a partial over at most kdrain x 128 <= 2^22 transactions is 4 x
// an integer <= 2^22, exact in f32), as in the single-database pass.
//
// Work: the units are (database, ta, tb) with ta <= tb, the 128 x 128 tiles of
// each database's item blocks, longest first (or the device plan's units,
// see batch_pair_plan_kernel).  Which units hold pairs depends on m'_d,
// known only on the device: a unit with 128 tb >= m'_d is empty, and every
// role of the CTA skips it alike.  CTA c takes units c, 2G - 1 - c, 2G + c,
// ... (G CTAs, the rounds alternating direction), so that the persistent
// grid ends nearly together.  A unit's K range runs in segments of at most kdrain
// stages; each segment is one accumulator run, and the two accumulator
// buffers let a segment's drain overlap the next segment's MMAs.
//
// CTA (416 threads):
//   warps 0-3   A producers, one row each (item block ta): copy the row's
//               bits DEPTH stages ahead into shared memory (cp.async, 64-byte
//               runs), expand each bit to an e4m3 byte and write the 128-byte
//               row into tensor memory (tcgen05.st, lane = row; the MMA reads
//               A from there).  On a diagonal tile (ta == tb) the B tile is
//               also the A operand, and these warps only arrive;
//   warps 4-7   B producers, one row each (item block tb): the same expansion
//               into the SWIZZLE_128B K-major B tile of the stage's ring slot;
//   warps 8-11  epilogue: per segment, tcgen05.ld the accumulator (warp q
//               reads lane quarter q = rows 32q .. 32q + 31), convert to
//               counts and write row a's counts for b > a: the first segment
//               of a unit stores, later ones add (a thread owns its row);
//   warp 12     one elected thread issues 4 MMAs (128 x N x 32, N = the
//               tile's columns rounded up to 16) per stage.
// Tensor memory: two 128-column f32 accumulators, then one 32-column A slot
// per ring stage.  Shared memory holds only the B ring, so the ring is deep
// (the MMA -> producer round trip, not bandwidth, bounds a stage when a
// tile's columns are few).  Rows outside the tile's items are zero; a B
// producer remembers which of its ring slots already hold its zero row and
// does not rewrite them.
// Every mbarrier wait is bounded; on expiry the CTA records FIM_E_TIMEOUT,
// lets its MMAs finish, frees its tensor memory and returns.
#include <algorithm>
#include <vector>

#include "fim_common.cuh"
#include "tc_util.cuh"

namespace {

using namespace fim_tc;

constexpr int BT = 128;                // tile side: items a (A rows), items b (B rows)
constexpr int KB = 128;                // transactions per stage = bytes per operand row
constexpr int BNPROD = 2 * BT;         // producer threads: A rows, then B rows
constexpr int BNEPI = 128;             // epilogue threads: one TMEM lane quarter per warp
constexpr int BTHREADS = BNPROD + BNEPI + 32;
constexpr int TILE_BYTES = BT * KB;    // 16 KB per operand tile and stage
constexpr uint32_t ACC_COLS = BT;      // one f32 accumulator: 128 columns; two buffers
constexpr uint32_t A_COL = 2 * ACC_COLS;  // A slot of ring stage q: columns [A_COL + 32 q, + 32)
constexpr uint32_t A_SLOT_COLS = KB / 4;
constexpr uint32_t BTMEM_COLS = 512;
constexpr int BKDRAIN_MAX = 32768;     // 2^22 transactions: partials stay <= 2^24
constexpr unsigned long long BWAIT_NS = 2000000000ull;

// STG expanded operand stages in the ring; DEPTH stages of raw bits staged
// ahead (a multiple of 4: copies go in quads of 4 stages).
template <int STG, int DEPTH>
struct __align__(1024) BtcSmem {
    static_assert(A_COL + STG * A_SLOT_COLS <= BTMEM_COLS, "tensor memory layout");
    uint8_t b[STG][TILE_BYTES];
    uint4 stg[DEPTH][BNPROD];          // raw bits: producer t's row, stage k at stg[k % DEPTH][t]
    uint64_t full[STG];
    uint64_t empty[STG];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t done;
    uint32_t tmem_base;
    int abort;
};

// Unit codes: a tile (d << 32 | ta << 16 | tb), or -- bit 63 set -- two
// databases of at most PACK_MAX frequent items sharing one diagonal tile
// (d1 << 32 | d2, d2 = PACK_NONE when d1 has no partner): rows and columns
// 0 .. 63 hold d1's items, 64 .. 127 d2's; the MMA's cross blocks are never
// read.
constexpr unsigned long long PACK = 1ull << 63;
constexpr uint32_t PACK_NONE = 0xFFFFFFFFu;
constexpr int PACK_MAX = BT / 2;

// What every role of the CTA derives from a unit code, identically.
struct BUnit {
    const DbDesc *D;   // the database (the first of a packed pair)
    const DbDesc *D2;  // a packed pair's second database, or null
    int ta, tb, mf, mf2, N;
    int64_t S;         // stages of 128 transactions (the longer database of a pair)
    int64_t S1, S2;    // a packed pair's own stage counts
    bool diag;
    bool empty;
    bool packed;
};

__device__ __forceinline__ BUnit decode_unit(const DbDesc *__restrict__ dbs, unsigned long long code) {
    BUnit u;
    u.packed = (code & PACK) != 0;
    if (u.packed) {
        const uint32_t d2 = (uint32_t)code;
        u.D = dbs + ((code >> 32) & 0x7FFFFFFFull);
        u.D2 = d2 != PACK_NONE ? dbs + d2 : nullptr;
        u.ta = u.tb = 0;
        u.mf = *(volatile const int32_t *)&u.D->mfreq;
        u.mf2 = u.D2 ? *(volatile const int32_t *)&u.D2->mfreq : 0;
        u.diag = true;
        u.empty = false;  // the plan packs only databases with pairs
        u.N = u.D2 ? PACK_MAX + ((u.mf2 + 15) & ~15) : (u.mf + 15) & ~15;
        u.S1 = (u.D->nw + 3) / 4;
        u.S2 = u.D2 ? (u.D2->nw + 3) / 4 : 0;
        u.S = u.S1 > u.S2 ? u.S1 : u.S2;
        return u;
    }
    u.D = dbs + (code >> 32);
    u.D2 = nullptr;
    u.ta = (int)((code >> 16) & 0xFFFFu);
    u.tb = (int)(code & 0xFFFFu);
    u.mf = *(volatile const int32_t *)&u.D->mfreq;  // written by the rank pass of this mine
    u.mf2 = 0;
    u.diag = u.ta == u.tb;
    u.empty = u.mf < 2 || u.D->maxlen == 1 || u.tb * BT >= u.mf;
    const int cols = u.empty ? 16 : min(BT, u.mf - u.tb * BT);
    u.N = (cols + 15) & ~15;
    u.S = (u.D->nw + 3) / 4;
    u.S1 = u.S;
    u.S2 = 0;
    return u;
}

template <typename S>
__device__ __forceinline__ bool bwait(S &s, uint64_t *b, uint32_t parity) {
    return mbar_wait_bounded(b, parity, &s.abort, BWAIT_NS);
}

// BG: stages a producer publishes per fence (2 or 4; a quad is 4 stages)
template <int STG, int DEPTH, int MINB, int BG>
__global__ void __launch_bounds__(BTHREADS, MINB)
batch_pairs_tc_kernel(const DbDesc *__restrict__ dbs, const unsigned long long *__restrict__ units,
                      int64_t n_units_host, const long long *__restrict__ n_units_dev,
                      const uint32_t *__restrict__ bm, const int32_t *__restrict__ perm_base,
                      int *__restrict__ pair_cnt, int kd, int *__restrict__ err) {
    static_assert(DEPTH % 4 == 0 && DEPTH >= 8, "raw bits go in quads, two or more in flight");
    static_assert(BG == 2 || BG == 4, "a quad publishes in two or one fences");
    static_assert(STG >= 2 * BG, "two publishing groups in flight");
    using Smem = BtcSmem<STG, DEPTH>;
    constexpr int BSTAGES = STG, BD = DEPTH;
    extern __shared__ uint8_t smem_raw[];
    Smem &s = *reinterpret_cast<Smem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the units the plan kernel wrote (this launch's stream, before it), or the host's
    const int64_t n_units = n_units_dev ? (int64_t)*n_units_dev : n_units_host;
    // CTA c's k-th unit: units come longest first, so the rounds alternate
    // direction (c, 2G - 1 - c, 2G + c, ...) to even out the CTAs' totals;
    // every role walks the same sequence
    const int64_t G = gridDim.x, c_ = blockIdx.x;
    auto unit_of = [G, c_](int64_t k) { return k * G + ((k & 1) ? G - 1 - c_ : c_); };

    if (threadIdx.x == 0) {
        for (int i = 0; i < BSTAGES; i++) { mbar_init(&s.full[i], BNPROD / 32); mbar_init(&s.empty[i], 1); }
        for (int i = 0; i < 2; i++) { mbar_init(&s.acc_full[i], 1); mbar_init(&s.acc_empty[i], BNEPI); }
        mbar_init(&s.done, 1);
        s.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&s.tmem_base)),
                     "r"(BTMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s.tmem_base;

    if (warp < BNPROD / 32) {
        // ---------------- producers: one operand row each ----------------
        const bool is_a = threadIdx.x < BT;
        const int r = threadIdx.x & (BT - 1);
        uint4 *const my = &s.stg[0][threadIdx.x];
        const int row0 = threadIdx.x - lane;  // the warp's first producer thread
        uint32_t zeroed = 0;                  // bit q: my row of ring slot q holds zeros
        int it = 0;                           // stages produced by this CTA (ring position)
        bool ok = true;
        for (int64_t k = 0, ui = unit_of(0); ui < n_units && ok; ui = unit_of(++k)) {
            const BUnit u = decode_unit(dbs, units[ui]);
            if (u.empty) continue;
            const bool store = !(is_a && u.diag);  // warp-uniform: a warp's rows are all A or all B
            // the row's database, item and stage count (a packed pair: rows
            // 0 .. 63 the first database's items, 64 .. 127 the second's)
            const DbDesc *const Dr = u.packed ? (r < PACK_MAX ? u.D : u.D2) : u.D;
            const int item = u.packed ? (r & (PACK_MAX - 1)) : (is_a ? u.ta : u.tb) * BT + r;
            const int mfr = u.packed ? (r < PACK_MAX ? u.mf : u.mf2) : u.mf;
            const int64_t lenr = u.packed ? (r < PACK_MAX ? u.S1 : u.S2) : u.S;
            const uint32_t *col =
                (store && Dr && item < mfr)
                    ? bm + Dr->bm_off + (int64_t)__ldg(perm_base + Dr->item_off + item) * Dr->nwp
                    : nullptr;
            const int64_t len = u.S;
            // stage k of the unit lives in stg[k % BD]; a quad of 4 stages is
            // refilled at a time, 4 lanes per row copying 64 contiguous bytes
            auto refill = [&](int64_t q0) {
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int piece = i * 32 + lane, rw = piece >> 2;
                    const int64_t k = q0 + (piece & 3);
                    const uint32_t *c = reinterpret_cast<const uint32_t *>(
                        __shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(col), rw));
                    const int64_t lr = __shfl_sync(0xffffffffu, lenr, rw);
                    if (c && k < lr) cp_async16(smem_addr(&s.stg[k % BD][row0 + rw]), c + k * 4);
                }
                cp_async_commit();
            };
#pragma unroll
            for (int q = 0; q < BD; q += 4) refill(q);
            for (int64_t q0 = 0; q0 < len && ok; q0 += 4) {
                cp_async_wait<BD / 4 - 1>();  // this lane's copies of quad q0 have landed ...
                __syncwarp();        // ... and so have the other lanes' (they filled my row)
#pragma unroll
                for (int64_t k0 = q0; k0 < q0 + 4; k0 += BG) {
                    const int cnt = (int)min64(BG, len - k0);
                    if (cnt <= 0 || !ok) break;
                    uint4 x[BG];
                    bool has[BG];  // my row holds bits at stage k0 + v (else a zero row)
#pragma unroll
                    for (int v = 0; v < BG; v++) {
                        has[v] = col && v < cnt && k0 + v < lenr;
                        x[v] = has[v] ? my[((k0 + v) % BD) * BNPROD] : make_uint4(0, 0, 0, 0);
                    }
                    bool wok = true;  // lane 0 waits for the warp
                    if (lane == 0) {
#pragma unroll
                        for (int v = 0; v < BG; v++)
                            if (v < cnt && wok) {
                                const int sl = (it + v) % BSTAGES;
                                wok = bwait(s, &s.empty[sl], ((uint32_t)((it + v) / BSTAGES) & 1u) ^ 1u);
                            }
                    }
                    ok = __shfl_sync(0xffffffffu, wok, 0);
                    if (!ok) break;
                    if (is_a) {
                        if (store) {  // off-diagonal tile: A rows into tensor memory
                            tc_fence_after();  // after the MMAs that read these slots
#pragma unroll
                            for (int v = 0; v < BG; v++)
                                if (v < cnt)
                                    store_row_tmem(tmem + ((uint32_t)(warp * 32) << 16) +
                                                       (A_COL + (uint32_t)((it + v) % BSTAGES) * A_SLOT_COLS),
                                                   x[v]);
                            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                            tc_fence_before();
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < BG; v++)
                            if (v < cnt) {
                                const int sl = (it + v) % BSTAGES;
                                if (has[v]) {
                                    store_row(s.b[sl], r, x[v]);
                                    zeroed &= ~(1u << sl);
                                } else if (!(zeroed & (1u << sl))) {
                                    zero_row(s.b[sl], r);
                                    zeroed |= 1u << sl;
                                }
                            }
                        fence_proxy_async();
                    }
                    __syncwarp();  // the warp's stores are fenced: lane 0 arrives for it
#pragma unroll
                    for (int v = 0; v < BG; v++)
                        if (v < cnt && lane == 0) mbar_arrive(&s.full[(it + v) % BSTAGES]);
                    it += cnt;
                }
                if (!ok) break;
                __syncwarp();  // every lane has consumed its row of quad q0
                refill(q0 + BD);
            }
            cp_async_wait<0>();  // the staging slots serve the next unit
        }
    } else if (warp < (BNPROD + BNEPI) / 32) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;  // TMEM lane quarter this warp may read
        int j = 0;               // segments drained by this CTA
        bool ok = true;
        for (int64_t k = 0, ui = unit_of(0); ui < n_units && ok; ui = unit_of(++k)) {
            const BUnit u = decode_unit(dbs, units[ui]);
            if (u.empty) continue;
            // my accumulator row: item a of database Da (a packed pair's rows
            // 64 .. 127 are the second database's, its columns 64 .. 127 too)
            const int lr = q * 32 + lane;
            const bool second = u.packed && lr >= PACK_MAX;
            const DbDesc *const Da = second ? u.D2 : u.D;
            const int a = u.packed ? (lr & (PACK_MAX - 1)) : u.ta * BT + lr;
            const int mfa = second ? u.mf2 : u.mf;
            const int coff = u.packed ? (second ? -PACK_MAX : 0) : u.tb * BT;  // column c holds item c + coff
            int *const row = Da ? pair_cnt + Da->pair_off + (int64_t)a * mfa : nullptr;
            for (int64_t st0 = 0; st0 < u.S; st0 += kd, j++) {
                const int buf = j & 1;
                // warp-uniform: tcgen05.ld below is a .sync.aligned warp instruction
                ok = __all_sync(0xffffffffu, bwait(s, &s.acc_full[buf], (uint32_t)(j >> 1) & 1u));
                if (!ok) break;
                tc_fence_after();
#pragma unroll 1
                for (int x = 0; x < u.N / 16; x++) {
                    uint32_t v[16];
                    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * ACC_COLS +
                                           (uint32_t)(x * 16);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15])
                        : "r"(taddr)
                        : "memory");
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (row && a < mfa) {
#pragma unroll
                        for (int c = 0; c < 16; c++) {
                            const int b = x * 16 + c + coff;
                            if (a < b && b < mfa) {
                                const int val = __float2int_rn(__uint_as_float(v[c])) >> 2;
                                row[b] = st0 == 0 ? val : row[b] + val;
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&s.acc_empty[buf]);
            }
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer ----------------
        bool ok = true;
        int it = 0, j = 0;
        for (int64_t k = 0, ui = unit_of(0); ui < n_units && ok; ui = unit_of(++k)) {
            const BUnit u = decode_unit(dbs, units[ui]);
            if (u.empty) continue;
            const uint32_t idesc = idesc_f8(BT, u.N);
            for (int64_t st0 = 0; st0 < u.S && ok; st0 += kd, j++) {
                const int64_t len = min64(kd, u.S - st0);
                const int buf = j & 1;
                // buffer buf's previous run has been drained
                if (!(ok = bwait(s, &s.acc_empty[buf], ((uint32_t)(j >> 1) & 1u) ^ 1u))) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)buf * ACC_COLS;
                for (int64_t k = 0; k < len; k++, it++) {
                    const int slot = it % BSTAGES;
                    if (!(ok = bwait(s, &s.full[slot], (uint32_t)(it / BSTAGES) & 1u))) break;
                    tc_fence_after();
                    const uint32_t b0 = smem_addr(s.b[slot]);
                    if (u.diag) {  // A is the B tile's 128 rows
#pragma unroll
                        for (int kk = 0; kk < KB / 32; kk++)
                            mma_f8(d, sdesc(b0 + kk * 32), sdesc(b0 + kk * 32), idesc, (k == 0 && kk == 0) ? 0u : 1u);
                    } else {
                        const uint32_t a0 = tmem + A_COL + (uint32_t)slot * A_SLOT_COLS;
#pragma unroll
                        for (int kk = 0; kk < KB / 32; kk++)  // 32 e4m3 elements = 8 columns per MMA
                            mma_f8_ts(d, a0 + 8u * kk, sdesc(b0 + kk * 32), idesc, (k == 0 && kk == 0) ? 0u : 1u);
                    }
                    mma_commit(&s.empty[slot]);
                }
                if (ok) mma_commit(&s.acc_full[buf]);
            }
        }
        // no MMA may be in flight when the tensor memory is freed
        mma_commit(&s.done);
        const unsigned long long t0 = globaltimer_ns();
        while (!mbar_try(&s.done, 0) && globaltimer_ns() - t0 < BWAIT_NS) {
        }
    }
    tc_fence_before();
    __syncthreads();
    if (s.abort && threadIdx.x == 0) atomicExch(err, FIM_E_TIMEOUT);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BTMEM_COLS)
                     : "memory");
    }
}

// Block-wide exclusive scan over 1024 threads; *total gets the block's sum.
__device__ long long block_scan_excl(long long v, long long *s_warp, long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const long long before = (warp > 0 ? s_warp[warp - 1] : 0) + x - v;
    *total = s_warp[31];
    __syncthreads();  // s_warp serves the next scan
    return before;
}

// The pair units of one group of databases, planned on the device once the
// rank pass has set every m'_d: ord[0 .. n) lists the group's databases in
// work order (most transactions first).  A database with 2 <= m'_d <=
// PACK_MAX shares a tile with the next such database in that order (so the
// two have about as many transactions); a larger one gets its upper-triangle
// tiles of 128 items; a database without pairs gets nothing.  Units are
// written in work order; *n_units receives their count.  One CTA of 1024
// threads; scratch holds 4 n ints and n long longs.
__global__ void __launch_bounds__(1024)
batch_pair_plan_kernel(const DbDesc *__restrict__ dbs, const int *__restrict__ ord, int n,
                       int *__restrict__ srank, long long *__restrict__ off, int *__restrict__ small_list,
                       unsigned long long *__restrict__ units, long long *__restrict__ n_units) {
    __shared__ long long s_warp[32];
    long long base_small = 0, base_units = 0;
    for (int c0 = 0; c0 < n; c0 += 1024) {
        const int i = c0 + (int)threadIdx.x;
        int small = 0;
        long long tiles = 0;
        if (i < n) {
            const DbDesc &D = dbs[ord[i]];
            const int mf = *(volatile const int32_t *)&D.mfreq;
            const bool live = mf >= 2 && D.maxlen != 1;
            small = live && mf <= PACK_MAX;
            if (live && !small) {
                const long long nt = (mf + BT - 1) / BT;
                tiles = nt * (nt + 1) / 2;
            }
        }
        long long t_small, t_units;
        const long long sr = block_scan_excl(small, s_warp, &t_small) + base_small;
        const long long cnt = small ? ((sr & 1) == 0 ? 1 : 0) : tiles;  // a pair opens at even ranks
        const long long o = block_scan_excl(cnt, s_warp, &t_units) + base_units;
        if (i < n) {
            srank[i] = small ? (int)sr : -1;
            off[i] = o;
            if (small) small_list[sr] = ord[i];
        }
        base_small += t_small;
        base_units += t_units;
    }
    __syncthreads();  // small_list is complete
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int d = ord[i], sr = srank[i];
        long long o = off[i];
        if (sr >= 0) {
            if ((sr & 1) == 0) {
                const uint32_t d2 = sr + 1 < base_small ? (uint32_t)small_list[sr + 1] : PACK_NONE;
                units[o] = PACK | ((unsigned long long)d << 32) | d2;
            }
        } else {
            const int mf = *(volatile const int32_t *)&dbs[d].mfreq;
            if (mf >= 2 && dbs[d].maxlen != 1) {
                const int nt = (mf + BT - 1) / BT;
                for (int ta = 0; ta < nt; ta++)
                    for (int tb = ta; tb < nt; tb++)
                        units[o++] = ((unsigned long long)d << 32) | ((unsigned long long)ta << 16) | (unsigned)tb;
            }
        }
    }
    if (threadIdx.x == 0) *n_units = base_units;
}

}  // namespace

// The batch's (database, tile) units in the order the pass takes them.  The
// upper-triangle tiles of a database's n_items (an upper bound of m'_d) are
// numbered in row order; the units go by tile number first -- every
// database's tile 0, then every tile 1, ... -- and within one tile number
// by descending stage count (ties by database).  Tile 0 holds pairs whenever
// m'_d >= 2, so the first units are all real work, longest first, and the
// round-robin deal gives every CTA a fair share of it; the later tile numbers
// are empty wherever m'_d is small.  The units of databases [d0, d1) are
// appended to `units`; returns false when there would be more than max_units.
bool batch_pairs_tc_units(const std::vector<DbDesc> &dbs, int d0, int d1, std::vector<unsigned long long> &units,
                          size_t max_units) {
    std::vector<int> order;
    size_t total = 0;
    int max_tiles = 0;
    for (int d = d0; d < d1; d++) {
        order.push_back(d);
        const int nt = (int)ceil_div64(dbs[d].m, BT);
        total += (size_t)nt * (size_t)(nt + 1) / 2;
        max_tiles = std::max(max_tiles, nt * (nt + 1) / 2);
    }
    if (units.size() + total > max_units) return false;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return dbs[x].nw > dbs[y].nw; });
    units.reserve(units.size() + total);
    for (int t = 0; t < max_tiles; t++)
        for (int d : order) {
            const int nt = (int)ceil_div64(dbs[d].m, BT);
            if (t >= nt * (nt + 1) / 2) continue;
            int ta = 0, r = t;  // tile t in row order: (ta, tb) with ta <= tb
            while (r >= nt - ta) { r -= nt - ta; ta++; }
            const int tb = ta + r;
            units.push_back(((unsigned long long)d << 32) | ((unsigned long long)ta << 16) | (unsigned)tb);
        }
    return true;
}

namespace {

template <int STG, int DEPTH, int MINB, int BG>
int launch_shape(fim_ctx *ctx, const DbDesc *d_dbs, const unsigned long long *d_units, int64_t n_units,
                 const long long *d_n_units, cudaStream_t st) {
    using Smem = BtcSmem<STG, DEPTH>;
    static_assert(sizeof(Smem) + 1024 <= 232448, "shared memory per CTA");
    // MINB CTAs share an SM: their tensor memory and shared memory must fit
    // it together
    static_assert(MINB * BTMEM_COLS <= 512, "tensor memory per SM");
    static_assert(MINB * (sizeof(Smem) + 2048) <= 233472, "CTAs per SM as planned");
    const int kd = ctx->pairs_kdrain > 0 ? ctx->pairs_kdrain : BKDRAIN_MAX;
    int64_t grid = ctx->pairs_split > 0 ? ctx->pairs_split : (int64_t)ctx->num_sms * MINB;
    if (grid > n_units) grid = n_units;
    // one CTA per SM when MINB is 1: more shared memory than half an SM
    // keeps a second CTA (and its tensor-memory allocation) off
    size_t smem = sizeof(Smem) + 1024;
    if (MINB == 1 && smem < 120 * 1024) smem = 120 * 1024;
    auto *kern = batch_pairs_tc_kernel<STG, DEPTH, MINB, BG>;
    FIM_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int *err = &ctx->counters.as<MineCounters>()->err;  // zeroed at the start of every batch
    ctx->launches++;
    kern<<<(unsigned)grid, BTHREADS, smem, st>>>(d_dbs, d_units, n_units, d_n_units, ctx->bm.as<uint32_t>(),
                                                 ctx->perm.as<int32_t>(), ctx->pair_cnt.as<int>(), kd, err);
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

}  // namespace

// Launch shapes of the batched tensor-core pair pass (the "batch_pairs_shape"
// knob): expanded operand stages in the ring, stages of raw bits staged
// ahead, CTAs per SM, stages a producer publishes per fence.
const int kBatchPairsShapes[][4] = {{8, 8, 1, 2}, {6, 8, 1, 2}, {8, 16, 1, 2}, {4, 8, 1, 2},
                                    {7, 12, 1, 2}, {8, 8, 1, 4}, {8, 16, 1, 4}};
const int kBatchPairsShapeCount = (int)(sizeof(kBatchPairsShapes) / sizeof(kBatchPairsShapes[0]));

int launch_batch_pairs_tc(fim_ctx *ctx, const DbDesc *d_dbs, const unsigned long long *d_units, int64_t n_units,
                          const long long *d_n_units, cudaStream_t st) {
    if (n_units <= 0) return FIM_OK;
    switch (ctx->batch_pairs_shape) {
        case 1: return launch_shape<6, 8, 1, 2>(ctx, d_dbs, d_units, n_units, d_n_units, st);
        case 2: return launch_shape<8, 16, 1, 2>(ctx, d_dbs, d_units, n_units, d_n_units, st);
        case 3: return launch_shape<4, 8, 1, 2>(ctx, d_dbs, d_units, n_units, d_n_units, st);
        case 4: return launch_shape<7, 12, 1, 2>(ctx, d_dbs, d_units, n_units, d_n_units, st);
        case 5: return launch_shape<8, 8, 1, 4>(ctx, d_dbs, d_units, n_units, d_n_units, st);
        case 6: return launch_shape<8, 16, 1, 4>(ctx, d_dbs, d_units, n_units, d_n_units, st);
        default: return launch_shape<8, 8, 1, 2>(ctx, d_dbs, d_units, n_units, d_n_units, st);
    }
}

int launch_batch_pair_plan(fim_ctx *ctx, const DbDesc *d_dbs, const int *d_ord, int n, unsigned long long *d_units,
                           long long *d_n_units, void *scratch, cudaStream_t st) {
    if (n <= 0) return FIM_OK;
    int *const srank = static_cast<int *>(scratch);
    int *const small_list = srank + n;
    long long *const off = reinterpret_cast<long long *>(small_list + n);  // 8n bytes in: aligned
    ctx->launches++;
    batch_pair_plan_kernel<<<1, 1024, 0, st>>>(d_dbs, d_ord, n, srank, off, small_list, d_units, d_n_units);
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

size_t batch_pair_plan_scratch(int n) {
    return sizeof(int) * 2 * (size_t)n + sizeof(long long) * (size_t)n;
}
