// k_batched.cu -- many independent databases in one pass of the pipeline.
//
// Every database d gets the three stages of Section III exactly as fim_mine
// gives one: bit columns (Eq. 1), singleton and pair supports with the
// threshold (Eq. 2-3, its own minsup), and the depth-first prefix extension.
// Here all databases share one launch per stage:
//   * a DbDesc table gives each database's CSR and its offsets into the
//     batch-wide arrays (bit columns, item supports/perm, pair counts, pair
//     bitset);
//   * each stage's grid is the concatenation of the databases' work units
//     (word blocks, item columns, pair tiles, pair rows); a CTA finds its
//     database in a unit -> database map (the build) or by binary search over
//     the prefix sums of those counts;
//   * the persistent DFS kernel takes root classes of all databases from one
//     queue (root_db tags them) and loads the task's database view;
//   * the compactor sorts by (database, size, items), so each database's
//     canonical results are one contiguous slice.
// Sizes that only the device knows (m' per database) never reach the host
// before the DFS ends, so build -> DFS is captured once in a CUDA graph and
// replayed for later batches of the same shape.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "fim_common.cuh"


namespace {

constexpr int WB = 32;     // words per build tile row
constexpr int TI = 64;     // pair tile side
constexpr int KW = 32;     // words per pair k-step
constexpr unsigned long long kTaskCap = 1ull << 20;
constexpr unsigned long long kCandPoolCap = 1ull << 24;

// largest d with prefix[d] <= x (prefix has n_db + 1 entries, prefix[0] = 0)
__device__ __forceinline__ int find_db(const int64_t *prefix, int n_db, int64_t x) {
    int lo = 0, hi = n_db;  // prefix[lo] <= x < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256)
batch_build_kernel(const DbDesc *__restrict__ dbs, int n_db, const int64_t *__restrict__ unit_prefix, int ib,
                   uint32_t *__restrict__ bm, int *__restrict__ flag) {
    extern __shared__ uint32_t tile[];  // [ib][WB]
    __shared__ int64_t s_ptr[WB * 32 + 1];
    const int d = find_db(unit_prefix, n_db, blockIdx.x);
    const DbDesc &D = dbs[d];
    const int64_t local = blockIdx.x - unit_prefix[d];
    const int nib = (D.m + ib - 1) / ib;
    const int64_t w0 = (local / nib) * WB;
    const int i0 = (int)(local % nib) * ib;
    const int icount = min(ib, D.m - i0);
    const int64_t n = D.n;
    const bool cmp = D.compact != 0;
    const int64_t nnz = n > 0 ? csr_off(D.indptr, cmp, n) : 0;
    const int64_t t0 = w0 * 32, t1 = min64(n, t0 + WB * 32);
    const int rows = t1 > t0 ? (int)(t1 - t0) : 0;
    for (int k = threadIdx.x; k < icount * WB; k += blockDim.x) tile[k] = 0u;
    if (rows > 0)
        for (int k = threadIdx.x; k <= rows; k += blockDim.x) s_ptr[k] = csr_off(D.indptr, cmp, t0 + k);
    __syncthreads();
    int bad = 0;
    if (rows > 0) {
        for (int k = threadIdx.x; k < rows; k += blockDim.x)
            if (s_ptr[k + 1] < s_ptr[k] || s_ptr[k] < 0 || s_ptr[k + 1] > nnz) bad = 1;
        const int64_t e0 = max64(0, s_ptr[0]), e1 = min64(nnz, s_ptr[rows]);
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const int32_t it = csr_id(D.indices, cmp, e);
            if (it < 0 || it >= D.m) { bad = 1; continue; }
            if (it < i0 || it >= i0 + icount) continue;
            int lo = 0, hi = rows;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_ptr[mid] <= e) lo = mid; else hi = mid;
            }
            atomicOr(&tile[(it - i0) * WB + (lo >> 5)], 1u << (lo & 31));
        }
    }
    if (bad) atomicExch(flag, 1);
    __syncthreads();
    uint32_t *col0 = bm + D.bm_off;
    for (int k = threadIdx.x; k < icount * WB; k += blockDim.x)
        col0[(int64_t)(i0 + k / WB) * D.nwp + w0 + k % WB] = tile[k];
}

// Databases with at most 1,024 items: one CTA per block of 32 x WBK
// transactions (WBK words of every column) of one database holds the
// block's words of every item column in shared memory, word-major with an odd
// pitch.  Lane i of a warp owns row i of a 32-row group (one tile word) and
// ORs bit i into its items' words with shared atomics -- no search for a
// row's position.  The block is then written out 16 bytes per thread, a
// column's WBK words by WBK/4 consecutive lanes (coalesced), and each
// column's popcount over the block rides along: a shuffle sum over those
// lanes, added into S(I_j) (Eq. 3), so no second pass reads the columns.
// Blocks past the last transaction hold padding words only and just write
// zeros.  A CTA finds its database in a unit -> database map.  The
// persistent form (one CTA per SM walking the units) serves host input read
// over the link, where it leaves each SM room for the pair pass of an earlier
// group of databases.
constexpr int BUILD_ROWS_THREADS = 512;
// What a build CTA needs of its unit, written per unit by the unit-map
// kernel: one 64-byte load instead of map -> database table -> prefix.
struct __align__(16) BuildUnit {
    const void *indptr;     // the database's CSR (wide, or compact)
    const void *indices;
    uint32_t *col0;         // its first bit column
    int64_t n;              // its transactions
    int64_t nwp;            // column pitch in words
    int64_t item_off;       // its first entry of the item supports
    int64_t w0;             // the unit's first word
    int32_t m;              // its items
    int32_t compact;        // 1: uint32 row offsets and uint16 item ids
};
static_assert(sizeof(BuildUnit) == 64, "one unit per 64 bytes");

template <int WBK, bool COAL, bool CMP>
__device__ __forceinline__ void build_rows_unit(const BuildUnit &D, uint32_t *__restrict__ sup,
                                                int *__restrict__ flag, uint32_t *tile) {
    static_assert(WBK % 4 == 0 && WBK / 4 <= 32 && 32 % (WBK / 4) == 0, "a column's chunks share a warp");
    constexpr int NWARP = BUILD_ROWS_THREADS / 32;
    constexpr int QPC = WBK / 4;  // 16-byte chunks of a column in this block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    using Id = typename std::conditional<CMP, unsigned short, int32_t>::type;
    const Id *const ids = static_cast<const Id *>(D.indices);
    const int m = D.m, ms = m | 1;  // odd pitch: the transposed reads below are conflict-free
    const int64_t w0 = D.w0;
    const int64_t n = D.n;
    uint32_t *const col0 = D.col0;
    const int64_t t0 = w0 * 32;
    if (t0 >= n) {  // padding words only
        for (int k = threadIdx.x; k < m * QPC; k += BUILD_ROWS_THREADS)
            *reinterpret_cast<uint4 *>(col0 + (int64_t)(k / QPC) * D.nwp + w0 + 4 * (k % QPC)) =
                make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    const int64_t nnz = csr_off(D.indptr, CMP, n);
    for (int k = threadIdx.x; k < WBK * ms / 4; k += BUILD_ROWS_THREADS)
        reinterpret_cast<uint4 *>(tile)[k] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    int bad = 0;
    if (COAL) {
        // a warp's 32 rows hold consecutive ids [A, B): the warp reads them
        // 32 at a time (coalesced, U loads in flight per lane) and finds each
        // id's row by a 5-step search over the rows' starts held by the lanes
        constexpr int U = 8;
        for (int g = warp; g < WBK; g += NWARP) {
            const int64_t r0 = t0 + 32 * g;
            if (r0 >= n) break;  // warp-uniform
            const int nrw = (int)min64(n - r0, 32);
            const int64_t a = csr_off(D.indptr, CMP, r0 + (lane < nrw ? lane : nrw));
            const int64_t B = csr_off(D.indptr, CMP, r0 + nrw);
            const int64_t A = __shfl_sync(0xffffffffu, a, 0);
            int64_t nx = __shfl_down_sync(0xffffffffu, a, 1);
            if (lane == 31) nx = B;
            const bool ok = A >= 0 && B >= A && B <= nnz && B - A < (1ll << 30) && (lane >= nrw || nx >= a);
            if (!__all_sync(0xffffffffu, ok)) {  // a malformed row: flagged, the word not read
                bad = 1;
                continue;
            }
            const int ar = (int)(a - A), span = (int)(B - A);  // lanes past the last row hold span
            const Id *const src = ids + A;
            uint32_t *const trow = tile + g * ms;
            for (int base = 0; base < span; base += 32 * U) {
                int32_t it[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int p = base + 32 * u + lane;
                    it[u] = p < span ? (int32_t)__ldg(src + p) : 0;
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    if (base + 32 * u >= span) break;  // warp-uniform
                    const int p = base + 32 * u + lane;
                    int r = 0;  // last row whose start is <= p
#pragma unroll
                    for (int st = 16; st > 0; st >>= 1) {
                        const int c = __shfl_sync(0xffffffffu, ar, r + st);
                        if (c <= p) r += st;
                    }
                    if (p < span) {
                        if ((unsigned)it[u] >= (unsigned)m) {
                            bad = 1;
                            continue;
                        }
                        atomicOr(trow + it[u], 1u << r);
                    }
                }
            }
        }
    } else {
        for (int g = warp; g < WBK; g += NWARP) {
            const int64_t r = t0 + 32 * g + lane;
            if (r < n) {
                int64_t e0 = csr_off(D.indptr, CMP, r), e1 = csr_off(D.indptr, CMP, r + 1);
                if (e1 < e0 || e0 < 0 || e1 > nnz) {  // a malformed row: flagged, not read
                    bad = 1;
                    e1 = e0;
                }
                uint32_t *const trow = tile + g * ms;
                const uint32_t bit = 1u << lane;
                // four independent loads in flight per lane
                for (int64_t e = e0; e < e1; e += 4) {
                    int32_t it[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) it[u] = e + u < e1 ? (int32_t)__ldg(ids + e + u) : 0;
#pragma unroll
                    for (int u = 0; u < 4; u++)
                        if (e + u < e1) {
                            if ((unsigned)it[u] >= (unsigned)m) {
                                bad = 1;
                                continue;
                            }
                            atomicOr(trow + it[u], bit);
                        }
                }
            }
        }
    }
    if (bad) atomicExch(flag, 1);
    __syncthreads();
    for (int base = 0; base < m * QPC; base += BUILD_ROWS_THREADS) {  // warp-uniform trips
        const int k = base + threadIdx.x;
        const int j = k / QPC, q = k % QPC;
        uint32_t c = 0;
        if (j < m) {
            uint4 v;
            v.x = tile[(4 * q + 0) * ms + j];
            v.y = tile[(4 * q + 1) * ms + j];
            v.z = tile[(4 * q + 2) * ms + j];
            v.w = tile[(4 * q + 3) * ms + j];
            *reinterpret_cast<uint4 *>(col0 + (int64_t)j * D.nwp + w0 + 4 * q) = v;
            c = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        }
#pragma unroll
        for (int o = QPC / 2; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (j < m && q == 0 && c) atomicAdd(&sup[D.item_off + j], c);
    }
}

template <int WBK, bool COAL, bool PERSIST>
__global__ void __launch_bounds__(BUILD_ROWS_THREADS)
batch_build_rows_kernel(const BuildUnit *__restrict__ units, int64_t unit_base, int64_t unit_end,
                        uint32_t *__restrict__ sup, int *__restrict__ flag) {
    extern __shared__ __align__(16) uint32_t tile[];  // [WBK][ms]
    auto one = [&](int64_t u) {
        const BuildUnit D = units[u];
        if (D.compact) build_rows_unit<WBK, COAL, true>(D, sup, flag, tile);
        else build_rows_unit<WBK, COAL, false>(D, sup, flag, tile);
    };
    if (!PERSIST) {
        one(unit_base + blockIdx.x);
        return;
    }
    for (int64_t u = unit_base + blockIdx.x; u < unit_end; u += gridDim.x) {
        one(u);
        __syncthreads();  // the tile has been written out before the next unit clears it
    }
}

using BuildRowsFn = void (*)(const BuildUnit *, int64_t, int64_t, uint32_t *, int *);
template <int WBK>
BuildRowsFn build_rows_fn_w(bool coal, bool persist) {
    return coal ? (persist ? batch_build_rows_kernel<WBK, true, true> : batch_build_rows_kernel<WBK, true, false>)
                : (persist ? batch_build_rows_kernel<WBK, false, true> : batch_build_rows_kernel<WBK, false, false>);
}
BuildRowsFn build_rows_fn(int wbk, bool coal, bool persist) {
    return wbk == 64 ? build_rows_fn_w<64>(coal, persist)
           : wbk == 16 ? build_rows_fn_w<16>(coal, persist) : build_rows_fn_w<32>(coal, persist);
}

// a group's window of the root arrays: where its finalize starts appending,
// and how many roots it appended
__global__ void window_begin_kernel(const MineCounters *__restrict__ ctr, RootWindow *__restrict__ w) {
    w->base = *(volatile const unsigned long long *)&ctr->n_roots;
    w->count = w->kept = w->ticket = 0;
}
__global__ void window_end_kernel(const MineCounters *__restrict__ ctr, RootWindow *__restrict__ w) {
    w->count = *(volatile const unsigned long long *)&ctr->n_roots - w->base;
}

// the rows build's unit table: one CTA per database writes its units
__global__ void batch_unit_db_kernel(const DbDesc *__restrict__ dbs, const int64_t *__restrict__ unit_prefix,
                                     int wbk, uint32_t *__restrict__ bm, BuildUnit *__restrict__ units) {
    const int d = blockIdx.x;
    const DbDesc &D = dbs[d];
    const int64_t u0 = unit_prefix[d];
    for (int64_t u = u0 + threadIdx.x; u < unit_prefix[d + 1]; u += blockDim.x) {
        BuildUnit b;
        b.indptr = D.indptr;
        b.indices = D.indices;
        b.col0 = bm + D.bm_off;
        b.n = D.n;
        b.nwp = D.nwp;
        b.item_off = D.item_off;
        b.w0 = (u - u0) * wbk;
        b.m = D.m;
        b.compact = D.compact;
        units[u] = b;
    }
}

// One CTA per item column of the batch: S(I_j) by popcount.
__global__ void __launch_bounds__(256)
batch_support_kernel(const DbDesc *__restrict__ dbs, int n_db, const int64_t *__restrict__ item_prefix,
                     const uint32_t *__restrict__ bm, uint32_t *__restrict__ sup) {
    const int d = find_db(item_prefix, n_db, blockIdx.x);
    const DbDesc &D = dbs[d];
    const int64_t j = blockIdx.x - item_prefix[d];
    const uint32_t *col = bm + D.bm_off + j * D.nwp;
    uint32_t c = 0;
    for (int64_t w = 4 * threadIdx.x; w < D.nwp; w += 4 * blockDim.x) {
        const uint4 v = ldg_u4(col + w);
        c += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
    }
    c = warp_sum_u32(c);
    __shared__ uint32_t s[8];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += s[k];
        sup[D.item_off + j] = t;
    }
}

// One warp per item: internal id = rank among the database's frequent items
// by (support, id); frequent items become singleton records.
__global__ void batch_rank_kernel(DbDesc *__restrict__ dbs, int n_db, const int64_t *__restrict__ item_prefix,
                                  int64_t n_items, const uint32_t *__restrict__ sup, int32_t *__restrict__ perm,
                                  MineCounters *ctr, unsigned long long *rec_off, uint32_t *rec_len,
                                  uint32_t *rec_sup, uint32_t *rec_items, uint32_t *rec_db,
                                  unsigned long long rec_cap, unsigned long long items_cap) {
    const int lane = threadIdx.x & 31;
    const int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gi >= n_items) return;
    const int d = find_db(item_prefix, n_db, gi);
    DbDesc &D = dbs[d];
    const int j = (int)(gi - D.item_off);
    const uint32_t *s = sup + D.item_off;
    const uint32_t sj = s[j];
    if (sj < D.thr) return;
    uint32_t below = 0;
    for (int i = lane; i < D.m; i += 32) {
        const uint32_t si = s[i];
        below += (si >= D.thr) && (si < sj || (si == sj && i < j));
    }
    below = warp_sum_u32(below);
    if (lane == 0) {
        perm[D.item_off + below] = j;
        atomicAdd(&D.mfreq, 1);
        const unsigned long long r = atomicAdd(&ctr->n_records, 1ull);
        const unsigned long long it = atomicAdd(&ctr->n_rec_items, 1ull);
        if (r < rec_cap && it < items_cap) {
            rec_off[r] = it;
            rec_len[r] = 1;
            rec_sup[r] = sj;
            rec_items[it] = below;
            rec_db[r] = (uint32_t)d;
        } else {
            atomicOr(&ctr->overflow, r < rec_cap ? 2 : 1);
        }
        if (D.maxlen == 0 || D.maxlen >= 1) atomicMax(&ctr->max_len, 1);
    }
}

// One CTA per database, the database's frequent items at most RANK_CAP:
// threads flag the frequent items, a block scan lists them in id order in
// shared memory, and each ranks its item among them by (support, id) -- the
// internal id (Eq. 3's threshold, then the relabelling of the miner).  The
// database's singleton records and m' are published with one global atomic
// per counter, not one per item.
constexpr int RANK_THREADS = 256;
constexpr int RANK_CAP = 4096;
__global__ void __launch_bounds__(RANK_THREADS)
batch_rank_db_kernel(DbDesc *__restrict__ dbs, int d0, const uint32_t *__restrict__ sup, int32_t *__restrict__ perm,
                     MineCounters *ctr, unsigned long long *rec_off, uint32_t *rec_len, uint32_t *rec_sup,
                     uint32_t *rec_items, uint32_t *rec_db, unsigned long long rec_cap,
                     unsigned long long items_cap) {
    __shared__ uint32_t f_sup[RANK_CAP];
    __shared__ int32_t f_id[RANK_CAP];
    __shared__ uint32_t s_warp[RANK_THREADS / 32 + 1];
    __shared__ unsigned long long s_base[2];
    __shared__ int s_nf;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = d0 + (int)blockIdx.x;
    DbDesc &D = dbs[d];
    const int m = D.m;
    const uint32_t *sp = sup + D.item_off;
    const uint32_t thr = D.thr;
    if (threadIdx.x == 0) s_nf = 0;
    __syncthreads();
    // compact the frequent items, ascending id, in chunks of RANK_THREADS
    for (int j0 = 0; j0 < m; j0 += RANK_THREADS) {
        const int j = j0 + threadIdx.x;
        const uint32_t sj = j < m ? sp[j] : 0u;
        const bool f = j < m && sj >= thr;
        const uint32_t bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) s_warp[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t acc = 0;
            for (int w = 0; w < RANK_THREADS / 32; w++) {
                const uint32_t t = s_warp[w];
                s_warp[w] = acc;
                acc += t;
            }
            s_warp[RANK_THREADS / 32] = acc;
        }
        __syncthreads();
        const int at = s_nf + (int)s_warp[warp] + __popc(bal & ((1u << lane) - 1u));
        if (f && at < RANK_CAP) {
            f_sup[at] = sj;
            f_id[at] = j;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_nf += (int)s_warp[RANK_THREADS / 32];
        __syncthreads();
    }
    const int mf = s_nf;  // <= RANK_CAP: the host picks this kernel only for m <= RANK_CAP
    if (threadIdx.x == 0) {
        D.mfreq = mf;
        s_base[0] = mf ? atomicAdd(&ctr->n_records, (unsigned long long)mf) : 0ull;
        s_base[1] = mf ? atomicAdd(&ctr->n_rec_items, (unsigned long long)mf) : 0ull;
        if (mf && (D.maxlen == 0 || D.maxlen >= 1)) atomicMax(&ctr->max_len, 1);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < mf; k += RANK_THREADS) {
        const uint32_t sk = f_sup[k];
        int below = 0;
        for (int i = 0; i < mf; i++) {  // every thread reads f_sup[i] at once: a broadcast
            const uint32_t si = f_sup[i];
            below += si < sk || (si == sk && i < k);
        }
        perm[D.item_off + below] = f_id[k];
        const unsigned long long r = s_base[0] + below, it = s_base[1] + below;
        if (r < rec_cap && it < items_cap) {
            rec_off[r] = it;
            rec_len[r] = 1;
            rec_sup[r] = sk;
            rec_items[it] = (uint32_t)below;
            rec_db[r] = (uint32_t)d;
        } else {
            atomicOr(&ctr->overflow, r < rec_cap ? 2 : 1);
        }
    }
}

// One CTA per database with at most FIN_CAP frequent items: the threshold
// on every pair (Eq. 3), the pair bitset, and the pair records and root
// classes.  A warp takes rows a; a first pass counts each row's frequent
// pairs and writes the bitset, a block scan gives each row its place, and a
// second pass writes the records: one global atomic per counter and
// database.
constexpr int FIN_THREADS = 512;
constexpr int FIN_CAP = 4096;
__global__ void __launch_bounds__(FIN_THREADS)
batch_finalize_db_kernel(const DbDesc *__restrict__ dbs, int d0, const int *__restrict__ pair_cnt,
                         uint32_t *__restrict__ pairbits, MineCounters *ctr, unsigned long long *rec_off,
                         uint32_t *rec_len, uint32_t *rec_sup, uint32_t *rec_items, uint32_t *rec_db,
                         unsigned long long rec_cap, unsigned long long items_cap, uint32_t *root_a,
                         uint32_t *root_b, uint32_t *root_sup, uint32_t *root_db) {
    __shared__ uint32_t s_off[FIN_CAP + 1];
    __shared__ uint32_t s_warp[FIN_THREADS / 32 + 1];
    __shared__ unsigned long long s_base[3];
    constexpr int NW = FIN_THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = d0 + (int)blockIdx.x;
    const DbDesc &D = dbs[d];
    const int mf = *(volatile const int32_t *)&D.mfreq;
    const int mpw = (mf + 31) / 32;
    const bool emit = D.maxlen == 0 || D.maxlen >= 2;
    const int *cnt = pair_cnt + D.pair_off;
    uint32_t *pb = pairbits + D.pb_off;
    // pass 1: bitset rows and per-row counts
    for (int a = warp; a < mf; a += NW) {
        const int *row = cnt + (int64_t)a * mf;
        uint32_t c = 0;
        for (int w = (a + 1) >> 5; w < mpw; w++) {
            const int b = w * 32 + lane;
            const bool f = emit && b > a && b < mf && (uint32_t)row[b] >= D.thr;
            const uint32_t bal = __ballot_sync(0xffffffffu, f);
            if (lane == 0) pb[(int64_t)a * mpw + w] = bal;
            c += __popc(bal);
        }
        for (int w = lane; w < ((a + 1) >> 5); w += 32) pb[(int64_t)a * mpw + w] = 0u;  // words left of a
        if (lane == 0) s_off[a] = c;
    }
    __syncthreads();
    // exclusive scan of the row counts (mf <= FIN_CAP: at most 8 per thread)
    constexpr int PER = (FIN_CAP + FIN_THREADS - 1) / FIN_THREADS;
    uint32_t v[PER], sum = 0;
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int a = threadIdx.x * PER + i;
        v[i] = a < mf ? s_off[a] : 0u;
        sum += v[i];
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int w = 0; w < NW; w++) {
            const uint32_t t = s_warp[w];
            s_warp[w] = acc;
            acc += t;
        }
        s_warp[NW] = acc;
    }
    __syncthreads();
    uint32_t run = s_warp[warp] + x - sum;
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int a = threadIdx.x * PER + i;
        if (a < mf) s_off[a] = run;
        run += v[i];
    }
    const uint32_t total = s_warp[NW];
    if (threadIdx.x == 0 && total) {
        s_base[0] = atomicAdd(&ctr->n_records, (unsigned long long)total);
        s_base[1] = atomicAdd(&ctr->n_rec_items, 2ull * total);
        s_base[2] = atomicAdd(&ctr->n_roots, (unsigned long long)total);
        atomicAdd((unsigned long long *)&ctr->pending, (unsigned long long)total);
        atomicMax(&ctr->max_len, 2);
    }
    __syncthreads();
    if (!total) return;
    // pass 2: the records, in (a, b) order within the database
    for (int a = warp; a < mf; a += NW) {
        const int *row = cnt + (int64_t)a * mf;
        uint32_t pos = s_off[a];
        for (int w = (a + 1) >> 5; w < mpw; w++) {
            const uint32_t bal = pb[(int64_t)a * mpw + w];
            if (!bal) continue;
            const int b = w * 32 + lane;
            if ((bal >> lane) & 1u) {
                const uint32_t p = pos + __popc(bal & ((1u << lane) - 1u));
                const uint32_t sv = (uint32_t)row[b];
                const unsigned long long r = s_base[0] + p, it = s_base[1] + 2ull * p, q = s_base[2] + p;
                if (r < rec_cap && it + 2 <= items_cap) {
                    rec_off[r] = it;
                    rec_len[r] = 2;
                    rec_sup[r] = sv;
                    rec_db[r] = (uint32_t)d;
                    rec_items[it] = (uint32_t)a;
                    rec_items[it + 1] = (uint32_t)b;
                } else {
                    atomicOr(&ctr->overflow, r < rec_cap ? 2 : 1);
                }
                root_a[q] = (uint32_t)a;
                root_b[q] = (uint32_t)b;
                root_sup[q] = sv;
                root_db[q] = (uint32_t)d;
            }
            pos += __popc(bal);
        }
    }
}

// Pair supports of a database with at most 64 frequent items, in one CTA:
// the threads cover only the upper-triangle 4 x 4 blocks of the m' x m'
// pair matrix (nb (nb + 1) / 2 of them, nb = ceil(m' / 4)), and the CTA's
// spare threads split the transactions into KG groups whose partial counts
// meet in shared memory.  Every 4 x 4 block holds at least one pair a < b.
__device__ void small_pairs(const DbDesc &D, int mf, const uint32_t *__restrict__ col0,
                            const int32_t *__restrict__ perm, int *__restrict__ out, uint32_t *smem) {
    __shared__ int64_t s_col[TI];
    const int nb = (mf + 3) >> 2;
    const int nblk = nb * (nb + 1) / 2;
    const int KG = 256 / nblk >= 4 ? 4 : (256 / nblk >= 2 ? 2 : 1);
    const int t = threadIdx.x;
    const bool act = t < nblk * KG;
    const int blk = t % nblk, kg = t / nblk;
    int bi = 0, r = blk;
    while (r >= nb - bi) { r -= nb - bi; bi++; }
    const int bj = bi + r;
    if (t < TI) s_col[t] = t < mf ? (int64_t)perm[t] * D.nwp : -1;
    uint32_t (*S)[KW][TI] = reinterpret_cast<uint32_t (*)[KW][TI]>(smem);  // [KG][KW][TI]
    uint32_t acc[4][4] = {};
    const int64_t step = (int64_t)KW * KG;  // divides the 128-word column padding
    for (int64_t k = 0; k < D.nw; k += step) {
        __syncthreads();
        // a thread copies 8 words (one 32-byte sector) of one row; consecutive
        // threads take consecutive rows, so the transposed stores are
        // conflict-free
        for (int e = t; e < KG * TI * (KW / 8); e += blockDim.x) {
            const int row = e % TI, q = (e / TI) % (KW / 8), g = e / (TI * (KW / 8));
            uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
            if (s_col[row] >= 0) {
                const uint32_t *src = col0 + s_col[row] + k + (int64_t)g * KW + 8 * q;
                v0 = ldg_u4(src);
                v1 = ldg_u4(src + 4);
            }
            const uint32_t w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
            for (int c = 0; c < 8; c++) S[g][8 * q + c][row] = w[c];
        }
        __syncthreads();
        if (act) {
#pragma unroll 8
            for (int kk = 0; kk < KW; kk++) {
                const uint4 a = *reinterpret_cast<const uint4 *>(&S[kg][kk][bi * 4]);
                const uint4 b = *reinterpret_cast<const uint4 *>(&S[kg][kk][bj * 4]);
                const uint32_t x[4] = {a.x, a.y, a.z, a.w}, y[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] += __popc(x[i] & y[j]);
            }
        }
    }
    // the KG partial counts meet in shared memory (the staging area, reused)
    int (*R)[TI] = reinterpret_cast<int (*)[TI]>(smem);
    __syncthreads();
    for (int e = t; e < TI * TI; e += blockDim.x) R[e / TI][e % TI] = 0;
    __syncthreads();
    if (act)
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (acc[i][j]) atomicAdd(&R[bi * 4 + i][bj * 4 + j], (int)acc[i][j]);
    __syncthreads();
    for (int e = t; e < mf * mf; e += blockDim.x) {
        const int a = e / mf, b = e % mf;
        if (a < b) out[e] = R[a][b];
    }
}

// Pair supports of one 64 x 64 tile of one database (CUDA cores, exact).
__global__ void __launch_bounds__(256)
batch_pairs_kernel(const DbDesc *__restrict__ dbs, int n_db, const int64_t *__restrict__ tile_prefix,
                   const uint32_t *__restrict__ bm, const int32_t *__restrict__ perm_base,
                   int *__restrict__ pair_cnt) {
    __shared__ __align__(16) uint32_t smem[4 * KW * TI];  // 32 KB
    uint32_t (*As)[TI] = reinterpret_cast<uint32_t (*)[TI]>(smem);
    uint32_t (*Bs)[TI] = reinterpret_cast<uint32_t (*)[TI]>(smem + KW * TI);
    const int d = find_db(tile_prefix, n_db, blockIdx.x);
    const DbDesc &D = dbs[d];
    const int mf = *(volatile const int32_t *)&D.mfreq;
    const int nt = (D.m + TI - 1) / TI;
    int idx = (int)(blockIdx.x - tile_prefix[d]), ta = 0;
    while (idx >= nt - ta) { idx -= nt - ta; ta++; }
    const int tb = ta + idx;
    if (tb * TI >= mf || D.maxlen == 1) return;
    const int32_t *perm = perm_base + D.item_off;
    const uint32_t *col0 = bm + D.bm_off;
    if (mf <= TI) {  // one tile: only its upper triangle, with the spare threads on K
        small_pairs(D, mf, col0, perm, pair_cnt + D.pair_off, smem);
        return;
    }
    const int t = threadIdx.x, lr = t & 63, lc = (t >> 6) * 8;
    const int ra = ta * TI + lr, rb = tb * TI + lr;
    const uint32_t *pa = ra < mf ? col0 + (int64_t)perm[ra] * D.nwp : nullptr;
    const uint32_t *pb = rb < mf ? col0 + (int64_t)perm[rb] * D.nwp : nullptr;
    const int ty = t >> 4, tx = t & 15;
    uint32_t acc[4][4] = {};
    for (int64_t k = 0; k < D.nw; k += KW) {
        uint4 a0 = make_uint4(0, 0, 0, 0), a1 = a0, b0 = a0, b1 = a0;
        if (pa) { a0 = ldg_u4(pa + k + lc); a1 = ldg_u4(pa + k + lc + 4); }
        if (pb) { b0 = ldg_u4(pb + k + lc); b1 = ldg_u4(pb + k + lc + 4); }
        __syncthreads();
        const uint32_t av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const uint32_t bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int q = 0; q < 8; q++) { As[lc + q][lr] = av[q]; Bs[lc + q][lr] = bv[q]; }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < KW; kk++) {
            const uint4 a = *reinterpret_cast<const uint4 *>(&As[kk][ty * 4]);
            const uint4 b = *reinterpret_cast<const uint4 *>(&Bs[kk][tx * 4]);
            const uint32_t x[4] = {a.x, a.y, a.z, a.w}, y[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] += __popc(x[i] & y[j]);
        }
    }
    int *out = pair_cnt + D.pair_off;
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int a = ta * TI + ty * 4 + i, b = tb * TI + tx * 4 + j;
            if (a < b && b < mf) out[(int64_t)a * mf + b] = (int)acc[i][j];
        }
}

// One warp per (database, row a): threshold, pair bitset, pair records, roots.
__global__ void __launch_bounds__(256)
batch_finalize_kernel(const DbDesc *__restrict__ dbs, int n_db, const int64_t *__restrict__ item_prefix,
                      int64_t n_items,
                      const int *__restrict__ pair_cnt, uint32_t *__restrict__ pairbits, MineCounters *ctr,
                      unsigned long long *rec_off, uint32_t *rec_len, uint32_t *rec_sup, uint32_t *rec_items,
                      uint32_t *rec_db, unsigned long long rec_cap, unsigned long long items_cap,
                      uint32_t *root_a, uint32_t *root_b, uint32_t *root_sup, uint32_t *root_db) {
    const int lane = threadIdx.x & 31;
    const int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gi >= n_items) return;
    const int d = find_db(item_prefix, n_db, gi);
    const DbDesc &D = dbs[d];
    const int a = (int)(gi - item_prefix[d]);
    const int mf = *(volatile const int32_t *)&D.mfreq;
    if (a >= mf) return;
    const int mpw = (mf + 31) / 32;
    const int *row = pair_cnt + D.pair_off + (int64_t)a * mf;
    const bool emit = D.maxlen == 0 || D.maxlen >= 2;
    for (int w = 0; w < mpw; w++) {
        const int b = w * 32 + lane;
        const uint32_t s = (b > a && b < mf) ? (uint32_t)row[b] : 0u;
        const bool f = emit && b > a && b < mf && s >= D.thr;
        const uint32_t bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) pairbits[D.pb_off + (int64_t)a * mpw + w] = bal;
        if (bal == 0) continue;
        const int cnt = __popc(bal);
        unsigned long long rbase = 0, ibase = 0, root = 0;
        if (lane == 0) {
            rbase = atomicAdd(&ctr->n_records, (unsigned long long)cnt);
            ibase = atomicAdd(&ctr->n_rec_items, 2ull * cnt);
            root = atomicAdd(&ctr->n_roots, (unsigned long long)cnt);
            atomicAdd((unsigned long long *)&ctr->pending, (unsigned long long)cnt);
            atomicMax(&ctr->max_len, 2);
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
                rec_db[r] = (uint32_t)d;
                rec_items[it] = (uint32_t)a;
                rec_items[it + 1] = (uint32_t)b;
            } else {
                atomicOr(&ctr->overflow, r < rec_cap ? 2 : 1);
            }
            root_a[root + pos] = (uint32_t)a;
            root_b[root + pos] = (uint32_t)b;
            root_sup[root + pos] = s;
            root_db[root + pos] = (uint32_t)d;
        }
    }
}

// Result slice of every database in the sorted output: count, scan, item base.
__global__ void db_count_kernel(const uint32_t *__restrict__ rec_db, unsigned long long R,
                                unsigned long long *__restrict__ cnt) {
    const unsigned long long r = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) {
        const uint32_t d = rec_db[r];
        if (d != 0xFFFFFFFFu) atomicAdd(&cnt[d], 1ull);  // holes carry no database
    }
}

__global__ void __launch_bounds__(1024)
db_scan_kernel(unsigned long long *__restrict__ a, int n, const unsigned long long *__restrict__ out_off,
               unsigned long long *__restrict__ item_start) {
    __shared__ unsigned long long s[1024];
    const int seg = (n + 1 + 1023) / 1024;
    const int b = threadIdx.x * seg, e = min(b + seg, n + 1);
    unsigned long long sum = 0;
    for (int i = b; i < e; i++) sum += (i < n) ? a[i] : 0ull;
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
        const unsigned long long v = (i < n) ? a[i] : 0ull;
        a[i] = run;  // exclusive: a[d] = first sorted record of database d; a[n] = R
        item_start[i] = out_off[run];
        run += v;
    }
}

__global__ void rebase_kernel(unsigned long long *__restrict__ off, uint64_t n, unsigned long long base) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) off[i] -= base;
}

struct Layout {
    std::vector<DbDesc> dbs;
    std::vector<int64_t> unit_prefix, item_prefix, tile_prefix;
    int64_t words = 0, items = 0, pairs = 0, pb = 0, root_cap = 0, nwp_max = 0, max_row_bound = 0;
    int m_max = 0, ib = 1;
};

// True when every range lies inside one page-locked host allocation that the
// GPU addresses at the host address itself (unified addressing): the start
// and the last byte of a range must be the same allocation (driver buffer
// id), so no pageable memory can sit inside it.
bool mapped_host_ranges(const std::vector<std::pair<const char *, size_t>> &runs) {
    static CUresult (*get_attrs)(unsigned, CUpointer_attribute *, void **, CUdeviceptr) = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPoint("cuPointerGetAttributes", &fn, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_attrs = reinterpret_cast<CUresult (*)(unsigned, CUpointer_attribute *, void **, CUdeviceptr)>(fn);
        cudaGetLastError();
    }
    if (!get_attrs || runs.empty()) return false;
    for (const auto &r : runs) {
        unsigned long long id[2] = {0, 0};
        for (int e = 0; e < 2; e++) {
            const char *p = e == 0 ? r.first : r.first + r.second - 1;
            cudaPointerAttributes a{};
            if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeHost ||
                a.devicePointer != (const void *)p) {
                cudaGetLastError();  // a query on unregistered memory leaves no sticky error
                return false;
            }
            CUpointer_attribute which = CU_POINTER_ATTRIBUTE_BUFFER_ID;
            void *out = &id[e];
            if (get_attrs(1, &which, &out, (CUdeviceptr)(uintptr_t)p) != CUDA_SUCCESS) return false;
        }
        if (id[0] == 0 || id[0] != id[1]) return false;
    }
    return true;
}

}  // namespace

extern "C" {

int fim_mine_batched(fim_ctx *ctx, int n_db, const fim_db_desc *in, uint32_t flags) {
    FIM_NVTX("fim_mine_batched");
    if (!ctx || n_db <= 0 || n_db > (1 << 20) || !in) return FIM_E_INVAL;
    if (flags & (FIM_TRACE | FIM_PAIRS_POPC)) {
        // traces are per single mine; the batched pair pass is the CUDA-core one
        if (flags & FIM_TRACE) return FIM_E_INVAL;
    }
    if ((flags & FIM_LEARNED) && !ctx->has_weights) return FIM_E_STATE;
    // pair supports on the tensor cores unless FIM_PAIRS_POPC asks for the
    // CUDA-core tiles
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FIM_E_CUDA;
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{dev_prev};
    cudaStream_t st = ctx->stream;
    const bool on_device = flags & FIM_INPUT_DEVICE;
    const uint32_t maxlen = flags >> 24;
    FIM_TRY(fim_finish_phase_times(ctx));  // before the events are recorded again
    ctx->mined = false;
    ctx->built = false;
    ctx->batch_mined = false;

    // ---- layout (host) -----------------------------------------------------
    Layout L;
    L.dbs.resize(n_db);
    L.unit_prefix.assign(n_db + 1, 0);
    L.item_prefix.assign(n_db + 1, 0);
    L.tile_prefix.assign(n_db + 1, 0);
    for (int d = 0; d < n_db; d++) L.m_max = in[d].n_items > L.m_max ? in[d].n_items : L.m_max;
    L.ib = L.m_max < 1024 ? (L.m_max > 0 ? L.m_max : 1) : 1024;
    // rows build (every database's columns fit one CTA's shared memory):
    // words per block as tuned, where the block's tile fits
    const bool rows_build = L.ib == L.m_max;
    int wbk = ctx->batch_build_block == 64 ? 64 : ctx->batch_build_block == 16 ? 16 : 32;
    if ((size_t)wbk * (size_t)(L.m_max | 1) * sizeof(uint32_t) > 227u * 1024u) wbk = 32;
    const int unit_words = rows_build ? wbk : WB;
    // the CSR's element types (FIM_CSR_COMPACT: uint32 row offsets, uint16 ids)
    const bool cmp = (flags & FIM_CSR_COMPACT) != 0;
    const size_t pb = csr_off_bytes(cmp), ib = csr_id_bytes(cmp);
    auto host_nnz = [cmp](const fim_db_desc &x) { return csr_off(x.indptr, cmp, x.n_trans); };
    int64_t host_nnz_total = 0, host_ptr_total = 0;
    for (int d = 0; d < n_db; d++) {
        const fim_db_desc &x = in[d];
        if (x.n_trans < 0 || x.n_trans > FIM_MAX_TRANS || x.n_items < 0 || x.n_items > FIM_MAX_ITEMS ||
            !x.indptr)
            return FIM_E_INVAL;
        if (!(flags & FIM_STRICT) && x.minsup == 0) return FIM_E_INVAL;
        DbDesc &D = L.dbs[d];
        D = DbDesc{};
        D.n = x.n_trans;
        D.m = x.n_items;
        D.nw = ceil_div64(D.n, 32);
        D.nwp = round_up64(D.nw, FIM_WORDS_ALIGN);
        uint64_t thr = (flags & FIM_STRICT) ? x.minsup + 1 : x.minsup;
        if ((flags & FIM_STRICT) && x.minsup == UINT64_MAX) thr = UINT64_MAX;
        D.thr = thr > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)thr;
        D.maxlen = maxlen;
        D.compact = cmp ? 1 : 0;
        D.bm_off = L.words;
        D.item_off = L.items;
        D.pair_off = L.pairs;
        D.pb_off = L.pb;
        L.words += (int64_t)D.m * D.nwp;
        L.items += D.m;
        L.pairs += (int64_t)D.m * D.m;
        L.pb += (int64_t)D.m * ceil_div64(D.m, 32);
        L.root_cap += (int64_t)D.m * (D.m > 0 ? D.m - 1 : 0) / 2;
        L.nwp_max = D.nwp > L.nwp_max ? D.nwp : L.nwp_max;
        const int nt = (int)ceil_div64(D.m, TI);
        L.unit_prefix[d + 1] = L.unit_prefix[d] + (D.m > 0 ? (D.nwp / unit_words) * ceil_div64(D.m, L.ib) : 0);
        L.item_prefix[d + 1] = L.items;
        L.tile_prefix[d + 1] = L.tile_prefix[d] + (int64_t)nt * (nt + 1) / 2;
        if (D.m > L.max_row_bound) L.max_row_bound = D.m;
        if (!on_device) {
            const int64_t nnz = host_nnz(x);
            if (csr_off(x.indptr, cmp, 0) != 0 || nnz < 0 || (nnz > 0 && !x.indices)) return FIM_E_INVAL;
            host_nnz_total += nnz;
            host_ptr_total += x.n_trans + 1;
        }
    }
    // ---- inputs: host CSRs in page-locked memory are read in place ----------
    // (the build kernel streams them over the host link, which caps copies
    // and in-kernel reads alike, so the upload and the build become one pass);
    // other host memory goes up in one staging copy per contiguous run
    bool mapped = false, streamed = false;
    if (!on_device && ctx->upload_mapped) {
        // contiguous host ranges of the indptr arrays and of the index arrays
        std::vector<std::pair<const char *, size_t>> rp, ri;
        auto note = [](std::vector<std::pair<const char *, size_t>> &runs, const void *p, size_t bytes) {
            if (!bytes) return;
            if (!runs.empty() && runs.back().first + runs.back().second == (const char *)p)
                runs.back().second += bytes;
            else
                runs.push_back({(const char *)p, bytes});
        };
        for (int d = 0; d < n_db && rp.size() + ri.size() <= 64; d++) {
            note(rp, in[d].indptr, pb * (size_t)(in[d].n_trans + 1));
            note(ri, in[d].indices, ib * (size_t)host_nnz(in[d]));
        }
        rp.insert(rp.end(), ri.begin(), ri.end());
        // page-locked: streamed up group by group inside the graph (copies
        // beside the mine), or read in place by the build
        const bool locked = rp.size() <= 64 && mapped_host_ranges(rp);
        streamed = locked && ctx->batch_stream_copies;
        mapped = locked && !streamed;
        if (mapped)
            for (int d = 0; d < n_db; d++) {
                L.dbs[d].indptr = in[d].indptr;  // unified addressing: the host address is the device address
                L.dbs[d].indices = in[d].indices;
            }
    }
    if (!on_device && !mapped) {
        FIM_TRY(fim_reserve(ctx, ctx->csr_ptr, pb * (size_t)(host_ptr_total ? host_ptr_total : 1)));
        FIM_TRY(fim_reserve(ctx, ctx->csr_idx, ib * (size_t)(host_nnz_total ? host_nnz_total : 1)));
        // databases whose arrays follow each other in host memory (one packed
        // buffer) go up in one copy per run instead of one per database
        struct Run { const char *src = nullptr; char *dst = nullptr; size_t bytes = 0; };
        Run rp, ri;
        auto flush = [&](Run &r) -> int {
            if (r.bytes) FIM_CUDA_TRY(cudaMemcpyAsync(r.dst, r.src, r.bytes, cudaMemcpyHostToDevice, st));
            r = Run{};
            return FIM_OK;
        };
        auto add = [&](Run &r, const void *src, void *dst, size_t bytes) -> int {
            if (!bytes) return FIM_OK;
            if (r.bytes && r.src + r.bytes == (const char *)src && r.dst + r.bytes == (char *)dst) {
                r.bytes += bytes;
                return FIM_OK;
            }
            FIM_TRY(flush(r));
            r.src = (const char *)src;
            r.dst = (char *)dst;
            r.bytes = bytes;
            return FIM_OK;
        };
        int64_t po = 0, io = 0;  // elements of the staging arrays
        char *const sp = ctx->csr_ptr.as<char>(), *const si = ctx->csr_idx.as<char>();
        for (int d = 0; d < n_db; d++) {
            const fim_db_desc &x = in[d];
            const int64_t nnz = host_nnz(x);
            if (!streamed) {  // streamed: the graph copies each group of databases
                FIM_TRY(add(rp, x.indptr, sp + pb * (size_t)po, pb * (size_t)(x.n_trans + 1)));
                if (nnz > 0) FIM_TRY(add(ri, x.indices, si + ib * (size_t)io, ib * (size_t)nnz));
            }
            L.dbs[d].indptr = sp + pb * (size_t)po;
            L.dbs[d].indices = si + ib * (size_t)io;
            po += x.n_trans + 1;
            io += nnz;
        }
        FIM_TRY(flush(rp));
        FIM_TRY(flush(ri));
    } else {
        for (int d = 0; d < n_db; d++) {
            L.dbs[d].indptr = in[d].indptr;
            L.dbs[d].indices = in[d].indices;
        }
    }
    const bool coal = ctx->batch_build_coal != 0;  // warp-coalesced id loads in the build
    // Pipelined groups of databases: group s is built and ranked on the ctx
    // stream while the pair pass of group s - 1 runs on the side stream.
    // Groups hold about equal transactions.  Only the fast paths pipeline:
    // rows build, per-database rank and finalize, tensor-core pairs.
    const bool pairs_tc_wanted = !(flags & FIM_PAIRS_POPC);
    // Automatic (batch_segments 0): with page-locked host input the link
    // bounds the mine, so eight groups: each group's upload (streamed) or
    // build reading host memory in place (mapped, the build then one CTA per
    // SM) runs beside the earlier groups' work; else one group.
    const int seg_want = ctx->batch_segments > 0 ? ctx->batch_segments : (mapped || streamed ? 8 : 1);
    int n_seg = (pairs_tc_wanted && rows_build && L.m_max <= RANK_CAP && L.m_max <= FIN_CAP && maxlen != 1)
                    ? seg_want : 1;
    if (n_seg > n_db) n_seg = n_db > 0 ? n_db : 1;
    std::vector<int> seg_db(n_seg + 1, 0);
    {
        int64_t total_n = 0;
        for (int d = 0; d < n_db; d++) total_n += L.dbs[d].n + 1;
        int64_t acc = 0;
        int s = 1;
        for (int d = 0; d < n_db && s < n_seg; d++) {
            acc += L.dbs[d].n + 1;
            if (acc * n_seg >= total_n * s) seg_db[s++] = d + 1;
        }
        while (s < n_seg) { seg_db[s] = seg_db[s - 1]; s++; }
        seg_db[n_seg] = n_db;
    }
    // the tensor-core pair pass's (database, tile) units, each group's longest first
    // (they depend only on each database's (m, words) and the grouping: the
    // last batch's are reused when those repeat)
    bool pairs_tc = pairs_tc_wanted;
    if (pairs_tc) {
        std::vector<int64_t> sig;
        sig.reserve(2 * (size_t)n_db + (size_t)n_seg + 2);
        sig.push_back(n_seg);
        for (int sg = 0; sg <= n_seg; sg++) sig.push_back(seg_db[sg]);
        for (int d = 0; d < n_db; d++) {
            sig.push_back(L.dbs[d].m);
            sig.push_back(L.dbs[d].nw);
        }
        if (sig != ctx->pair_units_sig) {
            ctx->pair_units_cache.clear();
            ctx->pair_seg_unit_cache.assign(n_seg + 1, 0);
            ctx->pair_units_ok = true;
            for (int sg = 0; sg < n_seg && ctx->pair_units_ok; sg++) {
                ctx->pair_units_ok = batch_pairs_tc_units(L.dbs, seg_db[sg], seg_db[sg + 1], ctx->pair_units_cache,
                                                          (size_t)1 << 24);
                ctx->pair_seg_unit_cache[sg + 1] = (int64_t)ctx->pair_units_cache.size();
            }
            // the device plan's database order: each group's, most transactions first
            ctx->pair_ord_cache.resize(n_db);
            for (int sg = 0; sg < n_seg; sg++) {
                for (int d = seg_db[sg]; d < seg_db[sg + 1]; d++) ctx->pair_ord_cache[d] = d;
                std::stable_sort(ctx->pair_ord_cache.begin() + seg_db[sg], ctx->pair_ord_cache.begin() + seg_db[sg + 1],
                                 [&](int x, int y) { return L.dbs[x].nw > L.dbs[y].nw; });
            }
            ctx->pair_units_sig.swap(sig);
        }
        pairs_tc = ctx->pair_units_ok;
    }
    const std::vector<unsigned long long> &pair_units = ctx->pair_units_cache;
    const std::vector<int64_t> &seg_unit = ctx->pair_seg_unit_cache;
    // pair units planned on the device after the rank pass (two small
    // databases to a tile); the host's units then only bound their number
    const bool pack = pairs_tc && ctx->batch_pairs_pack;
    if (!pairs_tc) {
        n_seg = 1;
        seg_db.assign({0, n_db});
    }
    const bool persist_build = mapped && n_seg > 1;
    // streamed uploads: each group's runs of contiguous host arrays
    struct HostCopy {
        const char *src;
        char *dst;
        size_t bytes;
    };
    std::vector<std::vector<HostCopy>> seg_copies(streamed ? n_seg : 0);
    for (int sg = 0; streamed && sg < n_seg; sg++) {
        std::vector<HostCopy> cp_ptr, cp_idx;
        auto note = [](std::vector<HostCopy> &v, const void *src, const void *dst, size_t bytes) {
            if (!bytes) return;
            if (!v.empty() && v.back().src + v.back().bytes == (const char *)src &&
                v.back().dst + v.back().bytes == (const char *)dst)
                v.back().bytes += bytes;
            else
                v.push_back({(const char *)src, (char *)dst, bytes});
        };
        for (int d = seg_db[sg]; d < seg_db[sg + 1]; d++) {
            note(cp_ptr, in[d].indptr, L.dbs[d].indptr, pb * (size_t)(in[d].n_trans + 1));
            note(cp_idx, in[d].indices, L.dbs[d].indices, ib * (size_t)host_nnz(in[d]));
        }
        seg_copies[sg] = cp_ptr;
        seg_copies[sg].insert(seg_copies[sg].end(), cp_idx.begin(), cp_idx.end());
    }
    // ---- device buffers -------------------------------------------------------
    const int workers = ctx->num_sms * ctx->dfs_ctas_per_sm;
    // databases of short columns: one warp per prefix-extension worker (CTAs
    // of eight, dfs_warp_ctas of them per SM); a stack deeper than WARP_DEPTH levels re-mines
    // the batch with CTA workers
    constexpr int kWarpDfsMaxWords = 4096, WARP_DEPTH = 24;
    const bool warp_dfs = ctx->dfs_warp && !ctx->force_cta_dfs && L.nwp_max <= kWarpDfsMaxWords;
    // pipelined groups: each group's roots planned and mined right after its
    // finalize, on the side stream, while later groups are uploaded and built
    const bool group_dfs = ctx->batch_group_dfs && n_seg > 1 && warp_dfs && (maxlen == 0 || maxlen >= 3);
    if (group_dfs) FIM_TRY(fim_reserve(ctx, ctx->batch_windows, sizeof(RootWindow) * (size_t)n_seg));
    const int n_warps = ctx->num_sms * ctx->dfs_warp_ctas * dfs_warp_per_cta();
    const int dfs_workers = warp_dfs ? n_warps : workers;
    int depth_cap = (int)(L.max_row_bound < 240 ? L.max_row_bound : 240);
    if (warp_dfs && depth_cap > WARP_DEPTH) depth_cap = WARP_DEPTH;
    if (depth_cap < 2) depth_cap = 2;
    const size_t per_level = (size_t)dfs_workers * (size_t)(L.nwp_max > 0 ? L.nwp_max : 1) * sizeof(uint32_t);
    while (depth_cap > 2 && per_level * (size_t)depth_cap > (8ull << 30)) depth_cap /= 2;
    const int64_t frame_pool = 4LL * (L.m_max > 0 ? L.m_max : 1) + 1024;
    const size_t tbl = sizeof(DbDesc) * (size_t)n_db;
    FIM_TRY(fim_reserve(ctx, ctx->dbdesc, tbl));
    FIM_TRY(fim_reserve(ctx, ctx->batch_prefix, sizeof(int64_t) * 3 * (size_t)(n_db + 1)));
    FIM_TRY(fim_reserve(ctx, ctx->bm, sizeof(uint32_t) * (size_t)(L.words ? L.words : 1)));
    FIM_TRY(fim_reserve(ctx, ctx->item_sup, sizeof(uint32_t) * (size_t)(L.items ? L.items : 1)));
    FIM_TRY(fim_reserve(ctx, ctx->perm, sizeof(int32_t) * (size_t)(L.items ? L.items : 1)));
    FIM_TRY(fim_reserve(ctx, ctx->pair_cnt, sizeof(int) * (size_t)(L.pairs ? L.pairs : 1)));
    FIM_TRY(fim_reserve(ctx, ctx->pairbits, sizeof(uint32_t) * (size_t)(L.pb ? L.pb : 1)));
    FIM_TRY(fim_reserve(ctx, ctx->roots, sizeof(uint32_t) * 4 * (size_t)(L.root_cap ? L.root_cap : 1)));
    FIM_TRY(fim_reserve(ctx, ctx->stack_bits, per_level * (size_t)depth_cap));
    FIM_TRY(fim_reserve(ctx, ctx->frame_items, sizeof(uint32_t) * (size_t)dfs_workers * frame_pool));
    FIM_TRY(fim_reserve(ctx, ctx->frame_sups, sizeof(uint32_t) * (size_t)dfs_workers * frame_pool));
    FIM_TRY(prepare_task_queue(ctx, sizeof(Task) * kTaskCap));
    FIM_TRY(fim_reserve(ctx, ctx->cand_pool, sizeof(uint32_t) * kCandPoolCap));
    FIM_TRY(reserve_root_plan(ctx, (size_t)(L.root_cap ? L.root_cap : 1)));
    // roots without candidates are dropped before the DFS; the others ordered
    // by the network's predicted work (FIM_LEARNED with learned_order) or as
    // root_sort says
    const int plan_mode = ((flags & FIM_LEARNED) && ctx->learned_order) ? 2 : ctx->root_sort;
    if (pairs_tc)
        FIM_TRY(fim_reserve(ctx, ctx->batch_units, sizeof(unsigned long long) * (pair_units.size() ? pair_units.size() : 1)));
    // plan buffer: 32 unit counts, the database order, the plan's scratch
    const size_t plan_ord_off = 32 * sizeof(long long);
    const size_t plan_scr_off = plan_ord_off + ((sizeof(int) * (size_t)n_db + 255) & ~(size_t)255);
    if (pack) FIM_TRY(fim_reserve(ctx, ctx->batch_plan, plan_scr_off + batch_pair_plan_scratch(n_db)));
    if (rows_build)
        FIM_TRY(fim_reserve(ctx, ctx->batch_unit_db,
                            sizeof(BuildUnit) * (size_t)(L.unit_prefix[n_db] ? L.unit_prefix[n_db] : 1)));
    if (ctx->rec_cap < (1ull << 22)) {
        ctx->rec_cap = 1ull << 22;
        ctx->rec_items_cap = 1ull << 24;
    }
    // the DbDesc table and prefix arrays: pinned host staging, re-uploaded per call
    std::vector<int64_t> pre(3 * (size_t)(n_db + 1));
    memcpy(pre.data(), L.unit_prefix.data(), sizeof(int64_t) * (n_db + 1));
    memcpy(pre.data() + (n_db + 1), L.item_prefix.data(), sizeof(int64_t) * (n_db + 1));
    memcpy(pre.data() + 2 * (n_db + 1), L.tile_prefix.data(), sizeof(int64_t) * (n_db + 1));
    const int64_t *d_unit = ctx->batch_prefix.as<int64_t>();
    const int64_t *d_item = d_unit + (n_db + 1);
    const int64_t *d_tile = d_item + (n_db + 1);
    MineCounters *d_ctr = ctx->counters.as<MineCounters>();
    DbDesc *d_dbs = ctx->dbdesc.as<DbDesc>();
    cudaEventRecord(ctx->ev[0], st);
    const uint64_t launches0 = ctx->launches;

    for (int attempt = 0; attempt < 4; attempt++) {
        FIM_TRY(fim_reserve(ctx, ctx->rec_off, sizeof(unsigned long long) * ctx->rec_cap));
        FIM_TRY(fim_reserve(ctx, ctx->rec_len, sizeof(uint32_t) * ctx->rec_cap));
        FIM_TRY(fim_reserve(ctx, ctx->rec_sup, sizeof(uint32_t) * ctx->rec_cap));
        FIM_TRY(fim_reserve(ctx, ctx->rec_db, sizeof(uint32_t) * ctx->rec_cap));
        FIM_TRY(fim_reserve(ctx, ctx->rec_items, sizeof(uint32_t) * ctx->rec_items_cap));
        // per-call inputs (outside the graph): descriptor table, prefixes,
        // pair units -- copied from ctx-held host copies, and only when their
        // bytes or their destination differ from the last copy
        auto upload = [&](std::vector<unsigned char> &last, std::pair<const void *, size_t> &last_buf,
                          const DevBuf &dst, const void *src, size_t bytes) -> int {
            const std::pair<const void *, size_t> buf{dst.p, dst.bytes};
            if (last_buf == buf && last.size() == bytes && memcmp(last.data(), src, bytes) == 0) return FIM_OK;
            last.assign((const unsigned char *)src, (const unsigned char *)src + bytes);
            last_buf = buf;
            FIM_CUDA_TRY(cudaMemcpyAsync(dst.p, last.data(), bytes, cudaMemcpyHostToDevice, st));
            return FIM_OK;
        };
        FIM_TRY(upload(ctx->up_desc, ctx->up_desc_buf, ctx->dbdesc, L.dbs.data(), tbl));
        FIM_TRY(upload(ctx->up_pre, ctx->up_pre_buf, ctx->batch_prefix, pre.data(), sizeof(int64_t) * pre.size()));
        if (pairs_tc && !pair_units.empty() && !pack)
            FIM_TRY(upload(ctx->up_units, ctx->up_units_buf, ctx->batch_units, pair_units.data(),
                           sizeof(unsigned long long) * pair_units.size()));
        if (pack) {
            DevBuf ord_buf{static_cast<char *>(ctx->batch_plan.p) + plan_ord_off, ctx->batch_plan.bytes};
            FIM_TRY(upload(ctx->up_ord, ctx->up_ord_buf, ord_buf, ctx->pair_ord_cache.data(), sizeof(int) * (size_t)n_db));
        }

        DfsParams p{};
        p.dbs = d_dbs;
        p.bm = ctx->bm.as<uint32_t>();
        p.perm = ctx->perm.as<int32_t>();
        p.pairbits = ctx->pairbits.as<uint32_t>();
        p.pair_cnt = ctx->pair_cnt.as<int>();
        p.item_sup = ctx->item_sup.as<uint32_t>();
        p.nwp_max = L.nwp_max > 0 ? L.nwp_max : 1;
        const size_t rc = (size_t)(L.root_cap ? L.root_cap : 1);
        uint32_t *roots = ctx->roots.as<uint32_t>();
        p.root_a = roots;
        p.root_b = roots + rc;
        p.root_sup = roots + 2 * rc;
        p.root_db = roots + 3 * rc;
        p.root_order = ctx->root_order.as<uint32_t>();
        p.tasks = ctx->tasks.as<Task>();
        p.task_cap = kTaskCap;
        p.cand_pool = ctx->cand_pool.as<uint32_t>();
        p.cand_pool_cap = kCandPoolCap;
        p.split_depth = (flags & FIM_NO_SPLIT) ? 0 : ctx->split_depth;
        p.stack_bits = ctx->stack_bits.as<uint32_t>();
        p.frame_items = ctx->frame_items.as<uint32_t>();
        p.frame_sups = ctx->frame_sups.as<uint32_t>();
        p.frame_pool = frame_pool;
        p.depth_cap = depth_cap;
        p.rec_off = ctx->rec_off.as<unsigned long long>();
        p.rec_len = ctx->rec_len.as<uint32_t>();
        p.rec_sup = ctx->rec_sup.as<uint32_t>();
        p.rec_items = ctx->rec_items.as<uint32_t>();
        p.rec_db = ctx->rec_db.as<uint32_t>();
        p.rec_cap = ctx->rec_cap;
        p.rec_items_cap = ctx->rec_items_cap;
        p.learned = (flags & FIM_LEARNED) ? 1 : 0;
        p.diffset_rule = (flags & FIM_DIFFSET_RULE) ? 1 : 0;
        p.mlp_w = ctx->mlp_wbf.as<__nv_bfloat16>();
        p.ctr = d_ctr;
        p.spin_limit = (unsigned long long)ctx->spin_limit_ms * 1000000ull;
        p.withhold_slot = -1;
        p.sparse_div = ctx->sparse_div > 0 ? ctx->sparse_div : 0;  // automatic: dense (small databases)
        p.epoch = ctx->epoch.as<uint32_t>();
        p.learned_kmin = ctx->learned_kmin;
        p.rec_chunk = ctx->rec_chunk;
        p.root_reverse = ctx->root_reverse;

        // graph key: everything the captured launches depend on, kept whole
        // and compared in full
        std::vector<unsigned char> &key = ctx->batch_graph_blob_next;
        key.clear();
        auto mix = [&key](const void *data, size_t n) {
            const unsigned char *b = (const unsigned char *)data;
            key.insert(key.end(), b, b + n);
        };
        mix(&n_db, sizeof(n_db));
        mix(&flags, sizeof(flags));
        mix(pre.data(), sizeof(int64_t) * pre.size());
        mix(&p, sizeof(p));
        mix(&L.ib, sizeof(L.ib));
        mix(&pairs_tc, sizeof(pairs_tc));
        mix(&wbk, sizeof(wbk));
        mix(&coal, sizeof(coal));
        mix(&persist_build, sizeof(persist_build));
        mix(&group_dfs, sizeof(group_dfs));
        if (group_dfs) {
            const void *wp = ctx->batch_windows.p;
            mix(&wp, sizeof(wp));
        }
        mix(&streamed, sizeof(streamed));
        for (const auto &v : seg_copies)
            for (const HostCopy &c : v) mix(&c, sizeof(c));
        const void *udb_ptr = ctx->batch_unit_db.p;
        mix(&udb_ptr, sizeof(udb_ptr));
        // every launch-shape knob the captured launches depend on
        const int shape[9] = {workers, ctx->dfs_block, ctx->pairs_kdrain, ctx->pairs_split, ctx->batch_pairs_shape,
                              ctx->dfs_ctas_per_sm, plan_mode, ctx->learned_order, n_seg};
        mix(&warp_dfs, sizeof(warp_dfs));
        mix(&ctx->dfs_warp_ctas, sizeof(ctx->dfs_warp_ctas));
        mix(shape, sizeof(shape));
        mix(&pack, sizeof(pack));
        if (pack) {
            const void *pp = ctx->batch_plan.p;
            mix(&pp, sizeof(pp));
        }
        if (pairs_tc) {
            const void *up = ctx->batch_units.p;
            mix(&up, sizeof(up));
            mix(pair_units.data(), sizeof(unsigned long long) * pair_units.size());
            const int64_t nu = (int64_t)pair_units.size();
            mix(&nu, sizeof(nu));
        }
        const size_t smem_build = (size_t)L.ib * WB * sizeof(uint32_t);
        FIM_CUDA_TRY(cudaFuncSetAttribute(batch_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem_build));
        const size_t smem_rows = (size_t)(L.m_max | 1) * wbk * sizeof(uint32_t);
        if (rows_build) {
            FIM_CUDA_TRY(cudaFuncSetAttribute(build_rows_fn(wbk, coal, persist_build),
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows));
        }
        const bool reuse = ctx->batch_graph_exec && ctx->batch_graph_blob == key;
        if (!reuse) {
            if (ctx->batch_graph_exec) {
                cudaGraphExecDestroy((cudaGraphExec_t)ctx->batch_graph_exec);
                ctx->batch_graph_exec = nullptr;
            }
            cudaGraph_t g = nullptr;
            if (n_seg > 1) {  // the side stream and the group events, made outside the capture
                FIM_TRY(fim_aux_stream(ctx));
                for (int sg = 0; sg <= n_seg; sg++)
                    if (!ctx->seg_ev[sg]) FIM_CUDA_TRY(cudaEventCreateWithFlags(&ctx->seg_ev[sg], cudaEventDisableTiming));
            }
            if (streamed) {  // the upload stream and its events
                if (!ctx->copy_stream) FIM_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
                for (int sg = 0; sg <= n_seg; sg++)
                    if (!ctx->copy_ev[sg])
                        FIM_CUDA_TRY(cudaEventCreateWithFlags(&ctx->copy_ev[sg], cudaEventDisableTiming));
            }
            FIM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            // phase boundaries as event-record nodes of the graph: graph start
            // (ev 7), after build + supports + rank (ev 1), after the pair
            // pass (ev 2); the DFS ends where the graph does (ev 3)
            cudaEventRecordWithFlags(ctx->ev[7], st, cudaEventRecordExternal);
            cudaMemsetAsync(d_ctr, 0, sizeof(MineCounters), st);
            cudaMemsetAsync(ctx->dev_flag.p, 0, sizeof(int), st);
            launch_epoch_bump(ctx);
            if (streamed) {
                // group sg's CSRs go up on the upload stream; its build waits
                // for copy_ev[sg] only, so later uploads overlap its work
                cudaEventRecord(ctx->copy_ev[n_seg], st);
                cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_ev[n_seg], 0);
                for (int sg = 0; sg < n_seg; sg++) {
                    for (const HostCopy &c : seg_copies[sg])
                        cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, ctx->copy_stream);
                    cudaEventRecord(ctx->copy_ev[sg], ctx->copy_stream);
                }
            }
            const int64_t units = L.unit_prefix[n_db], items = L.item_prefix[n_db], tiles = L.tile_prefix[n_db];
            // rows-per-thread build with fused supports when every database's
            // block of columns fits shared memory (ib == m_max <= 1,024)
            if (rows_build && items > 0)
                cudaMemsetAsync(ctx->item_sup.p, 0, sizeof(uint32_t) * (size_t)items, st);
            if (rows_build && units > 0)
                batch_unit_db_kernel<<<(unsigned)n_db, 256, 0, st>>>(d_dbs, d_unit, wbk, ctx->bm.as<uint32_t>(),
                                                                     ctx->batch_unit_db.as<BuildUnit>());
            auto build_rows = [&](int64_t u0, int64_t u1, cudaStream_t s_) {
                if (u1 <= u0) return;
                const unsigned grid = (unsigned)(u1 - u0);
                const BuildUnit *const bu = ctx->batch_unit_db.as<BuildUnit>();
                uint32_t *const sup = ctx->item_sup.as<uint32_t>();
                int *const flg = ctx->dev_flag.as<int>();
                const unsigned g = persist_build ? (unsigned)(u1 - u0 < ctx->num_sms ? u1 - u0 : ctx->num_sms) : grid;
                build_rows_fn(wbk, coal, persist_build)<<<g, BUILD_ROWS_THREADS, smem_rows, s_>>>(bu, u0, u1, sup,
                                                                                                 flg);
            };
            auto rank_db = [&](int da, int db_, cudaStream_t s_) {
                if (db_ > da)
                    batch_rank_db_kernel<<<(unsigned)(db_ - da), RANK_THREADS, 0, s_>>>(
                        d_dbs, da, ctx->item_sup.as<uint32_t>(), ctx->perm.as<int32_t>(), d_ctr, p.rec_off,
                        p.rec_len, p.rec_sup, p.rec_items, p.rec_db, p.rec_cap, p.rec_items_cap);
            };
            auto finalize_db = [&](int da, int db_, cudaStream_t s_) {
                if (db_ > da)
                    batch_finalize_db_kernel<<<(unsigned)(db_ - da), FIN_THREADS, 0, s_>>>(
                        d_dbs, da, ctx->pair_cnt.as<int>(), ctx->pairbits.as<uint32_t>(), d_ctr, p.rec_off,
                        p.rec_len, p.rec_sup, p.rec_items, p.rec_db, p.rec_cap, p.rec_items_cap, roots, roots + rc,
                        roots + 2 * rc, roots + 3 * rc);
            };
            int rc_pairs = FIM_OK;
            // group sg's tensor-core pair pass (planned on the device first
            // when packing; the host's units give the capacity)
            auto pair_pass = [&](int sg, cudaStream_t s_) -> int {
                unsigned long long *const u = ctx->batch_units.as<unsigned long long>() + seg_unit[sg];
                const int64_t cap = seg_unit[sg + 1] - seg_unit[sg];
                if (!pack) return launch_batch_pairs_tc(ctx, d_dbs, u, cap, nullptr, s_);
                char *const plan = static_cast<char *>(ctx->batch_plan.p);
                long long *const cnt = reinterpret_cast<long long *>(plan) + sg;
                const int *const ord = reinterpret_cast<const int *>(plan + plan_ord_off) + seg_db[sg];
                const int rc = launch_batch_pair_plan(ctx, d_dbs, ord, seg_db[sg + 1] - seg_db[sg], u, cnt,
                                                      plan + plan_scr_off, s_);
                return rc != FIM_OK ? rc : launch_batch_pairs_tc(ctx, d_dbs, u, cap, cnt, s_);
            };
            if (n_seg > 1) {
                // group s: build + rank on the ctx stream, then its pair pass
                // and finalize on the side stream, overlapping group s + 1's
                // build; the ctx stream joins the side stream before the DFS
                cudaStream_t aux = ctx->aux_stream;
                for (int sg = 0; sg < n_seg; sg++) {
                    const int da = seg_db[sg], db_ = seg_db[sg + 1];
                    if (streamed) cudaStreamWaitEvent(st, ctx->copy_ev[sg], 0);
                    build_rows(L.unit_prefix[da], L.unit_prefix[db_], st);
                    rank_db(da, db_, st);
                    cudaEventRecord(ctx->seg_ev[sg], st);
                    cudaStreamWaitEvent(aux, ctx->seg_ev[sg], 0);
                    if (rc_pairs == FIM_OK) rc_pairs = pair_pass(sg, aux);
                    RootWindow *const win = group_dfs ? ctx->batch_windows.as<RootWindow>() + sg : nullptr;
                    if (win) window_begin_kernel<<<1, 1, 0, aux>>>(d_ctr, win);
                    finalize_db(da, db_, aux);
                    if (win) {  // the group's own root plan and prefix extension, on the side stream
                        window_end_kernel<<<1, 1, 0, aux>>>(d_ctr, win);
                        if (rc_pairs == FIM_OK)
                            rc_pairs = launch_root_plan(ctx, d_ctr, rc, d_dbs, plan_mode, win, aux);
                        if (rc_pairs == FIM_OK) {
                            DfsParams pw = p;
                            pw.win = win;
                            rc_pairs = launch_dfs_warp(ctx, pw, n_warps, ctx->dfs_warp_ctas, aux);
                        }
                    }
                }
                cudaEventRecordWithFlags(ctx->ev[1], st, cudaEventRecordExternal);
                cudaEventRecord(ctx->seg_ev[n_seg], aux);
                cudaStreamWaitEvent(st, ctx->seg_ev[n_seg], 0);
            } else {
                if (streamed) cudaStreamWaitEvent(st, ctx->copy_ev[0], 0);
                if (units > 0) {
                    if (rows_build)
                        build_rows(0, units, st);
                    else
                        batch_build_kernel<<<(unsigned)units, 256, smem_build, st>>>(
                            d_dbs, n_db, d_unit, L.ib, ctx->bm.as<uint32_t>(), ctx->dev_flag.as<int>());
                }
                if (items > 0) {
                    if (!rows_build)
                        batch_support_kernel<<<(unsigned)items, 256, 0, st>>>(d_dbs, n_db, d_item,
                                                                              ctx->bm.as<uint32_t>(),
                                                                              ctx->item_sup.as<uint32_t>());
                    if (L.m_max <= RANK_CAP)
                        rank_db(0, n_db, st);
                    else
                        batch_rank_kernel<<<(unsigned)ceil_div64(items * 32, 256), 256, 0, st>>>(
                            d_dbs, n_db, d_item, items, ctx->item_sup.as<uint32_t>(), ctx->perm.as<int32_t>(), d_ctr,
                            p.rec_off, p.rec_len, p.rec_sup, p.rec_items, p.rec_db, p.rec_cap, p.rec_items_cap);
                }
                cudaEventRecordWithFlags(ctx->ev[1], st, cudaEventRecordExternal);
                if (tiles > 0 && maxlen != 1) {
                    if (pairs_tc)
                        rc_pairs = pair_pass(0, st);
                    else
                        batch_pairs_kernel<<<(unsigned)tiles, 256, 0, st>>>(d_dbs, n_db, d_tile,
                                                                            ctx->bm.as<uint32_t>(),
                                                                            ctx->perm.as<int32_t>(),
                                                                            ctx->pair_cnt.as<int>());
                    if (L.m_max <= FIN_CAP)
                        finalize_db(0, n_db, st);
                    else
                        batch_finalize_kernel<<<(unsigned)ceil_div64(items * 32, 256), 256, 0, st>>>(
                            d_dbs, n_db, d_item, items, ctx->pair_cnt.as<int>(), ctx->pairbits.as<uint32_t>(),
                            d_ctr, p.rec_off, p.rec_len, p.rec_sup, p.rec_items, p.rec_db, p.rec_cap,
                            p.rec_items_cap, roots, roots + rc, roots + 2 * rc, roots + 3 * rc);
                }
            }
            if (rc_pairs != FIM_OK) {
                cudaGraph_t junk = nullptr;
                cudaStreamEndCapture(st, &junk);
                if (junk) cudaGraphDestroy(junk);
                return rc_pairs;
            }
            cudaEventRecordWithFlags(ctx->ev[2], st, cudaEventRecordExternal);
            int rc_launch = FIM_OK;
            if (!group_dfs && (maxlen == 0 || maxlen >= 3)) {
                rc_launch = launch_root_plan(ctx, d_ctr, rc, d_dbs, plan_mode, nullptr, st);
                if (rc_launch == FIM_OK)
                    rc_launch = warp_dfs ? launch_dfs_warp(ctx, p, n_warps, ctx->dfs_warp_ctas, st)
                                         : launch_dfs(ctx, p, workers, ctx->dfs_block);
            }
            const cudaError_t ce = cudaStreamEndCapture(st, &g);
            if (rc_launch != FIM_OK) { if (g) cudaGraphDestroy(g); return rc_launch; }
            if (ce != cudaSuccess) { fim_set_cuda_error(ce, "capture", __FILE__, __LINE__); return FIM_E_CUDA; }
            cudaGraphExec_t ex = nullptr;
            // node priorities as captured: the side stream's pair passes go first
            const cudaError_t ie = cudaGraphInstantiate(&ex, g, cudaGraphInstantiateFlagUseNodePriority);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) { fim_set_cuda_error(ie, "instantiate", __FILE__, __LINE__); return FIM_E_CUDA; }
            ctx->batch_graph_exec = ex;
            ctx->batch_graph_blob.swap(key);
            ctx->batch_graph_launches = 10;  // unit map, build, rank, pairs, finalize, 3 root plan, DFS, epoch
        }
        FIM_CUDA_TRY(cudaGraphLaunch((cudaGraphExec_t)ctx->batch_graph_exec, st));
        ctx->launches += ctx->batch_graph_launches;
        cudaEventRecord(ctx->ev[3], st);
        int bad = 0;
        FIM_CUDA_TRY(cudaMemcpyAsync(&ctx->host_ctr, d_ctr, sizeof(MineCounters), cudaMemcpyDeviceToHost, st));
        FIM_CUDA_TRY(cudaMemcpyAsync(&bad, ctx->dev_flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        FIM_CUDA_TRY(cudaStreamSynchronize(st));
        if (bad) return FIM_E_INVAL;
        const MineCounters &c = ctx->host_ctr;
        if (c.err == FIM_E_STACK && warp_dfs) {
            // deeper than the warp workers' stack: the batch again with CTA workers
            ctx->force_cta_dfs = true;
            const int rc2 = fim_mine_batched(ctx, n_db, in, flags);
            ctx->force_cta_dfs = false;
            return rc2;
        }
        if (c.err != 0) return c.err;
        if (c.overflow) {
            ctx->rec_cap = c.n_records + c.n_records / 4 + 1024;
            ctx->rec_items_cap = c.n_rec_items + c.n_rec_items / 4 + 4096;
            continue;  // buffers grow; the new pointers give a new graph key
        }
        // ---- canonical order by (database, size, items) ----------------------
        FIM_TRY(launch_compact(ctx, c.n_records, c.n_records - c.rec_holes, n_db, L.m_max > 0 ? L.m_max : 1));
        FIM_TRY(fim_reserve(ctx, ctx->batch_slices, sizeof(unsigned long long) * 2 * (size_t)(n_db + 1)));
        unsigned long long *cnt = ctx->batch_slices.as<unsigned long long>();
        unsigned long long *istart = cnt + (n_db + 1);
        FIM_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (n_db + 1), st));
        if (c.n_records > 0) {
            ctx->launches += 2;
            db_count_kernel<<<(unsigned)ceil_div64((int64_t)c.n_records, 256), 256, 0, st>>>(
                ctx->rec_db.as<uint32_t>(), c.n_records, cnt);
            db_scan_kernel<<<1, 1024, 0, st>>>(cnt, n_db, ctx->out_off.as<unsigned long long>(), istart);
            FIM_CUDA_TRY(cudaGetLastError());
        } else {
            FIM_CUDA_TRY(cudaMemsetAsync(istart, 0, sizeof(unsigned long long) * (n_db + 1), st));
        }
        ctx->batch_set_start.resize(n_db + 1);
        ctx->batch_item_start.resize(n_db + 1);
        FIM_CUDA_TRY(cudaMemcpyAsync(ctx->batch_set_start.data(), cnt, sizeof(unsigned long long) * (n_db + 1),
                                     cudaMemcpyDeviceToHost, st));
        FIM_CUDA_TRY(cudaMemcpyAsync(ctx->batch_item_start.data(), istart,
                                     sizeof(unsigned long long) * (n_db + 1), cudaMemcpyDeviceToHost, st));
        cudaEventRecord(ctx->ev[4], st);
        FIM_CUDA_TRY(cudaStreamSynchronize(st));
        ctx->batch_n_db = n_db;
        ctx->batch_mined = true;
        fim_stats &s = ctx->stats;
        s.n_trans = 0;
        for (int d = 0; d < n_db; d++) s.n_trans += (uint64_t)in[d].n_trans;
        s.n_items = (uint64_t)L.items;
        s.n_sets = c.n_records - c.rec_holes;
        s.max_len = (uint64_t)c.max_len;
        s.supports_singletons = (uint64_t)L.items;
        s.supports_pairs = 0;  // sum over databases of m'(m'-1)/2: filled below
        s.supports_dfs = c.supports_dfs;
        s.dfs_words = c.dfs_words;
        s.dfs_bytes = c.dfs_bytes;
        s.dfs_touched_bytes = c.dfs_touched;
        s.classes = c.classes;
        s.tasks_pushed = c.pushed;
        s.diffset_classes = c.diffset;
        s.dfs_busy_ns = c.busy_ns;
        s.dfs_root_ns = c.root_ns;
        s.dfs_span_ns = c.t_last > c.t_first && c.t_first != 0 ? c.t_last - c.t_first : 0;
        s.dfs_workers = (uint64_t)dfs_workers;
        s.launches_build = 0;
        s.launches_mine = ctx->launches - launches0;
        s.pair_path = pairs_tc ? 1u : 0u;
        // phases of the graph: build + singleton supports + rank, pairs +
        // finalize, DFS; then the compaction outside the graph
        s.ms_build = s.ms_singletons = s.ms_pairs = s.ms_dfs = 0.f;
        if (cudaEventElapsedTime(&s.ms_build, ctx->ev[7], ctx->ev[1]) != cudaSuccess ||
            cudaEventElapsedTime(&s.ms_pairs, ctx->ev[1], ctx->ev[2]) != cudaSuccess ||
            cudaEventElapsedTime(&s.ms_dfs, ctx->ev[2], ctx->ev[3]) != cudaSuccess) {
            (void)cudaGetLastError();  // phase split unavailable: whole graph as the DFS
            s.ms_build = s.ms_pairs = 0.f;
            cudaEventElapsedTime(&s.ms_dfs, ctx->ev[0], ctx->ev[3]);
        }
        cudaEventElapsedTime(&s.ms_compact, ctx->ev[3], ctx->ev[4]);
        // m' per database (written by the device) for the pair-support count
        std::vector<DbDesc> back(n_db);
        FIM_CUDA_TRY(cudaMemcpy(back.data(), d_dbs, tbl, cudaMemcpyDeviceToHost));
        uint64_t mfsum = 0;
        for (int d = 0; d < n_db; d++) {
            const uint64_t mf = (uint64_t)back[d].mfreq;
            if (maxlen == 0 || maxlen >= 2) s.supports_pairs += mf * (mf > 0 ? mf - 1 : 0) / 2;
            mfsum += mf;
        }
        s.n_frequent_items = mfsum;
        if (ctx->bytes_held > s.peak_device_bytes) s.peak_device_bytes = ctx->bytes_held;
        return FIM_OK;
    }
    return FIM_E_NOMEM;
}

int fim_fetch_batched(fim_ctx *ctx, int db, uint64_t *n_sets, uint64_t *n_items_total, uint64_t *offsets,
                      uint32_t *items, uint32_t *supports, uint64_t cap_sets, uint64_t cap_items, uint32_t flags) {
    FIM_NVTX("fim_fetch_batched");
    if (!ctx || !n_sets || !n_items_total) return FIM_E_INVAL;
    if (!ctx->batch_mined) return FIM_E_STATE;
    if (db != FIM_ALL_DBS && (db < 0 || db >= ctx->batch_n_db)) return FIM_E_INVAL;
    const int nd = ctx->batch_n_db;
    const unsigned long long s0 = db == FIM_ALL_DBS ? 0ull : ctx->batch_set_start[db];
    const unsigned long long s1 = db == FIM_ALL_DBS ? ctx->batch_set_start[nd] : ctx->batch_set_start[db + 1];
    const unsigned long long i0 = db == FIM_ALL_DBS ? 0ull : ctx->batch_item_start[db];
    const unsigned long long i1 = db == FIM_ALL_DBS ? ctx->batch_item_start[nd] : ctx->batch_item_start[db + 1];
    *n_sets = s1 - s0;
    *n_items_total = i1 - i0;
    if (!offsets && !items && !supports) return FIM_OK;
    if (!offsets || !supports || (!items && i1 > i0)) return FIM_E_INVAL;
    if (cap_sets < s1 - s0 || cap_items < i1 - i0) return FIM_E_TOO_SMALL;
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FIM_E_CUDA;
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{dev_prev};
    cudaStream_t st = ctx->stream;
    const bool dev = flags & FIM_OUTPUT_DEVICE;
    const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    FIM_CUDA_TRY(cudaMemcpyAsync(offsets, ctx->out_off.as<unsigned long long>() + s0,
                                 sizeof(uint64_t) * (s1 - s0 + 1), k, st));
    if (i1 > i0)
        FIM_CUDA_TRY(cudaMemcpyAsync(items, ctx->out_items.as<uint32_t>() + i0, sizeof(uint32_t) * (i1 - i0), k, st));
    if (s1 > s0)
        FIM_CUDA_TRY(cudaMemcpyAsync(supports, ctx->out_sup.as<uint32_t>() + s0, sizeof(uint32_t) * (s1 - s0), k, st));
    if (dev) {
        ctx->launches++;
        rebase_kernel<<<(unsigned)ceil_div64((int64_t)(s1 - s0 + 1), 256), 256, 0, st>>>(
            (unsigned long long *)offsets, s1 - s0, i0);
        FIM_CUDA_TRY(cudaGetLastError());
    }
    FIM_CUDA_TRY(cudaStreamSynchronize(st));
    if (!dev)
        for (uint64_t q = 0; q <= s1 - s0; q++) offsets[q] -= i0;
    return FIM_OK;
}

int fim_batch_slices(fim_ctx *ctx, uint64_t *set_start, uint64_t cap) {
    FIM_NVTX("fim_batch_slices");
    if (!ctx || !set_start) return FIM_E_INVAL;
    if (!ctx->batch_mined) return FIM_E_STATE;
    if (cap < (uint64_t)ctx->batch_n_db + 1) return FIM_E_TOO_SMALL;
    for (int d = 0; d <= ctx->batch_n_db; d++) set_start[d] = ctx->batch_set_start[d];
    return FIM_OK;
}

}  // extern "C"
