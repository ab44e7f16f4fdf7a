// k_dfs.cu -- recursive prefix extension (Section III: the column AND "can
// be performed in sequence" for higher-order itemsets; the threshold test of
// Eq. 3 prunes every infrequent extension).
//
// Persistent kernel: each CTA is one depth-first worker.  Work arrives as
// tickets from one global counter.  Tickets below n_roots are the frequent
// pairs {a, b} (root prefix classes, of any database of the mine); later
// tickets are slots of a device queue that workers fill with prefix classes
// they split off while other workers wait.  Every wait is bounded
// (FIM_E_TIMEOUT, never a hang).
//
// A prefix class Y = X u {c} has its support S(Y), its parent X with S(X),
// and candidates e_1 < ... < e_k (later frequent siblings of c in X's class
// whose pair {c, e} is frequent), each with the known S(X u {e}).  One pass
// over the class streams, word by word,
//     b_Y = b_X AND col(c)                      (written to the worker's stack
//                                                when Y can have grandchildren)
//   dense:    S(Y u {e}) = popc(b_Y AND col(e))
//   diffset:  S(Y u {e}) = S(X u {e}) - popc(d_Y AND col(e)),  d_Y = b_X AND NOT col(c)
// The streamed operand (b_Y or d_Y) stays in registers; a lane skips the
// 16-byte load of col(e) where its operand words are all zero, so HBM serves
// only the 32-byte sectors that can contribute.  Per-warp popc sums are
// reduced with shuffles and combined in shared memory.  Frequent extensions
// become result records and the child list F.  The representation of each
// class (dense or diffset) is chosen by a closed-form size rule, by the
// scheduling MLP, or fixed to dense (the plain miner); it never changes a
// count.
#include "fim_common.cuh"

namespace {

constexpr int CB = 1024;                 // candidates per pass batch
constexpr int MAXSRC = FIM_TASK_MAXR + 1;
constexpr int MAXPATH = 256;             // longest itemset a worker tracks
constexpr int V = 2;                     // uint4 per lane per chunk (chunk = 256 words)
constexpr int CHUNK = 128 * V;
constexpr int NF = FIM_MLP_FEATURES;
constexpr int PCAP = 1024;               // perm entries a worker keeps in shared memory
constexpr unsigned ICH = 1024;           // item slots a worker reserves at a time

// The database of the task a worker is on.
struct DbView {
    const uint32_t *bm;
    const int32_t *perm;
    const uint32_t *pairbits;
    const int *pair_cnt;
    const uint32_t *item_sup;
    int64_t nwp, nw, n;
    int32_t mfreq, mpw;
    uint32_t thr, maxlen, id;
};

struct Smem {
    DbView db;
    int32_t perm_c[PCAP];                // the task database's perm[0 .. min(m', PCAP))
    const uint32_t *src[MAXSRC];
    const uint32_t *cptr[CB];
    uint32_t sup[CB];
    uint32_t path[MAXPATH];
    int nF[MAXPATH];
    int cur[MAXPATH];
    long long base[MAXPATH + 1];
    uint32_t supY[MAXPATH];              // support of the class at each level
    unsigned long long work[MAXPATH];    // candidate words ANDed in the subtree so far
    float feat[MAXPATH][NF];             // trace features of the class at each level
    float label[MAXPATH];                // measured representation label
    float mlp_w[FIM_MLP_PARAMS];         // scheduling MLP (bf16 values held as float)
    float y[2];                          // scheduling MLP output
    uint32_t scan[33];                   // block scan scratch (<= 32 warps)
    unsigned int sec_dense, sec_diff;    // nonzero 32-byte sectors (sparse parent: words) of b_Y and d_Y
    int nsrc;
    int diff;                            // 1: count through the diffset
    uint32_t *store;
    int store_sparse;                    // 1: store b_Y as its non-zero words (index, word)
    unsigned int zcount;                 // entries written by a sparse store
    int psparse;                         // 1: the parent b_X is stored sparse ...
    int pz;                              // ... as pz entries
    const uint32_t *pidx, *pval;         // ... word indices and words
    int lz[MAXPATH];                     // entries of each level's stored bitmap; -1 = dense
    unsigned long long n_roots;          // root count (fixed once the DFS runs)
    unsigned long long busy, root_busy, t_task;  // thread 0's worker timing
    // the worker's class statistics, summed by thread 0 and added to the
    // global counters once, at exit (per-class atomics on those shared words
    // delay every worker's ticket and record atomics on the same lines)
    unsigned long long n_sup, n_words, n_bytes, n_touched, n_classes, n_diff;
    int max_len;
    int err_seen;                        // last error flag read
    uint32_t epoch;                      // this mine's task epoch
    unsigned int iter;                   // classes since the worker started
    unsigned long long ticket;
    unsigned long long rbase, ibase;
    unsigned long long rec_next, rec_end;   // this worker's reserved record slots
    unsigned long long it_next, it_end;     // and item slots (thread 0 alone)
    int flag;
    int hungry;
    int kc;                              // candidates of the child being set up (-1: overflow)
    int ftot;                            // frequent candidates of a small batch
    int stop;
    int task_len;
    uint32_t task_sup;
    uint32_t task_db;
    int ncand;
    long long cand_off;
};

// Block-wide exclusive scan of v.  Returns the prefix; *total gets the sum.
template <int NT>
__device__ __forceinline__ uint32_t block_scan(Smem &s, uint32_t v, uint32_t *total) {
    constexpr int NWARP = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) s.scan[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int w = 0; w < NWARP; w++) {
            uint32_t t = s.scan[w];
            s.scan[w] = acc;
            acc += t;
        }
        s.scan[NWARP] = acc;
    }
    __syncthreads();
    *total = s.scan[NWARP];
    return s.scan[warp] + x - v;
}

__device__ __forceinline__ bool pairbit(const DbView &d, uint32_t a, uint32_t b) {
    return (__ldg(d.pairbits + (int64_t)a * d.mpw + (b >> 5)) >> (b & 31)) & 1u;
}

// Bit column of internal item `item` (< m') of the task's database: its
// perm entry from shared memory when cached, else from global memory.
__device__ __forceinline__ const uint32_t *column(const Smem &s, uint32_t item) {
    const int32_t j = item < (uint32_t)PCAP ? s.perm_c[item] : __ldg(s.db.perm + item);
    return s.db.bm + (int64_t)j * s.db.nwp;
}

__device__ void set_err(const DfsParams &p, int code) { atomicCAS(&p.ctr->err, 0, code); }

__device__ __forceinline__ bool nz4(uint4 a) { return (a.x | a.y | a.z | a.w) != 0u; }

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Nonzero 32-byte sectors among the warp's 16-byte lanes (lanes 2i, 2i+1
// share a sector).
__device__ __forceinline__ uint32_t warp_sectors(bool nz) {
    const uint32_t b = __ballot_sync(0xffffffffu, nz);
    return __popc((b | (b >> 1)) & 0x55555555u);
}

// Sparse store of b_Y: a level of the worker's stack holds word indices in
// its first half and the words in its second half.  Entries of one class
// are appended in any order (supports are order-free sums).
__device__ __forceinline__ void sparse_put4(const DfsParams &p, Smem &s, uint32_t *lv, int64_t half, uint4 y,
                                            int64_t pos, int lane) {
    const uint32_t w[4] = {y.x, y.y, y.z, y.w};
    const uint32_t c = (w[0] != 0u) + (w[1] != 0u) + (w[2] != 0u) + (w[3] != 0u);
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    uint32_t base = 0;
    if (lane == 31 && x) base = atomicAdd(&s.zcount, x);
    base = __shfl_sync(0xffffffffu, base, 31);
    uint32_t at = base + x - c;
#pragma unroll
    for (int q = 0; q < 4; q++)
        if (w[q]) {
            if (at < half) {
                lv[at] = (uint32_t)(pos + q);
                lv[half + at] = w[q];
            } else {
                set_err(p, FIM_E_STACK);
            }
            at++;
        }
}

template <int U>
__device__ __forceinline__ void sparse_put(const DfsParams &p, Smem &s, uint32_t *lv, int64_t half,
                                           const uint32_t *ix, const uint32_t *y, int lane) {
    uint32_t bal[U], cnt = 0;
#pragma unroll
    for (int u = 0; u < U; u++) {
        bal[u] = __ballot_sync(0xffffffffu, y[u] != 0u);
        cnt += __popc(bal[u]);
    }
    uint32_t base = 0;
    if (lane == 0 && cnt) base = atomicAdd(&s.zcount, cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int u = 0; u < U; u++) {
        if (y[u]) {
            const uint32_t at = base + __popc(bal[u] & lt);
            if (at < half) {
                lv[at] = ix[u];
                lv[half + at] = y[u];
            } else {
                set_err(p, FIM_E_STACK);
            }
        }
        base += __popc(bal[u]);
    }
}

// b_Y of support supY is stored sparse when its non-zero words (at most
// supY of them) are few: supY * sparse_div <= nw, and they fit half a level.
__device__ __forceinline__ int sparse_ok(const DfsParams &p, const DbView &db, uint32_t supY) {
    return p.sparse_div > 0 && (unsigned long long)supY * (unsigned)p.sparse_div <= (unsigned long long)db.nw &&
           (int64_t)supY <= p.nwp_max / 2;
}

// Thread 0: the view of database `db` from the mine-wide arrays.
__device__ void load_db(const DfsParams &p, Smem &s, uint32_t db) {
    const DbDesc &d = p.dbs[db];
    s.db.bm = p.bm + d.bm_off;
    s.db.perm = p.perm + d.item_off;
    s.db.item_sup = p.item_sup + d.item_off;
    s.db.pair_cnt = p.pair_cnt + d.pair_off;
    s.db.pairbits = p.pairbits + d.pb_off;
    s.db.nwp = d.nwp;
    s.db.nw = d.nw;
    s.db.n = d.n;
    s.db.mfreq = *(volatile const int32_t *)&d.mfreq;
    s.db.mpw = (s.db.mfreq + 31) / 32;
    s.db.thr = d.thr;
    s.db.maxlen = d.maxlen;
    s.db.id = db;
}

// One pass over a class: candidates cand[0..k) with parent supports
// psup[0..k) (both in the worker's frame pool), sources s.src[0..nsrc),
// optional store of b_Y, s.diff selects the diffset count (nsrc == 2).
// Frequent candidates are written compacted (item, support) to fi/fs and
// emitted as records with prefix s.path[0..plen).  Returns |F| (uniform).
// Dense pass over one candidate batch: the sources are whole bit columns or
// a dense b_X.  Warps = G candidate groups x (NWARP / G) chunk workers.
template <int NT>
__device__ __forceinline__ void dense_sweep(const DfsParams &p, Smem &s, int kb, bool first) {
    constexpr int NWARP = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nwp = s.db.nwp;
    const int nchunks = (int)((nwp + CHUNK - 1) / CHUNK);
    const int G = nchunks >= NWARP ? 1 : NWARP / nchunks;
    const int CW = NWARP / G;
    const int g = warp % G, cw = warp / G;
    const bool active = warp < G * CW;
    const int nsrc = s.nsrc;
    const bool diff = s.diff != 0;
    const bool two = nsrc == 2;
    uint32_t *store = first && g == 0 ? s.store : nullptr;
    const bool store_sparse = s.store_sparse != 0;
    const int64_t half = p.nwp_max / 2;
    const int b0 = first ? 0 : 1;
    if (active) {
            for (int q = cw; q < nchunks; q += CW) {
                const int64_t base = (int64_t)q * CHUNK + lane * 4;
                uint4 x[V];
                bool ok[V];
                uint32_t secd = 0, secf = 0;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const int64_t pos = base + v * 128;
                    ok[v] = pos < nwp;  // uniform across the warp (nwp % 128 == 0)
                    uint4 y = make_uint4(0, 0, 0, 0), f = y;
                    if (ok[v]) {
                        const uint4 s0 = ld_cg_u4(s.src[0] + pos);
                        y = s0;
                        if (two) {
                            const uint4 s1 = ld_cg_u4(s.src[1] + pos);
                            y = and4(s0, s1);
                            f = make_uint4(s0.x & ~s1.x, s0.y & ~s1.y, s0.z & ~s1.z, s0.w & ~s1.w);
                        }
                        // a popped task ANDs all of its prefix columns
                        for (int r = two ? 2 : 1; r < nsrc; r++) y = and4(y, ld_cg_u4(s.src[r] + pos));
                        if (store && b0 == 0 && g == 0) {
                            if (store_sparse) sparse_put4(p, s, store, half, y, pos, lane);
                            else *reinterpret_cast<uint4 *>(store + pos) = y;
                        }
                    }
                    x[v] = diff ? f : y;
                    if (ok[v] && b0 == 0 && g == 0) {
                        secd += warp_sectors(nz4(y));
                        secf += warp_sectors(nz4(f));
                    }
                }
                if (lane == 0 && (secd | secf)) {
                    atomicAdd(&s.sec_dense, secd);
                    atomicAdd(&s.sec_diff, secf);
                }
                bool any[V];
#pragma unroll
                for (int v = 0; v < V; v++) any[v] = ok[v] && nz4(x[v]);
                int c = g;
                for (; c + G < kb; c += 2 * G) {
                    const uint32_t *c0 = s.cptr[c], *c1 = s.cptr[c + G];
                    uint4 y0[V], y1[V];
#pragma unroll
                    for (int v = 0; v < V; v++) {
                        const int64_t pos = base + v * 128;
                        y0[v] = any[v] ? ldg_u4(c0 + pos) : make_uint4(0, 0, 0, 0);
                        y1[v] = any[v] ? ldg_u4(c1 + pos) : make_uint4(0, 0, 0, 0);
                    }
                    uint32_t n0 = 0, n1 = 0;
#pragma unroll
                    for (int v = 0; v < V; v++) { n0 += popc_and4(x[v], y0[v]); n1 += popc_and4(x[v], y1[v]); }
                    n0 = warp_sum_u32(n0);
                    n1 = warp_sum_u32(n1);
                    if (lane == 0) {
                        if (n0) atomicAdd(&s.sup[c], n0);
                        if (n1) atomicAdd(&s.sup[c + G], n1);
                    }
                }
                for (; c < kb; c += G) {
                    const uint32_t *c0 = s.cptr[c];
                    uint32_t n0 = 0;
#pragma unroll
                    for (int v = 0; v < V; v++) {
                        const int64_t pos = base + v * 128;
                        if (any[v]) n0 += popc_and4(x[v], ldg_u4(c0 + pos));
                    }
                    n0 = warp_sum_u32(n0);
                    if (lane == 0 && n0) atomicAdd(&s.sup[c], n0);
                }
            }
        }
}

// Pass over one candidate batch when b_X is stored as its pz non-zero words
// (index, word): b_Y and d_Y exist only there, so the pass gathers col(c) and
// col(e) at those word indices alone.  Warps = SG candidate groups x SCW
// entry workers; each lane takes U entries per step.
template <int NT>
__device__ __forceinline__ void sparse_sweep(const DfsParams &p, Smem &s, int kb, bool first) {
    constexpr int NWARP = NT / 32;
    constexpr int U = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pz = s.pz;
    const uint32_t *pidx = s.pidx, *pval = s.pval, *ext = s.src[1];
    const int wsteps = (pz + 32 * U - 1) / (32 * U);
    const int SG = wsteps >= NWARP ? 1 : NWARP / (wsteps > 0 ? wsteps : 1);
    const int SCW = NWARP / SG;
    const int sg = warp % SG, scw = warp / SG;
    const bool sactive = warp < SG * SCW;
    const bool diff = s.diff != 0;
    uint32_t *store = s.store;
    const int64_t half = p.nwp_max / 2;
    const int b0 = first ? 0 : 1;
    if (sactive) {
            // b_X is its pz non-zero words: b_Y and d_Y exist only there, so
            // the pass gathers col(c) and col(e) at those word indices alone
            for (int e0 = scw * 32 * U; e0 < pz; e0 += SCW * 32 * U) {
                uint32_t ix[U], pv[U], x[U], yv[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int t = e0 + u * 32 + lane;
                    ix[u] = t < pz ? __ldcg(pidx + t) : 0u;
                    pv[u] = t < pz ? __ldcg(pval + t) : 0u;
                }
                uint32_t secd = 0, secf = 0;
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const uint32_t cc = pv[u] ? __ldg(ext + ix[u]) : 0u;
                    yv[u] = pv[u] & cc;
                    const uint32_t fv = pv[u] & ~cc;
                    x[u] = diff ? fv : yv[u];
                    secd += __popc(__ballot_sync(0xffffffffu, yv[u] != 0u));
                    secf += __popc(__ballot_sync(0xffffffffu, fv != 0u));
                }
                if (b0 == 0 && sg == 0) {
                    if (lane == 0 && (secd | secf)) {
                        atomicAdd(&s.sec_dense, secd);
                        atomicAdd(&s.sec_diff, secf);
                    }
                    if (store) sparse_put<U>(p, s, store, half, ix, yv, lane);
                }
                int c = sg;
                for (; c + SG < kb; c += 2 * SG) {
                    const uint32_t *c0 = s.cptr[c], *c1 = s.cptr[c + SG];
                    uint32_t n0 = 0, n1 = 0;
#pragma unroll
                    for (int u = 0; u < U; u++)
                        if (x[u]) {
                            n0 += __popc(x[u] & __ldg(c0 + ix[u]));
                            n1 += __popc(x[u] & __ldg(c1 + ix[u]));
                        }
                    n0 = warp_sum_u32(n0);
                    n1 = warp_sum_u32(n1);
                    if (lane == 0) {
                        if (n0) atomicAdd(&s.sup[c], n0);
                        if (n1) atomicAdd(&s.sup[c + SG], n1);
                    }
                }
                for (; c < kb; c += SG) {
                    const uint32_t *c0 = s.cptr[c];
                    uint32_t n0 = 0;
#pragma unroll
                    for (int u = 0; u < U; u++)
                        if (x[u]) n0 += __popc(x[u] & __ldg(c0 + ix[u]));
                    n0 = warp_sum_u32(n0);
                    if (lane == 0 && n0) atomicAdd(&s.sup[c], n0);
                }
            }
        }
}

// Thread 0: record and item slots for tot itemsets of nitems items in all.
// A worker reserves slots in chunks (one returning global atomic per chunk,
// not per class); when a chunk cannot hold the class, its unused slots
// become holes -- records of length 0, which the compactor sorts after every
// itemset and leaves out -- and a new chunk is reserved.
__device__ __noinline__ void retire_records(const DfsParams &p, Smem &s) {
    const unsigned long long h = s.rec_end - s.rec_next;
    if (h) {
        for (unsigned long long r = s.rec_next; r < s.rec_end; r++)
            if (r < p.rec_cap) {
                p.rec_len[r] = 0u;
                p.rec_db[r] = 0xFFFFFFFFu;
            }
        atomicAdd(&p.ctr->rec_holes, h);
    }
    s.rec_next = s.rec_end;
}

__device__ __noinline__ void retire_slots(const DfsParams &p, Smem &s) {
    retire_records(p, s);
    if (s.it_end > s.it_next) atomicAdd(&p.ctr->item_holes, s.it_end - s.it_next);
    s.it_next = s.it_end;
}

__device__ __forceinline__ void reserve_slots(const DfsParams &p, Smem &s, unsigned tot, unsigned long long nitems,
                                           unsigned long long *rb, unsigned long long *ib) {
    if (s.rec_next + tot > s.rec_end) {
        retire_records(p, s);
        const unsigned long long want = tot > (unsigned)p.rec_chunk ? tot : (unsigned)p.rec_chunk;
        s.rec_next = atomicAdd(&p.ctr->n_records, want);
        s.rec_end = s.rec_next + want;
    }
    if (s.it_next + nitems > s.it_end) {
        if (s.it_end > s.it_next) atomicAdd(&p.ctr->item_holes, s.it_end - s.it_next);
        const unsigned long long want = nitems > ICH ? nitems : ICH;
        s.it_next = atomicAdd(&p.ctr->n_rec_items, want);
        s.it_end = s.it_next + want;
    }
    *rb = s.rec_next;
    *ib = s.it_next;
    s.rec_next += tot;
    s.it_next += nitems;
}

template <int NT>
__device__ int class_pass(const DfsParams &p, Smem &s, const uint32_t *cand, const uint32_t *psup,
                          int k, int plen, uint32_t *fi, uint32_t *fs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const DbView &db = s.db;
    const int nsrc = s.nsrc;
    const bool diff = s.diff != 0;
    uint32_t *store = s.store;
    const bool store_sparse = s.store_sparse != 0;
    const bool sparse_parent = s.psparse != 0;
    const int pz = sparse_parent ? s.pz : 0;
    int nF = 0;
    if (threadIdx.x == 0) { s.sec_dense = 0; s.sec_diff = 0; s.zcount = 0; }

    for (int b0 = 0; b0 < k; b0 += CB) {
        const int kb = min(CB, k - b0);
        for (int c = threadIdx.x; c < kb; c += NT) {
            s.cptr[c] = column(s, cand[b0 + c]);
            s.sup[c] = 0;
        }
        __syncthreads();
        if (sparse_parent) sparse_sweep<NT>(p, s, kb, b0 == 0);
        else dense_sweep<NT>(p, s, kb, b0 == 0);
        __syncthreads();
        if (kb <= 32) {
            // few candidates (the common case): warp 0 alone, one ballot, no
            // block-wide scan
            if (warp == 0) {
                uint32_t item = 0, sup = 0;
                bool f = false;
                if (lane < kb) {
                    item = cand[b0 + lane];
                    sup = diff ? psup[b0 + lane] - s.sup[lane] : s.sup[lane];
                    f = sup >= db.thr;
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, f);
                const uint32_t tot = __popc(bal);
                if (tot) {
                    unsigned long long rb = 0, ib = 0;
                    if (lane == 0) reserve_slots(p, s, tot, (unsigned long long)tot * (plen + 1), &rb, &ib);
                    rb = __shfl_sync(0xffffffffu, rb, 0);
                    ib = __shfl_sync(0xffffffffu, ib, 0);
                    if (f) {
                        const uint32_t pos = __popc(bal & ((1u << lane) - 1u));
                        fi[nF + pos] = item;
                        fs[nF + pos] = sup;
                        const unsigned long long r = rb + pos;
                        const unsigned long long it = ib + (unsigned long long)pos * (plen + 1);
                        if (r < p.rec_cap && it + plen + 1 <= p.rec_items_cap) {
                            p.rec_off[r] = it;
                            p.rec_len[r] = (uint32_t)(plen + 1);
                            p.rec_sup[r] = sup;
                            p.rec_db[r] = db.id;
                            for (int q = 0; q < plen; q++) p.rec_items[it + q] = s.path[q];
                            p.rec_items[it + plen] = item;
                        } else {
                            atomicOr(&p.ctr->overflow, r < p.rec_cap ? 2 : 1);
                        }
                    }
                }
                if (lane == 0) s.ftot = (int)tot;
            }
            __syncthreads();
            nF += s.ftot;
            continue;  // kb <= 32 < CB: this was the class's only batch
        }
        // compact the frequent candidates of this batch, in order
        for (int c0 = 0; c0 < kb; c0 += NT) {
            const int c = c0 + threadIdx.x;
            uint32_t item = 0, sup = 0, f = 0;
            if (c < kb) {
                item = cand[b0 + c];
                sup = diff ? psup[b0 + c] - s.sup[c] : s.sup[c];
                f = sup >= db.thr;
            }
            uint32_t tot;
            const uint32_t pos = block_scan<NT>(s, f, &tot);
            if (tot) {
                if (threadIdx.x == 0) reserve_slots(p, s, tot, (unsigned long long)tot * (plen + 1), &s.rbase, &s.ibase);
                __syncthreads();
                if (f) {
                    fi[nF + pos] = item;
                    fs[nF + pos] = sup;
                    const unsigned long long r = s.rbase + pos;
                    const unsigned long long it = s.ibase + (unsigned long long)pos * (plen + 1);
                    if (r < p.rec_cap && it + plen + 1 <= p.rec_items_cap) {
                        p.rec_off[r] = it;
                        p.rec_len[r] = (uint32_t)(plen + 1);
                        p.rec_sup[r] = sup;
                        p.rec_db[r] = db.id;
                        for (int q = 0; q < plen; q++) p.rec_items[it + q] = s.path[q];
                        p.rec_items[it + plen] = item;
                    } else {
                        atomicOr(&p.ctr->overflow, r < p.rec_cap ? 2 : 1);
                    }
                }
                nF += (int)tot;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        // algorithmic bytes are the dense operands whatever the representation
        const unsigned long long src_bytes = 4ull * db.nw * ((unsigned long long)nsrc + (store ? 1 : 0));
        const unsigned long long secs = diff ? s.sec_diff : s.sec_dense;
        // touched: a sparse parent reads (index, word) pairs and one sector of
        // col(c) per entry; a sparse store writes 8 bytes per entry
        const unsigned long long src_touched =
            sparse_parent ? 40ull * (unsigned long long)pz + (store ? 8ull * s.zcount : 0ull)
                          : 4ull * db.nw * ((unsigned long long)nsrc) +
                                (store ? (store_sparse ? 8ull * s.zcount : 4ull * db.nw) : 0ull);
        s.n_sup += (unsigned long long)k;
        s.n_words += (unsigned long long)k * (unsigned long long)db.nw;
        s.n_bytes += 4ull * db.nw * (unsigned long long)k + src_bytes;
        s.n_touched += 32ull * secs * (unsigned long long)k + src_touched;
        s.n_classes += 1ull;
        if (diff) s.n_diff += 1ull;
        if (nF > 0 && plen + 1 > s.max_len) s.max_len = plen + 1;
    }
    return nF;
}

// Features of class Y (support supY, parent support supX, k candidates with
// parent supports psup) -- the scheduling MLP's input, in a fixed order,
// each scaled to O(1) so that bf16 rounding of the input stays harmless.
__device__ void class_features(Smem &s, int ylen, uint32_t supY, uint32_t supX, const uint32_t *psup,
                               int k, float *out) {
    if (threadIdx.x < 32) {
        float acc = 0.f;
        for (int c = threadIdx.x; c < k; c += 32) acc += (float)psup[c];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) {
            const float sx = supX > 0 ? (float)supX : 1.f;
            const float sy = supY > 0 ? (float)supY : 1.f;
            out[0] = (float)ylen / 16.f;
            out[1] = log2f(1.f + (float)supY) / 32.f;
            out[2] = (float)supY / (float)(s.db.n > 0 ? s.db.n : 1);
            out[3] = log2f(1.f + (float)k) / 16.f;
            out[4] = (float)supY / sx;
            out[5] = k > 0 ? acc / ((float)k * sx) : 0.f;
            out[6] = log2f(1.f + (float)s.db.nw) / 32.f;
            out[7] = (float)s.db.thr / sy;
        }
    }
    __syncthreads();
}

// y = MLP(x) with bf16 weights and bf16-rounded activations, fp32 sums
// (the same arithmetic as the bf16 mode of fim_mlp_forward).  Result in s.y.
__device__ void mlp_infer(Smem &s, const float *x) {
    // shared-memory copy: W1 and W2 transposed ([in][out]) so that the lanes
    // of one warp read consecutive words; b1, b2, W3, b3 as stored
    const float *W1t = s.mlp_w, *b1 = W1t + 64 * 8, *W2t = b1 + 64, *b2 = W2t + 64 * 64, *W3 = b2 + 64,
                *b3 = W3 + 2 * 64;
    if (threadIdx.x < 32) {  // one warp; lane l owns hidden units l and l + 32
        const int l = threadIdx.x;
        float a0 = b1[l], a1 = b1[l + 32];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const float xi = bf16r(x[i]);
            a0 = fmaf(W1t[i * 64 + l], xi, a0);
            a1 = fmaf(W1t[i * 64 + l + 32], xi, a1);
        }
        const float h1a = bf16r(fmaxf(a0, 0.f)), h1b = bf16r(fmaxf(a1, 0.f));
        float c0 = b2[l], c1 = b2[l + 32];
#pragma unroll 8
        for (int i = 0; i < 32; i++) {  // inputs 0..31 (lane i's first unit), in order
            const float hi = __shfl_sync(0xffffffffu, h1a, i);
            c0 = fmaf(W2t[i * 64 + l], hi, c0);
            c1 = fmaf(W2t[i * 64 + l + 32], hi, c1);
        }
#pragma unroll 8
        for (int i = 0; i < 32; i++) {  // inputs 32..63
            const float hi = __shfl_sync(0xffffffffu, h1b, i);
            c0 = fmaf(W2t[(32 + i) * 64 + l], hi, c0);
            c1 = fmaf(W2t[(32 + i) * 64 + l + 32], hi, c1);
        }
        const float h2a = bf16r(fmaxf(c0, 0.f)), h2b = bf16r(fmaxf(c1, 0.f));
        float y0 = W3[l] * h2a + W3[l + 32] * h2b;
        float y1 = W3[64 + l] * h2a + W3[64 + l + 32] * h2b;
        for (int d = 16; d > 0; d >>= 1) {
            y0 += __shfl_xor_sync(0xffffffffu, y0, d);
            y1 += __shfl_xor_sync(0xffffffffu, y1, d);
        }
        if (l == 0) {
            s.y[0] = y0 + b3[0];
            s.y[1] = y1 + b3[1];
        }
    }
    __syncthreads();
}

// Representation of class Y before its pass: 1 = count through the diffset.
__device__ int choose_diff(const DfsParams &p, Smem &s, const float *feat, uint32_t supY, uint32_t supX,
                           bool infer) {
    if (p.learned) {
        if (!infer) return 0;  // too few candidates for the choice to matter: dense
        mlp_infer(s, feat);
        return s.y[1] > 0.f;
    }
    if (p.diffset_rule) return supX - supY < supY;  // |d_Y| < |b_Y| in bits
    return 0;
}

// Candidate list of the root class {a, b}: every c > b with {a,c} and {b,c}
// frequent, written ascending to out, with psup = S({a, c}).  Returns the
// count (all threads), or -1 if it does not fit.
template <int NT>
__device__ int root_candidates(const DfsParams &p, Smem &s, uint32_t a, uint32_t b, uint32_t *out,
                               uint32_t *psup, long long room) {
    const DbView &db = s.db;
    const uint32_t *ra = db.pairbits + (int64_t)a * db.mpw;
    const uint32_t *rb = db.pairbits + (int64_t)b * db.mpw;
    int n = 0;
    const int w0 = (int)(b >> 5);  // the word holding b; keep only c > b there
    for (int wb = w0; wb < db.mpw; wb += NT) {
        const int w = wb + threadIdx.x;
        uint32_t bits = 0;
        if (w < db.mpw) {
            bits = __ldg(ra + w) & __ldg(rb + w);
            if (w == w0) bits &= 0xFFFFFFFEu << (b & 31);
        }
        uint32_t tot;
        uint32_t pos = block_scan<NT>(s, __popc(bits), &tot);
        if (n + (long long)tot > room) { if (threadIdx.x == 0) set_err(p, FIM_E_STACK); return -1; }
        while (bits) {
            const int bit = __ffs(bits) - 1;
            bits &= bits - 1;
            const uint32_t c = (uint32_t)(w * 32 + bit);
            out[n + pos] = c;
            psup[n + pos] = (uint32_t)__ldg(db.pair_cnt + (int64_t)a * db.mfreq + c);
            pos++;
        }
        n += (int)tot;
        __syncthreads();
    }
    return n;
}

// Try to hand the child class (prefix s.path[0..plen) + item, candidates
// cand[0..k)) to the queue.  Returns true if it was published.
template <int NT>
__device__ bool try_push(const DfsParams &p, Smem &s, int plen, uint32_t item, uint32_t sup,
                         const uint32_t *cand, int k) {
    if (threadIdx.x == 0) {
        s.flag = 0;
        const unsigned long long off = atomicAdd(&p.ctr->pool_top, (unsigned long long)k);
        if (off + k <= p.cand_pool_cap) {
            const unsigned long long slot = atomicAdd(&p.ctr->qtail, 1ull);
            if (slot < p.task_cap) {
                s.flag = 1;
                s.cand_off = (long long)off;
                s.ticket = slot;
            }
        }
    }
    __syncthreads();
    if (!s.flag) return false;
    for (int c = threadIdx.x; c < k; c += NT) p.cand_pool[s.cand_off + c] = cand[c];
    __threadfence();  // every writer fences before the flag is raised
    __syncthreads();
    if (threadIdx.x == 0) {
        Task *t = p.tasks + s.ticket;
        for (int q = 0; q < plen; q++) t->items[q] = s.path[q];
        t->items[plen] = item;
        t->len = (uint32_t)(plen + 1);
        t->support = sup;
        t->n_cand = (uint32_t)k;
        t->cand_off = (unsigned long long)s.cand_off;
        t->prio = 0.f;
        t->db = s.db.id;
        atomicAdd((unsigned long long *)&p.ctr->pending, 1ull);
        atomicAdd(&p.ctr->pushed, 1ull);
        __threadfence();
        // (the fault-injection hook withholds one publish: the worker that
        // takes this slot, and every worker waiting for the queue to drain,
        // must give up at the spin limit)
        if ((long long)s.ticket != p.withhold_slot) atomicExch(&t->ready, s.epoch);
    }
    __syncthreads();
    return true;
}

// Close level L: its subtree is complete.  Write its trace row and pass its
// work up to level L-1.
__device__ void close_level(const DfsParams &p, Smem &s, int L) {
    if (threadIdx.x == 0) {
        if (p.trace) {
            const unsigned long long r = atomicAdd(&p.ctr->n_traces, 1ull);
            if (r < p.trace_cap) {
                for (int i = 0; i < NF; i++) p.trace_x[r * NF + i] = s.feat[L][i];
                p.trace_y[r * 2 + 0] = log2f(1.f + (float)s.work[L]);
                p.trace_y[r * 2 + 1] = s.label[L];
            }
        }
        if (L > 0) s.work[L - 1] += s.work[L];
    }
    __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT)
dfs_kernel(const DfsParams p) {
    extern __shared__ __align__(16) uint8_t dyn_smem[];
    Smem &s = *reinterpret_cast<Smem *>(dyn_smem);
    const int wid = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *fi = p.frame_items + (int64_t)wid * p.frame_pool;
    uint32_t *fs = p.frame_sups + (int64_t)wid * p.frame_pool;
    uint32_t *stk = p.stack_bits + (int64_t)wid * p.depth_cap * p.nwp_max;
    if (p.learned)
        for (int i = threadIdx.x; i < FIM_MLP_PARAMS; i += NT) {
            // W1 [64][8] and W2 [64][64] are stored [out][in]; keep them [in][out]
            int d = i;
            if (i < 64 * 8) d = (i % 8) * 64 + i / 8;
            else if (i >= 64 * 8 + 64 && i < 64 * 8 + 64 + 64 * 64) {
                const int k = i - (64 * 8 + 64);
                d = 64 * 8 + 64 + (k % 64) * 64 + k / 64;
            }
            s.mlp_w[d] = __bfloat162float(p.mlp_w[i]);
        }
    // thread 0's timing state lives in shared memory, not in every thread's registers
    if (threadIdx.x == 0) {
        s.busy = 0;
        s.root_busy = 0;
        atomicCAS(&p.ctr->t_first, 0ull, globaltimer_ns());
        s.n_roots = *(volatile unsigned long long *)&p.ctr->n_roots;  // final before the DFS starts
        s.epoch = *(volatile const uint32_t *)p.epoch;
        s.err_seen = 0;
        s.iter = 0;
        s.rec_next = s.rec_end = 0;
        s.it_next = s.it_end = 0;
        s.n_sup = s.n_words = s.n_bytes = s.n_touched = s.n_classes = s.n_diff = 0ull;
        s.max_len = 0;
    }

    while (true) {
        // ---- get the next task ---------------------------------------
        if (threadIdx.x == 0) {
            s.flag = 0;
            const unsigned long long t = atomicAdd(&p.ctr->ticket, 1ull);
            const unsigned long long nr = *(volatile unsigned long long *)&p.ctr->n_roots;
            if (*(volatile int *)&p.ctr->err != 0) {
                // an error ends the mine: take no more work
            } else if (t < nr) {
                // roots come out of the pair pass by ascending first item, i.e.
                // ascending item support; root_reverse hands out the pairs of
                // the most frequent items (the largest subtrees) first
                const unsigned long long tt = p.root_reverse ? nr - 1 - t : t;
                const unsigned long long rt = p.root_order ? p.root_order[tt] : tt;
                s.path[0] = p.root_a[rt];
                s.path[1] = p.root_b[rt];
                s.task_len = 2;
                s.task_sup = p.root_sup[rt];
                s.task_db = p.root_db ? p.root_db[rt] : 0u;
                s.ncand = -1;
                s.flag = 1;
            } else if (t - nr < p.task_cap) {
                Task *tk = p.tasks + (t - nr);
                unsigned long long spins = 0;
                const unsigned long long t_wait = globaltimer_ns();
                while (true) {
                    if (*(volatile uint32_t *)&tk->ready == s.epoch) {
                        __threadfence();
                        const int len = (int)*(volatile uint32_t *)&tk->len;
                        for (int q = 0; q < len; q++) s.path[q] = ((volatile uint32_t *)tk->items)[q];
                        s.task_len = len;
                        s.task_sup = *(volatile uint32_t *)&tk->support;
                        s.task_db = *(volatile uint32_t *)&tk->db;
                        s.ncand = (int)*(volatile uint32_t *)&tk->n_cand;
                        s.cand_off = (long long)*(volatile unsigned long long *)&tk->cand_off;
                        s.flag = 1;
                        break;
                    }
                    if (*(volatile long long *)&p.ctr->pending == 0) break;
                    if (*(volatile int *)&p.ctr->err != 0) break;
                    if ((++spins & 1023) == 0 && globaltimer_ns() - t_wait > p.spin_limit) {
                        set_err(p, FIM_E_TIMEOUT);
                        break;
                    }
                    __nanosleep(spins < 64 ? 64 : 512);
                }
            } else {
                // beyond the queue: nothing can arrive here; wait for the end
                unsigned long long spins = 0;
                const unsigned long long t_wait = globaltimer_ns();
                while (*(volatile long long *)&p.ctr->pending != 0 &&
                       *(volatile int *)&p.ctr->err == 0) {
                    if ((++spins & 1023) == 0 && globaltimer_ns() - t_wait > p.spin_limit) {
                        set_err(p, FIM_E_TIMEOUT);
                        break;
                    }
                    __nanosleep(512);
                }
            }
            if (s.flag) {
                load_db(p, s, s.task_db);
                s.t_task = globaltimer_ns();
            }
        }
        __syncthreads();
        if (!s.flag) break;
        // the task database's perm, for the column pointers of its classes
        // (the barriers of the candidate setup below publish it)
        for (int i = threadIdx.x; i < min(s.db.mfreq, PCAP); i += NT) s.perm_c[i] = __ldg(s.db.perm + i);

        // ---- level 0: the task's own class ---------------------------
        const int tlen = s.task_len;
        const bool root = s.ncand < 0;
        int k;
        if (root) {
            k = root_candidates<NT>(p, s, s.path[0], s.path[1], fi, fs, p.frame_pool);
        } else {
            k = s.ncand;
            if (k > p.frame_pool) { if (threadIdx.x == 0) set_err(p, FIM_E_STACK); k = -1; }
            else for (int c = threadIdx.x; c < k; c += NT) fi[c] = __ldcg(p.cand_pool + s.cand_off + c);
            __syncthreads();
        }
        const uint32_t maxlen = s.db.maxlen;
        const bool len_ok = maxlen == 0 || (uint32_t)tlen + 1 <= maxlen;
        if (k > 0 && len_ok) {
            // a root {a, b} has parent {a}: b_X = col(a), S(X) = S({a})
            const uint32_t supX =
                root ? (uint32_t)__ldg(s.db.item_sup + __ldg(s.db.perm + s.path[0])) : s.task_sup;
            // the network is consulted only where its choice can pay for the
            // inference: classes with at least learned_kmin candidates
            const bool infer = p.learned && root && k >= p.learned_kmin;
            if (p.trace || infer) class_features(s, tlen, s.task_sup, supX, fs, root ? k : 0, s.feat[0]);
            const int diff = root ? choose_diff(p, s, s.feat[0], s.task_sup, supX, infer) : 0;
            if (threadIdx.x == 0) {
                for (int r = 0; r < tlen; r++) s.src[r] = column(s, s.path[r]);
                s.nsrc = tlen;
                s.diff = diff;
                s.psparse = 0;
                // a root {a, b} whose parent column col(a) has a sparse copy
                // gathers col(b) and the candidates at col(a)'s non-zero words
                if (root && p.item_z) {
                    const int za = __ldg(p.item_z + s.path[0]);
                    if (za >= 0) {
                        s.psparse = 1;
                        s.pz = za;
                        s.pidx = p.item_idx + (int64_t)s.path[0] * p.item_cap;
                        s.pval = p.item_val + (int64_t)s.path[0] * p.item_cap;
                    }
                }
                s.store = k >= 2 ? stk : nullptr;
                // a sparse parent's child has no more entries than the parent
                // (item_cap <= half a stack level), so it is stored sparse too
                s.store_sparse = s.psparse || sparse_ok(p, s.db, s.task_sup);
                s.base[0] = 0;
                s.supY[0] = s.task_sup;
                s.work[0] = (unsigned long long)k * (unsigned long long)s.db.nw;
            }
            __syncthreads();
            // candidates live at fi[0..k), parent supports at fs[0..k); F_0
            // overwrites both in order
            int nF = class_pass<NT>(p, s, fi, fs, k, tlen, fi, fs);
            if (threadIdx.x == 0) {
                if (root) s.root_busy += globaltimer_ns() - s.t_task;
                s.lz[0] = (s.store && s.store_sparse) ? (int)s.zcount : -1;
                s.nF[0] = nF;
                s.cur[0] = 0;
                s.base[1] = nF;
                s.label[0] = (s.nsrc == 2 && s.sec_diff < s.sec_dense) ? 1.f : 0.f;
            }
            __syncthreads();
            int L = 0;
            while (L >= 0) {
                // the error flag is read with the queue counters at each push
                // decision; a class without one re-reads it every 16 classes.
                // The counters are loaded here, before the barrier and the
                // sibling gather, and first used after them: their round trip
                // overlaps that work instead of adding to it
                int q_err = 0;
                unsigned long long q_ticket = 0, q_tail = 0;
                if (threadIdx.x == 0) {
                    if ((++s.iter & 15u) == 0u) s.err_seen = *(volatile int *)&p.ctr->err;
                    s.stop = s.err_seen != 0;
                    if (tlen + L + 1 <= p.split_depth && tlen + L + 1 <= FIM_TASK_MAXR) {
                        q_err = *(volatile int *)&p.ctr->err;
                        q_ticket = *(volatile unsigned long long *)&p.ctr->ticket;
                        q_tail = *(volatile unsigned long long *)&p.ctr->qtail;
                    }
                }
                __syncthreads();
                if (s.stop) break;
                if (s.cur[L] >= s.nF[L]) {
                    close_level(p, s, L);
                    L--;
                    continue;
                }
                const int j = s.cur[L];  // thread 0 advances cur[L] after the barrier below
                const int plen = tlen + L;          // prefix length at level L
                const long long bL = s.base[L];
                const long long bC = s.base[L + 1]; // child's candidates go here
                const uint32_t citem = fi[bL + j];
                const uint32_t csup = fs[bL + j];
                // child candidates: later frequent siblings paired with citem,
                // each with its support in this class (the child's parent)
                int kc = 0;
                const int nFL = s.nF[L];
                const bool may_push = plen + 1 <= p.split_depth && plen + 1 <= FIM_TASK_MAXR;
                if (nFL - (j + 1) <= 32) {
                    // few siblings: warp 0 alone, compacted with a ballot
                    if (warp == 0) {
                        const int l = j + 1 + lane;
                        uint32_t d = 0, ds = 0;
                        bool f = false;
                        if (l < nFL) { d = fi[bL + l]; ds = fs[bL + l]; f = pairbit(s.db, citem, d); }
                        const uint32_t bal = __ballot_sync(0xffffffffu, f);
                        const int tot = __popc(bal);
                        if (bC + (long long)tot > p.frame_pool) {
                            if (lane == 0) { set_err(p, FIM_E_STACK); s.kc = -1; }
                        } else {
                            if (f) {
                                const int pos = __popc(bal & ((1u << lane) - 1u));
                                fi[bC + pos] = d;
                                fs[bC + pos] = ds;
                            }
                            if (lane == 0) s.kc = tot;
                        }
                    }
                } else {
                    bool overflow = false;
                    for (int l0 = j + 1; l0 < nFL; l0 += NT) {
                        const int l = l0 + threadIdx.x;
                        uint32_t d = 0, ds = 0, f = 0;
                        if (l < nFL) { d = fi[bL + l]; ds = fs[bL + l]; f = pairbit(s.db, citem, d); }
                        uint32_t tot;
                        const uint32_t pos = block_scan<NT>(s, f, &tot);
                        if (bC + kc + (long long)tot > p.frame_pool) { overflow = true; break; }
                        if (f) { fi[bC + kc + pos] = d; fs[bC + kc + pos] = ds; }
                        kc += (int)tot;
                    }
                    if (threadIdx.x == 0) {
                        if (overflow) set_err(p, FIM_E_STACK);
                        s.kc = overflow ? -1 : kc;
                    }
                }
                if (threadIdx.x == 0 && may_push) {
                    // the queue's hunger and the error flag, loaded at the top
                    // of this iteration, published by the barrier below
                    // (s.hungry, not s.flag: thread 0 rewrites s.flag inside
                    // try_push)
                    s.hungry = q_ticket > s.n_roots + q_tail;
                    s.err_seen = q_err;
                }
                __syncthreads();
                kc = s.kc;
                if (threadIdx.x == 0) s.cur[L] = j + 1;  // every thread has read cur[L]
                if (kc < 0) break;
                if (kc == 0) continue;
                if (maxlen && (uint32_t)plen + 2 > maxlen) continue;
                if (may_push && s.hungry && try_push<NT>(p, s, plen, citem, csup, fi + bC, kc)) continue;
                if (L + 1 >= p.depth_cap || plen + 1 >= MAXPATH) {
                    if (threadIdx.x == 0) set_err(p, FIM_E_STACK);
                    break;
                }
                // descend: b_child = b_parent AND col(citem)
                const uint32_t supX = s.supY[L];
                const bool infer = p.learned && kc >= p.learned_kmin;
                if (p.trace || infer) class_features(s, plen + 1, csup, supX, fs + bC, kc, s.feat[L + 1]);
                const int diff = choose_diff(p, s, s.feat[L + 1], csup, supX, infer);
                if (threadIdx.x == 0) {
                    uint32_t *lv = stk + (int64_t)L * p.nwp_max;  // b_X, the class at level L
                    s.path[plen] = citem;
                    s.src[0] = lv;
                    s.src[1] = column(s, citem);
                    s.nsrc = 2;
                    s.psparse = s.lz[L] >= 0;
                    s.pz = s.lz[L];
                    s.pidx = lv;
                    s.pval = lv + p.nwp_max / 2;
                    s.diff = diff;
                    s.store = kc >= 2 ? stk + (int64_t)(L + 1) * p.nwp_max : nullptr;
                    s.store_sparse = s.psparse || sparse_ok(p, s.db, csup);
                    s.supY[L + 1] = csup;
                    s.work[L + 1] = (unsigned long long)kc * (unsigned long long)s.db.nw;
                }
                __syncthreads();
                nF = class_pass<NT>(p, s, fi + bC, fs + bC, kc, plen + 1, fi + bC, fs + bC);
                if (threadIdx.x == 0) {
                    s.lz[L + 1] = (s.store && s.store_sparse) ? (int)s.zcount : -1;
                    s.nF[L + 1] = nF;
                    s.cur[L + 1] = 0;
                    s.base[L + 2] = bC + nF;
                    s.label[L + 1] = s.sec_diff < s.sec_dense ? 1.f : 0.f;
                }
                // (the barrier at the top of the loop publishes these)
                L++;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd((unsigned long long *)&p.ctr->pending, (unsigned long long)(-1ll));
            s.busy += globaltimer_ns() - s.t_task;
        }
    }
    if (threadIdx.x == 0) {
        retire_slots(p, s);  // the worker's unused slots become holes
        if (s.n_classes) {
            atomicAdd(&p.ctr->supports_dfs, s.n_sup);
            atomicAdd(&p.ctr->dfs_words, s.n_words);
            atomicAdd(&p.ctr->dfs_bytes, s.n_bytes);
            atomicAdd(&p.ctr->dfs_touched, s.n_touched);
            atomicAdd(&p.ctr->classes, s.n_classes);
            if (s.n_diff) atomicAdd(&p.ctr->diffset, s.n_diff);
        }
        if (s.max_len) atomicMax(&p.ctr->max_len, s.max_len);
        atomicAdd(&p.ctr->busy_ns, s.busy);
        atomicAdd(&p.ctr->root_ns, s.root_busy);
        atomicMax(&p.ctr->t_last, globaltimer_ns());
    }
}

// One CTA per frequent item i (internal id): if S(i) <= cap, its column's
// non-zero words go to [i * cap, i * cap + z) as (index, word), in any order.
__global__ void __launch_bounds__(256)
sparse_items_kernel(const uint32_t *__restrict__ bm, const int32_t *__restrict__ perm,
                    const uint32_t *__restrict__ item_sup, int64_t nwp, int64_t cap, uint32_t *__restrict__ idx,
                    uint32_t *__restrict__ val, int *__restrict__ z) {
    __shared__ unsigned int cnt;
    const int i = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const int32_t j = perm[i];
    if (item_sup[j] > (uint64_t)cap) {
        if (threadIdx.x == 0) z[i] = -1;
        return;
    }
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const uint32_t *col = bm + (int64_t)j * nwp;
    uint32_t *oi = idx + (int64_t)i * cap, *ov = val + (int64_t)i * cap;
    for (int64_t w0 = 0; w0 < nwp; w0 += 4 * 256) {  // nwp % 128 == 0: trips are warp-uniform
        const int64_t pos = w0 + 4 * threadIdx.x;
        const uint4 y = pos < nwp ? ldg_u4(col + pos) : make_uint4(0, 0, 0, 0);
        const uint32_t w[4] = {y.x, y.y, y.z, y.w};
        const uint32_t c = (w[0] != 0u) + (w[1] != 0u) + (w[2] != 0u) + (w[3] != 0u);
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        uint32_t base = 0;
        if (lane == 31 && x) base = atomicAdd(&cnt, x);
        base = __shfl_sync(0xffffffffu, base, 31);
        uint32_t at = base + x - c;
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (w[q]) {
                if (at < cap) {  // at most S(i) <= cap words are non-zero
                    oi[at] = (uint32_t)(pos + q);
                    ov[at] = w[q];
                }
                at++;
            }
    }
    __syncthreads();
    if (threadIdx.x == 0) z[i] = (int)cnt;
}

__global__ void epoch_bump_kernel(uint32_t *e) {
    const uint32_t v = *e + 1u;
    *e = v ? v : 1u;  // 0 marks a slot that was never published
}

}  // namespace

int prepare_task_queue(fim_ctx *ctx, size_t bytes) {
    void *old = ctx->tasks.p;
    FIM_TRY(fim_reserve(ctx, ctx->tasks, bytes));
    if (ctx->tasks.p != old) FIM_CUDA_TRY(cudaMemsetAsync(ctx->tasks.p, 0, ctx->tasks.bytes, ctx->stream));
    return FIM_OK;
}

int reserve_sparse_items(fim_ctx *ctx, int mf, int64_t cap) {
    if (mf <= 0) return FIM_OK;
    FIM_TRY(fim_reserve(ctx, ctx->sp_idx, sizeof(uint32_t) * (size_t)mf * (size_t)cap));
    FIM_TRY(fim_reserve(ctx, ctx->sp_val, sizeof(uint32_t) * (size_t)mf * (size_t)cap));
    FIM_TRY(fim_reserve(ctx, ctx->sp_z, sizeof(int) * (size_t)mf));
    return FIM_OK;
}

int launch_sparse_items(fim_ctx *ctx, int mf, int64_t cap, cudaStream_t st) {
    if (mf <= 0) return FIM_OK;
    ctx->launches++;
    sparse_items_kernel<<<mf, 256, 0, st>>>(ctx->bm.as<uint32_t>(), ctx->perm.as<int32_t>(),
                                                     ctx->item_sup.as<uint32_t>(), ctx->nwp, cap,
                                                     ctx->sp_idx.as<uint32_t>(), ctx->sp_val.as<uint32_t>(),
                                                     ctx->sp_z.as<int>());
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

int launch_epoch_bump(fim_ctx *ctx) {
    ctx->launches++;
    epoch_bump_kernel<<<1, 1, 0, ctx->stream>>>(ctx->epoch.as<uint32_t>());
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

int launch_dfs(fim_ctx *ctx, const DfsParams &p, int grid, int block) {
    if (grid <= 0) return FIM_OK;
    const size_t smem = sizeof(Smem);
    ctx->launches++;
    if (block == 256) {
        FIM_CUDA_TRY(cudaFuncSetAttribute(dfs_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        dfs_kernel<256><<<grid, 256, smem, ctx->stream>>>(p);
    } else {
        FIM_CUDA_TRY(cudaFuncSetAttribute(dfs_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        dfs_kernel<512><<<grid, 512, smem, ctx->stream>>>(p);
    }
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}
