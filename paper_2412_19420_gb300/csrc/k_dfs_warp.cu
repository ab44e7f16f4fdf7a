// k_dfs_warp.cu -- recursive prefix extension with one warp per worker, for
// databases whose bit columns are short.
//
// The same search as dfs_kernel (Section III: the column AND "in sequence",
// Eq. 3's threshold pruning every infrequent extension), laid out for classes
// whose prefix bitmap spans a few hundred words: a class's whole pass is a
// handful of 128-word chunks, so a CTA-wide worker spends its time in block
// barriers and serial bookkeeping.  Here every warp is an independent
// worker -- eight per CTA, no block barrier anywhere -- taking root classes
// {a, b} from the ticket counter (in the root plan's order) and mining each
// subtree depth-first to the end.  Per class:
//   b_Y = b_X AND col(c)   (recomputed chunk by chunk from the parent's
//                           stored bitmap; stored itself when Y has >= 2
//                           candidates, so its children can read it)
//   S(Y u {e}) = popc(b_Y AND col(e)) for every candidate e, 8 candidates per
//   sweep over the chunks, each lane one 16-byte slice of the prefix and of
//   each candidate, all loaded together; shuffle sums per candidate.
// Frequent extensions become result records and the child list.  The counts
// are exact integers; no representation choice, queue or splitting is needed
// at these sizes (the roots are many and come longest first).
#include "fim_common.cuh"

namespace {

constexpr int WW = 8;        // warps (workers) per CTA
constexpr int WMAXP = 64;    // longest itemset a warp worker tracks
constexpr int WG = 8;        // candidates counted per sweep of the prefix

struct WarpState {
    const uint32_t *bm;
    const int32_t *perm;
    const uint32_t *pairbits;
    const int *pair_cnt;
    const uint32_t *item_sup;
    int64_t nwp, nw;
    int32_t mfreq, mpw;
    uint32_t thr, maxlen, db;
    uint32_t path[WMAXP];
    int nF[WMAXP], cur[WMAXP];
    long long base[WMAXP + 1];
    // the worker's statistics, summed here by lane 0 and added to the global
    // counters once, at exit: per-class atomics on those few shared words
    // queued every worker's ticket and record atomics behind them
    unsigned long long n_sup, n_words, n_bytes, n_touched, n_classes, n_roots_done;
    int max_len;
};

__device__ __forceinline__ const uint32_t *wcol(const WarpState &s, uint32_t item) {
    return s.bm + (int64_t)__ldg(s.perm + item) * s.nwp;
}

__device__ __forceinline__ bool wpairbit(const WarpState &s, uint32_t a, uint32_t b) {
    return (__ldg(s.pairbits + (int64_t)a * s.mpw + (b >> 5)) >> (b & 31)) & 1u;
}

__device__ void wset_err(const DfsParams &p, int code) { atomicCAS(&p.ctr->err, 0, code); }

// One class pass: prefix b_Y = src0 AND src1 (word-aligned columns, zero
// padded to a multiple of 128 words), candidates cand[0..k) with parent
// supports; frequent ones compacted in order into fi/fs (which may alias
// cand/psup: a group's entries are read before any write reaches them) and
// emitted as records with prefix s.path[0..plen).  Returns |F| (uniform).
__device__ int warp_class_pass(const DfsParams &p, WarpState &s, const uint32_t *src0, const uint32_t *src1,
                               const uint32_t *cand, int k, int plen, uint32_t *store, uint32_t *fi,
                               uint32_t *fs) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = s.nw;
    int nF = 0;
    unsigned long long secs = 0;
    for (int g0 = 0; g0 < k; g0 += WG) {
        const int gn = min(WG, k - g0);
        // column pointers of this group's candidates (lane c looks up candidate c)
        uint32_t my_item = lane < gn ? cand[g0 + lane] : 0u;
        const uint32_t *my_col = lane < gn ? wcol(s, my_item) : nullptr;
        const uint32_t *cp[WG];
#pragma unroll
        for (int c = 0; c < WG; c++)
            cp[c] = reinterpret_cast<const uint32_t *>(
                __shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(my_col), c));
        uint32_t acc[WG];
#pragma unroll
        for (int c = 0; c < WG; c++) acc[c] = 0u;
        for (int64_t w0 = (int64_t)lane * 4; w0 - lane * 4 < nw; w0 += 128) {
            // the prefix's and the candidates' slices of this chunk are loaded
            // together: one memory round trip per chunk (these classes are
            // latency-bound, not bandwidth-bound)
            const uint4 s0 = ld_cg_u4(src0 + w0), s1 = ld_cg_u4(src1 + w0);
            uint4 cv[WG];
#pragma unroll
            for (int c = 0; c < WG; c++) cv[c] = c < gn ? ldg_u4(cp[c] + w0) : make_uint4(0u, 0u, 0u, 0u);
            const uint4 y = and4(s0, s1);
            if (g0 == 0) {
                if (store) *reinterpret_cast<uint4 *>(store + w0) = y;
                const uint32_t bz = __ballot_sync(0xffffffffu, (y.x | y.y | y.z | y.w) != 0u);
                secs += __popc((bz | (bz >> 1)) & 0x55555555u);  // non-zero 32-byte sectors
            }
#pragma unroll
            for (int c = 0; c < WG; c++) acc[c] += popc_and4(y, cv[c]);
        }
        // sums per candidate; lane c keeps candidate c's
        uint32_t mine = 0;
#pragma unroll
        for (int c = 0; c < WG; c++) {
            const uint32_t t = warp_sum_u32(acc[c]);
            if (lane == c) mine = t;
        }
        const bool f = lane < gn && mine >= s.thr;
        const uint32_t bal = __ballot_sync(0xffffffffu, f);
        const int tot = __popc(bal);
        if (tot) {
            unsigned long long rb = 0, ib = 0;
            if (lane == 0) {
                rb = atomicAdd(&p.ctr->n_records, (unsigned long long)tot);
                ib = atomicAdd(&p.ctr->n_rec_items, (unsigned long long)tot * (plen + 1));
            }
            rb = __shfl_sync(0xffffffffu, rb, 0);
            ib = __shfl_sync(0xffffffffu, ib, 0);
            if (f) {
                const int pos = __popc(bal & ((1u << lane) - 1u));
                fi[nF + pos] = my_item;
                fs[nF + pos] = mine;
                const unsigned long long r = rb + pos, it = ib + (unsigned long long)pos * (plen + 1);
                if (r < p.rec_cap && it + plen + 1 <= p.rec_items_cap) {
                    p.rec_off[r] = it;
                    p.rec_len[r] = (uint32_t)(plen + 1);
                    p.rec_sup[r] = mine;
                    p.rec_db[r] = s.db;
                    for (int q = 0; q < plen; q++) p.rec_items[it + q] = s.path[q];
                    p.rec_items[it + plen] = my_item;
                } else {
                    atomicOr(&p.ctr->overflow, r < p.rec_cap ? 2 : 1);
                }
            }
            nF += tot;
        }
        __syncwarp();
    }
    if (lane == 0) {
        const unsigned long long src_bytes = 4ull * nw * (2ull + (store ? 1ull : 0ull));
        s.n_sup += (unsigned long long)k;
        s.n_words += (unsigned long long)k * (unsigned long long)nw;
        s.n_bytes += 4ull * nw * (unsigned long long)k + src_bytes;
        s.n_touched += 32ull * secs * (unsigned long long)k + src_bytes;
        s.n_classes += 1ull;
        if (nF > 0 && plen + 1 > s.max_len) s.max_len = plen + 1;
    }
    return nF;
}

template <int MB>
__global__ void __launch_bounds__(WW * 32, MB)
dfs_warp_kernel(const DfsParams p) {
    __shared__ WarpState ws[WW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpState &s = ws[warp];
    const int64_t wid = (int64_t)blockIdx.x * WW + warp;
    uint32_t *fi = p.frame_items + wid * p.frame_pool;
    uint32_t *fs = p.frame_sups + wid * p.frame_pool;
    uint32_t *stk = p.stack_bits + wid * (int64_t)p.depth_cap * p.nwp_max;
    // the roots of a window (one group of databases), or all of them
    const unsigned long long nr = p.win ? *(volatile const unsigned long long *)&p.win->kept
                                        : *(volatile const unsigned long long *)&p.ctr->n_roots;
    const unsigned long long rbase = p.win ? p.win->base : 0ull;
    unsigned long long *const ticket = p.win ? &p.win->ticket : &p.ctr->ticket;
    unsigned long long busy = 0, t_task = 0;
    if (lane == 0) {
        atomicCAS(&p.ctr->t_first, 0ull, globaltimer_ns());
        s.n_sup = s.n_words = s.n_bytes = s.n_touched = s.n_classes = s.n_roots_done = 0ull;
        s.max_len = 0;
    }
    unsigned int iter = 0;
    // Roots are taken TCH at a time, and the next chunk's ticket is fetched
    // when a chunk starts: one contended atomic per TCH roots, its latency
    // hidden behind the chunk (with a ticket per root, a warp waited on the
    // counter about a third of its time).
    constexpr unsigned long long TCH = 4;
    unsigned long long t_cur = 0, t_end = 0, t_pref = 0;  // lane 0's chunk and the prefetched start
    int err = 0;
    // lane j < TCH holds root j of the current chunk: all of a chunk's root
    // records are loaded at once, not one dependent chain per root
    uint32_t my_a = 0, my_b = 0, my_db = 0;
    if (lane == 0) t_pref = atomicAdd(ticket, TCH);
    while (true) {
        unsigned long long t = 0;
        int fresh = 0, jr = 0;
        if (lane == 0) {
            if (t_cur >= t_end) {  // chunk done: take the prefetched one, prefetch the next
                t_cur = t_pref;
                t_end = t_pref + TCH;
                if (t_cur < nr) t_pref = atomicAdd(ticket, TCH);
                err = *(volatile int *)&p.ctr->err;
                fresh = 1;
            }
            jr = (int)(t_cur - (t_end - TCH));  // the root's place in its chunk
            t = t_cur++;
            t_task = globaltimer_ns();
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        err = __shfl_sync(0xffffffffu, err, 0);
        fresh = __shfl_sync(0xffffffffu, fresh, 0);
        jr = __shfl_sync(0xffffffffu, jr, 0);
        if (t >= nr || err) break;
        if (fresh) {  // t is the chunk's first root
            const unsigned long long tl = t + (unsigned long long)lane;
            if (lane < (int)TCH && tl < nr) {
                const unsigned long long tt = p.root_reverse ? nr - 1 - tl : tl;
                const unsigned long long rt = p.root_order ? p.root_order[rbase + tt] : rbase + tt;
                my_a = p.root_a[rt];
                my_b = p.root_b[rt];
                my_db = p.root_db ? p.root_db[rt] : 0u;
            }
        }
        const uint32_t a = __shfl_sync(0xffffffffu, my_a, jr), b = __shfl_sync(0xffffffffu, my_b, jr);
        const uint32_t dbi = __shfl_sync(0xffffffffu, my_db, jr);
        if (lane == 0) {
            const DbDesc &d = p.dbs[dbi];
            s.bm = p.bm + d.bm_off;
            s.perm = p.perm + d.item_off;
            s.item_sup = p.item_sup + d.item_off;
            s.pair_cnt = p.pair_cnt + d.pair_off;
            s.pairbits = p.pairbits + d.pb_off;
            s.nwp = d.nwp;
            s.nw = d.nw;
            s.mfreq = *(volatile const int32_t *)&d.mfreq;
            s.mpw = (s.mfreq + 31) / 32;
            s.thr = d.thr;
            s.maxlen = d.maxlen;
            s.db = dbi;
            s.path[0] = a;
            s.path[1] = b;
        }
        __syncwarp();
        const uint32_t maxlen = s.maxlen;
        // root candidates: c > b with {a, c} and {b, c} frequent, ascending,
        // with S({a, c}) -- lane = one word of the pair bitset rows at a time
        int k = 0;
        {
            const uint32_t *ra = s.pairbits + (int64_t)a * s.mpw, *rb = s.pairbits + (int64_t)b * s.mpw;
            const int w0 = (int)(b >> 5);
            for (int wb = w0; wb < s.mpw; wb += 32) {
                const int w = wb + lane;
                uint32_t bits = 0;
                if (w < s.mpw) {
                    bits = __ldg(ra + w) & __ldg(rb + w);
                    if (w == w0) bits &= 0xFFFFFFFEu << (b & 31);
                }
                const uint32_t cnt = __popc(bits);
                uint32_t x = cnt;  // inclusive scan of the counts over the lanes
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                const uint32_t tot = __shfl_sync(0xffffffffu, x, 31);
                if (k + (long long)tot > p.frame_pool) {
                    if (lane == 0) wset_err(p, FIM_E_STACK);
                    k = -1;
                    break;
                }
                uint32_t pos = k + x - cnt;
                while (bits) {
                    const uint32_t c = (uint32_t)(w * 32 + __ffs(bits) - 1);
                    bits &= bits - 1;
                    fi[pos] = c;
                    fs[pos] = (uint32_t)__ldg(s.pair_cnt + (int64_t)a * s.mfreq + c);
                    pos++;
                }
                k += (int)tot;
            }
        }
        __syncwarp();
        const bool len_ok = maxlen == 0 || 3 <= maxlen;
        if (k > 0 && len_ok) {
            // level 0: the root class {a, b}, b_Y = col(a) AND col(b)
            const uint32_t *ca = wcol(s, a), *cb = wcol(s, b);
            int nF = warp_class_pass(p, s, ca, cb, fi, k, 2, k >= 2 ? stk : nullptr, fi, fs);
            if (lane == 0) {
                s.nF[0] = nF;
                s.cur[0] = 0;
                s.base[0] = 0;
                s.base[1] = nF;
            }
            __syncwarp();
            int L = 0;
            while (L >= 0) {
                if ((++iter & 15u) == 0u) {
                    int e = 0;
                    if (lane == 0) e = *(volatile int *)&p.ctr->err;
                    if (__shfl_sync(0xffffffffu, e, 0)) break;
                }
                const int nFL = s.nF[L];
                const int j = s.cur[L];
                if (j >= nFL) {
                    L--;
                    continue;
                }
                const int plen = 2 + L;  // prefix length at level L
                const long long bL = s.base[L], bC = s.base[L + 1];
                const uint32_t citem = fi[bL + j];
                // child candidates: later frequent siblings paired with citem
                int kc = 0;
                for (int l0 = j + 1; l0 < nFL; l0 += 32) {
                    const int l = l0 + lane;
                    uint32_t d = 0, ds = 0;
                    bool f = false;
                    if (l < nFL) { d = fi[bL + l]; ds = fs[bL + l]; f = wpairbit(s, citem, d); }
                    const uint32_t bal = __ballot_sync(0xffffffffu, f);
                    if (bC + kc + (long long)__popc(bal) > p.frame_pool) {
                        kc = -1;
                        break;
                    }
                    if (f) {
                        const int pos = kc + __popc(bal & ((1u << lane) - 1u));
                        fi[bC + pos] = d;
                        fs[bC + pos] = ds;
                    }
                    kc += __popc(bal);
                }
                if (lane == 0) s.cur[L] = j + 1;
                __syncwarp();
                if (kc < 0) {
                    if (lane == 0) wset_err(p, FIM_E_STACK);
                    break;
                }
                if (kc == 0) continue;
                if (maxlen && (uint32_t)plen + 2 > maxlen) continue;
                if (L + 1 >= p.depth_cap || plen + 1 >= WMAXP) {
                    if (lane == 0) wset_err(p, FIM_E_STACK);
                    break;
                }
                if (lane == 0) s.path[plen] = citem;
                __syncwarp();
                // b_child = b_Y (level L of the stack) AND col(citem)
                const uint32_t *lv = stk + (int64_t)L * p.nwp_max;
                uint32_t *store = kc >= 2 ? stk + (int64_t)(L + 1) * p.nwp_max : nullptr;
                const int nFc = warp_class_pass(p, s, lv, wcol(s, citem), fi + bC, kc, plen + 1, store, fi + bC,
                                                fs + bC);
                if (lane == 0) {
                    s.nF[L + 1] = nFc;
                    s.cur[L + 1] = 0;
                    s.base[L + 2] = bC + nFc;
                }
                __syncwarp();
                L++;
            }
        }
        if (lane == 0) {
            s.n_roots_done += 1ull;
            busy += globaltimer_ns() - t_task;
        }
    }
    if (lane == 0) {
        if (s.n_roots_done) atomicAdd((unsigned long long *)&p.ctr->pending, 0ull - s.n_roots_done);
        if (s.n_classes) {
            atomicAdd(&p.ctr->supports_dfs, s.n_sup);
            atomicAdd(&p.ctr->dfs_words, s.n_words);
            atomicAdd(&p.ctr->dfs_bytes, s.n_bytes);
            atomicAdd(&p.ctr->dfs_touched, s.n_touched);
            atomicAdd(&p.ctr->classes, s.n_classes);
        }
        if (s.max_len) atomicMax(&p.ctr->max_len, s.max_len);
        atomicAdd(&p.ctr->busy_ns, busy);
        atomicMax(&p.ctr->t_last, globaltimer_ns());
    }
}

}  // namespace

// n_warps workers as CTAs of WW warps; ctas_per_sm (2 or 3) is the residency
// the registers are budgeted for: two CTAs an SM keep every candidate slice of
// a chunk in registers, three hold more workers and spill a little
int launch_dfs_warp(fim_ctx *ctx, const DfsParams &p, int n_warps, int ctas_per_sm, cudaStream_t st) {
    if (n_warps <= 0) return FIM_OK;
    ctx->launches++;
    const unsigned grid = (unsigned)ceil_div64(n_warps, WW);
    if (ctas_per_sm >= 3)
        dfs_warp_kernel<3><<<grid, WW * 32, 0, st>>>(p);
    else
        dfs_warp_kernel<2><<<grid, WW * 32, 0, st>>>(p);
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

int dfs_warp_max_depth() { return WMAXP - 2; }
int dfs_warp_per_cta() { return WW; }
