// k_dfs.cu -- recursive prefix extension (Section III: "the column AND
// operation can be performed in sequence" for higher-order itemsets; the
// threshold test of Eq. 3 prunes every infrequent extension).
//
// Persistent kernel: each CTA is one depth-first worker.  Work arrives as
// tickets from one global counter.  Tickets below n_roots are the frequent
// pairs {a, b} (root prefix classes); later tickets are slots of a device
// queue that workers fill with prefix classes they split off while other
// workers wait.  Every wait is bounded (FIM_E_TIMEOUT, never a hang).
//
// A prefix class is (prefix X, support S(X), candidates c_1 < ... < c_k), all
// candidates later than X's last item, each {x, c} frequent for x in X's last
// item (pair pruning).  One "pass" over the class computes, word by word,
//     b_X = AND of the class's sources (parent bitmap AND extension column)
//     S(X u {c}) = popc(b_X AND col(c))          for every candidate c
// with b_X held in registers (never re-read), candidate columns streamed from
// HBM with 128-bit loads, per-warp popc sums reduced by shuffles and combined
// in shared memory.  b_X is written to the worker's stack only when X can have
// grandchildren (k >= 2).  Frequent extensions become result records and the
// child list F; the worker then descends into F in order: child j gets the
// candidates {F_l : l > j, {F_j, F_l} frequent}.
#include "fim_common.cuh"

namespace {

constexpr int NT = 512;                  // threads per worker (CTA)
constexpr int NWARP = NT / 32;
constexpr int CB = 1024;                 // candidates per pass batch
constexpr int MAXSRC = FIM_TASK_MAXR + 1;
constexpr int MAXPATH = 256;             // longest itemset a worker tracks
constexpr int V = 2;                     // uint4 per lane per chunk (chunk = 256 words)
constexpr int CHUNK = 128 * V;

struct Smem {
    const uint32_t *src[MAXSRC];
    const uint32_t *cptr[CB];
    uint32_t sup[CB];
    uint32_t path[MAXPATH];
    int nF[MAXPATH];
    int cur[MAXPATH];
    long long base[MAXPATH + 1];
    uint32_t scan[NWARP + 1];
    int nsrc;
    uint32_t *store;
    unsigned long long ticket;
    unsigned long long rbase, ibase;
    int flag;
    int stop;
    int task_len;
    uint32_t task_sup;
    int ncand;
    long long cand_off;
};

// Block-wide exclusive scan of v (0/1 or small counts).  Returns the prefix;
// *total receives the sum.  All threads must call it.
__device__ __forceinline__ uint32_t block_scan(Smem &s, uint32_t v, uint32_t *total) {
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

__device__ __forceinline__ bool pairbit(const DfsParams &p, uint32_t a, uint32_t b) {
    return (__ldg(p.pairbits + (int64_t)a * p.mpw + (b >> 5)) >> (b & 31)) & 1u;
}

__device__ __forceinline__ const uint32_t *column(const DfsParams &p, uint32_t item) {
    return p.bm + (int64_t)__ldg(p.perm + item) * p.nwp;
}

__device__ void set_err(const DfsParams &p, int code) { atomicCAS(&p.ctr->err, 0, code); }

// One pass over a class: candidates cand[0..k) (global, in the worker's frame
// pool), sources in s.src[0..nsrc), optional store of b_X.  Frequent
// candidates are written compacted (item, support) to fi/fs and emitted as
// records with prefix s.path[0..plen).  Returns |F| (same in all threads).
__device__ int class_pass(const DfsParams &p, Smem &s, const uint32_t *cand, int k, int plen,
                          uint32_t *fi, uint32_t *fs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nwp = p.nwp;
    const int nchunks = (int)((nwp + CHUNK - 1) / CHUNK);
    // warps = G candidate groups x (NWARP / G) chunk workers
    const int G = nchunks >= NWARP ? 1 : NWARP / nchunks;
    const int CW = NWARP / G;
    const int g = warp % G, cw = warp / G;
    const bool active = warp < G * CW;
    const int nsrc = s.nsrc;
    uint32_t *store = s.store;
    int nF = 0;

    for (int b0 = 0; b0 < k; b0 += CB) {
        const int kb = min(CB, k - b0);
        for (int c = threadIdx.x; c < kb; c += NT) {
            s.cptr[c] = column(p, cand[b0 + c]);
            s.sup[c] = 0;
        }
        __syncthreads();
        if (active) {
            for (int q = cw; q < nchunks; q += CW) {
                const int64_t base = (int64_t)q * CHUNK + lane * 4;
                uint4 x[V];
                bool ok[V];
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const int64_t pos = base + v * 128;
                    ok[v] = pos < nwp;
                    x[v] = make_uint4(0, 0, 0, 0);
                    if (ok[v]) {
                        x[v] = ld_cg_u4(s.src[0] + pos);
                        for (int r = 1; r < nsrc; r++) x[v] = and4(x[v], ld_cg_u4(s.src[r] + pos));
                        if (store && b0 == 0 && g == 0)
                            *reinterpret_cast<uint4 *>(store + pos) = x[v];
                    }
                }
                int c = g;
                for (; c + G < kb; c += 2 * G) {
                    const uint32_t *c0 = s.cptr[c], *c1 = s.cptr[c + G];
                    uint4 y0[V], y1[V];
#pragma unroll
                    for (int v = 0; v < V; v++) {
                        const int64_t pos = base + v * 128;
                        y0[v] = ok[v] ? ldg_u4(c0 + pos) : make_uint4(0, 0, 0, 0);
                        y1[v] = ok[v] ? ldg_u4(c1 + pos) : make_uint4(0, 0, 0, 0);
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
                        if (ok[v]) n0 += popc_and4(x[v], ldg_u4(c0 + pos));
                    }
                    n0 = warp_sum_u32(n0);
                    if (lane == 0 && n0) atomicAdd(&s.sup[c], n0);
                }
            }
        }
        __syncthreads();
        // compact the frequent candidates of this batch, in order
        for (int c0 = 0; c0 < kb; c0 += NT) {
            const int c = c0 + threadIdx.x;
            uint32_t item = 0, sup = 0, f = 0;
            if (c < kb) {
                item = cand[b0 + c];
                sup = s.sup[c];
                f = sup >= p.thr;
            }
            uint32_t tot;
            const uint32_t pos = block_scan(s, f, &tot);
            if (tot) {
                if (threadIdx.x == 0) {
                    s.rbase = atomicAdd(&p.ctr->n_records, (unsigned long long)tot);
                    s.ibase = atomicAdd(&p.ctr->n_rec_items, (unsigned long long)tot * (plen + 1));
                }
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
        atomicAdd(&p.ctr->supports_dfs, (unsigned long long)k);
        atomicAdd(&p.ctr->dfs_words, (unsigned long long)k * (unsigned long long)p.nw);
        atomicAdd(&p.ctr->dfs_bytes, 4ull * p.nw * ((unsigned long long)k + nsrc + (store ? 1 : 0)));
        atomicAdd(&p.ctr->classes, 1ull);
        if (nF > 0) atomicMax(&p.ctr->max_len, plen + 1);
    }
    return nF;
}

// Candidate list of the root class {a, b}: every c > b with {a,c} and {b,c}
// frequent, written ascending to out.  Returns the count (all threads).
__device__ int root_candidates(const DfsParams &p, Smem &s, uint32_t a, uint32_t b, uint32_t *out,
                               long long room) {
    const uint32_t *ra = p.pairbits + (int64_t)a * p.mpw;
    const uint32_t *rb = p.pairbits + (int64_t)b * p.mpw;
    int n = 0;
    const int w0 = (int)(b >> 5);  // the word holding b; keep only c > b there
    for (int wb = w0; wb < p.mpw; wb += NT) {
        const int w = wb + threadIdx.x;
        uint32_t bits = 0;
        if (w < p.mpw) {
            bits = __ldg(ra + w) & __ldg(rb + w);
            if (w == w0) bits &= 0xFFFFFFFEu << (b & 31);
        }
        uint32_t tot;
        uint32_t pos = block_scan(s, __popc(bits), &tot);
        if (n + (long long)tot > room) { if (threadIdx.x == 0) set_err(p, FIM_E_STACK); return -1; }
        while (bits) {
            const int bit = __ffs(bits) - 1;
            bits &= bits - 1;
            out[n + pos++] = (uint32_t)(w * 32 + bit);
        }
        n += (int)tot;
        __syncthreads();
    }
    return n;
}

__device__ bool queue_hungry(const DfsParams &p) {
    const unsigned long long t = *(volatile unsigned long long *)&p.ctr->ticket;
    const unsigned long long q = *(volatile unsigned long long *)&p.ctr->qtail;
    const unsigned long long r = *(volatile unsigned long long *)&p.ctr->n_roots;
    return t > r + q;
}

// Try to hand the child class (prefix s.path[0..plen) + item, candidates
// cand[0..k)) to the queue.  Returns true if it was published.
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
        atomicAdd((unsigned long long *)&p.ctr->pending, 1ull);
        atomicAdd(&p.ctr->pushed, 1ull);
        __threadfence();
        atomicExch(&t->ready, 1u);
    }
    __syncthreads();
    return true;
}

__global__ void __launch_bounds__(NT, 2)
dfs_kernel(const DfsParams p) {
    __shared__ Smem s;
    const int wid = blockIdx.x;
    uint32_t *fi = p.frame_items + (int64_t)wid * p.frame_pool;
    uint32_t *fs = p.frame_sups + (int64_t)wid * p.frame_pool;
    uint32_t *stk = p.stack_bits + (int64_t)wid * p.depth_cap * p.nwp;

    while (true) {
        // ---- get the next task ---------------------------------------
        if (threadIdx.x == 0) {
            s.flag = 0;
            const unsigned long long t = atomicAdd(&p.ctr->ticket, 1ull);
            const unsigned long long nr = *(volatile unsigned long long *)&p.ctr->n_roots;
            if (*(volatile int *)&p.ctr->err != 0) {
                // an error ends the mine: take no more work
            } else if (t < nr) {
                s.path[0] = p.root_a[t];
                s.path[1] = p.root_b[t];
                s.task_len = 2;
                s.task_sup = p.root_sup[t];
                s.ncand = -1;
                s.flag = 1;
            } else if (t - nr < p.task_cap) {
                Task *tk = p.tasks + (t - nr);
                unsigned long long spins = 0;
                const unsigned long long t_wait = globaltimer_ns();
                while (true) {
                    if (*(volatile uint32_t *)&tk->ready) {
                        __threadfence();
                        const int len = (int)*(volatile uint32_t *)&tk->len;
                        for (int q = 0; q < len; q++) s.path[q] = ((volatile uint32_t *)tk->items)[q];
                        s.task_len = len;
                        s.task_sup = *(volatile uint32_t *)&tk->support;
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
        }
        __syncthreads();
        if (!s.flag) break;

        // ---- level 0: the task's own class ---------------------------
        const int tlen = s.task_len;
        int k;
        if (s.ncand < 0) {
            k = root_candidates(p, s, s.path[0], s.path[1], fi, p.frame_pool);
        } else {
            k = s.ncand;
            if (k > p.frame_pool) { if (threadIdx.x == 0) set_err(p, FIM_E_STACK); k = -1; }
            else for (int c = threadIdx.x; c < k; c += NT) fi[c] = __ldcg(p.cand_pool + s.cand_off + c);
            __syncthreads();
        }
        const bool len_ok = p.maxlen == 0 || (uint32_t)tlen + 1 <= p.maxlen;
        if (k > 0 && len_ok) {
            if (threadIdx.x == 0) {
                for (int r = 0; r < tlen; r++) s.src[r] = column(p, s.path[r]);
                s.nsrc = tlen;
                s.store = k >= 2 ? stk : nullptr;
                s.base[0] = 0;
            }
            __syncthreads();
            // candidates live at fi[0..k); F_0 overwrites them in order
            int nF = class_pass(p, s, fi, k, tlen, fi, fs);
            if (threadIdx.x == 0) { s.nF[0] = nF; s.cur[0] = 0; s.base[1] = nF; }
            __syncthreads();
            int L = 0;
            while (L >= 0) {
                if (threadIdx.x == 0) s.stop = *(volatile int *)&p.ctr->err != 0;
                __syncthreads();
                if (s.stop) break;
                if (s.cur[L] >= s.nF[L]) { L--; continue; }
                const int j = s.cur[L];
                __syncthreads();
                if (threadIdx.x == 0) s.cur[L] = j + 1;
                const int plen = tlen + L;          // prefix length at level L
                const long long bL = s.base[L];
                const long long bC = s.base[L + 1]; // child's candidates go here
                const uint32_t citem = fi[bL + j];
                const uint32_t csup = fs[bL + j];
                // child candidates: later frequent siblings paired with citem
                int kc = 0;
                const int nFL = s.nF[L];
                bool overflow = false;
                for (int l0 = j + 1; l0 < nFL; l0 += NT) {
                    const int l = l0 + threadIdx.x;
                    uint32_t d = 0, f = 0;
                    if (l < nFL) { d = fi[bL + l]; f = pairbit(p, citem, d); }
                    uint32_t tot;
                    const uint32_t pos = block_scan(s, f, &tot);
                    if (bC + kc + (long long)tot > p.frame_pool) { overflow = true; break; }
                    if (f) fi[bC + kc + pos] = d;
                    kc += (int)tot;
                }
                if (overflow) { if (threadIdx.x == 0) set_err(p, FIM_E_STACK); break; }
                __syncthreads();
                if (kc == 0) continue;
                if (p.maxlen && (uint32_t)plen + 2 > p.maxlen) continue;
                if (plen + 1 <= p.split_depth && plen + 1 <= FIM_TASK_MAXR) {
                    if (threadIdx.x == 0) s.flag = queue_hungry(p);
                    __syncthreads();
                    if (s.flag && try_push(p, s, plen, citem, csup, fi + bC, kc)) continue;
                }
                if (L + 1 >= p.depth_cap || plen + 1 >= MAXPATH) {
                    if (threadIdx.x == 0) set_err(p, FIM_E_STACK);
                    break;
                }
                // descend: b_child = b_parent AND col(citem)
                if (threadIdx.x == 0) {
                    s.path[plen] = citem;
                    s.src[0] = stk + (int64_t)L * p.nwp;
                    s.src[1] = column(p, citem);
                    s.nsrc = 2;
                    s.store = kc >= 2 ? stk + (int64_t)(L + 1) * p.nwp : nullptr;
                }
                __syncthreads();
                nF = class_pass(p, s, fi + bC, kc, plen + 1, fi + bC, fs + bC);
                if (threadIdx.x == 0) {
                    s.nF[L + 1] = nF;
                    s.cur[L + 1] = 0;
                    s.base[L + 2] = bC + nF;
                }
                __syncthreads();
                L++;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd((unsigned long long *)&p.ctr->pending, (unsigned long long)(-1ll));
        }
    }
}

}  // namespace

int launch_dfs(fim_ctx *ctx, const DfsParams &p, int grid, int block) {
    (void)block;
    if (grid <= 0) return FIM_OK;
    ctx->launches++;
    dfs_kernel<<<grid, NT, 0, ctx->stream>>>(p);
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

int dfs_threads() { return NT; }
