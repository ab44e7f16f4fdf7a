/*
 * fim.h -- C ABI of the GB300 Boolean-matrix frequent-itemset miner.
 *
 * The miner follows Section III of "A Matrix Logic Approach to Efficient
 * Frequent Itemset Discovery in Large Data Sets" (arXiv 2412.19420):
 *   matrix construction (Eq. 1)  -> fim_build_bitmaps
 *   support calculation (Eq. 2) and frequent-itemset extraction with the
 *   threshold test (Eq. 3)       -> fim_mine
 *   the frequent itemsets        -> fim_fetch_results
 *
 * Conventions shared by every entry point
 *   - Every call returns an int status: FIM_OK (0) or a negative FIM_E_* code.
 *     No C++ exception crosses this boundary.  fim_strerror() names a code.
 *   - A fim_ctx is bound to one CUDA device and one stream.  It owns every
 *     device allocation it makes; fim_destroy() releases them.  A ctx is not
 *     thread-safe: calls on one ctx must not overlap.
 *   - Pointers are plain host or device pointers, as each call's flags say.
 *     The library never keeps a caller's pointer after a call returns.
 *     Device inputs must be complete when a call is made: the ctx stream does
 *     not wait for work queued on other streams.  Calls that return results
 *     synchronise the ctx stream before returning.
 *   - Item ids are the caller's ids in [0, n_items); transaction order is the
 *     caller's row order (row i of the CSR is transaction T_i).
 *   - Supports are exact integer counts.  Results are canonical: items
 *     ascending inside each set, sets ordered by size then lexicographically.
 */
#ifndef FIM_H
#define FIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FIM_OK 0
#define FIM_E_INVAL (-1)     /* bad argument: malformed CSR, item >= n_items, minsup 0, ... */
#define FIM_E_NOMEM (-2)     /* device or host allocation failed                           */
#define FIM_E_CUDA (-3)      /* a CUDA runtime call failed                                 */
#define FIM_E_TIMEOUT (-4)   /* a bounded device-side wait ran out; the ctx stays usable   */
#define FIM_E_STACK (-5)     /* DFS stack budget too small for the itemset depth           */
#define FIM_E_TOO_SMALL (-6) /* caller's output buffer too small; required sizes returned  */
#define FIM_E_STATE (-7)     /* call out of order (mine before build, fetch before mine)   */
#define FIM_E_NODEV (-8)     /* no CUDA device / device id out of range                    */
#define FIM_E_CHECK (-9)     /* a "debug_checks" invariant failed (an internal error)      */

/* ---- flags ------------------------------------------------------------- */
/* All flags share one bit space, so that fim_mine_batched can take input
 * location and mine flags together. */
/* fim_build_bitmaps / fim_mine_batched: where the CSR arrays live */
#define FIM_INPUT_HOST 0u
#define FIM_INPUT_DEVICE 0x100u
/* fim_build_bitmaps / fim_mine_batched: the CSR's element types.  Default
 * (wide): indptr int64_t[n_trans + 1], indices int32_t[nnz].  Compact:
 * indptr uint32_t[n_trans + 1], indices uint16_t[nnz] -- the same matrix in
 * 2 + 4 / (items per row) bytes per item instead of 4 + 8 / (items per row),
 * for inputs with nnz < 2^32 (every item id fits: FIM_MAX_ITEMS < 2^16). */
#define FIM_CSR_COMPACT 0x400u

/* fim_mine / fim_mine_batched */
#define FIM_STRICT 0x1u       /* frequent iff S(X) > minsup (Eq. 3 literally); default S(X) >= minsup */
#define FIM_LEARNED 0x2u      /* the loaded MLP steers split/order/representation (never counts)    */
#define FIM_PAIRS_POPC 0x4u   /* 2-itemset pass on CUDA cores (AND+popc) instead of tensor cores    */
#define FIM_TRACE 0x8u        /* record one trace row per prefix class (features, subtree work)     */
#define FIM_DIFFSET_RULE 0x10u/* choose bitmap/diffset per class by the closed-form size rule       */
#define FIM_NO_SPLIT 0x20u    /* process every subtree inside the worker that found it              */
#define FIM_MAXLEN(k) (((uint32_t)(k) & 0xffu) << 24) /* longest itemset reported; 0 = unbounded */

/* fim_fetch_results / fim_fetch_batched: where the output buffers live */
#define FIM_OUTPUT_HOST 0u
#define FIM_OUTPUT_DEVICE 0x200u

/* ---- limits ------------------------------------------------------------ */
#define FIM_MAX_ITEMS 65535      /* n_items per database                           */
#define FIM_MAX_TRANS 2147483647 /* n_trans per database (supports fit in uint32)  */

typedef struct fim_ctx fim_ctx;

/* Per-mine counters, filled by fim_get_stats after fim_mine. */
typedef struct {
    uint64_t n_trans, n_items, n_frequent_items, n_sets, max_len;
    uint64_t supports_singletons; /* S(I_k) computed: n_items                      */
    uint64_t supports_pairs;      /* S(I_a n I_b) computed: m'(m'-1)/2 (Eq. 2)     */
    uint64_t supports_dfs;        /* supports of >= 3-itemsets computed by the DFS  */
    uint64_t dfs_words;           /* 32-bit candidate words ANDed by the DFS        */
    uint64_t dfs_bytes;           /* bytes the DFS kernel read/wrote algorithmically */
    uint64_t dfs_touched_bytes;   /* the same, counting only 32-byte sectors that can
                                     contribute (zero prefix words are skipped)     */
    uint64_t classes;             /* prefix classes expanded                        */
    uint64_t tasks_pushed;        /* classes handed to the device work queue        */
    uint64_t diffset_classes;     /* classes counted through a diffset              */
    uint64_t peak_device_bytes;   /* device memory held by the ctx                  */
    uint64_t launches_build;      /* kernels launched by the last fim_build_bitmaps */
    uint64_t launches_mine;       /* kernels launched by the last fim_mine          */
    uint64_t dfs_busy_ns;         /* DFS workers' time inside tasks, summed         */
    uint64_t dfs_span_ns;         /* first worker start to last worker exit         */
    uint64_t dfs_workers;         /* DFS workers (CTAs) of the launch               */
    uint64_t dfs_root_ns;         /* part of dfs_busy_ns spent in the root classes'
                                     own passes (candidate list + level-0 pass)     */
    float ms_build, ms_singletons, ms_pairs, ms_dfs, ms_compact; /* CUDA-event times */
    uint32_t pair_path;           /* 1 = tcgen05 tensor cores, 0 = CUDA-core popc   */
    uint32_t reserved;
} fim_stats;

/* One database of a batch (fim_mine_batched).  CSR as for fim_build_bitmaps;
 * the batch's flags say whether every database's arrays are wide or compact. */
typedef struct {
    const void *indptr;      /* [n_trans + 1]: int64_t, or uint32_t if FIM_CSR_COMPACT */
    const void *indices;     /* [indptr[n_trans]]: int32_t, or uint16_t if FIM_CSR_COMPACT */
    int64_t n_trans;
    int32_t n_items;
    int32_t pad;
    uint64_t minsup;         /* absolute count, >= 1 */
} fim_db_desc;

/* fim_create: make a context on `device` (CUDA ordinal).  `cuda_stream` is a
 * cudaStream_t to run on, or NULL for a stream the ctx creates and owns.
 * Errors: FIM_E_NODEV, FIM_E_CUDA, FIM_E_NOMEM, FIM_E_INVAL (out == NULL). */
int fim_create(fim_ctx **out, int device, void *cuda_stream);

/* fim_destroy: free every device and host allocation of the ctx (NULL ok). */
void fim_destroy(fim_ctx *ctx);

/* fim_build_bitmaps -- matrix construction, Eq. 1 (Section III):
 * M[i,j] = 1 iff item j occurs in transaction i.  The CSR gives transaction i
 * as indices[indptr[i] : indptr[i+1]]; repeated items inside a transaction
 * collapse (set membership), empty transactions are allowed and count toward
 * n_trans.  Input arrays are host pointers (FIM_INPUT_HOST) or device pointers
 * (FIM_INPUT_DEVICE), wide or compact (FIM_CSR_COMPACT: the element types
 * above); they are copied and may be freed when the call returns.
 * The ctx keeps the matrix as item-major bit columns: column j is
 * ceil(n_trans/32) uint32 words, bit (i mod 32) of word i/32 = M[i,j].
 * Errors: FIM_E_INVAL if indptr[0] != 0, indptr decreases, an item is outside
 * [0, n_items), n_items > FIM_MAX_ITEMS or n_trans > FIM_MAX_TRANS (the ctx
 * then holds no matrix); FIM_E_NOMEM; FIM_E_CUDA. */
int fim_build_bitmaps(fim_ctx *ctx, const void *indptr, const void *indices,
                      int64_t n_trans, int32_t n_items, uint32_t flags);

/* fim_mine -- support calculation and frequent-itemset extraction
 * (Eq. 2 generalised to any itemset by sequential column AND; Eq. 3):
 * finds every non-empty X with S(X) >= minsup (or S(X) > minsup under
 * FIM_STRICT), S(X) = popcount of the AND of X's bit columns.  Singletons by
 * column popcount, pairs by the A^T A contraction on tensor cores, larger sets
 * by a persistent depth-first prefix-extension kernel.  The result replaces
 * any earlier one held by the ctx.  Requires a prior fim_build_bitmaps.
 * Errors: FIM_E_STATE (no matrix), FIM_E_INVAL (minsup == 0 without
 * FIM_STRICT), FIM_E_NOMEM, FIM_E_TIMEOUT, FIM_E_CUDA. */
int fim_mine(fim_ctx *ctx, uint64_t minsup, uint32_t flags);

/* fim_fetch_results -- the frequent itemsets of the last fim_mine, canonical.
 * Always writes *n_sets and *n_items_total (sum of set sizes).  If offsets,
 * items and supports are all NULL it only reports the sizes.  Otherwise
 * offsets gets n_sets+1 entries (set q is items[offsets[q] : offsets[q+1]]),
 * items gets the caller's item ids, supports the exact counts; cap_sets and
 * cap_items give the capacities of supports/offsets-1 and items.
 * flags: FIM_OUTPUT_HOST (host buffers) or FIM_OUTPUT_DEVICE (device buffers).
 * Errors: FIM_E_STATE (nothing mined), FIM_E_TOO_SMALL (sizes still written),
 * FIM_E_INVAL, FIM_E_CUDA. */
int fim_fetch_results(fim_ctx *ctx, uint64_t *n_sets, uint64_t *n_items_total,
                      uint64_t *offsets, uint32_t *items, uint32_t *supports,
                      uint64_t cap_sets, uint64_t cap_items, uint32_t flags);

/* fim_get_stats: counters and phase times of the last fim_mine (or batch).
 * After fim_mine_batched the phases are those of the batch's graph: ms_build
 * covers the build with its fused singleton supports and the ranking
 * (ms_singletons is 0), ms_pairs the pair pass with its threshold, ms_dfs
 * the prefix extension, ms_compact the compaction after the graph. */
int fim_get_stats(const fim_ctx *ctx, fim_stats *out);

/* fim_set_tuning -- set one launch-shape parameter of the ctx; it applies to
 * later calls and never changes results.  Keys and ranges:
 *   "dfs_threads"      256, 512  threads of one DFS worker (CTA)
 *   "dfs_ctas_per_sm"  1..4      DFS workers per SM; dfs_threads x dfs_ctas_per_sm
 *                                must not exceed 1024 (FIM_E_INVAL otherwise)
 *   "split_depth"      0..8      longest prefix a worker may hand to the queue
 *   "root_reverse"     0, 1      hand out the root classes (frequent pairs) in
 *                                reverse order: pairs of the most frequent items
 *                                first (default 0)
 *   "learned_order"    0, 1      FIM_LEARNED also hands out the roots longest-
 *                                predicted-subtree first (default 0)
 *   "root_sort"        0, 1      without the network's order, hand out the roots
 *                                as the pair pass lists them (0) or most
 *                                candidates first (1, default).  Either way a root whose
 *                                class has no candidate is dropped before the
 *                                prefix extension starts
 *   "batch_segments"   0..16     fim_mine_batched pipelines this many groups of
 *                                databases (about equal transactions): a group's
 *                                pair pass runs while the next group is built;
 *                                0 (default) = eight groups for page-locked host
 *                                input (uploaded group by group, or read in place
 *                                by a build of one CTA per SM), else one
 *   "dfs_warp"         0, 1      fim_mine_batched with every database's columns at
 *                                most 4,096 words: one warp per prefix-extension
 *                                worker instead of one CTA (default 1)
 *   "dfs_warp_ctas"    2, 3      CTAs of eight such warp workers per SM (default 2)
 *   "record_chunk"     1..1024   result slots a prefix-extension worker reserves
 *                                at a time (default 1: exactly a class's sets);
 *                                the ones a worker leaves unused are sorted out
 *                                by the compaction
 *   "learned_kmin"     1..2^20   FIM_LEARNED consults the network only for classes
 *                                with at least this many candidates (default 8;
 *                                smaller ones are counted dense)
 *   "sparse_div"       -1..64    a class bitmap b_Y is kept as its non-zero words
 *                                when S(Y) x sparse_div <= nw (0 = always dense;
 *                                -1 = automatic, the default: 4 when the frequent
 *                                item columns exceed half of L2, else dense)
 *   "pairs_split"      0..4096   CTAs of the tensor-core pair pass, each taking an
 *                                equal share of the (tile, stage) space (0 = one per SM)
 *   "pairs_kdrain"     0..32768  128-transaction stages one accumulator sums before
 *                                it is drained (0 = 32768: partial sums stay <= 2^24,
 *                                exact in f32)
 *   "debug_checks"     0, 1      after fim_build_bitmaps, check on the device that
 *                                every pad bit and pad word of the columns is zero;
 *                                after fim_mine, that the output is canonical (sets
 *                                non-empty, items strictly ascending and < n_items,
 *                                supports at the threshold, sets strictly increasing
 *                                in (size, items) order); FIM_E_CHECK otherwise
 *                                (default 0)
 *   "spin_limit_ms"    1..600000 longest a device-side wait (the DFS work queue)
 *                                spins before the mine ends with FIM_E_TIMEOUT
 *                                (default 60000); the ctx stays usable
 *   "test_withhold_task" -1..2^20 fault injection for tests: the DFS never
 *                                publishes this work-queue slot, so the worker
 *                                that takes it (and the drain) must time out;
 *                                -1 (default) = off
 *   "upload_mapped"    0, 1      host input to fim_build_bitmaps and
 *                                fim_mine_batched that lives in page-locked, mapped
 *                                memory (cudaHostAlloc, cudaHostRegister) is read
 *                                by the build kernel in place over the host link,
 *                                without a staging copy (default 1; other host
 *                                memory is copied; a batch counts as page-locked
 *                                when its arrays form at most 64 contiguous runs,
 *                                each inside one such allocation)
 *   "batch_stream_copies" 0, 1   a page-locked host batch (as above) goes up by
 *                                copies of database groups inside the batch's
 *                                graph, each group's build starting when its copy
 *                                lands, beside the later groups' uploads (default
 *                                1); 0 = the build reads it in place
 *   "upload_chunks"    1..16     host input to fim_build_bitmaps: the indices go
 *                                up in this many chunks, each built as soon as it
 *                                lands (default 4; 1 = one copy, then the build)
 *   "upload_streams"   1, 2      copy streams the chunks alternate over (default 2)
 *   "compact_cluster"  0, 1      sort outputs small enough for one thread-block
 *                                cluster's shared memory in one launch (default 1)
 *   "batch_pairs_shape" 0..6     launch shape of fim_mine_batched's tensor-core
 *                                pair pass: (operand stages in the ring, stages of
 *                                raw bits staged ahead, CTAs per SM, stages per
 *                                producer fence) = 0 (8, 8, 1, 2), 1 (6, 8, 1, 2),
 *                                2 (8, 16, 1, 2), 3 (4, 8, 1, 2), 4 (7, 12, 1, 2),
 *                                5 (8, 8, 1, 4), 6 (8, 16, 1, 4); default 0
 *   "batch_build_block" 16, 32, 64  words of every column one CTA of
 *                                fim_mine_batched's build covers (32 x that many
 *                                transactions); a block that does not fit shared
 *                                memory falls back to the next smaller (default 32)
 *   "batch_pairs_pack" 0, 1      fim_mine_batched's tensor-core pair pass: its units
 *                                are planned on the device once m' is known, and two
 *                                databases with at most 64 frequent items (and about
 *                                as many transactions) share one 128 x 128 tile
 *                                (default 1); 0 = a tile per database
 *   "batch_group_dfs"  0, 1      fim_mine_batched with pipelined groups (more than
 *                                one): each group's root classes are planned and
 *                                mined (warp workers) right after its pair pass,
 *                                beside the later groups' uploads and builds
 *                                (default 1); 0 = one prefix extension after all
 *                                groups
 *   "batch_build_coal" 0, 1      fim_mine_batched's build: a warp reads its 32
 *                                rows' item ids 32 at a time (coalesced) and finds
 *                                each id's row among the lanes; 0 = lane-per-row
 *                                reads (default 1)
 * Errors: FIM_E_INVAL for an unknown key or an out-of-range value. */
int fim_set_tuning(fim_ctx *ctx, const char *key, int64_t value);

/* fim_mine_batched -- many independent databases in one persistent launch,
 * replayed from a captured CUDA graph when the same batch shape repeats.
 * dbs[d] describes database d (host or device CSR per flags &
 * FIM_INPUT_DEVICE); each is mined with its own dbs[d].minsup exactly as
 * fim_build_bitmaps + fim_mine would.  Results are fetched per database with
 * fim_fetch_batched.  Errors as fim_build_bitmaps and fim_mine, for any d. */
int fim_mine_batched(fim_ctx *ctx, int n_db, const fim_db_desc *dbs, uint32_t flags);

/* fim_fetch_batched -- results of database `db` of the last batch, with the
 * same contract as fim_fetch_results.  db = FIM_ALL_DBS returns every
 * database's results in one stream (sorted by database, then canonically),
 * offsets counted from the start of that stream; fim_batch_slices tells
 * where each database's sets begin. */
#define FIM_ALL_DBS (-1)
int fim_fetch_batched(fim_ctx *ctx, int db, uint64_t *n_sets, uint64_t *n_items_total,
                      uint64_t *offsets, uint32_t *items, uint32_t *supports,
                      uint64_t cap_sets, uint64_t cap_items, uint32_t flags);

/* fim_batch_slices: set_start[n_db + 1] (host) -- database d's sets are
 * set_start[d] .. set_start[d+1] - 1 of the FIM_ALL_DBS stream.
 * Errors: FIM_E_STATE (no batch mined), FIM_E_TOO_SMALL (cap < n_db + 1). */
int fim_batch_slices(fim_ctx *ctx, uint64_t *set_start, uint64_t cap);

/* ---- learned scheduler (8 -> 64 -> 64 -> 2 bf16 MLP) --------------------
 * The network predicts, per prefix class, log2(1 + subtree work) and the
 * logit of storing the class as a diffset.  It only steers scheduling and
 * representation; supports are always counted exactly.  The paper names an
 * adaptive, data-dependent choice of Boolean operation sequence and deep
 * models as directions (Sections I and V) without specifying a network.
 * Weight layout (float32, 4,866 values): W1[64][8], b1[64], W2[64][64],
 * b2[64], W3[2][64], b3[2]. */
#define FIM_MLP_PARAMS 4866
#define FIM_MLP_FEATURES 8

/* fim_sched_load_weights: copy host float32 weights into the ctx (bf16 for
 * inference).  Errors: FIM_E_INVAL if n_params != FIM_MLP_PARAMS. */
int fim_sched_load_weights(fim_ctx *ctx, const float *weights, size_t n_params);

/* fim_fetch_traces: trace rows of the last fim_mine run with FIM_TRACE.
 * features [n][8] and targets [n][2] (log2(1+subtree words), diffset label)
 * are host float32 buffers of capacity cap rows, or NULL to query *n_rows.
 * Errors: FIM_E_STATE, FIM_E_TOO_SMALL. */
int fim_fetch_traces(fim_ctx *ctx, uint64_t *n_rows, float *features, float *targets,
                     uint64_t cap);

/* fim_mlp_forward: y[B][2] = MLP(x[B][8]) with params[4866] (all DEVICE
 * float32 pointers).  bf16 != 0 rounds weights and activations to bf16 with
 * float32 accumulation (the inference precision); 0 computes in float32.
 * cache (device, B*(64+64+64+64) floats) keeps pre-activations for backward,
 * or NULL.  Runs on the ctx stream.  Errors: FIM_E_INVAL, FIM_E_CUDA. */
int fim_mlp_forward(fim_ctx *ctx, const float *params, const float *x, int64_t B,
                    float *y, float *cache, int bf16);

/* fim_mlp_backward: grad[4866] (device) = d loss / d params for the loss
 * mean_b[0.5 (y0-t0)^2 + softplus(y1) - t1 y1], from x, y, t (device) and
 * the cache of fim_mlp_forward with the same params.  Returns the loss in
 * *loss_out (host) when non-NULL.  Errors: FIM_E_INVAL, FIM_E_CUDA. */
int fim_mlp_backward(fim_ctx *ctx, const float *params, const float *x, const float *y,
                     const float *t, const float *cache, int64_t B, float *grad,
                     float *loss_out, int bf16);

/* fim_mlp_adam: one Adam step (bias-corrected, step counts from 1) on device
 * arrays params/m/v from grad.  Errors: FIM_E_INVAL, FIM_E_CUDA. */
int fim_mlp_adam(fim_ctx *ctx, float *params, const float *grad, float *m, float *v,
                 int step, float lr, float beta1, float beta2, float eps);

/* ---- one mine split over several GPUs ------------------------------------
 * The paper's decomposition of the matrix into parts mined separately and
 * merged (Section II), in the form that needs no communication during the
 * mine: after the pair pass, every frequent pair {a, b} (a < b in the
 * miner's internal item order) roots a prefix class holding the frequent sets
 * whose two smallest items are a and b; these classes partition the sets of
 * size >= 3.
 *
 * fim_mine_shard: fim_mine restricted to shard `shard` of n_shards (1 <=
 * n_shards <= FIM_MAX_SHARDS).  Every shard builds the same matrix and runs
 * the singleton and pair passes in full; the root classes, numbered in (a, b)
 * order, are dealt round-robin (class P to shard P mod n_shards), which every
 * shard derives identically from the pair bitsets, and the shard mines only
 * its own classes.  Shard 0 also
 * reports the frequent singletons and pairs.  The held output (canonical,
 * fetched with fim_fetch_results) is the shard's part: the parts of shards
 * 0 .. n_shards-1 are disjoint and their union is fim_mine's answer.
 * n_shards == 1 is fim_mine.  Errors: as fim_mine; FIM_E_INVAL for a shard
 * outside [0, n_shards) or n_shards outside [1, FIM_MAX_SHARDS]. */
#define FIM_MAX_SHARDS 1024
int fim_mine_shard(fim_ctx *ctx, uint64_t minsup, uint32_t flags, int shard, int n_shards);

/* fim_merge_results: replaces the ctx's held itemsets with the canonical
 * union of n_parts disjoint canonical lists -- the fim_fetch_results outputs
 * of the shards of one database.  Part p has n_sets[p] sets and
 * n_items_total[p] items: offsets[p] (n_sets[p] + 1 entries, first 0, last
 * n_items_total[p]), items[p] (the caller's ids, < n_items), supports[p].  All
 * arrays are host pointers (FIM_INPUT_HOST) or device pointers of the ctx's
 * GPU (FIM_INPUT_DEVICE); they are copied and may be freed on return.
 * n_trans is the database's transaction count (the n of lift in fim_rules).
 * The result is fetched with fim_fetch_results and feeds fim_rules, like a
 * mine's; fim_get_stats then reports the merge's n_sets, max_len,
 * ms_compact and launches_mine.  Parts that overlap give duplicate sets: the
 * call does not check.
 * Errors: FIM_E_INVAL (a NULL array, malformed offsets, a set longer than 255
 * items, an item >= n_items, n_trans or n_items out of range), FIM_E_NOMEM,
 * FIM_E_CUDA. */
int fim_merge_results(fim_ctx *ctx, int64_t n_trans, int32_t n_items, int n_parts,
                      const uint64_t *n_sets, const uint64_t *n_items_total,
                      const uint64_t *const *offsets, const uint32_t *const *items,
                      const uint32_t *const *supports, uint32_t flags);

/* ---- association rules -------------------------------------------------
 * Section IV.A names confidence and lift beside support as the measures the
 * mined itemsets are evaluated with; the paper prints no formula, so these
 * are the textbook ones.  For a frequent set Z, a nonempty proper subset X of
 * Z and Y = Z \ X, the rule X -> Y has
 *     conf(X -> Y) = S(Z) / S(X)
 *     lift(X -> Y) = conf(X -> Y) / (S(Y) / n) = S(Z) n / (S(X) S(Y))
 * with S the supports of Eq. 3 and n the transactions.
 *
 * fim_rules: from the itemsets held by the last fim_mine, builds on the device
 * every rule X -> Y with 2 <= |Z| <= max_len (0 = FIM_RULES_MAX_LEN) and
 * conf >= min_conf_ppm / 10^6, decided in integers: S(Z) * 10^6 >= min_conf_ppm
 * * S(X).  Rules are ordered by the index of Z in the canonical output, then by
 * ante_mask ascending; ante_mask bit i set means the i-th item of Z (its items
 * ascending) is in X, the others form Y.  conf is the double S(Z) / S(X); lift
 * is the double (S(Z) n) / (S(X) S(Y)) of the two exact integer products, each
 * rounded once to double, so results are reproducible bit for bit.  Sets
 * longer than max_len yield no rules (a set of size L has 2^L - 2 of them).
 * The rules stay in device memory of the ctx until the next fim_rules or
 * fim_mine; *n_rules gets their number.  Scratch: 8 bytes per held set and
 * 12 bytes per 32 candidate rules (sum of 2^|Z| - 2), plus 12 bytes per
 * candidate when there are at most 2^27 of them.
 * Errors: FIM_E_STATE (no fim_mine result held, or the held sets are not
 * downward closed), FIM_E_INVAL (min_conf_ppm > 10^6, max_len outside
 * {0} u [2, FIM_RULES_MAX_LEN], n_rules NULL), FIM_E_NOMEM (also when the
 * candidate rules' scratch does not fit), FIM_E_CUDA. */
#define FIM_RULES_MAX_LEN 20
int fim_rules(fim_ctx *ctx, uint32_t min_conf_ppm, int max_len, uint64_t *n_rules);

/* fim_rules_evaluated: the candidate rules the last fim_rules tested,
 * sum over the sets Z it covered of 2^|Z| - 2.  Errors as fim_fetch_rules. */
int fim_rules_evaluated(const fim_ctx *ctx, uint64_t *n_evaluated);

/* fim_fetch_rules: copies the rules of the last fim_rules (for the itemsets
 * still held) into caller buffers of cap entries each: set_index (uint64, the
 * index of Z in fim_fetch_results' order), ante_mask, conf, lift.  With all
 * four NULL it only writes *n_rules.  flags: FIM_OUTPUT_HOST or
 * FIM_OUTPUT_DEVICE.  Errors: FIM_E_STATE (no rules for the held itemsets),
 * FIM_E_TOO_SMALL (cap < *n_rules, which is still written), FIM_E_INVAL (some
 * but not all buffers NULL), FIM_E_CUDA. */
int fim_fetch_rules(fim_ctx *ctx, uint64_t *n_rules, uint64_t *set_index, uint32_t *ante_mask,
                    double *conf, double *lift, uint64_t cap, uint32_t flags);

/* ---- allocation-free entry point ---------------------------------------
 * The paper has no counterpart to this call.  It serves callers that cannot
 * allocate device memory while they use the library: processes whose own
 * memory pool owns every device byte and forbids allocations outside it, and
 * latency-critical paths that must not block in cudaMalloc/cudaFree (which
 * can synchronise the whole device).
 *
 * fim_pair_supports_noalloc: for the database given as a DEVICE CSR
 * (d_indptr[n_trans + 1], d_indices[d_indptr[n_trans]]), fills the
 * caller-owned DEVICE matrix d_pair_counts (uint32, n_items x n_items,
 * row-major): entry [a][b], a < b, is the pair support S(I_a n I_b) of Eq. 2,
 * entry [a][a] is S(I_a), entries below the diagonal are 0 -- the singleton
 * and pair supports fim_mine computes, without a threshold.  It runs on
 * cuda_stream (a cudaStream_t, NULL = the legacy default stream) of the
 * current device and returns when the work has finished: it synchronises
 * that stream twice (to read the CSR's element count d_indptr[n_trans], and
 * the validation flag), so it blocks the calling thread.
 * Memory: it calls no cudaMalloc, cudaFree or allocating library routine.
 * Its only scratch is a static device array of FIM_NOALLOC_MAX_BYTES that
 * every GPU which loads libfim holds until the process exits; the bit columns
 * of a database need n_items * 128 * ceil(n_trans / 1024) bytes of it.  The
 * first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture begins.  All calls share the array, which keeps the last call's
 * contents; each call rewrites every part of it that it reads, and clears the
 * output itself.  Calls whose GPU work overlaps (several streams or host
 * threads) race on the array and must be serialised by the caller.
 * Errors: FIM_E_INVAL for n_items > FIM_MAX_ITEMS or bit columns larger
 * than FIM_NOALLOC_MAX_BYTES (nothing is launched then), and for a malformed
 * CSR (indptr decreasing or outside [0, nnz], an item outside [0, n_items)),
 * which the counting kernels detect while they run: d_pair_counts then holds
 * no meaningful values, and the next call starts afresh; FIM_E_NODEV;
 * FIM_E_CUDA. */
#define FIM_NOALLOC_MAX_BYTES (64u << 20)
int fim_pair_supports_noalloc(const int64_t *d_indptr, const int32_t *d_indices, int64_t n_trans,
                              int32_t n_items, uint32_t *d_pair_counts, void *cuda_stream);

/* fim_probe: measurement probes for the counting kernels' rooflines, run on
 * the ctx's GPU and stream (two short launches, the second timed).
 *   which = 0: AND/popc word pairs per second over all SMs -- one LOP3, one
 *              POPC and one IADD per pair, the inner step of the pair and
 *              prefix-extension passes;
 *   which = 1: L2 read bandwidth in GB/s, 16-byte loads over a 32 MB buffer;
 *   which = 2: dense tcgen05 kind::f8f6f4 rate in TFLOP/s (e4m3 operands,
 *              f32 accumulator in tensor memory), in the pair pass's
 *              instruction shape 128 x 256 x 32 with A read from tensor
 *              memory: one CTA per SM, one thread issuing MMAs back to back;
 *   which = 3: the same with A read from shared memory;
 *   which = 4, 5: A from shared memory, N = 128 and N = 64 (the batched
 *              pair pass's tile widths for databases with few frequent items).
 * Errors: FIM_E_INVAL (unknown probe, result NULL), FIM_E_NOMEM, FIM_E_CUDA,
 * FIM_E_TIMEOUT (the MMA probe's bounded wait ran out). */
int fim_probe(fim_ctx *ctx, int which, double *result);

/* fim_minsup_from_ppm: ceil(n_trans * ppm / 1e6) in integers, at least 1:
 * the threshold of Eq. 3 given as a fraction of the transactions. */
uint64_t fim_minsup_from_ppm(int64_t n_trans, uint32_t ppm);

/* fim_strerror: static description of a status code. */
const char *fim_strerror(int status);

/* fim_version: ABI version (major << 16 | minor). */
uint32_t fim_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FIM_H */
