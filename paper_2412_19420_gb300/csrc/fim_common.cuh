// fim_common.cuh -- internal declarations shared by the miner's .cu files.
//
// Data layout in device memory (one database):
//   bm        uint32 [m][nwp]   item-major bit columns (Eq. 1): bit (i % 32) of
//                               word i / 32 of column j is M[i, j]; nwp = words per
//                               column padded to a multiple of 128 (512 B); pad
//                               bits and pad words are 0.
//   item_sup  uint32 [m]        S(I_j), column popcount (Eq. 3 aggregation)
//   perm      int32  [m']       internal id -> caller's item id.  Internal ids
//                               order the frequent items by (support, id) ascending.
//   pair_cnt  int32  [m'][m']   S(I_a n I_b) for a < b (Eq. 2), upper triangle
//   pairbits  uint32 [m'][mpw]  bit b of row a set iff a < b and {a,b} frequent
//   records   (off u64, len u32, sup u32) per frequent itemset + an item pool
//                               of internal ids; the compactor turns them into the
//                               canonical (offsets, items, supports) output.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include <utility>
#include <vector>

#include "../../include/fim.h"

#include <nvtx3/nvToolsExt.h>

// An NVTX range around an ABI call, visible to Nsight tools when one is
// attached (the header-only NVTX v3 API: no cost without a tool).
struct FimNvtxRange {
    explicit FimNvtxRange(const char *name) { nvtxRangePushA(name); }
    ~FimNvtxRange() { nvtxRangePop(); }
    FimNvtxRange(const FimNvtxRange &) = delete;
    FimNvtxRange &operator=(const FimNvtxRange &) = delete;
};
#define FIM_NVTX(name) FimNvtxRange fim_nvtx_range_(name)

#define FIM_WORDS_ALIGN 128  // column padding, in 32-bit words (512 bytes)

// ---------------------------------------------------------------- utilities
#define FIM_CUDA_TRY(expr)                                        \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) {                                  \
            fim_set_cuda_error(_e, #expr, __FILE__, __LINE__);    \
            return (_e == cudaErrorMemoryAllocation) ? FIM_E_NOMEM : FIM_E_CUDA; \
        }                                                         \
    } while (0)

#define FIM_TRY(expr)            \
    do {                         \
        int _r = (expr);         \
        if (_r != FIM_OK) return _r; \
    } while (0)

void fim_set_cuda_error(cudaError_t e, const char *what, const char *file, int line);

static inline int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }
static inline int64_t round_up64(int64_t a, int64_t b) { return ceil_div64(a, b) * b; }

// A grow-only device buffer owned by a ctx.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Device-side counters of one mine (kept in one small struct so a single
// memset clears them and a single copy reads them back).
struct MineCounters {
    unsigned long long n_records;    // frequent itemsets emitted
    unsigned long long n_rec_items;  // items emitted into the record pool
    unsigned long long supports_dfs; // supports evaluated by the DFS
    unsigned long long dfs_words;    // candidate words ANDed by the DFS
    unsigned long long dfs_bytes;    // algorithmic bytes moved by the DFS (dense operands)
    unsigned long long dfs_touched;  // bytes of the 32-byte sectors that can contribute
    unsigned long long classes;      // classes expanded
    unsigned long long pushed;       // tasks pushed to the queue
    unsigned long long diffset;      // classes counted via a diffset
    unsigned long long ticket;       // next work ticket
    unsigned long long qtail;        // next free queue slot
    unsigned long long pool_top;     // next free word of the candidate pool
    unsigned long long n_roots;      // frequent pairs (root classes)
    unsigned long long n_traces;     // trace rows written
    unsigned long long busy_ns;      // DFS workers' time inside tasks, summed
    unsigned long long t_first;      // DFS kernel span (%globaltimer): first start ...
    unsigned long long t_last;       // ... and last worker exit
    unsigned long long root_ns;      // workers' time in root classes' own passes, summed
    long long pending;               // tasks pushed but not finished
    int err;                         // FIM_OK or a FIM_E_* from the device
    int overflow;                    // bit 0 records, bit 1 items, bit 2 traces
    int max_len;                     // longest itemset emitted
    int m_freq;                      // m' (frequent items)
    int max_row_freq;                // most frequent items in one transaction
    int pad[3];
    // DFS workers reserve record and item slots in chunks; the slots a
    // worker leaves unused are holes (records of length 0, items nobody
    // references), left out of the canonical output
    unsigned long long rec_holes;
    unsigned long long item_holes;
};

// A pushed prefix class: items (internal ids) + support + candidate list.
#define FIM_TASK_MAXR 8  // longest prefix a queued task may carry
struct Task {
    uint32_t items[FIM_TASK_MAXR];
    uint32_t len;
    uint32_t support;
    uint32_t n_cand;
    uint32_t ready;            // epoch of the mine that published the slot
    unsigned long long cand_off;  // into the candidate pool
    float prio;                // predicted work (learned mode) or 0
    uint32_t db;               // database of the class
};

// One database of a mine: its CSR, sizes, and its offsets into the
// mine-wide arrays (bit columns, item supports / ranks / perm, pair counts,
// pair bitset).  fim_mine uses a one-entry table; fim_mine_batched one entry
// per database.  mfreq is written on the device by the ranking kernel.
struct DbDesc {
    const void *indptr;  // int64_t[n + 1], or uint32_t[n + 1] when compact
    const void *indices; // int32_t[nnz], or uint16_t[nnz] when compact
    int64_t n, nw, nwp;
    int64_t bm_off;      // words into the bit-column array
    int64_t item_off;    // entries into item_sup / rank / perm
    int64_t pair_off;    // entries into pair_cnt (m * m)
    int64_t pb_off;      // words into pairbits (m * ceil(m / 32))
    int32_t m;
    int32_t mfreq;
    uint32_t thr;
    uint32_t maxlen;
    int32_t compact;     // 1: the CSR is compact (FIM_CSR_COMPACT)
    int32_t pad;
};

// A CSR's row offset i and item id e, wide (int64 offsets, int32 ids) or
// compact (uint32 offsets, uint16 ids).
__host__ __device__ __forceinline__ int64_t csr_off(const void *indptr, bool compact, int64_t i) {
    return compact ? (int64_t) static_cast<const uint32_t *>(indptr)[i] : static_cast<const int64_t *>(indptr)[i];
}
#ifdef __CUDACC__
__device__ __forceinline__ int32_t csr_id(const void *indices, bool compact, int64_t e) {
    return compact ? (int32_t)__ldg(static_cast<const unsigned short *>(indices) + e)
                   : __ldg(static_cast<const int32_t *>(indices) + e);
}
#endif
inline size_t csr_off_bytes(bool compact) { return compact ? sizeof(uint32_t) : sizeof(int64_t); }
inline size_t csr_id_bytes(bool compact) { return compact ? sizeof(uint16_t) : sizeof(int32_t); }

// A window of the root arrays: the roots one group of a batch's databases
// appended (base, count), the part its root plan kept (kept, in
// root_order[base ..]) and the ticket counter of the prefix extension over
// them.
struct RootWindow {
    unsigned long long base, count, kept, ticket;
};

// One frame of a worker's DFS stack lives in global memory.
struct DfsParams {
    // mine-wide arrays; a database's part starts at its DbDesc offsets
    const DbDesc *dbs;
    const uint32_t *bm;
    const int32_t *perm;
    const uint32_t *pairbits;
    const int *pair_cnt;        // S({a,b}) for a < b, [m][m] per database
    const uint32_t *item_sup;   // S({j}) by caller id
    int64_t nwp_max;            // stack level stride (largest nwp of the mine)
    // roots: frequent pairs, visited in root_order (or index order if null)
    const uint32_t *root_a, *root_b, *root_sup, *root_db;
    const uint32_t *root_order;
    // queue
    Task *tasks;
    unsigned long long task_cap;
    uint32_t *cand_pool;
    unsigned long long cand_pool_cap;
    int split_depth;    // push children whose prefix length <= split_depth
    // per-worker stack
    uint32_t *stack_bits;   // [workers][depth][nwp]
    uint32_t *frame_items;  // [workers][pool]  F lists (internal ids)
    uint32_t *frame_sups;   // [workers][pool]
    int64_t frame_pool;     // entries per worker
    int depth_cap;          // levels per worker
    // results
    unsigned long long *rec_off;
    uint32_t *rec_len;
    uint32_t *rec_sup;
    uint32_t *rec_items;
    uint32_t *rec_db;
    unsigned long long rec_cap, rec_items_cap;
    // learned / traces
    const __nv_bfloat16 *mlp_w;  // bf16 weights or null
    const uint32_t *epoch;       // this mine's epoch (bumped on the stream before the DFS)
    // sparse item columns (single database): item i's non-zero words at
    // [i * item_cap, i * item_cap + item_z[i]) of item_idx / item_val, or
    // item_z[i] < 0 when the column is kept dense only; null = none
    const uint32_t *item_idx, *item_val;
    const int *item_z;
    int64_t item_cap;
    int learned;
    int diffset_rule;
    float *trace_x;          // [cap][8]
    float *trace_y;          // [cap][2]
    unsigned long long trace_cap;
    int trace;
    MineCounters *ctr;
    unsigned long long spin_limit;  // bounded waits (ns of %globaltimer)
    long long withhold_slot;        // test hook: this queue slot is never published (-1: none)
    int sparse_div;                 // store b_Y sparse when S(Y) * sparse_div <= nw (0: never)
    int learned_kmin;               // FIM_LEARNED consults the network for classes with >= this many candidates
    int rec_chunk;                  // record slots a DFS worker reserves at a time (1: exactly per class)
    int root_reverse;               // hand out the root classes in reverse emission order
    RootWindow *win;                // warp workers: only this window's roots (null: all of them)
};

// ---------------------------------------------------------------- the ctx
struct fim_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    // matrix
    bool built = false;
    int64_t n = 0;
    int32_t m = 0;
    int64_t nw = 0, nwp = 0;
    int max_row_len = 0;
    DevBuf csr_ptr, csr_idx;   // staging for host input
    DevBuf bm, item_sup, perm, rank, dev_flag;

    // mine
    bool mined = false;
    uint32_t mflags = 0;
    int32_t mfreq = 0;
    DevBuf pair_cnt, pairbits, roots;
    DevBuf tasks, cand_pool, stack_bits, frame_items, frame_sups;
    DevBuf epoch;               // uint32: mine counter; a task slot is live when ready == epoch
    DevBuf sp_idx, sp_val, sp_z; // sparse copies of low-support frequent item columns
    DevBuf rec_off, rec_len, rec_sup, rec_items, rec_db;
    DevBuf counters;            // MineCounters
    DevBuf dbdesc;              // DbDesc table of the mine
    DbDesc host_db{};           // host copy of a single-database table
    MineCounters host_ctr;
    unsigned long long rec_cap = 0, rec_items_cap = 0;

    // compactor
    DevBuf keys, idx_a, idx_b, hist, scan_tmp, kv_a, kv_b, scan_part;
    DevBuf out_off, out_items, out_sup;
    uint64_t out_sets = 0, out_items_total = 0;
    uint64_t mine_serial = 0;   // completed fim_mine calls; names the output held
    int64_t out_n = 0;          // transactions behind the held output
    int shard = 0, n_shards = 1; // prefix-class share of the mine in progress
    DevBuf shard_cost, merge_off;
    DevBuf probe_buf;           // measurement probes' buffer

    // association rules of the held output
    DevBuf rule_base, rule_part, rule_bits, rule_kbase;  // evaluation space, scans, keep words
    DevBuf rule_set, rule_mask, rule_conf, rule_lift, rule_sets;
    uint64_t rules_n = 0, rules_evaluated = 0;
    uint64_t rules_of = 0;      // mine_serial the rules belong to

    // learned scheduler
    DevBuf mlp_w32, mlp_wbf, mlp_scratch;
    DevBuf root_order, root_bucket, root_hist;
    bool has_weights = false;
    uint32_t cur_thr = 0;       // threshold of the mine in progress
    DevBuf trace_x, trace_y;
    unsigned long long trace_cap = 0;

    // batched mines: device prefix arrays, result slices, the captured graph
    DevBuf batch_prefix, batch_slices;
    DevBuf batch_units;         // (database, tile) units of the batched tensor-core pair pass
    DevBuf batch_unit_db;       // database of each unit of the batched rows build
    bool batch_mined = false;
    int batch_n_db = 0;
    std::vector<unsigned long long> batch_set_start, batch_item_start;
    void *batch_graph_exec = nullptr;   // cudaGraphExec_t
    std::vector<unsigned char> batch_graph_blob, batch_graph_blob_next;  // what the graph was captured for
    // the batched pair pass's units, kept while each database's (m, words)
    // and the grouping repeat
    std::vector<int64_t> pair_units_sig;
    std::vector<unsigned long long> pair_units_cache;
    std::vector<int64_t> pair_seg_unit_cache;
    std::vector<int> pair_ord_cache;  // each group's databases, most transactions first
    bool pair_units_ok = false;
    bool phase_times_pending = false;  // a single mine's ev[1..4] still to be read
    int batch_pairs_pack = 1;   // the batch's pair units planned on the device, small databases two to a tile
    int batch_group_dfs = 1;    // pipelined groups: each group's roots mined right after its finalize
    DevBuf batch_windows;       // those groups' root windows
    DevBuf batch_plan;          // that plan's unit counts, database order and scratch
    std::vector<unsigned char> up_ord;
    std::pair<const void *, size_t> up_ord_buf{};
    // what the batched mine last copied into dbdesc / batch_prefix /
    // batch_units, and that buffer's (address, capacity) then: a call whose
    // bytes and buffer repeat skips the copy (a buffer that grew is a new
    // one); a single-database mine, which writes dbdesc, clears up_desc
    std::vector<unsigned char> up_desc, up_pre, up_units;
    std::pair<const void *, size_t> up_desc_buf{}, up_pre_buf{}, up_units_buf{};
    uint64_t batch_graph_launches = 0;
    // compactor pass sequence, captured when a shape repeats
    // (two slots: a split mine alternates the shard's and the merge's shapes)
    void *compact_graph_exec[2] = {nullptr, nullptr}; // cudaGraphExec_t
    uint64_t compact_key[2] = {0, 0}, compact_graph_launches[2] = {0, 0};
    uint64_t compact_seen_key[2] = {0, 0};
    int compact_next = 0, compact_seen_next = 0;

    // tuning (autotuner may overwrite)
    int dfs_block = 256;
    int dfs_ctas_per_sm = 4;
    int split_depth = 8;
    int sparse_div = -1;        // -1: automatic (frequent columns vs L2)
    int learned_kmin = 8;
    int learned_order = 0;      // 1: FIM_LEARNED also orders roots longest-predicted-first
    int root_reverse = 0;
    int l2_bytes = 0;
    int pairs_split = 0;        // split-K factor of the tensor-core pair pass (0 = auto)
    int pairs_kdrain = 0;       // stages (x128 transactions) per exact drain (0 = 64)
    int batch_pairs_shape = 0;  // launch shape of the batched tensor-core pair pass
    int batch_build_block = 32; // words per column a batched build CTA covers (16, 32 or 64)
    int batch_build_coal = 1;   // batched build: a warp reads its rows' ids coalesced
    int root_sort = 1;          // root order without the network: 0 pair-pass order, 1 candidate count
    int rec_chunk = 1;          // record slots a DFS worker reserves at a time
    int batch_segments = 0;     // database groups the batch graph pipelines (build || pairs); 0 automatic
    int dfs_warp = 1;           // batches of short columns: one warp per prefix-extension worker
    int dfs_warp_ctas = 2;      // CTAs of warp workers per SM (2 or 3)
    bool force_cta_dfs = false; // set while a batch is re-mined with CTA workers
    cudaEvent_t seg_ev[18] = {};  // fork, join and per-group events of that pipeline
    int batch_stream_copies = 1;  // page-locked host batches go up group by group beside the mine
    cudaStream_t copy_stream = nullptr;  // those uploads
    cudaEvent_t copy_ev[18] = {};        // fork and per-group events of the uploads
    int compact_cluster = 1;    // small outputs: sort in one cluster launch
    int csort_cl[5] = {0, 0, 0, 0, 0};  // cluster size per key width (0 unknown, -1 none)
    int debug_checks = 0;       // device-side invariant checks after build and mine
    int spin_limit_ms = 60000;  // longest device-side wait before FIM_E_TIMEOUT
    int test_withhold_task = -1; // test hook: the DFS never publishes this queue slot
    int upload_mapped = 1;      // host input in pinned, mapped memory: build reads it in place
    int upload_chunks = 4;      // host input: index upload chunks overlapped with the build
    int upload_streams = 2;     // copy streams the chunks alternate over
    cudaStream_t up_stream[2] = {nullptr, nullptr};
    cudaStream_t aux_stream = nullptr;  // work that overlaps the pair pass
    cudaEvent_t aux_ev[2] = {};
    cudaEvent_t up_ev[16] = {};

    // stats + timing
    fim_stats stats{};
    cudaEvent_t ev[8] = {};
    size_t bytes_held = 0;
    uint64_t launches = 0;      // kernels this ctx has launched
};

int fim_reserve(fim_ctx *ctx, DevBuf &b, size_t bytes);
int fim_aux_stream(fim_ctx *ctx);  // create the side stream (highest priority) once
int fim_finish_phase_times(fim_ctx *ctx);  // the last single mine's phase times, once it has finished
void fim_release(fim_ctx *ctx, DevBuf &b);

// ---------------------------------------------------------------- launchers
// k_matrix.cu
// nnz < 0: read indptr[n] from the device.  h_indptr/h_indices (host input):
// the indices are uploaded into d_indices chunk by chunk, overlapping the build.
// compact: the CSR holds uint32 row offsets and uint16 item ids.
int launch_build_bitmaps(fim_ctx *ctx, const void *d_indptr, const void *d_indices, int64_t nnz,
                         const void *h_indptr, const void *h_indices, bool compact);
int launch_item_support(fim_ctx *ctx);
int launch_rank_items(fim_ctx *ctx, uint32_t thr, MineCounters *d_ctr);
int launch_emit_singletons(fim_ctx *ctx, MineCounters *d_ctr);
int launch_max_row_freq(fim_ctx *ctx, const int64_t *d_indptr, const int32_t *d_indices,
                        MineCounters *d_ctr);

// k_pairs.cu
int launch_pairs_popc(fim_ctx *ctx);
int launch_pairs_tc(fim_ctx *ctx);   // tcgen05; returns FIM_E_INVAL if unsupported
int launch_pairs_finalize(fim_ctx *ctx, uint32_t thr, MineCounters *d_ctr);

// k_dfs.cu
int launch_dfs(fim_ctx *ctx, const DfsParams &p, int grid, int block);
// Task slots carry the epoch of the mine that published them, so the queue
// needs no clearing between mines: bump the epoch (on the stream, so that a
// replayed graph bumps it too) and clear the slots only when the buffer is new.
int prepare_task_queue(fim_ctx *ctx, size_t bytes);
int launch_epoch_bump(fim_ctx *ctx);
// Sparse copies of the frequent item columns with S <= cap (single database).
// sparse copies of the low-support item columns for the root classes: the
// buffers first (host side), then the copy, on a stream of the caller's
int reserve_sparse_items(fim_ctx *ctx, int mf, int64_t cap);
int launch_sparse_items(fim_ctx *ctx, int mf, int64_t cap, cudaStream_t st);

// k_mlp.cu: learned root order (longest predicted subtree first)
// k_mlp.cu: drop the candidate-less roots, order the others (mode 0 about
// the pair pass's order, 1 by candidate count, 2 by the network's predicted
// subtree work); d_dbs = the batch's table, or null for a single database
int reserve_root_plan(fim_ctx *ctx, size_t root_cap);
// win (non-null): plan only the window's roots, leaving the root count to
// the groups that append after it
int launch_root_plan(fim_ctx *ctx, MineCounters *d_ctr, size_t root_cap, const DbDesc *d_dbs, int mode, RootWindow *win,
                     cudaStream_t st);

// k_compact.cu
// identity_items: the records already hold the caller's item ids (a merge)
// Sorts records [0, n_records) into the canonical output; n_valid of them are
// itemsets, the rest holes (length 0), which sort last and are left out.
int launch_compact(fim_ctx *ctx, uint64_t n_records, uint64_t n_valid, int n_db, int m_max,
                   bool identity_items = false);

// k_csort.cu: the compactor's sort of a small output in one cluster launch
int cluster_sort_plan(fim_ctx *ctx, uint64_t R, int kw, int *cl, int *cap, int *per);
int launch_cluster_sort(fim_ctx *ctx, const unsigned long long *keys, uint64_t R, int kw,
                        const std::vector<std::pair<int, int>> &passes, int cl, int cap, int per,
                        uint32_t *idx_out, cudaStream_t st);

// k_batch_pairs_tc.cu: the batch's pair supports on the tensor cores
bool batch_pairs_tc_units(const std::vector<DbDesc> &dbs, int d0, int d1, std::vector<unsigned long long> &units,
                          size_t max_units);
// d_n_units: the unit count written on the device by the plan kernel (null:
// n_units itself); n_units is then the capacity, which sizes the grid
int launch_batch_pairs_tc(fim_ctx *ctx, const DbDesc *d_dbs, const unsigned long long *d_units, int64_t n_units,
                          const long long *d_n_units, cudaStream_t st);
// Device plan of one group's pair units once m'_d is known: ord[0 .. n) the
// group's databases, most transactions first; databases with at most 64
// frequent items are packed two to a tile; *d_n_units gets the count.
// scratch: batch_pair_plan_scratch(n) bytes.
int launch_batch_pair_plan(fim_ctx *ctx, const DbDesc *d_dbs, const int *d_ord, int n, unsigned long long *d_units,
                           long long *d_n_units, void *scratch, cudaStream_t st);
size_t batch_pair_plan_scratch(int n);
extern const int kBatchPairsShapeCount;

// k_dfs_warp.cu: the prefix extension with one warp per worker
int launch_dfs_warp(fim_ctx *ctx, const DfsParams &p, int n_warps, int ctas_per_sm, cudaStream_t st);
int dfs_warp_max_depth();
int dfs_warp_per_cta();

// k_check.cu: the debug_checks invariants (FIM_E_CHECK when violated)
int run_check_pads(fim_ctx *ctx);
int run_check_output(fim_ctx *ctx, uint32_t thr);

// k_shard.cu: append the root classes shard `shard` of n_shards owns
int launch_shard_roots(fim_ctx *ctx, MineCounters *d_ctr, int shard, int n_shards);

// ---------------------------------------------------------------- device helpers
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint4 ldg_u4(const uint32_t *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

__device__ __forceinline__ uint4 ld_cg_u4(const uint32_t *p) {
    uint4 r;
    asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}

__device__ __forceinline__ uint32_t popc_and4(uint4 a, uint4 b) {
    return __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
}

__device__ __forceinline__ uint4 and4(uint4 a, uint4 b) {
    return make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
#endif
