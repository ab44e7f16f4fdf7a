// fim_api.cu -- the C ABI of include/fim.h: context, memory, and the order of
// the three stages of Section III (matrix construction, support calculation,
// frequent-itemset extraction).  No exception crosses the boundary; every
// entry point returns a FIM_* status.
#include <cstdio>
#include <cstring>
#include <new>

#include "fim_common.cuh"


namespace {

thread_local char g_last_cuda[256] = {0};

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

constexpr unsigned long long kTaskCap = 1ull << 20;
constexpr unsigned long long kCandPoolCap = 1ull << 24;
constexpr size_t kStackBudget = 8ull << 30;   // first try; grows on FIM_E_STACK
constexpr size_t kStackBudgetMax = 64ull << 30;

}  // namespace

void fim_set_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    snprintf(g_last_cuda, sizeof(g_last_cuda), "%s (%s) at %s:%d: %s", cudaGetErrorName(e), what,
             file, line, cudaGetErrorString(e));
    (void)cudaGetLastError();  // clear a sticky-free error so the ctx stays usable
}

// The ctx's side stream, at the device's highest priority: work put there
// (a group's pair pass beside the next group's build) is scheduled first
// where the two kernels compete for an SM.
int fim_aux_stream(fim_ctx *ctx) {
    if (ctx->aux_stream) return FIM_OK;
    int least = 0, greatest = 0;
    FIM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    FIM_CUDA_TRY(cudaStreamCreateWithPriority(&ctx->aux_stream, cudaStreamNonBlocking, greatest));
    return FIM_OK;
}

// Phase times of the last single-database mine, once its work has finished
// (events ev[1..4] of that mine; called before anything records them again).
int fim_finish_phase_times(fim_ctx *ctx) {
    if (!ctx->phase_times_pending) return FIM_OK;
    ctx->phase_times_pending = false;
    FIM_CUDA_TRY(cudaEventSynchronize(ctx->ev[4]));
    cudaEventElapsedTime(&ctx->stats.ms_pairs, ctx->ev[1], ctx->ev[2]);
    cudaEventElapsedTime(&ctx->stats.ms_dfs, ctx->ev[2], ctx->ev[3]);
    cudaEventElapsedTime(&ctx->stats.ms_compact, ctx->ev[3], ctx->ev[4]);
    return FIM_OK;
}

int fim_reserve(fim_ctx *ctx, DevBuf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (bytes <= b.bytes) return FIM_OK;
    if (b.p) {
        FIM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        cudaFree(b.p);
        ctx->bytes_held -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t nb = bytes + bytes / 4;
    nb = (nb + 255) & ~(size_t)255;
    cudaError_t e = cudaMalloc(&b.p, nb);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        e = cudaMalloc(&b.p, bytes);
        nb = bytes;
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            b.p = nullptr;
            return FIM_E_NOMEM;
        }
    }
    b.bytes = nb;
    ctx->bytes_held += nb;
    if (ctx->bytes_held > ctx->stats.peak_device_bytes) ctx->stats.peak_device_bytes = ctx->bytes_held;
    return FIM_OK;
}

void fim_release(fim_ctx *ctx, DevBuf &b) {
    if (b.p) {
        cudaFree(b.p);
        ctx->bytes_held -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

extern "C" {

uint32_t fim_version(void) { return (1u << 16) | 0u; }

const char *fim_strerror(int s) {
    switch (s) {
        case FIM_OK: return "ok";
        case FIM_E_INVAL: return "invalid argument or malformed database";
        case FIM_E_NOMEM: return "out of memory";
        case FIM_E_CUDA: return g_last_cuda[0] ? g_last_cuda : "CUDA error";
        case FIM_E_TIMEOUT: return "bounded device wait expired";
        case FIM_E_STACK: return "DFS stack budget exceeded";
        case FIM_E_TOO_SMALL: return "output buffer too small";
        case FIM_E_STATE: return "call out of order";
        case FIM_E_NODEV: return "no such CUDA device";
        case FIM_E_CHECK: return "a debug_checks invariant failed (internal error)";
        default: return "unknown status";
    }
}

uint64_t fim_minsup_from_ppm(int64_t n_trans, uint32_t ppm) {
    if (n_trans <= 0) return 1;
    const unsigned __int128 num = (unsigned __int128)(uint64_t)n_trans * ppm + 999999u;
    const uint64_t v = (uint64_t)(num / 1000000u);
    return v ? v : 1;
}

int fim_create(fim_ctx **out, int device, void *cuda_stream) {
    FIM_NVTX("fim_create");
    if (!out) return FIM_E_INVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
        (void)cudaGetLastError();
        return FIM_E_NODEV;
    }
    if (device < 0 || device >= ndev) return FIM_E_NODEV;
    DeviceGuard g(device);
    if (!g.ok) return FIM_E_CUDA;
    fim_ctx *ctx = new (std::nothrow) fim_ctx();
    if (!ctx) return FIM_E_NOMEM;
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&ctx->l2_bytes, cudaDevAttrL2CacheSize, device);
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return FIM_E_CUDA;
        }
        ctx->own_stream = true;
    }
    for (auto &e : ctx->ev) cudaEventCreate(&e);
    int rc = fim_reserve(ctx, ctx->counters, sizeof(MineCounters));
    if (rc == FIM_OK) rc = fim_reserve(ctx, ctx->dev_flag, 4 * sizeof(int));
    if (rc == FIM_OK) rc = fim_reserve(ctx, ctx->epoch, sizeof(uint32_t));
    if (rc == FIM_OK && cudaMemsetAsync(ctx->epoch.p, 0, sizeof(uint32_t), ctx->stream) != cudaSuccess) rc = FIM_E_CUDA;
    if (rc != FIM_OK) {
        fim_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return FIM_OK;
}

void fim_destroy(fim_ctx *ctx) {
    FIM_NVTX("fim_destroy");
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    DevBuf *all[] = {&ctx->csr_ptr, &ctx->csr_idx, &ctx->bm, &ctx->item_sup, &ctx->perm, &ctx->rank,
                     &ctx->dev_flag, &ctx->pair_cnt, &ctx->pairbits, &ctx->roots, &ctx->tasks,
                     &ctx->cand_pool, &ctx->stack_bits, &ctx->frame_items, &ctx->frame_sups,
                     &ctx->rec_off, &ctx->rec_len, &ctx->rec_sup, &ctx->rec_items, &ctx->counters,
                     &ctx->keys, &ctx->idx_a, &ctx->idx_b, &ctx->hist, &ctx->scan_tmp, &ctx->kv_a, &ctx->kv_b,
                     &ctx->scan_part, &ctx->out_off,
                     &ctx->out_items, &ctx->out_sup, &ctx->rule_base, &ctx->rule_part, &ctx->rule_bits,
                     &ctx->rule_kbase, &ctx->rule_set, &ctx->rule_mask,
                     &ctx->rule_conf, &ctx->rule_lift, &ctx->rule_sets, &ctx->probe_buf, &ctx->shard_cost, &ctx->merge_off, &ctx->mlp_w32, &ctx->mlp_wbf, &ctx->trace_x,
                     &ctx->trace_y, &ctx->mlp_scratch, &ctx->root_order, &ctx->root_bucket,
                     &ctx->root_hist, &ctx->rec_db, &ctx->dbdesc, &ctx->epoch, &ctx->sp_idx,
                     &ctx->sp_val, &ctx->sp_z};
    for (DevBuf *b : all) fim_release(ctx, *b);
    fim_release(ctx, ctx->batch_prefix);
    fim_release(ctx, ctx->batch_units);
    fim_release(ctx, ctx->batch_unit_db);
    fim_release(ctx, ctx->batch_plan);
    fim_release(ctx, ctx->batch_windows);
    fim_release(ctx, ctx->batch_slices);
    if (ctx->batch_graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)ctx->batch_graph_exec);
    for (void *g : ctx->compact_graph_exec)
        if (g) cudaGraphExecDestroy((cudaGraphExec_t)g);
    for (cudaStream_t u : ctx->up_stream)
        if (u) cudaStreamDestroy(u);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    for (cudaEvent_t e : ctx->seg_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (cudaEvent_t e : ctx->copy_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->aux_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->up_ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int fim_build_bitmaps(fim_ctx *ctx, const void *indptr, const void *indices, int64_t n_trans,
                      int32_t n_items, uint32_t flags) {
    FIM_NVTX("fim_build_bitmaps");
    if (!ctx) return FIM_E_INVAL;
    if (n_trans < 0 || n_trans > FIM_MAX_TRANS || n_items < 0 || n_items > FIM_MAX_ITEMS) return FIM_E_INVAL;
    if (!indptr) return FIM_E_INVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return FIM_E_CUDA;
    FIM_TRY(fim_finish_phase_times(ctx));  // before the events are recorded again
    ctx->built = false;
    ctx->mined = false;
    ctx->n = n_trans;
    ctx->m = n_items;
    ctx->nw = ceil_div64(n_trans, 32);
    ctx->nwp = round_up64(ctx->nw, FIM_WORDS_ALIGN);
    cudaStream_t st = ctx->stream;
    cudaEventRecord(ctx->ev[0], st);
    const uint64_t launches0 = ctx->launches;

    // the CSR's element types (FIM_CSR_COMPACT: uint32 row offsets, uint16 ids)
    const bool cmp = (flags & FIM_CSR_COMPACT) != 0;
    const size_t pb = csr_off_bytes(cmp), ib = csr_id_bytes(cmp);
    const void *d_ptr = indptr;
    const void *d_idx = indices;
    int64_t h_nnz = -1;
    bool mapped = false;  // pinned host CSR read by the build kernel in place
    if (!(flags & FIM_INPUT_DEVICE)) {
        const int64_t nnz = csr_off(indptr, cmp, n_trans);
        if (csr_off(indptr, cmp, 0) != 0 || nnz < 0 || (nnz > 0 && !indices)) return FIM_E_INVAL;
        if (ctx->upload_mapped) {
            // page-locked, mapped host memory is addressable from the GPU: the
            // kernel streams it over the host link, no staging copy
            cudaPointerAttributes ap{}, ai{};
            const bool ok_p = cudaPointerGetAttributes(&ap, indptr) == cudaSuccess &&
                              ap.type == cudaMemoryTypeHost && ap.devicePointer != nullptr;
            const bool ok_i = nnz == 0 || (cudaPointerGetAttributes(&ai, indices) == cudaSuccess &&
                                           ai.type == cudaMemoryTypeHost && ai.devicePointer != nullptr);
            cudaGetLastError();  // a query on unregistered memory leaves no sticky error
            if (ok_p && ok_i) {
                d_ptr = ap.devicePointer;
                d_idx = nnz ? ai.devicePointer : indices;
                h_nnz = nnz;
                mapped = true;
            }
        }
    }
    if (!(flags & FIM_INPUT_DEVICE) && !mapped) {
        const int64_t nnz = csr_off(indptr, cmp, n_trans);
        FIM_TRY(fim_reserve(ctx, ctx->csr_ptr, pb * (size_t)(n_trans + 1)));
        FIM_TRY(fim_reserve(ctx, ctx->csr_idx, ib * (size_t)(nnz > 0 ? nnz : 1)));
        FIM_CUDA_TRY(cudaMemcpyAsync(ctx->csr_ptr.p, indptr, pb * (size_t)(n_trans + 1), cudaMemcpyHostToDevice, st));
        // (the indices go up inside launch_build_bitmaps, overlapped with the build)
        d_ptr = ctx->csr_ptr.p;
        d_idx = ctx->csr_idx.p;
        h_nnz = nnz;
    }
    // device input: indptr[0] == 0 and indptr[n] >= 0 are checked by the build
    // kernel (no host round trip)
    const size_t mm = (size_t)(n_items > 0 ? n_items : 1);
    FIM_TRY(fim_reserve(ctx, ctx->bm, sizeof(uint32_t) * (size_t)ctx->nwp * mm));
    FIM_TRY(fim_reserve(ctx, ctx->item_sup, sizeof(uint32_t) * mm));
    FIM_TRY(fim_reserve(ctx, ctx->perm, sizeof(int32_t) * mm));
    FIM_TRY(fim_reserve(ctx, ctx->rank, sizeof(int32_t) * mm));
    if (flags & FIM_INPUT_DEVICE) FIM_TRY(launch_build_bitmaps(ctx, d_ptr, d_idx, -1, nullptr, nullptr, cmp));
    else if (mapped) FIM_TRY(launch_build_bitmaps(ctx, d_ptr, d_idx, h_nnz, nullptr, nullptr, cmp));
    else FIM_TRY(launch_build_bitmaps(ctx, d_ptr, d_idx, h_nnz, indptr, h_nnz > 0 ? indices : nullptr, cmp));
    cudaEventRecord(ctx->ev[1], st);
    FIM_TRY(launch_item_support(ctx));
    cudaEventRecord(ctx->ev[2], st);
    int flag[2] = {0, 0};
    FIM_CUDA_TRY(cudaMemcpyAsync(flag, ctx->dev_flag.p, sizeof(flag), cudaMemcpyDeviceToHost, st));
    FIM_CUDA_TRY(cudaStreamSynchronize(st));
    if (flag[0]) return FIM_E_INVAL;
    ctx->max_row_len = flag[1];
    cudaEventElapsedTime(&ctx->stats.ms_build, ctx->ev[0], ctx->ev[1]);
    cudaEventElapsedTime(&ctx->stats.ms_singletons, ctx->ev[1], ctx->ev[2]);
    if (ctx->debug_checks) FIM_TRY(run_check_pads(ctx));
    ctx->stats.launches_build = ctx->launches - launches0;
    ctx->built = true;
    return FIM_OK;
}

}  // extern "C"

namespace {

struct MineState {
    int depth_cap = 0;
    int64_t frame_pool = 0;
    size_t stack_budget = kStackBudget;
};

// One attempt at the whole mine with the current capacities.  Returns
// FIM_OK, or an error; *retry is set when a capacity must grow first.
int mine_once(fim_ctx *ctx, uint32_t thr, uint32_t flags, MineState &ms, bool *retry) {
    cudaStream_t st = ctx->stream;
    *retry = false;
    ctx->cur_thr = thr;
    if ((flags & FIM_LEARNED) && !ctx->has_weights) return FIM_E_STATE;
    MineCounters *d_ctr = ctx->counters.as<MineCounters>();
    FIM_CUDA_TRY(cudaMemsetAsync(d_ctr, 0, sizeof(MineCounters), st));
    cudaEventRecord(ctx->ev[0], st);
    FIM_TRY(launch_rank_items(ctx, thr, d_ctr));
    if (ctx->shard == 0) FIM_TRY(launch_emit_singletons(ctx, d_ctr));
    FIM_CUDA_TRY(cudaMemcpyAsync(&ctx->host_ctr, d_ctr, sizeof(MineCounters), cudaMemcpyDeviceToHost, st));
    FIM_CUDA_TRY(cudaStreamSynchronize(st));
    ctx->mfreq = ctx->host_ctr.m_freq;
    const int mf = ctx->mfreq;
    const uint32_t maxlen = flags >> 24;
    {   // the one-entry database table of a single-database mine (DFS, compactor)
        DbDesc &d = ctx->host_db;
        d = DbDesc{};
        d.n = ctx->n;
        d.nw = ctx->nw;
        d.nwp = ctx->nwp;
        d.m = ctx->m;
        d.mfreq = mf;
        d.thr = thr;
        d.maxlen = maxlen;
        FIM_TRY(fim_reserve(ctx, ctx->dbdesc, sizeof(DbDesc)));
        ctx->up_desc.clear();  // the batched mine's table is overwritten
        FIM_CUDA_TRY(cudaMemcpyAsync(ctx->dbdesc.p, &d, sizeof(DbDesc), cudaMemcpyHostToDevice, st));
    }
    cudaEventRecord(ctx->ev[1], st);
    const bool do_pairs = mf >= 2 && (maxlen == 0 || maxlen >= 2);
    const bool do_dfs = do_pairs && mf >= 3 && (maxlen == 0 || maxlen >= 3);
    // automatic: keep low-support classes sparse when the frequent item
    // columns do not fit in half of L2 (streaming whole columns from HBM
    // is latency-bound; from L2 the dense pass is as fast)
    const int sparse_div = ctx->sparse_div >= 0 ? ctx->sparse_div
                           : ((double)mf * (double)ctx->nwp * 4.0 > 0.5 * (double)ctx->l2_bytes ? 4 : 0);
    // sparse copies of the low-support item columns, for the root classes
    // (bounded: at most 1 GiB of (index, word) pairs); a child of a sparse
    // parent is stored sparse, so the copies must fit half a stack level.
    // They depend only on the ranking, so they are made on a side stream
    // while the pair pass runs (their kernel fits beside its CTAs).
    int64_t sp_cap = sparse_div > 0 ? ctx->nw / sparse_div : 0;
    if (sp_cap > ctx->nwp / 2) sp_cap = ctx->nwp / 2;
    const bool sp_items = do_dfs && sp_cap > 0 && (double)mf * (double)sp_cap * 8.0 <= (double)(1ull << 30);
    if (sp_items) {
        FIM_TRY(reserve_sparse_items(ctx, mf, sp_cap));
        FIM_TRY(fim_aux_stream(ctx));
        for (auto &e : ctx->aux_ev)
            if (!e) FIM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        FIM_CUDA_TRY(cudaEventRecord(ctx->aux_ev[0], st));
        FIM_CUDA_TRY(cudaStreamWaitEvent(ctx->aux_stream, ctx->aux_ev[0], 0));
    }
    ctx->stats.pair_path = 0;
    if (do_pairs) {
        const int mpw = (int)ceil_div64(mf, 32);
        const size_t npairs = (size_t)mf * (mf - 1) / 2;
        FIM_TRY(fim_reserve(ctx, ctx->pair_cnt, sizeof(int) * (size_t)mf * mf));
        FIM_TRY(fim_reserve(ctx, ctx->pairbits, sizeof(uint32_t) * (size_t)mf * mpw));
        FIM_TRY(fim_reserve(ctx, ctx->roots, sizeof(uint32_t) * 3 * npairs));
        int rc = FIM_E_INVAL;
        if (!(flags & FIM_PAIRS_POPC)) rc = launch_pairs_tc(ctx);
        if (rc == FIM_OK) ctx->stats.pair_path = 1;
        else FIM_TRY(launch_pairs_popc(ctx));
        if (sp_items) {  // launched after the pair pass, so that its CTAs take the SMs first
            FIM_TRY(launch_sparse_items(ctx, mf, sp_cap, ctx->aux_stream));
            FIM_CUDA_TRY(cudaEventRecord(ctx->aux_ev[1], ctx->aux_stream));
        }
        FIM_TRY(launch_pairs_finalize(ctx, thr, d_ctr));
        // a shard of a split mine takes only the root classes it owns
        if (ctx->n_shards > 1) FIM_TRY(launch_shard_roots(ctx, d_ctr, ctx->shard, ctx->n_shards));
    }
    cudaEventRecord(ctx->ev[2], st);
    if (do_dfs) {
        const int workers = ctx->num_sms * ctx->dfs_ctas_per_sm;
        // deepest class: a prefix can hold at most min(longest row, m') items
        int bound = ctx->max_row_len < mf ? ctx->max_row_len : mf;
        if (maxlen && (int)maxlen < bound) bound = (int)maxlen;
        if (bound > 240) bound = 240;  // the worker's shared-memory frame arrays hold 256 levels
        const int levels_needed = bound > 2 ? bound - 1 : 1;
        const size_t per_level = (size_t)workers * (size_t)ctx->nwp * sizeof(uint32_t);
        if (ms.depth_cap == 0) {
            size_t cap = ms.stack_budget / (per_level ? per_level : 1);
            ms.depth_cap = (int)(cap < (size_t)levels_needed ? cap : (size_t)levels_needed);
            if (ms.depth_cap < 2) ms.depth_cap = 2;
        }
        if (ms.frame_pool == 0) ms.frame_pool = 4LL * mf + 1024;
        FIM_TRY(fim_reserve(ctx, ctx->stack_bits, per_level * (size_t)ms.depth_cap));
        FIM_TRY(fim_reserve(ctx, ctx->frame_items, sizeof(uint32_t) * (size_t)workers * ms.frame_pool));
        FIM_TRY(fim_reserve(ctx, ctx->frame_sups, sizeof(uint32_t) * (size_t)workers * ms.frame_pool));
        FIM_TRY(prepare_task_queue(ctx, sizeof(Task) * kTaskCap));
        FIM_TRY(fim_reserve(ctx, ctx->cand_pool, sizeof(uint32_t) * kCandPoolCap));
        FIM_TRY(launch_epoch_bump(ctx));
        const size_t npairs = (size_t)mf * (mf - 1) / 2;
        DfsParams p{};
        p.dbs = ctx->dbdesc.as<DbDesc>();
        p.bm = ctx->bm.as<uint32_t>();
        p.perm = ctx->perm.as<int32_t>();
        p.pairbits = ctx->pairbits.as<uint32_t>();
        p.nwp_max = ctx->nwp;
        p.root_a = ctx->roots.as<uint32_t>();
        p.root_b = p.root_a + npairs;
        p.root_sup = p.root_a + 2 * npairs;
        p.root_db = nullptr;
        p.rec_db = ctx->rec_db.as<uint32_t>();
        p.tasks = ctx->tasks.as<Task>();
        p.task_cap = kTaskCap;
        p.cand_pool = ctx->cand_pool.as<uint32_t>();
        p.cand_pool_cap = kCandPoolCap;
        p.split_depth = (flags & FIM_NO_SPLIT) ? 0 : ctx->split_depth;
        p.stack_bits = ctx->stack_bits.as<uint32_t>();
        p.frame_items = ctx->frame_items.as<uint32_t>();
        p.frame_sups = ctx->frame_sups.as<uint32_t>();
        p.frame_pool = ms.frame_pool;
        p.depth_cap = ms.depth_cap;
        p.rec_off = ctx->rec_off.as<unsigned long long>();
        p.rec_len = ctx->rec_len.as<uint32_t>();
        p.rec_sup = ctx->rec_sup.as<uint32_t>();
        p.rec_items = ctx->rec_items.as<uint32_t>();
        p.rec_cap = ctx->rec_cap;
        p.rec_items_cap = ctx->rec_items_cap;
        p.ctr = d_ctr;
        p.spin_limit = (unsigned long long)ctx->spin_limit_ms * 1000000ull;
        p.withhold_slot = ctx->test_withhold_task;
        p.sparse_div = sparse_div;
        p.epoch = ctx->epoch.as<uint32_t>();
        p.learned_kmin = ctx->learned_kmin;
        p.rec_chunk = ctx->rec_chunk;
        p.root_reverse = ctx->root_reverse;
        if (sp_items) {
            FIM_CUDA_TRY(cudaStreamWaitEvent(st, ctx->aux_ev[1], 0));
            p.item_idx = ctx->sp_idx.as<uint32_t>();
            p.item_val = ctx->sp_val.as<uint32_t>();
            p.item_z = ctx->sp_z.as<int>();
            p.item_cap = sp_cap;
        }
        p.pair_cnt = ctx->pair_cnt.as<int>();
        p.item_sup = ctx->item_sup.as<uint32_t>();
        p.root_order = nullptr;
        p.learned = (flags & FIM_LEARNED) ? 1 : 0;
        p.diffset_rule = (flags & FIM_DIFFSET_RULE) ? 1 : 0;
        p.mlp_w = ctx->mlp_wbf.as<__nv_bfloat16>();
        {   // candidate-less roots dropped, the others ordered
            const int mode = (p.learned && ctx->learned_order) ? 2 : ctx->root_sort;
            FIM_TRY(reserve_root_plan(ctx, npairs));
            FIM_TRY(launch_root_plan(ctx, d_ctr, npairs, nullptr, mode, nullptr, st));
            p.root_order = ctx->root_order.as<uint32_t>();
        }
        p.trace = (flags & FIM_TRACE) ? 1 : 0;
        if (p.trace) {
            // complete subtree totals need every subtree inside one worker
            p.split_depth = 0;
            if (ctx->trace_cap == 0) ctx->trace_cap = 1ull << 21;
            FIM_TRY(fim_reserve(ctx, ctx->trace_x, sizeof(float) * FIM_MLP_FEATURES * ctx->trace_cap));
            FIM_TRY(fim_reserve(ctx, ctx->trace_y, sizeof(float) * 2 * ctx->trace_cap));
            p.trace_x = ctx->trace_x.as<float>();
            p.trace_y = ctx->trace_y.as<float>();
            p.trace_cap = ctx->trace_cap;
        }
        FIM_TRY(launch_dfs(ctx, p, workers, ctx->dfs_block));
    }
    cudaEventRecord(ctx->ev[3], st);
    FIM_CUDA_TRY(cudaMemcpyAsync(&ctx->host_ctr, d_ctr, sizeof(MineCounters), cudaMemcpyDeviceToHost, st));
    FIM_CUDA_TRY(cudaStreamSynchronize(st));
    const MineCounters &c = ctx->host_ctr;
    if (c.err == FIM_E_STACK) {
        if (ms.stack_budget >= kStackBudgetMax) return FIM_E_STACK;
        ms.stack_budget *= 2;
        ms.depth_cap = ms.depth_cap * 2 > 240 ? 240 : ms.depth_cap * 2;
        ms.frame_pool *= 2;
        *retry = true;
        return FIM_OK;
    }
    if (c.err != 0) return c.err;
    if (c.overflow) {
        ctx->rec_cap = c.n_records + c.n_records / 4 + 1024;
        ctx->rec_items_cap = c.n_rec_items + c.n_rec_items / 4 + 4096;
        FIM_TRY(fim_reserve(ctx, ctx->rec_off, sizeof(unsigned long long) * ctx->rec_cap));
        FIM_TRY(fim_reserve(ctx, ctx->rec_len, sizeof(uint32_t) * ctx->rec_cap));
        FIM_TRY(fim_reserve(ctx, ctx->rec_sup, sizeof(uint32_t) * ctx->rec_cap));
        FIM_TRY(fim_reserve(ctx, ctx->rec_items, sizeof(uint32_t) * ctx->rec_items_cap));
    FIM_TRY(fim_reserve(ctx, ctx->rec_db, sizeof(uint32_t) * ctx->rec_cap));
        *retry = true;
        return FIM_OK;
    }
    int lmax = c.max_len;
    if (ctx->shard == 0 && mf >= 1 && lmax < 1) lmax = 1;
    const unsigned long long n_sets = c.n_records - c.rec_holes;
    if (ctx->shard == 0 && n_sets > (unsigned long long)mf && lmax < 2) lmax = 2;
    ctx->host_ctr.max_len = lmax;
    FIM_TRY(launch_compact(ctx, c.n_records, n_sets, 1, ctx->m));
    cudaEventRecord(ctx->ev[4], st);
    FIM_CUDA_TRY(cudaGetLastError());
    // the mine returns with the compaction queued: the next call that reads
    // results (or these phase times) synchronises the stream first
    ctx->phase_times_pending = true;
    return FIM_OK;
}

}  // namespace

extern "C" {

int fim_mine(fim_ctx *ctx, uint64_t minsup, uint32_t flags) {
    FIM_NVTX("fim_mine");
    if (!ctx) return FIM_E_INVAL;
    if (!ctx->built) return FIM_E_STATE;
    if (!(flags & FIM_STRICT) && minsup == 0) return FIM_E_INVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return FIM_E_CUDA;
    FIM_TRY(fim_finish_phase_times(ctx));  // before the events are recorded again
    ctx->mined = false;
    ctx->mflags = flags;
    uint64_t thr64 = (flags & FIM_STRICT) ? minsup + 1 : minsup;
    if ((flags & FIM_STRICT) && minsup == UINT64_MAX) thr64 = UINT64_MAX;
    const uint32_t thr = thr64 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)thr64;
    if (ctx->rec_cap == 0) {
        ctx->rec_cap = 1ull << 20;
        ctx->rec_items_cap = 1ull << 23;
    }
    FIM_TRY(fim_reserve(ctx, ctx->rec_off, sizeof(unsigned long long) * ctx->rec_cap));
    FIM_TRY(fim_reserve(ctx, ctx->rec_len, sizeof(uint32_t) * ctx->rec_cap));
    FIM_TRY(fim_reserve(ctx, ctx->rec_sup, sizeof(uint32_t) * ctx->rec_cap));
    FIM_TRY(fim_reserve(ctx, ctx->rec_items, sizeof(uint32_t) * ctx->rec_items_cap));
    FIM_TRY(fim_reserve(ctx, ctx->rec_db, sizeof(uint32_t) * ctx->rec_cap));
    const uint64_t launches0 = ctx->launches;
    MineState ms;
    bool retry = true;
    for (int attempt = 0; retry && attempt < 8; attempt++) FIM_TRY(mine_once(ctx, thr, flags, ms, &retry));
    if (retry) return FIM_E_NOMEM;
    const MineCounters &c = ctx->host_ctr;
    fim_stats &s = ctx->stats;
    s.n_trans = (uint64_t)ctx->n;
    s.n_items = (uint64_t)ctx->m;
    s.n_frequent_items = (uint64_t)ctx->mfreq;
    s.n_sets = c.n_records - c.rec_holes;
    s.max_len = (uint64_t)c.max_len;
    s.supports_singletons = (uint64_t)ctx->m;
    const uint64_t mf = (uint64_t)ctx->mfreq;
    const uint32_t maxlen = flags >> 24;
    s.supports_pairs = (mf >= 2 && (maxlen == 0 || maxlen >= 2)) ? mf * (mf - 1) / 2 : 0;
    s.supports_dfs = c.supports_dfs;
    s.dfs_words = c.dfs_words;
    s.dfs_bytes = c.dfs_bytes;
    s.dfs_touched_bytes = c.dfs_touched;
    s.classes = c.classes;
    s.tasks_pushed = c.pushed;
    s.diffset_classes = c.diffset;
    s.launches_mine = ctx->launches - launches0;
    s.dfs_busy_ns = c.busy_ns;
    s.dfs_span_ns = c.t_last > c.t_first && c.t_first != 0 ? c.t_last - c.t_first : 0;
    s.dfs_workers = (uint64_t)ctx->num_sms * (uint64_t)ctx->dfs_ctas_per_sm;
    s.dfs_root_ns = c.root_ns;
    if (ctx->bytes_held > s.peak_device_bytes) s.peak_device_bytes = ctx->bytes_held;
    if (ctx->debug_checks) FIM_TRY(run_check_output(ctx, thr));
    ctx->out_n = ctx->n;
    ctx->mined = true;
    ctx->mine_serial++;
    return FIM_OK;
}

int fim_mine_shard(fim_ctx *ctx, uint64_t minsup, uint32_t flags, int shard, int n_shards) {
    FIM_NVTX("fim_mine_shard");
    if (!ctx || n_shards < 1 || n_shards > FIM_MAX_SHARDS || shard < 0 || shard >= n_shards) return FIM_E_INVAL;
    ctx->shard = shard;
    ctx->n_shards = n_shards;
    const int rc = fim_mine(ctx, minsup, flags);
    ctx->shard = 0;
    ctx->n_shards = 1;
    return rc;
}

int fim_fetch_results(fim_ctx *ctx, uint64_t *n_sets, uint64_t *n_items_total, uint64_t *offsets,
                      uint32_t *items, uint32_t *supports, uint64_t cap_sets, uint64_t cap_items,
                      uint32_t flags) {
    FIM_NVTX("fim_fetch_results");
    if (!ctx || !n_sets || !n_items_total) return FIM_E_INVAL;
    if (!ctx->mined) return FIM_E_STATE;
    *n_sets = ctx->out_sets;
    *n_items_total = ctx->out_items_total;
    if (!offsets && !items && !supports) return FIM_OK;
    if (!offsets || !supports || (!items && ctx->out_items_total)) return FIM_E_INVAL;
    if (cap_sets < ctx->out_sets || cap_items < ctx->out_items_total) return FIM_E_TOO_SMALL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return FIM_E_CUDA;
    const cudaMemcpyKind k = (flags & FIM_OUTPUT_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaStream_t st = ctx->stream;
    FIM_CUDA_TRY(cudaMemcpyAsync(offsets, ctx->out_off.p, sizeof(uint64_t) * (ctx->out_sets + 1), k, st));
    if (ctx->out_items_total)
        FIM_CUDA_TRY(cudaMemcpyAsync(items, ctx->out_items.p, sizeof(uint32_t) * ctx->out_items_total, k, st));
    if (ctx->out_sets)
        FIM_CUDA_TRY(cudaMemcpyAsync(supports, ctx->out_sup.p, sizeof(uint32_t) * ctx->out_sets, k, st));
    FIM_CUDA_TRY(cudaStreamSynchronize(st));
    return FIM_OK;
}

int fim_get_stats(const fim_ctx *ctx, fim_stats *out) {
    FIM_NVTX("fim_get_stats");
    if (!ctx || !out) return FIM_E_INVAL;
    // the ctx is the caller's own (non-const) object; the phase times of a
    // mine still in flight are read here, after it has finished
    FIM_TRY(fim_finish_phase_times(const_cast<fim_ctx *>(ctx)));
    *out = ctx->stats;
    return FIM_OK;
}

int fim_set_tuning(fim_ctx *ctx, const char *key, int64_t v) {
    FIM_NVTX("fim_set_tuning");
    if (!ctx || !key) return FIM_E_INVAL;
    struct Knob { const char *name; int *field; int64_t lo, hi; } knobs[] = {
        {"dfs_ctas_per_sm", &ctx->dfs_ctas_per_sm, 1, 4},
        {"dfs_threads", &ctx->dfs_block, 256, 512},
        {"split_depth", &ctx->split_depth, 0, FIM_TASK_MAXR},
        {"sparse_div", &ctx->sparse_div, -1, 64},
        {"learned_kmin", &ctx->learned_kmin, 1, 1 << 20},
        {"learned_order", &ctx->learned_order, 0, 1},
        {"root_reverse", &ctx->root_reverse, 0, 1},
        {"pairs_split", &ctx->pairs_split, 0, 4096},
        {"pairs_kdrain", &ctx->pairs_kdrain, 0, 32768},
        {"upload_chunks", &ctx->upload_chunks, 1, 16},
        {"compact_cluster", &ctx->compact_cluster, 0, 1},
        {"upload_mapped", &ctx->upload_mapped, 0, 1},
        {"batch_stream_copies", &ctx->batch_stream_copies, 0, 1},
        {"spin_limit_ms", &ctx->spin_limit_ms, 1, 600000},
        {"debug_checks", &ctx->debug_checks, 0, 1},
        {"test_withhold_task", &ctx->test_withhold_task, -1, 1 << 20},
        {"upload_streams", &ctx->upload_streams, 1, 2},
        {"batch_pairs_shape", &ctx->batch_pairs_shape, 0, kBatchPairsShapeCount - 1},
        {"batch_build_block", &ctx->batch_build_block, 16, 64},
        {"batch_build_coal", &ctx->batch_build_coal, 0, 1},
        {"batch_pairs_pack", &ctx->batch_pairs_pack, 0, 1},
        {"batch_group_dfs", &ctx->batch_group_dfs, 0, 1},
        {"root_sort", &ctx->root_sort, 0, 1},
        {"record_chunk", &ctx->rec_chunk, 1, 1024},
        {"batch_segments", &ctx->batch_segments, 0, 16},
        {"dfs_warp", &ctx->dfs_warp, 0, 1},
        {"dfs_warp_ctas", &ctx->dfs_warp_ctas, 2, 3},
    };
    for (const Knob &k : knobs)
        if (strcmp(k.name, key) == 0) {
            if (v < k.lo || v > k.hi) return FIM_E_INVAL;
            // the DFS worker exists in two widths; a worker is capped at 64
            // registers a thread, so at most 1024 worker threads fit an SM
            if (k.field == &ctx->dfs_block && v != 256 && v != 512) return FIM_E_INVAL;
            if (k.field == &ctx->batch_build_block && v != 16 && v != 32 && v != 64) return FIM_E_INVAL;
            const int64_t block = k.field == &ctx->dfs_block ? v : ctx->dfs_block;
            const int64_t per_sm = k.field == &ctx->dfs_ctas_per_sm ? v : ctx->dfs_ctas_per_sm;
            if (block * per_sm > 1024) return FIM_E_INVAL;
            *k.field = (int)v;
            return FIM_OK;
        }
    return FIM_E_INVAL;
}

}  // extern "C"
