// k_mlp.cu -- the scheduling MLP (8 -> 64 -> 64 -> 2): training kernels,
// inference for the root order, weight loading and trace export.
//
// The paper names choosing the Boolean-operation sequence from data
// characteristics and deep models as directions (Section I; Section V); the
// network itself is this miner's design.  It predicts, per prefix class,
// y0 = log2(1 + subtree candidate words) and y1 = logit(store as diffset).  It
// steers the order in which root classes are handed out and the
// representation a class is counted in; supports are always counted exactly.
//
// Arithmetic modes: bf16 = 0 computes in float32; bf16 = 1 rounds weights,
// inputs and hidden activations to bf16 and accumulates in float32 (the
// inference precision).  Parameter layout: W1[64][8] b1[64] W2[64][64] b2[64]
// W3[2][64] b3[2].  Loss: mean_b 0.5 (y0 - t0)^2 + softplus(y1) - t1 y1.
#include "fim_common.cuh"



namespace {

constexpr int P = FIM_MLP_PARAMS;
constexpr int OFF_B1 = 64 * 8, OFF_W2 = OFF_B1 + 64, OFF_B2 = OFF_W2 + 64 * 64, OFF_W3 = OFF_B2 + 64,
              OFF_B3 = OFF_W3 + 2 * 64;
constexpr int CACHE = 256;  // per sample: z1[64] z2[64] dz1[64] dz2[64]

__device__ __forceinline__ float rb(float x, int bf) { return bf ? __bfloat162float(__float2bfloat16_rn(x)) : x; }

__device__ void load_weights(float *w, const float *params, int bf) {
    for (int i = threadIdx.x; i < P; i += blockDim.x) w[i] = rb(params[i], bf);
    __syncthreads();
}

__global__ void __launch_bounds__(128)
mlp_forward_kernel(const float *__restrict__ params, const float *__restrict__ x, int64_t B,
                   float *__restrict__ y, float *__restrict__ cache, int bf) {
    __shared__ float w[P];
    load_weights(w, params, bf);
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float xi[8], h1[64];
#pragma unroll
    for (int k = 0; k < 8; k++) xi[k] = rb(x[b * 8 + k], bf);
    for (int i = 0; i < 64; i++) {
        float a = w[OFF_B1 + i];
#pragma unroll
        for (int k = 0; k < 8; k++) a = fmaf(w[i * 8 + k], xi[k], a);
        if (cache) cache[b * CACHE + i] = a;
        h1[i] = rb(fmaxf(a, 0.f), bf);
    }
    float y0 = w[OFF_B3], y1 = w[OFF_B3 + 1];
    for (int i = 0; i < 64; i++) {
        float a = w[OFF_B2 + i];
#pragma unroll 16
        for (int k = 0; k < 64; k++) a = fmaf(w[OFF_W2 + i * 64 + k], h1[k], a);
        if (cache) cache[b * CACHE + 64 + i] = a;
        const float h2 = rb(fmaxf(a, 0.f), bf);
        y0 = fmaf(w[OFF_W3 + i], h2, y0);
        y1 = fmaf(w[OFF_W3 + 64 + i], h2, y1);
    }
    y[b * 2 + 0] = y0;
    y[b * 2 + 1] = y1;
}

// Per sample: dz2 = (W3^T dy) * [z2 > 0], dz1 = (W2^T dz2) * [z1 > 0]; loss.
__global__ void __launch_bounds__(128)
mlp_backward_sample_kernel(const float *__restrict__ params, const float *__restrict__ y,
                           const float *__restrict__ t, float *__restrict__ cache, int64_t B,
                           float *__restrict__ loss_parts, int bf) {
    __shared__ float w[P];
    __shared__ float red[4];
    load_weights(w, params, bf);
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (b < B) {
        const float y0 = y[b * 2], y1 = y[b * 2 + 1], t0 = t[b * 2], t1 = t[b * 2 + 1];
        const float e = y0 - t0;
        l = 0.5f * e * e + fmaxf(y1, 0.f) + log1pf(expf(-fabsf(y1))) - t1 * y1;
        const float dy0 = e / (float)B, dy1 = (1.f / (1.f + expf(-y1)) - t1) / (float)B;
        float *c = cache + b * CACHE;
        float dz2[64];
        for (int i = 0; i < 64; i++) {
            const float g = w[OFF_W3 + i] * dy0 + w[OFF_W3 + 64 + i] * dy1;
            dz2[i] = c[64 + i] > 0.f ? g : 0.f;
            c[192 + i] = dz2[i];
        }
        for (int k = 0; k < 64; k++) {
            float g = 0.f;
#pragma unroll 16
            for (int i = 0; i < 64; i++) g = fmaf(w[OFF_W2 + i * 64 + k], dz2[i], g);
            c[128 + k] = c[k] > 0.f ? g : 0.f;
        }
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) loss_parts[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
}

// Partial weight gradients over a chunk of samples: thread j owns parameters
// j, j + 256, ...; every parameter's gradient is a sum over the batch of a
// product of a cached backward term and a forward activation.
constexpr int GCHUNK = 256;
__global__ void __launch_bounds__(256)
mlp_grad_partial_kernel(const float *__restrict__ x, const float *__restrict__ y, const float *__restrict__ t,
                        const float *__restrict__ cache, int64_t B, float *__restrict__ part, int bf) {
    __shared__ float sx[32][8], sz1[32][64], sz2[32][64], sd1[32][64], sd2[32][64], sdy[32][2];
    float acc[(P + 255) / 256];
#pragma unroll
    for (int q = 0; q < (P + 255) / 256; q++) acc[q] = 0.f;
    const int64_t b0 = (int64_t)blockIdx.x * GCHUNK;
    const int64_t b1 = min64(B, b0 + GCHUNK);
    for (int64_t s0 = b0; s0 < b1; s0 += 32) {
        const int ns = (int)min64(32, b1 - s0);
        __syncthreads();
        for (int i = threadIdx.x; i < ns * 64; i += 256) {
            const int r = i / 64, c = i % 64;
            const float *cc = cache + (s0 + r) * CACHE;
            sz1[r][c] = rb(fmaxf(cc[c], 0.f), bf);      // h1
            sz2[r][c] = rb(fmaxf(cc[64 + c], 0.f), bf); // h2
            sd1[r][c] = cc[128 + c];
            sd2[r][c] = cc[192 + c];
        }
        for (int i = threadIdx.x; i < ns * 8; i += 256) sx[i / 8][i % 8] = rb(x[(s0 + i / 8) * 8 + i % 8], bf);
        if (threadIdx.x < ns) {
            const int64_t bb = s0 + threadIdx.x;
            sdy[threadIdx.x][0] = (y[bb * 2] - t[bb * 2]) / (float)B;
            sdy[threadIdx.x][1] = (1.f / (1.f + expf(-y[bb * 2 + 1])) - t[bb * 2 + 1]) / (float)B;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < (P + 255) / 256; q++) {
            const int j = threadIdx.x + q * 256;
            if (j >= P) break;
            float a = acc[q];
            if (j < OFF_B1) {                 // W1[i][k] += dz1[i] x[k]
                const int i = j / 8, k = j % 8;
                for (int r = 0; r < ns; r++) a = fmaf(sd1[r][i], sx[r][k], a);
            } else if (j < OFF_W2) {          // b1[i] += dz1[i]
                const int i = j - OFF_B1;
                for (int r = 0; r < ns; r++) a += sd1[r][i];
            } else if (j < OFF_B2) {          // W2[i][k] += dz2[i] h1[k]
                const int i = (j - OFF_W2) / 64, k = (j - OFF_W2) % 64;
                for (int r = 0; r < ns; r++) a = fmaf(sd2[r][i], sz1[r][k], a);
            } else if (j < OFF_W3) {          // b2[i] += dz2[i]
                const int i = j - OFF_B2;
                for (int r = 0; r < ns; r++) a += sd2[r][i];
            } else if (j < OFF_B3) {          // W3[o][k] += dy[o] h2[k]
                const int o = (j - OFF_W3) / 64, k = (j - OFF_W3) % 64;
                for (int r = 0; r < ns; r++) a = fmaf(sdy[r][o], sz2[r][k], a);
            } else {                          // b3[o] += dy[o]
                const int o = j - OFF_B3;
                for (int r = 0; r < ns; r++) a += sdy[r][o];
            }
            acc[q] = a;
        }
    }
#pragma unroll
    for (int q = 0; q < (P + 255) / 256; q++) {
        const int j = threadIdx.x + q * 256;
        if (j < P) part[(int64_t)blockIdx.x * P + j] = acc[q];
    }
}

// grad[j] = sum over chunks of part[c][j] (fixed order: deterministic).
__global__ void mlp_grad_sum_kernel(const float *__restrict__ part, int nchunks, float *__restrict__ grad,
                                    const float *__restrict__ loss_parts, int nloss, float *__restrict__ loss) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < P) {
        float a = 0.f;
        for (int c = 0; c < nchunks; c++) a += part[(int64_t)c * P + j];
        grad[j] = a;
    }
    if (j == P) {
        float a = 0.f;
        for (int c = 0; c < nloss; c++) a += loss_parts[c];
        *loss = a;
    }
}

__global__ void mlp_adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                                float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P) return;
    const float gj = g[j];
    const float mj = b1 * m[j] + (1.f - b1) * gj;
    const float vj = b2 * v[j] + (1.f - b2) * gj * gj;
    m[j] = mj;
    v[j] = vj;
    w[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + eps);
}

__global__ void to_bf16_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ o) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < P) o[j] = __float2bfloat16_rn(w[j]);
}

// ---- root plan: drop the roots without candidates, order the rest ---------
// A root {a, b} roots the prefix class of the sets whose two smallest items
// are a and b; its candidates are the c > b with {a, c} and {b, c} frequent
// (a row AND of the pair bitsets).  A root without candidates has no subtree,
// so it is dropped before the prefix extension starts: no worker spends a
// task fetch on it.  The others are ordered by a bucket sort on a priority,
// largest first: the scheduling network's predicted subtree work (the bf16
// MLP's y0 on the root class's features, as the DFS computes them), or the
// candidate count, or none (bucket 0: about the pair pass's order).
constexpr int NBUCKET = 256;
constexpr uint8_t DROP = NBUCKET - 1;

struct RootView {
    const uint32_t *pairbits;
    const int *pair_cnt;
    const uint32_t *item_sup;
    const int32_t *perm;
    int64_t n, nw;
    int mf, mpw;
    uint32_t thr;
};

__global__ void __launch_bounds__(256)
root_plan_kernel(const uint32_t *__restrict__ root_a, const uint32_t *__restrict__ root_b,
                 const uint32_t *__restrict__ root_sup, const uint32_t *__restrict__ root_db,
                 const MineCounters *ctr, const RootWindow *win, const DbDesc *__restrict__ dbs, RootView single,
                 int mode, const __nv_bfloat16 *__restrict__ wbf, uint8_t *__restrict__ bucket,
                 uint32_t *__restrict__ hist) {
    __shared__ float w[P];
    __shared__ uint32_t h[NBUCKET];
    if (mode == 2)
        for (int i = threadIdx.x; i < P; i += blockDim.x) w[i] = __bfloat162float(wbf[i]);
    for (int i = threadIdx.x; i < NBUCKET; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const unsigned long long r0 = win ? win->base : 0ull, nr = win ? r0 + win->count : ctr->n_roots;
    for (unsigned long long r = r0 + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; r < nr;
         r += (unsigned long long)gridDim.x * blockDim.x) {
        RootView v = single;
        if (dbs) {  // a batch: the root's database
            const DbDesc &D = dbs[root_db[r]];
            v.mf = *(volatile const int32_t *)&D.mfreq;
            v.mpw = (v.mf + 31) / 32;
            v.pairbits = single.pairbits + D.pb_off;
            v.pair_cnt = single.pair_cnt + D.pair_off;
            v.item_sup = single.item_sup + D.item_off;
            v.perm = single.perm + D.item_off;
            v.n = D.n;
            v.nw = D.nw;
            v.thr = D.thr;
        }
        const uint32_t a = root_a[r], bb = root_b[r];
        const uint32_t *ra = v.pairbits + (int64_t)a * v.mpw, *rbp = v.pairbits + (int64_t)bb * v.mpw;
        int k = 0;
        float ps = 0.f;
        for (int wd = (int)(bb >> 5); wd < v.mpw; wd++) {
            uint32_t bits = ra[wd] & rbp[wd];
            if (wd == (int)(bb >> 5)) bits &= 0xFFFFFFFEu << (bb & 31);
            k += __popc(bits);
            if (mode == 2)
                while (bits) {
                    const int c = wd * 32 + __ffs(bits) - 1;
                    bits &= bits - 1;
                    ps += (float)v.pair_cnt[(int64_t)a * v.mf + c];
                }
        }
        uint8_t bq = DROP;
        if (k > 0 && mode == 1) {
            bq = (uint8_t)(254 - (k < 254 ? k : 254));  // more candidates first
        } else if (k > 0 && mode == 2) {
            const uint32_t sy = root_sup[r], sx = v.item_sup[v.perm[a]];
            const float fx = sx > 0 ? (float)sx : 1.f, fy = sy > 0 ? (float)sy : 1.f;
            // the DFS kernel's feature vector of the root class (same scaling)
            float x[8] = {2.f / 16.f, log2f(1.f + (float)sy) / 32.f, (float)sy / (float)(v.n > 0 ? v.n : 1),
                          log2f(1.f + (float)k) / 16.f, (float)sy / fx, ps / ((float)k * fx),
                          log2f(1.f + (float)v.nw) / 32.f, (float)v.thr / fy};
            float h1[64];
            for (int i = 0; i < 64; i++) {
                float acc = w[OFF_B1 + i];
                for (int q = 0; q < 8; q++) acc = fmaf(w[i * 8 + q], __bfloat162float(__float2bfloat16_rn(x[q])), acc);
                h1[i] = __bfloat162float(__float2bfloat16_rn(fmaxf(acc, 0.f)));
            }
            float y0 = w[OFF_B3];
            for (int i = 0; i < 64; i++) {
                float acc = w[OFF_B2 + i];
                for (int q = 0; q < 64; q++) acc = fmaf(w[OFF_W2 + i * 64 + q], h1[q], acc);
                y0 = fmaf(w[OFF_W3 + i], __bfloat162float(__float2bfloat16_rn(fmaxf(acc, 0.f))), y0);
            }
            int q = (int)lrintf(4.f * y0);  // predicted log2(1 + subtree words), quarter steps
            q = q < 0 ? 0 : (q > 254 ? 254 : q);
            bq = (uint8_t)(254 - q);  // most predicted work first
        } else if (k > 0) {
            bq = 0;
        }
        bucket[r] = bq;
        atomicAdd(&h[bq], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NBUCKET; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// Exclusive scan of the bucket counts; the dropped roots leave the root
// count (a window's kept count instead) and the pending-task count.
// hist[NBUCKET] keeps the count before.
__global__ void root_plan_scan_kernel(uint32_t *hist, MineCounters *ctr, RootWindow *win) {
    if (threadIdx.x == 0) {
        const unsigned long long total = win ? win->count : ctr->n_roots;
        const uint32_t dropped = hist[DROP];
        uint32_t acc = 0;
        for (int i = 0; i < NBUCKET; i++) { const uint32_t v = hist[i]; hist[i] = acc; acc += v; }
        hist[NBUCKET] = (uint32_t)total;
        if (win)
            win->kept = total - dropped;
        else
            ctr->n_roots = total - dropped;
        ctr->pending -= (long long)dropped;
    }
}

__global__ void root_plan_scatter_kernel(const uint8_t *__restrict__ bucket, uint32_t *__restrict__ hist,
                                         const RootWindow *win, uint32_t *__restrict__ order) {
    const unsigned long long r0 = win ? win->base : 0ull, nr = r0 + hist[NBUCKET];
    for (unsigned long long r = r0 + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; r < nr;
         r += (unsigned long long)gridDim.x * blockDim.x)
        if (bucket[r] != DROP) order[r0 + atomicAdd(&hist[bucket[r]], 1u)] = (uint32_t)r;
}

}  // namespace

int reserve_root_plan(fim_ctx *ctx, size_t root_cap) {
    FIM_TRY(fim_reserve(ctx, ctx->root_order, sizeof(uint32_t) * (root_cap ? root_cap : 1)));
    FIM_TRY(fim_reserve(ctx, ctx->root_bucket, root_cap ? root_cap : 1));
    FIM_TRY(fim_reserve(ctx, ctx->root_hist, sizeof(uint32_t) * (NBUCKET + 1)));
    return FIM_OK;
}

// (allocates nothing: it may run inside a stream capture once
// reserve_root_plan has sized the buffers)
int launch_root_plan(fim_ctx *ctx, MineCounters *d_ctr, size_t root_cap, const DbDesc *d_dbs, int mode,
                     RootWindow *win, cudaStream_t st) {
    if (mode == 2 && !ctx->has_weights) return FIM_E_STATE;
    FIM_CUDA_TRY(cudaMemsetAsync(ctx->root_hist.p, 0, sizeof(uint32_t) * (NBUCKET + 1), st));
    const uint32_t *roots = ctx->roots.as<uint32_t>();
    RootView v{};
    v.pairbits = ctx->pairbits.as<uint32_t>();
    v.pair_cnt = ctx->pair_cnt.as<int>();
    v.item_sup = ctx->item_sup.as<uint32_t>();
    v.perm = ctx->perm.as<int32_t>();
    if (!d_dbs) {
        v.mf = ctx->mfreq;
        v.mpw = (int)ceil_div64(v.mf, 32);
        v.n = ctx->n;
        v.nw = ctx->nw;
        v.thr = ctx->cur_thr;
    }
    // the root count is known only on the device: a grid-stride loop over at
    // most the capacity, with a grid of a few CTAs per SM
    int64_t grid = ceil_div64((int64_t)(root_cap ? root_cap : 1), 256);
    const int64_t resident = (int64_t)(ctx->num_sms > 0 ? ctx->num_sms : 1) * 8;
    if (grid > resident) grid = resident;
    ctx->launches += 3;
    root_plan_kernel<<<(unsigned)grid, 256, 0, st>>>(roots, roots + root_cap, roots + 2 * root_cap,
                                           d_dbs ? roots + 3 * root_cap : nullptr, d_ctr, win, d_dbs, v, mode,
                                           ctx->mlp_wbf.as<__nv_bfloat16>(), ctx->root_bucket.as<uint8_t>(),
                                           ctx->root_hist.as<uint32_t>());
    root_plan_scan_kernel<<<1, 32, 0, st>>>(ctx->root_hist.as<uint32_t>(), d_ctr, win);
    root_plan_scatter_kernel<<<(unsigned)grid, 256, 0, st>>>(ctx->root_bucket.as<uint8_t>(), ctx->root_hist.as<uint32_t>(),
                                                   win, ctx->root_order.as<uint32_t>());
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

extern "C" {

int fim_sched_load_weights(fim_ctx *ctx, const float *weights, size_t n_params) {
    FIM_NVTX("fim_sched_load_weights");
    if (!ctx || !weights || n_params != (size_t)P) return FIM_E_INVAL;
    FIM_TRY(fim_reserve(ctx, ctx->mlp_w32, sizeof(float) * P));
    FIM_TRY(fim_reserve(ctx, ctx->mlp_wbf, sizeof(__nv_bfloat16) * P));
    FIM_CUDA_TRY(cudaMemcpyAsync(ctx->mlp_w32.p, weights, sizeof(float) * P, cudaMemcpyHostToDevice, ctx->stream));
    ctx->launches++;
    to_bf16_kernel<<<(P + 255) / 256, 256, 0, ctx->stream>>>(ctx->mlp_w32.as<float>(),
                                                              ctx->mlp_wbf.as<__nv_bfloat16>());
    FIM_CUDA_TRY(cudaGetLastError());
    FIM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    ctx->has_weights = true;
    return FIM_OK;
}

int fim_fetch_traces(fim_ctx *ctx, uint64_t *n_rows, float *features, float *targets, uint64_t cap) {
    FIM_NVTX("fim_fetch_traces");
    if (!ctx || !n_rows) return FIM_E_INVAL;
    if (!ctx->mined || !(ctx->mflags & FIM_TRACE)) return FIM_E_STATE;
    unsigned long long n = ctx->host_ctr.n_traces;
    if (n > ctx->trace_cap) n = ctx->trace_cap;
    *n_rows = n;
    if (!features && !targets) return FIM_OK;
    if (!features || !targets) return FIM_E_INVAL;
    if (cap < n) return FIM_E_TOO_SMALL;
    if (n) {
        FIM_CUDA_TRY(cudaMemcpyAsync(features, ctx->trace_x.p, sizeof(float) * FIM_MLP_FEATURES * n,
                                     cudaMemcpyDeviceToHost, ctx->stream));
        FIM_CUDA_TRY(cudaMemcpyAsync(targets, ctx->trace_y.p, sizeof(float) * 2 * n, cudaMemcpyDeviceToHost,
                                     ctx->stream));
        FIM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    return FIM_OK;
}

int fim_mlp_forward(fim_ctx *ctx, const float *params, const float *x, int64_t B, float *y, float *cache,
                    int bf16) {
    FIM_NVTX("fim_mlp_forward");
    if (!ctx || !params || !x || !y || B < 0) return FIM_E_INVAL;
    if (B == 0) return FIM_OK;
    ctx->launches++;
    mlp_forward_kernel<<<(unsigned)ceil_div64(B, 128), 128, 0, ctx->stream>>>(params, x, B, y, cache, bf16 ? 1 : 0);
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

int fim_mlp_backward(fim_ctx *ctx, const float *params, const float *x, const float *y, const float *t,
                     const float *cache, int64_t B, float *grad, float *loss_out, int bf16) {
    FIM_NVTX("fim_mlp_backward");
    if (!ctx || !params || !x || !y || !t || !cache || !grad || B <= 0) return FIM_E_INVAL;
    const int nb = (int)ceil_div64(B, 128);
    const int nchunks = (int)ceil_div64(B, GCHUNK);
    FIM_TRY(fim_reserve(ctx, ctx->mlp_scratch, sizeof(float) * ((size_t)nchunks * P + nb + 1)));
    float *part = ctx->mlp_scratch.as<float>();
    float *loss_parts = part + (size_t)nchunks * P;
    float *loss = loss_parts + nb;
    const int bf = bf16 ? 1 : 0;
    ctx->launches += 3;
    mlp_backward_sample_kernel<<<nb, 128, 0, ctx->stream>>>(params, y, t, const_cast<float *>(cache), B, loss_parts, bf);
    mlp_grad_partial_kernel<<<nchunks, 256, 0, ctx->stream>>>(x, y, t, cache, B, part, bf);
    mlp_grad_sum_kernel<<<(P + 1 + 255) / 256, 256, 0, ctx->stream>>>(part, nchunks, grad, loss_parts, nb, loss);
    FIM_CUDA_TRY(cudaGetLastError());
    if (loss_out) {
        FIM_CUDA_TRY(cudaMemcpyAsync(loss_out, loss, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        FIM_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        *loss_out /= (float)B;
    }
    return FIM_OK;
}

int fim_mlp_adam(fim_ctx *ctx, float *params, const float *grad, float *m, float *v, int step, float lr,
                 float beta1, float beta2, float eps) {
    FIM_NVTX("fim_mlp_adam");
    if (!ctx || !params || !grad || !m || !v || step < 1) return FIM_E_INVAL;
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    ctx->launches++;
    mlp_adam_kernel<<<(P + 255) / 256, 256, 0, ctx->stream>>>(params, grad, m, v, lr, beta1, beta2, eps, c1, c2);
    FIM_CUDA_TRY(cudaGetLastError());
    return FIM_OK;
}

}  // extern "C"
