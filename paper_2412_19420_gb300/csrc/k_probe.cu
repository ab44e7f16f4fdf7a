// k_probe.cu -- measurement probes for the rooflines of the counting kernels.
//
// The AND/popc work of the pair and prefix-extension passes is one LOP3, one
// POPC and one IADD per 32-bit word pair; whether a pass can be ALU-bound
// depends on the POPC issue rate of the GPU, which is measured here rather
// than assumed.  The small workloads' operands live in L2, so their roofline
// is the L2 read bandwidth, also measured here.
#include "fim_common.cuh"

namespace {

constexpr int PROBE_T = 256;
constexpr int CHAINS = 8;  // independent accumulation chains per thread

// Every thread runs CHAINS independent (a & b ^ c) -> popc -> add chains for
// iters rounds; the operands change every round so nothing is hoisted.
__global__ void __launch_bounds__(PROBE_T)
popc_probe_kernel(uint32_t seed, int iters, unsigned long long *__restrict__ sink) {
    uint32_t a[CHAINS], acc[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) {
        a[c] = seed * (threadIdx.x + 1u) + 0x9E3779B9u * (uint32_t)(c + 1) + blockIdx.x;
        acc[c] = 0;
    }
    uint32_t b = seed ^ blockIdx.x, d = ~seed + threadIdx.x;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) {
            const uint32_t x = (a[c] & b) ^ d;  // one LOP3
            acc[c] += __popc(x);                // one POPC, one IADD
            a[c] += acc[c];                     // keeps the chain dependent
        }
        b = b * 1664525u + 1013904223u;
    }
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += acc[c];
    if (s == 0x7FFFFFFFu) atomicAdd(sink, 1ull);  // practically never: keeps the work live
}

// Reads a buffer that fits in L2 over and over, 16 bytes per load.
__global__ void __launch_bounds__(PROBE_T)
l2_probe_kernel(const uint4 *__restrict__ buf, unsigned long long n16, int reps,
                unsigned long long *__restrict__ sink) {
    uint32_t x = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * PROBE_T;
    for (int r = 0; r < reps; r++)
        for (unsigned long long i = (unsigned long long)blockIdx.x * PROBE_T + threadIdx.x; i < n16; i += stride) {
            const uint4 v = __ldcg(buf + i);
            x ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (x == 0x12345678u) atomicAdd(sink, 1ull);
}

}  // namespace

extern "C" {

int fim_probe(fim_ctx *ctx, int which, double *result) {
    FIM_NVTX("fim_probe");
    if (!ctx || !result || which < 0 || which > 1) return FIM_E_INVAL;
    *result = 0.0;
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FIM_E_CUDA;
    struct Restore { int d; ~Restore() { if (d >= 0) cudaSetDevice(d); } } restore{dev_prev};
    cudaStream_t st = ctx->stream;
    FIM_TRY(fim_reserve(ctx, ctx->probe_buf, 64u << 20));
    unsigned long long *sink = ctx->probe_buf.as<unsigned long long>();
    const unsigned grid = (unsigned)(ctx->num_sms > 0 ? ctx->num_sms : 1) * 8u;  // 2,048 threads per SM
    float ms = 0.f;
    double work = 0.0;
    for (int rep = 0; rep < 2; rep++) {  // the first run warms up, the second is timed
        cudaEventRecord(ctx->ev[5], st);
        if (which == 0) {
            const int iters = 4096;
            ctx->launches++;
            popc_probe_kernel<<<grid, PROBE_T, 0, st>>>(0x2545F491u + rep, iters, sink);
            work = (double)grid * PROBE_T * iters * CHAINS;  // word pairs (LOP3 + POPC + IADD each)
        } else {
            // 32 MB after the 64-byte sink: well inside the 126 MB L2
            const unsigned long long n16 = (32ull << 20) / 16;
            const int reps = 20;
            ctx->launches++;
            l2_probe_kernel<<<grid, PROBE_T, 0, st>>>(reinterpret_cast<const uint4 *>(ctx->probe_buf.as<char>() + 64),
                                                      n16, reps, sink);
            work = (double)n16 * 16.0 * reps;  // bytes read
        }
        cudaEventRecord(ctx->ev[6], st);
        FIM_CUDA_TRY(cudaGetLastError());
        FIM_CUDA_TRY(cudaEventSynchronize(ctx->ev[6]));
        cudaEventElapsedTime(&ms, ctx->ev[5], ctx->ev[6]);
    }
    if (ms <= 0.f) return FIM_E_CUDA;
    *result = which == 0 ? work / (ms * 1e-3) : work / (ms * 1e-3) / 1e9;
    return FIM_OK;
}

}  // extern "C"
