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

// ---- tcgen05 kind::f8f6f4 MMA rate -----------------------------------------
// One CTA per SM (the dynamic shared memory keeps a second one off), the
// pair pass's instruction shape: 128 x 256 x 32 e4m3 with an f32 accumulator
// in tensor memory, A either from tensor memory (the pair pass's off-diagonal
// tiles) or from a SWIZZLE_128B shared-memory tile (its diagonal tiles).  One
// elected thread issues `iters` MMAs back to back; the launch's time gives the
// dense rate the pair pass can reach.
constexpr int MP_THREADS = 128;
constexpr int MP_M = 128, MP_N = 256, MP_K = 32;
constexpr uint32_t MP_TMEM_COLS = 512;  // accumulator [0, 256), A at 256
constexpr unsigned long long MP_WAIT_NS = 2000000000ull;

struct __align__(1024) MmaProbeSmem {
    uint8_t b[MP_N * 128];  // 256 rows x 128 bytes (K = 128 e4m3), SWIZZLE_128B
    uint8_t a[MP_M * 128];
    uint64_t done;
    uint32_t tmem_base;
};

__device__ __forceinline__ uint32_t mp_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t mp_sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

__global__ void __launch_bounds__(MP_THREADS, 1)
mma_probe_kernel(int iters, int a_in_tmem, int n_cols, int *__restrict__ err) {
    extern __shared__ uint8_t raw[];
    MmaProbeSmem &s = *reinterpret_cast<MmaProbeSmem *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5;
    // operands: e4m3 2.0 in every other byte (the pair pass's 0/2 values)
    for (int i = threadIdx.x; i < (int)(sizeof(s.b) / 16); i += MP_THREADS)
        reinterpret_cast<uint4 *>(s.b)[i] = make_uint4(0x00400040u, 0x40000040u, 0x00404000u, 0x40400000u);
    for (int i = threadIdx.x; i < (int)(sizeof(s.a) / 16); i += MP_THREADS)
        reinterpret_cast<uint4 *>(s.a)[i] = make_uint4(0x40004000u, 0x00400040u, 0x40400000u, 0x00004040u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mp_smem(&s.done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(mp_smem(&s.tmem_base)),
                     "r"(MP_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s.tmem_base;
    const uint32_t a_col = MP_N;
    if (a_in_tmem) {  // each thread writes its row (lane) of A: 32 columns
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + a_col;
        const uint32_t v = 0x40004000u ^ (threadIdx.x & 1u ? 0x40404040u : 0u);
#pragma unroll
        for (int q = 0; q < 4; q++)
            asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr + 8u * q),
                         "r"(v)
                         : "memory");
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x == 0) {
        const uint32_t idesc = (1u << 4) | ((uint32_t)(n_cols >> 3) << 17) | ((uint32_t)(MP_M >> 4) << 24);
        const uint32_t b0 = mp_smem(s.b), a0 = mp_smem(s.a);
        for (int i = 0; i < iters; i++) {
            const uint32_t kk = (uint32_t)(i & 3), acc = i > 0 ? 1u : 0u;
            if (a_in_tmem)
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem),
                    "r"(tmem + a_col + 8u * kk), "l"(mp_sdesc(b0 + kk * 32)), "r"(idesc), "r"(acc)
                    : "memory");
            else
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(mp_sdesc(a0 + kk * 32)), "l"(mp_sdesc(b0 + kk * 32)), "r"(idesc), "r"(acc)
                    : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         mp_smem(&s.done))
                     : "memory");
        // bounded wait for the last MMA before the tensor memory is freed
        const unsigned long long t0 = globaltimer_ns();
        uint32_t ok = 0;
        while (!ok) {
            asm volatile(
                "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\nselp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok)
                : "r"(mp_smem(&s.done))
                : "memory");
            if (!ok && globaltimer_ns() - t0 > MP_WAIT_NS) {
                atomicExch(err, FIM_E_TIMEOUT);
                break;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MP_TMEM_COLS)
                     : "memory");
    }
}

}  // namespace

extern "C" {

int fim_probe(fim_ctx *ctx, int which, double *result) {
    FIM_NVTX("fim_probe");
    if (!ctx || !result || which < 0 || which > 5) return FIM_E_INVAL;
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
    const size_t mp_smem_bytes = sizeof(MmaProbeSmem) + 1024 + (64u << 10);  // > half an SM: one CTA each
    if (which >= 2) {
        FIM_CUDA_TRY(cudaFuncSetAttribute(mma_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)mp_smem_bytes));
        FIM_CUDA_TRY(cudaMemsetAsync(sink, 0, sizeof(int), st));
    }
    for (int rep = 0; rep < 2; rep++) {  // the first run warms up, the second is timed
        cudaEventRecord(ctx->ev[5], st);
        if (which >= 2) {
            // 2 x 128 x 256 x 32 flops per MMA; about 0.6 ms at the nominal rate
            const int iters = 8192;
            const int nsm = ctx->num_sms > 0 ? ctx->num_sms : 1;
            const size_t smem = mp_smem_bytes;
            ctx->launches++;
            // which 2, 3: N = 256 with A in tensor / shared memory; 4, 5: N = 128,
            // 64 with A in shared memory (the batched pair pass's small tiles)
            const int n_cols = which == 4 ? 128 : which == 5 ? 64 : MP_N;
            mma_probe_kernel<<<(unsigned)nsm, MP_THREADS, smem, st>>>(iters, which == 2 ? 1 : 0, n_cols,
                                                                    reinterpret_cast<int *>(sink));
            work = 2.0 * MP_M * n_cols * MP_K * (double)iters * nsm;  // flops
        } else if (which == 0) {
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
    if (which >= 2) {
        int e = 0;
        FIM_CUDA_TRY(cudaMemcpy(&e, sink, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) return e;
        *result = work / (ms * 1e-3) / 1e12;  // TFLOP/s
        return FIM_OK;
    }
    *result = which == 0 ? work / (ms * 1e-3) : work / (ms * 1e-3) / 1e9;
    return FIM_OK;
}

}  // extern "C"
