// Measured arithmetic peaks of the device, the denominators of the
// rooflines of the ALU-bound kernels (the moments' double-word folds and
// streaming, the solver, the FP32 sweep), and the rate of the warp-level
// TF32 tensor instruction.  Each probe is a kernel of independent dependency chains
// of one instruction (enough chains per thread and warps per SM to keep the
// pipe full), timed with CUDA events, best of five; the chains' results
// feed a store the compiler cannot drop.  Every loop has a fixed trip count.
#include <cuda_runtime.h>

#include "klr_common.cuh"

namespace klr {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;    // independent chains per thread
constexpr int kProbeUnroll = 16;   // chain steps per loop trip

__global__ void __launch_bounds__(kProbeThreads) probe_ffma_kernel(float* out, int iters, float b,
                                                                   float c) {
    float a[kProbeChains];
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) a[i] = 1e-3f * (float)(threadIdx.x + i);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int s = 0; s < kProbeUnroll; ++s)
#pragma unroll
            for (int i = 0; i < kProbeChains; ++i) a[i] = fmaf(a[i], b, c);
    }
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) sum += a[i];
    if (sum == -1.f) out[blockIdx.x] = sum;   // never true for these inputs
}

__global__ void __launch_bounds__(kProbeThreads) probe_ffma2_kernel(float* out, int iters, float b,
                                                                    float c) {
    f2p a[kProbeChains];
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i)
        a[i] = f2p_make(1e-3f * (float)(threadIdx.x + i), 2e-3f * (float)(threadIdx.x + i));
    const f2p bb = f2p_make(b, b), cc = f2p_make(c, c);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int s = 0; s < kProbeUnroll; ++s)
#pragma unroll
            for (int i = 0; i < kProbeChains; ++i)
                asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(bb), "l"(cc));
    }
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) {
        const float2 v = f2p_get(a[i]);
        sum += v.x + v.y;
    }
    if (sum == -1.f) out[blockIdx.x] = sum;
}

__global__ void __launch_bounds__(kProbeThreads) probe_dfma_kernel(double* out, int iters, double b,
                                                                   double c) {
    double a[kProbeChains];
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) a[i] = 1e-3 * (double)(threadIdx.x + i);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int s = 0; s < kProbeUnroll; ++s)
#pragma unroll
            for (int i = 0; i < kProbeChains; ++i) a[i] = fma(a[i], b, c);
    }
    double sum = 0.0;
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) sum += a[i];
    if (sum == -1.0) out[blockIdx.x] = sum;
}

// MUFU reciprocal: x -> 1/(x + c) keeps every chain in [1/2, 2]; the add (on
// the FP32 pipe, 8 times the reciprocal rate) keeps the assembler from
// cancelling a reciprocal of a reciprocal
__global__ void __launch_bounds__(kProbeThreads) probe_rcp_kernel(float* out, int iters, float c) {
    float a[kProbeChains];
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) a[i] = 1.f + 1e-3f * (float)(threadIdx.x + i);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int s = 0; s < kProbeUnroll; ++s)
#pragma unroll
            for (int i = 0; i < kProbeChains; ++i)
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(a[i]) : "f"(a[i] + c));
    }
    float sum = 0.f;
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) sum += a[i];
    if (sum == -1.f) out[blockIdx.x] = sum;
}

// TF32 mma.sync.m16n8k8 (the warp-level tensor path): four independent
// accumulator tiles per warp, the operands fixed small values, 2 * 16 * 8 * 8
// flop per instruction
__global__ void __launch_bounds__(kProbeThreads) probe_mma_tf32_kernel(float* out, int iters) {
    constexpr int NT = 4;
    float d[NT][4];
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int i = 0; i < 4; ++i) d[t][i] = 0.f;
    const uint32_t av = __float_as_uint(1e-6f * (float)(threadIdx.x & 7)) & 0xffffe000u;
    const uint32_t bv = __float_as_uint(1e-6f) & 0xffffe000u;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int t = 0; t < NT; ++t)
                asm volatile(
                    "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
                    "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
                    : "+f"(d[t][0]), "+f"(d[t][1]), "+f"(d[t][2]), "+f"(d[t][3])
                    : "r"(av), "r"(av), "r"(av), "r"(av), "r"(bv), "r"(bv));
    }
    float sum = 0.f;
#pragma unroll
    for (int t = 0; t < NT; ++t) sum += d[t][0] + d[t][1] + d[t][2] + d[t][3];
    if (sum == -1.f) out[blockIdx.x] = sum;
}

// best of `reps` timed launches of launch() after one untimed one, in ms
template <typename F>
klr_status time_best(cudaStream_t stream, int reps, F launch, float* best_ms) {
    cudaEvent_t a, b;
    KLR_CHECK_CUDA(cudaEventCreate(&a));
    KLR_CHECK_CUDA(cudaEventCreate(&b));
    launch();
    float best = 3.4e38f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(a, stream);
        launch();
        cudaEventRecord(b, stream);
        if (cudaEventSynchronize(b) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms > 0.f && ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (err != cudaSuccess) {
        set_error("peak probe: %s", cudaGetErrorString(err));
        return KLR_ECUDA;
    }
    *best_ms = best;
    return KLR_OK;
}

}  // namespace
}  // namespace klr

using namespace klr;

extern "C" {

klr_status klr_probe_peaks(klr_ctx* ctx, klr_peaks* out, void* stream_) {
    KLR_REQUIRE(ctx, "klr_probe_peaks: NULL context");
    KLR_REQUIRE(out, "klr_probe_peaks: NULL output");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    KLR_CHECK_CUDA(cudaSetDevice(c->device));
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    KLR_CHECK_CUDA(cudaStreamIsCapturing(stream, &cap));
    KLR_REQUIRE(cap == cudaStreamCaptureStatusNone, "klr_probe_peaks: stream is capturing");
    const int blocks = c->n_sm * 8;                 // 64 warps per SM
    const double threads = (double)blocks * kProbeThreads;
    const double steps = (double)kProbeUnroll * kProbeChains;
    void* sink = nullptr;
    KLR_CHECK_CUDA(cudaMalloc(&sink, sizeof(double) * blocks));
    klr_status st = KLR_OK;
    float ms = 0.f;
    const int it32 = 2048, it64 = 64, itr = 256, itm = 2048;
    do {
        st = time_best(stream, 5, [&] {
            probe_ffma_kernel<<<blocks, kProbeThreads, 0, stream>>>((float*)sink, it32, 0.999999f, 1e-6f);
        }, &ms);
        if (st != KLR_OK) break;
        out->fp32_fma_tflops = 2.0 * threads * steps * it32 / (ms * 1e-3) * 1e-12;
        st = time_best(stream, 5, [&] {
            probe_ffma2_kernel<<<blocks, kProbeThreads, 0, stream>>>((float*)sink, it32, 0.999999f, 1e-6f);
        }, &ms);
        if (st != KLR_OK) break;
        out->fp32x2_fma_tflops = 4.0 * threads * steps * it32 / (ms * 1e-3) * 1e-12;
        st = time_best(stream, 5, [&] {
            probe_dfma_kernel<<<blocks, kProbeThreads, 0, stream>>>((double*)sink, it64, 0.999999, 1e-6);
        }, &ms);
        if (st != KLR_OK) break;
        out->fp64_fma_tflops = 2.0 * threads * steps * it64 / (ms * 1e-3) * 1e-12;
        st = time_best(stream, 5, [&] {
            probe_rcp_kernel<<<blocks, kProbeThreads, 0, stream>>>((float*)sink, itr, 1e-7f);
        }, &ms);
        if (st != KLR_OK) break;
        out->mufu_rcp_tops = threads * steps * itr / (ms * 1e-3) * 1e-12;
        st = time_best(stream, 5, [&] {
            probe_mma_tf32_kernel<<<blocks, kProbeThreads, 0, stream>>>((float*)sink, itm);
        }, &ms);
        if (st != KLR_OK) break;
        out->tf32_mma_sync_tflops =
            2.0 * 16 * 8 * 8 * 16.0 * (threads / 32.0) * itm / (ms * 1e-3) * 1e-12;
    } while (false);
    cudaFree(sink);
    return st;
}

}  // extern "C"
