// peak.cu -- the measured FP32 rate that the roofline of the search kernel
// is taken against, and the measured FP64 rate for the plain FP64 join.
//
// The search kernel's distance arithmetic runs on the FP32 fused
// multiply-add pipe, in packed f32x2 instructions.  Its roofline therefore
// needs the rate at which this GPU actually retires FP32 FMAs, and whether
// the packed form raises it.  fma_rate_kernel runs independent FMA chains in
// every thread of a full-occupancy grid (eight chains per thread, enough to
// hide the pipe latency) with run-time operands, so nothing folds away; each
// thread stores its sums once at the end.  FLOPs count two per FMA lane.
#include <algorithm>
#include <cstdint>

#include "sj_internal.cuh"

namespace sj {

namespace {

constexpr int kChains = 8;

template <bool PACKED>
__global__ void __launch_bounds__(256) fma_rate_kernel(float *out, int iters, float a, float b) {
    const float seed = (float)(threadIdx.x & 7) * 1e-3f;
    if (PACKED) {
        unsigned long long acc[kChains], m, c;
        asm("mov.b64 %0, {%1, %1};" : "=l"(m) : "f"(a));
        asm("mov.b64 %0, {%1, %1};" : "=l"(c) : "f"(b));
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            const float s0 = seed + (float)k, s1 = seed - (float)k;
            asm("mov.b64 %0, {%1, %2};" : "=l"(acc[k]) : "f"(s0), "f"(s1));
        }
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[k]) : "l"(m), "l"(c));
        }
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            float x, y;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(acc[k]));
            s += x + y;
        }
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    } else {
        float acc[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = seed + (float)k;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(acc[k]) : "f"(a), "f"(b));
        }
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += acc[k];
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    }
}

// FP64 fused multiply-add chains (the plain FP64 join's pipe): the same
// structure in double precision.  GB300's FP64 rate is a small fraction of
// its FP32 rate, so the launch runs fewer iterations.
__global__ void __launch_bounds__(256) fma64_rate_kernel(double *out, int iters, double a, double b) {
    double acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (double)(threadIdx.x & 7) * 1e-3 + (double)k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k)
            asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(acc[k]) : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best of five timed launches (after one warm-up) of `launch` on stream s:
// the fastest launch's milliseconds, or a negative value when CUDA failed.
template <class F>
float best_of_five(cudaStream_t s, F launch) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = -1.0f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return -1.0f;
    }
    for (int rep = 0; rep < 6; ++rep) {
        float t = 0.0f;
        if (cudaEventRecord(e0, s) != cudaSuccess) { best = -1.0f; break; }
        launch();
        note_launch();
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            best = -1.0f;
            break;
        }
        if (rep > 0 && (best < 0.0f || t < best)) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return best;
}

}  // namespace

}  // namespace sj

using namespace sj;

extern "C" SJ_API sj_status sj_fp64_fma_rate(int device, double *tflops, double *ms) {
    if (!tflops || !ms || device < 0) return SJ_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SJ_ECUDA;
    }
    const int sms = sm_count(device);
    if (sms <= 0) return SJ_ECUDA;
    const int threads = 256, blocks = sms * 8;     // 2048 threads per SM
    const int iters = 1 << 12;
    double *out = nullptr;
    cudaStream_t s = nullptr;
    sj_status st = SJ_OK;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        st = SJ_ECUDA;
    float best = -1.0f;
    if (st == SJ_OK)
        best = best_of_five(s, [&]() { fma64_rate_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.999, 1e-3); });
    if (st == SJ_OK && best > 0.0f) {
        const double flops = 2.0 * (double)kChains * (double)iters * (double)blocks * threads;
        *ms = best;
        *tflops = flops / (best * 1e-3) / 1e12;
    } else {
        st = SJ_ECUDA;
    }
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    cudaGetLastError();
    return st;
}

extern "C" SJ_API sj_status sj_fp32_fma_rate(int device, int packed, double *tflops, double *ms) {
    if (!tflops || !ms || device < 0) return SJ_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return SJ_ECUDA;
    }
    const int sms = sm_count(device);
    if (sms <= 0) return SJ_ECUDA;
    const int threads = 256, blocks = sms * 8;     // 2048 threads per SM
    const int iters = 1 << 18;
    float *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sj_status st = SJ_OK;
    float best = 0.0f;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(float)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = SJ_ECUDA;
    }
    // one warm-up launch, then the best of five timed ones
    for (int rep = 0; rep < 6 && st == SJ_OK; ++rep) {
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = SJ_ECUDA; break; }
        if (packed)
            fma_rate_kernel<true><<<blocks, threads, 0, s>>>(out, iters, 0.999f, 1e-3f);
        else
            fma_rate_kernel<false><<<blocks, threads, 0, s>>>(out, iters, 0.999f, 1e-3f);
        note_launch();
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            st = SJ_ECUDA;
            break;
        }
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) { st = SJ_ECUDA; break; }
        if (rep > 0 && (best == 0.0f || t < best)) best = t;
    }
    if (st == SJ_OK && best > 0.0f) {
        const double lanes = packed ? 2.0 : 1.0;
        const double flops = 2.0 * lanes * (double)kChains * (double)iters * (double)blocks * threads;
        *ms = best;
        *tflops = flops / (best * 1e-3) / 1e12;
    } else if (st == SJ_OK) {
        st = SJ_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    cudaGetLastError();
    return st;
}
