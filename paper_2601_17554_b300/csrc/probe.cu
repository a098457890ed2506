// Unit-rate probes: the measured peaks that the attention roofline divides by
// (the MUFU base-2 exponential and the FP32 FMA pipe), taken on the device in
// use rather than quoted from a datasheet.  Each thread runs eight independent
// dependency chains so that throughput, not latency, limits the loop.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace mlpf {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_probe_ex2(float* out, float seed) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = seed * (float)(threadIdx.x + i) * 1e-6f;
    for (int n = 0; n < kIters; ++n) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[i]));
            x[i] = -0.5f * y;   // stays in [-0.5, 0]: 2^x in [0.7, 1]
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

// packed BF16 exponentials (ex2.approx.ftz.bf16x2): two results per instruction
__global__ void __launch_bounds__(kThreads) k_probe_ex2_bf16x2(float* out, float seed) {
    uint32_t x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        const float v = -seed * (float)(threadIdx.x + i) * 1e-6f;
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(x[i]) : "f"(v), "f"(v * 0.5f));
    }
    const uint32_t neg_half = 0xBF00BF00u;   // (-0.5, -0.5) in BF16
    const uint32_t zero = 0u;
    for (int n = 0; n < kIters; ++n) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            uint32_t y;
            asm volatile("ex2.approx.ftz.bf16x2 %0, %1;" : "=r"(y) : "r"(x[i]));
            asm volatile("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(x[i]) : "r"(y), "r"(neg_half), "r"(zero));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += __uint_as_float(x[i] << 16) + __uint_as_float(x[i] & 0xffff0000u);
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_probe_ffma(float* out, float seed) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = seed * (float)(threadIdx.x + i) * 1e-6f;
    const float a = 0.999f, b = 1e-3f;
    for (int n = 0; n < kIters; ++n) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[i]) : "f"(a), "f"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    out[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace
}  // namespace mlpf

using namespace mlpf;

static mlpf_status measure(int32_t device, double* ex2_per_s, double* ffma_per_s, double* ex2_bf16x2_per_s);

extern "C" mlpf_status mlpf_measure_unit_rates(int32_t device, double* ex2_per_s, double* ffma_per_s) {
    if (!ex2_per_s && !ffma_per_s) { set_error("no output requested"); return MLPF_E_INVALID; }
    return measure(device, ex2_per_s, ffma_per_s, nullptr);
}

extern "C" mlpf_status mlpf_measure_ex2_packed_rate(int32_t device, double* results_per_s) {
    if (!results_per_s) { set_error("no output requested"); return MLPF_E_INVALID; }
    return measure(device, nullptr, nullptr, results_per_s);
}

static mlpf_status measure(int32_t device, double* ex2_per_s, double* ffma_per_s, double* ex2_bf16x2_per_s) {
    if (cudaSetDevice(device) != cudaSuccess) { set_error("cudaSetDevice failed"); return MLPF_E_CUDA; }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) {
        set_error("cannot read the SM count");
        return MLPF_E_CUDA;
    }
    const int blocks = sms * 8;
    float* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mlpf_status rc = MLPF_OK;
    if (cudaMalloc(&out, sizeof(float) * blocks * kThreads) != cudaSuccess) { set_error("probe allocation failed"); return MLPF_E_OOM; }
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        set_error("probe stream/event creation failed");
        rc = MLPF_E_CUDA;
    }
    for (int kind = 0; kind < 3 && rc == MLPF_OK; ++kind) {
        double* dst = kind == 0 ? ex2_per_s : kind == 1 ? ffma_per_s : ex2_bf16x2_per_s;
        if (!dst) continue;
        float best = 1e30f;
        for (int rep = 0; rep < 4 && rc == MLPF_OK; ++rep) {   // the first run warms up
            cudaEventRecord(e0, st);
            if (kind == 0) k_probe_ex2<<<blocks, kThreads, 0, st>>>(out, 1.f);
            else if (kind == 1) k_probe_ffma<<<blocks, kThreads, 0, st>>>(out, 1.f);
            else k_probe_ex2_bf16x2<<<blocks, kThreads, 0, st>>>(out, 1.f);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) { set_error("probe kernel failed"); rc = MLPF_E_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = std::min(best, ms);
        }
        // results per second (two per packed instruction)
        if (rc == MLPF_OK) *dst = (double)blocks * kThreads * kIters * kChains * (kind == 2 ? 2 : 1) / (best * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    return rc;
}
