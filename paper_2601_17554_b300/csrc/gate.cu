// Student inference with per-event fallback to the full model: the student
// runs on every event; events whose per-element class confidence (max softmax),
// averaged or minimised over the event (MLPF_OPT_GATE_CONFIDENCE), is below a
// threshold are compacted into a new packed batch, run through the full
// (teacher) model and scattered back.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "internal.h"

namespace mlpf {
namespace {

// conf[e] = mean (mode 0) or minimum (mode 1) over the event's elements of the
// max softmax of the class scores; flag[e] = conf < thr
__global__ void __launch_bounds__(256) k_event_confidence(const int32_t* __restrict__ cu,
                                                          const float* __restrict__ logits, float thr,
                                                          int mode, int32_t* __restrict__ flag,
                                                          float* __restrict__ conf) {
    __shared__ float part[8];
    const int e = blockIdx.x;
    const int s = cu[e], t = cu[e + 1];
    float acc = mode == 1 ? 1.f : 0.f;
    for (int r = s + threadIdx.x; r < t; r += 256) {
        const float* l = logits + (size_t)r * 6;
        float m = l[0];
        for (int c = 1; c < 6; ++c) m = fmaxf(m, l[c]);
        float z = 0.f;
        for (int c = 0; c < 6; ++c) z += expf(l[c] - m);
        const float pmax = 1.f / z;   // max softmax = exp(m - m) / z
        acc = mode == 1 ? fminf(acc, pmax) : acc + pmax;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const float v = __shfl_xor_sync(0xffffffffu, acc, o);
        acc = mode == 1 ? fminf(acc, v) : acc + v;
    }
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = mode == 1 ? 1.f : 0.f;
        for (int i = 0; i < 8; ++i) a = mode == 1 ? fminf(a, part[i]) : a + part[i];
        const float cf = t <= s ? 1.f : (mode == 1 ? a : a / (float)(t - s));
        conf[e] = cf;
        flag[e] = cf < thr ? 1 : 0;
    }
}

// One CTA: sub_cu (packed offsets of the flagged events), src_event[i] (event of
// the i-th flagged one), meta = {n_sub, total_sub, max_n_sub}.
__global__ void __launch_bounds__(1024) k_compact_events(const int32_t* __restrict__ cu, const int32_t* __restrict__ flag,
                                                         int n_events, int32_t* __restrict__ sub_cu,
                                                         int32_t* __restrict__ src_event, int32_t* __restrict__ meta) {
    __shared__ int wsum[32], wcnt[32];
    __shared__ int carry_n, carry_t, maxn;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) { carry_n = 0; carry_t = 0; maxn = 0; sub_cu[0] = 0; }
    __syncthreads();
    for (int base = 0; base < n_events; base += 1024) {
        const int e = base + tid;
        const int f = e < n_events ? flag[e] : 0;
        const int n = f ? cu[e + 1] - cu[e] : 0;
        int ic = f, it = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, ic, o), b = __shfl_up_sync(0xffffffffu, it, o);
            if (lane >= o) { ic += a; it += b; }
        }
        if (lane == 31) { wcnt[wid] = ic; wsum[wid] = it; }
        __syncthreads();
        if (wid == 0) {
            int a = wcnt[lane], b = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, a, o), y = __shfl_up_sync(0xffffffffu, b, o);
                if (lane >= o) { a += x; b += y; }
            }
            wcnt[lane] = a;
            wsum[lane] = b;
        }
        __syncthreads();
        const int pre_c = carry_n + ic - f + (wid > 0 ? wcnt[wid - 1] : 0);
        const int pre_t = carry_t + it - n + (wid > 0 ? wsum[wid - 1] : 0);
        if (f) {
            src_event[pre_c] = e;
            sub_cu[pre_c + 1] = pre_t + n;
            atomicMax(&maxn, n);
        }
        __syncthreads();
        if (tid == 1023) { carry_n = pre_c + f; carry_t = pre_t + n; }
        __syncthreads();
    }
    if (tid == 0) {
        meta[0] = carry_n;
        meta[1] = carry_t;
        meta[2] = maxn;
    }
}

// Copy the rows of the flagged events: dir 0 gathers x into the sub-batch, dir 1
// scatters the teacher's logits/reg back.  One CTA per flagged event.
__global__ void k_move_rows(const int32_t* __restrict__ cu, const int32_t* __restrict__ sub_cu,
                            const int32_t* __restrict__ src_event, const float* __restrict__ x,
                            float* __restrict__ sub_x, const float* __restrict__ sub_lo,
                            const float* __restrict__ sub_rg, float* __restrict__ lo, float* __restrict__ rg,
                            int dir) {
    const int i = blockIdx.x;
    const int e = src_event[i];
    const int s = cu[e], n = cu[e + 1] - s, s2 = sub_cu[i];
    if (dir == 0) {
        for (int k = threadIdx.x; k < n * 42; k += blockDim.x) sub_x[(size_t)s2 * 42 + k] = x[(size_t)s * 42 + k];
    } else {
        for (int k = threadIdx.x; k < n * 6; k += blockDim.x) lo[(size_t)s * 6 + k] = sub_lo[(size_t)s2 * 6 + k];
        for (int k = threadIdx.x; k < n * 5; k += blockDim.x) rg[(size_t)s * 5 + k] = sub_rg[(size_t)s2 * 5 + k];
    }
}

}  // namespace
}  // namespace mlpf

using namespace mlpf;

struct mlpf_model {
    Model impl;
};

extern "C" mlpf_status mlpf_forward_gated(mlpf_model* student, mlpf_model* teacher, float threshold,
                                          int32_t student_precision, int32_t teacher_precision,
                                          const float* x, const int32_t* cu_seqlens, int32_t n_events,
                                          int32_t total, int32_t max_n, float* logits, float* reg,
                                          int32_t* cls, double* event_sums, int32_t* used_teacher,
                                          int32_t* n_fallback, void* stream) {
    if (!student || !teacher) { set_error("NULL model"); return MLPF_E_INVALID; }
    Model& sm = student->impl;
    if (sm.device != teacher->impl.device) { set_error("student and teacher on different devices"); return MLPF_E_INVALID; }
    if (sm.cfg.arch != teacher->impl.cfg.arch) {
        set_error("student and teacher must share the class-score layout (arch)");
        return MLPF_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    mlpf_status s = mlpf_forward(student, student_precision, x, cu_seqlens, n_events, total, max_n, logits, reg,
                                 nullptr, nullptr, stream);
    if (s != MLPF_OK) return s;
    if (n_fallback) *n_fallback = 0;
    if (total == 0 || n_events == 0) {
        if (event_sums && n_events > 0) cudaMemsetAsync(event_sums, 0, (size_t)n_events * 24, st);
        return MLPF_OK;
    }
    // gate buffers (owned by the student model, grown outside any capture)
    auto& gb = sm.gate;
    if ((size_t)total > gb.cap_total || (size_t)n_events > gb.cap_events) {
        if (gb.base) cudaFree(gb.base);
        gb = Model::Gate{};
        gb.cap_total = (size_t)total;
        gb.cap_events = (size_t)n_events;
        const size_t bytes = gb.cap_total * (42 + 6 + 5) * 4 + (gb.cap_events + 1) * 4 * 4 + 64 + 4096;
        if (cudaMalloc(&gb.base, bytes) != cudaSuccess) {
            gb = Model::Gate{};
            set_error("gate buffer allocation failed");
            return MLPF_E_OOM;
        }
        char* b = (char*)gb.base;
        gb.sub_x = (float*)b;
        gb.sub_lo = gb.sub_x + gb.cap_total * 42;
        gb.sub_rg = gb.sub_lo + gb.cap_total * 6;
        int32_t* ib = (int32_t*)(gb.sub_rg + gb.cap_total * 5);
        gb.flag = ib;
        gb.sub_cu = gb.flag + gb.cap_events + 1;
        gb.src = gb.sub_cu + gb.cap_events + 1;
        gb.meta = gb.src + gb.cap_events + 1;
        gb.conf = (float*)(gb.meta + 16);
    }
    k_event_confidence<<<n_events, 256, 0, st>>>(cu_seqlens, logits, threshold, sm.gate_confidence, gb.flag,
                                                  gb.conf);
    k_compact_events<<<1, 1024, 0, st>>>(cu_seqlens, gb.flag, n_events, gb.sub_cu, gb.src, gb.meta);
    int32_t meta[3];
    if (cudaMemcpyAsync(meta, gb.meta, sizeof(meta), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("gate: reading the fallback count failed");
        return MLPF_E_CUDA;
    }
    if (n_fallback) *n_fallback = meta[0];
    if (meta[0] > 0) {
        k_move_rows<<<meta[0], 256, 0, st>>>(cu_seqlens, gb.sub_cu, gb.src, x, gb.sub_x, nullptr, nullptr,
                                             nullptr, nullptr, 0);
        s = mlpf_forward(teacher, teacher_precision, gb.sub_x, gb.sub_cu, meta[0], meta[1], meta[2], gb.sub_lo,
                         gb.sub_rg, nullptr, nullptr, stream);
        if (s != MLPF_OK) return s;
        k_move_rows<<<meta[0], 256, 0, st>>>(cu_seqlens, gb.sub_cu, gb.src, nullptr, nullptr, gb.sub_lo, gb.sub_rg,
                                             logits, reg, 1);
    }
    if (used_teacher &&
        cudaMemcpyAsync(used_teacher, gb.flag, (size_t)n_events * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        set_error("gate: copying the fallback flags failed");
        return MLPF_E_CUDA;
    }
    if (run_event_sums(sm, cu_seqlens, n_events, logits, reg, cls, event_sums, sm.cfg.n_cls, st) < 0 ||
        cudaPeekAtLastError() != cudaSuccess) {
        set_error("gate: kernel launch failed");
        return MLPF_E_CUDA;
    }
    return MLPF_OK;
}
