// mlpf_forward_noalloc: the tensor-core forward with its scratch (the padded
// residual stream, Q/K/V/O, the block table and the attention work list) in a
// fixed file-scope device array instead of the model's cudaMalloc'd workspace.
//
// Who needs it: callers that must not allocate device memory at inference time,
// for example a framework module that runs under a memory budget owned by a
// caching allocator, or code that must not trigger a device allocation (and the
// implicit synchronisation it brings) inside its event loop.  The model itself
// (weights) is still created once by mlpf_load_weights.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"

namespace mlpf {
namespace {

constexpr int NA_MAX_TOTAL = 16384;  // elements per call
constexpr int NA_MAX_EVENTS = 64;    // events per call
constexpr int64_t NA_TPAD = ((NA_MAX_TOTAL + 64 * NA_MAX_EVENTS + 127) / 128) * 128;

constexpr size_t al(size_t v) { return (v + 1023) / 1024 * 1024; }
constexpr size_t NA_OFF_TZ = 0;
constexpr size_t NA_OFF_TQ = NA_OFF_TZ + al(NA_TPAD * 64 * 4);
constexpr size_t NA_OFF_TK = NA_OFF_TQ + al(NA_TPAD * 64 * 2);
constexpr size_t NA_OFF_TO = NA_OFF_TK + al(NA_TPAD * 64 * 2);
constexpr size_t NA_OFF_TVT = NA_OFF_TO + al(NA_TPAD * 64 * 2);
constexpr size_t NA_OFF_THP = NA_OFF_TVT + al(NA_TPAD * 64 * 2);
constexpr size_t NA_OFF_BLK = NA_OFF_THP + al(NA_TPAD * 64 * 2);
constexpr size_t NA_OFF_KMAX = NA_OFF_BLK + al((NA_TPAD / 64) * sizeof(int4));
constexpr size_t NA_OFF_ITEMS = NA_OFF_KMAX + al((NA_TPAD / 64) * 4 * sizeof(float));
constexpr size_t NA_OFF_CNT = NA_OFF_ITEMS + al((NA_TPAD / 128 + NA_MAX_EVENTS + 1) * sizeof(int4));
constexpr size_t NA_BYTES = NA_OFF_CNT + al(64 * sizeof(int));  // about 18.4 MB

}  // namespace
}  // namespace mlpf

// The scratch: one copy per GPU that loads the library, held until process exit.
static __device__ __align__(256) unsigned char g_mlpf_noalloc_scratch[mlpf::NA_BYTES];

namespace mlpf {
namespace {

struct NoallocDevice {
    bool ready = false;
    unsigned char* base = nullptr;  // device address of g_mlpf_noalloc_scratch
    CUtensorMap map_q, map_q64, map_k, map_o, map_vt, map_vt16, map_hp;   // every map the launch sequence uses
};
NoallocDevice g_na[64];
std::mutex g_na_mu;

// Workspace view of the static scratch (no allocation).
Workspace na_workspace(unsigned char* b) {
    Workspace w{};
    w.cap_total = NA_MAX_TOTAL;
    w.cap_events = NA_MAX_EVENTS;
    w.cap_tpad = NA_TPAD;
    w.base = b;
    w.bytes = NA_BYTES;
    w.tz = (float*)(b + NA_OFF_TZ);
    w.tq = (__nv_bfloat16*)(b + NA_OFF_TQ);
    w.tk = (__nv_bfloat16*)(b + NA_OFF_TK);
    w.to = (__nv_bfloat16*)(b + NA_OFF_TO);
    w.tvt = (__nv_bfloat16*)(b + NA_OFF_TVT);
    w.thp = (__nv_bfloat16*)(b + NA_OFF_THP);
    w.blk = (int4*)(b + NA_OFF_BLK);
    w.kmax = (float*)(b + NA_OFF_KMAX);
    w.items = (int4*)(b + NA_OFF_ITEMS);
    w.counters = (int*)(b + NA_OFF_CNT);
    return w;
}

}  // namespace
}  // namespace mlpf

using namespace mlpf;

extern "C" mlpf_status mlpf_forward_noalloc(mlpf_model* mm, int32_t precision, const float* x,
                                            const int32_t* cu_seqlens, int32_t n_events,
                                            int32_t total, int32_t max_n, float* logits,
                                            float* reg, int32_t* cls, double* event_sums,
                                            void* stream);

struct mlpf_model {
    Model impl;
};

extern "C" mlpf_status mlpf_forward_noalloc(mlpf_model* mm, int32_t precision, const float* x,
                                            const int32_t* cu_seqlens, int32_t n_events,
                                            int32_t total, int32_t max_n, float* logits,
                                            float* reg, int32_t* cls, double* event_sums,
                                            void* stream) {
    if (!mm) { set_error("model is NULL"); return MLPF_E_INVALID; }
    Model& m = mm->impl;
    if (precision != MLPF_BF16 && precision != MLPF_FP16) {
        set_error("mlpf_forward_noalloc runs the BF16 and FP16 tensor-core precisions only");
        return MLPF_E_UNSUPPORTED;
    }
    if (m.attn_window > 0) {
        set_error("mlpf_forward_noalloc has no scratch for windowed attention");
        return MLPF_E_UNSUPPORTED;
    }
    if (!m.tc_supported) {
        set_error("tensor-core path is built for d=64, 4 heads, FFN 256 models only");
        return MLPF_E_UNSUPPORTED;
    }
    if (n_events < 0 || total < 0 || max_n < 0 || max_n > 65536) { set_error("bad size"); return MLPF_E_INVALID; }
    if (total > NA_MAX_TOTAL || n_events > NA_MAX_EVENTS) {
        set_error("mlpf_forward_noalloc takes at most " + std::to_string(NA_MAX_TOTAL) + " elements and " +
                  std::to_string(NA_MAX_EVENTS) + " events per call (got " + std::to_string(total) +
                  " and " + std::to_string(n_events) + ")");
        return MLPF_E_INVALID;
    }
    if (total > 0 && (!x || !cu_seqlens || !logits || !reg || n_events == 0)) {
        set_error("NULL input or output pointer");
        return MLPF_E_INVALID;
    }
    if (total > 0 && ((uintptr_t)x & 7)) { set_error("x is not 8-byte aligned"); return MLPF_E_INVALID; }
    if (cudaSetDevice(m.device) != cudaSuccess) { set_error("cudaSetDevice failed"); return MLPF_E_CUDA; }
    if (m.device < 0 || m.device >= 64) { set_error("device index out of range"); return MLPF_E_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    if (total == 0) {
        if (event_sums && n_events > 0 &&
            cudaMemsetAsync(event_sums, 0, (size_t)n_events * 3 * sizeof(double), st) != cudaSuccess) {
            set_error("cudaMemsetAsync failed");
            return MLPF_E_CUDA;
        }
        return MLPF_OK;
    }
    NoallocDevice& nd = g_na[m.device];
    {
        // first call on this device: resolve the array's device address (a host-side
        // name is not a device pointer) and encode the tensor maps over it
        std::lock_guard<std::mutex> lock(g_na_mu);
        if (!nd.ready) {
            void* ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, g_mlpf_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                set_error(std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
                return MLPF_E_CUDA;
            }
            nd.base = (unsigned char*)ptr;
            Model tmp;
            tmp.ws = na_workspace(nd.base);
            if (!tc_make_maps(tmp)) return MLPF_E_CUDA;
            nd.map_q = tmp.ws.map_q;
            nd.map_q64 = tmp.ws.map_q64;   // 64-row Q tiles (attention variant 5)
            nd.map_k = tmp.ws.map_k;
            nd.map_o = tmp.ws.map_o;
            nd.map_vt = tmp.ws.map_vt;
            nd.map_vt16 = tmp.ws.map_vt16;   // 16-row V^T boxes (tensor-memory attention)
            nd.map_hp = tmp.ws.map_hp;
            nd.ready = true;
        }
    }
    // the same launch sequence on a workspace view of the static array; the model
    // itself is not modified (its own workspace and profiling state stay as they are)
    Workspace view = na_workspace(nd.base);
    view.map_q = nd.map_q;
    view.map_q64 = nd.map_q64;
    view.map_k = nd.map_k;
    view.map_o = nd.map_o;
    view.map_vt = nd.map_vt;
    view.map_vt16 = nd.map_vt16;
    view.map_hp = nd.map_hp;
    // no profiling events: creating them would allocate
    int64_t n = run_forward_tc(m, precision, x, cu_seqlens, n_events, total, max_n, logits, reg, st, &view, false);
    int64_t k = n < 0 ? -1 : run_event_sums(m, cu_seqlens, n_events, logits, reg, cls, event_sums, m.cfg.n_cls, st,
                                            false);
    if (n < 0 || k < 0) {
        set_error(std::string("kernel launch failed: ") + cudaGetErrorString(cudaGetLastError()));
        return MLPF_E_CUDA;
    }
    m.last_launches = n + k;
    return MLPF_OK;
}
