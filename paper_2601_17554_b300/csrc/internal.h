// Host-side internals shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "../../include/mlpf.h"

namespace mlpf {

void set_error(const std::string& msg);

// status bits written to the model's device status word
enum : unsigned {
    ST_TIMEOUT_ATTN = 1u,
    ST_TIMEOUT_GEMM = 2u,
    ST_NONFINITE = 4u,
};


// ---------------------------------------------------------------- weights
struct HostTensor {
    std::vector<int> shape;
    std::vector<float> data;
};

// fp32 device copies of every tensor (plain path) and prepared tensor-core images.
struct DeviceWeights {
    std::map<std::string, float*> f32;   // name -> device pointer (shared allocation)
    float* f32_base = nullptr;
    // FP32 path: concatenated QKV per layer, [3d, d] and [3d]
    std::vector<float*> wqkv_pid, bqkv_pid, wqkv_reg, bqkv_reg;
    // tensor-core path (d = 64 model only): 128B-swizzled weight images
    uint8_t* img_base = nullptr;
    std::map<std::string, uint8_t*> img_h;  // name -> device pointer of the FP16 image
    std::map<std::string, uint32_t> img_bytes;
    // wide tensor-core path: two-term FP16 images of every weight matrix, [N, 2 kp] with
    // kp = K padded to 64, keyed by the FP32 tensor's device pointer -> (image, kp)
    uint16_t* w16_base = nullptr;
    std::map<const float*, std::pair<const uint16_t*, int>> w16;
    // the wide path's QKV biases with the Q part times log2(e)/sqrt(dh) (its QKV weight
    // images carry the same factor), [3d] per layer
    float* wide_base = nullptr;
    std::vector<float*> bqkv_wide_pid, bqkv_wide_reg;
    float* tc_f32_base = nullptr;         // fused bias vectors for the tensor-core kernels
    std::map<std::string, float*> tcv;
    // FP8 E4M3 images (same layout, one byte per element) and per-tensor scales
    uint8_t* img8_base = nullptr;
    std::map<std::string, uint8_t*> img8;
    std::map<std::string, uint32_t> img8_bytes;
    std::map<std::string, float> w_scale;  // per-tensor weight scale (amax / 448)
};

// ---------------------------------------------------------------- workspace
struct Workspace {
    size_t cap_total = 0, cap_events = 0;
    int64_t cap_tpad = 0;   // padded-row capacity (multiple of 128)
    void* base = nullptr;
    size_t bytes = 0;
    // plain FP32 path
    float *z = nullptr, *zn = nullptr, *qkv = nullptr, *o = nullptr, *hid = nullptr;
    float *hpid = nullptr, *hreg = nullptr, *raw = nullptr;
    // tensor-core path (padded layout, rows of event e start at a multiple of 64)
    float* tz = nullptr;                 // [tpad, 64] residual stream fp32
    __nv_bfloat16 *tq = nullptr, *tk = nullptr, *to = nullptr, *tvt = nullptr, *thp = nullptr;
    int4* blk = nullptr;                 // per 64-row block: event, packed row, n valid
    float* kmax = nullptr;               // per 64-row block and head: largest K-row norm
    int4* items = nullptr;               // attention work items
    int* counters = nullptr;             // [0]=n_items [1]=tpad rows [2..3]=attn tickets
    CUtensorMap map_q, map_q64, map_k, map_o, map_vt, map_vt16, map_hp;   // map_vt16: 16-row V^T boxes
    // windowed attention: eta order of each event's elements (perm[r] = packed
    // row of the r-th element in that order), inputs and outputs in that order
    int32_t* perm = nullptr;
    float *xs = nullptr, *los = nullptr, *rgs = nullptr;
    // wide tensor-core path: two FP16 GEMM operand buffers [cap_total, the widest padded
    // input] (a layer's input and its hidden activations) and 16-bit Q | K | V [cap_total, 3 d]
    uint16_t* a16 = nullptr;
    uint16_t* b16 = nullptr;
    uint16_t* qkv16 = nullptr;
    // host-buffer entry point: device staging
    float *hx = nullptr, *hlogits = nullptr, *hreg_out = nullptr;
    int32_t *hcu = nullptr, *hcls = nullptr;
    double* hsums = nullptr;
    int32_t* hcu_chunks = nullptr;       // per-chunk cu_seqlens (each rebased to 0), back to back
};

struct GraphKey {
    int prec;
    const void *x, *cu, *lo, *rg, *cl, *su;
    int32_t n_events, total, max_n;
    const void* ws;   // base of the workspace the graph's kernels use
    bool operator<(const GraphKey& o) const;
};

// CUDA events around each kernel launch (MLPF_OPT_PROFILE); captured into
// graphs as external event-record nodes so replays re-record them.
struct Profile {
    std::vector<std::string> names;
    std::vector<cudaEvent_t> ev;  // 2 per launch
    int n = 0;
};

struct Model {
    int device = 0;
    mlpf_config cfg{};
    std::map<std::string, HostTensor> host;
    DeviceWeights w;
    Workspace ws;
    unsigned* status = nullptr;  // device status word
    int sm_count = 148;
    bool tc_supported = false;   // tensor-core path built for this configuration
    bool wide_supported = false; // generic-width tensor-core path (models the fused kernels do not cover)
    // options
    bool use_graphs = true;
    int64_t wait_limit_ns = 2000000000LL;
    bool debug_stall = false;
    int attn_ctas_per_sm = 1;
    // attention kernel variant per precision mode (BF16, FP16, E4M3), numbered as
    // MLPF_OPT_ATTN_VARIANT_* in mlpf.h; default: warp-level MMAs, 8 K/V stages
    int attn_variant[3] = {4, 4, 4};
    // windowed attention (0 = full): in eta order, query block b of 128 elements
    // attends to blocks b - attn_window .. b + attn_window
    int attn_window = 0;
    // gated inference (student models): event confidence = mean (0) or minimum (1)
    // of the per-element max softmax
    int gate_confidence = 0;
    // host-buffer forward: event chunks pipelined over copy-in, compute and copy-out
    int host_chunks = 8;
    // compute streams the chunks alternate over (2: odd chunks run on compute2 with
    // their own workspace ws_alt, so a chunk's attention tail overlaps the next chunk)
    int host_streams = 2;
    int wide_attn_kernel = 0;   // MLPF_OPT_WIDE_ATTN_KERNEL: 0 warp-level, 1 PV on tcgen05
    cudaStream_t copy_in = nullptr, copy_out = nullptr, compute2 = nullptr;
    Workspace ws_alt;
    std::vector<cudaEvent_t> chunk_ev;   // [0] start, [1] copies out done, then 2 per chunk
    int32_t* cu_pinned = nullptr;        // pinned host staging of the per-chunk cu_seqlens
    size_t cu_pinned_cap = 0;
    // anti-kt jet clustering scratch (mlpf_cluster_jets)
    void* jet_base = nullptr;
    size_t jet_bytes = 0;
    // FP8: activation slots (one per GEMM input) and their static scales s_a = amax / 448
    std::map<std::string, int> act_slot;
    std::vector<float> act_scale;
    bool fp8_ready = false;
    bool calibrating = false;       // 16-bit forward that records per-slot amax
    unsigned* amax_dev = nullptr;   // [64] max |activation| per slot (float bits)
    int embed_ctas_per_sm = 1;   // measured occupancy of the embedding kernels
    int64_t last_launches = 0;
    cudaStream_t cap_stream = nullptr;
    struct GraphEntry {
        cudaGraphExec_t exec;
        int64_t launches;
        Profile prof;
    };
    std::map<GraphKey, GraphEntry> graphs;
    // buffers of the gated (student + fallback) forward
    struct Gate {
        size_t cap_total = 0, cap_events = 0;
        void* base = nullptr;
        float *sub_x = nullptr, *sub_lo = nullptr, *sub_rg = nullptr, *conf = nullptr;
        int32_t *flag = nullptr, *sub_cu = nullptr, *src = nullptr, *meta = nullptr;
    } gate;
    bool profile = false;
    Profile* cur_prof = nullptr;   // profile being recorded by the launch sequence
    Profile direct_prof;           // profile of the last non-graph forward
    const Profile* last_prof = nullptr;
};

// Record the start / end of one kernel launch when profiling is on.
void prof_begin(Model& m, cudaStream_t st, const char* name);
void prof_end(Model& m, cudaStream_t st);

// launch sequences (return number of kernels launched, or -1 on launch error)
int64_t run_forward_f32(Model& m, const float* x, const int32_t* cu, int n_events, int total,
                        int max_n, float* logits, float* reg, cudaStream_t st);
// ws: the workspace the kernels use (NULL: the model's own); profile: record the
// per-kernel profiling events when the model's profiling option is on
int64_t run_forward_tc(Model& m, int prec, const float* x, const int32_t* cu, int n_events,
                       int total, int max_n, float* logits, float* reg, cudaStream_t st,
                       Workspace* ws = nullptr, bool profile = true);
void f32_eval_activation(const float* x, float* y, int n, int act, cudaStream_t st);
void tc_eval_activation(const float* x, float* y, int n, int act, cudaStream_t st);
// eta order / gather / scatter of the windowed-attention path (k_f32.cu)
int64_t run_eta_order(Model& m, const float* x, const int32_t* cu, int n_events, int total, cudaStream_t st);
void scatter_outputs(const int32_t* perm, const float* los, const float* rgs, float* logits, float* reg,
                     int total, cudaStream_t st);
int64_t run_event_sums(Model& m, const int32_t* cu, int n_events, const float* logits,
                       const float* reg, int32_t* cls, double* sums, int n_cls,
                       cudaStream_t st, bool profile = true);

// plain FP32 kernels shared with the training code (act: -1 none, 0 GELU, 1 ReLU)
void f32_linear(const float* X1, int ld1, int K1, const float* X2, int ld2, int K2, const float* W,
                const float* b, const float* R, int ldr, float* Y, int ldy, int T, int N, int act,
                cudaStream_t st);
void f32_layernorm(const float* X, const float* g, const float* b, float* Y, int T, int d, cudaStream_t st);
void f32_attention(const float* qkv, float* out, const int32_t* cu, int n_events, int max_n, int d,
                   int heads, float* lse, cudaStream_t st);
mlpf_status parse_blob_into(const uint8_t* p, size_t nbytes, Model& m);

// 16-bit tensor-core GEMM of the training step (k_gemm_tc.cu):
//   C[M, N] (op)= act(A[M, Kp] B[N, Kp]^T + bias) + R
// A, B row-major 16-bit (f16: FP16, else BF16), row strides lda, ldb (multiples of 8
// elements, bases 16-byte aligned), Kp a multiple of 64 with zeros beyond the true K.
// mode 0: C = ..., 1: C += ..., 2: C += ... split over K in chunks of kchunk (a multiple
// of 64; 0 = no split) with atomic adds; bias and R are added once (first split).  act:
// -1 none, 0 GELU, 1 ReLU.  C16 (or null): 16-bit copy of the result (mode 0; FP16 if
// c16_f16, else BF16) over max(N, c16_cols) columns, zeros beyond N; C may be null when
// only the 16-bit copy is wanted.  two_term: B is [N, 2 Kp] = [B_hi | B_lo] and the
// product is A (B_hi + B_lo)^T (weights carried as two 16-bit terms).  Returns
// false if a tensor map cannot be encoded.  Bounded waits set ST_TIMEOUT_GEMM in *status.
bool gemm_tc(int f16, const void* A, long lda, const void* B, long ldb, int M, int N, int Kp, float* C, long ldc,
             const float* bias, const float* R, long ldr, int act, int mode, int kchunk, uint16_t* C16, long ldc16,
             unsigned* status, uint64_t wait_ns, cudaStream_t st, int c16_f16 = 1, int two_term = 0,
             int c16_cols = 0);
// FP32 -> 16-bit operand copies: dst[r, c] = [s1 | s2][r, c] for c < k1 + k2, zero up to ldd
// (ldd even); cvt_16_t: dst[c, r] = src[r, c] for r < rows, c < cols, zero for rows <= r < ldd.
void cvt_16(const float* s1, long ld1, int k1, const float* s2, long ld2, int k2, int rows, uint16_t* dst, long ldd,
            int f16, cudaStream_t st);
void cvt_16_t(const float* src, long lds, int rows, int cols, uint16_t* dst, long ldd, int f16, cudaStream_t st);
// Two-term weight image [N, 2 kp]: columns 0.. the 16-bit rounding of W, columns kp.. the
// rounding of its residual (kp a multiple of 64), the B operand of a two_term gemm_tc.
void cvt_16_split(const float* W, long ldw, int N, int K, uint16_t* dst, int kp, int f16, cudaStream_t st);

// Varlen self-attention of the training step on the tensor cores (k_attn_train.cu):
// qkv [T, 3d] FP32 (Q | K | V, heads of dh = d / heads in {16, 32, 64}), out / dO [T, d],
// lse / D [T, heads] (natural-log log-sum-exp of the scaled scores; rowsum(dO o O)),
// dqkv [T, 3d].  16-bit operands (f16: FP16, else BF16), FP32 accumulation and
// statistics.  Return false for an unsupported head width.
bool attn_train_fwd_tc(int f16, const float* qkv, float* out, float* lse, const int32_t* cu, int n_events, int max_n,
                       int d, int heads, cudaStream_t st, int window = 0);
// sets the tensor-core GEMM kernels' shared-memory attributes (call outside graph capture)
void gemm_tc_prepare();
// generic-width tensor-core forward (k_f32.cu) and its weight images
bool wide_prepare_weights(Model& m);
int64_t run_forward_wide(Model& m, int prec, const float* x, const int32_t* cu, int n_events, int total, int max_n,
                         float* logits, float* reg, cudaStream_t st);
bool attn_train_bwd_tc(int f16, const float* qkv, const float* dO, const float* lse, const float* D, float* dqkv,
                       const int32_t* cu, int n_events, int max_n, int d, int heads, cudaStream_t st);
// Forward attention of the generic-width inference path on 16-bit Q | K | V [T, 3d] (FP16 if
// f16, else BF16); writes O as FP16 rows of stride ldo16 (the next GEMM's operand).
bool attn_fwd16(int f16, const uint16_t* qkv16, uint16_t* o16, int ldo16, const int32_t* cu, int n_events, int max_n,
                int d, int heads, cudaStream_t st, int window, int kernel, unsigned* status, uint64_t wait_ns);
void attn_fwd16_prepare();   // shared-memory attribute of the dh = 64 variant (outside capture)

// tensor-core path preparation (weights images, tensor maps)
bool tc_prepare_weights(Model& m);
bool tc_make_maps(Model& m);
int act_slot(Model& m, const std::string& name);

}  // namespace mlpf
