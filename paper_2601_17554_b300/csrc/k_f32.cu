// Plain FP32 path: SIMT FFMA kernels over the packed layout (no tensor cores,
// no TF32).  It is the precision reference on the GPU and the "plain" baseline
// the tensor-core path is measured against.  Also holds the per-event missing-pT
// sum kernel shared by every precision.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "internal.h"
#include "ptx.cuh"

namespace mlpf {

namespace {

constexpr int LIN_BM = 64, LIN_BN = 64, LIN_BK = 16;

__device__ __forceinline__ float act_fn(float v, int act) {
    if (act == 1) return fmaxf(v, 0.0f);
    if (act == 0) return 0.5f * v * (1.0f + erff(v * 0.70710678118654752f));
    return v;
}

// Y[r, n] = act(sum_k X[r, k] W[n, k] + b[n]) (+ R[r, n]); X = [X1 | X2] by columns.
// act: -1 none, 0 GELU, 1 ReLU.  R may alias Y (each element read then written
// by the same thread).
__global__ void __launch_bounds__(256) k_linear(const float* __restrict__ X1, int ld1, int K1,
                                                const float* __restrict__ X2, int ld2, int K2,
                                                const float* __restrict__ W,
                                                const float* __restrict__ b, const float* R,
                                                int ldr, float* Y, int ldy, int T, int N,
                                                int act) {
    __shared__ float As[LIN_BK][LIN_BM + 4];
    __shared__ float Ws[LIN_BK][LIN_BN + 4];
    const int K = K1 + K2;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = blockIdx.y * LIN_BM, n0 = blockIdx.x * LIN_BN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += LIN_BK) {
        for (int i = threadIdx.x; i < LIN_BM * LIN_BK; i += 256) {
            const int rr = i / LIN_BK, kk = i % LIN_BK;
            const int r = r0 + rr, k = k0 + kk;
            float v = 0.f;
            if (r < T && k < K) v = (k < K1) ? X1[(size_t)r * ld1 + k] : X2[(size_t)r * ld2 + (k - K1)];
            As[kk][rr] = v;
            const int n = n0 + rr;
            Ws[kk][rr] = (n < N && k < K) ? W[(size_t)n * K + k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < LIN_BK; ++kk) {
            float a[4], w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) w[j] = Ws[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty * 4 + i;
        if (r >= T) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float v = act_fn(acc[i][j] + b[n], act);
            if (R) v += R[(size_t)r * ldr + n];
            Y[(size_t)r * ldy + n] = v;
        }
    }
}

// LayerNorm over d columns, one warp per row (two-pass moments in FP32).
__global__ void k_layernorm(const float* __restrict__ X, const float* __restrict__ g,
                            const float* __restrict__ b, float* __restrict__ Y, int T, int d) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= T) return;
    const float* x = X + (size_t)row * d;
    float v[8];
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = lane + 32 * i;
        v[i] = (c < d) ? x[c] : 0.f;
        s += v[i];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float mu = s / d;
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = lane + 32 * i;
        const float t = (c < d) ? v[i] - mu : 0.f;
        q += t * t;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    const float rs = rsqrtf(q / d + 1e-5f);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = lane + 32 * i;
        if (c < d) Y[(size_t)row * d + c] = (v[i] - mu) * rs * g[c] + b[c];
    }
}

// The same LayerNorm writing FP16 rows of stride ldy (columns d .. ldy - 1 zero; ldy <= 256):
// the operand of the next GEMM of the generic-width tensor-core path.
__global__ void k_layernorm16(const float* __restrict__ X, const float* __restrict__ g, const float* __restrict__ b,
                              uint16_t* __restrict__ Y, int ldy, int T, int d) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= T) return;
    const float* x = X + (size_t)row * d;
    float v[8];
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = lane + 32 * i;
        v[i] = (c < d) ? x[c] : 0.f;
        s += v[i];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float mu = s / d;
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = lane + 32 * i;
        const float t = (c < d) ? v[i] - mu : 0.f;
        q += t * t;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    const float rs = rsqrtf(q / d + 1e-5f);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = lane + 32 * i;
        if (c < ldy) {
            const float y = c < d ? (v[i] - mu) * rs * g[c] + b[c] : 0.f;
            Y[(size_t)row * ldy + c] = (uint16_t)(pack_f16x2(y, 0.f) & 0xffffu);
        }
    }
}

// Self-attention within each event; one thread per query row, 64 keys per
// shared-memory tile, FP32 online softmax (exact expf).  qkv rows are
// [q | k | v] with head h in columns h*DH .. h*DH+DH-1 of each part.
// lse (optional, [T, heads]): log-sum-exp of each row's scaled scores, for the
// backward pass.
// window > 0: the query rows of 128-row block y (in the event's current order)
// attend to keys of blocks y - window .. y + window only.
template <int DH>
__global__ void __launch_bounds__(64) k_attention(const float* __restrict__ qkv,
                                                  float* __restrict__ out,
                                                  const int32_t* __restrict__ cu, int d,
                                                  float scale, float* __restrict__ lse, int window) {
    __shared__ float Ks[64][DH + 1];
    __shared__ float Vs[64][DH + 1];
    const int e = blockIdx.z, h = blockIdx.y;
    const int start = cu[e], n = cu[e + 1] - start;
    if (blockIdx.x * 64 >= n) return;
    const int qi = blockIdx.x * 64 + threadIdx.x;
    const bool active = qi < n;
    const int ld = 3 * d;
    float q[DH], acc[DH];
    float m = -INFINITY, l = 0.f;
#pragma unroll
    for (int c = 0; c < DH; ++c) {
        q[c] = active ? qkv[(size_t)(start + qi) * ld + h * DH + c] * scale : 0.f;
        acc[c] = 0.f;
    }
    int k_begin = 0, k_end = n;
    if (window > 0) {
        const int y = (blockIdx.x * 64) / 128;
        k_begin = max(0, (y - window) * 128);
        k_end = min(n, (y + window + 1) * 128);
    }
    for (int kb = k_begin; kb < k_end; kb += 64) {
        const int kj = kb + threadIdx.x;
        if (kj < k_end) {
            const float* kr = qkv + (size_t)(start + kj) * ld + d + h * DH;
            const float* vr = qkv + (size_t)(start + kj) * ld + 2 * d + h * DH;
#pragma unroll
            for (int c = 0; c < DH; ++c) {
                Ks[threadIdx.x][c] = kr[c];
                Vs[threadIdx.x][c] = vr[c];
            }
        }
        __syncthreads();
        const int cnt = min(64, k_end - kb);
        if (active) {
            float s[64];
            float mx = m;
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                if (j < cnt) {
                    float t = 0.f;
#pragma unroll
                    for (int c = 0; c < DH; ++c) t = fmaf(q[c], Ks[j][c], t);
                    s[j] = t;
                    mx = fmaxf(mx, t);
                }
            }
            const float alpha = expf(m - mx);
            l *= alpha;
#pragma unroll
            for (int c = 0; c < DH; ++c) acc[c] *= alpha;
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                if (j < cnt) {
                    const float p = expf(s[j] - mx);
                    l += p;
#pragma unroll
                    for (int c = 0; c < DH; ++c) acc[c] = fmaf(p, Vs[j][c], acc[c]);
                }
            }
            m = mx;
        }
        __syncthreads();
    }
    if (active) {
        const float inv = 1.0f / l;
#pragma unroll
        for (int c = 0; c < DH; ++c) out[(size_t)(start + qi) * d + h * DH + c] = acc[c] * inv;
        if (lse) lse[(size_t)(start + qi) * gridDim.y + h] = m + logf(l);
    }
}

// reg[r] = (pT_elem*exp(pT'), eta, sin, cos, E_elem*exp(E')), log pT_elem = x[r,8].
__global__ void k_decode(const float* __restrict__ x, const float* __restrict__ raw,
                         float* __restrict__ reg, int T) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= T) return;
    const float* a = raw + (size_t)r * 5;
    float* o = reg + (size_t)r * 5;
    o[0] = expf(x[(size_t)r * 42 + 8] + a[0]);
    o[1] = a[1];
    o[2] = a[2];
    o[3] = a[3];
    o[4] = expf(x[(size_t)r * 42 + 9] + a[4]);
}

// One block of ES_THREADS threads per event: class = argmax (lowest index on ties);
// FP64 sums of -px, -py and pT over elements with class != 0.  Threads stride
// over the event's rows; the partial sums are combined by a fixed xor
// butterfly per warp and then in warp order, so the result is deterministic (and
// does not depend on the other events of the batch).  512 threads: the largest
// events set the kernel's time, and 512-thread blocks of a 512-event batch are
// still resident at once (four per SM).
constexpr int ES_THREADS = 512, ES_WARPS = ES_THREADS / 32;
__global__ void __launch_bounds__(ES_THREADS) k_event_sums(const int32_t* __restrict__ cu, int n_events,
                                                    const float* __restrict__ logits,
                                                    const float* __restrict__ reg,
                                                    int32_t* __restrict__ cls_out,
                                                    double* __restrict__ sums, int n_cls,
                                                    int arch, unsigned* status) {
    __shared__ double part[3][ES_WARPS];
    __shared__ int bad;
    const int e = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    const int s = cu[e], t = cu[e + 1];
    double px = 0.0, py = 0.0, pt = 0.0;
    bool finite = true;
    for (int r = s + threadIdx.x; r < t; r += ES_THREADS) {
        const float* lo = logits + (size_t)r * n_cls;
        // arch 0: argmax of all scores (lowest index on ties); arch 1: a particle
        // where the binary logit (column 0) is > 0, PID = 1 + argmax of columns 1..
        const int c0 = arch == 1 ? 1 : 0;
        int best = c0;
        float bv = lo[c0];
        finite &= isfinite(lo[0]) && isfinite(bv);
        for (int c = c0 + 1; c < n_cls; ++c) {
            const float v = lo[c];
            finite &= isfinite(v);
            if (v > bv) { bv = v; best = c; }
        }
        if (arch == 1 && !(lo[0] > 0.f)) best = 0;
        const float* rg = reg + (size_t)r * 5;
#pragma unroll
        for (int c = 0; c < 5; ++c) finite &= isfinite(rg[c]);
        if (cls_out) cls_out[r] = best;
        if (best != 0) {
            // per-element terms in FP32 (this GPU's FP64 divide and square root are
            // slow), accumulated in FP64 in a fixed order
            const float p = rg[0], sn = rg[2], cs = rg[3];
            const float r2 = fmaf(sn, sn, cs * cs);
            if (r2 > 0.f) {
                const float inv = 1.0f / sqrtf(r2);
                px += (double)(p * (cs * inv));
                py += (double)(p * (sn * inv));
            }
            pt += (double)p;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        px += __shfl_xor_sync(0xffffffffu, px, o);
        py += __shfl_xor_sync(0xffffffffu, py, o);
        pt += __shfl_xor_sync(0xffffffffu, pt, o);
    }
    if (!finite) bad = 1;
    if (lane == 0) {
        part[0][wid] = px;
        part[1][wid] = py;
        part[2][wid] = pt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < ES_WARPS; ++w) {
            a0 += part[0][w];
            a1 += part[1][w];
            a2 += part[2][w];
        }
        if (bad) atomicOr(status, ST_NONFINITE);
        if (sums) {
            sums[(size_t)e * 3 + 0] = -a0;
            sums[(size_t)e * 3 + 1] = -a1;
            sums[(size_t)e * 3 + 2] = a2;
        }
    }
}

inline unsigned cdiv(long a, long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

static Model* g_model = nullptr;  // model of the launch sequence being recorded

static void linear(const float* X1, int ld1, int K1, const float* X2, int ld2, int K2,
                   const float* W, const float* b, const float* R, int ldr, float* Y, int ldy,
                   int T, int N, int act, cudaStream_t st, int64_t& n) {
    dim3 grid(cdiv(N, LIN_BN), cdiv(T, LIN_BM));
    prof_begin(*g_model, st, "f32_linear");
    k_linear<<<grid, 256, 0, st>>>(X1, ld1, K1, X2, ld2, K2, W, b, R, ldr, Y, ldy, T, N, act);
    prof_end(*g_model, st);
    ++n;
}

static void layernorm(const float* X, const float* g, const float* b, float* Y, int T, int d,
                      cudaStream_t st, int64_t& n) {
    prof_begin(*g_model, st, "f32_layernorm");
    k_layernorm<<<cdiv(T, 8), 256, 0, st>>>(X, g, b, Y, T, d);
    prof_end(*g_model, st);
    ++n;
}

// Per-type embedding (arch 1): rows of cluster-type elements take the cluster
// FFN's output.  Track-like types: track, GSF track, brem (one-hot x[0], x[5], x[6]).
__global__ void k_type_select(const float* __restrict__ x, const float* __restrict__ e_clu,
                              float* __restrict__ z, int T, int d) {
    const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (r >= T) return;
    const float* xr = x + (size_t)r * 42;
    if (xr[0] + xr[5] + xr[6] > 0.5f) return;
    for (int c = threadIdx.x & 31; c < d; c += 32) z[(size_t)r * d + c] = e_clu[(size_t)r * d + c];
}

int64_t run_forward_f32(Model& m, const float* x, const int32_t* cu, int n_events, int total,
                        int max_n, float* logits, float* reg, cudaStream_t st) {
    const mlpf_config& c = m.cfg;
    const int T = total, d = c.d, F = c.ffn, dh = d / c.heads, act = c.act;
    Workspace& w = m.ws;
    auto W = [&](const std::string& s) { return m.w.f32.at(s); };
    int64_t n = 0;
    g_model = &m;
    const float scale = 1.0f / sqrtf((float)dh);

    auto stack = [&](const char* prefix, int layers, std::vector<float*>& wqkv,
                     std::vector<float*>& bqkv, float* out) {
        for (int l = 0; l < layers; ++l) {
            const std::string p = std::string(prefix) + "." + std::to_string(l) + ".";
            layernorm(w.z, W(p + "ln1.g"), W(p + "ln1.b"), w.zn, T, d, st, n);
            linear(w.zn, d, d, nullptr, 0, 0, wqkv[l], bqkv[l], nullptr, 0, w.qkv, 3 * d, T, 3 * d,
                   -1, st, n);
            dim3 grid(cdiv(max_n, 64), c.heads, n_events);
            prof_begin(m, st, "f32_attention");
            if (dh == 16)
                k_attention<16><<<grid, 64, 0, st>>>(w.qkv, w.o, cu, d, scale, nullptr, m.attn_window);
            else if (dh == 32)
                k_attention<32><<<grid, 64, 0, st>>>(w.qkv, w.o, cu, d, scale, nullptr, m.attn_window);
            else
                k_attention<64><<<grid, 64, 0, st>>>(w.qkv, w.o, cu, d, scale, nullptr, m.attn_window);
            prof_end(m, st);
            ++n;
            linear(w.o, d, d, nullptr, 0, 0, W(p + "wo"), W(p + "bo"), w.z, d, w.z, d, T, d, -1, st,
                   n);
            layernorm(w.z, W(p + "ln2.g"), W(p + "ln2.b"), w.zn, T, d, st, n);
            linear(w.zn, d, d, nullptr, 0, 0, W(p + "ffn.w1"), W(p + "ffn.b1"), nullptr, 0, w.hid, F,
                   T, F, act, st, n);
            linear(w.hid, F, F, nullptr, 0, 0, W(p + "ffn.w2"), W(p + "ffn.b2"), w.z, d, w.z, d, T,
                   d, -1, st, n);
        }
        layernorm(w.z, W(std::string(prefix) + ".lnf.g"), W(std::string(prefix) + ".lnf.b"), out,
                  T, d, st, n);
    };

    auto mlp = [&](const float* in, int k_in, const char* p, float* out, int ldo, int n_out) {
        const std::string s(p);
        linear(in, k_in, k_in, nullptr, 0, 0, W(s + ".w1"), W(s + ".b1"), nullptr, 0, w.hid, d, T, d,
               act, st, n);
        linear(w.hid, d, d, nullptr, 0, 0, W(s + ".w2"), W(s + ".b2"), nullptr, 0, out, ldo, T, n_out,
               -1, st, n);
    };
    if (c.arch == 1) {
        // Sec. 5.3 as printed: track and cluster embeddings; two parallel stacks on
        // the embedding (kept in hreg while the classification stack runs)
        mlp(x, 42, "emb.trk", w.hreg, d, d);
        mlp(x, 42, "emb.clu", w.zn, d, d);
        prof_begin(m, st, "f32_type_select");
        k_type_select<<<cdiv(T, 8), 256, 0, st>>>(x, w.zn, w.hreg, T, d);
        prof_end(m, st);
        ++n;
        if (cudaMemcpyAsync(w.z, w.hreg, (size_t)T * d * sizeof(float), cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return -1;
        stack("pid", c.l_pid, m.w.wqkv_pid, m.w.bqkv_pid, w.hpid);
        if (cudaMemcpyAsync(w.z, w.hreg, (size_t)T * d * sizeof(float), cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return -1;
        stack("reg", c.l_reg, m.w.wqkv_reg, m.w.bqkv_reg, w.hreg);
        mlp(w.hpid, d, "head.bin", logits, c.n_cls, 1);
        mlp(w.hpid, d, "head.pid", logits + 1, c.n_cls, c.n_cls - 1);
    } else {
        mlp(x, 42, "emb", w.z, d, d);
        stack("pid", c.l_pid, m.w.wqkv_pid, m.w.bqkv_pid, w.hpid);
        linear(x, 42, 42, w.hpid, d, d, W("remb.w1"), W("remb.b1"), nullptr, 0, w.hid, d, T, d, act, st,
               n);
        linear(w.hid, d, d, nullptr, 0, 0, W("remb.w2"), W("remb.b2"), nullptr, 0, w.z, d, T, d, -1, st,
               n);
        stack("reg", c.l_reg, m.w.wqkv_reg, m.w.bqkv_reg, w.hreg);
        mlp(w.hpid, d, "head.cls", logits, c.n_cls, c.n_cls);
    }
    const char* names[4] = {"pt", "eta", "phi", "e"};
    const int widths[4] = {1, 1, 2, 1};
    int off = 0;
    for (int h = 0; h < 4; ++h) {
        mlp(w.hreg, d, (std::string("head.") + names[h]).c_str(), w.raw + off, 5, widths[h]);
        off += widths[h];
    }
    prof_begin(m, st, "f32_decode");
    k_decode<<<cdiv(T, 256), 256, 0, st>>>(x, w.raw, reg, T);
    prof_end(m, st);
    ++n;
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
    return n;
}

// ------------------------------------------------------------------ wide tensor-core path
// Forward of models outside the fused d = 64 kernels (any width with heads of 16, 32 or
// 64; both architectures) on the tensor cores: every linear layer is one tcgen05 GEMM
// (FP16 operands with two-term weights, FP32 accumulation, bias / activation / residual in
// its epilogue); the blocks' LayerNorms, the QKV GEMM, attention and the FFN's first GEMM
// hand their outputs to the next GEMM as 16-bit rows, the embedding and head inputs are
// converted; attention runs on warp-level MMAs (BF16 operands in the BF16 mode, FP16 in
// the FP16 mode; FP32 softmax statistics); LayerNorm moments, the residual stream and the
// decode stay FP32.  Same launch sequence as the plain path otherwise.
static constexpr uint64_t WIDE_WAIT_NS = 2000000000ull;

// y[T, N] = act([X1 | X2] W^T + b) (+ R) with two-term FP16 weights.  A16 (or null): the
// FP16 operand rows are already there (stride = W's padded K); otherwise [X1 | X2] is
// converted into the scratch first.  Y (or null): FP32 result; Y16 (or null): 16-bit copy
// (format c16_f16) of stride y16_ld, zero beyond N.
static void tlinear(Model& m, const uint16_t* A16, const float* X1, int ld1, int K1, const float* X2, int ld2, int K2,
                    const float* W, const float* b, const float* R, int ldr, float* Y, int ldy, int T, int N, int act,
                    cudaStream_t st, int64_t& n, bool& ok, uint16_t* Y16 = nullptr, int y16_ld = 0, int c16_f16 = 1) {
    const auto it = m.w.w16.find(W);
    if (it == m.w.w16.end()) {
        ok = false;
        return;
    }
    const int Kp = it->second.second;
    if (!A16) {
        prof_begin(m, st, "wide_cvt");
        cvt_16(X1, ld1, K1, X2, ld2, K2, T, m.ws.a16, Kp, 1, st);
        prof_end(m, st);
        ++n;
        A16 = m.ws.a16;
    }
    prof_begin(m, st, "wide_gemm");
    if (!gemm_tc(1, A16, Kp, it->second.first, 2 * Kp, T, N, Kp, Y, ldy, b, R, ldr, act, 0, 0, Y16, y16_ld, m.status,
                 WIDE_WAIT_NS, st, c16_f16, 1, y16_ld))
        ok = false;
    prof_end(m, st);
    ++n;
}

static void layernorm16(Model& m, const float* X, const float* g, const float* b, uint16_t* Y, int ldy, int T, int d,
                        cudaStream_t st, int64_t& n) {
    prof_begin(m, st, "wide_layernorm");
    k_layernorm16<<<cdiv(T, 8), 256, 0, st>>>(X, g, b, Y, ldy, T, d);
    prof_end(m, st);
    ++n;
}

int64_t run_forward_wide(Model& m, int prec, const float* x, const int32_t* cu, int n_events, int total, int max_n,
                         float* logits, float* reg, cudaStream_t st) {
    const mlpf_config& c = m.cfg;
    const int T = total, d = c.d, F = c.ffn, act = c.act;
    Workspace& w = m.ws;
    auto W = [&](const std::string& s) { return m.w.f32.at(s); };
    int64_t n = 0;
    bool ok = true;
    g_model = &m;
    const int Kd = (d + 63) / 64 * 64, Kf = (F + 63) / 64 * 64;   // padded operand widths
    auto stack = [&](const char* prefix, int layers, std::vector<float*>& wqkv, std::vector<float*>& bqkv,
                     float* out) {
        for (int l = 0; l < layers; ++l) {
            const std::string p = std::string(prefix) + "." + std::to_string(l) + ".";
            layernorm16(m, w.z, W(p + "ln1.g"), W(p + "ln1.b"), w.a16, Kd, T, d, st, n);
            // Q | K | V only as 16-bit values (the attention operands' format)
            tlinear(m, w.a16, nullptr, 0, d, nullptr, 0, 0, wqkv[l], bqkv[l], nullptr, 0, nullptr, 0, T, 3 * d, -1, st,
                    n, ok, w.qkv16, 3 * d, prec == MLPF_FP16);
            prof_begin(m, st, "wide_attention");
            if (!attn_fwd16(prec == MLPF_FP16, w.qkv16, w.a16, Kd, cu, n_events, max_n, d, c.heads, st, m.attn_window,
                            m.wide_attn_kernel, m.status, WIDE_WAIT_NS))
                ok = false;
            prof_end(m, st);
            ++n;
            tlinear(m, w.a16, nullptr, 0, d, nullptr, 0, 0, W(p + "wo"), W(p + "bo"), w.z, d, w.z, d, T, d, -1, st, n,
                    ok);
            layernorm16(m, w.z, W(p + "ln2.g"), W(p + "ln2.b"), w.a16, Kd, T, d, st, n);
            tlinear(m, w.a16, nullptr, 0, d, nullptr, 0, 0, W(p + "ffn.w1"), W(p + "ffn.b1"), nullptr, 0, nullptr, 0, T,
                    F, act, st, n, ok, w.b16, Kf);
            tlinear(m, w.b16, nullptr, 0, F, nullptr, 0, 0, W(p + "ffn.w2"), W(p + "ffn.b2"), w.z, d, w.z, d, T, d, -1,
                    st, n, ok);
        }
        layernorm(w.z, W(std::string(prefix) + ".lnf.g"), W(std::string(prefix) + ".lnf.b"), out, T, d, st, n);
    };
    auto mlp = [&](const float* in, int k_in, const char* p, float* out, int ldo, int n_out) {
        const std::string s(p);
        tlinear(m, nullptr, in, k_in, k_in, nullptr, 0, 0, W(s + ".w1"), W(s + ".b1"), nullptr, 0, nullptr, 0, T, d,
                act, st, n, ok, w.b16, Kd);
        tlinear(m, w.b16, nullptr, 0, d, nullptr, 0, 0, W(s + ".w2"), W(s + ".b2"), nullptr, 0, out, ldo, T, n_out, -1,
                st, n, ok);
    };
    if (c.arch == 1) {
        mlp(x, 42, "emb.trk", w.hreg, d, d);
        mlp(x, 42, "emb.clu", w.zn, d, d);
        prof_begin(m, st, "f32_type_select");
        k_type_select<<<cdiv(T, 8), 256, 0, st>>>(x, w.zn, w.hreg, T, d);
        prof_end(m, st);
        ++n;
        if (cudaMemcpyAsync(w.z, w.hreg, (size_t)T * d * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return -1;
        stack("pid", c.l_pid, m.w.wqkv_pid, m.w.bqkv_wide_pid, w.hpid);
        if (cudaMemcpyAsync(w.z, w.hreg, (size_t)T * d * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return -1;
        stack("reg", c.l_reg, m.w.wqkv_reg, m.w.bqkv_wide_reg, w.hreg);
        mlp(w.hpid, d, "head.bin", logits, c.n_cls, 1);
        mlp(w.hpid, d, "head.pid", logits + 1, c.n_cls, c.n_cls - 1);
    } else {
        mlp(x, 42, "emb", w.z, d, d);
        stack("pid", c.l_pid, m.w.wqkv_pid, m.w.bqkv_wide_pid, w.hpid);
        tlinear(m, nullptr, x, 42, 42, w.hpid, d, d, W("remb.w1"), W("remb.b1"), nullptr, 0, nullptr, 0, T, d, act, st,
                n, ok, w.b16, Kd);
        tlinear(m, w.b16, nullptr, 0, d, nullptr, 0, 0, W("remb.w2"), W("remb.b2"), nullptr, 0, w.z, d, T, d, -1, st, n,
                ok);
        stack("reg", c.l_reg, m.w.wqkv_reg, m.w.bqkv_wide_reg, w.hreg);
        mlp(w.hpid, d, "head.cls", logits, c.n_cls, c.n_cls);
    }
    const char* names[4] = {"pt", "eta", "phi", "e"};
    const int widths[4] = {1, 1, 2, 1};
    int off = 0;
    for (int h = 0; h < 4; ++h) {
        mlp(w.hreg, d, (std::string("head.") + names[h]).c_str(), w.raw + off, 5, widths[h]);
        off += widths[h];
    }
    prof_begin(m, st, "f32_decode");
    k_decode<<<cdiv(T, 256), 256, 0, st>>>(x, w.raw, reg, T);
    prof_end(m, st);
    ++n;
    if (!ok || cudaPeekAtLastError() != cudaSuccess) return -1;
    return n;
}

// v[i] *= s for i < n
__global__ void k_scale_prefix(float* __restrict__ v, long n, float s) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) v[i] *= s;
}

// Two-term FP16 images of every weight matrix the wide path multiplies (the weight as
// the sum of its FP16 rounding and the FP16 rounding of the remainder, about 22
// significant bits: the rounding of a weight shifts every element's output alike, which
// moves threshold decisions of a whole batch; activation roundings do not), each half
// padded with zeros to a multiple of 64 columns, keyed by the FP32 tensor's device pointer.
// The QKV images carry the Q rows times log2(e)/sqrt(dh), and so do the wide path's own
// copies of the QKV biases: the attention kernel takes its base-2 softmax exponent
// straight from Q K^T (one rounding of the scaled Q, in the GEMM's epilogue).
bool wide_prepare_weights(Model& m) {
    std::vector<std::pair<const float*, std::pair<int, int>>> mats;   // pointer, (N, K)
    for (const auto& kv : m.host)
        if (kv.second.shape.size() == 2) mats.push_back({m.w.f32.at(kv.first), {kv.second.shape[0], kv.second.shape[1]}});
    const int d = m.cfg.d;
    const float qscale = 1.4426950408889634f / sqrtf((float)(d / m.cfg.heads));
    std::vector<const float*> qkv(m.w.wqkv_pid.begin(), m.w.wqkv_pid.end());
    qkv.insert(qkv.end(), m.w.wqkv_reg.begin(), m.w.wqkv_reg.end());
    for (const float* p : qkv) mats.push_back({p, {3 * d, d}});
    size_t total = 0;
    for (const auto& mt : mats) total += (size_t)mt.second.first * 2 * ((mt.second.second + 63) / 64 * 64);
    if (cudaMalloc(&m.w.w16_base, total * sizeof(uint16_t)) != cudaSuccess) return false;
    // scaled QKV biases (kept) and one scaled QKV weight matrix at a time (scratch)
    const size_t nb = qkv.size() * 3 * (size_t)d;
    if (cudaMalloc(&m.w.wide_base, (nb + 3 * (size_t)d * d) * sizeof(float)) != cudaSuccess) return false;
    float* wtmp = m.w.wide_base + nb;
    for (size_t l = 0; l < qkv.size(); ++l) {
        const bool pid = l < m.w.wqkv_pid.size();
        const float* b = pid ? m.w.bqkv_pid[l] : m.w.bqkv_reg[l - m.w.wqkv_pid.size()];
        float* bw = m.w.wide_base + l * 3 * d;
        cudaMemcpy(bw, b, 3 * (size_t)d * sizeof(float), cudaMemcpyDeviceToDevice);
        k_scale_prefix<<<cdiv(d, 256), 256>>>(bw, d, qscale);
        (pid ? m.w.bqkv_wide_pid : m.w.bqkv_wide_reg).push_back(bw);
    }
    size_t off = 0;
    for (const auto& mt : mats) {
        const int N = mt.second.first, K = mt.second.second, Kp = (K + 63) / 64 * 64;
        uint16_t* dst = m.w.w16_base + off;
        const float* src = mt.first;
        if (std::find(qkv.begin(), qkv.end(), mt.first) != qkv.end()) {
            cudaMemcpy(wtmp, mt.first, 3 * (size_t)d * d * sizeof(float), cudaMemcpyDeviceToDevice);
            k_scale_prefix<<<cdiv(d * d, 256), 256>>>(wtmp, (long)d * d, qscale);
            src = wtmp;
        }
        cvt_16_split(src, K, N, K, dst, Kp, 1, 0);
        if (src == wtmp && cudaDeviceSynchronize() != cudaSuccess) return false;   // the scratch is reused
        m.w.w16[mt.first] = {dst, Kp};
        off += (size_t)N * 2 * Kp;
    }
    gemm_tc_prepare();
    attn_fwd16_prepare();
    return cudaDeviceSynchronize() == cudaSuccess;
}

void f32_linear(const float* X1, int ld1, int K1, const float* X2, int ld2, int K2, const float* W,
                const float* b, const float* R, int ldr, float* Y, int ldy, int T, int N, int act,
                cudaStream_t st) {
    if (T <= 0) return;
    dim3 grid(cdiv(N, LIN_BN), cdiv(T, LIN_BM));
    k_linear<<<grid, 256, 0, st>>>(X1, ld1, K1, X2, ld2, K2, W, b, R, ldr, Y, ldy, T, N, act);
}

void f32_layernorm(const float* X, const float* g, const float* b, float* Y, int T, int d, cudaStream_t st) {
    if (T <= 0) return;
    k_layernorm<<<cdiv(T, 8), 256, 0, st>>>(X, g, b, Y, T, d);
}

void f32_attention(const float* qkv, float* out, const int32_t* cu, int n_events, int max_n, int d,
                   int heads, float* lse, cudaStream_t st) {
    if (n_events <= 0 || max_n <= 0) return;
    const int dh = d / heads;
    const float scale = 1.0f / sqrtf((float)dh);
    dim3 grid(cdiv(max_n, 64), heads, n_events);
    if (dh == 16)
        k_attention<16><<<grid, 64, 0, st>>>(qkv, out, cu, d, scale, lse, 0);
    else if (dh == 32)
        k_attention<32><<<grid, 64, 0, st>>>(qkv, out, cu, d, scale, lse, 0);
    else
        k_attention<64><<<grid, 64, 0, st>>>(qkv, out, cu, d, scale, lse, 0);
}

__global__ void k_eval_act_f32(const float* __restrict__ x, float* __restrict__ y, int n, int act) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = act_fn(x[i], act);
}

void f32_eval_activation(const float* x, float* y, int n, int act, cudaStream_t st) {
    if (n > 0) k_eval_act_f32<<<(n + 255) / 256, 256, 0, st>>>(x, y, n, act);
}

// Eta order of each event's elements for windowed attention: one CTA per event
// sorts the 64-bit keys (sortable eta bits << 32 | position) with a bitonic
// network in shared memory (ties keep their input order), then writes perm and
// gathers the input rows in that order.  Events of up to kSortMax elements.
constexpr int kSortMax = 16384;
__global__ void __launch_bounds__(1024) k_eta_order(const float* __restrict__ x, const int32_t* __restrict__ cu,
                                                    int32_t* __restrict__ perm, float* __restrict__ xs) {
    extern __shared__ unsigned long long keys[];
    const int e = blockIdx.x;
    const int start = cu[e], n = min(cu[e + 1] - start, kSortMax);
    if (n <= 0) return;
    int np2 = 1;
    while (np2 < n) np2 <<= 1;
    for (int i = threadIdx.x; i < np2; i += blockDim.x) {
        unsigned long long k = ~0ull;
        if (i < n) {
            unsigned u = __float_as_uint(x[(size_t)(start + i) * 42 + 10]);
            u ^= (u & 0x80000000u) ? 0xffffffffu : 0x80000000u;   // order-preserving bits
            k = ((unsigned long long)u << 32) | (unsigned)i;
        }
        keys[i] = k;
    }
    __syncthreads();
    for (int size = 2; size <= np2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < np2; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const unsigned long long a = keys[i], b = keys[j];
                    const bool up = (i & size) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) perm[start + r] = start + (int)(keys[r] & 0xffffffffu);
    __syncthreads();
    for (int t = threadIdx.x; t < n * 42; t += blockDim.x) {
        const int r = t / 42, c = t - r * 42;
        xs[(size_t)(start + r) * 42 + c] = x[(size_t)(start + (int)(keys[r] & 0xffffffffu)) * 42 + c];
    }
}

__global__ void k_scatter_outputs(const int32_t* __restrict__ perm, const float* __restrict__ los,
                                  const float* __restrict__ rgs, float* __restrict__ logits,
                                  float* __restrict__ reg, int T) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= T) return;
    const int o = perm[r];
#pragma unroll
    for (int c = 0; c < 6; ++c) logits[(size_t)o * 6 + c] = los[(size_t)r * 6 + c];
#pragma unroll
    for (int c = 0; c < 5; ++c) reg[(size_t)o * 5 + c] = rgs[(size_t)r * 5 + c];
}

int64_t run_eta_order(Model& m, const float* x, const int32_t* cu, int n_events, int total, cudaStream_t st) {
    if (n_events <= 0 || total <= 0) return 0;
    static bool attr[64] = {};
    if (m.device >= 0 && m.device < 64 && !attr[m.device]) {
        cudaFuncSetAttribute(k_eta_order, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortMax * 8);
        attr[m.device] = true;
    }
    prof_begin(m, st, "eta_order");
    k_eta_order<<<n_events, 1024, kSortMax * 8, st>>>(x, cu, m.ws.perm, m.ws.xs);
    prof_end(m, st);
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
    return 1;
}

void scatter_outputs(const int32_t* perm, const float* los, const float* rgs, float* logits, float* reg, int total,
                     cudaStream_t st) {
    if (total > 0) k_scatter_outputs<<<cdiv(total, 256), 256, 0, st>>>(perm, los, rgs, logits, reg, total);
}

int64_t run_event_sums(Model& m, const int32_t* cu, int n_events, const float* logits,
                       const float* reg, int32_t* cls, double* sums, int n_cls,
                       cudaStream_t st, bool profile) {
    if (n_events <= 0 || (!cls && !sums)) return 0;
    if (profile) prof_begin(m, st, "event_sums");
    k_event_sums<<<n_events, ES_THREADS, 0, st>>>(cu, n_events, logits, reg, cls, sums, n_cls, m.cfg.arch, m.status);
    if (profile) prof_end(m, st);
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
    return 1;
}

}  // namespace mlpf
