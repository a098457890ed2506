// Tensor-core path of the MLPF forward (model width 64, 4 heads of 16, FFN 256):
//
//   k_schedule      one CTA: padded layout (each event starts at a multiple of 64
//                   rows), per-64-row block table, attention work list sorted by
//                   event size (longest first)
//   k_embed_qkv     per 128-row tile: element embedding FFN (Sec. 5.3) [or the
//                   regression-stack input FFN over concat(x, h_pid)], residual
//                   stream out, pre-LN, fused Q/K/V projection
//   k_attention     persistent varlen self-attention (Sec. 5.3, Eq. 4) with
//                   tcgen05 QK^T and PV, FP32 online softmax, one warpgroup per head
//   k_post          per 128-row tile: out-projection + residual, LN, FFN up, GELU,
//                   FFN down + residual, then either the next block's LN+QKV, the
//                   end of the PID stack (final LN, class head) or the end of the
//                   regression stack (final LN, four regression heads, decode)
//
// GEMM operands are BF16 in 128-byte-swizzled shared-memory tiles (TMA or
// per-thread swizzled stores), accumulators FP32 in TMEM; thread t of a CTA owns
// row t of each 128-row tile, so LayerNorm moments and softmax statistics are
// per-thread FP32 sums with no cross-thread reduction.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "ptx.cuh"

namespace mlpf {

namespace {

constexpr int D = 64;            // model width
constexpr int NH = 4;            // heads
constexpr int ROWS = 128;        // rows per tile (UMMA M)
constexpr int ATOM = ROWS * 128; // bytes of a [128 x 64] bf16 swizzled atom column
constexpr float LN_EPS = 1e-5f;
// Q is stored multiplied by log2(e) / sqrt(16) (head width 16): the attention
// kernels take the base-2 softmax exponent straight from Q K^T.
constexpr float kQScale = 0.25f * 1.4426950408889634f;

MLPF_DEV uint8_t* align1024(uint8_t* p) {
    return (uint8_t*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

// GELU(v) = v Phi(v) = v (1 + erf(v / sqrt 2)) / 2 with erf from the rational
// approximation of Abramowitz & Stegun, Handbook of Mathematical Functions,
// formula 7.1.26 (Hastings): for z >= 0, erf(z) = 1 - t (a1 + t (a2 + t (a3 + t (a4
// + t a5)))) e^(-z^2), t = 1 / (1 + p z), |error| <= 1.5e-7; erf(-z) = -erf(z).
// Two values at a time: the multiplies and multiply-adds are packed FP32x2 ops
// (one issue for both values), the reciprocal and the exponential run on the
// MUFU (approximate, ~1 ulp), which is idle in the GEMM epilogues.  The result is
// far below the 16-bit rounding of the operands it feeds.  Checked against the
// FP32 path's erff-based GELU by mlpf_eval_activation.
MLPF_DEV float2 gelu2_f(float va, float vb) {
    // Horner coefficients negated, so that the last step gives 1 - poly e directly
    const float2 kP = make_float2(0.3275911f, 0.3275911f), kNA1 = make_float2(-0.254829592f, -0.254829592f),
                 kNA2 = make_float2(0.284496736f, 0.284496736f), kNA3 = make_float2(-1.421413741f, -1.421413741f),
                 kNA4 = make_float2(1.453152027f, 1.453152027f), kNA5 = make_float2(-1.061405429f, -1.061405429f);
    const float2 one = make_float2(1.f, 1.f);
    const float2 v = make_float2(va, vb);
    // z = |v| / sqrt 2; -z^2 log2(e) = v^2 (-log2(e) / 2)
    const float2 z = __fmul2_rn(make_float2(fabsf(va), fabsf(vb)), make_float2(0.70710678118654752f, 0.70710678118654752f));
    const float2 den = __ffma2_rn(kP, z, one);
    const float2 w = __fmul2_rn(__fmul2_rn(v, v), make_float2(-0.72134752044448170f, -0.72134752044448170f));
    float2 t, e;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t.x) : "f"(den.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t.y) : "f"(den.y));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.x) : "f"(w.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.y) : "f"(w.y));
    float2 q = __ffma2_rn(t, kNA5, kNA4);
    q = __ffma2_rn(t, q, kNA3);
    q = __ffma2_rn(t, q, kNA2);
    q = __ffma2_rn(t, q, kNA1);
    q = __fmul2_rn(t, q);                       // -poly
    const float2 ea = __ffma2_rn(q, e, one);    // erf(|v| / sqrt 2)
    const float2 es = make_float2(copysignf(ea.x, va), copysignf(ea.y, vb));
    const float2 h = __fmul2_rn(v, make_float2(0.5f, 0.5f));
    return __ffma2_rn(h, es, h);                // v (1 + erf) / 2
}
// activation (0 GELU, 1 ReLU) of N (even) values in place
template <int N>
MLPF_DEV void act_n(float* v, int act) {
    if (act == 1) {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = fmaxf(v[i], 0.f);
    } else {
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            const float2 g = gelu2_f(v[i], v[i + 1]);
            v[i] = g.x;
            v[i + 1] = g.y;
        }
    }
}

// GEMM operand formats of the row-tile kernels.  A 128-byte swizzle atom holds
// 64 16-bit or 128 E4M3 K-elements; one K-step is 32 bytes in every format
// (16 elements of kind::f16, 32 of kind::f8f6f4).  A K=64 operand in E4M3 uses
// the first half of an atom (chunks 0..3); the rest stays zero.
// Precision modes (the FMT template parameter of the kernels):
//   FMT_BF16  attention in BF16 (Q, K, V^T, P; QK^T and PV on BF16 tensor cores),
//             every GEMM of the embedding, projections, FFNs and heads on FP16
//             operands: the per-stage rounding budget of the forward puts almost all
//             of the 16-bit error into the GEMM operands, almost none into the
//             attention products
//   FMT_FP16  FP16 everywhere
//   FMT_E4M3  E4M3 projection and FFN GEMMs (per-tensor scales), FP16 elsewhere
// The attention output O and h_pid are FP16 in every mode (GEMM A operands).
enum : int { FMT_BF16 = 0, FMT_FP16 = 1, FMT_E4M3 = 2 };
template <int FMT>
constexpr bool kIs8 = FMT == FMT_E4M3;
// format of Q, K, V^T and P (attention operands): FP16 unless BF16
template <int FMT>
constexpr bool kOutF16 = FMT != FMT_BF16;
// operand format of the projection and FFN GEMMs
template <int FMT>
constexpr int kGemm = FMT == FMT_BF16 ? FMT_FP16 : FMT;
// K-elements per 128-byte atom
template <int FMT>
constexpr int kAtomK = kIs8<FMT> ? 128 : 64;

// Issue a [128 x K] x [N x K]^T GEMM from swizzled smem tiles into TMEM columns.
// katoms: number of 128-byte atom columns in K.  b tile: N rows per atom column.
// accumulate: add to the existing accumulator from the first k-step on.
template <int FMT>
MLPF_DEV void issue_gemm(uint32_t d_tmem, const uint8_t* a, const uint8_t* b, int N, int katoms,
                         bool accumulate = false) {
    const uint32_t a0 = smem_u32(a), b0 = smem_u32(b);
    for (int kc = 0; kc < katoms * 4; ++kc) {
        const uint32_t ao = a0 + (kc >> 2) * ATOM + (kc & 3) * 32;
        const uint32_t bo = b0 + (kc >> 2) * (N * 128) + (kc & 3) * 32;
        const uint32_t acc = (kc > 0 || accumulate) ? 1u : 0u;
        if constexpr (kIs8<FMT>)
            mma_f8(d_tmem, sdesc_sw128(ao), sdesc_sw128(bo), idesc_e4m3(128, N), acc);
        else
            mma_f16(d_tmem, sdesc_sw128(ao), sdesc_sw128(bo), idesc_f16(128, N, FMT == FMT_FP16 ? 0u : 1u), acc);
    }
}

MLPF_DEV uint32_t pack_e4m3x4(float a, float b, float c, float d) {
    uint16_t lo, hi;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(b), "f"(a));
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(d), "f"(c));
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

// Store n (a multiple of 32) values of row r, starting at K-column k0, into the
// A-operand tile `tile` in format FMT (swizzled 128-byte rows; K-columns beyond
// one atom continue in the next atom column).  E4M3 values are v * qs.
// zero_hi (E4M3, K=64 operands): also clear the matching chunk of the unused
// upper half of the atom (the tile may hold other data there).
template <int FMT>
MLPF_DEV void st_op(uint8_t* tile, int r, const float* v, int n, int k0, float qs, bool zero_hi = false) {
    if constexpr (kIs8<FMT>) {
#pragma unroll
        for (int c = 0; c < n / 16; ++c) {
            const int k = k0 + 16 * c;
            const float* w = v + 16 * c;
            uint4 u;
            u.x = pack_e4m3x4(w[0] * qs, w[1] * qs, w[2] * qs, w[3] * qs);
            u.y = pack_e4m3x4(w[4] * qs, w[5] * qs, w[6] * qs, w[7] * qs);
            u.z = pack_e4m3x4(w[8] * qs, w[9] * qs, w[10] * qs, w[11] * qs);
            u.w = pack_e4m3x4(w[12] * qs, w[13] * qs, w[14] * qs, w[15] * qs);
            *(uint4*)(tile + (k >> 7) * ATOM + sw128_off(r, (k & 127) >> 4)) = u;
            if (zero_hi) *(uint4*)(tile + sw128_off(r, ((k & 127) >> 4) + 4)) = make_uint4(0, 0, 0, 0);
        }
    } else {
#pragma unroll
        for (int c = 0; c < n / 8; ++c) {
            const int k = k0 + 8 * c;
            const float* w = v + 8 * c;
            uint4 u;
            u.x = pack2<FMT == FMT_FP16>(w[0], w[1]);
            u.y = pack2<FMT == FMT_FP16>(w[2], w[3]);
            u.z = pack2<FMT == FMT_FP16>(w[4], w[5]);
            u.w = pack2<FMT == FMT_FP16>(w[6], w[7]);
            *(uint4*)(tile + (k >> 6) * ATOM + sw128_off(r, (k & 63) >> 3)) = u;
        }
    }
}



// Record max |v| of valid rows into amax[slot] (calibration of FP8 scales).
MLPF_DEV void record_amax(unsigned* amax, int slot, const float* v, int n, bool valid) {
    float mx = 0.f;
    for (int i = 0; i < n; ++i) mx = fmaxf(mx, fabsf(v[i]));
    unsigned u = valid ? __float_as_uint(mx) : 0u;
    u = __reduce_max_sync(0xffffffffu, u);
    if ((threadIdx.x & 31) == 0 && u) atomicMax(amax + slot, u);
}

struct RowInfo {
    bool valid;
    int prow;
};
MLPF_DEV RowInfo row_info(const int4* blk, int nblk, int p) {
    const int b = p >> 6;
    RowInfo ri{false, 0};
    if (b < nblk) {
        const int4 e = blk[b];
        ri.valid = (p & 63) < e.z;
        ri.prow = e.y + (p & 63);
    }
    return ri;
}

// ------------------------------------------------------------------ scheduler
// cu: [n_events+1].  blk[b] = {event, packed row of the block's first element,
// valid rows in the block, 0}.  items[i] = {padded row of the event's first
// element, query tile, N_e, event}, ordered by N_e descending.
// counters: [0] items, [1] padded rows, [2..33] attention tickets.
// Event sizes are clamped to [0, 65536] and every write is bounded by the
// workspace capacities, so offsets that break the contract cannot write out of
// bounds.
__global__ void __launch_bounds__(1024) k_schedule(const int32_t* __restrict__ cu, int n_events,
                                                   int4* __restrict__ blk,
                                                   int4* __restrict__ items,
                                                   int* __restrict__ counters, int cap_blocks,
                                                   int cap_items) {
    constexpr int NB = 1025;  // buckets by key-tile count (max_n <= 65536)
    __shared__ int hist[NB];
    __shared__ int wsum[32];
    __shared__ int carry;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < NB; i += 1024) hist[i] = 0;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int e = tid; e < n_events; e += 1024) {
        const int n = min(max(cu[e + 1] - cu[e], 0), 65536);
        if (n > 0) atomicAdd(&hist[(n + 63) >> 6], (n + 127) >> 7);
    }
    __syncthreads();
    {   // exclusive offsets, larger events first: a block-wide scan of buckets 1024 .. 1
        // (thread t takes bucket NB - 1 - t; bucket 0 holds no items, events of N = 0)
        const int b = NB - 1 - tid;
        const int c = hist[b];
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const int excl = incl - c + (wid > 0 ? wsum[wid - 1] : 0);
        hist[b] = excl;
        if (tid == 1023) {
            hist[0] = excl + c;
            counters[0] = excl + c;
        }
        __syncthreads();
    }
    for (int base = 0; base < n_events; base += 1024) {
        const int e = base + tid;
        const int n = e < n_events ? min(max(cu[e + 1] - cu[e], 0), 65536) : 0;
        const int nb = (n + 63) >> 6;
        int incl = nb;  // block-wide inclusive scan
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const int start = carry + incl - nb + (wid > 0 ? wsum[wid - 1] : 0);
        if (n > 0) {
            const int c0 = cu[e];
            for (int b = 0; b < nb && start + b < cap_blocks; ++b)
                blk[start + b] = make_int4(e, c0 + 64 * b, min(64, n - 64 * b), 0);
            const int nq = (n + 127) >> 7;
            const int pos = atomicAdd(&hist[nb], nq);
            // an event that does not fit the padded capacity gets no work
            const bool fits = start + nb <= cap_blocks;
            for (int qt = 0; qt < nq && pos + qt < cap_items; ++qt)
                items[pos + qt] = fits ? make_int4(start * 64, qt, n, e) : make_int4(0, 0, 0, e);
        }
        __syncthreads();
        if (tid == 1023) carry = start + nb;
        __syncthreads();
    }
    if (tid == 0) {
        counters[1] = min(carry, cap_blocks) * 64;
        counters[0] = min(counters[0], cap_items);
    }
    if (tid >= 2 && tid < 34) counters[tid] = 0;
}

// ------------------------------------------------------------ embed + QKV
struct EmbedParams {
    const float* x;
    const int4* blk;
    const int* counters;
    const uint8_t* w1;   // [64 x K1] image (K1: 42 -> one atom; 42 + 64 -> one E4M3 or two 16-bit atoms)
    const uint8_t* w2;   // [64 x 64]
    const uint8_t* wqkv; // [192 x 64]
    const float *b1, *b2, *lng, *lnb, *bqkv;
    const uint16_t* hp;  // MODE 1: h_pid rows (16-bit), read per thread in E4M3 mode and calibration
    float* z;
    uint16_t *q, *k, *vt;
    float* kmax;         // [64-row block][head] largest K-row norm (store_kmax)
    long ldvt;
    unsigned* status;
    uint64_t wait_ns;
    int act;
    // E4M3: qs[i] = 1/s_a of A operand i (input, hidden, LN1); ds[i] = s_a * s_w of GEMM i
    // (1 in the 16-bit formats)
    float qs[3], ds[3];
    unsigned* amax;      // calibration: max |A operand| of valid rows per slot, or NULL
    int slot[3];
};


// ------------------------------------------------------------ post-attention
struct PostParams {
    const float* x;
    const int4* blk;
    const int* counters;
    const uint8_t *wo, *wup, *wdn;  // [64x64], [256x64], [64x256]
    const uint8_t *wa, *wb;         // mode 0: wqkv [192x64]; 1: cls w1 [64x64], w2 [16x64];
                                    // 2: heads w1 [256x64], w2 [16x256]
    const float *bo, *ln2g, *ln2b, *bup, *bdn;
    const float *lng, *lnb;         // next LN1 (mode 0) or final LN (modes 1, 2)
    const float *ba, *bb;           // mode 0: bqkv (192); 1: cls b1 (64), b2 (16); 2: heads b1 (256), b2 (16)
    float* z;
    uint16_t *q, *k, *vt, *hp;
    float* kmax;                    // mode 0: [64-row block][head] largest K-row norm
    long ldvt;
    float* logits;
    float* reg;
    unsigned* status;
    uint64_t wait_ns;
    int act;
    // E4M3: qs = 1/s_a of the A operands (O, LN2, FFN hidden, a, b); ds = s_a * s_w of
    // the GEMMs (out-proj, FFN up, FFN down, a, b); 1 in the 16-bit formats
    float qs[5], ds[5];
    unsigned* amax;  // calibration: max |A operand| of valid rows per slot, or NULL
    int slot[5];
};

// parameter vector offsets (floats) in shared memory
constexpr int PV_BO = 0, PV_LN2G = 64, PV_LN2B = 128, PV_BUP = 192, PV_BDN = 448, PV_LNG = 512,
              PV_LNB = 576, PV_BA = 640, PV_BB = 896, PV_N = 912;
constexpr int PT_THREADS = 512;   // two teams x two warpgroups
// per team: sA (64-column operands) + sH (128 hidden columns: two 16-bit atoms, or one
// E4M3 atom followed by the 16-bit staging tile of the attention output)
constexpr uint32_t PT_TEAM_BYTES = 3 * ATOM;
constexpr int PT_RED_FLOATS = 2 * 2 * 128;            // per team: [pass][wg][row] LN partial sums

MLPF_DEV bool team_sync_or(int team, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, 256, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(1 + team)
        : "memory");
    return r != 0;
}

MLPF_DEV void team_bar(int team) {
    asm volatile("bar.sync %0, 256;" ::"r"(1 + team) : "memory");
}

// Largest K-row norm per head over each 64-row block of a 128-row tile: the
// attention kernel's bound on the scores of a key tile, |q . k| <= |q| max |k|
// (Cauchy-Schwarz), with 1 % added for the 16-bit rounding of the stored K.  Run
// by the 128 threads of warpgroup 1 (the K half) of a team, each with the squared
// per-head norms ss of its row (0 for padding rows); scratch: 16 floats of the
// team's shared memory that are free at this point.
MLPF_DEV void store_kmax(float (&ss)[4], float* scratch, int r, int team, float* kmax, int tile) {
#pragma unroll
    for (int hh = 0; hh < 4; ++hh)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss[hh] = fmaxf(ss[hh], __shfl_xor_sync(0xffffffffu, ss[hh], off));
    if ((r & 31) == 0) {
#pragma unroll
        for (int hh = 0; hh < 4; ++hh) scratch[(r >> 5) * 4 + hh] = ss[hh];
    }
    asm volatile("bar.sync %0, 128;" ::"r"(3 + team) : "memory");
    if (r < 8) {
        const int b = r >> 2, hh = r & 3;   // 64-row block b of the tile: warps 2b, 2b + 1
        kmax[(size_t)(2 * tile + b) * 4 + hh] = sqrtf(fmaxf(scratch[8 * b + hh], scratch[8 * b + 4 + hh])) * 1.01f;
    }
}
// squared norms of the two 16-channel heads in 32 values
MLPF_DEV void head_sq2(const float* u, float& s0, float& s1) {
    s0 = 0.f;
    s1 = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        s0 = fmaf(u[i], u[i], s0);
        s1 = fmaf(u[16 + i], u[16 + i], s1);
    }
}

// LayerNorm of a 64-column row whose columns are split between the two
// warpgroups of a team (32 each): two-pass FP32 moments, partial sums exchanged
// through shared memory.  z32/out32: this warpgroup's 32 columns.
MLPF_DEV void layernorm_split(const float* z32, float* out32, const float* g, const float* b, int wg,
                              int r, int team, float* red) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) s += z32[i];
    red[wg * 128 + r] = s;
    team_bar(team);
    s += red[(wg ^ 1) * 128 + r];
    const float mu = s * (1.0f / D);
    float q = 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const float t = z32[i] - mu;
        q = fmaf(t, t, q);
    }
    red[256 + wg * 128 + r] = q;
    team_bar(team);
    q += red[256 + (wg ^ 1) * 128 + r];
    const float rs = rsqrtf(q * (1.0f / D) + LN_EPS);
#pragma unroll
    for (int i = 0; i < 32; ++i) out32[i] = (z32[i] - mu) * rs * g[32 * wg + i] + b[32 * wg + i];
}

// FMT: GEMM operand format (BF16, FP16 or E4M3), FP32 accumulation in every case.
// The embedding FFN runs in FE (FP16 when FMT is E4M3: only the projection and FFN
// GEMMs of the encoder blocks use E4M3); the QKV projection runs in FMT.
// 256 threads: thread (wg, r) owns row r of the 128-row tile and, in every
// epilogue, the warpgroup's half of the columns; LayerNorm moments are combined
// through shared memory.
constexpr int EM_THREADS = 512;   // two teams (tiles in flight) x two warpgroups
constexpr int EV_N = 64 * 4 + 192;  // bias / LayerNorm floats of the embedding kernel
// Staging of a 64-row block's input rows (at most 64 x 168 contiguous bytes of x) widened
// to whole 16-byte granules: up to 15 bytes in front, the rest rounded up to 16.
constexpr uint32_t EM_XB = 16 * ((15 + 64 * 42 * 4 + 15) / 16);
template <int MODE, int FMT>  // MODE 0: input x (K = 42 -> 64); 1: concat(x, h_pid) (K = 106 -> 128)
__global__ void __launch_bounds__(EM_THREADS, 1) k_embed_qkv(const __grid_constant__ CUtensorMap map_hp,
                                                             EmbedParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    constexpr int FE = FMT_FP16;      // embedding FFN operands (16-bit in every mode)
    constexpr int G = kGemm<FMT>;     // QKV projection operands
    constexpr int KA = MODE == 0 ? 1 : 2;  // atoms of the first GEMM's A operand
    constexpr uint32_t W1B = 64 * 128 * KA, W2B = 64 * 128, WQB = 192 * 128;
    constexpr uint32_t TEAM_B = KA * ATOM + ATOM + 2 * 2 * 128 * 4;   // per team: sA, sH, LN sums
    constexpr bool TMA_HP = MODE == 1;
    constexpr bool F16 = kOutF16<FMT>;   // Q, K, V^T format
    const int tid = threadIdx.x;
    const int team = tid >> 8, wg = (tid >> 7) & 1, r = tid & 127;
    const bool leader = (tid & 255) == 0;
    uint8_t* sW1 = sm;
    uint8_t* sW2 = sW1 + W1B;
    uint8_t* sWq = sW2 + W2B;
    uint8_t* sA = sWq + WQB + team * TEAM_B;   // KA atom columns
    uint8_t* sH = sA + KA * ATOM;              // 1 atom column
    float* red = (float*)(sH + ATOM);          // [pass][wg][row] LayerNorm partial sums
    // bias and LayerNorm vectors: b1 [64], b2 [64], ln gain [64], ln shift [64], bqkv [192]
    float* pv = (float*)(sWq + WQB + 2 * TEAM_B);
    uint64_t* bars = (uint64_t*)(pv + EV_N);   // 0 weights; team t: 1 + 2t tma, 2 + 2t mma, 5 + t x rows
    uint64_t* tma_bar = &bars[1 + 2 * team];
    uint64_t* mma_bar = &bars[2 + 2 * team];
    uint64_t* x_bar = &bars[5 + team];
    uint32_t* tmem_hold = (uint32_t*)(bars + 8);
    int* abort_flag = (int*)(tmem_hold + 1);
    uint8_t* sX = (uint8_t*)(bars + 16) + team * 2 * EM_XB;   // the team's tile: two blocks of x rows

    if (tid == 0) {
        for (int i = 0; i < 7; ++i) mbar_init(&bars[i], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (tid < 32) {
        tmem_alloc(tmem_hold, 512);
        tmem_relinquish();
    }
    for (int i = tid; i < EV_N; i += EM_THREADS)
        pv[i] = i < 64 ? p.b1[i] : i < 128 ? p.b2[i - 64] : i < 192 ? p.lng[i - 128] : i < 256 ? p.lnb[i - 192]
                                                                                       : p.bqkv[i - 256] * (i < 320 ? kQScale : 1.f);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_hold + 256 * team;
    const uint32_t trow = tbase + ((uint32_t)(tid & 96) << 16);  // lane quarter of this warp
    volatile int* ab = abort_flag;

    if (tid == 0) {
        mbar_arrive_expect_tx(&bars[0], W1B + W2B + WQB);
        bulk_load(sW1, p.w1, W1B, &bars[0]);
        bulk_load(sW2, p.w2, W2B, &bars[0]);
        bulk_load(sWq, p.wqkv, WQB, &bars[0]);
    }
    bool fail = !mbar_wait(&bars[0], 0, ab, p.status, ST_TIMEOUT_GEMM, p.wait_ns);

    const int tpad = p.counters[1];
    const int nblk = tpad >> 6;
    const int ntiles = (tpad + ROWS - 1) / ROWS;
    uint32_t mph = 0, aph = 0, xph = 0;
    // The input rows of tile t: each of its two 64-row blocks holds consecutive packed rows,
    // one contiguous range of x, copied whole by the bulk-copy engine.  The range is widened
    // to whole 16-byte granules (a granule holding a byte of x lies in x's mapped page).
    // blk_of(t, e): the leader's copy of tile t's block entries (valid rows 0 past the end)
    auto blk_of = [&](int t, int4 (&e)[2]) {
#pragma unroll
        for (int b = 0; b < 2; ++b)
            e[b] = t < ntiles && 2 * t + b < nblk ? p.blk[2 * t + b] : make_int4(0, 0, 0, 0);
    };
    int x_issued = 0, h_issued = 0;   // leader: input-row copies and h_pid loads armed
    auto issue_x = [&](const int4 (&e)[2]) {
        ++x_issued;
        uint32_t bytes[2];
        const uint8_t* src[2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const uintptr_t a = (uintptr_t)(p.x + (size_t)e[b].y * 42);
            const uintptr_t a0 = a & ~(uintptr_t)15;
            const uintptr_t a1 = (a + (size_t)e[b].z * 168 + 15) & ~(uintptr_t)15;
            src[b] = (const uint8_t*)a0;
            bytes[b] = e[b].z > 0 ? (uint32_t)(a1 - a0) : 0u;
        }
        mbar_arrive_expect_tx(x_bar, bytes[0] + bytes[1]);
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (bytes[b]) bulk_load(sX + b * EM_XB, src[b], bytes[b], x_bar);
    };
    int4 enext[2];
    if (leader && blockIdx.x * 2 + team < ntiles) {
        blk_of(blockIdx.x * 2 + team, enext);
        issue_x(enext);
    }
    // the team syncs, its leader issues, everyone waits for the MMA; false on failure
    auto run_mma = [&](auto issue) -> bool {
        tc_fence_before();
        fence_proxy_async_smem();
        if (team_sync_or(team, fail)) return false;
        if (leader) {
            tc_fence_after();
            issue();
            mma_commit(mma_bar);
        }
        fail |= !mbar_wait(mma_bar, mph, ab, p.status, ST_TIMEOUT_GEMM, p.wait_ns);
        mph ^= 1;
        const bool stop = team_sync_or(team, fail);
        tc_fence_after();
        return !stop;
    };
    for (int tile = blockIdx.x * 2 + team; tile < ntiles; tile += 2 * gridDim.x) {
        if (team_sync_or(team, fail)) break;
        const int p0 = tile * ROWS;
        const int prow_pad = p0 + r;
        const RowInfo ri = row_info(p.blk, nblk, prow_pad);
        const bool more = tile + 2 * (int)gridDim.x < ntiles;
        if (leader && more) blk_of(tile + 2 * (int)gridDim.x, enext);   // used after the first GEMM
        if (TMA_HP && leader) {
            ++h_issued;
            mbar_arrive_expect_tx(tma_bar, ATOM);
            tma_load_2d(sA + ATOM, &map_hp, 0, p0, tma_bar);
            if (tile + 2 * (int)gridDim.x < ntiles) tma_prefetch_2d(&map_hp, 0, p0 + 2 * gridDim.x * ROWS);
        }
        float v[32];
        // this warpgroup's 32 of the row's 42 features (zero padded to 64), from the
        // staged block, at the row's offset from the block's first granule
        fail |= !mbar_wait(x_bar, xph, ab, p.status, ST_TIMEOUT_GEMM, p.wait_ns);
        xph ^= 1;
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
        if (ri.valid) {
            const uintptr_t a = (uintptr_t)(p.x + (size_t)(ri.prow - (r & 63)) * 42);
            const float2* src = (const float2*)(sX + (r >> 6) * EM_XB + (a & 15) + (r & 63) * 168 + 128 * wg);
            if (wg == 0) {
#pragma unroll
                for (int i = 0; i < 16; ++i) { const float2 t = src[i]; v[2 * i] = t.x; v[2 * i + 1] = t.y; }
            } else {
#pragma unroll
                for (int i = 0; i < 5; ++i) { const float2 t = src[i]; v[2 * i] = t.x; v[2 * i + 1] = t.y; }
            }
        }
        st_op<FE>(sA, r, v, 32, 32 * wg, 1.f);
        if (p.amax) {
            float amx = 0.f;
#pragma unroll
            for (int i = 0; i < 32; ++i) amx = fmaxf(amx, fabsf(v[i]));
            if (MODE == 1) {
                // this warpgroup's half of the h_pid row (16-bit, as the PID stack wrote it)
                const uint4* src = (const uint4*)(p.hp + (size_t)prow_pad * D + 32 * wg);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint4 u = src[c];
                    float a, b;
                    unpack2<true>(u.x, a, b); amx = fmaxf(amx, fmaxf(fabsf(a), fabsf(b)));
                    unpack2<true>(u.y, a, b); amx = fmaxf(amx, fmaxf(fabsf(a), fabsf(b)));
                    unpack2<true>(u.z, a, b); amx = fmaxf(amx, fmaxf(fabsf(a), fabsf(b)));
                    unpack2<true>(u.w, a, b); amx = fmaxf(amx, fmaxf(fabsf(a), fabsf(b)));
                }
            }
            record_amax(p.amax, p.slot[0], &amx, 1, ri.valid);
        }
        if (TMA_HP && leader) fail |= !mbar_wait(tma_bar, aph, ab, p.status, ST_TIMEOUT_GEMM, p.wait_ns);
        aph ^= 1;
        // embedding FFN, first layer
        if (!run_mma([&] { issue_gemm<FE>(tbase, sA, sW1, 64, KA); })) break;
        // every thread of the team has read its row: stage the team's next tile
        if (leader && more) issue_x(enext);
        tmem_ld32(trow + 32 * wg, v);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] += pv[32 * wg + i];
        act_n<32>(v, p.act);
        if (p.amax) record_amax(p.amax, p.slot[1], v, 32, ri.valid);
        st_op<FE>(sH, r, v, 32, 32 * wg, 1.f);
        // second layer: the residual stream, then LN1
        if (!run_mma([&] { issue_gemm<FE>(tbase, sH, sW2, 64, 1); })) break;
        tmem_ld32(trow + 32 * wg, v);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] += pv[64 + 32 * wg + i];
        {
            float4* zd = (float4*)(p.z + (size_t)prow_pad * D + 32 * wg);
#pragma unroll
            for (int i = 0; i < 8; ++i) zd[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
        layernorm_split(v, v, pv + 128, pv + 192, wg, r, team, red);
        if (p.amax) record_amax(p.amax, p.slot[2], v, 32, ri.valid);
        st_op<G>(sH, r, v, 32, 32 * wg, p.qs[2], true);
        // fused Q/K/V projection: warpgroup 0 stores Q and V^T columns 0-31,
        // warpgroup 1 stores K and V^T columns 32-63
        if (!run_mma([&] { issue_gemm<G>(tbase, sH, sWq, 192, 1); })) break;
        {
            const float ds = p.ds[2], dsqk = wg == 0 ? ds * kQScale : ds;
            float u[32], ss[4];
            uint16_t* dst = (wg == 0 ? p.q : p.k) + (size_t)prow_pad * D;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                tmem_ld32(trow + 64 * wg + 32 * h, u);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 32; ++i) u[i] = fmaf(u[i], dsqk, pv[256 + 64 * wg + 32 * h + i]);
                if (wg == 1) head_sq2(u, ss[2 * h], ss[2 * h + 1]);
                uint4* d4 = (uint4*)(dst + 32 * h);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    uint4 w4;
                    w4.x = pack2<F16>(u[8 * c + 0], u[8 * c + 1]);
                    w4.y = pack2<F16>(u[8 * c + 2], u[8 * c + 3]);
                    w4.z = pack2<F16>(u[8 * c + 4], u[8 * c + 5]);
                    w4.w = pack2<F16>(u[8 * c + 6], u[8 * c + 7]);
                    d4[c] = w4;
                }
            }
            if (wg == 1) {
#pragma unroll
                for (int hh = 0; hh < 4; ++hh) ss[hh] = ri.valid ? ss[hh] : 0.f;
                store_kmax(ss, red, r, team, p.kmax, tile);
            }
            tmem_ld32(trow + 128 + 32 * wg, u);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int ch = 32 * wg + i;
                const float t = ri.valid ? fmaf(u[i], ds, pv[256 + 128 + ch]) : 0.f;
                p.vt[(size_t)ch * p.ldvt + prow_pad] = (uint16_t)(pack2<F16>(t, 0.f) & 0xffffu);
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (*ab) {
        // let the copies still in flight land before the CTA exits: the last armed
        // phase of each barrier (bounded waits; a timed grace period only if one fails)
        bool landed = true;
        if (tid == 0) landed &= mbar_drain(&bars[0], 0, p.wait_ns);
        if (leader && x_issued > 0) landed &= mbar_drain(x_bar, (x_issued - 1) & 1, p.wait_ns);
        if (leader && h_issued > 0) landed &= mbar_drain(tma_bar, (h_issued - 1) & 1, p.wait_ns);
        if (!landed)
            for (int i = 0; i < 1000; ++i) __nanosleep(1000);
    }
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        tmem_dealloc(*tmem_hold, 512);
    }
}

template <int MODE, int FMT>  // 0: next layer LN1 + QKV; 1: end of PID stack; 2: end of regression stack
__global__ void __launch_bounds__(PT_THREADS, 1) k_post(const __grid_constant__ CUtensorMap map_o,
                                                        PostParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    // G: out-projection, FFN and QKV GEMMs; FH: output heads (FP16 in every mode)
    constexpr int G = kGemm<FMT>;
    constexpr int FH = FMT_FP16;
    constexpr bool F16 = kOutF16<FMT>;           // format of Q, K, V^T (O and h_pid: FP16)
    constexpr int HA = kIs8<G> ? 1 : 2;          // atoms of a 128-column FFN hidden operand
    constexpr int KA256 = 256 / kAtomK<G>;       // atoms of the 256-column FFN-down operand
    constexpr uint32_t WOB = 64 * 128, WUB = 256 * 128, WDB = KA256 * 64 * 128;
    constexpr uint32_t WAB = MODE == 0 ? 192 * 128 : (MODE == 1 ? 64 * 128 : 256 * 128);
    constexpr uint32_t WBB = MODE == 0 ? 0 : (MODE == 1 ? 16 * 128 : 4 * 16 * 128);
    uint8_t* sWo = sm;
    uint8_t* sWu = sWo + WOB;
    uint8_t* sWd = sWu + WUB;
    uint8_t* sWa = sWd + WDB;
    uint8_t* sWb = sWa + WAB;
    uint8_t* sTeam0 = sWb + ((WBB + 1023) & ~1023u);
    float* pv = (float*)(sTeam0 + 2 * PT_TEAM_BYTES);
    float* red_all = pv + PV_N;               // [team][PT_RED_FLOATS]
    uint64_t* bars = (uint64_t*)(red_all + 2 * PT_RED_FLOATS);  // 0 weights; team t: 1+2t tma, 2+2t mma
    uint32_t* tmem_hold = (uint32_t*)(bars + 6);
    int* abort_flag = (int*)(tmem_hold + 1);
    const int tid = threadIdx.x;
    const int team = tid >> 8, wg = (tid >> 7) & 1, r = tid & 127;
    const bool leader = (tid & 255) == 0;
    uint8_t* sA = sTeam0 + team * PT_TEAM_BYTES;
    uint8_t* sH = sA + ATOM;
    uint8_t* sO16 = kIs8<G> ? sA + 2 * ATOM : sA;  // where the attention output lands
    uint64_t* tma_bar = &bars[1 + 2 * team];
    uint64_t* mma_bar = &bars[2 + 2 * team];
    float* red = red_all + team * PT_RED_FLOATS;

    if (tid == 0) {
        for (int i = 0; i < 5; ++i) mbar_init(&bars[i], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (tid < 32) {
        tmem_alloc(tmem_hold, 512);
        tmem_relinquish();
    }
    // bias / LayerNorm vectors into shared memory
    for (int i = tid; i < PV_N; i += PT_THREADS) {
        float v = 0.f;
        if (i < PV_LN2G) v = p.bo[i - PV_BO];
        else if (i < PV_LN2B) v = p.ln2g[i - PV_LN2G];
        else if (i < PV_BUP) v = p.ln2b[i - PV_LN2B];
        else if (i < PV_BDN) v = p.bup[i - PV_BUP];
        else if (i < PV_LNG) v = p.bdn[i - PV_BDN];
        else if (i < PV_LNB) v = p.lng[i - PV_LNG];
        else if (i < PV_BA) v = p.lnb[i - PV_LNB];
        else if (i < PV_BB) {
            const int n = MODE == 0 ? 192 : (MODE == 1 ? 64 : 256);
            v = (i - PV_BA) < n ? p.ba[i - PV_BA] : 0.f;
            if (MODE == 0 && i - PV_BA < 64) v *= kQScale;   // Q bias
        } else v = MODE == 0 ? 0.f : p.bb[i - PV_BB];
        pv[i] = v;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_hold + 256 * team;
    const uint32_t trow = tbase + ((uint32_t)(tid & 96) << 16);
    volatile int* ab = abort_flag;
    if (tid == 0) {
        mbar_arrive_expect_tx(&bars[0], WOB + WUB + WDB + WAB + WBB);
        bulk_load(sWo, p.wo, WOB, &bars[0]);
        bulk_load(sWu, p.wup, WUB, &bars[0]);
        bulk_load(sWd, p.wdn, WDB, &bars[0]);
        bulk_load(sWa, p.wa, WAB, &bars[0]);
        if (WBB) bulk_load(sWb, p.wb, WBB, &bars[0]);
    }
    bool fail = !mbar_wait(&bars[0], 0, ab, p.status, ST_TIMEOUT_GEMM, p.wait_ns);

    const int tpad = p.counters[1];
    const int nblk = tpad >> 6;
    const int ntiles = (tpad + ROWS - 1) / ROWS;
    uint32_t mph = 0, aph = 0;
    int o_issued = 0;   // leader: attention-output tile loads armed
    // sync the team, let its leader issue MMAs, wait for them; false on failure
    auto run_mma = [&](auto issue) -> bool {
        tc_fence_before();
        fence_proxy_async_smem();
        if (team_sync_or(team, fail)) return false;
        if (leader) {
            tc_fence_after();
            issue();
            mma_commit(mma_bar);
        }
        fail |= !mbar_wait(mma_bar, mph, ab, p.status, ST_TIMEOUT_GEMM, p.wait_ns);
        mph ^= 1;
        const bool stop = team_sync_or(team, fail);
        tc_fence_after();
        return !stop;
    };
    for (int tile = blockIdx.x * 2 + team; tile < ntiles; tile += 2 * gridDim.x) {
        if (team_sync_or(team, fail)) break;
        const int pp = tile * ROWS + r;
        const RowInfo ri = row_info(p.blk, nblk, pp);
        if (leader) {
            ++o_issued;
            mbar_arrive_expect_tx(tma_bar, ATOM);
            tma_load_2d(sO16, &map_o, 0, tile * ROWS, tma_bar);
        }
        // the team's next attention-output tile into L2 (its TMA load is on the
        // critical path of the next tile)
        if (leader && tile + 2 * (int)gridDim.x < ntiles) tma_prefetch_2d(&map_o, 0, (tile + 2 * gridDim.x) * ROWS);
        float zr[32], v[32];   // this warpgroup's 32 columns of the residual row
        {
            const float4* zs = (const float4*)(p.z + (size_t)pp * D + 32 * wg);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 t = zs[i];
                zr[4 * i] = t.x; zr[4 * i + 1] = t.y; zr[4 * i + 2] = t.z; zr[4 * i + 3] = t.w;
            }
        }
        fail |= !mbar_wait(tma_bar, aph, ab, p.status, ST_TIMEOUT_GEMM, p.wait_ns);
        aph ^= 1;
        if (kIs8<G> || p.amax) {
            // this warpgroup's 32 columns of the attention output (16-bit swizzled tile)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint4 u = *(const uint4*)(sO16 + sw128_off(r, 4 * wg + c));
                unpack2<true>(u.x, v[8 * c], v[8 * c + 1]);
                unpack2<true>(u.y, v[8 * c + 2], v[8 * c + 3]);
                unpack2<true>(u.z, v[8 * c + 4], v[8 * c + 5]);
                unpack2<true>(u.w, v[8 * c + 6], v[8 * c + 7]);
            }
            if (p.amax) record_amax(p.amax, p.slot[0], v, 32, ri.valid);
            if constexpr (kIs8<G>) st_op<G>(sA, r, v, 32, 32 * wg, p.qs[0], true);
        }
        // out-projection + residual, LN2
        if (!run_mma([&] { issue_gemm<G>(tbase, sA, sWo, 64, 1); })) break;
        tmem_ld32(trow + 32 * wg, v);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 32; ++i) zr[i] += fmaf(v[i], p.ds[0], pv[PV_BO + 32 * wg + i]);
        // the element's log pT and log E for the decode at the end of the tile
        if (MODE == 2 && wg == 0 && ri.valid) prefetch_l2(p.x + (size_t)ri.prow * 42 + 8);
        layernorm_split(zr, v, pv + PV_LN2G, pv + PV_LN2B, wg, r, team, red);
        if (p.amax) record_amax(p.amax, p.slot[1], v, 32, ri.valid);
        st_op<G>(sA, r, v, 32, 32 * wg, p.qs[1], true);
        // FFN: two halves of 128 hidden columns, GELU, down-projection accumulated
        bool stop = false;
#pragma unroll 1
        for (int half = 0; half < 2 && !stop; ++half) {
            if (!run_mma([&] { issue_gemm<G>(tbase, sA, sWu + half * 128 * 128, 128, 1); })) { stop = true; break; }
#pragma unroll
            for (int q2 = 0; q2 < 2; ++q2) {
                tmem_ld32(trow + 64 * wg + 32 * q2, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    v[i] = fmaf(v[i], p.ds[1], pv[PV_BUP + 128 * half + 64 * wg + 32 * q2 + i]);
                act_n<32>(v, p.act);
                if (p.amax) record_amax(p.amax, p.slot[2], v, 32, ri.valid);
                st_op<G>(sH, r, v, 32, 64 * wg + 32 * q2, p.qs[2]);
            }
            if (!run_mma([&] { issue_gemm<G>(tbase + 128, sH, sWd + half * HA * 64 * 128, 64, HA, half > 0); })) {
                stop = true;
                break;
            }
        }
        if (stop) break;
        tmem_ld32(trow + 128 + 32 * wg, v);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 32; ++i) zr[i] += fmaf(v[i], p.ds[2], pv[PV_BDN + 32 * wg + i]);
        if (MODE == 0) {
            float4* zd = (float4*)(p.z + (size_t)pp * D + 32 * wg);
#pragma unroll
            for (int i = 0; i < 8; ++i) zd[i] = make_float4(zr[4 * i], zr[4 * i + 1], zr[4 * i + 2], zr[4 * i + 3]);
            layernorm_split(zr, v, pv + PV_LNG, pv + PV_LNB, wg, r, team, red);
            if (p.amax) record_amax(p.amax, p.slot[3], v, 32, ri.valid);
            st_op<G>(sA, r, v, 32, 32 * wg, p.qs[3], true);
            if (!run_mma([&] { issue_gemm<G>(tbase, sA, sWa, 192, 1); })) break;
            // wg 0: Q and V channels 0..31; wg 1: K and V channels 32..63
            uint16_t* qk = (wg == 0 ? p.q : p.k) + (size_t)pp * D;
            const float dsqk = wg == 0 ? p.ds[3] * kQScale : p.ds[3];
            float ss[4];
#pragma unroll
            for (int q2 = 0; q2 < 2; ++q2) {
                tmem_ld32(trow + 64 * wg + 32 * q2, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = fmaf(v[i], dsqk, pv[PV_BA + 64 * wg + 32 * q2 + i]);
                if (wg == 1) head_sq2(v, ss[2 * q2], ss[2 * q2 + 1]);
                uint4* d4 = (uint4*)(qk + 32 * q2);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    d4[c] = make_uint4(pack2<F16>(v[8 * c], v[8 * c + 1]), pack2<F16>(v[8 * c + 2], v[8 * c + 3]),
                                       pack2<F16>(v[8 * c + 4], v[8 * c + 5]), pack2<F16>(v[8 * c + 6], v[8 * c + 7]));
            }
            if (wg == 1) {
#pragma unroll
                for (int hh = 0; hh < 4; ++hh) ss[hh] = ri.valid ? ss[hh] : 0.f;
                store_kmax(ss, red, r, team, p.kmax, tile);
            }
            tmem_ld32(trow + 128 + 32 * wg, v);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float t = ri.valid ? fmaf(v[i], p.ds[3], pv[PV_BA + 128 + 32 * wg + i]) : 0.f;
                p.vt[(size_t)(32 * wg + i) * p.ldvt + pp] = (uint16_t)(pack2<F16>(t, 0.f) & 0xffffu);
            }
        } else if (MODE == 1) {
            layernorm_split(zr, v, pv + PV_LNG, pv + PV_LNB, wg, r, team, red);  // h_pid
            {
                uint4* d4 = (uint4*)(p.hp + (size_t)pp * D + 32 * wg);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    d4[c] = make_uint4(pack_f16x2(v[8 * c], v[8 * c + 1]), pack_f16x2(v[8 * c + 2], v[8 * c + 3]),
                                       pack_f16x2(v[8 * c + 4], v[8 * c + 5]), pack_f16x2(v[8 * c + 6], v[8 * c + 7]));
            }
            if (p.amax) record_amax(p.amax, p.slot[3], v, 32, ri.valid);
            st_op<FH>(sA, r, v, 32, 32 * wg, 1.f);
            if (!run_mma([&] { issue_gemm<FH>(tbase, sA, sWa, 64, 1); })) break;
            tmem_ld32(trow + 32 * wg, v);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] += pv[PV_BA + 32 * wg + i];
            act_n<32>(v, p.act);
            if (p.amax) record_amax(p.amax, p.slot[4], v, 32, ri.valid);
            st_op<FH>(sH, r, v, 32, 32 * wg, 1.f);
            if (!run_mma([&] { issue_gemm<FH>(tbase + 64, sH, sWb, 16, 1); })) break;
            if (wg == 0) {
                tmem_ld16(trow + 64, v);
                tmem_wait_ld();
                if (ri.valid) {
                    float2* lo = (float2*)(p.logits + (size_t)ri.prow * 6);
#pragma unroll
                    for (int c2 = 0; c2 < 3; ++c2)
                        lo[c2] = make_float2(v[2 * c2] + pv[PV_BB + 2 * c2], v[2 * c2 + 1] + pv[PV_BB + 2 * c2 + 1]);
                }
            }
        } else {
            layernorm_split(zr, v, pv + PV_LNG, pv + PV_LNB, wg, r, team, red);  // h_reg
            if (p.amax) record_amax(p.amax, p.slot[3], v, 32, ri.valid);
            st_op<FH>(sA, r, v, 32, 32 * wg, 1.f);
#pragma unroll 1
            for (int half = 0; half < 2 && !stop; ++half) {
                if (!run_mma([&] { issue_gemm<FH>(tbase, sA, sWa + half * 128 * 128, 128, 1); })) { stop = true; break; }
#pragma unroll
                for (int q2 = 0; q2 < 2; ++q2) {
                    tmem_ld32(trow + 64 * wg + 32 * q2, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        v[i] += pv[PV_BA + 128 * half + 64 * wg + 32 * q2 + i];
                    act_n<32>(v, p.act);
                    if (p.amax) record_amax(p.amax, p.slot[4], v, 32, ri.valid);
                    st_op<FH>(sH, r, v, 32, 64 * wg + 32 * q2, 1.f);
                }
                if (!run_mma([&] { issue_gemm<FH>(tbase + 128, sH, sWb + half * 2 * 16 * 128, 16, 2, half > 0); })) {
                    stop = true;
                    break;
                }
            }
            if (stop) break;
            if (wg == 0) {
                tmem_ld16(trow + 128, v);
                tmem_wait_ld();
                if (ri.valid) {
                    float o[5];
#pragma unroll
                    for (int c2 = 0; c2 < 5; ++c2) o[c2] = v[c2] + pv[PV_BB + c2];
                    const float* xr = p.x + (size_t)ri.prow * 42;
                    float* rg = p.reg + (size_t)ri.prow * 5;
                    rg[0] = expf(__ldg(xr + 8) + o[0]);
                    rg[1] = o[1];
                    rg[2] = o[2];
                    rg[3] = o[3];
                    rg[4] = expf(__ldg(xr + 9) + o[4]);
                }
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (*ab) {
        // the last armed phase of each copy barrier (bounded waits; a timed grace
        // period only if one fails)
        bool landed = true;
        if (tid == 0) landed &= mbar_drain(&bars[0], 0, p.wait_ns);
        if (leader && o_issued > 0) landed &= mbar_drain(tma_bar, (o_issued - 1) & 1, p.wait_ns);
        if (!landed)
            for (int i = 0; i < 1000; ++i) __nanosleep(1000);
    }
    __syncthreads();
    if (tid < 32) {
        tc_fence_after();
        tmem_dealloc(*tmem_hold, 512);
    }
}

// ------------------------------------------------------------- attention
// Varlen self-attention (Sec. 5.3, Eq. 4) within each event of the packed batch.
// Work items are (event, 128-query tile), longest events first; keys come in
// 64-row tiles of the same event (events start at 64-row boundaries of the padded
// layout, so a key tile never mixes events; padding keys are masked).  Two kernel
// families, chosen per batch by the autotuner: k_attention_tm (S and P in tensor
// memory, tcgen05 products) and k_attention_warp (warp-level MMAs).
constexpr uint32_t AT_QB = 128 * 128;   // Q tile bytes (128 rows x 64 ch, 16-bit)
constexpr uint32_t AT_KB = 64 * 128;    // K tile bytes (64 keys x 64 ch)
constexpr uint32_t AT_VB = 64 * 128;    // V^T tile bytes (64 ch x 64 keys)
struct AttnParams {
    const int4* items;
    int* counters;
    int layer;
    uint16_t* out;
    unsigned* status;
    uint64_t wait_ns;
    int debug_stall;
    int window;   // > 0: the query tile y attends to keys of 128-row blocks y - window .. y + window
    const float* kmax;   // [64-row block][head] largest K-row norm (warp-MMA kernel)
};

// Keys [kb, ke) of the event that query tile y (128 rows) attends to.
MLPF_DEV void key_range(int y, int n, int window, int& kb, int& ke) {
    kb = 0;
    ke = n;
    if (window > 0) {
        kb = max(0, (y - window) * ROWS);
        ke = min(n, (y + window + 1) * ROWS);
    }
}

// Largest excess (log2 units) of a tile's row max over the exponent reference
// before the tile is redone: P <= 16, far inside the FP16 and BF16 ranges.
constexpr float kStaleMax = 4.f;
// Largest exponent a key tile may reach without the maxima check (the warp
// kernel's bound path): P <= 2^15 inside the FP16 range (65504); with FP16
// operands P <= 2^13.5, so that the sum of a tile's four P values per key column
// (the row-sum operand, kTileSum) stays inside it too.
template <bool F16>
constexpr float kLimit = F16 ? 13.5f : 15.f;

MLPF_DEV float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// (d0, d1) = (a0, a1) * s + (t, t), one packed FP32x2 FMA
MLPF_DEV void ffma2_bcast(float& d0, float& d1, float a0, float a1, float s, float t) {
    uint64_t a, b, c, d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %1};" : "=l"(b) : "f"(s));
    asm("mov.b64 %0, {%1, %1};" : "=l"(c) : "f"(t));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d0), "=f"(d1) : "l"(d));
}

MLPF_DEV bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* ab, unsigned* status,
                        uint64_t wait_ns) {
    const bool ok = mbar_wait(bar, parity, ab, status, ST_TIMEOUT_ATTN, wait_ns);
    return __all_sync(0xffffffffu, ok);
}

// The TMA producer of the warp-level attention kernels (one thread): takes work
// items with the atomic ticket (a ticket is an item for QR = 128, or half of one for
// QR = 64; halves without query rows are skipped), loads each item's Q tile into one
// of two buffers and streams its 64-key K and V^T tiles with their per-head K-norm
// bounds through ST stages.  info[qb] carries the item (x < 0: no more items) to the
// consumers of Q buffer qb.  On an abort it lets the copies still in flight land.
template <int ST, int QR>
MLPF_DEV void attn_produce(const CUtensorMap* map_q, const CUtensorMap* map_k, const CUtensorMap* map_vt,
                           const AttnParams& p, uint8_t* sQ, uint8_t* sK, uint8_t* sV, float* kn,
                           uint64_t* q_full, uint64_t* q_empty, uint64_t* kv_full, uint64_t* kv_empty, int4* info,
                           volatile int* ab, int n_items, int* ticket) {
    constexpr uint32_t QB = QR * 128;
    tma_prefetch_map(map_q);
    tma_prefetch_map(map_k);
    tma_prefetch_map(map_vt);
    int q_it = 0, q_armed = 0;
    uint32_t g = 0;
    bool ok = true;
    while (ok) {
        const int t = atomicAdd(ticket, 1);
        const int item = QR == 128 ? t : t >> 1, half = QR == 128 ? 0 : t & 1;
        int4 it = make_int4(-1, 0, 0, 0);
        if (item < n_items) {
            it = p.items[item];
            it.w = half;
            if (it.z - it.y * ROWS - QR * half <= 0) continue;
        }
        const int qb = q_it & 1;
        if (q_it >= 2 && !mbar_wait(&q_empty[qb], ((q_it >> 1) - 1) & 1, ab, p.status, ST_TIMEOUT_ATTN, p.wait_ns))
            break;
        if (item >= n_items) {
            info[qb] = it;
            mbar_arrive(&q_full[qb]);
            break;
        }
        info[qb] = it;
        mbar_arrive_expect_tx(&q_full[qb], QB);
        tma_load_2d(sQ + qb * QB, map_q, 0, it.x + it.y * ROWS + QR * half, &q_full[qb]);
        ++q_armed;
        int kb, ke;
        key_range(it.y, it.z, p.window, kb, ke);
        const int nk = (ke - kb + 63) >> 6;
        for (int j = 0; j < nk; ++j, ++g) {
            const int s = (int)(g % ST);
            if (g >= ST && !mbar_wait(&kv_empty[s], ((g / ST) - 1) & 1, ab, p.status, ST_TIMEOUT_ATTN, p.wait_ns)) {
                ok = false;
                break;
            }
            // the tile's K and V^T and its per-head K-norm bounds (a 64-row block:
            // events start at 64-row boundaries, kb is a multiple of 128)
            mbar_arrive_expect_tx(&kv_full[s], AT_KB + AT_VB + 16);
            tma_load_2d(sK + s * AT_KB, map_k, 0, it.x + kb + 64 * j, &kv_full[s]);
            tma_load_2d(sV + s * AT_VB, map_vt, it.x + kb + 64 * j, 0, &kv_full[s]);
            bulk_load(kn + 4 * s, p.kmax + (size_t)(((it.x + kb) >> 6) + j) * 4, 16, &kv_full[s]);
        }
        ++q_it;
    }
    // on an abort, let the copies still in flight land before the CTA exits: wait
    // (bounded) for the last armed phase of every stage and Q buffer
    if (*ab) {
        bool landed = true;
        for (uint32_t t = g > ST ? g - ST : 0; t < g; ++t)
            landed &= mbar_drain(&kv_full[t % ST], (t / ST) & 1, p.wait_ns);
        for (int i = q_armed > 2 ? q_armed - 2 : 0; i < q_armed; ++i)
            landed &= mbar_drain(&q_full[i & 1], (i >> 1) & 1, p.wait_ns);
        if (!landed)   // a copy that never completes: a last, timed grace period
            for (int i = 0; i < 1000; ++i) __nanosleep(1000);
    }
}

// Attention with warp-level MMAs (m16n8k16).  With a head width of 16 the
// contractions are tiny (one K-step for QK^T, 16 keys per PV step) and the
// kernel is bound by the softmax; a 128-row tcgen05 MMA would tie the four
// warps of a warpgroup together at every key tile.  Here each warp owns 32
// query rows of one head end to end: S comes out of the MMA in registers, the
// exponentials are packed straight into the A fragments of the PV MMA, and the
// row sums are one more MMA against a constant block of ones, so the warps
// meet only at the K/V stage barriers.  Softmax rescaling is lazy: the exponent
// reference of a row is raised (and O, l rescaled) only when a 16-key step
// exceeds it by more than kStaleMax, so P <= 2^kStaleMax.  Q arrives scaled by
// kQScale and the QK^T MMA starts from the negated references, so its output is
// the exponent itself (no per-score multiply-add).
// QR: query rows per work item, 128 (one CTA per SM, 16 consumer warps) or 64
// (half items, two CTAs per SM of 8 consumer warps).
// HY (QR = 128 only): QK^T on the tensor cores instead: an MMA warp issues, per head
// and key tile, S = Q_h K_h^T (tcgen05, M 128, N 64, K 16) into one of two tensor-
// memory buffers per head (4 heads x 2 x 64 columns = 512), and each consumer warp
// loads its 32 rows of S with tcgen05.ld.16x256b, whose thread layout is the m16n8
// accumulator layout of the PV MMA's inputs; the references are subtracted with
// packed FP32 adds.  The QK^T MMAs (four of the ten warp-level MMAs per warp and
// 16-key step) leave the legacy tensor pipe, which bounds the kernel otherwise.
template <int QR, bool HY = false>
constexpr int aw_threads() { return NH * (QR / 32) * 32 + 32 + (HY ? 32 : 0); }   // consumers, TMA warp, MMA warp
template <int ST, int QR = 128>
struct AwLayout {
    static constexpr uint32_t QB = QR * 128;   // Q tile bytes
    static constexpr uint32_t OFF_K = 2 * QB;
    static constexpr uint32_t OFF_V = OFF_K + ST * AT_KB;
    static constexpr uint32_t OFF_BAR = OFF_V + ST * AT_VB;   // barriers, item info, flags (< 384 B)
    static constexpr uint32_t OFF_KN = OFF_BAR + 384;         // [ST][4] key-tile norm bounds (ST <= 8)
    static constexpr uint32_t SMEM = OFF_BAR + 512 + 1024;
};
static_assert((4 + 2 * 8 + 2 + 8 + 8 + 2) * 8 + 2 * 16 + 8 <= 384, "warp attention barrier area");

template <bool F16, int ST, int QR = 128, bool HY = false>
__global__ void __launch_bounds__(aw_threads<QR, HY>(), QR == 128 ? 1 : 2)
    k_attention_warp(const __grid_constant__ CUtensorMap map_q, const __grid_constant__ CUtensorMap map_k,
                     const __grid_constant__ CUtensorMap map_vt, AttnParams p) {
    static_assert(!HY || QR == 128, "tensor-memory scores need 128-row items");
    constexpr int RB = QR / 32;   // 32-row blocks (one per warp) per item
    constexpr int NW = NH * RB;   // consumer warps
    constexpr bool kTileSum = F16;   // bound path: one row-sum MMA per tile (FP16 operands)
    constexpr int SB = 1;   // 16-key steps per maxima check of the checked path (two: slower)
    constexpr uint32_t QB = AwLayout<ST, QR>::QB;
    using LY = AwLayout<ST, QR>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint8_t* sQ = sm;
    uint8_t* sK = sm + LY::OFF_K;
    uint8_t* sV = sm + LY::OFF_V;
    uint64_t* bars = (uint64_t*)(sm + LY::OFF_BAR);
    uint64_t* q_full = bars;            // [2]
    uint64_t* q_empty = bars + 2;       // [2], one arrival per consumer warp
    uint64_t* kv_full = bars + 4;       // [ST]
    uint64_t* kv_empty = kv_full + ST;  // [ST], one arrival per consumer warp
    uint64_t* never = kv_empty + ST;    // armed by nobody (debug stall)
    uint64_t* s_full = never + 2;       // HY: [head][buffer], MMA commit: S ready
    uint64_t* s_free = s_full + 8;      // HY: [head][buffer], one arrival per warp of the head
    uint64_t* drain = s_free + 8;       // HY: the MMA warp's exit
    int4* info = (int4*)(drain + 2);    // [2]
    int* abort_flag = (int*)(info + 2);
    uint32_t* tmem_hold = (uint32_t*)(abort_flag + 1);
    float* kn = (float*)(sm + LY::OFF_KN);   // per stage and head: largest K-row norm of the tile
    volatile int* ab = abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        // HY: Q and K/V stages are also released by the MMA warp's commits
        for (int i = 0; i < 2; ++i) { mbar_init(&q_full[i], 1); mbar_init(&q_empty[i], NW + (HY ? 1 : 0)); }
        for (int i = 0; i < ST; ++i) { mbar_init(&kv_full[i], 1); mbar_init(&kv_empty[i], NW + (HY ? 1 : 0)); }
        mbar_init(never, 1);
        if constexpr (HY) {
            for (int i = 0; i < 8; ++i) { mbar_init(&s_full[i], 1); mbar_init(&s_free[i], RB); }
            mbar_init(drain, 1);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (HY && warp == 0) {
        tmem_alloc(tmem_hold, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = HY ? *tmem_hold : 0u;
    const int n_items = p.counters[0];
    int* ticket = p.counters + 2 + p.layer;

    if (warp == NW) {
        // ------------------------------------------------ TMA producer (64-key stages)
        if (lane == 0)
            attn_produce<ST, QR>(&map_q, &map_k, &map_vt, p, sQ, sK, sV, kn, q_full, q_empty, kv_full, kv_empty,
                                 info, ab, n_items, ticket);
    } else if (HY && warp == NW + 1) {
        // ------------------------------------------------ HY: QK^T issue (one thread)
        if (lane == 0) {
            const uint32_t IQK = idesc_f16(128, 64, F16 ? 0u : 1u);
            int q_it = 0;
            uint32_t g = 0;
            bool ok = true;
            while (ok) {
                const int qb = q_it & 1;
                if (!mbar_wait(&q_full[qb], (q_it >> 1) & 1, ab, p.status, ST_TIMEOUT_ATTN, p.wait_ns)) break;
                const int4 it = info[qb];
                if (it.x < 0) break;
                int kb, ke;
                key_range(it.y, it.z, p.window, kb, ke);
                const int nk = (ke - kb + 63) >> 6;
                const uint32_t qa = smem_u32(sQ + qb * QB);
                for (int j = 0; j < nk && ok; ++j) {
                    const uint32_t t = g + j, s = t % ST, b = t & 1;
                    if (!mbar_wait(&kv_full[s], (t / ST) & 1, ab, p.status, ST_TIMEOUT_ATTN, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t ka = smem_u32(sK + s * AT_KB);
                    for (int h = 0; h < NH; ++h) {
                        // buffer b of head h: its four warps have read S of tile t - 2
                        if (t >= 2 && !mbar_wait(&s_free[2 * h + b], ((t >> 1) - 1) & 1, ab, p.status,
                                                 ST_TIMEOUT_ATTN, p.wait_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        mma_f16(tbase + h * 128 + b * 64, sdesc_sw128(qa + h * 32), sdesc_sw128(ka + h * 32), IQK, 0);
                        mma_commit(&s_full[2 * h + b]);
                    }
                    if (ok) mma_commit(&kv_empty[s]);
                }
                if (!ok) break;
                mma_commit(&q_empty[qb]);
                g += nk;
                ++q_it;
            }
            // every MMA issued complete before tensor memory and shared memory are released
            mma_commit(drain);
            mbar_drain(drain, 0, p.wait_ns);
        }
    } else {
        // ------------------------------------------------ warp: head h, query rows 32 rb .. 32 rb + 31
        // Fragments (m16n8k16): lane = 4 gq + tq; an accumulator holds rows gq
        // and gq + 8 of its 16-row tile at columns 2 tq, 2 tq + 1.
        const int h = warp / RB, rb = warp % RB;
        const int gq = lane >> 2, tq = lane & 3;
        const int mi = lane >> 3;                    // ldmatrix: matrix this lane addresses
        const uint32_t ONE2 = F16 ? 0x3C003C00u : 0x3F803F80u;
        (void)ONE2;
        const uint32_t sQa = smem_u32(sQ), sKa = smem_u32(sK), sVa = smem_u32(sV);
        // per-lane ldmatrix offsets: K rows (keys) + channel chunk; V^T rows (channels) + key chunk
        const int k_row = (lane & 7) + 8 * (mi >> 1), k_chunk = 2 * h + (mi & 1);
        const int v_row = h * 16 + (lane & 7) + 8 * (mi >> 1), v_sub = mi & 1;
        const uint32_t koff = sw128_off(k_row, k_chunk);   // K fragment offset of step 0
        int voff[4];   // this lane's V^T fragment offsets of the four 16-key steps
#pragma unroll
        for (int q = 0; q < 4; ++q) voff[q] = (int)sw128_off(v_row, 2 * q + v_sub);
        (void)voff;
        int q_it = 0;
        uint32_t g = 0;
        bool ok = true;
        while (ok) {
            const int qb = q_it & 1;
            if (!warp_wait(&q_full[qb], (q_it >> 1) & 1, ab, p.status, p.wait_ns)) break;
            const int4 it = info[qb];
            if (it.x < 0) break;
            if (p.debug_stall && !warp_wait(never, 0, ab, p.status, p.wait_ns)) break;
            int kb, ke;
            key_range(it.y, it.z, p.window, kb, ke);
            const int nk = (ke - kb + 63) >> 6;
            // Q fragments of the two 16-row tiles (one K-step: the head's 16 channels);
            // the second tile's rows are 16 further (same swizzle phase)
            const uint32_t qfa = sQa + qb * QB + sw128_off(rb * 32 + (lane & 15), 2 * h + (lane >> 4));
            uint32_t qa[2][4];
            auto load_q = [&]() {
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) ldsm_x4(qfa + 2048u * mt, qa[mt][0], qa[mt][1], qa[mt][2], qa[mt][3]);
            };
            // |q| of the fragment's rows (quad sums over the head's 16 channels), for
            // the key tiles' score bounds |q| max |k|; 1 % for the FP32 sums
            float qn[2][2];
            load_q();
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int hr = 0; hr < 2; ++hr) {
                    float a0, a1, a2, a3;
                    unpack2<F16>(qa[mt][hr], a0, a1);
                    unpack2<F16>(qa[mt][2 + hr], a2, a3);
                    float t = fmaf(a0, a0, fmaf(a1, a1, fmaf(a2, a2, a3 * a3)));
                    t += __shfl_xor_sync(0xffffffffu, t, 1);
                    t += __shfl_xor_sync(0xffffffffu, t, 2);
                    qn[mt][hr] = sqrtf(t) * 1.01f;
                }
            __syncwarp();
            if (lane == 0) mbar_arrive(&q_empty[qb]);
            // o: output accumulators; la: row sums (the ones-MMA accumulator, every
            // column holds its row's sum); nr: the negated exponent references of the
            // fragment's rows as an accumulator input, so that the QK^T MMA (Q
            // pre-scaled) yields the exponent S - ref itself.  The first block of
            // steps always sets the references.
            float o[2][2][4], la[2][4], nr[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    o[mt][0][e] = 0.f;
                    o[mt][1][e] = 0.f;
                    la[mt][e] = 0.f;
                    nr[mt][e] = 0.f;
                }
            }
            // HY: S - ref for keys 16q .. 16q+15 of global key tile t from the head's
            // tensor-memory buffer (t & 1): this warp's lanes 32 rb .. 32 rb + 31, the two
            // 16-row blocks in accumulator layout, then the negated references added
            auto s_tmem = [&](uint32_t t, int q, float (&dst)[2][2][4]) {
                const uint32_t col = tbase + h * 128 + (t & 1) * 64 + 16 * q;
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
                    tmem_ld16x256b_x2(col + ((uint32_t)(32 * rb + 16 * mt) << 16), &dst[mt][0][0]);
                tmem_wait_ld();
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const float2 n0 = make_float2(nr[mt][0], nr[mt][1]), n1 = make_float2(nr[mt][2], nr[mt][3]);
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        const float2 a = __fadd2_rn(make_float2(dst[mt][nt][0], dst[mt][nt][1]), n0);
                        const float2 c = __fadd2_rn(make_float2(dst[mt][nt][2], dst[mt][nt][3]), n1);
                        dst[mt][nt][0] = a.x;
                        dst[mt][nt][1] = a.y;
                        dst[mt][nt][2] = c.x;
                        dst[mt][nt][3] = c.y;
                    }
                }
            };
            // HY: S of tile t in tensor memory (before its first load) / read (after its last)
            auto s_wait = [&](uint32_t t) {
                return !HY || warp_wait(&s_full[2 * h + (t & 1)], (t >> 1) & 1, ab, p.status, p.wait_ns);
            };
            auto s_release = [&](uint32_t t) {
                if constexpr (HY) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&s_free[2 * h + (t & 1)]);
                }
            };
            // S - ref for keys 16q .. 16q+15 of the K tile at kbase (two 8-key column
            // tiles); the swizzle of rows 16q + k_row does not depend on q
            auto qkb = [&](uint32_t kbase, uint32_t t, int q, float (&dst)[2][2][4]) {
                if constexpr (HY) {
                    s_tmem(t, q, dst);
                } else {
                    uint32_t kf[4];
                    ldsm_x4(kbase + koff + 2048u * q, kf[0], kf[1], kf[2], kf[3]);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 2; ++nt)
                            mma16816_c<F16>(dst[mt][nt], qa[mt], kf[2 * nt], kf[2 * nt + 1], nr[mt]);
                }
            };
            // the four 16-key steps of a full tile on the bound path (no maxima, no vote)
            auto fast_tile = [&](uint32_t kbase, uint32_t vbase, uint32_t t) {
                // kTileSum: P summed over the tile's four steps (packed FP16 adds;
                // the bound keeps each P <= 2^13.5, the sum of four inside the FP16
                // range), then one row-sum MMA per tile instead of one per step
                // (1 % faster with FP16 operands; slower with BF16)
                uint32_t ps[2][4];
                // FP16 operands: S - ref accumulated in FP16 (the references are kept
                // FP16-representable, so every path uses the same values), whose f16x2
                // pairs are the exponent arguments as they stand
                uint32_t nr16[2][2];
                if constexpr (F16 && !HY) {
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        nr16[mt][0] = pack_f16x2(nr[mt][0], nr[mt][1]);
                        nr16[mt][1] = pack_f16x2(nr[mt][2], nr[mt][3]);
                    }
                }
                (void)nr16;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t vf[4], pa[2][4];
                    ldsm_x4(vbase + (uint32_t)voff[q], vf[0], vf[1], vf[2], vf[3]);
                    if constexpr (F16 && !HY) {
                        uint32_t kf[4];
                        ldsm_x4(kbase + koff + 2048u * q, kf[0], kf[1], kf[2], kf[3]);
#pragma unroll
                        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                            for (int nt = 0; nt < 2; ++nt) {
                                uint32_t h[2];
                                mma16816_h(h, qa[mt], kf[2 * nt], kf[2 * nt + 1], nr16[mt]);
                                pa[mt][2 * nt] = ex2_h2(h[0]);
                                pa[mt][2 * nt + 1] = ex2_h2(h[1]);
                            }
                    } else {
                        float sc[2][2][4];
                        qkb(kbase, t, q, sc);
#pragma unroll
                        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                            for (int hr = 0; hr < 2; ++hr) {
                                pa[mt][hr] = exp2_pair<F16>(sc[mt][0][2 * hr], sc[mt][0][2 * hr + 1]);
                                pa[mt][2 + hr] = exp2_pair<F16>(sc[mt][1][2 * hr], sc[mt][1][2 * hr + 1]);
                            }
                    }
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma16816<F16>(o[mt][0], pa[mt], vf[0], vf[1]);
                        mma16816<F16>(o[mt][1], pa[mt], vf[2], vf[3]);
                        if constexpr (kTileSum) {
#pragma unroll
                            for (int e = 0; e < 4; ++e) ps[mt][e] = q == 0 ? pa[mt][e] : add2<F16>(ps[mt][e], pa[mt][e]);
                        } else {
                            mma16816<F16>(la[mt], pa[mt], ONE2, ONE2);   // row sums
                        }
                    }
                }
                if constexpr (kTileSum) {
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) mma16816<F16>(la[mt], ps[mt], ONE2, ONE2);   // row sums
                }
            };
            for (int j = 0; j < nk; ++j, ++g) {
                // two full tiles on the bound path with one check and one branch
                // (halves the per-tile wait, check and release work); if the bound
                // fails, tile j falls through to the single-tile code below
                if (j > 0 && j + 1 < nk && ke - kb - 64 * (j + 1) >= 64) {
                    const uint32_t s0 = g % ST, s1 = (g + 1) % ST;
                    if (!warp_wait(&kv_full[s0], (g / ST) & 1, ab, p.status, p.wait_ns)) { ok = false; break; }
                    if (!warp_wait(&kv_full[s1], ((g + 1) / ST) & 1, ab, p.status, p.wait_ns)) { ok = false; break; }
                    const float km = fmaxf(kn[s0 * 4 + h], kn[s1 * 4 + h]);
                    bool over = false;
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int hr = 0; hr < 2; ++hr) over |= fmaf(qn[mt][hr], km, nr[mt][2 * hr]) > kLimit<F16>;
                    if (!__any_sync(0xffffffffu, over)) {
                        if (!s_wait(g)) { ok = false; break; }
                        tc_fence_after();
                        fast_tile(sKa + s0 * AT_KB, sVa + s0 * AT_VB, g);
                        s_release(g);
                        if (!s_wait(g + 1)) { ok = false; break; }
                        tc_fence_after();
                        fast_tile(sKa + s1 * AT_KB, sVa + s1 * AT_VB, g + 1);
                        s_release(g + 1);
                        __syncwarp();
                        if (lane == 0) {
                            mbar_arrive(&kv_empty[s0]);
                            mbar_arrive(&kv_empty[s1]);
                        }
                        ++j;
                        ++g;
                        continue;
                    }
                }
                const uint32_t s = g % ST;
                if (!warp_wait(&kv_full[s], (g / ST) & 1, ab, p.status, p.wait_ns)) { ok = false; break; }
                if (!s_wait(g)) { ok = false; break; }
                tc_fence_after();
                const int kvalid = ke - kb - 64 * j;
                const uint32_t kb = sKa + s * AT_KB, vb = sVa + s * AT_VB;
                // S - ref = Q K^T - ref for keys 16q .. 16q+15 (two 8-key column tiles);
                // the swizzle of rows 16q + k_row does not depend on q (16q is a
                // multiple of 8)
                auto qk = [&](int q, float (&dst)[2][2][4]) { qkb(kb, g, q, dst); };
                // Bound on the tile's scores, row by row: |q| max |k| <= ref + kLimit
                // for every row of the warp means P <= 2^kLimit without looking at
                // the maxima: the four 16-key steps then run without a vote or branch.
                // The first tile (it sets the references) and a ragged last tile take
                // the checked path.
                bool fast = false;
                if (j > 0 && kvalid >= 64) {
                    const float km = kn[s * 4 + h];
                    bool over = false;
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int hr = 0; hr < 2; ++hr) over |= fmaf(qn[mt][hr], km, nr[mt][2 * hr]) > kLimit<F16>;
                    fast = !__any_sync(0xffffffffu, over);
                }
                if (fast) {
                    fast_tile(kb, vb, g);
                } else {
                    // SB 16-key steps per maxima check: S of all of them first, one vote,
                    // then exponentials and PV (no branch between the steps of a block)
#pragma unroll
                    for (int q0 = 0; q0 < 4; q0 += SB) {
                        if (16 * q0 >= kvalid) break;   // warp-uniform
                        float sc[SB][2][2][4];
                        uint32_t vf[SB][4];
        #pragma unroll
                        for (int b = 0; b < SB; ++b) {
                            // V fragments (channels 0-7 / 8-15 of the head, keys 16q .. 16q+15)
                            // first: off the softmax's critical path
                            ldsm_x4(vb + (uint32_t)voff[q0 + b], vf[b][0], vf[b][1], vf[b][2], vf[b][3]);
                            qk(q0 + b, sc[b]);
                        }
                        if (16 * (q0 + SB) > kvalid) {   // ragged end of the event
#pragma unroll
                            for (int b = 0; b < SB; ++b)
#pragma unroll
                                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                                    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                                        for (int e = 0; e < 4; ++e)
                                            if (16 * (q0 + b) + 8 * nt + 2 * tq + (e & 1) >= kvalid)
                                                sc[b][mt][nt][e] = -INFINITY;
                        }
                        // P = 2^(S - ref) as the A fragments of PV (16 keys = one K-step).
                        uint32_t pa[SB][2][4];
                        auto exps = [&]() {
#pragma unroll
                            for (int b = 0; b < SB; ++b)
#pragma unroll
                                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                                    for (int hr = 0; hr < 2; ++hr) {
                                        pa[b][mt][hr] = exp2_pair<F16>(sc[b][mt][0][2 * hr], sc[b][mt][0][2 * hr + 1]);
                                        pa[b][mt][2 + hr] = exp2_pair<F16>(sc[b][mt][1][2 * hr], sc[b][mt][1][2 * hr + 1]);
                                    }
                        };
                        const bool first = j == 0 && q0 == 0;
                        float lm[2][2];
                        bool raise = first;
#pragma unroll
                        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                            for (int hr = 0; hr < 2; ++hr) {
                                float m = -INFINITY;
#pragma unroll
                                for (int b = 0; b < SB; ++b)
                                    m = fmaxf(m, max3f(fmaxf(sc[b][mt][0][2 * hr], sc[b][mt][0][2 * hr + 1]),
                                                       sc[b][mt][1][2 * hr], sc[b][mt][1][2 * hr + 1]));
                                lm[mt][hr] = m;
                                raise |= m > kStaleMax;
                            }
                        const bool raised = __any_sync(0xffffffffu, raise);
                        if (raised) {
                            // raise each row's reference by dr = (row max over the quad) - ref
                            // (never lowered after the first step), rescale O and l by 2^-dr
                            // and shift this block's exponents by -dr
#pragma unroll
                            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                                for (int hr = 0; hr < 2; ++hr) {
                                    float mx = lm[mt][hr];
                                    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
                                    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
                                    float dr = first ? mx : fmaxf(mx, 0.f);
                                    if constexpr (F16 && !HY) {
                                        // the new reference rounded to FP16 (the bound path's
                                        // FP16 accumulator input) and used as such everywhere
                                        const float nn = __half2float(__float2half_rn(nr[mt][2 * hr] - dr));
                                        dr = nr[mt][2 * hr] - nn;
                                        nr[mt][2 * hr] = nn;
                                        nr[mt][2 * hr + 1] = nn;
                                    } else {
                                        nr[mt][2 * hr] -= dr;
                                        nr[mt][2 * hr + 1] -= dr;
                                    }
                                    const float a = first ? 0.f : ex2_approx(-dr);
#pragma unroll
                                    for (int e = 0; e < 2; ++e) {
                                        o[mt][0][2 * hr + e] *= a;
                                        o[mt][1][2 * hr + e] *= a;
                                        la[mt][2 * hr + e] *= a;
#pragma unroll
                                        for (int b = 0; b < SB; ++b) {
                                            sc[b][mt][0][2 * hr + e] -= dr;
                                            sc[b][mt][1][2 * hr + e] -= dr;
                                        }
                                    }
                                }
                        }
                        exps();
#pragma unroll
                        for (int b = 0; b < SB; ++b)
#pragma unroll
                            for (int mt = 0; mt < 2; ++mt) {
                                mma16816<F16>(o[mt][0], pa[b][mt], vf[b][0], vf[b][1]);
                                mma16816<F16>(o[mt][1], pa[b][mt], vf[b][2], vf[b][3]);
                                mma16816<F16>(la[mt], pa[b][mt], ONE2, ONE2);   // row sums
                            }
                    }
                }
                s_release(g);
                __syncwarp();
                if (lane == 0) mbar_arrive(&kv_empty[s]);
            }
            if (!ok) break;
            const int qrow0 = it.x + it.y * ROWS + QR * it.w;   // it.w: half of the item (QR = 64)
            const int nrows = min(QR, it.z - it.y * ROWS - QR * it.w);
            // the event's padding rows (up to its next 64-row boundary) get O = 0, so
            // that every value the next kernels read is written by this forward
            const int npad = min(QR, ((it.z + 63) & ~63) - it.y * ROWS - QR * it.w);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int hr = 0; hr < 2; ++hr) {
                    const float l = la[mt][2 * hr];
                    const int r = rb * 32 + mt * 16 + gq + 8 * hr;
                    if (r < npad) {
                        const bool val = r < nrows;
                        const float inv = 1.0f / l;
                        uint32_t* dst = (uint32_t*)(p.out + (size_t)(qrow0 + r) * D + h * 16 + 2 * tq);
                        dst[0] = val ? pack_f16x2(o[mt][0][2 * hr] * inv, o[mt][0][2 * hr + 1] * inv) : 0u;
                        dst[4] = val ? pack_f16x2(o[mt][1][2 * hr] * inv, o[mt][1][2 * hr + 1] * inv) : 0u;
                    }
                }
            ++q_it;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (HY && warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, 512);
    }
}

// ------------------------------------ attention, warp-level QK^T, PV on tcgen05
// The warp-level kernel with the PV product and the row sums moved to the tensor
// cores.  Each consumer warp still owns 32 query rows of one head and computes
// S - ref with m16n8k16 MMAs (Q pre-scaled, the negated references as the
// accumulator input) and the packed exponentials, but writes P (16-bit pairs) into
// tensor memory with tcgen05.st.16x128b, whose thread layout is the MMA's A-fragment
// layout.  One MMA warp then accumulates O_h += P_h V_h and l_h += P_h 1 per head and
// 64-key tile (tcgen05, P as the tensor-memory A operand, M 128, N 16, K 64), so the
// legacy tensor pipe carries only the four QK^T MMAs of the ten per warp and 16-key
// step.  One MMA warp per head, so that a head's MMAs never wait for another head's
// warps.  P has three buffers per head (the warps write tile t while the MMAs of
// tiles t - 1 and t - 2 may still run); O and l stay in tensor memory for the whole
// item and are read once, at its end.  Tensor memory: P 4 heads x 3 buffers x 32
// columns, [O_h | l_h] 4 x 32 columns: all 512.
// Rescaling: one exponent reference per row for the whole tile, since the tile's P
// is summed by one MMA.  The bound path (|q| max |k| <= ref + kLimit for every row
// of the warp) runs the four steps straight through as in the warp-level kernel.
// Otherwise (the first tile of an item, a ragged last tile, a failed bound) the
// tile's row maxima are computed first (QK^T of every step, recomputed for the
// exponentials); the first tile sets the references, a later one raises a row's
// reference only when the row maximum exceeds it by more than kStaleMax, and then
// rescales the row's O and l in tensor memory once the previous tile's MMA is
// complete.  Steps wholly past the end of the event store P = 0.
constexpr int PT_NB = 3;                              // P buffers per head
constexpr int PT_ATT_THREADS = NH * 4 * 32 + 32 + NH * 32;   // 16 consumer warps, TMA warp, 4 MMA warps
template <int ST>
struct PtLayout {
    static constexpr uint32_t OFF_K = 2 * AT_QB;
    static constexpr uint32_t OFF_V = OFF_K + ST * AT_KB;
    static constexpr uint32_t OFF_ONES = OFF_V + ST * AT_VB;   // 16 rows of ones (row-sum B operand)
    static constexpr uint32_t OFF_BAR = OFF_ONES + 2048;      // barriers, item info, flags (< 512 B)
    static constexpr uint32_t OFF_KN = OFF_BAR + 512;         // [ST][4] key-tile norm bounds
    static constexpr uint32_t SMEM = OFF_KN + 8 * 16 + 1024;
};
// the item info (two int4) after the barriers, at a 16-byte aligned offset
constexpr uint32_t PT_INFO_OFF = 448;
static_assert((2 + 2 + 8 + 8 + 1 + 2 * NH * PT_NB + NH) * 8 <= PT_INFO_OFF, "PV-on-tcgen05 attention barriers");
static_assert(PT_INFO_OFF % 16 == 0 && PT_INFO_OFF + 2 * 16 + 8 <= 512, "PV-on-tcgen05 attention info area");

template <bool F16, int ST>
__global__ void __launch_bounds__(PT_ATT_THREADS, 1)
    k_attention_pt(const __grid_constant__ CUtensorMap map_q, const __grid_constant__ CUtensorMap map_k,
                   const __grid_constant__ CUtensorMap map_vt, AttnParams p) {
    constexpr int RB = 4;          // 32-row blocks (one per warp) per 128-row item
    constexpr int NW = NH * RB;    // consumer warps
    using LY = PtLayout<ST>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint8_t* sQ = sm;
    uint8_t* sK = sm + LY::OFF_K;
    uint8_t* sV = sm + LY::OFF_V;
    uint8_t* sOnes = sm + LY::OFF_ONES;
    uint64_t* bars = (uint64_t*)(sm + LY::OFF_BAR);
    uint64_t* q_full = bars;            // [2]
    uint64_t* q_empty = bars + 2;       // [2]: one arrival per consumer warp and per MMA warp
    uint64_t* kv_full = bars + 4;       // [ST]
    uint64_t* kv_empty = kv_full + ST;  // [ST]: one arrival per consumer warp, one commit per MMA warp
    uint64_t* never = kv_empty + ST;    // armed by nobody (debug stall)
    uint64_t* p_full = never + 1;             // [head][buffer]: one arrival per warp of the head
    uint64_t* p_free = p_full + NH * PT_NB;   // [head][buffer]: MMA commit, the tile's PV and row sums done
    uint64_t* drain = p_free + NH * PT_NB;    // [head]: the MMA warp's exit
    int4* info = (int4*)(sm + LY::OFF_BAR + PT_INFO_OFF);   // [2], 16-byte aligned
    int* abort_flag = (int*)(info + 2);
    uint32_t* tmem_hold = (uint32_t*)(abort_flag + 1);
    float* kn = (float*)(sm + LY::OFF_KN);
    volatile int* ab = abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) { mbar_init(&q_full[i], 1); mbar_init(&q_empty[i], NW + NH); }
        for (int i = 0; i < ST; ++i) { mbar_init(&kv_full[i], 1); mbar_init(&kv_empty[i], NW + NH); }
        mbar_init(never, 1);
        for (int i = 0; i < NH * PT_NB; ++i) { mbar_init(&p_full[i], RB); mbar_init(&p_free[i], 1); }
        for (int i = 0; i < NH; ++i) mbar_init(&drain[i], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    {   // the B operand of the row sums: 16 rows x 64 keys of ones
        const uint32_t one2 = F16 ? 0x3C003C00u : 0x3F803F80u;
        for (int i = tid; i < 512; i += PT_ATT_THREADS) ((uint32_t*)sOnes)[i] = one2;
        fence_proxy_async_smem();
    }
    if (warp == 0) {
        tmem_alloc(tmem_hold, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_hold;
    const int n_items = p.counters[0];
    int* ticket = p.counters + 2 + p.layer;
    // tensor-memory columns: P of head h, buffer b; O_h (16 columns) and l_h (16)
    auto colP = [](int h, uint32_t b) { return (uint32_t)(h * 32 * PT_NB) + b * 32u; };
    auto colO = [](int h) { return (uint32_t)(NH * 32 * PT_NB) + (uint32_t)(h * 32); };
    // tile t uses P buffer t % PT_NB; the k-th completion of a buffer's barriers is
    // its k-th tile, so the phase parity of tile t is (t / PT_NB) & 1
    auto pbuf = [](uint32_t t) { return t % PT_NB; };
    auto ppar = [](uint32_t t) { return (t / PT_NB) & 1u; };

    if (warp == NW) {
        // ------------------------------------------------ TMA producer (64-key stages)
        if (lane == 0)
            attn_produce<ST, 128>(&map_q, &map_k, &map_vt, p, sQ, sK, sV, kn, q_full, q_empty, kv_full, kv_empty,
                                  info, ab, n_items, ticket);
    } else if (warp > NW) {
        // ------------------------------------------------ PV and row-sum MMAs of head h (one thread)
        const int h = warp - NW - 1;
        if (lane == 0) {
            const uint32_t IPV = idesc_f16(128, 16, F16 ? 0u : 1u);
            const uint32_t onesa = smem_u32(sOnes);
            int q_it = 0;
            uint32_t g = 0;
            bool ok = true;
            while (ok) {
                const int qb = q_it & 1;
                if (!mbar_wait(&q_full[qb], (q_it >> 1) & 1, ab, p.status, ST_TIMEOUT_ATTN, p.wait_ns)) break;
                const int4 it = info[qb];
                mbar_arrive(&q_empty[qb]);   // info read (the MMAs do not read Q)
                if (it.x < 0) break;
                int kb, ke;
                key_range(it.y, it.z, p.window, kb, ke);
                const int nk = (ke - kb + 63) >> 6;
                for (int j = 0; j < nk && ok; ++j) {
                    const uint32_t t = g + j, s = t % ST, b = pbuf(t);
                    if (!mbar_wait(&kv_full[s], (t / ST) & 1, ab, p.status, ST_TIMEOUT_ATTN, p.wait_ns) ||
                        !mbar_wait(&p_full[PT_NB * h + b], ppar(t), ab, p.status, ST_TIMEOUT_ATTN, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t va = smem_u32(sV + s * AT_VB);
                    const uint32_t pa = tbase + colP(h, b), od = tbase + colO(h);
#pragma unroll
                    for (int kc = 0; kc < 4; ++kc) {
                        const uint32_t acc = (j > 0 || kc > 0) ? 1u : 0u;
                        mma_f16_ts(od, pa + 8 * kc, sdesc_sw128(va + h * 2048 + kc * 32), IPV, acc);
                        mma_f16_ts(od + 16, pa + 8 * kc, sdesc_sw128(onesa + kc * 32), IPV, acc);
                    }
                    mma_commit(&p_free[PT_NB * h + b]);
                    mma_commit(&kv_empty[s]);
                }
                if (!ok) break;
                g += nk;
                ++q_it;
            }
            // every MMA issued complete before tensor memory and shared memory are released
            mma_commit(&drain[h]);
            mbar_drain(&drain[h], 0, p.wait_ns);
        }
    } else {
        // ------------------------------------------------ warp: head h, query rows 32 rb .. 32 rb + 31
        const int h = warp / RB, rb = warp % RB;
        const int tq = lane & 3;
        const int mi = lane >> 3;
        const uint32_t sQa = smem_u32(sQ), sKa = smem_u32(sK);
        const int k_row = (lane & 7) + 8 * (mi >> 1), k_chunk = 2 * h + (mi & 1);
        const uint32_t koff = sw128_off(k_row, k_chunk);
        const uint32_t tlane = tbase + ((uint32_t)(32 * rb) << 16);   // this warp's lanes
        int q_it = 0;
        uint32_t g = 0;
        bool ok = true;
        while (ok) {
            const int qb = q_it & 1;
            if (!warp_wait(&q_full[qb], (q_it >> 1) & 1, ab, p.status, p.wait_ns)) break;
            const int4 it = info[qb];
            if (it.x < 0) break;
            if (p.debug_stall && !warp_wait(never, 0, ab, p.status, p.wait_ns)) break;
            int kb, ke;
            key_range(it.y, it.z, p.window, kb, ke);
            const int nk = (ke - kb + 63) >> 6;
            const uint32_t qfa = sQa + qb * AT_QB + sw128_off(rb * 32 + (lane & 15), 2 * h + (lane >> 4));
            uint32_t qa[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) ldsm_x4(qfa + 2048u * mt, qa[mt][0], qa[mt][1], qa[mt][2], qa[mt][3]);
            float qn[2][2];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int hr = 0; hr < 2; ++hr) {
                    float a0, a1, a2, a3;
                    unpack2<F16>(qa[mt][hr], a0, a1);
                    unpack2<F16>(qa[mt][2 + hr], a2, a3);
                    float t = fmaf(a0, a0, fmaf(a1, a1, fmaf(a2, a2, a3 * a3)));
                    t += __shfl_xor_sync(0xffffffffu, t, 1);
                    t += __shfl_xor_sync(0xffffffffu, t, 2);
                    qn[mt][hr] = sqrtf(t) * 1.01f;
                }
            __syncwarp();
            if (lane == 0) mbar_arrive(&q_empty[qb]);
            // nr: the negated exponent references of the fragment's rows, as the QK^T
            // MMA's accumulator input (its output is the exponent S - ref itself)
            float nr[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int e = 0; e < 4; ++e) nr[mt][e] = 0.f;
            // K fragments of step q (keys 16 q .. 16 q + 15) and S - ref from them
            auto kfrag = [&](uint32_t kbase, int q, uint32_t (&kf)[4]) {
                ldsm_x4(kbase + koff + 2048u * q, kf[0], kf[1], kf[2], kf[3]);
            };
            auto qk_f = [&](const uint32_t (&kf)[4], float (&dst)[2][2][4]) {
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) mma16816_c<F16>(dst[mt][nt], qa[mt], kf[2 * nt], kf[2 * nt + 1], nr[mt]);
            };
            auto qk = [&](uint32_t kbase, int q, float (&dst)[2][2][4]) {
                uint32_t kf[4];
                kfrag(kbase, q, kf);
                qk_f(kf, dst);
            };
            // P of step q into the columns pcol + 8 q .. + 7 (buffer of the tile), lanes
            // of the two 16-row blocks
            auto store_p = [&](uint32_t pcol, int q, const float (&sc)[2][2][4]) {
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    uint32_t pa[4];
#pragma unroll
                    for (int hr = 0; hr < 2; ++hr) {
                        pa[hr] = exp2_pair<F16>(sc[mt][0][2 * hr], sc[mt][0][2 * hr + 1]);
                        pa[2 + hr] = exp2_pair<F16>(sc[mt][1][2 * hr], sc[mt][1][2 * hr + 1]);
                    }
                    tmem_st16x128b_x2(pcol + ((uint32_t)(16 * mt) << 16) + 8 * q, pa);
                }
            };
            // the buffer of tile t may be written once the MMAs of tile t - PT_NB are complete
            auto p_acquire = [&](uint32_t t) {
                if (t < PT_NB) return true;
                const bool r = warp_wait(&p_free[PT_NB * h + pbuf(t)], ppar(t - PT_NB), ab, p.status, p.wait_ns);
                tc_fence_after();
                return r;
            };
            auto p_publish = [&](uint32_t t) {
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&p_full[PT_NB * h + pbuf(t)]);
            };
            // the four steps of a full tile on the bound path: the K fragments of every
            // step first (the loads stay ahead of the tensor-memory stores)
            auto fast_tile = [&](uint32_t kbase, uint32_t t) {
                uint32_t kf[4][4];
#pragma unroll
                for (int q = 0; q < 4; ++q) kfrag(kbase, q, kf[q]);
                const uint32_t pcol = tlane + colP(h, pbuf(t));
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float sc[2][2][4];
                    qk_f(kf[q], sc);
                    store_p(pcol, q, sc);
                }
            };
            for (int j = 0; j < nk; ++j, ++g) {
                // two full tiles on the bound path with one check and one branch
                if (j > 0 && j + 1 < nk && ke - kb - 64 * (j + 1) >= 64) {
                    const uint32_t s0 = g % ST, s1 = (g + 1) % ST;
                    if (!warp_wait(&kv_full[s0], (g / ST) & 1, ab, p.status, p.wait_ns)) { ok = false; break; }
                    if (!warp_wait(&kv_full[s1], ((g + 1) / ST) & 1, ab, p.status, p.wait_ns)) { ok = false; break; }
                    const float km = fmaxf(kn[s0 * 4 + h], kn[s1 * 4 + h]);
                    bool over = false;
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int hr = 0; hr < 2; ++hr) over |= fmaf(qn[mt][hr], km, nr[mt][2 * hr]) > kLimit<F16>;
                    if (!__any_sync(0xffffffffu, over)) {
                        if (!p_acquire(g)) { ok = false; break; }
                        fast_tile(sKa + s0 * AT_KB, g);
                        p_publish(g);
                        if (!p_acquire(g + 1)) { ok = false; break; }
                        fast_tile(sKa + s1 * AT_KB, g + 1);
                        p_publish(g + 1);
                        __syncwarp();
                        if (lane == 0) {
                            mbar_arrive(&kv_empty[s0]);
                            mbar_arrive(&kv_empty[s1]);
                        }
                        ++j;
                        ++g;
                        continue;
                    }
                }
                const uint32_t s = g % ST;
                if (!warp_wait(&kv_full[s], (g / ST) & 1, ab, p.status, p.wait_ns)) { ok = false; break; }
                const int kvalid = ke - kb - 64 * j;
                const uint32_t kbs = sKa + s * AT_KB;
                bool fast = false;
                if (j > 0 && kvalid >= 64) {
                    const float km = kn[s * 4 + h];
                    bool over = false;
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int hr = 0; hr < 2; ++hr) over |= fmaf(qn[mt][hr], km, nr[mt][2 * hr]) > kLimit<F16>;
                    fast = !__any_sync(0xffffffffu, over);
                }
                if (!p_acquire(g)) { ok = false; break; }
                if (fast) {
                    fast_tile(kbs, g);
                } else {
                    // the tile's row maxima (S - ref over its valid keys)
                    auto mask = [&](int q, float (&sc)[2][2][4]) {
                        if (16 * (q + 1) > kvalid) {
#pragma unroll
                            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                                    for (int e = 0; e < 4; ++e)
                                        if (16 * q + 8 * nt + 2 * tq + (e & 1) >= kvalid) sc[mt][nt][e] = -INFINITY;
                        }
                    };
                    float lm[2][2];
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) lm[mt][0] = lm[mt][1] = -INFINITY;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (16 * q >= kvalid) break;   // warp-uniform
                        float sc[2][2][4];
                        qk(kbs, q, sc);
                        mask(q, sc);
#pragma unroll
                        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                            for (int hr = 0; hr < 2; ++hr)
                                lm[mt][hr] = fmaxf(lm[mt][hr], max3f(fmaxf(sc[mt][0][2 * hr], sc[mt][0][2 * hr + 1]),
                                                                     sc[mt][1][2 * hr], sc[mt][1][2 * hr + 1]));
                    }
                    const bool first = j == 0;
                    bool raise = first;
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int hr = 0; hr < 2; ++hr) {
                            float mx = lm[mt][hr];
                            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
                            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
                            lm[mt][hr] = mx;
                            raise |= mx > kStaleMax;
                        }
                    if (__any_sync(0xffffffffu, raise)) {
                        // raise each row's reference by dr (the first tile: to its maximum;
                        // later: only upwards); a later tile rescales the row's O and l
                        float a[2][2];
#pragma unroll
                        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                            for (int hr = 0; hr < 2; ++hr) {
                                const float dr = first ? lm[mt][hr] : fmaxf(lm[mt][hr], 0.f);
                                a[mt][hr] = first ? 1.f : ex2_approx(-dr);
                                nr[mt][2 * hr] -= dr;
                                nr[mt][2 * hr + 1] -= dr;
                            }
                        if (!first) {
                            // O and l of tile t - 1 complete, then row (lane) of this warp scaled
                            if (!warp_wait(&p_free[PT_NB * h + pbuf(g - 1)], ppar(g - 1), ab, p.status, p.wait_ns)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            // the factor of row `lane` (16-row block lane / 16, half (lane / 8) & 1,
                            // fragment row lane & 7) is held by fragment lane 4 (lane & 7)
                            const int src = 4 * (lane & 7);
                            const float f00 = __shfl_sync(0xffffffffu, a[0][0], src);
                            const float f01 = __shfl_sync(0xffffffffu, a[0][1], src);
                            const float f10 = __shfl_sync(0xffffffffu, a[1][0], src);
                            const float f11 = __shfl_sync(0xffffffffu, a[1][1], src);
                            const float f = lane < 16 ? (lane < 8 ? f00 : f01) : (lane < 24 ? f10 : f11);
                            float ol[32];
                            tmem_ld32(tlane + colO(h), ol);
                            tmem_wait_ld();
                            uint32_t u[32];
#pragma unroll
                            for (int i = 0; i < 32; ++i) u[i] = __float_as_uint(ol[i] * f);
                            tmem_st32(tlane + colO(h), u);
                        }
                    }
                    // the exponentials with the tile's references; steps past the end of
                    // the event store P = 0
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float sc[2][2][4];
                        if (16 * q < kvalid) {
                            qk(kbs, q, sc);
                            mask(q, sc);
                        } else {
#pragma unroll
                            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                                    for (int e = 0; e < 4; ++e) sc[mt][nt][e] = -INFINITY;
                        }
                        store_p(tlane + colP(h, pbuf(g)), q, sc);
                    }
                }
                p_publish(g);
                __syncwarp();
                if (lane == 0) mbar_arrive(&kv_empty[s]);
            }
            if (!ok) break;
            // the item's output: O / l of row (lane) of this warp, head h
            const uint32_t tlast = g - 1;
            if (!warp_wait(&p_free[PT_NB * h + pbuf(tlast)], ppar(tlast), ab, p.status, p.wait_ns)) break;
            tc_fence_after();
            float ol[32];
            tmem_ld32(tlane + colO(h), ol);
            tmem_wait_ld();
            const int r = rb * 32 + lane;
            const int qrow0 = it.x + it.y * ROWS;
            // the event's padding rows (up to its next 64-row boundary) get O = 0, so
            // that every value the next kernels read is written by this forward
            if (r < min(ROWS, ((it.z + 63) & ~63) - it.y * ROWS)) {
                const float inv = 1.0f / ol[16];
                uint4 u0, u1;
                u0.x = pack_f16x2(ol[0] * inv, ol[1] * inv);
                u0.y = pack_f16x2(ol[2] * inv, ol[3] * inv);
                u0.z = pack_f16x2(ol[4] * inv, ol[5] * inv);
                u0.w = pack_f16x2(ol[6] * inv, ol[7] * inv);
                u1.x = pack_f16x2(ol[8] * inv, ol[9] * inv);
                u1.y = pack_f16x2(ol[10] * inv, ol[11] * inv);
                u1.z = pack_f16x2(ol[12] * inv, ol[13] * inv);
                u1.w = pack_f16x2(ol[14] * inv, ol[15] * inv);
                uint4* dst = (uint4*)(p.out + (size_t)(qrow0 + r) * D + h * 16);
                const bool val = r < it.z - it.y * ROWS;
                dst[0] = val ? u0 : make_uint4(0, 0, 0, 0);
                dst[1] = val ? u1 : make_uint4(0, 0, 0, 0);
            }
            ++q_it;
        }
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, 512);
    }
}

// ------------------------------------------------ attention, S and P in tensor memory
// Persistent, one CTA per SM: four softmax warpgroups (warpgroup h = head h; thread r
// owns query row r of the 128-row item), a TMA producer warp and an MMA warp.  Per
// head and 64-key tile the MMA warp computes S = Q_h K_h^T (tcgen05, Q and K from
// shared memory) into the head's S columns of tensor memory; the softmax threads
// load their row of S, write P = 2^(S - ref) in the 16-bit operand format into the
// head's P columns, and the MMA warp accumulates [O_h | l_h] += P [V_h | 1] with P
// as the tensor-memory A operand (M 128, N 32, K 64): P never passes through shared
// memory, and O and the row sums l stay in tensor memory for the whole item (read
// once, at its end).  Tensor memory per head: S 64 columns, P 32 (two 16-bit values
// per column), O 16, l 16 (every column the row sum); four heads, 512 columns.
// Each V^T stage holds, per head, the head's 16 V^T rows followed by 16 rows of ones,
// so one MMA gives the PV product and the row sums of the same rounded P.
// Rescaling is lazy as in the warp-level kernel: the first tile sets each row's
// exponent reference to the tile maximum; a later tile whose score bound |q| max|k|
// exceeds the reference by more than kLimit has its maxima computed, and a row whose
// maximum exceeds the reference by more than kStaleMax raises it and rescales its O
// and l in tensor memory.  BF16 exponentials are packed (ex2.bf16x2: two per MUFU
// operation), FP16 likewise (ex2.f16x2).  Every wait is bounded.
constexpr int TM_THREADS = NH * 128 + 64;        // 16 softmax warps, producer, MMA warp
constexpr uint32_t TM_VB = NH * 32 * 128;        // per stage: per head 16 V^T rows + 16 rows of ones
template <int ST>
struct TmLayout {
    static constexpr uint32_t OFF_K = 2 * AT_QB;
    static constexpr uint32_t OFF_V = OFF_K + ST * AT_KB;
    static constexpr uint32_t OFF_BAR = OFF_V + ST * TM_VB;   // barriers, item info, flags (< 512 B)
    static constexpr uint32_t OFF_KN = OFF_BAR + 512;         // [ST][4] key-tile norm bounds
    static constexpr uint32_t SMEM = OFF_KN + ST * 16 + 16 + 1024;
};

template <bool F16, int ST>
__global__ void __launch_bounds__(TM_THREADS, 1)
    k_attention_tm(const __grid_constant__ CUtensorMap map_q, const __grid_constant__ CUtensorMap map_k,
                   const __grid_constant__ CUtensorMap map_vt16, AttnParams p) {
    using LY = TmLayout<ST>;
    constexpr int NSW = NH * 4;                   // softmax warps
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint8_t* sQ = sm;
    uint8_t* sK = sm + LY::OFF_K;
    uint8_t* sV = sm + LY::OFF_V;
    uint64_t* bars = (uint64_t*)(sm + LY::OFF_BAR);
    uint64_t* q_full = bars;              // [2]  producer (tx)
    uint64_t* q_empty = bars + 2;         // [2]  MMA commit after the item's last QK^T
    uint64_t* kv_full = bars + 4;         // [ST] producer (tx)
    uint64_t* kv_empty = kv_full + ST;    // [ST] MMA commit after the tile's last MMA
    uint64_t* s_full = kv_empty + ST;     // [NH] MMA commit: S of the head's tile ready
    uint64_t* p_ready = s_full + NH;      // [NH] one arrival per softmax warp: P stored, S read
    uint64_t* pv_done = p_ready + NH;     // [NH] MMA commit: the head's [O | l] += P [V | 1] done
    uint64_t* o_free = pv_done + NH;      // [NH] one arrival per softmax warp: O, l read at item end
    uint64_t* drain = o_free + NH;        // MMA warp's exit: every issued MMA complete
    uint64_t* never = drain + 1;          // armed by nobody (debug stall)
    int4* info = (int4*)(never + 1);      // [2]
    uint32_t* tmem_hold = (uint32_t*)(info + 2);
    int* abort_flag = (int*)(tmem_hold + 1);
    float* kn = (float*)(sm + LY::OFF_KN);
    volatile int* ab = abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) { mbar_init(&q_full[i], 1); mbar_init(&q_empty[i], 1); }
        for (int i = 0; i < ST; ++i) { mbar_init(&kv_full[i], 1); mbar_init(&kv_empty[i], 1); }
        for (int h = 0; h < NH; ++h) {
            mbar_init(&s_full[h], 1);
            mbar_init(&p_ready[h], 4);
            mbar_init(&pv_done[h], 1);
            mbar_init(&o_free[h], 4);
        }
        mbar_init(drain, 1);
        mbar_init(never, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    {   // the rows of ones under each head's V^T rows, in every stage (B operand of the row sums)
        const uint32_t one2 = F16 ? 0x3C003C00u : 0x3F803F80u;
        for (int i = tid; i < ST * NH * 16 * 32; i += TM_THREADS) {
            const int s = i / (NH * 512), rem = i % (NH * 512), h = rem / 512, w = rem % 512;
            ((uint32_t*)(sV + s * TM_VB + h * 4096 + 2048))[w] = one2;
        }
        fence_proxy_async_smem();
    }
    if (warp == 0) {
        tmem_alloc(tmem_hold, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_hold;
    const int n_items = p.counters[0];
    int* ticket = p.counters + 2 + p.layer;

    if (warp == NSW) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            tma_prefetch_map(&map_q);
            tma_prefetch_map(&map_k);
            tma_prefetch_map(&map_vt16);
            int q_it = 0, q_armed = 0;
            uint32_t g = 0;
            bool ok = true;
            while (ok) {
                const int item = atomicAdd(ticket, 1);
                int4 it = make_int4(-1, 0, 0, 0);
                if (item < n_items) {
                    it = p.items[item];
                    if (it.z - it.y * ROWS <= 0) continue;   // an event the scheduler could not place
                }
                const int qb = q_it & 1;
                if (q_it >= 2 &&
                    !mbar_wait(&q_empty[qb], ((q_it >> 1) - 1) & 1, ab, p.status, ST_TIMEOUT_ATTN, p.wait_ns))
                    break;
                info[qb] = it;
                if (item >= n_items) {
                    mbar_arrive(&q_full[qb]);
                    break;
                }
                mbar_arrive_expect_tx(&q_full[qb], AT_QB);
                tma_load_2d(sQ + qb * AT_QB, &map_q, 0, it.x + it.y * ROWS, &q_full[qb]);
                ++q_armed;
                int kb, ke;
                key_range(it.y, it.z, p.window, kb, ke);
                const int nk = (ke - kb + 63) >> 6;
                for (int j = 0; j < nk; ++j, ++g) {
                    const int s = (int)(g % ST);
                    if (g >= ST &&
                        !mbar_wait(&kv_empty[s], ((g / ST) - 1) & 1, ab, p.status, ST_TIMEOUT_ATTN, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    const int key0 = it.x + kb + 64 * j;
                    mbar_arrive_expect_tx(&kv_full[s], AT_KB + NH * 2048 + 16);
                    tma_load_2d(sK + s * AT_KB, &map_k, 0, key0, &kv_full[s]);
#pragma unroll
                    for (int h = 0; h < NH; ++h)
                        tma_load_2d(sV + s * TM_VB + h * 4096, &map_vt16, key0, 16 * h, &kv_full[s]);
                    bulk_load(kn + 4 * s, p.kmax + (size_t)((key0 >> 6)) * 4, 16, &kv_full[s]);
                }
                ++q_it;
            }
            // on an abort, let the copies still in flight land before the CTA exits
            if (*ab) {
                for (uint32_t t = g > ST ? g - ST : 0; t < g; ++t)
                    mbar_drain(&kv_full[t % ST], (t / ST) & 1, p.wait_ns);
                for (int i = q_armed > 2 ? q_armed - 2 : 0; i < q_armed; ++i)
                    mbar_drain(&q_full[i & 1], (i >> 1) & 1, p.wait_ns);
            }
        }
    } else if (warp == NSW + 1) {
        // ------------------------------------------------ MMA issue (one thread)
        if (lane == 0) {
            const uint32_t fmt = F16 ? 0u : 1u;
            const uint32_t IQK = idesc_f16(128, 64, fmt), IPV = idesc_f16(128, 32, fmt);
            int q_it = 0;
            uint32_t g = 0;
            bool ok = true;
            auto W = [&](uint64_t* bar, uint32_t parity) {
                return mbar_wait(bar, parity, ab, p.status, ST_TIMEOUT_ATTN, p.wait_ns);
            };
            while (ok) {
                const int qb = q_it & 1;
                if (!W(&q_full[qb], (q_it >> 1) & 1)) break;
                const int4 it = info[qb];
                if (it.x < 0) break;
                int kb, ke;
                key_range(it.y, it.z, p.window, kb, ke);
                const int nk = (ke - kb + 63) >> 6;
                const uint32_t qa = smem_u32(sQ + qb * AT_QB);
                // S of the item's first tile, every head (the previous tile's P of each
                // head was read by its PV, issued after that head's p_ready)
                {
                    const uint32_t s = g % ST;
                    if (!W(&kv_full[s], (g / ST) & 1)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t ka = smem_u32(sK + s * AT_KB);
                    for (int h = 0; h < NH; ++h) {
                        mma_f16(tbase + h * 128, sdesc_sw128(qa + h * 32), sdesc_sw128(ka + h * 32), IQK, 0);
                        mma_commit(&s_full[h]);
                    }
                }
                for (int j = 0; j < nk && ok; ++j) {
                    const uint32_t t = g + j, s = t % ST;
                    const uint32_t va = smem_u32(sV + s * TM_VB);
                    const uint32_t ka1 = smem_u32(sK + ((t + 1) % ST) * AT_KB);
                    for (int h = 0; h < NH; ++h) {
                        if (!W(&p_ready[h], t & 1)) { ok = false; break; }
                        if (j == 0 && q_it > 0 && !W(&o_free[h], (q_it - 1) & 1)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t col = tbase + h * 128;
#pragma unroll
                        for (int kc = 0; kc < 4; ++kc)
                            mma_f16_ts(col + 96, col + 64 + 8 * kc, sdesc_sw128(va + h * 4096 + kc * 32), IPV,
                                       (j > 0 || kc > 0) ? 1u : 0u);
                        mma_commit(&pv_done[h]);
                        if (j + 1 < nk) {
                            if (h == 0 && !W(&kv_full[(t + 1) % ST], ((t + 1) / ST) & 1)) { ok = false; break; }
                            tc_fence_after();
                            mma_f16(col, sdesc_sw128(qa + h * 32), sdesc_sw128(ka1 + h * 32), IQK, 0);
                            mma_commit(&s_full[h]);
                        }
                    }
                    if (!ok) break;
                    mma_commit(&kv_empty[s]);
                }
                if (!ok) break;
                mma_commit(&q_empty[qb]);
                g += nk;
                ++q_it;
            }
            // every MMA issued by this thread complete before tensor memory is released
            mma_commit(drain);
            mbar_drain(drain, 0, p.wait_ns);
        }
    } else {
        // ------------------------------------------------ softmax: warpgroup h = head h
        const int h = warp >> 2;
        const int r = tid & 127;
        const uint32_t tl = tbase + ((uint32_t)((warp & 3) * 32) << 16) + h * 128;   // this warp's lanes
        const uint32_t tS = tl, tP = tl + 64, tO = tl + 96;
        int q_it = 0;
        uint32_t g = 0;
        bool ok = true;
        while (ok) {
            const int qb = q_it & 1;
            if (!warp_wait(&q_full[qb], (q_it >> 1) & 1, ab, p.status, p.wait_ns)) break;
            const int4 it = info[qb];
            if (it.x < 0) break;
            if (p.debug_stall && !warp_wait(never, 0, ab, p.status, p.wait_ns)) break;
            int kb, ke;
            key_range(it.y, it.z, p.window, kb, ke);
            const int nk = (ke - kb + 63) >> 6;
            // |q| of this row's head-h channels (1 % for the FP32 sums), for the key
            // tiles' score bounds |q| max|k|
            float qn;
            {
                const uint8_t* qrow = sQ + qb * AT_QB;
                const uint4 u0 = *(const uint4*)(qrow + sw128_off(r, 2 * h));
                const uint4 u1 = *(const uint4*)(qrow + sw128_off(r, 2 * h + 1));
                const uint32_t w8[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                float ss = 0.f;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float a, b;
                    unpack2<F16>(w8[i], a, b);
                    ss = fmaf(a, a, fmaf(b, b, ss));
                }
                qn = sqrtf(ss) * 1.01f;
            }
            float ref = 0.f;
            for (int j = 0; j < nk; ++j) {
                const uint32_t t = g + j, s = t % ST;
                if (!warp_wait(&s_full[h], t & 1, ab, p.status, p.wait_ns)) { ok = false; break; }
                if (!warp_wait(&kv_full[s], (t / ST) & 1, ab, p.status, p.wait_ns)) { ok = false; break; }
                tc_fence_after();
                const int kvalid = ke - kb - 64 * j;
                const bool full = kvalid >= 64;
                // the maxima are needed on the first tile (it sets the reference), on a
                // ragged tile and where the score bound does not hold
                const bool need = j == 0 || !full || fmaf(qn, kn[s * 4 + h], -ref) > kLimit<F16>;
                float sv[32];
                float m = -INFINITY;
                if (__any_sync(0xffffffffu, need)) {
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {
                        tmem_ld32(tS + 32 * hf, sv);
                        tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (!full && 32 * hf + i >= kvalid) sv[i] = -INFINITY;
#pragma unroll
                        for (int i = 0; i < 32; i += 2) m = max3f(m, sv[i], sv[i + 1]);
                    }
                }
                float nref = ref;
                bool redo = false;
                if (j == 0) {
                    nref = m;
                } else if (need && m - ref > kStaleMax) {
                    nref = m;
                    redo = true;
                }
                if (j > 0) {
                    // P(t-1) read and O, l final up to tile t-1 before P(t) is written
                    if (!warp_wait(&pv_done[h], (t - 1) & 1, ab, p.status, p.wait_ns)) { ok = false; break; }
                    tc_fence_after();
                    if (__any_sync(0xffffffffu, redo)) {
                        float ol[32];
                        tmem_ld32(tO, ol);
                        tmem_wait_ld();
                        const float a = redo ? ex2_approx(ref - nref) : 1.f;
                        uint32_t u[32];
#pragma unroll
                        for (int i = 0; i < 32; ++i) u[i] = __float_as_uint(ol[i] * a);
                        tmem_st32(tO, u);
                    }
                }
                ref = nref;
                // P = 2^(S - ref) into the head's P columns
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    tmem_ld32(tS + 32 * hf, sv);
                    tmem_wait_ld();
                    if (!full) {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (32 * hf + i >= kvalid) sv[i] = -INFINITY;
                    }
                    uint32_t pk[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        float x0, x1;
                        ffma2_bcast(x0, x1, sv[2 * i], sv[2 * i + 1], 1.f, -ref);
                        pk[i] = exp2_pair<F16>(x0, x1);
                    }
                    tmem_st16(tP + 16 * hf, pk);
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&p_ready[h]);
            }
            if (!ok) break;
            // the item's output: O / l of this row and head
            const uint32_t tlast = g + nk - 1;
            if (!warp_wait(&pv_done[h], tlast & 1, ab, p.status, p.wait_ns)) break;
            tc_fence_after();
            float ol[32];
            tmem_ld32(tO, ol);
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&o_free[h]);
            const int qrow0 = it.x + it.y * ROWS;
            // valid rows get O / l, the event's padding rows (up to its next 64-row
            // boundary) O = 0, so that every value the next kernels read is written here
            if (r < min(ROWS, ((it.z + 63) & ~63) - it.y * ROWS)) {
                const float inv = 1.0f / ol[16];
                uint4 u0, u1;
                u0.x = pack_f16x2(ol[0] * inv, ol[1] * inv);
                u0.y = pack_f16x2(ol[2] * inv, ol[3] * inv);
                u0.z = pack_f16x2(ol[4] * inv, ol[5] * inv);
                u0.w = pack_f16x2(ol[6] * inv, ol[7] * inv);
                u1.x = pack_f16x2(ol[8] * inv, ol[9] * inv);
                u1.y = pack_f16x2(ol[10] * inv, ol[11] * inv);
                u1.z = pack_f16x2(ol[12] * inv, ol[13] * inv);
                u1.w = pack_f16x2(ol[14] * inv, ol[15] * inv);
                uint4* dst = (uint4*)(p.out + (size_t)(qrow0 + r) * D + h * 16);
                const bool val = r < it.z - it.y * ROWS;
                dst[0] = val ? u0 : make_uint4(0, 0, 0, 0);
                dst[1] = val ? u1 : make_uint4(0, 0, 0, 0);
            }
            g += nk;
            ++q_it;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, 512);
    }
}

// the epilogues' activation on an array: thread i takes elements 2i and 2i + 1
__global__ void k_eval_act_tc(const float* __restrict__ x, float* __restrict__ y, int n, int act) {
    const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n) return;
    float v[2] = {x[i], i + 1 < n ? x[i + 1] : 0.f};
    act_n<2>(v, act);
    y[i] = v[0];
    if (i + 1 < n) y[i + 1] = v[1];
}

// ---------------------------------------------------------------- host side
uint32_t embed_smem(int mode, int fmt) {
    (void)fmt;
    const int ka = mode == 0 ? 1 : 2;
    // weights + two teams x (A operand, hidden tile, LayerNorm sums) + barriers + alignment;
    // at least 116 KB so that no two CTAs (512 TMEM columns each) share an SM
    const uint32_t need =
        64 * 128 * ka + 64 * 128 + 192 * 128 + 2 * (ka * ATOM + ATOM + 2 * 2 * 128 * 4) + EV_N * 4 + 128 +
        4 * EM_XB + 1024;
    return need < 116 * 1024 ? 116 * 1024 : need;
}
uint32_t post_smem(int mode, int fmt) {
    const uint32_t ka256 = fmt == FMT_E4M3 ? 2 : 4;
    const uint32_t wab = mode == 0 ? 192 * 128 : (mode == 1 ? 64 * 128 : 256 * 128);
    const uint32_t wbb = mode == 0 ? 0 : (mode == 1 ? 16 * 128 : 4 * 16 * 128);
    return 64 * 128 + 256 * 128 + ka256 * 64 * 128 + wab + ((wbb + 1023) & ~1023u) + 2 * PT_TEAM_BYTES +
           PV_N * 4 + 2 * PT_RED_FLOATS * 4 + 64 + 1024;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2-D map over a row-major 16-bit buffer (BF16 or FP16: TMA only moves bytes).
bool make_map_16(CUtensorMap* map, void* base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                 uint32_t box_outer) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Swizzled operand image of a weight matrix in format fmt:
// out[n][k'] = W[n][colmap(k')] (scaled by 1/scale for E4M3), zero padded.
// Atoms of 64 (16-bit) or 128 (E4M3) K-columns, each Npad rows of 128 bytes.
void build_image(std::vector<uint8_t>& out, int Npad, int Kpad, const std::vector<float>& W,
                 int N, int K, const std::vector<int>& colmap, const std::vector<int>& rowmap,
                 int fmt, float scale) {
    const int esz = fmt == FMT_E4M3 ? 1 : 2, ak = 128 / esz;
    out.assign((size_t)Npad * Kpad * esz, 0);
    const int atoms = Kpad / ak;
    for (int a = 0; a < atoms; ++a)
        for (int n = 0; n < Npad; ++n)
            for (int kk = 0; kk < ak; ++kk) {
                const int kp = a * ak + kk;
                const int src_k = colmap.empty() ? (kp < K ? kp : -1) : (kp < (int)colmap.size() ? colmap[kp] : -1);
                const int src_n = rowmap.empty() ? (n < N ? n : -1) : rowmap[n];
                float v = 0.f;
                if (src_k >= 0 && src_n >= 0) v = W[(size_t)src_n * K + src_k];
                const int byte = kk * esz;
                const size_t off = (size_t)a * Npad * 128 + (size_t)n * 128 +
                                   (size_t)((((byte >> 4) ^ (n & 7)) << 4)) + (byte & 15);
                if (fmt == FMT_E4M3) {
                    out[off] = (uint8_t)__nv_cvt_float_to_fp8(v / scale, __NV_SATFINITE, __NV_E4M3);
                } else if (fmt == FMT_FP16) {
                    const __half hv = __float2half_rn(v);
                    std::memcpy(&out[off], &hv, 2);
                } else {
                    const __nv_bfloat16 bv = __float2bfloat16_rn(v);
                    std::memcpy(&out[off], &bv, 2);
                }
            }
}

// Resident CTAs per SM of a kernel at its launch configuration (0 = cannot launch).
template <typename K>
int occupancy(K kernel, int threads, uint32_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) return 0;
    return n;
}

// Every kernel must fit one CTA per SM; the embedding and post kernels (512 TMEM
// columns each) must not share an SM with a second CTA.  Returns an
// empty string or a description of the kernels that do not fit.
template <int FMT>
std::string check_occupancy() {
    const int o_att[MLPF_ATTN_VARIANTS] = {
        occupancy(k_attention_tm<kOutF16<FMT>, 4>, TM_THREADS, TmLayout<4>::SMEM),
        occupancy(k_attention_tm<kOutF16<FMT>, 6>, TM_THREADS, TmLayout<6>::SMEM),
        occupancy(k_attention_tm<kOutF16<FMT>, 8>, TM_THREADS, TmLayout<8>::SMEM),
        occupancy(k_attention_warp<kOutF16<FMT>, 4>, aw_threads<128>(), AwLayout<4>::SMEM),
        occupancy(k_attention_warp<kOutF16<FMT>, 8>, aw_threads<128>(), AwLayout<8>::SMEM),
        occupancy(k_attention_warp<kOutF16<FMT>, 4, 64>, aw_threads<64>(), AwLayout<4, 64>::SMEM) / 2,
        occupancy(k_attention_warp<kOutF16<FMT>, 4, 128, true>, aw_threads<128, true>(), AwLayout<4>::SMEM),
        occupancy(k_attention_warp<kOutF16<FMT>, 8, 128, true>, aw_threads<128, true>(), AwLayout<8>::SMEM),
        occupancy(k_attention_pt<kOutF16<FMT>, 4>, PT_ATT_THREADS, PtLayout<4>::SMEM),
        occupancy(k_attention_pt<kOutF16<FMT>, 8>, PT_ATT_THREADS, PtLayout<8>::SMEM)};
    // the kernels that hold all 512 tensor-memory columns must not share an SM
    const int o_tm[] = {o_att[0], o_att[1], o_att[2], o_att[6], o_att[7], o_att[8], o_att[9]};
    for (int v : o_tm)
        if (v != 1)
            return "format " + std::to_string(FMT) + ": a tensor-memory attention kernel fits " + std::to_string(v) +
                   " CTAs per SM; ";
    const int o[6] = {*std::min_element(o_att, o_att + MLPF_ATTN_VARIANTS),
                      occupancy(k_post<0, FMT>, PT_THREADS, post_smem(0, FMT)),
                      occupancy(k_post<1, FMT>, PT_THREADS, post_smem(1, FMT)),
                      occupancy(k_post<2, FMT>, PT_THREADS, post_smem(2, FMT)),
                      occupancy(k_embed_qkv<0, FMT>, EM_THREADS, embed_smem(0, FMT)),
                      occupancy(k_embed_qkv<1, FMT>, EM_THREADS, embed_smem(1, FMT))};
    if (o[0] >= 1 && o[1] >= 1 && o[2] >= 1 && o[3] >= 1 && o[4] == 1 && o[5] == 1)
        return "";
    return "format " + std::to_string(FMT) + " CTAs/SM: attention " + std::to_string(o[0]) + ", post " +
           std::to_string(o[1]) + "/" + std::to_string(o[2]) + "/" + std::to_string(o[3]) + ", embed " +
           std::to_string(o[4]) + "/" + std::to_string(o[5]) + "; ";
}

template <int FMT>
void set_attrs() {
    cudaFuncSetAttribute(k_embed_qkv<0, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, embed_smem(0, FMT));
    cudaFuncSetAttribute(k_embed_qkv<1, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, embed_smem(1, FMT));
    cudaFuncSetAttribute(k_post<0, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, post_smem(0, FMT));
    cudaFuncSetAttribute(k_post<1, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, post_smem(1, FMT));
    cudaFuncSetAttribute(k_post<2, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, post_smem(2, FMT));
    cudaFuncSetAttribute(k_attention_tm<kOutF16<FMT>, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, TmLayout<4>::SMEM);
    cudaFuncSetAttribute(k_attention_tm<kOutF16<FMT>, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, TmLayout<6>::SMEM);
    cudaFuncSetAttribute(k_attention_tm<kOutF16<FMT>, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, TmLayout<8>::SMEM);
    cudaFuncSetAttribute(k_attention_warp<kOutF16<FMT>, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, AwLayout<4>::SMEM);
    cudaFuncSetAttribute(k_attention_warp<kOutF16<FMT>, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, AwLayout<8>::SMEM);
    cudaFuncSetAttribute(k_attention_warp<kOutF16<FMT>, 4, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, AwLayout<4, 64>::SMEM);
    cudaFuncSetAttribute(k_attention_warp<kOutF16<FMT>, 4, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, AwLayout<4>::SMEM);
    cudaFuncSetAttribute(k_attention_warp<kOutF16<FMT>, 8, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, AwLayout<8>::SMEM);
    cudaFuncSetAttribute(k_attention_pt<kOutF16<FMT>, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, PtLayout<4>::SMEM);
    cudaFuncSetAttribute(k_attention_pt<kOutF16<FMT>, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, PtLayout<8>::SMEM);
}

}  // namespace

void tc_eval_activation(const float* x, float* y, int n, int act, cudaStream_t st) {
    if (n > 0) k_eval_act_tc<<<((n + 1) / 2 + 255) / 256, 256, 0, st>>>(x, y, n, act);
}

bool tc_prepare_weights(Model& m) {
    const mlpf_config& c = m.cfg;
    auto H = [&](const std::string& s) -> const std::vector<float>& { return m.host.at(s).data; };
    struct Img {
        std::string name;
        std::vector<uint8_t> data[3];
        float scale;
    };
    std::vector<Img> imgs;
    std::vector<std::pair<std::string, std::vector<float>>> vecs;
    // Kpad16: padded K of the 16-bit image (E4M3: rounded up to 128)
    auto add = [&](const std::string& name, int Npad, int Kpad16, const std::vector<float>& W, int N, int K,
                   std::vector<int> colmap = {}, std::vector<int> rowmap = {}) {
        Img im;
        im.name = name;
        float amax = 0.f;
        for (float v : W) amax = std::max(amax, std::fabs(v));
        im.scale = amax > 0.f ? amax / 448.f : 1.f;  // per-tensor E4M3 scale
        build_image(im.data[FMT_FP16], Npad, Kpad16, W, N, K, colmap, rowmap, FMT_FP16, 1.f);
        build_image(im.data[FMT_E4M3], Npad, (Kpad16 + 127) / 128 * 128, W, N, K, colmap, rowmap, FMT_E4M3,
                    im.scale);
        imgs.push_back(std::move(im));
    };
    auto cat = [&](std::initializer_list<std::string> names, int pad_to = 0) {
        std::vector<float> v;
        for (auto& n : names) v.insert(v.end(), H(n).begin(), H(n).end());
        if ((int)v.size() < pad_to) v.resize(pad_to, 0.f);
        return v;
    };
    add("emb.w1", 64, 64, H("emb.w1"), 64, 42);
    add("emb.w2", 64, 64, H("emb.w2"), 64, 64);
    vecs.push_back({"emb.b1", H("emb.b1")});
    vecs.push_back({"emb.b2", H("emb.b2")});
    for (const char* s : {"pid", "reg"}) {
        const int L = std::string(s) == "pid" ? c.l_pid : c.l_reg;
        for (int l = 0; l < L; ++l) {
            const std::string p = std::string(s) + "." + std::to_string(l) + ".";
            std::vector<float> wqkv = cat({p + "wq", p + "wk", p + "wv"});
            add(p + "wqkv", 192, 64, wqkv, 192, 64);
            add(p + "wo", 64, 64, H(p + "wo"), 64, 64);
            add(p + "ffn.w1", 256, 64, H(p + "ffn.w1"), 256, 64);
            add(p + "ffn.w2", 64, 256, H(p + "ffn.w2"), 64, 256);
            vecs.push_back({p + "bqkv", cat({p + "bq", p + "bk", p + "bv"})});
            for (const char* v : {"bo", "ln1.g", "ln1.b", "ln2.g", "ln2.b", "ffn.b1", "ffn.b2"})
                vecs.push_back({p + v, H(p + v)});
        }
        vecs.push_back({std::string(s) + ".lnf.g", H(std::string(s) + ".lnf.g")});
        vecs.push_back({std::string(s) + ".lnf.b", H(std::string(s) + ".lnf.b")});
    }
    {
        // concat(x, h_pid): x in K-columns 0..41, h_pid in 64..127 (both formats)
        std::vector<int> colmap(128, -1);
        for (int k = 0; k < 42; ++k) colmap[k] = k;
        for (int k = 0; k < 64; ++k) colmap[64 + k] = 42 + k;
        add("remb.w1", 64, 128, H("remb.w1"), 64, 106, colmap);
        add("remb.w2", 64, 64, H("remb.w2"), 64, 64);
        vecs.push_back({"remb.b1", H("remb.b1")});
        vecs.push_back({"remb.b2", H("remb.b2")});
    }
    add("head.cls.w1", 64, 64, H("head.cls.w1"), 64, 64);
    add("head.cls.w2", 16, 64, H("head.cls.w2"), 6, 64);
    vecs.push_back({"head.cls.b1", H("head.cls.b1")});
    vecs.push_back({"head.cls.b2", cat({"head.cls.b2"}, 16)});
    {
        std::vector<float> w1 = cat({"head.pt.w1", "head.eta.w1", "head.phi.w1", "head.e.w1"});
        add("head.reg.w1", 256, 64, w1, 256, 64);
        // block-diagonal second layer: output o reads hidden block of its head
        std::vector<float> w2(5 * 256, 0.f);
        const char* names[4] = {"pt", "eta", "phi", "e"};
        int o = 0;
        for (int hh = 0; hh < 4; ++hh) {
            const auto& src = H(std::string("head.") + names[hh] + ".w2");
            const int k = (int)src.size() / 64;
            for (int r = 0; r < k; ++r, ++o)
                for (int i = 0; i < 64; ++i) w2[(size_t)o * 256 + hh * 64 + i] = src[(size_t)r * 64 + i];
        }
        add("head.reg.w2", 16, 256, w2, 5, 256);
        vecs.push_back({"head.reg.b1", cat({"head.pt.b1", "head.eta.b1", "head.phi.b1", "head.e.b1"})});
        vecs.push_back({"head.reg.b2", cat({"head.pt.b2", "head.eta.b2", "head.phi.b2", "head.e.b2"}, 16)});
    }
    size_t ib = 0, vb = 0;
    for (auto& i : imgs)
        for (int f = 1; f < 3; ++f) ib += (i.data[f].size() + 1023) / 1024 * 1024;
    for (auto& v : vecs) vb += (v.second.size() + 63) / 64 * 64;
    if (cudaMalloc(&m.w.img_base, ib) != cudaSuccess) { set_error("weight image allocation"); return false; }
    if (cudaMalloc(&m.w.tc_f32_base, vb * 4) != cudaSuccess) { set_error("bias allocation"); return false; }
    std::vector<uint8_t> hi(ib, 0);
    std::vector<float> hv(vb, 0.f);
    size_t o = 0;
    for (auto& i : imgs) {
        for (int f = 1; f < 3; ++f) {   // FP16 and E4M3 images (no mode runs a GEMM on BF16 operands)
            std::memcpy(&hi[o], i.data[f].data(), i.data[f].size());
            (f == FMT_FP16 ? m.w.img_h : m.w.img8)[i.name] = m.w.img_base + o;
            o += (i.data[f].size() + 1023) / 1024 * 1024;
        }
        m.w.w_scale[i.name] = i.scale;
    }
    o = 0;
    for (auto& v : vecs) {
        std::copy(v.second.begin(), v.second.end(), hv.begin() + o);
        m.w.tcv[v.first] = m.w.tc_f32_base + o;
        o += (v.second.size() + 63) / 64 * 64;
    }
    if (cudaMemcpy(m.w.img_base, hi.data(), ib, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m.w.tc_f32_base, hv.data(), vb * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("weight image upload");
        return false;
    }
    static bool attrs = false;
    if (!attrs) {
        set_attrs<FMT_BF16>();
        set_attrs<FMT_FP16>();
        set_attrs<FMT_E4M3>();
        attrs = true;
    }
    if (cudaGetLastError() != cudaSuccess) { set_error("kernel attribute setup"); return false; }
    m.embed_ctas_per_sm = std::max(1, std::min(occupancy(k_embed_qkv<1, FMT_BF16>, EM_THREADS, embed_smem(1, FMT_BF16)),
                                               occupancy(k_embed_qkv<1, FMT_FP16>, EM_THREADS, embed_smem(1, FMT_FP16))));
    const std::string occ = check_occupancy<FMT_BF16>() + check_occupancy<FMT_FP16>() + check_occupancy<FMT_E4M3>();
    if (!occ.empty()) {
        cudaGetLastError();
        set_error("a tensor-core kernel does not fit its launch configuration: " + occ);
        return false;
    }
    return true;
}

bool tc_make_maps(Model& m) {
    Workspace& w = m.ws;
    const uint64_t T = (uint64_t)w.cap_tpad;
    bool ok = make_map_16(&w.map_q, w.tq, 64, T, 64, 128) && make_map_16(&w.map_q64, w.tq, 64, T, 64, 64) &&
              make_map_16(&w.map_k, w.tk, 64, T, 64, 64) &&
              make_map_16(&w.map_o, w.to, 64, T, 64, 128) && make_map_16(&w.map_vt, w.tvt, T, 64, 64, 64) &&
              make_map_16(&w.map_vt16, w.tvt, T, 64, 64, 16) &&
              make_map_16(&w.map_hp, w.thp, 64, T, 64, 128);
    if (!ok) set_error("cuTensorMapEncodeTiled failed");
    return ok;
}

int act_slot(Model& m, const std::string& name) {
    auto it = m.act_slot.find(name);
    if (it != m.act_slot.end()) return it->second;
    const int i = (int)m.act_slot.size();
    m.act_slot[name] = i;
    if ((int)m.act_scale.size() <= i) m.act_scale.resize(i + 1, 1.f);
    return i;
}

template <int FMT>
static int64_t run_tc(Model& m, Workspace& w, bool profile, const float* x, const int32_t* cu, int n_events,
                      float* logits, float* reg, cudaStream_t st) {
    const mlpf_config& c = m.cfg;
    auto prof_begin = [&](Model& mm, cudaStream_t s, const char* name) {
        if (profile) mlpf::prof_begin(mm, s, name);
    };
    auto prof_end = [&](Model& mm, cudaStream_t s) {
        if (profile) mlpf::prof_end(mm, s);
    };
    auto V = [&](const std::string& s) { return (const float*)m.w.tcv.at(s); };
    // weight image of a GEMM in format f
    auto IF = [&](const std::string& s, int f) {
        return (const uint8_t*)(f == FMT_FP16 ? m.w.img_h : m.w.img8).at(s);
    };
    constexpr int FE = FMT_FP16;  // embedding FFNs and output heads (16-bit in every mode)
    auto I = [&](const std::string& s) { return IF(s, kGemm<FMT>); };
    auto IE = [&](const std::string& s) { return IF(s, FE); };
    // E4M3: 1/s_a of an activation slot and s_a * s_w of a GEMM (1 for 16-bit formats)
    auto QS = [&](const std::string& slot) { return FMT == FMT_E4M3 ? 1.f / m.act_scale[act_slot(m, slot)] : 1.f; };
    auto DS = [&](const std::string& slot, const std::string& wname) {
        return FMT == FMT_E4M3 ? m.act_scale[act_slot(m, slot)] * m.w.w_scale.at(wname) : 1.f;
    };
    unsigned* amax = m.calibrating ? m.amax_dev : nullptr;
    int64_t n = 0;
    const int grid = m.sm_count;
    prof_begin(m, st, "schedule");
    k_schedule<<<1, 1024, 0, st>>>(cu, n_events, w.blk, w.items, w.counters, (int)(w.cap_tpad / 64),
                                   (int)(w.cap_tpad / 128 + w.cap_events + 1));
    prof_end(m, st);
    ++n;
    auto attention = [&](int layer) {
        AttnParams ap{w.items, w.counters, layer, (uint16_t*)w.to, m.status, (uint64_t)m.wait_limit_ns,
                      m.debug_stall ? 1 : 0, m.attn_window, w.kmax};
        prof_begin(m, st, "attention");
        constexpr bool AF = kOutF16<FMT>;
        const dim3 g(grid * m.attn_ctas_per_sm);
        switch (m.attn_variant[FMT]) {
            case 0: k_attention_tm<AF, 4><<<g, TM_THREADS, TmLayout<4>::SMEM, st>>>(w.map_q, w.map_k, w.map_vt16, ap); break;
            case 1: k_attention_tm<AF, 6><<<g, TM_THREADS, TmLayout<6>::SMEM, st>>>(w.map_q, w.map_k, w.map_vt16, ap); break;
            case 2: k_attention_tm<AF, 8><<<g, TM_THREADS, TmLayout<8>::SMEM, st>>>(w.map_q, w.map_k, w.map_vt16, ap); break;
            case 3: k_attention_warp<AF, 4><<<g, aw_threads<128>(), AwLayout<4>::SMEM, st>>>(w.map_q, w.map_k, w.map_vt, ap); break;
            case 5: k_attention_warp<AF, 4, 64><<<2 * g.x, aw_threads<64>(), AwLayout<4, 64>::SMEM, st>>>(w.map_q64, w.map_k, w.map_vt, ap); break;
            case 6: k_attention_warp<AF, 4, 128, true><<<g, aw_threads<128, true>(), AwLayout<4>::SMEM, st>>>(w.map_q, w.map_k, w.map_vt, ap); break;
            case 7: k_attention_warp<AF, 8, 128, true><<<g, aw_threads<128, true>(), AwLayout<8>::SMEM, st>>>(w.map_q, w.map_k, w.map_vt, ap); break;
            case 8: k_attention_pt<AF, 4><<<g, PT_ATT_THREADS, PtLayout<4>::SMEM, st>>>(w.map_q, w.map_k, w.map_vt, ap); break;
            case 9: k_attention_pt<AF, 8><<<g, PT_ATT_THREADS, PtLayout<8>::SMEM, st>>>(w.map_q, w.map_k, w.map_vt, ap); break;
            default: k_attention_warp<AF, 8><<<g, aw_threads<128>(), AwLayout<8>::SMEM, st>>>(w.map_q, w.map_k, w.map_vt, ap); break;
        }
        prof_end(m, st);
        ++n;
    };
    auto embed = [&](int mode, const std::string& lp) {
        EmbedParams ep{};
        ep.x = x;
        ep.blk = w.blk;
        ep.counters = w.counters;
        const std::string e = mode == 0 ? "emb." : "remb.";
        ep.w1 = IE(e + "w1");
        ep.w2 = IE(e + "w2");
        ep.wqkv = I(lp + "wqkv");
        ep.b1 = V(e + "b1");
        ep.b2 = V(e + "b2");
        ep.lng = V(lp + "ln1.g");
        ep.lnb = V(lp + "ln1.b");
        ep.bqkv = V(lp + "bqkv");
        ep.hp = (const uint16_t*)w.thp;
        ep.z = w.tz;
        ep.q = (uint16_t*)w.tq;
        ep.k = (uint16_t*)w.tk;
        ep.vt = (uint16_t*)w.tvt;
        ep.kmax = w.kmax;
        ep.ldvt = w.cap_tpad;
        ep.status = m.status;
        ep.wait_ns = (uint64_t)m.wait_limit_ns;
        ep.act = c.act;
        const std::string s_in = mode == 0 ? "x" : "remb.in", s_h = e + "h", s_ln = lp + "ln1";
        ep.qs[0] = 1.f;  // the embedding FFN is 16-bit in every mode
        ep.qs[1] = 1.f;
        ep.qs[2] = QS(s_ln);
        ep.ds[0] = 1.f;
        ep.ds[1] = 1.f;
        ep.ds[2] = DS(s_ln, lp + "wqkv");
        ep.amax = amax;
        ep.slot[0] = act_slot(m, s_in);
        ep.slot[1] = act_slot(m, s_h);
        ep.slot[2] = act_slot(m, s_ln);
        prof_begin(m, st, mode == 0 ? "embed_qkv" : "reg_embed_qkv");
        if (mode == 0)
            k_embed_qkv<0, FMT><<<grid * m.embed_ctas_per_sm, EM_THREADS, embed_smem(0, FMT), st>>>(w.map_hp, ep);
        else
            k_embed_qkv<1, FMT><<<grid * m.embed_ctas_per_sm, EM_THREADS, embed_smem(1, FMT), st>>>(w.map_hp, ep);
        prof_end(m, st);
        ++n;
    };
    auto post = [&](int mode, const std::string& lp, const std::string& next) {
        PostParams pp{};
        pp.x = x;
        pp.blk = w.blk;
        pp.counters = w.counters;
        pp.wo = I(lp + "wo");
        pp.wup = I(lp + "ffn.w1");
        pp.wdn = I(lp + "ffn.w2");
        pp.bo = V(lp + "bo");
        pp.ln2g = V(lp + "ln2.g");
        pp.ln2b = V(lp + "ln2.b");
        pp.bup = V(lp + "ffn.b1");
        pp.bdn = V(lp + "ffn.b2");
        std::string s_a, s_b, w_a, w_b;
        if (mode == 0) {
            pp.wa = I(next + "wqkv");
            pp.wb = nullptr;
            pp.lng = V(next + "ln1.g");
            pp.lnb = V(next + "ln1.b");
            pp.ba = V(next + "bqkv");
            s_a = next + "ln1";
            w_a = next + "wqkv";
        } else if (mode == 1) {
            pp.wa = IE("head.cls.w1");
            pp.wb = IE("head.cls.w2");
            pp.lng = V("pid.lnf.g");
            pp.lnb = V("pid.lnf.b");
            pp.ba = V("head.cls.b1");
            pp.bb = V("head.cls.b2");
            s_a = "pid.lnf";
            s_b = "cls.h";
            w_a = "head.cls.w1";
            w_b = "head.cls.w2";
        } else {
            pp.wa = IE("head.reg.w1");
            pp.wb = IE("head.reg.w2");
            pp.lng = V("reg.lnf.g");
            pp.lnb = V("reg.lnf.b");
            pp.ba = V("head.reg.b1");
            pp.bb = V("head.reg.b2");
            s_a = "reg.lnf";
            s_b = "heads.h";
            w_a = "head.reg.w1";
            w_b = "head.reg.w2";
        }
        const std::string s_o = lp + "o", s_ln2 = lp + "ln2", s_ffn = lp + "ffn";
        pp.qs[0] = QS(s_o);
        pp.qs[1] = QS(s_ln2);
        pp.qs[2] = QS(s_ffn);
        // heads (modes 1, 2) are 16-bit in every mode
        pp.qs[3] = mode == 0 ? QS(s_a) : 1.f;
        pp.qs[4] = 1.f;
        pp.ds[0] = DS(s_o, lp + "wo");
        pp.ds[1] = DS(s_ln2, lp + "ffn.w1");
        pp.ds[2] = DS(s_ffn, lp + "ffn.w2");
        pp.ds[3] = mode == 0 ? DS(s_a, w_a) : 1.f;
        pp.ds[4] = 1.f;
        pp.amax = amax;
        pp.slot[0] = act_slot(m, s_o);
        pp.slot[1] = act_slot(m, s_ln2);
        pp.slot[2] = act_slot(m, s_ffn);
        pp.slot[3] = act_slot(m, s_a);
        pp.slot[4] = mode == 0 ? 0 : act_slot(m, s_b);
        pp.z = w.tz;
        pp.q = (uint16_t*)w.tq;
        pp.k = (uint16_t*)w.tk;
        pp.vt = (uint16_t*)w.tvt;
        pp.hp = (uint16_t*)w.thp;
        pp.kmax = w.kmax;
        pp.ldvt = w.cap_tpad;
        pp.logits = logits;
        pp.reg = reg;
        pp.status = m.status;
        pp.wait_ns = (uint64_t)m.wait_limit_ns;
        pp.act = c.act;
        prof_begin(m, st, mode == 0 ? "post_qkv" : (mode == 1 ? "post_cls_head" : "post_reg_heads"));
        if (mode == 0)
            k_post<0, FMT><<<grid, PT_THREADS, post_smem(0, FMT), st>>>(w.map_o, pp);
        else if (mode == 1)
            k_post<1, FMT><<<grid, PT_THREADS, post_smem(1, FMT), st>>>(w.map_o, pp);
        else
            k_post<2, FMT><<<grid, PT_THREADS, post_smem(2, FMT), st>>>(w.map_o, pp);
        prof_end(m, st);
        ++n;
    };
    int layer = 0;
    embed(0, "pid.0.");
    for (int l = 0; l < c.l_pid; ++l) {
        attention(layer++);
        const std::string lp = "pid." + std::to_string(l) + ".";
        if (l + 1 < c.l_pid)
            post(0, lp, "pid." + std::to_string(l + 1) + ".");
        else
            post(1, lp, "");
    }
    embed(1, "reg.0.");
    for (int l = 0; l < c.l_reg; ++l) {
        attention(layer++);
        const std::string lp = "reg." + std::to_string(l) + ".";
        if (l + 1 < c.l_reg)
            post(0, lp, "reg." + std::to_string(l + 1) + ".");
        else
            post(2, lp, "");
    }
    if (cudaPeekAtLastError() != cudaSuccess) return -1;
    return n;
}

int64_t run_forward_tc(Model& m, int prec, const float* x, const int32_t* cu, int n_events, int total,
                       int max_n, float* logits, float* reg, cudaStream_t st, Workspace* ws, bool profile) {
    (void)total;
    (void)max_n;
    Workspace& w = ws ? *ws : m.ws;
    if (prec == MLPF_FP8) return run_tc<FMT_E4M3>(m, w, profile, x, cu, n_events, logits, reg, st);
    return prec == MLPF_FP16 ? run_tc<FMT_FP16>(m, w, profile, x, cu, n_events, logits, reg, st)
                             : run_tc<FMT_BF16>(m, w, profile, x, cu, n_events, logits, reg, st);
}

}  // namespace mlpf
