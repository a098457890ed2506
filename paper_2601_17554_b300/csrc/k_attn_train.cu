// Varlen self-attention of the training step on the tensor cores (warp-level m16n8k16
// MMAs, BF16 or FP16 operands, FP32 accumulation and softmax statistics): forward with
// the rows' log-sum-exp kept for the backward, and the backward as two kernels that
// recompute the probabilities from Q, K and the log-sum-exp (Sec. 5.3, Eq. 4: per head
// softmax(Q K^T / sqrt(dh)) V within each event; its gradient
//   dV = P^T dO,  dP = dO V^T,  dS = P o (dP - rowsum(dO o O)),
//   dQ = dS K / sqrt(dh),  dK = dS^T Q / sqrt(dh)).
// Activations stay FP32 in HBM ([T, 3d] Q|K|V, [T, d] O and dO); each CTA converts the
// 64-row tiles it stages into shared memory.  One CTA per (64-row tile, head, event),
// four warps of 16 rows; scores in log2 units (Q pre-multiplied by log2(e)/sqrt(dh)).
#include <cuda_runtime.h>

#include "internal.h"
#include "ptx.cuh"

namespace mlpf {
namespace {

constexpr float kLog2e = 1.4426950408889634f;

// Stage rows r0 .. r0 + 63 of an event (rows >= n are zero) of DH columns starting at
// `col` of a row-major FP32 matrix (row stride ld) into shared memory as 16-bit values
// times `mul`, row stride DH + 8 elements (16-byte padded rows: conflict-free ldmatrix).
template <int DH, bool F16>
__device__ __forceinline__ void stage_tile(uint16_t* dst, const float* __restrict__ src, long ld, int col,
                                           int start, int r0, int n, float mul) {
    constexpr int LD = DH + 8, PER_ROW = DH / 4;
    for (int i = threadIdx.x; i < 64 * PER_ROW; i += 128) {
        const int r = i / PER_ROW, c4 = (i % PER_ROW) * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r0 + r < n) v = *reinterpret_cast<const float4*>(src + (long)(start + r0 + r) * ld + col + c4);
        uint2 p;
        p.x = pack2<F16>(v.x * mul, v.y * mul);
        p.y = pack2<F16>(v.z * mul, v.w * mul);
        *reinterpret_cast<uint2*>(dst + r * LD + c4) = p;
    }
}

// A fragment (16 x 16) of rows rb.., columns kc.. of a [rows][LD] tile
template <int LD>
__device__ __forceinline__ void load_a(const uint16_t* t, int rb, int kc, uint32_t* a) {
    const int l = threadIdx.x & 31;
    const uint16_t* p = t + (rb + (l & 7) + ((l >> 3) & 1) * 8) * LD + kc + (l >> 4) * 8;
    ldsm_x4(smem_u32(p), a[0], a[1], a[2], a[3]);
}
// B fragments of two n-tiles (n = nb .. nb + 15) for k = kc .. kc + 15 from a tile
// stored [n][k]: b[0], b[1] for n-tile 0, b[2], b[3] for n-tile 1
template <int LD>
__device__ __forceinline__ void load_b_nk(const uint16_t* t, int nb, int kc, uint32_t* b) {
    const int l = threadIdx.x & 31, i = l >> 3;
    const uint16_t* p = t + (nb + (l & 7) + (i >> 1) * 8) * LD + kc + (i & 1) * 8;
    ldsm_x4(smem_u32(p), b[0], b[1], b[2], b[3]);
}
// the same from a tile stored [k][n] (k = kb .. kb + 15, n = nc .. nc + 15)
template <int LD>
__device__ __forceinline__ void load_b_kn(const uint16_t* t, int kb, int nc, uint32_t* b) {
    const int l = threadIdx.x & 31, i = l >> 3;
    const uint16_t* p = t + (kb + (l & 7) + (i & 1) * 8) * LD + nc + (i >> 1) * 8;
    ldsm_x4_t(smem_u32(p), b[0], b[1], b[2], b[3]);
}
// accumulator fragments of n-tiles 2 kk and 2 kk + 1 -> A fragment for k = 16 kk ..
template <bool F16>
__device__ __forceinline__ void c_to_a(const float* c0, const float* c1, uint32_t* a) {
    a[0] = pack2<F16>(c0[0], c0[1]);
    a[1] = pack2<F16>(c0[2], c0[3]);
    a[2] = pack2<F16>(c1[0], c1[1]);
    a[3] = pack2<F16>(c1[2], c1[3]);
}

// S (16 rows x 64 columns, 8 n-tiles) = A (16 x DH, fragments a) times the tile `t`
// stored [n][k] (64 x DH)^T
template <int DH, bool F16>
__device__ __forceinline__ void scores(const uint32_t (*a)[4], const uint16_t* t, float (*s)[4]) {
    constexpr int LD = DH + 8;
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j][0] = s[j][1] = s[j][2] = s[j][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < DH / 16; ++kk)
#pragma unroll
        for (int np = 0; np < 4; ++np) {
            uint32_t b[4];
            load_b_nk<LD>(t, np * 16, kk * 16, b);
            mma16816<F16>(s[2 * np], a[kk], b[0], b[1]);
            mma16816<F16>(s[2 * np + 1], a[kk], b[2], b[3]);
        }
}
// acc (16 x DH) += P (16 x 64, accumulator fragments p) times the tile `t` stored [k][n]
template <int DH, bool F16>
__device__ __forceinline__ void accumulate(const float (*p)[4], const uint16_t* t, float (*acc)[4]) {
    constexpr int LD = DH + 8;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        uint32_t a[4];
        c_to_a<F16>(p[2 * kk], p[2 * kk + 1], a);
#pragma unroll
        for (int dp = 0; dp < DH / 16; ++dp) {
            uint32_t b[4];
            load_b_kn<LD>(t, kk * 16, dp * 16, b);
            mma16816<F16>(acc[2 * dp], a, b[0], b[1]);
            mma16816<F16>(acc[2 * dp + 1], a, b[2], b[3]);
        }
    }
}

// window > 0: the query rows of 128-row block y attend to the keys of blocks y - window ..
// y + window only (the eta-ordered block-banded reading of windowed attention)
template <int DH, bool F16>
__global__ void __launch_bounds__(128) k_attn_fwd_tc(const float* __restrict__ qkv, float* __restrict__ out,
                                                     float* __restrict__ lse, const int32_t* __restrict__ cu, int d,
                                                     float scale, int window) {
    constexpr int LD = DH + 8;
    __shared__ __align__(16) uint16_t Qs[64 * LD], Ks[64 * LD], Vs[64 * LD];
    const int e = blockIdx.z, h = blockIdx.y, H = gridDim.y;
    const int start = cu[e], n = cu[e + 1] - start, q0 = blockIdx.x * 64;
    if (q0 >= n) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    const long ld = 3L * d;
    stage_tile<DH, F16>(Qs, qkv, ld, h * DH, start, q0, n, scale * kLog2e);
    __syncthreads();
    uint32_t qa[DH / 16][4];
#pragma unroll
    for (int kk = 0; kk < DH / 16; ++kk) load_a<LD>(Qs, warp * 16, kk * 16, qa[kk]);
    float o[DH / 8][4] = {};
    float m[2] = {-INFINITY, -INFINITY}, l[2] = {0.f, 0.f};
    int kbeg = 0, kend = n;
    if (window > 0) {
        const int y = q0 / 128;
        kbeg = max(0, (y - window) * 128);
        kend = min(n, (y + window + 1) * 128);
    }
    for (int kb = kbeg; kb < kend; kb += 64) {
        __syncthreads();
        stage_tile<DH, F16>(Ks, qkv, ld, d + h * DH, start, kb, kend, 1.f);
        stage_tile<DH, F16>(Vs, qkv, ld, 2 * d + h * DH, start, kb, kend, 1.f);
        __syncthreads();
        float s[8][4];
        scores<DH, F16>(qa, Ks, s);
        float mx[2] = {m[0], m[1]};
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (kb + j * 8 + 2 * c + (u & 1) >= kend) s[j][u] = -INFINITY;
                mx[u >> 1] = fmaxf(mx[u >> 1], s[j][u]);
            }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            mx[r] = fmaxf(mx[r], __shfl_xor_sync(0xffffffffu, mx[r], 1));
            mx[r] = fmaxf(mx[r], __shfl_xor_sync(0xffffffffu, mx[r], 2));
        }
        const float al[2] = {ex2_approx(m[0] - mx[0]), ex2_approx(m[1] - mx[1])};
        l[0] *= al[0];
        l[1] *= al[1];
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                s[j][u] = ex2_approx(s[j][u] - mx[u >> 1]);
                l[u >> 1] += s[j][u];
            }
#pragma unroll
        for (int j = 0; j < DH / 8; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u) o[j][u] *= al[u >> 1];
        m[0] = mx[0];
        m[1] = mx[1];
        accumulate<DH, F16>(s, Vs, o);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        l[r] += __shfl_xor_sync(0xffffffffu, l[r], 1);
        l[r] += __shfl_xor_sync(0xffffffffu, l[r], 2);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int row = q0 + warp * 16 + g + 8 * r;
        if (row >= n) continue;
        const float inv = 1.f / l[r];
        float* orow = out + (long)(start + row) * d + h * DH;
#pragma unroll
        for (int j = 0; j < DH / 8; ++j)
            *reinterpret_cast<float2*>(orow + j * 8 + 2 * c) = make_float2(o[j][2 * r] * inv, o[j][2 * r + 1] * inv);
        if (lse && c == 0) lse[(long)(start + row) * H + h] = (m[r] + __log2f(l[r])) / kLog2e;
    }
}

// dQ: one CTA per 64 query rows; loops over the event's key tiles.
template <int DH, bool F16>
__global__ void __launch_bounds__(128) k_attn_dq_tc(const float* __restrict__ qkv, const float* __restrict__ dO,
                                                    const float* __restrict__ lse, const float* __restrict__ D,
                                                    float* __restrict__ dqkv, const int32_t* __restrict__ cu, int d,
                                                    float scale) {
    constexpr int LD = DH + 8;
    __shared__ __align__(16) uint16_t Qs[64 * LD], Gs[64 * LD], Ks[64 * LD], Vs[64 * LD];
    const int e = blockIdx.z, h = blockIdx.y, H = gridDim.y;
    const int start = cu[e], n = cu[e + 1] - start, q0 = blockIdx.x * 64;
    if (q0 >= n) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    const long ld = 3L * d;
    stage_tile<DH, F16>(Qs, qkv, ld, h * DH, start, q0, n, scale * kLog2e);
    stage_tile<DH, F16>(Gs, dO, d, h * DH, start, q0, n, 1.f);
    __syncthreads();
    uint32_t qa[DH / 16][4], ga[DH / 16][4];
#pragma unroll
    for (int kk = 0; kk < DH / 16; ++kk) {
        load_a<LD>(Qs, warp * 16, kk * 16, qa[kk]);
        load_a<LD>(Gs, warp * 16, kk * 16, ga[kk]);
    }
    float L2[2], Dr[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int row = q0 + warp * 16 + g + 8 * r;
        L2[r] = row < n ? lse[(long)(start + row) * H + h] * kLog2e : 0.f;
        Dr[r] = row < n ? D[(long)(start + row) * H + h] : 0.f;
    }
    float dq[DH / 8][4] = {};
    for (int kb = 0; kb < n; kb += 64) {
        __syncthreads();
        stage_tile<DH, F16>(Ks, qkv, ld, d + h * DH, start, kb, n, 1.f);
        stage_tile<DH, F16>(Vs, qkv, ld, 2 * d + h * DH, start, kb, n, 1.f);
        __syncthreads();
        float s[8][4], dp[8][4];
        scores<DH, F16>(qa, Ks, s);
        scores<DH, F16>(ga, Vs, dp);
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool valid = kb + j * 8 + 2 * c + (u & 1) < n;
                const float p = valid ? ex2_approx(s[j][u] - L2[u >> 1]) : 0.f;
                s[j][u] = p * (dp[j][u] - Dr[u >> 1]);   // dS
            }
        accumulate<DH, F16>(s, Ks, dq);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int row = q0 + warp * 16 + g + 8 * r;
        if (row >= n) continue;
        float* dst = dqkv + (long)(start + row) * ld + h * DH;
#pragma unroll
        for (int j = 0; j < DH / 8; ++j)
            *reinterpret_cast<float2*>(dst + j * 8 + 2 * c) = make_float2(dq[j][2 * r] * scale, dq[j][2 * r + 1] * scale);
    }
}

// dK, dV: one CTA per 64 key rows; loops over the event's query tiles.
template <int DH, bool F16>
__global__ void __launch_bounds__(128) k_attn_dkv_tc(const float* __restrict__ qkv, const float* __restrict__ dO,
                                                     const float* __restrict__ lse, const float* __restrict__ D,
                                                     float* __restrict__ dqkv, const int32_t* __restrict__ cu, int d,
                                                     float scale) {
    constexpr int LD = DH + 8;
    __shared__ __align__(16) uint16_t Ks[64 * LD], Vs[64 * LD], Qs[64 * LD], Gs[64 * LD];
    __shared__ float L2s[64], Ds[64];
    const int e = blockIdx.z, h = blockIdx.y, H = gridDim.y;
    const int start = cu[e], n = cu[e + 1] - start, k0 = blockIdx.x * 64;
    if (k0 >= n) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, c = lane & 3;
    const int g = lane >> 2;
    const long ld = 3L * d;
    stage_tile<DH, F16>(Ks, qkv, ld, d + h * DH, start, k0, n, 1.f);
    stage_tile<DH, F16>(Vs, qkv, ld, 2 * d + h * DH, start, k0, n, 1.f);
    __syncthreads();
    uint32_t ka[DH / 16][4], va[DH / 16][4];
#pragma unroll
    for (int kk = 0; kk < DH / 16; ++kk) {
        load_a<LD>(Ks, warp * 16, kk * 16, ka[kk]);
        load_a<LD>(Vs, warp * 16, kk * 16, va[kk]);
    }
    float dk[DH / 8][4] = {}, dv[DH / 8][4] = {};
    for (int qb = 0; qb < n; qb += 64) {
        __syncthreads();
        stage_tile<DH, F16>(Qs, qkv, ld, h * DH, start, qb, n, scale * kLog2e);
        stage_tile<DH, F16>(Gs, dO, d, h * DH, start, qb, n, 1.f);
        if (threadIdx.x < 64) {
            const int row = qb + threadIdx.x;
            L2s[threadIdx.x] = row < n ? lse[(long)(start + row) * H + h] * kLog2e : INFINITY;
            Ds[threadIdx.x] = row < n ? D[(long)(start + row) * H + h] : 0.f;
        }
        __syncthreads();
        float s[8][4], dp[8][4];
        scores<DH, F16>(ka, Qs, s);    // S^T: keys x queries
        scores<DH, F16>(va, Gs, dp);   // dP^T
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int qc = j * 8 + 2 * c + (u & 1);
                s[j][u] = ex2_approx(s[j][u] - L2s[qc]);   // P^T (0 for queries beyond the event)
                dp[j][u] = s[j][u] * (dp[j][u] - Ds[qc]);    // dS^T
            }
        accumulate<DH, F16>(s, Gs, dv);
        accumulate<DH, F16>(dp, Qs, dk);
    }
    (void)g;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int row = k0 + warp * 16 + (lane >> 2) + 8 * r;
        if (row >= n) continue;
        float* dst = dqkv + (long)(start + row) * ld + h * DH;
#pragma unroll
        for (int j = 0; j < DH / 8; ++j) {
            *reinterpret_cast<float2*>(dst + d + j * 8 + 2 * c) =
                make_float2(dk[j][2 * r] / kLog2e, dk[j][2 * r + 1] / kLog2e);
            *reinterpret_cast<float2*>(dst + 2 * d + j * 8 + 2 * c) = make_float2(dv[j][2 * r], dv[j][2 * r + 1]);
        }
    }
}

// Forward of the generic-width inference path on 16-bit Q | K | V ([T, 3d], written by the
// QKV GEMM's epilogue, Q pre-multiplied by log2(e)/sqrt(dh): the wide path folds that
// factor into the Q rows of its two-term QKV weights and biases): 128 query rows per CTA
// (eight warps of 16 rows), K / V tiles of 64 rows double-buffered with asynchronous
// copies.  The QK^T MMA starts from the rows' negated exponent references, so its output
// is the base-2 exponent itself; the references are raised lazily (the first tile sets
// them to the row maxima, a later tile only when a row maximum exceeds its reference by
// more than kRaise, so P <= 2^kRaise), P = 2^(S - ref) is taken two at a time with packed
// MUFU exponentials straight into the A fragments of the PV MMA, and the row sums are
// one more MMA of the same P against a block of ones (the sums of the rounded P that the
// PV product uses).  Writes O as FP16 rows of stride ldo16 (the operand of the output
// projection's GEMM).
template <int DH, bool F16>
__global__ void __launch_bounds__(256) k_attn_fwd16(const uint16_t* __restrict__ qkv16, uint16_t* __restrict__ o16,
                                                    int ldo16, const int32_t* __restrict__ cu, int d, int window) {
    constexpr int LD = DH + 8, CH = DH / 8;   // 16-byte chunks per row
    constexpr float kRaise = 4.f;
    extern __shared__ __align__(16) uint16_t att_smem[];   // (128 + 4 x 64) rows of LD
    uint16_t* Qs = att_smem;
    auto Kt = [&](int b) { return att_smem + (128 + 64 * b) * LD; };
    auto Vt = [&](int b) { return att_smem + (256 + 64 * b) * LD; };
    const int e = blockIdx.z, h = blockIdx.y;
    const int start = cu[e], n = cu[e + 1] - start, q0 = blockIdx.x * 128;
    if (q0 >= n) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
    const long ld = 3L * d;
    const uint32_t ONE2 = F16 ? 0x3C003C00u : 0x3F803F80u;
    int kbeg = 0, kend = n;
    if (window > 0) {
        const int y = q0 / 128;
        kbeg = max(0, (y - window) * 128);
        kend = min(n, (y + window + 1) * 128);
    }
    // rows r0 .. r0 + rows - 1 of column block col (rows at or beyond lim are zero)
    auto stage = [&](uint16_t* dst, int rows, int r0, int lim, int col) {
        for (int i = threadIdx.x; i < rows * CH; i += 256) {
            const int r = i / CH, ch = i % CH;
            const bool in = r0 + r < lim;
            const uint16_t* src = qkv16 + (long)(start + (in ? r0 + r : 0)) * ld + col + ch * 8;
            cp_async16(dst + r * LD + ch * 8, src, in ? 16u : 0u);
        }
    };
    stage(Qs, 128, q0, n, h * DH);
    stage(Kt(0), 64, kbeg, kend, d + h * DH);
    stage(Vt(0), 64, kbeg, kend, 2 * d + h * DH);
    cp_async_commit();
    float o[DH / 8][4] = {};
    float la[4] = {0.f, 0.f, 0.f, 0.f};   // row sums: the ones-MMA accumulator (every column its row's sum)
    float nr[4] = {0.f, 0.f, 0.f, 0.f};   // negated references of rows g (0, 1) and g + 8 (2, 3)
    uint32_t qa[DH / 16][4];
    int buf = 0;
    for (int kb = kbeg; kb < kend; kb += 64, buf ^= 1) {
        if (kb + 64 < kend) {
            stage(Kt(buf ^ 1), 64, kb + 64, kend, d + h * DH);
            stage(Vt(buf ^ 1), 64, kb + 64, kend, 2 * d + h * DH);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        if (kb == kbeg) {
#pragma unroll
            for (int kk = 0; kk < DH / 16; ++kk) load_a<LD>(Qs, warp * 16, kk * 16, qa[kk]);
        }
        // S - ref (16 rows x 64 keys, 8 n-tiles)
        float s[8][4];
        const uint16_t* kt = Kt(buf);
#pragma unroll
        for (int kk = 0; kk < DH / 16; ++kk)
#pragma unroll
            for (int np = 0; np < 4; ++np) {
                uint32_t b[4];
                load_b_nk<LD>(kt, np * 16, kk * 16, b);
                mma16816_c<F16>(s[2 * np], qa[kk], b[0], b[1], kk == 0 ? nr : s[2 * np]);
                mma16816_c<F16>(s[2 * np + 1], qa[kk], b[2], b[3], kk == 0 ? nr : s[2 * np + 1]);
            }
        if (kb + 64 > kend) {   // the event's last keys: mask the tile's tail
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (kb + j * 8 + 2 * c + (u & 1) >= kend) s[j][u] = -INFINITY;
        }
        // the tile's row maxima of S - ref; raise the references where needed
        float mr[2] = {-INFINITY, -INFINITY};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            mr[0] = fmaxf(mr[0], fmaxf(s[j][0], s[j][1]));
            mr[1] = fmaxf(mr[1], fmaxf(s[j][2], s[j][3]));
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            mr[r] = fmaxf(mr[r], __shfl_xor_sync(0xffffffffu, mr[r], 1));
            mr[r] = fmaxf(mr[r], __shfl_xor_sync(0xffffffffu, mr[r], 2));
        }
        const bool first = kb == kbeg;
        if (__any_sync(0xffffffffu, first || mr[0] > kRaise || mr[1] > kRaise)) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float dr = first ? mr[r] : fmaxf(mr[r], 0.f);
                const float al = first ? 1.f : ex2_approx(-dr);
                nr[2 * r] -= dr;
                nr[2 * r + 1] -= dr;
                la[2 * r] *= al;
                la[2 * r + 1] *= al;
#pragma unroll
                for (int j = 0; j < DH / 8; ++j) {
                    o[j][2 * r] *= al;
                    o[j][2 * r + 1] *= al;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    s[j][2 * r] -= dr;
                    s[j][2 * r + 1] -= dr;
                }
            }
        }
        // P = 2^(S - ref) as the A fragments of PV (16 keys per K-step), the row sums from
        // the same P
        const uint16_t* vt = Vt(buf);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t pa[4];
            pa[0] = exp2_pair<F16>(s[2 * kk][0], s[2 * kk][1]);
            pa[1] = exp2_pair<F16>(s[2 * kk][2], s[2 * kk][3]);
            pa[2] = exp2_pair<F16>(s[2 * kk + 1][0], s[2 * kk + 1][1]);
            pa[3] = exp2_pair<F16>(s[2 * kk + 1][2], s[2 * kk + 1][3]);
            mma16816<F16>(la, pa, ONE2, ONE2);
#pragma unroll
            for (int dp = 0; dp < DH / 16; ++dp) {
                uint32_t b[4];
                load_b_kn<LD>(vt, kk * 16, dp * 16, b);
                mma16816<F16>(o[2 * dp], pa, b[0], b[1]);
                mma16816<F16>(o[2 * dp + 1], pa, b[2], b[3]);
            }
        }
        __syncthreads();   // every warp is done with this buffer before it is refilled
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int row = q0 + warp * 16 + g + 8 * r;
        if (row >= n) continue;
        const float inv = 1.f / la[2 * r];
        uint32_t* orow = reinterpret_cast<uint32_t*>(o16 + (long)(start + row) * ldo16 + h * DH);
#pragma unroll
        for (int j = 0; j < DH / 8; ++j) orow[(j * 8 + 2 * c) / 2] = pack_f16x2(o[j][2 * r] * inv, o[j][2 * r + 1] * inv);
    }
}

// Generic-width attention with the PV products and the row sums on tcgen05 (heads of 16
// or 32, a multiple of four heads): one CTA per (event, 128 query rows, four heads).  The
// 16 consumer warps (warp 4 hl + rb: head hl of the group, query rows 32 rb .. 32 rb + 31,
// tensor-memory lanes of the same quarter) stage Q, K and V with asynchronous copies,
// compute S - ref with m16n8k16 MMAs (Q pre-scaled, the negated references as the
// accumulator input), take P = 2^(S - ref) with packed exponentials and store it into
// tensor memory with tcgen05.st.16x128b (the MMA A-fragment layout); each also transposes
// its 16 keys of the head's V tile into a K-major, 128-byte-swizzled V^T tile.  One MMA
// warp per head accumulates O_h += P_h V_h and l_h += P_h 1 per 64-key tile (tcgen05, P the
// tensor-memory A operand, M 128, K 64); O and l stay in tensor memory until the item
// ends.  P and V^T are double-buffered (tile j is written while the MMAs of tile j - 1
// run).  References: the first tile's row maxima (its QK^T is computed twice), then raised
// only when a 16-key step exceeds a row's reference by more than kRaise; such a raise
// (rare) rescales the tile's P already stored and, once the previous tile's MMAs are
// complete, the row's O and l in tensor memory.  On the legacy pipe only QK^T remains,
// which binds this kernel at heads of 32 when PV runs there too.  Every wait is bounded.
constexpr int WP_HG = 4;                           // heads per CTA
constexpr int WP_THREADS = 16 * 32 + WP_HG * 32;   // 16 consumer warps, 4 MMA warps
template <int DH>
struct WpLayout {
    static constexpr int LDQ = WP_HG * DH + 8;                        // staged row stride (elements)
    static constexpr uint32_t Q = 0;                                  // [128][LDQ]
    static constexpr uint32_t K = Q + 128 * LDQ * 2;                  // [2][64][LDQ]
    static constexpr uint32_t V = K + 2 * 64 * LDQ * 2;               // [2][64][LDQ], row-major
    static constexpr uint32_t VT = (V + 2 * 64 * LDQ * 2 + 1023) / 1024 * 1024;   // [2][HG][DH][128 B]
    static constexpr uint32_t VTB = WP_HG * DH * 128;                 // one V^T buffer
    static constexpr uint32_t ONES = VT + 2 * VTB;                    // [16][128 B]
    static constexpr uint32_t BAR = ONES + 2048;                      // barriers and flags
    static constexpr uint32_t SMEM = BAR + 256 + 1024;
    static constexpr int TCOLS = 128;   // tensor-memory columns per head: P 2 x 32, O DH, l 16 (aligned)
};

// named barrier `id` of n threads that returns whether any thread passed pred = true
__device__ __forceinline__ bool bar_any(int id, int n, bool pred) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r)
                 : "r"((uint32_t)pred), "r"(id), "r"(n)
                 : "memory");
    return r != 0;
}

template <int DH, bool F16>
__global__ void __launch_bounds__(WP_THREADS, 1)
    k_attn_wide_pt(const uint16_t* __restrict__ qkv16, uint16_t* __restrict__ o16, int ldo16,
                   const int32_t* __restrict__ cu, int d, int window, unsigned* status, uint64_t wait_ns) {
    using LY = WpLayout<DH>;
    constexpr int LDQ = LY::LDQ, CH = WP_HG * DH / 8;   // 16-byte chunks per staged row
    constexpr float kRaise = 4.f;
    static_assert(WP_HG * LY::TCOLS <= 512 && 64 + DH + 16 <= LY::TCOLS, "tensor-memory columns");
    extern __shared__ uint8_t wp_raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)wp_raw + 1023) & ~(uintptr_t)1023);
    uint16_t* Qs = (uint16_t*)(sm + LY::Q);
    auto Ks = [&](int b) { return (uint16_t*)(sm + LY::K) + b * 64 * LDQ; };
    auto Vs = [&](int b) { return (uint16_t*)(sm + LY::V) + b * 64 * LDQ; };
    uint8_t* VT = sm + LY::VT;
    uint64_t* bars = (uint64_t*)(sm + LY::BAR);
    uint64_t* p_full = bars;              // [head][buffer]: one arrival per warp of the head
    uint64_t* p_free = bars + 8;          // [head][buffer]: MMA commit
    uint64_t* drain = bars + 16;          // [head]: the MMA warp's exit
    int* abort_flag = (int*)(bars + 20);
    uint32_t* tmem_hold = (uint32_t*)(abort_flag + 1);
    volatile int* ab = abort_flag;
    const int e = blockIdx.z, hg = blockIdx.y;
    const int start = cu[e], n = cu[e + 1] - start, q0 = blockIdx.x * 128;
    if (q0 >= n) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long ld = 3L * d;
    int kbeg = 0, kend = n;
    if (window > 0) {
        const int y = q0 / 128;
        kbeg = max(0, (y - window) * 128);
        kend = min(n, (y + window + 1) * 128);
    }
    const int nk = (kend - kbeg + 63) / 64;
    if (tid == 0) {
        for (int i = 0; i < 8; ++i) { mbar_init(&p_full[i], 4); mbar_init(&p_free[i], 1); }
        for (int i = 0; i < WP_HG; ++i) mbar_init(&drain[i], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    {   // the B operand of the row sums: 16 rows x 64 keys of ones
        const uint32_t one2 = F16 ? 0x3C003C00u : 0x3F803F80u;
        for (int i = tid; i < 512; i += WP_THREADS) ((uint32_t*)(sm + LY::ONES))[i] = one2;
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
    auto colP = [](int hl, int b) { return (uint32_t)(hl * LY::TCOLS + 32 * b); };
    auto colO = [](int hl) { return (uint32_t)(hl * LY::TCOLS + 64); };
    auto vt_buf = [&](int b, int hl) { return VT + b * LY::VTB + hl * DH * 128; };

    if (warp >= 16) {
        // ------------------------------------------------ PV and row-sum MMAs of head hl
        const int hl = warp - 16;
        if (lane == 0) {
            const uint32_t IPV = idesc_f16(128, DH, F16 ? 0u : 1u), IL = idesc_f16(128, 16, F16 ? 0u : 1u);
            const uint32_t onesa = smem_u32(sm + LY::ONES);
            for (int j = 0; j < nk; ++j) {
                const int b = j & 1;
                if (!mbar_wait(&p_full[2 * hl + b], (j >> 1) & 1, ab, status, ST_TIMEOUT_ATTN, wait_ns)) break;
                tc_fence_after();
                const uint32_t pa = tbase + colP(hl, b), od = tbase + colO(hl);
                const uint32_t va = smem_u32(vt_buf(b, hl));
#pragma unroll
                for (int kc = 0; kc < 4; ++kc) {
                    const uint32_t acc = (j > 0 || kc > 0) ? 1u : 0u;
                    mma_f16_ts(od, pa + 8 * kc, sdesc_sw128(va + kc * 32), IPV, acc);
                    mma_f16_ts(od + DH, pa + 8 * kc, sdesc_sw128(onesa + kc * 32), IL, acc);
                }
                mma_commit(&p_free[2 * hl + b]);
            }
            mma_commit(&drain[hl]);
            mbar_drain(&drain[hl], 0, wait_ns);
        }
    } else {
        // ------------------------------------------------ consumer warp: head hl, rows 32 rb ..
        const int hl = warp >> 2, rb = warp & 3;
        const int c = lane & 3;
        const uint32_t tlane = tbase + ((uint32_t)(32 * rb) << 16);
        // rows r0 .. r0 + rows - 1 of the group's columns col0 .. (rows at or beyond lim are zero)
        auto stage = [&](uint16_t* dst, int rows, int r0, int lim, int col0) {
            for (int i = tid; i < rows * CH; i += 512) {
                const int r = i / CH, ch = i % CH;
                const bool in = r0 + r < lim;
                const uint16_t* src = qkv16 + (long)(start + (in ? r0 + r : 0)) * ld + col0 + ch * 8;
                cp_async16(dst + r * LDQ + ch * 8, src, in ? 16u : 0u);
            }
        };
        const int gcol = hg * WP_HG * DH;
        stage(Qs, 128, q0, n, gcol);
        stage(Ks(0), 64, kbeg, kend, d + gcol);
        stage(Vs(0), 64, kbeg, kend, 2 * d + gcol);
        cp_async_commit();
        float nr[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int u = 0; u < 4; ++u) nr[mt][u] = 0.f;
        uint32_t qa[2][DH / 16][4];
        bool ok = true;
        // S - ref of keys 16 q .. 16 q + 15 of the staged tile kt (two 8-key column tiles)
        auto qk = [&](const uint16_t* kt, int q, float (&s)[2][2][4]) {
#pragma unroll
            for (int kk = 0; kk < DH / 16; ++kk) {
                uint32_t b[4];
                load_b_nk<LDQ>(kt, 16 * q, hl * DH + 16 * kk, b);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma16816_c<F16>(s[mt][0], qa[mt][kk], b[0], b[1], kk == 0 ? nr[mt] : s[mt][0]);
                    mma16816_c<F16>(s[mt][1], qa[mt][kk], b[2], b[3], kk == 0 ? nr[mt] : s[mt][1]);
                }
            }
        };
        auto mask = [&](int q, int kvalid, float (&s)[2][2][4]) {
            if (16 * (q + 1) > kvalid) {
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (16 * q + 8 * nt + 2 * c + (u & 1) >= kvalid) s[mt][nt][u] = -INFINITY;
            }
        };
        // row maxima of a step (rows g, g + 8 of each 16-row block), over the quad
        auto rowmax = [&](const float (&s)[2][2][4], float (&mx)[2][2]) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int hr = 0; hr < 2; ++hr) {
                    float m = fmaxf(fmaxf(s[mt][0][2 * hr], s[mt][0][2 * hr + 1]),
                                    fmaxf(s[mt][1][2 * hr], s[mt][1][2 * hr + 1]));
                    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
                    mx[mt][hr] = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
                }
        };
        auto pack_p = [&](const float (&s)[2][2][4], int mt, uint32_t (&pa)[4]) {
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {
                pa[hr] = exp2_pair<F16>(s[mt][0][2 * hr], s[mt][0][2 * hr + 1]);
                pa[2 + hr] = exp2_pair<F16>(s[mt][1][2 * hr], s[mt][1][2 * hr + 1]);
            }
        };
        for (int j = 0; j < nk && ok; ++j) {
            const int kb = kbeg + 64 * j, b = j & 1, kvalid = kend - kb;
            if (j + 1 < nk) {
                stage(Ks(b ^ 1), 64, kb + 64, kend, d + gcol);
                stage(Vs(b ^ 1), 64, kb + 64, kend, 2 * d + gcol);
            }
            cp_async_commit();
            cp_async_wait<1>();
            if (bar_any(1, 512, !ok)) break;   // a failed wait anywhere: every consumer leaves
            if (j == 0) {
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int kk = 0; kk < DH / 16; ++kk) load_a<LDQ>(Qs, 32 * rb + 16 * mt, hl * DH + 16 * kk, qa[mt][kk]);
            }
            // P and V^T of buffer b: the MMAs of tile j - 2 are complete
            if (j >= 2) {
                ok = __all_sync(0xffffffffu, mbar_wait(&p_free[2 * hl + b], ((j >> 1) - 1) & 1, ab, status,
                                                        ST_TIMEOUT_ATTN, wait_ns));
                tc_fence_after();
            }
            if (ok) {
            // V^T of this warp's 16 keys: transposed 8 x 8 blocks (keys 16 rb + 8 kb2, channels
            // 8 cb) land as pairs of keys of one channel, stored into the swizzled K-major tile
            {
                const uint16_t* vs = Vs(b);
                uint8_t* vt = vt_buf(b, hl);
#pragma unroll
                for (int blk = 0; blk < DH / 8 * 2; blk += 4) {
                    const int mi = blk + (lane >> 3);               // this lane's matrix
                    const int kb2 = mi & 1, cb = mi >> 1;
                    const uint16_t* src = vs + (16 * rb + 8 * kb2 + (lane & 7)) * LDQ + hl * DH + 8 * cb;
                    uint32_t r[4];
                    ldsm_x4_t(smem_u32(src), r[0], r[1], r[2], r[3]);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int m2 = blk + i, kb3 = m2 & 1, cb3 = m2 >> 1;
                        const int ch = 8 * cb3 + (lane >> 2);             // channel = V^T row
                        const int chunk = 2 * rb + kb3;                    // 16-byte chunk of 8 keys
                        *(uint32_t*)(vt + ch * 128 + ((chunk ^ (ch & 7)) << 4) + 4 * (lane & 3)) = r[i];
                    }
                }
            }
            const uint16_t* kt = Ks(b);
            const uint32_t pcol = tlane + colP(hl, b);
            if (j == 0) {
                // the first tile sets the references to its row maxima
                float mx[2][2] = {{-INFINITY, -INFINITY}, {-INFINITY, -INFINITY}};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (16 * q >= kvalid) break;
                    float s[2][2][4], m2[2][2];
                    qk(kt, q, s);
                    mask(q, kvalid, s);
                    rowmax(s, m2);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int hr = 0; hr < 2; ++hr) mx[mt][hr] = fmaxf(mx[mt][hr], m2[mt][hr]);
                }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int hr = 0; hr < 2; ++hr) {
                        nr[mt][2 * hr] = -mx[mt][hr];
                        nr[mt][2 * hr + 1] = -mx[mt][hr];
                    }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float s[2][2][4];
                if (16 * q < kvalid) {
                    qk(kt, q, s);
                    mask(q, kvalid, s);
                } else {
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                            for (int u = 0; u < 4; ++u) s[mt][nt][u] = -INFINITY;
                }
                if (j > 0 && 16 * q < kvalid) {
                    // a raise is needed when any score of the warp exceeds its reference by
                    // more than kRaise: this thread's maximum and one vote; the rows' maxima
                    // only then
                    float tm = -INFINITY;
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 2; ++nt)
                            tm = fmaxf(tm, fmaxf(fmaxf(s[mt][nt][0], s[mt][nt][1]), fmaxf(s[mt][nt][2], s[mt][nt][3])));
                    if (__any_sync(0xffffffffu, tm > kRaise)) {
                        float mx[2][2];
                        rowmax(s, mx);
                        // raise the rows' references by dr >= 0; P of this tile's earlier
                        // steps, O and l (after the previous tile's MMAs) scale by 2^-dr
                        float al[2][2];
#pragma unroll
                        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                            for (int hr = 0; hr < 2; ++hr) {
                                const float dr = fmaxf(mx[mt][hr], 0.f);
                                al[mt][hr] = ex2_approx(-dr);
                                nr[mt][2 * hr] -= dr;
                                nr[mt][2 * hr + 1] -= dr;
#pragma unroll
                                for (int nt = 0; nt < 2; ++nt) {
                                    s[mt][nt][2 * hr] -= dr;
                                    s[mt][nt][2 * hr + 1] -= dr;
                                }
                            }
                        for (int q2 = 0; q2 < q; ++q2)
#pragma unroll
                            for (int mt = 0; mt < 2; ++mt) {
                                const uint32_t a = pcol + ((uint32_t)(16 * mt) << 16) + 8 * q2;
                                uint32_t u[4];
                                tmem_ld16x128b_x2(a, u);
                                tmem_wait_ld();
#pragma unroll
                                for (int i = 0; i < 4; ++i) {
                                    float x0, x1;
                                    unpack2<F16>(u[i], x0, x1);
                                    const float f = al[mt][i & 1];   // registers 0, 2: row g; 1, 3: row g + 8
                                    u[i] = pack2<F16>(x0 * f, x1 * f);
                                }
                                tmem_st16x128b_x2(a, u);
                            }
                        ok = __all_sync(0xffffffffu, mbar_wait(&p_free[2 * hl + (b ^ 1)], ((j - 1) >> 1) & 1, ab,
                                                                status, ST_TIMEOUT_ATTN, wait_ns));
                        if (!ok) break;
                        tc_fence_after();
                        // the factor of row `lane` (block lane / 16, half (lane / 8) & 1,
                        // fragment row lane & 7) is held by fragment lane 4 (lane & 7)
                        const int src = 4 * (lane & 7);
                        const float f00 = __shfl_sync(0xffffffffu, al[0][0], src);
                        const float f01 = __shfl_sync(0xffffffffu, al[0][1], src);
                        const float f10 = __shfl_sync(0xffffffffu, al[1][0], src);
                        const float f11 = __shfl_sync(0xffffffffu, al[1][1], src);
                        const float f = lane < 16 ? (lane < 8 ? f00 : f01) : (lane < 24 ? f10 : f11);
                        // O and l, 16 columns at a time
#pragma unroll 1
                        for (int c16 = 0; c16 < DH + 16; c16 += 16) {
                            float ol[16];
                            tmem_ld16(tlane + colO(hl) + c16, ol);
                            tmem_wait_ld();
                            uint32_t uo[16];
#pragma unroll
                            for (int i = 0; i < 16; ++i) uo[i] = __float_as_uint(ol[i] * f);
                            tmem_st16(tlane + colO(hl) + c16, uo);
                        }
                    }
                }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    uint32_t pa[4];
                    pack_p(s, mt, pa);
                    tmem_st16x128b_x2(pcol + ((uint32_t)(16 * mt) << 16) + 8 * q, pa);
                }
            }
            }
            if (ok) {   // publish P and V^T of tile j to the head's MMA warp
                fence_proxy_async_smem();
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&p_full[2 * hl + b]);
            }
            // every consumer is done with K(j), V(j) before they are refilled
            if (bar_any(1, 512, !ok)) break;
        }
        if (ok) {
            // the item's output: O / l of row `lane` of this warp
            const int jl = nk - 1;
            ok = mbar_wait(&p_free[2 * hl + (jl & 1)], (jl >> 1) & 1, ab, status, ST_TIMEOUT_ATTN, wait_ns);
            if (__all_sync(0xffffffffu, ok)) {
                tc_fence_after();
                float ol[DH + 16];
                if constexpr (DH == 32) {
                    tmem_ld32(tlane + colO(hl), ol);
                    tmem_ld16(tlane + colO(hl) + 32, ol + 32);
                } else {
                    tmem_ld32(tlane + colO(hl), ol);
                }
                tmem_wait_ld();
                const int row = q0 + 32 * rb + lane;
                if (row < n) {
                    const float inv = 1.f / ol[DH];
                    uint32_t* orow = reinterpret_cast<uint32_t*>(o16 + (long)(start + row) * ldo16 + hg * WP_HG * DH + hl * DH);
#pragma unroll
                    for (int i = 0; i < DH / 2; ++i) orow[i] = pack_f16x2(ol[2 * i] * inv, ol[2 * i + 1] * inv);
                }
            }
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

template <bool F16>
bool attn_tc_launch(int which, const float* qkv, const float* dO, float* out, float* lse, const float* D,
                    float* dqkv, const int32_t* cu, int n_events, int max_n, int d, int heads, cudaStream_t st,
                    int window) {
    const int dh = d / heads;
    const float scale = 1.f / sqrtf((float)dh);
    dim3 grid((max_n + 63) / 64, heads, n_events);
#define MLPF_ATTN_TC(DH)                                                                              \
    if (which == 0)                                                                                   \
        k_attn_fwd_tc<DH, F16><<<grid, 128, 0, st>>>(qkv, out, lse, cu, d, scale, window);            \
    else {                                                                                            \
        k_attn_dq_tc<DH, F16><<<grid, 128, 0, st>>>(qkv, dO, lse, D, dqkv, cu, d, scale);             \
        k_attn_dkv_tc<DH, F16><<<grid, 128, 0, st>>>(qkv, dO, lse, D, dqkv, cu, d, scale);            \
    }
    if (dh == 16) {
        MLPF_ATTN_TC(16)
    } else if (dh == 32) {
        MLPF_ATTN_TC(32)
    } else if (dh == 64) {
        MLPF_ATTN_TC(64)
    } else {
        return false;
    }
#undef MLPF_ATTN_TC
    return true;
}

}  // namespace

bool attn_train_fwd_tc(int f16, const float* qkv, float* out, float* lse, const int32_t* cu, int n_events, int max_n,
                       int d, int heads, cudaStream_t st, int window) {
    if (n_events <= 0 || max_n <= 0) return true;
    return f16 ? attn_tc_launch<true>(0, qkv, nullptr, out, lse, nullptr, nullptr, cu, n_events, max_n, d, heads, st,
                                      window)
               : attn_tc_launch<false>(0, qkv, nullptr, out, lse, nullptr, nullptr, cu, n_events, max_n, d, heads, st,
                                       window);
}

static constexpr int attn16_smem(int dh) { return 384 * (dh + 8) * 2; }

void attn_fwd16_prepare() {
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaFuncSetAttribute(k_attn_fwd16<64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, attn16_smem(64));
    cudaFuncSetAttribute(k_attn_fwd16<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, attn16_smem(64));
    cudaFuncSetAttribute(k_attn_wide_pt<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, WpLayout<16>::SMEM);
    cudaFuncSetAttribute(k_attn_wide_pt<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, WpLayout<16>::SMEM);
    cudaFuncSetAttribute(k_attn_wide_pt<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, WpLayout<32>::SMEM);
    cudaFuncSetAttribute(k_attn_wide_pt<32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, WpLayout<32>::SMEM);
    done[dev] = true;
}

bool attn_fwd16(int f16, const uint16_t* qkv16, uint16_t* o16, int ldo16, const int32_t* cu, int n_events, int max_n,
                int d, int heads, cudaStream_t st, int window, int kernel, unsigned* status, uint64_t wait_ns) {
    if (n_events <= 0 || max_n <= 0) return true;
    const int dh = d / heads;
    if (kernel == 1 && (dh == 16 || dh == 32) && heads % WP_HG == 0) {
        // PV and row sums on tcgen05
        dim3 gp((max_n + 127) / 128, heads / WP_HG, n_events);
#define MLPF_ATTN_PT(DH)                                                                                            \
    if (f16)                                                                                                        \
        k_attn_wide_pt<DH, true><<<gp, WP_THREADS, WpLayout<DH>::SMEM, st>>>(qkv16, o16, ldo16, cu, d, window, status, \
                                                                            wait_ns);                              \
    else                                                                                                            \
        k_attn_wide_pt<DH, false><<<gp, WP_THREADS, WpLayout<DH>::SMEM, st>>>(qkv16, o16, ldo16, cu, d, window,       \
                                                                             status, wait_ns);
        if (dh == 16) {
            MLPF_ATTN_PT(16)
        } else {
            MLPF_ATTN_PT(32)
        }
#undef MLPF_ATTN_PT
        return true;
    }
    dim3 grid((max_n + 127) / 128, heads, n_events);
#define MLPF_ATTN16(DH)                                                                               \
    if (f16)                                                                                          \
        k_attn_fwd16<DH, true><<<grid, 256, attn16_smem(DH), st>>>(qkv16, o16, ldo16, cu, d, window); \
    else                                                                                              \
        k_attn_fwd16<DH, false><<<grid, 256, attn16_smem(DH), st>>>(qkv16, o16, ldo16, cu, d, window);
    if (dh == 16) {
        MLPF_ATTN16(16)
    } else if (dh == 32) {
        MLPF_ATTN16(32)
    } else if (dh == 64) {
        MLPF_ATTN16(64)
    } else {
        return false;
    }
#undef MLPF_ATTN16
    return true;
}

bool attn_train_bwd_tc(int f16, const float* qkv, const float* dO, const float* lse, const float* D, float* dqkv,
                       const int32_t* cu, int n_events, int max_n, int d, int heads, cudaStream_t st) {
    if (n_events <= 0 || max_n <= 0) return true;
    return f16 ? attn_tc_launch<true>(1, qkv, dO, nullptr, const_cast<float*>(lse), D, dqkv, cu, n_events, max_n, d,
                                      heads, st, 0)
               : attn_tc_launch<false>(1, qkv, dO, nullptr, const_cast<float*>(lse), D, dqkv, cu, n_events, max_n, d,
                                       heads, st, 0);
}

}  // namespace mlpf
