// 16-bit tensor-core GEMM with a fused FP32 epilogue, for the linear layers of the training
// step and of the generic-width forward (Sec. 5.3: every layer of the model is a dense map
// y = x W^T + b; its backward needs dX = dY W and dW = dY^T X).  Each 128 x BN tile of
//     C (op)= act(A[M, Kp] B[N, Kp]^T + bias) + R
// with A and B row-major 16-bit (BF16 or FP16) in global memory, Kp a multiple of 64:
// TMA copies 128 x 64 and BN x 64 boxes (128-byte swizzle) into a ring of shared stages,
// one thread issues tcgen05.mma (M = 128, N = BN, K = 16 per instruction) into a
// BN-column FP32 accumulator in tensor memory, and four warps read it back with
// tcgen05.ld (thread = row) for the epilogue.  Split-K adds partial tiles with atomics
// (weight gradients, whose reduction runs over all elements of the batch).
// Every wait is bounded: on a timeout the CTA sets the status word, lets its copies and
// MMAs in flight land, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cuda_fp16.h>

#include "internal.h"
#include "ptx.cuh"

namespace mlpf {
namespace {

constexpr int TG_BM = 128;   // tile rows (M of one MMA)
constexpr int TG_BK = 64;    // K elements per stage: one 128-byte swizzle atom of 16-bit values

struct TgArgs {
    int M, N, Kp, kchunk;
    float* C;
    long ldc;
    uint16_t* C16;      // optional 16-bit copy of the result (mode 0 only)
    long ldc16;
    const float* bias;  // [N] or null (split 0 only)
    const float* R;     // residual [M, ldr] or null (split 0 only)
    long ldr;
    int mode;           // 0: C = ..., 1: C += ..., 2: C += ... with atomics (split-K)
    int act;            // -1 none, 0 GELU (erf), 1 ReLU: applied to (acc + bias), before R
    int f16;            // operand format: 1 FP16, 0 BF16
    int c16_f16;        // C16 format: 1 FP16, 0 BF16
    int c16_cols;       // C16 columns written (>= N: the padding columns beyond N get zeros)
    unsigned* status;
    uint64_t wait_ns;
};

// GELU x Phi(x) with erf from Abramowitz & Stegun 7.1.26 (|error of erf| <= 1.5e-7):
// erf(z) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-z^2), t = 1 / (1 + p z), z >= 0
__device__ __forceinline__ float gelu_as(float v) {
    const float z = fabsf(v) * 0.70710678118654752f;
    const float t = __fdividef(1.f, fmaf(0.3275911f, z, 1.f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                 0.254829592f);
    const float erf_abs = fmaf(-poly, ex2_approx(-z * z * 1.4426950408889634f), 1.f);
    return 0.5f * v * (1.f + copysignf(erf_abs, v));
}

__device__ __forceinline__ float tg_act(float v, int act) {
    if (act == 1) return fmaxf(v, 0.f);
    if (act == 0) return gelu_as(v);
    return v;
}

// TWO: the weight operand is two-term, B = [B_hi | B_lo] of 2 Kp columns; each K step
// multiplies the A tile by both terms into the same accumulator.
template <int BN, int ST, bool TWO = false>
struct TgLayout {
    static constexpr int A_BYTES = TG_BM * TG_BK * 2;
    static constexpr int B_BYTES = BN * TG_BK * 2;
    static constexpr int STAGE = A_BYTES + (TWO ? 2 : 1) * B_BYTES;   // multiple of 1024
    // full[ST], empty[ST], acc_full[2], acc_empty[2], drain
    static constexpr int OFF_BAR = ST * STAGE;
    static constexpr int OFF_MISC = OFF_BAR + (2 * ST + 5) * 8;
    static constexpr int BYTES = OFF_MISC + 64 + 1024;        // + alignment slack
    static constexpr uint32_t TMEM_COLS = 2 * BN;              // two accumulators
};

// The epilogue of one 32-column chunk of one row: bias, activation, residual, FP32 and
// 16-bit stores.  r: the row, nb: the chunk's first column, lead: the split that adds
// bias and residual.
__device__ __forceinline__ void red_add_v4(float* p, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ void tg_store_chunk(const TgArgs& g, float* v, int r, int nb, bool lead) {
    const int nn = max(0, min(32, g.N - nb));          // columns of the result
    const int n16 = max(0, min(32, g.c16_cols - nb));   // columns of the 16-bit copy (zero beyond N)
    if (nn == 32 && (nb & 3) == 0) {   // full chunk: 16-byte loads of bias and residual
        if (lead && g.bias && ((uintptr_t)g.bias & 15) == 0) {
            const float4* b4 = reinterpret_cast<const float4*>(g.bias + nb);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 b = __ldg(b4 + q);
                v[4 * q] += b.x;
                v[4 * q + 1] += b.y;
                v[4 * q + 2] += b.z;
                v[4 * q + 3] += b.w;
            }
        } else if (lead && g.bias) {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] += g.bias[nb + j];
        }
        if (g.act >= 0)
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = tg_act(v[j], g.act);
        if (lead && g.R && ((g.ldr & 3) == 0) && ((uintptr_t)g.R & 15) == 0) {
            const float4* r4 = reinterpret_cast<const float4*>(g.R + (long)r * g.ldr + nb);
            float4 rr[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) rr[q] = r4[q];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                v[4 * q] += rr[q].x;
                v[4 * q + 1] += rr[q].y;
                v[4 * q + 2] += rr[q].z;
                v[4 * q + 3] += rr[q].w;
            }
        } else if (lead && g.R) {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] += g.R[(long)r * g.ldr + nb + j];
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j >= nn) break;
            float y = v[j];
            if (lead && g.bias) y += g.bias[nb + j];
            y = tg_act(y, g.act);
            if (lead && g.R) y += g.R[(long)r * g.ldr + nb + j];
            v[j] = y;
        }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j)
        if (j >= nn) v[j] = 0.f;
    float* crow = g.C && nn > 0 ? g.C + (long)r * g.ldc + nb : nullptr;
    if (crow) {
        if (g.mode == 2 && nn == 32 && ((g.ldc | nb) & 3) == 0 && ((uintptr_t)g.C & 15) == 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                red_add_v4(crow + 4 * q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
        } else if (g.mode == 2) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (j < nn) atomicAdd(crow + j, v[j]);
        } else if (nn == 32 && ((g.ldc | nb) & 3) == 0 && ((uintptr_t)g.C & 15) == 0) {
            float4* c4 = (float4*)crow;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float4 o = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                if (g.mode == 1) {
                    const float4 p = c4[q];
                    o.x += p.x;
                    o.y += p.y;
                    o.z += p.z;
                    o.w += p.w;
                }
                c4[q] = o;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (j < nn) crow[j] = g.mode == 1 ? crow[j] + v[j] : v[j];
        }
    }
    if (g.C16 && n16 > 0) {
        uint16_t* hrow = g.C16 + (long)r * g.ldc16 + nb;
        if (n16 == 32 && ((g.ldc16 | nb) & 7) == 0 && ((uintptr_t)g.C16 & 15) == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint4 p;
                p.x = g.c16_f16 ? pack_f16x2(v[8 * q], v[8 * q + 1]) : pack_bf16x2(v[8 * q], v[8 * q + 1]);
                p.y = g.c16_f16 ? pack_f16x2(v[8 * q + 2], v[8 * q + 3]) : pack_bf16x2(v[8 * q + 2], v[8 * q + 3]);
                p.z = g.c16_f16 ? pack_f16x2(v[8 * q + 4], v[8 * q + 5]) : pack_bf16x2(v[8 * q + 4], v[8 * q + 5]);
                p.w = g.c16_f16 ? pack_f16x2(v[8 * q + 6], v[8 * q + 7]) : pack_bf16x2(v[8 * q + 6], v[8 * q + 7]);
                reinterpret_cast<uint4*>(hrow)[q] = p;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (j >= n16) break;
                const uint32_t p = g.c16_f16 ? pack_f16x2(v[j], 0.f) : pack_bf16x2(v[j], 0.f);
                hrow[j] = (uint16_t)(p & 0xffffu);
            }
        }
    }
}

// Persistent, warp-specialised: two CTAs per SM walk the tiles (n fastest, then m, then
// the K split) with stride gridDim.x.  Warp 0 (one lane) streams A and B boxes through
// an ST-deep ring of shared stages; warp 1 (one lane) issues the MMAs of a tile into one
// of two tensor-memory accumulators; warps 2-9 drain the other accumulator (the previous
// tile) through the epilogue meanwhile, warp w reading lanes 32 (w mod 4) .. + 31 and every
// other 32-column chunk (two warps per lane quarter).
template <int BN, int ST, bool TWO>
__global__ void __launch_bounds__(320, 2) k_gemm_tc(const __grid_constant__ CUtensorMap map_a,
                                                    const __grid_constant__ CUtensorMap map_b, TgArgs g,
                                                    int tiles_m, int tiles_n, int splits) {
    using L = TgLayout<BN, ST, TWO>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + L::OFF_BAR);
    uint64_t* empty = full + ST;
    uint64_t* acc_full = empty + ST;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_slot = (uint32_t*)(smem + L::OFF_MISC);
    volatile int* abort_flag = (volatile int*)(smem + L::OFF_MISC + 4);
    int* issued_s = (int*)(smem + L::OFF_MISC + 8);
    int* consumed_s = (int*)(smem + L::OFF_MISC + 12);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int per_split = tiles_m * tiles_n, total = per_split * splits;

    if (tid == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 8);   // one arrival per epilogue warp
        }
        mbar_init(drain, 1);
        fence_mbar_init();
        *abort_flag = 0;
        *issued_s = 0;
        *consumed_s = 0;
        tma_prefetch_map(&map_a);
        tma_prefetch_map(&map_b);
    }
    if (warp == 2) {
        tmem_alloc(tmem_slot, L::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    auto k_range = [&](int t, int& kbeg) {
        kbeg = (t / per_split) * g.kchunk;
        const int kend = min(g.Kp, kbeg + g.kchunk);
        return kend > kbeg ? (kend - kbeg) / TG_BK : 0;
    };

    if (warp == 0) {
        if (lane == 0) {   // TMA producer
            int it = 0;
            bool go = true;
            for (int t = blockIdx.x; t < total && go; t += gridDim.x) {
                const int rem = t % per_split, m0 = (rem / tiles_n) * TG_BM, n0 = (rem % tiles_n) * BN;
                int kbeg;
                const int nk = k_range(t, kbeg);
                for (int i = 0; i < nk; ++i, ++it) {
                    const int s = it % ST;
                    if (it >= ST && !mbar_wait(&empty[s], ((it / ST) - 1) & 1, abort_flag, g.status, ST_TIMEOUT_GEMM,
                                               g.wait_ns)) {
                        go = false;
                        break;
                    }
                    uint8_t* sa = smem + s * L::STAGE;
                    mbar_arrive_expect_tx(&full[s], L::STAGE);
                    tma_load_2d(sa, &map_a, kbeg + i * TG_BK, m0, &full[s]);
                    tma_load_2d(sa + L::A_BYTES, &map_b, kbeg + i * TG_BK, n0, &full[s]);
                    if constexpr (TWO)
                        tma_load_2d(sa + L::A_BYTES + L::B_BYTES, &map_b, g.Kp + kbeg + i * TG_BK, n0, &full[s]);
                }
            }
            *issued_s = it;
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            constexpr uint32_t idesc_bf = idesc_f16(TG_BM, BN, 1), idesc_h = idesc_f16(TG_BM, BN, 0);
            const uint32_t idesc = g.f16 ? idesc_h : idesc_bf;
            int it = 0, j = 0;
            bool go = true;
            for (int t = blockIdx.x; t < total && go; t += gridDim.x, ++j) {
                const int b = j & 1;
                int kbeg;
                const int nk = k_range(t, kbeg);
                if (j >= 2 && !mbar_wait(&acc_empty[b], ((j >> 1) - 1) & 1, abort_flag, g.status, ST_TIMEOUT_GEMM,
                                         g.wait_ns))
                    break;
                tc_fence_after();
                const uint32_t acc = tmem + b * BN;
                for (int i = 0; i < nk; ++i, ++it) {
                    const int s = it % ST;
                    if (!mbar_wait(&full[s], (it / ST) & 1, abort_flag, g.status, ST_TIMEOUT_GEMM, g.wait_ns)) {
                        go = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * L::STAGE), sb = sa + L::A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < TG_BK / 16; ++kk) {
                        mma_f16(acc, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), idesc, (i | kk) != 0);
                        if constexpr (TWO)
                            mma_f16(acc, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + L::B_BYTES + kk * 32), idesc, 1);
                    }
                    mma_commit(&empty[s]);
                }
                if (go) mma_commit(&acc_full[b]);
            }
            *consumed_s = it;
            mma_commit(drain);   // arrives once every MMA issued above has completed
        }
    } else {   // epilogue warps 2..9: two per lane quarter, alternate 32-column chunks
        const int q = warp & 3, half = (warp - 2) >> 2;
        int j = 0;
        for (int t = blockIdx.x; t < total; t += gridDim.x, ++j) {
            const int b = j & 1;
            const int split = t / per_split, rem = t % per_split;
            const int m0 = (rem / tiles_n) * TG_BM, n0 = (rem % tiles_n) * BN;
            int kbeg;
            const int nk = k_range(t, kbeg);
            const bool ok = mbar_wait(&acc_full[b], (j >> 1) & 1, abort_flag, g.status, ST_TIMEOUT_GEMM, g.wait_ns);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const int r = m0 + q * 32 + lane;
#pragma unroll 1
            for (int c = half; c < BN / 32; c += 2) {
                float v[32];
                __syncwarp();
                tmem_ld32(tmem + b * BN + ((uint32_t)(q * 32) << 16) + c * 32, v);
                tmem_wait_ld();
                const int nb = n0 + c * 32;
                if (r < g.M && nk > 0 && nb < max(g.N, g.c16_cols)) tg_store_chunk(g, v, r, nb, split == 0);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
    }
    __syncwarp();
    __syncthreads();
    if (tid == 0) {
        // let what is still in flight land before shared and tensor memory are released
        mbar_drain(drain, 0, g.wait_ns);
        if (*abort_flag)
            for (int i = *consumed_s; i < *issued_s; ++i) mbar_drain(&full[i % ST], (i / ST) & 1, g.wait_ns);
    }
    __syncthreads();
    if (warp == 2) tmem_dealloc(tmem, L::TMEM_COLS);
}

// 32 x 32 tile transpose through shared memory: dst[c, r] = src[r, c] for r < rows, c < cols;
// dst columns rows .. ldd - 1 of each written row are zero.  dst row c0 + c for the source
// column c (a column offset into a wider destination).
__global__ void k_cvt_t(const float* __restrict__ src, long lds, int rows, int cols, uint16_t* __restrict__ dst,
                        long ldd, int f16) {
    __shared__ float tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 256 threads: 8 rows per pass
    for (int i = ty; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + tx;
        tile[i][tx] = (r < rows && c < cols) ? src[(long)r * lds + c] : 0.f;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + tx;
        if (c < cols && r < ldd) {
            const float v = tile[tx][i];
            const uint32_t p = f16 ? pack_f16x2(v, 0.f) : pack_bf16x2(v, 0.f);
            dst[(long)c * ldd + r] = (uint16_t)(p & 0xffffu);
        }
    }
}

// dst[r, c] = src1[r, c] (c < k1), src2[r, c - k1] (k1 <= c < k1 + k2), 0 (up to ldd)
__global__ void k_cvt(const float* __restrict__ s1, long ld1, int k1, const float* __restrict__ s2, long ld2,
                      int k2, int rows, uint16_t* __restrict__ dst, long ldd, int f16) {
    const long n = (long)rows * (ldd / 2);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const long r = i / (ldd / 2);
        const int c = (int)(i % (ldd / 2)) * 2;
        float v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int cc = c + u;
            v[u] = cc < k1 ? s1[r * ld1 + cc] : (cc < k1 + k2 ? s2[r * ld2 + cc - k1] : 0.f);
        }
        ((uint32_t*)dst)[r * (ldd / 2) + c / 2] = f16 ? pack_f16x2(v[0], v[1]) : pack_bf16x2(v[0], v[1]);
    }
}

// Two-term 16-bit image of a weight matrix: dst[n, k] = rn16(W[n, k]) and
// dst[n, kp + k] = rn16(W[n, k] - rn16(W[n, k])) for k < K, zero elsewhere (row stride 2 kp).
__global__ void k_cvt_split(const float* __restrict__ W, long ldw, int N, int K, uint16_t* __restrict__ dst, int kp,
                            int f16) {
    const long n = (long)N * 2 * kp;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const long r = i / (2 * kp);
        const int c = (int)(i % (2 * kp)), k = c % kp;
        uint16_t out = 0;
        if (k < K) {
            const float w = W[r * ldw + k];
            const uint32_t hi = f16 ? pack_f16x2(w, 0.f) : pack_bf16x2(w, 0.f);
            if (c < kp) {
                out = (uint16_t)(hi & 0xffffu);
            } else {
                const float h = f16 ? __half2float(__ushort_as_half((unsigned short)(hi & 0xffffu)))
                                    : __bfloat162float(__ushort_as_bfloat16((unsigned short)(hi & 0xffffu)));
                const uint32_t lo = f16 ? pack_f16x2(w - h, 0.f) : pack_bf16x2(w - h, 0.f);
                out = (uint16_t)(lo & 0xffffu);
            }
        }
        dst[i] = out;
    }
}

typedef CUresult (*TgEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

TgEncodeFn tg_encode() {
    static TgEncodeFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (TgEncodeFn)p;
    }
    return fn;
}

// rows x Kp 16-bit matrix with row stride ld elements, boxes of box_rows x 64
bool tg_map(CUtensorMap* map, const void* base, long Kp, long rows, long ld, uint32_t box_rows) {
    TgEncodeFn fn = tg_encode();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)TG_BK, box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int ST, bool TWO = false>
void tg_launch(const CUtensorMap& ma, const CUtensorMap& mb, const TgArgs& a, int splits, int sms, cudaStream_t st) {
    using L = TgLayout<BN, ST, TWO>;
    const int tiles_m = (a.M + TG_BM - 1) / TG_BM, tiles_n = (std::max(a.N, a.c16_cols) + BN - 1) / BN;
    const long total = (long)tiles_m * tiles_n * splits;
    const int grid = (int)std::min<long>(total, sms);
    k_gemm_tc<BN, ST, TWO><<<grid, 320, L::BYTES, st>>>(ma, mb, a, tiles_m, tiles_n, splits);
}

template <int BN, int ST, bool TWO>
void tg_attr() {
    cudaFuncSetAttribute(k_gemm_tc<BN, ST, TWO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         TgLayout<BN, ST, TWO>::BYTES);
}

int g_sms[64] = {};

}  // namespace

void gemm_tc_prepare() {
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    // stages of 24-48 KB filling about 192 KB of shared memory: one CTA per SM
    tg_attr<64, 4, false>();
    tg_attr<128, 3, false>();
    tg_attr<64, 3, true>();
    tg_attr<128, 2, true>();
    cudaDeviceProp prop;
    g_sms[dev] = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.multiProcessorCount : 148;
    done[dev] = true;
}

bool gemm_tc(int f16, const void* A, long lda, const void* B, long ldb, int M, int N, int Kp, float* C, long ldc,
             const float* bias, const float* R, long ldr, int act, int mode, int kchunk, uint16_t* C16, long ldc16,
             unsigned* status, uint64_t wait_ns, cudaStream_t st, int c16_f16, int two_term, int c16_cols) {
    if (M <= 0 || N <= 0 || Kp <= 0) return true;
    const int Nt = std::max(N, C16 ? c16_cols : 0);
    const int BN = Nt <= 64 ? 64 : 128;
    CUtensorMap ma, mb;
    if (!tg_map(&ma, A, Kp, M, lda, TG_BM) || !tg_map(&mb, B, two_term ? 2L * Kp : Kp, N, ldb, BN)) return false;
    TgArgs a;
    a.M = M;
    a.N = N;
    a.Kp = Kp;
    if (kchunk <= 0 || kchunk >= Kp) kchunk = Kp;
    a.kchunk = kchunk;
    a.C = C;
    a.ldc = ldc;
    a.C16 = C16;
    a.ldc16 = ldc16;
    a.bias = bias;
    a.R = R;
    a.ldr = ldr;
    a.mode = mode;
    a.act = act;
    a.f16 = f16;
    a.c16_f16 = c16_f16;
    a.c16_cols = C16 ? std::max(c16_cols, N) : 0;
    a.status = status;
    a.wait_ns = wait_ns;
    const int splits = (Kp + kchunk - 1) / kchunk;
    int dev = 0;
    cudaGetDevice(&dev);
    const int sms = (dev >= 0 && dev < 64 && g_sms[dev] > 0) ? g_sms[dev] : 148;
    // stages of 24-48 KB filling about 96 KB of shared memory: two CTAs (each with two
    // accumulators of BN <= 128 columns) per SM
    if (two_term) {
        if (BN == 64)
            tg_launch<64, 3, true>(ma, mb, a, splits, 2 * sms, st);
        else
            tg_launch<128, 2, true>(ma, mb, a, splits, 2 * sms, st);
    } else if (BN == 64)
        tg_launch<64, 4>(ma, mb, a, splits, 2 * sms, st);
    else
        tg_launch<128, 3>(ma, mb, a, splits, 2 * sms, st);
    return true;
}

void cvt_16(const float* s1, long ld1, int k1, const float* s2, long ld2, int k2, int rows, uint16_t* dst, long ldd,
            int f16, cudaStream_t st) {
    const long n = (long)rows * (ldd / 2);
    if (n <= 0) return;
    const unsigned blocks = (unsigned)std::min<long>((n + 255) / 256, 148L * 16);
    k_cvt<<<blocks, 256, 0, st>>>(s1, ld1, k1, s2, ld2, k2, rows, dst, ldd, f16);
}

void cvt_16_split(const float* W, long ldw, int N, int K, uint16_t* dst, int kp, int f16, cudaStream_t st) {
    const long n = (long)N * 2 * kp;
    if (n <= 0) return;
    k_cvt_split<<<(unsigned)std::min<long>((n + 255) / 256, 148L * 16), 256, 0, st>>>(W, ldw, N, K, dst, kp, f16);
}

void cvt_16_t(const float* src, long lds, int rows, int cols, uint16_t* dst, long ldd, int f16, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return;
    dim3 grid((unsigned)((ldd + 31) / 32), (unsigned)((cols + 31) / 32));
    k_cvt_t<<<grid, 256, 0, st>>>(src, lds, rows, cols, dst, ldd, f16);
}

}  // namespace mlpf

using namespace mlpf;

extern "C" mlpf_status mlpf_gemm_tc(int32_t precision, const void* A, int64_t lda, const void* B, int64_t ldb,
                                    int32_t M, int32_t N, int32_t K, float* C, int64_t ldc, const float* bias,
                                    const float* R, int64_t ldr, int32_t act, int32_t mode, int32_t kchunk,
                                    uint32_t* status, void* stream) {
    if (precision != MLPF_BF16 && precision != MLPF_FP16) {
        set_error("mlpf_gemm_tc: precision must be MLPF_BF16 or MLPF_FP16");
        return MLPF_E_UNSUPPORTED;
    }
    if (!A || !B || !C || !status || M < 0 || N < 0 || K <= 0 || K % 64 || lda < K || ldb < K || lda % 8 ||
        ldb % 8 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ldc < N || mode < 0 || mode > 2 || act < -1 ||
        act > 1 || kchunk < 0 || kchunk % 64 || (R && ldr < N)) {
        set_error("mlpf_gemm_tc: bad arguments");
        return MLPF_E_INVALID;
    }
    gemm_tc_prepare();
    if (!gemm_tc(precision == MLPF_FP16, A, lda, B, ldb, M, N, K, C, ldc, bias, R, ldr, act, mode, kchunk, nullptr,
                 0, status, 2000000000ull, (cudaStream_t)stream)) {
        set_error("mlpf_gemm_tc: tensor map encoding failed");
        return MLPF_E_CUDA;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("mlpf_gemm_tc: ") + cudaGetErrorString(e));
        return MLPF_E_CUDA;
    }
    return MLPF_OK;
}
