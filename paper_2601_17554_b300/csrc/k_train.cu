// Training of a distilled (student) MLPF on per-element outputs of a full model:
// FP32 SIMT forward with saved activations, hand-written backward kernels
// (GEMM data and weight gradients, LayerNorm, GELU, varlen self-attention with
// the probabilities recomputed from the saved log-sum-exp), the fused
// distillation loss and the LAMB optimizer (You et al. 2019; the schedule of
// Sec. 5.3 is applied by the caller through the learning rate).
//
// Loss per element i (mean over the batch's elements):
//   KL(p_teacher || p_student) over the 6 classes
//   + sum over the 5 raw regression outputs (pT', eta, sin phi, cos phi, E') of
//     the squared difference, with the teacher's raw outputs recovered from its
//     decoded ones: pT' = log(pT / pT_elem), E' = log(E / E_elem) (Eq. 2).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace mlpf {
namespace {

inline unsigned cdivu(long a, long b) { return (unsigned)((a + b - 1) / b); }

__device__ __forceinline__ float gelu_fwd(float a) { return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float a) {
    // d/da [a Phi(a)] = Phi(a) + a phi(a)
    return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) + a * 0.3989422804014327f * expf(-0.5f * a * a);
}

__global__ void k_act_fwd(const float* __restrict__ a, float* __restrict__ h, long n, int act) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        h[i] = act == 1 ? fmaxf(a[i], 0.f) : gelu_fwd(a[i]);
}

__global__ void k_act_bwd(const float* __restrict__ a, const float* __restrict__ dh, float* __restrict__ da,
                          long n, int act) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        da[i] = dh[i] * (act == 1 ? (a[i] > 0.f ? 1.f : 0.f) : gelu_grad(a[i]));
}

// C[m, n] (+)= sum_k A(m, k) B(k, n), A(m, k) = A[m*lam + k*lak], B(k, n) = B[k*lbk + n*lbn].
// gridDim.z > 1 splits K into chunks of kchunk and adds partial results atomically
// (C must hold the value to add to).  accumulate = 0 overwrites C (single split only).
constexpr int GB = 64, GK = 16;
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, long lam,
                                              long lak, const float* __restrict__ B, long lbk, long lbn,
                                              float* C, long ldc, int accumulate, int kchunk) {
    __shared__ float As[GK][GB + 4];
    __shared__ float Bs[GK][GB + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * GB, n0 = blockIdx.x * GB;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    float acc[4][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += GK) {
        for (int i = threadIdx.x; i < GB * GK; i += 256) {
            int mm, kk;
            if (lak == 1) { kk = i % GK; mm = i / GK; } else { mm = i % GB; kk = i / GB; }
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < kend) ? A[(long)m * lam + (long)k * lak] : 0.f;
            int nn, kb;
            if (lbn == 1) { nn = i % GB; kb = i / GB; } else { kb = i % GK; nn = i / GK; }
            const int n = n0 + nn, k2 = k0 + kb;
            Bs[kb][nn] = (n < N && k2 < kend) ? B[(long)k2 * lbk + (long)n * lbn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float* c = C + (long)m * ldc + n;
            if (gridDim.z > 1)
                atomicAdd(c, acc[i][j]);
            else
                *c = accumulate ? *c + acc[i][j] : acc[i][j];
        }
    }
}

// out[n] += sum_t Y[t*ldy + n] (column sums; partial per block, then one atomic per column)
__global__ void k_colsum(const float* __restrict__ Y, long ldy, int T, int N, float* out, int rchunk) {
    __shared__ float part[8][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + lane;
    const int t0 = blockIdx.y * rchunk, t1 = min(T, t0 + rchunk);
    float s = 0.f;
    if (n < N)
        for (int t = t0 + w; t < t1; t += 8) s += Y[(long)t * ldy + n];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && n < N) {
        float a = 0.f;
        for (int i = 0; i < 8; ++i) a += part[i][lane];
        atomicAdd(out + n, a);
    }
}

// LayerNorm backward, one warp per row (d <= 256): dX (+)= d/dX of LN(X) applied to dY;
// dg += sum_t dY * xhat, db += sum_t dY (per-block partials, then atomics).
__global__ void __launch_bounds__(256) k_ln_bwd(const float* __restrict__ X, const float* __restrict__ g,
                                                const float* __restrict__ dY, float* dX, int accumulate,
                                                float* dg, float* db, int T, int d) {
    __shared__ float sg[8][256], sb[8][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float pg[8] = {}, pb[8] = {};
    for (int row = blockIdx.x * 8 + w; row < T; row += gridDim.x * 8) {
        const float* x = X + (long)row * d;
        const float* dy = dY + (long)row * d;
        float v[8], gy[8];
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = lane + 32 * i;
            v[i] = c < d ? x[c] : 0.f;
            s += v[i];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float mu = s / d;
        float q = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = lane + 32 * i;
            const float t = c < d ? v[i] - mu : 0.f;
            q += t * t;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        const float rs = rsqrtf(q / d + 1e-5f);
        float a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = lane + 32 * i;
            if (c < d) {
                const float xh = (v[i] - mu) * rs;
                const float dyv = dy[c];
                gy[i] = g[c] * dyv;
                a1 += gy[i];
                a2 += gy[i] * xh;
                pg[i] += dyv * xh;
                pb[i] += dyv;
                v[i] = xh;
            } else {
                gy[i] = 0.f;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        a1 /= d;
        a2 /= d;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int c = lane + 32 * i;
            if (c < d) {
                const float r = rs * (gy[i] - a1 - v[i] * a2);
                float* o = dX + (long)row * d + c;
                *o = accumulate ? *o + r : r;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int c = lane + 32 * i;
        if (c < 256) {
            sg[w][c] = pg[i];
            sb[w][c] = pb[i];
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < d; c += 256) {
        float a = 0.f, b = 0.f;
        for (int i = 0; i < 8; ++i) {
            a += sg[i][c];
            b += sb[i][c];
        }
        atomicAdd(dg + c, a);
        atomicAdd(db + c, b);
    }
}

// D[t, h] = sum_c dO[t, h*dh + c] * O[t, h*dh + c]
__global__ void k_attn_rowdot(const float* __restrict__ dO, const float* __restrict__ O, float* __restrict__ D,
                              int T, int d, int heads) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)T * heads) return;
    const int t = (int)(i / heads), h = (int)(i % heads), dh = d / heads;
    float s = 0.f;
    for (int c = 0; c < dh; ++c) s += dO[(long)t * d + h * dh + c] * O[(long)t * d + h * dh + c];
    D[i] = s;
}

// dQ of varlen self-attention: one thread per query row, keys in 64-row tiles.
// P_ij = exp(scale q_i.k_j - lse_i); dS_ij = P_ij (dO_i.v_j - D_i); dQ_i = scale sum_j dS_ij k_j.
template <int DH>
__global__ void __launch_bounds__(64) k_attn_bwd_dq(const float* __restrict__ qkv, const float* __restrict__ dO,
                                                    const float* __restrict__ lse, const float* __restrict__ D,
                                                    float* __restrict__ dqkv, const int32_t* __restrict__ cu,
                                                    int d, float scale) {
    __shared__ float Ks[64][DH + 1];
    __shared__ float Vs[64][DH + 1];
    const int e = blockIdx.z, h = blockIdx.y, H = gridDim.y;
    const int start = cu[e], n = cu[e + 1] - start;
    if (blockIdx.x * 64 >= n) return;
    const int qi = blockIdx.x * 64 + threadIdx.x;
    const bool active = qi < n;
    const int ld = 3 * d;
    float q[DH], g[DH], dq[DH];
    float L = 0.f, Dv = 0.f;
    if (active) {
        const long r = start + qi;
        for (int c = 0; c < DH; ++c) {
            q[c] = qkv[r * ld + h * DH + c] * scale;
            g[c] = dO[r * d + h * DH + c];
            dq[c] = 0.f;
        }
        L = lse[r * H + h];
        Dv = D[r * H + h];
    }
    for (int kb = 0; kb < n; kb += 64) {
        const int kj = kb + threadIdx.x;
        if (kj < n) {
            const long r = start + kj;
            for (int c = 0; c < DH; ++c) {
                Ks[threadIdx.x][c] = qkv[r * ld + d + h * DH + c];
                Vs[threadIdx.x][c] = qkv[r * ld + 2 * d + h * DH + c];
            }
        }
        __syncthreads();
        const int cnt = min(64, n - kb);
        if (active) {
            for (int j = 0; j < cnt; ++j) {
                float s = 0.f, dp = 0.f;
#pragma unroll
                for (int c = 0; c < DH; ++c) {
                    s = fmaf(q[c], Ks[j][c], s);
                    dp = fmaf(g[c], Vs[j][c], dp);
                }
                const float p = expf(s - L);
                const float ds = p * (dp - Dv);
#pragma unroll
                for (int c = 0; c < DH; ++c) dq[c] = fmaf(ds, Ks[j][c], dq[c]);
            }
        }
        __syncthreads();
    }
    if (active)
        for (int c = 0; c < DH; ++c) dqkv[(long)(start + qi) * ld + h * DH + c] = dq[c] * scale;
}

// dK, dV: one thread per key row, queries in 64-row tiles.
// dV_j = sum_i P_ij dO_i; dK_j = scale sum_i dS_ij q_i.
template <int DH>
__global__ void __launch_bounds__(64) k_attn_bwd_dkv(const float* __restrict__ qkv, const float* __restrict__ dO,
                                                     const float* __restrict__ lse, const float* __restrict__ D,
                                                     float* __restrict__ dqkv, const int32_t* __restrict__ cu,
                                                     int d, float scale) {
    __shared__ float Qs[64][DH + 1];
    __shared__ float Gs[64][DH + 1];
    __shared__ float Ls[64], Ds[64];
    const int e = blockIdx.z, h = blockIdx.y, H = gridDim.y;
    const int start = cu[e], n = cu[e + 1] - start;
    if (blockIdx.x * 64 >= n) return;
    const int kj = blockIdx.x * 64 + threadIdx.x;
    const bool active = kj < n;
    const int ld = 3 * d;
    float k[DH], v[DH], dk[DH], dv[DH];
    if (active) {
        const long r = start + kj;
        for (int c = 0; c < DH; ++c) {
            k[c] = qkv[r * ld + d + h * DH + c];
            v[c] = qkv[r * ld + 2 * d + h * DH + c];
            dk[c] = 0.f;
            dv[c] = 0.f;
        }
    }
    for (int qb = 0; qb < n; qb += 64) {
        const int qi = qb + threadIdx.x;
        if (qi < n) {
            const long r = start + qi;
            for (int c = 0; c < DH; ++c) {
                Qs[threadIdx.x][c] = qkv[r * ld + h * DH + c] * scale;
                Gs[threadIdx.x][c] = dO[r * d + h * DH + c];
            }
            Ls[threadIdx.x] = lse[r * H + h];
            Ds[threadIdx.x] = D[r * H + h];
        }
        __syncthreads();
        const int cnt = min(64, n - qb);
        if (active) {
            for (int i = 0; i < cnt; ++i) {
                float s = 0.f, dp = 0.f;
#pragma unroll
                for (int c = 0; c < DH; ++c) {
                    s = fmaf(Qs[i][c], k[c], s);
                    dp = fmaf(Gs[i][c], v[c], dp);
                }
                const float p = expf(s - Ls[i]);
                const float ds = p * (dp - Ds[i]);
#pragma unroll
                for (int c = 0; c < DH; ++c) {
                    dv[c] = fmaf(p, Gs[i][c], dv[c]);
                    dk[c] = fmaf(ds, Qs[i][c], dk[c]);
                }
            }
        }
        __syncthreads();
    }
    if (active) {
        const long r = start + kj;
        for (int c = 0; c < DH; ++c) {
            dqkv[r * ld + d + h * DH + c] = dk[c];
            dqkv[r * ld + 2 * d + h * DH + c] = dv[c];
        }
    }
}

// Distillation loss and its gradient w.r.t. the student's logits and raw outputs.
__global__ void __launch_bounds__(256) k_distill_loss(const float* __restrict__ sl, const float* __restrict__ sr,
                                                      const float* __restrict__ tl, const float* __restrict__ tr,
                                                      const float* __restrict__ x, int T, float invT,
                                                      float* __restrict__ dl, float* __restrict__ dr,
                                                      double* loss) {
    __shared__ double part[8];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double li = 0.0;
    if (t < T) {
        const float* a = sl + (long)t * 6;
        const float* b = tl + (long)t * 6;
        float ma = a[0], mb = b[0];
        for (int c = 1; c < 6; ++c) {
            ma = fmaxf(ma, a[c]);
            mb = fmaxf(mb, b[c]);
        }
        float za = 0.f, zb = 0.f;
        for (int c = 0; c < 6; ++c) {
            za += expf(a[c] - ma);
            zb += expf(b[c] - mb);
        }
        const float lza = logf(za), lzb = logf(zb);
        float kl = 0.f;
        for (int c = 0; c < 6; ++c) {
            const float lpa = a[c] - ma - lza, lpb = b[c] - mb - lzb;
            const float pb = expf(lpb);
            kl += pb * (lpb - lpa);
            dl[(long)t * 6 + c] = (expf(lpa) - pb) * invT;
        }
        const float* rs = sr + (long)t * 5;
        const float* rt = tr + (long)t * 5;
        float target[5];
        target[0] = logf(rt[0]) - x[(long)t * 42 + 8];
        target[1] = rt[1];
        target[2] = rt[2];
        target[3] = rt[3];
        target[4] = logf(rt[4]) - x[(long)t * 42 + 9];
        float mse = 0.f;
        for (int c = 0; c < 5; ++c) {
            const float df = rs[c] - target[c];
            mse += df * df;
            dr[(long)t * 5 + c] = 2.f * df * invT;
        }
        li = (double)(kl + mse) * invT;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) li += __shfl_xor_sync(0xffffffffu, li, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = li;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += part[i];
        atomicAdd(loss, s);
    }
}

// Supervised loss of Eq. 1 (printed architecture: logits = [binary, 5 PID]) and
// its gradient w.r.t. the logits and raw outputs, per element, mean over T:
//   beta BCE(b, sigmoid(z)) + b [ -(1 - p_t)^fg log p_t
//                                 + g (dpT'^2 + dE'^2) + delta (deta^2 + dsin^2 + dcos^2) ]
// b = [cls > 0], p_t = softmax(PID)[cls - 1], g = sqrt(pT target), pT' and E' targets
// by Eq. 2.  d/du_j of the focal term = c (delta_jk - p_j) with
// c = fg (1 - p_t)^(fg - 1) p_t log p_t - (1 - p_t)^fg.
__global__ void __launch_bounds__(256) k_supervised_loss(const float* __restrict__ lg, const float* __restrict__ raw,
                                                         const float* __restrict__ x, const int32_t* __restrict__ cls,
                                                         const float* __restrict__ regt, int T, float invT,
                                                         float beta, float fg, float delta,
                                                         float* __restrict__ dl, float* __restrict__ dr,
                                                         double* loss) {
    __shared__ double part[8];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double li = 0.0;
    if (t < T) {
        const float* l = lg + (long)t * 6;
        const int k = cls[t];
        const bool b = k > 0;
        const float z = l[0];
        const float bce = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))) - (b ? z : 0.f);
        const float sig = 1.f / (1.f + expf(-z));
        dl[(long)t * 6] = beta * (sig - (b ? 1.f : 0.f)) * invT;
        float lt = beta * bce;
        if (b) {
            float m = l[1];
            for (int c = 2; c < 6; ++c) m = fmaxf(m, l[c]);
            float zs = 0.f;
            for (int c = 1; c < 6; ++c) zs += expf(l[c] - m);
            const float lzs = logf(zs);
            const float logpt = l[k] - m - lzs, pt = expf(logpt), omp = 1.f - pt;
            const float ompg = powf(omp, fg);
            lt += -ompg * logpt;
            const float coef = fg * (fg == 0.f ? 0.f : powf(omp, fg - 1.f)) * pt * logpt - ompg;
            for (int c = 1; c < 6; ++c) {
                const float pj = expf(l[c] - m - lzs);
                dl[(long)t * 6 + c] = coef * ((c == k ? 1.f : 0.f) - pj) * invT;
            }
            const float* rt = regt + (long)t * 5;
            const float* rs = raw + (long)t * 5;
            const float g = sqrtf(rt[0]);
            float tgt[5], w[5] = {g, delta, delta, delta, g};
            tgt[0] = logf(rt[0]) - x[(long)t * 42 + 8];
            tgt[1] = rt[1];
            tgt[2] = rt[2];
            tgt[3] = rt[3];
            tgt[4] = logf(rt[4]) - x[(long)t * 42 + 9];
            for (int c = 0; c < 5; ++c) {
                const float df = rs[c] - tgt[c];
                lt += w[c] * df * df;
                dr[(long)t * 5 + c] = 2.f * w[c] * df * invT;
            }
        } else {
            for (int c = 1; c < 6; ++c) dl[(long)t * 6 + c] = 0.f;
            for (int c = 0; c < 5; ++c) dr[(long)t * 5 + c] = 0.f;
        }
        li = (double)lt * invT;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) li += __shfl_xor_sync(0xffffffffu, li, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = li;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += part[i];
        atomicAdd(loss, s);
    }
}

// Printed architecture: track-like elements (track, GSF track, brem; one-hot x[0],
// x[5], x[6]) take the track embedding.  merge: z = is_track ? et : ec.  split:
// dt = is_track ? d : 0, dc = is_track ? 0 : d (dt may alias d).
__device__ __forceinline__ bool is_track_row(const float* x, long r) {
    const float* xr = x + r * 42;
    return xr[0] + xr[5] + xr[6] > 0.5f;
}
__global__ void k_type_merge(const float* __restrict__ x, const float* __restrict__ et, const float* __restrict__ ec,
                             float* __restrict__ z, int T, int d) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)T * d) return;
    z[i] = is_track_row(x, i / d) ? et[i] : ec[i];
}
__global__ void k_type_split(const float* __restrict__ x, float* dt, float* __restrict__ dc, int T, int d) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long)T * d) return;
    const float v = dt[i];
    const bool trk = is_track_row(x, i / d);
    dt[i] = trk ? v : 0.f;
    dc[i] = trk ? 0.f : v;
}
__global__ void k_add(float* __restrict__ a, const float* __restrict__ b, long n) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] += b[i];
}

// LAMB: per chunk (tensor id, start, length) of the parameter vector.
__global__ void __launch_bounds__(256) k_lamb_moments(const float* __restrict__ w, float* __restrict__ g,
                                                      float* __restrict__ m, float* __restrict__ v,
                                                      const int4* __restrict__ chunks, double* wn2,
                                                      double* un2, float b1, float b2, float eps, float bc1,
                                                      float bc2, float wd) {
    __shared__ double s1[8], s2[8];
    const int4 ch = chunks[blockIdx.x];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < ch.z; i += 256) {
        const long k = (long)ch.y + i;
        const float gi = g[k];
        const float mi = b1 * m[k] + (1.f - b1) * gi;
        const float vi = b2 * v[k] + (1.f - b2) * gi * gi;
        m[k] = mi;
        v[k] = vi;
        const float u = (mi / bc1) / (sqrtf(vi / bc2) + eps) + wd * w[k];
        g[k] = u;
        a += (double)w[k] * w[k];
        b += (double)u * u;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s1[threadIdx.x >> 5] = a;
        s2[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x1 = 0.0, x2 = 0.0;
        for (int i = 0; i < 8; ++i) {
            x1 += s1[i];
            x2 += s2[i];
        }
        atomicAdd(wn2 + ch.x, x1);
        atomicAdd(un2 + ch.x, x2);
    }
}

__global__ void __launch_bounds__(256) k_lamb_apply(float* __restrict__ w, const float* __restrict__ u,
                                                    const int4* __restrict__ chunks, const double* wn2,
                                                    const double* un2, float lr) {
    const int4 ch = chunks[blockIdx.x];
    const double wn = sqrt(wn2[ch.x]), un = sqrt(un2[ch.x]);
    const float trust = (wn > 0.0 && un > 0.0) ? (float)(wn / un) : 1.f;
    for (int i = threadIdx.x; i < ch.z; i += 256) {
        const long k = (long)ch.y + i;
        w[k] -= lr * trust * u[k];
    }
}

}  // namespace

// ------------------------------------------------------------------ trainer
struct Trainer {
    Model m;                       // configuration and host copies of the initial tensors
    std::vector<std::string> names;
    std::vector<std::vector<int>> shapes;
    std::vector<size_t> offs, sizes;
    size_t n_params = 0;
    float *w = nullptr, *g = nullptr, *mom = nullptr, *var = nullptr;
    int4* chunks = nullptr;
    int n_chunks = 0;
    double* scratch = nullptr;     // [0] loss, [1..] per-tensor |w|^2, |u|^2
    long step = 0;
    // activation workspace
    size_t cap_rows = 0;
    float* act = nullptr;
    size_t act_floats = 0;
    // the batch whose activations the workspace holds after mlpf_trainer_forward (the
    // batch mlpf_trainer_backward must be called on); fwd_ok is cleared by any step
    bool fwd_ok = false;
    const float* fwd_x = nullptr;
    const int32_t* fwd_cu = nullptr;
    int32_t fwd_n = 0, fwd_total = 0;
    // GEMM arithmetic: MLPF_FP32 (SIMT FFMA) or 16-bit tensor-core operands (MLPF_BF16,
    // MLPF_FP16) with FP32 accumulation, FP32 master weights and FP32 activations
    int prec = MLPF_FP32;
    uint16_t* h16 = nullptr;       // operand scratch of the tensor-core GEMMs
    uint16_t *ha = nullptr, *hb = nullptr, *ht1 = nullptr, *ht2 = nullptr;
    size_t h16_rows = 0;
    unsigned* status = nullptr;    // device status word of the bounded waits
    bool tc_fail = false;          // a tensor map could not be encoded
};

namespace {

struct Acts {
    float *a1, *h1;                                   // embedding
    std::vector<float*> zp, zr;                       // residual snapshots per stack (L+1 each)
    std::vector<float*> ln1p, qkvp, op, lsep, zmp, ln2p, afp, hfp;  // per PID layer
    std::vector<float*> ln1r, qkvr, orr, lser, zmr, ln2r, afr, hfr; // per reg layer
    float *hp, *hreg, *ar, *hr, *ac, *hc, *logits, *raw;
    float *ah[4], *hh[4];
    // printed architecture: cluster embedding hidden/output, track embedding output,
    // PID head hidden (the binary head uses ac/hc)
    float *a1c, *h1c, *et, *ec, *ac2, *hc2;
    // backward
    float *dz, *dx1, *dx2, *dhp, *dhreg, *dlog, *draw, *D, *demb, *dsel;
};

size_t acts_layout(const mlpf_config& c, size_t T, Acts* A, float* base) {
    const size_t d = c.d, F = c.ffn, H = c.heads, W3 = std::max(3 * d, F);
    size_t off = 0;
    auto take = [&](size_t n) {
        float* p = base ? base + off : nullptr;
        off += (n * T + 63) / 64 * 64;
        return p;
    };
    Acts a;
    a.a1 = take(d);
    a.h1 = take(d);
    for (int l = 0; l <= c.l_pid; ++l) a.zp.push_back(take(d));
    for (int l = 0; l <= c.l_reg; ++l) a.zr.push_back(take(d));
    auto layer = [&](std::vector<float*>& ln1, std::vector<float*>& qkv, std::vector<float*>& o,
                     std::vector<float*>& lse, std::vector<float*>& zm, std::vector<float*>& ln2,
                     std::vector<float*>& af, std::vector<float*>& hf) {
        ln1.push_back(take(d));
        qkv.push_back(take(3 * d));
        o.push_back(take(d));
        lse.push_back(take(H));
        zm.push_back(take(d));
        ln2.push_back(take(d));
        af.push_back(take(F));
        hf.push_back(take(F));
    };
    for (int l = 0; l < c.l_pid; ++l) layer(a.ln1p, a.qkvp, a.op, a.lsep, a.zmp, a.ln2p, a.afp, a.hfp);
    for (int l = 0; l < c.l_reg; ++l) layer(a.ln1r, a.qkvr, a.orr, a.lser, a.zmr, a.ln2r, a.afr, a.hfr);
    a.hp = take(d);
    a.hreg = take(d);
    a.ar = take(d);
    a.hr = take(d);
    a.ac = take(d);
    a.hc = take(d);
    a.logits = take(6);
    a.raw = take(5);
    for (int k = 0; k < 4; ++k) {
        a.ah[k] = take(d);
        a.hh[k] = take(d);
    }
    const bool paper = c.arch == 1;
    a.a1c = paper ? take(d) : nullptr;
    a.h1c = paper ? take(d) : nullptr;
    a.et = paper ? take(d) : nullptr;
    a.ec = paper ? take(d) : nullptr;
    a.ac2 = paper ? take(d) : nullptr;
    a.hc2 = paper ? take(d) : nullptr;
    a.demb = paper ? take(d) : nullptr;
    a.dsel = paper ? take(d) : nullptr;
    a.dz = take(d);
    a.dx1 = take(W3);
    a.dx2 = take(W3);
    a.dhp = take(d);
    a.dhreg = take(d);
    a.dlog = take(6);
    a.draw = take(5);
    a.D = take(H);
    if (A) *A = a;
    return off;
}

const char* RH[4] = {"pt", "eta", "phi", "e"};
const int RW[4] = {1, 1, 2, 1};

}  // namespace

static float* P(Trainer& t, const std::string& n) {
    for (size_t i = 0; i < t.names.size(); ++i)
        if (t.names[i] == n) return t.w + t.offs[i];
    return nullptr;
}
static float* G(Trainer& t, const std::string& n) {
    for (size_t i = 0; i < t.names.size(); ++i)
        if (t.names[i] == n) return t.g + t.offs[i];
    return nullptr;
}

// dW[N, K] += dY[T, N]^T X[T, K] (ldy, ldx, ldw row strides); split over T
static void gemm_dw(const float* dY, long ldy, const float* X, long ldx, float* dW, long ldw, int T, int N, int K,
                    cudaStream_t st) {
    const int chunk = 4096;
    dim3 grid(cdivu(K, GB), cdivu(N, GB), cdivu(T, chunk));
    k_gemm<<<grid, 256, 0, st>>>(N, K, T, dY, 1, ldy, X, ldx, 1, dW, ldw, 1, chunk);
}
// dX[T, K] (+)= dY[T, N] W[N, K] with W row stride ldw (column offset in W via pointer)
static void gemm_dx(const float* dY, long ldy, const float* W, long ldw, float* dX, long ldx, int T, int N, int K,
                    int accumulate, cudaStream_t st) {
    dim3 grid(cdivu(K, GB), cdivu(T, GB), 1);
    k_gemm<<<grid, 256, 0, st>>>(T, K, N, dY, ldy, 1, W, ldw, 1, dX, ldx, accumulate, N);
}
static long r64(long v) { return (v + 63) / 64 * 64; }
static constexpr uint64_t TRAIN_WAIT_NS = 2000000000ull;   // 2 s per bounded wait

// y[T, N] = [X1 | X2] W^T + b (+ R): W row-major [N, K1 + K2]
static void lin(Trainer& t, const float* X1, int ld1, int K1, const float* X2, int ld2, int K2, const float* W,
                const float* b, const float* R, int ldr, float* Y, int ldy, int T, int N, cudaStream_t st) {
    if (t.prec == MLPF_FP32) {
        f32_linear(X1, ld1, K1, X2, ld2, K2, W, b, R, ldr, Y, ldy, T, N, -1, st);
        return;
    }
    const int f16 = t.prec == MLPF_FP16, K = K1 + K2;
    const long Kp = r64(K);
    cvt_16(X1, ld1, K1, X2, ld2, K2, T, t.ha, Kp, f16, st);
    cvt_16(W, K, K, nullptr, 0, 0, N, t.hb, Kp, f16, st);
    if (!gemm_tc(f16, t.ha, Kp, t.hb, Kp, T, N, (int)Kp, Y, ldy, b, R, ldr, -1, 0, 0, nullptr, 0, t.status,
                 TRAIN_WAIT_NS, st))
        t.tc_fail = true;
}
// dW[N, K] += dY[T, N]^T X[T, K]
static void dw(Trainer& t, const float* dY, long ldy, const float* X, long ldx, float* dW, long ldw, int T, int N,
               int K, cudaStream_t st) {
    if (t.prec == MLPF_FP32) {
        gemm_dw(dY, ldy, X, ldx, dW, ldw, T, N, K, st);
        return;
    }
    const int f16 = t.prec == MLPF_FP16;
    const long Tp = r64(T);
    cvt_16_t(dY, ldy, T, N, t.ht1, Tp, f16, st);   // [N, Tp]
    cvt_16_t(X, ldx, T, K, t.ht2, Tp, f16, st);    // [K, Tp]
    // split the reduction over the batch so that about two CTAs per SM work
    const long bn = K <= 64 ? 64 : (K <= 128 ? 128 : 256);   // the GEMM's tile width for N = K
    const long tiles = ((N + 127) / 128) * ((K + bn - 1) / bn);
    const long splits = std::max(1L, std::min(Tp / 512, 296 / std::max(1L, tiles)));
    const long kchunk = r64((Tp + splits - 1) / splits);
    if (!gemm_tc(f16, t.ht1, Tp, t.ht2, Tp, N, K, (int)Tp, dW, ldw, nullptr, nullptr, 0, -1, 2, (int)kchunk, nullptr,
                 0, t.status, TRAIN_WAIT_NS, st))
        t.tc_fail = true;
}
// dX[T, K] (+)= dY[T, N] W[N, K] (W row stride ldw)
static void dx(Trainer& t, const float* dY, long ldy, const float* W, long ldw, float* dX, long ldx, int T, int N,
               int K, int accumulate, cudaStream_t st) {
    if (t.prec == MLPF_FP32) {
        gemm_dx(dY, ldy, W, ldw, dX, ldx, T, N, K, accumulate, st);
        return;
    }
    const int f16 = t.prec == MLPF_FP16;
    const long Np = r64(N);
    cvt_16(dY, ldy, N, nullptr, 0, 0, T, t.ha, Np, f16, st);   // [T, Np]
    cvt_16_t(W, ldw, N, K, t.hb, Np, f16, st);                 // W^T: [K, Np]
    if (!gemm_tc(f16, t.ha, Np, t.hb, Np, T, K, (int)Np, dX, ldx, nullptr, nullptr, 0, -1, accumulate ? 1 : 0, 0,
                 nullptr, 0, t.status, TRAIN_WAIT_NS, st))
        t.tc_fail = true;
}
static void colsum(const float* Y, long ldy, int T, int N, float* out, cudaStream_t st) {
    const int rchunk = 2048;
    dim3 grid(cdivu(N, 32), cdivu(T, rchunk));
    k_colsum<<<grid, 256, 0, st>>>(Y, ldy, T, N, out, rchunk);
}
static void act_fwd(const float* a, float* h, long n, int act, cudaStream_t st) {
    k_act_fwd<<<(unsigned)std::min<long>(cdivu(n, 256), 148 * 16), 256, 0, st>>>(a, h, n, act);
}
static void act_bwd(const float* a, const float* dh, float* da, long n, int act, cudaStream_t st) {
    k_act_bwd<<<(unsigned)std::min<long>(cdivu(n, 256), 148 * 16), 256, 0, st>>>(a, dh, da, n, act);
}
static void ln_bwd(const float* X, const float* gam, const float* dY, float* dX, int acc, float* dg, float* db,
                   int T, int d, cudaStream_t st) {
    k_ln_bwd<<<std::min<unsigned>(cdivu(T, 8), 148 * 8), 256, 0, st>>>(X, gam, dY, dX, acc, dg, db, T, d);
}

// Forward of the whole model with every activation the backward pass needs.
static void train_forward(Trainer& t, const Acts& a, const float* x, const int32_t* cu, int n_events, int T,
                          int max_n, cudaStream_t st) {
    const mlpf_config& c = t.m.cfg;
    const int d = c.d, F = c.ffn, act = c.act;
    const bool paper = c.arch == 1;
    if (paper) {   // track and cluster embeddings, selected per element type
        lin(t, x, 42, 42, nullptr, 0, 0, P(t, "emb.trk.w1"), P(t, "emb.trk.b1"), nullptr, 0, a.a1, d, T, d, st);
        act_fwd(a.a1, a.h1, (long)T * d, act, st);
        lin(t, a.h1, d, d, nullptr, 0, 0, P(t, "emb.trk.w2"), P(t, "emb.trk.b2"), nullptr, 0, a.et, d, T, d, st);
        lin(t, x, 42, 42, nullptr, 0, 0, P(t, "emb.clu.w1"), P(t, "emb.clu.b1"), nullptr, 0, a.a1c, d, T, d, st);
        act_fwd(a.a1c, a.h1c, (long)T * d, act, st);
        lin(t, a.h1c, d, d, nullptr, 0, 0, P(t, "emb.clu.w2"), P(t, "emb.clu.b2"), nullptr, 0, a.ec, d, T, d, st);
        k_type_merge<<<cdivu((long)T * d, 256), 256, 0, st>>>(x, a.et, a.ec, a.zp[0], T, d);
        cudaMemcpyAsync(a.zr[0], a.zp[0], (size_t)T * d * sizeof(float), cudaMemcpyDeviceToDevice, st);
    } else {
        lin(t, x, 42, 42, nullptr, 0, 0, P(t, "emb.w1"), P(t, "emb.b1"), nullptr, 0, a.a1, d, T, d, st);
        act_fwd(a.a1, a.h1, (long)T * d, act, st);
        lin(t, a.h1, d, d, nullptr, 0, 0, P(t, "emb.w2"), P(t, "emb.b2"), nullptr, 0, a.zp[0], d, T, d, st);
    }
    auto stack = [&](const char* pre, int L, const std::vector<float*>& z, const std::vector<float*>& ln1,
                     const std::vector<float*>& qkv, const std::vector<float*>& o, const std::vector<float*>& lse,
                     const std::vector<float*>& zm, const std::vector<float*>& ln2, const std::vector<float*>& af,
                     const std::vector<float*>& hf, float* out) {
        for (int l = 0; l < L; ++l) {
            const std::string p = std::string(pre) + "." + std::to_string(l) + ".";
            f32_layernorm(z[l], P(t, p + "ln1.g"), P(t, p + "ln1.b"), ln1[l], T, d, st);
            const char* qn[3] = {"q", "k", "v"};
            for (int i = 0; i < 3; ++i)
                lin(t, ln1[l], d, d, nullptr, 0, 0, P(t, p + "w" + qn[i]), P(t, p + "b" + qn[i]), nullptr, 0,
                           qkv[l] + i * d, 3 * d, T, d, st);
            if (t.prec == MLPF_FP32)
                f32_attention(qkv[l], o[l], cu, n_events, max_n, d, c.heads, lse[l], st);
            else if (!attn_train_fwd_tc(t.prec == MLPF_FP16, qkv[l], o[l], lse[l], cu, n_events, max_n, d, c.heads,
                                        st))
                t.tc_fail = true;
            lin(t, o[l], d, d, nullptr, 0, 0, P(t, p + "wo"), P(t, p + "bo"), z[l], d, zm[l], d, T, d, st);
            f32_layernorm(zm[l], P(t, p + "ln2.g"), P(t, p + "ln2.b"), ln2[l], T, d, st);
            lin(t, ln2[l], d, d, nullptr, 0, 0, P(t, p + "ffn.w1"), P(t, p + "ffn.b1"), nullptr, 0, af[l], F, T, F,
                       st);
            act_fwd(af[l], hf[l], (long)T * F, act, st);
            lin(t, hf[l], F, F, nullptr, 0, 0, P(t, p + "ffn.w2"), P(t, p + "ffn.b2"), zm[l], d, z[l + 1], d, T, d,
                       st);
        }
        f32_layernorm(z[L], P(t, std::string(pre) + ".lnf.g"), P(t, std::string(pre) + ".lnf.b"), out, T, d, st);
    };
    stack("pid", c.l_pid, a.zp, a.ln1p, a.qkvp, a.op, a.lsep, a.zmp, a.ln2p, a.afp, a.hfp, a.hp);
    if (!paper) {
        lin(t, x, 42, 42, a.hp, d, d, P(t, "remb.w1"), P(t, "remb.b1"), nullptr, 0, a.ar, d, T, d, st);
        act_fwd(a.ar, a.hr, (long)T * d, act, st);
        lin(t, a.hr, d, d, nullptr, 0, 0, P(t, "remb.w2"), P(t, "remb.b2"), nullptr, 0, a.zr[0], d, T, d, st);
    }
    stack("reg", c.l_reg, a.zr, a.ln1r, a.qkvr, a.orr, a.lser, a.zmr, a.ln2r, a.afr, a.hfr, a.hreg);
    if (paper) {   // binary head -> logit column 0, PID head -> columns 1..5
        lin(t, a.hp, d, d, nullptr, 0, 0, P(t, "head.bin.w1"), P(t, "head.bin.b1"), nullptr, 0, a.ac, d, T, d, st);
        act_fwd(a.ac, a.hc, (long)T * d, act, st);
        lin(t, a.hc, d, d, nullptr, 0, 0, P(t, "head.bin.w2"), P(t, "head.bin.b2"), nullptr, 0, a.logits, 6, T, 1,
                   st);
        lin(t, a.hp, d, d, nullptr, 0, 0, P(t, "head.pid.w1"), P(t, "head.pid.b1"), nullptr, 0, a.ac2, d, T, d, st);
        act_fwd(a.ac2, a.hc2, (long)T * d, act, st);
        lin(t, a.hc2, d, d, nullptr, 0, 0, P(t, "head.pid.w2"), P(t, "head.pid.b2"), nullptr, 0, a.logits + 1, 6, T,
                   5, st);
    } else {
        lin(t, a.hp, d, d, nullptr, 0, 0, P(t, "head.cls.w1"), P(t, "head.cls.b1"), nullptr, 0, a.ac, d, T, d, st);
        act_fwd(a.ac, a.hc, (long)T * d, act, st);
        lin(t, a.hc, d, d, nullptr, 0, 0, P(t, "head.cls.w2"), P(t, "head.cls.b2"), nullptr, 0, a.logits, 6, T, 6,
                   st);
    }
    int off = 0;
    for (int k = 0; k < 4; ++k) {
        const std::string p = std::string("head.") + RH[k] + ".";
        lin(t, a.hreg, d, d, nullptr, 0, 0, P(t, p + "w1"), P(t, p + "b1"), nullptr, 0, a.ah[k], d, T, d, st);
        act_fwd(a.ah[k], a.hh[k], (long)T * d, act, st);
        lin(t, a.hh[k], d, d, nullptr, 0, 0, P(t, p + "w2"), P(t, p + "b2"), nullptr, 0, a.raw + off, 5, T, RW[k],
                   st);
        off += RW[k];
    }
}

// Backward from dlog/draw (set by the loss kernel) into t.g.
static void train_backward(Trainer& t, const Acts& a, const float* x, const int32_t* cu, int n_events, int T,
                           int max_n, cudaStream_t st) {
    const mlpf_config& c = t.m.cfg;
    const int d = c.d, F = c.ffn, act = c.act, H = c.heads, dh = d / H;
    const float scale = 1.0f / sqrtf((float)dh);
    // linear y = x W^T + b: weight, bias and (optionally) input gradients
    auto lin_bwd = [&](const float* dY, int ldy, const float* X, int ldx, const std::string& wn,
                       const std::string& bn, int N, int K, float* dX, int ldxo, int acc) {
        dw(t, dY, ldy, X, ldx, G(t, wn), K, T, N, K, st);
        colsum(dY, ldy, T, N, G(t, bn), st);
        if (dX) dx(t, dY, ldy, P(t, wn), K, dX, ldxo, T, N, K, acc, st);
    };
    const bool paper = c.arch == 1;
    if (paper) {   // binary head (logit column 0) and PID head (columns 1..5)
        lin_bwd(a.dlog, 6, a.hc, d, "head.bin.w2", "head.bin.b2", 1, d, a.dx1, d, 0);
        act_bwd(a.ac, a.dx1, a.dx2, (long)T * d, act, st);
        lin_bwd(a.dx2, d, a.hp, d, "head.bin.w1", "head.bin.b1", d, d, a.dhp, d, 0);
        lin_bwd(a.dlog + 1, 6, a.hc2, d, "head.pid.w2", "head.pid.b2", 5, d, a.dx1, d, 0);
        act_bwd(a.ac2, a.dx1, a.dx2, (long)T * d, act, st);
        lin_bwd(a.dx2, d, a.hp, d, "head.pid.w1", "head.pid.b1", d, d, a.dhp, d, 1);
    } else {   // class head
        lin_bwd(a.dlog, 6, a.hc, d, "head.cls.w2", "head.cls.b2", 6, d, a.dx1, d, 0);
        act_bwd(a.ac, a.dx1, a.dx2, (long)T * d, act, st);
        lin_bwd(a.dx2, d, a.hp, d, "head.cls.w1", "head.cls.b1", d, d, a.dhp, d, 0);
    }
    // regression heads
    int off = 0;
    for (int k = 0; k < 4; ++k) {
        const std::string p = std::string("head.") + RH[k] + ".";
        lin_bwd(a.draw + off, 5, a.hh[k], d, p + "w2", p + "b2", RW[k], d, a.dx1, d, 0);
        act_bwd(a.ah[k], a.dx1, a.dx2, (long)T * d, act, st);
        lin_bwd(a.dx2, d, a.hreg, d, p + "w1", p + "b1", d, d, a.dhreg, d, k > 0);
        off += RW[k];
    }
    auto stack_bwd = [&](const char* pre, int L, const std::vector<float*>& z, const std::vector<float*>& ln1,
                         const std::vector<float*>& qkv, const std::vector<float*>& o, const std::vector<float*>& lse,
                         const std::vector<float*>& zm, const std::vector<float*>& ln2,
                         const std::vector<float*>& af, const std::vector<float*>& hf, const float* dout) {
        ln_bwd(z[L], P(t, std::string(pre) + ".lnf.g"), dout, a.dz, 0, G(t, std::string(pre) + ".lnf.g"),
               G(t, std::string(pre) + ".lnf.b"), T, d, st);
        for (int l = L - 1; l >= 0; --l) {
            const std::string p = std::string(pre) + "." + std::to_string(l) + ".";
            // z[l+1] = zm + FFN(LN2(zm))
            lin_bwd(a.dz, d, hf[l], F, p + "ffn.w2", p + "ffn.b2", d, F, a.dx1, F, 0);
            act_bwd(af[l], a.dx1, a.dx2, (long)T * F, act, st);
            lin_bwd(a.dx2, F, ln2[l], d, p + "ffn.w1", p + "ffn.b1", F, d, a.dx1, d, 0);
            ln_bwd(zm[l], P(t, p + "ln2.g"), a.dx1, a.dz, 1, G(t, p + "ln2.g"), G(t, p + "ln2.b"), T, d, st);
            // zm = z[l] + MHA(LN1(z[l]))
            lin_bwd(a.dz, d, o[l], d, p + "wo", p + "bo", d, d, a.dx1, d, 0);   // dx1 = dO
            k_attn_rowdot<<<cdivu((long)T * H, 256), 256, 0, st>>>(a.dx1, o[l], a.D, T, d, H);
            dim3 grid(cdivu(max_n, 64), H, n_events);
            if (t.prec != MLPF_FP32) {
                if (!attn_train_bwd_tc(t.prec == MLPF_FP16, qkv[l], a.dx1, lse[l], a.D, a.dx2, cu, n_events, max_n, d,
                                       H, st))
                    t.tc_fail = true;
            } else if (dh == 16) {
                k_attn_bwd_dq<16><<<grid, 64, 0, st>>>(qkv[l], a.dx1, lse[l], a.D, a.dx2, cu, d, scale);
                k_attn_bwd_dkv<16><<<grid, 64, 0, st>>>(qkv[l], a.dx1, lse[l], a.D, a.dx2, cu, d, scale);
            } else if (dh == 32) {
                k_attn_bwd_dq<32><<<grid, 64, 0, st>>>(qkv[l], a.dx1, lse[l], a.D, a.dx2, cu, d, scale);
                k_attn_bwd_dkv<32><<<grid, 64, 0, st>>>(qkv[l], a.dx1, lse[l], a.D, a.dx2, cu, d, scale);
            } else {
                k_attn_bwd_dq<64><<<grid, 64, 0, st>>>(qkv[l], a.dx1, lse[l], a.D, a.dx2, cu, d, scale);
                k_attn_bwd_dkv<64><<<grid, 64, 0, st>>>(qkv[l], a.dx1, lse[l], a.D, a.dx2, cu, d, scale);
            }
            const char* qn[3] = {"q", "k", "v"};
            for (int i = 0; i < 3; ++i)  // dx1 <- dLN1 = sum of the three projections' input gradients
                lin_bwd(a.dx2 + i * d, 3 * d, ln1[l], d, p + "w" + qn[i], p + "b" + qn[i], d, d, a.dx1, d, i > 0);
            ln_bwd(z[l], P(t, p + "ln1.g"), a.dx1, a.dz, 1, G(t, p + "ln1.g"), G(t, p + "ln1.b"), T, d, st);
        }
    };
    stack_bwd("reg", c.l_reg, a.zr, a.ln1r, a.qkvr, a.orr, a.lser, a.zmr, a.ln2r, a.afr, a.hfr, a.dhreg);
    if (paper) {
        // both stacks read the embedding: its gradient is the sum of theirs
        cudaMemcpyAsync(a.demb, a.dz, (size_t)T * d * sizeof(float), cudaMemcpyDeviceToDevice, st);
        stack_bwd("pid", c.l_pid, a.zp, a.ln1p, a.qkvp, a.op, a.lsep, a.zmp, a.ln2p, a.afp, a.hfp, a.dhp);
        k_add<<<cdivu((long)T * d, 256), 256, 0, st>>>(a.demb, a.dz, (long)T * d);
        k_type_split<<<cdivu((long)T * d, 256), 256, 0, st>>>(x, a.demb, a.dsel, T, d);
        lin_bwd(a.demb, d, a.h1, d, "emb.trk.w2", "emb.trk.b2", d, d, a.dx1, d, 0);
        act_bwd(a.a1, a.dx1, a.dx2, (long)T * d, act, st);
        lin_bwd(a.dx2, d, x, 42, "emb.trk.w1", "emb.trk.b1", d, 42, nullptr, 0, 0);
        lin_bwd(a.dsel, d, a.h1c, d, "emb.clu.w2", "emb.clu.b2", d, d, a.dx1, d, 0);
        act_bwd(a.a1c, a.dx1, a.dx2, (long)T * d, act, st);
        lin_bwd(a.dx2, d, x, 42, "emb.clu.w1", "emb.clu.b1", d, 42, nullptr, 0, 0);
        return;
    }
    // regression-stack input FFN over concat(x, h_pid)
    lin_bwd(a.dz, d, a.hr, d, "remb.w2", "remb.b2", d, d, a.dx1, d, 0);
    act_bwd(a.ar, a.dx1, a.dx2, (long)T * d, act, st);
    {
        const int Kin = 42 + d;
        dw(t, a.dx2, d, x, 42, G(t, "remb.w1"), Kin, T, d, 42, st);
        dw(t, a.dx2, d, a.hp, d, G(t, "remb.w1") + 42, Kin, T, d, d, st);
        colsum(a.dx2, d, T, d, G(t, "remb.b1"), st);
        dx(t, a.dx2, d, P(t, "remb.w1") + 42, Kin, a.dhp, d, T, d, d, 1, st);
    }
    stack_bwd("pid", c.l_pid, a.zp, a.ln1p, a.qkvp, a.op, a.lsep, a.zmp, a.ln2p, a.afp, a.hfp, a.dhp);
    // embedding
    lin_bwd(a.dz, d, a.h1, d, "emb.w2", "emb.b2", d, d, a.dx1, d, 0);
    act_bwd(a.a1, a.dx1, a.dx2, (long)T * d, act, st);
    lin_bwd(a.dx2, d, x, 42, "emb.w1", "emb.b1", d, 42, nullptr, 0, 0);
}

}  // namespace mlpf

using namespace mlpf;

struct mlpf_trainer {
    Trainer t;
};

#define TCK(call)                                                                   \
    do {                                                                            \
        cudaError_t _e = (call);                                                    \
        if (_e != cudaSuccess) {                                                    \
            set_error(std::string(#call) + ": " + cudaGetErrorString(_e));          \
            return _e == cudaErrorMemoryAllocation ? MLPF_E_OOM : MLPF_E_CUDA;      \
        }                                                                           \
    } while (0)

// Operand scratch of the tensor-core GEMMs for `rows` rows: the widest GEMM operand
// (K or N up to max(42 + d, ffn), padded to 64) row-major, a weight image, and two
// transposed operands whose reduction runs over the rows.
static size_t h16_elems(const mlpf_config& c, size_t rows, size_t* kw_out = nullptr) {
    const size_t kw = (size_t)r64(std::max(42 + c.d, std::max(c.ffn, c.d)));
    if (kw_out) *kw_out = kw;
    return rows * kw + kw * kw + 2 * kw * (size_t)r64((long)rows);
}
static mlpf_status ensure_h16(Trainer& t) {
    if (t.prec == MLPF_FP32 || (t.h16 && t.h16_rows == t.cap_rows)) return MLPF_OK;
    if (t.h16) cudaFree(t.h16);
    t.h16 = nullptr;
    t.h16_rows = 0;
    size_t kw;
    const size_t n = h16_elems(t.m.cfg, t.cap_rows, &kw);
    TCK(cudaMalloc(&t.h16, n * sizeof(uint16_t)));
    t.h16_rows = t.cap_rows;
    t.ha = t.h16;
    t.hb = t.ha + t.cap_rows * kw;
    t.ht1 = t.hb + kw * kw;
    t.ht2 = t.ht1 + kw * (size_t)r64((long)t.cap_rows);
    return MLPF_OK;
}

// Activation workspace for `total` rows (grown, never shrunk).
static mlpf_status ensure_acts(Trainer& t, int32_t total) {
    if ((size_t)total > t.cap_rows) {
        const size_t rows = std::max<size_t>(total, t.cap_rows * 5 / 4);
        if (t.act) cudaFree(t.act);
        t.act = nullptr;
        t.cap_rows = 0;
        const size_t n = acts_layout(t.m.cfg, rows, nullptr, nullptr);
        TCK(cudaMalloc(&t.act, n * sizeof(float)));
        t.cap_rows = rows;
        t.act_floats = n;
    }
    return ensure_h16(t);
}

// Reads and clears the device status word (after a synchronization): MLPF_E_TIMEOUT if a
// bounded wait of a tensor-core GEMM ran out.
static mlpf_status trainer_status(Trainer& t) {
    unsigned h = 0;
    TCK(cudaMemcpy(&h, t.status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (h) {
        TCK(cudaMemset(t.status, 0, sizeof(unsigned)));
        set_error("a bounded wait in a training GEMM ran out");
        return MLPF_E_TIMEOUT;
    }
    return MLPF_OK;
}

// One step: forward, `loss` (fills a.dlog, a.draw and the loss accumulator), backward,
// optional LAMB update.
template <typename LossFn>
static mlpf_status trainer_step_impl(mlpf_trainer* tt, const float* x, const int32_t* cu, int32_t n_events,
                                     int32_t total, int32_t max_n, LossFn loss, float lr, int32_t update,
                                     float* grads_out, double* loss_out, void* stream) {
    Trainer& t = tt->t;
    cudaStream_t st = (cudaStream_t)stream;
    TCK(cudaSetDevice(t.m.device));
    t.fwd_ok = false;
    const mlpf_status rs = ensure_acts(t, total);
    if (rs != MLPF_OK) return rs;
    Acts a;
    acts_layout(t.m.cfg, t.cap_rows, &a, t.act);
    TCK(cudaMemsetAsync(t.g, 0, t.n_params * 4, st));
    TCK(cudaMemsetAsync(t.scratch, 0, (1 + 2 * t.names.size()) * sizeof(double), st));
    train_forward(t, a, x, cu, n_events, total, max_n, st);
    loss(a, st);
    train_backward(t, a, x, cu, n_events, total, max_n, st);
    if (grads_out) TCK(cudaMemcpyAsync(grads_out, t.g, t.n_params * 4, cudaMemcpyDeviceToDevice, st));
    if (update) {
        ++t.step;
        const float b1 = 0.9f, b2 = 0.999f;
        const float bc1 = 1.f - powf(b1, (float)t.step), bc2 = 1.f - powf(b2, (float)t.step);
        const size_t nt = t.names.size();
        k_lamb_moments<<<t.n_chunks, 256, 0, st>>>(t.w, t.g, t.mom, t.var, t.chunks, t.scratch + 1,
                                                   t.scratch + 1 + nt, b1, b2, 1e-6f, bc1, bc2, 0.f);
        k_lamb_apply<<<t.n_chunks, 256, 0, st>>>(t.w, t.g, t.chunks, t.scratch + 1, t.scratch + 1 + nt, lr);
    }
    TCK(cudaGetLastError());
    if (t.tc_fail) {
        t.tc_fail = false;
        set_error("a tensor-core kernel of the training step could not be launched (tensor map or head width)");
        return MLPF_E_CUDA;
    }
    if (loss_out) {
        TCK(cudaMemcpyAsync(loss_out, t.scratch, sizeof(double), cudaMemcpyDeviceToHost, st));
        TCK(cudaStreamSynchronize(st));
        return trainer_status(t);
    }
    return MLPF_OK;
}


extern "C" {

void mlpf_trainer_free(mlpf_trainer* tt) {
    if (!tt) return;
    Trainer& t = tt->t;
    cudaSetDevice(t.m.device);
    for (void* p : {(void*)t.w, (void*)t.g, (void*)t.mom, (void*)t.var, (void*)t.chunks, (void*)t.scratch,
                    (void*)t.act, (void*)t.h16, (void*)t.status})
        if (p) cudaFree(p);
    delete tt;
}

mlpf_status mlpf_trainer_create(const void* blob, size_t nbytes, int device, mlpf_trainer** out) {
    if (!blob || !out || nbytes < 48) { set_error("NULL or short blob"); return MLPF_E_INVALID; }
    *out = nullptr;
    auto* tt = new (std::nothrow) mlpf_trainer();
    if (!tt) { set_error("host allocation failed"); return MLPF_E_OOM; }
    Trainer& t = tt->t;
    t.m.device = device;
    mlpf_status s = parse_blob_into((const uint8_t*)blob, nbytes, t.m);
    if (s != MLPF_OK) { delete tt; return s; }
    const mlpf_config& c = t.m.cfg;
    if (c.d > 256 || c.ffn > 4096) { delete tt; set_error("unsupported trainer configuration"); return MLPF_E_UNSUPPORTED; }
    // parameter vector in blob order (names re-read from the blob; version 2 has an
    // arch word before the tensor count)
    {
        const uint8_t* p = (const uint8_t*)blob;
        int32_t version, h[11];
        std::memcpy(&version, p + 4, 4);
        const int nh = version == 1 ? 10 : 11;
        std::memcpy(h, p + 8, 4 * (size_t)nh);
        size_t off = 8 + 4 * (size_t)nh;
        for (int i = 0; i < h[nh - 1]; ++i) {
            char name[49];
            std::memcpy(name, p + off, 48);
            name[48] = 0;
            int32_t nd, s0, s1;
            std::memcpy(&nd, p + off + 48, 4);
            std::memcpy(&s0, p + off + 52, 4);
            std::memcpy(&s1, p + off + 56, 4);
            const size_t cnt = (size_t)s0 * (nd == 2 ? s1 : 1);
            t.names.push_back(name);
            t.shapes.push_back(nd == 2 ? std::vector<int>{s0, s1} : std::vector<int>{s0});
            t.offs.push_back(t.n_params);
            t.sizes.push_back(cnt);
            t.n_params += cnt;
            off += 60 + cnt * 4;
        }
    }
    if (cudaSetDevice(device) != cudaSuccess) { delete tt; set_error("cudaSetDevice failed"); return MLPF_E_CUDA; }
    std::vector<float> hw(t.n_params);
    for (size_t i = 0; i < t.names.size(); ++i) {
        const auto& src = t.m.host.at(t.names[i]).data;
        std::copy(src.begin(), src.end(), hw.begin() + t.offs[i]);
    }
    std::vector<int4> ch;
    for (size_t i = 0; i < t.names.size(); ++i)
        for (size_t s0 = 0; s0 < t.sizes[i]; s0 += 4096)
            ch.push_back(make_int4((int)i, (int)(t.offs[i] + s0), (int)std::min<size_t>(4096, t.sizes[i] - s0), 0));
    t.n_chunks = (int)ch.size();
    cudaError_t e = cudaSuccess;
    for (float** p : {&t.w, &t.g, &t.mom, &t.var})
        if (e == cudaSuccess) e = cudaMalloc(p, t.n_params * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&t.chunks, ch.size() * sizeof(int4));
    if (e == cudaSuccess) e = cudaMalloc(&t.scratch, (1 + 2 * t.names.size()) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&t.status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(t.status, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemcpy(t.w, hw.data(), t.n_params * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t.chunks, ch.data(), ch.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(t.mom, 0, t.n_params * 4);
    if (e == cudaSuccess) e = cudaMemset(t.var, 0, t.n_params * 4);
    if (e != cudaSuccess) {
        set_error(std::string("trainer allocation: ") + cudaGetErrorString(e));
        mlpf_trainer_free(tt);
        return e == cudaErrorMemoryAllocation ? MLPF_E_OOM : MLPF_E_CUDA;
    }
    *out = tt;
    return MLPF_OK;
}

int64_t mlpf_trainer_num_params(const mlpf_trainer* tt) { return tt ? (int64_t)tt->t.n_params : -1; }

mlpf_status mlpf_trainer_set_precision(mlpf_trainer* tt, int32_t precision) {
    if (!tt) { set_error("NULL trainer"); return MLPF_E_INVALID; }
    if (precision != MLPF_FP32 && precision != MLPF_BF16 && precision != MLPF_FP16) {
        set_error("trainer GEMM precision must be MLPF_FP32, MLPF_BF16 or MLPF_FP16");
        return MLPF_E_UNSUPPORTED;
    }
    Trainer& t = tt->t;
    t.prec = precision;
    t.fwd_ok = false;
    TCK(cudaSetDevice(t.m.device));
    gemm_tc_prepare();
    return ensure_h16(t);
}

mlpf_status mlpf_trainer_step(mlpf_trainer* tt, const float* x, const int32_t* cu, int32_t n_events,
                              int32_t total, int32_t max_n, const float* t_logits, const float* t_reg, float lr,
                              int32_t update, float* grads_out, double* loss_out, void* stream) {
    if (!tt || !x || !cu || !t_logits || !t_reg || total <= 0 || n_events <= 0 || max_n <= 0 || max_n > 65536) {
        set_error("bad trainer step arguments");
        return MLPF_E_INVALID;
    }
    if (tt->t.m.cfg.arch != 0) {
        set_error("the distillation loss is defined for the 6-class head (arch 0)");
        return MLPF_E_UNSUPPORTED;
    }
    double* acc = tt->t.scratch;
    auto loss = [&](const Acts& a, cudaStream_t st) {
        k_distill_loss<<<cdivu(total, 256), 256, 0, st>>>(a.logits, a.raw, t_logits, t_reg, x, total, 1.0f / total,
                                                          a.dlog, a.draw, acc);
    };
    return trainer_step_impl(tt, x, cu, n_events, total, max_n, loss, lr, update, grads_out, loss_out, stream);
}

mlpf_status mlpf_trainer_step_supervised(mlpf_trainer* tt, const float* x, const int32_t* cu, int32_t n_events,
                                         int32_t total, int32_t max_n, const int32_t* cls_target,
                                         const float* reg_target, float beta, float focal_gamma, float delta,
                                         float lr, int32_t update, float* grads_out, double* loss_out,
                                         void* stream) {
    if (!tt || !x || !cu || !cls_target || !reg_target || total <= 0 || n_events <= 0 || max_n <= 0 ||
        max_n > 65536 || !(beta >= 0.f) || !(focal_gamma >= 0.f) || !(delta >= 0.f)) {
        set_error("bad trainer step arguments");
        return MLPF_E_INVALID;
    }
    if (tt->t.m.cfg.arch != 1) {
        set_error("the supervised loss needs the binary + PID heads (arch 1)");
        return MLPF_E_UNSUPPORTED;
    }
    double* acc = tt->t.scratch;
    auto loss = [&](const Acts& a, cudaStream_t st) {
        k_supervised_loss<<<cdivu(total, 256), 256, 0, st>>>(a.logits, a.raw, x, cls_target, reg_target, total,
                                                             1.0f / total, beta, focal_gamma, delta, a.dlog, a.draw,
                                                             acc);
    };
    return trainer_step_impl(tt, x, cu, n_events, total, max_n, loss, lr, update, grads_out, loss_out, stream);
}

static mlpf_status check_batch(const mlpf_trainer* tt, const float* x, const int32_t* cu, int32_t n_events,
                               int32_t total, int32_t max_n) {
    if (!tt) { set_error("trainer is NULL"); return MLPF_E_INVALID; }
    if (n_events < 1 || total < 1 || max_n < 1 || max_n > 65536 || !x || !cu) {
        set_error("bad batch (the trainer needs at least one event and one element)");
        return MLPF_E_INVALID;
    }
    return MLPF_OK;
}

mlpf_status mlpf_trainer_forward(mlpf_trainer* tt, const float* x, const int32_t* cu, int32_t n_events,
                                 int32_t total, int32_t max_n, float* logits, float* raw, void* stream) {
    mlpf_status s = check_batch(tt, x, cu, n_events, total, max_n);
    if (s != MLPF_OK) return s;
    if (!logits || !raw) { set_error("NULL output"); return MLPF_E_INVALID; }
    Trainer& t = tt->t;
    cudaStream_t st = (cudaStream_t)stream;
    TCK(cudaSetDevice(t.m.device));
    t.fwd_ok = false;
    s = ensure_acts(t, total);
    if (s != MLPF_OK) return s;
    Acts a;
    acts_layout(t.m.cfg, t.cap_rows, &a, t.act);
    train_forward(t, a, x, cu, n_events, total, max_n, st);
    TCK(cudaMemcpyAsync(logits, a.logits, (size_t)total * 6 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    TCK(cudaMemcpyAsync(raw, a.raw, (size_t)total * 5 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    TCK(cudaGetLastError());
    t.fwd_ok = true;
    t.fwd_x = x;
    t.fwd_cu = cu;
    t.fwd_n = n_events;
    t.fwd_total = total;
    return MLPF_OK;
}

mlpf_status mlpf_trainer_backward(mlpf_trainer* tt, const float* x, const int32_t* cu, int32_t n_events,
                                  int32_t total, int32_t max_n, const float* dlogits, const float* draw,
                                  float* grads_out, void* stream) {
    mlpf_status s = check_batch(tt, x, cu, n_events, total, max_n);
    if (s != MLPF_OK) return s;
    if (!dlogits || !draw || !grads_out) { set_error("NULL gradient pointer"); return MLPF_E_INVALID; }
    Trainer& t = tt->t;
    if (!t.fwd_ok || t.fwd_x != x || t.fwd_cu != cu || t.fwd_n != n_events || t.fwd_total != total) {
        set_error("mlpf_trainer_backward needs the activations of mlpf_trainer_forward on the same batch "
                  "(no other forward or step in between)");
        return MLPF_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    TCK(cudaSetDevice(t.m.device));
    Acts a;
    acts_layout(t.m.cfg, t.cap_rows, &a, t.act);
    TCK(cudaMemcpyAsync(a.dlog, dlogits, (size_t)total * 6 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    TCK(cudaMemcpyAsync(a.draw, draw, (size_t)total * 5 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    TCK(cudaMemsetAsync(t.g, 0, t.n_params * 4, st));
    train_backward(t, a, x, cu, n_events, total, max_n, st);
    TCK(cudaMemcpyAsync(grads_out, t.g, t.n_params * 4, cudaMemcpyDeviceToDevice, st));
    TCK(cudaGetLastError());
    return MLPF_OK;
}

mlpf_status mlpf_trainer_params(mlpf_trainer* tt, float* get, const float* set, void* stream) {
    if (!tt) { set_error("trainer is NULL"); return MLPF_E_INVALID; }
    Trainer& t = tt->t;
    cudaStream_t st = (cudaStream_t)stream;
    TCK(cudaSetDevice(t.m.device));
    if (get) TCK(cudaMemcpyAsync(get, t.w, t.n_params * 4, cudaMemcpyDeviceToDevice, st));
    if (set) {
        TCK(cudaMemcpyAsync(t.w, set, t.n_params * 4, cudaMemcpyDeviceToDevice, st));
        t.fwd_ok = false;
    }
    return MLPF_OK;
}

mlpf_status mlpf_trainer_export(const mlpf_trainer* tt, void* blob, size_t cap, size_t* nbytes) {
    if (!tt || !nbytes) { set_error("NULL argument"); return MLPF_E_INVALID; }
    const Trainer& t = tt->t;
    const bool v2 = t.m.cfg.arch != 0;   // version 2 blobs carry the arch word
    const size_t need = (v2 ? 52 : 48) + t.names.size() * 60 + t.n_params * 4;
    *nbytes = need;
    if (!blob) return MLPF_OK;
    if (cap < need) { set_error("export buffer too small"); return MLPF_E_INVALID; }
    cudaSetDevice(t.m.device);
    std::vector<float> hw(t.n_params);
    if (cudaMemcpy(hw.data(), t.w, t.n_params * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("parameter download failed");
        return MLPF_E_CUDA;
    }
    uint8_t* p = (uint8_t*)blob;
    const mlpf_config& c = t.m.cfg;
    std::memcpy(p, "MLPF", 4);
    size_t off;
    if (v2) {
        const int32_t hdr[12] = {2, c.in_dim, c.d, c.heads, c.ffn, c.l_pid, c.l_reg, c.n_cls, c.n_reg, c.act,
                                 c.arch, (int32_t)t.names.size()};
        std::memcpy(p + 4, hdr, 48);
        off = 52;
    } else {
        const int32_t hdr[11] = {1, c.in_dim, c.d, c.heads, c.ffn, c.l_pid, c.l_reg, c.n_cls, c.n_reg, c.act,
                                 (int32_t)t.names.size()};
        std::memcpy(p + 4, hdr, 44);
        off = 48;
    }
    for (size_t i = 0; i < t.names.size(); ++i) {
        char name[48] = {0};
        std::strncpy(name, t.names[i].c_str(), 47);
        std::memcpy(p + off, name, 48);
        const int32_t rec[3] = {(int32_t)t.shapes[i].size(), t.shapes[i][0],
                                t.shapes[i].size() == 2 ? t.shapes[i][1] : 1};
        std::memcpy(p + off + 48, rec, 12);
        std::memcpy(p + off + 60, hw.data() + t.offs[i], t.sizes[i] * 4);
        off += 60 + t.sizes[i] * 4;
    }
    return MLPF_OK;
}

}  // extern "C"
