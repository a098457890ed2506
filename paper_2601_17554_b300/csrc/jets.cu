// Anti-kt jets of every event's reconstructed particles (the event-level step
// after the reconstruction: the paper clusters jets from the (ML)PF candidates
// with the anti-kt algorithm, R = 0.4 or 0.8, Sec. 3.3 and Sec. 6.2; no PUPPI
// weights, which need vertex information).
//
// Definitions (Cacciari, Salam, Soyez, JHEP 04 (2008) 063): particles are the
// elements with class != 0, pT > 0 and (sin phi, cos phi) != 0, massless;
// d_ij = min(pT_i^-2, pT_j^-2) dR_ij^2 / R^2, d_iB = pT_i^-2, dR^2 = dy^2 + dphi^2;
// the smallest distance either merges i and j (4-vector sum) or makes i a jet.
//
// One CTA per event.  Nearest-neighbour bookkeeping (Cacciari and Salam, "Dispelling
// the N^3 myth for the kt jet-finder", Phys. Lett. B 641 (2006) 57): if (a, b) is the
// pair of smallest d_ij with pT_a^-2 <= pT_b^-2, b is a's geometric nearest
// neighbour, so the smallest of all distances is min_i min(pT_i^-2 dR^2(i, NN_i) /
// R^2, pT_i^-2).  Each entry keeps its nearest neighbour; a step takes the block-wide
// minimum, merges or emits, and recomputes the neighbours of the entries whose
// neighbour left or moved.  Only neighbours within R count: for a pair at dR >= R,
// d_ij >= min(pT_i^-2, pT_j^-2), the softer entry's beam distance, which wins
// (ties go to the beam), so an entry without a neighbour within R takes d_iB.  The rapidity is taken from the running
// sums of E + pz = pT e^eta and E - pz = pT e^-eta (positive terms, no cancellation).
#include <cuda_runtime.h>

#include <climits>
#include <type_traits>
#include <string>

#include "internal.h"

namespace mlpf {
namespace {

constexpr int JT = 1024;        // threads per event (the per-step scans want the width:
                                // 256 threads 430 ms, 512 242 ms, 1024 166 ms per 512-event batch)
constexpr int JW = JT / 32;
constexpr int JLIST = 512;      // entries whose neighbour is recomputed in one step
// k_antikt_sm: events of at most JCAP elements keep the fields every step reads (y, phi,
// the entry distance dd, the squared distance d2 to the neighbour, the neighbour nn) in
// shared memory, 18 bytes per particle, with the particles sorted by rapidity (a pair at
// dy^2 >= R^2 is never within R, so the passes skip its azimuth and distance arithmetic);
// larger events run k_antikt on global memory, in input order.
constexpr int JCAP = 12288;
constexpr size_t kJetSmem = (size_t)JCAP * (4 * sizeof(float) + sizeof(int16_t));
constexpr int JG = 4;           // listed entries whose neighbours one block scan recomputes
constexpr int JT_SM = 1024;     // threads per event of k_antikt_sm
constexpr float kPiF = 3.14159265358979323846f;

struct JetScratch {
    float *y, *phi, *pinv, *px, *py, *ep, *em, *d2, *dd;   // per particle (local index in the event's rows)
    int *nn, *parent, *jid, *idx;
    unsigned char* act;
};

__device__ __forceinline__ float dr2(float ya, float pa, float yb, float pb) {
    const float dy = ya - yb;
    float dp = fabsf(pa - pb);
    if (dp > kPiF) dp = 2.f * kPiF - dp;
    return dy * dy + dp * dp;
}

// min(pT^-2 dR^2 / R^2, pT^-2): the entry's smallest distance (pair or beam)
__device__ __forceinline__ float entry_dist(float pinv, float d2, int nn, float inv_r2) {
    if (nn < 0) return pinv;
    const float pd = pinv * d2 * inv_r2;
    return pd < pinv ? pd : pinv;
}

__device__ __forceinline__ void argmin_pair(float& v, int& i, float ov, int oi) {
    if (ov < v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
    }
}

__device__ __forceinline__ void warp_argmin(float& v, int& i) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, off);
        const int oi = __shfl_xor_sync(0xffffffffu, i, off);
        argmin_pair(v, i, ov, oi);
    }
}

// the entry of smallest (value, index) over the block; every thread gets it
__device__ void block_argmin(float& v, int& i, float* sv, int* si) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_argmin(v, i);
    if (lane == 0) {
        sv[warp] = v;
        si[warp] = i;
    }
    __syncthreads();
    if (warp == 0) {
        v = lane < JW ? sv[lane] : INFINITY;
        i = lane < JW ? si[lane] : INT_MAX;
        warp_argmin(v, i);
        if (lane == 0) {
            sv[0] = v;
            si[0] = i;
        }
    }
    __syncthreads();
    v = sv[0];
    i = si[0];
    __syncthreads();
}

// nearest active neighbour within R of entry a over the entries m = m0, m0 + dm, ...
__device__ __forceinline__ void scan_neighbour(int a, int n, int m0, int dm, const JetScratch& S, int base,
                                               float r2, float& best, int& bj) {
    const float ya = S.y[base + a], pa = S.phi[base + a];
    best = INFINITY;
    bj = INT_MAX;
    for (int m = m0; m < n; m += dm) {
        if (m == a || !S.act[base + m]) continue;
        const float d = dr2(ya, pa, S.y[base + m], S.phi[base + m]);
        if (d < r2) argmin_pair(best, bj, d, m);
    }
}
__device__ __forceinline__ void set_neighbour(int a, float best, int bj, const JetScratch& S, int base,
                                              float inv_r2) {
    const int nn = bj == INT_MAX ? -1 : bj;
    S.nn[base + a] = nn;
    S.d2[base + a] = nn < 0 ? INFINITY : best;
    S.dd[base + a] = entry_dist(S.pinv[base + a], best, nn, inv_r2);
}
// one warp per entry
__device__ void warp_neighbour(int a, int n, const JetScratch& S, int base, float r2, float inv_r2) {
    float best;
    int bj;
    scan_neighbour(a, n, threadIdx.x & 31, 32, S, base, r2, best, bj);
    warp_argmin(best, bj);
    if ((threadIdx.x & 31) == 0) set_neighbour(a, best, bj, S, base, inv_r2);
}

__global__ void __launch_bounds__(JT) k_antikt(const float* __restrict__ reg, const int32_t* __restrict__ cls,
                                              const int32_t* __restrict__ cu, float r2, JetScratch S,
                                              float* __restrict__ jets, int32_t* __restrict__ n_jets,
                                              int32_t* __restrict__ jet_of) {
    __shared__ float sv[JW];
    __shared__ int si[JW];
    __shared__ int s_n, s_jets, s_cnt, s_over, s_j, s_beam;
    __shared__ int s_list[JLIST];
    const int ev = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = cu[ev], N = cu[ev + 1] - r0;
    if (N <= JCAP) return;   // k_antikt_sm takes this event
    const float inv_r2 = 1.f / r2;
    auto is_particle = [&](int row, float& pt, float& eta, float& s, float& c) {
        pt = reg[(size_t)row * 5];
        eta = reg[(size_t)row * 5 + 1];
        s = reg[(size_t)row * 5 + 2];
        c = reg[(size_t)row * 5 + 3];
        return cls[row] != 0 && pt > 0.f && (s * s + c * c) > 0.f;
    };
    // this event's rows of the scratch arrays (the per-step scans read them through
    // L1: keeping them in shared memory instead cost the L1 capacity and was slower)
    JetScratch L;
    L.y = S.y + r0; L.phi = S.phi + r0; L.pinv = S.pinv + r0; L.px = S.px + r0; L.py = S.py + r0;
    L.ep = S.ep + r0; L.em = S.em + r0; L.d2 = S.d2 + r0; L.dd = S.dd + r0; L.nn = S.nn + r0;
    L.parent = S.parent + r0; L.jid = S.jid + r0; L.idx = S.idx + r0; L.act = S.act + r0;
    if (tid == 0) {
        s_n = 0;
        s_jets = 0;
    }
    __syncthreads();
    // particles of the event, in input order (block-wide compaction by chunks)
    for (int c0 = 0; c0 < N; c0 += JT) {
        const int row = r0 + c0 + tid;
        bool f = false;
        float pt = 0.f, eta = 0.f, s = 0.f, c = 0.f;
        if (c0 + tid < N) {
            f = is_particle(row, pt, eta, s, c);
            if (jet_of) jet_of[row] = -1;
        }
        const unsigned b = __ballot_sync(0xffffffffu, f);
        if (lane == 0) si[warp] = __popc(b);
        __syncthreads();
        int off = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < JW; ++w) {
            off += w < warp ? si[w] : 0;
            tot += si[w];
        }
        if (f) {
            const int k = s_n + off + __popc(b & ((1u << lane) - 1u));
            const float r = sqrtf(s * s + c * c);
            const float px = pt * (c / r), py = pt * (s / r);
            L.idx[k] = row;
            L.px[k] = px;
            L.py[k] = py;
            L.ep[k] = pt * expf(eta);    // E + pz
            L.em[k] = pt * expf(-eta);   // E - pz
            L.y[k] = eta;                // massless: rapidity = pseudorapidity
            L.phi[k] = atan2f(s, c);
            L.pinv[k] = 1.f / (px * px + py * py);
            L.parent[k] = -1;
            L.jid[k] = -1;   // stays -1 only if the entry never clusters (non-finite input)
            L.act[k] = 1;
        }
        __syncthreads();
        if (tid == 0) s_n += tot;
        __syncthreads();
    }
    const int n = s_n;
    // nearest neighbours of all entries
    for (int a = warp; a < n; a += JW) warp_neighbour(a, n, L, 0, r2, inv_r2);
    __syncthreads();
    for (int step = 0; step < n; ++step) {   // every step removes one entry
        float bv = INFINITY;
        int bi = INT_MAX;
        for (int k = tid; k < n; k += JT)
            if (L.act[k]) argmin_pair(bv, bi, L.dd[k], k);
        block_argmin(bv, bi, sv, si);
        if (bi == INT_MAX) break;   // no active entry left (only for non-finite inputs)
        const int i = bi;
        if (tid == 0) {
            const int j = L.nn[i];
            const float pi = L.pinv[i];
            const bool beam = j < 0 || !(pi * L.d2[i] * inv_r2 < pi);
            s_j = j;
            s_beam = beam;
            s_cnt = 0;
            s_over = 0;
            if (beam) {   // i is a jet: (px, py, pz, E)
                const int t = s_jets++;
                float* o = jets + (size_t)(r0 + t) * 4;
                o[0] = L.px[i];
                o[1] = L.py[i];
                o[2] = 0.5f * (L.ep[i] - L.em[i]);
                o[3] = 0.5f * (L.ep[i] + L.em[i]);
                L.jid[i] = t;
                L.act[i] = 0;
            } else {      // merge into the lower index (E scheme)
                const int k = min(i, j), l = max(i, j);
                const float px = L.px[k] + L.px[l], py = L.py[k] + L.py[l];
                const float ep = L.ep[k] + L.ep[l], em = L.em[k] + L.em[l];
                L.px[k] = px;
                L.py[k] = py;
                L.ep[k] = ep;
                L.em[k] = em;
                L.y[k] = 0.5f * logf(ep / em);
                L.phi[k] = atan2f(py, px);
                L.pinv[k] = 1.f / (px * px + py * py);
                L.act[l] = 0;
                L.parent[l] = k;
                s_list[0] = k;
                s_cnt = 1;
            }
        }
        __syncthreads();
        const int j = s_j;
        const bool beam = s_beam;
        const int k = beam ? i : min(i, j);
        const float yk = L.y[k], pk = L.phi[k];
        // entries that lost their neighbour, or whose neighbour (the merged entry)
        // moved away, are listed; the others only check whether the merged entry is
        // now nearer
        for (int m = tid; m < n; m += JT) {
            if (!L.act[m] || (!beam && m == k)) continue;
            const int nm = L.nn[m];
            bool lost = beam ? nm == i : (nm == i || nm == j);
            if (lost && !beam && nm == k) {
                // the merged entry moved: still the nearest if it did not move away
                // (no other entry moved, and the entry it absorbed was not the nearest)
                const float d = dr2(L.y[m], L.phi[m], yk, pk);
                if (d < r2 && d <= L.d2[m]) {
                    L.d2[m] = d;
                    L.dd[m] = entry_dist(L.pinv[m], d, k, inv_r2);
                    lost = false;
                }
            } else if (!lost && !beam) {
                const float d = dr2(L.y[m], L.phi[m], yk, pk);
                if (d < r2 && (d < L.d2[m] || (d == L.d2[m] && k < nm))) {
                    L.nn[m] = k;
                    L.d2[m] = d;
                    L.dd[m] = entry_dist(L.pinv[m], d, k, inv_r2);
                }
            }
            if (lost) {
                const int slot = atomicAdd(&s_cnt, 1);
                if (slot < JLIST) s_list[slot] = m;
                else s_over = 1;
            }
        }
        __syncthreads();
        const int cnt = s_cnt;
        if (s_over) {
            for (int a = warp; a < n; a += JW)
                if (L.act[a]) warp_neighbour(a, n, L, 0, r2, inv_r2);
        } else if (cnt > JW) {   // one warp per entry
            for (int t = warp; t < cnt; t += JW) warp_neighbour(s_list[t], n, L, 0, r2, inv_r2);
        } else {                 // few entries: the whole block scans for each in turn
            for (int t = 0; t < cnt; ++t) {
                const int a = s_list[t];
                float best;
                int bj;
                scan_neighbour(a, n, tid, JT, L, 0, r2, best, bj);
                block_argmin(best, bj, sv, si);
                if (tid == 0) set_neighbour(a, best, bj, L, 0, inv_r2);
            }
        }
        __syncthreads();
    }
    // jet index of every particle: the entry its chain of merges ends in
    for (int m = tid; m < n; m += JT) {
        int root = m;
        while (L.parent[root] >= 0) root = L.parent[root];
        if (jet_of) jet_of[L.idx[m]] = L.jid[root];
    }
    if (tid == 0) n_jets[ev] = s_jets;
}

// The order in which the CTAs of a jet launch take the events: by element count,
// largest first (ties by event index).  One CTA per event and at most one CTA per SM
// (the shared-memory kernel), so the block scheduler hands the events out in this
// order as SMs become free: the longest-processing-time-first rule, which keeps the
// largest events off the end of the launch.  Bitonic sort of (count, event) keys in
// shared memory; a launch of more than JORDER events keeps the input order.
constexpr int JORDER = 4096;
__global__ void __launch_bounds__(1024) k_jet_order(const int32_t* __restrict__ cu, int n_events,
                                                    int32_t* __restrict__ order) {
    __shared__ unsigned long long key[JORDER];
    const int tid = threadIdx.x;
    if (n_events > JORDER) {
        for (int e = tid; e < n_events; e += blockDim.x) order[e] = e;
        return;
    }
    int M = 1;
    while (M < n_events) M <<= 1;
    for (int p = tid; p < M; p += blockDim.x) {
        // ascending keys: larger events first, then lower event index; padding last
        unsigned long long k = ~0ull;
        if (p < n_events) {
            const unsigned n = (unsigned)(cu[p + 1] - cu[p]);
            k = ((unsigned long long)(0x7fffffffu - n) << 32) | (unsigned)p;
        }
        key[p] = k;
    }
    __syncthreads();
    for (int kk = 2; kk <= M; kk <<= 1)
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int p = tid; p < M; p += blockDim.x) {
                const int q = p ^ jj;
                if (q > p) {
                    const unsigned long long a = key[p], b = key[q];
                    if ((a > b) == ((p & kk) == 0)) {
                        key[p] = b;
                        key[q] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int p = tid; p < n_events; p += blockDim.x) order[p] = (int32_t)(key[p] & 0xffffffffu);
}

// the entry of smallest (value, index) over the block, in every thread, with one
// barrier: each warp reduces the per-warp minima itself (sv is rewritten only after
// the caller's next barrier)
template <int NW>
__device__ void block_argmin_all(float& v, int& i, float* sv, int* si) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_argmin(v, i);
    if (lane == 0) {
        sv[warp] = v;
        si[warp] = i;
    }
    __syncthreads();
    v = lane < NW ? sv[lane] : INFINITY;
    i = lane < NW ? si[lane] : INT_MAX;
    warp_argmin(v, i);
}

// Anti-kt with the per-step fields in shared memory (the algorithm, order of merges
// and tie rules of k_antikt; see the top of this file).  An entry is inactive when
// its dd is NaN.  Each step: the block-wide minimum of dd (every thread carries the
// minimum over its own entries from the previous step's update pass), the merge or
// jet by thread 0, one pass in which every entry checks the merged entry and the
// entries that lost their neighbour are listed, and the neighbours of the listed
// entries recomputed, JG at a time per block scan.
template <int NT>
__global__ void __launch_bounds__(NT) k_antikt_sm(const float* __restrict__ reg, const int32_t* __restrict__ cls,
                                                 const int32_t* __restrict__ cu, float r2, JetScratch S,
                                                 float* __restrict__ jets, int32_t* __restrict__ n_jets,
                                                 int32_t* __restrict__ jet_of, const int32_t* __restrict__ order) {
    constexpr int NW = NT / 32;
    extern __shared__ float jsm[];
    float* sy = jsm;
    float* sphi = sy + JCAP;
    float* sdd = sphi + JCAP;
    float* sd2 = sdd + JCAP;
    int16_t* snn = (int16_t*)(sd2 + JCAP);
    __shared__ float sv[NW];
    __shared__ int si[NW];
    __shared__ float gv[2][NW * JG];   // group reductions, double-buffered
    __shared__ int gi[2][NW * JG];
    __shared__ int s_n, s_jets, s_cnt, s_over, s_j, s_beam;
    __shared__ int s_list[JLIST];
    __shared__ float bmin[JCAP / 32], bmax[JCAP / 32];   // y range of each block of 32 entries
    __shared__ int s_wlo[NW], s_whi[NW];                  // per warp: its lowest / highest near block
    const int ev = order[blockIdx.x], tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = cu[ev], N = cu[ev + 1] - r0;
    if (N > JCAP) return;   // k_antikt takes this event
    const float inv_r2 = 1.f / r2;
    JetScratch L;   // the cold fields in global memory (this event's rows)
    L.pinv = S.pinv + r0; L.px = S.px + r0; L.py = S.py + r0; L.ep = S.ep + r0; L.em = S.em + r0;
    L.parent = S.parent + r0; L.jid = S.jid + r0; L.idx = S.idx + r0;
    if (tid == 0) {
        s_n = 0;
        s_jets = 0;
    }
    __syncthreads();
    // the event's particles sorted by rapidity (= eta for massless particles): a warp's
    // consecutive entries are then close in y, and the per-step passes skip the distance
    // arithmetic of a whole warp whose entries are all at |dy| >= R.  Bitonic sort of
    // (key, element) over the next power of two >= N, keys +inf for the elements that are
    // not particles (they sort last), in the sdd / sd2 area (free until the neighbour pass)
    constexpr int SORTCAP = 16384;   // >= JCAP
    static_assert(SORTCAP >= JCAP && SORTCAP * 6 <= JCAP * 8, "sort area");
    float* skey = sdd;
    int16_t* sidx = (int16_t*)(sdd + SORTCAP);
    int M = 1;
    while (M < N) M <<= 1;
    for (int p = tid; p < M; p += NT) {
        float key = INFINITY;
        if (p < N) {
            const int row = r0 + p;
            const float pt = reg[(size_t)row * 5], eta = reg[(size_t)row * 5 + 1];
            const float s = reg[(size_t)row * 5 + 2], c = reg[(size_t)row * 5 + 3];
            if (cls[row] != 0 && pt > 0.f && (s * s + c * c) > 0.f) {
                key = eta == eta ? fminf(fmaxf(eta, -1e30f), 1e30f) : 0.f;
                atomicAdd(&s_n, 1);
            }
            if (jet_of) jet_of[row] = -1;
        }
        skey[p] = key;
        sidx[p] = (int16_t)p;
    }
    __syncthreads();
    for (int kk = 2; kk <= M; kk <<= 1)
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int p = tid; p < M; p += NT) {
                const int q = p ^ jj;
                if (q > p) {
                    const float a = skey[p], b = skey[q];
                    if ((a > b) == ((p & kk) == 0)) {
                        skey[p] = b;
                        skey[q] = a;
                        const int16_t t = sidx[p];
                        sidx[p] = sidx[q];
                        sidx[q] = t;
                    }
                }
            }
            __syncthreads();
        }
    const int n = s_n;
    // entry p = the p-th particle in rapidity order
    for (int p = tid; p < n; p += NT) {
        const int row = r0 + sidx[p];
        const float pt = reg[(size_t)row * 5], eta = reg[(size_t)row * 5 + 1];
        const float s = reg[(size_t)row * 5 + 2], c = reg[(size_t)row * 5 + 3];
        const float r = sqrtf(s * s + c * c);
        const float px = pt * (c / r), py = pt * (s / r);
        L.idx[p] = row;
        L.px[p] = px;
        L.py[p] = py;
        L.ep[p] = pt * expf(eta);    // E + pz
        L.em[p] = pt * expf(-eta);   // E - pz
        sy[p] = eta;                 // massless: rapidity = pseudorapidity
        sphi[p] = atan2f(s, c);
        L.pinv[p] = 1.f / (px * px + py * py);
        L.parent[p] = -1;
        L.jid[p] = -1;   // stays -1 only if the entry never clusters (non-finite input)
    }
    __syncthreads();
    for (int p = tid; p < n; p += NT) sdd[p] = 0.f;   // active (over the sort keys)
    // Blocks of 32 consecutive entries keep a conservative range of their rapidities
    // (widened when a merged entry moves, never narrowed; a y that is not finite has no
    // neighbour and is in no range).  The rescan of a group of listed entries runs over
    // the index range from the lowest to the highest block whose range comes within R
    // of one of them: the entries are sorted by rapidity, merged entries move little, so
    // that range is a small part of the event, and every thread still takes an equal
    // share of it.  Float rounding: a pair passes the dR^2 < R^2 test only if |dy| < R
    // (1 + 2^-22), below the widened R, and rounding is monotonic, so the inclusive test
    // keeps every such pair.
    const int nblk = (n + 31) >> 5;   // <= JCAP / 32 <= NT
    const float Rw = sqrtf(r2) * (1.f + 1e-5f) + 1e-6f;
    auto near1 = [&](int b, float y) { return y >= bmin[b] - Rw && y <= bmax[b] + Rw; };
    for (int b = tid; b < nblk; b += NT) {
        float lo = INFINITY, hi = -INFINITY;
        for (int m = 32 * b; m < min(n, 32 * b + 32); ++m) {
            lo = fminf(lo, sy[m]);
            hi = fmaxf(hi, sy[m]);
        }
        bmin[b] = lo;
        bmax[b] = hi;
    }
    __syncthreads();
    auto active = [&](int m) { const float d = sdd[m]; return d == d; };
    // nearest active neighbour within R of entry a over the entries m0, m0 + dm, ...
    auto scan = [&](int a, int m0, int dm, float& best, int& bj) {
        const float ya = sy[a], pa = sphi[a];
        best = INFINITY;
        bj = INT_MAX;
        for (int m = m0; m < n; m += dm) {
            if (m == a || !active(m)) continue;
            const float dy = ya - sy[m];
            if (dy * dy < r2) {   // else dR^2 >= dy^2 >= R^2
                const float d = dr2(ya, pa, sy[m], sphi[m]);
                if (d < r2) argmin_pair(best, bj, d, m);
            }
        }
    };
    auto set_nn = [&](int a, float best, int bj) {
        const int nn = bj == INT_MAX ? -1 : bj;
        snn[a] = (int16_t)nn;
        sd2[a] = nn < 0 ? INFINITY : best;
        sdd[a] = entry_dist(L.pinv[a], best, nn, inv_r2);
    };
    auto warp_nn = [&](int a) {
        float best;
        int bj;
        scan(a, lane, 32, best, bj);
        warp_argmin(best, bj);
        if (lane == 0) set_nn(a, best, bj);
    };
    // nearest neighbours of all entries (every entry is active here: dd = 0 or final)
    for (int a = warp; a < n; a += NW) warp_nn(a);
    __syncthreads();
    float bv = INFINITY;
    int bi = INT_MAX;
    for (int k = tid; k < n; k += NT) argmin_pair(bv, bi, sdd[k], k);
    int gbuf = 0;
    for (int step = 0; step < n; ++step) {   // every step removes one entry
        block_argmin_all<NW>(bv, bi, sv, si);
        if (bi == INT_MAX) break;   // no active entry left (only for non-finite inputs)
        const int i = bi;
        if (tid == 0) {
            const int j = snn[i];
            // every global field the step may need, in one round of loads (j's are i's
            // again when i has no neighbour)
            const int jj = j < 0 ? i : j;
            const float pi = L.pinv[i];
            const float pxi = L.px[i], pyi = L.py[i], epi = L.ep[i], emi = L.em[i];
            const float pxj = L.px[jj], pyj = L.py[jj], epj = L.ep[jj], emj = L.em[jj];
            const bool beam = j < 0 || !(pi * sd2[i] * inv_r2 < pi);
            s_j = j;
            s_beam = beam;
            s_cnt = 0;
            s_over = 0;
            if (beam) {   // i is a jet: (px, py, pz, E)
                const int t = s_jets++;
                float* o = jets + (size_t)(r0 + t) * 4;
                o[0] = pxi;
                o[1] = pyi;
                o[2] = 0.5f * (epi - emi);
                o[3] = 0.5f * (epi + emi);
                L.jid[i] = t;
                sdd[i] = __int_as_float(0x7fc00000);   // inactive
            } else {      // merge into the lower index (E scheme)
                const int k = min(i, j), l = max(i, j);
                const float px = pxi + pxj, py = pyi + pyj, ep = epi + epj, em = emi + emj;
                L.px[k] = px;
                L.py[k] = py;
                L.ep[k] = ep;
                L.em[k] = em;
                const float yk = 0.5f * logf(ep / em);
                sy[k] = yk;
                sphi[k] = atan2f(py, px);
                bmin[k >> 5] = fminf(bmin[k >> 5], yk);
                bmax[k >> 5] = fmaxf(bmax[k >> 5], yk);
                L.pinv[k] = 1.f / (px * px + py * py);
                sdd[l] = __int_as_float(0x7fc00000);
                L.parent[l] = k;
                s_list[0] = k;
                s_cnt = 1;
            }
        }
        __syncthreads();
        const int j = s_j;
        const bool beam = s_beam;
        const int k = beam ? i : min(i, j);
        const float yk = sy[k], pk = sphi[k];
        // entries that lost their neighbour, or whose neighbour (the merged entry) moved
        // away, are listed; the others check whether the merged entry is now nearer and
        // carry their distance into the next step's minimum
        bv = INFINITY;
        bi = INT_MAX;
        // compiled once for a jet step and once for a merge step (uniform over the step)
        auto update = [&](auto bc) {
            constexpr bool BEAM = decltype(bc)::value;
            for (int m = tid; m < n; m += NT) {
                float dm = sdd[m];
                if (!(dm == dm) || (!BEAM && m == k)) continue;
                const int nm = snn[m];
                bool lost = BEAM ? nm == i : (nm == i || nm == j);
                if constexpr (!BEAM) {
                    if (lost && nm == k) {
                        // the merged entry moved: still the nearest if it did not move away
                        // (no other entry moved, and the entry it absorbed was not the nearest)
                        const float d = dr2(sy[m], sphi[m], yk, pk);
                        if (d < r2 && d <= sd2[m]) {
                            sd2[m] = d;
                            dm = entry_dist(L.pinv[m], d, k, inv_r2);
                            sdd[m] = dm;
                            lost = false;
                        }
                    } else if (!lost) {
                        const float dy = sy[m] - yk;
                        if (dy * dy < r2) {   // else the merged entry is not within R
                            const float d = dr2(sy[m], sphi[m], yk, pk);
                            if (d < r2 && (d < sd2[m] || (d == sd2[m] && k < nm))) {
                                snn[m] = (int16_t)k;
                                sd2[m] = d;
                                dm = entry_dist(L.pinv[m], d, k, inv_r2);
                                sdd[m] = dm;
                            }
                        }
                    }
                }
                if (lost) {
                    const int slot = atomicAdd(&s_cnt, 1);
                    if (slot < JLIST) s_list[slot] = m;
                    else s_over = 1;
                } else {
                    argmin_pair(bv, bi, dm, m);
                }
            }
        };
        if (beam) update(std::true_type{});
        else update(std::false_type{});
        __syncthreads();
        const int cnt = s_cnt;
        if (s_over) {   // many entries lost their neighbour: recompute all, then the minimum
            for (int a = warp; a < n; a += NW)
                if (active(a)) warp_nn(a);
            __syncthreads();
            bv = INFINITY;
            bi = INT_MAX;
            for (int m = tid; m < n; m += NT)
                if (active(m)) argmin_pair(bv, bi, sdd[m], m);
        } else if (cnt > NW) {   // one warp per listed entry
            for (int t = warp; t < cnt; t += NW) warp_nn(s_list[t]);
            __syncthreads();
            for (int t = tid; t < cnt; t += NT) argmin_pair(bv, bi, sdd[s_list[t]], s_list[t]);
        } else {                 // JG listed entries per block scan
            for (int t0 = 0; t0 < cnt; t0 += JG) {
                int aa[JG];
                float ya[JG], pa[JG], best[JG];
                int bj[JG];
#pragma unroll
                for (int q = 0; q < JG; ++q) {
                    aa[q] = t0 + q < cnt ? s_list[t0 + q] : -1;
                    ya[q] = aa[q] >= 0 ? sy[aa[q]] : 0.f;
                    pa[q] = aa[q] >= 0 ? sphi[aa[q]] : 0.f;
                    best[q] = INFINITY;
                    bj[q] = INT_MAX;
                }
                // the listed entries' pT^-2 (global memory), loaded before the scan by the
                // thread that sets their neighbours after it
                float pin[JG];
#pragma unroll
                for (int q = 0; q < JG; ++q) pin[q] = tid == 0 && aa[q] >= 0 ? L.pinv[aa[q]] : 0.f;
                // the index range of the near blocks: per warp by ballot, then over the warps
                {
                    bool nb = false;
                    if (tid < nblk) {
#pragma unroll
                        for (int q = 0; q < JG; ++q) nb |= aa[q] >= 0 && near1(tid, ya[q]);
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, nb);
                    if (lane == 0) {
                        s_wlo[warp] = bal ? 32 * warp + __ffs(bal) - 1 : INT_MAX;
                        s_whi[warp] = bal ? 32 * warp + 31 - __clz(bal) : -1;
                    }
                }
                __syncthreads();
                int blo = lane < NW ? s_wlo[lane] : INT_MAX, bhi = lane < NW ? s_whi[lane] : -1;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    blo = min(blo, __shfl_xor_sync(0xffffffffu, blo, off));
                    bhi = max(bhi, __shfl_xor_sync(0xffffffffu, bhi, off));
                }
                const int m_end = min(n, 32 * (bhi + 1));
                const int g = min(JG, cnt - t0);
                // the scan with the group's G slots in use (most groups hold one or two
                // entries: about 1.7 entries are listed per step)
                auto scan_group = [&](auto gc) {
                    constexpr int G = decltype(gc)::value;
                    for (int m = (blo == INT_MAX ? n : 32 * blo) + tid; m < m_end; m += NT) {
                        if (!active(m)) continue;
                        const float ym = sy[m], pm = sphi[m];
#pragma unroll
                        for (int q = 0; q < G; ++q) {
                            if (aa[q] < 0 || m == aa[q]) continue;
                            const float dy = ya[q] - ym;
                            if (dy * dy < r2) {
                                const float d = dr2(ya[q], pa[q], ym, pm);
                                if (d < r2) argmin_pair(best[q], bj[q], d, m);
                            }
                        }
                    }
                };
                if (g == 1) scan_group(std::integral_constant<int, 1>{});
                else if (g == 2) scan_group(std::integral_constant<int, 2>{});
                else scan_group(std::integral_constant<int, JG>{});
#pragma unroll
                for (int q = 0; q < JG; ++q) {
                    if (q >= g) break;   // warp-uniform
                    warp_argmin(best[q], bj[q]);
                    if (lane == 0) {
                        gv[gbuf][warp * JG + q] = best[q];
                        gi[gbuf][warp * JG + q] = bj[q];
                    }
                }
                __syncthreads();
                if (warp == 0) {
#pragma unroll
                    for (int q = 0; q < JG; ++q) {
                        if (q >= g) break;
                        float v = lane < NW ? gv[gbuf][lane * JG + q] : INFINITY;
                        int ix = lane < NW ? gi[gbuf][lane * JG + q] : INT_MAX;
                        warp_argmin(v, ix);
                        if (lane == 0 && aa[q] >= 0) {
                            const int a = aa[q], nn = ix == INT_MAX ? -1 : ix;
                            const float dd = entry_dist(pin[q], v, nn, inv_r2);
                            snn[a] = (int16_t)nn;
                            sd2[a] = nn < 0 ? INFINITY : v;
                            sdd[a] = dd;
                            argmin_pair(bv, bi, dd, a);
                        }
                    }
                }
                gbuf ^= 1;
            }
        }
    }
    __syncthreads();
    // jet index of every particle: the entry its chain of merges ends in
    for (int m = tid; m < n; m += NT) {
        int root = m;
        while (L.parent[root] >= 0) root = L.parent[root];
        if (jet_of) jet_of[L.idx[m]] = L.jid[root];
    }
    if (tid == 0) n_jets[ev] = s_jets;
}

}  // namespace
}  // namespace mlpf

using namespace mlpf;

struct mlpf_model {
    Model impl;
};

extern "C" mlpf_status mlpf_cluster_jets(mlpf_model* mm, const float* reg, const int32_t* cls,
                                         const int32_t* cu_seqlens, int32_t n_events, int32_t total, float R,
                                         float* jets, int32_t* n_jets, int32_t* jet_of, void* stream) {
    if (!mm) { set_error("model is NULL"); return MLPF_E_INVALID; }
    if (n_events < 0 || total < 0) { set_error("negative size"); return MLPF_E_INVALID; }
    if (!(R > 0.f && R <= 2.f)) { set_error("jet distance parameter R must be in (0, 2]"); return MLPF_E_INVALID; }
    if (n_events > 0 && (!cu_seqlens || !n_jets)) { set_error("NULL cu_seqlens or n_jets"); return MLPF_E_INVALID; }
    if (total > 0 && (!reg || !cls || !jets)) { set_error("NULL reg, cls or jets"); return MLPF_E_INVALID; }
    if (n_events == 0) return MLPF_OK;
    Model& m = mm->impl;
    if (cudaSetDevice(m.device) != cudaSuccess) { set_error("cudaSetDevice failed"); return MLPF_E_CUDA; }
    // scratch: 13 words and 1 byte per element, then the events' launch order (one
    // word per event, 16-byte aligned), grown on demand
    const size_t cap = (size_t)(total > 0 ? total : 1);
    const size_t order_off = (cap * (13 * 4 + 1) + 15) & ~(size_t)15;
    const size_t need = order_off + (size_t)n_events * 4 + 256;
    if (m.jet_bytes < need) {
        if (m.jet_base) cudaFree(m.jet_base);
        m.jet_base = nullptr;
        m.jet_bytes = 0;
        const cudaError_t e = cudaMalloc(&m.jet_base, need);
        if (e != cudaSuccess) { set_error(std::string("jet scratch allocation: ") + cudaGetErrorString(e)); return MLPF_E_OOM; }
        m.jet_bytes = need;
    }
    float* f = (float*)m.jet_base;
    JetScratch S;
    S.y = f;
    S.phi = f + cap;
    S.pinv = f + 2 * cap;
    S.px = f + 3 * cap;
    S.py = f + 4 * cap;
    S.ep = f + 5 * cap;
    S.em = f + 6 * cap;
    S.d2 = f + 7 * cap;
    S.dd = f + 8 * cap;
    int* iw = (int*)(f + 9 * cap);
    S.nn = iw;
    S.parent = iw + cap;
    S.jid = iw + 2 * cap;
    S.idx = iw + 3 * cap;
    S.act = (unsigned char*)(iw + 4 * cap);
    int32_t* order = (int32_t*)((unsigned char*)m.jet_base + order_off);
    // events of at most JCAP elements in shared memory; larger ones (possible only when
    // the batch holds more than JCAP elements) on global memory
    k_jet_order<<<1, 1024, 0, (cudaStream_t)stream>>>(cu_seqlens, n_events, order);
    cudaFuncSetAttribute(k_antikt_sm<JT_SM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kJetSmem);
    k_antikt_sm<JT_SM><<<n_events, JT_SM, kJetSmem, (cudaStream_t)stream>>>(reg, cls, cu_seqlens, R * R, S, jets,
                                                                             n_jets, jet_of, order);
    if (total > JCAP)
        k_antikt<<<n_events, JT, 0, (cudaStream_t)stream>>>(reg, cls, cu_seqlens, R * R, S, jets, n_jets, jet_of);
    const cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) { set_error(std::string("jet kernel launch: ") + cudaGetErrorString(e)); return MLPF_E_CUDA; }
    return MLPF_OK;
}
