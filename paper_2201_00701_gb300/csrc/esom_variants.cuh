// The paper's alternative kernel designs, restated for sm_103a as ablation
// evidence (esom_knn_variant, esom_project_knn).  They compute what the
// library's own kernels compute, by the work split the paper compares:
//
//   k-NN (Section 4.2, "Available algorithms for k-NN"):
//   * Base: one thread per point; landmark rows read from global memory;
//     a sorted array of the k nearest, a new distance entering at its end
//     and moving towards the front past every larger one (insertion sort).
//   * Bitonic: S = next power of two >= k threads per point; each round the
//     S threads compute S distances, sort them with a bitonic network and
//     merge them into the S best so far with one bitonic comparator stage
//     and a bitonic merge, so only 2S candidates are ever held.  Here the
//     S-item blocks live in registers, one item a lane, and the network runs
//     on warp shuffles instead of shared memory.
//   Both rank the exact FP32 difference-form distances (the library's
//   dist2_row) by (distance, index), so their neighbours and distances are
//   the library's, bit for bit.
//
//   Projection (Section 4.3, "Registers"):
//   * one warp per point; the pairs u < v of the scored neighbours are
//     taken in 2x2 blocks (two u by two v) so that each loaded float4 of a
//     landmark row serves two pairs; D_uv = <X - L_u, L_v - L_u> /
//     |L_v - L_u|^2 by direct dot products (O(k^2 d) per point); privatised
//     per-lane sums reduced by warp shuffles; FP64 solve on lane 0.
//   The library's own projection instead derives D_uv from the exact
//   squared distances by the law of cosines and a table of squared landmark
//   distances (O(k^2) per point), one thread per point.  The two agree
//   within FP32 rounding, not bit for bit.
//
// Inputs are assumed finite (these are measurement variants; the library's
// own kernels define the behaviour for NaN and infinite coordinates).
#pragma once

#include "esom_fused.cuh"
#include "esom_variants.h"

namespace esom {

constexpr int kVarThreads = 256;
constexpr int kVarMaxK = 32;          // largest k of this build
constexpr int kVarWarps = kVarThreads / 32;

template <int D>
__device__ __forceinline__ void variant_point(const FusedArgs &a, long long row,
                                              float4 (&x)[D / 4]) {
    const float4 *xp = reinterpret_cast<const float4 *>(a.X) + row * (D / 4);
#pragma unroll
    for (int e = 0; e < D / 4; ++e) x[e] = centred(__ldg(xp + e), a.center, e);
}

// ---------------------------------------------------------------------------
// Base k-NN: one thread per point, insertion into a sorted array.

template <int D>
__global__ void __launch_bounds__(kVarThreads) knn_base_kernel(const FusedArgs a) {
    const long long row = (long long)blockIdx.x * kVarThreads + threadIdx.x;
    if (row >= a.n) return;
    float4 x[D / 4];
    variant_point<D>(a, row, x);
    const float4 *Lg = reinterpret_cast<const float4 *>(a.hi);
    const int k = a.k;
    float bd[kVarMaxK];
    int bi[kVarMaxK];
    int cnt = 0;
    for (int j = 0; j < a.L; ++j) {
        const float dd = dist2_row<D>(x, Lg, j);
        if (cnt == k && !(dd < bd[k - 1])) continue;
        // enter at the end, move front past larger distances; an equal
        // distance stays behind (it has the lower index)
        int p = cnt < k ? cnt++ : k - 1;
        while (p > 0 && bd[p - 1] > dd) {
            bd[p] = bd[p - 1];
            bi[p] = bi[p - 1];
            --p;
        }
        bd[p] = dd;
        bi[p] = j;
    }
    for (int t = 0; t < k; ++t) {
        a.idx[row * k + t] = bi[t];
        if (a.dist2) a.dist2[row * k + t] = bd[t];
    }
}

// ---------------------------------------------------------------------------
// Bitonic k-NN: segments of S lanes per point, one (distance, index) key a
// lane.  Keys are (distance bits << 32) | index; distances are >= 0, so key
// order is (distance, index) order.

__device__ __forceinline__ unsigned long long dist_key(float dd, int j) {
    return ((unsigned long long)__float_as_uint(dd) << 32) | (unsigned)j;
}

// one comparator stage across lanes `stride` apart: the lane keeps the
// smaller of the two keys where take_min, else the larger
__device__ __forceinline__ unsigned long long cmp_stage(unsigned long long v, int stride,
                                                        bool take_min) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, stride);
    return take_min ? (o < v ? o : v) : (o > v ? o : v);
}

// Bitonic sort of each S-lane segment (S a power of two <= 32; p = lane's
// position in its segment), ascending unless `desc`.  In the phase that
// builds sorted runs of `size`, runs whose position has bit `size` set are
// sorted the other way, so that pairs of runs form bitonic sequences.
__device__ __forceinline__ unsigned long long segment_sort(unsigned long long v, int p, int S,
                                                           bool desc) {
    for (int size = 2; size <= S; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const bool up = ((p & size) == 0) != desc;
            v = cmp_stage(v, stride, ((p & stride) == 0) == up);
        }
    return v;
}

// Bitonic sequence in each segment -> ascending.
__device__ __forceinline__ unsigned long long segment_merge(unsigned long long v, int p, int S) {
    for (int stride = S >> 1; stride > 0; stride >>= 1) v = cmp_stage(v, stride, (p & stride) == 0);
    return v;
}

template <int D>
__global__ void __launch_bounds__(kVarThreads) knn_bitonic_kernel(const FusedArgs a, int S) {
    const long long g = (long long)blockIdx.x * kVarThreads + threadIdx.x;
    // segments of a warp are consecutive points: a warp leaves as a whole
    if ((g & ~31ll) / S >= a.n) return;
    const long long row = g / S;
    const int p = (int)(g & (S - 1));
    const bool active = row < a.n;
    float4 x[D / 4];
    variant_point<D>(a, active ? row : a.n - 1, x);
    const float4 *Lg = reinterpret_cast<const float4 *>(a.hi);
    const int L = a.L;
    auto key_of = [&](int j) -> unsigned long long {
        return (active && j < L) ? dist_key(dist2_row<D>(x, Lg, j), j) : ~0ull;
    };
    // the first S landmarks, sorted, are the best block so far
    unsigned long long best = segment_sort(key_of(p), p, S, false);
    for (int base = S; base < L; base += S) {
        // the next S, sorted descending: min(best[p], next[p]) keeps the S
        // smallest of the 2S as a bitonic sequence, which one merge sorts
        const unsigned long long nk = segment_sort(key_of(base + p), p, S, true);
        best = segment_merge(nk < best ? nk : best, p, S);
    }
    if (active && p < a.k) {
        a.idx[row * a.k + p] = (int)(unsigned)(best & 0xffffffffu);
        if (a.dist2) a.dist2[row * a.k + p] = __uint_as_float((unsigned)(best >> 32));
    }
}

// ---------------------------------------------------------------------------
// Registers projection: one warp per point.

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__device__ __forceinline__ float dot4(float4 a, float4 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

__device__ __forceinline__ float4 sub4(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}

// One pair's share of the 2-D normal system (Section 3.1 step 3): the 2-D
// direction h = l_v - l_u, weight w = s_u s_v |h|^-2adjust, the point's
// coordinate D_uv on the line, and the terms (w / |h|^2) h h^T and
// w ((h . (l_u - l_0)) / |h|^2 + D_uv) h with 2-D positions relative to the
// nearest neighbour's l_0.
struct PairAcc {
    float a00, a01, a11, b0, b1;
};

__device__ __forceinline__ void add_pair(PairAcc &s, float p, float q, float2 lu, float2 lv,
                                         float2 l0, float su, float sv, float adjust) {
    const float hx = lv.x - lu.x, hy = lv.y - lu.y;
    const float r = fmaf(hx, hx, hy * hy);
    if (!(q > 0.f && r > 0.f)) return;
    const float ir = 1.0f / r;
    const float w = su * sv * (adjust == 1.f ? ir : exp2f(-adjust * log2f(r)));
    const float wr = w * ir;
    const float Duv = p / q;
    const float rhs = fmaf(fmaf(hx, lu.x - l0.x, hy * (lu.y - l0.y)), ir, Duv);
    s.a00 = fmaf(wr * hx, hx, s.a00);
    s.a01 = fmaf(wr * hx, hy, s.a01);
    s.a11 = fmaf(wr * hy, hy, s.a11);
    s.b0 = fmaf(w * rhs, hx, s.b0);
    s.b1 = fmaf(w * rhs, hy, s.b1);
}

template <int D>
__global__ void __launch_bounds__(kVarThreads) project_registers_kernel(const FusedArgs a) {
    __shared__ float s_ss[kVarWarps][kVarMaxK];
    __shared__ int s_ix[kVarWarps][kVarMaxK];
    __shared__ uint32_t s_nb[kVarWarps][kVarMaxK / 2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long row = (long long)blockIdx.x * kVarWarps + warp;
    if (row >= a.n) return;  // whole warps
    const unsigned full = 0xffffffffu;
    const int k = a.k, m = k - 1;
    const float4 *Lg = reinterpret_cast<const float4 *>(a.hi);
    const float2 *lo2 = reinterpret_cast<const float2 *>(a.lo);

    // neighbour t on lane t
    const bool have = lane < k;
    const int it = have ? min(max(a.idx[row * k + lane], 0), a.L - 1) : 0;
    const float dt = have ? a.dist2[row * k + lane] : 0.f;

    // Step 2: scores.  Mean and spread of the Euclidean distances of the m
    // scored neighbours with weights 1/(t+1); the exponential relative to
    // the nearest (a common factor that cancels in the solve) times the
    // cut-off that falls to 0 at the k-th.
    const float del = dt > 0.f ? sqrtf(dt) : 0.f;
    const float wt = lane < m ? 1.0f / (float)(lane + 1) : 0.f;
    const float wsum = warp_sum(wt);
    const float mean = warp_sum(wt * del) / wsum;
    const float dev = del - mean;
    const float sigma = sqrtf(warp_sum(wt * dev * dev) / wsum);
    const float d0 = __shfl_sync(full, del, 0), dk = __shfl_sync(full, del, k - 1);
    const bool flat = sigma <= kSigmaEps * fmaxf(mean, 1e-30f);
    const float inv_sigma = flat ? 0.f : a.boost / sigma;
    const float inv_dk = dk > 0.f ? 1.0f / dk : 0.f;
    float st = 0.f;
    if (lane < m) {
        const float f1 = flat ? 1.f : expf((d0 - del) * inv_sigma);
        const float z = kScoreEdge * (del * inv_dk - 1.f);
        const float f2 = dk > 0.f ? -expm1f(z) : 1.f;
        st = f1 * f2;
    }
    s_ss[warp][lane] = st;
    s_ix[warp][lane] = it;
    const int inext = __shfl_down_sync(full, it, 1);
    if ((lane & 1) == 0 && lane < kVarMaxK)
        s_nb[warp][lane >> 1] = (uint32_t)it | ((uint32_t)inext << 16);

    // 2-D positions relative to the nearest neighbour's
    const float2 l0 = lo2[__shfl_sync(full, it, 0)];
    __syncwarp();

    // Step 3: pairs u < v < m in blocks of two u by two v, the blocks of the
    // upper triangle dealt to the lanes in turn.
    const float4 *xp = reinterpret_cast<const float4 *>(a.X) + row * (D / 4);
    const int G = (m + 1) / 2;
    const int nblk = G * (G + 1) / 2;
    PairAcc acc = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int b = lane; b < nblk; b += 32) {
        int ga = 0, rem = b;
        while (rem >= G - ga) {
            rem -= G - ga;
            ++ga;
        }
        const int u[2] = {2 * ga, 2 * ga + 1};
        const int v[2] = {2 * (ga + rem), 2 * (ga + rem) + 1};
        int iu[2], iv[2], fu[2], fv[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            iu[c] = s_ix[warp][u[c]];
            iv[c] = s_ix[warp][v[c]];
            fu[c] = swz(D, iu[c]);
            fv[c] = swz(D, iv[c]);
        }
        float P[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, Q[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 4
        for (int e = 0; e < D / 4; ++e) {
            const float4 x4 = centred(__ldg(xp + e), a.center, e);
            float4 lu[2], lv[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                lu[c] = __ldg(Lg + (size_t)iu[c] * (D / 4) + (e ^ fu[c]));
                lv[c] = __ldg(Lg + (size_t)iv[c] * (D / 4) + (e ^ fv[c]));
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const float4 g = sub4(x4, lu[i]);
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const float4 h = sub4(lv[j], lu[i]);
                    P[i][j] += dot4(g, h);
                    Q[i][j] += dot4(h, h);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
                if (u[i] < v[j] && v[j] < m)
                    add_pair(acc, P[i][j], Q[i][j], lo2[iu[i]], lo2[iv[j]], l0,
                             s_ss[warp][u[i]], s_ss[warp][v[j]], a.adjust);
    }
    const float A00 = warp_sum(acc.a00), A01 = warp_sum(acc.a01), A11 = warp_sum(acc.a11);
    const float B0 = warp_sum(acc.b0), B1 = warp_sum(acc.b1);

    // Step 4: FP64 solve (the sums are the same on every lane); an
    // ill-conditioned system is recomputed in FP64 by the whole warp
    const double a00 = A00, a01 = A01, a11 = A11, b0 = B0, b1 = B1;
    const double det = a00 * a11 - a01 * a01;
    const double tr = a00 + a11;
    if (det > kDetRefine * tr * tr) {
        if (lane == 0)
            reinterpret_cast<float2 *>(a.out)[row] =
                make_float2((float)((b0 * a11 - a01 * b1) / det + (double)l0.x),
                            (float)((a00 * b1 - a01 * b0) / det + (double)l0.y));
    } else {
        const float2 r = refine_warp_point<D, kVarMaxK>(a.X, row, a.center, Lg, lo2, a.L, a.k,
                                                        a.boost, a.adjust);
        if (lane == 0) reinterpret_cast<float2 *>(a.out)[row] = r;
    }
}

template <int D>
cudaError_t launch_knn_base(const FusedArgs &a, cudaStream_t stream) {
    const long long blocks = (a.n + kVarThreads - 1) / kVarThreads;
    knn_base_kernel<D><<<(unsigned)blocks, kVarThreads, 0, stream>>>(a);
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_knn_bitonic(const FusedArgs &a, cudaStream_t stream) {
    const int S = next_pow2(a.k);
    const long long blocks = (a.n * S + kVarThreads - 1) / kVarThreads;
    knn_bitonic_kernel<D><<<(unsigned)blocks, kVarThreads, 0, stream>>>(a, S);
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_project_registers(const FusedArgs &a, cudaStream_t stream) {
    const long long blocks = (a.n + kVarWarps - 1) / kVarWarps;
    project_registers_kernel<D><<<(unsigned)blocks, kVarThreads, 0, stream>>>(a);
    return cudaGetLastError();
}

#define ESOM_DEFINE_VARIANTS(DV)                                                          \
    const VariantOps *variant_ops_d##DV() {                                               \
        static const VariantOps ops = {&launch_knn_base<DV>, &launch_knn_bitonic<DV>,     \
                                       &launch_project_registers<DV>};                    \
        return &ops;                                                                      \
    }

}  // namespace esom
