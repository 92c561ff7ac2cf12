// Fused EmbedSOM projection kernel for sm_103a (one launch per call).
//
// Per point (paper, Section 3.1 steps 1-4; Section 4.2 and 4.3):
//   1. k-NN over all L landmarks (squared Euclidean, ties to the lower
//      index).  The paper's GPU k-NN keeps the distances inside one fused
//      kernel instead of materialising a distance matrix (Section 4.2); so
//      does this one, and it also fuses the projection step, which the
//      paper ran as a second kernel behind an exchange buffer (Section 4.4).
//   2. scores from the sorted distances (largest for the nearest, 0 for the
//      k-th);
//   3. for each pair u < v of the k-1 scored neighbours, the coordinate D_uv
//      of the point's projection on the line L_u -> L_v and the matching
//      2-D operator d_uv, accumulated into the 2x2 normal system;
//   4. the 2x2 system solved by Cramer's rule in FP64.
//
// Work split (GB300-first, not the paper's Bitonic/Aligned kernels):
//   * one thread per point, 256 points per tile, persistent blocks striding
//     over tiles;
//   * the tile of points is copied global -> shared by one bulk TMA copy
//     (cp.async.bulk + mbarrier), prefetched one tile ahead;
//   * the landmarks (rows and squared norms) are copied by bulk TMA into
//     shared memory once per block when they fit, otherwise streamed in
//     chunks through two shared buffers; every thread reads the same
//     landmark at the same time, so each shared load is a broadcast;
//   * screening scan: |x|^2 + |l|^2 - 2 x.l in FP32 (one FMA per element),
//     packed with the landmark index into one 32-bit key (index in the low
//     mantissa bits), kept in a sorted register list of KC = k + spare
//     entries; keys below the current threshold go to a per-thread queue in
//     shared memory and are merged in warp-uniform flushes, in sorted blocks
//     of 8 with a bitonic merge network;
//   * exact re-rank: the listed candidates get their squared distance in the
//     FP32 difference form, are ordered by (distance, index), and a bound on
//     the screening error certifies that no landmark outside the list can
//     enter the k nearest; a point that fails the certificate is rescanned
//     exactly on its own;
//   * scores and the pair sums in FP32 registers (D_uv from the law of
//     cosines on the exact squared distances), 2-D coordinates relative to
//     the nearest neighbour's; only the determinant and the solve in FP64.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "esom_kernels.h"

namespace esom {

constexpr float kScoreEdge = 10.0f;     // steepness of the k-th-neighbour cut-off
constexpr float kSigmaEps = 1e-12f;     // spread below this * mean counts as zero
constexpr double kDetEps = 1e-10;       // det/trace^2 below this: rank-one solve
constexpr double kDetRefine = 1e-3;     // FP32 det/trace^2 below this: recompute in FP64
constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded mbarrier wait (2 s)
constexpr float kU = 5.9604645e-8f;     // 2^-24, unit roundoff of FP32

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy helpers (inline PTX).

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One bulk copy global -> shared, completing on `bar` (16-byte aligned
// addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The same test, but the hardware may suspend the thread until the phase
// completes, for up to 20 us, instead of answering at once: a waiting warp
// (the tensor-core kernel's producer most of all) then takes no issue slots
// from the warps that share its scheduler (measured 2.6% faster k-NN at
// d = 16, k = 20).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of `bar` to complete, giving up after `limit`
// ns (kWaitNs unless given; checked every 64 tries, so at most 64 x 20 us
// late).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit = kWaitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t it = 1; it < (1u << 28); ++it) {
        if (mbar_try_wait_sleep(bar, parity)) return true;
        if ((it & 63u) == 0 && global_ns() - t0 > limit) return false;
    }
    return false;
}

// Bulk copy of `bytes` into `dst`, split below the mbarrier transaction
// limit; the caller has armed `bar` for the total.
__device__ __forceinline__ void copy_pieces(void *dst, const void *src, uint32_t bytes,
                                            uint64_t *bar) {
    const uint32_t piece = 1u << 16;
    for (uint32_t off = 0; off < bytes; off += piece) {
        const uint32_t b = bytes - off < piece ? bytes - off : piece;
        bulk_g2s(static_cast<char *>(dst) + off, static_cast<const char *>(src) + off, b, bar);
    }
}

// Read-only global load that does not allocate in L1: for data read once
// (points, screened lists), so that it does not evict the landmark rows and
// pair-table entries other loads keep there.
__device__ __forceinline__ float4 ldg_stream(const float4 *p) {
    float4 r;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(p));
    return r;
}

// Reciprocal by the SFU (one instruction, relative error ~2^-23); used
// where a correctly rounded division is not needed.
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float log2f_fast(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float exp2f_fast(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// FP64 reciprocal: SFU seed refined by two Newton steps (full double
// precision for normal inputs), instead of the long division sequence.
__device__ __forceinline__ double drcp(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    r = r * fma(-x, r, 2.0);
    r = r * fma(-x, r, 2.0);
    return r;
}

// ---------------------------------------------------------------------------
// Screening keys: a 32-bit pattern whose high bits are the FP32 screening
// value and whose low `b` bits are the landmark index.  Read back as a float
// it is the value with its low mantissa bits replaced, so keys of different
// landmarks never tie and float min/max order them by value up to a
// relative perturbation below 2^(b-23).

__device__ __forceinline__ float make_key(float value, uint32_t j, uint32_t mask) {
    return __uint_as_float((__float_as_uint(value) & ~mask) | j);
}

// Batcher's odd-even merge sort network for any N, as a compile-time list of
// compare-exchange pairs, so that the unrolled loop indexes registers only.
template <int N>
struct SortNetwork {
    int lo[320], hi[320], count;
    constexpr SortNetwork() : lo(), hi(), count(0) {
        for (int p = 1; p < N; p += p)
            for (int k = p; k > 0; k /= 2)
                for (int j = k % p; j + k < N; j += k + k)
                    for (int i = 0; i < k; ++i)
                        if (i + j + k < N && (i + j) / (p + p) == (i + j + k) / (p + p)) {
                            lo[count] = i + j;
                            hi[count] = i + j + k;
                            ++count;
                        }
    }
};

template <int N>
__device__ __forceinline__ void key_sort(float (&a)[N]) {
    constexpr SortNetwork<N> net{};
    static_assert(net.count <= 320, "sorting network table too small");
#pragma unroll
    for (int c = 0; c < net.count; ++c) {
        const float x = a[net.lo[c]], y = a[net.hi[c]];
        a[net.lo[c]] = fminf(x, y);
        a[net.hi[c]] = fmaxf(x, y);
    }
}

template <int N>
__device__ __forceinline__ float at(const float (&a)[N], int pos) {
    float r = a[0];
#pragma unroll
    for (int t = 1; t < N; ++t)
        if (t == pos) r = a[t];
    return r;
}

// Threshold for queueing: a key at or above it cannot belong to the k
// nearest.  g is the k-th key's value widened by its quantisation; the
// screening/exact distance gap M is allowed on both sides.
__device__ __forceinline__ float push_threshold(float kth, float M, float q) {
    const float g = kth + 2.f * q * fabsf(kth);
    return g + 2.f * M + 4.f * q * (fabsf(g) + 2.f * M) + 1e-30f;
}

// Squared distance to landmark j (rows of L4, chunk-swizzled) in the FP32
// difference form with four partial sums (the exact distance that is
// reported and ranked).
template <int D>
__device__ __forceinline__ float dist2_row(const float4 (&x)[D / 4], const float4 *L4, int j) {
    const float4 *l = L4 + (size_t)j * (D / 4);
    const int f = swz(D, j);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
    for (int e = 0; e < D / 4; ++e) {
        const float4 q = l[e ^ f];
        const float dx = x[e].x - q.x, dy = x[e].y - q.y;
        const float dz = x[e].z - q.z, dw = x[e].w - q.w;
        a0 = fmaf(dx, dx, a0);
        a1 = fmaf(dy, dy, a1);
        a2 = fmaf(dz, dz, a2);
        a3 = fmaf(dw, dw, a3);
    }
    return (a0 + a1) + (a2 + a3);
}

// Screening value |x|^2 + |l|^2 - 2 x.l, accumulated as
// -2 (-(|x|^2 + |l|^2)/2 + x.l) in one FMA chain (hxx = -|x|^2/2; the
// scalings by -1/2 and -2 are exact).
template <int D>
__device__ __forceinline__ float screen_row(const float4 (&x)[D / 4], float hxx, float ll,
                                            const float4 *L4, int j) {
    const float4 *l = L4 + (size_t)j * (D / 4);
    const int f = swz(D, j);
    float a = fmaf(-0.5f, ll, hxx);
#pragma unroll
    for (int e = 0; e < D / 4; ++e) {
        const float4 q = l[e ^ f];
        a = fmaf(x[e].x, q.x, a);
        a = fmaf(x[e].y, q.y, a);
        a = fmaf(x[e].z, q.z, a);
        a = fmaf(x[e].w, q.w, a);
    }
    return -2.f * a;
}

struct ScanState {
    int qn;        // queued keys of this thread
    float thr;     // push threshold
};

__host__ __device__ constexpr int next_pow2(int x) {
    int p = 1;
    while (p < x) p += p;
    return p;
}

// keys (KC, ascending) <- the KC smallest of keys and q (8, ascending): the
// sequence [keys, +inf padding, q reversed] is bitonic, so one bitonic merge
// of its power-of-two length sorts it (compare-exchanges with the constant
// padding and those feeding only positions >= KC fold away).
template <int KC>
__device__ __forceinline__ void merge8(float (&keys)[KC], const float (&q)[8]) {
    constexpr int P = next_pow2(KC + 8);
    float s[P];
#pragma unroll
    for (int i = 0; i < P; ++i) s[i] = i < KC ? keys[i] : (i >= P - 8 ? q[P - 1 - i] : INFINITY);
#pragma unroll
    for (int len = P / 2; len >= 1; len /= 2)
#pragma unroll
        for (int i = 0; i < P; ++i)
            if ((i & len) == 0) {
                const float a = s[i], b = s[i + len];
                s[i] = fminf(a, b);
                s[i + len] = fmaxf(a, b);
            }
#pragma unroll
    for (int i = 0; i < KC; ++i) keys[i] = s[i];
}

// Merges every lane's queued keys into its list, in sorted blocks of 8 (a
// sorting network, then merge8; about half the operations of inserting the
// keys one by one), and recomputes the push threshold.
template <int KC, int QS = kThreads>
__device__ __forceinline__ void queue_flush(float (&keys)[KC], ScanState &st, const uint32_t *qk,
                                            int tid, int k, float M, float q) {
    const int mx = __reduce_max_sync(0xffffffffu, st.qn);
    for (int b = 0; b < mx; b += 8) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            v[i] = b + i < st.qn ? __uint_as_float(qk[(b + i) * QS + tid]) : INFINITY;
        key_sort<8>(v);
        merge8<KC>(keys, v);
    }
    st.qn = 0;
    st.thr = push_threshold(at<KC>(keys, k - 1), M, q);
}

// Screening values of NB consecutive landmarks j0.. of a chunk, with the NB
// FMA chains interleaved chunk by chunk (hxx = -|x|^2 / 2).  j0 is a
// multiple of 8, so the chunk swizzle of every row is known at compile time.
template <int D, int NB>
__device__ __forceinline__ void screen_block(const float4 (&x)[D / 4], float hxx,
                                             const float4 *L4, const float *Nc, int j0,
                                             float (&v)[NB]) {
#pragma unroll
    for (int jj = 0; jj < NB; ++jj) v[jj] = fmaf(-0.5f, Nc[j0 + jj], hxx);
#pragma unroll
    for (int e = 0; e < D / 4; ++e)
#pragma unroll
        for (int jj = 0; jj < NB; ++jj) {
            const float4 q = L4[(size_t)(j0 + jj) * (D / 4) + (e ^ swz(D, jj))];
            v[jj] = fmaf(x[e].x, q.x, v[jj]);
            v[jj] = fmaf(x[e].y, q.y, v[jj]);
            v[jj] = fmaf(x[e].z, q.z, v[jj]);
            v[jj] = fmaf(x[e].w, q.w, v[jj]);
        }
#pragma unroll
    for (int jj = 0; jj < NB; ++jj) v[jj] *= -2.f;
}

// Screens landmarks j_begin..cnt-1 of one shared-memory chunk (global
// indices base + j; base is a multiple of 8).  Single landmarks up to the
// next multiple of 8, then blocks of 8, then the tail; the queue is checked
// after every block and after each single-step run (at most 7 pushes).
template <int D, int KC>
__device__ __forceinline__ void push_key(float v, int jg, uint32_t mask, ScanState &st,
                                         uint32_t *qk, int tid) {
    const float key = make_key(v, (uint32_t)jg, mask);
    if (key < st.thr) {
        qk[st.qn * kThreads + tid] = __float_as_uint(key);
        ++st.qn;
    }
}

template <int D, int KC>
__device__ __forceinline__ void scan_chunk(const float4 (&x)[D / 4], float hxx, const float *Lc,
                                           const float *Nc, int j_begin, int cnt, int base,
                                           uint32_t mask, float (&keys)[KC], ScanState &st,
                                           uint32_t *qk, int tid, int k, float M, float q) {
    const float4 *L4 = reinterpret_cast<const float4 *>(Lc);
    for (int j = j_begin; j < cnt;) {
        if ((j & 7) == 0 && j + kCheck <= cnt) {
            float v[kCheck];
            screen_block<D, kCheck>(x, hxx, L4, Nc, j, v);
#pragma unroll
            for (int jj = 0; jj < kCheck; ++jj)
                push_key<D, KC>(v[jj], base + j + jj, mask, st, qk, tid);
            j += kCheck;
        } else {
            push_key<D, KC>(screen_row<D>(x, hxx, Nc[j], L4, j), base + j, mask, st, qk, tid);
            ++j;
        }
        if (__any_sync(0xffffffffu, st.qn > kQueue - kCheck))
            queue_flush<KC>(keys, st, qk, tid, k, M, q);
    }
}

// Exact k-NN of one point by a plain scan (the rare path when the screening
// certificate fails): difference-form distances, stable shift insertion.
// Out of line, on local copies, so that the hot path keeps its registers
// and its instruction footprint.
template <int D, int KK>
__device__ __noinline__ void exact_rescan(const float4 *xp, const float4 *Lg, int L, float *edp,
                                          int *eip) {
    float4 x[D / 4];
#pragma unroll
    for (int e = 0; e < D / 4; ++e) x[e] = xp[e];
    float ed[KK];
    int ei[KK];
#pragma unroll
    for (int t = 0; t < KK; ++t) {
        ed[t] = INFINITY;
        ei[t] = 0;
    }
    for (int j = 0; j < L; ++j) {
        const float d2 = dist2_row<D>(x, Lg, j);
        if (d2 < ed[KK - 1]) {
            bool c[KK];
#pragma unroll
            for (int t = 0; t < KK; ++t) c[t] = d2 < ed[t];
#pragma unroll
            for (int t = KK - 1; t > 0; --t) {
                ed[t] = c[t - 1] ? ed[t - 1] : (c[t] ? d2 : ed[t]);
                ei[t] = c[t - 1] ? ei[t - 1] : (c[t] ? j : ei[t]);
            }
            if (c[0]) {
                ed[0] = d2;
                ei[0] = j;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < KK; ++t) {
        edp[t] = ed[t];
        eip[t] = ei[t];
    }
}

// Orders cd/ci by (distance, index) with odd-even transposition passes (the
// rare path when screening left near ties out of order).  Out of line.
template <int KC>
__device__ __noinline__ void repair_order(float *cdp, int *cip) {
    float cd[KC];
    int ci[KC];
#pragma unroll
    for (int t = 0; t < KC; ++t) {
        cd[t] = cdp[t];
        ci[t] = cip[t];
    }
    for (int pass = 0; pass < KC; ++pass) {
#pragma unroll
        for (int t = 0; t + 1 < KC; ++t) {
            if ((t & 1) != (pass & 1)) continue;
            const bool sw = cd[t + 1] < cd[t] || (cd[t + 1] == cd[t] && ci[t + 1] < ci[t]);
            const float d0 = cd[t], d1 = cd[t + 1];
            const int i0 = ci[t], i1 = ci[t + 1];
            cd[t] = sw ? d1 : d0;
            cd[t + 1] = sw ? d0 : d1;
            ci[t] = sw ? i1 : i0;
            ci[t + 1] = sw ? i0 : i1;
        }
    }
#pragma unroll
    for (int t = 0; t < KC; ++t) {
        cdp[t] = cd[t];
        cip[t] = ci[t];
    }
}

// Exact re-rank of the screened list.  On return ed/ei hold the KK nearest
// listed candidates by (FP32 difference-form distance, index); returns false
// if the screening certificate fails (then the caller rescans).
// The keys come four at a time from key4(g) (keys 4g .. 4g + 3, ascending),
// so a caller can stream them from memory instead of holding all KC.
template <int D, int KC, int KK, class KEY4>
__device__ __forceinline__ bool rerank_keys(const float4 (&x)[D / 4], const KEY4 &key4,
                                            const float4 *Lg, uint32_t mask, int L, int k,
                                            float M, float q, float (&ed)[KK], int (&ei)[KK],
                                            float koff = 0.f, const int *lperm = nullptr) {
    static_assert(KC % 4 == 0, "list capacity is a multiple of 4");
    float cd[KC];
    int ci[KC];
    float last = INFINITY;
#pragma unroll
    for (int g = 0; g < KC / 4; ++g) {
        const float4 k4 = key4(g);
        const float kk[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int t = 4 * g + e;
            const bool valid = kk[e] < INFINITY;
            // (the min() only guards the row read; listed keys carry indices < L)
            const int j = valid ? min((int)(__float_as_uint(kk[e]) & mask), L - 1) : 0;
            // keys of a reordered screening carry internal positions
            ci[t] = lperm ? __ldg(lperm + j) : j;
            cd[t] = valid ? dist2_row<D>(x, Lg, ci[t]) : INFINITY;
        }
        if (g == KC / 4 - 1) last = k4.w;
    }
    // The screened order is the exact order except near ties; when it is
    // not, repair it (rare, out of line).
    bool sorted = true;
#pragma unroll
    for (int t = 0; t + 1 < KC; ++t)
        sorted = sorted && !(cd[t + 1] < cd[t] || (cd[t + 1] == cd[t] && ci[t + 1] < ci[t]));
    if (__builtin_expect(!sorted, 0)) {
        float tcd[KC];
        int tci[KC];
#pragma unroll
        for (int t = 0; t < KC; ++t) {
            tcd[t] = cd[t];
            tci[t] = ci[t];
        }
        repair_order<KC>(tcd, tci);
#pragma unroll
        for (int t = 0; t < KC; ++t) {
            cd[t] = tcd[t];
            ci[t] = tci[t];
        }
    }
#pragma unroll
    for (int t = 0; t < KK; ++t) {
        ed[t] = cd[t];
        ei[t] = ci[t];
    }
    // Every landmark left out has a key >= the last key in the list (or was
    // never queued, which push_threshold covers), so its exact distance is at
    // least last - 2q|last| - M.  Keys may be offset from distances by a
    // constant koff of the point (key = distance - koff, up to M).
    if (!(last < INFINITY)) return true;
    const float exact_k = at<KC>(cd, k - 1);
    return last - 2.f * q * fabsf(last) - M > exact_k - koff;
}

template <int D, int KC, int KK>
__device__ __forceinline__ bool rerank(const float4 (&x)[D / 4], const float (&keys)[KC],
                                       const float4 *Lg, uint32_t mask, int L, int k, float M,
                                       float q, float (&ed)[KK], int (&ei)[KK],
                                       float koff = 0.f, const int *lperm = nullptr) {
    return rerank_keys<D, KC, KK>(
        x,
        [&](int g) {
            return make_float4(keys[4 * g], keys[4 * g + 1], keys[4 * g + 2], keys[4 * g + 3]);
        },
        Lg, mask, L, k, M, q, ed, ei, koff, lperm);
}

// Writes one point's k neighbours (indices, and distances when dist2 is
// set) at row * k: 16-byte stores when k is a multiple of 4 and both arrays
// are 16-byte aligned (then every row is), else one value at a time.
template <int KK>
__device__ __forceinline__ void store_neighbours(int *idx, float *dist2, long long row, int k,
                                                 const int (&si)[KK], const float (&sd)[KK]) {
    const bool vec = (k & 3) == 0 && ((uintptr_t)idx & 15u) == 0 &&
                     ((uintptr_t)dist2 & 15u) == 0;
    if (vec) {
        int4 *ip = reinterpret_cast<int4 *>(idx + row * k);
        float4 *dp = reinterpret_cast<float4 *>(dist2 + row * k);
#pragma unroll
        for (int s = 0; s + 3 < KK; s += 4)
            if (s < k) {
                ip[s / 4] = make_int4(si[s], si[s + 1], si[s + 2], si[s + 3]);
                if (dist2) dp[s / 4] = make_float4(sd[s], sd[s + 1], sd[s + 2], sd[s + 3]);
            }
        return;
    }
#pragma unroll
    for (int s = 0; s < KK; ++s)
        if (s < k) {
            idx[row * k + s] = si[s];
            if (dist2) dist2[row * k + s] = sd[s];
        }
}

// Neighbour indices parked in this thread's own column of the queue buffer
// (32-bit words col[i * QS], QS = threads of the tile; word i holds ranks 2i
// and 2i+1 as 16-bit halves), so no other thread's words are touched.
template <int QS = kThreads>
__device__ __forceinline__ int nb_at(const uint32_t *col, int t) {
    return (int)((col[(t >> 1) * QS] >> ((t & 1) * 16)) & 0xFFFFu);
}

// ---------------------------------------------------------------------------
// Step 3: pair terms over u < v < m, accumulated into the normal system
// (A, b).  D_uv uses the law of cosines on the exact squared distances:
// <X - L_u, L_v - L_u> = (|X - L_u|^2 + |L_v - L_u|^2 - |X - L_v|^2) / 2.
// The constants of a landmark pair (pair_entry) depend only on the two
// landmarks; the handle tabulates them per landmark set (the pair table,
// built with pair_entry itself, or the table of |L_v - L_u|^2 alone for
// large L), and kernels without a table compute them from the rows.
// Every kernel that projects adds the same terms in the same order (u
// ascending, then v ascending) with pair_add, so all execution plans give
// the same bits whatever layout their neighbour data has.

// Where the pair constants come from.
enum PairMode : int {
    kPairTab2 = 0,  // a.ptab: the pair table, (1/q, 1/r) per landmark pair
    kPairTab1 = 1,  // a.qtab: q = |L_v - L_u|^2 per landmark pair
    kPairRows = 2,  // neither: q from the landmark rows in global memory
};

// |L_v - L_u|^2 in the FP32 difference form with four partial sums; the
// tables hold exactly these values (or values computed from them).  nlu is
// -L_u (so each difference is one packed add); the sums run two at a time on
// the packed FP32x2 pipe, each lane the same operation as the scalar form.
template <int D>
__device__ __forceinline__ float pair_q_neg(const float4 (&nlu)[D / 4], const float4 *Lv, int fv) {
    float2 q01 = make_float2(0.f, 0.f), q23 = make_float2(0.f, 0.f);
#pragma unroll
    for (int e = 0; e < D / 4; ++e) {
        const float4 lv = Lv[e ^ fv];
        const float2 exy = __fadd2_rn(make_float2(lv.x, lv.y), make_float2(nlu[e].x, nlu[e].y));
        const float2 ezw = __fadd2_rn(make_float2(lv.z, lv.w), make_float2(nlu[e].z, nlu[e].w));
        q01 = __ffma2_rn(exy, exy, q01);
        q23 = __ffma2_rn(ezw, ezw, q23);
    }
    return (q01.x + q01.y) + (q23.x + q23.y);
}

template <int D>
__device__ __forceinline__ float pair_q(const float4 (&lu)[D / 4], const float4 *Lv, int fv) {
    float4 nlu[D / 4];
#pragma unroll
    for (int e = 0; e < D / 4; ++e) nlu[e] = make_float4(-lu[e].x, -lu[e].y, -lu[e].z, -lu[e].w);
    return pair_q_neg<D>(nlu, Lv, fv);
}

// The constants of landmark pair (u, v) from q = |L_v - L_u|^2 and the 2-D
// operator h = l_v - l_u (absolute 2-D coordinates): (1/q, 1/|h|^2) by the
// SFU (relative error ~2^-23).  A pair that does not count (L_u = L_v, or
// l_u = l_v) gets 1/|h|^2 = 0, which zeroes its weight and so every term it
// adds; 1/q = 0 when q = 0 keeps its intermediates finite.
__device__ __forceinline__ float2 pair_entry(float qq, float hx, float hy) {
    const float r = fmaf(hx, hx, hy * hy);
    const float iq = qq > 0.f ? rcp_fast(qq) : 0.f;
    return make_float2(iq, (qq > 0.f && r > 0.f) ? rcp_fast(r) : 0.f);
}

struct NormalSys {
    float a00, a01, a11, b0, b1;
};

// One pair's terms, with u = l_u - l_0 (positions relative to the nearest
// neighbour's), h = l_v - l_u, hd = half the exact squared distances and
// e = pair_entry(...): the weight w = s_u s_v r^-adjust (1/r itself for
// adjust = 1, else by the SFU, relative error ~1e-6), D_uv, and
// w h h^T / r and w h (D_uv + <h, u>/r) added to the system.
template <bool ADJ1>
__device__ __forceinline__ void pair_add(float ux, float uy, float su, float hdu, float hx,
                                         float hy, float sv, float hdv, float2 e, float adjust,
                                         NormalSys &S) {
    const float ir = e.y;
    const float wr0 = ADJ1 ? ir : (ir > 0.f ? exp2f_fast(adjust * log2f_fast(ir)) : 0.f);
    const float w = su * sv * wr0;
    const float wr = w * ir;
    const float Duv = fmaf(hdu - hdv, e.x, 0.5f);
    const float rhs = fmaf(fmaf(hx, ux, hy * uy), ir, Duv);
    // the updates two at a time on the packed FP32x2 pipe
    const float2 h2 = make_float2(hx, hy);
    const float2 th = __fmul2_rn(make_float2(wr, wr), h2);  // (wr hx, wr hy)
    const float2 a0 = __ffma2_rn(make_float2(th.x, th.x), h2, make_float2(S.a00, S.a01));
    S.a00 = a0.x;
    S.a01 = a0.y;
    S.a11 = fmaf(th.y, hy, S.a11);
    const float wrhs = w * rhs;
    const float2 b = __ffma2_rn(make_float2(wrhs, wrhs), h2, make_float2(S.b0, S.b1));
    S.b0 = b.x;
    S.b1 = b.y;
}

template <int V> struct IntConst { static constexpr int value = V; };

// The pairs of one point whose neighbour indices sit in this thread's column
// of shared memory (nb_at) and whose scores and half distances are in
// registers (the fused and batched kernels); 2-D positions gathered from
// lo2; the pair constants from whichever table the arguments carry, else
// from the rows Lg.
template <int D, int KK, bool ADJ1, int QS = kThreads>
__device__ __forceinline__ void pair_sums_regs(const float (&hd)[KK], const float (&ss)[KK],
                                               const uint32_t *nb, int m, const float4 *Lg,
                                               const float2 *lo2, float2 l0, const FusedArgs &a,
                                               NormalSys &S) {
#pragma unroll 1
    for (int u = 0; u < m - 1; ++u) {
        const int iu = nb_at<QS>(nb, u);
        float su = ss[0], hdu = hd[0];
#pragma unroll
        for (int t = 1; t < KK; ++t)
            if (t == u) {
                su = ss[t];
                hdu = hd[t];
            }
        const float2 pu = lo2[iu];
        const float ux = pu.x - l0.x, uy = pu.y - l0.y;
        const float2 *trow = a.ptab ? a.ptab + (size_t)iu * a.L : nullptr;
        const float *qrow = a.qtab ? a.qtab + (size_t)iu * a.L : nullptr;
        const float4 *Lu = Lg + (size_t)iu * (D / 4);
        const int fu = swz(D, iu);
        float4 lu[D / 4];
#pragma unroll
        for (int e = 0; e < D / 4; ++e)
            lu[e] = (trow || qrow) ? make_float4(0.f, 0.f, 0.f, 0.f) : Lu[e ^ fu];
        // pair (u, v) for a compile-time v, so ss[v] and hd[v] stay registers
        const auto pair_v = [&](auto vc) {
            constexpr int v = decltype(vc)::value;
            if constexpr (v < KK) {
                if (v < m) {
                    const int iv = nb_at<QS>(nb, v);
                    const float2 pv = lo2[iv];
                    const float hx = pv.x - pu.x, hy = pv.y - pu.y;
                    const float2 e =
                        trow ? __ldg(trow + iv)
                             : pair_entry(qrow ? __ldg(qrow + iv)
                                               : pair_q<D>(lu, Lg + (size_t)iv * (D / 4),
                                                           swz(D, iv)),
                                          hx, hy);
                    pair_add<ADJ1>(ux, uy, su, hdu, hx, hy, ss[v], hd[v], e, a.adjust, S);
                }
            }
        };
        // v = u + 1, ..., m - 1 in ascending order: one jump to the first
        // pair of the row, then straight through (no per-slot v > u test)
        static_assert(KK <= 32, "list capacity above the pair cases");
        switch (u + 1) {
#define ESOM_PAIR_CASE(V) \
    case V:               \
        pair_v(IntConst<V>{}); \
        [[fallthrough]];
            ESOM_PAIR_CASE(1) ESOM_PAIR_CASE(2) ESOM_PAIR_CASE(3) ESOM_PAIR_CASE(4)
            ESOM_PAIR_CASE(5) ESOM_PAIR_CASE(6) ESOM_PAIR_CASE(7) ESOM_PAIR_CASE(8)
            ESOM_PAIR_CASE(9) ESOM_PAIR_CASE(10) ESOM_PAIR_CASE(11) ESOM_PAIR_CASE(12)
            ESOM_PAIR_CASE(13) ESOM_PAIR_CASE(14) ESOM_PAIR_CASE(15) ESOM_PAIR_CASE(16)
            ESOM_PAIR_CASE(17) ESOM_PAIR_CASE(18) ESOM_PAIR_CASE(19) ESOM_PAIR_CASE(20)
            ESOM_PAIR_CASE(21) ESOM_PAIR_CASE(22) ESOM_PAIR_CASE(23) ESOM_PAIR_CASE(24)
            ESOM_PAIR_CASE(25) ESOM_PAIR_CASE(26) ESOM_PAIR_CASE(27) ESOM_PAIR_CASE(28)
            ESOM_PAIR_CASE(29) ESOM_PAIR_CASE(30) ESOM_PAIR_CASE(31)
#undef ESOM_PAIR_CASE
            default:
                break;
        }
    }
}

// Stash words of the position-ordered pair table (POS): the landmark index
// in the low 16 bits, its position in the landmark order in the high 16.
__device__ __forceinline__ int stash_landmark(int w, bool pos) { return pos ? (w & 0xFFFF) : w; }
__device__ __forceinline__ int stash_column(int w, bool pos) { return pos ? (w >> 16) : w; }

// NG consecutive pairs (u, v0) .. (u, v0 + NG - 1) of the projection
// kernels' pair loop (all of them exist): the landmark indices from the
// stash column, then every table load of the group, then the pair terms.
// trow is u's table row; with POS its columns are landmark positions.
template <int NG, bool ADJ1, int MODE, int NT, bool POS>
__device__ __forceinline__ void pair_group(const float2 *sst, const int *sti, int v0,
                                           const float2 *trow, const float *qrow,
                                           const float2 *lo2, float2 pu, float ux, float uy,
                                           float2 uh, float adjust, NormalSys &S) {
    int iv[NG];
    float2 ev[NG];
#pragma unroll
    for (int j = 0; j < NG; ++j) iv[j] = sti[(v0 + j) * NT];
    // (cached in L1: the spatially ordered points of a warp share most of
    // their neighbours, so they reread the same entries)
#pragma unroll
    for (int j = 0; j < NG; ++j) {
        if (MODE == kPairTab2)
            ev[j] = __ldg(trow + stash_column(iv[j], POS));
        else
            ev[j].x = __ldg(qrow + iv[j]);
    }
#pragma unroll
    for (int j = 0; j < NG; ++j) {
        const float2 vh = sst[(v0 + j) * NT];
        const float2 pv = lo2[stash_landmark(iv[j], POS)];
        const float hx = pv.x - pu.x, hy = pv.y - pu.y;
        const float2 e = MODE == kPairTab2 ? ev[j] : pair_entry(ev[j].x, hx, hy);
        pair_add<ADJ1>(ux, uy, uh.x, uh.y, hx, hy, vh.x, vh.y, e, adjust, S);
    }
}

// The same pairs for the projection kernels, both loops at run time: each
// neighbour's score and half distance (sst, float2) and landmark index (sti)
// sit in this thread's columns of shared memory (stride NT), the 2-D
// positions in lo2; the pair constants of u's row come from the table in
// groups (pair_group) whose loads are issued before their pairs are summed
// (MODE kPairTab2 / kPairTab1), or are computed from the rows (kPairRows).
// Only the pairs u < v < m are visited, in ascending v.  With POS (table
// mode only) the stash words also carry the landmarks' positions and the
// constants come from the position-ordered table a.ptab_pos.
template <int D, bool ADJ1, int MODE, int NT, bool POS = false>
__device__ __forceinline__ void pair_sums_stash(const float2 *sst, const int *sti, int m,
                                                const float2 *lo2, float2 l0, const FusedArgs &a,
                                                NormalSys &S) {
    static_assert(!POS || MODE == kPairTab2, "positions index the pair table only");
    constexpr int G = 8;
#pragma unroll 1
    for (int u = 0; u < m - 1; ++u) {
        const float2 uh = sst[u * NT];  // (s_u, hd_u)
        const int wu = sti[u * NT];
        const int iu = stash_landmark(wu, POS);
        const float2 pu = lo2[iu];
        const float ux = pu.x - l0.x, uy = pu.y - l0.y;
        if constexpr (MODE == kPairRows) {
            const float4 *Lg = reinterpret_cast<const float4 *>(a.hi);
            const float4 *Lu = Lg + (size_t)iu * (D / 4);
            const int fu = swz(D, iu);
            float4 lu[D / 4];
#pragma unroll
            for (int e = 0; e < D / 4; ++e) lu[e] = __ldg(Lu + (e ^ fu));
#pragma unroll 1
            for (int v = u + 1; v < m; ++v) {
                const int iv = sti[v * NT];
                const float2 vh = sst[v * NT];
                const float2 pv = lo2[iv];
                const float hx = pv.x - pu.x, hy = pv.y - pu.y;
                const float qq = pair_q<D>(lu, Lg + (size_t)iv * (D / 4), swz(D, iv));
                pair_add<ADJ1>(ux, uy, uh.x, uh.y, hx, hy, vh.x, vh.y, pair_entry(qq, hx, hy),
                               a.adjust, S);
            }
        } else {
            const float2 *trow =
                MODE != kPairTab2 ? nullptr
                : POS             ? a.ptab_pos + (size_t)stash_column(wu, true) * a.L
                                  : a.ptab + (size_t)iu * a.L;
            const float *qrow = MODE == kPairTab1 ? a.qtab + (size_t)iu * a.L : nullptr;
            // whole groups of G, then one group each of 4, 2 and 1 as the
            // row's remainder asks: no slot runs past the row's last pair
            int v0 = u + 1;
#pragma unroll 1
            for (; v0 + G <= m; v0 += G)
                pair_group<G, ADJ1, MODE, NT, POS>(sst, sti, v0, trow, qrow, lo2, pu, ux, uy, uh,
                                              a.adjust, S);
            if (v0 + 4 <= m) {
                pair_group<4, ADJ1, MODE, NT, POS>(sst, sti, v0, trow, qrow, lo2, pu, ux, uy, uh,
                                              a.adjust, S);
                v0 += 4;
            }
            if (v0 + 2 <= m) {
                pair_group<2, ADJ1, MODE, NT, POS>(sst, sti, v0, trow, qrow, lo2, pu, ux, uy, uh,
                                              a.adjust, S);
                v0 += 2;
            }
            if (v0 < m)
                pair_group<1, ADJ1, MODE, NT, POS>(sst, sti, v0, trow, qrow, lo2, pu, ux, uy, uh,
                                              a.adjust, S);
        }
    }
}

// ---------------------------------------------------------------------------
// Step 2: scores from the exact squared distances of the k nearest.
// Distances are Euclidean; the weights of the mean and spread are 1/i over
// the m scored neighbours.  exp(boost (d_1 - d_i) / sigma) differs from
// exp(boost (mean - d_i) / sigma) by one common factor, which cancels in the
// solve, and it cannot overflow.  Euclidean distances by the SFU reciprocal
// square root (relative error ~2^-22, far below what the scores need).
template <int KK>
__device__ __forceinline__ void point_scores(const float (&sd)[KK], int k, float boost,
                                             float (&ss)[KK]) {
    const int m = k - 1;
    float del[KK];
#pragma unroll
    for (int t = 0; t < KK; ++t) del[t] = sd[t] > 0.f ? sd[t] * rsqrtf(sd[t]) : 0.f;
    float wsum = 0.f, mean = 0.f;
#pragma unroll
    for (int t = 0; t < KK; ++t)
        if (t < m) {
            const float w = 1.0f / (float)(t + 1);
            wsum += w;
            mean = fmaf(w, del[t], mean);
        }
    mean /= wsum;
    float var = 0.f;
#pragma unroll
    for (int t = 0; t < KK; ++t)
        if (t < m) {
            const float w = 1.0f / (float)(t + 1);
            const float dd = del[t] - mean;
            var = fmaf(w * dd, dd, var);
        }
    const float sigma = sqrtf(var / wsum);
    const float dk = at<KK>(del, k - 1);
    const bool flat = sigma <= kSigmaEps * fmaxf(mean, 1e-30f);
    const float inv_sigma = flat ? 0.f : boost / sigma;
    const float inv_dk = dk > 0.f ? 1.0f / dk : 0.f;
#pragma unroll
    for (int t = 0; t < KK; ++t) {
        float s = 0.f;
        if (t < m) {
            // SFU exponentials (relative error ~1e-6); 1 - e^z by its series
            // near z = 0, where the subtraction would cancel.
            const float f1 = flat ? 1.f : __expf((del[0] - del[t]) * inv_sigma);
            const float z = kScoreEdge * fmaf(del[t], inv_dk, -1.f);
            const float f2 = dk > 0.f ? (z > -0.03125f ? -z * fmaf(z, fmaf(z, 1.f / 6.f, 0.5f), 1.f)
                                                       : 1.f - __expf(z))
                                      : 1.f;
            s = f1 * f2;
        }
        ss[t] = s;
    }
}

// Where a point whose FP32 system is too ill-conditioned goes: its row is
// appended to a list that refine_kernel (refine_batch_kernel for the batched
// kernel) then recomputes in FP64.  Deferring it keeps the FP64 code, and
// the call it would need, out of the kernels' hot loops: a rare-path call
// there made them spill registers (measured 1.3-4x slower projections).
struct RefineSink {
    long long *list;
    unsigned *count;
    __device__ __forceinline__ void operator()(long long row) const {
        list[atomicAdd(count, 1u)] = row;
    }
};
struct BatchRefineSink {
    int2 *list;
    unsigned *count;
    int item;
    __device__ __forceinline__ void operator()(long long row) const {
        list[atomicAdd(count, 1u)] = make_int2(item, (int)row);
    }
};

// Step 4: FP64 solve of the normal system (coordinates relative to l0).  A
// system with det/trace^2 at or below kDetRefine goes to the sink (for an
// active point) and l0 stands in until the FP64 recomputation replaces it.
template <class SINK>
__device__ __forceinline__ float2 point_solve(const NormalSys &S, float2 l0, long long row,
                                              bool active, const SINK &sink) {
    const double a00 = S.a00, a01 = S.a01, a11 = S.a11, b0 = S.b0, b1 = S.b1;
    const double det = a00 * a11 - a01 * a01;
    const double tr = a00 + a11;
    if (__builtin_expect(det > kDetRefine * tr * tr, 1)) {
        const double id = drcp(det);
        const double px = (b0 * a11 - a01 * b1) * id;
        const double py = (a00 * b1 - a01 * b0) * id;
        return make_float2((float)(px + (double)l0.x), (float)(py + (double)l0.y));
    }
    if (active) sink(row);
    return l0;
}

// Steps 2-4 for one point whose landmark indices are in this thread's
// column of shared memory (nb_at(nb, t) for rank t) and whose exact squared
// distances are in sd (the fused and batched kernels).
template <int D, int KK, int QS = kThreads, class SINK>
__device__ __forceinline__ float2 project_point(const float (&sd)[KK], const uint32_t *nb,
                                                const float4 *Lg, const float2 *lo2,
                                                const FusedArgs &a, long long row, bool active,
                                                const SINK &sink) {
    const int m = a.k - 1;
    float ss[KK], hd[KK];
    point_scores<KK>(sd, a.k, a.boost, ss);
#pragma unroll
    for (int t = 0; t < KK; ++t) hd[t] = 0.5f * sd[t];
    // 2-D coordinates relative to the nearest neighbour's.
    const float2 l0 = lo2[nb_at<QS>(nb, 0)];
    NormalSys S = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (a.adjust == 1.f)
        pair_sums_regs<D, KK, true, QS>(hd, ss, nb, m, Lg, lo2, l0, a, S);
    else
        pair_sums_regs<D, KK, false, QS>(hd, ss, nb, m, Lg, lo2, l0, a, S);
    return point_solve(S, l0, row, active, sink);
}

// Steps 2-4 for one point of the projection kernels: neighbour indices and
// exact squared distances in registers (si, sd); each neighbour's score and
// half distance and its index go to this thread's stash columns sst / sti
// (stride NT) for the pair loop.
// With POS the index words also carry each landmark's position in the
// landmark order (a.ipos) for the position-ordered pair table.
template <int D, int KK, int MODE, int NT, bool POS = false, class SINK>
__device__ __forceinline__ float2 project_point_stash(const float (&sd)[KK], const int (&si)[KK],
                                                      float2 *sst, int *sti, const float2 *lo2,
                                                      const FusedArgs &a, long long row,
                                                      bool active, const SINK &sink) {
    const int m = a.k - 1;
    float ss[KK];
    point_scores<KK>(sd, a.k, a.boost, ss);
    const float2 l0 = lo2[si[0]];
#pragma unroll
    for (int t = 0; t < KK; ++t)
        if (t < m) {
            sst[t * NT] = make_float2(ss[t], 0.5f * sd[t]);
            sti[t * NT] = POS ? si[t] | (__ldg(a.ipos + si[t]) << 16) : si[t];
        }
    NormalSys S = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (a.adjust == 1.f)
        pair_sums_stash<D, true, MODE, NT, POS>(sst, sti, m, lo2, l0, a, S);
    else
        pair_sums_stash<D, false, MODE, NT, POS>(sst, sti, m, lo2, l0, a, S);
    return point_solve(S, l0, row, active, sink);
}

// ---------------------------------------------------------------------------

template <int D, int KC, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) fused_kernel(const FusedArgs a) {
    static_assert(D % 4 == 0 && D >= 4 && D <= 64, "D must be a multiple of 4 in [4, 64]");
    static_assert(KC >= 8 && KC <= 36 && KC % 4 == 0, "list capacity out of range");
    static_assert((KC - 4) / 2 <= kQueue, "neighbour indices must fit in the thread's queue column");
    constexpr int KK = KC - 4;  // largest k this capacity serves (>= 4 spare entries)
    extern __shared__ __align__(128) unsigned char smem[];
    // [0] points, [1],[2] landmarks, [3] the stall probe's (never completed)
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    volatile int &s_abort = *reinterpret_cast<int *>(smem + 64);
    float *sX = reinterpret_cast<float *>(smem + kBarrierBytes);
    const int nbufL = a.nchunks == 1 ? 1 : 2;
    const int chunk4 = (a.chunk + 3) & ~3;
    float *sL = sX + kThreads * D;                       // nbufL x chunk x D
    float *sN = sL + (size_t)nbufL * a.chunk * D;        // nbufL x chunk4 norms
    uint32_t *qk = reinterpret_cast<uint32_t *>(sN + (size_t)nbufL * chunk4);

    const int tid = threadIdx.x;
    const long long first = blockIdx.x;
    const long long my_tiles =
        first < a.ntiles ? (a.ntiles - 1 - first) / (long long)gridDim.x + 1 : 0;
    if (my_tiles == 0) return;
    const long long S = my_tiles * a.nchunks;  // chunk steps of this block (chunked mode)
    const size_t chunk_floats = (size_t)a.chunk * D;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        mbar_init(&bars[3], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    // Pending copies, tracked by thread 0 so that an abort can drain them.
    bool pendX = false, pendL0 = false, pendL1 = false;
    uint32_t parL0 = 0, parL1 = 0;
    auto issue_tile = [&](long long tile) {
        const long long r0 = tile * kThreads;
        const long long rows = a.n - r0 < kThreads ? a.n - r0 : kThreads;
        const uint32_t bytes = (uint32_t)(rows * D * sizeof(float));
        mbar_expect_tx(&bars[0], bytes);
        copy_pieces(sX, a.X + r0 * D, bytes, &bars[0]);
    };
    auto issue_chunk = [&](int c, int buf) {
        const int cnt = a.L - c * a.chunk < a.chunk ? a.L - c * a.chunk : a.chunk;
        const uint32_t rb = (uint32_t)((size_t)cnt * D * sizeof(float));
        const uint32_t nb = (uint32_t)(((cnt + 3) & ~3) * sizeof(float));
        mbar_expect_tx(&bars[1 + buf], rb + nb);
        copy_pieces(sL + buf * chunk_floats, a.hi + (size_t)c * chunk_floats, rb, &bars[1 + buf]);
        copy_pieces(sN + buf * chunk4, a.norms + (size_t)c * a.chunk, nb, &bars[1 + buf]);
    };
    if (tid == 0) {
        issue_tile(first);
        pendX = true;
        issue_chunk(0, 0);
        pendL0 = true;
        if (a.nchunks > 1 && S > 1) {
            issue_chunk(1 % a.nchunks, 1);
            pendL1 = true;
        }
    }

    uint32_t phX = 0;
    long long step = 0;
    bool ok = true;
    if (a.nchunks == 1) {
        ok = mbar_wait(&bars[1], 0);
        if (tid == 0 && ok) pendL0 = false;
    }
    const float4 *Lg = a.nchunks == 1 ? reinterpret_cast<const float4 *>(sL)
                                      : reinterpret_cast<const float4 *>(a.hi);
    const float2 *lo2 = reinterpret_cast<const float2 *>(a.lo);
    const float lmax = *a.lmax;
    const uint32_t mask = a.key_mask;
    const float q = a.key_quant;
    // |screening value - exact distance| <= kGamma (|x| + max |l|)^2: the
    // screening sum carries at most D + 2 roundings of partial sums bounded
    // by that square, plus the D-term norms |x|^2 and |l|^2 (2D), the
    // four-way difference form (D/4 + 5); 25% margin.
    constexpr float kGamma = (2.25f * D + 10.f) * kU * 1.25f;

    auto abort_block = [&]() {
        // Drain this block's own copies in flight (bounded), then leave.
        if (tid == 0) {
            atomicOr(a.status, kErrWaitTimeout);
            if (pendX) mbar_wait(&bars[0], phX);
            if (pendL0) mbar_wait(&bars[1], parL0);
            if (pendL1) mbar_wait(&bars[2], parL1);
        }
    };

    // Stall probe (tests of the timeout path only): a wait on a barrier that
    // nothing completes, bounded by stall_ns; the block then takes the same
    // abort path as for a copy that never lands (status bit, own copies
    // drained, no output written).
    if (a.stall_ns && !mbar_wait(&bars[3], 0, a.stall_ns)) s_abort = 1;

    long long tile = first;
    for (long long t = 0; t < my_tiles; ++t, tile += gridDim.x) {
        ok = mbar_wait(&bars[0], phX) && ok;
        if (!ok) s_abort = 1;
        const long long row0 = tile * kThreads;
        const int rows = (int)(a.n - row0 < kThreads ? a.n - row0 : kThreads);
        const bool active = tid < rows;
        float4 xr[D / 4];
        const float4 *xs = reinterpret_cast<const float4 *>(sX) + (size_t)tid * (D / 4);
#pragma unroll
        for (int e = 0; e < D / 4; ++e)
            xr[e] = active ? centred(xs[e], a.center, e) : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();  // point tile consumed; abort flag visible
        if (s_abort) {
            abort_block();
            return;
        }
        phX ^= 1;
        if (tid == 0) {
            pendX = false;
            if (t + 1 < my_tiles) {
                issue_tile(tile + gridDim.x);
                pendX = true;
            }
        }

        // Step 1a: screening scan.
        float xx = 0.f;
#pragma unroll
        for (int e = 0; e < D / 4; ++e) {
            xx = fmaf(xr[e].x, xr[e].x, xx);
            xx = fmaf(xr[e].y, xr[e].y, xx);
            xx = fmaf(xr[e].z, xr[e].z, xx);
            xx = fmaf(xr[e].w, xr[e].w, xx);
        }
        const float sx = sqrtf(xx) + lmax;
        const float M = kGamma * sx * sx;  // |screening value - exact distance| bound
        float keys[KC];
        ScanState st;
        st.qn = 0;
        st.thr = INFINITY;
        for (int c = 0; c < a.nchunks; ++c) {
            const int base = c * a.chunk;
            const int cnt = a.L - base < a.chunk ? a.L - base : a.chunk;
            const float *Lc = sL, *Nc = sN;
            int buf = 0;
            if (a.nchunks > 1) {
                buf = (int)(step & 1);
                const uint32_t par = (uint32_t)((step >> 1) & 1);
                if (!mbar_wait(&bars[1 + buf], par)) s_abort = 1;
                Lc = sL + buf * chunk_floats;
                Nc = sN + buf * chunk4;
            }
            int j_begin = 0;
            if (c == 0) {
                // The first KC landmarks go straight into the list, then one
                // sorting network (a chunk always holds at least KC
                // landmarks, or all of them).
                // KF = KC rounded up to 8 landmarks are screened as one
                // block and sorted; the KF - KC largest keys are dropped,
                // which the certificate covers like any key pushed out of
                // the list (they are >= its last key).
                constexpr int KF = (KC + 7) & ~7;
                const float4 *L4 = reinterpret_cast<const float4 *>(Lc);
                if (cnt >= KF) {
                    float v[KF];
                    screen_block<D, KF>(xr, -0.5f * xx, L4, Nc, 0, v);
#pragma unroll
                    for (int t2 = 0; t2 < KF; ++t2) v[t2] = make_key(v[t2], (uint32_t)t2, mask);
                    key_sort<KF>(v);
#pragma unroll
                    for (int t2 = 0; t2 < KC; ++t2) keys[t2] = v[t2];
                    j_begin = KF;
                } else {
#pragma unroll
                    for (int t2 = 0; t2 < KC; ++t2)
                        keys[t2] = t2 < cnt ? make_key(screen_row<D>(xr, -0.5f * xx, Nc[t2], L4,
                                                                     t2),
                                                       (uint32_t)t2, mask)
                                            : INFINITY;
                    key_sort<KC>(keys);
                    j_begin = KC < cnt ? KC : cnt;
                }
                st.thr = push_threshold(at<KC>(keys, a.k - 1), M, q);
            }
            scan_chunk<D, KC>(xr, -0.5f * xx, Lc, Nc, j_begin, cnt, base, mask, keys, st, qk, tid, a.k,
                              M, q);
            if (a.nchunks > 1) {
                __syncthreads();  // chunk buffer consumed; abort flag visible
                if (tid == 0) {
                    if (buf == 0) {
                        pendL0 = false;
                        parL0 ^= 1;
                    } else {
                        pendL1 = false;
                        parL1 ^= 1;
                    }
                }
                if (s_abort) {
                    abort_block();
                    return;
                }
                if (tid == 0 && step + 2 < S) {
                    issue_chunk((int)((step + 2) % a.nchunks), buf);
                    if (buf == 0)
                        pendL0 = true;
                    else
                        pendL1 = true;
                }
                ++step;
            }
        }
        queue_flush<KC>(keys, st, qk, tid, a.k, M, q);

        // Step 1b: exact re-rank of the list and its certificate.
        float sd[KK];
        int si[KK];
        const bool cert = rerank<D, KC, KK>(xr, keys, Lg, mask, a.L, a.k, M, q, sd, si);
        if (__builtin_expect(!cert, 0) && a.fail_list) {
            // deferred to rescan_kernel
            if (active) {
                atomicAdd(reinterpret_cast<unsigned *>(a.status) + 2, 1u);
                a.fail_list[atomicAdd(a.fail_count, 1u)] = row0 + tid;
            }
        } else if (__builtin_expect(!cert, 0)) {
            if (active) atomicAdd(reinterpret_cast<unsigned *>(a.status) + 2, 1u);
            float4 tx[D / 4];
            float tsd[KK];
            int tsi[KK];
#pragma unroll
            for (int e = 0; e < D / 4; ++e) tx[e] = xr[e];
            exact_rescan<D, KK>(tx, Lg, a.L, tsd, tsi);
#pragma unroll
            for (int t = 0; t < KK; ++t) {
                sd[t] = tsd[t];
                si[t] = tsi[t];
            }
        }

        if (a.mode == kKnn) {
            if (active) store_neighbours<KK>(a.idx, a.dist2, row0 + tid, a.k, si, sd);
            continue;
        }
        // The queue is empty now: park the neighbour indices in this thread's
        // own column of it (two 16-bit indices a word) to free registers for
        // the pair loop.
        uint32_t *nb = qk + tid;
#pragma unroll
        for (int s = 0; s < KK; s += 2)
            nb[(s >> 1) * kThreads] = (uint32_t)si[s] | ((uint32_t)si[s + 1] << 16);
        const float2 p = project_point<D, KK>(sd, nb, Lg, lo2, a, row0 + tid, active,
                                              RefineSink{a.refine_list, a.refine_count});
        if (active) reinterpret_cast<float2 *>(a.out)[row0 + tid] = p;
    }
}

// ---------------------------------------------------------------------------
// Batched form: several datasets of the same D and list capacity in one
// launch.  Each block takes a contiguous, cost-balanced range of the global
// tile list, so it switches dataset at most a few times; a dataset whose
// landmarks are resident is staged into shared memory when the block reaches
// its first tile, a chunked one is streamed chunk by chunk through the one
// landmark buffer.  The per-tile work is the single-launch kernel's.

template <int D, int KC, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) batch_kernel(const BatchArgs B) {
    constexpr int KK = KC - 4;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);  // [0] points, [1] landmarks
    volatile int &s_abort = *reinterpret_cast<int *>(smem + 64);
    float *sX = reinterpret_cast<float *>(smem + kBarrierBytes);
    const long long t0 = B.cta_begin[blockIdx.x], t1 = B.cta_begin[blockIdx.x + 1];
    if (t0 >= t1) return;
    // the landmark buffer holds the group's largest resident set or chunk
    int cap = 0;
    {
        const int i0 = B.tile_item[t0], i1 = B.tile_item[t1 - 1];
        for (int i = i0; i <= i1; ++i) cap = max(cap, B.items[i].chunk);
    }
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    uint32_t phX = 0, phL = 0;
    bool pendX = false, pendL = false;
    int cur = -1;  // dataset whose landmarks are resident in shared memory
    auto abort_block = [&]() {
        if (tid == 0) {
            atomicOr(B.status, kErrWaitTimeout);
            if (pendX) mbar_wait(&bars[0], phX);
            if (pendL) mbar_wait(&bars[1], phL);
        }
    };
    constexpr float kGamma = (2.25f * D + 10.f) * kU * 1.25f;

    for (long long t = t0; t < t1; ++t) {
        const int it = B.tile_item[t];
        const FusedArgs &a = B.items[it];
        const long long row0 = (t - B.tile_base[it]) * kThreads;
        const int rows = (int)(a.n - row0 < kThreads ? a.n - row0 : kThreads);
        float *sL = sX + kThreads * D;
        const int cap4 = (cap + 3) & ~3;
        float *sN = sL + (size_t)cap * D;
        uint32_t *qk = reinterpret_cast<uint32_t *>(sN + cap4);
        const size_t chunk_floats = (size_t)a.chunk * D;

        bool ok = true;
        if (a.nchunks == 1 && it != cur) {
            __syncthreads();  // the previous landmarks are no longer read
            if (tid == 0) {
                const uint32_t rb = (uint32_t)((size_t)a.L * D * sizeof(float));
                const uint32_t nb = (uint32_t)(((a.L + 3) & ~3) * sizeof(float));
                mbar_expect_tx(&bars[1], rb + nb);
                copy_pieces(sL, a.hi, rb, &bars[1]);
                copy_pieces(sN, a.norms, nb, &bars[1]);
                pendL = true;
            }
            ok = mbar_wait(&bars[1], phL);
            if (tid == 0 && ok) pendL = false;
            phL ^= 1;
            cur = it;
        }
        if (tid == 0) {
            const uint32_t bytes = (uint32_t)((size_t)rows * D * sizeof(float));
            mbar_expect_tx(&bars[0], bytes);
            copy_pieces(sX, a.X + row0 * D, bytes, &bars[0]);
            pendX = true;
        }
        ok = mbar_wait(&bars[0], phX) && ok;
        if (!ok) s_abort = 1;
        const bool active = tid < rows;
        float4 xr[D / 4];
        const float4 *xs = reinterpret_cast<const float4 *>(sX) + (size_t)tid * (D / 4);
#pragma unroll
        for (int e = 0; e < D / 4; ++e)
            xr[e] = active ? centred(xs[e], a.center, e) : make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();  // point tile consumed; abort flag visible
        if (s_abort) {
            abort_block();
            return;
        }
        phX ^= 1;
        if (tid == 0) pendX = false;

        float xx = 0.f;
#pragma unroll
        for (int e = 0; e < D / 4; ++e) {
            xx = fmaf(xr[e].x, xr[e].x, xx);
            xx = fmaf(xr[e].y, xr[e].y, xx);
            xx = fmaf(xr[e].z, xr[e].z, xx);
            xx = fmaf(xr[e].w, xr[e].w, xx);
        }
        const float sx = sqrtf(xx) + *a.lmax;
        const float M = kGamma * sx * sx;
        const uint32_t mask = a.key_mask;
        const float q = a.key_quant;
        float keys[KC];
        ScanState st;
        st.qn = 0;
        st.thr = INFINITY;
        for (int c = 0; c < a.nchunks; ++c) {
            const int base = c * a.chunk;
            const int cnt = a.L - base < a.chunk ? a.L - base : a.chunk;
            if (a.nchunks > 1) {
                __syncthreads();  // the previous chunk (or landmark set) is consumed
                if (tid == 0) {
                    const uint32_t rb = (uint32_t)((size_t)cnt * D * sizeof(float));
                    const uint32_t nb = (uint32_t)(((cnt + 3) & ~3) * sizeof(float));
                    mbar_expect_tx(&bars[1], rb + nb);
                    copy_pieces(sL, a.hi + (size_t)c * chunk_floats, rb, &bars[1]);
                    copy_pieces(sN, a.norms + (size_t)c * a.chunk, nb, &bars[1]);
                    pendL = true;
                }
                if (!mbar_wait(&bars[1], phL)) s_abort = 1;
                if (tid == 0) pendL = false;
                phL ^= 1;
                cur = -1;
            }
            int j_begin = 0;
            if (c == 0) {
                constexpr int KF = (KC + 7) & ~7;
                const float4 *L4 = reinterpret_cast<const float4 *>(sL);
                if (cnt >= KF) {
                    float v[KF];
                    screen_block<D, KF>(xr, -0.5f * xx, L4, sN, 0, v);
#pragma unroll
                    for (int t2 = 0; t2 < KF; ++t2) v[t2] = make_key(v[t2], (uint32_t)t2, mask);
                    key_sort<KF>(v);
#pragma unroll
                    for (int t2 = 0; t2 < KC; ++t2) keys[t2] = v[t2];
                    j_begin = KF;
                } else {
#pragma unroll
                    for (int t2 = 0; t2 < KC; ++t2)
                        keys[t2] = t2 < cnt ? make_key(screen_row<D>(xr, -0.5f * xx, sN[t2], L4,
                                                                     t2),
                                                       (uint32_t)t2, mask)
                                            : INFINITY;
                    key_sort<KC>(keys);
                    j_begin = KC < cnt ? KC : cnt;
                }
                st.thr = push_threshold(at<KC>(keys, a.k - 1), M, q);
            }
            scan_chunk<D, KC>(xr, -0.5f * xx, sL, sN, j_begin, cnt, base, mask, keys, st, qk, tid,
                              a.k, M, q);
        }
        if (a.nchunks > 1) {
            __syncthreads();
            if (s_abort) {
                abort_block();
                return;
            }
        }
        queue_flush<KC>(keys, st, qk, tid, a.k, M, q);

        const float4 *Lg = a.nchunks == 1 ? reinterpret_cast<const float4 *>(sL)
                                           : reinterpret_cast<const float4 *>(a.hi);
        float sd[KK];
        int si[KK];
        const bool cert = rerank<D, KC, KK>(xr, keys, Lg, mask, a.L, a.k, M, q, sd, si);
        if (__builtin_expect(!cert, 0)) {
            if (active) atomicAdd(reinterpret_cast<unsigned *>(B.status) + 2, 1u);
            float4 tx[D / 4];
            float tsd[KK];
            int tsi[KK];
#pragma unroll
            for (int e = 0; e < D / 4; ++e) tx[e] = xr[e];
            exact_rescan<D, KK>(tx, Lg, a.L, tsd, tsi);
#pragma unroll
            for (int t2 = 0; t2 < KK; ++t2) {
                sd[t2] = tsd[t2];
                si[t2] = tsi[t2];
            }
        }
        uint32_t *nb = qk + tid;
#pragma unroll
        for (int s2 = 0; s2 < KK; s2 += 2)
            nb[(s2 >> 1) * kThreads] = (uint32_t)si[s2] | ((uint32_t)si[s2 + 1] << 16);
        const float2 p = project_point<D, KK>(
            sd, nb, Lg, reinterpret_cast<const float2 *>(a.lo), a, row0 + tid, active,
            BatchRefineSink{B.refine_list, B.refine_count, it});
        if (active) reinterpret_cast<float2 *>(a.out)[row0 + tid] = p;
    }
}

// ---------------------------------------------------------------------------
// Steps 2-4 from given neighbours: one thread per point reads its k indices
// and exact squared distances (ascending, as a k-NN kernel wrote them) and
// projects.  Blocks of proj_threads(MODE); each thread keeps its
// neighbours' scores, half distances and indices in stash columns of shared
// memory for the pair loop (pair_sums_stash), with the pair constants from a
// table (the 2-D positions then copied into shared memory once per block) or
// computed from the rows in global memory (L above the tables' limit).

// Shared memory of the projection kernels: the stash columns and, with a
// table, the 2-D positions.
template <int KK, int MODE>
__device__ __forceinline__ void proj_smem_layout(unsigned char *smem, float2 **sst, int **sti,
                                                 float2 **lo) {
    constexpr int NT = proj_threads(MODE);
    unsigned char *p = smem + kBarrierBytes;
    *sst = reinterpret_cast<float2 *>(p);
    p += (size_t)KK * NT * sizeof(float2);
    *sti = reinterpret_cast<int *>(p);
    p += (size_t)KK * NT * sizeof(int);
    *lo = reinterpret_cast<float2 *>(p);
}

// Copies the 2-D positions into shared memory by bulk copies (every mode but
// kPairRows); false if the copy did not land in time (reported, drained).
template <int MODE>
__device__ __forceinline__ bool proj_stage(const FusedArgs &a, uint64_t *bar, float2 *lo) {
    if (MODE == kPairRows) return true;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        // (the handle's 2-D position buffer is padded to 16 bytes)
        const uint32_t lbytes = (uint32_t)(((size_t)a.L * 2 * sizeof(float) + 15) & ~(size_t)15);
        mbar_expect_tx(bar, lbytes);
        copy_pieces(lo, a.lo, lbytes, bar);
    }
    const bool ok = mbar_wait(bar, 0);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) {
            atomicOr(a.status, kErrWaitTimeout);
            mbar_wait(bar, 0);
        }
        return false;
    }
    return true;
}

template <int D, int KK, int MODE>
__device__ __forceinline__ void project_tiles(const FusedArgs &a, const float2 *lo2, float2 *sst,
                                              int *sti, int tid) {
    constexpr int NT = proj_threads(MODE);
    const long long ntiles = (a.n + NT - 1) / NT;
    const bool vec = (a.k & 3) == 0;  // rows of k entries are 16-byte aligned
    const long long nlist = a.rows_list ? (long long)*a.rows_count : 0;
    const long long ntl = a.rows_list ? (nlist + NT - 1) / NT : ntiles;
    for (long long tile = blockIdx.x; tile < ntl; tile += gridDim.x) {
        const long long pos = tile * NT + tid;
        const bool active = pos < (a.rows_list ? nlist : a.n);
        const long long row = !active       ? 0
                              : a.rows_list ? __ldg(a.rows_list + pos)
                              : a.perm      ? (long long)__ldg(a.perm + pos)
                                            : pos;
        float sd[KK];
        int si[KK];
        if (vec) {
            const int4 *ip = reinterpret_cast<const int4 *>(a.idx + (active ? row : 0) * a.k);
            const float4 *dp = reinterpret_cast<const float4 *>(a.dist2 + (active ? row : 0) * a.k);
#pragma unroll
            for (int t = 0; t < KK; t += 4) {
                const bool have = active && t < a.k;
                const int4 iv = have ? ip[t / 4] : make_int4(0, 0, 0, 0);
                const float4 dv = have ? dp[t / 4] : make_float4(0.f, 0.f, 0.f, 0.f);
                si[t] = iv.x;
                si[t + 1] = iv.y;
                si[t + 2] = iv.z;
                si[t + 3] = iv.w;
                sd[t] = dv.x;
                sd[t + 1] = dv.y;
                sd[t + 2] = dv.z;
                sd[t + 3] = dv.w;
            }
#pragma unroll
            for (int t = 0; t < KK; ++t) si[t] = min(max(si[t], 0), a.L - 1);
        } else {
#pragma unroll
            for (int t = 0; t < KK; ++t) {
                const bool have = active && t < a.k;
                si[t] = have ? min(max(a.idx[row * a.k + t], 0), a.L - 1) : 0;
                sd[t] = have ? a.dist2[row * a.k + t] : 0.f;
            }
        }
        const float2 p = project_point_stash<D, KK, MODE, NT>(
            sd, si, sst + tid, sti + tid, lo2, a, row, active,
            RefineSink{a.refine_list, a.refine_count});
        if (active) reinterpret_cast<float2 *>(a.out)[row] = p;
    }
}

template <int D, int KC, int MODE>
__global__ void __launch_bounds__(proj_threads(MODE), proj_min_blocks(KC)) project_kernel(const FusedArgs a) {
    constexpr int KK = KC - 4;
    constexpr int NT = proj_threads(MODE);
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    float2 *sst, *sLo;
    int *sti;
    proj_smem_layout<KK, MODE>(smem, &sst, &sti, &sLo);
    const int tid = threadIdx.x;
    const long long ntiles =
        a.rows_list ? ((long long)*a.rows_count + NT - 1) / NT : (a.n + NT - 1) / NT;
    if ((long long)blockIdx.x >= ntiles) return;
    if (!proj_stage<MODE>(a, bar, sLo)) return;
    project_tiles<D, KK, MODE>(
        a, MODE == kPairRows ? reinterpret_cast<const float2 *>(a.lo) : sLo, sst, sti, tid);
}

template <int D, int KC, int MODE>
cudaError_t launch_project(const FusedArgs &a, int grid, size_t smem, cudaStream_t stream) {
    project_kernel<D, KC, MODE><<<grid, proj_threads(MODE), smem, stream>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact re-rank of the screened lists of the tensor-core k-NN kernel: one
// thread per point (visited in the k-NN's order, a.perm, so that the
// threads of a warp read nearby rows), its KC keys from a.cand, the FP32
// difference-form distances of the listed landmarks from rows in shared
// memory (copied once per block by bulk TMA when they fit, a.nchunks == 1;
// else read from global memory), ordered by (distance, landmark index), and
// the certificate with the screening bound M = m_dot |x| max|l| + the FP32
// part (|x|^2 as the k-NN kernel summed it).  Certified lists go to a.idx /
// a.dist2; the others to a.fail_list for rescan_kernel.

template <int D, int KC, bool RES>
__device__ __forceinline__ void rerank_tiles(const FusedArgs &a, const float4 *Lg, int tid) {
    constexpr int KK = KC - 4;
    constexpr float kGamma = (2.25f * D + 10.f) * kU * 1.25f;
    const long long ntiles = (a.n + kThreads - 1) / kThreads;
    const float lmax = *a.lmax;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long pos = tile * kThreads + tid;
        const bool active = pos < a.n;
        const long long row = !active ? 0 : (a.perm ? (long long)__ldg(a.perm + pos) : pos);
        float4 xr[D / 4];
        const float4 *xp = reinterpret_cast<const float4 *>(a.X) + row * (D / 4);
        float xx = 0.f;
#pragma unroll
        for (int e = 0; e < D / 4; ++e) {
            xr[e] = active ? centred(__ldg(xp + e), a.center, e) : make_float4(0.f, 0.f, 0.f, 0.f);
            xx = fmaf(xr[e].x, xr[e].x, xx);
            xx = fmaf(xr[e].y, xr[e].y, xx);
            xx = fmaf(xr[e].z, xr[e].z, xx);
            xx = fmaf(xr[e].w, xr[e].w, xx);
        }
        const float xn = sqrtf(xx);
        const float sx = xn + lmax;
        const float M = a.m_dot * xn * lmax + 2.f * kGamma * sx * sx;
        float keys[KC];
        // (the screened lists are stored in the k-NN's visiting order)
        const float4 *cp = reinterpret_cast<const float4 *>(a.cand + (active ? pos : 0) * KC);
#pragma unroll
        for (int t = 0; t < KC; t += 4) {
            const float4 v = active ? __ldg(cp + t / 4) : make_float4(INFINITY, INFINITY, INFINITY,
                                                                     INFINITY);
            keys[t] = v.x;
            keys[t + 1] = v.y;
            keys[t + 2] = v.z;
            keys[t + 3] = v.w;
        }
        float sd[KK];
        int si[KK];
        const bool cert = rerank<D, KC, KK>(xr, keys, Lg, a.key_mask, a.L, a.k, M, a.key_quant, sd,
                                            si, xx, a.lperm);
        if (!active) continue;
        if (__builtin_expect(!cert, 0)) {
            // deferred: rescan_kernel finds this point's neighbours exactly
            atomicAdd(reinterpret_cast<unsigned *>(a.status) + 2, 1u);
            a.fail_list[atomicAdd(a.fail_count, 1u)] = row;
        }
        store_neighbours<KK>(a.idx, a.dist2, row, a.k, si, sd);
    }
}

template <int D, int KC>
__global__ void __launch_bounds__(kThreads) rerank_kernel(const FusedArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    float *sL = reinterpret_cast<float *>(smem + kBarrierBytes);
    const int tid = threadIdx.x;
    const long long ntiles = (a.n + kThreads - 1) / kThreads;
    if ((long long)blockIdx.x >= ntiles) return;
    if (a.nchunks == 1) {
        if (tid == 0) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0) {
            const uint32_t bytes = (uint32_t)((size_t)a.L * D * sizeof(float));
            mbar_expect_tx(bar, bytes);
            copy_pieces(sL, a.hi, bytes, bar);
        }
        const bool ok = mbar_wait(bar, 0);
        if (!__syncthreads_and(ok)) {
            // the copy did not land in time: report, drain it (bounded), leave
            if (tid == 0) {
                atomicOr(a.status, kErrWaitTimeout);
                mbar_wait(bar, 0);
            }
            return;
        }
        rerank_tiles<D, KC, true>(a, reinterpret_cast<const float4 *>(sL), tid);
    } else {
        rerank_tiles<D, KC, false>(a, reinterpret_cast<const float4 *>(a.hi), tid);
    }
}

template <int D, int KC>
cudaError_t launch_rerank(const FusedArgs &a, int grid, size_t smem, cudaStream_t stream) {
    rerank_kernel<D, KC><<<grid, kThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

// Exact re-rank and projection of the tensor-core k-NN's screened lists in
// one pass (the tensor-core plan of esom_project): one thread per point, in
// the k-NN's visiting order; the re-rank of rerank_tiles, then, for a
// certified list, steps 2-4 of the projection kernel with the neighbours
// still in registers, so no neighbour exchange buffer is written or read.
// The re-rank reads the landmark rows through the L1 cache.  A point whose
// certificate fails goes to a.fail_list; rescan_kernel and the projection
// kernel over that list finish it.  With the pair table in the landmark
// order (a.ptab_pos) a point's pair constants come from it: its neighbours
// sit close together in that order, so their entries of a table row share
// cache lines (same values as a.ptab, so the same bits).
template <int D, int KC, int MODE>
__global__ void __launch_bounds__(proj_threads(MODE), proj_min_blocks(KC))
    rerank_project_kernel(const FusedArgs a) {
    constexpr int KK = KC - 4;
    constexpr int NT = proj_threads(MODE);
    constexpr float kGamma = (2.25f * D + 10.f) * kU * 1.25f;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    float2 *sst, *sLo;
    int *sti;
    proj_smem_layout<KK, MODE>(smem, &sst, &sti, &sLo);
    const int tid = threadIdx.x;
    const long long ntiles = (a.n + NT - 1) / NT;
    if ((long long)blockIdx.x >= ntiles) return;
    if (!proj_stage<MODE>(a, bar, sLo)) return;
    const float2 *lo2 = MODE == kPairRows ? reinterpret_cast<const float2 *>(a.lo) : sLo;
    const float4 *Lg = reinterpret_cast<const float4 *>(a.hi);
    const float lmax = *a.lmax;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long pos = tile * NT + tid;
        const bool active = pos < a.n;
        const long long row = !active ? 0 : (a.perm ? (long long)__ldg(a.perm + pos) : pos);
        float4 xr[D / 4];
        const float4 *xp = reinterpret_cast<const float4 *>(a.X) + row * (D / 4);
        float xx = 0.f;
#pragma unroll
        for (int e = 0; e < D / 4; ++e) {
            xr[e] = active ? centred(ldg_stream(xp + e), a.center, e) : make_float4(0.f, 0.f, 0.f, 0.f);
            xx = fmaf(xr[e].x, xr[e].x, xx);
            xx = fmaf(xr[e].y, xr[e].y, xx);
            xx = fmaf(xr[e].z, xr[e].z, xx);
            xx = fmaf(xr[e].w, xr[e].w, xx);
        }
        const float xn = sqrtf(xx);
        const float sx = xn + lmax;
        const float M = a.m_dot * xn * lmax + 2.f * kGamma * sx * sx;
        // the screened keys streamed four at a time (not all KC live at once)
        const float4 *cp = reinterpret_cast<const float4 *>(a.cand + (active ? pos : 0) * KC);
        float sd[KK];
        int si[KK];
        const bool cert = rerank_keys<D, KC, KK>(
            xr,
            [&](int g) {
                return active ? ldg_stream(cp + g)
                              : make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
            },
            Lg, a.key_mask, a.L, a.k, M, a.key_quant, sd, si, xx, a.lperm);
        if (active && __builtin_expect(!cert, 0)) {
            atomicAdd(reinterpret_cast<unsigned *>(a.status) + 2, 1u);
            a.fail_list[atomicAdd(a.fail_count, 1u)] = row;
        }
        const bool proj = active && cert;
#pragma unroll
        for (int t = 0; t < KK; ++t) si[t] = min(max(si[t], 0), a.L - 1);
        float2 p;
        if (MODE == kPairTab2 && a.ptab_pos)
            p = project_point_stash<D, KK, MODE, NT, MODE == kPairTab2>(
                sd, si, sst + tid, sti + tid, lo2, a, row, proj,
                RefineSink{a.refine_list, a.refine_count});
        else
            p = project_point_stash<D, KK, MODE, NT>(sd, si, sst + tid, sti + tid, lo2, a, row,
                                                     proj,
                                                     RefineSink{a.refine_list, a.refine_count});
        if (proj) reinterpret_cast<float2 *>(a.out)[row] = p;
    }
}

template <int D, int KC, int MODE>
cudaError_t launch_rerank_project(const FusedArgs &a, int grid, size_t smem, cudaStream_t stream) {
    rerank_project_kernel<D, KC, MODE><<<grid, proj_threads(MODE), smem, stream>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact k-NN of the points whose screening certificate failed (deferred by
// the k-NN kernels to keep their warps on the fast path): FP32
// difference-form distances to all L landmarks (dist2_row, the same
// arithmetic as exact_rescan), each thread keeping the nearest KK of the
// landmarks it scans, then k rounds of a warp minimum over the lanes' heads.
// Keys are (distance bits << 32) | j: distances are >= 0, so their bit
// patterns order like the values and ties go to the lower index, as in
// exact_rescan.  With at most one failed point per block (the usual case:
// a handful of points a pass) the whole block scans one point, j = thread
// (mod 256), and warp 0 merges the eight warps' sorted lists from shared
// memory, which cuts the serial chain of landmark loads eightfold; with more,
// one warp scans each point, j = lane (mod 32).  Keys are unique, so both
// give the same neighbours.

__device__ __forceinline__ unsigned long long umin64(unsigned long long x, unsigned long long y) {
    return x < y ? x : y;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long x, unsigned long long y) {
    return x < y ? y : x;
}

// This thread's nearest KK (ascending keys) of the landmarks j0, j0 + step, ...
template <int D, int KK>
__device__ __forceinline__ void rescan_scan(const float4 (&x)[D / 4], const float4 *Lg, int L,
                                            int j0, int step, unsigned long long (&best)[KK]) {
#pragma unroll
    for (int t = 0; t < KK; ++t) best[t] = ~0ull;
    for (int j = j0; j < L; j += step) {
        const float d2 = dist2_row<D>(x, Lg, j);
        const unsigned long long key = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)j;
        if (key < best[KK - 1]) {
            unsigned long long prev = best[0];
            best[0] = umin64(key, best[0]);
#pragma unroll
            for (int t = 1; t < KK; ++t) {
                const unsigned long long cur = best[t];
                best[t] = umax64(prev, umin64(key, cur));
                prev = cur;
            }
        }
    }
}

// Round r of a warp's merge: the r-th smallest key over the lanes' lists
// (every lane gets it); the lane that held it pops its head.
template <int KK>
__device__ __forceinline__ unsigned long long warp_pop(unsigned long long (&best)[KK]) {
    unsigned long long m = best[0];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = umin64(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (best[0] == m) {  // keys are unique: one lane pops its head
#pragma unroll
        for (int t = 0; t + 1 < KK; ++t) best[t] = best[t + 1];
        best[KK - 1] = ~0ull;
    }
    return m;
}

// Landmarks per shared-memory chunk of the rescan kernel's warp-per-point
// mode (a multiple of 8: rows keep their chunk swizzle).
constexpr int kRescanChunk = 64;

template <int D, int KC>
__global__ void __launch_bounds__(256) rescan_kernel(const FusedArgs a) {
    constexpr int KK = KC - 4;
    constexpr int kWarps = 256 / 32;
    __shared__ unsigned long long s_top[kWarps][KK];
    const unsigned count = *reinterpret_cast<volatile const unsigned *>(a.fail_count);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float4 *Lg = reinterpret_cast<const float4 *>(a.hi);
    float4 x[D / 4];
    unsigned long long best[KK];
    if (count <= gridDim.x) {
        // block per point
        if (blockIdx.x >= count) return;  // whole blocks
        const long long row = a.fail_list[blockIdx.x];
        const float4 *xp = reinterpret_cast<const float4 *>(a.X) + row * (D / 4);
#pragma unroll
        for (int e = 0; e < D / 4; ++e) x[e] = centred(__ldg(xp + e), a.center, e);
        rescan_scan<D, KK>(x, Lg, a.L, threadIdx.x, 256, best);
        for (int r = 0; r < a.k; ++r) {
            const unsigned long long m = warp_pop<KK>(best);
            if (lane == 0) s_top[warp][r] = m;
        }
        __syncthreads();
        if (warp == 0) {
            // lane w < kWarps walks warp w's ascending list
            int pos = 0;
            unsigned long long head = lane < kWarps ? s_top[lane][0] : ~0ull;
            for (int r = 0; r < a.k; ++r) {
                unsigned long long m = head;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    m = umin64(m, __shfl_xor_sync(0xffffffffu, m, off));
                if (head == m && lane < kWarps) {
                    ++pos;
                    head = pos < a.k ? s_top[lane][pos] : ~0ull;
                }
                if (lane == 0) {
                    a.idx[row * a.k + r] = (int)(unsigned)(m & 0xffffffffu);
                    if (a.dist2) a.dist2[row * a.k + r] = __uint_as_float((unsigned)(m >> 32));
                }
            }
        }
        return;
    }
    // warp per point, the block's eight points at a time sharing each chunk
    // of landmark rows staged in shared memory (eight times fewer row reads
    // from L2 than each warp reading all L rows itself)
    __shared__ __align__(16) float4 s_rows[kRescanChunk * D / 4];
    const long long ngroups = ((long long)count + kWarps - 1) / kWarps;
    for (long long gq = blockIdx.x; gq < ngroups; gq += gridDim.x) {
        const long long w = gq * kWarps + warp;
        const bool act = w < (long long)count;
        const long long row = act ? a.fail_list[w] : 0;
        const float4 *xp = reinterpret_cast<const float4 *>(a.X) + row * (D / 4);
#pragma unroll
        for (int e = 0; e < D / 4; ++e)
            x[e] = act ? centred(__ldg(xp + e), a.center, e) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int t = 0; t < KK; ++t) best[t] = ~0ull;
        for (int c0 = 0; c0 < a.L; c0 += kRescanChunk) {
            const int cnt = a.L - c0 < kRescanChunk ? a.L - c0 : kRescanChunk;
            __syncthreads();  // the previous chunk is consumed
            for (int i = threadIdx.x; i < cnt * (D / 4); i += blockDim.x)
                s_rows[i] = __ldg(Lg + (size_t)c0 * (D / 4) + i);
            __syncthreads();
            // c0 is a multiple of 8, so a row keeps its chunk swizzle (swz
            // depends on the landmark index mod 8) and dist2_row gives the
            // same distance as from the global rows
            if (act)
                for (int j = lane; j < cnt; j += 32) {
                    const float d2 = dist2_row<D>(x, s_rows, j);
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)(c0 + j);
                    if (key < best[KK - 1]) {
                        unsigned long long prev = best[0];
                        best[0] = umin64(key, best[0]);
#pragma unroll
                        for (int t = 1; t < KK; ++t) {
                            const unsigned long long cur = best[t];
                            best[t] = umax64(prev, umin64(key, cur));
                            prev = cur;
                        }
                    }
                }
        }
        if (!act) continue;
        for (int r = 0; r < a.k; ++r) {
            const unsigned long long m = warp_pop<KK>(best);
            if (lane == 0) {
                a.idx[row * a.k + r] = (int)(unsigned)(m & 0xffffffffu);
                if (a.dist2) a.dist2[row * a.k + r] = __uint_as_float((unsigned)(m >> 32));
            }
        }
    }
}

template <int D, int KC>
cudaError_t launch_rescan(const FusedArgs &a, int grid, cudaStream_t stream) {
    rescan_kernel<D, KC><<<grid, 256, 0, stream>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Steps 1-4 of one point again with FP64 arithmetic, all 32 lanes of a warp
// sharing the work (the points whose FP32 normal system is ill-conditioned,
// det/trace^2 <= kDetRefine: its terms' rounding, ~1e-7 relative, is
// amplified by the condition number).  Called by every lane of the warp.
//   1. the exact k nearest (FP32 difference form, ties to the lower index:
//      the same neighbours as every k-NN path) by the warp scan of
//      rescan_kernel; lane i keeps rank i;
//   2. lane i: the squared distance of its neighbour in FP64 from the rows,
//      the score of reading R2 (weights 1/i over the m = k - 1 scored
//      neighbours, spread about the weighted mean, exp(boost (delta_1 -
//      delta_i) / sigma) times the cut-off factor) by warp sums;
//   3. the m (m - 1) / 2 pairs dealt to the lanes: D_uv = <X - L_u, L_v -
//      L_u> / q as an FP64 dot product, the weight s_u s_v r^-adjust, the
//      normal-system terms, summed over the warp;
//   4. the solve of reading R5: Cramer's rule if det > 1e-10 trace^2, else
//      the least-norm solution about the score-weighted centroid of the
//      scored 2-D landmarks (the plain mean if every score is 0), or that
//      centroid when A = 0.
// GB300's FP64 rate is low, so all 32 lanes issue useful FP64 work.
// Returns the coordinates on every lane.

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int D, int KK>
__device__ __noinline__ float2 refine_warp_point(const float *X, long long row,
                                                 const float *center, const float4 *Lg,
                                                 const float2 *lo2, int L, int k, float boost,
                                                 float adjust) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float4 x[D / 4];
    const float4 *xp = reinterpret_cast<const float4 *>(X) + row * (D / 4);
#pragma unroll
    for (int e = 0; e < D / 4; ++e) x[e] = centred(__ldg(xp + e), center, e);
    // 1. exact k nearest; lane r keeps rank r
    unsigned long long best[KK];
    rescan_scan<D, KK>(x, Lg, L, lane, 32, best);
    int j = 0;
    for (int r = 0; r < k; ++r) {
        const unsigned long long m = warp_pop<KK>(best);
        if (lane == r) j = (int)(unsigned)(m & 0xffffffffu);
    }
    // 2. distances and scores
    const int m = k - 1;
    const bool ranked = lane < k, scored = lane < m;
    double d2 = 0.0;
    if (ranked) {
        const float4 *l = Lg + (size_t)j * (D / 4);
        const int f = swz(D, j);
#pragma unroll
        for (int e = 0; e < D / 4; ++e) {
            const float4 q = l[e ^ f];
            const double t0 = (double)x[e].x - q.x, t1 = (double)x[e].y - q.y;
            const double t2 = (double)x[e].z - q.z, t3 = (double)x[e].w - q.w;
            d2 += t0 * t0 + t1 * t1 + t2 * t2 + t3 * t3;
        }
    }
    const double del = sqrt(d2);
    const double w = scored ? 1.0 / (double)(lane + 1) : 0.0;
    const double wsum = warp_sum_d(w);
    const double mean = warp_sum_d(w * del) / wsum;
    const double sigma = sqrt(warp_sum_d(w * (del - mean) * (del - mean)) / wsum);
    const double del0 = __shfl_sync(full, del, 0);
    const double dk = __shfl_sync(full, del, k - 1);
    const bool flat = sigma <= 1e-12 * fmax(mean, 1e-300);
    double s = 0.0;
    if (scored) {
        const double f1 = flat ? 1.0 : exp((double)boost * (del0 - del) / sigma);
        const double f2 = dk > 0.0 ? -expm1((double)kScoreEdge * (del / dk - 1.0)) : 1.0;
        s = f1 * f2;
    }
    const float2 l0 = lo2[__shfl_sync(full, j, 0)];
    const float2 lt = lo2[j];
    const double px = (double)lt.x - (double)l0.x, py = (double)lt.y - (double)l0.y;
    const double C0 = warp_sum_d(scored ? s * px : 0.0), C1 = warp_sum_d(scored ? s * py : 0.0);
    const double Ssum = warp_sum_d(s);
    const double M0 = warp_sum_d(scored ? px : 0.0), M1 = warp_sum_d(scored ? py : 0.0);
    // 3. pairs u < v < m dealt to the lanes
    double a00 = 0.0, a01 = 0.0, a11 = 0.0, b0 = 0.0, b1 = 0.0;
    const int P = m * (m - 1) / 2;
    for (int p0 = 0; p0 < P; p0 += 32) {
        const int p = p0 + lane;
        const bool valid = p < P;
        int u = 0, rem = valid ? p : 0;
        while (u < m - 1 && rem >= m - 1 - u) {
            rem -= m - 1 - u;
            ++u;
        }
        const int v = min(u + 1 + rem, 31);
        const int ju = __shfl_sync(full, j, u), jv = __shfl_sync(full, j, v);
        const double su = __shfl_sync(full, s, u), sv = __shfl_sync(full, s, v);
        const double pxu = __shfl_sync(full, px, u), pyu = __shfl_sync(full, py, u);
        const double pxv = __shfl_sync(full, px, v), pyv = __shfl_sync(full, py, v);
        if (!valid) continue;
        const float4 *Lu = Lg + (size_t)ju * (D / 4);
        const float4 *Lv = Lg + (size_t)jv * (D / 4);
        const int fu = swz(D, ju), fv = swz(D, jv);
        double q = 0.0, g = 0.0;
#pragma unroll
        for (int e = 0; e < D / 4; ++e) {
            const float4 cu = Lu[e ^ fu], cv = Lv[e ^ fv];
            const double e0 = (double)cv.x - cu.x, e1 = (double)cv.y - cu.y;
            const double e2 = (double)cv.z - cu.z, e3 = (double)cv.w - cu.w;
            q += e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3;
            g += ((double)x[e].x - cu.x) * e0 + ((double)x[e].y - cu.y) * e1 +
                 ((double)x[e].z - cu.z) * e2 + ((double)x[e].w - cu.w) * e3;
        }
        const double hx = pxv - pxu, hy = pyv - pyu;
        const double r = hx * hx + hy * hy;
        if (!(q > 0.0) || !(r > 0.0)) continue;
        const double wp = su * sv / (adjust == 1.f ? r : pow(r, (double)adjust));
        const double rhs = g / q + (hx * pxu + hy * pyu) / r;
        a00 += wp * hx * hx / r;
        a01 += wp * hx * hy / r;
        a11 += wp * hy * hy / r;
        b0 += wp * hx * rhs;
        b1 += wp * hy * rhs;
    }
    a00 = warp_sum_d(a00);
    a01 = warp_sum_d(a01);
    a11 = warp_sum_d(a11);
    b0 = warp_sum_d(b0);
    b1 = warp_sum_d(b1);
    // 4. solve
    const double det = a00 * a11 - a01 * a01, tr = a00 + a11;
    double rx, ry;
    if (det > kDetEps * tr * tr) {
        rx = (b0 * a11 - a01 * b1) / det;
        ry = (a00 * b1 - a01 * b0) / det;
    } else {
        const double c0 = Ssum > 0.0 ? C0 / Ssum : M0 / (double)m;
        const double c1 = Ssum > 0.0 ? C1 / Ssum : M1 / (double)m;
        rx = c0;
        ry = c1;
        if (tr > 0.0) {
            const double disc = sqrt((a00 - a11) * (a00 - a11) + 4.0 * a01 * a01);
            const double lam = 0.5 * (tr + disc);
            // major eigenvector: the better conditioned of two forms
            const double va0 = a01, va1 = lam - a00, vb0 = lam - a11, vb1 = a01;
            const double ga = va0 * va0 + va1 * va1, gb = vb0 * vb0 + vb1 * vb1;
            double v0 = ga >= gb ? va0 : vb0, v1 = ga >= gb ? va1 : vb1;
            double nn = ga >= gb ? ga : gb;
            if (nn == 0.0) {
                v0 = 1.0;
                v1 = 0.0;
                nn = 1.0;
            }
            nn = sqrt(nn);
            v0 /= nn;
            v1 /= nn;
            const double r0 = b0 - (a00 * c0 + a01 * c1);
            const double r1 = b1 - (a01 * c0 + a11 * c1);
            const double t = (v0 * r0 + v1 * r1) / lam;
            rx = c0 + t * v0;
            ry = c1 + t * v1;
        }
    }
    return make_float2((float)(rx + (double)l0.x), (float)(ry + (double)l0.y));
}

// The same recomputation with the 256 threads of a block on one point, for
// the refine kernels: each thread scans L/256 landmarks and the warps'
// lists are merged by warp 0 (as rescan_kernel's block mode), warp 0 then
// scores the neighbours (lane i = rank i), and the pairs are dealt to all
// threads, so a point takes a few microseconds instead of one warp's long
// chain of dependent loads and FP64 operations.  Every thread of the block
// calls it; returns the coordinates on every thread.
template <int D, int KK>
__device__ __noinline__ float2 refine_block_point(const float *X, long long row,
                                                  const float *center, const float4 *Lg,
                                                  const float2 *lo2, int L, int k, float boost,
                                                  float adjust) {
    constexpr int kWarps = 256 / 32;
    __shared__ unsigned long long s_top[kWarps][KK];
    __shared__ int s_j[32];
    __shared__ double s_s[32], s_px[32], s_py[32];
    __shared__ double s_red[kWarps][5];
    __shared__ double s_c[5];
    __shared__ float2 s_out;
    const unsigned full = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float4 x[D / 4];
    const float4 *xp = reinterpret_cast<const float4 *>(X) + row * (D / 4);
#pragma unroll
    for (int e = 0; e < D / 4; ++e) x[e] = centred(__ldg(xp + e), center, e);
    // 1. exact k nearest: every thread a slice, then the warps' lists merged
    unsigned long long best[KK];
    rescan_scan<D, KK>(x, Lg, L, tid, 256, best);
    for (int r = 0; r < k; ++r) {
        const unsigned long long m = warp_pop<KK>(best);
        if (lane == 0) s_top[warp][r] = m;
    }
    __syncthreads();
    const int m = k - 1;
    if (warp == 0) {
        int pos = 0, j = 0;
        unsigned long long head = lane < kWarps ? s_top[lane][0] : ~0ull;
        for (int r = 0; r < k; ++r) {
            unsigned long long mm = head;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) mm = umin64(mm, __shfl_xor_sync(full, mm, off));
            if (head == mm && lane < kWarps) {
                ++pos;
                head = pos < k ? s_top[lane][pos] : ~0ull;
            }
            if (lane == r) j = (int)(unsigned)(mm & 0xffffffffu);
        }
        // 2. distances and scores, lane i = rank i
        const bool ranked = lane < k, scored = lane < m;
        double d2 = 0.0;
        if (ranked) {
            const float4 *l = Lg + (size_t)j * (D / 4);
            const int f = swz(D, j);
#pragma unroll
            for (int e = 0; e < D / 4; ++e) {
                const float4 q = l[e ^ f];
                const double t0 = (double)x[e].x - q.x, t1 = (double)x[e].y - q.y;
                const double t2 = (double)x[e].z - q.z, t3 = (double)x[e].w - q.w;
                d2 += t0 * t0 + t1 * t1 + t2 * t2 + t3 * t3;
            }
        }
        const double del = sqrt(d2);
        const double w = scored ? 1.0 / (double)(lane + 1) : 0.0;
        const double wsum = warp_sum_d(w);
        const double mean = warp_sum_d(w * del) / wsum;
        const double sigma = sqrt(warp_sum_d(w * (del - mean) * (del - mean)) / wsum);
        const double del0 = __shfl_sync(full, del, 0);
        const double dk = __shfl_sync(full, del, k - 1);
        const bool flat = sigma <= 1e-12 * fmax(mean, 1e-300);
        double sc = 0.0;
        if (scored) {
            const double f1 = flat ? 1.0 : exp((double)boost * (del0 - del) / sigma);
            const double f2 = dk > 0.0 ? -expm1((double)kScoreEdge * (del / dk - 1.0)) : 1.0;
            sc = f1 * f2;
        }
        const float2 l0 = lo2[__shfl_sync(full, j, 0)];
        const float2 lt = lo2[j];
        const double px = (double)lt.x - (double)l0.x, py = (double)lt.y - (double)l0.y;
        const double C0 = warp_sum_d(scored ? sc * px : 0.0);
        const double C1 = warp_sum_d(scored ? sc * py : 0.0);
        const double Ssum = warp_sum_d(sc);
        const double M0 = warp_sum_d(scored ? px : 0.0), M1 = warp_sum_d(scored ? py : 0.0);
        s_j[lane] = j;
        s_s[lane] = sc;
        s_px[lane] = px;
        s_py[lane] = py;
        if (lane == 0) {
            s_c[0] = Ssum > 0.0 ? C0 / Ssum : M0 / (double)m;  // centroid (R5)
            s_c[1] = Ssum > 0.0 ? C1 / Ssum : M1 / (double)m;
            s_c[2] = l0.x;
            s_c[3] = l0.y;
        }
    }
    __syncthreads();
    // 3. pairs u < v < m dealt to the threads
    double a00 = 0.0, a01 = 0.0, a11 = 0.0, b0 = 0.0, b1 = 0.0;
    const int P = m * (m - 1) / 2;
    for (int p = tid; p < P; p += 256) {
        int u = 0, rem = p;
        while (rem >= m - 1 - u) {
            rem -= m - 1 - u;
            ++u;
        }
        const int v = u + 1 + rem;
        const int ju = s_j[u], jv = s_j[v];
        const float4 *Lu = Lg + (size_t)ju * (D / 4);
        const float4 *Lv = Lg + (size_t)jv * (D / 4);
        const int fu = swz(D, ju), fv = swz(D, jv);
        double q = 0.0, g = 0.0;
#pragma unroll
        for (int e = 0; e < D / 4; ++e) {
            const float4 cu = Lu[e ^ fu], cv = Lv[e ^ fv];
            const double e0 = (double)cv.x - cu.x, e1 = (double)cv.y - cu.y;
            const double e2 = (double)cv.z - cu.z, e3 = (double)cv.w - cu.w;
            q += e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3;
            g += ((double)x[e].x - cu.x) * e0 + ((double)x[e].y - cu.y) * e1 +
                 ((double)x[e].z - cu.z) * e2 + ((double)x[e].w - cu.w) * e3;
        }
        const double pxu = s_px[u], pyu = s_py[u];
        const double hx = s_px[v] - pxu, hy = s_py[v] - pyu;
        const double r = hx * hx + hy * hy;
        if (!(q > 0.0) || !(r > 0.0)) continue;
        const double wp = s_s[u] * s_s[v] / (adjust == 1.f ? r : pow(r, (double)adjust));
        const double rhs = g / q + (hx * pxu + hy * pyu) / r;
        a00 += wp * hx * hx / r;
        a01 += wp * hx * hy / r;
        a11 += wp * hy * hy / r;
        b0 += wp * hx * rhs;
        b1 += wp * hy * rhs;
    }
    a00 = warp_sum_d(a00);
    a01 = warp_sum_d(a01);
    a11 = warp_sum_d(a11);
    b0 = warp_sum_d(b0);
    b1 = warp_sum_d(b1);
    if (lane == 0) {
        s_red[warp][0] = a00;
        s_red[warp][1] = a01;
        s_red[warp][2] = a11;
        s_red[warp][3] = b0;
        s_red[warp][4] = b1;
    }
    __syncthreads();
    // 4. solve (reading R5)
    if (tid == 0) {
        double A00 = 0.0, A01 = 0.0, A11 = 0.0, B0 = 0.0, B1 = 0.0;
        for (int w = 0; w < kWarps; ++w) {
            A00 += s_red[w][0];
            A01 += s_red[w][1];
            A11 += s_red[w][2];
            B0 += s_red[w][3];
            B1 += s_red[w][4];
        }
        const double det = A00 * A11 - A01 * A01, tr = A00 + A11;
        double rx, ry;
        if (det > kDetEps * tr * tr) {
            rx = (B0 * A11 - A01 * B1) / det;
            ry = (A00 * B1 - A01 * B0) / det;
        } else {
            const double c0 = s_c[0], c1 = s_c[1];
            rx = c0;
            ry = c1;
            if (tr > 0.0) {
                const double disc = sqrt((A00 - A11) * (A00 - A11) + 4.0 * A01 * A01);
                const double lam = 0.5 * (tr + disc);
                const double va0 = A01, va1 = lam - A00, vb0 = lam - A11, vb1 = A01;
                const double ga = va0 * va0 + va1 * va1, gb = vb0 * vb0 + vb1 * vb1;
                double v0 = ga >= gb ? va0 : vb0, v1 = ga >= gb ? va1 : vb1;
                double nn = ga >= gb ? ga : gb;
                if (nn == 0.0) {
                    v0 = 1.0;
                    v1 = 0.0;
                    nn = 1.0;
                }
                nn = sqrt(nn);
                v0 /= nn;
                v1 /= nn;
                const double r0 = B0 - (A00 * c0 + A01 * c1);
                const double r1 = B1 - (A01 * c0 + A11 * c1);
                const double t = (v0 * r0 + v1 * r1) / lam;
                rx = c0 + t * v0;
                ry = c1 + t * v1;
            }
        }
        s_out = make_float2((float)(rx + s_c[2]), (float)(ry + s_c[3]));
    }
    __syncthreads();
    const float2 res = s_out;
    __syncthreads();  // s_out and the other arrays may be reused by the next point
    return res;
}

// One block per row of a.refine_list (count *a.refine_count): the FP64
// recomputation of the point, written to a.out.
template <int D, int KC>
__global__ void __launch_bounds__(256) refine_kernel(const FusedArgs a) {
    constexpr int KK = KC - 4;
    const unsigned count = *reinterpret_cast<volatile const unsigned *>(a.refine_count);
    for (long long w = blockIdx.x; w < (long long)count; w += gridDim.x) {
        const long long row = a.refine_list[w];
        const float2 p = refine_block_point<D, KK>(a.X, row, a.center,
                                                   reinterpret_cast<const float4 *>(a.hi),
                                                   reinterpret_cast<const float2 *>(a.lo), a.L,
                                                   a.k, a.boost, a.adjust);
        if (threadIdx.x == 0) {
            reinterpret_cast<float2 *>(a.out)[row] = p;
            atomicAdd(reinterpret_cast<unsigned *>(a.status) + 5, 1u);  // stats: refines
        }
    }
}

// The same for the batched kernel: entries (dataset, row).
template <int D, int KC>
__global__ void __launch_bounds__(256) refine_batch_kernel(const BatchArgs B) {
    constexpr int KK = KC - 4;
    const unsigned count = *reinterpret_cast<volatile const unsigned *>(B.refine_count);
    for (long long w = blockIdx.x; w < (long long)count; w += gridDim.x) {
        const int2 e = B.refine_list[w];
        const FusedArgs &a = B.items[e.x];
        const float2 p = refine_block_point<D, KK>(a.X, e.y, a.center,
                                                   reinterpret_cast<const float4 *>(a.hi),
                                                   reinterpret_cast<const float2 *>(a.lo), a.L,
                                                   a.k, a.boost, a.adjust);
        if (threadIdx.x == 0) {
            reinterpret_cast<float2 *>(a.out)[e.y] = p;
            atomicAdd(reinterpret_cast<unsigned *>(B.status) + 5, 1u);  // stats: refines
        }
    }
}

template <int D, int KC>
cudaError_t launch_refine(const FusedArgs &a, int grid, cudaStream_t stream) {
    refine_kernel<D, KC><<<grid, 256, 0, stream>>>(a);
    return cudaGetLastError();
}

template <int D, int KC>
cudaError_t launch_refine_batch(const BatchArgs &b, int grid, cudaStream_t stream) {
    refine_batch_kernel<D, KC><<<grid, 256, 0, stream>>>(b);
    return cudaGetLastError();
}

// One thread per ordered pair (u, v) of landmarks: the pair table
// (pair_entry of the loop's own pair_q and the 2-D operator) when ptab is
// given, else the table of squared landmark distances (pair_q alone).
template <int D>
__global__ void landmark_pair_kernel(const float *__restrict__ hi, const float *__restrict__ lo,
                                     int L, float2 *__restrict__ ptab, float *__restrict__ qtab) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)L * L) return;
    const int u = (int)(t / L), v = (int)(t - (long long)u * L);
    const float4 *Lg = reinterpret_cast<const float4 *>(hi);
    const float4 *Lu = Lg + (size_t)u * (D / 4);
    const int fu = swz(D, u);
    float4 lu[D / 4];
#pragma unroll
    for (int e = 0; e < D / 4; ++e) lu[e] = __ldg(Lu + (e ^ fu));
    const float qq = pair_q<D>(lu, Lg + (size_t)v * (D / 4), swz(D, v));
    if (ptab) {
        const float2 pu = reinterpret_cast<const float2 *>(lo)[u];
        const float2 pv = reinterpret_cast<const float2 *>(lo)[v];
        ptab[t] = pair_entry(qq, pv.x - pu.x, pv.y - pu.y);
    } else {
        qtab[t] = qq;
    }
}

template <int D>
cudaError_t launch_pair_table(const float *hi, const float *lo, int L, float2 *ptab, float *qtab,
                              cudaStream_t stream) {
    const long long pairs = (long long)L * L;
    landmark_pair_kernel<D><<<(unsigned)((pairs + 255) / 256), 256, 0, stream>>>(hi, lo, L, ptab,
                                                                                qtab);
    return cudaGetLastError();
}

template <int D, int KC, int MINB>
cudaError_t launch_batch(const BatchArgs &b, int grid, size_t smem, cudaStream_t stream) {
    batch_kernel<D, KC, MINB><<<grid, kThreads, smem, stream>>>(b);
    return cudaGetLastError();
}

template <int D, int KC, int MINB>
cudaError_t launch_fused(const FusedArgs &a, int grid, size_t smem, cudaStream_t stream) {
    fused_kernel<D, KC, MINB><<<grid, kThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int D, int KC>
struct Instance {
    // Two resident blocks per SM (<= 128 registers a thread) where the list
    // and the point rows fit without spilling; one otherwise.
    static constexpr int kMinBlocks = (D <= 16 && KC <= 24) ? 2 : 1;
    static const KernelOps ops;
};

template <int D, int KC>
const KernelOps Instance<D, KC>::ops = {
    reinterpret_cast<const void *>(&fused_kernel<D, KC, Instance<D, KC>::kMinBlocks>), KC,
    &launch_fused<D, KC, Instance<D, KC>::kMinBlocks>,
    reinterpret_cast<const void *>(&batch_kernel<D, KC, Instance<D, KC>::kMinBlocks>),
    &launch_batch<D, KC, Instance<D, KC>::kMinBlocks>, &launch_pair_table<D>,
    {reinterpret_cast<const void *>(&project_kernel<D, KC, kPairTab2>),
     reinterpret_cast<const void *>(&project_kernel<D, KC, kPairTab1>),
     reinterpret_cast<const void *>(&project_kernel<D, KC, kPairRows>)},
    {&launch_project<D, KC, kPairTab2>, &launch_project<D, KC, kPairTab1>,
     &launch_project<D, KC, kPairRows>},
    &launch_rescan<D, KC>,
    reinterpret_cast<const void *>(&rerank_kernel<D, KC>), &launch_rerank<D, KC>,
    {reinterpret_cast<const void *>(&rerank_project_kernel<D, KC, kPairTab2>),
     reinterpret_cast<const void *>(&rerank_project_kernel<D, KC, kPairTab1>),
     reinterpret_cast<const void *>(&rerank_project_kernel<D, KC, kPairRows>)},
    {&launch_rerank_project<D, KC, kPairTab2>, &launch_rerank_project<D, KC, kPairTab1>,
     &launch_rerank_project<D, KC, kPairRows>},
    &launch_refine<D, KC>, &launch_refine_batch<D, KC>};

// Table of the list capacities instantiated for each D.
#define ESOM_DEFINE_D(DV)                                            \
    const KernelOps *kernel_ops_d##DV(int kc) {                      \
        switch (kc) {                                                \
            case 8: return &Instance<DV, 8>::ops;                    \
            case 12: return &Instance<DV, 12>::ops;                  \
            case 16: return &Instance<DV, 16>::ops;                  \
            case 20: return &Instance<DV, 20>::ops;                  \
            case 24: return &Instance<DV, 24>::ops;                  \
            case 28: return &Instance<DV, 28>::ops;                  \
            case 32: return &Instance<DV, 32>::ops;                  \
            case 36: return &Instance<DV, 36>::ops;                  \
            default: return nullptr;                                 \
        }                                                            \
    }

}  // namespace esom
