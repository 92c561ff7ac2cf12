// Fused EmbedSOM projection kernel for sm_103a (one launch per call).
//
// Per point (paper, Section 3.1 steps 1-4; Section 4.2 and 4.3):
//   1. k-NN over all L landmarks (squared Euclidean, FP32, ties to the lower
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
//   * the landmarks are copied by bulk TMA into shared memory once per block
//     when they fit (L*D*4 <= chunk budget), otherwise streamed in chunks
//     through two shared buffers; every thread reads the same landmark at
//     the same time, so each shared load is a broadcast;
//   * the k-NN list lives in registers, sorted, with compile-time capacity
//     KC >= k; new distances below the current k-th are appended to a small
//     per-thread queue in shared memory and merged into the list in
//     warp-uniform flushes, so the insertion network runs in lock-step;
//   * scores and the pair sums run in FP32 registers, with the 2-D landmark
//     coordinates taken relative to the nearest neighbour's (the fit is
//     shift-equivariant) to keep the FP32 sums small; only the determinant
//     and the solve are FP64.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "esom_kernels.h"

namespace esom {

constexpr float kScoreEdge = 10.0f;     // steepness of the k-th-neighbour cut-off
constexpr float kSigmaEps = 1e-12f;     // spread below this * mean counts as zero
constexpr double kDetEps = 1e-10;       // det/trace^2 below this: rank-one solve
constexpr double kDetRecheck = 1e-4;    // FP32 det/trace^2 below this: recompute it
constexpr unsigned long long kWaitNs = 2000000000ull;  // bounded mbarrier wait (2 s)

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

// Waits for phase `parity` of `bar` to complete, giving up after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t it = 1; it < (1u << 28); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0 && global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

// Issues the bulk copy of `bytes` into `dst` and arms `bar` for it; large
// copies are split into pieces below the mbarrier transaction limit.
__device__ __forceinline__ void issue_copy(void *dst, const void *src, uint32_t bytes,
                                           uint64_t *bar) {
    mbar_expect_tx(bar, bytes);
    const uint32_t piece = 1u << 16;
    for (uint32_t off = 0; off < bytes; off += piece) {
        const uint32_t b = bytes - off < piece ? bytes - off : piece;
        bulk_g2s(static_cast<char *>(dst) + off, static_cast<const char *>(src) + off, b, bar);
    }
}

// ---------------------------------------------------------------------------
// Register-resident sorted k-NN list.

template <int KC>
__device__ __forceinline__ void list_insert(float (&sd)[KC], int (&si)[KC], float v, int vi) {
    // Shift insertion: every slot at or after the new entry's position takes
    // its predecessor, so existing entries keep their order.  Candidates
    // arrive in increasing landmark index and go behind every entry of equal
    // distance, which keeps the list sorted by (distance, index).  All the
    // comparisons are independent of each other (no chain through the list).
    bool c[KC];
#pragma unroll
    for (int t = 0; t < KC; ++t) c[t] = v < sd[t];
#pragma unroll
    for (int t = KC - 1; t > 0; --t) {
        sd[t] = c[t - 1] ? sd[t - 1] : (c[t] ? v : sd[t]);
        si[t] = c[t - 1] ? si[t - 1] : (c[t] ? vi : si[t]);
    }
    sd[0] = c[0] ? v : sd[0];
    si[0] = c[0] ? vi : si[0];
}

template <int KC>
__device__ __forceinline__ float list_at(const float (&a)[KC], int pos) {
    float r = a[0];
#pragma unroll
    for (int t = 1; t < KC; ++t)
        if (t == pos) r = a[t];
    return r;
}

// Merges this thread's queued candidates into its list; the warp runs as
// many insertion rounds as its fullest queue needs.
template <int KC>
__device__ __forceinline__ void queue_flush(float (&sd)[KC], int (&si)[KC], int &qn, float &thr,
                                            const float *qd, const int *qi, int tid, int k) {
    const int mx = __reduce_max_sync(0xffffffffu, qn);
    for (int i = 0; i < mx; ++i) {
        float v = INFINITY;
        int vi = 0;
        if (i < qn) {
            v = qd[i * kThreads + tid];
            vi = qi[i * kThreads + tid];
        }
        list_insert<KC>(sd, si, v, vi);
    }
    qn = 0;
    thr = list_at<KC>(sd, k - 1);
}

template <int D>
__device__ __forceinline__ float dist2_row(const float4 (&x)[D / 4], const float4 *l) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
    for (int e = 0; e < D / 4; ++e) {
        const float4 q = l[e];
        const float dx = x[e].x - q.x, dy = x[e].y - q.y;
        const float dz = x[e].z - q.z, dw = x[e].w - q.w;
        a0 = fmaf(dx, dx, a0);
        a1 = fmaf(dy, dy, a1);
        a2 = fmaf(dz, dz, a2);
        a3 = fmaf(dw, dw, a3);
    }
    return (a0 + a1) + (a2 + a3);
}

// Scans `cnt` landmarks of one shared-memory chunk (global indices base..).
template <int D, int KC>
__device__ __forceinline__ void scan_chunk(const float4 (&x)[D / 4], const float *Lc, int cnt,
                                           int base, float (&sd)[KC], int (&si)[KC], int &qn,
                                           float &thr, float *qd, int *qi, int tid, int k) {
    const float4 *L4 = reinterpret_cast<const float4 *>(Lc);
    for (int j0 = 0; j0 < cnt; j0 += kCheck) {
        if (j0 + kCheck <= cnt) {
#pragma unroll
            for (int jj = 0; jj < kCheck; ++jj) {
                const float d2 = dist2_row<D>(x, L4 + (size_t)(j0 + jj) * (D / 4));
                if (d2 < thr) {
                    qd[qn * kThreads + tid] = d2;
                    qi[qn * kThreads + tid] = base + j0 + jj;
                    ++qn;
                }
            }
        } else {
            for (int j = j0; j < cnt; ++j) {
                const float d2 = dist2_row<D>(x, L4 + (size_t)j * (D / 4));
                if (d2 < thr) {
                    qd[qn * kThreads + tid] = d2;
                    qi[qn * kThreads + tid] = base + j;
                    ++qn;
                }
            }
        }
        if (__any_sync(0xffffffffu, qn > kQueue - kCheck))
            queue_flush<KC>(sd, si, qn, thr, qd, qi, tid, k);
    }
}

// ---------------------------------------------------------------------------
// Step 3: pair terms over u < v < m.  PASS 0 accumulates the normal system
// (A, b); PASS 1 accumulates rho = sum w (h.n)^2 / r for a unit 2-D direction
// n (the Rayleigh quotient n^T A n) and skips the work only PASS 0 needs.

template <int D, int KC, int PASS>
__device__ __forceinline__ void pair_sums(const float4 (&x)[D / 4], const int (&si)[KC],
                                          const float (&ss)[KC], int m, const float4 *Lg,
                                          const float2 *lo2, float2 l0, const FusedArgs &a,
                                          float nx, float ny, float &A00, float &A01,
                                          float &A11, float &B0, float &B1, float &rho) {
#pragma unroll 1
    for (int u = 0; u < m - 1; ++u) {
        int iu = si[0];
        float su = ss[0];
#pragma unroll
        for (int t = 1; t < KC; ++t)
            if (t == u) {
                iu = si[t];
                su = ss[t];
            }
        const float4 *Lu = Lg + (size_t)iu * (D / 4);
        float4 lu[D / 4], y[D / 4];
#pragma unroll
        for (int e = 0; e < D / 4; ++e) {
            lu[e] = Lu[e];
            y[e] = make_float4(x[e].x - lu[e].x, x[e].y - lu[e].y, x[e].z - lu[e].z,
                               x[e].w - lu[e].w);
        }
        const float2 lut = __ldg(&lo2[iu]);
        const float lux = lut.x - l0.x, luy = lut.y - l0.y;  // l_u relative to l_0
#pragma unroll
        for (int v = 1; v < KC; ++v) {
            if (v > u && v < m) {
                const float4 *Lv = Lg + (size_t)si[v] * (D / 4);
                float q0 = 0.f, q1 = 0.f, n0 = 0.f, n1 = 0.f;
#pragma unroll
                for (int e = 0; e < D / 4; ++e) {
                    const float4 lv = Lv[e];
                    const float ex = lv.x - lu[e].x, ey = lv.y - lu[e].y;
                    const float ez = lv.z - lu[e].z, ew = lv.w - lu[e].w;
                    q0 = fmaf(ex, ex, q0);
                    q1 = fmaf(ey, ey, q1);
                    q0 = fmaf(ez, ez, q0);
                    q1 = fmaf(ew, ew, q1);
                    n0 = fmaf(y[e].x, ex, n0);
                    n1 = fmaf(y[e].y, ey, n1);
                    n0 = fmaf(y[e].z, ez, n0);
                    n1 = fmaf(y[e].w, ew, n1);
                }
                const float q = q0 + q1, num = n0 + n1;
                const float2 lvt = __ldg(&lo2[si[v]]);
                const float hx = lvt.x - lut.x, hy = lvt.y - lut.y;
                const float r = fmaf(hx, hx, hy * hy);
                if (q > 0.f && r > 0.f) {
                    const float Duv = num * __frcp_rn(q);
                    const float ir = __frcp_rn(r);
                    float w = su * ss[v];
                    if (a.adjust_mode == 1)
                        w *= ir;
                    else if (a.adjust_mode == 0)
                        w *= exp2f(-a.adjust * log2f(r));
                    const float wr = w * ir;
                    if (PASS == 0) {
                        const float rhs = fmaf(fmaf(hx, lux, hy * luy), ir, Duv);
                        A00 = fmaf(wr * hx, hx, A00);
                        A01 = fmaf(wr * hx, hy, A01);
                        A11 = fmaf(wr * hy, hy, A11);
                        const float wrhs = w * rhs;
                        B0 = fmaf(wrhs, hx, B0);
                        B1 = fmaf(wrhs, hy, B1);
                    } else {
                        const float t = fmaf(hx, nx, hy * ny);
                        rho = fmaf(wr * t, t, rho);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Steps 2-4 for one point: scores, pair sums, FP64 solve.

template <int D, int KC>
__device__ __forceinline__ float2 project_point(const float4 (&x)[D / 4], const float (&sd)[KC],
                                                const int (&si)[KC], const float4 *Lg,
                                                const float2 *lo2, const FusedArgs &a) {
    const int k = a.k, m = k - 1;

    // Step 2: scores.  Distances are Euclidean; the weights of the mean and
    // spread are 1/i over the m scored neighbours.  exp(boost (d_1 - d_i) /
    // sigma) differs from exp(boost (mean - d_i) / sigma) by one common
    // factor, which cancels in the solve, and it cannot overflow.
    float del[KC];
#pragma unroll
    for (int t = 0; t < KC; ++t) del[t] = sqrtf(sd[t]);
    float wsum = 0.f, mean = 0.f;
#pragma unroll
    for (int t = 0; t < KC; ++t)
        if (t < m) {
            const float w = 1.0f / (float)(t + 1);
            wsum += w;
            mean = fmaf(w, del[t], mean);
        }
    mean /= wsum;
    float var = 0.f;
#pragma unroll
    for (int t = 0; t < KC; ++t)
        if (t < m) {
            const float w = 1.0f / (float)(t + 1);
            const float dd = del[t] - mean;
            var = fmaf(w * dd, dd, var);
        }
    const float sigma = sqrtf(var / wsum);
    const float dk = list_at<KC>(del, k - 1);
    const bool flat = sigma <= kSigmaEps * fmaxf(mean, 1e-30f);
    const float inv_sigma = flat ? 0.f : a.boost / sigma;
    const float inv_dk = dk > 0.f ? 1.0f / dk : 0.f;
    float ss[KC];
#pragma unroll
    for (int t = 0; t < KC; ++t) {
        float s = 0.f;
        if (t < m) {
            const float f1 = flat ? 1.f : expf((del[0] - del[t]) * inv_sigma);
            const float f2 = dk > 0.f ? -expm1f(kScoreEdge * fmaf(del[t], inv_dk, -1.f)) : 1.f;
            s = f1 * f2;
        }
        ss[t] = s;
    }

    // 2-D coordinates relative to the nearest neighbour's.
    const float2 l0 = __ldg(&lo2[si[0]]);
    float C0 = 0.f, C1 = 0.f, Ssum = 0.f, M0 = 0.f, M1 = 0.f;
#pragma unroll
    for (int t = 0; t < KC; ++t)
        if (t < m) {
            const float2 lt = __ldg(&lo2[si[t]]);
            const float px = lt.x - l0.x, py = lt.y - l0.y;
            C0 = fmaf(ss[t], px, C0);
            C1 = fmaf(ss[t], py, C1);
            Ssum += ss[t];
            M0 += px;
            M1 += py;
        }

    // Step 3: pair terms, u < v < m.
    float A00 = 0.f, A01 = 0.f, A11 = 0.f, B0 = 0.f, B1 = 0.f, rho = 0.f;
    pair_sums<D, KC, 0>(x, si, ss, m, Lg, lo2, l0, a, 0.f, 0.f, A00, A01, A11, B0, B1, rho);

    // Step 4: FP64 solve.
    const double a00 = A00, a01 = A01, a11 = A11, b0 = B0, b1 = B1;
    double det = a00 * a11 - a01 * a01;
    const double tr = a00 + a11;
    if (tr > 0.0 && det <= kDetRecheck * tr * tr) {
        // A00 A11 - A01^2 from FP32 sums cannot resolve det/trace^2 below
        // ~1e-6.  Recompute the small eigenvalue as the Rayleigh quotient
        // n^T A n along the minor eigenvector n of the FP32 matrix: a sum of
        // non-negative terms w (h.n)^2 / r over the pairs, free of
        // cancellation, and accurate to second order in the error of n.
        const double disc = sqrt((a00 - a11) * (a00 - a11) + 4.0 * a01 * a01);
        const double lmax = 0.5 * (tr + disc);
        // two candidate major eigenvectors; take the better conditioned one
        const double va0 = a01, va1 = lmax - a00, vb0 = lmax - a11, vb1 = a01;
        const double na = va0 * va0 + va1 * va1, nb = vb0 * vb0 + vb1 * vb1;
        const double v0 = na >= nb ? va0 : vb0, v1 = na >= nb ? va1 : vb1;
        const double nn = sqrt(na >= nb ? na : nb);
        if (nn > 0.0) {
            // minor direction: the major one turned by 90 degrees
            float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f, z4 = 0.f;
            pair_sums<D, KC, 1>(x, si, ss, m, Lg, lo2, l0, a, (float)(-v1 / nn), (float)(v0 / nn),
                                z0, z1, z2, z3, z4, rho);
            const double lmin = (double)rho;
            det = lmin * (tr - lmin);
        }
    }
    double px, py;
    if (det > kDetEps * tr * tr) {
        const double id = 1.0 / det;
        px = (b0 * a11 - a01 * b1) * id;
        py = (a00 * b1 - a01 * b0) * id;
    } else {
        // Rank one (or zero): least-norm solution about the score-weighted
        // centroid of the scored 2-D landmarks (plain mean if all scores are 0).
        double c0, c1;
        if (Ssum > 0.f) {
            c0 = (double)C0 / (double)Ssum;
            c1 = (double)C1 / (double)Ssum;
        } else {
            c0 = (double)M0 / (double)m;
            c1 = (double)M1 / (double)m;
        }
        if (tr == 0.0) {
            px = c0;
            py = c1;
        } else {
            const double disc = sqrt((a00 - a11) * (a00 - a11) + 4.0 * a01 * a01);
            const double lam = 0.5 * (tr + disc);
            double va0 = a01, va1 = lam - a00, vb0 = lam - a11, vb1 = a01;
            const double na = va0 * va0 + va1 * va1, nb = vb0 * vb0 + vb1 * vb1;
            double v0 = na >= nb ? va0 : vb0, v1 = na >= nb ? va1 : vb1;
            double nn = na >= nb ? na : nb;
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
            px = c0 + t * v0;
            py = c1 + t * v1;
        }
    }
    return make_float2((float)(px + (double)l0.x), (float)(py + (double)l0.y));
}

// ---------------------------------------------------------------------------

template <int D, int KC, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) fused_kernel(const FusedArgs a) {
    static_assert(D % 4 == 0 && D >= 4 && D <= 64, "D must be a multiple of 4 in [4, 64]");
    static_assert(KC >= 2 && KC <= 32, "list capacity out of range");
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);  // [0] points, [1],[2] landmarks
    float *sX = reinterpret_cast<float *>(smem + kBarrierBytes);
    float *sL = sX + kThreads * D;
    const int nbufL = a.nchunks == 1 ? 1 : 2;
    float *qd = sL + (size_t)nbufL * a.chunk * D;
    int *qi = reinterpret_cast<int *>(qd + kQueue * kThreads);
    volatile int &s_abort = *reinterpret_cast<int *>(smem + 64);

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
        issue_copy(sX, a.X + r0 * D, (uint32_t)(rows * D * sizeof(float)), &bars[0]);
    };
    auto issue_chunk = [&](int c, int buf) {
        const int cnt = a.L - c * a.chunk < a.chunk ? a.L - c * a.chunk : a.chunk;
        issue_copy(sL + buf * chunk_floats, a.hi + (size_t)c * chunk_floats,
                   (uint32_t)((size_t)cnt * D * sizeof(float)), &bars[1 + buf]);
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

    auto abort_block = [&]() {
        // Drain this block's own copies in flight (bounded), then leave.
        if (tid == 0) {
            atomicOr(a.status, kErrWaitTimeout);
            if (pendX) mbar_wait(&bars[0], phX);
            if (pendL0) mbar_wait(&bars[1], parL0);
            if (pendL1) mbar_wait(&bars[2], parL1);
        }
    };

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
        for (int e = 0; e < D / 4; ++e) xr[e] = active ? xs[e] : make_float4(0.f, 0.f, 0.f, 0.f);
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

        // Step 1: k-NN.
        float sd[KC];
        int si[KC];
#pragma unroll
        for (int s = 0; s < KC; ++s) {
            sd[s] = INFINITY;
            si[s] = 0;
        }
        float thr = INFINITY;
        int qn = 0;
        for (int c = 0; c < a.nchunks; ++c) {
            const int base = c * a.chunk;
            const int cnt = a.L - base < a.chunk ? a.L - base : a.chunk;
            const float *Lc = sL;
            int buf = 0;
            if (a.nchunks > 1) {
                buf = (int)(step & 1);
                const uint32_t par = (uint32_t)((step >> 1) & 1);
                if (!mbar_wait(&bars[1 + buf], par)) s_abort = 1;
                Lc = sL + buf * chunk_floats;
            }
            scan_chunk<D, KC>(xr, Lc, cnt, base, sd, si, qn, thr, qd, qi, tid, a.k);
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
        queue_flush<KC>(sd, si, qn, thr, qd, qi, tid, a.k);

        if (a.mode == kKnn) {
            if (active) {
                const long long row = row0 + tid;
#pragma unroll
                for (int s = 0; s < KC; ++s)
                    if (s < a.k) {
                        a.idx[row * a.k + s] = si[s];
                        if (a.dist2) a.dist2[row * a.k + s] = sd[s];
                    }
            }
            continue;
        }
        const float2 p = project_point<D, KC>(xr, sd, si, Lg, lo2, a);
        if (active) reinterpret_cast<float2 *>(a.out)[row0 + tid] = p;
    }
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
    static constexpr int kMinBlocks = (D <= 16 && KC <= 20) || (D <= 8 && KC <= 24) ? 2 : 1;
    static const KernelOps ops;
};

template <int D, int KC>
const KernelOps Instance<D, KC>::ops = {
    reinterpret_cast<const void *>(&fused_kernel<D, KC, Instance<D, KC>::kMinBlocks>), KC,
    &launch_fused<D, KC, Instance<D, KC>::kMinBlocks>};

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
            default: return nullptr;                                 \
        }                                                            \
    }

}  // namespace esom
