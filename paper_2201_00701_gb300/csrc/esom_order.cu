// Spatial orderings for the tensor-core screened k-NN.
//
// The tensor-core k-NN computes all L screening values of a point (Section
// 4.2's distance block as one contraction), but only the few below the
// point's current threshold need selection work (key, test, queue push,
// merge).  Two orderings make those few cluster, so that a warp can skip a
// whole group of 32 values after one minimum and one vote:
//   * landmarks: a balanced recursive split of the landmark set along each
//     group's principal direction (power iteration) into chunks of kTcN,
//     the chunks the MMA consumes; internal position j' of the screening
//     holds landmark lperm[j'];
//   * points: each point's home is the chunk with the nearest centroid; the
//     points of a pass are visited grouped by home (a bucket sort that keeps
//     the input order inside a bucket), so the 128 points of a tile lie near
//     each other, and a tile visits the chunks nearest its home chunk first,
//     which tightens every point's threshold early.
// Results do not depend on either order: the screened list is certified and
// re-ranked by exact distance with the original landmark indices.
#include <cuda_runtime.h>
#include <stdint.h>

#include "esom_kernels.h"

namespace esom {

namespace {

constexpr int kOrderThreads = 1024;
constexpr int kOrderWarps = kOrderThreads / 32;
constexpr int kPowerIters = 8;

// Logical coordinate t of landmark row j (rows are stored with their 16-byte
// pieces swizzled, see swz).
__device__ __forceinline__ float row_elem(const float *hi, int j, int D, int t) {
    const int e = t >> 2;
    return hi[(size_t)j * D + (((e ^ swz(D, j)) << 2) | (t & 3))];
}

// Order-preserving map of a float to an unsigned integer.
__device__ __forceinline__ uint32_t float_order_bits(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float warp_allsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sort key of a landmark during the split: node (16 bits), projection on the
// node's principal direction (32 bits), index (16 bits; L <= kOrderMaxL).
__device__ __forceinline__ unsigned long long order_key(int node, uint32_t proj, int j) {
    return ((unsigned long long)node << 48) | ((unsigned long long)proj << 16) |
           (unsigned long long)(unsigned)j;
}

}  // namespace

// One block: the landmark order lperm (internal position -> landmark).  The
// node list holds contiguous ranges of the current order; a node of more
// than kTcN landmarks is split into a left part of a multiple of kTcN
// landmarks (about half) and the rest, by their projections on the node's
// principal direction (power iteration from the axis of largest variance),
// so that every leaf but the last is a full chunk.  All reductions run in a
// fixed order: the order is deterministic.
__global__ void __launch_bounds__(kOrderThreads) landmark_order_kernel(
    const float *__restrict__ hi, int L, int D, int Lp, int *__restrict__ lperm) {
    extern __shared__ unsigned long long skey[];  // Lp keys
    __shared__ float red[kOrderWarps][64];
    __shared__ float mu[64], vv[64];
    __shared__ int ns[2][kOrderMaxL / kTcN + 1], nz[2][kOrderMaxL / kTcN + 1];
    __shared__ int ncount[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < Lp; i += kOrderThreads)
        skey[i] = i < L ? order_key(0, 0u, i) : ~0ull;  // padding sorts last
    if (tid == 0) {
        ns[0][0] = 0;
        nz[0][0] = L;
        ncount[0] = 1;
    }
    __syncthreads();
    int cur = 0;
    for (int level = 0; level < 16; ++level) {
        const int cnt = ncount[cur];
        bool any_split = false;
        for (int nd = 0; nd < cnt; ++nd)
            any_split = any_split || nz[cur][nd] > kTcN;
        if (!any_split) break;
        for (int nd = 0; nd < cnt; ++nd) {
            const int s0 = ns[cur][nd], m = nz[cur][nd];
            if (m <= kTcN) {
                for (int i = tid; i < m; i += kOrderThreads)
                    skey[s0 + i] = order_key(nd, 0u, (int)(skey[s0 + i] & 0xFFFFu));
                continue;
            }
            // mean and spread per coordinate (lane: coordinates lane, lane + 32)
            float a0 = 0.f, a1 = 0.f, q0 = 0.f, q1 = 0.f;
            for (int i = warp; i < m; i += kOrderWarps) {
                const int j = (int)(skey[s0 + i] & 0xFFFFu);
                const float x0 = lane < D ? row_elem(hi, j, D, lane) : 0.f;
                const float x1 = lane + 32 < D ? row_elem(hi, j, D, lane + 32) : 0.f;
                a0 += x0;
                a1 += x1;
                q0 = fmaf(x0, x0, q0);
                q1 = fmaf(x1, x1, q1);
            }
            red[warp][lane] = a0;
            red[warp][lane + 32] = a1;
            __syncthreads();
            if (tid < 64) {
                float s = 0.f;
                for (int w = 0; w < kOrderWarps; ++w) s += red[w][tid];
                mu[tid] = s / (float)m;
            }
            __syncthreads();
            red[warp][lane] = q0;
            red[warp][lane + 32] = q1;
            __syncthreads();
            if (tid < 64) {
                float s = 0.f;
                for (int w = 0; w < kOrderWarps; ++w) s += red[w][tid];
                vv[tid] = tid < D ? s / (float)m - mu[tid] * mu[tid] : -1.f;
            }
            __syncthreads();
            if (warp == 0) {
                // start: the axis of largest variance, tilted slightly so it
                // is not orthogonal to the principal direction
                float best = vv[lane], b1 = vv[lane + 32];
                int bi = lane;
                if (b1 > best) {
                    best = b1;
                    bi = lane + 32;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                }
                __syncwarp();
                vv[lane] = lane < D ? (lane == bi ? 1.f : 1e-3f) : 0.f;
                vv[lane + 32] = lane + 32 < D ? (lane + 32 == bi ? 1.f : 1e-3f) : 0.f;
            }
            __syncthreads();
            for (int it = 0; it < kPowerIters; ++it) {
                float c0 = 0.f, c1 = 0.f;
                const float v0 = vv[lane], v1 = vv[lane + 32];
                const float m0 = mu[lane], m1 = mu[lane + 32];
                for (int i = warp; i < m; i += kOrderWarps) {
                    const int j = (int)(skey[s0 + i] & 0xFFFFu);
                    const float y0 = lane < D ? row_elem(hi, j, D, lane) - m0 : 0.f;
                    const float y1 = lane + 32 < D ? row_elem(hi, j, D, lane + 32) - m1 : 0.f;
                    const float dot = warp_allsum(fmaf(y0, v0, y1 * v1));
                    c0 = fmaf(y0, dot, c0);
                    c1 = fmaf(y1, dot, c1);
                }
                red[warp][lane] = c0;
                red[warp][lane + 32] = c1;
                __syncthreads();
                if (warp == 0) {
                    float s0v = 0.f, s1v = 0.f;
                    for (int w = 0; w < kOrderWarps; ++w) {
                        s0v += red[w][lane];
                        s1v += red[w][lane + 32];
                    }
                    const float nrm = warp_allsum(fmaf(s0v, s0v, s1v * s1v));
                    if (nrm > 0.f) {
                        const float inv = rsqrtf(nrm);
                        vv[lane] = s0v * inv;
                        vv[lane + 32] = s1v * inv;
                    }
                }
                __syncthreads();
            }
            {
                const float v0 = vv[lane], v1 = vv[lane + 32];
                const float m0 = mu[lane], m1 = mu[lane + 32];
                for (int i = warp; i < m; i += kOrderWarps) {
                    const int j = (int)(skey[s0 + i] & 0xFFFFu);
                    const float y0 = lane < D ? row_elem(hi, j, D, lane) - m0 : 0.f;
                    const float y1 = lane + 32 < D ? row_elem(hi, j, D, lane + 32) - m1 : 0.f;
                    const float p = warp_allsum(fmaf(y0, v0, y1 * v1));
                    __syncwarp();
                    if (lane == 0) skey[s0 + i] = order_key(nd, float_order_bits(p), j);
                }
            }
            __syncthreads();
        }
        __syncthreads();
        // bitonic sort of all keys: nodes stay contiguous and in order, each
        // node sorted by its projections
        for (int k = 2; k <= Lp; k <<= 1)
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = tid; i < Lp; i += kOrderThreads) {
                    const int ix = i ^ jj;
                    if (ix > i) {
                        const unsigned long long a = skey[i], b = skey[ix];
                        const bool up = (i & k) == 0;
                        if ((a > b) == up) {
                            skey[i] = b;
                            skey[ix] = a;
                        }
                    }
                }
                __syncthreads();
            }
        if (tid == 0) {
            const int nxt = cur ^ 1;
            int c2 = 0;
            for (int nd = 0; nd < cnt; ++nd) {
                const int s0 = ns[cur][nd], m = nz[cur][nd];
                if (m > kTcN) {
                    const int nl = ((m / kTcN + 1) / 2) * kTcN;
                    ns[nxt][c2] = s0;
                    nz[nxt][c2++] = nl;
                    ns[nxt][c2] = s0 + nl;
                    nz[nxt][c2++] = m - nl;
                } else {
                    ns[nxt][c2] = s0;
                    nz[nxt][c2++] = m;
                }
            }
            ncount[nxt] = c2;
        }
        __syncthreads();
        cur ^= 1;
    }
    for (int i = tid; i < L; i += kOrderThreads) lperm[i] = (int)(skey[i] & 0xFFFFu);
}

// Block c: centroid of chunk c (its landmarks in the internal order) and the
// squared norms in the internal order (NaN padding to a multiple of kTcN).
__global__ void chunk_center_kernel(const float *__restrict__ hi, const float *__restrict__ norms,
                                    const int *__restrict__ lperm, int L, int D,
                                    float *__restrict__ centers, float *__restrict__ norms_int) {
    const int c = blockIdx.x, t = threadIdx.x;  // kTcN threads
    const int j0 = c * kTcN;
    const int cnt = L - j0 < kTcN ? L - j0 : kTcN;
    const int jp = j0 + t;
    norms_int[jp] = jp < L ? norms[lperm[jp]] : __int_as_float(0x7fc00000);
    if (t < D) {
        float s = 0.f;
        for (int i = 0; i < cnt; ++i) s += row_elem(hi, lperm[j0 + i], D, t);
        centers[(size_t)c * D + t] = s / (float)cnt;
    }
}

// Block c: the chunks ordered by the distance of their centroids from chunk
// c's (ties to the lower chunk), corder[c * nch + r].
__global__ void chunk_visit_order_kernel(const float *__restrict__ centers, int nch, int D,
                                         unsigned short *__restrict__ corder) {
    __shared__ unsigned long long key[kOrderMaxL / kTcN];
    const int c = blockIdx.x, t = threadIdx.x;  // kOrderMaxL / kTcN threads
    constexpr int P = kOrderMaxL / kTcN;
    if (t < nch) {
        float s = 0.f;
        for (int i = 0; i < D; ++i) {
            const float d = centers[(size_t)t * D + i] - centers[(size_t)c * D + i];
            s = fmaf(d, d, s);
        }
        key[t] = ((unsigned long long)float_order_bits(s) << 32) | (unsigned)t;
    } else {
        key[t] = ~0ull;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            const int ix = t ^ jj;
            if (ix > t) {
                const unsigned long long a = key[t], b = key[ix];
                const bool up = (t & k) == 0;
                if ((a > b) == up) {
                    key[t] = b;
                    key[ix] = a;
                }
            }
            __syncthreads();
        }
    if (t < nch) corder[(size_t)c * nch + t] = (unsigned short)(key[t] & 0xFFFFu);
}

cudaError_t launch_landmark_order(const float *hi, const float *norms, int L, int D, int *lperm,
                                  float *centers, float *norms_int, unsigned short *corder,
                                  cudaStream_t stream, bool reorder) {
    if (L > kOrderMaxL || L < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (reorder) {
        int Lp = 1;
        while (Lp < L) Lp <<= 1;
        if (Lp < 2) Lp = 2;
        const size_t smem = (size_t)Lp * sizeof(unsigned long long);
        e = cudaFuncSetAttribute(landmark_order_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        landmark_order_kernel<<<1, kOrderThreads, smem, stream>>>(hi, L, D, Lp, lperm);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int nch = (L + kTcN - 1) / kTcN;
    chunk_center_kernel<<<nch, kTcN, 0, stream>>>(hi, norms, lperm, L, D, centers, norms_int);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    chunk_visit_order_kernel<<<nch, kOrderMaxL / kTcN, 0, stream>>>(centers, nch, D, corder);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Points of one pass grouped by home chunk.  Block b owns the contiguous
// range [b P, (b + 1) P) of the pass's points.

// home[i] = the chunk with the nearest centroid (FP32, ties to the lower
// chunk); counts[b * nch + c] = how many of block b's points have home c.
template <int D>
__global__ void point_home_kernel(const float *__restrict__ X, long long n, int per_block,
                                  const float *__restrict__ centers, int nch,
                                  const float *__restrict__ center,
                                  unsigned short *__restrict__ home, int *__restrict__ counts) {
    extern __shared__ float sc[];  // nch x D centroids
    __shared__ int hist[kOrderMaxL / kTcN];
    const int tid = threadIdx.x;
    for (int i = tid; i < nch * D; i += blockDim.x) sc[i] = centers[i];
    for (int i = tid; i < nch; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const long long p0 = (long long)blockIdx.x * per_block;
    const long long p1 = p0 + per_block < n ? p0 + per_block : n;
    for (long long i = p0 + tid; i < p1; i += blockDim.x) {
        float4 x[D / 4];
        const float4 *xp = reinterpret_cast<const float4 *>(X + (size_t)i * D);
#pragma unroll
        for (int e = 0; e < D / 4; ++e) x[e] = centred(__ldg(xp + e), center, e);
        float best = INFINITY;
        int bc = 0;
        for (int c = 0; c < nch; ++c) {
            const float4 *cc = reinterpret_cast<const float4 *>(sc + c * D);
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int e = 0; e < D / 4; ++e) {
                const float4 q = cc[e];
                const float d0 = x[e].x - q.x, d1 = x[e].y - q.y;
                const float d2 = x[e].z - q.z, d3 = x[e].w - q.w;
                s0 = fmaf(d0, d0, s0);
                s1 = fmaf(d1, d1, s1);
                s0 = fmaf(d2, d2, s0);
                s1 = fmaf(d3, d3, s1);
            }
            const float s = s0 + s1;
            if (s < best) {
                best = s;
                bc = c;
            }
        }
        home[i] = (unsigned short)bc;
        atomicAdd(&hist[bc], 1);
    }
    __syncthreads();
    for (int c = tid; c < nch; c += blockDim.x) counts[(size_t)blockIdx.x * nch + c] = hist[c];
}

// perm[pos] = the point at visiting position pos: buckets by home in chunk
// order, inside a bucket by block and then by position in the block (so the
// input order is kept); tile_home[t] = home of the point at position 128 t.
__global__ void point_scatter_kernel(long long n, int per_block, int nblocks, int nch,
                                     const unsigned short *__restrict__ home,
                                     const int *__restrict__ counts, int *__restrict__ perm,
                                     unsigned short *__restrict__ tile_home) {
    constexpr int P = kOrderMaxL / kTcN;
    __shared__ int base[P], total[P];
    __shared__ int wcnt[8][P];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;  // 256 threads
    for (int c = tid; c < nch; c += blockDim.x) {
        int tot = 0, before = 0;
        for (int b = 0; b < nblocks; ++b) {
            const int v = counts[(size_t)b * nch + c];
            tot += v;
            if (b < (int)blockIdx.x) before += v;
        }
        total[c] = tot;
        base[c] = before;
    }
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int c = 0; c < nch; ++c) {
            const int t = total[c];
            base[c] += run;
            run += t;
        }
    }
    for (int i = tid; i < 8 * P; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const long long p0 = (long long)blockIdx.x * per_block;
    const long long p1 = p0 + per_block < n ? p0 + per_block : n;
    for (long long r0 = p0; r0 < p1; r0 += blockDim.x) {
        const long long i = r0 + tid;
        const bool act = i < p1;
        const int c = act ? (int)home[i] : -1 - lane;  // inactive lanes match nobody
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (act && rank == 0) wcnt[warp][c] = __popc(peers);
        __syncthreads();
        if (act) {
            int off = base[c] + rank;
            for (int w = 0; w < warp; ++w) off += wcnt[w][c];
            perm[off] = (int)i;
            if ((off & (kTcRows - 1)) == 0) tile_home[off / kTcRows] = (unsigned short)c;
        }
        __syncthreads();
        for (int c2 = tid; c2 < nch; c2 += blockDim.x) {
            int s = 0;
            for (int w = 0; w < 8; ++w) {
                s += wcnt[w][c2];
                wcnt[w][c2] = 0;
            }
            base[c2] += s;
        }
        __syncthreads();
    }
}

cudaError_t launch_point_order(const float *X, long long n, int D, const float *centers, int nch,
                               const float *center, unsigned short *home, int *counts,
                               int nblocks, int *perm, unsigned short *tile_home,
                               cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    if (nch > kOrderMaxL / kTcN || D % 4 != 0 || D < 4 || D > 64) return cudaErrorInvalidValue;
    long long per = (n + nblocks - 1) / nblocks;
    per = (per + 255) / 256 * 256;
    const int nb = (int)((n + per - 1) / per);
    const size_t smem = (size_t)nch * D * sizeof(float);
    switch (D) {
#define ESOM_HOME_CASE(DV)                                                                    \
    case DV:                                                                                  \
        point_home_kernel<DV><<<nb, 256, smem, stream>>>(X, n, (int)per, centers, nch, center, \
                                                         home, counts);                       \
        break;
        ESOM_HOME_CASE(4) ESOM_HOME_CASE(8) ESOM_HOME_CASE(12) ESOM_HOME_CASE(16)
        ESOM_HOME_CASE(20) ESOM_HOME_CASE(24) ESOM_HOME_CASE(28) ESOM_HOME_CASE(32)
        ESOM_HOME_CASE(36) ESOM_HOME_CASE(40) ESOM_HOME_CASE(44) ESOM_HOME_CASE(48)
        ESOM_HOME_CASE(52) ESOM_HOME_CASE(56) ESOM_HOME_CASE(60) ESOM_HOME_CASE(64)
#undef ESOM_HOME_CASE
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    point_scatter_kernel<<<nb, 256, 0, stream>>>(n, (int)per, nb, nch, home, counts, perm,
                                                 tile_home);
    return cudaGetLastError();
}

// ipos[lperm[i]] = i, one thread per position.
__global__ void landmark_rank_kernel(const int *__restrict__ lperm, int L, int *__restrict__ ipos) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L) ipos[lperm[i]] = i;
}

// ptab_pos[i * L + j] = ptab[lperm[i] * L + lperm[j]]: one block row per
// position i (grid.y), threads over j; the source row is read in the order
// lperm gives, the destination row written contiguously.
__global__ void pair_table_positions_kernel(const float2 *__restrict__ ptab,
                                            const int *__restrict__ lperm, int L,
                                            float2 *__restrict__ ptab_pos) {
    const int i = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L || j >= L) return;
    const size_t src = (size_t)__ldg(lperm + i) * L;
    ptab_pos[(size_t)i * L + j] = __ldg(ptab + src + __ldg(lperm + j));
}

cudaError_t launch_pair_table_positions(const float2 *ptab, const int *lperm, int L,
                                        float2 *ptab_pos, int *ipos, cudaStream_t stream) {
    if (L < 1) return cudaSuccess;
    landmark_rank_kernel<<<(L + 255) / 256, 256, 0, stream>>>(lperm, L, ipos);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((L + 255) / 256), (unsigned)L);
    pair_table_positions_kernel<<<grid, 256, 0, stream>>>(ptab, lperm, L, ptab_pos);
    return cudaGetLastError();
}

}  // namespace esom
