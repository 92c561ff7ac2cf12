// C ABI of libesom (declared in include/esom.h): handles, argument checks,
// landmark staging, launch configuration and the host-buffer pipeline.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "esom.h"
#include "esom_ctx.h"
#include "esom_kernels.h"
#include "esom_variants.h"

using esom::FusedArgs;
using esom::KernelOps;

namespace {

thread_local char g_last_error[512] = "";

esom_status fail(esom_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

esom_status cuda_fail(cudaError_t e, const char *what) {
    return fail(ESOM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Points per chunk of the host-buffer pipeline.
// Host-buffer pipeline: points move in chunks of at most kHostChunk (one
// k-NN pass), the first and the last of one wave of the handle's k-NN kernel
// (its resident blocks x the points of a tile), so that only a small input
// copy precedes the first launch and a small output copy follows the last
// one, and neither edge chunk leaves a partial wave; every other copy
// overlaps a launch.
constexpr long long kHostChunk = 1 << 19;

long long host_chunk(long long p0, long long n, long long edge) {
    const long long left = n - p0;
    if (p0 == 0) return left < edge ? left : edge;
    if (left <= edge) return left;
    return left - edge < kHostChunk ? left - edge : kHostChunk;
}

// Operand precision of a tensor-core screening mode.
int tc_prec(int screening) { return screening == ESOM_SCREEN_BF16 ? esom::kTcBf16 : esom::kTcTf32; }

}  // namespace

namespace esom {
void fill_args(const esom_ctx *h, const float *points, long long n, float *out, float boost,
               float adjust, FusedArgs *a) {
    memset(a, 0, sizeof(*a));
    a->X = points;
    a->n = n;
    a->hi = h->hi;
    a->lo = h->lo;
    a->norms = h->norms;
    a->lmax = reinterpret_cast<const float *>(h->status + 1);
    key_layout(h->L, &a->key_mask, &a->key_quant);
    a->L = h->L;
    a->k = h->k;
    a->boost = boost;
    a->adjust = adjust;
    a->out = out;
    a->mode = kProject;
    a->chunk = h->chunk;
    a->nchunks = h->nchunks;
    a->ntiles = (n + kThreads - 1) / kThreads;
    a->status = h->status;
    a->img = h->img;
    // the pair constants from the handle's table (whichever it keeps)
    a->ptab = h->ptab;
    a->qtab = h->qtab;
    // (current whenever screening is on: build_screening refreshes it)
    a->ptab_pos = h->screening && h->order_on ? h->ptab_pos : nullptr;
    a->ipos = a->ptab_pos ? h->ipos : nullptr;
    a->center = h->centered ? h->center : nullptr;
    a->tc_chunks = (h->L + kTcN - 1) / kTcN;
    a->refine_list = h->refine_list;
    a->refine_count = reinterpret_cast<unsigned *>(h->status) + 4;
}

int set_error(int s, const char *msg) {
    snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
    return s;
}

// One thread per landmark: squared norm (FMA chain, logical order), the
// running maximum of the norms (non-negative floats order like their bit
// patterns), and the row rewritten in place with its chunks swizzled.
__global__ void landmark_prep_kernel(float *__restrict__ hi, int L, int D,
                                     float *__restrict__ norms, float *__restrict__ lmax,
                                     int padded, const float *__restrict__ center) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= padded) return;
    if (j >= L) {
        // padding: NaN, so a screening value built from it never passes a
        // threshold (every comparison with NaN is false)
        norms[j] = __int_as_float(0x7fc00000);
        return;
    }
    float4 *row = reinterpret_cast<float4 *>(hi + (size_t)j * D);
    float4 buf[16];
    const int c = D / 4;
    float s = 0.f;
    for (int e = 0; e < c; ++e) {
        buf[e] = centred(row[e], center, e);
        s = fmaf(buf[e].x, buf[e].x, s);
        s = fmaf(buf[e].y, buf[e].y, s);
        s = fmaf(buf[e].z, buf[e].z, s);
        s = fmaf(buf[e].w, buf[e].w, s);
    }
    const int f = swz(D, j);
    for (int e = 0; e < c; ++e) row[e ^ f] = buf[e];
    norms[j] = s;
    atomicMax(reinterpret_cast<int *>(lmax), __float_as_int(sqrtf(s)));
}

cudaError_t launch_landmark_prep(float *hi, int L, int D, float *norms, float *lmax,
                                 cudaStream_t stream, int pad, const float *center) {
    const int padded = (L + pad - 1) / pad * pad;
    landmark_prep_kernel<<<(padded + 255) / 256, 256, 0, stream>>>(hi, L, D, norms, lmax,
                                                                   padded, center);
    return cudaGetLastError();
}

// One thread per coordinate: the landmarks' mean, summed in FP64 in landmark
// order (deterministic), rounded to the nearest integer.
__global__ void landmark_center_kernel(const float *__restrict__ hi, int L, int D,
                                       float *__restrict__ center) {
    const int i = threadIdx.x;
    if (i >= D) return;
    double sum = 0.0;
    for (int j = 0; j < L; ++j) sum += (double)hi[(size_t)j * D + i];
    center[i] = (float)rint(sum / (double)L);
}

cudaError_t launch_landmark_center(const float *hi, int L, int D, float *center,
                                   cudaStream_t stream) {
    landmark_center_kernel<<<1, 64, 0, stream>>>(hi, L, D, center);
    return cudaGetLastError();
}

// One thread per 16-byte piece of a chunk image: piece c of column block blk
// of landmark j holds row bytes blk * row_bytes + 16 c .. + 15 of the split
// row -- high parts (the rounding of each value to TF32 or BF16, nearest) in
// the first half of the image, low parts (the rounding of the remainder) in
// the second -- zero beyond d and for rows beyond L.  The rows of hi are
// chunk-swizzled (logical chunk e at e ^ swz(D, j)).
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t bf16_rn(float x) {
    unsigned short r;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(r) : "f"(x));
    return r;
}

__global__ void tc_image_kernel(const float *__restrict__ hi, int L, int D,
                                unsigned char *__restrict__ img, int Lpad, int prec,
                                const int *__restrict__ lperm) {
    const int eb = tc_elem_bytes(prec);
    const int rb = tc_row_bytes(D, prec), nb = tc_nblk(D, prec), ppb = rb / 16;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)Lpad * nb * ppb) return;
    const int c = (int)(t % ppb);
    const int blk = (int)((t / ppb) % nb);
    const int j = (int)(t / ppb / nb);
    const int b0 = blk * rb + 16 * c;  // first byte of the piece in the split row
    uint4 h = make_uint4(0u, 0u, 0u, 0u), l = h;
    for (int q = 0; q < 4 / eb; ++q) {
        const int e = b0 / (4 * eb) + q;  // float4 index of the row
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < L && e < D / 4) {
            // internal position j holds landmark lperm[j] (the spatial order)
            const int src = lperm ? lperm[j] : j;
            v = reinterpret_cast<const float4 *>(hi + (size_t)src * D)[e ^ swz(D, src)];
        }
        const float a[4] = {v.x, v.y, v.z, v.w};
        uint32_t hw[4], lw[4];
        for (int i = 0; i < 4; ++i) {
            if (prec == kTcBf16) {
                hw[i] = bf16_rn(a[i]);
                lw[i] = bf16_rn(a[i] - __uint_as_float(hw[i] << 16));
            } else {
                const float hf = tf32_rna(a[i]);
                hw[i] = __float_as_uint(hf);
                lw[i] = __float_as_uint(tf32_rna(a[i] - hf));
            }
        }
        if (prec == kTcBf16) {
            const uint32_t h0 = hw[0] | (hw[1] << 16), h1 = hw[2] | (hw[3] << 16);
            const uint32_t l0 = lw[0] | (lw[1] << 16), l1 = lw[2] | (lw[3] << 16);
            if (q == 0) {
                h.x = h0; h.y = h1; l.x = l0; l.y = l1;
            } else {
                h.z = h0; h.w = h1; l.z = l0; l.w = l1;
            }
        } else {
            h = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            l = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
    }
    unsigned char *chunk = img + (size_t)(j / kTcN) * tc_chunk_bytes(D, prec);
    const unsigned off = tc_image_offset(D, kTcN, j % kTcN, blk, c, prec);
    *reinterpret_cast<uint4 *>(chunk + off) = h;
    *reinterpret_cast<uint4 *>(chunk + tc_chunk_bytes(D, prec) / 2 + off) = l;
}

cudaError_t launch_tc_image(const float *hi, int L, int D, unsigned char *img, int prec,
                            cudaStream_t stream, const int *lperm) {
    const int Lpad = (L + kTcN - 1) / kTcN * kTcN;
    const long long threads =
        (long long)Lpad * tc_nblk(D, prec) * (tc_row_bytes(D, prec) / 16);
    tc_image_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(hi, L, D, img, Lpad,
                                                                           prec, lperm);
    return cudaGetLastError();
}
}  // namespace esom



namespace {

esom_status configure(esom_ctx *h) {
    const int chunk = esom::landmark_chunk(h->L, h->d, h->forced_chunk);
    const int nchunks = (h->L + chunk - 1) / chunk;
    const size_t smem = esom::fused_smem_bytes(h->d, chunk, nchunks);
    // The attribute belongs to the kernel, shared by all handles: allow the
    // device's opt-in maximum so no handle can shrink another's limit.
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(shared memory opt-in)");
    if (smem > (size_t)optin)
        return fail(ESOM_EUNSUPPORTED, "needs %zu bytes of shared memory per block, device has %d",
                    smem, optin);
    e = cudaFuncSetAttribute(h->ops->func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(shared memory)");
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, h->ops->func, esom::kThreads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (bps < 1)
        return fail(ESOM_EUNSUPPORTED, "launch does not fit on an SM (shared %zu bytes)", smem);
    h->chunk = chunk;
    h->nchunks = nchunks;
    h->smem = smem;
    h->blocks_per_sm = bps;
    return ESOM_OK;
}

// The tensor-core screening's landmark operands for the current landmarks:
// the spatial order (when on), then the split chunk images in that order.
cudaError_t build_screening(esom_ctx *h, int prec, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (h->order_on) {
        // a handle that keeps its order (the frame server's sessions, whose
        // landmarks move a little per frame) recomputes it only the first time
        const bool reorder = !h->keep_order || !h->order_valid;
        e = esom::launch_landmark_order(h->hi, h->norms, h->L, h->d, h->lperm, h->centers,
                                        h->norms_int, h->corder, st, reorder);
        if (e == cudaSuccess) h->order_valid = 1;
    }
    if (e == cudaSuccess)
        e = esom::launch_tc_image(h->hi, h->L, h->d, h->img, prec, st,
                                  h->order_on ? h->lperm : nullptr);
    // the pair table of the current landmarks, moved into the same order
    if (e == cudaSuccess && h->order_on && h->ptab_pos)
        e = esom::launch_pair_table_positions(h->ptab, h->lperm, h->L, h->ptab_pos, h->ipos, st);
    return e;
}

// Largest landmark rows (bytes) the re-rank kernel keeps in shared memory.
constexpr size_t kRerankResidentBytes = 100 * 1024;

esom_status check_device(const esom_ctx *h) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (cur != h->dev)
        return fail(ESOM_EINVAL, "handle belongs to device %d but device %d is current", h->dev,
                    cur);
    return ESOM_OK;
}

// Which projection kernel the handle's tables call for (PairMode: 0 pair
// table, 1 squared-distance table, 2 neither).
int proj_mode(const esom_ctx *h) { return h->ptab ? 0 : h->qtab ? 1 : 2; }

// Kernel timing (esom_set_timing): CUDA events on the launching stream
// around each kernel, folded into per-kind totals when the ring of event
// pairs fills or when the totals are read.
void time_fold(esom_ctx *h) {
    for (int i = 0; i < h->tcount; ++i) {
        float ms = 0.f;
        if (cudaEventSynchronize(h->tev[i][1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, h->tev[i][0], h->tev[i][1]) == cudaSuccess) {
            h->tms[h->tkind[i]] += ms;
            h->tlaunch[h->tkind[i]] += 1;
        }
    }
    h->tcount = 0;
}

struct KernelTimer {
    esom_ctx *h;
    cudaStream_t st;
    int slot = -1;
    KernelTimer(esom_ctx *h_, int kind, cudaStream_t s) : h(h_), st(s) {
        if (!h->timing) return;
        if (h->tcount == esom_ctx::kTimed) time_fold(h);
        slot = h->tcount++;
        h->tkind[slot] = kind;
        cudaEventRecord(h->tev[slot][0], st);
    }
    ~KernelTimer() {
        if (slot >= 0) cudaEventRecord(h->tev[slot][1], st);
    }
};

// Projection from given neighbours by the library's kernel (one thread per
// point, distance table), the launch the split path makes after its k-NN.
// The FP64 recomputation of the rows the projection just listed (one warp a
// row), and the reset of the list for the next launch is the caller's.
cudaError_t launch_refine(esom_ctx *h, const FusedArgs &p, cudaStream_t stream) {
    return h->ops->launch_refine(p, 2 * h->num_sms, stream);
}

esom_status launch_projection(esom_ctx *h, FusedArgs p0, cudaStream_t stream) {
    p0.ptab = h->ptab;
    p0.qtab = h->qtab;
    p0.mode = esom::kProject;
    const int pm = proj_mode(h);
    unsigned *rcount = reinterpret_cast<unsigned *>(h->status) + 4;
    // passes of at most kTcPass points: the refine list holds one pass
    for (long long off = 0; off < p0.n; off += esom::kTcPass) {
        FusedArgs p = p0;
        p.n = p0.n - off < esom::kTcPass ? p0.n - off : esom::kTcPass;
        p.X = p0.X + off * h->d;
        p.idx = p0.idx + off * h->k;
        p.dist2 = p0.dist2 + off * h->k;
        p.out = p0.out + off * 2;
        if (off > 0) p.perm = nullptr;  // a visiting order covers one pass
        cudaError_t e = cudaMemsetAsync(rcount, 0, sizeof(unsigned), stream);
        if (e == cudaSuccess) {
            p.ntiles = (p.n + esom::proj_threads(pm) - 1) / esom::proj_threads(pm);
            long long grid = (long long)h->proj_blocks_per_sm * h->num_sms;
            if (grid > p.ntiles) grid = p.ntiles;
            KernelTimer kt(h, ESOM_KERNEL_PROJECT, stream);
            e = h->ops->launch_proj[pm](p, (int)grid, h->proj_smem, stream);
        }
        if (e == cudaSuccess) {
            KernelTimer kt(h, ESOM_KERNEL_REFINE, stream);
            e = launch_refine(h, p, stream);
        }
        h->launches += 2;
        if (e != cudaSuccess) return cuda_fail(e, "projection kernel launch");
    }
    return ESOM_OK;
}

esom_status launch(esom_ctx *h, const float *points, long long n, float *out, int *idx,
                   float *dist2, float boost, float adjust, int mode, cudaStream_t stream) {
    FusedArgs a;
    esom::fill_args(h, points, n, out, boost, adjust, &a);
    a.idx = idx;
    a.dist2 = dist2;
    a.mode = mode;
    cudaError_t e = cudaSuccess;
    if (h->screening || (h->split && mode == esom::kProject)) {
        // Split execution: the k-NN kernel (tensor-core or plain); for a
        // projection, in passes of kTcPass points through the handle's
        // neighbour scratch, each followed by the projection kernel.
        // Points whose certificate fails go to the handle's fail list (the
        // count lives in status word 3) and are resolved by the warp-per-point
        // rescan kernel after the pass; a pass holds at most kTcPass points.
        unsigned *fail_count = reinterpret_cast<unsigned *>(h->status) + 3;
        // proj_out (tensor-core plans, projection): the exact re-rank and the
        // projection run as one kernel writing proj_out, and the points whose
        // certificate failed are projected after their rescan
        auto knn = [&](FusedArgs k, long long cnt, float *proj_out) -> cudaError_t {
            k.mode = esom::kKnn;
            k.fail_list = h->fail_list;
            k.fail_count = fail_count;
            // status words 3 and 4: the fail count and the refine count
            cudaError_t r = cudaMemsetAsync(fail_count, 0, 2 * sizeof(unsigned), stream);
            if (r != cudaSuccess) return r;
            if (h->screening) {
                // points grouped by home chunk; the tensor-core k-NN writes
                // screened lists, re-ranked exactly by the next kernel
                FusedArgs t = k;
                t.m_dot = esom::tc_dot_bound(h->d, tc_prec(h->screening));
                t.cand = h->cand;
                if (h->order_on) {
                    KernelTimer kt(h, ESOM_KERNEL_ORDER, stream);
                    r = esom::launch_point_order(k.X, cnt, h->d, h->centers,
                                                 (h->L + esom::kTcN - 1) / esom::kTcN, k.center,
                                                 h->home, h->counts, esom::kOrderBlocks, h->perm,
                                                 h->tile_home, stream);
                    if (r != cudaSuccess) return r;
                    h->launches += 2;
                    t.perm = h->perm;
                    t.tile_home = h->tile_home;
                    t.corder = h->corder;
                    t.lperm = h->lperm;
                    t.norms = h->norms_int;
                }
                const long long tiles = (cnt + esom::kTcRows - 1) / esom::kTcRows;
                long long grid = (long long)h->tc_blocks_per_sm * h->num_sms;
                if (grid > tiles) grid = tiles;
                {
                    KernelTimer kt(h, ESOM_KERNEL_TC_KNN, stream);
                    r = h->tc->launch(t, (int)grid, h->tc_smem, stream);
                }
                if (r != cudaSuccess) return r;
                ++h->launches;
                if (proj_out) {
                    const int pm = proj_mode(h);
                    FusedArgs rp = t;
                    rp.mode = esom::kProject;
                    rp.out = proj_out;
                    rp.norms = h->norms;
                    const long long ptiles =
                        (cnt + esom::proj_threads(pm) - 1) / esom::proj_threads(pm);
                    long long pgrid = (long long)h->rproj_blocks_per_sm * h->num_sms;
                    if (pgrid > ptiles) pgrid = ptiles;
                    {
                        KernelTimer kt(h, ESOM_KERNEL_RERANK_PROJECT, stream);
                        r = h->ops->launch_rproj[pm](rp, (int)pgrid, h->proj_smem, stream);
                    }
                    if (r != cudaSuccess) return r;
                    {
                        KernelTimer kt(h, ESOM_KERNEL_RESCAN, stream);
                        r = h->ops->launch_rescan(k, 2 * h->num_sms, stream);
                    }
                    if (r != cudaSuccess) return r;
                    // the failed points, from their rescanned neighbours
                    FusedArgs pf = k;
                    pf.mode = esom::kProject;
                    pf.out = proj_out;
                    pf.perm = nullptr;
                    pf.rows_list = h->fail_list;
                    pf.rows_count = fail_count;
                    {
                        KernelTimer kt(h, ESOM_KERNEL_PROJECT, stream);
                        r = h->ops->launch_proj[pm](pf, h->num_sms, h->proj_smem, stream);
                    }
                    if (r != cudaSuccess) return r;
                    h->launches += 4;  // re-rank + projection, rescan, projection, refine
                    KernelTimer kt(h, ESOM_KERNEL_REFINE, stream);
                    return launch_refine(h, pf, stream);
                }
                FusedArgs rr = t;
                rr.norms = h->norms;
                rr.nchunks = h->rerank_smem > esom::rerank_smem_bytes(h->d, h->L, false) ? 1 : 2;
                const long long rtiles = (cnt + esom::kThreads - 1) / esom::kThreads;
                long long rgrid = (long long)h->rerank_blocks_per_sm * h->num_sms;
                if (rgrid > rtiles) rgrid = rtiles;
                KernelTimer kt(h, ESOM_KERNEL_RERANK, stream);
                r = h->ops->launch_rerank(rr, (int)rgrid, h->rerank_smem, stream);
                ++h->launches;
            } else {
                k.ntiles = (cnt + esom::kThreads - 1) / esom::kThreads;
                long long grid = (long long)h->blocks_per_sm * h->num_sms;
                if (grid > k.ntiles) grid = k.ntiles;
                KernelTimer kt(h, ESOM_KERNEL_FUSED, stream);
                r = h->ops->launch(k, (int)grid, h->smem, stream);
                ++h->launches;
            }
            if (r != cudaSuccess) return r;
            ++h->launches;
            KernelTimer kt(h, ESOM_KERNEL_RESCAN, stream);
            return h->ops->launch_rescan(k, 2 * h->num_sms, stream);
        };
        if (mode == esom::kKnn) {
            for (long long off = 0; off < n && e == cudaSuccess; off += esom::kTcPass) {
                const long long cnt = n - off < esom::kTcPass ? n - off : esom::kTcPass;
                FusedArgs k = a;
                k.X = points + off * h->d;
                k.n = cnt;
                k.idx = idx + off * h->k;
                k.dist2 = dist2 ? dist2 + off * h->k : nullptr;
                e = knn(k, cnt, nullptr);
            }
        } else {
            for (long long off = 0; off < n && e == cudaSuccess; off += esom::kTcPass) {
                const long long cnt = n - off < esom::kTcPass ? n - off : esom::kTcPass;
                FusedArgs k = a;
                k.X = points + off * h->d;
                k.n = cnt;
                k.idx = h->tc_idx;
                k.dist2 = h->tc_d2;
                if (h->screening) {
                    e = knn(k, cnt, out + off * 2);
                    continue;
                }
                e = knn(k, cnt, nullptr);
                if (e != cudaSuccess) break;
                FusedArgs p = k;
                p.out = out + off * 2;
                // the points in the k-NN's visiting order: neighbouring
                // threads then share landmark rows and table rows
                p.perm = h->screening && h->order_on ? h->perm : nullptr;
                // rows resident when they fit the configured shared memory;
                // the projection kernel reads the distance table whenever
                // there is one (measured 22% faster than recomputing from
                // resident rows at mixture30_d16; the values are the same)
                const esom_status ps = launch_projection(h, p, stream);
                if (ps != ESOM_OK) return ps;
            }
        }
    } else {
        // the fused kernel, in passes of at most kTcPass points (the refine
        // list holds one pass), each projection followed by the FP64
        // recomputation of the points it listed
        unsigned *rcount = reinterpret_cast<unsigned *>(h->status) + 4;
        for (long long off = 0; off < n && e == cudaSuccess; off += esom::kTcPass) {
            FusedArgs f = a;
            f.n = n - off < esom::kTcPass ? n - off : esom::kTcPass;
            f.X = points + off * h->d;
            if (mode == esom::kKnn) {
                f.idx = idx + off * h->k;
                f.dist2 = dist2 ? dist2 + off * h->k : nullptr;
            } else {
                f.out = out + off * 2;
            }
            f.ntiles = (f.n + esom::kThreads - 1) / esom::kThreads;
            long long grid = (long long)h->blocks_per_sm * h->num_sms;
            if (grid > f.ntiles) grid = f.ntiles;
            f.stall_ns = h->stall_ns;
            h->stall_ns = 0;
            if (mode == esom::kProject) e = cudaMemsetAsync(rcount, 0, sizeof(unsigned), stream);
            if (e == cudaSuccess) {
                KernelTimer kt(h, ESOM_KERNEL_FUSED, stream);
                e = h->ops->launch(f, (int)grid, h->smem, stream);
            }
            if (e == cudaSuccess && mode == esom::kProject) {
                KernelTimer kt(h, ESOM_KERNEL_REFINE, stream);
                e = launch_refine(h, f, stream);
            }
            h->launches += mode == esom::kProject ? 2 : 1;
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    h->points += (uint64_t)n;
    return ESOM_OK;
}

esom_status check_common(esom_ctx *h, const float *points, long long n) {
    if (!h) return fail(ESOM_EINVAL, "null handle");
    if (n < 0) return fail(ESOM_EINVAL, "n = %lld < 0", n);
    if (h->version == 0) return fail(ESOM_ENOLANDMARKS, "esom_set_landmarks has not been called");
    if (n > 0 && !points) return fail(ESOM_EINVAL, "null points");
    if (((uintptr_t)points & 15u) != 0)
        return fail(ESOM_EALIGN, "points must be 16-byte aligned");
    return check_device(h);
}

}  // namespace

extern "C" {

esom_status esom_create(int d, int L, int k, esom_handle *out) {
    if (!out) return fail(ESOM_EINVAL, "null output handle pointer");
    *out = nullptr;
    if (d < 1 || d > ESOM_MAX_D) return fail(ESOM_EINVAL, "d = %d outside [1, %d]", d, ESOM_MAX_D);
    if (d % 4 != 0) return fail(ESOM_EALIGN, "d = %d is not a multiple of 4", d);
    if (L < 1 || L > ESOM_MAX_L) return fail(ESOM_EINVAL, "L = %d outside [1, %d]", L, ESOM_MAX_L);
    if (k < 2 || k > L) return fail(ESOM_EINVAL, "k = %d outside [2, L = %d]", k, L);
    if (k > ESOM_MAX_K) return fail(ESOM_EUNSUPPORTED, "k = %d above %d", k, ESOM_MAX_K);
    const int kc = esom::list_capacity(k);
    const KernelOps *ops = esom::kernel_ops(d, kc);
    if (!ops) return fail(ESOM_EUNSUPPORTED, "no kernel for d = %d, k = %d", d, k);

    esom_ctx *h = new (std::nothrow) esom_ctx;
    if (!h) return fail(ESOM_ENOMEM, "host allocation of the handle failed");
    h->d = d;
    h->L = L;
    h->k = k;
    h->kc = kc;
    h->ops = ops;
    cudaError_t e = cudaGetDevice(&h->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "device query");
    }
    e = cudaMalloc(&h->hi, (size_t)L * d * sizeof(float));
    // 2-D positions padded to 16 bytes, so they can be bulk-copied whole
    if (e == cudaSuccess) e = cudaMalloc(&h->lo, ((size_t)L * 2 * sizeof(float) + 15) & ~(size_t)15);
    if (e == cudaSuccess)
        e = cudaMalloc(&h->norms, (size_t)((L + esom::kTcN - 1) / esom::kTcN * esom::kTcN) *
                                      sizeof(float));
    if (e == cudaSuccess && L <= esom::kPtabMaxL)
        e = cudaMalloc(&h->ptab, (size_t)L * L * sizeof(float2));
    else if (e == cudaSuccess && L <= esom::kQtabMaxL)
        e = cudaMalloc(&h->qtab, (size_t)L * L * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->refine_list, (size_t)esom::kTcPass * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->status, 256);
    if (e == cudaSuccess) e = cudaMemset(h->status, 0, 256);
    if (e != cudaSuccess) {
        esom_destroy(h);
        return fail(ESOM_ENOMEM, "device allocation: %s", cudaGetErrorString(e));
    }
    esom_status s = configure(h);
    if (s != ESOM_OK) {
        esom_destroy(h);
        return s;
    }
    *out = h;
    return ESOM_OK;
}

esom_status esom_set_landmarks(esom_handle h, const float *hi, const float *lo,
                               esom_stream_t stream) {
    if (!h) return fail(ESOM_EINVAL, "null handle");
    if (!hi || !lo) return fail(ESOM_EINVAL, "null landmark pointer");
    esom_status s = check_device(h);
    if (s != ESOM_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(h->hi, hi, (size_t)h->L * h->d * sizeof(float),
                                    cudaMemcpyDefault, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->lo, lo, (size_t)h->L * 2 * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->status + 1, 0, sizeof(float), st);
    // centring: the centre of these landmarks, subtracted from the rows here
    // and from the points by every kernel
    h->centered = h->centering;
    if (e == cudaSuccess && h->centered)
        e = esom::launch_landmark_center(h->hi, h->L, h->d, h->center, st);
    if (e == cudaSuccess) e = esom::launch_landmark_prep(h->hi, h->L, h->d, h->norms,
                                                         reinterpret_cast<float *>(h->status + 1), st,
                                                         esom::kTcN,
                                                         h->centered ? h->center : nullptr);
    if (e == cudaSuccess && (h->ptab || h->qtab))
        e = h->ops->launch_pair_table(h->hi, h->lo, h->L, h->ptab, h->qtab, st);
    if (e == cudaSuccess && h->screening) e = build_screening(h, tc_prec(h->screening), st);
    if (e != cudaSuccess) return cuda_fail(e, "landmark copy");
    ++h->version;
    return ESOM_OK;
}

uint64_t esom_landmark_version(esom_handle h) { return h ? h->version : 0; }

esom_status esom_project(esom_handle h, const float *points, int64_t n, float *out, float boost,
                         float adjust, esom_stream_t stream) {
    esom_status s = check_common(h, points, n);
    if (s != ESOM_OK) return s;
    if (n > 0 && !out) return fail(ESOM_EINVAL, "null out");
    if (((uintptr_t)out & 7u) != 0) return fail(ESOM_EALIGN, "out must be 8-byte aligned");
    if (!(boost > 0.0f) || !(boost < INFINITY)) return fail(ESOM_EINVAL, "boost must be > 0");
    if (!(adjust >= 0.0f) || !(adjust < INFINITY)) return fail(ESOM_EINVAL, "adjust must be >= 0");
    if (n == 0) return ESOM_OK;
    return launch(h, points, n, out, nullptr, nullptr, boost, adjust, esom::kProject,
                  reinterpret_cast<cudaStream_t>(stream));
}

esom_status esom_knn(esom_handle h, const float *points, int64_t n, int32_t *idx, float *dist2,
                     esom_stream_t stream) {
    esom_status s = check_common(h, points, n);
    if (s != ESOM_OK) return s;
    if (n > 0 && !idx) return fail(ESOM_EINVAL, "null idx");
    if (((uintptr_t)idx & 3u) != 0 || ((uintptr_t)dist2 & 3u) != 0)
        return fail(ESOM_EALIGN, "idx and dist2 must be 4-byte aligned");
    if (n == 0) return ESOM_OK;
    return launch(h, points, n, nullptr, idx, dist2, 1.0f, 1.0f, esom::kKnn,
                  reinterpret_cast<cudaStream_t>(stream));
}

esom_status esom_project_host(esom_handle h, const float *points_host, int64_t n,
                              float *out_host, float boost, float adjust, esom_stream_t stream) {
    if (!h) return fail(ESOM_EINVAL, "null handle");
    if (n < 0) return fail(ESOM_EINVAL, "n = %lld < 0", (long long)n);
    if (h->version == 0) return fail(ESOM_ENOLANDMARKS, "esom_set_landmarks has not been called");
    if (n > 0 && (!points_host || !out_host)) return fail(ESOM_EINVAL, "null host buffer");
    if (!(boost > 0.0f) || !(boost < INFINITY)) return fail(ESOM_EINVAL, "boost must be > 0");
    if (!(adjust >= 0.0f) || !(adjust < INFINITY)) return fail(ESOM_EINVAL, "adjust must be >= 0");
    esom_status s = check_device(h);
    if (s != ESOM_OK) return s;
    if (n == 0) return ESOM_OK;
    std::lock_guard<std::mutex> lock(h->host_mu);
    cudaError_t e = cudaSuccess;
    const size_t xbytes = (size_t)kHostChunk * h->d * sizeof(float);
    const size_t obytes = (size_t)kHostChunk * 2 * sizeof(float);
    if (!h->stage_x[0]) {
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaMalloc(&h->stage_x[b], xbytes);
            if (e == cudaSuccess) e = cudaMalloc(&h->stage_out[b], obytes);
        }
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_out, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaEventCreateWithFlags(&h->ev_in[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_comp[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_free[b], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(ESOM_ENOMEM, "staging set-up: %s", cudaGetErrorString(e));
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // Order the pipeline after the caller's earlier work on `stream`.
    e = cudaEventRecord(h->ev_start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_in, h->ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_out, h->ev_start, 0);
    if (e != cudaSuccess) return cuda_fail(e, "pipeline ordering");
    bool used[2] = {false, false};
    int c = 0;
    long long edge = h->screening ? (long long)h->tc_blocks_per_sm * h->num_sms * esom::kTcRows
                                  : (long long)h->blocks_per_sm * h->num_sms * esom::kThreads;
    if (edge < 1 || edge > kHostChunk) edge = kHostChunk;
    long long cnt = 0;
    for (long long p0 = 0; p0 < n; p0 += cnt, ++c) {
        const int b = c & 1;
        cnt = host_chunk(p0, n, edge);
        // input copy waits until the previous result in this buffer left the device
        if (used[b]) e = cudaStreamWaitEvent(h->s_in, h->ev_free[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->stage_x[b], points_host + p0 * h->d,
                                (size_t)cnt * h->d * sizeof(float), cudaMemcpyHostToDevice,
                                h->s_in);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[b], h->s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->ev_in[b], 0);
        if (e != cudaSuccess) return cuda_fail(e, "host pipeline (input)");
        s = launch(h, h->stage_x[b], cnt, h->stage_out[b], nullptr, nullptr, boost, adjust,
                   esom::kProject, st);
        if (s != ESOM_OK) return s;
        e = cudaEventRecord(h->ev_comp[b], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_out, h->ev_comp[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out_host + p0 * 2, h->stage_out[b], (size_t)cnt * 2 * sizeof(float),
                                cudaMemcpyDeviceToHost, h->s_out);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_free[b], h->s_out);
        if (e != cudaSuccess) return cuda_fail(e, "host pipeline (output)");
        used[b] = true;
    }
    // The caller's stream reaches this point only after every result copy.
    for (int b = 0; b < 2; ++b)
        if (used[b]) {
            e = cudaStreamWaitEvent(st, h->ev_free[b], 0);
            if (e != cudaSuccess) return cuda_fail(e, "host pipeline (join)");
        }
    return ESOM_OK;
}

esom_status esom_device_status(esom_handle h, esom_stream_t stream) {
    if (!h) return fail(ESOM_EINVAL, "null handle");
    esom_status s = check_device(h);
    if (s != ESOM_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int flag = 0;
    e = cudaMemcpy(&flag, h->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (flag != 0) {
        e = cudaMemset(h->status, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "status clear");
        return fail(ESOM_EDEVICE, "device error flags 0x%x (bounded wait ran out)", flag);
    }
    return ESOM_OK;
}

esom_status esom_get_stats(esom_handle h, esom_stream_t stream, esom_stats *out, int reset) {
    if (!h || !out) return fail(ESOM_EINVAL, "null argument");
    esom_status s = check_device(h);
    if (s != ESOM_OK) return s;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    unsigned words[6] = {0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(words, h->status, sizeof(words), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "stats read");
    out->points = h->points;
    out->rescans = words[2];
    out->refines = words[5];
    out->launches = h->launches;
    if (reset) {
        h->launches = 0;
        e = cudaMemset(h->status + 2, 0, sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemset(h->status + 5, 0, sizeof(unsigned));
        if (e != cudaSuccess) return cuda_fail(e, "stats reset");
        h->points = 0;
    }
    return ESOM_OK;
}

esom_status esom_set_timing(esom_handle h, int on) {
    if (!h) return fail(ESOM_EINVAL, "null handle");
    esom_status s = check_device(h);
    if (s != ESOM_OK) return s;
    if (on && !h->tev[0][0]) {
        for (int i = 0; i < esom_ctx::kTimed; ++i)
            for (int j = 0; j < 2; ++j) {
                const cudaError_t e = cudaEventCreate(&h->tev[i][j]);
                if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate (kernel timing)");
            }
    }
    h->timing = on ? 1 : 0;
    return ESOM_OK;
}

esom_status esom_get_timing(esom_handle h, esom_stream_t stream, esom_kernel_times *out,
                            int reset) {
    if (!h || !out) return fail(ESOM_EINVAL, "null argument");
    esom_status s = check_device(h);
    if (s != ESOM_OK) return s;
    const cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    time_fold(h);
    for (int i = 0; i < ESOM_KERNEL_KINDS; ++i) {
        out->launches[i] = h->tlaunch[i];
        out->ms[i] = h->tms[i];
        if (reset) {
            h->tlaunch[i] = 0;
            h->tms[i] = 0.0;
        }
    }
    return ESOM_OK;
}

esom_status esom_set_landmark_chunk(esom_handle h, int chunk) {
    if (!h) return fail(ESOM_EINVAL, "null handle");
    if (chunk < 0) return fail(ESOM_EINVAL, "chunk = %d < 0", chunk);
    const int old = h->forced_chunk;
    h->forced_chunk = chunk;
    esom_status s = configure(h);
    if (s != ESOM_OK) {
        h->forced_chunk = old;
        configure(h);
    }
    return s;
}

esom_status esom_get_config(esom_handle h, esom_config *cfg) {
    if (!h || !cfg) return fail(ESOM_EINVAL, "null argument");
    cfg->d = h->d;
    cfg->L = h->L;
    cfg->k = h->k;
    cfg->kc = h->kc;
    cfg->threads_per_block = esom::kThreads;
    cfg->blocks_per_sm = h->blocks_per_sm;
    cfg->num_sms = h->num_sms;
    cfg->landmark_chunk = h->chunk;
    cfg->landmark_chunks = h->nchunks;
    cfg->shared_bytes = (int)h->smem;
    cfg->screening = h->screening;
    cfg->plan = h->screening == ESOM_SCREEN_BF16   ? ESOM_PLAN_BF16
                : h->screening == ESOM_SCREEN_TF32 ? ESOM_PLAN_TF32
                : h->split                          ? ESOM_PLAN_SPLIT
                                                    : ESOM_PLAN_FUSED;
    if (h->screening) {
        // the tensor-core k-NN kernel (the projection kernel that follows it
        // uses 256 threads and the landmark rows of the plain kernel)
        cfg->threads_per_block = esom::kTcThreads;
        cfg->blocks_per_sm = h->tc_blocks_per_sm;
        cfg->landmark_chunk = esom::kTcN;
        cfg->landmark_chunks = (h->L + esom::kTcN - 1) / esom::kTcN;
        cfg->shared_bytes = (int)h->tc_smem;
    }
    return ESOM_OK;
}

namespace {
// Configures the projection-from-neighbours kernel and allocates the
// neighbour scratch of the split (two-kernel) execution.
// Launch configuration of the projection kernel (steps 2-4 from given
// neighbours).
esom_status prepare_projection(esom_ctx *h) {
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(shared memory opt-in)");
    const int pm = proj_mode(h);
    const size_t psmem = esom::project_smem_bytes(h->L, h->kc, pm);
    if (psmem > (size_t)optin)
        return fail(ESOM_EUNSUPPORTED, "projection needs %zu bytes of shared memory", psmem);
    const void *fn = h->ops->proj_func[pm];
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(projection shared memory)");
    int pbps = 0, rbps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pbps, fn, esom::proj_threads(pm), psmem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (pbps < 1) return fail(ESOM_EUNSUPPORTED, "projection launch does not fit on an SM");
    // the re-rank + projection kernel of the tensor-core plans (same shared
    // memory layout)
    const void *rfn = h->ops->rproj_func[pm];
    e = cudaFuncSetAttribute(rfn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rbps, rfn, esom::proj_threads(pm),
                                                          psmem);
    if (e != cudaSuccess) return cuda_fail(e, "re-rank projection kernel configuration");
    if (rbps < 1) return fail(ESOM_EUNSUPPORTED, "re-rank projection launch does not fit on an SM");
    h->proj_smem = psmem;
    h->proj_blocks_per_sm = pbps;
    h->rproj_blocks_per_sm = rbps;
    return ESOM_OK;
}

// The split execution: the projection kernel's configuration and the
// neighbour scratch of one pass.
esom_status prepare_split(esom_ctx *h) {
    esom_status s = prepare_projection(h);
    if (s != ESOM_OK) return s;
    cudaError_t e = cudaSuccess;
    if (!h->tc_idx) {
        e = cudaMalloc(&h->tc_idx, (size_t)esom::kTcPass * h->k * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&h->tc_d2, (size_t)esom::kTcPass * h->k * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&h->fail_list, (size_t)esom::kTcPass * sizeof(long long));
        if (e != cudaSuccess) {
            cudaFree(h->tc_idx);
            cudaFree(h->tc_d2);
            cudaFree(h->fail_list);
            h->tc_idx = nullptr;
            h->tc_d2 = nullptr;
            h->fail_list = nullptr;
            return fail(ESOM_ENOMEM, "device allocation of the neighbour scratch: %s",
                        cudaGetErrorString(e));
        }
    }
    return ESOM_OK;
}

}  // namespace

esom_status esom_knn_variant(esom_handle h, int variant, const float *points, int64_t n,
                             int32_t *idx, float *dist2, esom_stream_t stream) {
    esom_status s = check_common(h, points, n);
    if (s != ESOM_OK) return s;
    if (variant != ESOM_KNN_BASE && variant != ESOM_KNN_BITONIC)
        return fail(ESOM_EINVAL, "unknown k-NN variant %d", variant);
    if (n > 0 && !idx) return fail(ESOM_EINVAL, "null idx");
    if (((uintptr_t)idx & 3u) != 0 || ((uintptr_t)dist2 & 3u) != 0)
        return fail(ESOM_EALIGN, "idx and dist2 must be 4-byte aligned");
    if (n == 0) return ESOM_OK;
    const esom::VariantOps *v = esom::variant_ops(h->d);
    if (!v) return fail(ESOM_EUNSUPPORTED, "no variant kernels for d = %d", h->d);
    FusedArgs a;
    esom::fill_args(h, points, n, nullptr, 1.0f, 1.0f, &a);
    a.idx = idx;
    a.dist2 = dist2;
    a.mode = esom::kKnn;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const cudaError_t e = variant == ESOM_KNN_BASE ? v->knn_base(a, st) : v->knn_bitonic(a, st);
    if (e != cudaSuccess) return cuda_fail(e, "k-NN variant launch");
    return ESOM_OK;
}

esom_status esom_project_knn(esom_handle h, int variant, const float *points, int64_t n,
                             const int32_t *idx, const float *dist2, float *out, float boost,
                             float adjust, esom_stream_t stream) {
    esom_status s = check_common(h, points, n);
    if (s != ESOM_OK) return s;
    if (variant != ESOM_PROJ_TABLE && variant != ESOM_PROJ_REGISTERS)
        return fail(ESOM_EINVAL, "unknown projection variant %d", variant);
    if (n > 0 && (!idx || !dist2 || !out)) return fail(ESOM_EINVAL, "null idx, dist2 or out");
    if ((((uintptr_t)idx | (uintptr_t)dist2) & 15u) != 0)
        return fail(ESOM_EALIGN, "idx and dist2 must be 16-byte aligned");
    if (((uintptr_t)out & 7u) != 0) return fail(ESOM_EALIGN, "out must be 8-byte aligned");
    if (!(boost > 0.0f) || !(boost < INFINITY)) return fail(ESOM_EINVAL, "boost must be > 0");
    if (!(adjust >= 0.0f) || !(adjust < INFINITY)) return fail(ESOM_EINVAL, "adjust must be >= 0");
    if (n == 0) return ESOM_OK;
    FusedArgs p;
    esom::fill_args(h, points, n, out, boost, adjust, &p);
    p.idx = const_cast<int *>(idx);
    p.dist2 = const_cast<float *>(dist2);
    p.mode = esom::kProject;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (variant == ESOM_PROJ_TABLE) {
        if (h->proj_smem == 0) {
            s = prepare_projection(h);
            if (s != ESOM_OK) return s;
        }
        s = launch_projection(h, p, st);
        if (s != ESOM_OK) return s;
    } else {
        const esom::VariantOps *v = esom::variant_ops(h->d);
        if (!v) return fail(ESOM_EUNSUPPORTED, "no variant kernels for d = %d", h->d);
        const cudaError_t e = v->project_registers(p, st);
        if (e != cudaSuccess) return cuda_fail(e, "projection variant launch");
    }
    h->points += (uint64_t)n;
    return ESOM_OK;
}

esom_status esom_set_centering(esom_handle h, int on) {
    if (!h) return fail(ESOM_EINVAL, "null handle");
    esom_status s = check_device(h);
    if (s != ESOM_OK) return s;
    if (on && !h->center) {
        const cudaError_t e = cudaMalloc(&h->center, ESOM_MAX_D * sizeof(float));
        if (e != cudaSuccess) {
            h->center = nullptr;
            return fail(ESOM_ENOMEM, "device allocation of the centre: %s", cudaGetErrorString(e));
        }
    }
    h->centering = on ? 1 : 0;
    return ESOM_OK;
}

esom_status esom_set_split(esom_handle h, int on) {
    if (!h) return fail(ESOM_EINVAL, "null handle");
    esom_status s = check_device(h);
    if (s != ESOM_OK) return s;
    if (on) {
        s = prepare_split(h);
        if (s != ESOM_OK) return s;
    }
    h->split = on ? 1 : 0;
    return ESOM_OK;
}

esom_status esom_tune(esom_handle h, const float *points, int64_t n, float *out, float boost,
                      float adjust, esom_stream_t stream, int *plan) {
    esom_status s = check_common(h, points, n);
    if (s != ESOM_OK) return s;
    if (n < 1 || !out) return fail(ESOM_EINVAL, "esom_tune needs n >= 1 points and an output");
    const long long m = n < esom::kTcPass ? n : esom::kTcPass;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    const int old_screening = h->screening, old_split = h->split;
    int best = -1;
    float best_ms = 0.f;
    for (int p = ESOM_PLAN_FUSED; p <= ESOM_PLAN_BF16; ++p) {
        s = esom_set_screening(h, p == ESOM_PLAN_TF32 ? ESOM_SCREEN_TF32
                                  : p == ESOM_PLAN_BF16 ? ESOM_SCREEN_BF16 : ESOM_SCREEN_FP32,
                               stream);
        if (s == ESOM_OK) s = esom_set_split(h, p == ESOM_PLAN_SPLIT);
        if (s != ESOM_OK) continue;  // plan unavailable here (e.g. no tensor-core kernel)
        float total = 0.f;
        for (int r = 0; r < 3 && s == ESOM_OK; ++r) {
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) s = esom_project(h, points, m, out, boost, adjust, stream);
            if (s == ESOM_OK && e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (s == ESOM_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (s == ESOM_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) s = cuda_fail(e, "tuning run");
            if (r > 0) total += ms;  // the first run warms up
        }
        if (s == ESOM_OK && (best < 0 || total < best_ms)) {
            best = p;
            best_ms = total;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0) {
        esom_set_screening(h, old_screening, stream);
        esom_set_split(h, old_split);
        return fail(ESOM_ECUDA, "no execution plan ran");
    }
    s = esom_set_screening(h, best == ESOM_PLAN_TF32 ? ESOM_SCREEN_TF32
                              : best == ESOM_PLAN_BF16 ? ESOM_SCREEN_BF16 : ESOM_SCREEN_FP32,
                           stream);
    if (s == ESOM_OK) s = esom_set_split(h, best == ESOM_PLAN_SPLIT);
    if (s == ESOM_OK && plan) *plan = best;
    return s;
}

esom_status esom_set_screening(esom_handle h, int mode, esom_stream_t stream) {
    if (!h) return fail(ESOM_EINVAL, "null handle");
    if (mode != ESOM_SCREEN_FP32 && mode != ESOM_SCREEN_TF32 && mode != ESOM_SCREEN_BF16)
        return fail(ESOM_EINVAL, "unknown screening mode %d", mode);
    esom_status s = check_device(h);
    if (s != ESOM_OK) return s;
    if (mode == ESOM_SCREEN_FP32) {
        h->screening = 0;
        return ESOM_OK;
    }
    const int prec = tc_prec(mode);
    const esom::TcOps *tc = esom::tc_ops(h->d, h->kc, prec);
    if (!tc) return fail(ESOM_EUNSUPPORTED, "no tensor-core kernel for d = %d, k = %d", h->d, h->k);
    int major = 0, minor = 0;
    cudaError_t e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, h->dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(compute capability)");
    if (major != 10 || minor != 3)
        return fail(ESOM_EUNSUPPORTED, "tensor-core screening needs sm_103 (device is sm_%d%d)",
                    major, minor);
    const size_t smem = esom::tc_smem_bytes(h->d, h->kc, prec);
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(shared memory opt-in)");
    if (smem > (size_t)optin)
        return fail(ESOM_EUNSUPPORTED, "needs %zu bytes of shared memory per block, device has %d",
                    smem, optin);
    e = cudaFuncSetAttribute(tc->func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(shared memory)");
    // Resident blocks per SM from the kernel's registers (allocated per warp
    // in units of 256) and shared memory (plus the 1 KiB the driver reserves
    // per block), at most 512 / kTcCols for the TMEM columns.
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, tc->func);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    int smem_sm = 0, regs_sm = 0;
    e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, h->dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(SM resources)");
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
    int bps = regs_sm / (warp_regs * (esom::kTcThreads / 32));
    const int by_smem = smem_sm / (int)(smem + 1024);
    if (by_smem < bps) bps = by_smem;
    if (bps * esom::kTcCols > 512) bps = 512 / esom::kTcCols;
    if (bps < 1) return fail(ESOM_EUNSUPPORTED, "tensor-core launch does not fit on an SM");
    // the projection kernel that follows each k-NN pass
    s = prepare_split(h);
    if (s != ESOM_OK) return s;
    if (!h->img) {
        // sized for TF32, the larger of the two image formats
        const size_t bytes = (size_t)((h->L + esom::kTcN - 1) / esom::kTcN) *
                             esom::tc_chunk_bytes(h->d, esom::kTcTf32);
        e = cudaMalloc(&h->img, bytes);
        if (e != cudaSuccess) {
            h->img = nullptr;
            return fail(ESOM_ENOMEM, "device allocation of the landmark images: %s",
                        cudaGetErrorString(e));
        }
    }
    // the exact re-rank of the screened lists, and its candidate buffer
    {
        const bool res = (size_t)h->L * h->d * sizeof(float) <= kRerankResidentBytes;
        const size_t rsmem = esom::rerank_smem_bytes(h->d, h->L, res);
        e = cudaFuncSetAttribute(h->ops->rerank_func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin);
        int rbps = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rbps, h->ops->rerank_func,
                                                              esom::kThreads, rsmem);
        if (e != cudaSuccess) return cuda_fail(e, "re-rank kernel configuration");
        if (rbps < 1) return fail(ESOM_EUNSUPPORTED, "re-rank launch does not fit on an SM");
        h->rerank_smem = rsmem;
        h->rerank_blocks_per_sm = rbps;
    }
    const int nch = (h->L + esom::kTcN - 1) / esom::kTcN;
    if (!h->cand) {
        e = cudaMalloc(&h->cand, (size_t)esom::kTcPass * h->kc * sizeof(float));
        if (e != cudaSuccess) {
            h->cand = nullptr;
            return fail(ESOM_ENOMEM, "device allocation of the candidate lists: %s",
                        cudaGetErrorString(e));
        }
    }
    if (h->L <= esom::kOrderMaxL && !h->lperm) {
        e = cudaMalloc(&h->lperm, (size_t)h->L * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&h->centers, (size_t)nch * h->d * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&h->norms_int, (size_t)nch * esom::kTcN * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&h->corder, (size_t)nch * nch * sizeof(unsigned short));
        if (e == cudaSuccess) e = cudaMalloc(&h->home, (size_t)esom::kTcPass * sizeof(unsigned short));
        if (e == cudaSuccess)
            e = cudaMalloc(&h->counts, (size_t)esom::kOrderBlocks * nch * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&h->perm, (size_t)esom::kTcPass * sizeof(int));
        if (e == cudaSuccess)
            e = cudaMalloc(&h->tile_home,
                           (size_t)(esom::kTcPass / esom::kTcRows) * sizeof(unsigned short));
        if (e == cudaSuccess && h->ptab)
            e = cudaMalloc(&h->ptab_pos, (size_t)h->L * h->L * sizeof(float2));
        if (e == cudaSuccess && h->ptab) e = cudaMalloc(&h->ipos, (size_t)h->L * sizeof(int));
        if (e != cudaSuccess) {
            cudaFree(h->ptab_pos);
            cudaFree(h->ipos);
            h->ptab_pos = nullptr;
            h->ipos = nullptr;
            cudaFree(h->lperm);
            cudaFree(h->centers);
            cudaFree(h->norms_int);
            cudaFree(h->corder);
            cudaFree(h->home);
            cudaFree(h->counts);
            cudaFree(h->perm);
            cudaFree(h->tile_home);
            h->lperm = nullptr;
            h->centers = h->norms_int = nullptr;
            h->corder = h->home = h->tile_home = nullptr;
            h->counts = h->perm = nullptr;
            return fail(ESOM_ENOMEM, "device allocation of the screening orders: %s",
                        cudaGetErrorString(e));
        }
    }
    h->order_on = h->lperm != nullptr;
    if (h->version > 0) {
        e = build_screening(h, prec, reinterpret_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) return cuda_fail(e, "landmark image build");
    }
    h->tc = tc;
    h->tc_smem = smem;
    h->tc_blocks_per_sm = bps;
    h->screening = mode;
    return ESOM_OK;
}

esom_status esom_destroy(esom_handle h) {
    if (!h) return ESOM_OK;
    cudaFree(h->hi);
    cudaFree(h->lo);
    cudaFree(h->norms);
    cudaFree(h->status);
    cudaFree(h->refine_list);
    cudaFree(h->img);
    cudaFree(h->qtab);
    cudaFree(h->ptab);
    cudaFree(h->ptab_pos);
    cudaFree(h->ipos);
    for (int i = 0; i < esom_ctx::kTimed; ++i)
        for (int j = 0; j < 2; ++j)
            if (h->tev[i][j]) cudaEventDestroy(h->tev[i][j]);
    cudaFree(h->tc_idx);
    cudaFree(h->tc_d2);
    cudaFree(h->fail_list);
    cudaFree(h->center);
    cudaFree(h->cand);
    cudaFree(h->lperm);
    cudaFree(h->centers);
    cudaFree(h->norms_int);
    cudaFree(h->corder);
    cudaFree(h->home);
    cudaFree(h->counts);
    cudaFree(h->perm);
    cudaFree(h->tile_home);
    for (int b = 0; b < 2; ++b) {
        cudaFree(h->stage_x[b]);
        cudaFree(h->stage_out[b]);
        if (h->ev_in[b]) cudaEventDestroy(h->ev_in[b]);
        if (h->ev_comp[b]) cudaEventDestroy(h->ev_comp[b]);
        if (h->ev_free[b]) cudaEventDestroy(h->ev_free[b]);
    }
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->s_in) cudaStreamDestroy(h->s_in);
    if (h->s_out) cudaStreamDestroy(h->s_out);
    delete h;
    return ESOM_OK;
}

esom_status esom_test_stall(esom_handle h, int64_t limit_ns) {
    if (!h) return fail(ESOM_EINVAL, "null handle");
    if (limit_ns < 1000 || limit_ns > 2000000000)
        return fail(ESOM_EINVAL, "limit_ns = %lld outside [1e3, 2e9]", (long long)limit_ns);
    if (h->screening || h->split)
        return fail(ESOM_EINVAL, "the stall probe needs the fused plan (ESOM_PLAN_FUSED)");
    h->stall_ns = (unsigned long long)limit_ns;
    return ESOM_OK;
}

esom_status esom_selftest_drcp(const double *x, int64_t n, double *rcp, double *div,
                               esom_stream_t stream) {
    if (n < 0) return fail(ESOM_EINVAL, "n < 0");
    if (n == 0) return ESOM_OK;
    if (!x || !rcp || !div) return fail(ESOM_EINVAL, "null pointer");
    const cudaError_t e = esom::launch_drcp_selftest(x, n, rcp, div,
                                                     reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ESOM_OK : cuda_fail(e, "drcp self-test launch");
}

esom_status esom_selftest_tc_products(esom_handle h, const float *points, int64_t n, float *T,
                                      esom_stream_t stream) {
    esom_status s = check_common(h, points, n);
    if (s != ESOM_OK) return s;
    if (!h->screening) return fail(ESOM_EINVAL, "tensor-core screening is off");
    if (n > esom::kTcPass) return fail(ESOM_EINVAL, "n = %lld above %lld", (long long)n,
                                       esom::kTcPass);
    if (n == 0) return ESOM_OK;
    if (!T || ((uintptr_t)T & 15u) != 0) return fail(ESOM_EALIGN, "T must be 16-byte aligned");
    const int prec = tc_prec(h->screening);
    const esom::TcOps *op = esom::tc_dump_ops(h->d, prec);
    if (!op) return fail(ESOM_EUNSUPPORTED, "no tensor-core kernel for d = %d", h->d);
    const size_t smem = esom::tc_smem_bytes(h->d, 8, prec);
    cudaError_t e = cudaFuncSetAttribute(op->func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(shared memory)");
    FusedArgs a;
    esom::fill_args(h, points, n, nullptr, 1.f, 1.f, &a);
    a.mode = esom::kKnn;
    a.dist2 = T;
    a.lperm = h->order_on ? h->lperm : nullptr;  // the images are in this order
    const long long tiles = (n + esom::kTcRows - 1) / esom::kTcRows;
    const int grid = (int)(tiles < h->num_sms ? tiles : h->num_sms);
    e = op->launch(a, grid, smem, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ESOM_OK : cuda_fail(e, "tensor-core product dump launch");
}

const char *esom_last_error(void) { return g_last_error; }

const char *esom_status_string(esom_status s) {
    switch (s) {
        case ESOM_OK: return "ESOM_OK";
        case ESOM_EINVAL: return "ESOM_EINVAL";
        case ESOM_ENOMEM: return "ESOM_ENOMEM";
        case ESOM_EALIGN: return "ESOM_EALIGN";
        case ESOM_ENOLANDMARKS: return "ESOM_ENOLANDMARKS";
        case ESOM_ECUDA: return "ESOM_ECUDA";
        case ESOM_EUNSUPPORTED: return "ESOM_EUNSUPPORTED";
        case ESOM_EDEVICE: return "ESOM_EDEVICE";
    }
    return "ESOM_UNKNOWN";
}

}  // extern "C"
