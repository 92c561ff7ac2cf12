// Tensor-core screened k-NN kernel for sm_103a (tcgen05, TF32).
//
// Step 1 of the projection with the same result as the plain fused kernel
// (esom_fused.cuh), computed with the distance block on the tensor cores;
// esom_project follows it with project_kernel (steps 2-4 from the
// neighbours), as the paper runs k-NN and projection as two kernels with an
// exchange buffer (Section 4.4).  The paper's k-NN spends its
// time in the g x d distance block (Section 4.2, and Section 5's remark that
// the k-NN cost grows with g d); here that block is a dense contraction of a
// tile of 128 points with chunks of 64 landmarks:
//
//   T = X_tile . L_chunk^T        (tcgen05.mma kind::tf32, FP32 accumulators
//                                  in tensor memory, operands in shared
//                                  memory in the 128-byte-swizzled K-major
//                                  layout)
//   v_j = |L_j|^2 - 2 T_j         (screening value = |X - L_j|^2 - |X|^2,
//                                  up to the screening error)
//
// Each operand is split into two TF32 parts, x = x_hi + x_lo (x_hi the TF32
// rounding of x, x_lo that of the remainder), and T accumulates the three
// products x_hi l_hi + x_lo l_hi + x_hi l_lo: the dropped terms are below
// 2^-21 relative, so the screening error is of the order of an FP32 dot
// product's and the certificate almost never fails.
//
// Each selection thread owns one point (one TMEM lane), reads its 64 values
// of a chunk with two tcgen05.ld, keys them like the plain kernel (value
// with the landmark index in the low mantissa bits) and keeps the KC
// smallest.  The list is then re-ranked with exact FP32 difference-form
// distances, and a bound on the screening error certifies that no landmark
// outside the list can be among the k nearest; a point that fails is
// appended to a list that rescan_kernel (one warp per point) then resolves
// with an exact scan.
// So the neighbours and their distances are the plain kernel's, bit for
// bit (and so are the coordinates projected from them); the screening
// precision only decides how often a point is rescanned.
//
// Roles: warps 0-3 select (thread t <-> point row t <-> TMEM lane t); warp 4
// is the producer: one lane streams the landmark chunk images through a ring
// of shared-memory stages by bulk copies (cp.async.bulk + mbarrier) and
// issues the MMAs into two TMEM accumulator buffers, so the MMA of chunk c+1
// overlaps the selection of chunk c.  As soon as a tile's last chunk has
// been read (every MMA of the tile is then complete), the selection threads
// write the next tile's operand (split rows) into the one point buffer and
// only then re-rank the current tile, so the next tile's MMAs overlap that
// work.  Every
// wait is bounded; on a timeout the block raises the status word, drains
// its own copies and MMAs and frees its tensor memory.
#pragma once

#include "esom_fused.cuh"

namespace esom {

// ---------------------------------------------------------------------------
// tcgen05 / tensor-memory helpers (inline PTX).

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in a swizzled
// layout: 8-row groups SBO bytes apart, the leading byte offset unused for
// these layouts (1), descriptor version 1, layout type 2 (128-byte swizzle)
// or 4 (64-byte swizzle).  The operand base is 1024-byte aligned; a K step
// inside the row moves the start address by its bytes.
template <int ROWB>
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
    constexpr uint64_t kLayout = ROWB == 128 ? 2 : 4;
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)((8 * ROWB) >> 4) << 32) | ((uint64_t)1 << 46) | (kLayout << 61);
}

// Instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B both
// TF32 (bits 7-9 and 10-12 = 2, kind::tf32) or both BF16 (= 1, kind::f16),
// both K-major, N / 8 at bits 17-22, M / 16 at bits 24-28.
template <int PREC>
__host__ __device__ constexpr uint32_t tc_idesc() {
    return (1u << 4) | ((PREC == kTcBf16 ? 1u : 2u) << 7) | ((PREC == kTcBf16 ? 1u : 2u) << 10) |
           ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void mma_split(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    if (PREC == kTcBf16)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
}

// FP32 -> BF16, round to nearest even; and back (exact).
__device__ __forceinline__ uint32_t to_bf16_bits(float x) {
    unsigned short r;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float bf16_bits_to_f32(uint32_t b) { return __uint_as_float(b << 16); }

// Splits four values into BF16 high and low parts, packed two a word
// (element 2w in the low half of word w, as the MMA reads K-contiguous
// 16-bit elements).
__device__ __forceinline__ void split_bf16x4(float4 v, uint2 &hi, uint2 &lo) {
    const float a[4] = {v.x, v.y, v.z, v.w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h[i] = to_bf16_bits(a[i]);
        l[i] = to_bf16_bits(a[i] - bf16_bits_to_f32(h[i]));
    }
    hi = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
    lo = make_uint2(l[0] | (l[1] << 16), l[2] | (l[3] << 16));
}

// Arrives on `bar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane, waited for inside
// the same statement.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
        "[%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Smallest of three floats in one instruction (a NaN operand is ignored).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// FP32 -> TF32, round to nearest (ties away from zero); low 13 bits zero.
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// ---------------------------------------------------------------------------

// DUMP (tests of the error bound only): instead of selecting, every
// selection thread writes the raw accumulator values T_j of its point for all
// landmarks to a.dist2 (row-major, tc_chunks * kTcN per point).
template <int D, int KC, int PREC, bool DUMP = false>
__global__ void __launch_bounds__(kTcThreads, tc_minb(D, KC)) tc_kernel(const FusedArgs a) {
    static_assert(D % 4 == 0 && D >= 4 && D <= 64, "D must be a multiple of 4 in [4, 64]");
    static_assert(KC >= 8 && KC <= 36 && KC % 4 == 0, "list capacity out of range");
    constexpr int EB = tc_elem_bytes(PREC);      // bytes of an operand element
    constexpr int RB = tc_row_bytes(D, PREC);    // bytes of a row per column block
    constexpr int NB = tc_nblk(D, PREC);
    constexpr int PPB = RB / 16;                 // 16-byte pieces per block row
    constexpr int KPB = RB / 32;                 // K steps (32 bytes) per block row
    constexpr int S = tc_stages(D, PREC);
    constexpr int KS = (D * EB + 31) / 32;       // MMA K steps of 32 bytes
    constexpr uint32_t kAPart = kTcRows * RB * NB;  // x_hi (then x_lo) of a tile
    constexpr uint32_t kBPart = kTcN * RB * NB;     // l_hi (then l_lo) of a chunk
    constexpr uint32_t kBBytes = 2 * kBPart;
    constexpr uint32_t kIdesc = tc_idesc<PREC>();
    constexpr int QS = kTcRows;  // queue stride: one column per selection thread
    constexpr int QC = tc_queue(D, KC);   // queue capacity (keys a thread)
    constexpr int QI = tc_check(D, KC);   // values pushed between fullness checks
    static_assert(QI == 16 || QI == 32, "fullness checks every 16 or 32 values");
    constexpr int KF = ((KC + 7) & ~7) < 32 ? ((KC + 7) & ~7) : 32;  // first sorted block

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    unsigned char *sA = base;                      // point tile: x_hi, x_lo
    unsigned char *sB = base + 2 * kAPart;         // S landmark chunk stages
    uint32_t *qk = reinterpret_cast<uint32_t *>(sB + S * kBBytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(qk + QC * kTcRows);
    uint64_t *l_full = bars, *l_empty = bars + S;
    uint64_t *t_full = bars + 2 * S, *t_empty = bars + 2 * S + 2;
    uint64_t *a_ready = bars + 2 * S + 4, *done_bar = bars + 2 * S + 5;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + 2 * S + 8);
    volatile int *s_abort = reinterpret_cast<volatile int *>(s_tmem + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long ntiles = (a.n + kTcRows - 1) / kTcRows;
    const long long first = blockIdx.x;
    const long long my_tiles =
        first < ntiles ? (ntiles - 1 - first) / (long long)gridDim.x + 1 : 0;
    if (my_tiles == 0) return;  // whole block, before any barrier or TMEM use
    const int nch = a.tc_chunks;

    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&l_full[i], 1);
            mbar_init(&l_empty[i], 1);
        }
        mbar_init(&t_full[0], 1);
        mbar_init(&t_full[1], 1);
        mbar_init(&t_empty[0], 4);
        mbar_init(&t_empty[1], 4);
        mbar_init(a_ready, 4);
        mbar_init(done_bar, 1);
        fence_mbar_init();
        *s_abort = 0;
    }
    if (warp == 4) {
        tmem_alloc(s_tmem, kTcCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    auto raise_abort = [&]() {
        *s_abort = 1;
        atomicOr(a.status, kErrWaitTimeout);
    };
    // The landmark chunk a tile visits at step r: in the order of chunk
    // distance from the tile's home chunk when the points are grouped by
    // home, else chunk r.
    auto chunk_of = [&](long long tile, int r) -> int {
        if (!a.corder) return r;
        return (int)__ldg(a.corder + (size_t)__ldg(a.tile_home + tile) * nch + r);
    };

    if (warp == 4) {
        // ------------------------------------------------------------------
        // Producer: lane 0 streams chunk images and issues the MMAs.
        if (lane == 0) {
            const long long total = my_tiles * nch;
            long long issued = 0, landed = 0;
            auto issue = [&](long long g) {
                const int s = (int)(g % S);
                const int c = chunk_of(first + (g / nch) * gridDim.x, (int)(g % nch));
                mbar_expect_tx(&l_full[s], kBBytes);
                bulk_g2s(sB + (size_t)s * kBBytes, a.img + (size_t)c * kBBytes, kBBytes,
                         &l_full[s]);
            };
            for (; issued < total && issued < S; ++issued) issue(issued);
            bool ok = true;
            long long g = 0;
            const uint32_t ahi = smem_u32(sA), alo = ahi + kAPart;
            for (long long i = 0; i < my_tiles && ok; ++i) {
                if (!mbar_wait(a_ready, (uint32_t)(i & 1))) {
                    ok = false;
                    break;
                }
                for (int c = 0; c < nch; ++c, ++g) {
                    const int s = (int)(g % S), tb = (int)(g & 1);
                    if (*s_abort || !mbar_wait(&l_full[s], (uint32_t)((g / S) & 1))) {
                        ok = false;
                        break;
                    }
                    landed = g + 1;
                    if (!mbar_wait(&t_empty[tb], (uint32_t)(((g >> 1) & 1) ^ 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t bhi = smem_u32(sB + (size_t)s * kBBytes), blo = bhi + kBPart;
                    const uint32_t dt = tmem + (uint32_t)(tb * kTcN);
#pragma unroll
                    for (int ks = 0; ks < KS; ++ks) {
                        const uint32_t ka = (uint32_t)((ks / KPB) * kTcRows * RB + (ks % KPB) * 32);
                        const uint32_t kb = (uint32_t)((ks / KPB) * kTcN * RB + (ks % KPB) * 32);
                        mma_split<PREC>(dt, sw_desc<RB>(ahi + ka), sw_desc<RB>(bhi + kb), kIdesc,
                                        ks > 0 ? 1u : 0u);
                        mma_split<PREC>(dt, sw_desc<RB>(alo + ka), sw_desc<RB>(bhi + kb), kIdesc,
                                        1u);
                        mma_split<PREC>(dt, sw_desc<RB>(ahi + ka), sw_desc<RB>(blo + kb), kIdesc,
                                        1u);
                    }
                    mma_commit(&t_full[tb]);
                    mma_commit(&l_empty[s]);
                    // Refill the stage of the previous step (its MMA was
                    // issued one step ago) with the chunk S steps after it.
                    if (g >= 1 && g - 1 + S < total && issued == g - 1 + S) {
                        const long long h = g - 1;
                        if (!mbar_wait(&l_empty[h % S], (uint32_t)((h / S) & 1))) {
                            ok = false;
                            break;
                        }
                        issue(issued++);
                    }
                }
            }
            if (!ok) raise_abort();
            // Drain: every MMA issued, then every copy issued but not waited.
            mma_commit(done_bar);
            mbar_wait(done_bar, 0);
            for (long long h = landed; h < issued; ++h)
                mbar_wait(&l_full[h % S], (uint32_t)((h / S) & 1));
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------------
        // Selection: thread tid owns row tid of every tile of this block.
        const uint32_t mask = a.key_mask;
        const float q = a.key_quant;
        const float lmax = *a.lmax;
        const uint32_t my_lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        constexpr float kGamma = (2.25f * D + 10.f) * kU * 1.25f;

        // Writes this thread's row of tile `tile`, split into high and low
        // parts (TF32 or BF16, swizzled), into the point buffer and returns
        // |x|^2 (FP32, exact row).
        auto write_tile = [&](long long tile) -> float {
            const long long pos = tile * kTcRows + tid;
            const bool act = pos < a.n;
            const long long row = act && a.perm ? (long long)__ldg(a.perm + pos) : pos;
            const float4 *xp = reinterpret_cast<const float4 *>(a.X) + (act ? row : 0) * (D / 4);
            float xx = 0.f;
#pragma unroll
            for (int blk = 0; blk < NB; ++blk)
#pragma unroll
                for (int c = 0; c < PPB; ++c) {
                    const int b0 = blk * RB + 16 * c;  // first byte of the piece in the row
                    if (b0 >= 32 * KS) continue;       // pieces the MMA K steps do not read
                    uint4 h = make_uint4(0u, 0u, 0u, 0u), l = h;
#pragma unroll
                    for (int q = 0; q < 4 / EB; ++q) {  // float4s of x in this piece
                        const int e = b0 / (4 * EB) + q;  // float4 index of the row
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (e < D / 4 && act) {
                            v = centred(__ldg(xp + e), a.center, e);
                            xx = fmaf(v.x, v.x, xx);
                            xx = fmaf(v.y, v.y, xx);
                            xx = fmaf(v.z, v.z, xx);
                            xx = fmaf(v.w, v.w, xx);
                        }
                        if (PREC == kTcBf16) {
                            uint2 hh, ll;
                            split_bf16x4(v, hh, ll);
                            if (q == 0) {
                                h.x = hh.x; h.y = hh.y; l.x = ll.x; l.y = ll.y;
                            } else {
                                h.z = hh.x; h.w = hh.y; l.z = ll.x; l.w = ll.y;
                            }
                        } else {
                            const float4 hv = make_float4(to_tf32(v.x), to_tf32(v.y),
                                                          to_tf32(v.z), to_tf32(v.w));
                            const float4 lv =
                                make_float4(to_tf32(v.x - hv.x), to_tf32(v.y - hv.y),
                                            to_tf32(v.z - hv.z), to_tf32(v.w - hv.w));
                            h = make_uint4(__float_as_uint(hv.x), __float_as_uint(hv.y),
                                           __float_as_uint(hv.z), __float_as_uint(hv.w));
                            l = make_uint4(__float_as_uint(lv.x), __float_as_uint(lv.y),
                                           __float_as_uint(lv.z), __float_as_uint(lv.w));
                        }
                    }
                    const unsigned off = tc_image_offset(D, kTcRows, tid, blk, c, PREC);
                    *reinterpret_cast<uint4 *>(sA + off) = h;
                    *reinterpret_cast<uint4 *>(sA + kAPart + off) = l;
                }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(a_ready);
            return xx;
        };

        // Keys of 32 values of chunk base (columns h32 .. h32 + 31) into the
        // queue: half a packed FMA for the screening value, the key, the
        // threshold test and a predicated push.  Padding columns (beyond L) have NaN
        // norms, so they never pass.  Every QI values the queue is flushed
        // when a lane may not have room for QI more.
        auto push32 = [&](float (&v)[32], int jbase, float (&keys)[KC], ScanState &st,
                          float M) {
            const float4 *N4 = reinterpret_cast<const float4 *>(a.norms + jbase);
            // screening values two at a time on the packed FP32x2 pipe (each
            // lane the same fma as fmaf(-2, v, |l|^2))
#pragma unroll
            for (int jb = 0; jb < 32; jb += 4) {
                const float4 n4 = __ldg(N4 + jb / 4);
                const float2 s01 = __ffma2_rn(make_float2(v[jb], v[jb + 1]),
                                              make_float2(-2.f, -2.f), make_float2(n4.x, n4.y));
                const float2 s23 = __ffma2_rn(make_float2(v[jb + 2], v[jb + 3]),
                                              make_float2(-2.f, -2.f), make_float2(n4.z, n4.w));
                v[jb] = s01.x;
                v[jb + 1] = s01.y;
                v[jb + 2] = s23.x;
                v[jb + 3] = s23.y;
            }
            // In groups of 8 landmarks: a group is skipped when no lane of
            // the warp can queue one of its values.  A key differs from its
            // value v by at most q|v|, and v - q|v| grows with v, so the
            // group's smallest key is at least vmin - q|vmin|; with the
            // points grouped by home (a.perm) the lanes of a warp are near
            // each other and most groups are skipped.
            float thr = st.thr;
            uint32_t *qp = qk + st.qn * QS + tid;
#pragma unroll
            for (int g8 = 0; g8 < 32; g8 += 8) {
                const float vmin = fminf(fmin3(fmin3(v[g8], v[g8 + 1], v[g8 + 2]),
                                               fmin3(v[g8 + 3], v[g8 + 4], v[g8 + 5]), v[g8 + 6]),
                                         v[g8 + 7]);
                if (__any_sync(0xffffffffu, fmaf(-q, fabsf(vmin), vmin) < thr)) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float key =
                            make_key(v[g8 + e], (uint32_t)(jbase + g8 + e), mask);
                        if (key < thr) {
                            *qp = __float_as_uint(key);
                            qp += QS;
                        }
                    }
                }
                // after the check no lane holds more than QC - QI keys, so
                // the next QI values fit
                if ((QI == 16 && g8 == 8) || g8 == 24) {
                    st.qn = (int)((qp - (qk + tid)) / QS);
                    if (__any_sync(0xffffffffu, st.qn > QC - QI))
                        queue_flush<KC, QS>(keys, st, qk, tid, a.k, M, q);
                    qp = qk + st.qn * QS + tid;
                    thr = st.thr;
                }
            }
        };

        bool ok = true;
        float xx_next = write_tile(first);
        long long g = 0;
        long long tile = first;
        for (long long i = 0; i < my_tiles && ok; ++i, tile += gridDim.x) {
            const long long pos = tile * kTcRows + tid;
            const bool active = pos < a.n;
            const long long row = active && a.perm ? (long long)__ldg(a.perm + pos) : pos;
            const float xx = xx_next;
            const float xn = sqrtf(xx);
            const float sx = xn + lmax;
            // |v_j - (exact FP32 distance - |x|^2)| <= M
            const float M = a.m_dot * xn * lmax + 2.f * kGamma * sx * sx;

            float keys[KC];
            ScanState st;
            st.qn = 0;
            st.thr = INFINITY;
#pragma unroll 1
            for (int c = 0; c < nch; ++c, ++g) {
                const int tb = (int)(g & 1);
                const bool w = mbar_wait(&t_full[tb], (uint32_t)((g >> 1) & 1));
                if (!__all_sync(0xffffffffu, w)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int base = chunk_of(tile, c) * kTcN;  // first internal index
                const uint32_t col = my_lane_addr + (uint32_t)(tb * kTcN);
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    float v[32];
                    tmem_ld32(col + (uint32_t)(32 * h), v);
                    if (h == 1) {
                        // both halves are in registers: release the buffer
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&t_empty[tb]);
                    }
                    if (DUMP) {
                        // at the landmark's own column (internal position
                        // j' holds landmark lperm[j'])
                        if (active) {
                            float *o = a.dist2 + row * (long long)(nch * kTcN);
#pragma unroll
                            for (int t = 0; t < 32; ++t) {
                                const int jp = base + 32 * h + t;
                                o[a.lperm && jp < a.L ? __ldg(a.lperm + jp) : jp] = v[t];
                            }
                        }
                    } else if (c == 0 && h == 0) {
                        // The first KF values go straight into the list (one
                        // sorting network; padding columns sort last); any
                        // beyond KC are dropped, which the certificate covers
                        // like any key pushed out.  The rest of the half is
                        // pushed.
                        const int cnt = a.L - base < kTcN ? a.L - base : kTcN;
                        float kv[KF];
#pragma unroll
                        for (int t = 0; t < KF; ++t)
                            kv[t] = t < cnt ? make_key(fmaf(-2.f, v[t], __ldg(a.norms + base + t)),
                                                       (uint32_t)(base + t), mask)
                                            : INFINITY;
                        key_sort<KF>(kv);
#pragma unroll
                        for (int t = 0; t < KC; ++t) keys[t] = t < KF ? kv[t] : INFINITY;
                        st.thr = push_threshold(at<KC>(keys, a.k - 1), M, q);
#pragma unroll
                        for (int t = KF; t < 32; ++t) {
                            const float key = make_key(fmaf(-2.f, v[t], __ldg(a.norms + base + t)),
                                                       (uint32_t)(base + t), mask);
                            if (key < st.thr) {
                                qk[st.qn * QS + tid] = __float_as_uint(key);
                                ++st.qn;
                            }
                        }
                        queue_flush<KC, QS>(keys, st, qk, tid, a.k, M, q);
                    } else {
                        push32(v, base + 32 * h, keys, st, M);
                    }
                }
            }
            if (!ok) break;
            // Every MMA of this tile has completed (its last chunk has been
            // read): the next tile's operand replaces this one's, so that its
            // MMAs run while this tile is re-ranked.
            if (i + 1 < my_tiles) xx_next = write_tile(tile + gridDim.x);
            if (DUMP) continue;
            queue_flush<KC, QS>(keys, st, qk, tid, a.k, M, q);

            // The screened list goes to the candidate buffer; rerank_kernel
            // computes its exact distances from rows in shared memory (an
            // in-kernel re-rank gathering the rows from L2 took 37% of this
            // kernel's time).
            if (active) {
                // stored in the visiting order: a warp's lists are contiguous
                float4 *cp = reinterpret_cast<float4 *>(a.cand + pos * KC);
#pragma unroll
                for (int t = 0; t < KC; t += 4)
                    cp[t / 4] = make_float4(keys[t], keys[t + 1], keys[t + 2], keys[t + 3]);
            }
        }
        if (!ok) raise_abort();
    }

    // Teardown: every MMA has completed (the producer waited for its last
    // commit) and every tensor-memory read has been waited for.
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        tmem_dealloc(tmem, kTcCols);
    }
}

template <int D, int KC, int PREC, bool DUMP = false>
cudaError_t launch_tc(const FusedArgs &a, int grid, size_t smem, cudaStream_t stream) {
    tc_kernel<D, KC, PREC, DUMP><<<grid, kTcThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

template <int D, int KC, int PREC>
struct TcInstance {
    static const TcOps ops;
};

template <int D, int KC, int PREC>
const TcOps TcInstance<D, KC, PREC>::ops = {
    reinterpret_cast<const void *>(&tc_kernel<D, KC, PREC>), KC, &launch_tc<D, KC, PREC>};

#define ESOM_TC_CASES(DV, P)                                         \
    switch (kc) {                                                    \
        case 8: return &TcInstance<DV, 8, P>::ops;                   \
        case 12: return &TcInstance<DV, 12, P>::ops;                 \
        case 16: return &TcInstance<DV, 16, P>::ops;                 \
        case 20: return &TcInstance<DV, 20, P>::ops;                 \
        case 24: return &TcInstance<DV, 24, P>::ops;                 \
        case 28: return &TcInstance<DV, 28, P>::ops;                 \
        case 32: return &TcInstance<DV, 32, P>::ops;                 \
        case 36: return &TcInstance<DV, 36, P>::ops;                 \
        default: return nullptr;                                     \
    }

template <int D, int PREC>
struct TcDumpInstance {
    static const TcOps ops;
};

template <int D, int PREC>
const TcOps TcDumpInstance<D, PREC>::ops = {
    reinterpret_cast<const void *>(&tc_kernel<D, 8, PREC, true>), 8,
    &launch_tc<D, 8, PREC, true>};

#define ESOM_DEFINE_TC_D(DV)                                         \
    const TcOps *tc_ops_d##DV(int kc, int prec) {                    \
        if (prec == kTcBf16) {                                       \
            ESOM_TC_CASES(DV, kTcBf16)                               \
        }                                                            \
        ESOM_TC_CASES(DV, kTcTf32)                                   \
    }                                                                \
    const TcOps *tc_dump_ops_d##DV(int prec) {                       \
        return prec == kTcBf16 ? &TcDumpInstance<DV, kTcBf16>::ops   \
                               : &TcDumpInstance<DV, kTcTf32>::ops;  \
    }

}  // namespace esom
