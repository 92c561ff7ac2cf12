// Internal interface between the C ABI (esom_api.cu) and the kernel
// instantiations (esom_k_d*.cu).  Not installed; not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace esom {

constexpr int kThreads = 256;      // threads per block = points per tile
constexpr int kQueue = 24;         // per-thread candidate queue capacity (keys)
constexpr int kCheck = 8;          // landmarks scanned between queue checks
constexpr int kBarrierBytes = 128; // mbarrier area at the start of shared memory

// Device-side error bits written to the handle's status word.
constexpr int kErrWaitTimeout = 1;

enum Mode : int { kProject = 0, kKnn = 1 };

struct FusedArgs {
    const float *X;       // n x D points (16-byte aligned)
    long long n;
    const float *hi;      // L x D landmarks (library-owned, 256-byte aligned)
    const float *lo;      // L x 2 landmarks (library-owned)
    const float *norms;   // squared norms of the L landmarks, padded to a multiple of 4
    const float *lmax;    // largest landmark norm (one float)
    int L, k;
    float boost, adjust;
    float *out;           // n x 2 (project)
    int *idx;             // n x k (knn)
    float *dist2;         // n x k (knn, nullable)
    int mode;             // Mode
    int chunk;            // landmarks per shared-memory chunk
    int nchunks;          // ceil(L / chunk); 1 = resident
    long long ntiles;     // ceil(n / kThreads)
    unsigned key_mask;    // low bits of a screening key that hold the landmark index
    float key_quant;      // 2^(bits - 23): relative perturbation of a key
    int *status;          // device status words: [0] error bits, [2] rescan count
    const unsigned char *img;  // tensor-core screening: landmark chunk images
    int tc_chunks;        // ceil(L / kTcN) chunks in img
    // pair constants of the projection (pair_entry): the pair table of
    // (1/q, 1/r) per landmark pair, or the L x L table of q = |L_v - L_u|^2
    // (pair_q values) for larger L; both null: computed from the rows
    const float2 *ptab;
    const float *qtab;
    // the pair table with rows and columns in the spatial landmark order
    // (ptab_pos[i * L + j] = ptab[lperm[i] * L + lperm[j]]) and each
    // landmark's position in that order (ipos[lperm[i]] = i): the re-rank +
    // projection kernel gathers a point's pair constants from it, so that
    // neighbouring landmarks' entries share cache lines; null: ptab
    const float2 *ptab_pos;
    const int *ipos;
    // k-NN mode: when set, a point whose screening certificate fails is not
    // rescanned in line but appended (row index) to fail_list, counted in
    // *fail_count; rescan_kernel then finds its neighbours exactly
    long long *fail_list;
    unsigned *fail_count;
    // when set, the landmark rows are stored centred on this point (d floats,
    // 16-byte aligned) and every kernel subtracts it from the points it loads
    const float *center;
    // fused kernel only, for tests of the timeout path: when nonzero, every
    // block first waits on a barrier that nothing completes and gives up
    // after this many ns (see esom_test_stall)
    unsigned long long stall_ns;
    // tensor-core k-NN with spatial orders (all null: natural order): the
    // visiting order of the points, each tile's home chunk, the chunks'
    // visiting orders, and the landmark of each internal screening position
    // (a.norms then holds the norms in the internal order)
    const int *perm;
    const unsigned short *tile_home;
    const unsigned short *corder;
    const int *lperm;
    // tensor-core k-NN: the screened list of each point (KC keys, ascending,
    // at row * KC), re-ranked exactly by rerank_kernel; m_dot = the
    // tensor-core part of the screening error per unit |x| max|l|
    // (tc_dot_bound)
    float *cand;
    float m_dot;
    // projection: rows whose FP32 normal system is too ill-conditioned are
    // appended here (count in *refine_count) for refine_kernel
    long long *refine_list;
    unsigned *refine_count;
    // projection kernel: when set, it projects only the rows listed here
    // (*rows_count of them; e.g. the points whose certificate failed)
    const long long *rows_list;
    const unsigned *rows_count;
};

// x - c, four at a time (c may be null: no centring).
__device__ __forceinline__ float4 centred(float4 x, const float *c, int e) {
    if (!c) return x;
    const float4 v = __ldg(reinterpret_cast<const float4 *>(c) + e);
    return make_float4(x.x - v.x, x.y - v.y, x.z - v.z, x.w - v.w);
}

// Many datasets of one (D, list capacity) in one launch: every block walks a
// contiguous range [cta_begin[b], cta_begin[b+1]) of the global tile list;
// tile t belongs to dataset tile_item[t], whose local tile index is
// t - tile_base[item].
struct BatchArgs {
    const FusedArgs *items;     // per dataset (mode = project), device memory
    const long long *tile_base; // first global tile of each dataset
    const int *tile_item;       // dataset of each global tile
    const long long *cta_begin; // grid + 1 range boundaries
    int *status;                // error bits, as for a single launch
    int2 *refine_list;          // (dataset, row) of ill-conditioned points
    unsigned *refine_count;
};

struct KernelOps {
    const void *func;     // the __global__ function (for attributes / occupancy)
    int kc;               // compile-time list capacity
    cudaError_t (*launch)(const FusedArgs &, int grid, size_t smem, cudaStream_t);
    const void *batch_func;
    cudaError_t (*launch_batch)(const BatchArgs &, int grid, size_t smem, cudaStream_t);
    // Fills the pair table ptab[u * L + v] = pair_entry(q, l_v - l_u) when
    // ptab is given, else qtab[u * L + v] = q, with q = |L_v - L_u|^2 from
    // the (chunk-swizzled) rows of hi by the pair loop's own arithmetic
    // (pair_q), so the tables hold exactly the values the loop would compute.
    cudaError_t (*launch_pair_table)(const float *hi, const float *lo, int L, float2 *ptab,
                                     float *qtab, cudaStream_t);
    // Projection from given neighbours (FusedArgs idx / dist2, k per point):
    // steps 2-4 of the fused kernel in blocks of kProjThreads, one kernel per
    // source of the pair constants (index: PairMode of esom_fused.cuh;
    // shared memory: project_smem_bytes).
    const void *proj_func[3];
    cudaError_t (*launch_proj[3])(const FusedArgs &, int grid, size_t smem, cudaStream_t);
    // Exact k-NN of the rows in a.fail_list (one warp per row), written to
    // a.idx / a.dist2 like the k-NN kernels do.
    cudaError_t (*launch_rescan)(const FusedArgs &, int grid, cudaStream_t);
    // Exact re-rank of the tensor-core k-NN's screened lists (a.cand):
    // FP32 difference-form distances (rows in shared memory when
    // a.nchunks == 1, rerank_smem_bytes), order by (distance, landmark), the
    // certificate; writes a.idx / a.dist2, failed rows to a.fail_list.
    const void *rerank_func;
    cudaError_t (*launch_rerank)(const FusedArgs &, int grid, size_t smem, cudaStream_t);
    // Exact re-rank and projection in one kernel (the tensor-core plan's
    // projection, blocks of kProjThreads, one kernel per PairMode, shared
    // memory project_smem_bytes): certified points are projected at once,
    // the others go to a.fail_list.
    const void *rproj_func[3];
    cudaError_t (*launch_rproj[3])(const FusedArgs &, int grid, size_t smem, cudaStream_t);
    // FP64 recomputation, one block a point, of the rows in a.refine_list
    // (B.refine_list for the batched kernel), written to the outputs.
    cudaError_t (*launch_refine)(const FusedArgs &, int grid, cudaStream_t);
    cudaError_t (*launch_refine_batch)(const BatchArgs &, int grid, cudaStream_t);
};


inline size_t rerank_smem_bytes(int D, int L, bool resident) {
    return kBarrierBytes + (resident ? (size_t)L * D * sizeof(float) : 0);
}

// Returns the instantiation for dimension D and list capacity kc, or nullptr.
const KernelOps *kernel_ops(int D, int kc);

// Largest L for which a handle keeps the pair table (8 bytes a landmark
// pair: 32 MiB at 2048), and the L x L table of squared landmark distances
// (64 MiB at 4096); above both the pair loop computes its constants.
constexpr int kPtabMaxL = 2048;
constexpr int kQtabMaxL = 4096;

// Threads (= points) per block of the projection kernels, and the resident
// blocks per SM they are compiled for (list capacity kc: five blocks, at most
// 102 registers a thread, up to k = 20; four above, where the lists need
// more registers).
constexpr int kProjThreads = 128;
__host__ __device__ constexpr int proj_threads(int) { return kProjThreads; }
__host__ __device__ constexpr int proj_min_blocks(int kc) { return kc <= 24 ? 5 : 4; }


// ---------------------------------------------------------------------------
// Tensor-core screening (tcgen05, TF32): tiles of kTcRows points (the MMA's M
// and the TMEM lanes), landmark chunks of kTcN (the MMA's N); one block =
// four selection warps (one thread per point) and one producer warp that
// streams landmark chunk images and issues the MMAs.  The kernel finds the k
// nearest; a second kernel (project_kernel) projects from them.
constexpr int kTcRows = 128;
constexpr int kTcN = 64;
constexpr int kTcThreads = 160;
constexpr int kTcCols = 2 * kTcN;  // TMEM columns: two accumulator buffers

// Operand precision of the tensor-core screening: split TF32 (4-byte
// elements, kind::tf32) or split BF16 (2-byte elements, kind::f16).
enum TcPrec : int { kTcTf32 = 0, kTcBf16 = 1 };
__host__ __device__ constexpr int tc_elem_bytes(int prec) { return prec == kTcBf16 ? 2 : 4; }

// Operand layout: rows of tc_row_bytes per column block (64 bytes with the
// 64-byte swizzle when a row's d elements fit, else 128 bytes with the
// 128-byte swizzle), tc_nblk column blocks; pipeline stages of the landmark
// ring; resident blocks per SM the launch aims for.  One MMA K step reads 32
// bytes of a row (8 TF32 or 16 BF16 values).
__host__ __device__ constexpr int tc_row_bytes(int D, int prec = kTcTf32) {
    return D * tc_elem_bytes(prec) <= 64 ? 64 : 128;
}
__host__ __device__ constexpr int tc_nblk(int D, int prec = kTcTf32) {
    return D * tc_elem_bytes(prec) <= 64 ? 1 : (D * tc_elem_bytes(prec) + 127) / 128;
}
__host__ __device__ constexpr int tc_stages(int D, int prec = kTcTf32) {
    return D * tc_elem_bytes(prec) <= 128 ? 3 : 2;
}
__host__ __device__ constexpr int tc_minb(int D, int KC) { return D <= 16 ? (KC <= 16 ? 4 : 3) : 2; }

// Candidate queue of the tensor-core k-NN kernel: its capacity (keys per
// selection thread) and the values pushed between two fullness checks.  A
// queue of 48 checked once per tensor-memory load of 32 values flushes
// rarely (measured 9% faster k-NN than 24 / 16 at d = 16, k = 20); four
// blocks per SM (d <= 16, k <= 12) leave shared memory for 24 / 16 only.
__host__ __device__ constexpr int tc_queue(int D, int KC) { return tc_minb(D, KC) >= 4 ? 24 : 48; }
__host__ __device__ constexpr int tc_check(int D, int KC) { return tc_minb(D, KC) >= 4 ? 16 : 32; }

// Bound on the tensor-core part of the screening error per unit |X| max|L|.
// With x_hi the rounding of x to p significant bits (p = 11 for TF32, 8 for
// BF16) and x_lo that of x - x_hi: |x - x_hi| <= 2^-p |x| and
// |x - x_hi - x_lo| <= 2^-2p |x|, so the dropped terms x_lo l_lo and the two
// remainders are <= 3 2^-2p |x_i||l_i| per coordinate; the 3D products are
// exact in FP32 and accumulated with at most 3D + 1 roundings (2^-23 each,
// relative to the sum of |products| <= |x||l|).  Twice that in
// v_j = |L_j|^2 - 2 T_j, and a factor 2 of margin.  (Measured on the GPU:
// at most 0.103 of this bound, on rows spanning 2^-10 .. 2^10.)
__host__ __device__ constexpr float tc_dot_bound(int D, int prec) {
    return 4.f * (3.f * (prec == kTcBf16 ? 1.5258789e-5f : 2.3841858e-7f) +
                  (float)(3 * D + 1) * 1.1920929e-7f);
}

// Bytes of one chunk image: the high parts of kTcN rows, then the low
// parts, in the swizzled K-major order the MMA reads (see tc_image_offset).
__host__ __device__ inline size_t tc_chunk_bytes(int D, int prec = kTcTf32) {
    return (size_t)2 * kTcN * tc_row_bytes(D, prec) * tc_nblk(D, prec);
}

// Byte offset of 16-byte piece c of column block blk of row r inside an
// operand of `rows` rows (base aligned to 1024 bytes): 8-row groups of
// 8 * row_bytes, piece c of row r at slot c ^ (r mod 8) (128-byte swizzle)
// or c ^ ((r / 2) mod 4) (64-byte swizzle).
__host__ __device__ inline unsigned tc_image_offset(int D, int rows, int r, int blk, int c,
                                                    int prec = kTcTf32) {
    const int rb = tc_row_bytes(D, prec);
    const int sw = rb == 64 ? ((r >> 1) & 3) : (r & 7);
    return (unsigned)(blk * rows * rb + (r >> 3) * 8 * rb + (r & 7) * rb + ((c ^ sw) << 4));
}

inline size_t tc_smem_bytes(int D, int KC, int prec = kTcTf32) {
    const size_t rb = (size_t)tc_row_bytes(D, prec) * tc_nblk(D, prec);
    return 1024                                  // alignment slack
           + 2 * (size_t)kTcRows * rb            // point tile (high and low parts)
           + (size_t)tc_stages(D, prec) * tc_chunk_bytes(D, prec)  // landmark chunk ring
           + (size_t)tc_queue(D, KC) * kTcRows * 4  // candidate queue
           + 256;                                // barriers, TMEM address, flags
}

// Spatial orders of the tensor-core screening (esom_order.cu), used when
// L <= kOrderMaxL: the landmark order lperm (internal position -> landmark,
// chunks of kTcN along principal directions), the chunk centroids (nch x D),
// the squared norms in the internal order (NaN padding) and each chunk's
// visiting order (corder[c * nch + r], the chunks by centroid distance).
constexpr int kOrderMaxL = 8192;
// With reorder false the landmark order lperm is kept (it only sets the
// speed of the screening, never its result) and only the centroids, the
// internal-order norms and the visiting orders are recomputed.
cudaError_t launch_landmark_order(const float *hi, const float *norms, int L, int D, int *lperm,
                                  float *centers, float *norms_int, unsigned short *corder,
                                  cudaStream_t stream, bool reorder = true);
// The pair table in the landmark order lperm (ptab_pos[i * L + j] =
// ptab[lperm[i] * L + lperm[j]], the same entries moved) and the inverse
// order (ipos[lperm[i]] = i), for L <= kPtabMaxL.
cudaError_t launch_pair_table_positions(const float2 *ptab, const int *lperm, int L,
                                        float2 *ptab_pos, int *ipos, cudaStream_t stream);
// The points of one pass grouped by home chunk (nearest centroid):
// perm[pos] = point at visiting position pos, tile_home[t] = home chunk of
// position kTcRows t; home (n) and counts (nblocks * nch) are scratch.
constexpr int kOrderBlocks = 304;
cudaError_t launch_point_order(const float *X, long long n, int D, const float *centers, int nch,
                               const float *center, unsigned short *home, int *counts,
                               int nblocks, int *perm, unsigned short *tile_home,
                               cudaStream_t stream);

// Points per tensor-core k-NN pass of esom_project: the pass writes their
// neighbours (k indices and squared distances each) to the handle's scratch,
// the projection kernel reads them.
constexpr long long kTcPass = 1 << 20;

struct TcOps {
    const void *func;
    int kc;
    cudaError_t (*launch)(const FusedArgs &, int grid, size_t smem, cudaStream_t);
};


// Shared memory of the projection kernels (pair mode `mode`, PairMode of
// esom_fused.cuh) for list capacity kc: the stash columns (a float2 and an
// index per neighbour and thread) and, with a table (modes 0, 1), the 2-D
// positions.
inline size_t project_smem_bytes(int L, int kc, int mode) {
    const size_t lo = ((size_t)L * 2 * sizeof(float) + 15) & ~(size_t)15;
    const size_t kk = (size_t)(kc - 4);
    return kBarrierBytes + kk * kProjThreads * (8 + 4) + (mode != 2 ? lo : 0);
}

// Tensor-core instantiation for D, list capacity kc and precision, or
// nullptr.
const TcOps *tc_ops(int D, int kc, int prec);
// The tensor-core kernel in its accumulator-dump form (list capacity 8):
// writes the raw values T_j = x . l_j of every point and landmark to
// a.dist2 (tc_chunks * kTcN per point) instead of selecting; for tests of
// the screening error bound.
const TcOps *tc_dump_ops(int D, int prec);

// Builds the split chunk images of the landmarks (precision prec) from the
// (chunk-swizzled) rows of hi: ceil(L / kTcN) images of tc_chunk_bytes(D,
// prec), rows beyond L zero; with lperm, internal position j holds landmark
// lperm[j].
cudaError_t launch_tc_image(const float *hi, int L, int D, unsigned char *img, int prec,
                            cudaStream_t stream, const int *lperm = nullptr);

// rcp[i] = the FP64 reciprocal the 2x2 solve uses (drcp), div[i] = 1.0 / x[i]
// by CUDA's division, for i < n (device pointers).
cudaError_t launch_drcp_selftest(const double *x, long long n, double *rcp, double *div,
                                 cudaStream_t stream);

// Records `msg` as this host thread's last error message; returns s.
int set_error(int s, const char *msg);

// Squared landmark norms (norms[j], j < L; NaN padding up to a multiple of
// `pad`, itself a multiple of 4), the largest norm (*lmax, which must hold 0
// on entry), and the rows of hi swizzled in place (see swz) -- after
// subtracting `center` from them when it is given.
cudaError_t launch_landmark_prep(float *hi, int L, int D, float *norms, float *lmax,
                                 cudaStream_t stream, int pad = 4, const float *center = nullptr);

// center[i] = the landmarks' mean coordinate i rounded to an integer (FP64
// sums in landmark order; integers keep integer-valued data exact).
cudaError_t launch_landmark_center(const float *hi, int L, int D, float *center,
                                   cudaStream_t stream);

// Landmark rows are stored with their 16-byte chunks permuted: logical chunk
// e of row j sits at physical chunk e ^ swz(j), with g = gcd(d/4, 8) and
// swz(j) = (j / (8/g)) mod g.  Rows are d*4 bytes apart, so without the
// permutation the same chunk of different rows falls on few of the eight
// 16-byte bank groups; with it, any eight consecutive rows use all eight,
// and the random-row gathers of the re-rank and the pair loop see ~2.6-way
// instead of up to 8-way conflicts.  swz depends only on j mod 8.
__host__ __device__ inline int swz_groups(int D) {
    const int c = D / 4;
    return (c % 8 == 0) ? 8 : (c % 4 == 0) ? 4 : (c % 2 == 0) ? 2 : 1;
}
__host__ __device__ inline int swz(int D, int j) {
    const int g = swz_groups(D);
    return (j / (8 / g)) & (g - 1);
}

// List capacity for k neighbours: k plus at least four spare entries, a
// multiple of 4, at least 8.
inline int list_capacity(int k) {
    int kc = ((k + 4 + 3) / 4) * 4;
    return kc < 8 ? 8 : kc;
}

// Screening-key layout for L landmarks.
inline void key_layout(int L, unsigned *mask, float *quant) {
    int b = 1;
    while ((1 << b) < L) ++b;
    *mask = (1u << b) - 1u;
    *quant = ldexpf(1.0f, b - 23);
}

inline size_t fused_smem_bytes(int D, int chunk, int nchunks) {
    const size_t nbuf = nchunks == 1 ? 1 : 2;
    size_t s = kBarrierBytes;
    s += (size_t)kThreads * D * sizeof(float);                // point tile
    s += nbuf * chunk * D * sizeof(float);                    // landmark rows
    s += nbuf * (size_t)((chunk + 3) & ~3) * sizeof(float);   // landmark norms
    s += (size_t)kQueue * kThreads * sizeof(unsigned);        // candidate queue
    return s;
}

// Shared memory of the batched kernel: one landmark buffer of `chunk` rows
// (the largest resident set or chunk of the group).
inline size_t batch_smem_bytes(int D, int chunk) {
    size_t s = kBarrierBytes;
    s += (size_t)kThreads * D * sizeof(float);
    s += (size_t)chunk * D * sizeof(float);
    s += (size_t)((chunk + 3) & ~3) * sizeof(float);
    s += (size_t)kQueue * kThreads * sizeof(unsigned);
    return s;
}

// Landmarks per shared-memory chunk: all of them when rows and norms fit in
// 72 KiB (resident), otherwise a multiple of 8 filling 32 KiB per buffer;
// `forced` > 0 overrides (rounded up to a multiple of 8).  A multiple of 8
// keeps local and global landmark indices equal modulo 8 (see swz).
inline int landmark_chunk(int L, int D, int forced) {
    const size_t per = (size_t)D * sizeof(float) + sizeof(float);
    if (forced > 0) {
        int c = (forced + 7) & ~7;
        return c >= L ? L : c;
    }
    if ((size_t)L * per <= 72 * 1024) return L;
    int c = (int)((32 * 1024) / per) & ~7;
    return c < 48 ? 48 : c;
}

}  // namespace esom
