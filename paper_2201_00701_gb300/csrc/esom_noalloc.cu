// esom_project_noalloc: the fused projection for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// owned by its own pool allocator (a foreign cudaMalloc would bypass the pool's
// budget and fragment it), or an interactive frame loop where cudaMalloc and
// cudaFree must be avoided because they can synchronise the whole device and
// stall the frame.  Such callers cannot create a handle (esom_create
// allocates).  This entry point instead keeps its scratch -- the staged copy
// of the landmarks and the kernel's status word -- in one file-scope
// __device__ array of fixed size, which every GPU that loads the library holds
// until the process exits.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "esom.h"
#include "esom_kernels.h"

namespace {

constexpr size_t kScratchFloats = ESOM_NOALLOC_SCRATCH_BYTES / sizeof(float);
constexpr size_t kStatusFloats = 64;  // first 256 bytes: the status words
// rows the scratch must keep for the list of ill-conditioned points of one
// pass (recomputed in FP64 after the pass); the rest of the scratch raises
// the pass size up to a handle's
constexpr size_t kMinRefineRows = 8192;
constexpr int kMaxDevices = 64;

}  // namespace

static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

namespace {

std::mutex g_setup_mu;
float *g_scratch_addr[kMaxDevices] = {};

esom_status noalloc_fail(esom_status s, const char *msg) {
    return static_cast<esom_status>(esom::set_error(s, msg));
}

// Device address of the scratch array on `dev` (which must be current).  In
// host code the array's name is only a host-side stand-in, so the address is
// looked up once per device with cudaGetSymbolAddress and cached.
cudaError_t scratch_address(int dev, float **out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" esom_status esom_project_noalloc(const float *points, int64_t n, const float *hi,
                                            const float *lo, int d, int L, int k, float *out,
                                            float boost, float adjust, esom_stream_t stream) {
    if (d < 4 || d > ESOM_MAX_D || d % 4 != 0)
        return noalloc_fail(ESOM_EINVAL, "d must be a multiple of 4 in [4, 64]");
    if (L < 2 || k < 2 || k > L) return noalloc_fail(ESOM_EINVAL, "need 2 <= k <= L");
    // the same code as esom_create for a k no kernel is built for
    if (k > ESOM_MAX_K) return noalloc_fail(ESOM_EUNSUPPORTED, "k above ESOM_MAX_K (32)");
    if (L > ESOM_MAX_L ||
        (size_t)L * (size_t)d + (size_t)((2 * L + 3) & ~3) + (size_t)((L + 3) & ~3) +
                kStatusFloats + 2 * kMinRefineRows > kScratchFloats)
        return noalloc_fail(ESOM_EINVAL,
                            "landmarks exceed the no-alloc scratch: need (L*(d+2) + L rounded up "
                            "to 4)*4 + 256 + 65536 bytes <= ESOM_NOALLOC_SCRATCH_BYTES");
    if (n < 0) return noalloc_fail(ESOM_EINVAL, "n < 0");
    if (!hi || !lo) return noalloc_fail(ESOM_EINVAL, "null landmark pointer");
    if (n > 0 && (!points || !out)) return noalloc_fail(ESOM_EINVAL, "null points or out");
    if (((uintptr_t)points & 15u) != 0) return noalloc_fail(ESOM_EALIGN, "points not 16-byte aligned");
    if (((uintptr_t)out & 7u) != 0) return noalloc_fail(ESOM_EALIGN, "out not 8-byte aligned");
    if (!(boost > 0.0f) || !(boost < INFINITY)) return noalloc_fail(ESOM_EINVAL, "boost must be > 0");
    if (!(adjust >= 0.0f) || !(adjust < INFINITY))
        return noalloc_fail(ESOM_EINVAL, "adjust must be >= 0");
    if (n == 0) return ESOM_OK;

    const esom::KernelOps *ops = esom::kernel_ops(d, esom::list_capacity(k));
    if (!ops) return noalloc_fail(ESOM_EUNSUPPORTED, "no kernel for this (d, k)");

    int dev = 0, sms = 0, optin = 0, bps = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(ESOM_ECUDA, "cudaGetDevice failed");
    float *scratch = nullptr;
    e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return noalloc_fail(ESOM_ECUDA, cudaGetErrorString(e));

    // Launch shape as for a handle.
    const int chunk = esom::landmark_chunk(L, d, 0);
    const int nchunks = (L + chunk - 1) / chunk;
    const size_t smem = esom::fused_smem_bytes(d, chunk, nchunks);
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess && smem > (size_t)optin) return noalloc_fail(ESOM_EUNSUPPORTED, "shared memory");
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ops->func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, ops->func, esom::kThreads, smem);
    if (e != cudaSuccess) return noalloc_fail(ESOM_ECUDA, cudaGetErrorString(e));
    if (bps < 1) return noalloc_fail(ESOM_EUNSUPPORTED, "launch does not fit on an SM");

    // Scratch layout (every part 16-byte aligned): [status words: error
    // bits, largest norm, rescans, -, refine-list length | landmarks L x d |
    // 2-D landmarks L x 2 | squared norms, L rounded up to 4 | refine list,
    // the rest].
    int *status = reinterpret_cast<int *>(scratch);
    float *s_lmax = scratch + 1;
    float *s_hi = scratch + kStatusFloats;
    float *s_lo = s_hi + (size_t)L * d;
    float *s_norms = s_lo + (size_t)((2 * L + 3) & ~3);  // 16-byte aligned for the bulk copy
    float *s_list = s_norms + (size_t)((L + 3) & ~3);
    long long *refine_list = reinterpret_cast<long long *>(s_list);
    unsigned *refine_count = reinterpret_cast<unsigned *>(status) + 4;
    long long pass = (long long)((kScratchFloats - (size_t)(s_list - scratch)) / 2);
    if (pass > esom::kTcPass) pass = esom::kTcPass;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(status, 0, 2 * sizeof(int), st);  // status and max norm start at zero
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s_hi, hi, (size_t)L * d * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s_lo, lo, (size_t)L * 2 * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = esom::launch_landmark_prep(s_hi, L, d, s_norms, s_lmax, st);
    if (e != cudaSuccess) return noalloc_fail(ESOM_ECUDA, cudaGetErrorString(e));

    esom::FusedArgs a;
    memset(&a, 0, sizeof(a));
    a.X = points;
    a.n = n;
    a.hi = s_hi;
    a.lo = s_lo;
    a.norms = s_norms;
    a.lmax = s_lmax;
    esom::key_layout(L, &a.key_mask, &a.key_quant);
    a.L = L;
    a.k = k;
    a.boost = boost;
    a.adjust = adjust;
    a.mode = esom::kProject;
    a.chunk = chunk;
    a.nchunks = nchunks;
    a.status = status;
    a.refine_list = refine_list;
    a.refine_count = refine_count;
    // passes that the refine list can hold, each followed by the FP64
    // recomputation of the points it listed
    for (long long off = 0; off < n && e == cudaSuccess; off += pass) {
        a.n = n - off < pass ? n - off : pass;
        a.X = points + off * d;
        a.out = out + off * 2;
        a.ntiles = (a.n + esom::kThreads - 1) / esom::kThreads;
        long long grid = (long long)bps * sms;
        if (grid > a.ntiles) grid = a.ntiles;
        e = cudaMemsetAsync(refine_count, 0, sizeof(unsigned), st);
        if (e == cudaSuccess) e = ops->launch(a, (int)grid, smem, st);
        if (e == cudaSuccess) e = ops->launch_refine(a, 2 * sms, st);
    }
    if (e != cudaSuccess) return noalloc_fail(ESOM_ECUDA, cudaGetErrorString(e));
    return ESOM_OK;
}
