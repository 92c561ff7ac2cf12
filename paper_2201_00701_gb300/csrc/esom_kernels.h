// Internal interface between the C ABI (esom_api.cu) and the kernel
// instantiations (esom_k_d*.cu).  Not installed; not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace esom {

constexpr int kThreads = 256;      // threads per block = points per tile
constexpr int kQueue = 16;         // per-thread candidate queue capacity
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
    int L, k;
    float boost, adjust;
    int adjust_mode;      // 0 general, 1 adjust == 1, 2 adjust == 0
    float *out;           // n x 2 (project)
    int *idx;             // n x k (knn)
    float *dist2;         // n x k (knn, nullable)
    int mode;             // Mode
    int chunk;            // landmarks per shared-memory chunk
    int nchunks;          // ceil(L / chunk); 1 = resident
    long long ntiles;     // ceil(n / kThreads)
    int *status;          // device status word (error bits)
};

struct KernelOps {
    const void *func;     // the __global__ function (for attributes / occupancy)
    int kc;               // compile-time list capacity
    cudaError_t (*launch)(const FusedArgs &, int grid, size_t smem, cudaStream_t);
};

// Returns the instantiation for dimension D and list capacity kc, or nullptr.
const KernelOps *kernel_ops(int D, int kc);

// Records `msg` as this host thread's last error message; returns s.
int set_error(int s, const char *msg);

inline size_t fused_smem_bytes(int D, int chunk, int nchunks) {
    size_t s = kBarrierBytes;
    s += (size_t)kThreads * D * sizeof(float);                    // point tile
    s += (size_t)(nchunks == 1 ? 1 : 2) * chunk * D * sizeof(float); // landmark chunk(s)
    s += (size_t)2 * kQueue * kThreads * sizeof(float);           // candidate queue
    return s;
}

}  // namespace esom
