// Handle state shared by the C ABI translation units (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "esom.h"
#include "esom_kernels.h"

struct esom_ctx {
    int d = 0, L = 0, k = 0, kc = 0, dev = 0;
    float *hi = nullptr;   // L x d
    float *lo = nullptr;   // L x 2
    float *norms = nullptr; // squared landmark norms, zero-padded to a multiple of kTcN
    // device status words: [0] error bits, [1] the largest norm (float),
    // [2] rescans since the stats reset, [3] certificate failures of the
    // current pass, [4] refine-list length of the current pass
    int *status = nullptr;
    long long *refine_list = nullptr;  // rows of one pass for the FP64 recomputation
    // pair constants of the projection per landmark pair: the pair table
    // (L <= kPtabMaxL), else the squared landmark distances (L <= kQtabMaxL)
    float2 *ptab = nullptr;
    float *qtab = nullptr;
    uint64_t version = 0;
    const esom::KernelOps *ops = nullptr;
    int num_sms = 0;
    int forced_chunk = 0;
    // esom_test_stall: limit (ns) of the probe wait of the next fused-kernel
    // launch; 0 = none (the launch consumes it)
    unsigned long long stall_ns = 0;
    uint64_t points = 0;   // points handed to the kernels since the last stats reset
    uint64_t launches = 0; // kernels launched for esom_project / esom_knn since then
    // kernel timing (esom_set_timing): a ring of event pairs on the launching
    // stream, the kind of kernel of each, per-kind totals
    static constexpr int kTimed = 256;
    int timing = 0, tcount = 0;
    cudaEvent_t tev[kTimed][2] = {};
    int tkind[kTimed] = {};
    double tms[ESOM_KERNEL_KINDS] = {};
    uint64_t tlaunch[ESOM_KERNEL_KINDS] = {};
    // launch configuration (derived from L, d and the chunk choice)
    int chunk = 0, nchunks = 0, blocks_per_sm = 0;
    size_t smem = 0;
    // tensor-core screening (esom_set_screening); img holds the landmark
    // chunk images while it is on
    int screening = 0;
    int split = 0;  // k-NN kernel + projection kernel instead of the fused one
    // centring (esom_set_centering): requested, and in effect for the
    // landmarks now stored (set by esom_set_landmarks)
    int centering = 0, centered = 0;
    float *center = nullptr;  // ESOM_MAX_D floats
    const esom::TcOps *tc = nullptr;
    unsigned char *img = nullptr;
    int tc_blocks_per_sm = 0;
    size_t tc_smem = 0;
    // neighbours of one k-NN pass (kTcPass x k) for the projection kernel
    int *tc_idx = nullptr;
    float *tc_d2 = nullptr;
    long long *fail_list = nullptr;  // rows whose certificate failed (kTcPass)
    int proj_blocks_per_sm = 0, rproj_blocks_per_sm = 0;
    size_t proj_smem = 0;
    // tensor-core k-NN: screened lists of one pass (kTcPass x kc keys) and
    // the exact re-rank kernel's configuration
    float *cand = nullptr;
    int rerank_blocks_per_sm = 0;
    size_t rerank_smem = 0;
    // spatial orders of the tensor-core screening (L <= kOrderMaxL):
    // landmark order, chunk centroids, norms in the internal order, chunk
    // visiting orders; per pass: point homes, block counts, visiting order
    // of the points, home chunk of each tile
    int order_on = 0;
    // keep_order: reuse the landmark order on later landmark sets (set by the
    // frame server); order_valid: lperm holds an order of this handle
    int keep_order = 0, order_valid = 0;
    int *lperm = nullptr;
    // the pair table in the landmark order lperm and the inverse order
    // (with ptab and the orders), rebuilt with the tensor-core operands
    float2 *ptab_pos = nullptr;
    int *ipos = nullptr;
    float *centers = nullptr;
    float *norms_int = nullptr;
    unsigned short *corder = nullptr;
    unsigned short *home = nullptr;
    int *counts = nullptr;
    int *perm = nullptr;
    unsigned short *tile_home = nullptr;
    // host-buffer pipeline state (created on first use)
    float *stage_x[2] = {nullptr, nullptr};
    float *stage_out[2] = {nullptr, nullptr};
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr},
                ev_free[2] = {nullptr, nullptr}, ev_start = nullptr;
    std::mutex host_mu;
};

namespace esom {
// Fills the per-launch arguments for `n` points of handle h (mode project).
void fill_args(const esom_ctx *h, const float *points, long long n, float *out, float boost,
               float adjust, FusedArgs *a);
}  // namespace esom
