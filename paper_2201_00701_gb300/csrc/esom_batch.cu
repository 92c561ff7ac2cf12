// Batched projection of many datasets (C ABI in include/esom.h).
//
// A batch is planned once: its datasets are grouped by (d, list capacity),
// each group becomes one launch of the batched kernel, and the group's tiles
// (256 points each) are split into contiguous ranges of about equal
// estimated cost, one range per block.  An optional autotuner times the
// candidate launch shapes of every group on the batch itself and keeps the
// fastest.  esom_batch_run replays the plan; esom_batch_run_graph replays it
// from a CUDA graph captured on first use.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "esom.h"
#include "esom_ctx.h"
#include "esom_kernels.h"

using esom::BatchArgs;
using esom::FusedArgs;
using esom::KernelOps;

namespace {

esom_status bfail(esom_status s, const char *msg) {
    return static_cast<esom_status>(esom::set_error(s, msg));
}

esom_status bcuda(cudaError_t e, const char *what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return bfail(ESOM_ECUDA, buf);
}

// One launch shape of a group.
struct Shape {
    int forced_chunk;   // 0: each dataset's own choice; > 0: stream landmarks in chunks of this
    int blocks_per_sm;  // blocks per SM (1 .. occupancy limit)
    int separate = 0;   // 1: each dataset by its own single-dataset launch
};

struct Group {
    int D = 0, kc = 0;
    const KernelOps *ops = nullptr;
    std::vector<int> items;          // indices into the batch's item list
    std::vector<FusedArgs> args;     // per dataset (host copy)
    std::vector<long long> tile_base, cost;
    std::vector<int> tile_item;
    long long tiles = 0;
    // device copies
    FusedArgs *d_items = nullptr;
    long long *d_tile_base = nullptr, *d_cta_begin = nullptr;
    int *d_tile_item = nullptr;
    int2 *d_refine = nullptr;        // (dataset, row) of ill-conditioned points
    int grid = 0;
    size_t smem = 0;
    Shape shape{0, 0};
    float tuned_ms = -1.f;
};

}  // namespace

// Status words of a batch: [0] error bits, [2] rescans, then one
// refine-list count per group from kGroupCountWord on.
constexpr int kGroupCountWord = 16;
constexpr int kStatusWords = 1024;

struct esom_batch_ctx {
    int dev = 0, num_sms = 0, optin = 0;
    std::vector<esom_batch_item> items;
    std::vector<Group> groups;
    int *status = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string plan;
};

namespace {

// Estimated cost of one point of a dataset (FP32 instructions): screening
// scan, list upkeep, re-rank and pair loop.
long long point_cost(const esom_ctx *h) {
    const long long m = h->k - 1;
    return (long long)h->L * (h->d + 6) + (long long)h->kc * (2LL * h->d + 8) +
           m * (m - 1) / 2 * (2LL * h->d + 40) + 200;
}

// Applies a launch shape: per-dataset chunking, shared memory, grid and the
// cost-balanced tile ranges (uploaded to the device); or, for `separate`,
// each dataset's own launch configuration.
esom_status apply_shape(esom_batch_ctx *b, Group &g, const Shape &sh) {
    if (sh.separate) {
        for (size_t i = 0; i < g.items.size(); ++i) {
            const esom_ctx *h = b->items[g.items[i]].landmarks;
            FusedArgs &a = g.args[i];
            a.chunk = h->chunk;
            a.nchunks = h->nchunks;
            a.ptab = h->ptab;
            a.qtab = h->qtab;
        }
        g.shape = Shape{0, 0, 1};
        g.grid = 0;
        g.smem = 0;
        return ESOM_OK;
    }
    int cap = 0;
    for (size_t i = 0; i < g.items.size(); ++i) {
        const esom_ctx *h = b->items[g.items[i]].landmarks;
        FusedArgs &a = g.args[i];
        int chunk = h->chunk;
        if (sh.forced_chunk > 0 && h->L > sh.forced_chunk)
            chunk = esom::landmark_chunk(h->L, h->d, sh.forced_chunk);
        a.chunk = chunk;
        a.nchunks = (h->L + chunk - 1) / chunk;
        a.ptab = h->ptab;
        a.qtab = h->qtab;
        cap = std::max(cap, chunk);
    }
    const size_t smem = esom::batch_smem_bytes(g.D, cap);
    if (smem > (size_t)b->optin) return bfail(ESOM_EUNSUPPORTED, "batch: shared memory");
    cudaError_t e = cudaFuncSetAttribute(g.ops->batch_func,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, b->optin);
    int bps = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, g.ops->batch_func,
                                                           esom::kThreads, smem);
    if (e != cudaSuccess) return bcuda(e, "batch occupancy");
    if (bps < 1) return bfail(ESOM_EUNSUPPORTED, "batch: block does not fit on an SM");
    const int use = sh.blocks_per_sm > 0 ? std::min(sh.blocks_per_sm, bps) : bps;
    long long grid = (long long)use * b->num_sms;
    if (grid > g.tiles) grid = g.tiles;
    // cost-balanced contiguous ranges
    long long total = 0;
    for (long long t = 0; t < g.tiles; ++t) total += g.cost[t];
    std::vector<long long> begin((size_t)grid + 1, g.tiles);
    begin[0] = 0;
    long long acc = 0, t = 0;
    for (long long c = 1; c < grid; ++c) {
        const long long target = (total * c + grid - 1) / grid;
        while (t < g.tiles && acc + g.cost[t] <= target) acc += g.cost[t++];
        begin[(size_t)c] = t;
    }
    e = cudaMemcpy(g.d_items, g.args.data(), g.args.size() * sizeof(FusedArgs),
                   cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        cudaFree(g.d_cta_begin);
        g.d_cta_begin = nullptr;
        e = cudaMalloc(&g.d_cta_begin, begin.size() * sizeof(long long));
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(g.d_cta_begin, begin.data(), begin.size() * sizeof(long long),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(e, "batch plan upload");
    g.grid = (int)grid;
    g.smem = smem;
    g.shape = Shape{sh.forced_chunk, use, 0};
    return ESOM_OK;
}

esom_status launch_group(esom_batch_ctx *b, const Group &g, cudaStream_t st) {
    if (g.tiles == 0) return ESOM_OK;
    const int gi = (int)(&g - b->groups.data());
    if (g.shape.separate) {
        // each dataset through its handle's own execution plan (fused,
        // split or tensor-core, as set on the handle or chosen by esom_tune)
        for (size_t i = 0; i < g.items.size(); ++i) {
            const esom_batch_item &it = b->items[g.items[i]];
            if (it.n == 0) continue;
            const esom_status s = esom_project(it.landmarks, it.points, it.n, it.out, it.boost,
                                               it.adjust, reinterpret_cast<esom_stream_t>(st));
            if (s != ESOM_OK) return s;
        }
        return ESOM_OK;
    }
    BatchArgs a;
    a.items = g.d_items;
    a.tile_base = g.d_tile_base;
    a.tile_item = g.d_tile_item;
    a.cta_begin = g.d_cta_begin;
    a.status = b->status;
    // points whose FP32 system is too ill-conditioned: listed by the group's
    // launch, recomputed in FP64 right after it
    a.refine_list = g.d_refine;
    // each group its own count (groups may run concurrently in a graph)
    a.refine_count = reinterpret_cast<unsigned *>(b->status) + kGroupCountWord + gi;
    cudaError_t e = cudaMemsetAsync(a.refine_count, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = g.ops->launch_batch(a, g.grid, g.smem, st);
    if (e == cudaSuccess) e = g.ops->launch_refine_batch(a, 2 * b->num_sms, st);
    return e == cudaSuccess ? ESOM_OK : bcuda(e, "batch launch");
}

// Times candidate shapes of one group on the batch itself; keeps the best.
esom_status autotune(esom_batch_ctx *b, Group &g) {
    std::vector<Shape> cands;
    for (int fc : {0, 512, 256})
        for (int bps : {0, 1}) cands.push_back(Shape{fc, bps, 0});
    cands.push_back(Shape{0, 0, 1});
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Shape best_shape{0, 0, 0};
    for (const Shape &c : cands) {
        if (apply_shape(b, g, c) != ESOM_OK) continue;
        float ms = 0.f, tot = 0.f;
        bool ok = true;
        for (int r = 0; r < 3 && ok; ++r) {
            cudaEventRecord(e0, 0);
            ok = launch_group(b, g, 0) == ESOM_OK;
            cudaEventRecord(e1, 0);
            ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) tot += ms;
        }
        if (ok && tot < best) {
            best = tot;
            best_shape = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    esom_status s = apply_shape(b, g, best_shape);
    g.tuned_ms = best / 2.f;
    return s;
}

void describe(esom_batch_ctx *b) {
    std::string out = "{\"groups\": [";
    char buf[320];
    for (size_t i = 0; i < b->groups.size(); ++i) {
        const Group &g = b->groups[i];
        snprintf(buf, sizeof(buf),
                 "%s{\"d\": %d, \"kc\": %d, \"datasets\": %zu, \"tiles\": %lld, \"grid\": %d, "
                 "\"shared_bytes\": %zu, \"forced_chunk\": %d, \"blocks_per_sm\": %d, "
                 "\"separate\": %d, \"tuned_ms\": %.4f}",
                 i ? ", " : "", g.D, g.kc, g.items.size(), g.tiles, g.grid, g.smem,
                 g.shape.forced_chunk, g.shape.blocks_per_sm, g.shape.separate, g.tuned_ms);
        out += buf;
    }
    out += "]}";
    b->plan = out;
}

}  // namespace

extern "C" {

esom_status esom_batch_create(const esom_batch_item *items, int count, int autotune_flag,
                              esom_batch *out) {
    if (!out) return bfail(ESOM_EINVAL, "null output pointer");
    *out = nullptr;
    if (count < 1 || !items) return bfail(ESOM_EINVAL, "empty batch");
    esom_batch_ctx *b = new (std::nothrow) esom_batch_ctx;
    if (!b) return bfail(ESOM_ENOMEM, "host allocation");
    cudaError_t e = cudaGetDevice(&b->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&b->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->dev);
    if (e != cudaSuccess) {
        delete b;
        return bcuda(e, "device query");
    }
    b->items.assign(items, items + count);
    std::map<std::pair<int, int>, int> gidx;
    for (int i = 0; i < count; ++i) {
        const esom_batch_item &it = items[i];
        const esom_ctx *h = it.landmarks;
        esom_status s = ESOM_OK;
        if (!h) s = bfail(ESOM_EINVAL, "batch item without a handle");
        else if (h->dev != b->dev) s = bfail(ESOM_EINVAL, "batch item on another device");
        else if (h->version == 0) s = bfail(ESOM_ENOLANDMARKS, "batch item without landmarks");
        else if (it.n < 0) s = bfail(ESOM_EINVAL, "batch item with n < 0");
        else if (it.n > 0 && (!it.points || !it.out)) s = bfail(ESOM_EINVAL, "null buffer");
        else if (((uintptr_t)it.points & 15u) || ((uintptr_t)it.out & 7u))
            s = bfail(ESOM_EALIGN, "points must be 16-byte and out 8-byte aligned");
        else if (!(it.boost > 0.f) || !(it.adjust >= 0.f)) s = bfail(ESOM_EINVAL, "boost/adjust");
        if (s != ESOM_OK) {
            delete b;
            return s;
        }
        const auto key = std::make_pair(h->d, h->kc);
        if (!gidx.count(key)) {
            gidx[key] = (int)b->groups.size();
            b->groups.emplace_back();
            b->groups.back().D = h->d;
            b->groups.back().kc = h->kc;
            b->groups.back().ops = h->ops;
        }
        b->groups[(size_t)gidx[key]].items.push_back(i);
    }
    e = cudaMalloc(&b->status, kStatusWords * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, kStatusWords * sizeof(int));
    esom_status s = e == cudaSuccess ? ESOM_OK : bcuda(e, "batch status");
    for (Group &g : b->groups) {
        if (s != ESOM_OK) break;
        for (int idx : g.items) {
            const esom_batch_item &it = b->items[(size_t)idx];
            const esom_ctx *h = it.landmarks;
            FusedArgs a;
            esom::fill_args(h, it.points, it.n, it.out, it.boost, it.adjust, &a);
            a.status = b->status;
            g.tile_base.push_back(g.tiles);
            const long long nt = (it.n + esom::kThreads - 1) / esom::kThreads;
            const long long pc = point_cost(h);
            for (long long t = 0; t < nt; ++t) {
                g.tile_item.push_back((int)g.args.size());
                const long long rows = std::min<long long>(esom::kThreads, it.n - t * esom::kThreads);
                g.cost.push_back(rows * pc);
            }
            g.tiles += nt;
            g.args.push_back(a);
        }
        long long group_points = 0;
        for (const FusedArgs &fa : g.args) group_points += fa.n;
        e = cudaMalloc(&g.d_items, g.args.size() * sizeof(FusedArgs));
        if (e == cudaSuccess)
            e = cudaMalloc(&g.d_refine, (size_t)(group_points > 0 ? group_points : 1) * sizeof(int2));
        if (e == cudaSuccess) e = cudaMalloc(&g.d_tile_base, g.tile_base.size() * sizeof(long long));
        if (e == cudaSuccess && g.tiles > 0) e = cudaMalloc(&g.d_tile_item, g.tile_item.size() * sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemcpy(g.d_tile_base, g.tile_base.data(), g.tile_base.size() * sizeof(long long),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess && g.tiles > 0)
            e = cudaMemcpy(g.d_tile_item, g.tile_item.data(), g.tile_item.size() * sizeof(int),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            s = bcuda(e, "batch plan allocation");
            break;
        }
        if (g.tiles == 0) continue;
        s = autotune_flag ? autotune(b, g) : apply_shape(b, g, Shape{0, 0, 0});
    }
    if (s != ESOM_OK) {
        esom_batch_destroy(b);
        return s;
    }
    describe(b);
    *out = b;
    return ESOM_OK;
}

esom_status esom_batch_run(esom_batch b, esom_stream_t stream) {
    if (!b) return bfail(ESOM_EINVAL, "null batch");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (const Group &g : b->groups) {
        esom_status s = launch_group(b, g, st);
        if (s != ESOM_OK) return s;
    }
    return ESOM_OK;
}

// Launches the batch's work as independent branches forked from and joined
// back into the capture stream: each group's batched launch on a branch of
// its own, and the datasets that run through their own handles (separate
// shapes) on one branch per handle (datasets sharing a handle share its
// scratch, so they stay in order on that branch).  The branches have no
// data in common, so the graph lets their kernels overlap on the GPU.
esom_status capture_branches(esom_batch_ctx *b, cudaStream_t cap) {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::map<const esom_ctx *, size_t> by_handle;
    cudaEvent_t fork = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(fork, cap);
    auto branch = [&](size_t *idx) -> cudaError_t {
        cudaStream_t bs;
        cudaError_t r = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
        if (r != cudaSuccess) return r;
        streams.push_back(bs);
        *idx = streams.size() - 1;
        return cudaStreamWaitEvent(bs, fork, 0);
    };
    esom_status s = e == cudaSuccess ? ESOM_OK : bcuda(e, "batch graph fork");
    for (const Group &g : b->groups) {
        if (s != ESOM_OK || g.tiles == 0) continue;
        if (!g.shape.separate) {
            size_t bi = 0;
            e = branch(&bi);
            s = e == cudaSuccess ? launch_group(b, g, streams[bi]) : bcuda(e, "batch branch");
            continue;
        }
        for (int idx : g.items) {
            const esom_batch_item &it = b->items[(size_t)idx];
            if (it.n == 0 || s != ESOM_OK) continue;
            auto f = by_handle.find(it.landmarks);
            size_t bi = 0;
            if (f == by_handle.end()) {
                e = branch(&bi);
                if (e != cudaSuccess) {
                    s = bcuda(e, "batch branch");
                    break;
                }
                by_handle[it.landmarks] = bi;
            } else {
                bi = f->second;
            }
            s = esom_project(it.landmarks, it.points, it.n, it.out, it.boost, it.adjust,
                             reinterpret_cast<esom_stream_t>(streams[bi]));
        }
    }
    // join every branch back into the capture stream
    for (cudaStream_t bs : streams) {
        cudaEvent_t j = nullptr;
        cudaError_t r = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        if (r == cudaSuccess) r = cudaEventRecord(j, bs);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(cap, j, 0);
        if (j) events.push_back(j);
        if (r != cudaSuccess && s == ESOM_OK) s = bcuda(r, "batch graph join");
    }
    for (cudaEvent_t j : events) cudaEventDestroy(j);
    for (cudaStream_t bs : streams) cudaStreamDestroy(bs);
    if (fork) cudaEventDestroy(fork);
    return s;
}

esom_status esom_batch_run_graph(esom_batch b, esom_stream_t stream) {
    if (!b) return bfail(ESOM_EINVAL, "null batch");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!b->exec) {
        cudaStream_t cap;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bcuda(e, "capture stream");
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        esom_status s = e == cudaSuccess ? capture_branches(b, cap) : bcuda(e, "begin capture");
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (s != ESOM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (e2 != cudaSuccess) return bcuda(e2, "end capture");
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            return bcuda(e, "graph instantiate");
        }
        b->graph = graph;
    }
    const cudaError_t e = cudaGraphLaunch(b->exec, st);
    return e == cudaSuccess ? ESOM_OK : bcuda(e, "graph launch");
}

const char *esom_batch_plan(esom_batch b) { return b ? b->plan.c_str() : ""; }

esom_status esom_batch_destroy(esom_batch b) {
    if (!b) return ESOM_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (Group &g : b->groups) {
        cudaFree(g.d_items);
        cudaFree(g.d_tile_base);
        cudaFree(g.d_tile_item);
        cudaFree(g.d_cta_begin);
        cudaFree(g.d_refine);
    }
    cudaFree(b->status);
    delete b;
    return ESOM_OK;
}

}  // extern "C"
