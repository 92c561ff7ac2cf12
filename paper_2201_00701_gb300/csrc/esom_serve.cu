// SOM landmark update and the frame-serving runtime (C ABI in include/esom.h).
//
// The paper's interactive use (Section 3.2.2 and Section 5.1) trains the
// high-dimensional landmarks as SOM weights while the user watches, and
// re-projects every point each frame.  A frame here is: one SOM step on a
// minibatch of the session's own points (best-matching landmark by the k-NN
// kernel, neighbourhood-weighted batch update), a landmark refresh, and the
// projection of all the session's points.
//
// The server keeps sessions resident on the device, admits a session only if
// its device memory fits the budget, and runs frames with continuous
// batching: up to `max_inflight` frames of different sessions are on the GPU
// at once (each on its session's stream, so they overlap), frames of one
// session run in order, and a frame starts as soon as a slot frees.  Frame
// completion times are read from GPU events against a reference event, so
// latency does not depend on how often the host polls.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <mutex>
#include <vector>

#include "esom.h"
#include "esom_ctx.h"
#include "esom_fused.cuh"
#include "esom_kernels.h"

namespace {

esom_status sfail(esom_status s, const char *msg) {
    return static_cast<esom_status>(esom::set_error(s, msg));
}

esom_status scuda(cudaError_t e, const char *what) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    return sfail(ESOM_ECUDA, buf);
}

// One warp per landmark j: h = exp(-|l_j - l_b(x)|^2 / (2 sigma^2)) over the
// minibatch, then L_j += alpha (sum h x / sum h - L_j).
template <int D>
__global__ void som_update_kernel(float *__restrict__ hi, const float2 *__restrict__ lo, int L,
                                  const float *__restrict__ batch, const int *__restrict__ bmu,
                                  int bmu_stride, int b, float alpha, float inv2s2) {
    const int j = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= L) return;
    const float2 lj = lo[j];
    float acc[D];
#pragma unroll
    for (int t = 0; t < D; ++t) acc[t] = 0.f;
    float hs = 0.f;
    for (int x = lane; x < b; x += 32) {
        const int bi = bmu[(size_t)x * bmu_stride];
        if ((unsigned)bi >= (unsigned)L) continue;  // not a landmark: the point is skipped
        const float2 li = lo[bi];
        const float dx = lj.x - li.x, dy = lj.y - li.y;
        const float h = expf(-(dx * dx + dy * dy) * inv2s2);
        hs += h;
        const float4 *row = reinterpret_cast<const float4 *>(batch + (size_t)x * D);
#pragma unroll
        for (int e = 0; e < D / 4; ++e) {
            const float4 v = row[e];
            acc[4 * e] = fmaf(h, v.x, acc[4 * e]);
            acc[4 * e + 1] = fmaf(h, v.y, acc[4 * e + 1]);
            acc[4 * e + 2] = fmaf(h, v.z, acc[4 * e + 2]);
            acc[4 * e + 3] = fmaf(h, v.w, acc[4 * e + 3]);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        hs += __shfl_xor_sync(0xffffffffu, hs, off);
#pragma unroll
        for (int t = 0; t < D; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], off);
    }
    if (hs > 1e-30f) {
        const float ih = 1.f / hs;
#pragma unroll
        for (int t = 0; t < D; ++t)
            if ((t & 31) == lane) {
                float *p = hi + (size_t)j * D + t;
                *p = fmaf(alpha, fmaf(acc[t], ih, -*p), *p);
            }
    }
}

template <int D>
cudaError_t launch_som(float *hi, const float *lo, int L, const float *batch, const int *bmu,
                       int stride, int b, float alpha, float sigma, cudaStream_t st) {
    const int threads = 256;
    const int blocks = (int)(((size_t)L * 32 + threads - 1) / threads);
    som_update_kernel<D><<<blocks, threads, 0, st>>>(hi, reinterpret_cast<const float2 *>(lo), L,
                                                     batch, bmu, stride, b, alpha,
                                                     0.5f / (sigma * sigma));
    return cudaGetLastError();
}

cudaError_t som_dispatch(int d, float *hi, const float *lo, int L, const float *batch,
                         const int *bmu, int stride, int b, float alpha, float sigma,
                         cudaStream_t st) {
    switch (d) {
#define ESOM_SOM_CASE(DV) \
    case DV: return launch_som<DV>(hi, lo, L, batch, bmu, stride, b, alpha, sigma, st);
        ESOM_SOM_CASE(4) ESOM_SOM_CASE(8) ESOM_SOM_CASE(12) ESOM_SOM_CASE(16)
        ESOM_SOM_CASE(20) ESOM_SOM_CASE(24) ESOM_SOM_CASE(28) ESOM_SOM_CASE(32)
        ESOM_SOM_CASE(36) ESOM_SOM_CASE(40) ESOM_SOM_CASE(44) ESOM_SOM_CASE(48)
        ESOM_SOM_CASE(52) ESOM_SOM_CASE(56) ESOM_SOM_CASE(60) ESOM_SOM_CASE(64)
#undef ESOM_SOM_CASE
        default: return cudaErrorInvalidValue;
    }
}

// Best-matching landmark of each minibatch point: the nearest landmark by
// the exact FP32 difference-form distance of the projection kernels
// (dist2_row on the handle's rows, centred like theirs), ties to the lower
// index -- the first column esom_knn returns, in one launch instead of a
// k-NN pass.  One thread per point; the block streams the rows through
// shared memory in chunks of 64 (a multiple of 8, so each row keeps its
// chunk swizzle).
constexpr int kBmuThreads = 256;
constexpr int kBmuChunk = 64;

template <int D>
__global__ void __launch_bounds__(kBmuThreads) bmu_kernel(const float *__restrict__ X, int b,
                                                          const float *__restrict__ hi, int L,
                                                          const float *__restrict__ center,
                                                          int *__restrict__ bmu) {
    __shared__ __align__(16) float4 rows[kBmuChunk * D / 4];
    const int p = blockIdx.x * kBmuThreads + threadIdx.x;
    const bool act = p < b;
    float4 x[D / 4];
    const float4 *xp = reinterpret_cast<const float4 *>(X) + (size_t)(act ? p : 0) * (D / 4);
#pragma unroll
    for (int e = 0; e < D / 4; ++e) x[e] = esom::centred(__ldg(xp + e), center, e);
    const float4 *Lg = reinterpret_cast<const float4 *>(hi);
    float best = INFINITY;
    int bi = 0;
    for (int c0 = 0; c0 < L; c0 += kBmuChunk) {
        const int cnt = L - c0 < kBmuChunk ? L - c0 : kBmuChunk;
        __syncthreads();
        for (int i = threadIdx.x; i < cnt * (D / 4); i += kBmuThreads)
            rows[i] = __ldg(Lg + (size_t)c0 * (D / 4) + i);
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const float d2 = esom::dist2_row<D>(x, rows, j);
            if (d2 < best) {
                best = d2;
                bi = c0 + j;
            }
        }
    }
    if (act) bmu[p] = bi;
}

cudaError_t bmu_dispatch(int d, const float *X, int b, const float *hi, int L, const float *center,
                         int *bmu, cudaStream_t st) {
    const int blocks = (b + kBmuThreads - 1) / kBmuThreads;
    switch (d) {
#define ESOM_BMU_CASE(DV) \
    case DV: bmu_kernel<DV><<<blocks, kBmuThreads, 0, st>>>(X, b, hi, L, center, bmu); break;
        ESOM_BMU_CASE(4) ESOM_BMU_CASE(8) ESOM_BMU_CASE(12) ESOM_BMU_CASE(16)
        ESOM_BMU_CASE(20) ESOM_BMU_CASE(24) ESOM_BMU_CASE(28) ESOM_BMU_CASE(32)
        ESOM_BMU_CASE(36) ESOM_BMU_CASE(40) ESOM_BMU_CASE(44) ESOM_BMU_CASE(48)
        ESOM_BMU_CASE(52) ESOM_BMU_CASE(56) ESOM_BMU_CASE(60) ESOM_BMU_CASE(64)
#undef ESOM_BMU_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Counter-based choice of the minibatch window of frame f (splitmix64).
uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

struct Frame {
    uint64_t id;
    double arrival;
};

struct Session {
    esom_session_desc desc{};
    esom_handle h = nullptr;
    float *points = nullptr, *out = nullptr, *hi = nullptr, *lo = nullptr;
    int *bmu = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    size_t bytes = 0;
    std::deque<Frame> queue;
    bool inflight = false;
    std::vector<Frame> current;  // frames the work in flight completes
    int plan = -1;               // ESOM_PLAN_* chosen by esom_tune (automatic screening)
    std::deque<esom_frame_done> finished;  // completed, not yet reported
    uint64_t submitted = 0, completed = 0;
};

}  // namespace

struct esom_server_ctx {
    uint64_t budget = 0, used = 0;
    int max_inflight = 1, inflight = 0, dev = 0;
    int coalesce = 0;  // run a session's queued frames' SOM steps, then one projection
    int screening = ESOM_SCREEN_FP32;  // screening mode of the sessions' handles
    std::vector<Session *> sessions;
    cudaEvent_t ref = nullptr;
    std::chrono::steady_clock::time_point t0;
    double ref_host = 0.0;
    std::mutex mu;
};

namespace {

double host_now(const esom_server_ctx *s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// One SOM step of frame f of session ss on its stream: k-NN of the frame's
// minibatch window, the update, the landmark refresh.
esom_status som_frame_step(Session &ss, const Frame &f) {
    const esom_session_desc &d = ss.desc;
    cudaStream_t st = ss.stream;
    const esom_stream_t est = reinterpret_cast<esom_stream_t>(st);
    esom_status r = ESOM_OK;
    if (d.minibatch > 0 && d.alpha > 0.f) {
        const int64_t b = d.minibatch < d.n ? d.minibatch : d.n;
        const uint64_t span = (uint64_t)(d.n - b) + 1;
        const int64_t off = (int64_t)(mix64(d.seed ^ (f.id * 0x100000001b3ull)) % span);
        // best-matching landmarks of the window (esom_knn's first column)
        cudaError_t e = bmu_dispatch(d.d, ss.points + off * d.d, (int)b, ss.h->hi, d.L,
                                     ss.h->centered ? ss.h->center : nullptr, ss.bmu, st);
        if (e != cudaSuccess) return scuda(e, "best-matching landmarks");
        e = som_dispatch(d.d, ss.hi, ss.lo, d.L, ss.points + off * d.d, ss.bmu, 1, (int)b,
                         d.alpha, d.sigma, st);
        if (e != cudaSuccess) return scuda(e, "SOM update");
        r = esom_set_landmarks(ss.h, ss.hi, ss.lo, est);
        if (r != ESOM_OK) return r;
    }
    return ESOM_OK;
}

// Enqueues the queue's front frame of session ss -- or, when the server
// coalesces, every queued frame: their SOM steps in order, then one
// projection, which all of them complete with -- and the completion event.
esom_status launch_frames(esom_server_ctx *s, Session &ss) {
    const esom_session_desc &d = ss.desc;
    ss.current.clear();
    do {
        ss.current.push_back(ss.queue.front());
        ss.queue.pop_front();
        esom_status r = som_frame_step(ss, ss.current.back());
        if (r != ESOM_OK) return r;
    } while (s->coalesce && !ss.queue.empty());
    esom_status r = esom_project(ss.h, ss.points, d.n, ss.out, d.boost, d.adjust,
                                 reinterpret_cast<esom_stream_t>(ss.stream));
    if (r != ESOM_OK) return r;
    const cudaError_t e = cudaEventRecord(ss.done, ss.stream);
    if (e != cudaSuccess) return scuda(e, "frame event");
    ss.inflight = true;
    ++s->inflight;
    return ESOM_OK;
}

// Starts queued frames while slots are free, oldest arrival first.
esom_status fill_slots(esom_server_ctx *s) {
    while (s->inflight < s->max_inflight) {
        Session *best = nullptr;
        for (Session *ss : s->sessions)
            if (!ss->inflight && !ss->queue.empty() &&
                (!best || ss->queue.front().arrival < best->queue.front().arrival))
                best = ss;
        if (!best) break;
        esom_status r = launch_frames(s, *best);
        if (r != ESOM_OK) return r;
    }
    return ESOM_OK;
}

void free_session(Session *ss) {
    if (!ss) return;
    if (ss->stream) cudaStreamSynchronize(ss->stream);
    esom_destroy(ss->h);
    cudaFree(ss->points);
    cudaFree(ss->out);
    cudaFree(ss->hi);
    cudaFree(ss->lo);
    cudaFree(ss->bmu);
    if (ss->done) cudaEventDestroy(ss->done);
    if (ss->stream) cudaStreamDestroy(ss->stream);
    delete ss;
}

}  // namespace

extern "C" {

esom_status esom_som_update(float *hi, const float *lo, int d, int L, const float *batch,
                            const int32_t *bmu, int bmu_stride, int64_t b, float alpha,
                            float sigma, esom_stream_t stream) {
    if (!hi || !lo || (b > 0 && (!batch || !bmu))) return sfail(ESOM_EINVAL, "null pointer");
    if (d < 4 || d > ESOM_MAX_D || d % 4) return sfail(ESOM_EINVAL, "d must be a multiple of 4 in [4, 64]");
    if (L < 1 || b < 0 || b > (1 << 30) || bmu_stride < 1) return sfail(ESOM_EINVAL, "sizes");
    if (!(sigma > 0.f) || !(alpha >= 0.f)) return sfail(ESOM_EINVAL, "sigma > 0, alpha >= 0");
    if (((uintptr_t)batch & 15u) || ((uintptr_t)lo & 7u))
        return sfail(ESOM_EALIGN, "batch 16-byte and lo 8-byte aligned");
    if (b == 0 || alpha == 0.f) return ESOM_OK;
    const cudaError_t e = som_dispatch(d, hi, lo, L, batch, bmu, bmu_stride, (int)b, alpha, sigma,
                                       reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? ESOM_OK : scuda(e, "SOM update");
}

esom_status esom_server_create(uint64_t budget_bytes, int max_inflight, esom_server *out) {
    if (!out) return sfail(ESOM_EINVAL, "null output");
    *out = nullptr;
    if (max_inflight < 1) return sfail(ESOM_EINVAL, "max_inflight < 1");
    esom_server_ctx *s = new (std::nothrow) esom_server_ctx;
    if (!s) return sfail(ESOM_ENOMEM, "host allocation");
    s->budget = budget_bytes;
    s->max_inflight = max_inflight;
    cudaError_t e = cudaGetDevice(&s->dev);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ref);
    if (e == cudaSuccess) e = cudaEventRecord(s->ref, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(s->ref);
    if (e != cudaSuccess) {
        delete s;
        return scuda(e, "server set-up");
    }
    s->t0 = std::chrono::steady_clock::now();
    s->ref_host = 0.0;
    *out = s;
    return ESOM_OK;
}

double esom_server_now(esom_server s) { return s ? host_now(s) : 0.0; }

esom_status esom_server_set_screening(esom_server s, int mode) {
    if (!s) return sfail(ESOM_EINVAL, "null server");
    if (mode != ESOM_SCREEN_FP32 && mode != ESOM_SCREEN_TF32 && mode != ESOM_SCREEN_BF16 &&
        mode != ESOM_SCREEN_AUTO)
        return sfail(ESOM_EINVAL, "unknown screening mode");
    std::lock_guard<std::mutex> lock(s->mu);
    if (!s->sessions.empty()) return sfail(ESOM_EINVAL, "set the screening mode before adding sessions");
    s->screening = mode;
    return ESOM_OK;
}

esom_status esom_server_set_coalescing(esom_server s, int on) {
    if (!s) return sfail(ESOM_EINVAL, "null server");
    std::lock_guard<std::mutex> lock(s->mu);
    s->coalesce = on ? 1 : 0;
    return ESOM_OK;
}

esom_status esom_server_add_session(esom_server s, const esom_session_desc *desc,
                                    const float *points, const float *hi, const float *lo,
                                    int *session) {
    if (!s || !desc || !session || !points || !hi || !lo) return sfail(ESOM_EINVAL, "null argument");
    const esom_session_desc &d = *desc;
    if (d.n < 1 || d.minibatch < 0 || !(d.boost > 0.f) || !(d.adjust >= 0.f) ||
        (d.minibatch > 0 && d.alpha > 0.f && !(d.sigma > 0.f)))
        return sfail(ESOM_EINVAL, "session description");
    std::lock_guard<std::mutex> lock(s->mu);
    // resident points and output, the session's landmark copy and the
    // handle's (rows, 2-D positions, norms, squared-distance table), the
    // minibatch k-NN indices
    const size_t qtab = d.L <= esom::kPtabMaxL   ? (size_t)d.L * d.L * 8
                        : d.L <= esom::kQtabMaxL ? (size_t)d.L * d.L * 4
                                                 : 0;
    // tensor-core screening: landmark images and the neighbour scratch
    const size_t img = s->screening != ESOM_SCREEN_FP32
                           ? (size_t)((d.L + esom::kTcN - 1) / esom::kTcN) *
                                     esom::tc_chunk_bytes(d.d, esom::kTcTf32) +
                                 (size_t)esom::kTcPass * (d.k * 8 + (d.k + 8) * 4) +
                                 // the pair table in the landmark order
                                 (d.L <= esom::kPtabMaxL ? (size_t)d.L * d.L * 8 + d.L * 4 : 0)
                           : 0;
    const size_t bytes = (size_t)d.n * d.d * 4 + (size_t)d.n * 8 + (size_t)d.L * (d.d + 2) * 4 * 2 +
                         (size_t)((d.L + 63) & ~63) * 4 + qtab + img +
                         (size_t)d.minibatch * d.k * 4 + 4096;
    if (s->used + bytes > s->budget)
        return sfail(ESOM_ENOMEM, "session refused: device memory budget exceeded");
    Session *ss = new (std::nothrow) Session;
    if (!ss) return sfail(ESOM_ENOMEM, "host allocation");
    ss->desc = d;
    ss->bytes = bytes;
    esom_status r = esom_create(d.d, d.L, d.k, &ss->h);
    if (r == ESOM_OK && (s->screening == ESOM_SCREEN_TF32 || s->screening == ESOM_SCREEN_BF16))
        r = esom_set_screening(ss->h, s->screening, nullptr);
    cudaError_t e = cudaSuccess;
    if (r == ESOM_OK) {
        e = cudaMalloc(&ss->points, (size_t)d.n * d.d * 4);
        if (e == cudaSuccess) e = cudaMalloc(&ss->out, (size_t)d.n * 8);
        if (e == cudaSuccess) e = cudaMalloc(&ss->hi, (size_t)d.L * d.d * 4);
        if (e == cudaSuccess) e = cudaMalloc(&ss->lo, (size_t)d.L * 8);
        if (e == cudaSuccess) e = cudaMalloc(&ss->bmu, (size_t)(d.minibatch > 0 ? d.minibatch : 1) * d.k * 4);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ss->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&ss->done);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ss->points, points, (size_t)d.n * d.d * 4, cudaMemcpyDefault, ss->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ss->hi, hi, (size_t)d.L * d.d * 4, cudaMemcpyDefault, ss->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ss->lo, lo, (size_t)d.L * 8, cudaMemcpyDefault, ss->stream);
        if (e == cudaSuccess) {
            r = esom_set_landmarks(ss->h, ss->hi, ss->lo, reinterpret_cast<esom_stream_t>(ss->stream));
        }
        if (e == cudaSuccess && r == ESOM_OK) e = cudaStreamSynchronize(ss->stream);
        if (e == cudaSuccess && r == ESOM_OK && s->screening == ESOM_SCREEN_AUTO)
            r = esom_tune(ss->h, ss->points, d.n, ss->out, d.boost, d.adjust,
                          reinterpret_cast<esom_stream_t>(ss->stream), &ss->plan);
        // a frame's SOM step moves the landmarks a little: the spatial order
        // of the tensor-core screening (computed at admission) is kept, so a
        // frame's landmark refresh does not pay for a new one
        if (r == ESOM_OK) ss->h->keep_order = 1;
    }
    if (r != ESOM_OK || e != cudaSuccess) {
        free_session(ss);
        return r != ESOM_OK ? r : sfail(ESOM_ENOMEM, "session allocation");
    }
    s->used += bytes;
    *session = (int)s->sessions.size();
    s->sessions.push_back(ss);
    return ESOM_OK;
}

esom_status esom_server_submit(esom_server s, int session, double arrival) {
    if (!s || session < 0 || session >= (int)s->sessions.size() || !s->sessions[(size_t)session])
        return sfail(ESOM_EINVAL, "no such session");
    std::lock_guard<std::mutex> lock(s->mu);
    Session &ss = *s->sessions[(size_t)session];
    ss.queue.push_back(Frame{ss.submitted++, arrival});
    return fill_slots(s);
}

esom_status esom_server_poll(esom_server s, int wait_all, esom_frame_done *done, int max,
                             int *count) {
    if (!s || !count || (max > 0 && !done)) return sfail(ESOM_EINVAL, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    *count = 0;
    for (;;) {
        for (size_t i = 0; i < s->sessions.size(); ++i) {
            Session *ss = s->sessions[i];
            if (!ss || !ss->inflight) continue;
            cudaError_t q = wait_all ? cudaEventSynchronize(ss->done) : cudaEventQuery(ss->done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return scuda(q, "frame completion");
            float ms = 0.f;
            cudaError_t e = cudaEventElapsedTime(&ms, s->ref, ss->done);
            if (e != cudaSuccess) return scuda(e, "frame timing");
            for (const Frame &f : ss->current) {
                esom_frame_done o;
                o.session = (int)i;
                o.frame = f.id;
                o.arrival = f.arrival;
                o.completion = s->ref_host + ms / 1e3;
                ss->finished.push_back(o);
            }
            ss->completed += ss->current.size();
            ss->current.clear();
            ss->inflight = false;
            --s->inflight;
        }
        esom_status r = fill_slots(s);
        if (r != ESOM_OK) return r;
        // report completed frames, oldest completion first within a session
        for (Session *ss : s->sessions)
            while (ss && !ss->finished.empty() && *count < max) {
                done[(*count)++] = ss->finished.front();
                ss->finished.pop_front();
            }
        bool pending = s->inflight > 0;
        for (Session *ss : s->sessions)
            if (ss && !ss->queue.empty()) pending = true;
        if (!wait_all || !pending || *count >= max) break;
    }
    return ESOM_OK;
}

esom_status esom_server_session_output(esom_server s, int session, const float **out,
                                       uint64_t *frames) {
    if (!s || session < 0 || session >= (int)s->sessions.size() || !s->sessions[(size_t)session])
        return sfail(ESOM_EINVAL, "no such session");
    std::lock_guard<std::mutex> lock(s->mu);
    const Session &ss = *s->sessions[(size_t)session];
    if (out) *out = ss.out;
    if (frames) *frames = ss.completed;
    return ESOM_OK;
}

esom_status esom_server_memory(esom_server s, uint64_t *used, uint64_t *budget) {
    if (!s) return sfail(ESOM_EINVAL, "null server");
    if (used) *used = s->used;
    if (budget) *budget = s->budget;
    return ESOM_OK;
}

esom_status esom_server_destroy(esom_server s) {
    if (!s) return ESOM_OK;
    for (Session *ss : s->sessions) free_session(ss);
    if (s->ref) cudaEventDestroy(s->ref);
    delete s;
    return ESOM_OK;
}

}  // extern "C"
