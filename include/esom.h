/*
 * esom.h -- C ABI of the GB300 EmbedSOM projection library (libesom.so).
 *
 * The library maps n high-dimensional points to 2-D with the EmbedSOM
 * projection (paper: "Scalable semi-supervised dimensionality reduction with
 * GPU-accelerated EmbedSOM", Section 3.1, steps 1-4; GPU form in Section 4:
 * the k-NN step of Section 4.2 and the projection step of Section 4.3, run
 * as in Section 4.4 but fused into one kernel).
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers (for example from torch's
 *     data_ptr()) to contiguous, row-major float32 / int32 data, unless the
 *     entry point says otherwise.  The caller owns every buffer it passes;
 *     the library never frees caller memory.
 *   - `stream` is a cudaStream_t (a CUstream_st*); NULL is the legacy
 *     default stream.  Calls are asynchronous on that stream, make no host
 *     synchronisation and allocate nothing after esom_create /
 *     esom_set_landmarks (esom_project_host allocates its staging buffers on
 *     its first call).
 *   - A handle is bound to the device that was current at esom_create;
 *     calls made while another device is current return ESOM_EINVAL.
 *   - Every call checks its arguments first and launches nothing when they
 *     are invalid; the message of the last failure on the calling host
 *     thread is returned by esom_last_error().
 *   - n == 0 returns ESOM_OK without launching.
 *   - NaN or Inf inputs give unspecified output values, never a fault.
 */
#ifndef ESOM_H
#define ESOM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct esom_ctx *esom_handle;
typedef struct CUstream_st *esom_stream_t; /* same type as cudaStream_t */

typedef enum {
    ESOM_OK = 0,
    ESOM_EINVAL = -1,        /* bad argument (size, range, null pointer, device) */
    ESOM_ENOMEM = -2,        /* device or host allocation failed */
    ESOM_EALIGN = -3,        /* pointer not 16-byte aligned, or d not a multiple of 4 */
    ESOM_ENOLANDMARKS = -4,  /* esom_set_landmarks has not been called */
    ESOM_ECUDA = -5,         /* a CUDA runtime call or launch failed */
    ESOM_EUNSUPPORTED = -6,  /* (d, k) outside what this build instantiates */
    ESOM_EDEVICE = -7        /* a kernel reported a device-side error (bounded wait ran out) */
} esom_status;

/* Limits of this build: d is a multiple of 4 in [4, ESOM_MAX_D];
 * 2 <= k <= min(L, ESOM_MAX_K); 1 <= L <= ESOM_MAX_L. */
#define ESOM_MAX_D 64
#define ESOM_MAX_K 32
#define ESOM_MAX_L 65536

/* Creates a projection context for points of dimension d, L landmarks and k
 * neighbours (Section 3.1 step 1 requires 3 <= k <= L; k = 2 is accepted as
 * a degenerate case whose result is the nearest landmark's 2-D position).
 * Allocates the device copies of the landmarks, their squared norms, a
 * device status word and, for L <= 4096, an L x L table of squared landmark
 * distances (L*L*4 bytes: 64 MiB at L = 4096) on the current device.  On
 * success *out receives the handle. */
esom_status esom_create(int d, int L, int k, esom_handle *out);

/* Copies the landmarks into the handle (Section 3.1: L is g x d, l is g x 2;
 * the paper's g is L here).  hi: L x d float32, lo: L x 2 float32, host or
 * device pointers (copied with cudaMemcpyDefault on `stream`).  The caller
 * keeps ownership and may reuse the buffers once the copy has run on the
 * stream.  Small kernels on the same stream then compute the landmarks'
 * squared norms for the screening scan and, for L <= 4096, the table of
 * squared distances |L_u - L_v|^2 that the pair loop of step 3 reads (the
 * values the loop would otherwise compute per point, bit for bit).  Each
 * call increments the landmark version.  Projections queued on other streams are not ordered against this
 * copy by the library. */
esom_status esom_set_landmarks(esom_handle h, const float *hi, const float *lo,
                               esom_stream_t stream);

/* Landmark version: 0 before the first esom_set_landmarks, then 1, 2, ... */
uint64_t esom_landmark_version(esom_handle h);

/* EmbedSOM projection (Section 3.1 steps 1-4; Section 4.3):
 *   points: n x d float32, 16-byte aligned (ESOM_EALIGN otherwise);
 *   out:    n x 2 float32, 8-byte aligned, receives x_i = (x, y);
 *   boost > 0: sharpness of the distance-to-score map (step 2);
 *   adjust >= 0: pair weight s_u s_v / |l_v - l_u|^(2 adjust); adjust = 1 is
 *     exactly the objective printed in step 4.
 * One fused kernel per call: k-NN by an FP32 screening scan whose
 * candidates are re-ranked exactly in FP32 (the k nearest are those of the
 * FP32 difference-form distance, certified by an error bound), scores and
 * pair terms in FP32, the 2x2 determinant and solve in FP64.  Inputs whose
 * squared distances overflow FP32 give unspecified output. */
esom_status esom_project(esom_handle h, const float *points, int64_t n, float *out,
                         float boost, float adjust, esom_stream_t stream);

/* k-NN step alone (Section 3.1 step 1; Section 4.2):
 *   points: n x d float32, 16-byte aligned;
 *   idx:    n x k int32, landmark indices in ascending distance, ties to the
 *           lower index;
 *   dist2:  n x k float32, squared Euclidean distances (nullable). */
esom_status esom_knn(esom_handle h, const float *points, int64_t n, int32_t *idx,
                     float *dist2, esom_stream_t stream);

/* esom_project for HOST buffers: points_host (n x d) and out_host (n x 2)
 * are host pointers (pinned memory gives overlapped copies; pageable memory
 * works but copies synchronously).  The points are streamed through device
 * staging buffers owned by the handle in chunks, with host-to-device copies,
 * projection and device-to-host copies of successive chunks overlapped on
 * `stream` and two internal streams.  Returns after enqueueing; out_host is
 * complete when `stream` reaches this point (synchronise it before reading).
 * The staging buffers (2 x chunk x (d + 2) x 4 bytes) are allocated on the
 * first call and kept until esom_destroy. */
esom_status esom_project_host(esom_handle h, const float *points_host, int64_t n,
                              float *out_host, float boost, float adjust,
                              esom_stream_t stream);

/* Waits for `stream`, then reports and clears any device-side error flag
 * that a kernel of this handle raised (a bounded wait on an mbarrier that
 * ran out): ESOM_EDEVICE if one was raised, ESOM_OK otherwise. */
esom_status esom_device_status(esom_handle h, esom_stream_t stream);

/* Counters kept by a handle's kernels. */
typedef struct {
    uint64_t points;    /* points projected or searched */
    uint64_t rescans;   /* points whose screening certificate failed, so their k
                           nearest were found by an exact rescan (slower path) */
    uint64_t refines;   /* points whose FP32 normal system was too ill-conditioned
                           (det/trace^2 <= 1e-3), so steps 1-4 were recomputed
                           in FP64 (slower path) */
    uint64_t launches;  /* kernels this library launched for esom_project,
                           esom_project_host and esom_knn calls of the handle */
} esom_stats;

/* Waits for `stream`, then returns the handle's counters accumulated since
 * esom_create or the last reset; reset != 0 zeroes them afterwards. */
esom_status esom_get_stats(esom_handle h, esom_stream_t stream, esom_stats *out, int reset);

/* Kernel timing, for measurement (no counterpart in the paper).  With
 * esom_set_timing(h, 1) the handle brackets every kernel it launches for
 * esom_project, esom_project_host and esom_knn with CUDA events on the
 * launching stream (allocated on the first call: 2 x 256 events) and adds
 * each kernel's duration to the total of its kind; esom_get_timing waits for
 * `stream` and returns the totals (reset != 0 zeroes them).  Timing adds one
 * event record on each side of every kernel; it is off by default.
 * Errors: ESOM_EINVAL, ESOM_ECUDA. */
#define ESOM_KERNEL_ORDER 0          /* spatial order of the points (two kernels) */
#define ESOM_KERNEL_TC_KNN 1         /* tensor-core screened k-NN */
#define ESOM_KERNEL_RERANK_PROJECT 2 /* exact re-rank + projection (tensor-core plans) */
#define ESOM_KERNEL_RERANK 3         /* exact re-rank alone (esom_knn, tensor-core plans) */
#define ESOM_KERNEL_RESCAN 4         /* exact rescan of points whose certificate failed */
#define ESOM_KERNEL_PROJECT 5        /* projection from given neighbours */
#define ESOM_KERNEL_REFINE 6         /* FP64 recomputation of ill-conditioned points */
#define ESOM_KERNEL_FUSED 7          /* plain FP32 kernel (fused plan, or the split
                                        plan's k-NN) */
#define ESOM_KERNEL_KINDS 8
typedef struct {
    uint64_t launches[ESOM_KERNEL_KINDS];
    double ms[ESOM_KERNEL_KINDS];
} esom_kernel_times;
esom_status esom_set_timing(esom_handle h, int on);
esom_status esom_get_timing(esom_handle h, esom_stream_t stream, esom_kernel_times *out,
                            int reset);

/* Forces the number of landmarks per shared-memory chunk (0 restores the
 * automatic choice: all landmarks resident when L*d*4 <= 64 KiB, otherwise
 * 32 KiB chunks streamed through two buffers).  Lets tests drive the
 * chunked path with small L; also a tuning knob. */
esom_status esom_set_landmark_chunk(esom_handle h, int chunk);

/* Launch configuration chosen for this handle (for tests and tuning). */
typedef struct {
    int d, L, k, kc;            /* kc: compile-time capacity of the k-NN list */
    int threads_per_block;      /* points per tile = threads per block */
    int blocks_per_sm, num_sms;
    int landmark_chunk;         /* landmarks per shared-memory chunk */
    int landmark_chunks;        /* 1: all landmarks resident in shared memory */
    int shared_bytes;           /* dynamic shared memory per block */
    int screening;              /* ESOM_SCREEN_* in effect (the other fields then
                                   describe the tensor-core launch: 160 threads,
                                   128 points a tile, 64-landmark chunks) */
    int plan;                   /* ESOM_PLAN_* of esom_project */
} esom_config;

esom_status esom_get_config(esom_handle h, esom_config *cfg);

/* ---------------------------------------------------------------------------
 * Screening precision of the k-NN distance block (Section 4.2's fused
 * distance + selection; the block is the g x d term of the cost).
 *   ESOM_SCREEN_FP32  the default: FP32 CUDA-core scan.
 *   ESOM_SCREEN_TF32  the distance block X . L^T runs on the tensor cores
 *                     (tcgen05, FP32 accumulation in tensor memory, 128
 *                     points by 64 landmarks an MMA tile) with operands
 *                     split into two TF32 parts, x = x_hi + x_lo, and the
 *                     three products x_hi l_hi + x_lo l_hi + x_hi l_lo
 *                     (screening error ~2^-21 relative, like FP32's).
 *   ESOM_SCREEN_BF16  the same with BF16 parts (kind::f16; half the operand
 *                     bytes, screening error ~2^-14 relative: more points
 *                     fail the certificate and are rescanned).
 * Either way the listed candidates are re-ranked with exact FP32 distances
 * and a bound on the screening error certifies that no other landmark can be
 * among the k nearest (a point that fails is rescanned exactly; see
 * esom_get_stats), so both modes return the same neighbours, distances and
 * coordinates, bit for bit; the mode only changes speed.
 * With TF32, esom_project runs the tensor-core k-NN kernel and then a
 * re-rank and projection kernel over passes of 2^20 points, exchanging the
 * screened candidate lists through scratch buffers of the handle (2^20 *
 * (k + 4 .. 8) * 4 bytes, and 2^20 * k * 8 bytes for the neighbours of the
 * few points whose certificate fails): projections
 * of one handle on different streams must then not overlap.
 * Switching to TF32 allocates the landmark images (2 * ceil(L/64) * 64 *
 * row bytes, row bytes = 64 for d <= 16, else 128 * ceil(d/32)) and the
 * scratch, kept until esom_destroy, and, if landmarks are set, builds the
 * images on `stream`; later esom_set_landmarks calls rebuild them.
 * Errors: ESOM_EINVAL (unknown mode), ESOM_EUNSUPPORTED (device is not
 * sm_103, or no kernel for this d and k), ESOM_ENOMEM, ESOM_ECUDA.
 * esom_batch_* and esom_project_noalloc always screen in FP32. */
#define ESOM_SCREEN_FP32 0
#define ESOM_SCREEN_TF32 1
#define ESOM_SCREEN_BF16 2
esom_status esom_set_screening(esom_handle h, int mode, esom_stream_t stream);

/* on != 0: esom_project with FP32 screening runs as two kernels, as the
 * paper's pipeline does (Section 4.4): the k-NN kernel writes each point's
 * neighbours to the handle's scratch (2^20 * k * 8 bytes, allocated here),
 * then the projection kernel reads them, in passes of 2^20 points; on = 0:
 * one fused kernel (the default).  Same results either way; projections of
 * one handle on different streams must not overlap while split (the
 * scratch is shared).  Tensor-core screening always runs split.
 * Errors: ESOM_ENOMEM, ESOM_EUNSUPPORTED, ESOM_ECUDA. */
esom_status esom_set_split(esom_handle h, int on);

/* The paper's alternative kernel designs, for ablation (Section 4.2 k-NN
 * algorithms, Section 4.3 projection algorithms).
 *
 * esom_knn_variant: the k nearest landmarks of each point, as esom_knn
 * returns them (same layout, same indices and distances bit for bit: the
 * exact FP32 squared distances ranked by (distance, index)), computed by
 *   ESOM_KNN_BASE     one thread per point, insertion into a sorted array
 *                     of k, landmark rows from global memory;
 *   ESOM_KNN_BITONIC  next_pow2(k) threads per point, bitonic sort of each
 *                     block of that many distances and a bitonic merge into
 *                     the best block so far.
 * idx (n x k int32) and dist2 (n x k float, nullable) are device memory,
 * 4-byte aligned; points as for esom_project.  Finite inputs only.
 *
 * esom_project_knn: steps 2-4 (scores, pair sums, solve) from neighbours
 * the caller gives (idx, dist2: n x k, device memory, 16-byte aligned, the
 * exact squared distances esom_knn returns, ascending), writing out (n x 2):
 *   ESOM_PROJ_TABLE      the library's projection kernel: one thread per
 *                        point, D_uv from the law of cosines and the table
 *                        of squared landmark distances; with esom_knn's
 *                        neighbours the result equals esom_project's bits;
 *   ESOM_PROJ_REGISTERS  one warp per point, pairs in 2 x 2 blocks, D_uv by
 *                        direct dot products over d; equal to the former
 *                        within FP32 rounding.
 * Indices outside [0, L) are clamped.  Errors: ESOM_EINVAL (unknown
 * variant, null pointer, boost/adjust as for esom_project), ESOM_EALIGN. */
#define ESOM_KNN_BASE 1
#define ESOM_KNN_BITONIC 2
#define ESOM_PROJ_TABLE 0
#define ESOM_PROJ_REGISTERS 1
esom_status esom_knn_variant(esom_handle h, int variant, const float *points, int64_t n,
                             int32_t *idx, float *dist2, esom_stream_t stream);
esom_status esom_project_knn(esom_handle h, int variant, const float *points, int64_t n,
                             const int32_t *idx, const float *dist2, float *out, float boost,
                             float adjust, esom_stream_t stream);

/* on != 0: from the next esom_set_landmarks on, the handle centres the data
 * on c = the landmarks' mean rounded to integers: it stores the landmark
 * rows minus c and every kernel subtracts c from the points it loads
 * (distances do not change; FP32 rounding does, slightly).  The screening
 * error bound grows with |x| max|l|, so data far from the origin fail the
 * certificate often and are rescanned; centred, they do not.  Integer c
 * keeps integer-valued data exact.  Off by default.  All plans of the
 * handle agree bit for bit either way, and esom_batch_* groups follow the
 * setting of each member's landmark handle; esom_project_noalloc does not
 * centre.  Errors: ESOM_ENOMEM. */
esom_status esom_set_centering(esom_handle h, int on);

/* Execution plans of esom_project: one fused FP32 kernel, FP32 k-NN kernel +
 * projection kernel, tensor-core k-NN (TF32 or BF16) + projection kernel.  All give the
 * same bits; which is fastest depends on d, L and k (tensor cores pay at
 * large L, the split at small L). */
#define ESOM_PLAN_FUSED 0
#define ESOM_PLAN_SPLIT 1
#define ESOM_PLAN_TF32 2
#define ESOM_PLAN_BF16 3
/* Autotuner: times each plan on the first min(n, 2^20) of `points` (device,
 * n x d) three times on `stream`, writing their coordinates to `out`
 * (n x 2 device), keeps the fastest for the handle (as if set with
 * esom_set_screening / esom_set_split) and stores it in *plan (nullable).
 * Synchronises the stream.  Plans that cannot run here are skipped.
 * Errors: those of esom_project; ESOM_ECUDA if no plan ran. */
esom_status esom_tune(esom_handle h, const float *points, int64_t n, float *out, float boost,
                      float adjust, esom_stream_t stream, int *plan);

/* ---------------------------------------------------------------------------
 * Batched projection: many datasets of uneven n, d and L through one plan.
 * Each item names a handle whose landmarks it uses (d, L and k come from the
 * handle), its points (n x d device, 16-byte aligned), its output (n x 2
 * device, 8-byte aligned) and boost/adjust.  The plan groups items by (d, k
 * capacity); each group is ONE launch of a persistent kernel whose blocks
 * walk contiguous, cost-balanced ranges of the group's 256-point tiles.
 * Handles and buffers must stay valid while the plan exists; landmark
 * updates through the handles are picked up by later runs.  The paper has
 * no batched form (its benchmark runs one dataset at a time, Section 4.1). */
typedef struct esom_batch_ctx *esom_batch;

typedef struct {
    esom_handle landmarks;
    const float *points;
    int64_t n;
    float *out;
    float boost, adjust;
} esom_batch_item;

/* Builds the plan (allocates its device tables).  autotune != 0 times
 * candidate launch shapes of every group on the batch itself (running it a
 * few times, so the outputs are written) and keeps the fastest: landmark
 * chunking (each dataset's own, or forced chunks of 512 or 256), blocks per
 * SM (occupancy limit or 1), or one esom_project per dataset through its
 * handle's own execution plan (for large datasets, and for handles tuned to
 * the tensor-core plan, the persistent group launch may not pay).  The
 * persistent group launch screens in FP32 with the fused kernel whatever
 * the handles' settings; all shapes give the same bits. */
esom_status esom_batch_create(const esom_batch_item *items, int count, int autotune,
                              esom_batch *out);

/* Enqueues the plan's launches (one per group, or one per dataset of a
 * group whose chosen shape is separate launches) on `stream`. */
esom_status esom_batch_run(esom_batch b, esom_stream_t stream);

/* Same as esom_batch_run, replayed from a CUDA graph captured on the first
 * call (one graph launch per run). */
esom_status esom_batch_run_graph(esom_batch b, esom_stream_t stream);

/* JSON description of the plan: groups, tiles, grid, chosen shape. */
const char *esom_batch_plan(esom_batch b);

esom_status esom_batch_destroy(esom_batch b);

/* ---------------------------------------------------------------------------
 * SOM landmark update (Section 3.2.2: the high-dimensional landmarks are
 * trained as SOM weights on the topology of the 2-D landmarks, with a
 * neighbourhood width sigma and a learning rate alpha).  One batch step:
 *   L_j += alpha * ( sum_x h(j, b(x)) x / sum_x h(j, b(x)) - L_j ),
 *   h(j, i) = exp(-|l_j - l_i|^2 / (2 sigma^2)),
 * over the minibatch points x with best-matching landmarks b(x) =
 * bmu[x * bmu_stride] (for example column 0 of esom_knn's idx, stride k);
 * entries outside [0, L) skip their point; landmarks whose neighbourhood
 * weight sums to below 1e-30 (FP32) are left unchanged.
 * hi: L x d device, row-major, updated in place (the caller owns it; pass it
 * to esom_set_landmarks afterwards to project with the new rows);
 * lo: L x 2 device, 8-byte aligned; batch: b x d device, 16-byte aligned;
 * all three and bmu stay owned by the caller.  Asynchronous on `stream`.
 * Errors: ESOM_EINVAL for null pointers, d not a multiple of 4 in [4, 64],
 * L < 1, b < 0 or > 2^30, bmu_stride < 1, sigma <= 0 or alpha < 0;
 * ESOM_EALIGN for misaligned batch or lo; ESOM_ECUDA for a launch error.
 * b = 0 or alpha = 0 changes nothing.  The paper gives no formula for the
 * step; this batch form is this library's reading. */
esom_status esom_som_update(float *hi, const float *lo, int d, int L, const float *batch,
                            const int32_t *bmu, int bmu_stride, int64_t b, float alpha,
                            float sigma, esom_stream_t stream);

/* ---------------------------------------------------------------------------
 * Frame server: sessions with resident points; each frame request runs one
 * SOM step on a minibatch window of the session's points (chosen by a
 * counter-based hash of the seed and the frame number), refreshes the
 * handle's landmarks and re-projects all the session's points (the paper
 * re-projects every point each frame, Section 5.1 and Section 6).
 * Continuous batching: up to max_inflight frames of different sessions run
 * at once (one stream per session, so they overlap on the GPU); a session's
 * frames run in order; queued frames start, oldest arrival first, as slots
 * free up.  A session is admitted only if its device memory fits the
 * budget (ESOM_ENOMEM otherwise).  Times are seconds on the server's clock
 * (esom_server_now); completion times come from GPU events. */
typedef struct esom_server_ctx *esom_server;

typedef struct {
    int d, L, k;
    int64_t n;
    float boost, adjust;
    float alpha, sigma;  /* SOM step; alpha = 0 or minibatch = 0: projection only */
    int minibatch;
    uint64_t seed;
} esom_session_desc;

typedef struct {
    int session;
    uint64_t frame;
    double arrival, completion;
} esom_frame_done;

/* A server on the current device.  budget_bytes: the device memory that
 * admitted sessions may hold together; max_inflight >= 1: frames on the GPU
 * at once.  ESOM_EINVAL for max_inflight < 1, ESOM_ECUDA if the device
 * cannot be set up.  The server is not thread-safe across create/destroy;
 * submit/poll/session_output may be called from several host threads. */
esom_status esom_server_create(uint64_t budget_bytes, int max_inflight, esom_server *out);
/* Admits one session.  points (n x d), hi (L x d), lo (L x 2), float32
 * row-major, host or device: copied into device memory the server owns
 * before the call returns (the caller may free them).  ESOM_ENOMEM when the
 * session's device footprint (points, output, two landmark copies, norms,
 * minibatch indices) would take the server past its budget (nothing is
 * allocated then) or an allocation fails; ESOM_EINVAL for a bad
 * description (n < 1, minibatch < 0, boost <= 0, adjust < 0, sigma <= 0
 * with a SOM step, or d, L, k that esom_create rejects).  *session gets a
 * small integer id, 0, 1, ... in admission order. */
esom_status esom_server_add_session(esom_server s, const esom_session_desc *desc,
                                    const float *points, const float *hi, const float *lo,
                                    int *session);
double esom_server_now(esom_server s);
/* Queues one frame of `session` that arrived at time `arrival`. */
esom_status esom_server_submit(esom_server s, int session, double arrival);
/* Coalescing (off by default): when a session's frames have queued up
 * behind its frame in flight, start them together -- their SOM steps in
 * order, then one projection that completes all of them.  The landmarks
 * follow the same trajectory as frame by frame, so the output after the
 * last frame is the same; only the intermediate projections are skipped
 * (an interactive view shows the newest one).  Keeps latency bounded when
 * frames arrive faster than the GPU projects them. */
esom_status esom_server_set_coalescing(esom_server s, int on);
/* Screening of the handles of sessions added from now on: ESOM_SCREEN_FP32,
 * ESOM_SCREEN_TF32, ESOM_SCREEN_BF16, or ESOM_SCREEN_AUTO (each session's
 * handle is tuned with esom_tune on its own points when it is admitted);
 * only before the first
 * esom_server_add_session (ESOM_EINVAL after).  Results are the same in any
 * mode; TF32 and AUTO add the landmark images and the neighbour scratch to
 * each session's footprint. */
#define ESOM_SCREEN_AUTO 3
esom_status esom_server_set_screening(esom_server s, int mode);
/* Collects finished frames (up to max) and starts queued ones in free
 * slots; wait_all != 0 blocks until every queued frame has finished (or
 * max records were filled). */
esom_status esom_server_poll(esom_server s, int wait_all, esom_frame_done *done, int max,
                             int *count);
/* Device pointer to the session's latest coordinates (n x 2 float32, owned
 * by the server, valid until esom_server_destroy; read it only when no
 * frame of the session is in flight) and the number of frames it has
 * completed. */
esom_status esom_server_session_output(esom_server s, int session, const float **out,
                                       uint64_t *frames);
esom_status esom_server_memory(esom_server s, uint64_t *used, uint64_t *budget);
esom_status esom_server_destroy(esom_server s);

/* Projection without any device allocation, for callers that cannot call
 * cudaMalloc (for example an application whose device memory all belongs to
 * its own pool allocator, or a frame loop that must not risk the device-wide
 * synchronisation cudaMalloc/cudaFree can cause).  The paper has no
 * counterpart: this is a deployment variant of esom_project.
 *
 * The caller passes everything esom_create / esom_set_landmarks /
 * esom_project would take: points (n x d, 16-byte aligned device pointer),
 * hi (L x d) and lo (L x 2) landmarks (host or device pointers), d, L, k,
 * out (n x 2, 8-byte aligned device pointer), boost, adjust and the stream.
 * The function allocates nothing.  Its scratch -- a staged copy of the
 * landmarks, their squared norms and the kernel's status word -- lives in
 * one fixed ESOM_NOALLOC_SCRATCH_BYTES array in device memory that every GPU
 * that loads the library holds until the process exits.  The rest of the
 * array holds the list of points whose normal system needs the FP64
 * recomputation; the points are projected in passes that list fits (at least
 * 8192 points a pass).  Landmark sets with (L * (d + 2) + L rounded up to a
 * multiple of 4) * 4 + 256 + 65536 bytes above ESOM_NOALLOC_SCRATCH_BYTES are
 * rejected with ESOM_EINVAL before anything is queued.
 *
 * The first call on a device looks up that device's address of the scratch
 * array (cudaGetSymbolAddress, with the device current); make that first call
 * before any stream capture.  Every call shares the one array and leaves its
 * landmarks there; the status word is cleared at the start of each call.
 * Calls whose work overlaps on the GPU (on different streams, or from several
 * host threads) race on the scratch and give undefined results: serialise
 * them.  A bounded wait inside the kernel that runs out (2 s; a sign of a
 * stalled device) makes the kernel record it in the scratch status word and
 * leave its remaining points unwritten: this call does not report it, and
 * `out` is then undefined.
 * Errors: ESOM_EINVAL (bad d, L, k, n, pointers, boost or adjust; landmarks
 * beyond the scratch), ESOM_EALIGN, ESOM_EUNSUPPORTED (k > ESOM_MAX_K, no
 * kernel for d and k, or the launch does not fit), ESOM_ECUDA. */
#define ESOM_NOALLOC_SCRATCH_BYTES (4u << 20)
esom_status esom_project_noalloc(const float *points, int64_t n, const float *hi,
                                 const float *lo, int d, int L, int k, float *out,
                                 float boost, float adjust, esom_stream_t stream);

/* ---------------------------------------------------------------------------
 * Test hooks (no counterpart in the paper).
 *
 * esom_test_stall: arms the next launch of the fused kernel of this handle
 * (plan ESOM_PLAN_FUSED; esom_project or esom_knn) to exercise its timeout
 * path: every block first waits on a barrier that nothing completes and
 * gives up after limit_ns (1e3 <= limit_ns <= 2e9), then takes the path of a
 * bounded wait that ran out -- it records the timeout in the device status
 * word, waits for its own copies in flight and returns without writing its
 * points.  esom_device_status then returns ESOM_EDEVICE; the handle and the
 * context stay usable.  One launch consumes the probe.
 * Errors: ESOM_EINVAL (null handle, limit out of range, plan not fused).
 *
 * esom_selftest_drcp: for i < n, rcp[i] = the FP64 reciprocal the 2x2 solve
 * of esom_project uses (Section 3.1 step 4: Cramer's rule divides by the
 * determinant; here an SFU approximation refined by two Newton steps) and
 * div[i] = 1.0 / x[i] by CUDA's division, on `stream`.  x, rcp and div are
 * device pointers to n doubles.  Errors: ESOM_EINVAL, ESOM_ECUDA. */
esom_status esom_test_stall(esom_handle h, int64_t limit_ns);

/* esom_selftest_tc_products: the raw tensor-core values behind the screened
 * k-NN (Section 4.2: the distance block; here a tcgen05 contraction of split
 * TF32 or BF16 operands with FP32 accumulation), for tests of its error
 * bound.  Needs tensor-core screening on (esom_set_screening).  For each of
 * the n points (n <= 2^20; device, as for esom_project) writes
 * T[i * Lc + j] = the accumulated x_i . L_j for j < Lc = 64 ceil(L / 64)
 * (landmarks beyond L are zero rows) to T (device, n * Lc floats, 16-byte
 * aligned).  Errors: ESOM_EINVAL, ESOM_EALIGN, ESOM_ENOLANDMARKS,
 * ESOM_EUNSUPPORTED, ESOM_ECUDA. */
esom_status esom_selftest_tc_products(esom_handle h, const float *points, int64_t n, float *T,
                                      esom_stream_t stream);
esom_status esom_selftest_drcp(const double *x, int64_t n, double *rcp, double *div,
                               esom_stream_t stream);

/* Releases the handle's device buffers.  Pending work on streams that use
 * the handle must have completed. NULL is accepted. */
esom_status esom_destroy(esom_handle h);

/* Message of the last non-OK status returned on this host thread. */
const char *esom_last_error(void);

/* Constant name of a status code. */
const char *esom_status_string(esom_status s);

#ifdef __cplusplus
}
#endif

#endif /* ESOM_H */
