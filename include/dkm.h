/*
 * dkm.h -- C ABI of libdkm: GB300-native indexed k-means (Lloyd's algorithm
 * with index-based batch pruning) for 2D / 3D float32 points.
 *
 * Method: Dask-means, arXiv 2412.02244.
 *   - Eq. 1 / Section II-A: k-means minimises the sum of squared errors
 *     (SSE); Lloyd's algorithm alternates assignment (nearest centroid) and
 *     update (cluster mean).
 *   - Section II-B: index-based acceleration returns exactly Lloyd's result.
 *   - Section IV-A ("Pruning Mechanisms", Eq. for the ball-node test, the
 *     two-nearest gap test and the kNN bounds inherited from parent nodes):
 *     a group of spatially close points is assigned in batch after pruning
 *     centroids with distance bounds; here the groups are Morton-ordered
 *     tiles with axis-aligned bounding boxes and the centroid index is a
 *     uniform grid rebuilt every iteration.
 *   - Section V-A (memory-tunable index, Eq. for f under a memory budget):
 *     the centroid grid's cell size grows until the index fits
 *     dkm_options.mem_budget_bytes.
 *   - Algorithm 1: the outer loop (build the centroid index, assign, refine
 *     c_j = sv(j)/|S_j|) is dkm_run / dkm_fit.
 *
 * Conventions (every function):
 *   - Array arguments may be device pointers (cudaMalloc / torch CUDA
 *     tensors) or host pointers (pageable or pinned); the library detects
 *     which with cudaPointerGetAttributes and copies host data through its
 *     own device buffers.  The caller owns every array it passes.
 *   - Points are row-major n x d float32 (d = 2 or 3); centroids are
 *     row-major k x d float32; labels are int32 in [0, k), in the caller's
 *     original point order.
 *   - Work is enqueued on dkm_options.stream (a cudaStream_t; NULL = the
 *     legacy default stream).  Each call returns after its host-visible
 *     outputs (sse, iterations, changed) are written; device outputs are
 *     ready in stream order.
 *   - No exception crosses the ABI.  Every function returns a dkm_status;
 *     dkm_last_error() gives the message of the calling thread's last
 *     failure.
 *   - Ties go to the lowest centroid index; an empty cluster keeps its
 *     previous centroid.
 */
#ifndef DKM_H_
#define DKM_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DKM_API __attribute__((visibility("default")))
#else
#define DKM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DKM_OK = 0,
    DKM_EINVAL = 1,     /* bad argument, non-finite input, label out of range */
    DKM_ENOMEM = 2,     /* device allocation failed, or the index cannot fit the budget */
    DKM_ECUDA = 3,      /* a CUDA runtime call failed (message in dkm_last_error) */
    DKM_ETIMEOUT = 4,   /* a bounded device-side wait gave up */
    DKM_EINTERNAL = 5   /* an internal consistency check failed */
} dkm_status;

enum {
    DKM_ALGO_INDEXED = 0,   /* Morton tiles + centroid grid pruning (the method) */
    DKM_ALGO_BRUTE = 1      /* plain Lloyd: every point against every centroid */
};

typedef struct {
    /* Cap, in bytes, on the per-iteration centroid index (the grid's cell
     * counters and buckets, both parities).  The planner coarsens the grid
     * until it fits, like the paper's memory-tunable leaf capacity.
     * 0 = default (64 MiB). */
    size_t mem_budget_bytes;
    /* Target grid cells per centroid before the budget cap (default 1.0). */
    float cells_per_centroid;
    /* DKM_ALGO_INDEXED (default) or DKM_ALGO_BRUTE. */
    int algo;
    /* dkm_run / dkm_fit: 1 = stop after the first assignment pass that
     * changes no label (default); 0 = always run max_iter passes. */
    int early_stop;
    /* Per-kernel CUDA events, read back by dkm_last_timings: 0 = off;
     * 1 = around the kernels of every fifth pass (every pass of a run of up
     * to five); n >= 2 = one pass in each n (the middle one of each n; the
     * middle pass of a run shorter than n).  Each profiled pass costs a run
     * some launch overlap (tens of us). */
    int profile;
    /* cudaStream_t to enqueue on; NULL = legacy default stream. */
    void* stream;
} dkm_options;

/* Grid plan for a point set (host-only arithmetic, no GPU needed). */
typedef struct {
    int dims[3];            /* cells per axis (dims[2] = 1 when d = 2) */
    float cell;             /* cell edge length */
    float origin[3];        /* low corner of the grid */
    int bucket_cap;         /* centroid slots per cell before the overflow list */
    int64_t cells;          /* dims[0]*dims[1]*dims[2] */
    size_t index_bytes;     /* bytes of the per-iteration centroid index */
    size_t scratch_bytes;   /* all device scratch a context of this size owns */
} dkm_plan_info;

typedef struct {
    float setup_ms;         /* last dkm_setup: bbox, Morton sort, tile boxes */
    float iterations_ms;    /* last dkm_run: all passes (graph launch) */
    float search_ms;        /* mean per profiled pass: candidate search */
    float assign_ms;        /* mean per profiled pass: assignment + accumulation kernel */
    float update_ms;        /* mean per profiled pass: centroid update + grid rebuild */
    float finalize_ms;      /* last dkm_run: label un-permute + final SSE */
    int passes;             /* profiled passes the means cover (opts.profile) */
} dkm_timings;

typedef struct {
    double evals_per_point;     /* candidate distance evaluations per point, last pass */
    double candidates_per_tile; /* mean tile candidate-list length, last pass */
    int64_t fallback_tiles;     /* tiles whose candidate list overflowed, last pass */
    int64_t stayed_tiles;       /* tiles that passed the stay test, last pass */
    int64_t grid_overflow;      /* centroids placed in the overflow list, last rebuild */
    int64_t tiles;              /* tiles of the point index (<= 256 points each) */
    int tile_level;             /* Morton level whose cubes bound the tiles */
    int passes;                 /* assignment passes of the last dkm_run */
    int64_t stayed_points;      /* points that passed the point stay test, last pass */
} dkm_stats;

typedef struct dkm_ctx dkm_ctx;

/* Fill *opts with the defaults above. */
DKM_API void dkm_default_options(dkm_options* opts);

/* Static string for a status code. */
DKM_API const char* dkm_status_string(dkm_status s);

/* Message of the calling thread's last failing call ("" if none). */
DKM_API const char* dkm_last_error(void);

/*
 * Plan the centroid grid for n points of dimension d with bounding box
 * [bbox_lo, bbox_hi] (d floats each) and k centroids, under opts'
 * memory budget (Section V-A analog).  Pure host arithmetic.
 * DKM_EINVAL on bad sizes; DKM_ENOMEM if even a single cell exceeds the
 * budget.
 */
DKM_API dkm_status dkm_plan(int64_t n, int d, int k, const float* bbox_lo, const float* bbox_hi,
                    const dkm_options* opts, dkm_plan_info* out);

/*
 * Create a context for n points of dimension d and k clusters, allocate
 * its device scratch and build the point index (dkm_setup) from points
 * (n x d).  The library keeps its own sorted copy; the caller may free
 * points afterwards.  opts may be NULL (defaults).
 * Errors: DKM_EINVAL (d not 2/3, n < 1, k < 1, k > n, null pointer,
 * non-finite point), DKM_ENOMEM, DKM_ECUDA, DKM_ETIMEOUT (as dkm_setup).
 * On error *out is NULL.
 */
DKM_API dkm_status dkm_create(dkm_ctx** out, const float* points, int64_t n, int d, int k,
                      const dkm_options* opts);

/*
 * Rebuild the point index (bounding box, Morton sort into tiles, tile
 * boxes -- the analog of building the spatial-vector Ball-tree once,
 * Algorithm 1 first step) for a new set of n x d points of the context's
 * size.  Errors: DKM_EINVAL (null, non-finite), DKM_ECUDA, DKM_ETIMEOUT
 * (a radix-sort pass waits, with a bounded number of polls, for the
 * digit counts of the CTAs before it; it gave up -- the context then needs
 * a new dkm_setup).
 */
DKM_API dkm_status dkm_setup(dkm_ctx* ctx, const float* points);

/*
 * One assignment pass (Section II-A assignment step, pruned as in Section
 * IV-A): labels[i] = index of the nearest of the k x d centroids.
 * labels (n, original order) may be NULL.  sse_out (nullable) receives
 * sum_i min_j ||p_i - c_j||^2 for these centroids.  changed_out (nullable)
 * receives how many labels differ from this context's previous pass (all n
 * on the first).  The per-cluster sums of this pass are kept for
 * dkm_update(ctx, NULL, ...).
 */
DKM_API dkm_status dkm_assign(dkm_ctx* ctx, const float* centroids, int32_t* labels,
                      double* sse_out, int64_t* changed_out);

/*
 * One update step (Algorithm 1 refine: c_j = mean of the points labelled
 * j; an empty cluster keeps its centroid).  labels (n, original order):
 * the labelling to average; NULL = the labels of the last dkm_assign on
 * this context, whose sums are reused.  centroids_inout (k x d): the
 * previous centroids on entry, the new ones on return.  counts (k,
 * nullable) receives the cluster sizes.  DKM_EINVAL if a label is out of
 * range (centroids_inout is then left unchanged) or if labels is NULL
 * before any dkm_assign.
 */
DKM_API dkm_status dkm_update(dkm_ctx* ctx, const int32_t* labels, float* centroids_inout,
                      int32_t* counts);

/*
 * Lloyd's loop on the context's points (Algorithm 1): up to max_iter
 * passes of assignment + update, starting from init_centroids (k x d).
 * With opts.early_stop the loop ends after the first pass that changes no
 * label.  iterations_out = passes executed.  centroids_out (k x d) = the
 * centroids after the last update; labels_out (n) = the last pass's
 * labels; sse_out = SSE of those labels against centroids_out.
 * max_iter = 0 labels the points against init_centroids (no update) and
 * returns them unchanged.  Outputs other than iterations_out may be NULL.
 */
DKM_API dkm_status dkm_run(dkm_ctx* ctx, const float* init_centroids, int max_iter,
                   float* centroids_out, int32_t* labels_out, int* iterations_out,
                   double* sse_out);

/*
 * One-shot k-means: dkm_create + dkm_run + dkm_destroy.  opts may be NULL.
 * The run's kernels are launched directly on the stream (a context's
 * dkm_run captures them into a CUDA graph that later runs relaunch); the
 * results are the same bit for bit.
 */
DKM_API dkm_status dkm_fit(const float* points, int64_t n, int d, int k, const float* init_centroids,
                   int max_iter, float* centroids_out, int32_t* labels_out,
                   int* iterations_out, double* sse_out, const dkm_options* opts);

/*
 * Batched contexts: B independent k-means problems ("clouds") in one
 * context, run together -- every kernel of a pass covers the tiles of all
 * clouds, so a pass is one launch per kernel whatever B is, and the whole
 * loop is one CUDA graph.  Each cloud has its own point index (Morton
 * order and tiles on its own bounding box), its own centroid grid (cells
 * ~ cells_per_centroid * k_b, all clouds' grids together under
 * mem_budget_bytes), its own fixed-point scale and its own early stop.
 * The paper runs one problem at a time; a batch of B clouds gives exactly
 * the B results of B separate runs.
 *
 * points: concatenated clouds, n_total x d (host or device);
 * offsets: B + 1 int64 (host or device), offsets[0] = 0, cloud b =
 *   rows offsets[b] .. offsets[b+1] - 1, every cloud non-empty;
 * ks: B int32 (host or device), 1 <= ks[b] <= points of cloud b;
 * centroid arrays (init, output): sum(ks) x d, cloud after cloud;
 * labels: n_total int32, cloud-local centroid index (0 .. ks[b] - 1);
 * iterations_out (B int32) and sse_out (B double), host or device,
 *   nullable: passes executed and final SSE of each cloud.
 * 1 <= B <= 65535.  For B > 1 the sort key keeps the cloud index in its top
 * ceil(log2 B) bits, so each cloud's Morton code gets fewer bits per axis
 * (7 in 3D at B = 512); the results do not depend on it.
 * The single-cloud functions accept batched contexts too: dkm_assign
 * returns the total SSE and change count, dkm_run the largest pass count
 * and the total SSE, dkm_get_plan cloud 0's grid with the total cell count.
 * Errors as dkm_create / dkm_run, plus DKM_EINVAL for bad offsets or ks.
 */
DKM_API dkm_status dkm_create_batched(dkm_ctx** out, const float* points, const int64_t* offsets,
                                      int B, int d, const int32_t* ks, const dkm_options* opts);
DKM_API dkm_status dkm_run_batched(dkm_ctx* ctx, const float* init_centroids, int max_iter,
                                   float* centroids_out, int32_t* labels_out,
                                   int32_t* iterations_out, double* sse_out);
DKM_API dkm_status dkm_fit_batched(const float* points, const int64_t* offsets, int B, int d,
                                   const int32_t* ks, const float* init_centroids, int max_iter,
                                   float* centroids_out, int32_t* labels_out,
                                   int32_t* iterations_out, double* sse_out,
                                   const dkm_options* opts);

/*
 * Index tuning of a context.  None of these settings changes which centroid
 * is nearest to a point (the labels of a given centroid set are exact
 * whatever the index); they change how much work the pruning does.  The
 * tile cut also regroups the per-tile fixed-point sums of the update, so
 * centroids computed under different cuts may differ in their last bits
 * (far inside the update's error bound).  The paper fits a cost model for
 * its memory/leaf-capacity choice (Section V-A); here the choice is
 * measured instead.
 */
typedef struct {
    /* grid cells per centroid before the memory-budget cap, in
     * (0, max(4, opts.cells_per_centroid)] */
    float cells_per_centroid;
    /* a cloud's tiles are cut at the finest Morton cubes that add at most
     * its 256-point windows / tile_cut_div tiles; 1 .. 1024 (default 2) */
    int tile_cut_div;
    /* tile candidate lists longer than this are filtered again per row of
     * 64 points (default 48; >= 256 turns the row filter off) */
    int row_filter_min;
    /* candidate lists up to this length (0 .. 32) are sorted by their box
     * lower bound and evaluated with an early exit once the bound exceeds
     * every point's current best (the kNN pruning rule); default 0 (off) */
    int sort_max;
    /* hierarchical tiles: groups of this many consecutive tiles of a cloud
     * share one candidate search over the union of their boxes, and each
     * tile narrows the group's list with its own box; 1 .. 32, default 1
     * (every tile searches on its own) */
    int tile_group;
    /* the bound layer (Section IV-A): 1 = before searching, a tile whose
     * points all had label a in the last pass keeps a for every point when
     * its box lies within half the distance from c_a to the nearest other
     * centroid (maxd(box, c_a) < cb[a] / 2, Eq. interbound; cb from a grid
     * kNN(2) over the centroids after each update, started inside a run
     * from the bound ub = cb[j] + Delta[j] + max(Delta) of Eq. ub); such a
     * tile skips the grid search.  2 = also the point test of Eq.
     * interbound1 in the assignment: a point within cb[a] / 2 of its last
     * centroid keeps it, and a row of 64 points that all keep theirs skips
     * the candidate evaluation.  Only with tile_group = 1; default 0 */
    int stay_test;
    /* dkm_autotune only: mean ms per Lloyd pass of the chosen setting and
     * of the setting the context had before, configurations timed, and
     * whether the choice came from the process-wide cache (nothing timed) */
    float ms_per_pass;
    float ms_per_pass_before;
    int trials;
    int from_cache;
} dkm_tuning;

/* Current setting of a context (timing fields 0). */
DKM_API dkm_status dkm_get_tuning(const dkm_ctx* ctx, dkm_tuning* out);

/* Apply a setting (the timing fields are ignored); re-plans the grids and
 * re-cuts the tiles as needed.  DKM_EINVAL for values out of range. */
DKM_API dkm_status dkm_set_tuning(dkm_ctx* ctx, const dkm_tuning* tuning);

/*
 * Measure and apply the fastest setting for this context: coordinate
 * descent over cells_per_centroid {0.5, 1, 2, 4}, tile_cut_div
 * {1, 2, 4, 8, 16, 32}, row_filter_min {16, 32, 48, 96, 256}, sort_max
 * {0, 16, 32}, tile_group {1, 2, 4, 8, 16} and stay_test {0, 1, 2}, each
 * setting timed (CUDA events, best of two) over `passes` Lloyd passes
 * (1 .. 64, no early stop) from init_centroids.  The context's labels and
 * centroids are overwritten by those runs.  With use_cache = 1 a setting
 * found before in this process for the same workload shape (d, number of
 * clouds, and the rounded log2 of the mean points and centroids per cloud)
 * is applied without timing.  out (nullable) receives the choice.
 */
DKM_API dkm_status dkm_autotune(dkm_ctx* ctx, const float* init_centroids, int passes,
                                int use_cache, dkm_tuning* out);

/* Device bytes the context owns, and how many of them are the per-iteration
 * centroid index.  Either pointer may be NULL. */
DKM_API dkm_status dkm_query_memory(const dkm_ctx* ctx, size_t* device_bytes, size_t* index_bytes);

/* Plan the context was built with. */
DKM_API dkm_status dkm_get_plan(const dkm_ctx* ctx, dkm_plan_info* out);

/* Timings of the last dkm_setup / dkm_run (needs opts.profile; otherwise
 * 0).  CUDA events are recorded around the kernels of the profiled passes
 * only (opts.profile), so profiling adds few graph nodes; the setup time is
 * read out here (this call may wait for the last dkm_setup to finish). */
DKM_API dkm_status dkm_last_timings(dkm_ctx* ctx, dkm_timings* out);

/* Pruning counters of the last pass (reads device counters; synchronises
 * the context's stream). */
DKM_API dkm_status dkm_last_stats(dkm_ctx* ctx, dkm_stats* out);

/* Free the context and its device memory.  NULL is a no-op. */
DKM_API void dkm_destroy(dkm_ctx* ctx);

/*
 * Differentiable losses of a batch of B point clouds (the differentiable
 * extension of Eq. 1).  Cloud b holds points[offsets[b] .. offsets[b+1])
 * (rows of the n_total x d array points); every cloud has k centroids
 * (1 <= k <= 1024), stored cloud after cloud as B x k x d arrays.
 * points, init_centroids, ckpt and the gradient arrays are device
 * pointers; offsets (B + 1, offsets[0] = 0, every cloud non-empty), tau (B),
 * loss (B) and dloss (B) may be host or device pointers.  Work runs on
 * stream (a cudaStream_t; NULL = legacy default stream); each call returns
 * after its outputs are written.  Scratch comes from the stream-ordered
 * allocator (cudaMallocAsync) and is released before returning.
 *
 * Soft k-means with T unrolled steps at a fixed temperature tau[b]:
 *   w^t_ij = softmax_j(-||p_i - c^t_j||^2 / tau),
 *   c^{t+1}_j = sum_i w^t_ij p_i / sum_i w^t_ij   (a centroid whose weights
 *     all underflow to zero in FP32 keeps its position, and the backward
 *     passes the gradient of c^{t+1}_j on to c^t_j unchanged),
 *   loss[b] = sum_ij w^T_ij ||p_i - c^T_j||^2.
 * dkm_soft_forward writes the centroids of every step into ckpt
 * (B x (T+1) x k x d, step-major: ckpt[t] is B x k x d) and the loss.
 * Optionally (both device pointers, nullable) it also keeps per step the
 * two softmax statistics of every point, stats (T x 2 x n_total floats:
 * min_j ||p_i - c^t_j||^2, then 1 / the softmax normaliser), and the
 * weight sums of every centroid, norms (T x B x k floats) -- O(n) per step,
 * not the n x k weights.
 * dkm_soft_backward takes the checkpoints and the upstream gradient
 * dloss[b] = dOut/dloss[b] and writes dOut/dpoints (n_total x d) and
 * dOut/dinit_centroids (B x k x d), recomputing the weights of each step
 * from ckpt instead of storing them; given the forward's stats and norms
 * (both, else neither) it skips recomputing them, with the same result
 * bit for bit.  tau is a constant of the loss.
 * Errors: DKM_EINVAL (sizes, offsets, null pointers), DKM_ECUDA.
 */
DKM_API dkm_status dkm_soft_forward(const float* points, const int64_t* offsets, int B, int d,
                                    int k, const float* init_centroids, int T, const float* tau,
                                    float* ckpt, double* loss, float* stats, float* norms,
                                    void* stream);
DKM_API dkm_status dkm_soft_backward(const float* points, const int64_t* offsets, int B, int d,
                                     int k, const float* ckpt, int T, const float* tau,
                                     const double* dloss, const float* stats, const float* norms,
                                     float* grad_points, float* grad_init, void* stream);

/*
 * Hard SSE of each cloud, Eq. 1 with the nearest centroid (lowest index on
 * ties): loss[b] = sum_i min_j ||p_i - c_j||^2, with optional labels (n_total,
 * cloud-local centroid index), dloss/dpoints = 2 (p_i - c_a(i)) and
 * dloss/dcentroids_j = -2 sum_{a(i)=j} (p_i - c_j).  Same layout and pointer
 * rules as dkm_soft_forward; labels, loss and both gradients may be NULL.
 */
DKM_API dkm_status dkm_hard_sse(const float* points, const int64_t* offsets, int B, int d, int k,
                                const float* centroids, int32_t* labels, double* loss,
                                float* grad_points, float* grad_centroids, void* stream);

/*
 * Backward of the hard SSE for an upstream gradient dloss[b] = dOut/dloss[b]
 * (B doubles, host or device): given the labels the forward returned
 * (n_total int32, cloud-local, device), writes
 *   grad_points[i]     = dloss[b] * 2 (p_i - c_a(i)),
 *   grad_centroids[j]  = dloss[b] * -2 sum_{a(i)=j} (p_i - c_j),
 * either of them nullable.  Same layout and pointer rules as
 * dkm_soft_forward.  Errors: DKM_EINVAL (sizes, null pointers, a label
 * outside [0, k): the gradient rows of such points are 0), DKM_ECUDA.
 */
DKM_API dkm_status dkm_hard_sse_backward(const float* points, const int64_t* offsets, int B,
                                         int d, int k, const float* centroids,
                                         const int32_t* labels, const double* dloss,
                                         float* grad_points, float* grad_centroids,
                                         void* stream);

/*
 * Temperature of the soft loss per cloud: tau[b] = frac * ||hi_b - lo_b||^2,
 * the squared diagonal of cloud b's bounding box (FP32 box corners, FP64
 * sum of squares, rounded to FP32).  The default of the differentiable
 * workload is frac = 0.01.  points (device), offsets and tau (B floats)
 * host or device.  Errors: DKM_EINVAL (sizes, offsets, null pointers,
 * frac <= 0), DKM_ECUDA.
 */
DKM_API dkm_status dkm_soft_temperature(const float* points, const int64_t* offsets, int B, int d,
                                        double frac, float* tau, void* stream);

/* Largest k dkm_lloyd_step_noalloc accepts (its fixed scratch holds k
 * cluster accumulators of 32 bytes each, about 2 MiB in all). */
#define DKM_NOALLOC_MAX_K 65536

/*
 * One Lloyd step (brute-force assignment of every point, then the update)
 * that allocates no device memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code that
 * runs inside a host framework which owns all device memory through its
 * own allocator, or a latency-critical loop where cudaMalloc / cudaFree
 * would synchronise the device.
 *
 * points (n x d), centroids (k x d): device pointers, read.
 * centroids_out (k x d): device pointer, written with the cluster means
 *   (an empty cluster keeps its centroid); must not alias centroids.
 * labels (n): device pointer, written, nearest centroid of each point
 *   (ties to the lowest index), in input order.
 * sse_out (nullable): host pointer, receives the SSE of the labels against
 *   the input centroids; the call then waits for the stream.
 * stream: cudaStream_t (NULL = legacy default stream).
 *
 * Scratch: one fixed device array inside the library (per-cluster sums for
 * up to DKM_NOALLOC_MAX_K clusters, SSE counters, a bounding box).  Every
 * GPU that loads the library holds it until the process exits.  The first
 * call on a device looks up that array's device address on the current
 * device (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Each call clears what must start at zero.  All calls share the
 * one array, so calls that overlap on the GPU (other streams, other host
 * threads) race; serialise them.
 * A NaN or infinite coordinate in points or centroids is detected on the
 * GPU: every label is then set to -1, centroids_out receives centroids
 * unchanged, and the SSE is NaN.  With sse_out the call reads that result
 * back and returns DKM_EINVAL; without it the call returns before the GPU
 * has looked at the data, so the caller must check the labels.
 * Errors: DKM_EINVAL (d not 2/3, n < 1, k < 1 or k > DKM_NOALLOC_MAX_K,
 * null pointer) before any GPU work, or non-finite input (with sse_out);
 * DKM_ECUDA.
 */
DKM_API dkm_status dkm_lloyd_step_noalloc(const float* points, int64_t n, int d, int k,
                                          const float* centroids, float* centroids_out,
                                          int32_t* labels, double* sse_out, void* stream);

/*
 * Device peaks for roofline reporting (no counterpart in the paper).  The
 * brute-force assignment and the soft k-means passes are bound by FP32
 * arithmetic, not by memory; their achieved rate is reported against the
 * FP32 FMA throughput measured here: FMA-chain kernels (eight independent
 * chains per thread, eight 256-thread CTAs per SM), scalar fmaf and packed
 * f32x2, each timed with CUDA events after a warm-up launch.  An FMA counts
 * as two floating-point operations.  Runs on the current device and
 * stream (NULL = legacy default); allocates a small output buffer with the
 * stream-ordered allocator.  Errors: DKM_EINVAL (null out), DKM_ECUDA.
 */
typedef struct {
    int sm_count;               /* multiprocessors of the current device */
    int sm_clock_mhz;           /* its rated maximum SM clock */
    double fp32_fma_tflops;     /* measured, scalar FFMA */
    double fp32x2_fma_tflops;   /* measured, packed f32x2 FFMA */
    float scalar_ms;            /* duration of the timed scalar launch */
    float packed_ms;            /* duration of the timed packed launch */
} dkm_peaks;

DKM_API dkm_status dkm_device_peaks(dkm_peaks* out, void* stream);

/*
 * Self-test of the library's one device-side wait: the radix sort of
 * dkm_setup, whose CTAs wait (decoupled look-back) for the digit counts of
 * the CTAs before them.  Runs one sort pass on 8,192 keys whose only CTA
 * is handed the second tile, so the count it waits for is never published:
 * the wait must give up by itself (after about a second) and report it.
 * The points are then gathered by the partly written order, as dkm_setup
 * does before it reads the error flag; the slots the pass never wrote hold
 * out-of-range indices, which the gather must clamp.
 * Allocates and frees its own small device buffers on a private stream.
 * seconds_out (nullable, host): the wall time of the pass.
 * Returns DKM_OK if the wait ended and was reported; DKM_EINTERNAL if the
 * pass ended without reporting; DKM_ECUDA.
 */
DKM_API dkm_status dkm_selftest_wait(double* seconds_out);

#ifdef __cplusplus
}
#endif

#endif /* DKM_H_ */
