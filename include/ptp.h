/*
 * ptp.h -- C ABI of the GB300 (sm_103a) Parallel Toplesets Propagation
 * library: approximate geodesic distance maps on triangle meshes
 * (Romero Calla, Fuentes Perez, Montenegro, "A minimalistic approach for
 * fast computation of geodesic distances on triangular meshes").
 *
 * Problem (Sec. 3.1, "Discrete distance maps"): given a triangle mesh
 * T = (V, E, F) and a source set S subset of V, compute d_S : V -> R, the
 * geodesic distance from every vertex to S.
 *
 * Pipeline, one call per stage:
 *   ptp_mesh_create   vertices + faces -> device mesh with the
 *                     vertex -> incident-triangle lists;
 *   ptp_toplesets     sources -> toplesets V_r (breadth-first levels,
 *                     Sec. 4.1 Definition) and the mesh renumbered in
 *                     topleset order (Sec. 4.3);
 *   ptp_distance      the PTP iteration over the sliding update band
 *                     (Sec. 4.2, Eq. lower_band / upper_band) into a
 *                     caller-owned device buffer in the ORIGINAL vertex order.
 *   ptp_geodesic      all three stages in one call (host or device buffers).
 *
 * Conventions shared by every entry point:
 *  - Every function returns a ptp_status; PTP_OK is 0.
 *  - Streams: `stream` is a cudaStream_t passed as an opaque pointer
 *    (NULL = the legacy default stream).  Work is enqueued on it; a function
 *    only blocks where its comment says so.
 *  - Pointers: `ptr_kind` says whether array arguments are host memory
 *    (PTP_HOST) or device memory of the current device (PTP_DEVICE).  Inputs
 *    are copied; the caller keeps ownership of every buffer it passes.
 *  - Handles are opaque, own their device memory (stream-ordered
 *    allocations on the creating stream) and are released by the matching
 *    *_destroy.  A handle may be used from one host thread at a time.
 *  - Indices are 0-based int32; vertex positions are float32 xyz triples.
 */
#ifndef PTP_H
#define PTP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ptp_status {
    PTP_OK = 0,
    PTP_ERR_ARG = 1,             /* null pointer, bad size or bad parameter        */
    PTP_ERR_INDEX = 2,           /* a face or source index is out of range         */
    PTP_ERR_DEGENERATE_FACE = 3, /* a face repeats a vertex                         */
    PTP_ERR_CUDA = 4,            /* a CUDA runtime call failed                      */
    PTP_ERR_NOT_CONVERGED = 5,   /* max_iter reached; the distances are written     */
    PTP_ERR_TIMEOUT = 6,         /* a device-side wait hit its limit; kernel exited */
    PTP_ERR_NOMEM = 7,           /* device allocation failed                        */
    PTP_ERR_TOO_LARGE = 8        /* a size exceeds this entry point's limit         */
} ptp_status;

enum { PTP_HOST = 0, PTP_DEVICE = 1 };

typedef struct ptp_mesh ptp_mesh;
typedef struct ptp_toplesets_s ptp_toplesets_t;
typedef struct ptp_batch_s ptp_batch_t;

/* Parameters of ptp_distance.  Fill with ptp_params_default first. */
typedef struct ptp_params {
    double eps;        /* relative-change threshold of Eq. lower_band (Sec. 4.2);
                          the paper uses 1e-3 in all experiments                   */
    double eps_abs;    /* absolute slack: a vertex of V_{i_{k-1}} passes when
                          |d_k - d_{k-1}| < eps * d_{k-1} + eps_abs or the change
                          is exactly 0 (paper: eps_abs = 0)                        */
    int64_t max_iter;  /* iteration cap; 0 = 8 * rho + 64                          */
    int32_t block;     /* threads per CTA of the window kernel: 0 = 512, else a
                          multiple of 32 in [64, 512] (see ptp_autotune)        */
    int32_t grid;      /* CTAs of the window kernel; 0 = all co-resident CTAs      */
    int32_t band_mode; /* 0: the paper's dynamic band (Eq. lower_band); 1: the
                          fixed band of the complexity analysis (Sec. 6.1), lower
                          bound ceil(k / 2), no convergence test; 2: the learned
                          multi-advance band (an extension; the paper has no
                          counterpart): the bottom topleset is tested as in
                          Eq. lower_band and, besides it, the toplesets above it
                          that the learned schedule marks due are tested as one
                          group; when both pass, the lower bound moves past all
                          of them at once instead of by one.  A wrong prediction
                          costs iterations, never the test.  Meant for fixpoint
                          runs (a small eps such as 1e-7), where the result
                          equals the dynamic band's within rounding.  Needs
                          `schedule` (ptp_distance) or `mlp_half`
                          (ptp_distance_from_sources); single-source entry points
                          only                                                      */
    int32_t reserved;  /* must be 0                                                */
    void *trace;       /* optional DEVICE buffer of trace_cap ptp_trace_rec, one per
                          iteration, or NULL                                       */
    int64_t trace_cap;
    void *ev_begin;    /* optional cudaEvent_t recorded on `stream` right before the
                          window kernel, or NULL                                   */
    void *ev_end;      /* optional cudaEvent_t recorded right after it, or NULL     */
    const int32_t *schedule; /* optional DEVICE array [rho] from ptp_mlp_infer.
                          band_mode 0: for each topleset i, the number of
                          iterations the band's lower bound is expected to stay
                          at i; the test of Eq. lower_band is skipped until that
                          many iterations have passed, then applied as usual
                          every iteration (NULL: test every iteration).
                          band_mode 2: for each topleset r, the iterations after
                          it enters the band (at iteration r) until it is
                          expected to have converged; r joins the tested group
                          from iteration r + max(schedule[r], 1) on            */
    const void *mlp_half;   /* band_mode 2 in ptp_distance_from_sources: DEVICE
                          array of PTP_MLP_NPARAM FP16 weights of the schedule
                          MLP.  The launch computes each topleset's window
                          features while it copies it into topleset order and
                          infers its schedule before the iteration reaches it,
                          with the same arithmetic as ptp_window_features +
                          ptp_mlp_infer, so the two paths run the same
                          iteration                                             */
    float mlp_margin;       /* margin of that inference (see ptp_mlp_infer)       */
    int32_t reserved2;      /* must be 0                                           */
    int32_t *conv_trace;    /* optional DEVICE array [rho] (ptp_distance only),
                          filled with -1 by the caller: for each topleset, the
                          last iteration in which one of its vertices failed
                          the relative-change test (the schedule MLP's training
                          target)                                               */
} ptp_params;

/* One record per PTP iteration k (written only when params.trace is set). */
typedef struct ptp_trace_rec {
    int32_t i;         /* lower band bound used at iteration k, i_{k-1}            */
    int32_t j;         /* upper band bound j_k (Eq. upper_band)                    */
    int32_t active;    /* band vertices recomputed (some neighbour changed)        */
    int32_t changed;   /* band vertices whose distance changed                     */
    float maxrel;      /* max relative change over V_{i_{k-1}}                     */
    int32_t advanced;  /* i_k - i_{k-1}: 1 if Eq. lower_band advanced the band,
                          more when band_mode 2 retired a tested group          */
    double errsum;     /* FP64 sum of relative changes over V_{i_{k-1}}            */
} ptp_trace_rec;

typedef struct ptp_stats {
    int64_t iterations;      /* K, iterations run                                   */
    int64_t band_updates;    /* sum over k of |B_k minus S| (the paper's work count) */
    int64_t active_updates;  /* vertex updates actually recomputed                  */
    int64_t changed;         /* vertex updates that lowered the distance            */
    int64_t fp64_solves;     /* triangle solves taken in FP64 (near-degenerate)     */
    int32_t rho;             /* number of toplesets                                 */
    int32_t status;          /* ptp_status of the device-side run                   */
    int64_t checks;          /* iterations that applied the test of Eq. lower_band  */
} ptp_stats;

/* Human-readable name of a status code (static storage). */
const char *ptp_status_str(ptp_status s);

/* Defaults: eps = 1e-3 and eps_abs = 0 (Sec. 4.2, the paper's setting),
 * max_iter = 0 (auto), block = grid = 0 (auto), band_mode = 0, no trace, no
 * events. */
ptp_status ptp_params_default(ptp_params *p);

/* Number of CUDA kernel launches this library has issued in this process
 * (all devices, all entry points).  Never blocks. */
int64_t ptp_kernel_launches(void);

/* Return to the driver the device memory the library keeps for reuse.
 * Every buffer the library allocates comes from its own stream-ordered
 * memory pool per device, which keeps freed memory mapped so that the next
 * call does not map it again; this trims those pools to what is still in
 * use (nothing, once every handle is destroyed and its stream has
 * finished).  Never blocks on a stream; PTP_ERR_CUDA on a CUDA error. */
ptp_status ptp_release_memory(void);

/*
 * Build the device mesh (Sec. 3.1, T = (V, E, F); Sec. 4.3 stores it as a
 * compact half-edge structure, here as vertex -> incident-triangle lists).
 *  xyz    [n_verts * 3] float32, row-major vertex positions.
 *  faces  [n_faces * 3] int32, 0-based, either orientation.
 *  Validates every face: PTP_ERR_INDEX (index outside [0, n_verts)),
 *  PTP_ERR_DEGENERATE_FACE (a face repeats a vertex), PTP_ERR_ARG
 *  (null pointer, n_verts < 3, n_faces < 1, or more than 2^31 - 1 corners).
 *  Blocks until validation has finished on `stream`.
 */
ptp_status ptp_mesh_create(const float *xyz, int64_t n_verts, const int32_t *faces, int64_t n_faces,
                           int ptr_kind, void *stream, ptp_mesh **out);

/* Bounding-box diagonal of the vertices (the "mesh diameter" used for error
 * tolerances), vertex and face counts.  Any output pointer may be NULL. */
ptp_status ptp_mesh_info(const ptp_mesh *mesh, int64_t *n_verts, int64_t *n_faces, double *diameter);

/* Release the mesh.  Destroy every ptp_toplesets_t made from it first. */
ptp_status ptp_mesh_destroy(ptp_mesh *mesh);

/*
 * Toplesets from the source set S (Sec. 4.1, Definition: V_0 = S and V_r the
 * not yet visited neighbours of V_{r-1}), computed by a breadth-first search
 * on the device, and the mesh renumbered so that V_0, V_1, ... occupy
 * consecutive index ranges (Sec. 4.3, reordering for coalesced access).
 *  sources  [m] int32 vertex indices, m >= 1; duplicates are allowed.
 *  PTP_ERR_INDEX if a source is outside [0, n_verts); PTP_ERR_ARG if m < 1.
 *  Vertices not reachable from S are placed after the last topleset and get
 *  +inf from ptp_distance.  The order inside one topleset is unspecified.
 *  Asynchronous apart from the source validation, which reads the sources
 *  on the host (a device `sources` array is copied to the host first).
 *  The mesh must outlive the returned handle.
 */
ptp_status ptp_toplesets(ptp_mesh *mesh, const int32_t *sources, int32_t m, int ptr_kind, void *stream,
                         ptp_toplesets_t **out);

/*
 * Topleset layout, for inspection.  Blocks on `stream`.  Outputs (any may be
 * NULL): rho, the number of toplesets; n_reached, the vertices reachable
 * from S; off_dev, device array [rho + 1] of topleset start offsets in the
 * renumbered order; perm_dev, device array [n_verts] mapping renumbered
 * index -> original index.  The device arrays belong to the handle.
 */
ptp_status ptp_toplesets_info(ptp_toplesets_t *tops, void *stream, int32_t *rho, int32_t *n_reached,
                              const int32_t **off_dev, const int32_t **perm_dev);

ptp_status ptp_toplesets_destroy(ptp_toplesets_t *tops);

/*
 * PTP (Sec. 4.2): d_0 = +inf except d_0(S) = 0; iteration k recomputes, from
 * d_{k-1} only, every non-source vertex of the band
 * B = V_{i_{k-1}} u ... u V_{j_k} as the minimum of its old value and the
 * update step (Sec. 3.2, planar Eikonal solve under the monotonicity
 * condition Q X^T n < 0, else the edge fallback) over its incident
 * triangles; j_k = min(k, rho - 1) (Eq. upper_band) and i_k = i_{k-1} + 1
 * when every vertex of V_{i_{k-1}} passed the relative-change test
 * (Eq. lower_band); the run stops when i_k > rho - 1.
 *  d_out   caller-owned DEVICE buffer of n_verts float32, ORIGINAL order;
 *          unreachable vertices get +inf.
 *  stats   NULL: fully asynchronous.  Non-NULL: blocks on `stream` and fills
 *          the statistics; the return value is then the device-side status
 *          (PTP_OK, PTP_ERR_NOT_CONVERGED with d_out written, or
 *          PTP_ERR_TIMEOUT).
 * Per-call scratch (two distance buffers, per-vertex change stamps) is a
 * stream-ordered allocation released on `stream` before returning.
 * Calls on the same handle must not overlap in time.
 */
ptp_status ptp_distance(ptp_toplesets_t *tops, const ptp_params *params, float *d_out, void *stream,
                        ptp_stats *stats);

/*
 * ptp_distance_from_sources -- the whole map from a mesh and a source set in
 * one launch, the toplesets being built while the iteration runs.
 *
 * Computes what ptp_toplesets followed by ptp_distance computes (Sec. 4.1,
 * Sec. 4.2; the same iterates, hence bit-identical distances), but the BFS
 * runs inside the window launch: a few CTAs expand the toplesets level by
 * level, a few more put each finished level into topleset order (Sec. 4.3:
 * slots remapped to positions, geometry copied), and the others iterate,
 * each iteration k waiting (on the device) only until V_0 .. V_k are in
 * place.  The distances are gathered back to the original order at the end.
 * (The multi-source calls, ptp_voronoi and ptp_fps, run the same launch
 * without the rearrangement, as the paper's multi-source GPU runs do, Sec.
 * 5.1: the band is walked through the BFS queue in the original order.)
 *  sources   [m] vertex indices (ptr_kind), m >= 1; repeats are ignored.
 *  d_out     [n_verts] float32 DEVICE, original order; +inf if unreachable.
 *  params    as ptp_distance; schedule must be NULL (PTP_ERR_ARG); the
 *            events, when set, bracket the fused kernel.
 * Asynchronous unless stats is non-NULL or the sources are DEVICE pointers
 * (they are validated on the host).  Errors: PTP_ERR_ARG, PTP_ERR_INDEX, and
 * the statuses of ptp_distance.  stats->rho is the number of toplesets.
 */
ptp_status ptp_distance_from_sources(ptp_mesh *mesh, const int32_t *sources, int32_t m, int ptr_kind,
                                     const ptp_params *params, float *d_out, void *stream, ptp_stats *stats);

/*
 * ptp_distance_noalloc -- ptp_distance for callers that may not allocate.
 * (An addition of this library; the paper has no counterpart.)
 *
 * ptp_distance takes its per-call scratch (two distance buffers and two
 * per-vertex change stamps, 16 bytes per vertex) from a stream-ordered
 * allocation.  Some callers cannot allocate once their set-up is done: a
 * real-time loop that must not wait for the allocator or grow a memory pool,
 * or a host application that hands every byte of device memory out through
 * its own allocator and forbids libraries from calling cudaMalloc.  Such a
 * caller creates the mesh and its toplesets at set-up and then answers
 * distance queries with this entry point, which calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *
 * Scratch: a file-scope device array sized for PTP_NOALLOC_MAX_VERTS
 * vertices (16 MiB + 256 bytes).  It belongs to the library's device code,
 * so every GPU on which the process uses the library holds it until the
 * process exits, whether or not this entry point is ever called: plain
 * ptp_distance users pay these 16 MiB per device too.  A handle with more
 * vertices is rejected with PTP_ERR_TOO_LARGE.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and caches it per device ordinal; make that first call
 * before any stream capture.  The cache assumes the device's primary
 * context (the one the CUDA runtime uses) stays alive: after
 * cudaDeviceReset, or with another context made current, the cached
 * address is stale and must not be used.  Every call shares the one
 * array per device and overwrites what the last call left there, so calls
 * whose work overlaps on the GPU (another stream, another host thread) race;
 * serialise them.  Arguments, results, blocking and statuses are those of
 * ptp_distance, except that ptp_last_stats does not see these calls: pass
 * `stats` to get their statistics.
 */
#define PTP_NOALLOC_MAX_VERTS 1048576
ptp_status ptp_distance_noalloc(ptp_toplesets_t *tops, const ptp_params *params, float *d_out, void *stream,
                                ptp_stats *stats);

/*
 * Batched maps: up to PTP_BATCH_MAX independent single-source problems
 * (different meshes, different sources, different sizes) solved by one
 * persistent launch.  Each map follows the iteration of Sec. 4.2 with its
 * own window (Eq. lower_band / upper_band) and its own iteration count, so
 * every map's distances are bit for bit those ptp_distance returns for it
 * alone; the maps share one grid barrier per iteration, which on meshes too
 * small to fill the GPU turns many latency-bound launches into one.  (An
 * addition of this library: the paper runs one map at a time.)
 *
 * ptp_batch_create copies the count toplesets handles' renumbered layouts
 * into one concatenated device layout (208 bytes per vertex plus 8 per
 * corner) on `stream` and blocks until the copy is done; the handles may be
 * destroyed afterwards.  Handles built on other streams (the toplesets of
 * independent meshes can be built concurrently, each BFS occupying one
 * 8-SM cluster) must be complete before the call: join those streams to
 * `stream` first, or synchronise them.  All handles must live on
 * one device, with fewer than 2^26 vertices and 2^31 corners in total
 * (PTP_ERR_TOO_LARGE otherwise); count in [1, PTP_BATCH_MAX] (PTP_ERR_ARG).
 * The handle belongs to the caller: ptp_batch_destroy frees it, after its
 * work on the creation stream has finished.
 *
 * ptp_distance_batch runs the maps with `params` shared by all of them
 * (eps, eps_abs, max_iter, grid, band_mode and the events as in
 * ptp_distance; trace and schedule must be NULL, else PTP_ERR_ARG).
 *  d_out   host array of count DEVICE pointers; d_out[b] receives map b's
 *          [n_verts_b] float32 distances in its mesh's vertex order.
 *  stats   NULL or an array of count records: per map iterations,
 *          band_updates, rho, status and checks; active_updates, changed and
 *          fp64_solves hold the batch totals.
 * Blocks until the launch has finished (it reads every map's status).
 * Returns PTP_OK when every map converged, PTP_ERR_NOT_CONVERGED when some
 * map reached max_iter (all distances written), PTP_ERR_TIMEOUT when a
 * device-side wait hit its limit.
 */
#define PTP_BATCH_MAX 32
ptp_status ptp_batch_create(ptp_toplesets_t *const *tops, int32_t count, void *stream, ptp_batch_t **out);
ptp_status ptp_distance_batch(ptp_batch_t *batch, const ptp_params *params, float *const *d_out, void *stream,
                              ptp_stats *stats);
ptp_status ptp_batch_destroy(ptp_batch_t *batch);

/*
 * Launch-shape autotuner for ptp_distance or ptp_distance_batch (an addition
 * of this library; the paper has no counterpart).  The iteration of Sec. 4.2
 * fixes what is computed; the threads per CTA and the number of CTAs of the
 * window kernel only change how fast, and every shape gives bit-identical
 * distances.  Exactly one of tops / batch is non-NULL.  Each candidate shape
 * (CTAs of 512, 256, 128 threads; all co-resident CTAs, one per SM, 1/2, 1/4
 * and 1/8 of the SMs, 8 CTAs) runs the caller's problem `reps` times (0 = 3,
 * at most 100) with the other fields of *params, timed on `stream` by CUDA
 * events around the window kernel; the median decides.  The fastest shape is
 * written to params->block and params->grid and, if result is non-NULL, to
 * *result.  Trial outputs go to a scratch allocation, so no output buffer
 * of the caller is written; ptp_last_stats(tops) afterwards describes the
 * last trial run.  Blocks.  Returns the first failing status of a trial run
 * (PTP_ERR_NOT_CONVERGED counts as success).
 */
typedef struct ptp_tune_result {
    int32_t block;     /* threads per CTA of the fastest shape              */
    int32_t grid;      /* CTAs of the fastest shape                         */
    float ms;          /* its median window-kernel time                     */
    float ms_default;  /* median time of the default shape (512, all CTAs)  */
    int32_t tried;     /* shapes timed                                      */
} ptp_tune_result;
ptp_status ptp_autotune(ptp_toplesets_t *tops, ptp_batch_t *batch, ptp_params *params, int32_t reps, void *stream,
                        ptp_tune_result *result);

/*
 * Self-test of the device-side wait limit (an addition of this library).
 * Every wait in the library's kernels (grid barriers, the fused launch's
 * waits for toplesets) gives up after a limit, flags PTP_ERR_TIMEOUT and
 * returns, leaving the context usable.  This launches two CTAs that wait at
 * a barrier sized for three, so the wait can only end by its limit of
 * `cycles` SM clock cycles (1000 .. 4e9; else PTP_ERR_ARG).  Blocks.
 * Returns PTP_ERR_TIMEOUT when the limit worked.
 */
ptp_status ptp_selftest_wait_limit(int64_t cycles, void *stream);

/*
 * Geodesic Voronoi regions (Sec. 5.3, Voronoi diagrams from farthest-point
 * samples): one multi-source PTP map from the m seeds (Sec. 6.1.5, multi-source
 * problem; as in the paper's multi-source runs the vertices are not
 * rearranged), where every vertex also carries the index (0..m-1) of the seed
 * its distance came from: the label of the closer neighbour of the triangle
 * that gave its final value.
 *  seeds      [m] vertex indices (ptr_kind), m >= 1; a repeated seed keeps its
 *             first index.
 *  d_out      [n_verts] float32 DEVICE, distance to the nearest seed.
 *  label_out  [n_verts] int32 DEVICE, seed index, -1 where unreachable.
 *  The map is one launch that builds the toplesets while the window runs
 *  (40 B per vertex of scratch besides the distances and labels).
 *  Blocks only when stats is non-NULL (as ptp_distance).
 */
ptp_status ptp_voronoi(ptp_mesh *mesh, const int32_t *seeds, int32_t m, int ptr_kind, const ptp_params *params,
                       float *d_out, int32_t *label_out, void *stream, ptp_stats *stats);

/*
 * Farthest-point sampling (Sec. 5.3 and App. A): S_1 = {first};
 * S_{i+1} = S_i + argmax_v d_{S_i}(v), each d_{S_i} a full multi-source PTP
 * map from all samples so far (ties: the smallest vertex index; an
 * unreachable vertex counts as infinitely far).  Everything stays on the
 * device: the argmax, the sample list and the source count are device data,
 * and with use_graph != 0 one sampling step is captured once as a CUDA graph
 * and relaunched for every sample.  Each map is one launch that builds the
 * toplesets while the window runs.
 *  samples_out  [n_samples] int32 DEVICE: first, then the chosen samples.
 *  d_out        [n_verts] float32 DEVICE or NULL: distance to all n_samples
 *               samples (one more map).
 *  stats        NULL or totals over all maps (iterations, updates; rho of the
 *               last map; status = the worst status seen).  Blocks.
 */
ptp_status ptp_fps(ptp_mesh *mesh, int32_t first, int32_t n_samples, const ptp_params *params, int32_t *samples_out,
                   float *d_out, int use_graph, void *stream, ptp_stats *stats);

/*
 * Learned iteration schedule (an extension of the method; the paper has no
 * counterpart).  A multilayer perceptron 6 -> 32 -> 32 -> 1 (ReLU) with FP16
 * weights and FP32 accumulation predicts, per topleset window, log2 of the
 * number of iterations the band's lower bound stays at that topleset.
 * Parameters: PTP_MLP_NPARAM values, flat, in the order W1[32][6], b1[32],
 * W2[32][32], b2[32], W3[32], b3 (FP32 master copy; FP16 copy as IEEE
 * binary16 bit patterns).
 */
#define PTP_MLP_NPARAM 1313
#define PTP_WINDOW_FEATURES 6

/* Per-topleset window features [rho][6] (DEVICE float32): log2(|V_r|+1)/20,
 * ring-edge length mean and std over V_r relative to the mesh mean, the
 * smallest triangle angle at V_r's vertices, std/mean of the Euclidean
 * distance from the first source over V_r (how far the topleset is from a
 * sphere around the source, i.e. from the distance isocurves, which the paper
 * ties to the iteration count, Sec. 5.2), and r / rho.  feat_out must hold
 * 6 * n_verts floats.  Asynchronous. */
ptp_status ptp_window_features(ptp_toplesets_t *tops, float *feat_out, void *stream);

/* Schedule from features: sched_out[s] = clamp(floor(2^(y_s - margin)), 1,
 * cap) for s < count (or < *count_dev when count_dev is non-NULL, a DEVICE
 * int32, e.g. &info[0] = rho).  All arrays DEVICE.  Asynchronous. */
ptp_status ptp_mlp_infer(const uint16_t *w_half, const float *feat, int32_t count, const int32_t *count_dev,
                         float margin, int32_t cap, int32_t *sched_out, void *stream);

/* One fused forward + backward pass over `count` samples (X [count][6],
 * targets Y [count], DEVICE): adds d(loss)/d(params) to grad [PTP_MLP_NPARAM]
 * and the loss sum((y - t)^2) / count to *loss (if non-NULL).  Asynchronous. */
ptp_status ptp_mlp_grad(const uint16_t *w_half, const float *X, const float *Y, int32_t count, float *grad,
                        float *loss, void *stream);

/* Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step >= 1) on the FP32 master
 * weights with moments m, v; refreshes w_half and zeroes grad.  DEVICE. */
ptp_status ptp_mlp_adam(float *w_master, uint16_t *w_half, float *m, float *v, float *grad, float lr, int32_t step,
                        void *stream);

/* FP32 parameters -> FP16 copy.  DEVICE. */
ptp_status ptp_mlp_to_half(const float *w, uint16_t *w_half, void *stream);

/* Statistics of the last ptp_distance call on this handle.  Blocks on
 * `stream`.  Returns that call's device-side status. */
ptp_status ptp_last_stats(ptp_toplesets_t *tops, void *stream, ptp_stats *stats);

/*
 * All stages in one call: mesh, then the map with the toplesets built inside
 * the window launch (ptp_distance_from_sources; with a schedule,
 * ptp_toplesets + ptp_distance), then release.  The distances are those of
 * ptp_toplesets + ptp_distance.
 *  ptr_kind applies to xyz, faces, sources AND d_out (host d_out is filled
 *  by a device-to-host copy before returning).  Blocks on `stream`.
 */
ptp_status ptp_geodesic(const float *xyz, int64_t n_verts, const int32_t *faces, int64_t n_faces,
                        const int32_t *sources, int32_t m, int ptr_kind, const ptp_params *params,
                        float *d_out, void *stream, ptp_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* PTP_H */
