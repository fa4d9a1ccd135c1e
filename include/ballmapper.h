/*
 * ballmapper.h -- C-ABI of the GB300 exact Ball Mapper library (libballmapper.so).
 *
 * The operations follow the paper's statement of the problem:
 *   - the exact range oracle R_r(q) = { x in X : d(q,x) < r }            (Sec. 5, Def. 5.1)     
 *   - the greedy epsilon-net: while a point is uncovered, select one,     (Sec. 2.2)
 *     add it to the landmark set and cover its open ball; the point
 *     selected is always the smallest uncovered index
 *   - ball memberships X_i = X intersect B(l_i, eps), full open balls     (Sec. 2.3; ball definition Sec. 2.1)
 *   - the Ball Mapper graph = 1-skeleton of the nerve: an edge {i,j}      (Sec. 2.1 nerve; Sec. 5.2, Def. 5.6)
 *     for every landmark pair whose balls share a data point
 * The metric is Euclidean (Sec. 6.1).  Distances are decided exactly: the
 * result equals the one obtained with FP64 squared distances summed in
 * coordinate order, for any finite float32 input.
 *
 * Conventions shared by every entry point
 *   - Points are float32, row-major, n rows of d contiguous coordinates.
 *   - By default every pointer argument (inputs and outputs) is DEVICE
 *     memory of the current CUDA device and all work is ordered on
 *     opt->stream.  With opt->host_io != 0, inputs are host pointers (copied
 *     in on the stream) and outputs are returned in host memory; the call
 *     then returns only after the stream work is complete.
 *   - Outputs are allocated by the library (opt->alloc / opt->free when
 *     given, else cudaMallocAsync / cudaFreeAsync on the stream, or malloc
 *     for host outputs) and released by the caller with bm_csr_free /
 *     bm_graph_free, passing the same options.
 *   - The caller keeps ownership of its inputs; they are only read.
 *   - Every call returns a bm_status; nothing throws across the ABI.  On
 *     error the output struct is zeroed, nothing is leaked, and
 *     bm_last_error() returns a thread-local message.
 *   - Ids are int32: n must be below 2^31.  Identical inputs give identical
 *     output bytes.
 */
#ifndef BALLMAPPER_H
#define BALLMAPPER_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BM_API __attribute__((visibility("default")))
#else
#define BM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BM_OK = 0,
    BM_ERR_ARG = 1,        /* invalid argument (null pointer, n or d out of range, eps not finite > 0, NaN/Inf input) */
    BM_ERR_CUDA = 2,       /* a CUDA runtime call failed; see bm_last_error() */
    BM_ERR_NOMEM = 3,      /* an allocation failed */
    BM_ERR_CAPACITY = 4,   /* an output exceeds a hard limit (e.g. more than 2^31-1 edges) */
    BM_ERR_TIMEOUT = 5,    /* a bounded device-side wait expired; the context is still usable */
    BM_ERR_UNSUPPORTED = 6 /* the device is not sm_103 (GB300) or lacks a needed feature */
} bm_status;

/* Distance-tile arithmetic.  All are exact: pairs whose approximate value
 * lies within the proven error band of eps^2 are re-decided in FP64, so the
 * results are identical on every path; the paths differ in speed and in how
 * many pairs fall into the band. */
typedef enum {
    BM_PATH_TC_SPLIT3 = 0, /* tcgen05 tensor cores: BF16 hi/lo split, three products, FP32 accumulation in TMEM */
    BM_PATH_FP32 = 1,      /* plain FP32 CUDA-core tiles (comparison path) */
    BM_PATH_TC_FP16 = 2,   /* tcgen05 tensor cores: one FP16 product on coordinates scaled by a power of two,
                            * FP32 accumulation; about 3x fewer tensor-core operations than the split with a
                            * band about 2^6 times wider (best when eps^2 is far from most squared distances) */
    BM_PATH_TC_AUTO = 3    /* default.  bm_build: the first greedy step runs on TC_SPLIT3; its band rate times
                            * the ratio of the two proven band widths predicts the fp16 band, and the greedy
                            * continues on TC_FP16 when that prediction is below 5e-5 of the tile pairs,
                            * returning to TC_SPLIT3 (once) if the measured fp16 band exceeds 2e-4;
                            * bm_build_batched: the same first-step choice per instance, made before the
                            * graph (no return inside it); range queries: TC_SPLIT3.  stats.path reports
                            * the path the build finished on. */
} bm_path;

/* Translation of the tensor-core operands.  D(q, x) is unchanged when every point and
 * query moves by the same vector c, while the proven error band grows with the operands'
 * norms (Sec. 3.2: the expanded form ||q||^2 + ||x||^2 - 2 q.x loses precision when the
 * norms dwarf the distances).  The tensor-core tiles may therefore work on fl(x - c), c the
 * mean of a sample of the points (up to 65,536 rows); results are identical either way
 * (the FP64 recheck takes the original coordinates), only the band width changes. */
typedef enum {
    BM_CENTRE_AUTO = 0,    /* default: translate when the call has at least 65,536 points, takes a
                            * tensor-core path without an inverted-file or graph index, and c shrinks
                            * the sample's largest squared norm by 5 % or more */
    BM_CENTRE_ALWAYS = 1,  /* translate whenever a tensor-core path without an index is taken */
    BM_CENTRE_OFF = 2      /* never translate */
} bm_centring;

/* Allocation callbacks: return device (or, for host outputs, ignored) memory
 * of at least `bytes` bytes ordered on `stream`; NULL signals failure.  Without them the
 * library allocates stream-ordered from a pool of its own per device and context, which
 * keeps up to 64 GiB of freed memory mapped for later calls (outputs handed to the caller
 * return to it through bm_csr_free / bm_graph_free). */
typedef void* (*bm_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*bm_free_fn)(void* ptr, void* stream, void* ctx);

typedef struct {
    void* stream;          /* cudaStream_t; NULL = legacy default stream */
    int32_t path;          /* bm_path */
    int32_t host_io;       /* 0: device pointers in and out; 1: host pointers in and out */
    int32_t batch;         /* largest greedy batch (candidates per step), multiple of 32: 32..16384 for
                              bm_build and the index builds, 32..2048 for bm_build_batched;
                              0 = 16384 (bm_build; 8192 for bm_build_ivf and bm_build_gidx).
                              The batch starts at min(batch, 256), doubles while 90 % of the
                              candidates become landmarks (99 % past 2048, 99.5 % past 4096) and
                              halves below 50 % (90 % past 2048). */
    int32_t skip_edges;    /* bm_build: 1 = landmarks and memberships only (no nerve pass) */
    bm_alloc_fn alloc;     /* optional device allocator for outputs and scratch */
    bm_free_fn free;
    void* alloc_ctx;
    int32_t want_dists;    /* bm_build, bm_range_query, bm_build_ivf, bm_ivf_range_query: 1 = also return
                              the distance of every stored pair (bm_csr.dists) and its measured error
                              (bm_stats.dist_max_rel_err); bm_build_batched rejects it (BM_ERR_ARG) */
    int32_t centring;      /* bm_centring (bm_build, bm_range_query and bm_build_batched, per instance;
                              other values: BM_ERR_ARG); the calls built on these follow it too */
} bm_options;

typedef struct {
    int64_t distance_evals;   /* algorithmic exact decisions: rows x n (memberships / range query) */
    int64_t tile_pairs;       /* pairs evaluated by the distance tiles, speculative candidates included */
    int64_t band_pairs;       /* pairs re-decided in FP64 (inside the error band) */
    int64_t greedy_steps;     /* candidate batches processed by the greedy */
    int64_t candidates;       /* candidates examined by the greedy */
    int64_t edge_pairs;       /* (i<j) landmark pairs emitted by the nerve pass before deduplication */
    double ms_prep, ms_greedy, ms_members, ms_edges, ms_total;  /* device time per phase */
    float band_delta;         /* half-width of the error band used (in units of (eps^2 - D)/2) */
    int32_t path;             /* bm_path actually used */
    double ms_sweep;          /* device time of the distance-tile launches (CUDA events on the stream) */
    int64_t sweep_launches;   /* distance-tile kernel launches */
    int64_t kernel_launches;  /* all kernel launches of the call */
    double recheck_rate;      /* band_pairs / tile_pairs: the fraction of tile decisions re-taken in FP64 */
    double dist_max_rel_err;  /* with want_dists: max over reported distances of |dist - sqrt(D)| / sqrt(D),
                                 D the FP64 squared distance in coordinate order (the CPU oracle's value);
                                 the rounding of sqrt(D) to float bounds it by 2^-24; 0 otherwise */
    int32_t truncated;        /* graph index: 1 when a query stopped at its visit cap */
    int32_t centred;          /* 1 when the tensor-core operands were those of the translated points */
} bm_stats;

typedef struct {
    int64_t rows;       /* number of rows */
    int64_t nnz;        /* number of stored ids */
    int64_t* offsets;   /* rows + 1 entries; row r is ids[offsets[r] .. offsets[r+1]) */
    int32_t* ids;       /* point ids, ascending within each row */
    int32_t on_host;    /* 1 when offsets/ids/dists are host memory */
    int32_t reserved0;
    float* dists;       /* NULL unless opt->want_dists: nnz entries, dists[e] = d(q_row, X[ids[e]]) as the
                           float nearest to the FP64 root of the FP64 squared distance summed in
                           coordinate order (relative error <= 2^-24 against that FP64 distance) */
} bm_csr;

typedef struct {
    int64_t n_landmarks;
    int32_t* landmarks;   /* point ids in greedy order (strictly increasing) */
    bm_csr members;       /* row i = R_eps(landmarks[i]), the full open ball */
    int64_t n_edges;
    int32_t* edges;       /* 2 * n_edges landmark ordinals (i, j), i < j, lexicographic, unique */
    int32_t on_host;
    int32_t reserved0;
    bm_stats stats;
} bm_graph;

/* Fill *opt with defaults (default stream, automatic tensor-core path, device I/O). */
BM_API void bm_options_init(bm_options* opt);

/* Exact range query, Sec. 5, Def. 5.1: out row j = { i : ||X_i - Q_j|| < eps }.
 * X: n x d float32; Q: m x d float32; eps > 0 finite.  n = 0 or m = 0 give
 * empty rows (X or Q may then be NULL).  stats may be NULL. */
BM_API bm_status bm_range_query(const float* X, int64_t n, int32_t d, const float* Q, int64_t m,
                         float eps, const bm_options* opt, bm_csr* out, bm_stats* stats);

/* Ball Mapper construction, Sec. 2.2 (greedy epsilon-net in index order),
 * Sec. 2.3 (full-ball memberships) and Sec. 2.1 / Sec. 5.2 (nerve edges).
 * n = 0 gives an empty graph. */
BM_API bm_status bm_build(const float* X, int64_t n, int32_t d, float eps, const bm_options* opt,
                   bm_graph* out);

/* k-th nearest-neighbour distance of every point, the point itself counted first
 * (the target-occupancy rule of Sec. 6.1): kdist[i] = sqrt(D_(k)(i)), D_(1) <= D_(2) <= ...
 * the FP64 squared distances (coordinate order) from X_i to all n points, X_i included.
 * Exact: equal to the FP64 value of that definition for any finite float32 input.
 *   X: n x d float32 (n >= 1); 1 <= k <= min(n, 1024);
 *   kdist: n doubles (device memory; host memory with opt->host_io), written.
 * Arithmetic: a proven upper bound of each row's k-th squared distance from a strided
 * sample of the points (CUDA cores), a range query of every point with its own radius
 * on the distance tiles (opt->path; automatic and fp16 run the bf16 split), then the
 * k-th smallest FP64 squared distance of each ball.  stats may be NULL. */
BM_API bm_status bm_knn_dist(const float* X, int64_t n, int32_t d, int32_t k, const bm_options* opt, double* kdist,
                             bm_stats* stats);

/* Target-occupancy scale (Sec. 6.1): *eps = median over the points of bm_knn_dist's
 * values (for even n the mean of the two middle values), returned in host memory. */
BM_API bm_status bm_occupancy_eps(const float* X, int64_t n, int32_t d, int32_t k, const bm_options* opt,
                                  double* eps, bm_stats* stats);

/* Ball Mapper on farthest-point landmarks (Sec. 2.2, the deterministic alternative to
 * the greedy): L = {first}; repeatedly the point farthest from L (the smallest index
 * among equal distances) joins L while its distance to L is at least eps (open balls:
 * a point at exactly eps is not covered, so the paper's "> eps" is taken as ">=" here,
 * the rule under which every point ends inside an open ball).  Landmarks are returned
 * in selection order (out->landmarks[0] == first); memberships are the full open balls
 * in that order and edges use those ordinals (i < j, lexicographic), as in bm_build.
 * Distances are decided exactly (FP64 in coordinate order).  0 <= first < n (n = 0
 * gives an empty graph).  stats.greedy_steps = selection passes, ms_greedy includes them. */
BM_API bm_status bm_build_fps(const float* X, int64_t n, int32_t d, float eps, int64_t first, const bm_options* opt,
                              bm_graph* out);

/* Coloring (Sec. 2.3): out[i] = statistic of f over CSR row i (the ball X_i):
 *   BM_COLOR_MEAN (FP64 sum / |X_i|; the summation order is unspecified, so the value
 *   may differ from a sequential sum by (|X_i| - 1) 2^-53 sum |f|), BM_COLOR_MEDIAN (the
 *   middle value, or for an even count the mean of the two middle values), BM_COLOR_MIN,
 *   BM_COLOR_MAX.  An empty row gets NaN.
 *   offsets (rows + 1, int64), ids (int32, in [0, n)), f (n float32, finite), out (rows
 *   doubles): device memory, or host memory with opt->host_io.  BM_ERR_ARG for an id out
 *   of range or a non-finite f. */
typedef enum { BM_COLOR_MEAN = 0, BM_COLOR_MEDIAN = 1, BM_COLOR_MIN = 2, BM_COLOR_MAX = 3 } bm_color_stat;
BM_API bm_status bm_color(const int64_t* offsets, const int32_t* ids, int64_t rows, const float* f, int64_t n,
                          int32_t stat, const bm_options* opt, double* out);

/* One problem of a batched build: n x d float32 points (device memory; host
 * memory with host_io) and its own eps. */
typedef struct {
    const float* X;
    int64_t n;
    int32_t d;
    float eps;
    int32_t batch;       /* largest greedy batch of this instance, multiple of 32 in [32, 2048];
                            0 = opt->batch (an autotuned per-(d, n) table fills it) */
    int32_t reserved0;
} bm_instance;

/* Many independent Ball Mapper builds (each exactly bm_build's result: Sec. 2.2
 * greedy, Sec. 2.3 memberships, Sec. 5.2 nerve) in one call.  The paper builds
 * one complex at a time; this entry point exists to fill the GPU with many
 * small problems.  The greedy loops of all instances run inside one CUDA graph
 * launched once: a device-side WHILE loop per instance, the loops side by side,
 * each iteration one greedy step that decides on the device whether another is
 * needed.  Prep runs before the graph; CSR and nerve edges after it, for all
 * instances at once.  An instance whose step buffers overflow inside the graph
 * is finished by the host-driven loop with larger buffers (same result).
 *   inst:     count instances (count >= 0); each validated like bm_build.
 *   opt:      stream, path, host_io, skip_edges, alloc/free as for bm_build;
 *             batch = largest candidate batch per step of instances whose own
 *             batch is 0 (0 = 1024).  With the automatic path every instance's
 *             first greedy step runs on the bf16 split before the graph, and the
 *             instance continues on fp16 inside the graph when its measured band
 *             predicts a small fp16 band (the rule of bm_build's automatic path);
 *             stats.path reports each instance's choice.
 *   outs:     count graphs, caller-owned array; each filled like bm_build's out.
 *             stats.ms_total of every instance is the time of the whole call,
 *             ms_prep that of the prep of all instances, ms_greedy that of the
 *             graph launch, ms_members that of the tails (host resume of
 *             overflowed instances, then CSR and nerve edges of all instances as
 *             one renumbered build); ms_edges, ms_sweep and edge_pairs stay 0.
 *             The instances together may hold at most 2^31 - 1 points and
 *             landmarks (BM_ERR_CAPACITY otherwise).
 *   statuses: optional, count entries: BM_OK, or the status of the instance
 *             that failed.
 * On error every outs[i] is zeroed (nothing leaks) and the first failing
 * status is returned; bm_last_error names the instance. */
BM_API bm_status bm_build_batched(const bm_instance* inst, int32_t count, const bm_options* opt, bm_graph* outs,
                                  int32_t* statuses);

/* ---- Tensor-core tile configuration (no counterpart in the paper: it tunes how
 * the distance tiles of Sec. 3.2 map onto the GB300's tensor cores).
 * For a point dimension d the tiles use K extent d_pad (a multiple of ck, >= d;
 * the operands are zero-padded to it), K chunks of ck bf16 per shared-memory
 * stage (16, 32 or 64), point tiles of nt rows (64, 128 or 256) held in bbuf
 * buffers, and astg stages of query chunks.  Only shapes compiled into the
 * library are accepted (bm_tile_shapes lists them, d_pad = 0 there), and an override
 * must fit the shared memory of both tensor-core representations.  Results
 * never depend on the configuration; speed does.  Settings are process-wide,
 * guarded by a lock, and read when a call prepares its operands. */
typedef struct {
    int32_t d_pad;
    int32_t ck;
    int32_t nt;
    int32_t bbuf;
    int32_t astg;
} bm_tile_config;

/* Writes up to max compiled shapes into out (out may be NULL); returns how many exist. */
BM_API int32_t bm_tile_shapes(bm_tile_config* out, int32_t max);
/* The configuration used for dimension d (an override if set, else the built-in choice). */
BM_API bm_status bm_get_tile_config(int32_t d, bm_tile_config* out);
/* Override the configuration for dimension d; cfg = NULL restores the built-in
 * choice.  BM_ERR_ARG (with the reason in bm_last_error) for a configuration
 * that is not compiled, does not fit in shared memory, or pads d wrongly. */
BM_API bm_status bm_set_tile_config(int32_t d, const bm_tile_config* cfg);

/* Nerve-edge deduplication (Sec. 5.2): witnessed landmark pairs are made unique
 * either in a bitmap of landmark rows (chosen when the bitmap is at most 64
 * bytes per witnessed pair) or by sorting the pair keys.  bytes bounds the
 * bitmap of one chunk of rows (default 1 GiB, 0 restores it; a negative value
 * always sorts).  Process-wide; returns the previous setting.  Results do not
 * depend on it. */
BM_API int64_t bm_set_nerve_bitmap_bytes(int64_t bytes);

/* The proven half-width of the error band (Sec. 3.2: the tiles evaluate
 * v = q.x - phi_q - phi_x = (eps^2 - D)/2 from the expanded form, in FP32 on the
 * tensor cores or the CUDA cores), in units of v: the library decides a pair on the
 * tiles only where the accumulator lies farther than this from the decision point, and
 * re-decides the rest in FP64.  path: BM_PATH_TC_SPLIT3, BM_PATH_TC_FP16 or BM_PATH_FP32;
 * d: dimension; d_pad: the padded K extent of the tiles (bm_get_tile_config; d for the
 * FP32 path); n_a, n_b: bounds on the norms of the query and point rows; phi_a, phi_b:
 * bounds on their |phi| (on the fp16 path all four in the operands' scaled units).  The
 * library uses it per query row (n_a, phi_a of the row) against the points' maxima.  Host
 * function, no device needed; a negative or non-finite input gives a non-finite result. */
BM_API double bm_band_halfwidth(int32_t path, int32_t d, int32_t d_pad, double n_a, double n_b, double phi_a,
                                double phi_b);

/* ---- Inverted-file index: the paper's non-exhaustive approximate oracle (Sec. 5.4;
 * nprobe cells searched per query, Sec. 6.1).  Points are grouped into nlist
 * k-means cells; a query examines only the points of its nprobe nearest cells
 * and decides membership exactly, so every returned point is a true member
 * (conservative oracle, Def. 5.14: no false positives, Sec. 5.3).
 * Cells: `iters` Lloyd iterations on `sample` points (0 = min(n, 262144))
 * drawn by a seeded Fisher-Yates shuffle (splitmix64); the first nlist
 * sampled points initialise the centroids; a point's cell is its nearest
 * centroid (ties to the lowest id); centroids are FP64 means of their
 * members in point order; an empty cell keeps its centroid.
 * The index refers to X (device) until freed; with opt->host_io it keeps a
 * device copy.  Its buffers come from opt's allocator. */
typedef struct bm_ivf bm_ivf;

BM_API bm_status bm_ivf_train(const float* X, int64_t n, int32_t d, int32_t nlist, int32_t iters, int64_t sample,
                              uint64_t seed, const bm_options* opt, bm_ivf** out);
BM_API void bm_ivf_free(bm_ivf* idx);
/* Shape and device arrays of the index: cell of each point (n), centroids (nlist x d). */
BM_API bm_status bm_ivf_info(const bm_ivf* idx, int64_t* n, int32_t* d, int32_t* nlist, const int32_t** cell_of,
                             const float** centroids);
/* out row j = { i : cell(i) among the nprobe cells nearest to Q_j, ||X_i - Q_j|| < eps }.
 * probes: optional device int32 array (m x nprobe) receiving each query's cells. */
BM_API bm_status bm_ivf_range_query(const bm_ivf* idx, const float* Q, int64_t m, float eps, int32_t nprobe,
                                    const bm_options* opt, bm_csr* out, int32_t* probes, bm_stats* stats);
/* Ball Mapper with the inverted-file oracle (Sec. 6.2 modes).  landmarks != NULL:
 * fixed-landmark mode (their balls and nerve through the index; landmarks is
 * device memory, or host memory with opt->host_io).  landmarks == NULL:
 * end-to-end mode (the greedy of Sec. 2.2 driven by the index's range sets). */
BM_API bm_status bm_build_ivf(const bm_ivf* idx, float eps, int32_t nprobe, const int32_t* landmarks,
                              int64_t n_landmarks, const bm_options* opt, bm_graph* out);

/* ---- Proximity-graph index: the paper's graph-based non-exhaustive oracle (Sec. 5.4:
 * a query examines only the part of a proximity graph its traversal visits, and decides
 * membership with the exact distance, so every returned point is a true member --
 * false negatives only, no false positives; the breadth of the search is the efSearch
 * of Sec. 6.1, here ef).
 * Graph: every point's M nearest other points (by FP64 squared distance, then id),
 * made undirected; adjacency lists ascend by id.
 * Query (one warp per query, distances FP64 in coordinate order, candidates ordered by
 * (distance, id)): the nearest of n_entries entry points floor(t n / n_entries); a beam
 * of at most ef visited nodes, the best unexpanded one expanded until all are expanded;
 * then every visited node inside the ball that was not expanded is expanded in visit
 * order; at most max_visits visits per query (0 = 4096; stats.truncated reports a query
 * that stopped there).  The row is the visited points strictly inside eps.
 * The index refers to X (device) until freed; with opt->host_io it keeps a device copy.
 *   bm_gidx_build: 1 <= M <= min(n - 1, 1023); n_entries in [1, n] (0 = min(n, 64)).
 *   ef in [1, 256]; max_visits in [1, 2^24]. */
typedef struct bm_gidx bm_gidx;

BM_API bm_status bm_gidx_build(const float* X, int64_t n, int32_t d, int32_t M, int32_t n_entries,
                               const bm_options* opt, bm_gidx** out);
BM_API void bm_gidx_free(bm_gidx* idx);
/* Shape and device arrays of the graph: adj_off (n + 1), adj (n_adj neighbour ids). */
BM_API bm_status bm_gidx_info(const bm_gidx* idx, int64_t* n, int32_t* d, int64_t* n_adj, const int64_t** adj_off,
                              const int32_t** adj);
/* out row j = the points with d(X_i, Q_j) < eps among those the search for Q_j visits. */
BM_API bm_status bm_gidx_range_query(const bm_gidx* idx, const float* Q, int64_t m, float eps, int32_t ef,
                                     int64_t max_visits, const bm_options* opt, bm_csr* out, bm_stats* stats);
/* Ball Mapper with the graph oracle (Sec. 6.2 modes): landmarks != NULL: fixed-landmark
 * mode (device memory, host with opt->host_io); NULL: the greedy of Sec. 2.2 driven by
 * the index's range sets (a point is covered when a landmark's search finds it). */
BM_API bm_status bm_build_gidx(const bm_gidx* idx, float eps, int32_t ef, int64_t max_visits,
                               const int32_t* landmarks, int64_t n_landmarks, const bm_options* opt, bm_graph* out);

/* Release outputs (safe on zeroed structs); pass the options used to create them. */
BM_API void bm_csr_free(bm_csr* csr, const bm_options* opt);
BM_API void bm_graph_free(bm_graph* g, const bm_options* opt);

BM_API const char* bm_status_string(bm_status s);
BM_API const char* bm_last_error(void);

/* Range COUNT without any allocation: counts[j] = |{ i : ||X_i - Q_j|| < eps }|.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot allocate device memory when they call (allocation-free real-time
 * code, code running inside another allocator's callback, a fixed memory
 * budget).  It works in a 32 MiB scratch area compiled into the library (held
 * by every GPU that loads it until process exit) plus the caller's arrays:
 *   X: n x d, Q: m x d float32 device arrays; counts: m int64 device array
 *   (written, previous contents ignored); stream: cudaStream_t or NULL.
 * Limits: n + m <= 4,194,304 (else BM_ERR_CAPACITY, nothing launched); at most
 * 2,097,120 pairs may fall in the error band (else BM_ERR_CAPACITY); eps <= 1e19
 * (else BM_ERR_ARG).  NaN or Inf in X or Q: BM_ERR_ARG.
 * The first call in a CUDA context on a device looks up the scratch's device
 * address (again after a cudaDeviceReset), so make it before any stream
 * capture begins.  Calls share the scratch: calls whose GPU work overlaps
 * (other streams or threads) race and must be serialised by the caller.  The
 * call synchronises `stream` before returning. */
BM_API bm_status bm_range_count_noalloc(const float* X, int64_t n, int32_t d, const float* Q, int64_t m,
                                        float eps, void* stream, int64_t* counts);

/* Library version as major*10000 + minor*100 + patch. */
BM_API int32_t bm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BALLMAPPER_H */
