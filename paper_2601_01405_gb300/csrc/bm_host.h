// bm_host.h -- host-side internal interfaces of libballmapper (not part of the C-ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "ballmapper.h"
#include "bm_common.cuh"

namespace bm {

// Scratch/output allocator bound to one call: caller callbacks when given,
// else stream-ordered cudaMallocAsync.  Frees whatever it still holds on
// destruction (outputs are detached with take()).
// Device memory of one call, freed (stream-ordered) when the Arena dies.  In
// slab mode requests up to 16 MB are carved from a few blocks (4 MB, doubling
// up to 64 MB): one allocator call per block instead of one per buffer;
// release() does not return slab memory and slab buffers cannot be taken.
// Larger requests stay buffers of their own in both modes.
class Arena {
public:
    Arena(const bm_options* opt, cudaStream_t s, bool slab = false) : opt_(opt), stream_(s), slab_(slab) {}
    ~Arena();
    void* get(size_t bytes);          // nullptr on failure; 256-byte aligned
    void* get_standalone(size_t bytes);   // a buffer of its own even in slab mode
    void release(void* p);            // free now (standalone buffers only)
    bool take(void* p);               // detach a standalone output (caller frees it later)
    const bm_options* options() const { return opt_; }
private:
    void* raw(size_t bytes);
    const bm_options* opt_;
    cudaStream_t stream_;
    bool slab_;
    std::vector<void*> ptrs_;         // standalone buffers
    std::vector<void*> slabs_;        // slab blocks
    char* cur_ = nullptr;
    size_t left_ = 0, next_ = 4u << 20;
    static constexpr size_t kSlabMax = 16u << 20;
};

void device_free(const bm_options* opt, cudaStream_t s, void* p);
// Identifier of the current CUDA context (0 when the driver cannot report one).
unsigned long long current_context_id();

// Launch with programmatic stream serialization (the kernel must begin with pdl_wait();
// see bm_common.cuh), so that its launch overlaps the predecessor kernel's tail.  Inside a
// stream capture the launch is an ordinary one.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;   // unknown: take the ordinary launch
    }
    cfg.attrs = cs == cudaStreamCaptureStatusNone ? attr : nullptr;
    cfg.numAttrs = cs == cudaStreamCaptureStatusNone ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// Kernel launches issued by the current thread (reported in bm_stats).
extern thread_local long long g_kernel_launches;
inline void note_launch() { ++g_kernel_launches; }

// Failure carried up to the C-ABI.
struct Failure {
    bm_status status;
    std::string msg;
};

// One side of the distance tiles after preparation.
struct Prepared {
    const float* x = nullptr;          // rows x d float32 (device)
    long long rows = 0;
    int d = 0;
    float* phi = nullptr;              // ||x||^2 / 2 - eps^2 / 4, rounded to float
    __nv_bfloat16* hi = nullptr;       // rows x d_pad: bf16(x)
    __nv_bfloat16* lo = nullptr;       // rows x d_pad: bf16(x - bf16(x))
    __nv_bfloat16* aug = nullptr;      // rows x 16: the -phi pieces and ones (see prep kernel)
    int d_pad = 0;
    int ck = 0, nt = 0, bbuf = 0, astg = 0;   // tensor-core tile shape chosen for this d
    int prec = 0;                      // kPrecNone / kPrecSplit (bf16 hi, lo) / kPrecFp16 (fp16 in hi, no lo)
    int scale_exp = 0;                 // fp16: operands hold x * 2^scale_exp
    const float* centre = nullptr;     // d floats (device) or null: the tensor-core operands, phi and the
                                       // norms are those of fl(x - centre); x itself stays untranslated
};
constexpr int kPrecNone = 0, kPrecSplit = 1, kPrecFp16 = 2;

// Tensor-core tile configuration for one point dimension d: padded K extent
// (a multiple of ck, >= d), K chunk per shared-memory stage, point-tile width,
// point-tile buffers and query-chunk stages.
struct TileConfig {
    int d_pad, ck, nt, bbuf, astg;
};
// prod: tensor-core products per coordinate (3 for the bf16 split, 1 for fp16)
TileConfig tile_config_for(int d, int prod = 3);   // the override for d if one is set, else the built-in choice
TileConfig tile_config_builtin(int d, int prod = 3);
bool tile_config_check(int d, const TileConfig& c, std::string* why, int prod = 3);
bool tile_config_set(int d, const TileConfig* c, std::string* why);   // nullptr: back to the built-in choice
int tile_shapes(TileConfig* out, int max);  // the compiled (ck, nt, bbuf, astg) shapes, d_pad = 0

// prep.cu
// row_r2 (optional, query side): per-row squared radius; phi = ||x||^2/2 - row_r2[r]/2
// (the whole radius on this side; the point side is then prepared with eps2 = 0)
cudaError_t launch_prep(const float* x, long long rows, int d, double eps2, bool a_side, bool want_tc,
                        Prepared& out, unsigned* max_norm_bits, int* bad_flag, cudaStream_t s,
                        const double* row_r2 = nullptr);
cudaError_t launch_delta(DeviceState* st, int path, int d, int d_pad, double eps2, bool same_sets,
                         cudaStream_t s, int scale_exp = 0);
// Centre of the tensor-core operands: the mean of a sample of the rows of x (d floats into
// centre), set to 0 unless it shrinks the sample's largest squared norm by 5 % (force: kept
// always); *centred (device) receives 1 when kept.  partial: kCentreBlocks * d doubles,
// maxima: 2 unsigned (device scratch).
constexpr int kCentreBlocks = 152 * 8;
cudaError_t launch_centre(const float* x, long long rows, int d, bool force, double* partial, unsigned* maxima,
                          float* centre, int* centred, cudaStream_t s);
// fp16 operands of an already prepared set (hi, aug allocated as 2-byte arrays)
cudaError_t launch_prep16(const float* x, long long rows, int d, double eps2, bool a_side, int scale_exp,
                          Prepared& p, cudaStream_t s);
int fp16_scale_exp(double max_norm, double eps);
// Proven band half-width of a path in its operand units (see bm_prep.cu)
__host__ __device__ double band_halfwidth(int path, int d, int d_pad, double eps2, double Na, double Nb,
                                          int scale_exp);
// The same bound for explicit bounds Pa, Pb on |phi| of the two sides (operand units)
__host__ __device__ double band_halfwidth_core(int path, int d, int d_pad, double Na, double Nb, double Pa,
                                               double Pb);
// The per-row delta' entries of an augmentation (A side: column 6; B side: 1 in column 6,
// the point's own delta'_row in column 7), once the points' maximum norm is in st.
// eps2: the radius the set was prepared with (0 for the points of a k-NN sweep);
// row_r2: a k-NN sweep's per-query squared radii (A side), else null.
cudaError_t launch_set_aug_delta(const DeviceState* st, Prepared& p, double eps2, bool a_side, cudaStream_t s,
                                 const double* row_r2 = nullptr);

struct IvfIndex;
struct GraphIndex;

// tile_fp32.cu
struct SweepDesc {
    const Prepared* a;           // query / candidate rows
    const Prepared* b;           // points
    long long a_rows_max;        // rows the launch covers
    const int* a_rows_dev;       // when non-null: active rows read on device (greedy)
    const DeviceState* st;       // delta, done flag
    bool check_done;             // skip work when st->done
    double eps2;
    HitSink sink;
    // inverted-file mode: scan only the nprobe cells nearest to each row
    const IvfIndex* ivf = nullptr;
    const float* ivf_phi_perm = nullptr;
    int nprobe = 0;
    int* ivf_probes_out = nullptr;   // optional: where to leave each row's probed cells
    // per-row squared radius (k-NN sweeps): the band recheck decides D < row_eps2[row]
    const double* row_eps2 = nullptr;
    // graph-index mode: the rows' balls are searched through the proximity graph
    const GraphIndex* gidx = nullptr;
    int gidx_ef = 0;
    long long gidx_max_visits = 0;
    // inverted-file scan on the tensor cores: the padded cell-ordered point operands
    const Prepared* ivf_b_pad = nullptr;
    // table mode of the tensor-core tiles (work items, A row -> query, source row -> point)
    const TcItem* tc_items = nullptr;
    const long long* tc_items_count = nullptr;
    const int* tc_a_map = nullptr;
    const int* tc_b_ids = nullptr;
};
cudaError_t launch_sweep_fp32(const SweepDesc& s, cudaStream_t stream);

// tile_tc.cu
bool tc_supported();             // device is sm_103 and the kernel loaded
// grid_out: CTAs launched (= hit segments written when s.sink.seg_counts is set)
cudaError_t launch_sweep_tc(const SweepDesc& s, cudaStream_t stream, std::string* why, int* grid_out);
int device_sm_count();
// Gather the per-CTA hit and band segments of one sweep into dst / band_dst
// (one launch); *count_out / *band_count_out = entries kept.  A segment longer
// than seg_cap sets overflow_bit in st->error (and st->done when
// stop_on_overflow) and records its length in st->max_seg.
cudaError_t launch_compact_segments(const unsigned long long* src, const unsigned long long* band_src,
                                    unsigned long long seg_cap, const unsigned long long* seg_counts,
                                    const unsigned long long* band_seg_counts, int nseg, unsigned long long* dst,
                                    unsigned long long* band_dst, unsigned long long* count_out,
                                    unsigned long long* band_count_out, DeviceState* st, int overflow_bit,
                                    bool check_done, bool stop_on_overflow, cudaStream_t s);

// greedy.cu
struct GreedyBuffers {
    DeviceState* st;
    unsigned* covered;            // ceil(n/32) words
    int* slot_of;                 // n, -1 when not a candidate of the current step
    int* cand_ids;                // S
    int* ordinal;                 // S: landmark ordinal of a slot, -1 when not a landmark
    unsigned* conflict;           // S x S/32
    unsigned* row_any;            // S/32
    int* landmarks;               // n
    Prepared cand;                // gathered candidate rows (x, phi, hi, lo, aug)
    unsigned long long* step_keys;
    unsigned long long step_cap;
    unsigned long long* mem_keys;
    unsigned long long mem_cap;
};
cudaError_t launch_greedy_select(const GreedyBuffers& g, const Prepared& pts, int S, bool want_tc,
                                 cudaStream_t s);
cudaError_t launch_greedy_gather(const GreedyBuffers& g, const Prepared& pts, int S, bool want_tc, cudaStream_t s);
cudaError_t launch_greedy_resolve(const GreedyBuffers& g, int S, cudaStream_t s);
cudaError_t launch_greedy_apply(const GreedyBuffers& g, cudaStream_t s);
cudaError_t launch_greedy_continue(const GreedyBuffers& g, cudaGraphConditionalHandle h, unsigned* iterations,
                                   unsigned max_iterations, cudaStream_t s);
cudaError_t launch_greedy_rollback(const GreedyBuffers& g, cudaStream_t s);

// sort.cu
cudaError_t exclusive_scan_i64(const long long* in, long long* out, long long n, Arena& ar,
                               cudaStream_t s);  // out[0..n], out[n] = total
cudaError_t radix_sort_u64(unsigned long long* keys, unsigned long long* tmp, long long n,
                           const std::vector<int>& shifts, Arena& ar, cudaStream_t s,
                           unsigned long long** result);
int bits_for(long long v);  // bits needed to represent v (>= 0)
std::vector<int> digit_shifts(int lo_bits, int hi_bits);  // 8-bit digit shifts covering [0,lo) and [32,32+hi)

// ivf.cu: inverted-file index (Sec. 5.4 IndexIVFFlat-style cells) and its scan.
struct IvfIndex {
    long long n = 0;
    int d = 0;
    int nlist = 0;
    const float* X = nullptr;          // the indexed points (device, row-major), by id
    float* centroids = nullptr;        // nlist x d
    float* cnorm = nullptr;            // nlist: ||c||^2 (float)
    long long* cell_off = nullptr;     // nlist + 1
    int* cell_ids = nullptr;           // n: point ids grouped by cell, ascending within a cell
    int* cell_of = nullptr;            // n: cell of each point
    float* xperm = nullptr;            // n x d: rows of X in cell order
    float* xnorm = nullptr;            // n: ||x||^2 of the rows of X (by id, float)
    bm_options opt;                    // allocator of the index's buffers
    float* owned_x = nullptr;          // device copy of X when the index was built from host memory
    // tensor-core scan: the cell-ordered points with every cell padded to a multiple of 256
    // rows (zero rows after its points), so that point tiles never straddle two cells
    long long* pad_off = nullptr;      // nlist + 1: first padded row of each cell
    float* xpad = nullptr;             // npad x d
    long long npad = 0;
    long long max_cell_tiles = 0;      // largest padded cell / 256
};
// pad_off = exclusive scan of the cell sizes (off[c+1] - off[c]) rounded up to `unit`
cudaError_t launch_cell_pad_offsets(const long long* off, int nlist, int unit, long long* counts, long long* pad_off,
                                    Arena& ar, cudaStream_t s);
// xpad row pad_off[c] + j = xperm row cell_off[c] + j for j < the cell's size, zeros after
cudaError_t launch_pad_rows(const float* xperm, const long long* cell_off, const long long* pad_off, int nlist,
                            long long npad, int d, float* xpad, cudaStream_t s);
// The tensor-core scan's layout for one sweep (queries grouped by probed cell, cq_off /
// cq_rows): the padded query operands (A hi / lo / aug rows copied from `a`, zero rows
// for padding; a_map = query of each padded row or -1) and the work items (per cell:
// its point tiles x groups of up to 16 query tiles).  items_count (device) = items made.
cudaError_t launch_ivf_tc_layout(const IvfIndex& ix, int NT, const long long* cq_off, const int* cq_rows,
                                 const Prepared& a, Prepared& apad, int* a_map, long long* pa_off, long long* cnt,
                                 TcItem* items, long long* item_off, Arena& ar, cudaStream_t s);

// Nearest centroid per row (FP32 expansion ||x||^2 + ||c||^2 - 2 x.c, ties to the
// lowest centroid id): best[r] = (float bits of the distance << 32) | centroid.
cudaError_t launch_nearest_centroid(const float* rows, const int* row_ids, long long nrows, const float* rnorm,
                                    const float* cent, const float* cnorm, int nlist, int d,
                                    unsigned long long* best, cudaStream_t s);
cudaError_t launch_row_norms(const float* x, long long rows, int d, float* out, cudaStream_t s);
cudaError_t launch_cell_means(const float* rows, const long long* off, const int* members, int nlist, int d,
                              float* cent, cudaStream_t s);
cudaError_t launch_unpack_cells(const unsigned long long* best, const int* row_ids, long long n, int* cell_of,
                                unsigned long long* keys, cudaStream_t s);
cudaError_t launch_gather_rows(const float* x, const int* ids, long long rows, int d, float* out, cudaStream_t s);
// top-nprobe centroids of each query row (direct FP32 distances, ties to the lowest id)
cudaError_t launch_probe_select(const float* A, long long rows_max, const int* rows_dev, const IvfIndex& ix,
                                int nprobe, int* probes, cudaStream_t s);
// group (row, probe) pairs by cell: cq_off[nlist+1], cq_rows; tile_off[nlist+1] over 64 x 64 tiles
cudaError_t launch_group_probes(const int* probes, long long rows_max, const int* rows_dev, int nprobe,
                                const IvfIndex& ix, long long* cnt, long long* cq_off, int* cq_rows,
                                long long* tile_off, Arena& ar, cudaStream_t s);
// scan the probed cells: hits -> sink (global counters), band pairs -> sink.band_keys
cudaError_t launch_ivf_scan(const float* A, const float* phiA, const IvfIndex& ix, const float* phi_perm,
                            const long long* cq_off, const int* cq_rows, const long long* tile_off,
                            const DeviceState* st, bool check_done, const HitSink& sink, cudaStream_t s);

// recheck.cu: FP64 re-decision of the band pairs; confirmed hits are appended
// to keys through *count (book: the greedy's candidate-conflict bookkeeping).
cudaError_t launch_band_recheck(DeviceState* st, const unsigned long long* band, unsigned long long band_cap,
                                const float* ax, const float* bx, int d, double eps2, unsigned long long* keys,
                                unsigned long long* count, unsigned long long cap, const HitSink& book,
                                bool check_done, int overflow_bit, bool stop_on_overflow, cudaStream_t s,
                                const double* row_eps2 = nullptr);

// dists.cu: dists[e] = float(sqrt(D)) for every CSR entry, D the FP64 squared distance
// in coordinate order between the row's query (qx + r d, or X + qidx[r] d) and X[ids[e]];
// the largest relative error against sqrt(D) is atomicMax'ed into *max_err_bits (double bits).
cudaError_t launch_member_dists(const float* qx, const int* qidx, const float* X, int d, const long long* offsets,
                                long long rows, const int* ids, long long nnz, float* dists,
                                unsigned long long* max_err_bits, cudaStream_t s);

// knn.cu: k-th nearest-neighbour distances (Sec. 6.1 target occupancy)
// Pass 1: rho[q] = a squared radius strictly above the k-th smallest FP64 squared
// distance from X[q] to the sample {X[j * stride] : j < s} (s >= k), itself a bound on
// the k-th smallest over all points; *rho_max_bits = max rho (double bits); *bad |= 1
// when a bound is not finite.  Shared memory: 8 k doubles per block (k <= 1024).
cudaError_t launch_knn_bound(const float* X, long long n, int d, long long stride, long long s, int k, double* rho,
                             unsigned long long* rho_max_bits, int* bad, cudaStream_t st);
// Pass 3: D[e] = FP64 squared distance of CSR entry e to its row's point X[row]; kdist[r]
// = sqrt of the k-th smallest D of row r (*bad |= 2 when a row holds fewer than k).
// exclude_self: rank among the entries other than the row's own point; kD (optional):
// the k-th smallest squared distance itself.
cudaError_t launch_knn_select(const float* X, int d, const long long* offsets, long long rows, const int* ids,
                              long long nnz, double* D, int k, double* kdist, int* bad, cudaStream_t st,
                              bool exclude_self = false, double* kD = nullptr);

// fps.cu: farthest point sampling (Sec. 2.2), one kernel per landmark inside a graph
// WHILE loop (the last block to finish a pass appends the landmark and sets the loop
// condition).  mind: n doubles (the FP64 squared distance to the landmark set).
struct FpsState {
    long long count;                 // landmarks so far
    long long last;                  // the newest landmark
    int done;                        // 1 once no point is at distance >= eps
    int error;                       // 1 when the iteration bound was passed
    unsigned long long iterations;   // passes run
    double last_dist2;               // squared distance of the newest landmark to the set before it
};
int fps_grid(long long n);           // blocks of a pass (the size of the partial arrays)
cudaError_t launch_fps_init(double* mind, long long n, int* landmarks, FpsState* st, long long first, cudaStream_t s);
cudaError_t launch_fps_step(const float* X, long long n, int d, double eps2, double* mind, int* landmarks, FpsState* st,
                            double* part_v, int* part_i, unsigned* ticket, cudaGraphConditionalHandle h, bool use_graph,
                            cudaStream_t s);
cudaError_t launch_finite_check(const float* X, long long count, int* bad, cudaStream_t s);

// color.cu: coloring (Sec. 2.3) of every CSR row; stat 0 mean, 1 median, 2 min, 3 max;
// *bad |= 1 for an id outside [0, n), |= 2 for a non-finite f.
cudaError_t launch_color(const long long* offsets, const int* ids, long long rows, const float* f, long long n, int stat,
                         double* out, int* bad, cudaStream_t s);

// gidx.cu: the proximity-graph index (Sec. 5.4, graph-based non-exhaustive search).
struct GraphIndex {
    long long n = 0;
    int d = 0;
    int M = 0;                        // nearest neighbours per point before symmetrisation
    int E = 0;                        // entry points floor(t n / E), t < E
    const float* X = nullptr;         // the indexed points (device)
    long long* adj_off = nullptr;     // n + 1
    int* adj = nullptr;               // undirected adjacency, ascending per node
    long long n_adj = 0;
    bm_options opt;                   // allocator of the index's buffers
    float* owned_x = nullptr;         // device copy of X when built from host memory
};
// nbr[r M + t]: row r's M nearest other points (ball entries with D < DM, then D == DM in id order)
cudaError_t launch_knn_ids(const long long* offsets, const int* ids, const double* D, const double* DM, long long rows,
                           int M, int* nbr, int* bad, cudaStream_t s);
cudaError_t launch_arc_keys(const int* nbr, long long n, int M, unsigned long long* keys, cudaStream_t s);
// out = the distinct keys of the sorted array keys (count at pos[n] after the scan)
cudaError_t launch_unique_sorted(const unsigned long long* keys, long long n, long long* flags, long long* pos,
                                 unsigned long long* out, Arena& ar, cudaStream_t s);
// rows of sd (candidates or queries) searched through gx; in-range visited points are
// emitted as (row << 32 | point) keys (count, cap; greedy bookkeeping from sd.sink)
cudaError_t launch_graph_search(const SweepDesc& sd, const GraphIndex& gx, DeviceState* st, unsigned long long* count,
                                unsigned long long cap, int overflow_bit, bool greedy, Arena& ar, cudaStream_t s,
                                unsigned long long* visits, int* truncated);

// graph.cu
cudaError_t launch_csr_from_sorted(const unsigned long long* keys, long long nnz, long long rows,
                                   long long* offsets, int* ids, cudaStream_t s);
struct EdgeResult {
    int* edges = nullptr;
    long long n_edges = 0;
    long long pairs = 0;
};
// sorted_keys: memberships (ordinal << 32 | point) sorted; moff: their CSR row offsets (L + 1).
bool build_edges(const unsigned long long* sorted_keys, const long long* moff, long long nnz, long long n_points,
                 long long n_landmarks, Arena& ar, cudaStream_t s, EdgeResult& out, Failure& f);

// The stages of build_edges, for callers that run them over many builds with
// one host synchronisation per stage: transpose (pair counts per landmark in
// lpre), then per chunk of landmark rows emit (distinct count at *count_dev)
// and scatter, then release.
constexpr long long kEdgeChunkPairs = 1LL << 28;   // sort path: emitted pairs per chunk (32 B of scratch each)
// bitmap path: bitmap bytes per chunk (process-wide; < 0 disables the bitmap path)
long long edges_bitmap_budget();
long long edges_set_bitmap_budget(long long bytes);   // returns the previous value; 0 = default (1 GiB)
struct EdgeJob {
    const unsigned long long* keys = nullptr;   // sorted membership keys (ordinal << 32 | point)
    const long long* moff = nullptr;            // their CSR row offsets (L + 1)
    long long nnz = 0, n = 0, L = 0;
    bool bitmap = false;                        // deduplicate with a row bitmap (else by sorting)
    unsigned long long* tsorted = nullptr;     // swapped keys, sorted (stage 1 only)
    long long* toff = nullptr;                 // point -> covering landmarks (CSR)
    int* tlist = nullptr;
    int* tpos = nullptr;                       // nnz: position of membership e (row-major) in tlist
    long long* lpre = nullptr;                 // L + 1: exclusive scan of the pairs per smaller landmark
    unsigned long long* sorted = nullptr;      // sort path: sorted pair keys of the chunk
    unsigned* bits = nullptr;                  // bitmap path: rows of the chunk, W words each
    long long* pos = nullptr;                  // scan of first-of-run flags / of per-row bit counts
    const long long* count_dev = nullptr;      // distinct pairs of the chunk (device)
    int* bad = nullptr;                        // bitmap path: nonzero when an input broke a CSR invariant
};
bool edges_check(const EdgeJob& j, cudaStream_t s, Failure& f);   // synchronises; fails when *bad is set
bool edges_transpose(EdgeJob& j, Arena& ar, cudaStream_t s, Failure& f);
bool edges_choose_bitmap(long long L, long long P);   // bitmap when it is no larger than 64 bytes per pair
long long edges_bitmap_rows(long long L);              // landmark rows per bitmap chunk
bool edges_emit(EdgeJob& j, int i0, int i1, long long Pc, Arena& ar, cudaStream_t s, Failure& f);
bool edges_scatter(EdgeJob& j, int i0, int i1, long long Pc, int* dst, Arena& ar, cudaStream_t s, Failure& f);
void edges_release(EdgeJob& j, Arena& ar);

// batch.cu -- the tail of a batched build as one build over all instances
struct BatchSplit {        // one instance's share of the global results
    long long* offsets;    // rows + 1 (output)
    int* ids;              // nnz (output)
    int* edges;            // 2 n_edges (output)
    long long row_base, rows, pt_base, nnz, edge0, n_edges;
};
cudaError_t launch_gather_batch_keys(const unsigned long long* const* srcs, const long long* key_off,
                                     const long long* row_base, const long long* pt_base, int count,
                                     long long total, unsigned long long* dst, cudaStream_t s);
cudaError_t launch_edge_bounds(const int* edges, long long E, const long long* row_base, int count, long long* bounds,
                               cudaStream_t s);
cudaError_t launch_split_batch(const BatchSplit* parts, int count, const long long* goff, const int* gids,
                               const int* gedges, cudaStream_t s);

}  // namespace bm
