// bm_api.cu -- the C-ABI of libballmapper: argument checks, buffer management,
// phase orchestration on the caller's stream, and error reporting.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "bm_host.h"

namespace bm {

thread_local std::string g_last_error;
thread_local long long g_kernel_launches = 0;

void device_free(const bm_options* opt, cudaStream_t s, void* p) {
    if (!p) return;
    if (opt && opt->free) opt->free(p, (void*)s, opt->alloc_ctx);
    else cudaFreeAsync(p, s);
}

// Identifier of the current CUDA context (0 when the driver cannot report one).
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (PFN_cuCtxGetCurrent_v4000)p;
        else
            cudaGetLastError();
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PFN_cuCtxGetId_v12000)p;
        else
            cudaGetLastError();
        looked_up = true;
    }
    if (!get_current || !get_id) return 0ull;
    CUcontext ctx = nullptr;
    unsigned long long id = 0ull;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0ull;
    return id;
}


namespace {
// The library's own stream-ordered pool per device (used when the caller gives no
// allocator).  It keeps up to kPoolKeepBytes of freed memory mapped across
// synchronisations, so that a call does not map its scratch afresh after the previous
// call's memory went back to the driver (the default pool keeps nothing).  Keyed on the
// context, like any device resource: a context created after a reset gets its own pool.
constexpr unsigned long long kPoolKeepBytes = 64ull << 30;
std::mutex g_pool_mu;
std::vector<std::pair<unsigned long long, cudaMemPool_t>> g_pools;   // (context id, pool)

cudaMemPool_t library_pool() {
    const unsigned long long id = current_context_id();
    if (id == 0) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto& e : g_pools)
        if (e.first == id) return e.second;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    unsigned long long keep = kPoolKeepBytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaGetLastError();
    g_pools.emplace_back(id, pool);
    return pool;
}
}  // namespace

Arena::~Arena() {
    for (void* p : ptrs_) device_free(opt_, stream_, p);
    for (void* p : slabs_) device_free(opt_, stream_, p);
}

void* Arena::raw(size_t bytes) {
    void* p = nullptr;
    if (opt_ && opt_->alloc) {
        p = opt_->alloc(bytes, (void*)stream_, opt_->alloc_ctx);
    } else if (cudaMemPool_t pool = library_pool()) {
        if (cudaMallocFromPoolAsync(&p, bytes, pool, stream_) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    } else if (cudaMallocAsync(&p, bytes, stream_) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void* Arena::get(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    if (slab_ && bytes <= kSlabMax) {
        if (bytes > left_) {
            const size_t block = std::max(bytes, next_);
            char* b = (char*)raw(block);
            if (!b) return nullptr;
            slabs_.push_back(b);
            cur_ = b;
            left_ = block;
            next_ = std::min<size_t>(2 * next_, 64u << 20);
        }
        void* p = cur_;
        cur_ += bytes;
        left_ -= bytes;
        return p;
    }
    return get_standalone(bytes);
}

void* Arena::get_standalone(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    void* p = raw(bytes);
    if (p) ptrs_.push_back(p);
    return p;
}

void Arena::release(void* p) {
    if (!p) return;
    auto it = std::find(ptrs_.begin(), ptrs_.end(), p);
    if (it != ptrs_.end()) {
        ptrs_.erase(it);
        device_free(opt_, stream_, p);
    }
}

bool Arena::take(void* p) {
    auto it = std::find(ptrs_.begin(), ptrs_.end(), p);
    if (it == ptrs_.end()) return false;
    ptrs_.erase(it);
    return true;
}

namespace {

struct Call {
    bm_options opt;
    cudaStream_t stream;
};

bm_status fail(bm_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

#define TRY_CUDA(expr)                                                                  \
    do {                                                                                \
        cudaError_t e__ = (expr);                                                       \
        if (e__ != cudaSuccess) {                                                       \
            cudaGetLastError();                                                         \
            return fail(e__ == cudaErrorMemoryAllocation ? BM_ERR_NOMEM : BM_ERR_CUDA,  \
                        std::string(#expr) + ": " + cudaGetErrorString(e__));           \
        }                                                                               \
    } while (0)

// Synchronise with the stream; a failure names the stage whose work was in flight.
#define TRY_SYNC(stream, stage)                                                         \
    do {                                                                                \
        cudaError_t e__ = cudaStreamSynchronize(stream);                                \
        if (e__ != cudaSuccess) {                                                       \
            cudaGetLastError();                                                         \
            return fail(BM_ERR_CUDA, std::string("after ") + (stage) + ": " + cudaGetErrorString(e__)); \
        }                                                                               \
    } while (0)

#define ALLOC(ptr, type, count)                                                         \
    do {                                                                                \
        ptr = (type*)ar.get(sizeof(type) * (size_t)(count));                           \
        if (!ptr) return fail(BM_ERR_NOMEM, "allocation of " #ptr " failed (" +         \
                                                std::to_string(sizeof(type) * (size_t)(count)) + " bytes)"); \
    } while (0)

bm_status check_device(int path) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BM_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3)
        return fail(BM_ERR_UNSUPPORTED, "libballmapper is built for sm_103 (GB300); device is sm_" +
                                            std::to_string(major) + std::to_string(minor));
    if (path != BM_PATH_FP32 && path != BM_PATH_TC_SPLIT3 && path != BM_PATH_TC_FP16 && path != BM_PATH_TC_AUTO)
        return fail(BM_ERR_ARG, "unknown path");
    return BM_OK;
}

bm_status validate_points(const float* X, long long n, int d, const char* name) {
    if (n < 0 || n > 0x7fffffffLL) return fail(BM_ERR_ARG, std::string(name) + ": row count out of range [0, 2^31-1]");
    if (d < 1 || d > 65536) return fail(BM_ERR_ARG, "d out of range [1, 65536]");
    if (n > 0 && X == nullptr) return fail(BM_ERR_ARG, std::string(name) + " is NULL");
    return BM_OK;
}

// Largest greedy batch of a single build (the resolve kernel's conflict walk holds 16384
// candidates).
constexpr int kMaxBatch = 16384;

bm_status validate_centring(int c) {
    if (c != BM_CENTRE_AUTO && c != BM_CENTRE_ALWAYS && c != BM_CENTRE_OFF)
        return fail(BM_ERR_ARG, "centring must be BM_CENTRE_AUTO, BM_CENTRE_ALWAYS or BM_CENTRE_OFF");
    return BM_OK;
}

bm_status validate_eps(float eps) {
    if (!std::isfinite(eps) || !(eps > 0.f)) return fail(BM_ERR_ARG, "eps must be finite and > 0");
    return BM_OK;
}

// Largest greedy batch: 0 (the default) or a multiple of 32 in [32, max].
bm_status validate_batch(int S, int max) {
    if (S != 0 && (S < 32 || S > max || S % 32))
        return fail(BM_ERR_ARG, "batch must be a multiple of 32 in [32, " + std::to_string(max) + "]");
    return BM_OK;
}

struct Timer {
    cudaEvent_t ev[8];
    int used = 0;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {
        for (auto& e : ev) e = nullptr;
    }
    ~Timer() {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
    void mark() {
        if (used < 8 && cudaEventCreate(&ev[used]) == cudaSuccess) {
            cudaEventRecord(ev[used], s);
            ++used;
        }
    }
    double ms(int a, int b) {
        if (a >= used || b >= used) return 0.0;
        float t = 0.f;
        cudaEventSynchronize(ev[b]);
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
};

// Copy `bytes` of device memory into a fresh host buffer (malloc).
bool to_host(void** dst, const void* src, size_t bytes, cudaStream_t s) {
    *dst = std::malloc(bytes ? bytes : 1);
    if (!*dst) return false;
    if (bytes && cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
    return true;
}

const float* stage_input(const float* X, long long rows, int d, bool host_io, Arena& ar, cudaStream_t s,
                         bm_status* st) {
    *st = BM_OK;
    if (!host_io || rows == 0) return X;
    float* dX = (float*)ar.get(sizeof(float) * (size_t)rows * d);
    if (!dX) {
        *st = fail(BM_ERR_NOMEM, "device copy of host input failed to allocate");
        return nullptr;
    }
    if (cudaMemcpyAsync(dX, X, sizeof(float) * (size_t)rows * d, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        *st = fail(BM_ERR_CUDA, "host to device copy failed");
        return nullptr;
    }
    return dX;
}

bool is_tc_path(int path) { return path == BM_PATH_TC_SPLIT3 || path == BM_PATH_TC_FP16; }

float float_from_bits(unsigned u) {
    float f;
    std::memcpy(&f, &u, sizeof(f));
    return f;
}

int prec_for(int path) {
    return path == BM_PATH_TC_SPLIT3 ? kPrecSplit : (path == BM_PATH_TC_FP16 ? kPrecFp16 : kPrecNone);
}

// Allocate and fill the tile operands of one point set: phi and norms always; the
// bf16 split (kPrecSplit) here; the fp16 operands (kPrecFp16) only once the scale
// is known (finish_fp16, after the norms have been read back).
bm_status prepare(const float* x, long long rows, int d, double eps2, bool a_side, int prec, Arena& ar,
                  unsigned* max_norm_bits, int* bad, cudaStream_t s, Prepared& p, const double* row_r2 = nullptr,
                  const float* centre = nullptr) {
    p.x = x;
    p.rows = rows;
    p.d = d;
    p.prec = prec;
    p.centre = prec != kPrecNone ? centre : nullptr;
    const TileConfig tcfg = tile_config_for(d, prec == kPrecFp16 ? 1 : 3);
    p.d_pad = tcfg.d_pad;
    p.ck = tcfg.ck;
    p.nt = tcfg.nt;
    p.bbuf = tcfg.bbuf;
    p.astg = tcfg.astg;
    ALLOC(p.phi, float, std::max<long long>(rows, 1));
    if (prec != kPrecNone) {
        ALLOC(p.hi, __nv_bfloat16, std::max<long long>(rows, 1) * p.d_pad);   // bf16 or fp16 bits
        ALLOC(p.aug, __nv_bfloat16, std::max<long long>(rows, 1) * 16);
    }
    if (prec == kPrecSplit) ALLOC(p.lo, __nv_bfloat16, std::max<long long>(rows, 1) * p.d_pad);
    TRY_CUDA(launch_prep(x, rows, d, eps2, a_side, prec == kPrecSplit, p, max_norm_bits, bad, s, row_r2));
    return BM_OK;
}

// Centre of the tensor-core operands of a call over the points x (null: none), as
// opt.centring asks; the device's choice lands in st->centred.  Lives in the call's arena.
constexpr long long kCentreMinRows = 65536;

bm_status operand_centre(const float* x, long long rows, int d, const bm_options& opt, DeviceState* st, Arena& ar,
                         cudaStream_t s, const float** centre) {
    *centre = nullptr;
    if (opt.centring == BM_CENTRE_OFF || rows <= 0 || d > 512) return BM_OK;   // the tiles take d <= 512
    if (opt.centring != BM_CENTRE_ALWAYS && rows < kCentreMinRows) return BM_OK;
    float* c;
    double* partial;
    unsigned* maxima;
    ALLOC(c, float, d);
    ALLOC(partial, double, (long long)kCentreBlocks * d);
    ALLOC(maxima, unsigned, 2);
    TRY_CUDA(launch_centre(x, rows, d, opt.centring == BM_CENTRE_ALWAYS, partial, maxima, c, &st->centred, s));
    *centre = c;
    return BM_OK;
}

// After the norms are known on the host: fp16 operands at the chosen scale (fp16 path
// only), the band half-width, and the per-row delta' entries of both sides'
// augmentation (tensor-core paths).  pts: the B side (points); qry: the A side
// (queries), or null.
bm_status finish_prep(DeviceState* st, int path, int d, double eps2, double eps, bool same_sets, float max_norm,
                      Prepared* pts, Prepared* qry, cudaStream_t s) {
    int e = 0;
    if (path == BM_PATH_TC_FP16) {
        e = fp16_scale_exp((double)max_norm, eps);
        TRY_CUDA(launch_prep16(pts->x, pts->rows, d, eps2, false, e, *pts, s));
        if (qry) TRY_CUDA(launch_prep16(qry->x, qry->rows, d, eps2, true, e, *qry, s));
    }
    TRY_CUDA(launch_delta(st, path, d, pts->d_pad, eps2, same_sets, s, e));
    if (pts->prec != kPrecNone) TRY_CUDA(launch_set_aug_delta(st, *pts, eps2, false, s));
    if (qry && qry->prec != kPrecNone) TRY_CUDA(launch_set_aug_delta(st, *qry, eps2, true, s));
    return BM_OK;
}

bm_status run_sweep(const SweepDesc& sd, int path, cudaStream_t s, int* grid) {
    *grid = 0;
    if (path == BM_PATH_FP32) {
        TRY_CUDA(launch_sweep_fp32(sd, s));
        return BM_OK;
    }
    std::string why;
    cudaError_t e = launch_sweep_tc(sd, s, &why, grid);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BM_ERR_CUDA, "tensor-core sweep: " + why + " (" + cudaGetErrorString(e) + ")");
    }
    return BM_OK;
}

// Hit and band-pair buffers of one sweep.  The tensor-core tiles write per-CTA
// segments (raw, raw_band) that are compacted into keys / band; the FP32 tiles
// write keys / band directly.
struct SweepOut {
    unsigned long long* keys = nullptr;
    unsigned long long* band = nullptr;
    unsigned long long* raw = nullptr;
    unsigned long long* raw_band = nullptr;
    unsigned long long* seg_counts = nullptr;
    unsigned long long* band_seg_counts = nullptr;
    unsigned long long cap = 0;
};

bm_status alloc_sweep_out(Arena& ar, bool tc, unsigned long long cap, int sms, SweepOut& o) {
    o.cap = cap;
    ALLOC(o.keys, unsigned long long, cap);
    ALLOC(o.band, unsigned long long, cap);
    if (tc) {
        ALLOC(o.raw, unsigned long long, cap);
        ALLOC(o.raw_band, unsigned long long, cap);
        ALLOC(o.seg_counts, unsigned long long, sms);
        ALLOC(o.band_seg_counts, unsigned long long, sms);
    }
    return BM_OK;
}

void release_sweep_out(Arena& ar, SweepOut& o, bool keep_keys) {
    if (!keep_keys) ar.release(o.keys);
    ar.release(o.band);
    ar.release(o.raw);
    ar.release(o.raw_band);
    ar.release(o.seg_counts);
    ar.release(o.band_seg_counts);
    o = SweepOut();
}

struct SweepTimer;

}  // namespace
}  // namespace bm

namespace bm {
namespace {

struct HostState {
    DeviceState* pinned = nullptr;
    HostState() {
        if (cudaMallocHost(&pinned, sizeof(DeviceState)) != cudaSuccess) {
            cudaGetLastError();
            pinned = nullptr;
        }
    }
    ~HostState() {
        if (pinned) cudaFreeHost(pinned);
    }
};

// Device time of the distance-tile launches: an event pair around each launch,
// summed whenever the host synchronises with the stream anyway.
struct SweepTimer {
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    double ms = 0.0;
    long long launches = 0;
    cudaStream_t s;
    bool on = true;   // off while a stream is being captured into a graph
    explicit SweepTimer(cudaStream_t st) : s(st) {}
    ~SweepTimer() {
        for (auto e : ev) cudaEventDestroy(e);
    }
    void mark() {
        if (!on) return;
        if (used == ev.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return;
            }
            ev.push_back(e);
        }
        cudaEventRecord(ev[used++], s);
    }
    void before() { mark(); }
    void after() {
        mark();
        ++launches;
    }
    void collect() {  // the stream has been synchronised
        for (size_t i = 0; i + 1 < used; i += 2) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ev[i], ev[i + 1]) == cudaSuccess) ms += t;
            else cudaGetLastError();
        }
        used = 0;
    }
};

// One distance sweep: tiles, compaction of the per-CTA segments (tensor-core
// path), FP64 recheck of the band pairs.  sd.sink must already carry the
// greedy bookkeeping (or none) and the statistics pointers.  Hits end up in
// o.keys with their number in *count.
bm_status ivf_sweep(SweepDesc& sd, DeviceState* st, Arena& ar, bool greedy, cudaStream_t s) {
    const IvfIndex& ix = *sd.ivf;
    const long long rows_max = sd.a_rows_max;
    int* probes = sd.ivf_probes_out;
    if (!probes) ALLOC(probes, int, std::max<long long>(rows_max * sd.nprobe, 1));
    long long *cnt, *cq_off, *tile_off;
    int* cq_rows;
    ALLOC(cnt, long long, ix.nlist + 1);
    ALLOC(cq_off, long long, ix.nlist + 1);
    ALLOC(tile_off, long long, ix.nlist + 1);
    ALLOC(cq_rows, int, std::max<long long>(rows_max * sd.nprobe, 1));
    TRY_CUDA(launch_probe_select(sd.a->x, rows_max, sd.a_rows_dev, ix, sd.nprobe, probes, s));
    TRY_CUDA(launch_group_probes(probes, rows_max, sd.a_rows_dev, sd.nprobe, ix, cnt, cq_off, cq_rows, tile_off, ar,
                                 s));
    TRY_CUDA(launch_ivf_scan(sd.a->x, sd.a->phi, ix, sd.ivf_phi_perm, cq_off, cq_rows, tile_off, st, greedy, sd.sink,
                             s));
    ar.release(cq_rows);
    ar.release(tile_off);
    ar.release(cq_off);
    ar.release(cnt);
    if (probes != sd.ivf_probes_out) ar.release(probes);
    return BM_OK;
}

// The inverted-file scan on the tensor-core tiles: queries grouped by probed cell, both
// sides laid out by cell in whole tiles, the tile kernel in table mode (one item = a
// cell's point tile against a group of its query tiles), then the usual compaction and
// FP64 recheck of the band pairs (keys hold query and point ids).
bm_status ivf_sweep_tc(SweepDesc& sd, DeviceState* st, int path, SweepOut& o, unsigned long long* count,
                       int overflow_bit, bool greedy, int sms, SweepTimer& stimer, cudaStream_t s, Arena& ar) {
    const IvfIndex& ix = *sd.ivf;
    const Prepared& bp = *sd.ivf_b_pad;
    const long long rows_max = sd.a_rows_max;
    int* probes = sd.ivf_probes_out;
    if (!probes) ALLOC(probes, int, std::max<long long>(rows_max * sd.nprobe, 1));
    long long *cnt, *cq_off, *tile_off, *pa_off, *item_off;
    int *cq_rows, *a_map;
    ALLOC(cnt, long long, ix.nlist + 1);
    ALLOC(cq_off, long long, ix.nlist + 1);
    ALLOC(tile_off, long long, ix.nlist + 1);
    ALLOC(pa_off, long long, ix.nlist + 1);
    ALLOC(item_off, long long, ix.nlist + 1);
    ALLOC(cq_rows, int, std::max<long long>(rows_max * sd.nprobe, 1));
    TRY_CUDA(launch_probe_select(sd.a->x, rows_max, sd.a_rows_dev, ix, sd.nprobe, probes, s));
    TRY_CUDA(launch_group_probes(probes, rows_max, sd.a_rows_dev, sd.nprobe, ix, cnt, cq_off, cq_rows, tile_off, ar,
                                 s));
    // padded query operands: every (query, probe) pair plus at most 127 padding rows per cell
    Prepared apad = *sd.a;
    apad.rows = rows_max * sd.nprobe + 127LL * ix.nlist;
    ALLOC(apad.hi, __nv_bfloat16, apad.rows * apad.d_pad);
    apad.lo = nullptr;
    if (sd.a->lo) ALLOC(apad.lo, __nv_bfloat16, apad.rows * apad.d_pad);
    ALLOC(apad.aug, __nv_bfloat16, apad.rows * 16);
    ALLOC(a_map, int, apad.rows);
    const int NT = bp.nt;
    const long long bmax = ix.max_cell_tiles * (256 / NT);
    const long long item_cap = bmax * ((rows_max * sd.nprobe / 128 + ix.nlist) / 16 + 1) + ix.npad / NT + 1;
    TcItem* items;
    ALLOC(items, TcItem, item_cap);
    TRY_CUDA(launch_ivf_tc_layout(ix, NT, cq_off, cq_rows, *sd.a, apad, a_map, pa_off, cnt, items, item_off, ar, s));
    SweepDesc sd2 = sd;
    sd2.a = &apad;
    sd2.b = &bp;
    sd2.a_rows_max = apad.rows;
    sd2.a_rows_dev = nullptr;
    sd2.ivf = nullptr;
    sd2.tc_items = items;
    sd2.tc_items_count = item_off + ix.nlist;
    sd2.tc_a_map = a_map;
    sd2.tc_b_ids = ix.cell_ids;
    sd2.sink.count = count;
    sd2.sink.cap = o.cap;
    sd2.sink.band_n = &st->band_n;
    sd2.sink.band_cap = o.cap;
    sd2.sink.keys = o.raw;
    sd2.sink.band_keys = o.raw_band;
    sd2.sink.seg_counts = o.seg_counts;
    sd2.sink.band_seg_counts = o.band_seg_counts;
    sd2.sink.seg_cap = o.cap / sms;
    stimer.before();
    int grid = 0;
    bm_status rs = run_sweep(sd2, path, s, &grid);
    stimer.after();
    if (rs != BM_OK) return rs;
    TRY_CUDA(launch_compact_segments(o.raw, o.raw_band, sd2.sink.seg_cap, o.seg_counts, o.band_seg_counts, grid, o.keys,
                                     o.band, count, &st->band_n, st, overflow_bit, greedy, greedy, s));
    TRY_CUDA(launch_band_recheck(st, o.band, o.cap, sd.a->x, ix.X, ix.d, sd.eps2, o.keys, count, o.cap, sd.sink,
                                 greedy, overflow_bit, greedy, s));
    ar.release(items);
    ar.release(a_map);
    ar.release(apad.aug);
    ar.release(apad.lo);
    ar.release(apad.hi);
    ar.release(cq_rows);
    ar.release(item_off);
    ar.release(pa_off);
    ar.release(tile_off);
    ar.release(cq_off);
    ar.release(cnt);
    if (probes != sd.ivf_probes_out) ar.release(probes);
    return BM_OK;
}

bm_status sweep_stage(SweepDesc& sd, DeviceState* st, int path, SweepOut& o, unsigned long long* count,
                      int overflow_bit, bool greedy, int sms, SweepTimer& stimer, cudaStream_t s, Arena& ar) {
    if (sd.gidx) {   // proximity-graph search: exact decisions on the visited points, no band
        sd.sink.keys = o.keys;
        sd.sink.count = count;
        sd.sink.cap = o.cap;
        sd.sink.seg_counts = nullptr;
        sd.sink.band_seg_counts = nullptr;
        stimer.before();
        const cudaError_t e = launch_graph_search(sd, *sd.gidx, st, count, o.cap, overflow_bit, greedy, ar, s,
                                                  &st->tile_pairs, &st->gidx_truncated);
        stimer.after();
        TRY_CUDA(e);
        return BM_OK;
    }
    if (sd.ivf && sd.ivf_b_pad) {   // inverted-file scan on the tensor-core tiles
        return ivf_sweep_tc(sd, st, path, o, count, overflow_bit, greedy, sms, stimer, s, ar);
    }
    if (sd.ivf) {   // inverted-file scan: FP32 tiles over the probed cells, global counters
        sd.sink.count = count;
        sd.sink.cap = o.cap;
        sd.sink.band_n = &st->band_n;
        sd.sink.band_cap = o.cap;
        sd.sink.keys = o.keys;
        sd.sink.band_keys = o.band;
        sd.sink.seg_counts = nullptr;
        sd.sink.band_seg_counts = nullptr;
        stimer.before();
        bm_status rs = ivf_sweep(sd, st, ar, greedy, s);
        stimer.after();
        if (rs != BM_OK) return rs;
        TRY_CUDA(launch_band_recheck(st, o.band, o.cap, sd.a->x, sd.ivf->X, sd.ivf->d, sd.eps2, o.keys, count, o.cap,
                                     sd.sink, greedy, overflow_bit, greedy, s));
        return BM_OK;
    }
    const bool tc = is_tc_path(path);
    sd.sink.count = count;
    sd.sink.cap = o.cap;
    sd.sink.band_n = &st->band_n;
    sd.sink.band_cap = o.cap;
    if (tc) {
        sd.sink.keys = o.raw;
        sd.sink.band_keys = o.raw_band;
        sd.sink.seg_counts = o.seg_counts;
        sd.sink.band_seg_counts = o.band_seg_counts;
        sd.sink.seg_cap = o.cap / sms;
    } else {
        sd.sink.keys = o.keys;
        sd.sink.band_keys = o.band;
        sd.sink.seg_counts = nullptr;
        sd.sink.band_seg_counts = nullptr;
        sd.sink.seg_cap = 0;
    }
    stimer.before();
    int grid = 0;
    bm_status rs = run_sweep(sd, path, s, &grid);
    stimer.after();
    if (rs != BM_OK) return rs;
    if (tc) {
        TRY_CUDA(launch_compact_segments(o.raw, o.raw_band, sd.sink.seg_cap, o.seg_counts, o.band_seg_counts, grid,
                                         o.keys, o.band, count, &st->band_n, st, overflow_bit, greedy, greedy, s));
    }
    TRY_CUDA(launch_band_recheck(st, o.band, o.cap, sd.a->x, sd.b->x, sd.b->d, sd.eps2, o.keys, count, o.cap, sd.sink,
                                 greedy, overflow_bit, greedy, s, sd.row_eps2));
    return BM_OK;
}

bm_status read_state(const DeviceState* dst, HostState& hs, DeviceState& out, cudaStream_t s) {
    if (!hs.pinned) return fail(BM_ERR_NOMEM, "pinned state buffer");
    TRY_CUDA(cudaMemcpyAsync(hs.pinned, dst, sizeof(DeviceState), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    out = *hs.pinned;
    return BM_OK;
}

// Reported distances of a CSR (want_dists): allocates *dists and a device error slot
// (*err_dev, zeroed), launches the kernel; the error is read later with read_err.
bm_status csr_dists(Arena& ar, cudaStream_t s, const float* qx, const int* qidx, const float* X, int d,
                    const long long* offsets, long long rows, const int* ids, long long nnz, float** dists,
                    unsigned long long** err_dev) {
    ALLOC(*dists, float, std::max<long long>(nnz, 1));
    ALLOC(*err_dev, unsigned long long, 1);
    TRY_CUDA(cudaMemsetAsync(*err_dev, 0, sizeof(unsigned long long), s));
    TRY_CUDA(launch_member_dists(qx, qidx, X, d, offsets, rows, ids, nnz, *dists, *err_dev, s));
    return BM_OK;
}

bm_status read_err(const unsigned long long* err_dev, cudaStream_t s, double* out) {
    *out = 0.0;
    if (!err_dev) return BM_OK;
    unsigned long long bits = 0;
    TRY_CUDA(cudaMemcpyAsync(&bits, err_dev, sizeof(bits), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    std::memcpy(out, &bits, sizeof(double));
    return BM_OK;
}

// The greedy + membership part of bm_build.  Returns BM_OK with *retry set when
// a buffer was too small (capacities are updated for the next attempt).
// Buffers and sweep description of one greedy build.
struct GreedyCtx {
    GreedyBuffers g;
    SweepOut so;
    SweepDesc sd;
    int S = 0, sms = 0, path = 0;
    bool tc = false;
    // automatic path: the first step runs on the bf16 split; its band rate, scaled by
    // the ratio of the two paths' proven band widths, predicts the fp16 band; the
    // greedy moves to fp16 when that prediction is small and back (once) when the
    // measured fp16 band is not
    bool auto_switch = false;
    int auto_phase = 0;              // 0: deciding on the split, 1: on fp16, watching, 2: settled
    double eps2 = 0.0, eps = 0.0;
    std::vector<int> switches;       // greedy steps at which the path changed
    unsigned long long band0 = 0, pairs0 = 0;
};

// Band pairs per tile pair above which the fp16 tiles lose to the split: a band
// pair costs an FP64 distance (~0.35-0.7 ns at d = 64-128 on GB300), while the fp16
// tiles save ~0.1 ps per pair.
constexpr double kAutoBandFraction = 2e-4;
constexpr double kAutoPredictFraction = 5e-5;   // move to fp16 below this predicted rate

bm_status greedy_setup(const Prepared& pts, double eps2, int path, int S, Arena& ar, cudaStream_t s, DeviceState* st,
                       unsigned long long step_cap, unsigned long long mem_cap, const IvfIndex* ivf,
                       const float* phi_perm, int nprobe, GreedyCtx& c) {
    const long long n = pts.rows;
    const int d = pts.d;
    const bool tc = is_tc_path(path);
    c.S = S;
    c.path = path;
    c.tc = tc;
    c.eps2 = eps2;
    c.eps = std::sqrt(eps2);
    GreedyBuffers& g = c.g;
    g.st = st;
    const long long words_n = (n + 31) / 32;
    const int words = S / 32;
    ALLOC(g.covered, unsigned, words_n);
    TRY_CUDA(cudaMemsetAsync(g.covered, 0, sizeof(unsigned) * words_n, s));
    ALLOC(g.slot_of, int, n);
    TRY_CUDA(cudaMemsetAsync(g.slot_of, 0xff, sizeof(int) * n, s));
    ALLOC(g.cand_ids, int, S);
    ALLOC(g.ordinal, int, S);
    ALLOC(g.conflict, unsigned, (long long)S * words);
    TRY_CUDA(cudaMemsetAsync(g.conflict, 0, sizeof(unsigned) * S * words, s));
    ALLOC(g.row_any, unsigned, words);
    TRY_CUDA(cudaMemsetAsync(g.row_any, 0, sizeof(unsigned) * words, s));
    ALLOC(g.landmarks, int, n);
    float* cx;
    ALLOC(cx, float, (long long)S * d);
    g.cand.x = cx;
    g.cand.rows = S;
    g.cand.d = d;
    g.cand.d_pad = pts.d_pad;
    g.cand.ck = pts.ck;
    g.cand.nt = pts.nt;
    g.cand.bbuf = pts.bbuf;
    g.cand.astg = pts.astg;
    g.cand.prec = pts.prec;
    g.cand.scale_exp = pts.scale_exp;
    ALLOC(g.cand.phi, float, S);
    if (tc) {
        ALLOC(g.cand.hi, __nv_bfloat16, (long long)S * pts.d_pad);
        ALLOC(g.cand.aug, __nv_bfloat16, (long long)S * 16);
        TRY_CUDA(cudaMemsetAsync(g.cand.hi, 0, sizeof(__nv_bfloat16) * S * pts.d_pad, s));
        TRY_CUDA(cudaMemsetAsync(g.cand.aug, 0, sizeof(__nv_bfloat16) * S * 16, s));
        if (pts.prec == kPrecSplit) {
            ALLOC(g.cand.lo, __nv_bfloat16, (long long)S * pts.d_pad);
            TRY_CUDA(cudaMemsetAsync(g.cand.lo, 0, sizeof(__nv_bfloat16) * S * pts.d_pad, s));
        }
    }
    c.sms = device_sm_count();
    bm_status ars = alloc_sweep_out(ar, tc, step_cap, c.sms, c.so);
    if (ars != BM_OK) return ars;
    g.step_keys = c.so.keys;
    g.step_cap = step_cap;
    ALLOC(g.mem_keys, unsigned long long, mem_cap);
    g.mem_cap = mem_cap;

    SweepDesc& sd = c.sd;
    sd = SweepDesc();
    sd.a = &g.cand;
    sd.b = &pts;
    sd.a_rows_max = S;
    sd.a_rows_dev = &st->cand_count;
    sd.st = st;
    sd.check_done = true;
    sd.eps2 = eps2;
    sd.sink.slot_of = g.slot_of;
    sd.sink.conflict = g.conflict;
    sd.sink.row_any = g.row_any;
    sd.sink.conflict_words = words;
    sd.sink.band_count = &st->band_pairs;
    sd.sink.pair_count = &st->tile_pairs;
    sd.ivf = ivf;
    sd.ivf_phi_perm = phi_perm;
    sd.nprobe = nprobe;
    return BM_OK;
}

// One greedy step: select, gather, sweep (+ compaction and recheck), resolve, apply.
// Only kernel launches, so the step can also be captured into a graph body.
bm_status greedy_enqueue_step(GreedyCtx& c, const Prepared& pts, Arena& ar, SweepTimer& stimer, cudaStream_t s) {
    DeviceState* st = c.g.st;
    TRY_CUDA(launch_greedy_select(c.g, pts, c.S, c.tc, s));
    TRY_CUDA(launch_greedy_gather(c.g, pts, c.S, c.tc, s));
    bm_status rs = sweep_stage(c.sd, st, c.path, c.so, &st->step_hits, kErrStepOverflow, true, c.sms, stimer, s, ar);
    if (rs != BM_OK) return rs;
    TRY_CUDA(launch_greedy_resolve(c.g, c.S, s));
    TRY_CUDA(launch_greedy_apply(c.g, s));
    return BM_OK;
}

// Host-driven greedy loop: enqueue steps in growing chunks, read the state, grow
// an overflowing buffer and redo the step, until no uncovered point remains.
// With resume set the first state read comes before any new step (the steps so
// far ran elsewhere, e.g. in a graph).
// Move a greedy in progress to another tensor-core representation: new operands
// of the points (replacing the old ones), candidate operand rows to match, the new
// band half-width and the points' per-row delta' entries.  Every step is exact on either
// path.
bm_status switch_path(GreedyCtx& c, Prepared& pts, Arena& ar, cudaStream_t s, int to, float max_norm, int step) {
    DeviceState* st = c.g.st;
    Prepared p2;
    int e = 0;
    if (to == BM_PATH_TC_SPLIT3) {
        int* bad;
        ALLOC(bad, int, 1);
        TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
        bm_status rs = prepare(pts.x, pts.rows, pts.d, c.eps2, false, kPrecSplit, ar, &st->max_norm_bits, bad, s, p2,
                               nullptr, pts.centre);
        if (rs != BM_OK) return rs;
        ar.release(pts.phi);
    } else {
        p2 = pts;   // same rows, phi and norms
        p2.prec = kPrecFp16;
        const TileConfig t = tile_config_for(pts.d, 1);
        p2.d_pad = t.d_pad;
        p2.ck = t.ck;
        p2.nt = t.nt;
        p2.bbuf = t.bbuf;
        p2.astg = t.astg;
        p2.lo = nullptr;
        ALLOC(p2.hi, __nv_bfloat16, std::max<long long>(pts.rows, 1) * p2.d_pad);
        ALLOC(p2.aug, __nv_bfloat16, std::max<long long>(pts.rows, 1) * 16);
        e = fp16_scale_exp((double)max_norm, c.eps);
        TRY_CUDA(launch_prep16(p2.x, p2.rows, p2.d, c.eps2, false, e, p2, s));
    }
    ar.release(pts.hi);
    ar.release(pts.lo);
    ar.release(pts.aug);
    pts = p2;   // c.sd.b points at pts
    const int S = c.S;
    Prepared& cand = c.g.cand;
    ar.release(cand.hi);
    ar.release(cand.lo);
    ar.release(cand.aug);
    cand.lo = nullptr;
    ALLOC(cand.hi, __nv_bfloat16, (long long)S * pts.d_pad);
    ALLOC(cand.aug, __nv_bfloat16, (long long)S * 16);
    TRY_CUDA(cudaMemsetAsync(cand.hi, 0, sizeof(__nv_bfloat16) * S * pts.d_pad, s));
    TRY_CUDA(cudaMemsetAsync(cand.aug, 0, sizeof(__nv_bfloat16) * S * 16, s));
    if (to == BM_PATH_TC_SPLIT3) {
        ALLOC(cand.lo, __nv_bfloat16, (long long)S * pts.d_pad);
        TRY_CUDA(cudaMemsetAsync(cand.lo, 0, sizeof(__nv_bfloat16) * S * pts.d_pad, s));
    }
    cand.d_pad = pts.d_pad;
    cand.ck = pts.ck;
    cand.nt = pts.nt;
    cand.bbuf = pts.bbuf;
    cand.astg = pts.astg;
    cand.prec = pts.prec;
    cand.scale_exp = pts.scale_exp;
    TRY_CUDA(launch_delta(st, to, pts.d, pts.d_pad, c.eps2, true, s, e));
    TRY_CUDA(launch_set_aug_delta(st, pts, c.eps2, false, s));
    c.path = to;
    c.switches.push_back(step);
    return BM_OK;
}

bm_status greedy_drive(GreedyCtx& c, Prepared& pts, Arena& ar, cudaStream_t s, HostState& hs,
                       unsigned long long& step_cap, unsigned long long& mem_cap, DeviceState& h,
                       SweepTimer& stimer, bool resume) {
    GreedyBuffers& g = c.g;
    DeviceState* st = g.st;
    // the automatic path looks at the band after the first step already
    int chunk = c.auto_switch ? 1 : 2;
    int regrows = 0;
    bool enqueue = !resume;
    while (true) {
        for (int i = 0; enqueue && i < chunk; ++i) {
            bm_status rs = greedy_enqueue_step(c, pts, ar, stimer, s);
            if (rs != BM_OK) return rs;
        }
        enqueue = true;
        bm_status rs = read_state(st, hs, h, s);
        if (rs != BM_OK) return rs;
        stimer.collect();
        if (h.error & kErrTimeout) return fail(BM_ERR_TIMEOUT, "a bounded device wait expired in the distance tiles");
        if (h.error & kErrLoopLimit) return fail(BM_ERR_CUDA, "device-side greedy loop passed its iteration bound");
        if (h.error & (kErrStepOverflow | kErrMemberOverflow)) {
            // a step stopped before committing anything: grow the buffer and redo it
            if (++regrows > 64) return fail(BM_ERR_CAPACITY, "greedy buffers kept overflowing");
            if (h.error & kErrStepOverflow) {
                const unsigned long long need =
                    std::max<unsigned long long>(h.max_seg * (unsigned long long)c.sms,
                                                 std::max(h.step_hits, h.band_n)) * 3 / 2;
                step_cap = std::max<unsigned long long>(need, 2 * step_cap);
                release_sweep_out(ar, c.so, false);
                bm_status rs2 = alloc_sweep_out(ar, c.tc, step_cap, c.sms, c.so);
                if (rs2 != BM_OK) return rs2;
                g.step_keys = c.so.keys;
                g.step_cap = step_cap;
            }
            if (h.error & kErrMemberOverflow) {
                const unsigned long long need = std::max<unsigned long long>(2 * mem_cap, (h.mem_count + h.step_hits) * 3 / 2);
                unsigned long long* nk;
                ALLOC(nk, unsigned long long, need);
                if (h.mem_count)
                    TRY_CUDA(cudaMemcpyAsync(nk, g.mem_keys, sizeof(unsigned long long) * h.mem_count,
                                             cudaMemcpyDeviceToDevice, s));
                ar.release(g.mem_keys);
                g.mem_keys = nk;
                g.mem_cap = mem_cap = need;
            }
            TRY_CUDA(launch_greedy_rollback(g, s));
            continue;
        }
        if (h.done) break;
        if (c.auto_switch && c.auto_phase < 2) {
            const unsigned long long db = h.band_pairs - c.band0, dp = h.tile_pairs - c.pairs0;
            c.band0 = h.band_pairs;
            c.pairs0 = h.tile_pairs;
            const float nmax = float_from_bits(h.max_norm_bits);
            if (dp > 0 && c.auto_phase == 0) {
                const int e = fp16_scale_exp((double)nmax, c.eps);
                const double d16 = band_halfwidth(BM_PATH_TC_FP16, pts.d, tile_config_for(pts.d, 1).d_pad, c.eps2,
                                                  nmax, nmax, e) * std::ldexp(1.0, -2 * e);
                const double d3 = band_halfwidth(BM_PATH_TC_SPLIT3, pts.d, pts.d_pad, c.eps2, nmax, nmax, 0);
                const double predicted = (double)db / (double)dp * (d16 / d3);
                if (predicted < kAutoPredictFraction) {
                    bm_status rs2 = switch_path(c, pts, ar, s, BM_PATH_TC_FP16, nmax, (int)h.steps);
                    if (rs2 != BM_OK) return rs2;
                    c.auto_phase = 1;
                } else {
                    c.auto_phase = 2;
                }
            } else if (dp > 0 && c.auto_phase == 1) {
                if ((double)db > kAutoBandFraction * (double)dp) {
                    bm_status rs2 = switch_path(c, pts, ar, s, BM_PATH_TC_SPLIT3, nmax, (int)h.steps);
                    if (rs2 != BM_OK) return rs2;
                    c.auto_phase = 2;
                }
            }
        }
        chunk = std::min(chunk * 2, 64);
    }
    return BM_OK;
}

bm_status greedy_pass(Prepared& pts, double eps2, int path, bool auto_switch, int S, Arena& ar, cudaStream_t s,
                      DeviceState* st, HostState& hs, unsigned long long& step_cap, unsigned long long& mem_cap,
                      bool* retry, int** landmarks_out, unsigned long long** mem_keys_out, DeviceState& final_state,
                      SweepTimer& stimer, const IvfIndex* ivf, const float* phi_perm, int nprobe, int* path_used,
                      const GraphIndex* gidx = nullptr, int ef = 0, long long max_visits = 0,
                      const Prepared* ivf_b_pad = nullptr) {
    *retry = false;
    GreedyCtx c;
    bm_status rs = greedy_setup(pts, eps2, path, S, ar, s, st, step_cap, mem_cap, ivf, phi_perm, nprobe, c);
    if (rs != BM_OK) return rs;
    c.sd.gidx = gidx;
    c.sd.gidx_ef = ef;
    c.sd.gidx_max_visits = max_visits;
    c.sd.ivf_b_pad = ivf_b_pad;
    c.auto_switch = auto_switch;
    rs = greedy_drive(c, pts, ar, s, hs, step_cap, mem_cap, final_state, stimer, false);
    if (rs != BM_OK) return rs;
    release_sweep_out(ar, c.so, false);
    *landmarks_out = c.g.landmarks;
    *mem_keys_out = c.g.mem_keys;
    *path_used = c.path;
    return BM_OK;
}

}  // namespace
}  // namespace bm

using namespace bm;

namespace bm {
namespace {

// Range query R_eps(q) for every row q of Q over the points X (exact), or over the
// cells an inverted-file index probes for q (conservative).  Arguments validated.
// row_r2 (device, m entries; optional): a squared radius per query row instead of eps^2
// (k-NN sweeps; r2_max is its maximum); the tensor-core rows then use the bf16 split.
bm_status range_core(const float* X, long long n, int d, const float* Q, long long m, float eps, const bm_options& opt,
                     const IvfIndex* ivf, int nprobe, int* probes_out, bm_csr* out, bm_stats* stats,
                     const double* row_r2 = nullptr, double r2_max = 0.0, unsigned long long cap_hint = 0,
                     const GraphIndex* gidx = nullptr, int ef = 0, long long max_visits = 0) {
    std::memset(out, 0, sizeof(*out));
    if (stats) std::memset(stats, 0, sizeof(*stats));
    cudaStream_t s = (cudaStream_t)opt.stream;
    const bool host_io = opt.host_io != 0;
    const double eps2 = row_r2 ? 0.0 : (double)eps * (double)eps;
    // automatic path: a single sweep cannot change course, so range queries take the split
    const int req = (opt.path == BM_PATH_TC_AUTO || (row_r2 && opt.path == BM_PATH_TC_FP16))
                        ? (int)BM_PATH_TC_SPLIT3 : opt.path;
    // the inverted file scans on the tensor cores unless the FP32 path is asked for
    const bool tc = is_tc_path(req) && gidx == nullptr && !(ivf && row_r2);
    const int path = gidx ? (int)BM_PATH_FP32 : (tc ? req : (ivf ? (int)BM_PATH_FP32 : req));
    Timer tm(s);
    tm.mark();
    SweepTimer stimer(s);
    const long long launches0 = g_kernel_launches;
    bm_status rs = BM_OK;
    long long nnz = 0;
    long long* offsets = nullptr;
    int* ids = nullptr;
    unsigned long long band = 0, pairs = 0;
    float delta = 0.f;
    float* dists = nullptr;
    unsigned long long* err_dev = nullptr;
    double dist_err = 0.0;
    int truncated = 0, centred = 0;
    {
        Arena ar(&opt, s);
        const float* dX = (ivf || gidx) ? X : stage_input(X, n, d, host_io, ar, s, &rs);
        if (rs != BM_OK) return rs;
        const float* dQ = stage_input(Q, m, d, host_io, ar, s, &rs);
        if (rs != BM_OK) return rs;
        ALLOC(offsets, long long, m + 1);
        if (m == 0 || n == 0) {
            TRY_CUDA(cudaMemsetAsync(offsets, 0, sizeof(long long) * (m + 1), s));
            ALLOC(ids, int, 1);
        } else {
            DeviceState* st;
            ALLOC(st, DeviceState, 1);
            TRY_CUDA(cudaMemsetAsync(st, 0, sizeof(DeviceState), s));
            int* bad;
            ALLOC(bad, int, 1);
            TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
            Prepared px, pq;
            // inverted-file mode: the points enter the tiles in cell order
            const int prec = tc ? prec_for(path) : kPrecNone;
            const float* bsrc = ivf ? (tc ? ivf->xpad : ivf->xperm) : dX;
            const long long brows = (ivf && tc) ? ivf->npad : n;
            // the tensor-core tiles without an index may take translated operands (same centre
            // for points and queries)
            const float* centre = nullptr;
            if (tc && !ivf) {
                rs = operand_centre(dX, n, d, opt, st, ar, s, &centre);
                if (rs != BM_OK) return rs;
            }
            rs = prepare(bsrc, brows, d, eps2, false, prec, ar, &st->max_norm_bits, bad, s, px, nullptr, centre);
            if (rs != BM_OK) return rs;
            rs = prepare(dQ, m, d, eps2, true, prec, ar, &st->max_norm_q_bits, bad, s, pq, row_r2, centre);
            if (rs != BM_OK) return rs;
            int hbad = 0;
            unsigned hnorm[2] = {0u, 0u};
            TRY_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
            TRY_CUDA(cudaMemcpyAsync(hnorm, &st->max_norm_bits, sizeof(hnorm), cudaMemcpyDeviceToHost, s));
            TRY_CUDA(cudaStreamSynchronize(s));
            if (hbad) return fail(BM_ERR_ARG, "input holds NaN or Inf");
            {
                float nx, nq;
                std::memcpy(&nx, &hnorm[0], sizeof(float));
                std::memcpy(&nq, &hnorm[1], sizeof(float));
                if (row_r2) {
                    // |phi_q| <= max(N_q^2, r2_max) / 2 (the whole radius on the query side),
                    // |phi_x| <= N_x^2 / 2; delta rounded up to float
                    const double Nq = nq, Nx = nx;
                    const double dl = band_halfwidth_core(path, d, px.d_pad, Nq, Nx, 0.5 * std::max(Nq * Nq, r2_max),
                                                          0.5 * Nx * Nx);
                    float df = (float)dl;
                    if ((double)df < dl) df = std::nextafter(df, INFINITY);
                    TRY_CUDA(cudaMemcpyAsync(&st->delta, &df, sizeof(float), cudaMemcpyHostToDevice, s));
                    TRY_CUDA(cudaStreamSynchronize(s));
                    if (px.prec != kPrecNone) {
                        TRY_CUDA(launch_set_aug_delta(st, px, eps2, false, s));
                        TRY_CUDA(launch_set_aug_delta(st, pq, eps2, true, s, row_r2));
                    }
                } else {
                    rs = finish_prep(st, path, d, eps2, (double)eps, false, std::max(nx, nq), &px, &pq, s);
                    if (rs != BM_OK) return rs;
                }
            }
            unsigned long long cap = (unsigned long long)std::min<long long>(std::max<long long>(n, m) * 4 + (1 << 20),
                                                                              (long long)n * m);
            if (tc) cap = std::max<unsigned long long>(cap, (unsigned long long)device_sm_count() * 4096);
            if (cap_hint) cap = std::max<unsigned long long>(cap, std::min<unsigned long long>(cap_hint, (unsigned long long)n * m));
            HostState hs;
            DeviceState h;
            unsigned long long* keys = nullptr;
            const int sms = device_sm_count();
            for (int attempt = 0; attempt < 3; ++attempt) {
                SweepOut so;
                rs = alloc_sweep_out(ar, tc, cap, sms, so);
                if (rs != BM_OK) return rs;
                SweepDesc sd;
                sd.a = &pq;
                sd.b = &px;
                sd.a_rows_max = m;
                sd.a_rows_dev = nullptr;
                sd.st = st;
                sd.check_done = false;
                sd.eps2 = eps2;
                sd.sink = HitSink();
                sd.sink.band_count = &st->band_pairs;
                sd.sink.pair_count = &st->tile_pairs;
                sd.ivf = ivf;
                sd.ivf_phi_perm = px.phi;
                sd.nprobe = nprobe;
                sd.ivf_probes_out = probes_out;
                sd.row_eps2 = row_r2;
                sd.gidx = gidx;
                sd.gidx_ef = ef;
                sd.gidx_max_visits = max_visits;
                sd.ivf_b_pad = (ivf && tc) ? &px : nullptr;
                rs = sweep_stage(sd, st, path, so, &st->hit_count, kErrHitOverflow, false, sms, stimer, s, ar);
                if (rs != BM_OK) return rs;
                rs = read_state(st, hs, h, s);
                if (rs != BM_OK) return rs;
                stimer.collect();
                if (h.error & kErrTimeout) return fail(BM_ERR_TIMEOUT, "a bounded device wait expired");
                const bool overflow = (h.error & kErrHitOverflow) != 0 || h.hit_count > cap || h.band_n > cap;
                keys = so.keys;
                release_sweep_out(ar, so, !overflow);
                if (!overflow) break;
                if (attempt == 2) return fail(BM_ERR_CAPACITY, "range query hit buffer kept overflowing");
                cap = std::max<unsigned long long>(
                    2 * cap, std::max(h.max_seg * (unsigned long long)sms, std::max(h.hit_count, h.band_n)) * 5 / 4 + 1024);
                TRY_CUDA(cudaMemsetAsync(&st->error, 0, sizeof(int), s));
                TRY_CUDA(cudaMemsetAsync(&st->max_seg, 0, sizeof(unsigned long long), s));
                TRY_CUDA(cudaMemsetAsync(&st->band_n, 0, sizeof(unsigned long long), s));
                TRY_CUDA(cudaMemsetAsync(&st->hit_count, 0, sizeof(unsigned long long), s));
                TRY_CUDA(cudaMemsetAsync(&st->band_pairs, 0, sizeof(unsigned long long), s));
                TRY_CUDA(cudaMemsetAsync(&st->tile_pairs, 0, sizeof(unsigned long long), s));
            }
            nnz = (long long)h.hit_count;
            band = h.band_pairs;
            pairs = h.tile_pairs;
            delta = h.delta;
            truncated = h.gidx_truncated;
            centred = h.centred;
            unsigned long long* tmp;
            ALLOC(tmp, unsigned long long, std::max<long long>(nnz, 1));
            unsigned long long* sorted = nullptr;
            TRY_CUDA(radix_sort_u64(keys, tmp, nnz, digit_shifts(bits_for(n - 1), bits_for(m - 1)), ar, s, &sorted));
            ALLOC(ids, int, std::max<long long>(nnz, 1));
            TRY_CUDA(launch_csr_from_sorted(sorted, nnz, m, offsets, ids, s));
        }
        if (opt.want_dists) {
            if (nnz == 0) {
                ALLOC(dists, float, 1);
            } else {
                rs = csr_dists(ar, s, dQ, nullptr, dX, d, offsets, m, ids, nnz, &dists, &err_dev);
                if (rs != BM_OK) return rs;
            }
        }
        if (host_io) {
            void *ho = nullptr, *hi = nullptr, *hd = nullptr;
            if (!to_host(&ho, offsets, sizeof(long long) * (m + 1), s) ||
                !to_host(&hi, ids, sizeof(int) * std::max<long long>(nnz, 1), s) ||
                (dists && !to_host(&hd, dists, sizeof(float) * std::max<long long>(nnz, 1), s))) {
                std::free(ho);
                std::free(hi);
                std::free(hd);
                return fail(BM_ERR_CUDA, "device to host copy of the result failed");
            }
            TRY_CUDA(cudaStreamSynchronize(s));
            offsets = (long long*)ho;
            ids = (int*)hi;
            dists = (float*)hd;
            out->on_host = 1;
        } else {
            ar.take(offsets);
            ar.take(ids);
            if (dists && !ar.take(dists)) return fail(BM_ERR_NOMEM, "distance buffer could not be handed over");
        }
        rs = read_err(err_dev, s, &dist_err);
        if (rs != BM_OK) return rs;
    }
    tm.mark();
    out->rows = m;
    out->nnz = nnz;
    out->offsets = (int64_t*)offsets;
    out->ids = ids;
    out->dists = dists;
    if (stats) {
        stats->distance_evals = (int64_t)n * m;
        stats->tile_pairs = (int64_t)pairs;
        stats->band_pairs = (int64_t)band;
        stats->ms_total = tm.ms(0, 1);
        stats->band_delta = delta;
        stats->path = path;
        stats->ms_sweep = stimer.ms;
        stats->sweep_launches = stimer.launches;
        stats->kernel_launches = g_kernel_launches - launches0;
        stats->recheck_rate = pairs ? (double)band / (double)pairs : 0.0;
        stats->dist_max_rel_err = dist_err;
        stats->truncated = truncated;
        stats->centred = centred;
    }
    return BM_OK;
}

// k-th nearest-neighbour distance of every point, itself counted first (Sec. 6.1), and
// optionally their median (the target-occupancy eps).  kdist: n doubles (device, or host
// with host_io; may be NULL when only eps is wanted).  Arguments validated.
bm_status knn_core(const float* X, long long n, int d, int k, const bm_options& opt, double* kdist, double* eps_out,
                   bm_stats* stats) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    cudaStream_t s = (cudaStream_t)opt.stream;
    const bool host_io = opt.host_io != 0;
    Timer tm(s);
    tm.mark();
    const long long launches0 = g_kernel_launches;
    bm_stats rst;
    std::memset(&rst, 0, sizeof(rst));
    long long nnz = 0;
    {
        Arena ar(&opt, s);
        bm_status rs = BM_OK;
        const float* dX = stage_input(X, n, d, host_io, ar, s, &rs);
        if (rs != BM_OK) return rs;
        // pass 1: per-row upper bounds from a strided sample of at least k points (about
        // n / 16 of them, at least 8 k, at most 65,536): a row's ball then holds about
        // k n / s points
        long long target = std::max<long long>(8LL * k, n / 16);
        target = std::max<long long>(std::min<long long>(target, 65536), k);
        const long long stride = target >= n ? 1 : n / target;
        const long long sN = (n + stride - 1) / stride;
        double* rho;
        unsigned long long* rmax;
        int* bad;
        ALLOC(rho, double, n);
        ALLOC(rmax, unsigned long long, 1);
        ALLOC(bad, int, 1);
        TRY_CUDA(cudaMemsetAsync(rmax, 0, sizeof(unsigned long long), s));
        TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
        TRY_CUDA(launch_knn_bound(dX, n, d, stride, sN, k, rho, rmax, bad, s));
        int hbad = 0;
        unsigned long long hmax = 0;
        TRY_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        TRY_CUDA(cudaMemcpyAsync(&hmax, rmax, sizeof(hmax), cudaMemcpyDeviceToHost, s));
        TRY_CUDA(cudaStreamSynchronize(s));
        if (hbad) return fail(BM_ERR_ARG, "input holds NaN or Inf, or squared distances that overflow float");
        double r2_max;
        std::memcpy(&r2_max, &hmax, sizeof(double));
        // pass 2: range query of every point with its own squared radius (exact)
        bm_options o2 = opt;
        o2.host_io = 0;
        o2.want_dists = 0;
        bm_csr csr;
        const double expect = 1.5 * (double)n * (double)k * ((double)n / (double)sN) + 2.0 * (double)n;
        const unsigned long long hint = (unsigned long long)std::min(expect, (double)n * (double)n);
        rs = range_core(dX, n, d, dX, n, 1.0f, o2, nullptr, 0, nullptr, &csr, &rst, rho, r2_max, hint);
        if (rs != BM_OK) return rs;
        struct CsrGuard {
            bm_csr* c;
            const bm_options* o;
            ~CsrGuard() { bm_csr_free(c, o); }
        } guard{&csr, &o2};
        nnz = csr.nnz;
        // pass 3: the k-th smallest FP64 squared distance of every row
        double* D;
        ALLOC(D, double, std::max<long long>(nnz, 1));
        double* kd = (kdist && !host_io) ? kdist : nullptr;
        if (!kd) ALLOC(kd, double, n);
        TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
        TRY_CUDA(launch_knn_select(dX, d, (const long long*)csr.offsets, n, csr.ids, nnz, D, k, kd, bad, s));
        ar.release(D);
        if (eps_out) {
            // median: radix sort of the bit patterns (non-negative doubles order like them)
            unsigned long long *keys, *tmp, *sorted = nullptr;
            ALLOC(keys, unsigned long long, n);
            ALLOC(tmp, unsigned long long, n);
            TRY_CUDA(cudaMemcpyAsync(keys, kd, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            TRY_CUDA(radix_sort_u64(keys, tmp, n, digit_shifts(32, 32), ar, s, &sorted));
            double mid[2] = {0.0, 0.0};
            const long long i1 = n / 2, i0 = (n % 2) ? i1 : i1 - 1;
            TRY_CUDA(cudaMemcpyAsync(&mid[0], sorted + i0, sizeof(double), cudaMemcpyDeviceToHost, s));
            TRY_CUDA(cudaMemcpyAsync(&mid[1], sorted + i1, sizeof(double), cudaMemcpyDeviceToHost, s));
            TRY_CUDA(cudaStreamSynchronize(s));
            *eps_out = (n % 2) ? mid[1] : (mid[0] + mid[1]) * 0.5;
        }
        if (kdist && host_io) TRY_CUDA(cudaMemcpyAsync(kdist, kd, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        TRY_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        TRY_CUDA(cudaStreamSynchronize(s));
        if (hbad) return fail(BM_ERR_CUDA, "k-NN select: a row's ball held fewer than k points");
    }
    tm.mark();
    if (stats) {
        *stats = rst;
        stats->distance_evals = (int64_t)n * n;
        stats->ms_total = tm.ms(0, 1);
        stats->kernel_launches = g_kernel_launches - launches0;
        stats->candidates = nnz;   // points examined by the select (the rows' balls)
    }
    return BM_OK;
}


}  // namespace
}  // namespace bm

namespace bm {
namespace {

// Memberships (ordinal << 32 | point keys) to the CSR of full balls, then the
// nerve edges (skipped with opt.skip_edges).  mem_keys is released.
bm_status members_and_edges(Arena& ar, cudaStream_t s, const bm_options& opt, long long n, long long L,
                            long long nnz, unsigned long long* mem_keys, Timer* tm, long long** offsets_out,
                            int** ids_out, int** edges_out, long long* E_out, long long* edge_pairs) {
    unsigned long long* tmp;
    ALLOC(tmp, unsigned long long, std::max<long long>(nnz, 1));
    unsigned long long* sorted = nullptr;
    TRY_CUDA(radix_sort_u64(mem_keys, tmp, nnz, digit_shifts(bits_for(n - 1), bits_for(L - 1)), ar, s, &sorted));
    long long* offsets;
    int* ids;
    ALLOC(offsets, long long, L + 1);
    ALLOC(ids, int, std::max<long long>(nnz, 1));
    TRY_CUDA(launch_csr_from_sorted(sorted, nnz, L, offsets, ids, s));
    if (tm) tm->mark();  // CSR done
    Failure f{BM_OK, ""};
    EdgeResult er;
    if (!opt.skip_edges && !build_edges(sorted, offsets, nnz, n, L, ar, s, er, f)) return fail(f.status, f.msg);
    int* edges = er.edges;
    if (!edges) ALLOC(edges, int, 2);
    if (tm) tm->mark();  // edges done
    ar.release(tmp);
    ar.release(mem_keys);
    *offsets_out = offsets;
    *ids_out = ids;
    *edges_out = edges;
    *E_out = er.n_edges;
    *edge_pairs = er.pairs;
    return BM_OK;
}

// Move the result arrays into *g: copied to malloc'd host buffers (host_io) or
// handed over as device buffers that the caller frees with bm_graph_free.
bm_status hand_over(Arena& ar, cudaStream_t s, bool host_io, int* landmarks, long long* offsets, int* ids,
                    int* edges, long long L, long long nnz, long long E, bm_graph& g, float* dists = nullptr) {
    if (host_io) {
        void *hl = nullptr, *ho = nullptr, *hi = nullptr, *he = nullptr, *hd = nullptr;
        bool ok = to_host(&hl, landmarks, sizeof(int) * std::max<long long>(L, 1), s) &&
                  to_host(&ho, offsets, sizeof(long long) * (L + 1), s) &&
                  to_host(&hi, ids, sizeof(int) * std::max<long long>(nnz, 1), s) &&
                  to_host(&he, edges, sizeof(int) * 2 * std::max<long long>(E, 1), s) &&
                  (!dists || to_host(&hd, dists, sizeof(float) * std::max<long long>(nnz, 1), s));
        if (ok && cudaStreamSynchronize(s) != cudaSuccess) ok = false;
        if (!ok) {
            std::free(hl); std::free(ho); std::free(hi); std::free(he); std::free(hd);
            cudaGetLastError();
            return fail(BM_ERR_CUDA, "device to host copy of the result failed");
        }
        g.landmarks = (int*)hl;
        g.members.offsets = (int64_t*)ho;
        g.members.ids = (int*)hi;
        g.members.dists = (float*)hd;
        g.edges = (int*)he;
        g.on_host = 1;
        g.members.on_host = 1;
    } else {
        // buffers carved from a slab are copied into buffers of their own
        auto own = [&](void* p, size_t bytes, bm_status* rs) -> void* {
            if (ar.take(p)) return p;
            void* q = ar.get_standalone(bytes);
            if (!q || !ar.take(q)) {
                *rs = fail(BM_ERR_NOMEM, "allocation of a result buffer failed");
                return nullptr;
            }
            if (cudaMemcpyAsync(q, p, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                cudaGetLastError();
                device_free(ar.options(), s, q);
                *rs = fail(BM_ERR_CUDA, "device copy of a result buffer failed");
                return nullptr;
            }
            return q;
        };
        bm_status rs = BM_OK;
        void* ol = own(landmarks, sizeof(int) * std::max<long long>(L, 1), &rs);
        void* oo = rs == BM_OK ? own(offsets, sizeof(long long) * (L + 1), &rs) : nullptr;
        void* oi = rs == BM_OK ? own(ids, sizeof(int) * std::max<long long>(nnz, 1), &rs) : nullptr;
        void* oe = rs == BM_OK ? own(edges, sizeof(int) * 2 * std::max<long long>(E, 1), &rs) : nullptr;
        void* od = rs == BM_OK && dists ? own(dists, sizeof(float) * std::max<long long>(nnz, 1), &rs) : nullptr;
        if (rs != BM_OK) {
            device_free(ar.options(), s, ol);
            device_free(ar.options(), s, oo);
            device_free(ar.options(), s, oi);
            device_free(ar.options(), s, oe);
            return rs;
        }
        g.landmarks = (int*)ol;
        g.members.offsets = (int64_t*)oo;
        g.members.ids = (int*)oi;
        g.members.dists = (float*)od;
        g.edges = (int*)oe;
    }
    g.n_landmarks = L;
    g.members.rows = L;
    g.members.nnz = nnz;
    g.n_edges = E;
    return BM_OK;
}

// Ball Mapper of the points X (n x d): greedy landmarks (or the given fixed ones),
// full-ball memberships, nerve edges.  With an inverted-file index the balls are
// the index's conservative range sets (Sec. 5.3-5.4); otherwise they are exact.
bm_status build_graph(const float* X, long long n, int d, float eps, const bm_options& opt, const IvfIndex* ivf,
                      int nprobe, const int* fixed_lm, long long nL, bm_graph* out, const GraphIndex* gidx = nullptr,
                      int ef = 0, long long max_visits = 0) {
    std::memset(out, 0, sizeof(*out));
    int S = opt.batch;
    if (S == 0) S = (ivf || gidx) ? 8192 : kMaxBatch;
    if (S < 32 || S > kMaxBatch || S % 32)
        return fail(BM_ERR_ARG, "batch must be a multiple of 32 in [32, " + std::to_string(kMaxBatch) + "]");
    cudaStream_t s = (cudaStream_t)opt.stream;
    const bool host_io = opt.host_io != 0;
    const double eps2 = (double)eps * (double)eps;
    // automatic path: the greedy starts on the split and picks its path after the
    // first step (greedy_drive)
    const bool auto_switch = opt.path == BM_PATH_TC_AUTO && ivf == nullptr && gidx == nullptr && fixed_lm == nullptr;
    // fixed landmarks sweep once: the automatic path and fp16 take the bf16 split
    const int req = (opt.path == BM_PATH_TC_AUTO || (fixed_lm && opt.path == BM_PATH_TC_FP16))
                        ? (int)BM_PATH_TC_SPLIT3 : opt.path;
    const bool tc = is_tc_path(req) && gidx == nullptr;
    int path = gidx ? (int)BM_PATH_FP32 : req;
    Timer tm(s);
    tm.mark();  // 0
    SweepTimer stimer(s);
    const long long launches0 = g_kernel_launches;
    bm_status rs = BM_OK;
    bm_graph g;
    std::memset(&g, 0, sizeof(g));
    DeviceState fin;
    std::memset(&fin, 0, sizeof(fin));
    long long edge_pairs = 0;
    unsigned long long* err_dev = nullptr;
    double dist_err = 0.0;
    {
        Arena ar(&opt, s);
        const float* dX = (ivf || gidx) ? X : stage_input(X, n, d, host_io, ar, s, &rs);
        if (rs != BM_OK) return rs;
        int* landmarks = nullptr;
        long long* offsets = nullptr;
        int* ids = nullptr;
        int* edges = nullptr;
        long long L = 0, nnz = 0, E = 0;
        if (n == 0) {
            ALLOC(landmarks, int, 1);
            ALLOC(offsets, long long, 1);
            TRY_CUDA(cudaMemsetAsync(offsets, 0, sizeof(long long), s));
            ALLOC(ids, int, 1);
            ALLOC(edges, int, 2);
            tm.mark(); tm.mark(); tm.mark(); tm.mark();
        } else {
            DeviceState* st;
            ALLOC(st, DeviceState, 1);
            int* bad;
            ALLOC(bad, int, 1);
            TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
            TRY_CUDA(cudaMemsetAsync(st, 0, sizeof(DeviceState), s));
            Prepared px;
            const float* centre = nullptr;   // translated tensor-core operands (not with an index)
            if (tc && !ivf) {
                rs = operand_centre(dX, n, d, opt, st, ar, s, &centre);
                if (rs != BM_OK) return rs;
            }
            rs = prepare(dX, n, d, eps2, false, tc ? prec_for(path) : kPrecNone, ar, &st->max_norm_bits, bad, s, px,
                         nullptr, centre);
            if (rs != BM_OK) return rs;
            // inverted-file mode: the cell-ordered copy of the points for the scan (phi for the
            // FP32 scan; the padded tensor-core operands otherwise)
            Prepared pperm;
            if (ivf && !tc) {
                rs = prepare(ivf->xperm, n, d, eps2, false, kPrecNone, ar, &st->max_norm_bits, bad, s, pperm);
                if (rs != BM_OK) return rs;
            }
            if (ivf && tc) {
                rs = prepare(ivf->xpad, ivf->npad, d, eps2, false, prec_for(path), ar, &st->max_norm_bits, bad, s,
                             pperm);
                if (rs != BM_OK) return rs;
            }
            const Prepared* b_pad = (ivf && tc) ? &pperm : nullptr;
            int hbad = 0;
            unsigned hnorm = 0u;
            TRY_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
            TRY_CUDA(cudaMemcpyAsync(&hnorm, &st->max_norm_bits, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
            TRY_CUDA(cudaStreamSynchronize(s));
            if (hbad) return fail(BM_ERR_ARG, "input holds NaN or Inf");
            {
                float nx;
                std::memcpy(&nx, &hnorm, sizeof(float));
                rs = finish_prep(st, path, d, eps2, (double)eps, true, nx, &px, nullptr, s);
                if (rs != BM_OK) return rs;
                if (b_pad) TRY_CUDA(launch_set_aug_delta(st, pperm, eps2, false, s));
            }
            tm.mark();  // 1: prep done
            unsigned long long step_cap = (unsigned long long)std::min<long long>((long long)S * n, 1LL << 22);
            if (tc) step_cap = std::max<unsigned long long>(step_cap, (unsigned long long)device_sm_count() * 2048);
            unsigned long long mem_cap = (unsigned long long)std::max<long long>(4 * n, 1LL << 20);
            HostState hs;
            unsigned long long* mem_keys = nullptr;
            if (fixed_lm) {
                // fixed landmarks: their balls through the index, one scan of all rows
                ALLOC(landmarks, int, std::max<long long>(nL, 1));
                if (nL) TRY_CUDA(cudaMemcpyAsync(landmarks, fixed_lm, sizeof(int) * nL,
                                                 host_io ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
                float* qx;
                ALLOC(qx, float, std::max<long long>(nL, 1) * d);
                TRY_CUDA(launch_gather_rows(dX, landmarks, nL, d, qx, s));
                Prepared pq;
                rs = prepare(qx, nL, d, eps2, true, tc ? prec_for(path) : kPrecNone, ar, &st->max_norm_q_bits, bad, s,
                             pq, nullptr, centre);
                if (rs != BM_OK) return rs;
                if (tc) TRY_CUDA(launch_set_aug_delta(st, pq, eps2, true, s));   // the landmark rows' delta'
                const int sms = device_sm_count();
                unsigned long long cap = (unsigned long long)std::max<long long>(4 * n, 1LL << 20);
                if (tc) cap = std::max<unsigned long long>(cap, (unsigned long long)sms * 4096);
                for (int attempt = 0; attempt < 3; ++attempt) {
                    SweepOut so;
                    rs = alloc_sweep_out(ar, tc, cap, sms, so);
                    if (rs != BM_OK) return rs;
                    SweepDesc sd;
                    sd.a = &pq;
                    sd.b = &px;
                    sd.a_rows_max = nL;
                    sd.a_rows_dev = nullptr;
                    sd.st = st;
                    sd.check_done = false;
                    sd.eps2 = eps2;
                    sd.sink = HitSink();
                    sd.sink.band_count = &st->band_pairs;
                    sd.sink.pair_count = &st->tile_pairs;
                    sd.ivf = ivf;
                    sd.ivf_phi_perm = pperm.phi;
                    sd.nprobe = nprobe;
                    sd.gidx = gidx;
                    sd.gidx_ef = ef;
                    sd.gidx_max_visits = max_visits;
                    sd.ivf_b_pad = b_pad;
                    rs = sweep_stage(sd, st, path, so, &st->mem_count, kErrHitOverflow, false, sms, stimer, s, ar);
                    if (rs != BM_OK) return rs;
                    rs = read_state(st, hs, fin, s);
                    if (rs != BM_OK) return rs;
                    stimer.collect();
                    const bool overflow = (fin.error & kErrHitOverflow) != 0 || fin.mem_count > cap || fin.band_n > cap;
                    mem_keys = so.keys;
                    release_sweep_out(ar, so, !overflow);
                    if (!overflow) break;
                    if (attempt == 2) return fail(BM_ERR_CAPACITY, "membership buffer kept overflowing");
                    cap = std::max<unsigned long long>(
                        2 * cap, std::max(fin.max_seg * (unsigned long long)sms, std::max(fin.mem_count, fin.band_n)) *
                                     5 / 4 + 1024);
                    TRY_CUDA(cudaMemsetAsync(&st->error, 0, sizeof(int), s));
                    TRY_CUDA(cudaMemsetAsync(&st->max_seg, 0, sizeof(unsigned long long), s));
                    TRY_CUDA(cudaMemsetAsync(&st->band_n, 0, sizeof(unsigned long long), s));
                    TRY_CUDA(cudaMemsetAsync(&st->mem_count, 0, sizeof(unsigned long long), s));
                }
                fin.n_landmarks = (int)nL;
                ar.release(qx);
            } else {
                for (int attempt = 0; attempt < 6; ++attempt) {
                    bool retry = false;
                    TRY_CUDA(cudaMemsetAsync(st, 0, offsetof(DeviceState, max_norm_bits), s));
                    {
                        const int s_first = S < 256 ? S : 256;   // the batch grows while candidates survive
                        TRY_CUDA(cudaMemcpyAsync(&st->s_next, &s_first, sizeof(int), cudaMemcpyHostToDevice, s));
                        TRY_CUDA(cudaStreamSynchronize(s));
                    }
                    int path_used = path;
                    rs = greedy_pass(px, eps2, path, auto_switch, S, ar, s, st, hs, step_cap, mem_cap, &retry,
                                     &landmarks, &mem_keys, fin, stimer, ivf, ivf ? pperm.phi : nullptr, nprobe,
                                     &path_used, gidx, ef, max_visits, b_pad);
                    if (rs != BM_OK) return rs;
                    path = path_used;
                    if (!retry) break;
                    if (attempt == 5) return fail(BM_ERR_CAPACITY, "greedy buffers kept overflowing");
                }
            }
            tm.mark();  // 2: greedy (with memberships) done
            L = fin.n_landmarks;
            nnz = (long long)fin.mem_count;
            rs = members_and_edges(ar, s, opt, n, L, nnz, mem_keys, &tm, &offsets, &ids, &edges, &E, &edge_pairs);
            if (rs != BM_OK) return rs;
        }
        float* dists = nullptr;
        if (opt.want_dists) {
            if (n == 0) {
                ALLOC(dists, float, 1);
            } else {
                rs = csr_dists(ar, s, nullptr, landmarks, dX, d, offsets, L, ids, nnz, &dists, &err_dev);
                if (rs != BM_OK) return rs;
            }
        }
        rs = hand_over(ar, s, host_io, landmarks, offsets, ids, edges, L, nnz, E, g, dists);
        if (rs != BM_OK) return rs;
        rs = read_err(err_dev, s, &dist_err);
        if (rs != BM_OK) return rs;
    }
    tm.mark();  // 5
    g.stats.distance_evals = (int64_t)g.n_landmarks * n;
    g.stats.tile_pairs = (int64_t)fin.tile_pairs;
    g.stats.band_pairs = (int64_t)fin.band_pairs;
    g.stats.greedy_steps = (int64_t)fin.steps;
    g.stats.candidates = (int64_t)fin.candidates;
    g.stats.edge_pairs = edge_pairs;
    g.stats.ms_prep = tm.ms(0, 1);
    g.stats.ms_greedy = tm.ms(1, 2);
    g.stats.ms_members = tm.ms(2, 3);
    g.stats.ms_edges = tm.ms(3, 4);
    g.stats.ms_total = tm.ms(0, 5);
    g.stats.band_delta = fin.delta;
    g.stats.path = path;
    g.stats.ms_sweep = stimer.ms;
    g.stats.sweep_launches = stimer.launches;
    g.stats.kernel_launches = g_kernel_launches - launches0;
    g.stats.recheck_rate = fin.tile_pairs ? (double)fin.band_pairs / (double)fin.tile_pairs : 0.0;
    g.stats.dist_max_rel_err = dist_err;
    g.stats.truncated = fin.gidx_truncated;
    g.stats.centred = fin.centred;
    *out = g;
    return BM_OK;
}


// ---- Batched builds: the greedy loops of many instances in one CUDA graph.

// Page-locked host array (asynchronous device-to-host copies land here).
struct PinnedI64 {
    long long* p = nullptr;
    explicit PinnedI64(int count) {
        if (cudaMallocHost(&p, sizeof(long long) * (size_t)std::max(count, 1)) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    ~PinnedI64() {
        if (p) cudaFreeHost(p);
    }
};

struct BatchItem {
    Arena* ar = nullptr;   // the batch's shared scratch arena
    long long n = 0;
    int d = 0;
    double eps2 = 0.0;
    DeviceState* st = nullptr;
    Prepared px;
    GreedyCtx gc;
    unsigned long long step_cap = 0, mem_cap = 0;
    long long body_kernels = 0;
};

struct GraphGuard {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    ~GraphGuard() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
    }
};

// Stage and prepare one instance's points; its DeviceState is sts[i] (zeroed).
bm_status batch_prep(BatchItem& it, const bm_instance& in, const bm_options& opt, bool tc, int path,
                     DeviceState* st, int* bad, cudaStream_t s) {
    Arena& ar = *it.ar;
    bm_status rs = BM_OK;
    const float* dX = stage_input(in.X, in.n, in.d, opt.host_io != 0, ar, s, &rs);
    if (rs != BM_OK) return rs;
    it.st = st;
    const float* centre = nullptr;
    if (tc) {
        rs = operand_centre(dX, in.n, in.d, opt, st, ar, s, &centre);
        if (rs != BM_OK) return rs;
    }
    rs = prepare(dX, in.n, in.d, it.eps2, false, tc ? prec_for(path) : kPrecNone, ar, &st->max_norm_bits, bad, s,
                 it.px, nullptr, centre);
    if (rs != BM_OK) return rs;
    return BM_OK;
}

// Capture one greedy step plus the loop condition into the body of a WHILE node.
bm_status batch_capture(BatchItem& it, GraphGuard& gg, unsigned* iterations, SweepTimer& stimer) {
    cudaGraphConditionalHandle h;
    TRY_CUDA(cudaGraphConditionalHandleCreate(&h, gg.graph, 1u, cudaGraphCondAssignDefault));
    // zero-initialised storage (the union in the struct has no default constructor)
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    std::memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    TRY_CUDA(cudaGraphAddNode(&node, gg.graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    TRY_CUDA(cudaStreamBeginCaptureToGraph(gg.cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    const long long k0 = g_kernel_launches;
    bm_status rs = greedy_enqueue_step(it.gc, it.px, *it.ar, stimer, gg.cs);
    cudaError_t le = cudaSuccess;
    const unsigned max_iterations = (unsigned)std::min<long long>(it.n + 2, 0x7fffffffLL);
    if (rs == BM_OK) le = launch_greedy_continue(it.gc.g, h, iterations, max_iterations, gg.cs);
    cudaGraph_t captured = nullptr;
    cudaError_t ee = cudaStreamEndCapture(gg.cs, &captured);
    it.body_kernels = g_kernel_launches - k0;
    if (rs != BM_OK) return rs;
    TRY_CUDA(le);
    TRY_CUDA(ee);
    return BM_OK;
}

bm_status build_batched(const bm_instance* inst, int count, const bm_options& opt, bm_graph* outs,
                        int32_t* statuses, int* failed) {
    *failed = -1;
    int S = opt.batch;
    if (S == 0) S = 1024;
    if (S < 32 || S > 2048 || S % 32) return fail(BM_ERR_ARG, "batch must be a multiple of 32 in [32, 2048]");
    cudaStream_t s = (cudaStream_t)opt.stream;
    const bool host_io = opt.host_io != 0;
    // automatic path: every instance starts on the split; its first step (run before the
    // graph) decides whether its loop inside the graph runs on fp16
    const bool auto_path = opt.path == BM_PATH_TC_AUTO;
    const int path = auto_path ? (int)BM_PATH_TC_SPLIT3 : opt.path;
    const bool tc = is_tc_path(path);
    Timer tm(s);
    tm.mark();  // 0
    SweepTimer stimer(s);
    stimer.on = false;  // no event records inside graph bodies
    Arena ar(&opt, s);  // batch-wide state
    // One slab arena for the scratch of every instance: a few 64 MB blocks instead of
    // several blocks per instance (each block is one call of the caller's allocator)
    std::unique_ptr<Arena> scratch(new Arena(&opt, s, true));
    std::vector<BatchItem> items(count);
    DeviceState* sts;
    int* bads;
    unsigned* iters;
    ALLOC(sts, DeviceState, std::max(count, 1));
    ALLOC(bads, int, std::max(count, 1));
    ALLOC(iters, unsigned, std::max(count, 1));
    TRY_CUDA(cudaMemsetAsync(sts, 0, sizeof(DeviceState) * std::max(count, 1), s));
    TRY_CUDA(cudaMemsetAsync(bads, 0, sizeof(int) * std::max(count, 1), s));
    TRY_CUDA(cudaMemsetAsync(iters, 0, sizeof(unsigned) * std::max(count, 1), s));
    const int sms = device_sm_count();
    auto tag = [&](int i, bm_status rs) {
        *failed = i;
        if (statuses) statuses[i] = rs;
        g_last_error = "instance " + std::to_string(i) + ": " + g_last_error;
        return rs;
    };
    // 1. prep of every instance
    for (int i = 0; i < count; ++i) {
        BatchItem& it = items[i];
        it.ar = scratch.get();
        it.n = inst[i].n;
        it.d = inst[i].d;
        it.eps2 = (double)inst[i].eps * (double)inst[i].eps;
        if (it.n == 0) continue;
        bm_status rs = batch_prep(it, inst[i], opt, tc, path, sts + i, bads + i, s);
        if (rs != BM_OK) return tag(i, rs);
    }
    std::vector<float> norms(std::max(count, 1), 0.f);
    {
        std::vector<int> hbad(std::max(count, 1));
        std::vector<DeviceState> hs0(std::max(count, 1));
        TRY_CUDA(cudaMemcpyAsync(hbad.data(), bads, sizeof(int) * std::max(count, 1), cudaMemcpyDeviceToHost, s));
        TRY_CUDA(cudaMemcpyAsync(hs0.data(), sts, sizeof(DeviceState) * std::max(count, 1), cudaMemcpyDeviceToHost, s));
        TRY_SYNC(s, "prep of all instances");
        for (int i = 0; i < count; ++i)
            if (hbad[i]) return tag(i, fail(BM_ERR_ARG, "input holds NaN or Inf"));
        for (int i = 0; i < count; ++i) {   // fp16 operands at each instance's scale, band half-width
            BatchItem& it = items[i];
            if (it.n == 0) continue;
            float nx;
            std::memcpy(&nx, &hs0[i].max_norm_bits, sizeof(float));
            norms[i] = nx;
            bm_status rs = finish_prep(it.st, path, it.d, it.eps2, (double)inst[i].eps, true, nx, &it.px, nullptr, s);
            if (rs != BM_OK) return tag(i, rs);
        }
    }
    tm.mark();  // 1: prep done
    // 2. greedy buffers (the state starts zeroed: the first step requests 32 candidates);
    //    each instance's largest batch is its own (an autotuned table) or opt.batch
    for (int i = 0; i < count; ++i) {
        BatchItem& it = items[i];
        if (it.n == 0) continue;
        const int Si = inst[i].batch ? inst[i].batch : S;
        it.step_cap = (unsigned long long)std::min<long long>(std::max<long long>(32 * it.n, 1LL << 16), 1LL << 22);
        if (tc) it.step_cap = std::max<unsigned long long>(it.step_cap, (unsigned long long)sms * 2048);
        it.mem_cap = (unsigned long long)std::max<long long>(4 * it.n, 1LL << 16);
        bm_status rs = greedy_setup(it.px, it.eps2, path, Si, *it.ar, s, it.st, it.step_cap, it.mem_cap, nullptr,
                                    nullptr, 0, it.gc);
        if (rs != BM_OK) return tag(i, rs);
    }
    // 2b. automatic path: the first step of every instance on the split, then each instance
    //     picks its representation for the graph from its band (as greedy_drive's first step)
    if (auto_path) {
        for (int i = 0; i < count; ++i) {
            BatchItem& it = items[i];
            if (it.n == 0) continue;
            bm_status rs = greedy_enqueue_step(it.gc, it.px, *it.ar, stimer, s);
            if (rs != BM_OK) return tag(i, rs);
        }
        std::vector<DeviceState> h1(std::max(count, 1));
        TRY_CUDA(cudaMemcpyAsync(h1.data(), sts, sizeof(DeviceState) * std::max(count, 1), cudaMemcpyDeviceToHost, s));
        TRY_SYNC(s, "the first greedy step of all instances");
        for (int i = 0; i < count; ++i) {
            BatchItem& it = items[i];
            if (it.n == 0 || h1[i].done || h1[i].error || h1[i].tile_pairs == 0) continue;
            const double eps = std::sqrt(it.eps2);
            const int e = fp16_scale_exp((double)norms[i], eps);
            const double d16 = band_halfwidth(BM_PATH_TC_FP16, it.d, tile_config_for(it.d, 1).d_pad, it.eps2, norms[i],
                                              norms[i], e) * std::ldexp(1.0, -2 * e);
            const double d3 = band_halfwidth(BM_PATH_TC_SPLIT3, it.d, it.px.d_pad, it.eps2, norms[i], norms[i], 0);
            const double predicted = (double)h1[i].band_pairs / (double)h1[i].tile_pairs * (d16 / d3);
            if (predicted < kAutoPredictFraction) {
                bm_status rs = switch_path(it.gc, it.px, *it.ar, s, BM_PATH_TC_FP16, norms[i], 1);
                if (rs != BM_OK) return tag(i, rs);
            }
        }
    }
    // 3. one graph: a WHILE node per instance, no edges between them
    {
        GraphGuard gg;
        TRY_CUDA(cudaStreamCreateWithFlags(&gg.cs, cudaStreamNonBlocking));
        TRY_CUDA(cudaGraphCreate(&gg.graph, 0));
        int nodes = 0;
        for (int i = 0; i < count; ++i) {
            BatchItem& it = items[i];
            if (it.n == 0) continue;
            bm_status rs = batch_capture(it, gg, iters + i, stimer);
            if (rs != BM_OK) return tag(i, rs);
            ++nodes;
        }
        if (nodes) {
            TRY_CUDA(cudaGraphInstantiate(&gg.exec, gg.graph, 0));
            tm.mark();  // 2: graph built
            TRY_CUDA(cudaGraphLaunch(gg.exec, s));
        } else {
            tm.mark();
        }
        tm.mark();  // 3: graph done
        TRY_SYNC(s, "the graph of greedy loops");
    }
    // 4. states; an instance stopped inside the graph (buffer overflow) is finished by
    //    the host loop
    std::vector<unsigned> hiters(std::max(count, 1));
    std::vector<DeviceState> hst(std::max(count, 1));
    TRY_CUDA(cudaMemcpyAsync(hiters.data(), iters, sizeof(unsigned) * std::max(count, 1), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaMemcpyAsync(hst.data(), sts, sizeof(DeviceState) * std::max(count, 1), cudaMemcpyDeviceToHost, s));
    TRY_SYNC(s, "reading the instance states");
    std::vector<long long> executed(std::max(count, 1), 0);
    {
        HostState hs;
        for (int i = 0; i < count; ++i) {
            BatchItem& it = items[i];
            if (it.n == 0) continue;
            executed[i] = (long long)hiters[i] * it.body_kernels;
            if (!hst[i].done || hst[i].error) {
                const long long k0 = g_kernel_launches;
                bm_status rs = greedy_drive(it.gc, it.px, *it.ar, s, hs, it.step_cap, it.mem_cap, hst[i], stimer, true);
                if (rs != BM_OK) return tag(i, rs);
                executed[i] += g_kernel_launches - k0;
            }
            release_sweep_out(*it.ar, it.gc.so, false);
        }
    }
    // 5. the tails as one build: memberships of all instances renumbered into global
    //    rows and points, then one sort, one CSR and one nerve pass (bm_batch.cu)
    std::vector<int> live;   // instances with points
    for (int i = 0; i < count; ++i)
        if (items[i].n > 0) live.push_back(i);
    const int nl = (int)live.size();
    std::vector<long long> row_base(nl + 1, 0), pt_base(nl + 1, 0), key_off(nl + 1, 0);
    std::vector<const unsigned long long*> srcs(std::max(nl, 1), nullptr);
    for (int k = 0; k < nl; ++k) {
        const int i = live[k];
        row_base[k + 1] = row_base[k] + hst[i].n_landmarks;
        pt_base[k + 1] = pt_base[k] + items[i].n;
        key_off[k + 1] = key_off[k] + (long long)hst[i].mem_count;
        srcs[k] = items[i].gc.g.mem_keys;
    }
    const long long L_all = row_base[nl], n_all = pt_base[nl], nnz_all = key_off[nl];
    if (n_all > 0x7fffffffLL || L_all > 0x7fffffffLL)
        return fail(BM_ERR_CAPACITY, "a batch holds more than 2^31-1 points or landmarks in total; split it");
    long long *d_rb, *d_pb, *d_ko, *d_bounds;
    const unsigned long long** d_srcs;
    ALLOC(d_rb, long long, nl + 1);
    ALLOC(d_pb, long long, nl + 1);
    ALLOC(d_ko, long long, nl + 1);
    ALLOC(d_bounds, long long, nl + 1);
    ALLOC(d_srcs, const unsigned long long*, std::max(nl, 1));
    TRY_CUDA(cudaMemcpyAsync(d_rb, row_base.data(), sizeof(long long) * (nl + 1), cudaMemcpyHostToDevice, s));
    TRY_CUDA(cudaMemcpyAsync(d_pb, pt_base.data(), sizeof(long long) * (nl + 1), cudaMemcpyHostToDevice, s));
    TRY_CUDA(cudaMemcpyAsync(d_ko, key_off.data(), sizeof(long long) * (nl + 1), cudaMemcpyHostToDevice, s));
    TRY_CUDA(cudaMemcpyAsync(d_srcs, srcs.data(), sizeof(void*) * std::max(nl, 1), cudaMemcpyHostToDevice, s));
    unsigned long long* gkeys;
    ALLOC(gkeys, unsigned long long, std::max<long long>(nnz_all, 1));
    TRY_CUDA(launch_gather_batch_keys(d_srcs, d_ko, d_rb, d_pb, nl, nnz_all, gkeys, s));
    long long* goff = nullptr;
    int* gids = nullptr;
    int* gedges = nullptr;
    long long E_all = 0, pairs_all = 0;
    if (nl > 0) {
        bm_status rs = members_and_edges(ar, s, opt, n_all, L_all, nnz_all, gkeys, nullptr, &goff, &gids, &gedges,
                                         &E_all, &pairs_all);
        if (rs != BM_OK) return rs;
        TRY_CUDA(launch_edge_bounds(gedges, E_all, d_rb, nl, d_bounds, s));
    }
    std::vector<long long> bounds(nl + 1, 0);
    TRY_CUDA(cudaMemcpyAsync(bounds.data(), d_bounds, sizeof(long long) * (nl + 1), cudaMemcpyDeviceToHost, s));
    TRY_SYNC(s, "the membership and nerve passes over all instances");
    // 6. per-instance outputs cut from the global results
    std::vector<BatchSplit> parts(std::max(nl, 1));
    for (int k = 0; k < nl; ++k) {
        const int i = live[k];
        Arena& iar = *items[i].ar;
        BatchSplit& p = parts[k];
        p.row_base = row_base[k];
        p.rows = row_base[k + 1] - row_base[k];
        p.pt_base = pt_base[k];
        p.nnz = key_off[k + 1] - key_off[k];
        p.edge0 = bounds[k];
        p.n_edges = bounds[k + 1] - bounds[k];
        p.offsets = (long long*)iar.get_standalone(sizeof(long long) * (p.rows + 1));
        p.ids = (int*)iar.get_standalone(sizeof(int) * std::max<long long>(p.nnz, 1));
        p.edges = (int*)iar.get_standalone(sizeof(int) * 2 * std::max<long long>(p.n_edges, 1));
        if (!p.offsets || !p.ids || !p.edges) return tag(i, fail(BM_ERR_NOMEM, "result buffers"));
    }
    BatchSplit* d_parts;
    ALLOC(d_parts, BatchSplit, std::max(nl, 1));
    TRY_CUDA(cudaMemcpyAsync(d_parts, parts.data(), sizeof(BatchSplit) * std::max(nl, 1), cudaMemcpyHostToDevice, s));
    if (nl > 0) TRY_CUDA(launch_split_batch(d_parts, nl, goff, gids, gedges, s));
    int k = 0;
    for (int i = 0; i < count; ++i) {
        BatchItem& it = items[i];
        Arena& iar = *it.ar;
        bm_graph g;
        std::memset(&g, 0, sizeof(g));
        bm_status rs;
        if (it.n == 0) {
            int* lm = (int*)iar.get(sizeof(int));
            long long* off = (long long*)iar.get(sizeof(long long));
            int* ids = (int*)iar.get(sizeof(int));
            int* edges = (int*)iar.get(2 * sizeof(int));
            if (!lm || !off || !ids || !edges) return tag(i, fail(BM_ERR_NOMEM, "empty result"));
            if (cudaMemsetAsync(off, 0, sizeof(long long), s) != cudaSuccess) {
                cudaGetLastError();
                return tag(i, fail(BM_ERR_CUDA, "memset"));
            }
            rs = hand_over(iar, s, host_io, lm, off, ids, edges, 0, 0, 0, g);
        } else {
            const BatchSplit& p = parts[k++];
            rs = hand_over(iar, s, host_io, it.gc.g.landmarks, p.offsets, p.ids, p.edges, p.rows, p.nnz, p.n_edges, g);
        }
        if (rs != BM_OK) return tag(i, rs);
        const DeviceState& fin = hst[i];
        g.stats.distance_evals = (int64_t)g.n_landmarks * it.n;
        g.stats.tile_pairs = (int64_t)fin.tile_pairs;
        g.stats.band_pairs = (int64_t)fin.band_pairs;
        g.stats.greedy_steps = (int64_t)fin.steps;
        g.stats.candidates = (int64_t)fin.candidates;
        g.stats.edge_pairs = 0;   // witnessed pairs are counted for the whole batch only
        g.stats.band_delta = fin.delta;
        g.stats.centred = fin.centred;
        g.stats.path = it.n ? it.gc.path : path;
        g.stats.kernel_launches = executed[i];
        outs[i] = g;
        if (statuses) statuses[i] = BM_OK;
    }
    TRY_SYNC(s, "the split of the results");
    scratch.reset();   // every instance's scratch
    tm.mark();  // 4
    const double total = tm.ms(0, 4), prep = tm.ms(0, 1), graph = tm.ms(2, 3), tail = tm.ms(3, 4);
    for (int i = 0; i < count; ++i) {
        outs[i].stats.ms_total = total;
        outs[i].stats.ms_prep = prep;
        outs[i].stats.ms_greedy = graph;
        outs[i].stats.ms_members = tail;
    }
    return BM_OK;
}

// Ball Mapper on farthest-point landmarks (Sec. 2.2): the selection loop as one graph
// launch (a WHILE node repeating the pass kernel), then memberships and edges of those
// landmarks through the fixed-landmark build.  Arguments validated, n >= 1.
bm_status fps_build(const float* X, long long n, int d, float eps, long long first, const bm_options& opt,
                    bm_graph* out) {
    cudaStream_t s = (cudaStream_t)opt.stream;
    const bool host_io = opt.host_io != 0;
    const double eps2 = (double)eps * (double)eps;
    Timer tm(s);
    tm.mark();
    const long long launches0 = g_kernel_launches;
    Arena ar(&opt, s);
    bm_status rs = BM_OK;
    const float* dX = stage_input(X, n, d, host_io, ar, s, &rs);
    if (rs != BM_OK) return rs;
    int* bad;
    ALLOC(bad, int, 1);
    TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    TRY_CUDA(launch_finite_check(dX, n * d, bad, s));
    int hbad = 0;
    TRY_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    if (hbad) return fail(BM_ERR_ARG, "input holds NaN or Inf");
    double* mind;
    int* lm;
    FpsState* st;
    double* part_v;
    int* part_i;
    unsigned* ticket;
    const int G = fps_grid(n);
    ALLOC(mind, double, n);
    ALLOC(lm, int, n);
    ALLOC(st, FpsState, 1);
    ALLOC(part_v, double, G);
    ALLOC(part_i, int, G);
    ALLOC(ticket, unsigned, 1);
    TRY_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s));
    TRY_CUDA(launch_fps_init(mind, n, lm, st, first, s));
    tm.mark();  // 1: set-up done
    {
        GraphGuard gg;
        TRY_CUDA(cudaStreamCreateWithFlags(&gg.cs, cudaStreamNonBlocking));
        TRY_CUDA(cudaGraphCreate(&gg.graph, 0));
        cudaGraphConditionalHandle h;
        TRY_CUDA(cudaGraphConditionalHandleCreate(&h, gg.graph, 1u, cudaGraphCondAssignDefault));
        alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
        std::memset(cp_raw, 0, sizeof(cp_raw));
        cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        TRY_CUDA(cudaGraphAddNode(&node, gg.graph, nullptr, nullptr, 0, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        TRY_CUDA(cudaStreamBeginCaptureToGraph(gg.cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        const cudaError_t le = launch_fps_step(dX, n, d, eps2, mind, lm, st, part_v, part_i, ticket, h, true, gg.cs);
        cudaGraph_t captured = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(gg.cs, &captured);
        TRY_CUDA(le);
        TRY_CUDA(ee);
        TRY_CUDA(cudaGraphInstantiate(&gg.exec, gg.graph, 0));
        TRY_CUDA(cudaGraphLaunch(gg.exec, s));
        TRY_SYNC(s, "the farthest-point selection loop");
    }
    tm.mark();  // 2: selection done
    FpsState hst;
    TRY_CUDA(cudaMemcpyAsync(&hst, st, sizeof(FpsState), cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    if (hst.error) return fail(BM_ERR_CUDA, "farthest-point loop passed its iteration bound");
    const long long L = hst.count;
    std::vector<int> hl;
    const int32_t* fixed = lm;
    if (host_io) {   // the fixed-landmark build reads host landmarks in host I/O mode
        hl.resize((size_t)std::max<long long>(L, 1));
        TRY_CUDA(cudaMemcpyAsync(hl.data(), lm, sizeof(int) * L, cudaMemcpyDeviceToHost, s));
        TRY_CUDA(cudaStreamSynchronize(s));
        fixed = hl.data();
    }
    rs = build_graph(X, n, d, eps, opt, nullptr, 0, fixed, L, out);
    if (rs != BM_OK) return rs;
    const double ms_sel = tm.ms(1, 2), ms_setup = tm.ms(0, 1);
    out->stats.greedy_steps = (int64_t)hst.iterations;
    out->stats.candidates = (int64_t)hst.iterations * n;   // points examined by the passes
    out->stats.ms_greedy += ms_sel;
    out->stats.ms_prep += ms_setup;
    out->stats.ms_total += ms_sel + ms_setup;
    out->stats.kernel_launches = g_kernel_launches - launches0 + (int64_t)hst.iterations - 1;
    return BM_OK;
}

}  // namespace
}  // namespace bm

extern "C" {

void bm_options_init(bm_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->path = BM_PATH_TC_AUTO;
}

const char* bm_status_string(bm_status s) {
    switch (s) {
        case BM_OK: return "ok";
        case BM_ERR_ARG: return "invalid argument";
        case BM_ERR_CUDA: return "CUDA error";
        case BM_ERR_NOMEM: return "out of memory";
        case BM_ERR_CAPACITY: return "capacity exceeded";
        case BM_ERR_TIMEOUT: return "device wait timed out";
        case BM_ERR_UNSUPPORTED: return "unsupported device";
    }
    return "unknown status";
}

const char* bm_last_error(void) { return g_last_error.c_str(); }

int32_t bm_version(void) { return 100; }

void bm_csr_free(bm_csr* csr, const bm_options* opt) {
    if (!csr) return;
    if (csr->on_host) {
        std::free(csr->offsets);
        std::free(csr->ids);
        std::free(csr->dists);
    } else {
        cudaStream_t s = opt ? (cudaStream_t)opt->stream : nullptr;
        device_free(opt, s, csr->offsets);
        device_free(opt, s, csr->ids);
        device_free(opt, s, csr->dists);
    }
    std::memset(csr, 0, sizeof(*csr));
}

void bm_graph_free(bm_graph* g, const bm_options* opt) {
    if (!g) return;
    if (g->on_host) {
        std::free(g->landmarks);
        std::free(g->edges);
    } else {
        cudaStream_t s = opt ? (cudaStream_t)opt->stream : nullptr;
        device_free(opt, s, g->landmarks);
        device_free(opt, s, g->edges);
    }
    bm_csr_free(&g->members, opt);
    std::memset(g, 0, sizeof(*g));
}

bm_status bm_range_query(const float* X, int64_t n, int32_t d, const float* Q, int64_t m, float eps,
                         const bm_options* opt_in, bm_csr* out, bm_stats* stats) {
    if (!out) return fail(BM_ERR_ARG, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    if (stats) std::memset(stats, 0, sizeof(*stats));
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    bm_status vs = validate_points(X, n, d, "X");
    if (vs != BM_OK) return vs;
    vs = validate_points(Q, m, d, "Q");
    if (vs != BM_OK) return vs;
    vs = validate_eps(eps);
    if (vs != BM_OK) return vs;
    vs = validate_centring(opt.centring);
    if (vs != BM_OK) return vs;
    vs = check_device(opt.path);
    if (vs != BM_OK) return vs;
    return range_core(X, n, d, Q, m, eps, opt, nullptr, 0, nullptr, out, stats);
}

bm_status bm_build(const float* X, int64_t n, int32_t d, float eps, const bm_options* opt_in, bm_graph* out) {
    if (!out) return fail(BM_ERR_ARG, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    bm_status vs = validate_points(X, n, d, "X");
    if (vs != BM_OK) return vs;
    vs = validate_eps(eps);
    if (vs != BM_OK) return vs;
    vs = validate_batch(opt.batch, kMaxBatch);   // arguments first, then the device
    if (vs != BM_OK) return vs;
    vs = validate_centring(opt.centring);
    if (vs != BM_OK) return vs;
    vs = check_device(opt.path);
    if (vs != BM_OK) return vs;
    return build_graph(X, n, d, eps, opt, nullptr, 0, nullptr, 0, out);
}

bm_status bm_build_fps(const float* X, int64_t n, int32_t d, float eps, int64_t first, const bm_options* opt_in,
                       bm_graph* out) {
    if (!out) return fail(BM_ERR_ARG, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    bm_status vs = validate_points(X, n, d, "X");
    if (vs != BM_OK) return vs;
    vs = validate_eps(eps);
    if (vs != BM_OK) return vs;
    if (n > 0 && (first < 0 || first >= n)) return fail(BM_ERR_ARG, "first must be in [0, n)");
    vs = check_device(opt.path);
    if (vs != BM_OK) return vs;
    if (n == 0) return build_graph(X, 0, d, eps, opt, nullptr, 0, nullptr, 0, out);
    bm_status rs = fps_build(X, n, d, eps, first, opt, out);
    if (rs != BM_OK) {
        const std::string msg = g_last_error;
        bm_graph_free(out, &opt);
        g_last_error = msg;
    }
    return rs;
}

bm_status bm_color(const int64_t* offsets, const int32_t* ids, int64_t rows, const float* f, int64_t n, int32_t stat,
                   const bm_options* opt_in, double* out) {
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    if (rows < 0 || n < 0 || n > 0x7fffffffLL) return fail(BM_ERR_ARG, "rows or n out of range");
    if (stat < BM_COLOR_MEAN || stat > BM_COLOR_MAX) return fail(BM_ERR_ARG, "unknown coloring statistic");
    if (rows > 0 && (!offsets || !out)) return fail(BM_ERR_ARG, "offsets or out is NULL");
    if (n > 0 && !f) return fail(BM_ERR_ARG, "f is NULL");
    bm_status vs = check_device(opt.path);
    if (vs != BM_OK) return vs;
    if (rows == 0) return BM_OK;
    cudaStream_t s = (cudaStream_t)opt.stream;
    const bool host_io = opt.host_io != 0;
    Arena ar(&opt, s);
    const long long* doff = (const long long*)offsets;
    const int* dids = ids;
    const float* df = f;
    double* dout = out;
    if (host_io) {
        const long long nnz = offsets[rows];
        if (nnz < 0 || offsets[0] < 0 || offsets[0] > nnz) return fail(BM_ERR_ARG, "offsets are not a CSR");
        if (nnz > 0 && !ids) return fail(BM_ERR_ARG, "ids is NULL");
        long long* o;
        int* i;
        float* fv;
        ALLOC(o, long long, rows + 1);
        ALLOC(i, int, std::max<long long>(nnz, 1));
        ALLOC(fv, float, std::max<long long>(n, 1));
        ALLOC(dout, double, rows);
        TRY_CUDA(cudaMemcpyAsync(o, offsets, sizeof(long long) * (rows + 1), cudaMemcpyHostToDevice, s));
        if (nnz) TRY_CUDA(cudaMemcpyAsync(i, ids, sizeof(int) * nnz, cudaMemcpyHostToDevice, s));
        if (n) TRY_CUDA(cudaMemcpyAsync(fv, f, sizeof(float) * n, cudaMemcpyHostToDevice, s));
        doff = o;
        dids = i;
        df = fv;
    }
    int* bad;
    ALLOC(bad, int, 1);
    TRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    TRY_CUDA(launch_color(doff, dids, rows, df, n, stat, dout, bad, s));
    int hbad = 0;
    TRY_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (host_io) TRY_CUDA(cudaMemcpyAsync(out, dout, sizeof(double) * rows, cudaMemcpyDeviceToHost, s));
    TRY_CUDA(cudaStreamSynchronize(s));
    if (hbad & 2) return fail(BM_ERR_ARG, "f holds NaN or Inf");
    if (hbad & 1) return fail(BM_ERR_ARG, "a membership id lies outside [0, n)");
    return BM_OK;
}

static bm_status validate_knn(const float* X, int64_t n, int32_t d, int32_t k, const bm_options& opt) {
    bm_status vs = validate_points(X, n, d, "X");
    if (vs != BM_OK) return vs;
    if (n < 1) return fail(BM_ERR_ARG, "the k-th nearest neighbour needs n >= 1");
    if (k < 1 || k > n || k > 1024) return fail(BM_ERR_ARG, "k must be in [1, min(n, 1024)]");
    return check_device(opt.path);
}

bm_status bm_knn_dist(const float* X, int64_t n, int32_t d, int32_t k, const bm_options* opt_in, double* kdist,
                      bm_stats* stats) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (!kdist) return fail(BM_ERR_ARG, "kdist is NULL");
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    bm_status vs = validate_knn(X, n, d, k, opt);
    if (vs != BM_OK) return vs;
    return knn_core(X, n, d, k, opt, kdist, nullptr, stats);
}

bm_status bm_occupancy_eps(const float* X, int64_t n, int32_t d, int32_t k, const bm_options* opt_in, double* eps,
                           bm_stats* stats) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (!eps) return fail(BM_ERR_ARG, "eps is NULL");
    *eps = 0.0;
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    bm_status vs = validate_knn(X, n, d, k, opt);
    if (vs != BM_OK) return vs;
    return knn_core(X, n, d, k, opt, nullptr, eps, stats);
}

int64_t bm_set_nerve_bitmap_bytes(int64_t bytes) { return edges_set_bitmap_budget(bytes); }

double bm_band_halfwidth(int32_t path, int32_t d, int32_t d_pad, double n_a, double n_b, double phi_a,
                         double phi_b) {
    return band_halfwidth_core(path, d, d_pad, n_a, n_b, phi_a, phi_b);
}

int32_t bm_tile_shapes(bm_tile_config* out, int32_t max) {
    std::vector<TileConfig> v(64);
    const int n = tile_shapes(v.data(), (int)v.size());
    for (int i = 0; out && i < n && i < max; ++i) out[i] = {v[i].d_pad, v[i].ck, v[i].nt, v[i].bbuf, v[i].astg};
    return n;
}

bm_status bm_get_tile_config(int32_t d, bm_tile_config* out) {
    if (!out) return fail(BM_ERR_ARG, "out is NULL");
    if (d < 1 || d > 65536) return fail(BM_ERR_ARG, "d out of range [1, 65536]");
    const TileConfig c = tile_config_for(d);
    *out = {c.d_pad, c.ck, c.nt, c.bbuf, c.astg};
    return BM_OK;
}

bm_status bm_set_tile_config(int32_t d, const bm_tile_config* cfg) {
    if (d < 1 || d > 65536) return fail(BM_ERR_ARG, "d out of range [1, 65536]");
    std::string why;
    if (cfg) {
        const TileConfig c = {cfg->d_pad, cfg->ck, cfg->nt, cfg->bbuf, cfg->astg};
        if (!tile_config_set(d, &c, &why)) return fail(BM_ERR_ARG, "tile configuration rejected: " + why);
    } else {
        tile_config_set(d, nullptr, &why);
    }
    return BM_OK;
}

bm_status bm_build_batched(const bm_instance* inst, int32_t count, const bm_options* opt_in, bm_graph* outs,
                           int32_t* statuses) {
    if (count < 0) return fail(BM_ERR_ARG, "count < 0");
    if (count > 0 && (!inst || !outs)) return fail(BM_ERR_ARG, "inst or outs is NULL");
    for (int i = 0; i < count; ++i) std::memset(&outs[i], 0, sizeof(bm_graph));
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    for (int i = 0; i < count; ++i) {
        if (statuses) statuses[i] = BM_OK;
        bm_status vs = validate_points(inst[i].X, inst[i].n, inst[i].d, "X");
        if (vs == BM_OK) vs = validate_eps(inst[i].eps);
        if (vs == BM_OK) vs = validate_batch(inst[i].batch, 2048);
        if (vs != BM_OK) {
            if (statuses) statuses[i] = vs;
            g_last_error = "instance " + std::to_string(i) + ": " + g_last_error;
            return vs;
        }
    }
    bm_status vs = validate_batch(opt.batch, 2048);   // arguments first, then the device
    if (vs == BM_OK) vs = validate_centring(opt.centring);
    if (vs != BM_OK) return vs;
    if (opt.want_dists) return fail(BM_ERR_ARG, "bm_build_batched does not return distances (want_dists)");
    vs = check_device(opt.path);
    if (vs != BM_OK) return vs;
    if (count == 0) return BM_OK;
    int failed = -1;
    bm_status rs = build_batched(inst, count, opt, outs, statuses, &failed);
    if (rs != BM_OK) {
        const std::string msg = g_last_error;
        for (int i = 0; i < count; ++i) bm_graph_free(&outs[i], &opt);
        g_last_error = msg;
    }
    return rs;
}

// ------------------------------------------------------------------ inverted file
struct bm_ivf {
    bm::IvfIndex ix;
};

namespace {

// Buffers that live as long as the index: the caller's allocator, else cudaMallocAsync.
void* persistent_alloc(const bm_options& opt, size_t bytes, std::vector<void*>& held) {
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (opt.alloc) p = opt.alloc(bytes, opt.stream, opt.alloc_ctx);
    else if (cudaMallocAsync(&p, bytes, (cudaStream_t)opt.stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) held.push_back(p);
    return p;
}

void free_index(bm_ivf* h) {
    if (!h) return;
    IvfIndex& ix = h->ix;
    void* bufs[] = {ix.centroids, ix.cnorm, ix.cell_off, ix.cell_ids, ix.cell_of, ix.xperm, ix.xnorm, ix.owned_x,
                    ix.pad_off, ix.xpad};
    for (void* b : bufs) device_free(&ix.opt, (cudaStream_t)ix.opt.stream, b);
    delete h;
}

// splitmix64 (Steele, Lea, Flood 2014): the seeded stream of the k-means sample.
uint64_t splitmix64(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

bm_status bm_ivf_train(const float* X, int64_t n, int32_t d, int32_t nlist, int32_t iters, int64_t sample,
                       uint64_t seed, const bm_options* opt_in, bm_ivf** out) {
    if (!out) return fail(BM_ERR_ARG, "out is NULL");
    *out = nullptr;
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    bm_status vs = validate_points(X, n, d, "X");
    if (vs != BM_OK) return vs;
    if (n < 1) return fail(BM_ERR_ARG, "the index needs at least one point");
    if (nlist < 1 || nlist > 4096 || nlist > n) return fail(BM_ERR_ARG, "nlist must be in [1, min(n, 4096)]");
    if (iters < 0 || iters > 1000) return fail(BM_ERR_ARG, "iters must be in [0, 1000]");
    if (sample == 0) sample = std::min<int64_t>(n, 262144);
    if (sample < nlist || sample > n) return fail(BM_ERR_ARG, "sample must be in [nlist, n]");
    vs = check_device(BM_PATH_FP32);
    if (vs != BM_OK) return vs;
    cudaStream_t s = (cudaStream_t)opt.stream;
    bm_ivf* h = new (std::nothrow) bm_ivf;
    if (!h) return fail(BM_ERR_NOMEM, "index handle");
    IvfIndex& ix = h->ix;
    ix.n = n;
    ix.d = d;
    ix.nlist = nlist;
    ix.opt = opt;
    ix.opt.host_io = 0;
    std::vector<void*> held;
    auto bail = [&](bm_status st, const std::string& msg) {
        free_index(h);
        return fail(st, msg);
    };
#define PALLOC(ptr, type, count)                                                                  \
    do {                                                                                          \
        ptr = (type*)persistent_alloc(ix.opt, sizeof(type) * (size_t)(count), held);              \
        if (!ptr) return bail(BM_ERR_NOMEM, "allocation of the index's " #ptr " failed");          \
    } while (0)
#define PTRY(expr)                                                                                \
    do {                                                                                          \
        cudaError_t e__ = (expr);                                                                 \
        if (e__ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                   \
            return bail(BM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e__));         \
        }                                                                                         \
    } while (0)
    {
        Arena ar(&opt, s);
        if (opt.host_io) {
            PALLOC(ix.owned_x, float, n * d);
            PTRY(cudaMemcpyAsync(ix.owned_x, X, sizeof(float) * n * d, cudaMemcpyHostToDevice, s));
            ix.X = ix.owned_x;
        } else {
            ix.X = X;
        }
        // seeded sample: the first `sample` positions of a Fisher-Yates shuffle of 0..n-1;
        // its first nlist points initialise the centroids
        std::vector<int> perm((size_t)n);
        for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = (int)i;
        uint64_t st64 = seed;
        for (int64_t i = 0; i < sample; ++i) {
            const int64_t j = i + (int64_t)(splitmix64(st64) % (uint64_t)(n - i));
            std::swap(perm[(size_t)i], perm[(size_t)j]);
        }
        int* dsample = (int*)ar.get(sizeof(int) * (size_t)sample);
        if (!dsample) return bail(BM_ERR_NOMEM, "sample ids");
        PTRY(cudaMemcpyAsync(dsample, perm.data(), sizeof(int) * (size_t)sample, cudaMemcpyHostToDevice, s));
        PALLOC(ix.xnorm, float, n);
        PTRY(launch_row_norms(ix.X, n, d, ix.xnorm, s));
        PALLOC(ix.centroids, float, (long long)nlist * d);
        PALLOC(ix.cnorm, float, nlist);
        PTRY(launch_gather_rows(ix.X, dsample, nlist, d, ix.centroids, s));
        const size_t big = (size_t)std::max<int64_t>(n, sample);
        unsigned long long* best = (unsigned long long*)ar.get(sizeof(unsigned long long) * big);
        unsigned long long* keys = (unsigned long long*)ar.get(sizeof(unsigned long long) * big);
        unsigned long long* tmp = (unsigned long long*)ar.get(sizeof(unsigned long long) * big);
        long long* moff = (long long*)ar.get(sizeof(long long) * (nlist + 1));
        int* mids = (int*)ar.get(sizeof(int) * (size_t)sample);
        if (!best || !keys || !tmp || !moff || !mids) return bail(BM_ERR_NOMEM, "k-means scratch");
        const std::vector<int> shifts = digit_shifts(bits_for(n - 1), bits_for(nlist - 1));
        for (int it = 0; it < iters; ++it) {   // Lloyd iterations on the sample
            PTRY(launch_row_norms(ix.centroids, nlist, d, ix.cnorm, s));
            PTRY(launch_nearest_centroid(ix.X, dsample, sample, ix.xnorm, ix.centroids, ix.cnorm, nlist, d, best, s));
            PTRY(launch_unpack_cells(best, dsample, sample, nullptr, keys, s));
            unsigned long long* sorted = nullptr;
            PTRY(radix_sort_u64(keys, tmp, sample, shifts, ar, s, &sorted));
            PTRY(launch_csr_from_sorted(sorted, sample, nlist, moff, mids, s));
            PTRY(launch_cell_means(ix.X, moff, mids, nlist, d, ix.centroids, s));
        }
        // every point joins its nearest centroid; cells in point order
        PTRY(launch_row_norms(ix.centroids, nlist, d, ix.cnorm, s));
        PTRY(launch_nearest_centroid(ix.X, nullptr, n, ix.xnorm, ix.centroids, ix.cnorm, nlist, d, best, s));
        PALLOC(ix.cell_of, int, n);
        PTRY(launch_unpack_cells(best, nullptr, n, ix.cell_of, keys, s));
        unsigned long long* sorted = nullptr;
        PTRY(radix_sort_u64(keys, tmp, n, shifts, ar, s, &sorted));
        PALLOC(ix.cell_off, long long, nlist + 1);
        PALLOC(ix.cell_ids, int, n);
        PTRY(launch_csr_from_sorted(sorted, n, nlist, ix.cell_off, ix.cell_ids, s));
        PALLOC(ix.xperm, float, n * d);
        PTRY(launch_gather_rows(ix.X, ix.cell_ids, n, d, ix.xperm, s));
        // the tensor-core scan's layout: every cell padded to a multiple of 256 rows
        PALLOC(ix.pad_off, long long, nlist + 1);
        long long* pcnt = (long long*)ar.get(sizeof(long long) * (nlist + 1));
        if (!pcnt) return bail(BM_ERR_NOMEM, "padding scratch");
        PTRY(launch_cell_pad_offsets(ix.cell_off, nlist, 256, pcnt, ix.pad_off, ar, s));
        std::vector<long long> hpo((size_t)nlist + 1);
        PTRY(cudaMemcpyAsync(hpo.data(), ix.pad_off, sizeof(long long) * (nlist + 1), cudaMemcpyDeviceToHost, s));
        PTRY(cudaStreamSynchronize(s));
        ix.npad = hpo[(size_t)nlist];
        for (int c = 0; c < nlist; ++c)
            ix.max_cell_tiles = std::max<long long>(ix.max_cell_tiles, (hpo[(size_t)c + 1] - hpo[(size_t)c]) / 256);
        PALLOC(ix.xpad, float, std::max<long long>(ix.npad, 1) * d);
        PTRY(launch_pad_rows(ix.xperm, ix.cell_off, ix.pad_off, nlist, ix.npad, d, ix.xpad, s));
        PTRY(cudaStreamSynchronize(s));
    }
#undef PALLOC
#undef PTRY
    *out = h;
    return BM_OK;
}

void bm_ivf_free(bm_ivf* idx) { free_index(idx); }

bm_status bm_ivf_info(const bm_ivf* idx, int64_t* n, int32_t* d, int32_t* nlist, const int32_t** cell_of,
                      const float** centroids) {
    if (!idx) return fail(BM_ERR_ARG, "index is NULL");
    if (n) *n = idx->ix.n;
    if (d) *d = idx->ix.d;
    if (nlist) *nlist = idx->ix.nlist;
    if (cell_of) *cell_of = idx->ix.cell_of;
    if (centroids) *centroids = idx->ix.centroids;
    return BM_OK;
}

bm_status bm_ivf_range_query(const bm_ivf* idx, const float* Q, int64_t m, float eps, int32_t nprobe,
                             const bm_options* opt_in, bm_csr* out, int32_t* probes, bm_stats* stats) {
    if (!out) return fail(BM_ERR_ARG, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    if (!idx) return fail(BM_ERR_ARG, "index is NULL");
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    const IvfIndex& ix = idx->ix;
    bm_status vs = validate_points(Q, m, ix.d, "Q");
    if (vs != BM_OK) return vs;
    vs = validate_eps(eps);
    if (vs != BM_OK) return vs;
    if (nprobe < 1 || nprobe > ix.nlist) return fail(BM_ERR_ARG, "nprobe must be in [1, nlist]");
    vs = check_device(BM_PATH_FP32);
    if (vs != BM_OK) return vs;
    return range_core(ix.X, ix.n, ix.d, Q, m, eps, opt, &ix, nprobe, probes, out, stats);
}

bm_status bm_build_ivf(const bm_ivf* idx, float eps, int32_t nprobe, const int32_t* landmarks, int64_t n_landmarks,
                       const bm_options* opt_in, bm_graph* out) {
    if (!out) return fail(BM_ERR_ARG, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    if (!idx) return fail(BM_ERR_ARG, "index is NULL");
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    const IvfIndex& ix = idx->ix;
    bm_status vs = validate_eps(eps);
    if (vs != BM_OK) return vs;
    if (nprobe < 1 || nprobe > ix.nlist) return fail(BM_ERR_ARG, "nprobe must be in [1, nlist]");
    if (landmarks && (n_landmarks < 0 || n_landmarks > ix.n)) return fail(BM_ERR_ARG, "n_landmarks out of range");
    vs = check_device(BM_PATH_FP32);
    if (vs != BM_OK) return vs;
    return build_graph(ix.X, ix.n, ix.d, eps, opt, &ix, nprobe, landmarks, landmarks ? n_landmarks : 0, out);
}

}  // extern "C"

// ------------------------------------------------------------------ graph index
struct bm_gidx {
    bm::GraphIndex gx;
};

namespace {

void free_gidx(bm_gidx* h) {
    if (!h) return;
    GraphIndex& gx = h->gx;
    void* bufs[] = {gx.adj_off, gx.adj, gx.owned_x};
    for (void* b : bufs) device_free(&gx.opt, (cudaStream_t)gx.opt.stream, b);
    delete h;
}

}  // namespace

bm_status bm_gidx_build(const float* X, int64_t n, int32_t d, int32_t M, int32_t n_entries, const bm_options* opt_in,
                        bm_gidx** out) {
    if (!out) return fail(BM_ERR_ARG, "out is NULL");
    *out = nullptr;
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    bm_status vs = validate_points(X, n, d, "X");
    if (vs != BM_OK) return vs;
    if (n < 2) return fail(BM_ERR_ARG, "the graph index needs at least two points");
    if (M < 1 || M >= n || M > 1023) return fail(BM_ERR_ARG, "M must be in [1, min(n - 1, 1023)]");
    if (n_entries == 0) n_entries = (int32_t)std::min<int64_t>(n, 64);
    if (n_entries < 1 || n_entries > n) return fail(BM_ERR_ARG, "n_entries must be in [1, n]");
    vs = check_device(opt.path);
    if (vs != BM_OK) return vs;
    cudaStream_t s = (cudaStream_t)opt.stream;
    bm_gidx* h = new (std::nothrow) bm_gidx;
    if (!h) return fail(BM_ERR_NOMEM, "index handle");
    GraphIndex& gx = h->gx;
    gx.n = n;
    gx.d = d;
    gx.M = M;
    gx.E = n_entries;
    gx.opt = opt;
    gx.opt.host_io = 0;
    gx.opt.want_dists = 0;
    std::vector<void*> held;
    auto bail = [&](bm_status st, const std::string& msg) {
        free_gidx(h);
        return fail(st, msg);
    };
#define PALLOC(ptr, type, count)                                                                  \
    do {                                                                                          \
        ptr = (type*)persistent_alloc(gx.opt, sizeof(type) * (size_t)(count), held);              \
        if (!ptr) return bail(BM_ERR_NOMEM, "allocation of the index's " #ptr " failed");          \
    } while (0)
#define PTRY(expr)                                                                                \
    do {                                                                                          \
        cudaError_t e__ = (expr);                                                                 \
        if (e__ != cudaSuccess) {                                                                 \
            cudaGetLastError();                                                                   \
            return bail(BM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e__));         \
        }                                                                                         \
    } while (0)
    {
        Arena ar(&opt, s);
        if (opt.host_io) {
            PALLOC(gx.owned_x, float, n * d);
            PTRY(cudaMemcpyAsync(gx.owned_x, X, sizeof(float) * n * d, cudaMemcpyHostToDevice, s));
            gx.X = gx.owned_x;
        } else {
            gx.X = X;
        }
        // the M + 1 nearest points of every row (itself included): per-row radius from the
        // sampled bound, exact range query, then the M nearest others by (D, id)
        const int k = M + 1;
        long long target = std::max<long long>(8LL * k, n / 16);
        target = std::max<long long>(std::min<long long>(target, 65536), k);
        const long long stride = target >= n ? 1 : n / target;
        const long long sN = (n + stride - 1) / stride;
        double* rho = (double*)ar.get(sizeof(double) * n);
        unsigned long long* rmax = (unsigned long long*)ar.get(sizeof(unsigned long long));
        int* bad = (int*)ar.get(sizeof(int));
        if (!rho || !rmax || !bad) return bail(BM_ERR_NOMEM, "graph index scratch");
        PTRY(cudaMemsetAsync(rmax, 0, sizeof(unsigned long long), s));
        PTRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
        PTRY(launch_knn_bound(gx.X, n, d, stride, sN, k, rho, rmax, bad, s));
        int hbad = 0;
        unsigned long long hmax = 0;
        PTRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        PTRY(cudaMemcpyAsync(&hmax, rmax, sizeof(hmax), cudaMemcpyDeviceToHost, s));
        PTRY(cudaStreamSynchronize(s));
        if (hbad) return bail(BM_ERR_ARG, "input holds NaN or Inf, or squared distances that overflow float");
        double r2_max;
        std::memcpy(&r2_max, &hmax, sizeof(double));
        bm_options o2 = gx.opt;
        bm_csr csr;
        const double expect = 1.5 * (double)n * (double)k * ((double)n / (double)sN) + 2.0 * (double)n;
        const unsigned long long hint = (unsigned long long)std::min(expect, (double)n * (double)n);
        bm_status rs = range_core(gx.X, n, d, gx.X, n, 1.0f, o2, nullptr, 0, nullptr, &csr, nullptr, rho, r2_max, hint);
        if (rs != BM_OK) {
            const std::string msg = g_last_error;
            free_gidx(h);
            return fail(rs, msg);
        }
        struct CsrGuard {
            bm_csr* c;
            const bm_options* o;
            ~CsrGuard() { bm_csr_free(c, o); }
        } guard{&csr, &o2};
        const long long nnz = csr.nnz;
        double* D = (double*)ar.get(sizeof(double) * std::max<long long>(nnz, 1));
        double* DM = (double*)ar.get(sizeof(double) * n);
        int* nbr = (int*)ar.get(sizeof(int) * n * M);
        if (!D || !DM || !nbr) return bail(BM_ERR_NOMEM, "graph index scratch");
        PTRY(launch_knn_select(gx.X, d, (const long long*)csr.offsets, n, csr.ids, nnz, D, M, nullptr, bad, s, true,
                               DM));
        PTRY(launch_knn_ids((const long long*)csr.offsets, csr.ids, D, DM, n, M, nbr, bad, s));
        // undirected adjacency: arcs and their reverses, sorted, deduplicated, as CSR
        const long long na = 2 * n * M;
        unsigned long long* keys = (unsigned long long*)ar.get(sizeof(unsigned long long) * na);
        unsigned long long* tmp = (unsigned long long*)ar.get(sizeof(unsigned long long) * na);
        long long* flags = (long long*)ar.get(sizeof(long long) * na);
        long long* pos = (long long*)ar.get(sizeof(long long) * (na + 1));
        if (!keys || !tmp || !flags || !pos) return bail(BM_ERR_NOMEM, "graph index scratch");
        PTRY(launch_arc_keys(nbr, n, M, keys, s));
        unsigned long long* sorted = nullptr;
        PTRY(radix_sort_u64(keys, tmp, na, digit_shifts(bits_for(n - 1), bits_for(n - 1)), ar, s, &sorted));
        unsigned long long* uniq = sorted == keys ? tmp : keys;
        PTRY(launch_unique_sorted(sorted, na, flags, pos, uniq, ar, s));
        long long nu = 0;
        PTRY(cudaMemcpyAsync(&nu, pos + na, sizeof(long long), cudaMemcpyDeviceToHost, s));
        PTRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        PTRY(cudaStreamSynchronize(s));
        if (hbad) return bail(BM_ERR_CUDA, "graph index: a row's ball held fewer than M other points");
        PALLOC(gx.adj_off, long long, n + 1);
        PALLOC(gx.adj, int, std::max<long long>(nu, 1));
        PTRY(launch_csr_from_sorted(uniq, nu, n, gx.adj_off, gx.adj, s));
        gx.n_adj = nu;
        PTRY(cudaStreamSynchronize(s));
    }
#undef PALLOC
#undef PTRY
    *out = h;
    return BM_OK;
}

void bm_gidx_free(bm_gidx* idx) { free_gidx(idx); }

bm_status bm_gidx_info(const bm_gidx* idx, int64_t* n, int32_t* d, int64_t* n_adj, const int64_t** adj_off,
                       const int32_t** adj) {
    if (!idx) return fail(BM_ERR_ARG, "index is NULL");
    const GraphIndex& gx = idx->gx;
    if (n) *n = gx.n;
    if (d) *d = gx.d;
    if (n_adj) *n_adj = gx.n_adj;
    if (adj_off) *adj_off = (const int64_t*)gx.adj_off;
    if (adj) *adj = gx.adj;
    return BM_OK;
}

static bm_status validate_search(int32_t ef, int64_t* max_visits) {
    if (ef < 1 || ef > 256) return fail(BM_ERR_ARG, "ef must be in [1, 256]");
    if (*max_visits == 0) *max_visits = 4096;
    if (*max_visits < 1 || *max_visits > (1LL << 24)) return fail(BM_ERR_ARG, "max_visits must be in [1, 2^24]");
    return BM_OK;
}

bm_status bm_gidx_range_query(const bm_gidx* idx, const float* Q, int64_t m, float eps, int32_t ef,
                              int64_t max_visits, const bm_options* opt_in, bm_csr* out, bm_stats* stats) {
    if (!out) return fail(BM_ERR_ARG, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (!idx) return fail(BM_ERR_ARG, "index is NULL");
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    const GraphIndex& gx = idx->gx;
    bm_status vs = validate_points(Q, m, gx.d, "Q");
    if (vs == BM_OK) vs = validate_eps(eps);
    if (vs == BM_OK) vs = validate_search(ef, &max_visits);
    if (vs != BM_OK) return vs;
    vs = check_device(opt.path);
    if (vs != BM_OK) return vs;
    return range_core(gx.X, gx.n, gx.d, Q, m, eps, opt, nullptr, 0, nullptr, out, stats, nullptr, 0.0, 0, &gx, ef,
                      max_visits);
}

bm_status bm_build_gidx(const bm_gidx* idx, float eps, int32_t ef, int64_t max_visits, const int32_t* landmarks,
                        int64_t n_landmarks, const bm_options* opt_in, bm_graph* out) {
    if (!out) return fail(BM_ERR_ARG, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    if (!idx) return fail(BM_ERR_ARG, "index is NULL");
    bm_options opt;
    bm_options_init(&opt);
    if (opt_in) opt = *opt_in;
    const GraphIndex& gx = idx->gx;
    bm_status vs = validate_eps(eps);
    if (vs == BM_OK) vs = validate_search(ef, &max_visits);
    if (vs != BM_OK) return vs;
    if (landmarks && (n_landmarks < 0 || n_landmarks > gx.n)) return fail(BM_ERR_ARG, "n_landmarks out of range");
    vs = validate_batch(opt.batch, kMaxBatch);
    if (vs != BM_OK) return vs;
    vs = check_device(opt.path);
    if (vs != BM_OK) return vs;
    return build_graph(gx.X, gx.n, gx.d, eps, opt, nullptr, 0, landmarks, landmarks ? n_landmarks : 0, out, &gx, ef,
                       max_visits);
}
