// bm_host.h -- host-side internal interfaces of libballmapper (not part of the C-ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ballmapper.h"
#include "bm_common.cuh"

namespace bm {

// Scratch/output allocator bound to one call: caller callbacks when given,
// else stream-ordered cudaMallocAsync.  Frees whatever it still holds on
// destruction (outputs are detached with take()).
class Arena {
public:
    Arena(const bm_options* opt, cudaStream_t s) : opt_(opt), stream_(s) {}
    ~Arena();
    void* get(size_t bytes);          // nullptr on failure; 256-byte aligned
    void release(void* p);            // free now
    void take(void* p);               // detach an output (caller frees it later)
private:
    const bm_options* opt_;
    cudaStream_t stream_;
    std::vector<void*> ptrs_;
};

void device_free(const bm_options* opt, cudaStream_t s, void* p);

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
};

int tc_pad_dim(int d);  // padded K extent of the tensor-core operands for dimension d

// prep.cu
cudaError_t launch_prep(const float* x, long long rows, int d, double eps2, bool a_side, bool want_tc,
                        Prepared& out, unsigned* max_norm_bits, int* bad_flag, cudaStream_t s);
cudaError_t launch_delta(DeviceState* st, int path, int d, int d_pad, double eps2, bool same_sets,
                         cudaStream_t s);

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
cudaError_t launch_greedy_rollback(const GreedyBuffers& g, cudaStream_t s);

// sort.cu
cudaError_t exclusive_scan_i64(const long long* in, long long* out, long long n, Arena& ar,
                               cudaStream_t s);  // out[0..n], out[n] = total
cudaError_t radix_sort_u64(unsigned long long* keys, unsigned long long* tmp, long long n,
                           const std::vector<int>& shifts, Arena& ar, cudaStream_t s,
                           unsigned long long** result);
int bits_for(long long v);  // bits needed to represent v (>= 0)
std::vector<int> digit_shifts(int lo_bits, int hi_bits);  // 8-bit digit shifts covering [0,lo) and [32,32+hi)

// recheck.cu: FP64 re-decision of the band pairs; confirmed hits are appended
// to keys through *count (book: the greedy's candidate-conflict bookkeeping).
cudaError_t launch_band_recheck(DeviceState* st, const unsigned long long* band, unsigned long long band_cap,
                                const float* ax, const float* bx, int d, double eps2, unsigned long long* keys,
                                unsigned long long* count, unsigned long long cap, const HitSink& book,
                                bool check_done, int overflow_bit, bool stop_on_overflow, cudaStream_t s);

// graph.cu
cudaError_t launch_csr_from_sorted(const unsigned long long* keys, long long nnz, long long rows,
                                   long long* offsets, int* ids, cudaStream_t s);
struct EdgeResult {
    int* edges = nullptr;
    long long n_edges = 0;
    long long pairs = 0;
};
bool build_edges(const unsigned long long* sorted_keys, long long nnz, long long n_points,
                 long long n_landmarks, Arena& ar, cudaStream_t s, EdgeResult& out, Failure& f);

}  // namespace bm
