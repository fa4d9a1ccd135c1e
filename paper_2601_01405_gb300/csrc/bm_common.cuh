// bm_common.cuh -- device-side definitions shared by the kernels of libballmapper.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace bm {

constexpr unsigned kFull = 0xffffffffu;

// Error bits raised by kernels into DeviceState::error.
enum : int {
    kErrStepOverflow = 1,    // a greedy step produced more hits than its buffer holds
    kErrMemberOverflow = 2,  // membership keys exceeded their buffer (recoverable)
    kErrTimeout = 4,         // a bounded wait expired
    kErrHitOverflow = 8,     // range-query hits exceeded their buffer (recoverable)
    kErrLoopLimit = 16,      // a device-side greedy loop ran more iterations than it can need
};

// Device-resident state of one build.  Written only by the library's kernels
// and read back by the host between batches of greedy steps.
struct DeviceState {
    long long scan_pos;              // smallest index not yet examined by the greedy
    int cand_count;                  // candidates of the current step
    int n_landmarks;                 // landmarks so far
    int done;                        // 1 once no uncovered point remains
    int error;                       // kErr* bits
    unsigned long long step_hits;    // hits appended by the current step's sweep
    unsigned long long mem_count;    // membership keys produced so far
    unsigned long long steps;        // greedy steps executed
    unsigned long long band_pairs;   // pairs re-decided in FP64
    unsigned long long tile_pairs;   // pairs evaluated by the tiles
    unsigned long long candidates;   // candidates examined
    unsigned long long hit_count;    // range-query hits
    unsigned int max_norm_bits;      // float bits of max ||x|| over the points
    unsigned int max_norm_q_bits;    // float bits of max ||q|| over the queries
    float delta;                     // band half-width in units of (eps^2 - D)/2
    int pad0;
    unsigned long long max_seg;      // largest per-CTA hit segment seen by a compaction
    unsigned long long band_n;       // band pairs awaiting the FP64 recheck (current sweep)
    long long step_start_pos;        // scan_pos at the start of the current greedy step
    int s_cur;                       // candidates requested by the current step
    int s_next;                      // candidates the next step requests (adapted to the survival rate)
    int gidx_truncated;              // a graph-index search stopped at its visit cap
    int centred;                     // 1 when the tensor-core operands are those of translated rows
};

// One work item of the tensor-core tiles in table mode (the inverted-file scan): the
// point tile b_tile (NT rows of the padded cell-ordered operands) against query tiles
// a_tile0 .. a_tile0 + a_count - 1 (128 rows each of the padded query operands).
// Rows below a_end hold queries; columns below col_end hold points, column c being
// source row src0 + (c - b_col0) of the cell order.
struct TcItem {
    long long b_tile;
    int a_tile0;
    int a_count;
    long long a_end;
    long long col_end;
    long long b_col0;
    long long src0;
};

// Where a distance tile delivers its (row, point) hits.
//   key = (uint64 row << 32) | point
// In greedy mode (slot_of != nullptr) a hit whose point is itself a candidate
// of a later slot also sets conflict[row][slot] and row_any[row].
struct HitSink {
    unsigned long long* keys;
    unsigned long long* count;
    unsigned long long cap;
    const int* slot_of;
    unsigned* conflict;
    unsigned* row_any;
    int conflict_words;
    int pad0;
    unsigned long long* band_count;
    unsigned long long* pair_count;
    // Segmented mode (persistent tile kernels): CTA b appends to
    // keys[b * seg_cap ..) through a shared-memory counter and publishes its
    // count in seg_counts[b]; a compaction pass makes the keys contiguous.
    unsigned long long* seg_counts;
    unsigned long long seg_cap;
    // Pairs inside the error band, (row << 32 | point), re-decided in FP64 by
    // the band recheck kernel: contiguous (band_keys/band_n/band_cap) or
    // segmented like the hits (band_seg_counts, seg_cap per CTA).
    unsigned long long* band_keys;
    unsigned long long* band_n;
    unsigned long long band_cap;
    unsigned long long* band_seg_counts;
};

// FP64 squared distance in coordinate order with separately rounded multiply
// and add: the value every exact decision of the library is taken on.
__device__ __forceinline__ double exact_sqdist(const float* __restrict__ a,
                                               const float* __restrict__ b, int d) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = __dsub_rn((double)a[i], (double)b[i]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Programmatic dependent launch: a kernel launched with launch_pdl may be scheduled while
// its predecessor in the stream still runs; pdl_wait blocks until that predecessor has
// completed and its memory operations are visible (a no-op for an ordinary launch), and
// pdl_trigger lets the next kernel be scheduled once every block of this one has issued
// it.  Step kernels call both first thing, before touching any global memory.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Warp-aggregated reservation of `cnt` slots in a global counter.  Must be
// called by all 32 lanes of the warp.  Returns the lane's first slot.
__device__ __forceinline__ unsigned long long warp_reserve(unsigned long long* counter, unsigned cnt) {
    const unsigned lane = lane_id();
    unsigned x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(kFull, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    const unsigned total = __shfl_sync(kFull, x, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, (unsigned long long)total);
    base = __shfl_sync(kFull, base, 31);
    return base + (x - cnt);
}

// Same as warp_reserve for a 32-bit counter (the per-CTA shared-memory counters).
__device__ __forceinline__ unsigned warp_reserve32(unsigned* counter, unsigned cnt) {
    const unsigned lane = lane_id();
    unsigned x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(kFull, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    const unsigned total = __shfl_sync(kFull, x, 31);
    unsigned base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, total);
    base = __shfl_sync(kFull, base, 31);
    return base + (x - cnt);
}

// Emit the hits of one lane: `mask` bit j set means (row, col0 + cols[j]) is a hit.
// All 32 lanes must call it.  Handles the greedy conflict bookkeeping.
__device__ __forceinline__ void emit_hits_row(const HitSink& sink, unsigned row, const unsigned* cols,
                                              unsigned long long mask) {
    const unsigned cnt = __popcll(mask);
    unsigned long long pos = warp_reserve(sink.count, cnt);
    while (mask) {
        const int j = __ffsll(mask) - 1;
        mask &= mask - 1;
        const unsigned col = cols[j];
        if (pos < sink.cap) sink.keys[pos] = ((unsigned long long)row << 32) | col;
        ++pos;
        if (sink.slot_of) {
            const int s = sink.slot_of[col];
            if (s > (int)row) {
                atomicOr(&sink.conflict[(size_t)row * sink.conflict_words + (s >> 5)], 1u << (s & 31));
                atomicOr(&sink.row_any[row >> 5], 1u << (row & 31));
            }
        }
    }
}

// Same as emit_hits_row for a run of 32 consecutive columns col0 .. col0+31.
__device__ __forceinline__ void emit_hits_run(const HitSink& sink, unsigned row, unsigned col0, unsigned mask) {
    const unsigned cnt = __popc(mask);
    unsigned long long pos = warp_reserve(sink.count, cnt);
    while (mask) {
        const int j = __ffs(mask) - 1;
        mask &= mask - 1;
        const unsigned col = col0 + (unsigned)j;
        if (pos < sink.cap) sink.keys[pos] = ((unsigned long long)row << 32) | col;
        ++pos;
        if (sink.slot_of) {
            const int s = sink.slot_of[col];
            if (s > (int)row) {
                atomicOr(&sink.conflict[(size_t)row * sink.conflict_words + (s >> 5)], 1u << (s & 31));
                atomicOr(&sink.row_any[row >> 5], 1u << (row & 31));
            }
        }
    }
}

// Segmented-mode emission: reserve from the CTA's shared-memory counter
// `ctr` (generic pointer) and write into the CTA's own key segment.
__device__ __forceinline__ void emit_hits_run_seg(const HitSink& sink, unsigned long long* seg_keys,
                                                  unsigned* ctr, unsigned row, unsigned col0,
                                                  unsigned mask) {
    const unsigned cnt = __popc(mask);
    unsigned long long pos = warp_reserve32(ctr, cnt);
    while (mask) {
        const int j = __ffs(mask) - 1;
        mask &= mask - 1;
        const unsigned col = col0 + (unsigned)j;
        if (pos < sink.seg_cap) seg_keys[pos] = ((unsigned long long)row << 32) | col;
        ++pos;
        if (sink.slot_of) {
            const int s = sink.slot_of[col];
            if (s > (int)row) {
                atomicOr(&sink.conflict[(size_t)row * sink.conflict_words + (s >> 5)], 1u << (s & 31));
                atomicOr(&sink.row_any[row >> 5], 1u << (row & 31));
            }
        }
    }
}

// Append (row, col0 + j) for every set bit j of mask to keys, reserving from a
// global 64-bit counter (ctr64) or a shared 32-bit one (ctr32), no bookkeeping.
// All 32 lanes must call it.
__device__ __forceinline__ void emit_plain_run(unsigned long long* keys, unsigned long long* ctr64, unsigned* ctr32,
                                               unsigned long long cap, unsigned row, unsigned col0, unsigned mask) {
    unsigned long long pos = ctr32 ? (unsigned long long)warp_reserve32(ctr32, __popc(mask))
                                   : warp_reserve(ctr64, __popc(mask));
    while (mask) {
        const int j = __ffs(mask) - 1;
        mask &= mask - 1;
        if (pos < cap) keys[pos] = ((unsigned long long)row << 32) | (col0 + (unsigned)j);
        ++pos;
    }
}

// FP64 squared distance in coordinate order, four coordinates per load
// (rows 16-byte aligned, d a multiple of 4); same arithmetic as exact_sqdist.
__device__ __forceinline__ double exact_sqdist4(const float* __restrict__ a, const float* __restrict__ b, int d) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    double s = 0.0;
#pragma unroll 4
    for (int i = 0; i < d / 4; ++i) {
        const float4 x = a4[i], y = b4[i];
        double t;
        t = __dsub_rn((double)x.x, (double)y.x); s = __dadd_rn(s, __dmul_rn(t, t));
        t = __dsub_rn((double)x.y, (double)y.y); s = __dadd_rn(s, __dmul_rn(t, t));
        t = __dsub_rn((double)x.z, (double)y.z); s = __dadd_rn(s, __dmul_rn(t, t));
        t = __dsub_rn((double)x.w, (double)y.w); s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// Block-wide exclusive scan of one int per thread (blockDim.x multiple of 32, <= 1024).
__device__ __forceinline__ int block_exclusive_scan(int v, int* smem32, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem32[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? smem32[lane] : 0;
        int t = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        smem32[lane] = t - w;           // exclusive prefix of warp totals
        if (lane == 31) smem32[32] = t;  // grand total
    }
    __syncthreads();
    const int res = smem32[warp] + x - v;
    total = smem32[32];
    __syncthreads();
    return res;
}

}  // namespace bm
