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
