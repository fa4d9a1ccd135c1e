// bm_recheck.cu -- K(b-rc): FP64 re-decision of the pairs inside the error band.
//
// The distance tiles decide every pair whose approximate value lies outside
// [-delta, delta] (v = (eps^2 - D)/2) and list the rest.  Here each listed
// pair gets the exact test D(q,x) < eps^2 with D summed in FP64 in coordinate
// order -- the same arithmetic as the CPU oracle -- which turns the tiles into
// an exact range oracle (verified range set, Sec. 5.3).  A first FP32 pass on
// the direct differences (relative error ~(d+2) 2^-24 of D, no cancellation)
// settles every pair whose eps^2 lies clearly outside the interval that must
// contain the FP64 value; only the rest pay for FP64, which GB300 runs at a
// small fraction of its FP32 rate.  One thread per pair, four coordinates per
// load when the rows allow it; confirmed members are appended to the hit keys
// (with the greedy's candidate-conflict bookkeeping).
#include <cmath>

#include "bm_host.h"

namespace bm {

namespace {

// FP32 squared distance by direct differences (no norm expansion, so no
// cancellation): t_i = fl(a_i - b_i), D32 = FMA-accumulated sum of t_i^2.  All
// terms are non-negative, so |D32 - D| <= gamma_{d+2} D (u = 2^-24) plus an
// absolute d 2^-125 for squares below the normal range.
__device__ __forceinline__ float sqdist32(const float* __restrict__ a, const float* __restrict__ b, int d, int vec4) {
    float s = 0.f;
    if (vec4) {
        const float4* a4 = reinterpret_cast<const float4*>(a);
        const float4* b4 = reinterpret_cast<const float4*>(b);
#pragma unroll 4
        for (int i = 0; i < d / 4; ++i) {
            const float4 x = a4[i], y = b4[i];
            float t = __fsub_rn(x.x, y.x); s = __fmaf_rn(t, t, s);
            t = __fsub_rn(x.y, y.y); s = __fmaf_rn(t, t, s);
            t = __fsub_rn(x.z, y.z); s = __fmaf_rn(t, t, s);
            t = __fsub_rn(x.w, y.w); s = __fmaf_rn(t, t, s);
        }
    } else {
        for (int i = 0; i < d; ++i) {
            const float t = __fsub_rn(a[i], b[i]);
            s = __fmaf_rn(t, t, s);
        }
    }
    return s;
}

__global__ void __launch_bounds__(256) band_recheck_kernel(
    DeviceState* st, const unsigned long long* __restrict__ band, unsigned long long band_cap,
    const float* __restrict__ ax, const float* __restrict__ bx, int d, double eps2, unsigned long long* keys,
    unsigned long long* count, unsigned long long cap, const int* slot_of, unsigned* conflict, unsigned* row_any,
    int words, int check_done, int overflow_bit, int stop_on_overflow, int vec4, double c_lo, double c_hi,
    double abs_slack, const double* __restrict__ row_eps2) {
    pdl_wait();
    pdl_trigger();
    if (check_done && st->done) return;
    const unsigned long long nb_raw = st->band_n;
    const unsigned long long nb = nb_raw < band_cap ? nb_raw : band_cap;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(&st->band_pairs, nb_raw);
        if (nb_raw > band_cap || *count > cap) {
            atomicOr(&st->error, overflow_bit);
            if (stop_on_overflow) st->done = 1;
        }
    }
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < nb;
         i0 += stride) {
        const unsigned long long i = i0 + lane;
        unsigned long long key = 0;
        bool hit = false;
        if (i < nb) {
            key = band[i];
            const unsigned long long row = key >> 32, col = key & 0xffffffffull;
            const float* a = ax + row * (unsigned long long)d;
            const float* b = bx + col * (unsigned long long)d;
            const double r2 = row_eps2 ? row_eps2[row] : eps2;
            // filter: decided in FP32 when eps^2 lies outside the interval that must hold
            // the FP64 value; otherwise the FP64 evaluation (the oracle's arithmetic) decides
            const float s32 = sqdist32(a, b, d, vec4);
            bool decided = false;
            if (s32 <= 3.0e38f) {
                const double D32 = (double)s32;
                if ((D32 + abs_slack) * c_hi < r2) {
                    hit = true;
                    decided = true;
                } else if ((D32 - abs_slack) * c_lo >= r2) {
                    decided = true;
                }
            }
            if (!decided) {
                const double D = vec4 ? exact_sqdist4(a, b, d) : exact_sqdist(a, b, d);
                hit = D < r2;
            }
        }
        unsigned long long pos = warp_reserve(count, hit ? 1u : 0u);
        if (hit) {
            if (pos < cap) {
                keys[pos] = key;
            } else {
                atomicOr(&st->error, overflow_bit);
                if (stop_on_overflow) st->done = 1;
            }
            if (slot_of) {
                const unsigned row = (unsigned)(key >> 32), col = (unsigned)(key & 0xffffffffull);
                const int s = slot_of[col];
                if (s > (int)row) {
                    atomicOr(&conflict[(size_t)row * words + (s >> 5)], 1u << (s & 31));
                    atomicOr(&row_any[row >> 5], 1u << (row & 31));
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_band_recheck(DeviceState* st, const unsigned long long* band, unsigned long long band_cap,
                                const float* ax, const float* bx, int d, double eps2, unsigned long long* keys,
                                unsigned long long* count, unsigned long long cap, const HitSink& book,
                                bool check_done, int overflow_bit, bool stop_on_overflow, cudaStream_t s,
                                const double* row_eps2) {
    const int vec4 = (d % 4 == 0) && ((uintptr_t)ax % 16 == 0) && ((uintptr_t)bx % 16 == 0);
    // D64 (FP64, the oracle's arithmetic) lies in [(D32 - abs) c_lo, (D32 + abs) c_hi]:
    // D in [(D32 - abs)/(1 + g32), (D32 + abs)/(1 - g32)] and |D64 - D| <= g64 D, with
    // g = gamma_{d+2} = (d+2)u / (1 - (d+2)u); the factors 1 -+ 2^-50 cover the rounding
    // of these constants and of the two FP64 operations that apply them.
    const double u32 = std::ldexp(1.0, -24), u64 = std::ldexp(1.0, -53);
    const double g32 = (d + 2) * u32 / (1.0 - (d + 2) * u32), g64 = (d + 2) * u64 / (1.0 - (d + 2) * u64);
    const double c_lo = (1.0 - g64) / (1.0 + g32) * (1.0 - std::ldexp(1.0, -50));
    const double c_hi = (1.0 + g64) / (1.0 - g32) * (1.0 + std::ldexp(1.0, -50));
    const double abs_slack = d * std::ldexp(1.0, -125);
    note_launch();
    return launch_pdl(band_recheck_kernel, dim3(device_sm_count() * 4), dim3(256), 0, s, st, band, band_cap, ax, bx, d,
                      eps2, keys, count, cap, book.slot_of, book.conflict, book.row_any, book.conflict_words,
                      check_done ? 1 : 0, overflow_bit, stop_on_overflow ? 1 : 0, vec4, c_lo, c_hi, abs_slack,
                      row_eps2);
}

}  // namespace bm
