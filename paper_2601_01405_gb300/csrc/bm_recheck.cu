// bm_recheck.cu -- K(b-rc): FP64 re-decision of the pairs inside the error band.
//
// The distance tiles decide every pair whose approximate value lies outside
// [-delta, delta] (v = (eps^2 - D)/2) and list the rest.  Here each listed
// pair gets the exact test D(q,x) < eps^2 with D summed in FP64 in coordinate
// order -- the same arithmetic as the CPU oracle -- which turns the tiles into
// an exact range oracle (verified range set, Sec. 5.3).  One thread per pair,
// four coordinates per load when the rows allow it; confirmed members are
// appended to the hit keys (with the greedy's candidate-conflict bookkeeping).
#include "bm_host.h"

namespace bm {

namespace {

__global__ void __launch_bounds__(256) band_recheck_kernel(
    DeviceState* st, const unsigned long long* __restrict__ band, unsigned long long band_cap,
    const float* __restrict__ ax, const float* __restrict__ bx, int d, double eps2, unsigned long long* keys,
    unsigned long long* count, unsigned long long cap, const int* slot_of, unsigned* conflict, unsigned* row_any,
    int words, int check_done, int overflow_bit, int stop_on_overflow, int vec4) {
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
            const double D = vec4 ? exact_sqdist4(a, b, d) : exact_sqdist(a, b, d);
            hit = D < eps2;
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
                                bool check_done, int overflow_bit, bool stop_on_overflow, cudaStream_t s) {
    const int vec4 = (d % 4 == 0) && ((uintptr_t)ax % 16 == 0) && ((uintptr_t)bx % 16 == 0);
    note_launch();
    band_recheck_kernel<<<device_sm_count() * 4, 256, 0, s>>>(st, band, band_cap, ax, bx, d, eps2, keys, count, cap,
                                                             book.slot_of, book.conflict, book.row_any,
                                                             book.conflict_words, check_done ? 1 : 0, overflow_bit,
                                                             stop_on_overflow ? 1 : 0, vec4);
    return cudaGetLastError();
}

}  // namespace bm
