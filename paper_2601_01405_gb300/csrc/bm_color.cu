// bm_color.cu -- coloring of a Ball Mapper graph (Sec. 2.3).
//
// A coloring assigns to landmark l_i a summary of a per-point function f over
// its ball X_i = X intersect B(l_i, eps): the mean (the choice the paper
// prints), the median, the minimum or the maximum (named there as colorings
// that stay between the ball's smallest and largest value).  Input is the
// membership CSR of any build (row i = the ids of X_i) and f (float32, one
// value per point); output is one double per row (NaN for an empty row).
//
//   mean, min, max: one warp per row; the FP64 sum is accumulated per lane and
//     tree-reduced, so it differs from a sequential sum only by rounding
//     (|error| <= (m - 1) 2^-53 sum |f| for m members);
//   median: one block per row, the middle order statistic(s) by an 8-bit radix
//     select on order-preserving 32-bit keys of f (exact; an even count takes
//     the mean of the two middle values, (a + b) / 2 in FP64).
// Ids outside [0, n) are not dereferenced: the row gets NaN and *bad is set.
#include "bm_host.h"

namespace bm {

namespace {

// float -> unsigned key with the same order (negative values flipped)
__device__ __forceinline__ unsigned order_key(float v) {
    const unsigned u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_value(unsigned k) {
    const unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

__global__ void __launch_bounds__(256) color_warp_kernel(const long long* __restrict__ offsets,
                                                         const int* __restrict__ ids, long long rows,
                                                         const float* __restrict__ f, long long n, int stat,
                                                         double* __restrict__ out, int* bad) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        const long long b = offsets[r], e = offsets[r + 1];
        double acc = stat == 0 ? 0.0 : (stat == 2 ? INFINITY : -INFINITY);
        bool oob = false;
        for (long long j = b + lane; j < e; j += 32) {
            const int id = ids[j];
            if (id < 0 || (long long)id >= n) {
                oob = true;
                continue;
            }
            const double v = (double)f[id];
            if (stat == 0) acc += v;
            else if (stat == 2) acc = fmin(acc, v);
            else acc = fmax(acc, v);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(kFull, acc, o);
            if (stat == 0) acc += w;
            else if (stat == 2) acc = fmin(acc, w);
            else acc = fmax(acc, w);
        }
        oob = __any_sync(kFull, oob);
        if (lane == 0) {
            if (oob) atomicOr(bad, 1);
            out[r] = (e == b || oob) ? NAN : (stat == 0 ? acc / (double)(e - b) : acc);
        }
    }
}

// The rank-th smallest key of the row (0-based), block-wide radix select; all threads
// of the block must call it.
__device__ unsigned select_key(const int* __restrict__ ids, const float* __restrict__ f, long long b, long long e,
                               unsigned rank, unsigned* hist, unsigned* s_prefix, unsigned* s_rank) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        *s_prefix = 0u;
        *s_rank = rank;
    }
    unsigned mask = 0u;
    for (int shift = 24; shift >= 0; shift -= 8) {
        hist[threadIdx.x] = 0u;
        __syncthreads();
        const unsigned prefix = *s_prefix;
        for (long long j = b + threadIdx.x; j < e; j += blockDim.x) {
            const unsigned key = order_key(f[ids[j]]);
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (warp == 0) {
            unsigned c[8], sum = 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[q] = hist[lane * 8 + q];
                sum += c[q];
            }
            unsigned incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned rk = *s_rank, excl = incl - sum;
            if (excl <= rk && rk < incl) {
                unsigned acc = excl;
                int bin = lane * 8;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (rk < acc + c[q]) { bin = lane * 8 + q; break; }
                    acc += c[q];
                }
                *s_rank = rk - acc;
                *s_prefix = prefix | ((unsigned)bin << shift);
            }
        }
        mask |= 255u << shift;
        __syncthreads();
    }
    const unsigned k = *s_prefix;
    __syncthreads();
    return k;
}

__global__ void __launch_bounds__(256) color_median_kernel(const long long* __restrict__ offsets,
                                                           const int* __restrict__ ids, long long rows,
                                                           const float* __restrict__ f, long long n,
                                                           double* __restrict__ out, int* bad) {
    __shared__ unsigned hist[256];
    __shared__ unsigned s_prefix, s_rank;
    __shared__ int s_oob;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const long long b = offsets[r], e = offsets[r + 1];
        if (threadIdx.x == 0) s_oob = 0;
        __syncthreads();
        for (long long j = b + threadIdx.x; j < e; j += blockDim.x)
            if (ids[j] < 0 || (long long)ids[j] >= n) s_oob = 1;
        __syncthreads();
        if (e == b || s_oob) {
            if (threadIdx.x == 0) {
                out[r] = NAN;
                if (s_oob) atomicOr(bad, 1);
            }
            __syncthreads();
            continue;
        }
        const long long m = e - b;
        const unsigned hi = select_key(ids, f, b, e, (unsigned)(m / 2), hist, &s_prefix, &s_rank);
        double med = (double)key_value(hi);
        if (m % 2 == 0) {
            const unsigned lo = select_key(ids, f, b, e, (unsigned)(m / 2 - 1), hist, &s_prefix, &s_rank);
            med = ((double)key_value(lo) + med) / 2.0;
        }
        if (threadIdx.x == 0) out[r] = med;
        __syncthreads();
    }
}

__global__ void color_finite_kernel(const float* __restrict__ f, long long n, int* bad) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool b = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) b |= !isfinite(f[i]);
    if (__any_sync(kFull, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 2);
}

}  // namespace

cudaError_t launch_color(const long long* offsets, const int* ids, long long rows, const float* f, long long n, int stat,
                         double* out, int* bad, cudaStream_t s) {
    const long long cap = (long long)device_sm_count() * 8;
    if (n > 0) {
        long long g = (n + 255) / 256;
        note_launch();
        color_finite_kernel<<<(unsigned)(g < cap ? g : cap), 256, 0, s>>>(f, n, bad);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (rows == 0) return cudaSuccess;
    if (stat == 1) {
        note_launch();
        color_median_kernel<<<(unsigned)(rows < cap ? rows : cap), 256, 0, s>>>(offsets, ids, rows, f, n, out, bad);
    } else {
        long long g = (rows + 7) / 8;
        note_launch();
        color_warp_kernel<<<(unsigned)(g < cap ? g : cap), 256, 0, s>>>(offsets, ids, rows, f, n, stat, out, bad);
    }
    return cudaGetLastError();
}

}  // namespace bm
