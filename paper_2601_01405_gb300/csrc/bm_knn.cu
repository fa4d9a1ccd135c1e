// bm_knn.cu -- k-th nearest-neighbour distances and the target-occupancy scale.
//
// Sec. 6.1 chooses eps per dataset as the median, over all points, of the
// distance to the k-th nearest neighbour, the point itself counted first.
// Exactly: for point i let D_(1) <= D_(2) <= ... be the FP64 squared distances
// (coordinate order, the oracle's arithmetic) to all n points, i included
// (D = 0); r_k(i) = sqrt(D_(k)); eps = median_i r_k(i) (mean of the two middle
// values for even n).
//
// The GPU computes D_(k) exactly in three passes:
//   1. bound (this file, CUDA cores): over a strided sample S of the points, an
//      FP32 direct-difference squared distance per pair, raised to a proven
//      upper bound of the FP64 value; the k-th smallest bound over S is >= the
//      k-th smallest FP64 distance over S >= D_(k) over all points.  Its next
//      double up is the row's squared radius rho_i (strictly above D_(k)).
//   2. a range query with the per-row radius rho_i on the tensor-core tiles
//      (exact: band pairs re-decided in FP64): the row's hits are exactly the
//      points with D < rho_i, a set that holds every point with D <= D_(k),
//      hence at least k points and the k smallest distances.
//   3. select (this file): the FP64 squared distances of a row's hits, and
//      their k-th smallest by a radix select on the bit patterns (non-negative
//      doubles order like their bits).
// The median is taken after a radix sort of the n values.
#include "bm_host.h"

namespace bm {

namespace {

constexpr int kBoundWarps = 8;

// Pass 1: one warp per query row.  The warp keeps the k smallest bounds seen so
// far in shared memory (unordered) with their maximum tau: the first k sample
// points fill the slots, later ones replace the maximum when smaller.
__global__ void __launch_bounds__(kBoundWarps * 32) knn_bound_kernel(
    const float* __restrict__ X, long long n, int d, long long stride, long long s, int k, int vec4, double c_hi,
    double abs_slack, double* __restrict__ rho, unsigned long long* rho_max_bits, int* bad) {
    extern __shared__ double s_top[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* top = s_top + (size_t)warp * k;
    const long long warps_total = (long long)gridDim.x * kBoundWarps;
    double row_max = 0.0;
    for (long long q = (long long)blockIdx.x * kBoundWarps + warp; q < n; q += warps_total) {
        const float* xq = X + q * d;
        double tau = 0.0;
        int tau_pos = 0;
        for (long long t0 = 0; t0 < s; t0 += 32) {
            const long long t = t0 + lane;
            double ub = INFINITY;
            if (t < s) {
                const float* xp = X + t * stride * d;
                float acc = 0.f;
                if (vec4) {
                    const float4* a4 = reinterpret_cast<const float4*>(xq);
                    const float4* b4 = reinterpret_cast<const float4*>(xp);
                    for (int i = 0; i < d / 4; ++i) {
                        const float4 a = a4[i], b = b4[i];
                        float u = __fsub_rn(a.x, b.x); acc = __fmaf_rn(u, u, acc);
                        u = __fsub_rn(a.y, b.y); acc = __fmaf_rn(u, u, acc);
                        u = __fsub_rn(a.z, b.z); acc = __fmaf_rn(u, u, acc);
                        u = __fsub_rn(a.w, b.w); acc = __fmaf_rn(u, u, acc);
                    }
                } else {
                    for (int i = 0; i < d; ++i) {
                        const float u = __fsub_rn(xq[i], xp[i]);
                        acc = __fmaf_rn(u, u, acc);
                    }
                }
                ub = (acc <= 3.0e38f) ? ((double)acc + abs_slack) * c_hi : INFINITY;
            }
            if (t0 < k) {
                // filling: slots t0 .. t0 + 31 (those below k)
                if (t < k) top[t] = ub;
                if (t0 + 32 >= k || t0 + 32 >= s) {
                    __syncwarp();
                    // tau = max over the k slots, and where it sits
                    double m = -1.0;
                    int mp = 0;
                    for (int j = lane; j < k; j += 32)
                        if (top[j] > m) { m = top[j]; mp = j; }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const double om = __shfl_xor_sync(kFull, m, o);
                        const int op = __shfl_xor_sync(kFull, mp, o);
                        if (om > m || (om == m && op < mp)) { m = om; mp = op; }
                    }
                    tau = m;
                    tau_pos = mp;
                    // the lanes of this round past the k slots compete below
                    if (t < k) ub = INFINITY;
                } else {
                    continue;
                }
            }
            unsigned want = __ballot_sync(kFull, ub < tau);
            while (want) {
                const int src = __ffs(want) - 1;
                want &= want - 1;
                const double v = __shfl_sync(kFull, ub, src);
                if (!(v < tau)) continue;   // tau fell since the ballot
                if (lane == 0) top[tau_pos] = v;
                __syncwarp();
                double m = -1.0;
                int mp = 0;
                for (int j = lane; j < k; j += 32)
                    if (top[j] > m) { m = top[j]; mp = j; }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double om = __shfl_xor_sync(kFull, m, o);
                    const int op = __shfl_xor_sync(kFull, mp, o);
                    if (om > m || (om == m && op < mp)) { m = om; mp = op; }
                }
                tau = m;
                tau_pos = mp;
            }
        }
        __syncwarp();
        if (lane == 0) {
            if (!(tau < INFINITY)) {
                atomicOr(bad, 1);
                rho[q] = 0.0;
            } else {
                // strictly above the bound, so the range query's strict test keeps D_(k)
                const double r = nextafter(tau, INFINITY);
                rho[q] = r;
                row_max = fmax(row_max, r);
            }
        }
    }
    if (lane == 0 && row_max > 0.0) atomicMax(rho_max_bits, (unsigned long long)__double_as_longlong(row_max));
}

// FP64 squared distance of every CSR entry to its row's query point X[row]
// (coordinate order, the oracle's arithmetic).
__global__ void __launch_bounds__(256) csr_sqdist_kernel(const float* __restrict__ X, int d, int vec4,
                                                         const long long* __restrict__ offsets, long long rows,
                                                         const int* __restrict__ ids, long long nnz,
                                                         double* __restrict__ D) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        long long lo = 0, hi = rows;
        while (hi - lo > 1) {
            const long long mid = (lo + hi) >> 1;
            if (offsets[mid] <= e) lo = mid;
            else hi = mid;
        }
        const float* q = X + lo * d;
        const float* x = X + (long long)ids[e] * d;
        D[e] = vec4 ? exact_sqdist4(q, x, d) : exact_sqdist(q, x, d);
    }
}

// Pass 3: one block per row (grid-stride), the k-th smallest of the row's FP64
// values by an 8-bit radix select on their bit patterns (eight passes, high
// digit first).  kdist[r] = sqrt of it.  A row with fewer than k values sets *bad.
__global__ void __launch_bounds__(256) kth_select_kernel(const double* __restrict__ D, const int* __restrict__ ids,
                                                         const long long* __restrict__ offsets, long long rows, int k,
                                                         int exclude_self, double* __restrict__ kdist,
                                                         double* __restrict__ kD, int* bad) {
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ int s_rank;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const long long e0 = offsets[r], e1 = offsets[r + 1];
        if (e1 - e0 < k + exclude_self) {
            if (threadIdx.x == 0) {
                atomicOr(bad, 2);
                if (kdist) kdist[r] = -1.0;
                if (kD) kD[r] = -1.0;
            }
            continue;
        }
        if (threadIdx.x == 0) {
            s_prefix = 0ull;
            s_rank = k - 1;
        }
        unsigned long long mask = 0ull;
        for (int shift = 56; shift >= 0; shift -= 8) {
            hist[threadIdx.x] = 0u;
            __syncthreads();
            const unsigned long long prefix = s_prefix;
            for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
                if (exclude_self && ids[e] == (int)r) continue;
                const unsigned long long key = (unsigned long long)__double_as_longlong(D[e]);
                if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
            }
            __syncthreads();
            if (warp == 0) {
                // the bin holding rank s_rank: 8 bins per lane, then a warp scan of lane sums
                unsigned c[8], sum = 0u;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    c[b] = hist[lane * 8 + b];
                    sum += c[b];
                }
                unsigned incl = sum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                const int rank = s_rank;
                const unsigned excl = incl - sum;
                const bool mine = excl <= (unsigned)rank && (unsigned)rank < incl;
                if (mine) {
                    unsigned acc = excl;
                    int bin = lane * 8;
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        if ((unsigned)rank < acc + c[b]) { bin = lane * 8 + b; break; }
                        acc += c[b];
                    }
                    s_rank = rank - (int)acc;
                    s_prefix = prefix | ((unsigned long long)bin << shift);
                }
            }
            mask |= 255ull << shift;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double v = __longlong_as_double((long long)s_prefix);
            if (kdist) kdist[r] = __dsqrt_rn(v);
            if (kD) kD[r] = v;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_knn_bound(const float* X, long long n, int d, long long stride, long long s, int k, double* rho,
                             unsigned long long* rho_max_bits, int* bad, cudaStream_t st) {
    const int vec4 = (d % 4 == 0) && ((uintptr_t)X % 16 == 0);
    // an upper bound of the FP64 value from the FP32 one: D32 relative error <= gamma_{d+2}
    // (u = 2^-24, direct differences), FP64 value within gamma_{d+2} (u = 2^-53) of the
    // exact one, 2^-50 for the rounding of the constant and of its application
    const double u32 = ldexp(1.0, -24), u64 = ldexp(1.0, -53);
    const double g32 = (d + 2) * u32 / (1.0 - (d + 2) * u32), g64 = (d + 2) * u64 / (1.0 - (d + 2) * u64);
    const double c_hi = (1.0 + g64) / (1.0 - g32) * (1.0 + ldexp(1.0, -50));
    const double abs_slack = d * ldexp(1.0, -125);
    const size_t smem = (size_t)kBoundWarps * k * sizeof(double);
    static size_t attr = 0;
    if (smem > 48 * 1024 && attr < smem) {
        cudaError_t e = cudaFuncSetAttribute(knn_bound_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    long long blocks = (n + kBoundWarps - 1) / kBoundWarps;
    const long long cap = (long long)device_sm_count() * 8;
    if (blocks > cap) blocks = cap;
    note_launch();
    knn_bound_kernel<<<(unsigned)blocks, kBoundWarps * 32, smem, st>>>(X, n, d, stride, s, k, vec4, c_hi, abs_slack,
                                                                      rho, rho_max_bits, bad);
    return cudaGetLastError();
}

cudaError_t launch_knn_select(const float* X, int d, const long long* offsets, long long rows, const int* ids,
                              long long nnz, double* D, int k, double* kdist, int* bad, cudaStream_t st,
                              bool exclude_self, double* kD) {
    if (rows == 0) return cudaSuccess;
    const int vec4 = (d % 4 == 0) && ((uintptr_t)X % 16 == 0);
    long long blocks = (nnz + 255) / 256;
    const long long cap = (long long)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    note_launch();
    csr_sqdist_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, d, vec4, offsets, rows, ids, nnz, D);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long long sb = rows < (long long)device_sm_count() * 8 ? rows : (long long)device_sm_count() * 8;
    note_launch();
    kth_select_kernel<<<(unsigned)sb, 256, 0, st>>>(D, ids, offsets, rows, k, exclude_self ? 1 : 0, kdist, kD, bad);
    return cudaGetLastError();
}

}  // namespace bm
