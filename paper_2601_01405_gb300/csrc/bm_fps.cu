// bm_fps.cu -- farthest point sampling epsilon-net (Sec. 2.2).
//
// Starting from a given landmark, the procedure repeatedly takes the point
// farthest from the landmark set, x* = argmax_x min_{l in L} d(x, l), and adds
// it while that distance is at least eps (open balls: a point at exactly eps is
// not covered, so it must become a landmark; the smallest index wins among
// equal maxima).  The result is unique for the data, eps and the first
// landmark.
//
// Every iteration is one pass over the points: m(x) = min(m(x), D(x, l_new))
// with D the FP64 squared distance in coordinate order (the oracle's value),
// then an argmax.  A pass is a matrix-vector product (one new landmark against
// all points), bound by HBM bandwidth, so it runs on CUDA cores:
//   * FP32 filter: D32 on direct differences bounds the FP64 value from below;
//     when that bound is already >= m(x) nothing changes and no FP64 work is
//     done (m only decreases, so most points leave after the first passes);
//   * argmax per block, then the last block to finish (a ticket counter) reduces
//     the block results, appends the landmark or stops, and sets the loop
//     condition of the CUDA-graph WHILE node that repeats the kernel -- the
//     whole procedure is one graph launch, with no host round trip per landmark.
// The loop is bounded: past n + 2 iterations the kernel stops it with an error.
#include <climits>

#include "bm_host.h"

namespace bm {

namespace {

constexpr int kFpsThreads = 256;

__device__ __forceinline__ float fps_sqdist32(const float* __restrict__ a, const float* __restrict__ b, int d,
                                              int vec4) {
    float s = 0.f;
    if (vec4) {
        const float4* a4 = reinterpret_cast<const float4*>(a);
        const float4* b4 = reinterpret_cast<const float4*>(b);
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

// (value, index) argmax with the smallest index among equal values
__device__ __forceinline__ void arg_better(double& v, int& i, double ov, int oi) {
    if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
    }
}

__global__ void __launch_bounds__(kFpsThreads) fps_step_kernel(
    const float* __restrict__ X, long long n, int d, int vec4, double eps2, double c_lo, double abs_slack,
    double* __restrict__ mind, int* __restrict__ landmarks, FpsState* st, double* part_v, int* part_i,
    unsigned* ticket, cudaGraphConditionalHandle h, int use_graph) {
    __shared__ double s_v[kFpsThreads / 32];
    __shared__ int s_i[kFpsThreads / 32];
    __shared__ bool s_last;
    if (st->done) {
        if (use_graph && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
        return;
    }
    const long long cur = st->last;
    const float* c = X + cur * d;
    double bv = -1.0;
    int bi = INT_MAX;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const float* p = X + x * d;
        double m = mind[x];
        const float s32 = fps_sqdist32(p, c, d, vec4);
        // lower bound of the FP64 value: nothing to do when it cannot go below m
        const bool settled = s32 <= 3.0e38f && ((double)s32 - abs_slack) * c_lo >= m;
        if (!settled) {
            const double D = vec4 ? exact_sqdist4(p, c, d) : exact_sqdist(p, c, d);
            if (D < m) {
                m = D;
                mind[x] = D;
            }
        }
        arg_better(bv, bi, m, (int)x);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) arg_better(bv, bi, __shfl_xor_sync(kFull, bv, o), __shfl_xor_sync(kFull, bi, o));
    if (lane == 0) {
        s_v[warp] = bv;
        s_i[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kFpsThreads / 32; ++w) arg_better(bv, bi, s_v[w], s_i[w]);
        part_v[blockIdx.x] = bv;
        part_i[blockIdx.x] = bi;
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // the last block: every other block's result is visible (fence before its ticket)
    __threadfence();
    bv = -1.0;
    bi = INT_MAX;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const double v = *(volatile double*)&part_v[b];
        const int i = *(volatile int*)&part_i[b];
        arg_better(bv, bi, v, i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) arg_better(bv, bi, __shfl_xor_sync(kFull, bv, o), __shfl_xor_sync(kFull, bi, o));
    if (lane == 0) {
        s_v[warp] = bv;
        s_i[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kFpsThreads / 32; ++w) arg_better(bv, bi, s_v[w], s_i[w]);
        st->iterations += 1;
        unsigned go = 0u;
        if (st->iterations > (unsigned long long)n + 2ull) {
            st->error = 1;
            st->done = 1;
        } else if (bv >= eps2 && st->count < n && bi < n) {
            landmarks[st->count] = bi;
            st->count += 1;
            st->last = bi;
            st->last_dist2 = bv;
            go = 1u;
        } else {
            st->done = 1;
        }
        *ticket = 0u;
        if (use_graph) cudaGraphSetConditional(h, go);
    }
}

__global__ void fps_init_kernel(double* mind, long long n, int* landmarks, FpsState* st, long long first) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) mind[x] = INFINITY;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        landmarks[0] = (int)first;
        st->count = 1;
        st->last = first;
        st->done = 0;
        st->error = 0;
        st->iterations = 0;
        st->last_dist2 = 0.0;
    }
}

__global__ void finite_check_kernel(const float* __restrict__ X, long long count, int* bad) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool b = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        b |= !isfinite(X[i]);
    if (__any_sync(kFull, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

}  // namespace

int fps_grid(long long n) {
    long long g = (n + kFpsThreads - 1) / kFpsThreads;
    const long long cap = (long long)device_sm_count() * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_fps_init(double* mind, long long n, int* landmarks, FpsState* st, long long first, cudaStream_t s) {
    note_launch();
    fps_init_kernel<<<(unsigned)fps_grid(n), kFpsThreads, 0, s>>>(mind, n, landmarks, st, first);
    return cudaGetLastError();
}

cudaError_t launch_fps_step(const float* X, long long n, int d, double eps2, double* mind, int* landmarks, FpsState* st,
                            double* part_v, int* part_i, unsigned* ticket, cudaGraphConditionalHandle h, bool use_graph,
                            cudaStream_t s) {
    const int vec4 = (d % 4 == 0) && ((uintptr_t)X % 16 == 0);
    // D64 >= (D32 - abs) c_lo: the same interval as the band recheck's FP32 filter
    const double u32 = ldexp(1.0, -24), u64 = ldexp(1.0, -53);
    const double g32 = (d + 2) * u32 / (1.0 - (d + 2) * u32), g64 = (d + 2) * u64 / (1.0 - (d + 2) * u64);
    const double c_lo = (1.0 - g64) / (1.0 + g32) * (1.0 - ldexp(1.0, -50));
    const double abs_slack = d * ldexp(1.0, -125);
    note_launch();
    fps_step_kernel<<<(unsigned)fps_grid(n), kFpsThreads, 0, s>>>(X, n, d, vec4, eps2, c_lo, abs_slack, mind,
                                                                  landmarks, st, part_v, part_i, ticket, h,
                                                                  use_graph ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_finite_check(const float* X, long long count, int* bad, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    long long g = (count + 255) / 256;
    if (g > (long long)device_sm_count() * 8) g = (long long)device_sm_count() * 8;
    note_launch();
    finite_check_kernel<<<(unsigned)g, 256, 0, s>>>(X, count, bad);
    return cudaGetLastError();
}

}  // namespace bm
