// bm_dists.cu -- reported distances of a membership or range-query CSR.
//
// For every stored pair (row r, point x) of a CSR whose rows are balls
// R_eps(q_r) (Sec. 5, Def. 5.1; memberships X_i, Sec. 2.3), the distance
// d(q_r, x) is reported as a float: the FP64 squared distance in coordinate
// order (the arithmetic every exact decision of the library is taken on, the
// same as the CPU oracle's), its correctly rounded FP64 square root, rounded
// once more to float.  The relative error against the FP64 distance is thus at
// most 2^-24; the kernel measures it for every entry and keeps the largest, so
// each call reports the error it actually made.
#include "bm_host.h"

namespace bm {

namespace {

__global__ void __launch_bounds__(256) member_dists_kernel(const float* __restrict__ qx, const int* __restrict__ qidx,
                                                           const float* __restrict__ X, int d, int vec4,
                                                           const long long* __restrict__ offsets, long long rows,
                                                           const int* __restrict__ ids, long long nnz,
                                                           float* __restrict__ dists,
                                                           unsigned long long* max_err_bits) {
    double worst = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        // the row holding entry e: the largest r with offsets[r] <= e (empty rows skipped)
        long long lo = 0, hi = rows;
        while (hi - lo > 1) {
            const long long mid = (lo + hi) >> 1;
            if (offsets[mid] <= e) lo = mid;
            else hi = mid;
        }
        const float* q = qidx ? X + (long long)qidx[lo] * d : qx + lo * d;
        const float* x = X + (long long)ids[e] * d;
        const double D = vec4 ? exact_sqdist4(q, x, d) : exact_sqdist(q, x, d);
        const double r = __dsqrt_rn(D);
        const float f = __double2float_rn(r);
        dists[e] = f;
        const double err = r > 0.0 ? fabs((double)f - r) / r : (f == 0.f ? 0.0 : 1.0);
        worst = fmax(worst, err);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(kFull, worst, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0 && worst > 0.0)
        atomicMax(max_err_bits, (unsigned long long)__double_as_longlong(worst));
}

}  // namespace

cudaError_t launch_member_dists(const float* qx, const int* qidx, const float* X, int d, const long long* offsets,
                                long long rows, const int* ids, long long nnz, float* dists,
                                unsigned long long* max_err_bits, cudaStream_t s) {
    if (nnz == 0 || rows == 0) return cudaSuccess;
    const float* qbase = qidx ? X : qx;
    const int vec4 = (d % 4 == 0) && ((uintptr_t)X % 16 == 0) && ((uintptr_t)qbase % 16 == 0);
    long long blocks = (nnz + 255) / 256;
    if (blocks > (long long)device_sm_count() * 16) blocks = (long long)device_sm_count() * 16;
    note_launch();
    member_dists_kernel<<<(unsigned)blocks, 256, 0, s>>>(qx, qidx, X, d, vec4, offsets, rows, ids, nnz, dists,
                                                        max_err_bits);
    return cudaGetLastError();
}

}  // namespace bm
