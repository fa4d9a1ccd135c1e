// bm_prep.cu -- K0: per-point preparation for the distance tiles.
//
// The decision d(q,x) < eps (open ball, Sec. 2.1; exact range set, Sec. 5, Def. 5.1) is
// taken on the algebraic form of Sec. 3.2:
//     D(q,x) = ||q||^2 + ||x||^2 - 2 q.x,
// rewritten as   v = q.x - phi_q - phi_x,   phi = ||.||^2/2 - eps^2/4,
// so that  x in R_eps(q)  <=>  v = (eps^2 - D)/2 > 0.
// The norms are computed once per point here (the paper: computed once per
// query, precomputed and stored per data point) and the inner product is left
// to the tiles.
//
// For the tensor-core path each coordinate is split exactly-or-nearly into
// two bf16 values, x = hi + lo (hi = bf16(x), lo = bf16(x - hi)), and phi is
// carried into the K dimension by a 16-wide augmentation block so that the
// FP32 accumulator already holds v:
//   B side (points):   aug = [1, 1, 1, -p1, -p2, -p3, 1, delta'_x, 0 ...]
//   A side (queries):  aug = [-p1, -p2, -p3, 1, 1, 1, delta'_q, 0, 0 ...]
// with phi ~ p1 + p2 + p3 (three bf16 pieces of the FP64 value) and delta'_q the query
// row's band half-width rounded up to the operand type (set_aug_rows, once the points'
// maximum norm is known; delta'_x, the same for a point, is what a greedy candidate
// carries), so the accumulator holds v + delta'_q and the tiles classify by its sign.  The tensor-core operands may be those of the translated rows x - c
// (launch_centre below); phi and the norms are then the translated rows' too.
#include <cuda_fp16.h>

#include <cmath>

#include "bm_host.h"

namespace bm {

// One warp per group of 32 rows.  The coordinates are read coalesced (row by row, 32
// columns at a time) and staged in shared memory, so that each lane then owns one row's
// FP64 sum of squares: one FP64 multiply-add per coordinate and no cross-lane FP64
// reduction (FP64 throughput is the limit of this kernel on GB300).  The bf16 split, phi
// (FP64, rounded to float) and the augmentation row are written as before.
constexpr int kPrepWarps = 8;

__device__ __forceinline__ int aug_pos(int col, int a_side) {
    return a_side ? col : (col < 3 ? col + 3 : (col < 6 ? col - 3 : col));
}

__global__ void __launch_bounds__(256) prep_kernel(const float* __restrict__ x, long long rows, int d,
                                                   double eps2, const double* __restrict__ row_r2,
                                                   int a_side, int want_tc,
                                                   const float* __restrict__ centre,
                                                   float* __restrict__ phi_out,
                                                   __nv_bfloat16* __restrict__ hi,
                                                   __nv_bfloat16* __restrict__ lo,
                                                   __nv_bfloat16* __restrict__ aug, int d_pad,
                                                   unsigned* max_norm_bits, int* bad_flag) {
    __shared__ float tile[kPrepWarps][32][33];
    __shared__ float s_max[kPrepWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int D = want_tc ? d_pad : d;   // columns summed (zeros past d) and, for the tiles, written
    float my_max = 0.f;
    bool bad = false;
    const long long groups = (rows + 31) / 32;
    for (long long gi = (long long)blockIdx.x * kPrepWarps + warp; gi < groups; gi += (long long)gridDim.x * kPrepWarps) {
        const long long r0 = gi * 32;
        double s = 0.0;
        for (int c0 = 0; c0 < D; c0 += 32) {
            const int i = c0 + lane;
            const float ci = (centre && i < d) ? centre[i] : 0.f;
            for (int rr = 0; rr < 32; ++rr) {
                const long long r = r0 + rr;
                float v = 0.f;
                if (r < rows && i < d) {
                    v = x[r * d + i];
                    if (!isfinite(v)) bad = true;
                    v = __fsub_rn(v, ci);   // x' = fl(x - c); exact when c = 0
                }
                if (want_tc && r < rows && i < D) {
                    const __nv_bfloat16 h = __float2bfloat16_rn(v);
                    hi[r * d_pad + i] = h;
                    lo[r * d_pad + i] = __float2bfloat16_rn(v - __bfloat162float(h));
                }
                tile[warp][rr][lane] = v;
            }
            __syncwarp();
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                const double v = (double)tile[warp][lane][j];
                s += v * v;
            }
            __syncwarp();
        }
        const long long r = r0 + lane;
        if (r < rows) {
            // per-row radius (query side of a k-NN sweep): the whole r^2 on this side
            const double phi = row_r2 ? 0.5 * s - 0.5 * row_r2[r] : 0.5 * s - 0.25 * eps2;
            phi_out[r] = (float)phi;
            if (want_tc) {
                const __nv_bfloat16 p1 = __double2bfloat16(phi);
                const double r1 = phi - (double)__bfloat162float(p1);
                const __nv_bfloat16 p2 = __double2bfloat16(r1);
                const double r2 = r1 - (double)__bfloat162float(p2);
                const __nv_bfloat16 p3 = __double2bfloat16(r2);
                const __nv_bfloat16 one = __float2bfloat16_rn(1.f);
                const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
                const __nv_bfloat16 top = __ushort_as_bfloat16((unsigned short)0x7F7Fu);   // largest finite
                // pos < 3: the -p pieces; 3 <= pos < 6: ones (A side layout; B side swaps halves);
                // column 6: the query's +delta'_row (A side) against 1 (B side); column 7 (B side):
                // the point's own delta'_row for the greedy's candidates.  Until set_aug_rows
                // writes them, the delta' entries hold the largest finite value (every pair
                // in the band: exact, only slow)
                __align__(16) __nv_bfloat16 a[16];
#pragma unroll
                for (int col = 0; col < 16; ++col) {
                    const int pos = aug_pos(col, a_side);
                    a[col] = pos == 0 ? __hneg(p1) : pos == 1 ? __hneg(p2) : pos == 2 ? __hneg(p3)
                           : pos < 6 ? one
                           : pos == 6 ? (a_side ? top : one)
                           : (pos == 7 && !a_side) ? top : zero;
                }
                uint4* dst = reinterpret_cast<uint4*>(aug + r * 16);
                dst[0] = reinterpret_cast<const uint4*>(a)[0];
                dst[1] = reinterpret_cast<const uint4*>(a)[1];
            }
            my_max = fmaxf(my_max, __fsqrt_ru(__double2float_ru(s)));   // an upper bound of the norm
        }
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicExch(bad_flag, 1);
    // block max -> one atomic per block (norms are >= 0, so float bits order as unsigned)
    for (int o = 16; o > 0; o >>= 1) my_max = fmaxf(my_max, __shfl_xor_sync(kFull, my_max, o));
    if (lane == 0) s_max[warp] = my_max;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < kPrepWarps; ++w) m = fmaxf(m, s_max[w]);
        atomicMax(max_norm_bits, __float_as_uint(m));
    }
}

// FP16 operands (BM_PATH_TC_FP16), of the translated rows x = fl(x_in - c) when a centre
// is given: xs = x 2^e (exact in FP64), hi = fp16(xs) rounded to
// nearest, and the augmentation block with three fp16 pieces of
// phi_s = ||xs||^2 / 2 - eps^2 4^e / 4 (FP64), in the same positions as the bf16 block.
// The scale 2^e keeps every operand and phi piece inside the fp16 range.
__global__ void __launch_bounds__(256) prep16_kernel(const float* __restrict__ x, long long rows, int d, int d_pad,
                                                     int scale_exp, double eps2s, int a_side,
                                                     const float* __restrict__ centre,
                                                     __half* __restrict__ hi, __half* __restrict__ aug) {
    __shared__ float tile[kPrepWarps][32][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double scale = ldexp(1.0, scale_exp);
    // x 2^e is exact in float (and so is its fp16 rounding) while 2^e is a normal float
    const bool fscale = scale_exp >= -120 && scale_exp <= 120;
    const float scalef = fscale ? ldexpf(1.f, scale_exp) : 1.f;
    const long long groups = (rows + 31) / 32;
    for (long long gi = (long long)blockIdx.x * kPrepWarps + warp; gi < groups; gi += (long long)gridDim.x * kPrepWarps) {
        const long long r0 = gi * 32;
        double s = 0.0;   // sum of x_i^2; the scaled sum is s 4^e, exactly
        for (int c0 = 0; c0 < d_pad; c0 += 32) {
            const int i = c0 + lane;
            const float ci = (centre && i < d) ? centre[i] : 0.f;
            for (int rr = 0; rr < 32; ++rr) {
                const long long r = r0 + rr;
                const float v = (r < rows && i < d) ? __fsub_rn(x[r * d + i], ci) : 0.f;
                if (r < rows && i < d_pad)
                    hi[r * d_pad + i] = fscale ? __float2half_rn(v * scalef) : __double2half((double)v * scale);
                tile[warp][rr][lane] = v;
            }
            __syncwarp();
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                const double v = (double)tile[warp][lane][j];
                s += v * v;
            }
            __syncwarp();
        }
        const long long r = r0 + lane;
        if (r < rows) {
            const double phi = 0.5 * (s * scale * scale) - 0.25 * eps2s;
            const __half p1 = __double2half(phi);
            const double r1 = phi - (double)__half2float(p1);
            const __half p2 = __double2half(r1);
            const double r2 = r1 - (double)__half2float(p2);
            const __half p3 = __double2half(r2);
            const __half one = __float2half_rn(1.f), zero = __float2half_rn(0.f);
            const __half top = __ushort_as_half((unsigned short)0x7BFFu);   // largest finite
            __align__(16) __half a[16];
#pragma unroll
            for (int col = 0; col < 16; ++col) {
                const int pos = aug_pos(col, a_side);
                a[col] = pos == 0 ? __hneg(p1) : pos == 1 ? __hneg(p2) : pos == 2 ? __hneg(p3)
                       : pos < 6 ? one
                       : pos == 6 ? (a_side ? top : one)
                       : (pos == 7 && !a_side) ? top : zero;
            }
            uint4* dst = reinterpret_cast<uint4*>(aug + r * 16);
            dst[0] = reinterpret_cast<const uint4*>(a)[0];
            dst[1] = reinterpret_cast<const uint4*>(a)[1];
        }
    }
}

cudaError_t launch_prep16(const float* x, long long rows, int d, double eps2, bool a_side, int scale_exp,
                          Prepared& p, cudaStream_t s) {
    if (rows == 0) return cudaSuccess;
    long long blocks = (rows + 255) / 256;   // 8 warps of 32-row groups per block
    if (blocks > 152 * 16) blocks = 152 * 16;
    const double scale = ldexp(1.0, scale_exp);
    p.scale_exp = scale_exp;
    note_launch();
    prep16_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, rows, d, p.d_pad, scale_exp, eps2 * scale * scale,
                                                   a_side ? 1 : 0, p.centre, reinterpret_cast<__half*>(p.hi),
                                                   reinterpret_cast<__half*>(p.aug));
    return cudaGetLastError();
}

// Power-of-two scale for the fp16 operands: max(N, eps) * 2^e < 128, so that every
// scaled coordinate and |phi_s| <= 3 * 128^2 / 4 stay far inside the fp16 range.
int fp16_scale_exp(double max_norm, double eps) {
    const double m = max_norm > eps ? max_norm : eps;
    if (!(m > 0.0) || !std::isfinite(m)) return 0;
    int k = 0;
    std::frexp(m, &k);   // m < 2^k
    return 7 - k;
}

cudaError_t launch_prep(const float* x, long long rows, int d, double eps2, bool a_side, bool want_tc,
                        Prepared& out, unsigned* max_norm_bits, int* bad_flag, cudaStream_t s, const double* row_r2) {
    if (rows == 0) return cudaSuccess;
    long long blocks = (rows + 255) / 256;   // 8 warps of 32-row groups per block
    if (blocks > 152 * 16) blocks = 152 * 16;
    note_launch();
    // out.centre is set for every tensor-core set (split or fp16): the norms and phi measured
    // here must be those of the translated rows the tiles see
    prep_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, rows, d, eps2, row_r2, a_side ? 1 : 0, want_tc ? 1 : 0,
                                                 out.centre, out.phi, out.hi, out.lo, out.aug, out.d_pad,
                                                 max_norm_bits, bad_flag);
    return cudaGetLastError();
}

// ---- Translation of the tensor-core operands.
// D(q, x) does not change when both sides move by the same c, while the proven band
// half-width grows with the operands' norms (N_a N_b and |phi|, see below).  Data whose
// mean lies far from the origin (the Swiss roll, for one) get a band several times wider
// than their spread requires, so the tiles may take x' = fl(x - c) with c the mean of a
// sample of the points.  The FP64 recheck keeps the original coordinates, so no decision
// depends on c; the band bound charges the rounding of x - c.
constexpr long long kCentreSample = 65536;

// Row of sample k (m samples spread evenly over the rows; all rows when m = rows).
__device__ __forceinline__ long long sample_row(long long k, long long m, long long rows) {
    return (long long)(((unsigned long long)k * (unsigned long long)rows) / (unsigned long long)m);
}

// Block b sums its share of the sampled rows per column in FP64 (fixed partition, order
// and reduction tree, so the centre is the same on every run; kCentreBlocks = 1216 blocks
// leave ~54 of 65,536 sampled rows to a block).  Warp w of the block takes rows k0 + w,
// k0 + w + 8, ...; lane l the columns 32 c + l of each row (all chunks of a row loaded
// together, coalesced); the eight warp sums of a column are added in warp order.
constexpr int kCentreWarps = 8;
constexpr int kCentreChunks = 16;   // 32-column chunks: d <= 512 (the tensor-core tiles' limit)

__global__ void __launch_bounds__(kCentreWarps * 32) centre_partial_kernel(const float* __restrict__ x, long long rows,
                                                                          int d, long long m,
                                                                          double* __restrict__ partial) {
    __shared__ double s_sum[kCentreWarps][kCentreChunks * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long k0 = (long long)blockIdx.x * m / gridDim.x, k1 = (long long)(blockIdx.x + 1) * m / gridDim.x;
    double acc[kCentreChunks];
#pragma unroll
    for (int c = 0; c < kCentreChunks; ++c) acc[c] = 0.0;
    const int nch = (d + 31) >> 5;   // chunks that hold columns (FP64 adds only for those)
    for (long long k = k0 + warp; k < k1; k += kCentreWarps) {   // every column of a row in flight at once
        const float* row = x + sample_row(k, m, rows) * d;
        float v[kCentreChunks];
#pragma unroll
        for (int c = 0; c < kCentreChunks; ++c) v[c] = c < nch && c * 32 + lane < d ? row[c * 32 + lane] : 0.f;
#pragma unroll
        for (int c = 0; c < kCentreChunks; ++c)
            if (c < nch) acc[c] += (double)v[c];
    }
#pragma unroll
    for (int c = 0; c < kCentreChunks; ++c) s_sum[warp][c * 32 + lane] = acc[c];
    __syncthreads();
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < kCentreWarps; ++w) t += s_sum[w][j];
        partial[(long long)blockIdx.x * d + j] = t;
    }
}

// c = the sample mean rounded to float (0 where it is not finite), one warp per column
// (the block partials split over the lanes and added in a fixed tree); clears the two
// maxima that centre_gain_kernel fills.
__global__ void __launch_bounds__(256) centre_mean_kernel(const double* __restrict__ partial, int blocks, int d,
                                                          long long m, float* __restrict__ centre,
                                                          unsigned* maxima) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        maxima[0] = 0u;
        maxima[1] = 0u;
    }
    if (j >= d) return;
    double s = 0.0;
    for (int b = lane; b < blocks; b += 32) s += partial[(long long)b * d + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) {
        const float c = (float)(s / (double)m);
        centre[j] = isfinite(c) ? c : 0.f;
    }
}

// Largest squared norm over the sampled rows before (maxima[0]) and after (maxima[1])
// the translation, in FP32: an estimate that only decides whether to translate (the band
// bound uses the norms the prep kernels compute in FP64).  One warp per sampled row, one
// atomic per block.
__global__ void __launch_bounds__(256) centre_gain_kernel(const float* __restrict__ x, long long rows, int d,
                                                          long long m, const float* __restrict__ centre,
                                                          unsigned* maxima) {
    __shared__ float s_max[2][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    float m0 = 0.f, m1 = 0.f;
    for (long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < m; k += warps) {
        const float* row = x + sample_row(k, m, rows) * d;
        float s0 = 0.f, s1 = 0.f;
        for (int j = lane; j < d; j += 32) {
            const float v = row[j], t = v - centre[j];
            s0 = fmaf(v, v, s0);
            s1 = fmaf(t, t, s1);
        }
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(kFull, s0, o);
            s1 += __shfl_xor_sync(kFull, s1, o);
        }
        m0 = fmaxf(m0, s0);
        m1 = fmaxf(m1, s1);
    }
    if (lane == 0) {
        s_max[0][warp] = m0;
        s_max[1][warp] = m1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // squares are >= +0, so float bits order as unsigned
        for (int w = 1; w < 8; ++w) {
            m0 = fmaxf(m0, s_max[0][w]);
            m1 = fmaxf(m1, s_max[1][w]);
        }
        atomicMax(&maxima[0], __float_as_uint(m0));
        atomicMax(&maxima[1], __float_as_uint(m1));
    }
}

// Keep c only where it shrinks the sample's largest squared norm by 5 % or more (always
// when forced); otherwise c = 0.  *centred records the choice.
__global__ void centre_decide_kernel(float* centre, int d, const unsigned* maxima, int force, int* centred) {
    __shared__ int s_keep;
    if (threadIdx.x == 0) {
        const float n0 = __uint_as_float(maxima[0]), n1 = __uint_as_float(maxima[1]);
        s_keep = force || (isfinite(n0) && n1 <= 0.95f * n0);
        *centred = s_keep;
    }
    __syncthreads();
    if (!s_keep)
        for (int j = threadIdx.x; j < d; j += blockDim.x) centre[j] = 0.f;
}

cudaError_t launch_centre(const float* x, long long rows, int d, bool force, double* partial, unsigned* maxima,
                          float* centre, int* centred, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    if (d > kCentreChunks * 32) return cudaErrorInvalidValue;
    const long long m = rows < kCentreSample ? rows : kCentreSample;
    note_launch();
    centre_partial_kernel<<<kCentreBlocks, kCentreWarps * 32, 0, s>>>(x, rows, d, m, partial);
    note_launch();
    centre_mean_kernel<<<(unsigned)((d + 7) / 8), 256, 0, s>>>(partial, kCentreBlocks, d, m, centre, maxima);
    if (!force) {
        const long long blocks = (m + 7) / 8 < 152 * 16 ? (m + 7) / 8 : 152 * 16;   // ~4 sampled rows per warp
        note_launch();
        centre_gain_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, rows, d, m, centre, maxima);
    }
    note_launch();
    centre_decide_kernel<<<1, 256, 0, s>>>(centre, d, maxima, force ? 1 : 0, centred);
    return cudaGetLastError();
}

// Half-width of the error band, in units of v = (eps^2 - D)/2.
//
// N_a, N_b: max norms of the two sides; Phi = max |phi| <= max(N^2/2 - eps^2/4, eps^2/4).
//
// FP32 path: s = q.x by a chain of d FMAs, |s^ - s| <= gamma_d sum|q_i x_i| <= gamma_d N_a N_b
// (u = 2^-24); phi rounded to float (u |phi| each) and two subtractions (u |.| each).
//     delta = 2 (d + 8) 2^-23 (N_a N_b + Phi_a + Phi_b)
//
// Tensor-core path: K = 3 d_pad + 7 accumulated terms (hi.hi, lo.hi, hi.lo, the six
// phi-piece products and 1 x delta'), each exact in FP32; the accumulation order and rounding of
// tcgen05 are not specified, so every one of the K-1 additions (and one alignment
// truncation per term) is charged 2^-23 of the sum of magnitudes:
//     |acc - T| <= 2 K 2^-23 (1.02 N_a N_b + 1.01 (Phi_a + Phi_b)).
// Dropped lo.lo products: <= 2^-16 N_a N_b.  bf16 rounding of lo (inputs that are not
// multiples of 2^-k with |m| < 2^16): <= 2 * 2^-16 N_a N_b.  Three-piece phi: 2^-24 |phi|.
//     delta = 2 [2 K 2^-23 (1.02 N_a N_b + 1.01 (Phi_a + Phi_b)) + 3 2^-16 N_a N_b
//                + 2^-23 (Phi_a + Phi_b)]
// Both bounds carry a safety factor of 2 and a tiny absolute term for underflow.
//
// FP16 path (operands scaled by 2^e; N, Phi and delta in scaled units): with
// hi = fp16(x), |x - hi| <= 2^-11 |x| + 2^-25 (normal / subnormal rounding), so
// |q.x - hq.hx| <= 2^-10 (1 + 2^-10) N_a N_b + 2^-24 sqrt(d_pad) (N_a + N_b) + d_pad 2^-49;
// products hq.hx are exact in FP32; K = d_pad + 7 accumulated terms charged as above;
// three fp16 phi pieces: 2^-33 |phi| + 2^-25 each; FP64 phi: 2^-42 N^2.
//     delta = 2 [E_rep + 2 K 2^-23 (1.002 N_a N_b + 1.001 (Phi_a + Phi_b) + 2^-24 sqrt(d_pad)(N_a + N_b))
//                + 2^-33 (Phi_a + Phi_b) + 2^-22 + 2^-42 (N_a^2 + N_b^2)]
//
// Translated operands (both tensor-core paths): the tiles see x' = fl(x - c) on both
// sides (c = 0: x' = x).  With e = x' - (x - c), |e_i| <= u |x'_i| / (1 - u) (u = 2^-24), so
// the squared distance they approximate, D' = ||a' - b'||^2, differs from D by
// |D' - D| <= 2 ||a' - b'|| (||e_a|| + ||e_b||) (1 + 3u) + (||e_a|| + ||e_b||)^2
//          <= 2.0001 u (N_a + N_b)^2,
// N the norms of the translated rows (the ones the prep kernels measure); v moves by half
// of that, so both bounds add E_ctr = 1.01 2^-24 (N_a + N_b)^2 inside the brackets.
// The bound itself, in the units of the operands (scaled by 2^scale_exp on the fp16
// path); Na, Nb are the unscaled max norms.  Used by the device (delta_kernel) and by
// the host's choice of path.
// The bound for given (scaled) max norms Na, Nb and (scaled) bounds Pa, Pb on |phi| of
// the two sides.
__host__ __device__ double band_halfwidth_core(int path, int d, int d_pad, double Na, double Nb, double Pa,
                                               double Pb) {
    const double u23 = 1.0 / 8388608.0, u16 = 1.0 / 65536.0;
    double delta;
    if (path == BM_PATH_FP32) {
        delta = 2.0 * (d + 8) * u23 * (Na * Nb + Pa + Pb);
    } else if (path == BM_PATH_TC_FP16) {
        const double rd = sqrt((double)d_pad), K = d_pad + 7.0;
        const double u24 = u23 * 0.5;
        const double e_rep = ldexp(1.0 + ldexp(1.0, -10), -10) * Na * Nb + u24 * rd * (Na + Nb) + d_pad * ldexp(1.0, -49);
        const double e_acc = 2.0 * K * u23 * (1.002 * Na * Nb + 1.001 * (Pa + Pb) + u24 * rd * (Na + Nb));
        const double e_aug = ldexp(1.0, -33) * (Pa + Pb) + ldexp(1.0, -22);
        const double e_phi = ldexp(1.0, -42) * (Na * Na + Nb * Nb);
        const double e_ctr = 1.01 * u23 * 0.5 * (Na + Nb) * (Na + Nb);
        delta = 2.0 * (e_rep + e_acc + e_aug + e_phi + e_ctr);
    } else {
        const double K = 3.0 * d_pad + 7.0;
        const double e_ctr = 1.01 * u23 * 0.5 * (Na + Nb) * (Na + Nb);
        delta = 2.0 * (2.0 * K * u23 * (1.02 * Na * Nb + 1.01 * (Pa + Pb)) + 3.0 * u16 * Na * Nb +
                       u23 * (Pa + Pb) + e_ctr);
    }
    return delta + 1e-30;
}

__host__ __device__ double band_halfwidth(int path, int d, int d_pad, double eps2, double Na, double Nb,
                                          int scale_exp) {
    const double sc = ldexp(1.0, scale_exp);
    Na *= sc;
    Nb *= sc;
    const double e2 = eps2 * sc * sc;
    const double Pa = fmax(Na * Na * 0.5 - 0.25 * e2, 0.25 * e2);
    const double Pb = fmax(Nb * Nb * 0.5 - 0.25 * e2, 0.25 * e2);
    return band_halfwidth_core(path, d, d_pad, Na, Nb, Pa, Pb);
}

__global__ void delta_kernel(DeviceState* st, int path, int d, int d_pad, double eps2, int same_sets,
                             int scale_exp) {
    const double Nb = (double)__uint_as_float(st->max_norm_bits);
    const double Na = same_sets ? Nb : (double)__uint_as_float(st->max_norm_q_bits);
    st->delta = __double2float_ru(band_halfwidth(path, d, d_pad, eps2, Na, Nb, scale_exp));
}

// Band half-width of one query row: its own norm and |phi| against the points' maxima
// (the bound above holds pair by pair with N_a the row's norm: every term is a product of
// the two sides' magnitudes, and the points enter through their maxima only).  phi_f is
// the row's phi rounded to float (the FP64 value lies within 2^-24 |phi_f| / (1 - 2^-24));
// its squared norm is 2 phi + r2 (r2 = eps^2 / 2, or a k-NN row's own squared radius), so
// N_a^2 <= 2 phi_f + 2^-22 |phi_f| + r2 and |phi| <= (1 + 2^-22) |phi_f|.  Unscaled inputs;
// the result in the units of the operands (scaled by 2^scale_exp on the fp16 path).  The
// bound is evaluated in FP64 row by row: read off as coefficients of N_a and N_a^2 it
// would lose its low-order terms to cancellation when the norms are large.
__device__ double band_halfwidth_row(int path, int d, int d_pad, double phi_f, double r2, double Nb, double Pb,
                                     int scale_exp) {
    const double sc = ldexp(1.0, scale_exp);
    const double n2 = 2.0 * phi_f + ldexp(fabs(phi_f), -22) + r2;
    const double Na = (double)__fsqrt_ru(__double2float_ru(fmax(n2, 0.0)));   // rounded up (FP32: cheap)
    const double Pa = fabs(phi_f) * (1.0 + ldexp(1.0, -22));
    return band_halfwidth_core(path, d, d_pad, Na * sc, Nb * sc, Pa * sc * sc, Pb * sc * sc);
}

// The delta' entries of an augmentation block once the points' maximum norm is known:
// a query row (A side) gets +delta'_row in column 6; a point (B side) gets 1 in column 6 and
// its own delta'_row in column 7 (what it carries as a greedy candidate; against the
// queries' 0 in column 7 it adds nothing).  delta'_row = the row's half-width rounded up
// to the operand type; the tiles compare the accumulator with 2 delta'_row, so every row
// has the narrowest band its own norm allows.  row_r2 (queries of a k-NN sweep): each
// row's squared radius, the points' side then prepared with eps^2 = 0.
__global__ void set_aug_rows_kernel(const DeviceState* st, const float* __restrict__ phi,
                                    const double* __restrict__ row_r2, long long rows, int path, int d, int d_pad,
                                    double eps2, int scale_exp, int a_side, unsigned short* aug) {
    const double Nb = (double)__uint_as_float(st->max_norm_bits);
    const double Pb = fmax(Nb * Nb * 0.5 - 0.25 * eps2, 0.25 * eps2);
    const bool fp16 = path == BM_PATH_TC_FP16;
    const unsigned short one = fp16 ? __half_as_ushort(__float2half_rn(1.f))
                                    : __bfloat16_as_ushort(__float2bfloat16_rn(1.f));
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
        const double r2 = row_r2 ? row_r2[r] : 0.5 * eps2;
        const double dl = band_halfwidth_row(path, d, d_pad, (double)phi[r], r2, Nb, Pb, scale_exp);
        const float df = __double2float_ru(dl);
        const unsigned short bits = fp16 ? __half_as_ushort(__float2half_ru(df))
                                         : __bfloat16_as_ushort(__float2bfloat16_ru(df));
        if (a_side) {
            aug[r * 16 + 6] = bits;
        } else {
            aug[r * 16 + 6] = one;
            aug[r * 16 + 7] = bits;
        }
    }
}

cudaError_t launch_set_aug_delta(const DeviceState* st, Prepared& p, double eps2, bool a_side, cudaStream_t s,
                                 const double* row_r2) {
    if (p.rows == 0 || p.aug == nullptr || p.prec == kPrecNone) return cudaSuccess;
    long long blocks = (p.rows + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    const int path = p.prec == kPrecFp16 ? (int)BM_PATH_TC_FP16 : (int)BM_PATH_TC_SPLIT3;
    note_launch();
    set_aug_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(st, p.phi, row_r2, p.rows, path, p.d, p.d_pad, eps2,
                                                         p.prec == kPrecFp16 ? p.scale_exp : 0, a_side ? 1 : 0,
                                                         reinterpret_cast<unsigned short*>(p.aug));
    return cudaGetLastError();
}

cudaError_t launch_delta(DeviceState* st, int path, int d, int d_pad, double eps2, bool same_sets,
                         cudaStream_t s, int scale_exp) {
    note_launch();
    delta_kernel<<<1, 1, 0, s>>>(st, path, d, d_pad, eps2, same_sets ? 1 : 0, scale_exp);
    return cudaGetLastError();
}

}  // namespace bm
