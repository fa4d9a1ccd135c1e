// bm_tile_fp32.cu -- K(b0): plain FP32 CUDA-core distance tiles (comparison path).
//
// Computes, for every (query row a, point b) of a 128 x 128 tile, the inner
// product a.b by a chain of FP32 fused multiply-adds in coordinate order
// (Sec. 3.2: the inner product dominates the cost of a range query) and then
//     v = a.b - phi_a - phi_b  =  (eps^2 - D)/2   up to rounding.
// Pairs with v > delta are members of the open ball, pairs with v < -delta
// are not, and the rest are listed for the FP64 recheck kernel (the verified
// range set of Sec. 5.3: candidates plus an exact check).  delta bounds the
// FP32 error (see the delta kernel).
#include "bm_host.h"

namespace bm {

namespace {

constexpr int BM = 128, BN = 128, BK = 16, NT = 256;

struct Fp32Args {
    const float* A;
    const float* phiA;
    long long a_rows_max;
    const int* a_rows_dev;
    const float* B;
    const float* phiB;
    long long n;
    int d;
    int check_done;
    double eps2;
    long long a_tiles;
    const DeviceState* st;
    HitSink sink;
};

__global__ void __launch_bounds__(NT, 2) sweep_fp32_kernel(Fp32Args p) {
    if (p.check_done && p.st->done) return;
    const long long a_rows = p.a_rows_dev ? (long long)*p.a_rows_dev : p.a_rows_max;
    const long long tile = blockIdx.x;
    const long long at = tile % p.a_tiles, bt = tile / p.a_tiles;
    const long long a0 = at * BM, b0 = bt * BN;
    if (a0 >= a_rows || b0 >= p.n) return;

    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ __align__(16) float Bs[2][BK][BN + 4];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int d = p.d;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    float ra[8], rb[8];
    auto load_regs = [&](int k0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = tid + i * NT;
            const int r = e >> 4, k = e & 15;
            const long long ar = a0 + r, br = b0 + r;
            const int kk = k0 + k;
            ra[i] = (ar < a_rows && kk < d) ? p.A[ar * d + kk] : 0.f;
            rb[i] = (br < p.n && kk < d) ? p.B[br * d + kk] : 0.f;
        }
    };
    auto store_smem = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = tid + i * NT;
            const int r = e >> 4, k = e & 15;
            As[buf][k][r] = ra[i];
            Bs[buf][k][r] = rb[i];
        }
    };

    const int ktiles = (d + BK - 1) / BK;
    load_regs(0);
    store_smem(0);
    __syncthreads();
    for (int kt = 0; kt < ktiles; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < ktiles) load_regs((kt + 1) * BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            float av[8], bv[8];
            const float4 a_lo = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
            const float4 a_hi = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
            const float4 b_lo = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
            const float4 b_hi = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
            av[0] = a_lo.x; av[1] = a_lo.y; av[2] = a_lo.z; av[3] = a_lo.w;
            av[4] = a_hi.x; av[5] = a_hi.y; av[6] = a_hi.z; av[7] = a_hi.w;
            bv[0] = b_lo.x; bv[1] = b_lo.y; bv[2] = b_lo.z; bv[3] = b_lo.w;
            bv[4] = b_hi.x; bv[5] = b_hi.y; bv[6] = b_hi.z; bv[7] = b_hi.w;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (kt + 1 < ktiles) {
            store_smem(buf ^ 1);
        }
        __syncthreads();
    }

    // ---- epilogue: classify, re-decide the band in FP64, emit hits ----
    const float delta = p.st->delta;
    unsigned cols[8];
    float phib[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const long long c = b0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
        cols[j] = (unsigned)c;
        phib[j] = c < p.n ? p.phiB[c] : 0.f;
    }
    float phia[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const long long r = a0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        phia[i] = r < a_rows ? p.phiA[r] : 0.f;
    }
    // bit (8 i + j) of hit / band describes pair (row i, column j) of this thread
    unsigned long long hit = 0, band = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const long long r = a0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool ok = r < a_rows && (long long)cols[j] < p.n;
            const float v = (acc[i][j] - phia[i]) - phib[j];
            if (ok && v > delta) hit |= 1ull << (8 * i + j);
            else if (ok && v >= -delta) band |= 1ull << (8 * i + j);
        }
    }
#pragma unroll 1
    for (int i = 0; i < 8; ++i) {
        const long long r = a0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        const unsigned long long hm = (hit >> (8 * i)) & 0xffull, bmk = (band >> (8 * i)) & 0xffull;
        if (__any_sync(kFull, hm != 0ull)) emit_hits_row(p.sink, (unsigned)r, cols, hm);
        if (__any_sync(kFull, bmk != 0ull)) {   // band pairs go to the FP64 recheck kernel
            unsigned long long pos = warp_reserve(p.sink.band_n, __popcll(bmk));
            unsigned long long m = bmk;
            while (m) {
                const int j = __ffsll(m) - 1;
                m &= m - 1;
                if (pos < p.sink.band_cap) p.sink.band_keys[pos] = ((unsigned long long)r << 32) | cols[j];
                ++pos;
            }
        }
    }
    if (tid == 0) {
        const long long ra_ = (a_rows - a0) < BM ? (a_rows - a0) : BM;
        const long long rb_ = (p.n - b0) < BN ? (p.n - b0) : BN;
        atomicAdd(p.sink.pair_count, (unsigned long long)(ra_ * rb_));
    }
}

}  // namespace

cudaError_t launch_sweep_fp32(const SweepDesc& s, cudaStream_t stream) {
    if (s.a_rows_max == 0 || s.b->rows == 0) return cudaSuccess;
    Fp32Args p;
    p.A = s.a->x;
    p.phiA = s.a->phi;
    p.a_rows_max = s.a_rows_max;
    p.a_rows_dev = s.a_rows_dev;
    p.B = s.b->x;
    p.phiB = s.b->phi;
    p.n = s.b->rows;
    p.d = s.b->d;
    p.check_done = s.check_done ? 1 : 0;
    p.eps2 = s.eps2;
    p.a_tiles = (s.a_rows_max + BM - 1) / BM;
    p.st = s.st;
    p.sink = s.sink;
    const long long b_tiles = (s.b->rows + BN - 1) / BN;
    const long long tiles = p.a_tiles * b_tiles;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    note_launch();
    sweep_fp32_kernel<<<(unsigned)tiles, NT, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace bm
