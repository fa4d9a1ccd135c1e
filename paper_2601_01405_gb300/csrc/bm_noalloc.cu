// bm_noalloc.cu -- bm_range_count_noalloc: an entry point that allocates nothing.
//
// Some callers cannot allocate device memory at the time they need an answer:
// real-time services that forbid allocation after start-up, callers that live
// inside another allocator's callback, and callers held to a fixed memory
// budget.  For them this file offers a range COUNT, |R_eps(q)| for every query
// row q, that works entirely in a fixed scratch area compiled into the
// library, plus the output array the caller passes.
//
// The scratch is one file-scope __device__ array of kScratchBytes (32 MiB).
// Every GPU that loads this module keeps it until the process exits.  All
// calls share it: a call leaves its contents behind and the next call clears
// what must start at zero, and calls whose GPU work overlaps (two streams,
// two host threads) race on it.  The host reaches the array only through the
// device address returned by cudaGetSymbolAddress.  That address is looked up
// by the first call made in a CUDA context on a device (so that call should
// happen before any stream capture begins) and kept per context: a context
// created after a cudaDeviceReset gets its own lookup.
//
// Arithmetic: the same exact decision as the other entry points -- FP32 tiles
// with the proven error band, band pairs re-decided by the FP64 squared
// distance in coordinate order.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "bm_host.h"

namespace bm {

namespace {

constexpr size_t kScratchBytes = 32ull << 20;
constexpr long long kMaxRows = 4ll << 20;                 // n + m
constexpr size_t kStateBytes = 256;
constexpr size_t kPhiBytes = (size_t)kMaxRows * sizeof(float);
constexpr unsigned long long kBandCap = (kScratchBytes - kStateBytes - kPhiBytes) / sizeof(unsigned long long);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

static_assert(sizeof(DeviceState) <= kStateBytes, "state block too small");

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// Counting variant of the FP32 distance tile: 64 query rows x 64 points,
// 4 x 4 pairs per thread; members are counted per row, band pairs listed.
__global__ void __launch_bounds__(NT) count_tile_kernel(const float* __restrict__ A, const float* __restrict__ phiA,
                                                        long long m, const float* __restrict__ B,
                                                        const float* __restrict__ phiB, long long n, int d,
                                                        long long a_tiles, DeviceState* st,
                                                        unsigned long long* band, unsigned long long band_cap,
                                                        long long* counts) {
    const long long tile = blockIdx.x;
    const long long a0 = (tile % a_tiles) * BM, b0 = (tile / a_tiles) * BN;
    if (a0 >= m || b0 >= n) return;
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < d; k0 += BK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = tid + i * NT, r = e >> 4, k = e & 15;
            As[k][r] = (a0 + r < m && k0 + k < d) ? A[(a0 + r) * d + k0 + k] : 0.f;
            Bs[k][r] = (b0 + r < n && k0 + k < d) ? B[(b0 + r) * d + k0 + k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(As[k][ty * 4 + i], Bs[k][tx * 4 + j], acc[i][j]);
        __syncthreads();
    }
    const float delta = st->delta;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long r = a0 + ty * 4 + i;
        unsigned hits = 0;
        unsigned bandm = 0;
        if (r < m) {
            const float pa = phiA[r];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long c = b0 + tx * 4 + j;
                if (c >= n) continue;
                const float v = (acc[i][j] - pa) - phiB[c];
                if (v > delta) ++hits;
                else if (v >= -delta) bandm |= 1u << j;
            }
            if (hits) atomicAdd((unsigned long long*)&counts[r], (unsigned long long)hits);
        }
        if (__any_sync(kFull, bandm != 0u)) {
            unsigned long long pos = warp_reserve(&st->band_n, __popc(bandm));
            while (bandm) {
                const int j = __ffs(bandm) - 1;
                bandm &= bandm - 1;
                if (pos < band_cap) band[pos] = ((unsigned long long)r << 32) | (unsigned)(b0 + tx * 4 + j);
                ++pos;
            }
        }
    }
}

__global__ void count_recheck_kernel(DeviceState* st, const unsigned long long* band, unsigned long long band_cap,
                                     const float* __restrict__ A, const float* __restrict__ B, int d, double eps2,
                                     long long* counts) {
    const unsigned long long nb = st->band_n < band_cap ? st->band_n : band_cap;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += stride) {
        const unsigned long long key = band[i];
        const unsigned long long r = key >> 32, c = key & 0xffffffffull;
        if (exact_sqdist(A + r * d, B + c * d, d) < eps2) atomicAdd((unsigned long long*)&counts[r], 1ull);
    }
}

// Largest eps accepted: eps^2 / 4 enters phi, which is stored as a float; above
// about 3.7e19 it overflows and every pair would land in the error band.
constexpr float kMaxEps = 1.0e19f;

// Scratch address per device, valid for the CUDA context it was looked up in.
struct ScratchSlot {
    unsigned long long ctx_id;
    void* addr;
};
std::mutex g_setup_mutex;
ScratchSlot g_slot[64] = {};

}  // namespace

// the library's thread-local error message (defined with the other entry points)
extern thread_local std::string g_last_error;

namespace {
bm_status fail(bm_status s, const char* msg) {
    g_last_error = msg;
    return s;
}
}  // namespace

}  // namespace bm

using namespace bm;

extern "C" bm_status bm_range_count_noalloc(const float* X, int64_t n, int32_t d, const float* Q, int64_t m,
                                            float eps, void* stream, int64_t* counts) {
    if (n < 0 || m < 0 || n > 0x7fffffffLL || m > 0x7fffffffLL) return fail(BM_ERR_ARG, "row counts out of range");
    if (d < 1 || d > 65536) return fail(BM_ERR_ARG, "d out of range [1, 65536]");
    if (!(eps > 0.f) || eps != eps || eps > 3.4e38f) return fail(BM_ERR_ARG, "eps must be finite and > 0");
    if (eps > kMaxEps) return fail(BM_ERR_ARG, "bm_range_count_noalloc: eps above 1e19 is not supported");
    if (n + m > kMaxRows)
        return fail(BM_ERR_CAPACITY, "bm_range_count_noalloc: n + m exceeds its fixed scratch limit of 4194304 rows");
    if ((n > 0 && !X) || (m > 0 && (!Q || !counts))) return fail(BM_ERR_ARG, "NULL input or output");
    cudaStream_t s = (cudaStream_t)stream;
    if (m == 0) return BM_OK;
    if (cudaMemsetAsync(counts, 0, sizeof(int64_t) * (size_t)m, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(BM_ERR_CUDA, "clearing the counts failed");
    }
    if (n == 0) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(BM_ERR_CUDA, "stream synchronisation failed");
        return BM_OK;
    }
    // once per device and context: the device address of the scratch array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return fail(BM_ERR_CUDA, "no current CUDA device");
    }
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        const unsigned long long ctx = current_context_id();
        ScratchSlot& slot = g_slot[dev];
        if (!slot.addr || ctx == 0ull || slot.ctx_id != ctx) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                slot.addr = nullptr;
                return fail(BM_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch failed");
            }
            slot.addr = p;
            slot.ctx_id = ctx;
        }
        base = (unsigned char*)slot.addr;
    }
    DeviceState* st = (DeviceState*)base;
    float* phiX = (float*)(base + kStateBytes);
    float* phiQ = phiX + n;
    unsigned long long* band = (unsigned long long*)(base + kStateBytes + kPhiBytes);
    const double eps2 = (double)eps * (double)eps;
    bool ok = cudaMemsetAsync(st, 0, sizeof(DeviceState), s) == cudaSuccess;
    int* bad = &st->pad0;  // reused as the NaN flag of this call (cleared above)
    Prepared px, pq;
    px.x = X; px.rows = n; px.d = d; px.phi = phiX;
    pq.x = Q; pq.rows = m; pq.d = d; pq.phi = phiQ;
    ok = ok && launch_prep(X, n, d, eps2, false, false, px, &st->max_norm_bits, bad, s) == cudaSuccess;
    ok = ok && launch_prep(Q, m, d, eps2, true, false, pq, &st->max_norm_q_bits, bad, s) == cudaSuccess;
    ok = ok && launch_delta(st, BM_PATH_FP32, d, d, eps2, false, s) == cudaSuccess;
    // n + m <= 2^22 rows keeps a_tiles * b_tiles below 2^30 blocks
    const long long a_tiles = (m + BM - 1) / BM, b_tiles = (n + BN - 1) / BN;
    if (ok) {
        count_tile_kernel<<<(unsigned)(a_tiles * b_tiles), NT, 0, s>>>(Q, phiQ, m, X, phiX, n, d, a_tiles, st, band,
                                                                     kBandCap, (long long*)counts);
        ok = cudaGetLastError() == cudaSuccess;
    }
    if (ok) {
        count_recheck_kernel<<<608, 256, 0, s>>>(st, band, kBandCap, Q, X, d, eps2, (long long*)counts);
        ok = cudaGetLastError() == cudaSuccess;
    }
    DeviceState h;
    ok = ok && cudaMemcpyAsync(&h, st, sizeof(DeviceState), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return fail(BM_ERR_CUDA, "a CUDA call of bm_range_count_noalloc failed");
    }
    if (h.pad0) return fail(BM_ERR_ARG, "input holds NaN or Inf");
    if (h.band_n > kBandCap)
        return fail(BM_ERR_CAPACITY, "bm_range_count_noalloc: more boundary pairs than its fixed scratch holds");
    return BM_OK;
}
