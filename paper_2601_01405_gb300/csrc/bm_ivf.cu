// bm_ivf.cu -- inverted-file range queries (K(f)): the paper's non-exhaustive index.
//
// Sec. 5.4 reads an inverted-file index as a candidate generator: the data set is
// divided into cells, a query examines only the points of selected cells, and
// membership is decided with the exact distance, so the oracle is conservative
// (Def. 5.14): no false positives, possibly false negatives (Sec. 5.3).  Sec. 6.1
// uses such an index with nprobe cells searched per query.
//
// Cells come from k-means (Lloyd iterations on a sample of the points); every
// point belongs to its nearest centroid.  A query probes its nprobe nearest
// centroids.  The scan groups (query, cell) pairs by cell so that each cell's
// points are streamed once for all the queries that probe it, evaluates 64 x 64
// FP32 tiles with the same proven error band as the exact path, and lists band
// pairs for the FP64 recheck kernel.  Determinism: centroid sums are FP64 in
// point-index order, ties in every argmin go to the lowest id.
#include <cfloat>

#include "bm_host.h"

namespace bm {

namespace {

constexpr int TB = 64, TK = 16, TT = 256;

unsigned grid1(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

__global__ void row_norms_kernel(const float* __restrict__ x, long long rows, int d, float* __restrict__ out) {
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        float s = 0.f;
        for (int i = lane; i < d; i += 32) s = fmaf(x[r * d + i], x[r * d + i], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (lane == 0) out[r] = s;
    }
}

// rows (optionally gathered through row_ids) x centroids in 64 x 64 tiles; each
// thread keeps the best of its 4 centroids per row and publishes it with an
// atomicMin on the packed (distance bits, centroid id).
__global__ void __launch_bounds__(TT) nearest_centroid_kernel(const float* __restrict__ R, const int* __restrict__ rid,
                                                             long long nrows, const float* __restrict__ rnorm,
                                                             const float* __restrict__ C, const float* __restrict__ cnorm,
                                                             int nlist, int d, long long ctiles,
                                                             unsigned long long* best) {
    const long long r0 = (blockIdx.x / ctiles) * TB, c0 = (blockIdx.x % ctiles) * TB;
    if (r0 >= nrows) return;
    __shared__ float Rs[TK][TB + 4];
    __shared__ float Cs[TK][TB + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < d; k0 += TK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = tid + i * TT, r = e >> 4, k = e & 15;
            const long long rr = r0 + r;
            const long long src = rr < nrows ? (rid ? (long long)rid[rr] : rr) : 0;
            Rs[k][r] = (rr < nrows && k0 + k < d) ? R[src * d + k0 + k] : 0.f;
            Cs[k][r] = (c0 + r < nlist && k0 + k < d) ? C[(c0 + r) * d + k0 + k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; ++k)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(Rs[k][ty * 4 + i], Cs[k][tx * 4 + j], acc[i][j]);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long r = r0 + ty * 4 + i;
        if (r >= nrows) continue;
        const float rn = rnorm[rid ? rid[r] : r];
        unsigned long long b = ~0ull;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long c = c0 + tx * 4 + j;
            if (c >= nlist) continue;
            float D = __fsub_rn(__fadd_rn(rn, cnorm[c]), __fmul_rn(2.f, acc[i][j]));
            D = D > 0.f ? D : 0.f;
            const unsigned long long key = ((unsigned long long)__float_as_uint(D) << 32) | (unsigned)c;
            b = key < b ? key : b;
        }
        if (b != ~0ull) atomicMin(&best[r], b);
    }
}

// New centroid = mean of its members (FP64, in member order); empty cell keeps its centroid.
__global__ void cell_means_kernel(const float* __restrict__ rows, const long long* __restrict__ off,
                                  const int* __restrict__ members, int nlist, int d, float* __restrict__ cent) {
    const int c = blockIdx.x;
    if (c >= nlist) return;
    const long long b = off[c], e = off[c + 1];
    if (e == b) return;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (long long p = b; p < e; ++p) s += (double)rows[(long long)members[p] * d + j];
        cent[(long long)c * d + j] = (float)(s / (double)(e - b));
    }
}

// (cell << 32 | point id) keys from the packed nearest-centroid results.
__global__ void unpack_cells_kernel(const unsigned long long* best, const int* row_ids, long long n, int* cell_of,
                                    unsigned long long* keys) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned c = (unsigned)(best[i] & 0xffffffffull);
        if (cell_of) cell_of[i] = (int)c;
        const unsigned id = row_ids ? (unsigned)row_ids[i] : (unsigned)i;
        if (keys) keys[i] = ((unsigned long long)c << 32) | id;
    }
}

__global__ void gather_rows_kernel(const float* __restrict__ x, const int* __restrict__ ids, long long rows, int d,
                                   float* __restrict__ out) {
    const long long total = rows * d;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const long long r = e / d, j = e - r * d;
        out[e] = x[(long long)ids[r] * d + j];
    }
}

// One block per query row: distances to all centroids with the very arithmetic of
// the cell assignment (row norm by the same lane-strided reduction, dot products
// with FMAs in coordinate order, the same rounded combination), so a point's own
// cell is always among its probes; bitonic sort of the packed (distance bits, id)
// keys in shared memory, the first nprobe ids kept.
__global__ void __launch_bounds__(256) probe_select_kernel(const float* __restrict__ A, long long rows_max,
                                                          const int* rows_dev, const float* __restrict__ C,
                                                          const float* __restrict__ cnorm, int nlist, int d,
                                                          int nprobe, int* probes) {
    extern __shared__ unsigned long long s_keys[];   // P2 keys, then d floats
    __shared__ float s_qn;
    const long long rows = rows_dev ? (long long)*rows_dev : rows_max;
    int P2 = 1;
    while (P2 < nlist) P2 <<= 1;
    float* q = reinterpret_cast<float*>(s_keys + P2);
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        for (int j = threadIdx.x; j < d; j += blockDim.x) q[j] = A[r * d + j];
        __syncthreads();
        if (threadIdx.x < 32) {
            float sq = 0.f;
            for (int i = threadIdx.x; i < d; i += 32) sq = fmaf(q[i], q[i], sq);
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(kFull, sq, o);
            if (threadIdx.x == 0) s_qn = sq;
        }
        __syncthreads();
        const float qn = s_qn;
        for (int c = threadIdx.x; c < P2; c += blockDim.x) {
            unsigned long long key = ~0ull;
            if (c < nlist) {
                float acc = 0.f;
                for (int j = 0; j < d; ++j) acc = fmaf(q[j], C[(long long)c * d + j], acc);
                float D = __fsub_rn(__fadd_rn(qn, cnorm[c]), __fmul_rn(2.f, acc));
                D = D > 0.f ? D : 0.f;
                key = ((unsigned long long)__float_as_uint(D) << 32) | (unsigned)c;
            }
            s_keys[c] = key;
        }
        __syncthreads();
        for (int k = 2; k <= P2; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < P2; i += blockDim.x) {
                    const int l = i ^ j;
                    if (l > i) {
                        const unsigned long long a = s_keys[i], b = s_keys[l];
                        const bool up = (i & k) == 0;
                        if ((a > b) == up) {
                            s_keys[i] = b;
                            s_keys[l] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int t = threadIdx.x; t < nprobe; t += blockDim.x)
            probes[r * nprobe + t] = (int)(unsigned)(s_keys[t] & 0xffffffffull);
        __syncthreads();
    }
}

__global__ void probe_count_kernel(const int* probes, long long rows_max, const int* rows_dev, int nprobe,
                                   long long* cnt) {
    const long long rows = rows_dev ? (long long)*rows_dev : rows_max;
    const long long total = rows * nprobe;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride)
        atomicAdd((unsigned long long*)&cnt[probes[e]], 1ull);
}

__global__ void probe_fill_kernel(const int* probes, long long rows_max, const int* rows_dev, int nprobe,
                                  const long long* cq_off, long long* cursor, int* cq_rows) {
    const long long rows = rows_dev ? (long long)*rows_dev : rows_max;
    const long long total = rows * nprobe;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int c = probes[e];
        const long long slot = (long long)atomicAdd((unsigned long long*)&cursor[c], 1ull);
        cq_rows[cq_off[c] + slot] = (int)(e / nprobe);
    }
}

__global__ void tile_counts_kernel(const long long* cq_off, const long long* cell_off, int nlist, long long* tiles) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nlist) return;
    const long long nq = cq_off[c + 1] - cq_off[c], nx = cell_off[c + 1] - cell_off[c];
    tiles[c] = ((nq + TB - 1) / TB) * ((nx + TB - 1) / TB);
}

// Persistent scan over the (cell, query tile, point tile) work list.
__global__ void __launch_bounds__(TT) ivf_scan_kernel(const float* __restrict__ A, const float* __restrict__ phiA,
                                                     const float* __restrict__ xperm, const float* __restrict__ phiX,
                                                     const int* __restrict__ cell_ids,
                                                     const long long* __restrict__ cell_off,
                                                     const long long* __restrict__ cq_off,
                                                     const int* __restrict__ cq_rows,
                                                     const long long* __restrict__ tile_off, int nlist, int d,
                                                     const DeviceState* st, int check_done, HitSink sink) {
    if (check_done && st->done) return;
    __shared__ float As[TK][TB + 4];
    __shared__ float Bs[TK][TB + 4];
    __shared__ int s_row[TB];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long long total = tile_off[nlist];
    const float delta = st->delta;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        int lo = 0, hi = nlist - 1;   // cell c with tile_off[c] <= t < tile_off[c + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_off[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        const int c = lo;
        const long long nq = cq_off[c + 1] - cq_off[c], nx = cell_off[c + 1] - cell_off[c];
        const long long xtiles = (nx + TB - 1) / TB, local = t - tile_off[c];
        const long long q0 = (local / xtiles) * TB, x0 = (local % xtiles) * TB;
        if (tid < TB) s_row[tid] = q0 + tid < nq ? cq_rows[cq_off[c] + q0 + tid] : -1;
        __syncthreads();
        float acc[4][4] = {};
        for (int k0 = 0; k0 < d; k0 += TK) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int e = tid + i * TT, r = e >> 4, k = e & 15;
                const int ar = s_row[r];
                As[k][r] = (ar >= 0 && k0 + k < d) ? A[(long long)ar * d + k0 + k] : 0.f;
                const long long xp = cell_off[c] + x0 + r;
                Bs[k][r] = (x0 + r < nx && k0 + k < d) ? xperm[xp * d + k0 + k] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < TK; ++k)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(As[k][ty * 4 + i], Bs[k][tx * 4 + j], acc[i][j]);
            __syncthreads();
        }
        unsigned cols[4];
        float phib[4];
        bool colok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long xi = x0 + tx * 4 + j;
            colok[j] = xi < nx;
            const long long xp = cell_off[c] + (colok[j] ? xi : 0);
            cols[j] = (unsigned)cell_ids[xp];
            phib[j] = phiX[xp];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int ar = s_row[ty * 4 + i];
            unsigned long long hit = 0, band = 0;
            if (ar >= 0) {
                const float pa = phiA[ar];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (!colok[j]) continue;
                    const float v = (acc[i][j] - pa) - phib[j];
                    if (v > delta) hit |= 1ull << j;
                    else if (v >= -delta) band |= 1ull << j;
                }
            }
            if (__any_sync(kFull, hit != 0ull)) emit_hits_row(sink, (unsigned)ar, cols, hit);
            if (__any_sync(kFull, band != 0ull)) {
                unsigned long long pos = warp_reserve(sink.band_n, __popcll(band));
                unsigned long long m = band;
                while (m) {
                    const int j = __ffsll(m) - 1;
                    m &= m - 1;
                    if (pos < sink.band_cap) sink.band_keys[pos] = ((unsigned long long)(unsigned)ar << 32) | cols[j];
                    ++pos;
                }
            }
        }
        if (tid == 0) {
            const long long ra = (nq - q0) < TB ? (nq - q0) : TB;
            const long long rb = (nx - x0) < TB ? (nx - x0) : TB;
            atomicAdd(sink.pair_count, (unsigned long long)(ra * rb));
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_row_norms(const float* x, long long rows, int d, float* out, cudaStream_t s) {
    if (rows == 0) return cudaSuccess;
    note_launch();
    row_norms_kernel<<<grid1(rows * 32, 256), 256, 0, s>>>(x, rows, d, out);
    return cudaGetLastError();
}

cudaError_t launch_nearest_centroid(const float* rows, const int* row_ids, long long nrows, const float* rnorm,
                                    const float* cent, const float* cnorm, int nlist, int d,
                                    unsigned long long* best, cudaStream_t s) {
    if (nrows == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(best, 0xff, sizeof(unsigned long long) * nrows, s);
    if (e != cudaSuccess) return e;
    const long long ctiles = (nlist + TB - 1) / TB, rtiles = (nrows + TB - 1) / TB;
    if (rtiles * ctiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    note_launch();
    nearest_centroid_kernel<<<(unsigned)(rtiles * ctiles), TT, 0, s>>>(rows, row_ids, nrows, rnorm, cent, cnorm,
                                                                      nlist, d, ctiles, best);
    return cudaGetLastError();
}

cudaError_t launch_cell_means(const float* rows, const long long* off, const int* members, int nlist, int d,
                              float* cent, cudaStream_t s) {
    note_launch();
    cell_means_kernel<<<nlist, 128, 0, s>>>(rows, off, members, nlist, d, cent);
    return cudaGetLastError();
}

cudaError_t launch_unpack_cells(const unsigned long long* best, const int* row_ids, long long n, int* cell_of,
                                unsigned long long* keys, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    note_launch();
    unpack_cells_kernel<<<grid1(n, 256), 256, 0, s>>>(best, row_ids, n, cell_of, keys);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const float* x, const int* ids, long long rows, int d, float* out, cudaStream_t s) {
    if (rows == 0) return cudaSuccess;
    note_launch();
    gather_rows_kernel<<<grid1(rows * d, 256), 256, 0, s>>>(x, ids, rows, d, out);
    return cudaGetLastError();
}

cudaError_t launch_probe_select(const float* A, long long rows_max, const int* rows_dev, const IvfIndex& ix,
                                int nprobe, int* probes, cudaStream_t s) {
    if (rows_max == 0) return cudaSuccess;
    int P2 = 1;
    while (P2 < ix.nlist) P2 <<= 1;
    const size_t smem = sizeof(unsigned long long) * P2 + sizeof(float) * ix.d;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(probe_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const long long grid = rows_max < 152 * 8 ? rows_max : 152 * 8;
    note_launch();
    probe_select_kernel<<<(unsigned)grid, 256, smem, s>>>(A, rows_max, rows_dev, ix.centroids, ix.cnorm, ix.nlist,
                                                          ix.d, nprobe, probes);
    return cudaGetLastError();
}

cudaError_t launch_group_probes(const int* probes, long long rows_max, const int* rows_dev, int nprobe,
                                const IvfIndex& ix, long long* cnt, long long* cq_off, int* cq_rows,
                                long long* tile_off, Arena& ar, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(long long) * (ix.nlist + 1), s);
    if (e != cudaSuccess) return e;
    note_launch();
    probe_count_kernel<<<grid1(rows_max * nprobe, 256), 256, 0, s>>>(probes, rows_max, rows_dev, nprobe, cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan_i64(cnt, cq_off, ix.nlist, ar, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(long long) * (ix.nlist + 1), s)) != cudaSuccess) return e;
    note_launch();
    probe_fill_kernel<<<grid1(rows_max * nprobe, 256), 256, 0, s>>>(probes, rows_max, rows_dev, nprobe, cq_off, cnt,
                                                                     cq_rows);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    note_launch();
    tile_counts_kernel<<<(ix.nlist + 255) / 256, 256, 0, s>>>(cq_off, ix.cell_off, ix.nlist, cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return exclusive_scan_i64(cnt, tile_off, ix.nlist, ar, s);
}

cudaError_t launch_ivf_scan(const float* A, const float* phiA, const IvfIndex& ix, const float* phi_perm,
                            const long long* cq_off, const int* cq_rows, const long long* tile_off,
                            const DeviceState* st, bool check_done, const HitSink& sink, cudaStream_t s) {
    note_launch();
    ivf_scan_kernel<<<152 * 8, TT, 0, s>>>(A, phiA, ix.xperm, phi_perm, ix.cell_ids, ix.cell_off, cq_off, cq_rows,
                                          tile_off, ix.nlist, ix.d, st, check_done ? 1 : 0, sink);
    return cudaGetLastError();
}

}  // namespace bm

// ---------------------------------------------------------------- tensor-core scan layout
//
// The tensor-core tiles stream a point tile of NT rows against up to 16 query tiles of
// 128 rows.  For the inverted file the points of a cell and the queries that probe it
// must meet in the same tiles, so both sides are laid out by cell with every cell padded
// to whole tiles: points (once per index) to multiples of 256 rows, the (query, probe)
// pairs of a sweep to multiples of 128 rows.  A work item is one point tile of a cell
// against a group of that cell's query tiles; the kernel maps padded A rows to queries
// (a_map) and padded columns back to point ids through the cell order.

namespace bm {

namespace {

__global__ void pad_counts_kernel(const long long* off, int nlist, int unit, long long* counts) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nlist) return;
    const long long sz = off[c + 1] - off[c];
    counts[c] = (sz + unit - 1) / unit * unit;
}

__device__ __forceinline__ int cell_of_row(const long long* off, int nlist, long long r) {
    int lo = 0, hi = nlist - 1;   // largest c with off[c] <= r
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= r) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void pad_rows_kernel(const float* __restrict__ xperm, const long long* __restrict__ cell_off,
                                const long long* __restrict__ pad_off, int nlist, long long npad, int d,
                                float* __restrict__ xpad) {
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < npad; r += warps) {
        const int c = cell_of_row(pad_off, nlist, r);
        const long long j = r - pad_off[c], nx = cell_off[c + 1] - cell_off[c];
        const float* src = j < nx ? xperm + (cell_off[c] + j) * d : nullptr;
        for (int i = lane; i < d; i += 32) xpad[r * d + i] = src ? src[i] : 0.f;
    }
}

// One warp per padded query row: its query (or -1) and its operand rows.
__global__ void gather_query_pad_kernel(const long long* __restrict__ pa_off, const long long* __restrict__ cq_off,
                                        const int* __restrict__ cq_rows, int nlist,
                                        const unsigned* __restrict__ hi, const unsigned* __restrict__ lo,
                                        const unsigned* __restrict__ aug, int words, unsigned* __restrict__ ohi,
                                        unsigned* __restrict__ olo, unsigned* __restrict__ oaug, int* __restrict__ a_map) {
    const long long total = pa_off[nlist];
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < total; r += warps) {
        const int c = cell_of_row(pa_off, nlist, r);
        const long long j = r - pa_off[c], nq = cq_off[c + 1] - cq_off[c];
        const int q = j < nq ? cq_rows[cq_off[c] + j] : -1;
        if (lane == 0) a_map[r] = q;
        for (int i = lane; i < words; i += 32) {
            ohi[r * words + i] = q >= 0 ? hi[(long long)q * words + i] : 0u;
            if (olo) olo[r * words + i] = q >= 0 ? lo[(long long)q * words + i] : 0u;
        }
        if (lane < 8) oaug[r * 8 + lane] = q >= 0 ? aug[(long long)q * 8 + lane] : 0u;
    }
}

__global__ void item_counts_kernel(const long long* cq_off, const long long* cell_off, const long long* pad_off,
                                   int nlist, int NT, long long* counts) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nlist) return;
    const long long nq = cq_off[c + 1] - cq_off[c], nx = cell_off[c + 1] - cell_off[c];
    const long long b_tiles = (pad_off[c + 1] - pad_off[c]) / NT, a_tiles = (nq + 127) / 128;
    counts[c] = (nq > 0 && nx > 0) ? b_tiles * ((a_tiles + 15) / 16) : 0;
}

__global__ void item_fill_kernel(const long long* cq_off, const long long* cell_off, const long long* pad_off,
                                 const long long* pa_off, const long long* item_off, int nlist, int NT, TcItem* items) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nlist) return;
    const long long nq = cq_off[c + 1] - cq_off[c], nx = cell_off[c + 1] - cell_off[c];
    const long long k0 = item_off[c], k1 = item_off[c + 1];
    if (k1 == k0) return;
    const long long b_tiles = (pad_off[c + 1] - pad_off[c]) / NT, a_tiles = (nq + 127) / 128;
    const long long groups = (a_tiles + 15) / 16;
    for (long long k = k0; k < k1; ++k) {
        const long long local = k - k0, u = local / groups, g = local % groups;
        TcItem it;
        it.b_tile = pad_off[c] / NT + u;
        it.a_tile0 = (int)(pa_off[c] / 128 + g * 16);
        it.a_count = (int)((a_tiles - g * 16) < 16 ? (a_tiles - g * 16) : 16);
        it.a_end = pa_off[c] + nq;
        it.col_end = pad_off[c] + nx;
        it.b_col0 = pad_off[c];
        it.src0 = cell_off[c];
        items[k] = it;
    }
}

unsigned grid_rows(long long n, int per_block) {
    long long b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

}  // namespace

cudaError_t launch_cell_pad_offsets(const long long* off, int nlist, int unit, long long* counts, long long* pad_off,
                                    Arena& ar, cudaStream_t s) {
    note_launch();
    pad_counts_kernel<<<(nlist + 255) / 256, 256, 0, s>>>(off, nlist, unit, counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return exclusive_scan_i64(counts, pad_off, nlist, ar, s);
}

cudaError_t launch_pad_rows(const float* xperm, const long long* cell_off, const long long* pad_off, int nlist,
                            long long npad, int d, float* xpad, cudaStream_t s) {
    if (npad == 0) return cudaSuccess;
    note_launch();
    pad_rows_kernel<<<grid_rows(npad, 8), 256, 0, s>>>(xperm, cell_off, pad_off, nlist, npad, d, xpad);
    return cudaGetLastError();
}

cudaError_t launch_ivf_tc_layout(const IvfIndex& ix, int NT, const long long* cq_off, const int* cq_rows,
                                 const Prepared& a, Prepared& apad, int* a_map, long long* pa_off, long long* cnt,
                                 TcItem* items, long long* item_off, Arena& ar, cudaStream_t s) {
    cudaError_t e = launch_cell_pad_offsets(cq_off, ix.nlist, 128, cnt, pa_off, ar, s);
    if (e != cudaSuccess) return e;
    note_launch();
    gather_query_pad_kernel<<<grid_rows(apad.rows, 8), 256, 0, s>>>(
        pa_off, cq_off, cq_rows, ix.nlist, reinterpret_cast<const unsigned*>(a.hi),
        reinterpret_cast<const unsigned*>(a.lo), reinterpret_cast<const unsigned*>(a.aug), a.d_pad / 2,
        reinterpret_cast<unsigned*>(apad.hi), reinterpret_cast<unsigned*>(apad.lo),
        reinterpret_cast<unsigned*>(apad.aug), a_map);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    note_launch();
    item_counts_kernel<<<(ix.nlist + 255) / 256, 256, 0, s>>>(cq_off, ix.cell_off, ix.pad_off, ix.nlist, NT, cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan_i64(cnt, item_off, ix.nlist, ar, s)) != cudaSuccess) return e;
    note_launch();
    item_fill_kernel<<<(ix.nlist + 255) / 256, 256, 0, s>>>(cq_off, ix.cell_off, ix.pad_off, pa_off, item_off, ix.nlist,
                                                            NT, items);
    return cudaGetLastError();
}

}  // namespace bm
