// bm_batch.cu -- the tail of a batched build as one build over all instances.
//
// The instances' point sets are disjoint, so their memberships can be renumbered
// into one Ball Mapper: landmark rows and points get global numbers (row_base[k] +
// ordinal, pt_base[k] + point) and the union is sorted, turned into CSR and into
// nerve edges by the regular passes in one go (no witnessed pair can join two
// instances, and the lexicographic edge order keeps every instance's edges
// contiguous).  These kernels build the global key array and cut the global
// results back into per-instance outputs.
#include "bm_host.h"

namespace bm {

namespace {

// Index of the segment holding position g: largest k with off[k] <= g (off has count + 1
// ascending entries, off[0] = 0).
__device__ __forceinline__ int segment_of(const long long* off, int count, long long g) {
    int lo = 0, hi = count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void gather_batch_keys_kernel(const unsigned long long* const* srcs, const long long* key_off,
                                         const long long* row_base, const long long* pt_base, int count,
                                         unsigned long long* dst) {
    const long long total = key_off[count];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        const int k = segment_of(key_off, count, g);
        const unsigned long long key = srcs[k][g - key_off[k]];
        const unsigned long long row = (unsigned long long)row_base[k] + (key >> 32);
        const unsigned long long pt = (unsigned long long)pt_base[k] + (key & 0xffffffffull);
        dst[g] = (row << 32) | pt;
    }
}

// bounds[k] = first edge whose smaller landmark is >= row_base[k] (k = 0 .. count).
__global__ void edge_bounds_kernel(const int* edges, long long E, const long long* row_base, int count,
                                   long long* bounds) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > count) return;
    const long long key = row_base[k];
    long long lo = 0, hi = E;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if ((long long)edges[2 * mid] < key) lo = mid + 1;
        else hi = mid;
    }
    bounds[k] = lo;
}

// blockIdx.y = instance: its CSR offsets (rebased), ids (local point numbers) and
// edges (local landmark ordinals) from the global results.
__global__ void split_batch_kernel(const BatchSplit* parts, const long long* goff, const int* gids,
                                   const int* gedges) {
    const BatchSplit p = parts[blockIdx.y];
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long base = goff[p.row_base];
    for (long long j = t0; j <= p.rows; j += stride) p.offsets[j] = goff[p.row_base + j] - base;
    for (long long t = t0; t < p.nnz; t += stride) p.ids[t] = (int)((long long)gids[base + t] - p.pt_base);
    for (long long e = t0; e < p.n_edges; e += stride) {
        p.edges[2 * e] = (int)((long long)gedges[2 * (p.edge0 + e)] - p.row_base);
        p.edges[2 * e + 1] = (int)((long long)gedges[2 * (p.edge0 + e) + 1] - p.row_base);
    }
}

unsigned grid_cover(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

}  // namespace

cudaError_t launch_gather_batch_keys(const unsigned long long* const* srcs, const long long* key_off,
                                     const long long* row_base, const long long* pt_base, int count,
                                     long long total, unsigned long long* dst, cudaStream_t s) {
    if (total == 0) return cudaSuccess;
    note_launch();
    gather_batch_keys_kernel<<<grid_cover(total, 256), 256, 0, s>>>(srcs, key_off, row_base, pt_base, count, dst);
    return cudaGetLastError();
}

cudaError_t launch_edge_bounds(const int* edges, long long E, const long long* row_base, int count, long long* bounds,
                               cudaStream_t s) {
    note_launch();
    edge_bounds_kernel<<<(count + 1 + 255) / 256, 256, 0, s>>>(edges, E, row_base, count, bounds);
    return cudaGetLastError();
}

cudaError_t launch_split_batch(const BatchSplit* parts, int count, const long long* goff, const int* gids,
                               const int* gedges, cudaStream_t s) {
    for (int k0 = 0; k0 < count; k0 += 65535) {   // grid y is limited to 65535 instances per launch
        const int c = count - k0 < 65535 ? count - k0 : 65535;
        note_launch();
        split_batch_kernel<<<dim3(64, (unsigned)c), 256, 0, s>>>(parts + k0, goff, gids, gedges);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace bm
