// bm_sort.cu -- device-wide exclusive scan and LSD radix sort of 64-bit keys.
//
// Used to order membership keys (landmark << 32 | point) into CSR rows and to
// deduplicate nerve edge keys (i << 32 | j).  Radix sort: 8-bit digits,
// reduce-then-scan: per-tile digit histograms, one exclusive scan over the
// digit-major count table, then a stable scatter in which each tile ranks
// its keys by digit with warp match masks.
#include "bm_host.h"

namespace bm {

int bits_for(long long v) {
    int b = 0;
    while (b < 63 && (1LL << b) <= v) ++b;
    return b;
}

std::vector<int> digit_shifts(int lo_bits, int hi_bits) {
    std::vector<int> s;
    for (int b = 0; b < lo_bits; b += 8) s.push_back(b);
    for (int b = 0; b < hi_bits; b += 8) s.push_back(32 + b);
    return s;
}

namespace {

constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_scan_excl(T v, T* sm, T& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? sm[lane] : T(0);
        T t = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        sm[lane] = t - w;
        if (lane == 31) sm[32] = t;
    }
    __syncthreads();
    T r = sm[warp] + x - v;
    total = sm[32];
    __syncthreads();
    return r;
}

// Phase 1/3 of the scan: each block scans kScanTile elements; with add != nullptr
// it adds the block's carried-in offset and writes the exclusive result.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_tile_kernel(const T* in, T* out, long long n, T* block_sums,
                                                                 const T* add) {
    __shared__ T sm[33];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    T v[kScanItems];
    T local = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : T(0);
        local += v[i];
    }
    T total;
    T excl = block_scan_excl<T>(local, sm, total);
    if (add == nullptr) {
        if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
        return;
    }
    T run = excl + add[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (base <= n - 1 && base + kScanItems >= n) out[n] = run;  // grand total
}

template <typename T>
cudaError_t exclusive_scan(const T* in, T* out, long long n, Arena& ar, cudaStream_t s) {
    // out has n + 1 entries; out[n] = total
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(T), s);
    const long long blocks = (n + kScanTile - 1) / kScanTile;
    T* sums = (T*)ar.get(sizeof(T) * (blocks + 1));
    if (!sums) return cudaErrorMemoryAllocation;
    note_launch();
    scan_tile_kernel<T><<<(unsigned)blocks, kScanThreads, 0, s>>>(in, nullptr, n, sums, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    T* sums_scan = (T*)ar.get(sizeof(T) * (blocks + 1));
    if (!sums_scan) return cudaErrorMemoryAllocation;
    if (blocks == 1) {
        e = cudaMemsetAsync(sums_scan, 0, sizeof(T), s);
    } else {
        e = exclusive_scan<T>(sums, sums_scan, blocks, ar, s);
    }
    if (e != cudaSuccess) return e;
    note_launch();
    scan_tile_kernel<T><<<(unsigned)blocks, kScanThreads, 0, s>>>(in, out, n, nullptr, sums_scan);
    e = cudaGetLastError();
    ar.release(sums_scan);
    ar.release(sums);
    return e;
}

// ---------------------------------------------------------------- radix sort
constexpr int kRadixThreads = 256, kRadixItems = 16, kRadixTile = kRadixThreads * kRadixItems;
constexpr int kWarps = kRadixThreads / 32;

__global__ void __launch_bounds__(kRadixThreads) radix_hist_kernel(const unsigned long long* keys, long long n,
                                                                   int shift, unsigned* counts, long long tiles) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kRadixTile;
    for (int i = threadIdx.x; i < kRadixTile; i += kRadixThreads) {
        const long long k = base + i;
        if (k < n) atomicAdd(&h[(unsigned)(keys[k] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(long long)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kRadixThreads) radix_scatter_kernel(const unsigned long long* keys,
                                                                      unsigned long long* out, long long n,
                                                                      int shift, const unsigned* offsets,
                                                                      long long tiles) {
    __shared__ unsigned running[256];
    __shared__ unsigned wh[kWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    running[tid] = offsets[(long long)tid * tiles + blockIdx.x];
    const long long base = (long long)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixItems; ++r) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) wh[w][tid] = 0;
        __syncthreads();
        const long long idx = base + (long long)r * kRadixThreads + tid;
        const bool valid = idx < n;
        const unsigned long long key = valid ? keys[idx] : 0ull;
        const unsigned digit = valid ? ((unsigned)(key >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(kFull, digit);
        const unsigned rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wh[warp][digit] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned pre = 0;
            for (int w = 0; w < warp; ++w) pre += wh[w][digit];
            out[running[digit] + pre + rank] = key;
        }
        __syncthreads();
        unsigned add = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) add += wh[w][tid];
        running[tid] += add;
        __syncthreads();
    }
}

}  // namespace

cudaError_t exclusive_scan_i64(const long long* in, long long* out, long long n, Arena& ar, cudaStream_t s) {
    return exclusive_scan<long long>(in, out, n, ar, s);
}

// Sorts keys[0..n) by the 8-bit digits at `shifts` (least significant first).
// *result points to whichever of keys/tmp holds the sorted keys.
cudaError_t radix_sort_u64(unsigned long long* keys, unsigned long long* tmp, long long n,
                           const std::vector<int>& shifts, Arena& ar, cudaStream_t s,
                           unsigned long long** result) {
    *result = keys;
    if (n <= 1 || shifts.empty()) return cudaSuccess;
    if (n >= (1LL << 32)) return cudaErrorInvalidValue;
    const long long tiles = (n + kRadixTile - 1) / kRadixTile;
    const long long cn = 256 * tiles;
    unsigned* counts = (unsigned*)ar.get(sizeof(unsigned) * cn);
    unsigned* offs = (unsigned*)ar.get(sizeof(unsigned) * (cn + 1));
    if (!counts || !offs) return cudaErrorMemoryAllocation;
    unsigned long long* src = keys;
    unsigned long long* dst = tmp;
    for (int sh : shifts) {
        note_launch();
        radix_hist_kernel<<<(unsigned)tiles, kRadixThreads, 0, s>>>(src, n, sh, counts, tiles);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = exclusive_scan<unsigned>(counts, offs, cn, ar, s);
        if (e != cudaSuccess) return e;
        note_launch();
        radix_scatter_kernel<<<(unsigned)tiles, kRadixThreads, 0, s>>>(src, dst, n, sh, offs, tiles);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        unsigned long long* t = src;
        src = dst;
        dst = t;
    }
    ar.release(offs);
    ar.release(counts);
    *result = src;
    return cudaSuccess;
}

}  // namespace bm
