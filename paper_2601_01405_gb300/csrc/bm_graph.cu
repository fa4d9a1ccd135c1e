// bm_graph.cu -- K(c) CSR membership compaction and K(d) nerve edges.
//
// K(c): membership keys (row << 32 | point), sorted, become CSR rows: row
// offsets are the positions where the row part changes, ids the low halves.
//
// K(d): the Ball Mapper graph is the 1-skeleton of the nerve (Sec. 2.1,
// Sec. 5.2, Def. 5.6): {i, j} is an edge iff some point lies in both balls.  Every
// point x covered by c_x balls witnesses the c_x (c_x - 1) / 2 pairs of its
// covering landmarks, so the edge set is the deduplicated union of those
// pairs.  Steps: transpose the memberships (point -> ascending covering
// landmarks, by a radix sort of swapped keys); count the witnessed pairs per
// smaller landmark and cut the landmark range into chunks of at most 2^28
// pairs; per chunk emit (i << 32 | j) keys, radix sort, keep the first key of
// every run and append.  Chunks ascend in i, so the edges come out
// lexicographic.
#include "bm_host.h"

namespace bm {

namespace {

__global__ void csr_offsets_kernel(const unsigned long long* keys, long long nnz, long long rows,
                                   long long* offsets, int* ids) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride) {
        const unsigned long long k = keys[i];
        const long long r = (long long)(k >> 32);
        ids[i] = (int)(unsigned)(k & 0xffffffffull);
        const long long rp = i == 0 ? -1 : (long long)(keys[i - 1] >> 32);
        for (long long q = rp + 1; q <= r; ++q) offsets[q] = i;
        if (i == nnz - 1)
            for (long long q = r + 1; q <= rows; ++q) offsets[q] = nnz;
    }
}

__global__ void fill_i64_kernel(long long* p, long long n, long long v) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = v;
}

// (row << 32 | point) -> (point << 32 | row): the transposed membership keys.
__global__ void swap_keys_kernel(const unsigned long long* keys, long long nnz, unsigned long long* out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride) {
        const unsigned long long k = keys[i];
        out[i] = (k << 32) | (k >> 32);
    }
}

// Pairs (i, j), i < j, that point x witnesses with landmark i as the smaller
// ordinal: entry a of x's sorted cover list (length c) starts c - 1 - a pairs.
__global__ void landmark_pair_counts_kernel(const unsigned long long* tkeys, const long long* toff,
                                            const int* tlist, long long nnz, unsigned long long* plc) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const long long x = (long long)(tkeys[e] >> 32);
        const long long c = toff[x + 1] - toff[x], a = e - toff[x];
        if (c - 1 - a > 0) atomicAdd(&plc[tlist[e]], (unsigned long long)(c - 1 - a));
    }
}

// First position in sorted v[lo, hi) with v[pos] >= key.
__device__ __forceinline__ long long lower_bound_i32(const int* v, long long lo, long long hi, int key) {
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (v[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Per point: the number of its pairs whose smaller landmark lies in [i0, i1).
__global__ void chunk_pair_counts_kernel(const long long* toff, const int* tlist, long long n, int i0, int i1,
                                         long long* pc) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const long long b0 = toff[x], c = toff[x + 1] - b0;
        long long cnt = 0;
        if (c >= 2) {
            const long long p0 = lower_bound_i32(tlist, b0, b0 + c, i0) - b0;
            const long long p1 = lower_bound_i32(tlist, b0, b0 + c, i1) - b0;
            const long long k = p1 - p0;   // entries p0 .. p1-1 start (c-1-a) pairs each
            cnt = k * (c - 1) - (p0 + p1 - 1) * k / 2;
        }
        pc[x] = cnt;
    }
}

// One warp per point: keys ((i - i0) << 32 | j) for the pairs counted above.
__global__ void emit_chunk_pairs_kernel(const long long* toff, const int* tlist, long long n, int i0, int i1,
                                        const long long* poff, unsigned long long* pairs) {
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (long long x = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); x < n; x += warps) {
        const long long b0 = toff[x];
        const int c = (int)(toff[x + 1] - b0);
        if (c < 2) continue;
        const int p0 = (int)(lower_bound_i32(tlist, b0, b0 + c, i0) - b0);
        const int p1 = (int)(lower_bound_i32(tlist, b0, b0 + c, i1) - b0);
        long long o = poff[x];
        for (int a = p0; a < p1; ++a) {
            const unsigned hi = (unsigned)(tlist[b0 + a] - i0);
            for (int b = a + 1 + lane; b < c; b += 32)
                pairs[o + (b - a - 1)] = ((unsigned long long)hi << 32) | (unsigned)tlist[b0 + b];
            o += c - 1 - a;
        }
    }
}

__global__ void unique_flags_kernel(const unsigned long long* keys, long long n, long long* flags) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void unique_scatter_kernel(const unsigned long long* keys, long long n, const long long* pos, int i0,
                                      int* edges) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (i == 0 || keys[i] != keys[i - 1]) {
            const long long o = pos[i];
            edges[2 * o] = i0 + (int)(keys[i] >> 32);
            edges[2 * o + 1] = (int)(keys[i] & 0xffffffffull);
        }
    }
}

// Gathers per-CTA segments into one contiguous array.  Blocks [0, nseg) handle
// the hit segments, blocks [nseg, 2 nseg) the band segments of the same sweep.
// Each block first loads all segment counts into shared memory and takes its
// prefix with a block scan.
__global__ void __launch_bounds__(256) compact_segments_kernel(
    const unsigned long long* src, const unsigned long long* band_src, unsigned long long seg_cap,
    const unsigned long long* seg_counts, const unsigned long long* band_seg_counts, int nseg,
    unsigned long long* dst, unsigned long long* band_dst, unsigned long long* count_out,
    unsigned long long* band_count_out, DeviceState* st, int overflow_bit, int check_done, int stop_on_overflow) {
    if (check_done && st->done) return;
    __shared__ unsigned long long s_cnt[256];
    __shared__ unsigned long long s_pre, s_mine;
    const bool band = (int)blockIdx.x >= nseg;
    const int seg = band ? (int)blockIdx.x - nseg : (int)blockIdx.x;
    const unsigned long long* counts = band ? band_seg_counts : seg_counts;
    for (int q = threadIdx.x; q < 256; q += blockDim.x) {
        unsigned long long c = q < nseg ? counts[q] : 0ull;
        if (q < nseg && c > seg_cap) {
            if (q == seg) {
                atomicOr(&st->error, overflow_bit);
                atomicMax(&st->max_seg, c);
                if (stop_on_overflow) st->done = 1;
            }
            c = seg_cap;
        }
        s_cnt[q] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long pre = 0, tot = 0;
        for (int q = 0; q < nseg; ++q) {
            if (q < seg) pre += s_cnt[q];
            tot += s_cnt[q];
        }
        s_pre = pre;
        s_mine = s_cnt[seg];
        if (seg == nseg - 1) *(band ? band_count_out : count_out) = tot;
    }
    __syncthreads();
    const unsigned long long* in = (band ? band_src : src) + (unsigned long long)seg * seg_cap;
    unsigned long long* out = (band ? band_dst : dst) + s_pre;
    for (unsigned long long i = threadIdx.x; i < s_mine; i += blockDim.x) out[i] = in[i];
}

unsigned grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

}  // namespace

cudaError_t launch_csr_from_sorted(const unsigned long long* keys, long long nnz, long long rows, long long* offsets,
                                   int* ids, cudaStream_t s) {
    if (nnz == 0) {
        note_launch();
        fill_i64_kernel<<<grid_for(rows + 1, 256), 256, 0, s>>>(offsets, rows + 1, 0);
        return cudaGetLastError();
    }
    note_launch();
    csr_offsets_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(keys, nnz, rows, offsets, ids);
    return cudaGetLastError();
}

cudaError_t launch_compact_segments(const unsigned long long* src, const unsigned long long* band_src,
                                    unsigned long long seg_cap, const unsigned long long* seg_counts,
                                    const unsigned long long* band_seg_counts, int nseg, unsigned long long* dst,
                                    unsigned long long* band_dst, unsigned long long* count_out,
                                    unsigned long long* band_count_out, DeviceState* st, int overflow_bit,
                                    bool check_done, bool stop_on_overflow, cudaStream_t s) {
    if (nseg <= 0) return cudaSuccess;
    if (nseg > 256) return cudaErrorInvalidValue;
    note_launch();
    compact_segments_kernel<<<2 * nseg, 256, 0, s>>>(src, band_src, seg_cap, seg_counts, band_seg_counts, nseg, dst,
                                                      band_dst, count_out, band_count_out, st, overflow_bit,
                                                      check_done ? 1 : 0, stop_on_overflow ? 1 : 0);
    return cudaGetLastError();
}

#define BM_TRY(expr)                                                   \
    do {                                                               \
        cudaError_t e__ = (expr);                                      \
        if (e__ != cudaSuccess) {                                      \
            f.status = BM_ERR_CUDA;                                    \
            f.msg = std::string(#expr) + ": " + cudaGetErrorString(e__); \
            return false;                                              \
        }                                                              \
    } while (0)

#define BM_ALLOC(ptr, type, count)                                     \
    do {                                                               \
        ptr = (type*)ar.get(sizeof(type) * (size_t)(count));           \
        if (!ptr) {                                                    \
            f.status = BM_ERR_NOMEM;                                   \
            f.msg = "allocation of " #ptr " failed";                   \
            return false;                                              \
        }                                                              \
    } while (0)

bool build_edges(const unsigned long long* keys, long long nnz, long long n, long long L, Arena& ar,
                 cudaStream_t s, EdgeResult& out, Failure& f) {
    out = EdgeResult();
    if (nnz == 0 || L < 2) return true;
    // 1. point -> covering landmarks, ascending (transpose by a radix sort of swapped keys)
    unsigned long long *tk, *tk2;
    BM_ALLOC(tk, unsigned long long, nnz);
    BM_ALLOC(tk2, unsigned long long, nnz);
    note_launch();
    swap_keys_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(keys, nnz, tk);
    BM_TRY(cudaGetLastError());
    unsigned long long* tsorted = nullptr;
    BM_TRY(radix_sort_u64(tk, tk2, nnz, digit_shifts(bits_for(L - 1), bits_for(n - 1)), ar, s, &tsorted));
    long long* toff;
    BM_ALLOC(toff, long long, n + 1);
    int* tlist;
    BM_ALLOC(tlist, int, nnz);
    BM_TRY(launch_csr_from_sorted(tsorted, nnz, n, toff, tlist, s));
    // 2. pairs per smaller landmark -> landmark-range chunks of bounded size
    unsigned long long* plc;
    BM_ALLOC(plc, unsigned long long, L + 1);
    BM_TRY(cudaMemsetAsync(plc, 0, sizeof(unsigned long long) * (L + 1), s));
    note_launch();
    landmark_pair_counts_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(tsorted, toff, tlist, nnz, plc);
    BM_TRY(cudaGetLastError());
    long long* lpre;
    BM_ALLOC(lpre, long long, L + 1);
    BM_TRY(exclusive_scan_i64((const long long*)plc, lpre, L, ar, s));
    std::vector<long long> hpre((size_t)L + 1);
    BM_TRY(cudaMemcpyAsync(hpre.data(), lpre, sizeof(long long) * (L + 1), cudaMemcpyDeviceToHost, s));
    BM_TRY(cudaStreamSynchronize(s));
    ar.release(lpre);
    ar.release(plc);
    ar.release(tk2);
    ar.release(tk);
    const long long P = hpre[(size_t)L];
    out.pairs = P;
    if (P == 0) return true;
    const long long kBudget = 1LL << 28;   // emitted pairs per chunk (32 B of scratch each)
    std::vector<std::pair<int, int>> chunks;
    for (long long i0 = 0; i0 < L;) {
        long long i1 = i0 + 1;
        // largest i1 with pairs(i0, i1) <= budget (at least one landmark)
        long long lo = i0 + 1, hi = L;
        while (lo < hi) {
            const long long mid = (lo + hi + 1) / 2;
            if (hpre[(size_t)mid] - hpre[(size_t)i0] <= kBudget) lo = mid;
            else hi = mid - 1;
        }
        i1 = lo;
        if (hpre[(size_t)i1] - hpre[(size_t)i0] >= (1LL << 32)) {
            f.status = BM_ERR_CAPACITY;
            f.msg = "nerve pass: one landmark witnesses more than 2^32 pairs";
            return false;
        }
        chunks.emplace_back((int)i0, (int)i1);
        i0 = i1;
    }
    // 3. per chunk: count, emit, radix sort, deduplicate, append (chunks ascend in i)
    long long* pc;
    BM_ALLOC(pc, long long, n + 1);
    long long* poff;
    BM_ALLOC(poff, long long, n + 1);
    int* edges = nullptr;
    long long E = 0, cap = 0;
    for (const auto& ch : chunks) {
        const int i0 = ch.first, i1 = ch.second;
        const long long Pc = hpre[(size_t)i1] - hpre[(size_t)i0];
        if (Pc == 0) continue;
        note_launch();
        chunk_pair_counts_kernel<<<grid_for(n, 256), 256, 0, s>>>(toff, tlist, n, i0, i1, pc);
        BM_TRY(cudaGetLastError());
        BM_TRY(exclusive_scan_i64(pc, poff, n, ar, s));
        unsigned long long *pairs, *tmp;
        BM_ALLOC(pairs, unsigned long long, Pc);
        BM_ALLOC(tmp, unsigned long long, Pc);
        note_launch();
        emit_chunk_pairs_kernel<<<grid_for(n * 32, 256), 256, 0, s>>>(toff, tlist, n, i0, i1, poff, pairs);
        BM_TRY(cudaGetLastError());
        unsigned long long* sorted = nullptr;
        BM_TRY(radix_sort_u64(pairs, tmp, Pc, digit_shifts(bits_for(L - 1), bits_for(i1 - i0 - 1)), ar, s, &sorted));
        long long* flags;
        BM_ALLOC(flags, long long, Pc);
        long long* pos;
        BM_ALLOC(pos, long long, Pc + 1);
        note_launch();
        unique_flags_kernel<<<grid_for(Pc, 256), 256, 0, s>>>(sorted, Pc, flags);
        BM_TRY(cudaGetLastError());
        BM_TRY(exclusive_scan_i64(flags, pos, Pc, ar, s));
        long long Ec = 0;
        BM_TRY(cudaMemcpyAsync(&Ec, pos + Pc, sizeof(long long), cudaMemcpyDeviceToHost, s));
        BM_TRY(cudaStreamSynchronize(s));
        if (E + Ec > 0x7fffffffLL) {
            f.status = BM_ERR_CAPACITY;
            f.msg = "more than 2^31-1 edges";
            return false;
        }
        if (E + Ec > cap) {   // grow the output (doubling), keeping the edges so far
            long long ncap = std::max<long long>(E + Ec, 2 * cap);
            int* ne;
            BM_ALLOC(ne, int, 2 * ncap);
            if (E) BM_TRY(cudaMemcpyAsync(ne, edges, sizeof(int) * 2 * E, cudaMemcpyDeviceToDevice, s));
            ar.release(edges);
            edges = ne;
            cap = ncap;
        }
        note_launch();
        unique_scatter_kernel<<<grid_for(Pc, 256), 256, 0, s>>>(sorted, Pc, pos, i0, edges + 2 * E);
        BM_TRY(cudaGetLastError());
        E += Ec;
        ar.release(pos);
        ar.release(flags);
        ar.release(tmp);
        ar.release(pairs);
    }
    ar.release(poff);
    ar.release(pc);
    ar.release(tlist);
    ar.release(toff);
    out.edges = edges;
    out.n_edges = E;
    return true;
}

}  // namespace bm
