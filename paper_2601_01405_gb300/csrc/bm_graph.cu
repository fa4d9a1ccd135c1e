// bm_graph.cu -- K(c) CSR membership compaction and K(d) nerve edges.
//
// K(c): membership keys (row << 32 | point), sorted, become CSR rows: row
// offsets are the positions where the row part changes, ids the low halves.
//
// K(d): the Ball Mapper graph is the 1-skeleton of the nerve (Sec. 2.1,
// Sec. 5.2, Def. 5.6): {i, j} is an edge iff some point lies in both balls.  Every
// point x covered by c_x balls witnesses the c_x (c_x - 1) / 2 pairs of its
// covering landmarks, so the edge set is the deduplicated union of those
// pairs.  Steps: transpose the memberships (point -> covering landmarks),
// count and prefix-sum the pairs per point, emit (i << 32 | j) keys with
// i < j, radix sort, keep the first key of every run.
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

__global__ void count_points_kernel(const unsigned long long* keys, long long nnz, long long* cnt) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride)
        atomicAdd((unsigned long long*)&cnt[keys[i] & 0xffffffffull], 1ull);
}

__global__ void scatter_transpose_kernel(const unsigned long long* keys, long long nnz, const long long* toff,
                                         long long* cursor, int* tlist) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride) {
        const unsigned long long k = keys[i];
        const long long pt = (long long)(k & 0xffffffffull);
        const long long slot = (long long)atomicAdd((unsigned long long*)&cursor[pt], 1ull);
        tlist[toff[pt] + slot] = (int)(k >> 32);
    }
}

__global__ void pair_counts_kernel(const long long* toff, long long n, long long* pc) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const long long c = toff[i + 1] - toff[i];
        pc[i] = c * (c - 1) / 2;
    }
}

// One warp per point: all pairs (a < b) of its covering landmarks.
__global__ void emit_pairs_kernel(const long long* toff, const int* tlist, long long n, const long long* poff,
                                  unsigned long long* pairs) {
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (long long pt = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pt < n; pt += warps) {
        const long long b0 = toff[pt];
        const int c = (int)(toff[pt + 1] - b0);
        if (c < 2) continue;
        long long o = poff[pt];
        for (int a = 0; a < c - 1; ++a) {
            const unsigned la = (unsigned)tlist[b0 + a];
            for (int b = a + 1 + lane; b < c; b += 32) {
                const unsigned lb = (unsigned)tlist[b0 + b];
                const unsigned lo = la < lb ? la : lb, hi = la < lb ? lb : la;
                pairs[o + (b - a - 1)] = ((unsigned long long)lo << 32) | hi;
            }
            o += c - 1 - a;
        }
    }
}

__global__ void unique_flags_kernel(const unsigned long long* keys, long long n, long long* flags) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void unique_scatter_kernel(const unsigned long long* keys, long long n, const long long* pos,
                                      int* edges) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (i == 0 || keys[i] != keys[i - 1]) {
            const long long o = pos[i];
            edges[2 * o] = (int)(keys[i] >> 32);
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
    long long* cnt;
    BM_ALLOC(cnt, long long, n + 1);
    BM_TRY(cudaMemsetAsync(cnt, 0, sizeof(long long) * (n + 1), s));
    note_launch();
    count_points_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(keys, nnz, cnt);
    BM_TRY(cudaGetLastError());
    long long* toff;
    BM_ALLOC(toff, long long, n + 1);
    BM_TRY(exclusive_scan_i64(cnt, toff, n, ar, s));
    int* tlist;
    BM_ALLOC(tlist, int, nnz);
    BM_TRY(cudaMemsetAsync(cnt, 0, sizeof(long long) * (n + 1), s));
    note_launch();
    scatter_transpose_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(keys, nnz, toff, cnt, tlist);
    BM_TRY(cudaGetLastError());
    note_launch();
    pair_counts_kernel<<<grid_for(n, 256), 256, 0, s>>>(toff, n, cnt);
    BM_TRY(cudaGetLastError());
    long long* poff;
    BM_ALLOC(poff, long long, n + 1);
    BM_TRY(exclusive_scan_i64(cnt, poff, n, ar, s));
    long long P = 0;
    BM_TRY(cudaMemcpyAsync(&P, poff + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    BM_TRY(cudaStreamSynchronize(s));
    out.pairs = P;
    if (P == 0) return true;
    if (P >= (1LL << 32)) {
        f.status = BM_ERR_CAPACITY;
        f.msg = "nerve pass: " + std::to_string(P) + " witnessed pairs exceed one sort (2^32 keys)";
        return false;
    }
    unsigned long long *pairs, *tmp;
    BM_ALLOC(pairs, unsigned long long, P);
    BM_ALLOC(tmp, unsigned long long, P);
    note_launch();
    emit_pairs_kernel<<<grid_for(n * 32, 256), 256, 0, s>>>(toff, tlist, n, poff, pairs);
    BM_TRY(cudaGetLastError());
    ar.release(tlist);
    const int lb = bits_for(L - 1);
    unsigned long long* sorted = nullptr;
    BM_TRY(radix_sort_u64(pairs, tmp, P, digit_shifts(lb, lb), ar, s, &sorted));
    long long* flags;
    BM_ALLOC(flags, long long, P);
    long long* pos;
    BM_ALLOC(pos, long long, P + 1);
    note_launch();
    unique_flags_kernel<<<grid_for(P, 256), 256, 0, s>>>(sorted, P, flags);
    BM_TRY(cudaGetLastError());
    BM_TRY(exclusive_scan_i64(flags, pos, P, ar, s));
    long long E = 0;
    BM_TRY(cudaMemcpyAsync(&E, pos + P, sizeof(long long), cudaMemcpyDeviceToHost, s));
    BM_TRY(cudaStreamSynchronize(s));
    if (E > 0x7fffffffLL) {
        f.status = BM_ERR_CAPACITY;
        f.msg = "more than 2^31-1 edges";
        return false;
    }
    int* edges;
    BM_ALLOC(edges, int, 2 * E);
    note_launch();
    unique_scatter_kernel<<<grid_for(P, 256), 256, 0, s>>>(sorted, P, pos, edges);
    BM_TRY(cudaGetLastError());
    ar.release(pos);
    ar.release(flags);
    ar.release(tmp);
    ar.release(pairs);
    ar.release(poff);
    ar.release(toff);
    ar.release(cnt);
    out.edges = edges;
    out.n_edges = E;
    return true;
}

}  // namespace bm
