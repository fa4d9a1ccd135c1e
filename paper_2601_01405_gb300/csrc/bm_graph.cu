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
// landmarks, by a radix sort of swapped keys) and count the witnessed pairs per
// smaller landmark.  Then one of two deduplications, chosen by size:
//   bitmap  (dense witnesses): the landmark rows are cut into chunks whose
//           L-bit rows fit a bitmap budget; every witnessed pair sets bit j of
//           row i (warp-aggregated atomicOr); each row's set bits, read in
//           order, are its edges.  Memory and work are independent of how often
//           a pair is witnessed.
//   sort    (sparse witnesses): chunks of at most 2^28 pairs; emit
//           (i << 32 | j) keys, radix sort, keep the first key of every run.
// Chunks ascend in i, so the edges come out lexicographic either way.
#include <atomic>
#include <string>

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

// (row << 32 | point) at index e -> (point << 32 | e): sorted stably on the point alone,
// these give every point's cover list in landmark order (e ascends with the landmark)
// and, through e, where each membership sits in it.
__global__ void point_index_keys_kernel(const unsigned long long* keys, long long nnz, unsigned long long* out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
        out[e] = (keys[e] << 32) | (unsigned long long)e;
}

// tlist holds the membership index e at each cover-list position p: record tpos[e] = p and
// replace it by e's landmark.
__global__ void cover_from_index_kernel(const unsigned long long* keys, long long nnz, int* tlist, int* tpos) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
        const long long e = (long long)(unsigned)tlist[p];
        tpos[e] = (int)p;
        tlist[p] = (int)(keys[e] >> 32);
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

// Bitmap deduplication.  One warp per membership (i, x) of landmark rows
// [i0, i1), taken in row order from the sorted membership keys (entries
// moff[i0] .. moff[i1]): the warp finds i in x's ascending cover list (binary
// search) and every later entry j of that list sets bit j of row i - i0 (W
// 32-bit words per row).  Walking the memberships in row order keeps the rows
// being written few and L2-resident.  Lanes take consecutive entries
// (ascending j), so lanes on the same word are contiguous: a segmented OR over
// the run leaves the union with its first lane, which issues one atomicOr.
// Inputs that break the CSR invariants (an index outside its array, i missing
// from x's list) are not dereferenced: the kernel records them in *bad and
// skips the entry.
__global__ void nerve_bits_kernel(const unsigned long long* keys, const long long* moff, const long long* toff,
                                  const int* tlist, const int* tpos, long long nnz, long long n, int i0, int i1,
                                  long long W, unsigned* bits, int* bad) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long e0 = moff[i0], e1 = moff[i1];
    if (e0 < 0 || e1 > nnz || e0 > e1) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(bad, 16);
        return;
    }
    for (long long e = e0 + (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < e1; e += warps) {
        const unsigned long long key = keys[e];
        const int i = (int)(key >> 32);
        const long long x = (long long)(key & 0xffffffffull);
        if (i < i0 || i >= i1 || x >= n) {
            if (lane == 0) atomicOr(bad, 1);
            continue;
        }
        const long long b0 = toff[x], end = toff[x + 1];
        if (b0 < 0 || end > nnz || b0 >= end) {
            if (lane == 0) atomicOr(bad, 2);
            continue;
        }
        const long long t = tpos[e];   // where membership e sits in x's cover list
        if (t < b0 || t >= end || tlist[t] != i) {
            if (lane == 0) atomicOr(bad, 32);
            continue;
        }
        unsigned* row = bits + (long long)(i - i0) * W;
        for (long long base = t + 1; base < end; base += 32) {
            const long long b = base + lane;
            const bool valid = b < end;
            int j = valid ? tlist[b] : 0;
            if (valid && (j <= i || (long long)(j >> 5) >= W)) {   // cover lists ascend and stay below L
                atomicOr(bad, 4);
                j = 0;
            }
            const bool ok = valid && j > i;
            const int word = ok ? (j >> 5) : -1 - lane;   // skipped lanes never join a run
            unsigned acc = ok ? (1u << (j & 31)) : 0u;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned v = __shfl_down_sync(kFull, acc, off);
                const int w = __shfl_down_sync(kFull, word, off);
                if (lane + off < 32 && w == word) acc |= v;
            }
            const int wprev = __shfl_up_sync(kFull, word, 1);
            if (ok && (lane == 0 || wprev != word)) atomicOr(row + word, acc);
        }
    }
}

// Row-per-block bitmap emission (rows of up to 51,200 words): a block takes landmark
// rows i from a counter and builds row i in shared memory from the memberships (i, x)
// and the later entries j of each x's cover list (shared-memory atomicOr, one per run
// of lanes on a word, as above), then stores the row's non-zero words.  No global
// atomics, and a heavy row never spreads its bits over L2.  Same input checks as
// nerve_bits_kernel.
__global__ void __launch_bounds__(512) nerve_rows_kernel(const unsigned long long* keys, const long long* moff,
                                                         const long long* toff, const int* tlist, const int* tpos,
                                                         long long nnz, long long n, int i0, int i1, long long W,
                                                         unsigned* bits, int* bad, int* next_row) {
    extern __shared__ unsigned srow[];
    __shared__ int s_row;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (long long w = threadIdx.x; w < W; w += blockDim.x) srow[w] = 0u;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_row = atomicAdd(next_row, 1);
        __syncthreads();
        const long long i = (long long)i0 + s_row;
        if (i >= i1) break;
        const long long e0 = moff[i], e1 = moff[i + 1];
        if (e0 < 0 || e1 > nnz || e0 > e1) {
            if (threadIdx.x == 0) atomicOr(bad, 16);
            continue;
        }
        // 32 memberships per warp at a time: their look-ups (the point, its cover list's
        // extent, where i sits in it) are one load per lane, issued together; then the
        // warp walks the 32 suffixes one after the other
        for (long long eb = e0 + (long long)warp * 32; eb < e1; eb += (long long)nwarps * 32) {
            const long long e = eb + lane;
            long long t = 0, end = 0;
            bool good = false;
            if (e < e1) {
                const unsigned long long key = keys[e];
                const long long x = (long long)(key & 0xffffffffull);
                if ((long long)(key >> 32) != i || x >= n) {
                    atomicOr(bad, 1);
                } else {
                    const long long b0 = toff[x];
                    end = toff[x + 1];
                    if (b0 < 0 || end > nnz || b0 >= end) {
                        atomicOr(bad, 2);
                    } else {
                        t = tpos[e];   // where membership e sits in x's cover list
                        if (t < b0 || t >= end || tlist[t] != (int)i) atomicOr(bad, 32);
                        else good = true;
                    }
                }
            }
            for (unsigned mm = __ballot_sync(kFull, good); mm; mm &= mm - 1) {
                const int m = __ffs(mm) - 1;
                const long long tm = __shfl_sync(kFull, t, m), endm = __shfl_sync(kFull, end, m);
                // four loads in flight per lane before the bits are combined
                for (long long base = tm + 1; base < endm; base += 128) {
                    int jv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const long long b = base + u * 32 + lane;
                        jv[u] = b < endm ? tlist[b] : 0;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (base + u * 32 >= endm) break;   // warp-uniform
                        const bool valid = base + u * 32 + lane < endm;
                        int j = jv[u];
                        if (valid && (j <= (int)i || (long long)(j >> 5) >= W)) {
                            atomicOr(bad, 4);
                            j = 0;
                        }
                        const bool ok = valid && j > (int)i;
                        const int word = ok ? (j >> 5) : -1 - lane;
                        unsigned acc = ok ? (1u << (j & 31)) : 0u;
#pragma unroll
                        for (int off = 1; off < 32; off <<= 1) {
                            const unsigned v = __shfl_down_sync(kFull, acc, off);
                            const int w = __shfl_down_sync(kFull, word, off);
                            if (lane + off < 32 && w == word) acc |= v;
                        }
                        const int wprev = __shfl_up_sync(kFull, word, 1);
                        if (ok && (lane == 0 || wprev != word)) atomicOr(&srow[word], acc);
                    }
                }
            }
        }
        __syncthreads();
        unsigned* row = bits + (i - i0) * W;
        for (long long w = ((i + 1) >> 5) + threadIdx.x; w < W; w += blockDim.x) {
            const unsigned v = srow[w];
            if (v) {
                row[w] = v;
                srow[w] = 0u;
            }
        }
    }
}

// Set bits per bitmap row (one warp per row).
__global__ void bitrow_counts_kernel(const unsigned* bits, long long R, long long W, long long* cnt) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < R; r += warps) {
        const unsigned* row = bits + r * W;
        long long c = 0;
        for (long long w = lane; w < W; w += 32) c += __popc(row[w]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        if (lane == 0) cnt[r] = c;
    }
}

// Position of the r-th (0-based) set bit of v (popcount bisection).
__device__ __forceinline__ int nth_set_bit(unsigned v, int r) {
    int pos = 0;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const unsigned low = (1u << sh) - 1u;
        const int c = __popc(v & low);
        if (r >= c) {
            r -= c;
            v >>= sh;
            pos += sh;
        } else {
            v &= low;
        }
    }
    return pos;
}

// Row r's set bits, in ascending order, become edges (i0 + r, j) at positions
// roff[r] ... (one warp per row).  Per 32 words the warp scans the popcounts and
// writes the group's edges with consecutive lanes on consecutive slots: slot k's
// word is found by bisection over the scanned counts, its bit by nth_set_bit.
__global__ void bitrow_extract_kernel(const unsigned* bits, long long R, long long W, int i0, const long long* roff,
                                      int* edges, int* bad) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long total = roff[R];
    int2* out = reinterpret_cast<int2*>(edges);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < R; r += warps) {
        const unsigned* row = bits + r * W;
        long long pos = roff[r];
        const int i = i0 + (int)r;
        for (long long w0 = ((long long)i + 1) >> 5 & ~31LL; w0 < W; w0 += 32) {
            const unsigned word = (w0 + lane < W) ? row[w0 + lane] : 0u;
            const int c = __popc(word);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const int T = __shfl_sync(kFull, incl, 31);
            for (int kb = 0; kb < T; kb += 32) {
                const int k = kb + lane;
                int owner = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int v = __shfl_sync(kFull, incl, owner + step - 1);
                    if (v <= k) owner += step;
                }
                const unsigned ow = __shfl_sync(kFull, word, owner & 31);
                const int before = __shfl_sync(kFull, incl - c, owner & 31);
                if (k < T) {
                    const long long o = pos + k;
                    if (o < total) out[o] = make_int2(i, (int)((w0 + owner) * 32) + nth_set_bit(ow, k - before));
                    else atomicOr(bad, 8);
                }
            }
            pos += T;
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
    pdl_wait();
    pdl_trigger();
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
    return launch_pdl(compact_segments_kernel, dim3(2 * nseg), dim3(256), 0, s, src, band_src, seg_cap, seg_counts,
                      band_seg_counts, nseg, dst, band_dst, count_out, band_count_out, st, overflow_bit,
                      check_done ? 1 : 0, stop_on_overflow ? 1 : 0);
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

// Stage 1: point -> covering landmarks (transpose by a stable radix sort of
// (point, membership index) keys on the point bits: the memberships are in landmark
// order, so each cover list comes out ascending), the position of every membership in
// its cover list (j.tpos), pairs per smaller landmark and their exclusive scan j.lpre
// (L + 1).
bool edges_transpose(EdgeJob& j, Arena& ar, cudaStream_t s, Failure& f) {
    const long long nnz = j.nnz, n = j.n, L = j.L;
    unsigned long long *tk, *tk2;
    BM_ALLOC(tk, unsigned long long, nnz);
    BM_ALLOC(tk2, unsigned long long, nnz);
    note_launch();
    point_index_keys_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(j.keys, nnz, tk);
    BM_TRY(cudaGetLastError());
    BM_TRY(radix_sort_u64(tk, tk2, nnz, digit_shifts(0, bits_for(n - 1)), ar, s, &j.tsorted));
    BM_ALLOC(j.toff, long long, n + 1);
    BM_ALLOC(j.tlist, int, nnz);
    BM_ALLOC(j.tpos, int, nnz);
    BM_TRY(launch_csr_from_sorted(j.tsorted, nnz, n, j.toff, j.tlist, s));
    note_launch();
    cover_from_index_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(j.keys, nnz, j.tlist, j.tpos);
    BM_TRY(cudaGetLastError());
    unsigned long long* plc;
    BM_ALLOC(plc, unsigned long long, L + 1);
    BM_TRY(cudaMemsetAsync(plc, 0, sizeof(unsigned long long) * (L + 1), s));
    note_launch();
    landmark_pair_counts_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(j.tsorted, j.toff, j.tlist, nnz, plc);
    BM_TRY(cudaGetLastError());
    BM_ALLOC(j.lpre, long long, L + 1);
    BM_TRY(exclusive_scan_i64((const long long*)plc, j.lpre, L, ar, s));
    ar.release(plc);
    ar.release(tk);   // the sorted swapped keys (one of the two) are not needed after this
    ar.release(tk2);
    j.tsorted = nullptr;
    return true;
}

namespace {
constexpr long long kDefaultBitmapBytes = 1LL << 30;
std::atomic<long long> g_bitmap_bytes{kDefaultBitmapBytes};
}  // namespace

long long edges_bitmap_budget() { return g_bitmap_bytes.load(); }

long long edges_set_bitmap_budget(long long bytes) {
    return g_bitmap_bytes.exchange(bytes == 0 ? kDefaultBitmapBytes : bytes);
}

long long edges_bitmap_words(long long L) { return (L + 31) / 32; }

constexpr long long kRowBlockWords = 51200;   // 200 KB of shared memory per row block

bool edges_choose_bitmap(long long L, long long P) {
    if (edges_bitmap_budget() < 0) return false;
    const double bytes = (double)L * (double)edges_bitmap_words(L) * 4.0;
    return bytes <= 64.0 * (double)P;
}

long long edges_bitmap_rows(long long L) {
    const long long row_bytes = edges_bitmap_words(L) * 4;
    return std::max<long long>(1, std::min<long long>(L, edges_bitmap_budget() / row_bytes));
}

// Stage 2: deduplicate the Pc pairs (i, j), i in [i0, i1), witnessed by the
// points.  Afterwards *j.count_dev (device) is the number of distinct pairs.
bool edges_emit(EdgeJob& j, int i0, int i1, long long Pc, Arena& ar, cudaStream_t s, Failure& f) {
    const long long n = j.n, L = j.L;
    if (j.bitmap) {
        const long long R = i1 - i0, W = edges_bitmap_words(L);
        BM_ALLOC(j.bits, unsigned, R * W);
        BM_TRY(cudaMemsetAsync(j.bits, 0, sizeof(unsigned) * R * W, s));
        if (!j.bad) {
            BM_ALLOC(j.bad, int, 1);
            BM_TRY(cudaMemsetAsync(j.bad, 0, sizeof(int), s));
        }
        if (W <= kRowBlockWords) {
            // rows built in shared memory, one block per row at a time
            static bool attr_set = false;
            if (!attr_set) {
                BM_TRY(cudaFuncSetAttribute(nerve_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)(kRowBlockWords * sizeof(unsigned))));
                attr_set = true;
            }
            int* next_row;
            BM_ALLOC(next_row, int, 1);
            BM_TRY(cudaMemsetAsync(next_row, 0, sizeof(int), s));
            const int per_sm = W * 4 <= 48 * 1024 ? 4 : (W * 4 <= 100 * 1024 ? 2 : 1);
            note_launch();
            nerve_rows_kernel<<<(unsigned)(device_sm_count() * per_sm), 512, (size_t)W * sizeof(unsigned), s>>>(
                j.keys, j.moff, j.toff, j.tlist, j.tpos, j.nnz, n, i0, i1, W, j.bits, j.bad, next_row);
            BM_TRY(cudaGetLastError());
        } else {
            note_launch();
            nerve_bits_kernel<<<grid_for(j.nnz * 32, 256), 256, 0, s>>>(j.keys, j.moff, j.toff, j.tlist, j.tpos, j.nnz,
                                                                         n, i0, i1, W, j.bits, j.bad);
            BM_TRY(cudaGetLastError());
        }
        long long* cnt;
        BM_ALLOC(cnt, long long, R + 1);
        note_launch();
        bitrow_counts_kernel<<<grid_for(R * 32, 256), 256, 0, s>>>(j.bits, R, W, cnt);
        BM_TRY(cudaGetLastError());
        BM_ALLOC(j.pos, long long, R + 1);
        BM_TRY(exclusive_scan_i64(cnt, j.pos, R, ar, s));
        ar.release(cnt);
        j.count_dev = j.pos + R;
        return true;
    }
    long long *pc, *poff;
    BM_ALLOC(pc, long long, n + 1);
    BM_ALLOC(poff, long long, n + 1);
    note_launch();
    chunk_pair_counts_kernel<<<grid_for(n, 256), 256, 0, s>>>(j.toff, j.tlist, n, i0, i1, pc);
    BM_TRY(cudaGetLastError());
    BM_TRY(exclusive_scan_i64(pc, poff, n, ar, s));
    unsigned long long *pairs, *tmp;
    BM_ALLOC(pairs, unsigned long long, Pc);
    BM_ALLOC(tmp, unsigned long long, Pc);
    note_launch();
    emit_chunk_pairs_kernel<<<grid_for(n * 32, 256), 256, 0, s>>>(j.toff, j.tlist, n, i0, i1, poff, pairs);
    BM_TRY(cudaGetLastError());
    BM_TRY(radix_sort_u64(pairs, tmp, Pc, digit_shifts(bits_for(L - 1), bits_for(i1 - i0 - 1)), ar, s, &j.sorted));
    long long* flags;
    BM_ALLOC(flags, long long, Pc);
    BM_ALLOC(j.pos, long long, Pc + 1);
    note_launch();
    unique_flags_kernel<<<grid_for(Pc, 256), 256, 0, s>>>(j.sorted, Pc, flags);
    BM_TRY(cudaGetLastError());
    BM_TRY(exclusive_scan_i64(flags, j.pos, Pc, ar, s));
    ar.release(flags);
    ar.release(j.sorted == pairs ? tmp : pairs);
    ar.release(poff);
    ar.release(pc);
    j.count_dev = j.pos + Pc;
    return true;
}

// Stage 3: write the distinct pairs of stage 2 (as landmark ordinals) to dst.
bool edges_scatter(EdgeJob& j, int i0, int i1, long long Pc, int* dst, Arena& ar, cudaStream_t s, Failure& f) {
    note_launch();
    if (j.bitmap) {
        const long long R = i1 - i0;
        bitrow_extract_kernel<<<grid_for(R * 32, 256), 256, 0, s>>>(j.bits, R, edges_bitmap_words(j.L), i0, j.pos,
                                                                    dst, j.bad);
    } else {
        unique_scatter_kernel<<<grid_for(Pc, 256), 256, 0, s>>>(j.sorted, Pc, j.pos, i0, dst);
    }
    BM_TRY(cudaGetLastError());
    ar.release(j.pos);
    ar.release(j.sorted);
    ar.release(j.bits);
    j.pos = nullptr;
    j.sorted = nullptr;
    j.bits = nullptr;
    j.count_dev = nullptr;
    return true;
}

bool edges_check(const EdgeJob& j, cudaStream_t s, Failure& f) {
    if (!j.bad) return true;
    int hb = 0;
    BM_TRY(cudaMemcpyAsync(&hb, j.bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    BM_TRY(cudaStreamSynchronize(s));
    if (hb) {
        f.status = BM_ERR_CUDA;
        f.msg = "nerve pass: a cover list broke its invariants (code " + std::to_string(hb) + ")";
        return false;
    }
    return true;
}

void edges_release(EdgeJob& j, Arena& ar) {
    ar.release(j.tsorted);
    ar.release(j.toff);
    ar.release(j.tlist);
    ar.release(j.tpos);
    ar.release(j.lpre);
    ar.release(j.bad);
    j.tsorted = nullptr;
    j.toff = nullptr;
    j.tlist = nullptr;
    j.tpos = nullptr;
    j.lpre = nullptr;
    j.bad = nullptr;
}

bool build_edges(const unsigned long long* keys, const long long* moff, long long nnz, long long n, long long L,
                 Arena& ar, cudaStream_t s, EdgeResult& out, Failure& f) {
    out = EdgeResult();
    if (nnz == 0 || L < 2) return true;
    EdgeJob j;
    j.keys = keys;
    j.moff = moff;
    j.nnz = nnz;
    j.n = n;
    j.L = L;
    if (!edges_transpose(j, ar, s, f)) return false;
    // the pair total first; the per-landmark prefix (8 (L + 1) bytes, 54 MB for a batch of
    // 6.7M landmarks) comes to the host only where the sort path needs several chunks
    long long P = 0;
    BM_TRY(cudaMemcpyAsync(&P, j.lpre + L, sizeof(long long), cudaMemcpyDeviceToHost, s));
    BM_TRY(cudaStreamSynchronize(s));
    out.pairs = P;
    if (P == 0) {
        edges_release(j, ar);
        return true;
    }
    j.bitmap = edges_choose_bitmap(L, P);
    std::vector<std::pair<int, int>> chunks;
    std::vector<long long> cpre;   // pairs before each chunk's first landmark, then P
    if (j.bitmap) {
        const long long R = edges_bitmap_rows(L);
        for (long long i0 = 0; i0 < L; i0 += R) chunks.emplace_back((int)i0, (int)std::min(L, i0 + R));
        cpre.resize(chunks.size() + 1);
        for (size_t c = 0; c < chunks.size(); ++c)
            BM_TRY(cudaMemcpyAsync(&cpre[c], j.lpre + chunks[c].first, sizeof(long long), cudaMemcpyDeviceToHost, s));
        cpre[chunks.size()] = P;
        BM_TRY(cudaStreamSynchronize(s));
    } else if (P <= kEdgeChunkPairs) {
        chunks.emplace_back(0, (int)L);
        cpre = {0, P};
    } else {
        std::vector<long long> hpre((size_t)L + 1);
        BM_TRY(cudaMemcpyAsync(hpre.data(), j.lpre, sizeof(long long) * (L + 1), cudaMemcpyDeviceToHost, s));
        BM_TRY(cudaStreamSynchronize(s));
        for (long long i0 = 0; i0 < L;) {
            // largest i1 with pairs(i0, i1) <= budget (at least one landmark)
            long long lo = i0 + 1, hi = L;
            while (lo < hi) {
                const long long mid = (lo + hi + 1) / 2;
                if (hpre[(size_t)mid] - hpre[(size_t)i0] <= kEdgeChunkPairs) lo = mid;
                else hi = mid - 1;
            }
            const long long i1 = lo;
            if (hpre[(size_t)i1] - hpre[(size_t)i0] >= (1LL << 32)) {
                f.status = BM_ERR_CAPACITY;
                f.msg = "nerve pass: one landmark witnesses more than 2^32 pairs";
                return false;
            }
            chunks.emplace_back((int)i0, (int)i1);
            cpre.push_back(hpre[(size_t)i0]);
            i0 = i1;
        }
        cpre.push_back(P);
    }
    // per chunk: deduplicate, then append (chunks ascend in i)
    int* edges = nullptr;
    long long E = 0, cap = 0;
    for (size_t c = 0; c < chunks.size(); ++c) {
        const int i0 = chunks[c].first, i1 = chunks[c].second;
        const long long Pc = cpre[c + 1] - cpre[c];
        if (Pc == 0) continue;
        if (!edges_emit(j, i0, i1, Pc, ar, s, f)) return false;
        long long Ec = 0;
        BM_TRY(cudaMemcpyAsync(&Ec, j.count_dev, sizeof(long long), cudaMemcpyDeviceToHost, s));
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
        if (!edges_scatter(j, i0, i1, Pc, edges + 2 * E, ar, s, f)) return false;
        E += Ec;
    }
    if (!edges_check(j, s, f)) return false;
    edges_release(j, ar);
    out.edges = edges;
    out.n_edges = E;
    return true;
}

}  // namespace bm
