// bm_gidx.cu -- graph-based conservative range oracle (Sec. 5.4).
//
// The paper's second family of non-exhaustive indexes searches a proximity
// graph: a query examines only the points its partial traversal visits, and
// decides membership with the exact distance, so no point outside the ball is
// ever returned (false negatives only).  This file builds the graph and runs
// the traversal, GPU-native and deterministic:
//
//   graph   every point's M nearest other points, by (FP64 squared distance, id)
//           (from the exact k-NN machinery: per-row radius range query, then an
//           ordered selection), made undirected (the arcs and their reverses,
//           sorted and deduplicated); adjacency lists ascend by id.
//   query   one warp per query row, all distances FP64 in coordinate order:
//           1. entry: the nearest of E entry points floor(t n / E);
//           2. beam: a sorted list of at most ef visited nodes in shared memory;
//              the best unexpanded one is expanded (its neighbours, in
//              adjacency order, are visited once and enter the list when it has
//              room or they beat its worst); until every listed node is expanded;
//           3. range expansion: visited nodes inside the ball that were not
//              expanded are expanded in visit order (first in, first out);
//           at most max_visits visits per query.  Visited nodes are kept in a
//           per-query open-addressing table in global memory.
//   The row is every visited node with D < r^2; it is emitted as (row << 32 |
//   point) keys through the same sink as the distance tiles (with the greedy's
//   candidate-conflict bookkeeping), so range queries, fixed-landmark builds and
//   the greedy itself run through this index unchanged.
#include <algorithm>
#include <climits>

#include "bm_host.h"

namespace bm {

namespace {

constexpr int kSearchWarps = 4;   // warps (queries) per block
constexpr int kMaxEf = 256;

// ---------------------------------------------------------------- graph construction

// One warp per row: the M nearest other points of row r among its ball's entries
// (ids ascending, FP64 squared distances D), by (D, id).  DM = the M-th smallest D
// among the entries other than r; the row keeps every entry with D < DM and, in id
// order, the first ones with D == DM until M are kept.  *bad |= 4 when a row holds
// fewer than M others.
__global__ void __launch_bounds__(256) knn_ids_kernel(const long long* __restrict__ offsets,
                                                      const int* __restrict__ ids, const double* __restrict__ D,
                                                      const double* __restrict__ DM, long long rows, int M,
                                                      int* __restrict__ nbr, int* bad) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        const long long e0 = offsets[r], e1 = offsets[r + 1];
        const double dm = DM[r];
        // how many strictly below DM (they are all kept)
        int less = 0;
        for (long long e = e0 + lane; e < e1; e += 32)
            if (ids[e] != (int)r && D[e] < dm) ++less;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) less += __shfl_xor_sync(kFull, less, o);
        int need_eq = M - less;   // entries equal to DM still to take, smallest ids first
        int kept = 0;
        const unsigned below = (1u << lane) - 1u;
        for (long long b = e0; b < e1; b += 32) {
            const long long e = b + lane;
            const bool valid = e < e1 && ids[e] != (int)r;
            const double v = valid ? D[e] : INFINITY;
            const bool eq = valid && v == dm;
            const unsigned eqb = __ballot_sync(kFull, eq);
            const bool take = (valid && v < dm) || (eq && __popc(eqb & below) < need_eq);
            const int ne = __popc(eqb);
            need_eq -= ne < need_eq ? ne : (need_eq > 0 ? need_eq : 0);
            const unsigned tb = __ballot_sync(kFull, take);
            const int pos = kept + __popc(tb & below);
            if (take && pos < M) nbr[r * M + pos] = ids[e];
            kept += __popc(tb);
        }
        if (lane == 0 && kept < M) {
            atomicOr(bad, 4);
            for (int t = kept; t < M; ++t) nbr[r * M + t] = (int)r;
        }
    }
}

// arcs (i, nbr) and their reverses as keys (a << 32 | b)
__global__ void arc_keys_kernel(const int* __restrict__ nbr, long long n, int M, unsigned long long* keys) {
    const long long total = n * M;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const unsigned long long i = (unsigned long long)(t / M), j = (unsigned)nbr[t];
        keys[2 * t] = (i << 32) | j;
        keys[2 * t + 1] = (j << 32) | i;
    }
}

__global__ void first_of_run_kernel(const unsigned long long* __restrict__ keys, long long n, long long* flags) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void compact_runs_kernel(const unsigned long long* __restrict__ keys, long long n,
                                    const long long* __restrict__ pos, unsigned long long* out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        if (i == 0 || keys[i] != keys[i - 1]) out[pos[i]] = keys[i];
}

// ---------------------------------------------------------------- search

__device__ __forceinline__ unsigned hash_id(int v, unsigned mask) {
    unsigned h = (unsigned)v * 0x9E3779B1u;
    h ^= h >> 15;
    return h & mask;
}

__device__ __forceinline__ bool table_has(const int* tab, unsigned mask, int v) {
    unsigned s = hash_id(v, mask);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const int x = tab[s];
        if (x == v) return true;
        if (x == -1) return false;
        s = (s + 1) & mask;
    }
    return false;
}

__device__ __forceinline__ void table_put(int* tab, unsigned mask, int v) {
    unsigned s = hash_id(v, mask);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const int old = atomicCAS(&tab[s], -1, v);
        if (old == -1 || old == v) return;
        s = (s + 1) & mask;
    }
}

struct BeamEntry {
    double D;
    int id;
    int slot;
};

__device__ __forceinline__ bool beam_less(double da, int ia, double db, int ib) {
    return da < db || (da == db && ia < ib);
}

struct SearchArgs {
    const float* Q;             // query rows (candidate rows in greedy mode)
    long long rows_max;
    const int* rows_dev;        // greedy: active rows on the device
    long long row0;             // first row of this launch (chunking)
    const float* X;
    long long n;
    int d;
    const long long* adj_off;
    const int* adj;
    int E, ef;
    long long max_visits;
    unsigned table_mask;        // table slots - 1
    double eps2;
    int* table;                 // per chunk row: table_mask + 1 ints (cleared here)
    int* vis_id;                // per chunk row: max_visits
    double* vis_D;
    unsigned char* vis_exp;
    const DeviceState* st;
    int check_done;
    HitSink sink;
    unsigned long long* visits; // total visits (statistics)
    int* truncated;             // set when a query reached max_visits
};

// Insert (D, v, slot) into the sorted beam of n_ entries (capacity ef); the whole warp calls it.
__device__ __forceinline__ void beam_insert(BeamEntry* R, int& nR, int ef, double D, int v, int slot) {
    const int lane = threadIdx.x & 31;
    if (nR == ef && !beam_less(D, v, R[nR - 1].D, R[nR - 1].id)) return;
    // position: entries less than the key
    int p = 0;
    for (int b = 0; b < nR; b += 32) {
        const int i = b + lane;
        const bool lt = i < nR && beam_less(R[i].D, R[i].id, D, v);
        p += __popc(__ballot_sync(kFull, lt));
    }
    const int last = nR < ef ? nR : ef - 1;   // entries [p, last) move one place up
    BeamEntry tmp[kMaxEf / 32];
#pragma unroll
    for (int k = 0; k < kMaxEf / 32; ++k) {
        const int i = p + k * 32 + lane;
        if (i < last) tmp[k] = R[i];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < kMaxEf / 32; ++k) {
        const int i = p + k * 32 + lane;
        if (i < last) R[i + 1] = tmp[k];
    }
    __syncwarp();
    if (lane == 0) {
        R[p].D = D;
        R[p].id = v;
        R[p].slot = slot;
    }
    __syncwarp();
    if (nR < ef) ++nR;
}

__global__ void __launch_bounds__(kSearchWarps * 32) graph_search_kernel(SearchArgs a) {
    __shared__ BeamEntry s_R[kSearchWarps][kMaxEf];
    if (a.check_done && a.st->done) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long rows = a.rows_dev ? (long long)*a.rows_dev : a.rows_max;
    const long long local = (long long)blockIdx.x * kSearchWarps + w;   // row within this chunk
    const long long row = a.row0 + local;
    if (row >= rows) return;
    BeamEntry* R = s_R[w];
    int* tab = a.table + local * (long long)(a.table_mask + 1);
    int* vid = a.vis_id + local * a.max_visits;
    double* vD = a.vis_D + local * a.max_visits;
    unsigned char* vexp = a.vis_exp + local * a.max_visits;
    for (unsigned s = lane; s <= a.table_mask; s += 32) tab[s] = -1;
    __syncwarp();
    const float* q = a.Q + row * a.d;
    const int d = a.d;
    // 1. entry: the nearest entry point by (D, id)
    double bd = INFINITY;
    int bi = INT_MAX;
    for (int t = lane; t < a.E; t += 32) {
        const long long e = (long long)t * a.n / a.E;
        const double D = exact_sqdist(q, a.X + e * d, d);
        if (beam_less(D, (int)e, bd, bi)) { bd = D; bi = (int)e; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double od = __shfl_xor_sync(kFull, bd, o);
        const int oi = __shfl_xor_sync(kFull, bi, o);
        if (beam_less(od, oi, bd, bi)) { bd = od; bi = oi; }
    }
    long long nv = 1;
    if (lane == 0) {
        table_put(tab, a.table_mask, bi);
        vid[0] = bi;
        vD[0] = bd;
        vexp[0] = 0;
        R[0].D = bd;
        R[0].id = bi;
        R[0].slot = 0;
    }
    __syncwarp();
    int nR = 1;
    bool capped = false;
    // expand node c: visit its unvisited neighbours in adjacency order (up to the cap);
    // in the beam phase they are offered to the beam in that order
    auto expand = [&](int c, bool beam) {
        const long long a0 = a.adj_off[c], a1 = a.adj_off[c + 1];
        for (long long b = a0; b < a1 && nv < a.max_visits; b += 32) {
            const long long e = b + lane;
            const int v = e < a1 ? a.adj[e] : -1;
            const bool fresh = v >= 0 && !table_has(tab, a.table_mask, v);
            const unsigned fb = __ballot_sync(kFull, fresh);
            const long long rank = __popc(fb & ((1u << lane) - 1u));
            const bool allowed = fresh && nv + rank < a.max_visits;
            const unsigned ab = __ballot_sync(kFull, allowed);
            if (__popc(ab) < __popc(fb)) capped = true;
            double D = INFINITY;
            if (allowed) {
                D = exact_sqdist(q, a.X + (long long)v * d, d);
                table_put(tab, a.table_mask, v);
                vid[nv + rank] = v;
                vD[nv + rank] = D;
                vexp[nv + rank] = 0;
            }
            __syncwarp();
            if (beam) {
                unsigned m = ab;
                while (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1;
                    const double Ds = __shfl_sync(kFull, D, src);
                    const int vs = __shfl_sync(kFull, v, src);
                    const int slot = (int)(nv + __popc(ab & ((1u << src) - 1u)));
                    beam_insert(R, nR, a.ef, Ds, vs, slot);
                }
            }
            nv += __popc(ab);
        }
    };
    // 2. beam phase
    while (true) {
        int pick = -1;
        for (int b = 0; b < nR && pick < 0; b += 32) {
            const int i = b + lane;
            const bool un = i < nR && vexp[R[i].slot] == 0;
            const unsigned ub = __ballot_sync(kFull, un);
            if (ub) pick = b + __ffs(ub) - 1;
        }
        if (pick < 0) break;
        const int c = R[pick].id;
        if (lane == 0) vexp[R[pick].slot] = 1;
        __syncwarp();
        expand(c, true);
    }
    // 3. range expansion in visit order
    for (long long h = 0; h < nv; ++h) {
        if (!(vD[h] < a.eps2) || vexp[h]) continue;
        if (lane == 0) vexp[h] = 1;
        __syncwarp();
        expand(vid[h], false);
    }
    // emit the in-range visited nodes
    for (long long b = 0; b < nv; b += 32) {
        const long long h = b + lane;
        const bool in = h < nv && vD[h] < a.eps2;
        const int col = in ? vid[h] : 0;
        const unsigned long long pos = warp_reserve(a.sink.count, in ? 1u : 0u);
        if (in) {
            if (pos < a.sink.cap) a.sink.keys[pos] = ((unsigned long long)row << 32) | (unsigned)col;
            if (a.sink.slot_of) {
                const int s = a.sink.slot_of[col];
                if (s > (int)row) {
                    atomicOr(&a.sink.conflict[(size_t)row * a.sink.conflict_words + (s >> 5)], 1u << (s & 31));
                    atomicOr(&a.sink.row_any[row >> 5], 1u << (row & 31));
                }
            }
        }
    }
    if (lane == 0) {
        atomicAdd(a.visits, (unsigned long long)nv);
        if (capped) atomicOr(a.truncated, 1);
    }
}

// after all chunks: the hit count must fit the sink
__global__ void search_overflow_kernel(DeviceState* st, const unsigned long long* count, unsigned long long cap,
                                       int overflow_bit, int stop) {
    if (*count > cap) {
        atomicOr(&st->error, overflow_bit);
        if (stop) st->done = 1;
    }
}

}  // namespace

cudaError_t launch_knn_ids(const long long* offsets, const int* ids, const double* D, const double* DM, long long rows,
                           int M, int* nbr, int* bad, cudaStream_t s) {
    if (rows == 0) return cudaSuccess;
    long long g = (rows + 7) / 8;
    const long long cap = (long long)device_sm_count() * 16;
    note_launch();
    knn_ids_kernel<<<(unsigned)(g < cap ? g : cap), 256, 0, s>>>(offsets, ids, D, DM, rows, M, nbr, bad);
    return cudaGetLastError();
}

cudaError_t launch_arc_keys(const int* nbr, long long n, int M, unsigned long long* keys, cudaStream_t s) {
    long long g = (n * M + 255) / 256;
    const long long cap = (long long)device_sm_count() * 16;
    note_launch();
    arc_keys_kernel<<<(unsigned)(g < cap ? g : cap), 256, 0, s>>>(nbr, n, M, keys);
    return cudaGetLastError();
}

cudaError_t launch_unique_sorted(const unsigned long long* keys, long long n, long long* flags, long long* pos,
                                 unsigned long long* out, Arena& ar, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    long long g = (n + 255) / 256;
    const long long cap = (long long)device_sm_count() * 16;
    note_launch();
    first_of_run_kernel<<<(unsigned)(g < cap ? g : cap), 256, 0, s>>>(keys, n, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = exclusive_scan_i64(flags, pos, n, ar, s);
    if (e != cudaSuccess) return e;
    note_launch();
    compact_runs_kernel<<<(unsigned)(g < cap ? g : cap), 256, 0, s>>>(keys, n, pos, out);
    return cudaGetLastError();
}

long long graph_search_chunk_rows(long long max_visits, unsigned table_slots) {
    // per row: table ints + visit ids, D and flags; keep one chunk near 1 GiB
    const long long per = (long long)table_slots * 4 + max_visits * (4 + 8 + 1);
    long long rows = (1LL << 30) / (per > 0 ? per : 1);
    if (rows < kSearchWarps) rows = kSearchWarps;
    if (rows > 65536) rows = 65536;
    return rows / kSearchWarps * kSearchWarps;
}

cudaError_t launch_graph_search(const SweepDesc& sd, const GraphIndex& gx, DeviceState* st, unsigned long long* count,
                                unsigned long long cap, int overflow_bit, bool greedy, Arena& ar, cudaStream_t s,
                                unsigned long long* visits, int* truncated) {
    const long long rows_max = sd.a_rows_max;
    if (rows_max == 0 || gx.n == 0) return cudaSuccess;
    unsigned slots = 64;
    while ((long long)slots < 2 * sd.gidx_max_visits) slots <<= 1;
    const long long chunk = std::min<long long>(graph_search_chunk_rows(sd.gidx_max_visits, slots),
                                                (rows_max + kSearchWarps - 1) / kSearchWarps * kSearchWarps);
    int* table = (int*)ar.get(sizeof(int) * (size_t)chunk * slots);
    int* vid = (int*)ar.get(sizeof(int) * (size_t)chunk * sd.gidx_max_visits);
    double* vD = (double*)ar.get(sizeof(double) * (size_t)chunk * sd.gidx_max_visits);
    unsigned char* vexp = (unsigned char*)ar.get((size_t)chunk * sd.gidx_max_visits);
    if (!table || !vid || !vD || !vexp) return cudaErrorMemoryAllocation;
    SearchArgs a;
    a.Q = sd.a->x;
    a.rows_max = rows_max;
    a.rows_dev = sd.a_rows_dev;
    a.X = gx.X;
    a.n = gx.n;
    a.d = gx.d;
    a.adj_off = gx.adj_off;
    a.adj = gx.adj;
    a.E = gx.E;
    a.ef = sd.gidx_ef;
    a.max_visits = sd.gidx_max_visits;
    a.table_mask = slots - 1;
    a.eps2 = sd.eps2;
    a.table = table;
    a.vis_id = vid;
    a.vis_D = vD;
    a.vis_exp = vexp;
    a.st = st;
    a.check_done = greedy ? 1 : 0;
    a.sink = sd.sink;
    a.sink.count = count;
    a.sink.cap = cap;
    a.visits = visits;
    a.truncated = truncated;
    for (long long r0 = 0; r0 < rows_max; r0 += chunk) {
        a.row0 = r0;
        const long long rows = std::min(chunk, rows_max - r0);
        note_launch();
        graph_search_kernel<<<(unsigned)((rows + kSearchWarps - 1) / kSearchWarps), kSearchWarps * 32, 0, s>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    note_launch();
    search_overflow_kernel<<<1, 1, 0, s>>>(st, count, cap, overflow_bit, greedy ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    ar.release(vexp);
    ar.release(vD);
    ar.release(vid);
    ar.release(table);
    return e;
}

}  // namespace bm
