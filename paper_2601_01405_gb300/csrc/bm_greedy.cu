// bm_greedy.cu -- K(a): block-greedy epsilon-net in index order.
//
// The greedy of Sec. 2.2 selects an uncovered point, adds it to the landmark
// set and covers its open ball, until no point is uncovered.  With the
// smallest uncovered index selected every time, x is a landmark exactly when
// no landmark l < x has d(l, x) < eps.  One step of this implementation
// processes a block of the next S uncovered points ("candidates") at once:
//
//   select  (1 CTA)   next S uncovered ids in index order, gather their rows
//   sweep   (grid)    candidates x all points with the distance tiles: the
//                     full open ball of every candidate, plus an S x S bit
//                     matrix conflict[k][s] = "candidate k covers candidate s", s > k
//   resolve (1 warp)  walk the candidates in index order; a candidate is a
//                     landmark iff no earlier landmark candidate covers it,
//                     which is the sequential rule restricted to the block
//   apply   (grid)    keep the balls of the new landmarks: mark their points
//                     covered and append (landmark ordinal, point) keys
//
// The balls computed in the sweep are the full balls X_i of Sec. 2.3, so the
// membership lists come out of the greedy with no second pass.
#include "bm_host.h"

namespace bm {

namespace {

constexpr int kSelThreads = 1024;

__global__ void __launch_bounds__(kSelThreads) greedy_select_kernel(
    DeviceState* st, const unsigned* __restrict__ covered, long long n, int S, int* slot_of,
    int* cand_ids, unsigned* conflict, unsigned* row_any, int words, const float* __restrict__ X,
    const float* __restrict__ phi, int d, float* cand_x, float* cand_phi, int want_tc,
    const __nv_bfloat16* __restrict__ H, const __nv_bfloat16* __restrict__ Lo,
    const __nv_bfloat16* __restrict__ Aug, int d_pad, __nv_bfloat16* cH, __nv_bfloat16* cLo,
    __nv_bfloat16* cAug) {
    if (st->done) return;
    if (st->error & kErrTimeout) {  // a bounded wait expired in a previous step: stop the loop
        if (threadIdx.x == 0) st->done = 1;
        return;
    }
    __shared__ int s_scan[33];
    __shared__ int s_found;
    __shared__ long long s_pos;
    const int tid = threadIdx.x;

    // 1. undo the previous step's bookkeeping
    const int prev = st->cand_count;
    for (int i = tid; i < prev; i += kSelThreads) slot_of[cand_ids[i]] = -1;
    for (int i = tid; i < prev * words; i += kSelThreads) conflict[i] = 0;
    for (int i = tid; i < words; i += kSelThreads) row_any[i] = 0;
    if (tid == 0) {
        s_found = 0;
        s_pos = st->scan_pos;
    }
    __syncthreads();

    // 2. next S uncovered ids in index order (bitmap scan, 1024 words per round)
    while (true) {
        const int found = s_found;
        const long long pos = s_pos;
        if (found >= S || pos >= n) break;
        const long long w0 = pos >> 5;
        const long long w = w0 + tid;
        unsigned bits = 0;
        if (w * 32 < n) {
            bits = ~covered[w];
            if (w == w0) bits &= 0xffffffffu << (pos & 31);
            const long long rem = n - w * 32;
            if (rem < 32) bits &= (1u << rem) - 1u;
        }
        int total;
        const int excl = block_exclusive_scan(__popc(bits), s_scan, total);
        int slot = found + excl;
        while (bits && slot < S) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            cand_ids[slot++] = (int)(w * 32 + b);
        }
        __syncthreads();
        if (tid == 0) {
            const int nf = found + total;
            if (nf >= S) {
                s_found = S;
                s_pos = (long long)cand_ids[S - 1] + 1;
            } else {
                s_found = nf;
                s_pos = (w0 + kSelThreads) * 32;
            }
        }
        __syncthreads();
    }
    const int found = s_found;
    if (tid == 0) {
        st->cand_count = found;
        st->scan_pos = s_pos < n ? s_pos : n;
        st->step_hits = 0;
        st->candidates += (unsigned long long)found;
        if (found == 0) st->done = 1;
        else st->steps += 1;
    }
    // 3. register the candidates and gather their rows
    for (int s = tid; s < found; s += kSelThreads) slot_of[cand_ids[s]] = s;
    for (long long e = tid; e < (long long)found * d; e += kSelThreads) {
        const int s = (int)(e / d), i = (int)(e % d);
        cand_x[e] = X[(long long)cand_ids[s] * d + i];
    }
    for (int s = tid; s < found; s += kSelThreads) cand_phi[s] = phi[cand_ids[s]];
    if (want_tc) {
        for (long long e = tid; e < (long long)found * d_pad; e += kSelThreads) {
            const int s = (int)(e / d_pad), i = (int)(e % d_pad);
            const long long src = (long long)cand_ids[s] * d_pad + i;
            cH[e] = H[src];
            cLo[e] = Lo[src];
        }
        // A-side augmentation = B-side row with its halves [0,3) and [3,6) swapped
        for (long long e = tid; e < (long long)found * 16; e += kSelThreads) {
            const int s = (int)(e >> 4), i = (int)(e & 15);
            const int src = i < 3 ? i + 3 : (i < 6 ? i - 3 : i);
            cAug[e] = Aug[(long long)cand_ids[s] * 16 + src];
        }
    }
}

// One warp.  Rows of the conflict matrix that hold any bit were flagged in
// row_any by the sweep; they are staged in shared memory first, then walked
// in index order.  Candidate k is a landmark iff no earlier landmark
// candidate covers it (its bit is clear in the running 'killed' set).
__global__ void __launch_bounds__(256) greedy_resolve_kernel(DeviceState* st, const unsigned* conflict,
                                                             const unsigned* row_any, int words,
                                                             const int* cand_ids, int* ordinal,
                                                             int* landmarks) {
    if (st->done) return;
    extern __shared__ unsigned s_rows[];   // S x words
    const int c = st->cand_count;
    const int tid = threadIdx.x, lane = tid & 31;
    // stage flagged rows
    for (int e = tid; e < c * words; e += blockDim.x) {
        const int k = e / words;
        s_rows[e] = ((row_any[k >> 5] >> (k & 31)) & 1u) ? conflict[e] : 0u;
    }
    __syncthreads();
    if (tid >= 32) return;
    unsigned killed = 0;  // lane owns word 'lane' of the killed set
    for (int w = 0; w < words; ++w) {
        unsigned m = row_any[w];
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const int k = w * 32 + b;
            if (k >= c) break;
            const unsigned kw = __shfl_sync(kFull, killed, w);
            if ((kw >> b) & 1u) continue;
            if (lane < words) killed |= s_rows[k * words + lane];
        }
    }
    // alive = not killed; ordinals by prefix count in slot order
    const int base = st->n_landmarks;
    int running = 0;
    for (int w = 0; w < words; ++w) {
        const unsigned kw = __shfl_sync(kFull, killed, w);
        unsigned valid = (w * 32 + 32 <= c) ? kFull : (w * 32 >= c ? 0u : ((1u << (c - w * 32)) - 1u));
        const unsigned alive = ~kw & valid;
        const int k = w * 32 + lane;
        if (k < c) {
            const bool a = (alive >> lane) & 1u;
            const int rank = running + __popc(alive & ((1u << lane) - 1u));
            ordinal[k] = a ? base + rank : -1;
            if (a) landmarks[base + rank] = cand_ids[k];
        }
        running += __popc(alive);
    }
    if (lane == 0) st->n_landmarks = base + running;
}

__global__ void __launch_bounds__(256) greedy_apply_kernel(DeviceState* st, const unsigned long long* step_keys,
                                                           unsigned long long step_cap, const int* ordinal,
                                                           unsigned* covered, unsigned long long* mem_keys,
                                                           unsigned long long mem_cap) {
    if (st->done) return;
    const unsigned long long cnt = st->step_hits;
    if (cnt > step_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            atomicOr(&st->error, kErrStepOverflow);
            st->done = 1;
        }
        return;
    }
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    // loop bound rounded to whole warps so that every lane reaches warp_reserve
    for (unsigned long long i0 = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         i0 < cnt; i0 += stride) {
        const unsigned long long i = i0 + lane_id();
        unsigned long long key = 0;
        int ord = -1;
        if (i < cnt) {
            key = step_keys[i];
            ord = ordinal[key >> 32];
        }
        const unsigned pt = (unsigned)(key & 0xffffffffull);
        if (ord >= 0) atomicOr(&covered[pt >> 5], 1u << (pt & 31));
        unsigned long long pos = warp_reserve(&st->mem_count, ord >= 0 ? 1u : 0u);
        if (ord >= 0) {
            if (pos < mem_cap) mem_keys[pos] = ((unsigned long long)(unsigned)ord << 32) | pt;
            else atomicOr(&st->error, kErrMemberOverflow);
        }
    }
}

}  // namespace

cudaError_t launch_greedy_select(const GreedyBuffers& g, const Prepared& pts, int S, bool want_tc,
                                 cudaStream_t s) {
    const int words = S / 32;
    note_launch();
    greedy_select_kernel<<<1, kSelThreads, 0, s>>>(
        g.st, g.covered, pts.rows, S, g.slot_of, g.cand_ids, g.conflict, g.row_any, words, pts.x, pts.phi,
        pts.d, const_cast<float*>(g.cand.x), g.cand.phi, want_tc ? 1 : 0,
        pts.hi, pts.lo, pts.aug, pts.d_pad, g.cand.hi, g.cand.lo, g.cand.aug);
    return cudaGetLastError();
}

cudaError_t launch_greedy_resolve(const GreedyBuffers& g, int S, cudaStream_t s) {
    const int words = S / 32;
    const size_t smem = (size_t)S * words * sizeof(unsigned);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(greedy_resolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             32 * 1024 * 4);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    note_launch();
    greedy_resolve_kernel<<<1, 256, smem, s>>>(g.st, g.conflict, g.row_any, words, g.cand_ids, g.ordinal,
                                               g.landmarks);
    return cudaGetLastError();
}

cudaError_t launch_greedy_apply(const GreedyBuffers& g, cudaStream_t s) {
    note_launch();
    greedy_apply_kernel<<<152 * 8, 256, 0, s>>>(g.st, g.step_keys, g.step_cap, g.ordinal, g.covered, g.mem_keys,
                                                 g.mem_cap);
    return cudaGetLastError();
}

}  // namespace bm
