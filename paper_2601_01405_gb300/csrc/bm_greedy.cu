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
    DeviceState* st, const unsigned* __restrict__ covered, long long n, int S, int* __restrict__ slot_of,
    int* __restrict__ cand_ids, unsigned* __restrict__ conflict, unsigned* __restrict__ row_any, int words,
    const float* __restrict__ X,
    const float* __restrict__ phi, int d, float* cand_x, float* cand_phi, int want_tc,
    const __nv_bfloat16* __restrict__ H, const __nv_bfloat16* __restrict__ Lo,
    const __nv_bfloat16* __restrict__ Aug, int d_pad, __nv_bfloat16* cH, __nv_bfloat16* cLo,
    __nv_bfloat16* cAug) {
    pdl_wait();
    pdl_trigger();
    if (st->done) return;
    if (st->error & kErrTimeout) {  // a bounded wait expired in a previous step: stop the loop
        if (threadIdx.x == 0) st->done = 1;
        return;
    }
    __shared__ int s_scan[33];
    __shared__ int s_found;
    __shared__ long long s_pos;
    const int tid = threadIdx.x;

    // 1. undo the previous step's bookkeeping: conflict bits live only in the rows
    //    flagged in row_any and in their first ceil(prev / 32) words (columns are
    //    candidate slots), so only those are cleared
    const int prev = st->cand_count;
    const int prev_words = (prev + 31) >> 5;
#pragma unroll 4
    for (int i = tid; i < prev; i += kSelThreads) slot_of[cand_ids[i]] = -1;
#pragma unroll 4
    for (int k = tid; k < prev; k += kSelThreads)
        if ((row_any[k >> 5] >> (k & 31)) & 1u)
            for (int w = 0; w < prev_words; ++w) conflict[(size_t)k * words + w] = 0;
    __syncthreads();
    for (int i = tid; i < words; i += kSelThreads) row_any[i] = 0;
    __shared__ int s_req;
    if (tid == 0) {
        s_found = 0;
        s_pos = st->scan_pos;
        st->step_start_pos = st->scan_pos;   // lets the host redo this step with larger buffers
        int req = st->s_next;
        req = req < 32 ? 32 : (req > S ? S : req);
        s_req = req;
        st->s_cur = req;
    }
    __syncthreads();
    S = s_req;   // this step's batch: adapted between 32 and the buffer size

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
        while (bits && slot < S) {   // 3. register each candidate as it is found
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int id = (int)(w * 32 + b);
            cand_ids[slot] = id;
            slot_of[id] = slot;
            ++slot;
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
        st->band_n = 0;
        st->candidates += (unsigned long long)found;
        if (found == 0) st->done = 1;
        else st->steps += 1;
    }
    // (the candidates' rows are gathered by greedy_gather_kernel)
}

// One warp per candidate: copy its float32 row, phi and, for the tensor-core
// paths, its 16-bit operand rows (bf16 hi and lo, or fp16 hi alone) and A-side
// augmentation (the B-side row with the halves [0,3) and [3,6) swapped and the point's
// own delta'_row in column 6) into
// the contiguous candidate operands.
__global__ void __launch_bounds__(256) greedy_gather_kernel(
    const DeviceState* st, const int* __restrict__ cand_ids, const float* __restrict__ X,
    const float* __restrict__ phi, int d, float* __restrict__ cand_x, float* __restrict__ cand_phi, int want_tc,
    const unsigned* __restrict__ H, const unsigned* __restrict__ Lo, const unsigned short* __restrict__ Aug,
    int d_pad, unsigned* __restrict__ cH, unsigned* __restrict__ cLo, unsigned short* __restrict__ cAug) {
    pdl_wait();
    pdl_trigger();
    if (st->done) return;
    const int s = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (s >= st->cand_count) return;
    const long long id = cand_ids[s];
    for (int i = lane; i < d; i += 32) cand_x[(long long)s * d + i] = X[id * d + i];
    if (lane == 0) cand_phi[s] = phi[id];
    if (want_tc) {
        const int w = d_pad / 2;  // bf16 pairs per row
        for (int i = lane; i < w; i += 32) {
            cH[(long long)s * w + i] = H[id * w + i];
            if (Lo) cLo[(long long)s * w + i] = Lo[id * w + i];   // no lo half in fp16 mode
        }
        if (lane < 16) {
            // A-side layout from the point's B-side block: the halves [0,3) and [3,6) swapped,
            // column 6 = the point's own +delta'_row (its column 7) against the points' 1,
            // column 7 = 0
            const int src = lane < 3 ? lane + 3 : (lane < 6 ? lane - 3 : (lane == 6 ? 7 : lane));
            cAug[(long long)s * 16 + lane] = lane == 7 ? (unsigned short)0 : Aug[id * 16 + src];
        }
    }
}

// Rows of the conflict matrix that hold any bit were flagged in row_any by
// the sweep; flagged rows are staged in shared memory (as many as fit; the rest
// are read from global memory).  One warp then walks the flagged candidates in
// index order: candidate k is a landmark iff no earlier landmark candidate
// covers it (its bit is clear in the running 'killed' set, up to 16 words per
// lane: word lane + 32 h, as many as this step's batch needs).  Finally every thread assigns ordinals in parallel,
// and the next step's batch size follows the survival rate (fewer wasted
// candidate rows on dense data, larger batches where balls are small).
constexpr int kMaxWords = 512;   // batches of up to 16384 candidates

// Warp 0 of the resolve: the flagged rows (a bit in row_any among the first c slots) in
// index order into s_flag_row; returns their count.  H: words per lane, cw <= 32 H, so the
// loops cover only the words this step's batch can use.
template <int H>
__device__ __forceinline__ int resolve_flags(const unsigned* row_any, int words, int c, int* s_flag_row, int lane) {
    int base = 0;
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int w = lane + 32 * h;
        unsigned a = w < words ? row_any[w] : 0u;
        if (w * 32 >= c) a = 0u;
        else if (w * 32 + 32 > c) a &= (1u << (c - w * 32)) - 1u;
        const int cnt = __popc(a);
        int x = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        const int first = base + x - cnt;
        unsigned m = a;
        int k = first;
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            s_flag_row[k++] = w * 32 + b;
        }
        base += __shfl_sync(kFull, x, 31);
    }
    return base;
}

// Warp 0 of the resolve: walk the flagged candidates in index order with the running
// 'killed' set (word lane + 32 h in killed[h]), then the alive words and the alive count
// before each word; returns the number of landmarks.
template <int H>
__device__ __forceinline__ int resolve_walk(const unsigned* conflict, int words, int c, int cw,
                                            const int* s_flag_row, int nflag, const unsigned* s_rows, int staged,
                                            unsigned* s_alive, int* s_rank_of_word, int lane) {
    unsigned killed[H];
#pragma unroll
    for (int h = 0; h < H; ++h) killed[h] = 0u;
    for (int f = 0; f < nflag; ++f) {
        const int k = s_flag_row[f], w = k >> 5;
        unsigned mine = killed[0];   // this lane's copy of word (w mod 32) + 32 h, h = w / 32
#pragma unroll
        for (int h = 1; h < H; ++h)
            if ((w >> 5) == h) mine = killed[h];
        const unsigned kw = __shfl_sync(kFull, mine, w & 31);
        if ((kw >> (k & 31)) & 1u) continue;
        const unsigned* row = f < staged ? s_rows + (size_t)f * cw : conflict + (size_t)k * words;
#pragma unroll
        for (int h = 0; h < H; ++h)
            if (lane + 32 * h < cw) killed[h] |= row[lane + 32 * h];
    }
    int base = 0;
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int w = lane + 32 * h;
        const unsigned valid = (w * 32 + 32 <= c) ? kFull : (w * 32 >= c ? 0u : ((1u << (c - w * 32)) - 1u));
        const unsigned alive = ~killed[h] & valid;
        s_alive[w] = alive;
        const int cnt = __popc(alive);
        int x = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        s_rank_of_word[w] = base + x - cnt;   // alive count before word w
        base += __shfl_sync(kFull, x, 31);
    }
    return base;
}

// Dynamic shared memory: the flagged row ids (s_max ints), then the staged rows
// (stage_words words).
__global__ void __launch_bounds__(1024) greedy_resolve_kernel(DeviceState* st, const unsigned* conflict,
                                                             const unsigned* row_any, int words,
                                                             const int* __restrict__ cand_ids,
                                                             int* __restrict__ ordinal,
                                                             int* __restrict__ landmarks, unsigned long long mem_cap,
                                                             int stage_words, int s_max) {
    pdl_wait();
    pdl_trigger();
    if (st->done) return;
    // the new memberships are a subset of this step's hits: stop before anything
    // is committed if they might not fit (the host grows the buffer and redoes the step)
    if (st->mem_count + st->step_hits > mem_cap) {
        if (threadIdx.x == 0) {
            atomicOr(&st->error, kErrMemberOverflow);
            st->done = 1;
        }
        return;
    }
    extern __shared__ unsigned s_dyn[];
    int* s_flag_row = reinterpret_cast<int*>(s_dyn);   // flagged rows in index order (at most s_max)
    unsigned* s_rows = s_dyn + s_max;                  // staged flagged rows, cw words each
    __shared__ int s_rank_of_word[kMaxWords + 1];
    __shared__ unsigned s_alive[kMaxWords];
    __shared__ int s_nflag;
    const int c = st->cand_count;
    const int cw = (c + 31) >> 5;   // words of a conflict row that can hold bits (slots < c)
    const int H = cw <= 32 ? 1 : cw <= 64 ? 2 : cw <= 128 ? 4 : cw <= 256 ? 8 : 16;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        int nf;
        switch (H) {
            case 1: nf = resolve_flags<1>(row_any, words, c, s_flag_row, lane); break;
            case 2: nf = resolve_flags<2>(row_any, words, c, s_flag_row, lane); break;
            case 4: nf = resolve_flags<4>(row_any, words, c, s_flag_row, lane); break;
            case 8: nf = resolve_flags<8>(row_any, words, c, s_flag_row, lane); break;
            default: nf = resolve_flags<16>(row_any, words, c, s_flag_row, lane); break;
        }
        if (lane == 0) s_nflag = nf;
    }
    __syncthreads();
    const int nflag = s_nflag;
    const int stage_rows = cw > 0 ? stage_words / cw : 0;
    const int staged = nflag < stage_rows ? nflag : stage_rows;
    for (int e = tid; e < staged * cw; e += blockDim.x) {
        const int f = e / cw, wi = e - f * cw;
        s_rows[e] = conflict[(size_t)s_flag_row[f] * words + wi];
    }
    __syncthreads();
    if (tid < 32) {
        int alive;
        switch (H) {
            case 1: alive = resolve_walk<1>(conflict, words, c, cw, s_flag_row, nflag, s_rows, staged, s_alive,
                                            s_rank_of_word, lane); break;
            case 2: alive = resolve_walk<2>(conflict, words, c, cw, s_flag_row, nflag, s_rows, staged, s_alive,
                                            s_rank_of_word, lane); break;
            case 4: alive = resolve_walk<4>(conflict, words, c, cw, s_flag_row, nflag, s_rows, staged, s_alive,
                                            s_rank_of_word, lane); break;
            case 8: alive = resolve_walk<8>(conflict, words, c, cw, s_flag_row, nflag, s_rows, staged, s_alive,
                                            s_rank_of_word, lane); break;
            default: alive = resolve_walk<16>(conflict, words, c, cw, s_flag_row, nflag, s_rows, staged, s_alive,
                                              s_rank_of_word, lane); break;
        }
        if (lane == 0) s_rank_of_word[kMaxWords] = alive;
    }
    __syncthreads();
    const int base_l = st->n_landmarks;
#pragma unroll 4
    for (int k = tid; k < c; k += blockDim.x) {   // the candidate id loads of four rounds in flight
        const int id = cand_ids[k];
        const unsigned aw = s_alive[k >> 5];
        const bool a = (aw >> (k & 31)) & 1u;
        const int rank = s_rank_of_word[k >> 5] + __popc(aw & ((1u << (k & 31)) - 1u));
        ordinal[k] = a ? base_l + rank : -1;
        if (a) landmarks[base_l + rank] = id;
    }
    __syncthreads();
    if (tid == 0) {
        const int alive = s_rank_of_word[kMaxWords];
        st->n_landmarks = base_l + alive;
        // next batch: double while at least 90 % of a full batch survives (99 % past
        // 2048 candidates, 99.5 % past 4096: past 2048 a wasted row costs more than
        // the per-step work that doubling saves), halve below 50 % (90 % past 2048)
        const int cur = st->s_cur;
        int nxt = cur;
        const bool grow = cur < 2048 ? 10 * alive >= 9 * c : (cur < 4096 ? 100 * alive >= 99 * c
                                                                          : 1000 * alive >= 995 * c);
        if (c == cur && grow) nxt = cur * 2;
        else if (2 * alive < c || (cur > 2048 && 10 * alive < 9 * c)) nxt = cur / 2;
        nxt = nxt < 32 ? 32 : (nxt > s_max ? s_max : nxt);
        st->s_next = nxt;
    }
}

__global__ void __launch_bounds__(256) greedy_apply_kernel(DeviceState* st, const unsigned long long* step_keys,
                                                           unsigned long long step_cap, const int* ordinal,
                                                           unsigned* covered, unsigned long long* mem_keys,
                                                           unsigned long long mem_cap) {
    pdl_wait();
    pdl_trigger();
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
    return launch_pdl(greedy_select_kernel, dim3(1), dim3(kSelThreads), 0, s,
        g.st, (const unsigned*)g.covered, pts.rows, S, g.slot_of, g.cand_ids, g.conflict, g.row_any, words,
        (const float*)pts.x, (const float*)pts.phi, pts.d, const_cast<float*>(g.cand.x), g.cand.phi, want_tc ? 1 : 0,
        (const __nv_bfloat16*)pts.hi, (const __nv_bfloat16*)pts.lo, (const __nv_bfloat16*)pts.aug, pts.d_pad,
        g.cand.hi, g.cand.lo, g.cand.aug);
}

// Undo the bookkeeping of a step stopped by a buffer overflow so that the next
// select kernel picks the same candidates again.
__global__ void greedy_rollback_kernel(DeviceState* st) {
    st->scan_pos = st->step_start_pos;
    st->steps -= 1;
    st->candidates -= (unsigned long long)st->cand_count;
    st->done = 0;
    st->error = 0;
    st->max_seg = 0;
    st->step_hits = 0;
    st->band_n = 0;
}

cudaError_t launch_greedy_rollback(const GreedyBuffers& g, cudaStream_t s) {
    note_launch();
    greedy_rollback_kernel<<<1, 1, 0, s>>>(g.st);
    return cudaGetLastError();
}

cudaError_t launch_greedy_gather(const GreedyBuffers& g, const Prepared& pts, int S, bool want_tc, cudaStream_t s) {
    note_launch();
    return launch_pdl(greedy_gather_kernel, dim3((S + 7) / 8), dim3(256), 0, s,
        (const DeviceState*)g.st, (const int*)g.cand_ids, (const float*)pts.x, (const float*)pts.phi, pts.d,
        const_cast<float*>(g.cand.x), g.cand.phi, want_tc ? 1 : 0,
        reinterpret_cast<const unsigned*>(pts.hi), reinterpret_cast<const unsigned*>(pts.lo),
        reinterpret_cast<const unsigned short*>(pts.aug), pts.d_pad, reinterpret_cast<unsigned*>(g.cand.hi),
        reinterpret_cast<unsigned*>(g.cand.lo), reinterpret_cast<unsigned short*>(g.cand.aug));
}

cudaError_t launch_greedy_resolve(const GreedyBuffers& g, int S, cudaStream_t s) {
    if (S > kMaxWords * 32) return cudaErrorInvalidValue;
    const int words = S / 32;
    constexpr size_t kStageBytes = 128 * 1024;
    constexpr size_t kMaxSmem = kStageBytes + sizeof(int) * kMaxWords * 32;
    const size_t full = (size_t)S * words * sizeof(unsigned);   // every row of the largest batch
    const size_t stage = full < kStageBytes ? full : kStageBytes;
    const size_t smem = sizeof(int) * (size_t)S + stage;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(greedy_resolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kMaxSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    note_launch();
    return launch_pdl(greedy_resolve_kernel, dim3(1), dim3(1024), smem, s, g.st, (const unsigned*)g.conflict,
                      (const unsigned*)g.row_any, words, (const int*)g.cand_ids, g.ordinal, g.landmarks, g.mem_cap,
                      (int)(stage / sizeof(unsigned)), S);
}

// Loop condition of a greedy build run as a graph WHILE node: another step while
// points remain uncovered and no step stopped on an error (an overflowing step
// sets done as well, and the host resumes the build with larger buffers).
// Every step with a candidate makes at least one landmark, so n + 1 iterations
// always suffice; past max_iterations the loop stops with kErrLoopLimit.
__global__ void greedy_continue_kernel(DeviceState* st, cudaGraphConditionalHandle h, unsigned* iterations,
                                       unsigned max_iterations) {
    const unsigned it = ++*iterations;
    unsigned go = (st->done || st->error) ? 0u : 1u;
    if (go && it >= max_iterations) {
        st->error |= kErrLoopLimit;
        st->done = 1;
        go = 0u;
    }
    cudaGraphSetConditional(h, go);
}

cudaError_t launch_greedy_continue(const GreedyBuffers& g, cudaGraphConditionalHandle h, unsigned* iterations,
                                   unsigned max_iterations, cudaStream_t s) {
    note_launch();
    greedy_continue_kernel<<<1, 1, 0, s>>>(g.st, h, iterations, max_iterations);
    return cudaGetLastError();
}

cudaError_t launch_greedy_apply(const GreedyBuffers& g, cudaStream_t s) {
    note_launch();
    return launch_pdl(greedy_apply_kernel, dim3(152 * 8), dim3(256), 0, s, g.st,
                      (const unsigned long long*)g.step_keys, g.step_cap, (const int*)g.ordinal, g.covered,
                      g.mem_keys, g.mem_cap);
}

}  // namespace bm
