// bm_tile_tc_kernel.cuh -- the tcgen05 distance-tile kernel and its launch templates,
// shared by bm_tile_tc.cu (dense sweeps) and bm_tile_tc_table.cu (table mode, the
// inverted-file scan), which instantiate the two modes in separate translation units.
//
//
// Decision rule (open ball, Sec. 2.1; exact range set, Sec. 5, Def. 5.1): x is in
// R_eps(q) iff D(q,x) < eps^2.  Following the algebraic decomposition of
// Sec. 3.2 the tile evaluates, for 128 query rows x NT points,
//     v = q.x - phi_q - phi_x = (eps^2 - D)/2,      phi = ||.||^2/2 - eps^2/4
// as one FP32 accumulation in tensor memory:
//     q.x ~ hi_q.hi_x + lo_q.hi_x + hi_q.lo_x      (bf16 split products, exact in FP32)
//     - phi_q - phi_x + delta'_q                   (the 16-wide augmentation block)
// with delta'_q the query row's own proven error bound (rounded up), so that pairs with
// v > delta'_q are members, v < -delta'_q are not, and the band in between is listed for
// the FP64 recheck kernel (verified range set, Sec. 5.3).
//
// Kernel organisation (one CTA per SM, persistent over work items):
//   warp 0  TMA producer: one point tile (B, NT rows x all K) per work item,
//           then the K chunks of up to 16 query tiles (A, 128 rows each)
//           through a ring of shared-memory stages
//   warp 1  allocates tensor memory; lane 0 issues tcgen05.mma (M=128, N=NT,
//           K=16 per instruction) into one of two TMEM accumulators
//   warp 10 for one-stage query tiles (fp16), a second issuer: warps 1 and 10 take
//           alternate tiles, each with its own accumulator, so one thread's barrier
//           work per tile overlaps the other's MMAs
//   warps 2-9  epilogue: tcgen05.ld of the accumulator (one TMEM lane = one
//           query row per thread; two warps per lane quarter, each on half of
//           the columns, all loads in flight before one wait), classification
//           and warp-aggregated emission of hits and band pairs
// Every mbarrier wait is bounded in time; on expiry the kernel records
// kErrTimeout, drains its in-flight copies and MMAs, frees TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <string>

#include "bm_host.h"

namespace bm {
namespace tc {


constexpr int kThreads = 352;   // producer, MMA issuer, 8 epilogue warps, second MMA issuer
constexpr int kIssuer2 = kThreads / 32 - 1;   // the second MMA-issuing warp
constexpr int kEpiWarps = 8;
constexpr int kMaxGroup = 16;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s
constexpr unsigned long long kDrainNs = 200000000ull;  // 0.2 s

struct TcArgs {
    CUtensorMap a_hi, a_lo, a_aug, b_hi, b_lo, b_aug;
    const float* ax;      // query rows, float32 (band recheck)
    const float* bx;      // points, float32 (band recheck)
    long long a_rows_max;
    const int* a_rows_dev;
    long long n;
    int d;
    int d_pad;
    int check_done;
    int pad0;
    double eps2;
    DeviceState* st;
    HitSink sink;
    // table mode (inverted-file scan): work items from a device table; A row r holds the
    // query a_map[r], B column c of an item is point b_ids[src0 + c - b_col0]
    const TcItem* items;
    const long long* items_count;
    const int* a_map;
    const int* b_ids;
    // the A operand's augmentation rows (16 entries each): column 6 holds each row's +delta'
    const unsigned short* a_aug_rows;
};

struct Ctl {
    unsigned long long b_full[2], b_empty[2];
    unsigned long long a_full[16], a_empty[16];
    unsigned long long t_full[2], t_empty[2];
    unsigned long long drain;
    unsigned tmem_base;
    int abort_flag;
    unsigned seg_used;   // hits appended by this CTA (segmented mode)
    unsigned band_used;  // band pairs appended by this CTA (segmented mode)
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait.  Returns false when the CTA is aborting or the bound expired.
__device__ __forceinline__ bool bar_wait_at(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* gerr) {
    if (bar_try(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (true) {
        if (bar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            atomicOr(gerr, kErrTimeout);
            return false;
        }
    }
}

__device__ __forceinline__ bool bar_wait(unsigned long long* b, uint32_t parity, volatile int* abort_flag,
                                         int* gerr) {
    return bar_wait_at(su32(b), parity, abort_flag, gerr);
}

// Bounded wait used while draining; ignores the abort flag.
__device__ __forceinline__ void bar_drain(unsigned long long* b, uint32_t parity) {
    const uint32_t bar = su32(b);
    const unsigned long long t0 = gtimer();
    while (!bar_try(bar, parity) && gtimer() - t0 < kDrainNs) {
    }
}

__device__ __forceinline__ void bar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(unsigned long long* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, unsigned long long* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// Shared-memory matrix descriptor (tcgen05): K-major operand with a swizzle
// atom of 8 rows x `span` bytes; atoms are stacked every 8*span bytes.
__device__ __forceinline__ unsigned long long sdesc(uint32_t addr, uint32_t span) {
    const uint32_t layout = span == 128 ? 2u : (span == 64 ? 4u : 6u);  // SW128 / SW64 / SW32
    return (unsigned long long)((addr & 0x3FFFFu) >> 4) | (1ull << 16) |
           ((unsigned long long)((8u * span) >> 4) << 32) | (1ull << 46) | ((unsigned long long)layout << 61);
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16 (or both F16), both K-major.
__host__ __device__ constexpr uint32_t idesc_f16kind(int M, int N, bool bf16) {
    return (1u << 4) | (bf16 ? (1u << 7) | (1u << 10) : 0u) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, unsigned long long a, unsigned long long b, uint32_t idesc,
                                    uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit_at(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) { mma_commit_at(su32(bar)); }

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// All of a warp's 32-column TMEM loads for one tile and the wait for them in one asm
// statement.  The destination registers of tcgen05.ld hold the data only after
// tcgen05.wait::ld; as separate statements the compiler would be free to move or spill
// them in between (saving values that have not landed), so loads and wait stay fused.
// The loads are the reducing form (.red.max): m[c] is the largest of the 32 values of
// chunk c in this thread's row, so a row's "all negative" test is m[c] < 0 with no
// per-element work.
template <int K>
__device__ __forceinline__ void tmem_ld_all(uint32_t taddr, uint32_t (&r)[K][32], float (&m)[K]);

template <>
__device__ __forceinline__ void tmem_ld_all<1>(uint32_t taddr, uint32_t (&r)[1][32], float (&m)[1]) {
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %32, [%33];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]), "=r"(r[0][6]), "=r"(r[0][7]), "=r"(r[0][8]), "=r"(r[0][9]), "=r"(r[0][10]), "=r"(r[0][11]), "=r"(r[0][12]), "=r"(r[0][13]), "=r"(r[0][14]), "=r"(r[0][15]), "=r"(r[0][16]), "=r"(r[0][17]), "=r"(r[0][18]), "=r"(r[0][19]), "=r"(r[0][20]), "=r"(r[0][21]), "=r"(r[0][22]), "=r"(r[0][23]), "=r"(r[0][24]), "=r"(r[0][25]), "=r"(r[0][26]), "=r"(r[0][27]), "=r"(r[0][28]), "=r"(r[0][29]), "=r"(r[0][30]), "=r"(r[0][31]),
          "=f"(m[0])
        : "r"(taddr + 0u)
        : "memory");
}

template <>
__device__ __forceinline__ void tmem_ld_all<2>(uint32_t taddr, uint32_t (&r)[2][32], float (&m)[2]) {
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %64, [%66];\n"
        "tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, %65, [%67];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]), "=r"(r[0][6]), "=r"(r[0][7]), "=r"(r[0][8]), "=r"(r[0][9]), "=r"(r[0][10]), "=r"(r[0][11]), "=r"(r[0][12]), "=r"(r[0][13]), "=r"(r[0][14]), "=r"(r[0][15]), "=r"(r[0][16]), "=r"(r[0][17]), "=r"(r[0][18]), "=r"(r[0][19]), "=r"(r[0][20]), "=r"(r[0][21]), "=r"(r[0][22]), "=r"(r[0][23]), "=r"(r[0][24]), "=r"(r[0][25]), "=r"(r[0][26]), "=r"(r[0][27]), "=r"(r[0][28]), "=r"(r[0][29]), "=r"(r[0][30]), "=r"(r[0][31]),
          "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]), "=r"(r[1][3]), "=r"(r[1][4]), "=r"(r[1][5]), "=r"(r[1][6]), "=r"(r[1][7]), "=r"(r[1][8]), "=r"(r[1][9]), "=r"(r[1][10]), "=r"(r[1][11]), "=r"(r[1][12]), "=r"(r[1][13]), "=r"(r[1][14]), "=r"(r[1][15]), "=r"(r[1][16]), "=r"(r[1][17]), "=r"(r[1][18]), "=r"(r[1][19]), "=r"(r[1][20]), "=r"(r[1][21]), "=r"(r[1][22]), "=r"(r[1][23]), "=r"(r[1][24]), "=r"(r[1][25]), "=r"(r[1][26]), "=r"(r[1][27]), "=r"(r[1][28]), "=r"(r[1][29]), "=r"(r[1][30]), "=r"(r[1][31]),
          "=f"(m[0]), "=f"(m[1])
        : "r"(taddr + 0u), "r"(taddr + 32u)
        : "memory");
}

template <>
__device__ __forceinline__ void tmem_ld_all<4>(uint32_t taddr, uint32_t (&r)[4][32], float (&m)[4]) {
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %128, [%132];\n"
        "tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, %129, [%133];\n"
        "tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 {%64,%65,%66,%67,%68,%69,%70,%71,%72,%73,%74,%75,%76,%77,%78,%79,%80,%81,%82,%83,%84,%85,%86,%87,%88,%89,%90,%91,%92,%93,%94,%95}, %130, [%134];\n"
        "tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 {%96,%97,%98,%99,%100,%101,%102,%103,%104,%105,%106,%107,%108,%109,%110,%111,%112,%113,%114,%115,%116,%117,%118,%119,%120,%121,%122,%123,%124,%125,%126,%127}, %131, [%135];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0][0]), "=r"(r[0][1]), "=r"(r[0][2]), "=r"(r[0][3]), "=r"(r[0][4]), "=r"(r[0][5]), "=r"(r[0][6]), "=r"(r[0][7]), "=r"(r[0][8]), "=r"(r[0][9]), "=r"(r[0][10]), "=r"(r[0][11]), "=r"(r[0][12]), "=r"(r[0][13]), "=r"(r[0][14]), "=r"(r[0][15]), "=r"(r[0][16]), "=r"(r[0][17]), "=r"(r[0][18]), "=r"(r[0][19]), "=r"(r[0][20]), "=r"(r[0][21]), "=r"(r[0][22]), "=r"(r[0][23]), "=r"(r[0][24]), "=r"(r[0][25]), "=r"(r[0][26]), "=r"(r[0][27]), "=r"(r[0][28]), "=r"(r[0][29]), "=r"(r[0][30]), "=r"(r[0][31]),
          "=r"(r[1][0]), "=r"(r[1][1]), "=r"(r[1][2]), "=r"(r[1][3]), "=r"(r[1][4]), "=r"(r[1][5]), "=r"(r[1][6]), "=r"(r[1][7]), "=r"(r[1][8]), "=r"(r[1][9]), "=r"(r[1][10]), "=r"(r[1][11]), "=r"(r[1][12]), "=r"(r[1][13]), "=r"(r[1][14]), "=r"(r[1][15]), "=r"(r[1][16]), "=r"(r[1][17]), "=r"(r[1][18]), "=r"(r[1][19]), "=r"(r[1][20]), "=r"(r[1][21]), "=r"(r[1][22]), "=r"(r[1][23]), "=r"(r[1][24]), "=r"(r[1][25]), "=r"(r[1][26]), "=r"(r[1][27]), "=r"(r[1][28]), "=r"(r[1][29]), "=r"(r[1][30]), "=r"(r[1][31]),
          "=r"(r[2][0]), "=r"(r[2][1]), "=r"(r[2][2]), "=r"(r[2][3]), "=r"(r[2][4]), "=r"(r[2][5]), "=r"(r[2][6]), "=r"(r[2][7]), "=r"(r[2][8]), "=r"(r[2][9]), "=r"(r[2][10]), "=r"(r[2][11]), "=r"(r[2][12]), "=r"(r[2][13]), "=r"(r[2][14]), "=r"(r[2][15]), "=r"(r[2][16]), "=r"(r[2][17]), "=r"(r[2][18]), "=r"(r[2][19]), "=r"(r[2][20]), "=r"(r[2][21]), "=r"(r[2][22]), "=r"(r[2][23]), "=r"(r[2][24]), "=r"(r[2][25]), "=r"(r[2][26]), "=r"(r[2][27]), "=r"(r[2][28]), "=r"(r[2][29]), "=r"(r[2][30]), "=r"(r[2][31]),
          "=r"(r[3][0]), "=r"(r[3][1]), "=r"(r[3][2]), "=r"(r[3][3]), "=r"(r[3][4]), "=r"(r[3][5]), "=r"(r[3][6]), "=r"(r[3][7]), "=r"(r[3][8]), "=r"(r[3][9]), "=r"(r[3][10]), "=r"(r[3][11]), "=r"(r[3][12]), "=r"(r[3][13]), "=r"(r[3][14]), "=r"(r[3][15]), "=r"(r[3][16]), "=r"(r[3][17]), "=r"(r[3][18]), "=r"(r[3][19]), "=r"(r[3][20]), "=r"(r[3][21]), "=r"(r[3][22]), "=r"(r[3][23]), "=r"(r[3][24]), "=r"(r[3][25]), "=r"(r[3][26]), "=r"(r[3][27]), "=r"(r[3][28]), "=r"(r[3][29]), "=r"(r[3][30]), "=r"(r[3][31]),
          "=f"(m[0]), "=f"(m[1]), "=f"(m[2]), "=f"(m[3])
        : "r"(taddr + 0u), "r"(taddr + 32u), "r"(taddr + 64u), "r"(taddr + 96u)
        : "memory");
}


// Byte sizes of the shared-memory regions for a configuration.  PROD = 3: the
// point tile holds hi and lo chunks (bf16 split); PROD = 1: hi chunks only (fp16).
struct Layout {
    int CK, NT, BBUF, ASTG, nc, cps;
    uint32_t a_chunk, a_stage, b_chunk, b_aug, b_bytes, b_stride, a_off, ctl_off, total;
};

__host__ __device__ inline Layout make_layout(int CK, int NT, int BBUF, int ASTG, int d_pad, int PROD = 3) {
    Layout L;
    L.CK = CK;
    L.NT = NT;
    L.BBUF = BBUF;
    L.ASTG = ASTG;
    L.nc = d_pad / CK;
    L.a_chunk = 128u * CK * 2u;
    L.b_chunk = (uint32_t)NT * CK * 2u;
    L.b_aug = (uint32_t)NT * 32u;
    L.b_bytes = (PROD == 3 ? 2u : 1u) * L.nc * L.b_chunk + L.b_aug;
    L.b_stride = (L.b_bytes + 1023u) & ~1023u;
    // fp16: a stage holds cps K chunks of the query tile (both chunks of a d_pad = 128
    // tile with 64-wide chunks, else one) and the last stage also its augmentation
    // block, so a tile costs one stage hand-off where the split pays nc + 1
    L.cps = (PROD == 1 && L.nc == 2 && CK == 64) ? 2 : 1;
    L.a_stage = L.cps * L.a_chunk + (PROD == 1 ? 128u * 32u : 0u);
    L.a_off = BBUF * L.b_stride;
    L.ctl_off = L.a_off + ASTG * L.a_stage;
    L.total = L.ctl_off + 1024u + 1024u;  // control block + alignment slack
    return L;
}

// TABLE: work items come from a device table (inverted-file scan) instead of the dense
// (point tile x query-tile group) enumeration; a template parameter so that the dense
// instantiations carry none of its code.
template <int CK, int NT, int BBUF, int ASTG, int PROD, int CPS, bool TABLE>
__global__ void __launch_bounds__(kThreads, 1) sweep_tc_kernel(const __grid_constant__ TcArgs p) {
    const bool seg_mode = p.sink.seg_counts != nullptr;
    if (seg_mode && threadIdx.x == 0) {
        p.sink.seg_counts[blockIdx.x] = 0;
        p.sink.band_seg_counts[blockIdx.x] = 0;
    }
    if (p.check_done && p.st->done) return;
    const long long a_rows = p.a_rows_dev ? (long long)*p.a_rows_dev : p.a_rows_max;
    if (a_rows <= 0 || p.n <= 0) return;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const Layout L = make_layout(CK, NT, BBUF, ASTG, p.d_pad, PROD);
    const int nc = L.nc;
    const int nq = PROD == 3 ? 2 * nc : nc;   // query-tile chunks before the augmentation chunk
    constexpr int cps = CPS;   // = L.cps (the dispatch picks the instantiation that matches)
    const int nstage = PROD == 3 ? nq + 1 : (nc + cps - 1) / cps;   // shared-memory stages per query tile
    // One-stage query tiles (fp16: d_pad = CK, or d_pad = 2 CK in one stage) are five
    // (nine) MMAs; the issuing thread's per-tile barrier work does not overlap its own
    // MMAs, so two warps issue alternate tiles (tile T into accumulator T mod 2).
    const bool dual = PROD == 1 && nstage == 1;
    Ctl* ctl = reinterpret_cast<Ctl*>(smem + L.ctl_off);
    const uint32_t sbase = su32(smem);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long a_tiles = (a_rows + 127) / 128;
    const int G = (int)(a_tiles < kMaxGroup ? a_tiles : kMaxGroup);
    const long long n_groups = (a_tiles + G - 1) / G;
    const long long b_tiles = (p.n + NT - 1) / NT;
    constexpr bool table = TABLE;
    const long long items = table ? *p.items_count : b_tiles * n_groups;
    constexpr uint32_t kTmemCols = 2 * NT;
    constexpr uint32_t kIdesc = idesc_f16kind(128, NT, PROD == 3);
    constexpr uint32_t kSpan = CK * 2;
    int* gerr = &p.st->error;

    if (threadIdx.x == 0) {
        for (int i = 0; i < BBUF; ++i) {
            bar_init(&ctl->b_full[i], 1);
            bar_init(&ctl->b_empty[i], dual ? 2 : 1);   // both issuers release the point tile
        }
        for (int i = 0; i < ASTG; ++i) {
            bar_init(&ctl->a_full[i], 1);
            bar_init(&ctl->a_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            bar_init(&ctl->t_full[i], 1);
            bar_init(&ctl->t_empty[i], kEpiWarps);
        }
        bar_init(&ctl->drain, dual ? 2 : 1);
        ctl->abort_flag = 0;
        ctl->seg_used = 0;
        ctl->band_used = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&ctl->tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = ctl->tmem_base;
    volatile int* abort_flag = &ctl->abort_flag;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            uint32_t a_st = 0, a_ph = 0, b_buf = 0, b_ph = 0;
            bool ok = true;
            // parity of the last load issued into each stage / buffer (for draining)
            int a_last[ASTG], b_last[BBUF];
            for (int i = 0; i < ASTG; ++i) a_last[i] = -1;
            for (int i = 0; i < BBUF; ++i) b_last[i] = -1;
            for (long long item = blockIdx.x; ok && item < items; item += gridDim.x) {
                long long bt, at0, at1;
                if (table) {
                    const TcItem& it = p.items[item];
                    bt = it.b_tile;
                    at0 = it.a_tile0;
                    at1 = at0 + it.a_count;
                } else {
                    const long long g = item % n_groups;
                    bt = item / n_groups;
                    at0 = g * G;
                    at1 = (at0 + G < a_tiles) ? at0 + G : a_tiles;
                }
                const int yb = (int)(bt * NT);
                if (!bar_wait(&ctl->b_empty[b_buf], b_ph ^ 1, abort_flag, gerr)) { ok = false; break; }
                bar_expect_tx(&ctl->b_full[b_buf], L.b_bytes);
                const uint32_t bb = sbase + b_buf * L.b_stride;
                for (int c = 0; c < nc; ++c) {
                    tma_load(bb + c * L.b_chunk, &p.b_hi, &ctl->b_full[b_buf], c * CK, yb);
                    if (PROD == 3) tma_load(bb + (nc + c) * L.b_chunk, &p.b_lo, &ctl->b_full[b_buf], c * CK, yb);
                }
                tma_load(bb + nq * L.b_chunk, &p.b_aug, &ctl->b_full[b_buf], 0, yb);
                b_last[b_buf] = (int)b_ph;
                if (++b_buf == BBUF) { b_buf = 0; b_ph ^= 1; }
                for (long long at = at0; ok && at < at1; ++at) {
                    const int ya = (int)(at * 128);
                    for (int q = 0; q < nstage; ++q) {
                        if (!bar_wait(&ctl->a_empty[a_st], a_ph ^ 1, abort_flag, gerr)) { ok = false; break; }
                        const uint32_t dst = sbase + L.a_off + a_st * L.a_stage;
                        if (PROD == 1) {
                            const bool last = q == nstage - 1;
                            const int c0 = q * cps, c1 = (c0 + cps < nc) ? c0 + cps : nc;
                            bar_expect_tx(&ctl->a_full[a_st], (c1 - c0) * L.a_chunk + (last ? 128u * 32u : 0u));
                            for (int c = c0; c < c1; ++c)
                                tma_load(dst + (c - c0) * L.a_chunk, &p.a_hi, &ctl->a_full[a_st], c * CK, ya);
                            if (last) tma_load(dst + (c1 - c0) * L.a_chunk, &p.a_aug, &ctl->a_full[a_st], 0, ya);
                        } else if (q < nc) {
                            bar_expect_tx(&ctl->a_full[a_st], L.a_chunk);
                            tma_load(dst, &p.a_hi, &ctl->a_full[a_st], q * CK, ya);
                        } else if (q < nq) {
                            bar_expect_tx(&ctl->a_full[a_st], L.a_chunk);
                            tma_load(dst, &p.a_lo, &ctl->a_full[a_st], (q - nc) * CK, ya);
                        } else {
                            bar_expect_tx(&ctl->a_full[a_st], 128u * 32u);
                            tma_load(dst, &p.a_aug, &ctl->a_full[a_st], 0, ya);
                        }
                        a_last[a_st] = (int)a_ph;
                        if (++a_st == ASTG) { a_st = 0; a_ph ^= 1; }
                    }
                }
            }
            // drain: every issued copy has landed before shared memory is released
            for (int i = 0; i < ASTG; ++i)
                if (a_last[i] >= 0) bar_drain(&ctl->a_full[i], (uint32_t)a_last[i]);
            for (int i = 0; i < BBUF; ++i)
                if (b_last[i] >= 0) bar_drain(&ctl->b_full[i], (uint32_t)b_last[i]);
        }
    } else if (warp == 1 || warp == kIssuer2) {
        // ------------------------------------------------------------ MMA issuers
        // Descriptors are formed once per stage / point tile (a descriptor's address
        // field is the byte address / 16: offsets add to it), barrier addresses once.
        if (lane == 0 && (warp == 1 || dual)) {
            uint32_t a_st = 0, a_ph = 0, b_buf = 0, b_ph = 0, t_buf = 0, t_ph = 0;
            bool ok = true;
            const uint32_t a_full0 = su32(&ctl->a_full[0]), a_empty0 = su32(&ctl->a_empty[0]);
            const uint32_t t_full0 = su32(&ctl->t_full[0]), t_empty0 = su32(&ctl->t_empty[0]);
            const unsigned long long ad0 = sdesc(sbase + L.a_off, kSpan);
            const unsigned long long aaug0 = sdesc(sbase + L.a_off + nc * L.a_chunk, 32);
            const unsigned long long achunk = L.a_chunk >> 4, bchunk = L.b_chunk >> 4;
            const unsigned long long aaug_split0 = sdesc(sbase + L.a_off, 32);   // split: aug stage
            const unsigned long long astep = L.a_stage >> 4;
            uint32_t t_seq = 0;   // dual issue: tiles of this CTA before the current item
            for (long long item = blockIdx.x; ok && item < items; item += gridDim.x) {
                long long at0, at1;
                if (table) {
                    at0 = p.items[item].a_tile0;
                    at1 = at0 + p.items[item].a_count;
                } else {
                    const long long g = item % n_groups;
                    at0 = g * G;
                    at1 = (at0 + G < a_tiles) ? at0 + G : a_tiles;
                }
                if (!bar_wait(&ctl->b_full[b_buf], b_ph, abort_flag, gerr)) { ok = false; break; }
                fence_after();
                const uint32_t bb = sbase + b_buf * L.b_stride;
                if (dual) {
                    // tiles T of this CTA in order; this warp issues those with T mod 2 = me
                    const uint32_t me = warp == 1 ? 0u : 1u;
                    const unsigned long long bd = sdesc(bb, kSpan), baug = sdesc(bb + nq * L.b_chunk, 32);
                    const uint32_t nt = (uint32_t)(at1 - at0);
                    for (uint32_t i = (me ^ t_seq) & 1u; i < nt; i += 2) {
                        const uint32_t tt = t_seq + i;
                        const uint32_t st = tt % ASTG, sph = (tt / ASTG) & 1u, tph = (tt >> 1) & 1u;
                        if (!bar_wait_at(t_empty0 + 8u * me, tph ^ 1u, abort_flag, gerr) ||
                            !bar_wait_at(a_full0 + 8u * st, sph, abort_flag, gerr)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint32_t dacc = tmem + me * NT;
                        const unsigned long long ad = ad0 + st * astep, aaug = aaug0 + st * astep;
#pragma unroll
                        for (int c = 0; c < CPS; ++c) {
                            if (c >= nc) break;
#pragma unroll
                            for (int k = 0; k < CK / 16; ++k)
                                mma(dacc, ad + c * achunk + 2 * k, bd + c * bchunk + 2 * k, kIdesc, c > 0 || k > 0);
                        }
                        mma(dacc, aaug, baug, kIdesc, 1);
                        mma_commit_at(a_empty0 + 8u * st);
                        mma_commit_at(t_full0 + 8u * me);
                    }
                    if (!ok) break;
                    t_seq += nt;
                    mma_commit(&ctl->b_empty[b_buf]);
                    if (++b_buf == BBUF) { b_buf = 0; b_ph ^= 1; }
                    continue;
                }
                if constexpr (PROD == 3) {
                    // bf16 split: per query tile nc hi stages (A hi x B hi and A hi x B lo),
                    // nc lo stages (A lo x B hi) and the augmentation stage; descriptors
                    // from per-stage / per-point-tile bases
                    const unsigned long long bd = sdesc(bb, kSpan), baug = sdesc(bb + nq * L.b_chunk, 32);
                    for (long long ia = 0; ia < at1 - at0; ++ia) {
                        if (!bar_wait_at(t_empty0 + 8u * t_buf, t_ph ^ 1, abort_flag, gerr)) { ok = false; break; }
                        const uint32_t dacc = tmem + t_buf * NT;
                        for (int q = 0; q < nstage; ++q) {
                            if (!bar_wait_at(a_full0 + 8u * a_st, a_ph, abort_flag, gerr)) { ok = false; break; }
                            fence_after();
                            const unsigned long long ad = ad0 + a_st * astep;
                            if (q < nc) {
                                const unsigned long long bh = bd + q * bchunk, bl = bd + (nc + q) * bchunk;
#pragma unroll
                                for (int k = 0; k < CK / 16; ++k) {
                                    mma(dacc, ad + 2 * k, bh + 2 * k, kIdesc, q > 0 || k > 0);
                                    mma(dacc, ad + 2 * k, bl + 2 * k, kIdesc, 1);
                                }
                            } else if (q < nq) {
                                const unsigned long long bh = bd + (q - nc) * bchunk;
#pragma unroll
                                for (int k = 0; k < CK / 16; ++k) mma(dacc, ad + 2 * k, bh + 2 * k, kIdesc, 1);
                            } else {
                                mma(dacc, aaug_split0 + a_st * astep, baug, kIdesc, 1);
                            }
                            mma_commit_at(a_empty0 + 8u * a_st);
                            if (++a_st == ASTG) { a_st = 0; a_ph ^= 1; }
                        }
                        if (!ok) break;
                        mma_commit_at(t_full0 + 8u * t_buf);
                        if (++t_buf == 2) { t_buf = 0; t_ph ^= 1; }
                    }
                } else {
                    // fp16 with one K chunk per stage over several stages (d_pad > CK): the
                    // augmentation block rides in the last stage
                    for (long long ia = 0; ok && ia < at1 - at0; ++ia) {
                        if (!bar_wait(&ctl->t_empty[t_buf], t_ph ^ 1, abort_flag, gerr)) { ok = false; break; }
                        fence_after();
                        const uint32_t dacc = tmem + t_buf * NT;
                        uint32_t acc = 0;
                        for (int q = 0; q < nstage; ++q) {
                            if (!bar_wait(&ctl->a_full[a_st], a_ph, abort_flag, gerr)) { ok = false; break; }
                            fence_after();
                            const uint32_t aa = sbase + L.a_off + a_st * L.a_stage;
#pragma unroll
                            for (int k = 0; k < CK / 16; ++k) {
                                mma(dacc, sdesc(aa + k * 32, kSpan), sdesc(bb + q * L.b_chunk + k * 32, kSpan), kIdesc,
                                    acc);
                                acc = 1;
                            }
                            if (q == nstage - 1)
                                mma(dacc, sdesc(aa + L.a_chunk, 32), sdesc(bb + nq * L.b_chunk, 32), kIdesc, 1);
                            mma_commit(&ctl->a_empty[a_st]);
                            if (++a_st == ASTG) { a_st = 0; a_ph ^= 1; }
                        }
                        if (!ok) break;
                        mma_commit(&ctl->t_full[t_buf]);
                        if (++t_buf == 2) { t_buf = 0; t_ph ^= 1; }
                    }
                }
                if (!ok) break;
                mma_commit(&ctl->b_empty[b_buf]);
                if (++b_buf == BBUF) { b_buf = 0; b_ph ^= 1; }
            }
            // drain: all issued MMAs complete before TMEM / shared memory are released
            mma_commit(&ctl->drain);
            bar_drain(&ctl->drain, 0);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        // warp w reads TMEM lanes 32*(w%4) .. +31 (the tcgen05.ld lane rule);
        // warps 2-5 take the first half of the columns, warps 6-9 the second.
        constexpr int kChunks = NT / 64;            // 32-column loads per warp per tile
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        // Column 6 of the query rows' augmentation carries +delta'_row (the row's band half-width
        // rounded up to the operand type) against the points' 1, so the accumulator holds
        // acc = v + delta'_row: acc < 0 (sign bit set) decides "not a member", acc > 2 delta'_row
        // decides "member", the rest is the band.  The split tiles (dense, wide bands) read
        // each row's delta'_row; the fp16 tiles take the threshold 2 delta' of the largest
        // half-width instead (acc > 2 delta' >= 2 delta'_row is still a member, and their
        // epilogue, the kernel's bottleneck, keeps no per-row load).
        constexpr bool row_thr = PROD == 3;
        const float thr_all = 2.f * __half2float(__float2half_ru(p.st->delta));
        const unsigned long long seg_off = seg_mode ? (unsigned long long)blockIdx.x * p.sink.seg_cap : 0ull;
        unsigned long long* seg_keys = p.sink.keys + seg_off;
        unsigned long long* band_keys = p.sink.band_keys + seg_off;
        const unsigned long long band_cap = seg_mode ? p.sink.seg_cap : p.sink.band_cap;
        uint32_t t_buf = 0, t_ph = 0;
        unsigned long long pairs_local = 0;
        bool ok = true;
        for (long long item = blockIdx.x; ok && item < items; item += gridDim.x) {
            long long bt, at0, at1, a_end = a_rows, col_end = p.n, b_col0 = 0, src0 = 0;
            if (table) {
                const TcItem it = p.items[item];
                bt = it.b_tile;
                at0 = it.a_tile0;
                at1 = at0 + it.a_count;
                a_end = it.a_end;
                col_end = it.col_end;
                b_col0 = it.b_col0;
                src0 = it.src0;
            } else {
                const long long g = item % n_groups;
                bt = item / n_groups;
                at0 = g * G;
                at1 = (at0 + G < a_tiles) ? at0 + G : a_tiles;
            }
            const long long col_base = bt * NT + half * (NT / 2);
            for (long long at = at0; at < at1; ++at) {
                const long long row = at * 128 + quarter * 32 + lane;
                const bool row_ok = row < a_end;
                // this row's threshold (split tiles), loaded before the wait for the accumulator
                const unsigned short dbits = row_thr && row_ok ? p.a_aug_rows[row * 16 + 6] : (unsigned short)0;
                const bool w = __all_sync(kFull, bar_wait(&ctl->t_full[t_buf], t_ph, abort_flag, gerr));
                if (!w) { ok = false; break; }
                fence_after();
                // the query this A row holds (table mode) and the key's row part
                const long long qid = table ? (row_ok ? (long long)p.a_map[row] : -1) : row;
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + t_buf * NT + half * (NT / 2);
                uint32_t r[kChunks][32];
                float cmax[kChunks];
                tmem_ld_all<kChunks>(taddr, r, cmax);
                // the accumulator is read: hand the TMEM buffer back to the MMA warp
                fence_before();
                __syncwarp();
                if (lane == 0) bar_arrive(&ctl->t_empty[t_buf]);
                if (++t_buf == 2) { t_buf = 0; t_ph ^= 1; }
                // fast path: every value of this thread's row below zero (the chunk maxima of
                // the reducing loads) for the whole warp -> nothing to emit.  A chunk holding
                // -0 (or NaN) is not "below zero" and takes the sign-bit path below.
                float rmax = cmax[0];
#pragma unroll
                for (int j = 1; j < kChunks; ++j) rmax = fmaxf(rmax, cmax[j]);
                const bool quiet = !row_ok || rmax < 0.f;
                if (__all_sync(kFull, quiet)) {
                    if (threadIdx.x == 64) {
                        const long long ra = (a_end - at * 128) < 128 ? (a_end - at * 128) : 128;
                        const long long rb = (col_end - bt * NT) < NT ? (col_end - bt * NT) : NT;
                        if (!table || (ra > 0 && rb > 0)) pairs_local += (unsigned long long)(ra * rb);
                    }
                    continue;
                }
                // classification: per 32-column chunk a hit mask (acc > hit_thr) and a band
                // mask (0 <= acc <= hit_thr), bit i = column col0 + i.  Sign bits are
                // gathered with funnel shifts (bit i of the mask from register i); the sign
                // of thr - acc is set exactly when acc > thr (a rounded difference keeps the
                // sign of the exact one, and is +0 only when they are equal).
                const float hit_thr = row_thr ? 2.f * __bfloat162float(__ushort_as_bfloat16(dbits)) : thr_all;
                unsigned hitm[kChunks], bandm[kChunks];
                unsigned nh = 0, nb = 0;
#pragma unroll
                for (int j = 0; j < kChunks; ++j) {
                    hitm[j] = 0u;
                    bandm[j] = 0u;
                    if (row_ok && !(cmax[j] < 0.f)) {
                        const long long left = col_end - (col_base + j * 32);
                        const unsigned valid = left >= 32 ? kFull : (left <= 0 ? 0u : (1u << left) - 1u);
                        unsigned sgn = 0u;
#pragma unroll
                        for (int i = 31; i >= 0; --i) sgn = __funnelshift_l(r[j][i], sgn, 1);
                        const unsigned near_ = ~sgn & valid;
                        unsigned gt = 0u;
                        if (near_) {
#pragma unroll
                            for (int i = 31; i >= 0; --i)
                                gt = __funnelshift_l(__float_as_uint(hit_thr - __uint_as_float(r[j][i])), gt, 1);
                        }
                        hitm[j] = gt & near_;
                        bandm[j] = near_ & ~gt;
                        nh += __popc(hitm[j]);
                        nb += __popc(bandm[j]);
                    }
                }
                // emission: one reservation per warp and tile for both kinds (counts packed
                // as hits << 16 | band, each at most 128 per lane), then each lane writes its keys
                const unsigned packed = (nh << 16) | nb;
                if (__any_sync(kFull, packed != 0u)) {
                    unsigned incl = packed;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const unsigned y = __shfl_up_sync(kFull, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const unsigned tot = __shfl_sync(kFull, incl, 31);
                    unsigned long long hbase = 0, bbase = 0;
                    if (lane == 31) {
                        if (seg_mode) {
                            if (tot >> 16) hbase = atomicAdd(&ctl->seg_used, tot >> 16);
                            if (tot & 0xffffu) bbase = atomicAdd(&ctl->band_used, tot & 0xffffu);
                        } else {
                            if (tot >> 16) hbase = atomicAdd(p.sink.count, (unsigned long long)(tot >> 16));
                            if (tot & 0xffffu) bbase = atomicAdd(p.sink.band_n, (unsigned long long)(tot & 0xffffu));
                        }
                    }
                    hbase = __shfl_sync(kFull, hbase, 31);
                    bbase = __shfl_sync(kFull, bbase, 31);
                    const unsigned excl = incl - packed;
                    unsigned long long hpos = hbase + (excl >> 16), bpos = bbase + (excl & 0xffffu);
                    unsigned long long* hkeys = seg_mode ? seg_keys : p.sink.keys;
                    const unsigned long long hcap = seg_mode ? p.sink.seg_cap : p.sink.cap;
                    const unsigned long long rowkey = (unsigned long long)(unsigned)qid << 32;
#pragma unroll
                    for (int j = 0; j < kChunks; ++j) {
                        const unsigned col0 = (unsigned)(col_base + j * 32);
                        unsigned m = bandm[j];
                        while (m) {
                            const int b = __ffs(m) - 1;
                            m &= m - 1;
                            unsigned col = col0 + (unsigned)b;
                            if (table) col = (unsigned)p.b_ids[src0 + ((long long)col - b_col0)];
                            if (bpos < band_cap) band_keys[bpos] = rowkey | col;
                            ++bpos;
                        }
                        m = hitm[j];
                        while (m) {
                            const int b = __ffs(m) - 1;
                            m &= m - 1;
                            unsigned col = col0 + (unsigned)b;
                            if (table) col = (unsigned)p.b_ids[src0 + ((long long)col - b_col0)];
                            if (hpos < hcap) hkeys[hpos] = rowkey | col;
                            ++hpos;
                            if (p.sink.slot_of) {   // greedy: a later candidate covered by this one
                                const int sl = p.sink.slot_of[col];
                                const int qr = (int)qid;
                                if (sl > qr) {
                                    atomicOr(&p.sink.conflict[(size_t)qr * p.sink.conflict_words + (sl >> 5)],
                                             1u << (sl & 31));
                                    atomicOr(&p.sink.row_any[qr >> 5], 1u << (qr & 31));
                                }
                            }
                        }
                    }
                }
                if (threadIdx.x == 64) {
                    const long long ra = (a_end - at * 128) < 128 ? (a_end - at * 128) : 128;
                    const long long rb = (col_end - bt * NT) < NT ? (col_end - bt * NT) : NT;
                    if (!table || (ra > 0 && rb > 0)) pairs_local += (unsigned long long)(ra * rb);
                }
            }
        }
        if (threadIdx.x == 64 && pairs_local) atomicAdd(p.sink.pair_count, pairs_local);
    }

    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
    if (seg_mode && threadIdx.x == 0) {
        p.sink.seg_counts[blockIdx.x] = ctl->seg_used;
        p.sink.band_seg_counts[blockIdx.x] = ctl->band_used;
    }
}


// The compiled tile shapes (CK, NT, BBUF, ASTG).
#define BM_TC_SHAPES(X) \
    X(16, 256, 2, 8)    \
    X(32, 256, 2, 8)    \
    X(32, 256, 1, 8)    \
    X(32, 128, 2, 8)    \
    X(64, 256, 2, 5)    \
    X(64, 256, 1, 5)    \
    X(64, 128, 2, 5)    \
    X(64, 128, 1, 4)    \
    X(64, 64, 1, 4)     \
    X(64, 256, 1, 3)    \
    X(64, 256, 2, 2)

template <int CK, int NT, int BBUF, int ASTG, int PROD, int CPS, bool TABLE>
cudaError_t launch_cfg(TcArgs& args, long long a_rows_max, cudaStream_t stream, std::string* why, int* grid_out) {
    const Layout L0 = make_layout(CK, NT, BBUF, ASTG, args.d_pad, PROD);
    if (L0.cps != CPS) {
        if (why) *why = "tile instantiation does not match the stage layout";
        return cudaErrorInvalidValue;
    }
    // at least 120 KB so that two CTAs never share an SM (each holds 2*NT TMEM columns)
    Layout L = L0;
    if (L.total < 120u * 1024u) L.total = 120u * 1024u;
    auto kern = sweep_tc_kernel<CK, NT, BBUF, ASTG, PROD, CPS, TABLE>;
    static int attr_bytes = 0;
    if (attr_bytes < (int)L.total) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
        if (e != cudaSuccess) {
            if (why) *why = "cannot reserve shared memory";
            return e;
        }
        attr_bytes = (int)L.total;
    }
    const long long a_tiles = (a_rows_max + 127) / 128;
    const long long G = a_tiles < kMaxGroup ? a_tiles : kMaxGroup;
    const long long items = ((args.n + NT - 1) / NT) * ((a_tiles + G - 1) / G);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // table mode: the item count is on the device; every SM takes part
    const long long grid = args.items ? sms : (items < sms ? items : sms);
    *grid_out = (int)(grid > 0 ? grid : 0);
    if (grid <= 0) return cudaSuccess;
    note_launch();
    kern<<<(unsigned)grid, kThreads, L.total, stream>>>(args);
    return cudaGetLastError();
}

// fp16 whole-tile stages exist for 64-wide K chunks only (d_pad = 128).
template <int CK, int NT, int BBUF, int ASTG, bool TABLE>
cudaError_t launch_whole(TcArgs& args, long long a_rows_max, cudaStream_t stream, std::string* why, int* grid_out) {
    if constexpr (CK == 64) {
        return launch_cfg<CK, NT, BBUF, ASTG, 1, 2, TABLE>(args, a_rows_max, stream, why, grid_out);
    } else {
        if (why) *why = "whole-tile stages need 64-wide K chunks";
        return cudaErrorInvalidValue;
    }
}

// Launch the instantiation of a tile configuration: the bf16 split (three products), fp16
// with one K chunk per stage, or fp16 with the whole query tile in one stage.
template <bool TABLE>
cudaError_t dispatch(const TileConfig& cfg, bool fp16, bool whole, TcArgs& args, long long a_rows_max,
                     cudaStream_t stream, std::string* why, int* grid_out) {
#define BM_X(a, b, c, d)                                                                                \
    if (cfg.ck == a && cfg.nt == b && cfg.bbuf == c && cfg.astg == d)                                   \
        return !fp16    ? launch_cfg<a, b, c, d, 3, 1, TABLE>(args, a_rows_max, stream, why, grid_out)   \
               : !whole ? launch_cfg<a, b, c, d, 1, 1, TABLE>(args, a_rows_max, stream, why, grid_out) \
                        : launch_whole<a, b, c, d, TABLE>(args, a_rows_max, stream, why, grid_out);
    BM_TC_SHAPES(BM_X)
#undef BM_X
    if (why) *why = "tile shape not compiled";
    return cudaErrorNotSupported;
}

}  // namespace tc
}  // namespace bm
