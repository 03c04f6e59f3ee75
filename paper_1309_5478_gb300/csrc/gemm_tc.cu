// Fused tensor-core distance GEMM + quick multi-select (the chosen form).
//
// Paper: Methods, "Distance calculation" (distances from the product X^T Y and the
// norms, ranked by d'_ij = |y_j|^2 - 2 x_i.y_j) and "GPU-based quick multi-select"
// (per-row selection with warp ballot/popc partitions). The paper materialises the
// M x N matrix in global memory between the two; here the selection runs in the
// GEMM's epilogue, so the matrix never leaves the chip.
//
// Structure (one persistent CTA per SM, 10 warps):
//   warp 0     TMA producer: 128 x 64 query tiles (A) and 256 x 64 corpus tiles (B),
//              128-byte swizzle, into a 4-stage shared-memory ring (mbarrier full/empty)
//   warp 1     allocates 512 TMEM columns (two 128 x 256 FP32 accumulators) and issues
//              tcgen05.mma (BF16 kind::f16, or FP8 e4m3 kind::f8f6f4) from one thread;
//              tcgen05.commit releases smem stages and publishes finished accumulators
//   warps 2-9  epilogue: two warps per TMEM lane quarter (32 query rows, one per lane),
//              each taking half of every tile's columns; tcgen05.ld 32 columns at a time,
//              v = |c_j|^2 - 2 acc (FP8: acc scaled back), and a key (v, j) that passes the
//              row's running threshold is appended to the row's candidate list in global
//              memory (L2-resident): the first warp fills it from the front, the second
//              from the back. When a list nears its capacity, the quick multi-select
//              (select_core.cuh) shrinks it and the threshold falls to
//              max(v_(k+m), v_(k) + 2E_i) (speculatively to lower ranks while only part
//              of the corpus has been swept), so the list always holds every point whose
//              exact distance can still be among the row's k smallest.
//   warps 10-11 exact re-rank (rerank_core.cuh) of the row blocks this CTA has finished,
//              while the other warps sweep the next one: the re-rank gathers FP32 corpus
//              rows from HBM while the tensor cores are busy, so the two overlap. They stop
//              once the epilogue has finished the CTA's last row block; the rows they have
//              not reached by then are left to the re-rank launch that follows the kernel.
// Work: row blocks of 128 queries; each CTA sweeps all corpus tiles of a row block
// (the candidate state of a row lives in one CTA), then hands the rows' lists to the
// re-rank (which reduces them to the band) and takes the next row block.
// Every wait is bounded (p.wait_limit polls); on expiry the kernel records KNN_ETIMEOUT in
// a status word, stops issuing work, waits (bounded) for its own copies and frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "engine.h"
#include "internal.h"
#include "rerank_core.cuh"
#include "select_core.cuh"
#include "tc_fused.h"

namespace knn {
namespace {

constexpr int TC_BM = 128;
constexpr int TC_BN = 256;
constexpr int TC_BK_BYTES = 128;  // one 128-byte swizzle row per stage: 64 BF16 or 128 FP8 values
constexpr int A_BYTES = TC_BM * TC_BK_BYTES;  // 16 KB

// Tile configurations (corpus columns per tile BN):
//   256: 128 x 256 tiles, two 256-column accumulators (all 512 TMEM columns), one CTA of
//        12 warps an SM (producer, MMA issuer, 8 epilogue warps, 2 re-rank warps);
//   128: 128 x 128 tiles, two 128-column accumulators (256 TMEM columns), 10 warps a CTA and
//        two CTAs an SM, so 16 epilogue warps share an SM (batched launches only).
template <int BN>
struct Tile {
    static constexpr int B_BYTES = BN * TC_BK_BYTES;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr uint32_t TMEM_COLS = 2u * BN;
    static constexpr int THREADS = BN == 256 ? 384 : 320;
    static constexpr int CTAS_PER_SM = BN == 256 ? 1 : 2;
};
constexpr int TC_THREADS = Tile<TC_BN>::THREADS;
constexpr int STAGE_BYTES = Tile<TC_BN>::STAGE_BYTES;
// dynamic shared memory a CTA may use: the SM's 228 KB less 1 KB reserved per CTA, shared by
// the CTAs of an SM
constexpr size_t smem_budget(int bn) { return bn == 256 ? 232448 : (233472 - 2 * 1024) / 2; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false when the limit expired or another warp already gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, long long limit) {
    for (long long i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

// The same wait taken by a whole warp: every lane observes the phase, and all lanes
// return the same answer (a warp that gives up leaves together).
__device__ __forceinline__ bool mbar_wait_all(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                              long long limit) {
    for (long long i = 0; i < limit; ++i) {
        if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
        if ((i & 255) == 255 && __any_sync(0xffffffffu, *abort_flag != 0)) return false;
    }
    if (lane_id() == 0) *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr & 0x3ffffu) >> 4);
    d |= static_cast<uint64_t>(1) << 16;            // leading byte offset (unused for swizzled K-major)
    d |= static_cast<uint64_t>(1024 >> 4) << 32;    // stride byte offset: 8 rows x 128 B
    d |= static_cast<uint64_t>(1) << 46;            // descriptor version
    d |= static_cast<uint64_t>(2) << 61;            // SWIZZLE_128B
    return d;
}

// Instruction descriptor: FP32 accumulator, K-major A and B, M = 128, N = BN.
template <int P, int BN>
__host__ __device__ constexpr uint32_t idesc() {
    // bits 4-5 D format (1 = F32); 7-9 A format, 10-12 B format (kind::f16: 1 = BF16;
    // kind::f8f6f4: 0 = E4M3); 15/16 A/B major (0 = K); 17-22 N >> 3; 24-28 M >> 4.
    return (1u << 4) | ((P == P_BF16 ? 1u : 0u) << 7) | ((P == P_BF16 ? 1u : 0u) << 10) |
           (static_cast<uint32_t>(BN >> 3) << 17) | (static_cast<uint32_t>(TC_BM >> 4) << 24);
}

template <int P, int BN>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    if constexpr (P == P_BF16) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc<P, BN>()), "r"(accumulate));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc<P, BN>()), "r"(accumulate));
    }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Issues a 32-column TMEM load; the registers are valid only after tmem_ld_wait().
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    tmem_ld32_issue(taddr, r);
    tmem_ld_wait();
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

constexpr int MAX_STAGES = 4;

constexpr int EPI_WARPS = 8;   // two per TMEM lane quarter; each takes half of every tile's columns
constexpr int RR_WARPS = 2;    // re-rank warps (warps 2 + EPI_WARPS ...)
constexpr int RR_P = 512;      // keys per re-rank warp buffer: longer lists are left to the re-rank launch
constexpr int RAW_LIST_MAX = 512;  // longest list handed to the re-rank without a trim
constexpr int HIST_WORDS = 36; // histogram of the sampled select (33 buckets used)

// Per-epilogue-warp working arrays for the quick multi-select of one row's list (the keys
// stay in the global list): the 32-bit values A and a histogram in shared memory; the
// rarely used auxiliary arrays in global scratch (L2-resident).
struct EpiSmem {
    uint32_t* A;        // shared: cap values
    uint32_t* hist;     // shared: HIST_WORDS
    uint32_t* B;        // global: cap values (sampled two-rank select), then tmp (cap values)
    uint64_t* scratch;  // global: exact 64-bit path (2 cap keys + reference list); B aliases its front
};

// Shared candidate-list state of the 128 rows of the current row block. Both warps of a
// lane quarter insert into the same list of a row without atomics: the warp of the first
// column half fills it from the front, the other from the back; a shrink compacts both
// segments to the front.
struct RowState {
    uint16_t* cnt;    // [128][2] keys at the front and at the back of the list
    uint64_t* tau;    // [128] threshold key: every key left out is > tau
    float* tauf;      // [128] float form of tau for the column filter (tau_filter)
    uint32_t* flags;  // [128] RS_TRUNC | RS_SPEC
};
constexpr uint32_t RS_TRUNC = 1u;  // the list was truncated
constexpr uint32_t RS_SPEC = 2u;   // a speculative shrink lowered the threshold


__host__ __device__ constexpr size_t epi_warp_bytes(int cap) {
    return static_cast<size_t>(cap) * 4 + HIST_WORDS * 4;
}
constexpr size_t ROWSTATE_BYTES = 128 * (4 + 8 + 4 + 4);

__host__ __device__ constexpr size_t cn_bytes(int precision, int bn = TC_BN) {
    return static_cast<size_t>(precision == P_FP8 ? 2 : 1) * 2 * bn * 4;
}

// Re-rank warps' shared memory: a key buffer and an FP64 tie buffer each, and counters.
constexpr size_t RR_BYTES = RR_WARPS * (static_cast<size_t>(RR_P + TIE_MAX) * 8 + RC_COUNT * 8);
// mbarriers, TMEM address, abort flag, completion count, and the epilogue pairs' wait results
constexpr size_t BAR_BYTES = 192;

__host__ __device__ constexpr size_t tc_smem_bytes(int cap, int stages, int precision, bool rr, int bn = TC_BN) {
    return 1024 /* alignment slack */ + static_cast<size_t>(stages) * (A_BYTES + bn * TC_BK_BYTES) +
           EPI_WARPS * epi_warp_bytes(cap) + cn_bytes(precision, bn) + ROWSTATE_BYTES + BAR_BYTES + (rr ? RR_BYTES : 0);
}

__host__ __device__ constexpr size_t scratch_words_per_warp(int cap) {
    return 2 * static_cast<size_t>(cap) + SEG_MAX;
}


// One work item's view of its problem: the row block `rb` of a problem, with the
// problem's tensor maps, sizes and arrays.
struct Item {
    const CUtensorMap* tmA;
    const CUtensorMap* tmB;
    int64_t M, N;
    int rb, nk, nct;
    int t0, nsw;      // first corpus tile of the sweep and tiles swept (symmetric form: t0 = rb / 2)
    int k, km, cap;
    int spec, perm_a;
    float spec_d2;
    const float* qnorm2;
    int64_t self_offset;
    const int32_t* self_col;
    const float* cnorm2;
    const float* E;
    const float* thr;
    const float* q_inv_scale;
    const float* c_inv_scale;
    uint64_t* cand;
    int32_t* count;
    uint64_t* bound;
    uint32_t* flags;
};

// Row block of the CTA's work item `it` (non-batched launch). The symmetric form's row
// blocks have sweeps of decreasing length, so every other full wave of items is dealt
// in reverse CTA order, which pairs long sweeps with short ones on each CTA.
__device__ __forceinline__ int item_rb(const FusedParams& p, int it) {
    if (!p.sym) return it;
    const int g = static_cast<int>(gridDim.x);
    const int w = it / g, b = it - w * g;
    return ((w & 1) && (w + 1) * g <= p.n_items) ? w * g + (g - 1 - b) : it;
}

template <bool BATCHED, int BN>
__device__ __forceinline__ Item get_item(const FusedParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB,
                                         int it) {
    Item im;
    if constexpr (!BATCHED) {
        im.tmA = tmA;
        im.tmB = tmB;
        im.M = p.M;
        im.N = p.N;
        im.rb = item_rb(p, it);
        im.nk = p.k_bytes / TC_BK_BYTES;
        im.k = p.k;
        im.km = p.km;
        im.cap = p.cap;
        im.self_offset = p.self_offset;
        im.self_col = p.self_col;
        im.cnorm2 = p.cnorm2;
        im.E = p.E;
        im.thr = p.thr;
        im.q_inv_scale = p.q_inv_scale;
        im.c_inv_scale = p.c_inv_scale;
        im.cand = p.cand;
        im.count = p.count;
        im.bound = p.bound;
        im.flags = p.flags;
        im.spec = p.spec;
        im.perm_a = p.perm_a > 1 ? p.perm_a : 1;
        im.spec_d2 = p.qnorm2 ? p.spec_d2 : F_INF;
        im.qnorm2 = p.qnorm2;
    } else {
        const FusedWork w = p.work[it];
        const FusedProblem& q = p.problems[w.problem];
        im.tmA = &q.tmA;
        im.tmB = &q.tmB;
        im.M = q.M;
        im.N = q.N;
        im.rb = w.rb;
        im.nk = q.k_bytes / TC_BK_BYTES;
        im.k = q.k;
        im.km = q.km;
        im.cap = q.cap;
        im.self_offset = q.self_offset;
        im.self_col = nullptr;
        im.cnorm2 = q.cnorm2;
        im.E = q.E;
        im.thr = q.thr;
        im.q_inv_scale = q.q_inv_scale;
        im.c_inv_scale = q.c_inv_scale;
        im.cand = q.cand;
        im.count = q.count;
        im.bound = q.bound;
        im.flags = q.flags;
        im.spec = q.spec;
        im.perm_a = 1;
        im.spec_d2 = F_INF;
        im.qnorm2 = nullptr;
    }
    im.nct = static_cast<int>((im.N + BN - 1) / BN);
    im.t0 = (!BATCHED && p.sym) ? im.rb >> 1 : 0;
    im.nsw = im.nct - im.t0;
    return im;
}

// Corpus tile swept at step ct of a row block's sweep.
__device__ __forceinline__ int tile_at(const Item& im, int ct) {
    return im.perm_a == 1 ? im.t0 + ct : static_cast<int>((static_cast<int64_t>(ct) * im.perm_a) % im.nct);
}

// Warp-cooperative shrink of the candidate list of row r (of the block) during the
// sweep, the out-of-line path behind shrink_mid_fast: a value of a 32-key sample of the
// list, sorted across the lanes, is taken as the threshold when counting over the list
// shows that at least rkm values lie at or below it and at least rk lie at or below it
// minus the window (so it is >= max(v_rkm, v_rk + window) and the list still holds the
// band of those ranks), preferring the smallest such sample value. If no sample value
// passes, or the threshold would keep more than keep_max keys, the two ranks are found by
// the sampled two-rank select, and when more than keep_max keys still remain the exact
// 64-bit quick multi-select keeps the keep_trunc smallest (truncation). The list's two
// segments (front and back) are read into registers, KPL keys per lane (cap <= 32 KPL), and
// the survivors are compacted to the front. Ranks below (k, k + m) make the shrink
// speculative (RS_SPEC is recorded when it lowers the threshold).
template <int KPL>
__device__ __noinline__ void shrink_row_k(const Item& p, const EpiSmem& es, const RowState& rs, int r, int64_t grow,
                                          float window, int rk, int rkm, int keep_max, int keep_trunc) {
    const int lane = static_cast<int>(lane_id());
    const uint32_t lt_mask = lanemask_lt();
    const int n0 = rs.cnt[2 * r];
    const int n = n0 + rs.cnt[2 * r + 1];
    const uint64_t t = rs.tau[r];
    uint64_t* gbuf = p.cand + grow * p.cap;
    uint64_t key[KPL];
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
        const int i = q * 32 + lane;
        const int pos = i < n0 ? i : p.cap - 1 - (i - n0);
        key[q] = i < n ? __ldcg(reinterpret_cast<const unsigned long long*>(gbuf) + pos) : KEY_MAX;
    }
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
        const int i = q * 32 + lane;
        if (i < n) es.A[i] = static_cast<uint32_t>(key[q] >> 32);
    }
    __syncwarp();
    const int kk = rk < n ? rk : n;
    const int kme = rkm < n ? rkm : n;
    uint64_t band = KEY_MAX;
    bool have_band = false;
    if (n >= rkm) {
        // sample of the list's values, sorted across the lanes
        const uint32_t smp = warp_sort32(es.A[(static_cast<int64_t>(lane) * n) >> 5]);
        // number of values <= x over the whole list
        auto count_le = [&](uint32_t x) {
            int c = 0;
#pragma unroll
            for (int q = 0; q < KPL; ++q) c += (q * 32 + lane < n && static_cast<uint32_t>(key[q] >> 32) <= x) ? 1 : 0;
            return __reduce_add_sync(0xffffffffu, static_cast<uint32_t>(c));
        };
        auto passes = [&](uint32_t cand) {
            if (count_le(cand) < static_cast<uint32_t>(kme)) return false;
            if (window <= 0.f) return true;
            return count_le(float_to_ord(ord_to_float(cand) - window)) >= static_cast<uint32_t>(kk);
        };
        int s0 = (32 * kme + n - 1) / n;  // the sample position expected to hold about rkm values
        s0 = s0 > 31 ? 31 : s0;
        int sel = -1;
        if (passes(__shfl_sync(0xffffffffu, smp, s0))) {
            sel = s0;
            while (sel > 0 && passes(__shfl_sync(0xffffffffu, smp, sel - 1))) --sel;
        } else {
            for (int s1 = s0 + 1; s1 < 32; ++s1)
                if (passes(__shfl_sync(0xffffffffu, smp, s1))) {
                    sel = s1;
                    break;
                }
        }
        if (sel >= 0) {
            band = key_ceiling(ord_to_float(__shfl_sync(0xffffffffu, smp, sel)));
            have_band = true;
        }
    }
    if (!have_band && n >= rkm) {
        uint32_t o_k = 0, o_km = 0;
        (void)two_ranks_sampled(es.A, es.B, es.B + p.cap, es.hist, n, kk - 1, kme - 1, o_k, o_km);
        float bv = ord_to_float(o_km);
        if (window > 0.f) bv = fmaxf(bv, ord_to_float(o_k) + window);
        band = key_ceiling(bv);
    }
    uint64_t nt = band < t ? band : t;
    int keep = 0;
#pragma unroll
    for (int q = 0; q < KPL; ++q) keep += (q * 32 + lane < n && key[q] <= nt) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
    if (have_band && keep > keep_max && n >= rkm) {
        // the sample value keeps too much: the exact ranks before the exact path
        uint32_t o_k = 0, o_km = 0;
        (void)two_ranks_sampled(es.A, es.B, es.B + p.cap, es.hist, n, kk - 1, kme - 1, o_k, o_km);
        float bv = ord_to_float(o_km);
        if (window > 0.f) bv = fmaxf(bv, ord_to_float(o_k) + window);
        band = key_ceiling(bv);
        nt = band < t ? band : t;
        keep = 0;
#pragma unroll
        for (int q = 0; q < KPL; ++q) keep += (q * 32 + lane < n && key[q] <= nt) ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
    }
    int nn;
    bool tr = false;
    if (keep <= keep_max) {
        nn = 0;
#pragma unroll
        for (int q = 0; q < KPL; ++q) {
            const bool kp = q * 32 + lane < n && key[q] <= nt;
            const uint32_t b = __ballot_sync(0xffffffffu, kp);
            if (kp) gbuf[nn + __popc(b & lt_mask)] = key[q];
            nn += __popc(b);
        }
    } else {
        // exact path on 64-bit keys in global scratch (ties at the threshold value)
        uint64_t* sA = es.scratch;
        uint64_t* sB = sA + p.cap;
        int* seg_s = reinterpret_cast<int*>(sB + p.cap);
        uint32_t* seg_e = reinterpret_cast<uint32_t*>(seg_s + SEG_MAX);
#pragma unroll
        for (int q = 0; q < KPL; ++q)
            if (q * 32 + lane < n) sA[q * 32 + lane] = key[q];
        __syncwarp();
        CompactResult res = compact_row(sA, sB, seg_s, seg_e, n, rk, rkm, window, t, keep_max, keep_trunc);
        if (res.ok) {
            for (int i = lane; i < res.n; i += 32) gbuf[i] = sA[i];
            nn = res.n;
            nt = res.tau;
            tr = res.truncated;
            band = res.band;
        } else {
            // reference list overflow: keep the first keys of the list and give up the
            // bound, so the row cannot be certified and goes to the exact fallback
            nn = n < keep_trunc ? n : keep_trunc;
#pragma unroll
            for (int q = 0; q < KPL; ++q)
                if (q * 32 + lane < nn) gbuf[q * 32 + lane] = key[q];
            nt = 0ull;
            tr = true;
        }
    }
    const uint32_t fl = rs.flags[r];
    const bool speculated = (rk < p.k || rkm < p.km) && nt < t;
    __syncwarp();
    if (lane == 0) {
        rs.cnt[2 * r] = static_cast<uint16_t>(nn);
        rs.cnt[2 * r + 1] = 0;
        rs.tau[r] = nt;
        rs.tauf[r] = tau_filter(nt);
        rs.flags[r] = fl | (tr ? RS_TRUNC : 0u) | (speculated ? RS_SPEC : 0u);
    }
    (void)band;
    __syncwarp();
}


// Fast path of a shrink of row r (inline, compact code): the sampled threshold search
// of shrink_row_k and the ballot compaction. When the sampled band would keep more than
// keep_max keys it is refined to the exact band edge by bisection; if that still keeps
// too many (or no sample value reaches the ranks), the list is truncated instead at
// the largest sample value that keeps at most keep_trunc keys, found by a binary search
// over the sorted sample, and the row is marked truncated there (every key dropped is
// above that value; the re-rank certificate decides). Returns false, with the list and
// the row state untouched, when no such value exists (keep_trunc = 0 disables truncation);
// the caller then runs shrink_row_k. Only the list's n keys are counted and kept: the
// padding of the register copy is KEY_MAX, which a threshold still open admits (a list
// that no sample value reduces and that needs no truncation keeps its n keys).
template <int KPL>
__device__ __forceinline__ bool shrink_mid_fast_body(const Item& p, const EpiSmem& es, const RowState& rs, int r,
                                                     int64_t grow, float window, int rk, int rkm, int keep_max,
                                                     int keep_trunc) {
    const int lane = static_cast<int>(lane_id());
    const int n0 = rs.cnt[2 * r];
    const int n = n0 + rs.cnt[2 * r + 1];
    if (n < rkm) return false;
    const uint64_t t = rs.tau[r];
    uint64_t* gbuf = p.cand + grow * p.cap;
    uint64_t key[KPL];
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
        const int i = q * 32 + lane;
        const int pos = i < n0 ? i : p.cap - 1 - (i - n0);
        key[q] = i < n ? __ldcg(reinterpret_cast<const unsigned long long*>(gbuf) + pos) : KEY_MAX;
    }
#pragma unroll
    for (int q = 0; q < KPL; ++q)
        if (q * 32 + lane < n) es.A[q * 32 + lane] = static_cast<uint32_t>(key[q] >> 32);
    __syncwarp();
    const uint32_t smp = warp_sort32(es.A[(lane * n) >> 5]);
    auto count_le = [&](uint32_t x) {
        int c = 0;
#pragma unroll
        for (int q = 0; q < KPL; ++q) c += static_cast<uint32_t>(key[q] >> 32) <= x ? 1 : 0;  // padding is KEY_MAX
        return static_cast<int>(__reduce_add_sync(0xffffffffu, static_cast<uint32_t>(c)));
    };
    auto passes = [&](uint32_t cand) {
        if (count_le(cand) < rkm) return false;
        return window <= 0.f || count_le(float_to_ord(ord_to_float(cand) - window)) >= rk;
    };
    int s0 = (32 * rkm + n - 1) / n;
    s0 = s0 > 31 ? 31 : s0;
    int sel = -1;
    if (passes(__shfl_sync(0xffffffffu, smp, s0))) {
        sel = s0;
        while (sel > 0 && passes(__shfl_sync(0xffffffffu, smp, sel - 1))) --sel;
    } else {
        for (int s1 = s0 + 1; s1 < 32 && sel < 0; ++s1)
            if (passes(__shfl_sync(0xffffffffu, smp, s1))) sel = s1;
    }
    uint64_t nt = t;
    int keep = n + 1;
    bool trunc = false;
    if (sel >= 0) {
        const uint64_t band = key_ceiling(ord_to_float(__shfl_sync(0xffffffffu, smp, sel)));
        nt = band < t ? band : t;
        keep = 0;
#pragma unroll
        for (int q = 0; q < KPL; ++q) keep += (q * 32 + lane < n && key[q] <= nt) ? 1 : 0;
        keep = static_cast<int>(__reduce_add_sync(0xffffffffu, static_cast<uint32_t>(keep)));
    }
    if (sel >= 0 && keep > keep_max) {
        // the sample value overshoots the band by up to one sample gap: the exact band edge
        // is the smallest value passing, found by bisection on the ordered values between
        // the last failing sample value and the passing one
        uint32_t lo_v = sel > 0 ? __shfl_sync(0xffffffffu, smp, sel - 1) : 0u;  // fails (or below all)
        uint32_t hi_v = __shfl_sync(0xffffffffu, smp, sel);                       // passes
        while (hi_v - lo_v > 1u) {
            const uint32_t mid = lo_v + ((hi_v - lo_v) >> 1);
            if (passes(mid)) hi_v = mid; else lo_v = mid;
        }
        const uint64_t band = key_ceiling(ord_to_float(hi_v));
        nt = band < t ? band : t;
        keep = 0;
#pragma unroll
        for (int q = 0; q < KPL; ++q) keep += (q * 32 + lane < n && key[q] <= nt) ? 1 : 0;
        keep = static_cast<int>(__reduce_add_sync(0xffffffffu, static_cast<uint32_t>(keep)));
    }
    if (keep > keep_max) {
        // the band does not fit: truncate at the largest sample value keeping <= keep_trunc
        int lo = 0, hi = (sel >= 0 ? sel : 32) - 1, best = -1;
        while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            if (count_le(__shfl_sync(0xffffffffu, smp, mid)) <= keep_trunc) {
                best = mid;
                lo = mid + 1;
            } else {
                hi = mid - 1;
            }
        }
        if (best < 0) return false;
        const uint64_t tt = key_ceiling(ord_to_float(__shfl_sync(0xffffffffu, smp, best)));
        nt = tt < t ? tt : t;
        trunc = true;
    }
    const uint32_t lt_mask = lanemask_lt();
    int nn = 0;
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
        const bool kp = q * 32 + lane < n && key[q] <= nt;
        const uint32_t b = __ballot_sync(0xffffffffu, kp);
        if (kp) gbuf[nn + __popc(b & lt_mask)] = key[q];
        nn += __popc(b);
    }
    const bool speculated = (rk < p.k || rkm < p.km) && nt < t;
    __syncwarp();
    if (lane == 0) {
        rs.cnt[2 * r] = static_cast<uint16_t>(nn);
        rs.cnt[2 * r + 1] = 0;
        rs.tau[r] = nt;
        rs.tauf[r] = tau_filter(nt);
        rs.flags[r] |= (speculated ? RS_SPEC : 0u) | (trunc ? RS_TRUNC : 0u);
    }
    __syncwarp();
    return true;
}

// Out-of-line copy for the longest-list variant (48 keys a lane): its keys would otherwise
// count against the register allocation of the whole epilogue loop, which then spills inside
// its filter, while at a shrink only a few of the loop's values are live (lists of 1248 keys
// in a batch: fused launch 112 -> 108 ms).
template <int KPL>
__device__ __noinline__ bool shrink_mid_fast_call(const Item& p, const EpiSmem& es, const RowState& rs, int r,
                                                  int64_t grow, float window, int rk, int rkm, int keep_max,
                                                  int keep_trunc) {
    return shrink_mid_fast_body<KPL>(p, es, rs, r, grow, window, rk, rkm, keep_max, keep_trunc);
}

template <int KPL>
__device__ __forceinline__ bool shrink_mid_fast(const Item& p, const EpiSmem& es, const RowState& rs, int r,
                                                int64_t grow, float window, int rk, int rkm, int keep_max,
                                                int keep_trunc) {
    if constexpr (KPL > 32)
        return shrink_mid_fast_call<KPL>(p, es, rs, r, grow, window, rk, rkm, keep_max, keep_trunc);
    else
        return shrink_mid_fast_body<KPL>(p, es, rs, r, grow, window, rk, rkm, keep_max, keep_trunc);
}

// Value of r[t] for a lane-dependent t (0..31) by a 5-level select tree (no local memory).
__device__ __forceinline__ uint32_t select32(const uint32_t (&r)[32], int t) {
    uint32_t a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = (t & 16) ? r[i + 16] : r[i];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (t & 8) ? a[i + 8] : a[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = (t & 4) ? a[i + 4] : a[i];
#pragma unroll
    for (int i = 0; i < 2; ++i) a[i] = (t & 2) ? a[i + 2] : a[i];
    return (t & 1) ? a[1] : a[0];
}

// Packed FP32 pairs (sm_100 and later): each half is rounded exactly like its scalar
// counterpart, so results match fmaf / __fmul_rn bit for bit.
__device__ __forceinline__ void fma2(float& d0, float& d1, float a0, float a1, float b0, float b1, float c0,
                                     float c1) {
    asm("{\n .reg .b64 A, B, C, D;\n mov.b64 A, {%2, %3};\n mov.b64 B, {%4, %5};\n mov.b64 C, {%6, %7};\n"
        " fma.rn.f32x2 D, A, B, C;\n mov.b64 {%0, %1}, D;\n}\n"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1), "f"(c0), "f"(c1));
}
__device__ __forceinline__ void mul2(float& d0, float& d1, float a0, float a1, float b0, float b1) {
    asm("{\n .reg .b64 A, B, D;\n mov.b64 A, {%2, %3};\n mov.b64 B, {%4, %5};\n"
        " mul.rn.f32x2 D, A, B;\n mov.b64 {%0, %1}, D;\n}\n"
        : "=f"(d0), "=f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
// Three-input minimum (a NaN operand is ignored, as with fminf).
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// The transposed direction of the symmetric graph form for one thread's row i: on a tile
// past row i's own super-block, a column j with v_ij <= tau_j (i.e. squared distance
// <= sym_t) also belongs in row j's inbox, as the key (d'_ji, i).
struct SymCtx {
    bool on;              // this tile feeds the transposed pairs (warp-uniform)
    float tau_j;          // sym_t - |x_i|^2 (-inf for rows past M)
    float qi;             // |x_i|^2
    uint32_t row;         // i
    uint64_t* inbox;
    int32_t* inbox_cnt;
    int32_t cap_in;
};

// Filters one 32-column chunk of the accumulator into the row's candidate list. The
// ranking values v = |c_j|^2 - 2 acc (FP8: acc scaled back first) replace the accumulator
// bits in r (packed pair arithmetic); a tree of three-input minimums gives the lane's
// smallest value, and one warp vote ends the chunk when no lane has a value at or below
// its row's threshold, the common case once thresholds have settled. Otherwise the lanes
// build their survivor masks and take one survivor per round, its value picked from r
// by a select tree, appending it to the lane's segment of the row's list (slot
// base + dir * cnt); the warp runs as many rounds as its lane with the most survivors.
// In the symmetric form the same vote also admits the transposed pairs (sym), which are
// appended to the column rows' inboxes with an atomic slot each; their key value
// (v - |x_j|^2) + |x_i|^2 carries two more roundings than a row's own values, which the
// error bound of symmetric problems includes.
template <int P>
__device__ __forceinline__ void filter_chunk(uint32_t (&r)[32], const float* cn, const float* cs, float qscale,
                                             int64_t j0, int64_t self, float tau_f, uint64_t* gbuf, int& cnt,
                                             int base, int dir, uint32_t& inserted, const SymCtx& sym) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 c = reinterpret_cast<const float4*>(cn)[q];
        float a0 = __uint_as_float(r[4 * q]), a1 = __uint_as_float(r[4 * q + 1]);
        float a2 = __uint_as_float(r[4 * q + 2]), a3 = __uint_as_float(r[4 * q + 3]);
        if constexpr (P == P_FP8) {
            const float4 sc = reinterpret_cast<const float4*>(cs)[q];
            float s0, s1, s2, s3;
            mul2(s0, s1, sc.x, sc.y, qscale, qscale);
            mul2(s2, s3, sc.z, sc.w, qscale, qscale);
            mul2(a0, a1, a0, a1, s0, s1);
            mul2(a2, a3, a2, a3, s2, s3);
        }
        float v0, v1, v2, v3;
        fma2(v0, v1, a0, a1, -2.f, -2.f, c.x, c.y);
        fma2(v2, v3, a2, a3, -2.f, -2.f, c.z, c.w);
        r[4 * q] = __float_as_uint(v0);
        r[4 * q + 1] = __float_as_uint(v1);
        r[4 * q + 2] = __float_as_uint(v2);
        r[4 * q + 3] = __float_as_uint(v3);
    }
    // lane minimum over the 32 values: 10 + 4 + 1 + 1 three- and two-input minimums
    float m[11];
#pragma unroll
    for (int i = 0; i < 10; ++i)
        m[i] = min3f(__uint_as_float(r[3 * i]), __uint_as_float(r[3 * i + 1]), __uint_as_float(r[3 * i + 2]));
    m[10] = fminf(__uint_as_float(r[30]), __uint_as_float(r[31]));
    const float mn = fminf(min3f(min3f(m[0], m[1], m[2]), min3f(m[3], m[4], m[5]), min3f(m[6], m[7], m[8])),
                           fminf(m[9], m[10]));
    const bool any_j = sym.on && __any_sync(0xffffffffu, mn <= sym.tau_j);
    if (any_j) {
        uint32_t mj = 0;
#pragma unroll
        for (int e = 0; e < 32; ++e) mj |= (__uint_as_float(r[e]) <= sym.tau_j) ? (1u << e) : 0u;
        const uint32_t rounds_j = __reduce_max_sync(0xffffffffu, static_cast<uint32_t>(__popc(mj)));
        inserted += static_cast<uint32_t>(__popc(mj));
        for (uint32_t it = 0; it < rounds_j; ++it) {
            const int t = (__ffs(mj) - 1) & 31;
            const bool has = mj != 0u;
            mj &= mj - 1u;
            const float v = __uint_as_float(select32(r, t));
            if (has) {
                const int64_t j = j0 + t;
                const float u = __fadd_rn(__fsub_rn(v, cn[t]), sym.qi);
                const int slot = atomicAdd(sym.inbox_cnt + j, 1);
                if (slot < sym.cap_in) sym.inbox[j * sym.cap_in + slot] = make_key(u, sym.row);
            }
        }
    }
    if (!__any_sync(0xffffffffu, mn <= tau_f)) return;
    uint32_t m8[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        uint32_t mq = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) mq |= (__uint_as_float(r[q * 4 + e]) <= tau_f) ? (1u << e) : 0u;
        m8[q] = mq << (4 * q);
    }
    uint32_t mask = ((m8[0] | m8[1]) | (m8[2] | m8[3])) | ((m8[4] | m8[5]) | (m8[6] | m8[7]));
    const uint64_t ds = static_cast<uint64_t>(self - j0);
    if (ds < 32u) mask &= ~(1u << ds);
    const uint32_t rounds = __reduce_max_sync(0xffffffffu, static_cast<uint32_t>(__popc(mask)));
    inserted += static_cast<uint32_t>(__popc(mask));
    const uint32_t jlo = static_cast<uint32_t>(j0);
    for (uint32_t it = 0; it < rounds; ++it) {
        const int t = (__ffs(mask) - 1) & 31;
        const bool has = mask != 0u;
        mask &= mask - 1u;
        const float v = __uint_as_float(select32(r, t));
        if (has) {
            gbuf[base + dir * cnt] = make_key(v, jlo + static_cast<uint32_t>(t));
            ++cnt;
        }
    }
}

__device__ __forceinline__ void pair_barrier(int quarter) {
    // named barrier 1 + quarter, shared by the two epilogue warps of that lane quarter
    asm volatile("bar.sync %0, 64;" ::"r"(1 + quarter) : "memory");
}

// Waits (bounded) until the epilogue warps' completion count reaches `target` (each
// epilogue warp adds one per finished row block). Called by the whole warp; lane 0 polls.
// False when the kernel is giving up.
__device__ __forceinline__ bool wait_epilogue(const volatile int* ep_done, int target, volatile int* abort_flag,
                                              long long limit) {
    int ok = 0;
    if (lane_id() == 0) {
        for (long long i = 0;; ++i) {
            if (*ep_done >= target) {
                __threadfence_block();  // the lists, counts and flags written before the count was raised
                ok = 1;
                break;
            }
            if (*abort_flag) break;
            if (i >= limit) {
                *abort_flag = 1;
                break;
            }
            __nanosleep(256);
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

template <int P, bool BATCHED, int KPL, int BN>
__global__ void __launch_bounds__(Tile<BN>::THREADS, Tile<BN>::CTAS_PER_SM)
    fused_gemm_select_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                             const FusedParams params) {
    const FusedParams& p = params;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~static_cast<uintptr_t>(1023));
    const int nst = p.stages;
    unsigned char* stage_base = smem;
    constexpr int STAGE = Tile<BN>::STAGE_BYTES;
    unsigned char* epi_base = smem + nst * STAGE;
    float* cn_smem = reinterpret_cast<float*>(epi_base + EPI_WARPS * epi_warp_bytes(p.cap_max));  // [2][BN] (+ scales)
    unsigned char* rs_base = reinterpret_cast<unsigned char*>(cn_smem) + cn_bytes(P, BN);
    RowState rs;
    rs.tau = reinterpret_cast<uint64_t*>(rs_base);
    rs.cnt = reinterpret_cast<uint16_t*>(rs.tau + 128);
    rs.tauf = reinterpret_cast<float*>(rs.cnt + 2 * 128);
    rs.flags = reinterpret_cast<uint32_t*>(rs.tauf + 128);
    uint64_t* bars = reinterpret_cast<uint64_t*>(rs_base + ROWSTATE_BYTES);
    uint64_t* full = bars;                        // [MAX_STAGES]
    uint64_t* empty = bars + MAX_STAGES;          // [MAX_STAGES]
    uint64_t* acc_full = bars + 2 * MAX_STAGES;   // [2]
    uint64_t* acc_empty = acc_full + 2;           // [2]
    uint64_t* drain = acc_empty + 2;              // [1]: completion of every MMA issued
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    int* ep_done = reinterpret_cast<int*>(tmem_holder + 2);  // epilogue warps' finished row blocks
    volatile int* pair_ok = reinterpret_cast<volatile int*>(reinterpret_cast<unsigned char*>(bars) + 128);  // [8]
    unsigned char* rr_base = reinterpret_cast<unsigned char*>(bars) + BAR_BYTES;  // RR_BYTES when p.rr_on
    const long long wait_limit = p.wait_limit > 0 ? p.wait_limit : (1ll << 26);

    const int warp = static_cast<int>(threadIdx.x / 32);
    const uint32_t lane = lane_id();
    const int n_items = p.n_items;
    constexpr uint32_t CN_TX = static_cast<uint32_t>(cn_bytes(P, BN) / 2);  // bytes staged per tile

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 2);  // the norms' copy (arrive + bytes) and the MMA commit
            mbar_init(&acc_empty[a], EPI_WARPS);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        *ep_done = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(Tile<BN>::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    if (warp == 0) {
        // ------------------------------ TMA producer ------------------------------
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            bool ok = true;
            const int kx = TC_BK_BYTES / (P == P_BF16 ? 2 : 1);
            for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
                const Item im = get_item<BATCHED, BN>(p, &tmA, &tmB, it);
                for (int ct = 0; ct < im.nsw && ok; ++ct) {
                    for (int ks = 0; ks < im.nk; ++ks) {
                        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, wait_limit)) {
                            ok = false;
                            break;
                        }
                        unsigned char* a = stage_base + s * STAGE;
                        mbar_expect_tx(&full[s], STAGE);
                        tma_load_2d(a, im.tmA, &full[s], ks * kx, im.rb * TC_BM);
                        tma_load_2d(a + A_BYTES, im.tmB, &full[s], ks * kx, tile_at(im, ct) * BN);
                        if (++s == nst) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                }
            }
            if (ok) {
                // drain: every stage filled has been consumed
                for (int i = 0; i < nst; ++i) {
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, wait_limit)) break;
                    if (++s == nst) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            } else {
                // gave up: still let the copies already issued land before the CTA exits
                for (int i = 0; i < nst; ++i) {
                    if (--s < 0) {
                        s = nst - 1;
                        ph ^= 1u;
                    }
                    for (int spin = 0; spin < (1 << 20); ++spin)
                        if (mbar_try_wait(&full[s], ph)) break;
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------ MMA issuer --------------------------------
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            int tile = 0;
            bool ok = true;
            int copy_acc = -1;  // accumulator whose norms copy is in flight without its commit
            uint32_t copy_ph = 0;
            const int k_per_mma = 32;  // bytes of K per instruction: 16 BF16 or 32 FP8 values
            for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
                const Item im = get_item<BATCHED, BN>(p, &tmA, &tmB, it);
                for (int ct = 0; ct < im.nsw && ok; ++ct, ++tile) {
                    const int acc = tile & 1;
                    const uint32_t acc_ph = static_cast<uint32_t>((tile >> 1) & 1);
                    if (!mbar_wait(&acc_empty[acc], acc_ph ^ 1u, abort_flag, wait_limit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // stage this tile's corpus norms (and FP8 scales) for the epilogue
                    mbar_expect_tx(&acc_full[acc], CN_TX);
                    copy_acc = acc;
                    copy_ph = acc_ph;
                    const int64_t cphys = static_cast<int64_t>(tile_at(im, ct)) * BN;
                    bulk_copy_g2s(cn_smem + acc * BN, im.cnorm2 + cphys, BN * 4, &acc_full[acc]);
                    if constexpr (P == P_FP8)
                        bulk_copy_g2s(cn_smem + 2 * BN + acc * BN, im.c_inv_scale + cphys, BN * 4,
                                      &acc_full[acc]);
                    const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * BN);
                    for (int ks = 0; ks < im.nk; ++ks) {
                        if (!mbar_wait(&full[s], ph, abort_flag, wait_limit)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a_addr = smem_u32(stage_base + s * STAGE);
                        const uint32_t b_addr = a_addr + A_BYTES;
#pragma unroll
                        for (int kk = 0; kk < TC_BK_BYTES / k_per_mma; ++kk) {
                            umma<P, BN>(d_tmem, sdesc(a_addr + kk * k_per_mma), sdesc(b_addr + kk * k_per_mma),
                                    (ks | kk) != 0 ? 1u : 0u);
                        }
                        umma_commit(&empty[s]);
                        if (++s == nst) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                    if (ok) {
                        umma_commit(&acc_full[acc]);
                        copy_acc = -1;
                    }
                }
            }
            if (!ok && copy_acc >= 0) {
                // gave up after staging a tile's norms: arrive in place of the missing commit
                // and let the copy land before the CTA exits
                mbar_arrive(&acc_full[copy_acc]);
                for (int spin = 0; spin < (1 << 20); ++spin)
                    if (mbar_try_wait(&acc_full[copy_acc], copy_ph)) break;
            }
            // every MMA issued completes before the TMEM is freed
            umma_commit(drain);
            for (int spin = 0; spin < (1 << 20); ++spin)
                if (mbar_try_wait(drain, 0)) break;
        }
        __syncwarp();
    } else if (warp < 2 + EPI_WARPS) {
        // ------------------------------ epilogue ----------------------------------
        const int ew = warp - 2;                  // epilogue warp 0..7
        const int quarter = warp & 3;             // TMEM lane quarter this warp may read
        const int half = ew >> 2;                 // which half of every tile's columns
        const int partner_bit = half;             // rows of the quarter this warp compacts: parity == half
        const int row_in_block = quarter * 32 + static_cast<int>(lane);
        EpiSmem es;
        unsigned char* mine = epi_base + static_cast<size_t>(ew) * epi_warp_bytes(p.cap_max);
        es.A = reinterpret_cast<uint32_t*>(mine);
        es.hist = es.A + p.cap_max;
        es.scratch = p.scratch + (static_cast<size_t>(blockIdx.x) * EPI_WARPS + ew) * scratch_words_per_warp(p.cap_max);
        es.B = reinterpret_cast<uint32_t*>(es.scratch);
        int tile = 0;
        bool ok = true;
        uint32_t inserted = 0;  // this lane's insertions (its rows)
        for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
            const Item p = get_item<BATCHED, BN>(params, &tmA, &tmB, it);
            const int rb = p.rb;
            const int nct = p.nsw;
            // room for one half-tile of insertions from both warps: 2 x 64 per row
            const int trigger = p.cap - 128;
            const int keep_mid = p.cap - 160 > p.km ? p.cap - 160 : p.km;
            const int trunc_mid = p.cap / 2 > p.km ? p.cap / 2 : p.km;
            const int64_t grow = static_cast<int64_t>(rb) * TC_BM + row_in_block;
            const bool valid = grow < p.M;
            const int64_t self = !valid ? -1
                                 : p.self_col ? static_cast<int64_t>(p.self_col[grow])
                                 : (p.self_offset >= 0 ? grow + p.self_offset : -1);
            uint64_t tau_thr = KEY_MAX;
            if (valid && p.thr) {
                const float t = p.thr[grow];
                if (t == t && t < F_INF) tau_thr = key_ceiling(t);
            }
            uint32_t flags0 = 0u;
            if (valid && p.spec_d2 < F_INF) {
                // speculative start: a squared distance every row's band is expected to lie below
                const uint64_t ts = key_ceiling(p.spec_d2 - p.qnorm2[grow]);
                if (ts < tau_thr) {
                    tau_thr = ts;
                    flags0 = RS_SPEC;
                }
            }
            if (half == 0) {
                rs.cnt[2 * row_in_block] = 0;
                rs.cnt[2 * row_in_block + 1] = 0;
                rs.tau[row_in_block] = valid ? tau_thr : 0ull;
                rs.tauf[row_in_block] = valid ? tau_filter(tau_thr) : -F_INF;
                rs.flags[row_in_block] = flags0;
            }
            pair_barrier(quarter);
            float tau_f = rs.tauf[row_in_block];
            const float qscale = (P == P_FP8 && valid) ? p.q_inv_scale[grow] : 1.f;
            uint64_t* gbuf = valid ? p.cand + grow * p.cap : nullptr;
            // this warp's segment of the row's list: front (first column half) or back
            const int seg_base = half ? p.cap - 1 : 0;
            const int seg_dir = half ? -1 : 1;
            int my_cnt = 0;
            const float my_window = (valid && p.E) ? 2.f * p.E[grow] : 0.f;  // shuffled to the shrinking warp
            SymCtx sym{};
            const bool sym_item = !BATCHED && params.sym;
            if (sym_item) {
                sym.qi = valid ? p.qnorm2[grow] : 0.f;
                sym.tau_j = valid ? params.sym_t - sym.qi : -F_INF;
                sym.row = static_cast<uint32_t>(grow);
                sym.inbox = params.inbox;
                sym.inbox_cnt = params.inbox_cnt;
                sym.cap_in = params.cap_in;
            }

            for (int ct = 0; ct < nct; ++ct, ++tile) {
                const int acc = tile & 1;
                const uint32_t acc_ph = static_cast<uint32_t>((tile >> 1) & 1);
                // the two warps of a lane quarter meet at named barriers: a warp whose wait
                // gives up still takes the tile's first one, where the pair decides together
                const bool got = mbar_wait_all(&acc_full[acc], acc_ph, abort_flag, wait_limit);
                if (got) tc_fence_after();
                const int c0 = half * (BN / 2);  // first column of this warp's half
                const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                                       static_cast<uint32_t>(acc * BN + c0);
                const float* cn = cn_smem + acc * BN + c0;
                const float* cs = cn_smem + 2 * BN + acc * BN + c0;
                const int64_t jt = static_cast<int64_t>(tile_at(p, ct)) * BN + c0;
                sym.on = sym_item && ct > 0;  // past the row block's own super-block
                uint32_t ra[32], rb2[32];
#pragma unroll 1
                // each step covers 64 columns of each warp's half: two steps a 256-column
                // tile, one a 128-column tile
                for (int hs = 0; hs < BN / 128; ++hs) {
                    if (got) {
                        if constexpr (BN == TC_BN) {
                            // two chunks of 32 columns, the second load overlapping the first filter
                            tmem_ld32(taddr + hs * 64, ra);
                            tmem_ld32_issue(taddr + hs * 64 + 32, rb2);
                            filter_chunk<P>(ra, cn + hs * 64, cs + hs * 64, qscale, jt + hs * 64, self, tau_f, gbuf,
                                            my_cnt, seg_base, seg_dir, inserted, sym);
                            tmem_ld_wait();
                            filter_chunk<P>(rb2, cn + hs * 64 + 32, cs + hs * 64 + 32, qscale, jt + hs * 64 + 32,
                                            self, tau_f, gbuf, my_cnt, seg_base, seg_dir, inserted, sym);
                        } else {
                            // two CTAs an SM: one chunk's registers at a time (the SM's other
                            // CTA covers the load latency)
                            tmem_ld32(taddr + hs * 64, ra);
                            filter_chunk<P>(ra, cn + hs * 64, cs + hs * 64, qscale, jt + hs * 64, self, tau_f, gbuf,
                                            my_cnt, seg_base, seg_dir, inserted, sym);
                            tmem_ld32(taddr + hs * 64 + 32, ra);
                            filter_chunk<P>(ra, cn + hs * 64 + 32, cs + hs * 64 + 32, qscale, jt + hs * 64 + 32,
                                            self, tau_f, gbuf, my_cnt, seg_base, seg_dir, inserted, sym);
                        }
                        if (hs == BN / 128 - 1) {
                            // accumulator and staged norms of this tile no longer needed by this warp
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&acc_empty[acc]);
                        }
                    }
                    // both warps of the quarter have finished this half-tile: shrink full lists
                    rs.cnt[2 * row_in_block + half] = static_cast<uint16_t>(my_cnt);
                    if (hs == 0 && lane == 0) pair_ok[2 * quarter + half] = got ? 1 : 0;
                    pair_barrier(quarter);
                    if (hs == 0 && !(pair_ok[2 * quarter] && pair_ok[2 * quarter + 1])) {
                        ok = false;  // both warps of the pair leave here, after the same barriers
                        break;
                    }
                    const int total = rs.cnt[2 * row_in_block] + rs.cnt[2 * row_in_block + 1];
                    uint32_t need = __ballot_sync(0xffffffffu, valid && total > trigger);
                    need &= partner_bit ? 0xaaaaaaaau : 0x55555555u;
                    if (need) {
                        // target ranks: speculative while only part of the corpus has been seen
                        const int64_t seen = static_cast<int64_t>(ct) * BN + (hs + 1) * 128;
                        const int rk = p.spec ? spec_rank(p.k, seen, p.N) : p.k;
                        const int rkm = p.spec ? spec_rank(p.km, seen, p.N) : p.km;
                        while (need) {
                            const int owner = __ffs(need) - 1;
                            need &= need - 1;
                            const int64_t g = static_cast<int64_t>(rb) * TC_BM + quarter * 32 + owner;
                            const float w = __shfl_sync(0xffffffffu, my_window, owner);
                            if (!shrink_mid_fast<KPL>(p, es, rs, quarter * 32 + owner, g, w, rk, rkm, keep_mid,
                                                      trunc_mid))
                                shrink_row_k<KPL>(p, es, rs, quarter * 32 + owner, g, w, rk, rkm, keep_mid, trunc_mid);
                        }
                    }
                    pair_barrier(quarter);
                    tau_f = rs.tauf[row_in_block];
                    my_cnt = rs.cnt[2 * row_in_block + half];
                }
                if (!ok) break;
            }
            if (!ok) break;
            // row block done: each row's list (both segments, every key <= its threshold)
            // goes to the re-rank, which reduces it to the band of the k-th and (k+m)-th.
            // Lists longer than RAW_LIST_MAX are trimmed here first (to a sampled band
            // threshold, like a shrink with the ranks k and k + m, never truncating), so
            // that the re-rank mostly sorts at most RAW_LIST_MAX keys per row.
            {
                const int total = rs.cnt[2 * row_in_block] + rs.cnt[2 * row_in_block + 1];
                uint32_t need = __ballot_sync(0xffffffffu, valid && total > RAW_LIST_MAX);
                need &= partner_bit ? 0xaaaaaaaau : 0x55555555u;
                while (need) {
                    const int owner = __ffs(need) - 1;
                    need &= need - 1;
                    const int64_t g = static_cast<int64_t>(rb) * TC_BM + quarter * 32 + owner;
                    const float w = __shfl_sync(0xffffffffu, my_window, owner);
                    if (!shrink_mid_fast<KPL>(p, es, rs, quarter * 32 + owner, g, w, p.k, p.km, p.cap, 0))
                        shrink_row_k<KPL>(p, es, rs, quarter * 32 + owner, g, w, p.k, p.km, p.cap, p.cap);
                }
                pair_barrier(quarter);
            }
            if (half == 0 && valid) {
                const int c0 = rs.cnt[2 * row_in_block], c1 = rs.cnt[2 * row_in_block + 1];
                const uint32_t rfl = rs.flags[row_in_block];
                uint32_t fl = ROW_RAW_LIST | ((rfl & RS_TRUNC) ? ROW_TRUNCATED : 0u) |
                              ((rfl & RS_SPEC) ? ROW_SPECULATIVE : 0u);
                // a supplied threshold drops every key above it: the list is truncated there
                // and the re-rank certificate decides whether it held the answer; fewer than
                // k survivors is a miss outright
                if (p.thr) {
                    const float t = p.thr[grow];
                    if (t == t && t < F_INF) {
                        if (params.thr_bound) {
                            // a bound, not a guess: fewer than k keys is no miss, and a list whose
                            // threshold never fell below the bound holds every key at or below it
                            fl |= ROW_TRUNCATED | (rs.tau[row_in_block] >= key_ceiling(t) ? ROW_BOUNDED : 0u);
                        } else {
                            fl |= ROW_TRUNCATED | (c0 + c1 < p.k ? ROW_THRESHOLD_MISS : 0u);
                        }
                    }
                }
                uint64_t bnd = rs.tau[row_in_block];
                if (sym_item) {
                    // keys of the transposed pairs left out have value above sym_t - |x_i|^2 - delta
                    // (delta: the filter's and the key's roundings, each below 2^-24 of a magnitude
                    // of at most 3 max|x|^2 or sym_t)
                    const float c2max = __uint_as_float(*params.c2max_bits);
                    const float delta = 0x1p-20f * (c2max + fabsf(params.sym_t));
                    const uint64_t bi = key_ceiling(__fsub_rd(__fsub_rd(params.sym_t, sym.qi), delta));
                    bnd = bi < bnd ? bi : bnd;
                }
                p.count[grow] = c0 | (c1 << 16);
                p.bound[grow] = bnd;
                p.flags[grow] = fl;
            }
            // the next row block reinitialises the row state only after both warps are done
            pair_barrier(quarter);
            // this warp is done with the row block: the re-rank warps may take it once all are
            if (lane == 0) {
                __threadfence_block();
                atomicAdd(ep_done, 1);
            }
        }
        if (!ok && lane == 0) atomicExch(p.status, static_cast<int>(KNN_ETIMEOUT));
        if (params.inserted) {
            const uint32_t w = __reduce_add_sync(0xffffffffu, inserted);
            if (lane == 0 && w) atomicAdd(params.inserted, static_cast<unsigned long long>(w));
        }
    } else if (!BATCHED && p.rr_on) {
        // ------------------------------ re-rank -----------------------------------
        // The rows of every row block the epilogue has finished, while it sweeps the next
        // one; the CTA's last row block (and any rows not reached when the epilogue ends)
        // are left to the re-rank launch after the kernel, which skips rows marked done.
        const int rw = warp - 2 - EPI_WARPS;
        uint64_t* K = reinterpret_cast<uint64_t*>(rr_base) + static_cast<size_t>(rw) * (RR_P + TIE_MAX);
        double* T64 = reinterpret_cast<double*>(K + RR_P);
        unsigned long long* cnt =
            reinterpret_cast<unsigned long long*>(rr_base + RR_WARPS * static_cast<size_t>(RR_P + TIE_MAX) * 8) +
            rw * RC_COUNT;
        if (lane < RC_COUNT) cnt[lane] = 0ull;
        __syncwarp();
        const int mine = (n_items - static_cast<int>(blockIdx.x) + static_cast<int>(gridDim.x) - 1) /
                         static_cast<int>(gridDim.x);
        const int all_done = EPI_WARPS * mine;
        bool go = true;
        int j = 0;
        for (int it = blockIdx.x; it < n_items && go; it += gridDim.x, ++j) {
            if (!wait_epilogue(ep_done, EPI_WARPS * (j + 1), abort_flag, wait_limit)) break;
            for (int r = rw; r < TC_BM; r += RR_WARPS) {
                const int done = __shfl_sync(0xffffffffu, *reinterpret_cast<volatile int*>(ep_done), 0);
                if (done >= all_done) {
                    go = false;
                    break;
                }
                const int64_t grow = static_cast<int64_t>(item_rb(p, it)) * TC_BM + r;
                if (grow >= p.M) break;
                if (row_keys(p.rr, grow) > RR_P) continue;
                rerank_row<true, 4, 0>(p.rr, grow, RR_P, K, T64, cnt, lane);
            }
        }
        __syncwarp();
        if (lane == 0) flush_rerank_counts(p.rr.counters, cnt, true);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(Tile<BN>::TMEM_COLS)
                     : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicExch(p.status, static_cast<int>(KNN_ETIMEOUT));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
        else
            cudaGetLastError();
    }
    return fn;
}

bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t row_bytes, int box_rows, int elem_bytes) {
    auto fn = encode_fn();
    if (!fn) return false;
    const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(row_bytes / elem_bytes), static_cast<cuuint64_t>(rows)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(row_bytes)};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(TC_BK_BYTES / elem_bytes), static_cast<cuuint32_t>(box_rows)};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool fused_available() {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaGetLastError();
    return major == 10 && minor == 3 && encode_fn() != nullptr;
}

int fused_cap(int k, int km) {
    (void)k;
    int c = 2 * km + 160;
    c = (c + 31) / 32 * 32;
    return c < 448 ? 448 : c;
}

int fused_stages(int cap, int precision, bool rr, int bn) {
    if (cap > FUSED_CAP_MAX) return 0;  // a list is staged as at most 48 keys per lane
    if (bn == 128 && cap > 512) return 0;  // the two-CTA tile exists for the 16-keys-a-lane lists only
    for (int st = MAX_STAGES; st >= 2; --st)
        if (tc_smem_bytes(cap, st, precision, rr, bn) <= smem_budget(bn)) return st;
    return 0;
}

size_t fused_scratch_words(int cap, int grid) {
    return scratch_words_per_warp(cap) * EPI_WARPS * static_cast<size_t>(grid);
}

bool encode_problem_maps(FusedProblem* prob, const void* xq, const void* xc, int precision, int bn) {
    const int elem = precision == P_BF16 ? 2 : 1;
    return make_map(&prob->tmA, xq, prob->M, prob->k_bytes, TC_BM, elem) &&
           make_map(&prob->tmB, xc, prob->N, prob->k_bytes, bn, elem);
}

// Kernel instantiation for a precision, a launch form and the list capacity (keys
// per lane of the register-staged shrink: 16 up to 512 keys, 32 up to 1024, 48 up to 1536).
// The 128-column tile exists for batched launches with lists of at most 512 keys.
template <bool BATCHED>
void (*fused_kernel(int precision, int cap_max, int bn))(const CUtensorMap, const CUtensorMap, const FusedParams) {
    if constexpr (BATCHED) {
        if (bn == 128)
            return precision == P_BF16 ? fused_gemm_select_kernel<P_BF16, true, 16, 128>
                                       : fused_gemm_select_kernel<P_FP8, true, 16, 128>;
    }
    if (precision == P_BF16)
        return cap_max > 1024 ? fused_gemm_select_kernel<P_BF16, BATCHED, 48, TC_BN>
               : cap_max > 512 ? fused_gemm_select_kernel<P_BF16, BATCHED, 32, TC_BN>
                               : fused_gemm_select_kernel<P_BF16, BATCHED, 16, TC_BN>;
    return cap_max > 1024 ? fused_gemm_select_kernel<P_FP8, BATCHED, 48, TC_BN>
           : cap_max > 512 ? fused_gemm_select_kernel<P_FP8, BATCHED, 32, TC_BN>
                           : fused_gemm_select_kernel<P_FP8, BATCHED, 16, TC_BN>;
}

cudaError_t launch_fused_batched(const FusedParams& p, int precision, int grid, cudaStream_t st, int bn) {
    if (p.n_items <= 0) return cudaSuccess;
    if (p.cap_max > FUSED_CAP_MAX || (bn != TC_BN && (bn != 128 || p.cap_max > 512))) return cudaErrorInvalidValue;
    CUtensorMap dummy{};
    const size_t smem = tc_smem_bytes(p.cap_max, p.stages, precision, false, bn);
    if (smem > smem_budget(bn)) return cudaErrorInvalidValue;
    auto kern = fused_kernel<true>(precision, p.cap_max, bn);
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(kern), static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, bn == 128 ? Tile<128>::THREADS : Tile<TC_BN>::THREADS, smem, st>>>(dummy, dummy, p);
    return cudaGetLastError();
}

cudaError_t launch_fused(const FusedParams& p, int precision, int grid, cudaStream_t st) {
    if (p.M <= 0) return cudaSuccess;
    if (p.cap_max > FUSED_CAP_MAX) return cudaErrorInvalidValue;
    const int elem = precision == P_BF16 ? 2 : 1;
    CUtensorMap ta, tb;
    if (!make_map(&ta, p.xq, p.M, p.k_bytes, TC_BM, elem)) return cudaErrorInvalidValue;
    if (!make_map(&tb, p.xc, p.N, p.k_bytes, TC_BN, elem)) return cudaErrorInvalidValue;
    const size_t smem = tc_smem_bytes(p.cap_max, p.stages, precision, p.rr_on != 0);
    if (smem > 232448) return cudaErrorInvalidValue;
    auto kern = fused_kernel<false>(precision, p.cap_max, TC_BN);
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(kern), static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, TC_THREADS, smem, st>>>(ta, tb, p);
    return cudaGetLastError();
}

}  // namespace knn
