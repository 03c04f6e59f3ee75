// Unfused quick multi-select over a materialised distance matrix.
//
// Paper: Methods, "GPU-based quick multi-select". One warp owns one row of the
// distance matrix. The row is streamed once from HBM with coalesced 16-byte loads;
// a running threshold tau acts as the pivot of that first partition: each 32-wide
// group votes with a ballot on "key <= tau" and the survivors are written, at
// offsets taken from popc of the lower lanes' bits, into a shared-memory buffer
// (the left part; the right part is discarded since only the K smallest are
// wanted, the K < L branch of the recursion). When the buffer fills, the warp runs
// the quick multi-select of select_core.cuh on it (ballot partitions, ping-pong
// between two shared-memory arrays, a reference list instead of copies) to find the
// k-th and (k+m)-th smallest keys, and tau shrinks to
//     max(key_(k+m), ceiling(value(key_k) + window)),
// where window is twice the row's bound on the error of the matrix values. Every key
// dropped is therefore larger than the final tau, and the kept keys include every
// point whose exact distance can still be among the k smallest (the band argument
// in the design notes). Output per row: the candidate keys, their count, tau
// (every left-out key is > tau) and flags.
#include <atomic>
#include <cstdlib>

#include "internal.h"
#include "select_core.cuh"

namespace knn {
namespace {

constexpr int SEL_U = 8;                 // 16-byte loads per lane per step
constexpr int STEP = 32 * 4 * SEL_U;     // values per warp and step
constexpr int BW = 8;                    // warps per row of the block-per-row select

struct RowBuffers {
    uint64_t* A;
    uint64_t* B;
    int* seg_s;
    uint32_t* seg_e;
};

__host__ __device__ constexpr size_t warp_smem_bytes(int bufk) {
    return static_cast<size_t>(bufk) * 16 + static_cast<size_t>(SEG_MAX) * 8;
}

// One step of a row into v (value 4u + c of a lane is column base + (32u + lane) 4 + c).
// Full steps of 16-byte aligned rows take 16-byte streaming loads; the last step is
// loaded value by value, NaN past the row end (NaN never passes a threshold compare).
template <bool VEC>
__device__ __forceinline__ void load_step(const float* rowp, int64_t N, int64_t base, float (&v)[4 * SEL_U]) {
    const uint32_t lane = lane_id();
    if (VEC && base + STEP <= N) {
#pragma unroll
        for (int u = 0; u < SEL_U; ++u) {
            const float4 f = ldg_stream_f4(rowp + base + (static_cast<int64_t>(u) * 32 + lane) * 4);
            v[4 * u] = f.x;
            v[4 * u + 1] = f.y;
            v[4 * u + 2] = f.z;
            v[4 * u + 3] = f.w;
        }
    } else {
#pragma unroll
        for (int u = 0; u < SEL_U; ++u)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t idx = base + (static_cast<int64_t>(u) * 32 + lane) * 4 + c;
                v[4 * u + c] = idx < N ? rowp[idx] : __int_as_float(0x7fffffff);
            }
    }
}

// Three-input minimum (a NaN operand is ignored, as with fminf).
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// v[t] for a lane-dependent t (0..31) by a 5-level select tree (no local memory).
__device__ __forceinline__ float select32f(const float (&v)[32], int t) {
    float a[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = (t & 16) ? v[i + 16] : v[i];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (t & 8) ? a[i + 8] : a[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = (t & 4) ? a[i + 4] : a[i];
#pragma unroll
    for (int i = 0; i < 2; ++i) a[i] = (t & 2) ? a[i + 2] : a[i];
    return (t & 1) ? a[1] : a[0];
}

// Survivor bits of a lane's 32 values of a step (bit 4u + c), value <= thr, the
// excluded self column cleared. NaN never passes.
__device__ __forceinline__ uint32_t step_bits(const float (&v)[32], float thr, int64_t base, int64_t self_col) {
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) m |= (v[i] <= thr) ? (1u << i) : 0u;
    const uint64_t off = static_cast<uint64_t>(self_col - base);
    if (off < static_cast<uint64_t>(STEP) && static_cast<uint32_t>((off & 127) >> 2) == lane_id())
        m &= ~(1u << (((off >> 7) << 2) + (off & 3)));
    return m;
}

// Fast path of a shrink of A[0, n) (shared memory): a 32-key sample of the values,
// sorted across the lanes, proposes thresholds; the smallest sample value with at least
// rkm values at or below it and at least rk at or below it minus the window is taken (so
// it is >= max(v_rkm, v_rk + window)), clamped by tau, and the keys above it are
// compacted away in place with ballot/popc. Returns false, leaving A untouched, when no
// sample value passes or more than keep_max keys would remain.
__device__ __forceinline__ bool shrink_fast(uint64_t* A, int& n, uint64_t& tau, int rk, int rkm, float window,
                                            int keep_max) {
    const uint32_t lane = lane_id();
    if (n < rkm) return false;
    const uint32_t smp = warp_sort32(static_cast<uint32_t>(A[(static_cast<int64_t>(lane) * n) >> 5] >> 32));
    auto count_le = [&](uint32_t x) {
        int c = 0;
        for (int i = static_cast<int>(lane); i < n; i += 32) c += static_cast<uint32_t>(A[i] >> 32) <= x ? 1 : 0;
        return __reduce_add_sync(0xffffffffu, static_cast<uint32_t>(c));
    };
    auto passes = [&](uint32_t cand) {
        if (count_le(cand) < static_cast<uint32_t>(rkm)) return false;
        return window <= 0.f || count_le(float_to_ord(ord_to_float(cand) - window)) >= static_cast<uint32_t>(rk);
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
    if (sel < 0) return false;
    const uint64_t band = key_ceiling(ord_to_float(__shfl_sync(0xffffffffu, smp, sel)));
    const uint64_t nt = band < tau ? band : tau;
    int keep = 0;
    for (int i = static_cast<int>(lane); i < n; i += 32) keep += A[i] <= nt ? 1 : 0;
    keep = static_cast<int>(__reduce_add_sync(0xffffffffu, static_cast<uint32_t>(keep)));
    if (keep > keep_max) return false;
    // in place: a lane writes at or below the positions this round has already read
    const uint32_t lt = lanemask_lt();
    int nn = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + static_cast<int>(lane);
        const uint64_t key = i < n ? A[i] : KEY_MAX;
        const bool kp = key <= nt;
        const uint32_t b = __ballot_sync(0xffffffffu, kp);
        if (kp) A[nn + __popc(b & lt)] = key;
        nn += __popc(b);
    }
    __syncwarp();
    n = nn;
    tau = nt;
    return true;
}

// Streams one row, keeping keys <= tau in A. The next step's loads are issued before the
// current step is filtered. Per step a lane takes the minimum of its 32 values and one
// warp vote decides whether any lane may hold a survivor; only then are survivor bits
// built and inserted, one per lane and round at ballot/popc offsets, the buffer shrunk
// first whenever a round could overflow it (speculative ranks while only part of the
// row has been seen). When the sampled shrink cannot decide, the scan leaves its loop,
// runs the exact quick multi-select and resumes the same step with the survivor bits it
// had not inserted yet (the hot loop holds no call). Returns false on a reference-list
// overflow. n, tau, truncated are updated in place.
template <bool VEC, bool CHECK_NAN>
__device__ __forceinline__ bool scan_row(const float* rowp, int64_t N, int64_t self_col, const RowBuffers& rb,
                                         int bufk, int k, int km, float window, bool spec, int& n, uint64_t& tau,
                                         bool& truncated, bool& nan_seen, bool& spec_used) {
    const uint32_t lane = lane_id();
    const uint32_t lt = lanemask_lt();
    const int keep_mid = bufk - 160 > km ? bufk - 160 : km;
    const int trunc_mid = (bufk / 2) > km ? bufk / 2 : km;
    float thr = tau_filter(tau);
    float cur[4 * SEL_U], nxt[4 * SEL_U];
    int64_t base = 0;
    uint32_t pending = 0;  // survivor bits of step `base` left when the scan stopped for an exact shrink
    bool resume = false;
    while (base < N) {
        bool need_exact = false;
        int rk = k, rkm = km;
        load_step<VEC>(rowp, N, base, cur);
        for (; base < N; base += STEP) {
            if (base + STEP < N) load_step<VEC>(rowp, N, base + STEP, nxt);
            uint32_t mask;
            if (resume) {
                mask = pending & step_bits(cur, thr, base, self_col);
                resume = false;
            } else {
                if (CHECK_NAN) {
                    bool bad = false;
                    if (base + STEP <= N) {
#pragma unroll
                        for (int i = 0; i < 32; ++i) bad |= cur[i] != cur[i];
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            bad |= (cur[i] != cur[i]) && (base + ((i >> 2) * 32 + lane) * 4 + (i & 3) < N);
                    }
                    nan_seen |= bad;
                }
                float m[11];
#pragma unroll
                for (int i = 0; i < 10; ++i) m[i] = min3f(cur[3 * i], cur[3 * i + 1], cur[3 * i + 2]);
                m[10] = fminf(cur[30], cur[31]);
                const float mn = fminf(
                    min3f(min3f(m[0], m[1], m[2]), min3f(m[3], m[4], m[5]), min3f(m[6], m[7], m[8])),
                    fminf(m[9], m[10]));
                mask = __any_sync(0xffffffffu, mn <= thr) ? step_bits(cur, thr, base, self_col) : 0u;
            }
            while (__any_sync(0xffffffffu, mask != 0u)) {
                if (n + 32 > bufk) {
                    // a round could overflow the buffer: shrink first
                    rk = spec ? spec_rank(k, base, N) : k;
                    rkm = spec ? spec_rank(km, base, N) : km;
                    const uint64_t before = tau;
                    if (!shrink_fast(rb.A, n, tau, rk, rkm, window, keep_mid)) {
                        need_exact = true;
                        pending = mask;
                        break;
                    }
                    if ((rk < k || rkm < km) && tau < before) spec_used = true;
                    thr = tau_filter(tau);
                    mask &= step_bits(cur, thr, base, self_col);
                    continue;
                }
                const int t = (__ffs(mask) - 1) & 31;
                const bool has = mask != 0u;
                mask &= mask - 1u;
                const float v = select32f(cur, t);
                const uint32_t b = __ballot_sync(0xffffffffu, has);
                if (has)
                    rb.A[n + __popc(b & lt)] =
                        make_key(v, static_cast<uint32_t>(base + ((t >> 2) * 32 + lane) * 4 + (t & 3)));
                n += __popc(b);
            }
            if (need_exact) break;
#pragma unroll
            for (int i = 0; i < 32; ++i) cur[i] = nxt[i];
        }
        if (!need_exact) break;
        // exact quick multi-select shrink, then resume step `base` with the pending bits
        __syncwarp();
        const uint64_t before = tau;
        CompactResult r = compact_row(rb.A, rb.B, rb.seg_s, rb.seg_e, n, rk, rkm, window, tau, keep_mid, trunc_mid);
        if (!r.ok) return false;
        n = r.n;
        tau = r.tau;
        truncated |= r.truncated;
        if ((rk < k || rkm < km) && tau < before) spec_used = true;
        thr = tau_filter(tau);
        resume = true;
    }
    __syncwarp();
    return true;
}

template <bool VEC, bool CHECK_NAN, bool TOPK>
__global__ void __launch_bounds__(256, 2) select_rows_kernel(SelectParams p, int bufk, int64_t self_offset, int32_t* __restrict__ out_idx,
                                   float* __restrict__ out_val) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = static_cast<int>(threadIdx.x / 32);
    const int warps = static_cast<int>(blockDim.x / 32);
    const int64_t row = static_cast<int64_t>(blockIdx.x) * warps + warp;
    if (row >= p.M) return;
    const uint32_t lane = lane_id();
    unsigned char* mine = smem_raw + static_cast<size_t>(warp) * warp_smem_bytes(bufk);
    RowBuffers rb;
    rb.A = reinterpret_cast<uint64_t*>(mine);
    rb.B = rb.A + bufk;
    rb.seg_s = reinterpret_cast<int*>(rb.B + bufk);
    rb.seg_e = reinterpret_cast<uint32_t*>(rb.seg_s + SEG_MAX);

    const float* rowp = p.D + row * p.ldd;
    const float window = p.E ? 2.f * p.E[row] : 0.f;
    const int64_t self_col = p.self_col ? static_cast<int64_t>(p.self_col[row])
                                        : (self_offset >= 0 ? row + self_offset : -1);
    uint64_t tau_thr = KEY_MAX;
    if (p.thr) {
        const float t = p.thr[row];
        if (t == t && t < F_INF) tau_thr = key_ceiling(t);
    }
    uint32_t flags = 0;
    bool nan_seen = false;
    bool spec = p.spec != 0;
    for (int attempt = 0; attempt < 3; ++attempt) {
        int n = 0;
        uint64_t tau = tau_thr;
        bool truncated = false;
        bool spec_used = false;
        bool ok = scan_row<VEC, CHECK_NAN>(rowp, p.N, self_col, rb, bufk, p.k, p.km, window, spec, n, tau,
                                           truncated, nan_seen, spec_used);
        CompactResult r{};
        if (ok && n > 0) {
            r = compact_row(rb.A, rb.B, rb.seg_s, rb.seg_e, n, p.k, p.km, window, tau, p.cap, p.cap);
            ok = r.ok;
        } else {
            r.n = 0;
            r.tau = tau;
            r.band = KEY_MAX;
            r.ok = ok;
        }
        if (ok && spec_used && (r.band > tau || n < p.km)) {
            // a speculative threshold cut into the band: select the row again without it
            spec = false;
            continue;
        }
        if (!ok) {
            flags |= ROW_SELECT_ERROR;
            r.n = 0;
        }
        truncated |= r.truncated;
        if (tau_thr != KEY_MAX && ok && (r.n < p.k || r.band > tau_thr)) {
            // the supplied threshold cut into the answer or its band: plain multi-select instead
            flags |= ROW_THRESHOLD_MISS;
            tau_thr = KEY_MAX;
            continue;
        }
        if (CHECK_NAN && __any_sync(0xffffffffu, nan_seen)) flags |= ROW_SELECT_ERROR;
        if constexpr (TOPK) {
            const int kk = r.n < p.k ? r.n : p.k;
            const int P = pow2_ceil(kk > 1 ? kk : 1);
            for (int i = static_cast<int>(lane); i < P; i += 32)
                if (i >= kk) rb.A[i] = KEY_MAX;
            __syncwarp();
            warp_bitonic_sort_smem(rb.A, P);
            for (int i = static_cast<int>(lane); i < p.k; i += 32) {
                const bool have = i < kk;
                out_idx[row * p.k + i] = have ? static_cast<int32_t>(key_idx(rb.A[i])) : -1;
                out_val[row * p.k + i] = have ? key_val(rb.A[i]) : F_INF;
            }
            if (lane == 0) p.flags[row] = flags | (truncated ? ROW_TRUNCATED : 0u);
        } else {
            uint64_t* dst = p.cand + row * p.cap;
            for (int i = static_cast<int>(lane); i < r.n; i += 32) dst[i] = rb.A[i];
            if (lane == 0) {
                p.count[row] = r.n;
                p.bound[row] = r.tau;
                p.flags[row] = flags | (truncated ? ROW_TRUNCATED : 0u);
            }
        }
        return;
    }
}

template <bool VEC, bool CHECK_NAN, bool TOPK>
cudaError_t launch_variant(const SelectParams& p, int bufk, int64_t self_offset, int32_t* out_idx, float* out_val,
                           cudaStream_t st) {
    const size_t per_warp = warp_smem_bytes(bufk);
    int warps = static_cast<int>((96u * 1024u) / per_warp);
    if (warps > 8) warps = 8;
    if (warps < 1) warps = 1;
    const size_t smem = per_warp * warps;
    auto kern = select_rows_kernel<VEC, CHECK_NAN, TOPK>;
    // the attribute is per device and only grows: set it when this device has not seen this size
    static std::atomic<int> smem_set[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || static_cast<int>(smem) > smem_set[dev].load(std::memory_order_relaxed)) {
        e = raise_smem_limit(reinterpret_cast<const void*>(kern), static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) smem_set[dev].store(static_cast<int>(smem), std::memory_order_relaxed);
    }
    const int64_t blocks = (p.M + warps - 1) / warps;
    kern<<<static_cast<unsigned>(blocks), warps * 32, smem, st>>>(p, bufk, self_offset, out_idx, out_val);
    return cudaGetLastError();
}

int choose_bufk(int km, int cap) {
    int want = 2 * km + 288;
    if (want < cap + 64) want = cap + 64;
    int b = pow2_ceil(want);
    return b < 512 ? 512 : b;
}

}  // namespace

// self_offset < 0: nothing excluded; otherwise column row + self_offset is skipped.
cudaError_t launch_select_ex(const SelectParams& p, int64_t self_offset, bool check_nan, cudaStream_t st) {
    if (p.M <= 0) return cudaSuccess;
    const int bufk = choose_bufk(p.km, p.cap);
    const bool vec = (p.ldd % 4 == 0) && (reinterpret_cast<uintptr_t>(p.D) % 16 == 0);
    if (vec) {
        return check_nan ? launch_variant<true, true, false>(p, bufk, self_offset, nullptr, nullptr, st)
                         : launch_variant<true, false, false>(p, bufk, self_offset, nullptr, nullptr, st);
    }
    return check_nan ? launch_variant<false, true, false>(p, bufk, self_offset, nullptr, nullptr, st)
                     : launch_variant<false, false, false>(p, bufk, self_offset, nullptr, nullptr, st);
}

cudaError_t launch_select(const SelectParams& p, cudaStream_t st) { return launch_select_ex(p, -1, false, st); }

namespace {
// Merge of a row's S segment answers (k (value, segment-local index) pairs each) into the
// row's k smallest: one warp per row sorts the S k keys (value, global index) in shared
// memory; the order is the unsplit select's order.
__global__ void select_merge_kernel(const int32_t* __restrict__ seg_idx, const float* __restrict__ seg_val,
                                    const uint32_t* __restrict__ seg_flags, int64_t M, int32_t S, int32_t k,
                                    int64_t seg_len, int32_t P, int32_t* __restrict__ out_idx,
                                    float* __restrict__ out_val, uint32_t* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = static_cast<int>(threadIdx.x / 32);
    const int64_t row = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + warp;
    if (row >= M) return;
    const uint32_t lane = lane_id();
    uint64_t* K = reinterpret_cast<uint64_t*>(smem_raw) + static_cast<size_t>(warp) * P;
    const int n = S * k;
    uint32_t fl = 0;
    for (int i = static_cast<int>(lane); i < P; i += 32) {
        if (i < n) {
            const int s = i / k;
            const int64_t src = (row * S + s) * static_cast<int64_t>(k) + (i - s * k);
            const int32_t j = seg_idx[src];
            K[i] = j < 0 ? KEY_MAX : make_key(seg_val[src], static_cast<uint32_t>(j + s * seg_len));
        } else {
            K[i] = KEY_MAX;
        }
    }
    for (int s = static_cast<int>(lane); s < S; s += 32) fl |= seg_flags[row * S + s];
    fl = __reduce_or_sync(0xffffffffu, fl);
    __syncwarp();
    warp_bitonic_sort_smem(K, P);
    for (int i = static_cast<int>(lane); i < k; i += 32) {
        const bool have = K[i] != KEY_MAX;
        out_idx[row * k + i] = have ? static_cast<int32_t>(key_idx(K[i])) : -1;
        out_val[row * k + i] = have ? key_val(K[i]) : F_INF;
    }
    if (lane == 0) flags[row] = fl;
}
}  // namespace

namespace {
// Row r's answer from a select over the concatenation of its S segment answers: column c of
// that concatenation is entry c mod k of segment c / k, whose segment-local index gets the
// segment's offset. The concatenation keeps equal values in increasing global index order,
// so the lower-index tie rule carries over.
__global__ void select_remap_kernel(const int32_t* __restrict__ merged_col, const int32_t* __restrict__ seg_idx,
                                    const uint32_t* __restrict__ seg_flags, int64_t M, int32_t S, int32_t k,
                                    int64_t seg_len, int32_t* __restrict__ out_idx, uint32_t* __restrict__ flags) {
    const int64_t row = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
    if (row >= M) return;
    const uint32_t lane = lane_id();
    for (int i = static_cast<int>(lane); i < k; i += 32) {
        const int32_t c = merged_col[row * k + i];
        int32_t j = -1;
        if (c >= 0) {
            const int32_t s = c / k;
            const int32_t js = seg_idx[row * S * static_cast<int64_t>(k) + c];
            j = js < 0 ? -1 : static_cast<int32_t>(js + s * seg_len);
        }
        out_idx[row * k + i] = j;
    }
    uint32_t fl = 0;
    for (int s = static_cast<int>(lane); s < S; s += 32) fl |= seg_flags[row * S + s];
    fl = __reduce_or_sync(0xffffffffu, fl);
    if (lane == 0) flags[row] |= fl;
}
}  // namespace

cudaError_t launch_select_remap(const int32_t* merged_col, const int32_t* seg_idx, const uint32_t* seg_flags,
                                int64_t M, int32_t S, int32_t k, int64_t seg_len, int32_t* out_idx, uint32_t* flags,
                                cudaStream_t st) {
    if (M <= 0) return cudaSuccess;
    const int warps = 8;
    select_remap_kernel<<<static_cast<unsigned>((M + warps - 1) / warps), warps * 32, 0, st>>>(
        merged_col, seg_idx, seg_flags, M, S, k, seg_len, out_idx, flags);
    return cudaGetLastError();
}

int select_split_segments(int64_t M, int64_t N, int64_t ldd, int32_t k, const void* D) {
    // few rows: one warp per row would leave most of the GPU idle (the paper switches to a
    // thread block per row for few queries); dense rows split into S equal segments
    constexpr int64_t WARPS_WANTED = 152 * 16;
    const int64_t wr = select_prefers_block(M, k) ? BW : 1;  // warps per row
    if (ldd != N || M * wr * 4 >= WARPS_WANTED || reinterpret_cast<uintptr_t>(D) % 16 != 0) return 1;
    int S = 1;
    while (S < 64 && M * wr * S * 2 <= WARPS_WANTED && N % (2 * S) == 0 && (N / (2 * S)) % 4 == 0 &&
           N / (2 * S) >= 8192 && N / (2 * S) >= 8 * static_cast<int64_t>(k))
        S *= 2;
    return S;
}

cudaError_t launch_select_merge(const int32_t* seg_idx, const float* seg_val, const uint32_t* seg_flags, int64_t M,
                                int32_t S, int32_t k, int64_t seg_len, int32_t* out_idx, float* out_val,
                                uint32_t* flags, cudaStream_t st) {
    if (M <= 0) return cudaSuccess;
    const int P = pow2_ceil(S * k > 32 ? S * k : 32);
    const int warps = 4;
    const size_t smem = static_cast<size_t>(warps) * P * 8;
    cudaError_t e = raise_smem_limit(reinterpret_cast<const void*>(select_merge_kernel), static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    select_merge_kernel<<<static_cast<unsigned>((M + warps - 1) / warps), warps * 32, smem, st>>>(
        seg_idx, seg_val, seg_flags, M, S, k, seg_len, P, out_idx, out_val, flags);
    return cudaGetLastError();
}

int select_spec(int64_t N) {
    if (const char* e = std::getenv("KNN_SPECULATE")) return std::atoi(e) != 0 && N >= 2 * 32 * 4 * SEL_U ? 1 : 0;
    return N >= 16384 ? 1 : 0;
}

namespace {
// ---------------------------------------------------------------------------
// Block-per-row select (the paper's variant for long rows and few queries): the
// BW warps of a CTA share one candidate buffer, so a large k costs one buffer per
// row instead of one per warp.
// ---------------------------------------------------------------------------
constexpr int BSEG_MAX = 48;   // kept-part references before they are gathered back into A

struct BlockShared {
    int cnt[BW];               // per-warp counts (survivors, or keys < pivot in a partition)
    int cnt2[BW];              // keys > pivot in a partition
    int seg_lo[BSEG_MAX];      // kept position ranges whose keys live in B
    int seg_hi[BSEG_MAX];
    uint64_t key;              // broadcast of a selected key
    uint32_t nan;
};

__host__ __device__ constexpr size_t block_smem_bytes(int bufk) {
    return static_cast<size_t>(bufk) * 16 + sizeof(BlockShared);
}

int block_bufk(int k) {
    int want = 2 * k + 288;
    if (want < k + STEP) want = k + STEP;
    return pow2_ceil(want);
}

// Gathers the kept ranges recorded in B back into A (positions unchanged).
__device__ __forceinline__ void block_gather_segments(uint64_t* A, const uint64_t* B, BlockShared& sh, int nseg) {
    for (int t = 0; t < nseg; ++t)
        for (int i = sh.seg_lo[t] + static_cast<int>(threadIdx.x); i < sh.seg_hi[t]; i += blockDim.x) A[i] = B[i];
}

// Block-wide quick multi-select: afterwards A[0, r + 1) holds the r + 1 smallest keys of
// A[0, n) (unique keys, any order); returns the largest of them (rank r). Each step
// partitions the live range around a pivot into the other array: every warp counts the
// keys below and above the pivot in its slice, an inter-warp prefix of the counts gives
// each warp its write offsets, and the warp writes with ballot/popc (smaller keys from
// the left end, larger from the right end). Recursion continues on the side holding
// rank r; a left part that stays kept is recorded by reference, not copied. All threads
// of the block call it.
__device__ uint64_t block_select_prefix(uint64_t* A, uint64_t* B, int n, int r, BlockShared& sh) {
    const int warp = static_cast<int>(threadIdx.x >> 5);
    const uint32_t lane = lane_id();
    const uint32_t lt_mask = lanemask_lt();
    int lo = 0, hi = n, nseg = 0;
    bool in_b = false;
    uint64_t result = KEY_MAX;
    for (int guard = 0; guard < 1 << 20; ++guard) {
        const int len = hi - lo;
        uint64_t* src = in_b ? B : A;
        uint64_t* dst = in_b ? A : B;
        if (len <= 32) {
            if (warp == 0) {
                uint64_t v = static_cast<int>(lane) < len ? src[lo + lane] : KEY_MAX;
                v = warp_sort32(v);
                if (static_cast<int>(lane) < len) src[lo + lane] = v;
                const uint64_t kr = shfl_u64(v, r - lo);
                if (lane == 0) sh.key = kr;
            }
            if (in_b && threadIdx.x == 0) {
                sh.seg_lo[nseg] = lo;
                sh.seg_hi[nseg] = r + 1;
            }
            nseg += in_b ? 1 : 0;
            __syncthreads();
            result = sh.key;
            break;
        }
        const uint32_t h0 = mix32(static_cast<uint32_t>(lo) * 0x9e3779b1u + static_cast<uint32_t>(hi) +
                                  static_cast<uint32_t>(guard) * 0x85ebca6bu);
        const uint32_t ul = static_cast<uint32_t>(len);
        const uint64_t pivot =
            median3(src[lo + h0 % ul], src[lo + mix32(h0) % ul], src[lo + mix32(h0 ^ 0x5bd1e995u) % ul]);
        const int cs = ((len + BW - 1) / BW + 31) & ~31;
        const int w0 = lo + warp * cs;
        const int w1 = min(hi, w0 + cs);
        int nl = 0, ng = 0;
        for (int i = w0 + static_cast<int>(lane); i < w1; i += 32) {
            const uint64_t v = src[i];
            nl += v < pivot ? 1 : 0;
            ng += v > pivot ? 1 : 0;
        }
        nl = static_cast<int>(__reduce_add_sync(0xffffffffu, static_cast<uint32_t>(nl)));
        ng = static_cast<int>(__reduce_add_sync(0xffffffffu, static_cast<uint32_t>(ng)));
        if (lane == 0) {
            sh.cnt[warp] = nl;
            sh.cnt2[warp] = ng;
        }
        __syncthreads();
        int off_l = 0, off_g = 0, tot_l = 0;
#pragma unroll
        for (int w = 0; w < BW; ++w) {
            off_l += w < warp ? sh.cnt[w] : 0;
            off_g += w < warp ? sh.cnt2[w] : 0;
            tot_l += sh.cnt[w];
        }
        int wl = lo + off_l, wg = hi - 1 - off_g;
        for (int i0 = w0; i0 < w1; i0 += 32) {
            const int i = i0 + static_cast<int>(lane);
            const uint64_t v = i < w1 ? src[i] : pivot;
            const bool l = i < w1 && v < pivot;
            const bool g = i < w1 && v > pivot;
            const uint32_t bl = __ballot_sync(0xffffffffu, l);
            const uint32_t bg = __ballot_sync(0xffffffffu, g);
            if (l) dst[wl + __popc(bl & lt_mask)] = v;
            if (g) dst[wg - __popc(bg & lt_mask)] = v;
            if (i < w1 && v == pivot) dst[lo + tot_l] = v;
            wl += __popc(bl);
            wg -= __popc(bg);
        }
        __syncthreads();
        const int m = lo + tot_l;  // the pivot's position (its rank)
        if (r < m) {
            hi = m;
            in_b = !in_b;
            continue;
        }
        // [lo, m] is kept; it lives in dst
        if (!in_b) {  // dst is B
            if (threadIdx.x == 0) {
                sh.seg_lo[nseg] = lo;
                sh.seg_hi[nseg] = m + 1;
            }
            ++nseg;
        }
        if (r == m) {
            result = pivot;
            break;
        }
        lo = m + 1;
        in_b = !in_b;
        if (nseg == BSEG_MAX) {
            __syncthreads();
            block_gather_segments(A, B, sh, nseg);
            nseg = 0;
            __syncthreads();
        }
    }
    __syncthreads();
    block_gather_segments(A, B, sh, nseg);
    __syncthreads();
    return result;
}

// Ascending bitonic sort of A[0, P) by the whole block (P a power of two).
__device__ __forceinline__ void block_bitonic_sort(uint64_t* A, int P) {
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = static_cast<int>(threadIdx.x); i < (P >> 1); i += blockDim.x) {
                const int pos = 2 * i - (i & (stride - 1));
                const int other = pos + stride;
                const bool up = (pos & size) == 0;
                const uint64_t a = A[pos], b = A[other];
                if ((a > b) == up) {
                    A[pos] = b;
                    A[other] = a;
                }
            }
            __syncthreads();
        }
}

// Inserts a warp's survivor bits at A[at, ...) (ballot/popc offsets, one key per lane and round).
__device__ __forceinline__ void block_insert(uint64_t* A, const float (&cur)[32], uint32_t mask, int at, int64_t base) {
    const uint32_t lane = lane_id();
    const uint32_t lt = lanemask_lt();
    while (__any_sync(0xffffffffu, mask != 0u)) {
        const int t = (__ffs(mask) - 1) & 31;
        const bool has = mask != 0u;
        mask &= mask - 1u;
        const float v = select32f(cur, t);
        const uint32_t b = __ballot_sync(0xffffffffu, has);
        if (has) A[at + __popc(b & lt)] = make_key(v, static_cast<uint32_t>(base + ((t >> 2) * 32 + lane) * 4 + (t & 3)));
        at += __popc(b);
    }
}

// The k smallest of each row as sorted (index, value) pairs; one CTA of BW warps per row.
// A chunk of BW steps is filtered against the running threshold (the k-th smallest key
// so far), all warps' survivors are inserted at once when they fit, else warp by warp
// with a block-wide select in between; the row ends with a select of rank k - 1 and a
// block bitonic sort. Later chunks only hold larger columns, as the threshold filter needs.
template <bool VEC>
__global__ void __launch_bounds__(BW * 32) select_block_rows_kernel(SelectParams p, int bufk, int32_t* __restrict__ out_idx,
                                                                   float* __restrict__ out_val) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* A = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* B = A + bufk;
    BlockShared& sh = *reinterpret_cast<BlockShared*>(B + bufk);
    const int warp = static_cast<int>(threadIdx.x >> 5);
    const uint32_t lane = lane_id();
    const int64_t row = blockIdx.x;
    const float* rowp = p.D + row * p.ldd;
    const int64_t N = p.N;
    const int k = p.k;
    if (threadIdx.x == 0) sh.nan = 0;
    int n = 0;
    float thr = F_INF;
    bool nan_seen = false;
    for (int64_t cbase = 0; cbase < N; cbase += static_cast<int64_t>(BW) * STEP) {
        const int64_t base = cbase + static_cast<int64_t>(warp) * STEP;
        float cur[4 * SEL_U];
        uint32_t mask = 0;
        if (base < N) {
            load_step<VEC>(rowp, N, base, cur);
#pragma unroll
            for (int i = 0; i < 32; ++i)
                nan_seen |= (cur[i] != cur[i]) && (base + ((i >> 2) * 32 + lane) * 4 + (i & 3) < N);
            mask = step_bits(cur, thr, base, -1);
        }
        int c = static_cast<int>(__reduce_add_sync(0xffffffffu, static_cast<uint32_t>(__popc(mask))));
        if (lane == 0) sh.cnt[warp] = c;
        __syncthreads();
        int total = 0;
#pragma unroll
        for (int w = 0; w < BW; ++w) total += sh.cnt[w];
        if (n + total > bufk && n > k) {
            // shrink first, then filter the chunk again with the tighter threshold
            __syncthreads();  // every warp has read the counts the select overwrites
            const uint64_t tau = block_select_prefix(A, B, n, k - 1, sh);
            n = k;
            thr = tau_filter(tau);
            if (base < N) mask &= step_bits(cur, thr, base, -1);
            c = static_cast<int>(__reduce_add_sync(0xffffffffu, static_cast<uint32_t>(__popc(mask))));
            if (lane == 0) sh.cnt[warp] = c;
            __syncthreads();
            total = 0;
#pragma unroll
            for (int w = 0; w < BW; ++w) total += sh.cnt[w];
        }
        if (n + total <= bufk) {
            int at = n;
#pragma unroll
            for (int w = 0; w < BW; ++w) at += w < warp ? sh.cnt[w] : 0;
            block_insert(A, cur, mask, at, base);
            n += total;
        } else {
            // a loose threshold (the row's first chunks): warp by warp, shrinking in between
            for (int w = 0; w < BW; ++w) {
                int cw = sh.cnt[w];
                if (n + cw > bufk) {
                    __syncthreads();
                    const uint64_t tau = block_select_prefix(A, B, n, k - 1, sh);
                    n = k;
                    thr = tau_filter(tau);
                    if (base < N) mask &= step_bits(cur, thr, base, -1);
                    c = static_cast<int>(__reduce_add_sync(0xffffffffu, static_cast<uint32_t>(__popc(mask))));
                    if (lane == 0 && warp >= w) sh.cnt[warp] = c;
                    __syncthreads();
                    cw = sh.cnt[w];
                }
                if (warp == w) {
                    block_insert(A, cur, mask, n, base);
                    mask = 0;
                }
                n += cw;
            }
        }
        __syncthreads();
    }
    if (__any_sync(0xffffffffu, nan_seen) && lane == 0) atomicOr(&sh.nan, 1u);
    if (n > k) {
        block_select_prefix(A, B, n, k - 1, sh);
        n = k;
    }
    const int P = pow2_ceil(n > 1 ? n : 1);
    for (int i = n + static_cast<int>(threadIdx.x); i < P; i += blockDim.x) A[i] = KEY_MAX;
    __syncthreads();
    block_bitonic_sort(A, P);
    for (int i = static_cast<int>(threadIdx.x); i < k; i += blockDim.x) {
        const bool have = i < n;
        out_idx[row * k + i] = have ? static_cast<int32_t>(key_idx(A[i])) : -1;
        out_val[row * k + i] = have ? key_val(A[i]) : F_INF;
    }
    if (threadIdx.x == 0) p.flags[row] = sh.nan ? ROW_SELECT_ERROR : 0u;
}

template <bool VEC>
cudaError_t launch_block_variant(const SelectParams& p, int bufk, int32_t* out_idx, float* out_val, cudaStream_t st) {
    const size_t smem = block_smem_bytes(bufk);
    auto kern = select_block_rows_kernel<VEC>;
    static std::atomic<int> smem_set[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || static_cast<int>(smem) > smem_set[dev].load(std::memory_order_relaxed)) {
        e = raise_smem_limit(reinterpret_cast<const void*>(kern), static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) smem_set[dev].store(static_cast<int>(smem), std::memory_order_relaxed);
    }
    kern<<<static_cast<unsigned>(p.M), BW * 32, smem, st>>>(p, bufk, out_idx, out_val);
    return cudaGetLastError();
}
}  // namespace

int select_block_k() {
    const char* e = std::getenv("KNN_SELECT_BLOCK_K");
    return e ? std::atoi(e) : 128;
}

bool select_prefers_block(int64_t M, int32_t k) {
    const int bk = select_block_k();
    return bk > 0 && (k >= bk || M <= 64);
}

cudaError_t launch_select_topk(const SelectParams& p, int32_t* out_idx, float* out_val, cudaStream_t st) {
    if (p.M <= 0) return cudaSuccess;
    const bool vec4 = (p.ldd % 4 == 0) && (reinterpret_cast<uintptr_t>(p.D) % 16 == 0);
    if (p.block && !p.E && !p.thr && !p.self_col && p.M <= 0x7fffffff) {
        const int bufk = block_bufk(p.k);
        return vec4 ? launch_block_variant<true>(p, bufk, out_idx, out_val, st)
                    : launch_block_variant<false>(p, bufk, out_idx, out_val, st);
    }
    const int bufk = choose_bufk(p.k, p.k);
    const bool vec = (p.ldd % 4 == 0) && (reinterpret_cast<uintptr_t>(p.D) % 16 == 0);
    return vec ? launch_variant<true, true, true>(p, bufk, -1, out_idx, out_val, st)
               : launch_variant<false, true, true>(p, bufk, -1, out_idx, out_val, st);
}

}  // namespace knn
