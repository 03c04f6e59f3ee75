// Warp-level quick multi-select building blocks (device code, header-only so that
// the unfused select kernel and the fused GEMM epilogue share them).
//
// Paper: Methods, "GPU-based quick multi-select".
//   - One warp owns one row ("each array is handled by a single thread warp").
//   - A partition reads each element once into a register, votes with a warp ballot
//     on "element >= pivot", and derives every lane's destination from a popc of the
//     ballot bits of the lower lanes: elements below the pivot are written from the
//     left end of the auxiliary array, the others from the right end. No prefix sum,
//     no second read. Two running counters (the paper's g_< and g_>=) give the warp's
//     write offsets.
//   - Input and auxiliary arrays swap roles after each partition ("ping-pong"), and
//     rather than copying data back, a list of references (start, end, which array)
//     records where every part of the row lives.
//   - Recursion: with L elements left of the pivot and K wanted, K < L continues on the
//     left part, K > L keeps the left part and continues on the right with K - L.
// Deviations for GB300 (reasons in the design notes):
//   - the partition is three-way (< pivot, == pivot, > pivot), so that a pivot equal
//     to the minimum still makes progress (the two-way rule can loop forever there);
//   - keys are 64-bit (value, index) pairs, unique within a row, so the answer is
//     unique and ties go to the lower index;
//   - the pivot is the median of the segment's first, middle and last keys
//     (the paper does not say how it picks pivots);
//   - segments of at most 32 keys are finished with a 32-lane bitonic network.
#pragma once

#include "common.cuh"

namespace knn {

// Speculative thresholds (running-threshold selections over a stream of columns).
// Having seen a fraction f of a row's columns, a mid-stream shrink may aim at ranks
// max(SPEC_RMIN, SPEC_ALPHA * f * r) instead of r (r = k and k + m): for columns in
// random order the final list then still holds about SPEC_ALPHA * r keys, while far fewer
// keys are inserted before the threshold settles. Every caller checks at the end of the
// row whether the band it needed lies inside the threshold it ended with, and otherwise
// treats the row as truncated there or selects it again without speculation.
constexpr float SPEC_ALPHA = 3.f;
constexpr int SPEC_RMIN = 16;

__device__ __forceinline__ int spec_rank(int r, int64_t seen, int64_t N) {
    const float t = ceilf(SPEC_ALPHA * static_cast<float>(r) * (static_cast<float>(seen) / static_cast<float>(N)));
    const int s = t > static_cast<float>(SPEC_RMIN) ? static_cast<int>(t) : SPEC_RMIN;
    return s < r ? s : r;
}

// Float threshold for a running-threshold filter: v <= tau_filter(tau) exactly when
// key(v, j) <= tau, for every column j after the ones tau was built from (columns are
// visited in increasing order; a value tied with a non-ceiling threshold key is then
// above it, so the float just below tau's value is used).
__device__ __forceinline__ float tau_filter(uint64_t tau) {
    if ((tau >> 32) == 0xffffffffull) return F_INF;
    const float v = key_val(tau);
    return static_cast<uint32_t>(tau) == 0xffffffffu ? v : nextafterf(v, -F_INF);
}

constexpr int SEG_MAX = 128;        // references kept per warp
constexpr uint32_t SEG_IN_B = 1u << 30;
constexpr uint32_t SEG_SORTED = 1u << 31;
constexpr uint32_t SEG_END_MASK = SEG_IN_B - 1;

template <typename K>
__device__ __forceinline__ K shfl_key(K v, int src);
template <>
__device__ __forceinline__ uint32_t shfl_key<uint32_t>(uint32_t v, int src) {
    return __shfl_sync(0xffffffffu, v, src);
}
template <>
__device__ __forceinline__ uint64_t shfl_key<uint64_t>(uint64_t v, int src) {
    return shfl_u64(v, src);
}

template <typename K>
__device__ __forceinline__ K shfl_xor_key(K v, int m) {
    if constexpr (sizeof(K) == 8) {
        return __shfl_xor_sync(0xffffffffu, static_cast<unsigned long long>(v), m);
    } else {
        return __shfl_xor_sync(0xffffffffu, v, m);
    }
}

// Ascending bitonic sort of one key per lane across the warp.
template <typename K>
__device__ __forceinline__ K warp_sort32(K v) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            K o = shfl_xor_key(v, j);
            const bool up = (lane & k) == 0 || k == 32;
            const bool lower = (lane & j) == 0;
            v = (lower == up) ? (o < v ? o : v) : (o > v ? o : v);
        }
    }
    return v;
}

// Integer mixing (xorshift-multiply rounds) for pivot positions.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x = (x ^ (x >> 16)) * 0x7feb352du;
    x = (x ^ (x >> 15)) * 0x846ca68bu;
    return x ^ (x >> 16);
}

template <typename K>
__device__ __forceinline__ K median3(K a, K b, K c) {
    K lo = a < b ? a : b, hi = a < b ? b : a;
    K m = hi < c ? hi : c;
    return lo > m ? lo : m;
}

// Three-way ballot partition of src[s, e) around `pivot` into dst[s, e):
// dst = [keys < pivot][keys == pivot][keys > pivot]. Returns the sizes of the first
// two parts. All 32 lanes must call it with the same arguments.
template <typename K>
__device__ __forceinline__ void partition3(const K* src, K* dst, int s, int e, K pivot, int& nlt, int& neq) {
    const uint32_t lane = lane_id();
    const uint32_t lt_mask = lanemask_lt();
    int g_lt = 0, g_gt = 0, g_eq = 0;  // the paper's running counters
    for (int base = s; base < e; base += 32) {
        const int i = base + static_cast<int>(lane);
        const bool valid = i < e;
        const K v = valid ? src[i] : K(0);
        const bool lt = valid && v < pivot;
        const bool gt = valid && v > pivot;
        const uint32_t b_lt = __ballot_sync(0xffffffffu, lt);
        const uint32_t b_gt = __ballot_sync(0xffffffffu, gt);
        const uint32_t b_eq = __ballot_sync(0xffffffffu, valid && !lt && !gt);
        if (lt) dst[s + g_lt + __popc(b_lt & lt_mask)] = v;
        if (gt) dst[e - 1 - g_gt - __popc(b_gt & lt_mask)] = v;
        g_lt += __popc(b_lt);
        g_gt += __popc(b_gt);
        g_eq += __popc(b_eq);
    }
    for (int t = static_cast<int>(lane); t < g_eq; t += 32) dst[s + g_lt + t] = pivot;
    __syncwarp();
    nlt = g_lt;
    neq = g_eq;
}

// Key of rank r (0-based) among a[0, n) (duplicates allowed). a and b are both
// clobbered (b is the auxiliary array).
template <typename K>
__device__ K warp_rank_select(K* a, K* b, int n, int r) {
    K* src = a;
    K* dst = b;
    int lo = 0, hi = n;
    const uint32_t lane = lane_id();
    for (int guard = 0; guard < 4096; ++guard) {
        const int len = hi - lo;
        if (len <= 32) {
            K v = static_cast<int>(lane) < len ? src[lo + lane] : static_cast<K>(~K(0));
            v = warp_sort32(v);
            return shfl_key(v, r - lo);
        }
        const uint32_t h0 = mix32(static_cast<uint32_t>(lo) * 0x9e3779b1u + static_cast<uint32_t>(hi) +
                                  static_cast<uint32_t>(guard) * 0x85ebca6bu);
        const uint32_t ul = static_cast<uint32_t>(len);
        const K pivot = median3(src[lo + h0 % ul], src[lo + mix32(h0) % ul], src[lo + mix32(h0 ^ 0x5bd1e995u) % ul]);
        int nlt, neq;
        partition3(src, dst, lo, hi, pivot, nlt, neq);
        if (r < lo + nlt) {
            hi = lo + nlt;
        } else if (r < lo + nlt + neq) {
            return pivot;
        } else {
            lo = lo + nlt + neq;
        }
        K* t = src;
        src = dst;
        dst = t;
    }
    return src[r];  // unreachable: every partition removes at least the pivot
}

// Reference list over a row's keys held in two arrays A and B: every position p in
// [0, n) belongs to exactly one segment, and the segment says which array holds the
// live key for p. Keys are unique, so the segment of position p holds exactly the
// keys of ranks [start, end).
struct SegRefs {
    int* start;     // shared or global, SEG_MAX entries
    uint32_t* end;  // end | SEG_IN_B | SEG_SORTED
    int count;      // warp-uniform
};

__device__ __forceinline__ void seg_init(SegRefs& s, int n) {
    if (lane_id() == 0) {
        s.start[0] = 0;
        s.end[0] = static_cast<uint32_t>(n);
    }
    s.count = 1;
    __syncwarp();
}

// Returns the key of rank r; refines the reference list. Returns false (and leaves
// *out untouched) when the list is full.
__device__ __forceinline__ bool seg_rank(SegRefs& s, uint64_t* A, uint64_t* B, int r, uint64_t* out) {
    const uint32_t lane = lane_id();
    for (int guard = 0; guard < 4096; ++guard) {
        // find the segment holding position r
        int found = -1;
        for (int base = 0; base < s.count && found < 0; base += 32) {
            const int t = base + static_cast<int>(lane);
            bool hit = false;
            if (t < s.count) {
                const int st = s.start[t];
                const int en = static_cast<int>(s.end[t] & SEG_END_MASK);
                hit = st <= r && r < en;
            }
            const uint32_t b = __ballot_sync(0xffffffffu, hit);
            if (b) found = base + __ffs(b) - 1;
        }
        if (found < 0) return false;
        const int st = s.start[found];
        const uint32_t ef = s.end[found];
        const int en = static_cast<int>(ef & SEG_END_MASK);
        uint64_t* src = (ef & SEG_IN_B) ? B : A;
        uint64_t* dst = (ef & SEG_IN_B) ? A : B;
        const int len = en - st;
        if ((ef & SEG_SORTED) || len == 1) {
            *out = src[r];
            return true;
        }
        if (len <= 32) {
            uint64_t v = static_cast<int>(lane) < len ? src[st + lane] : KEY_MAX;
            v = warp_sort32(v);
            if (static_cast<int>(lane) < len) src[st + lane] = v;
            if (lane == 0) s.end[found] = ef | SEG_SORTED;
            __syncwarp();
            *out = shfl_key(v, r - st);
            return true;
        }
        if (s.count + 2 > SEG_MAX) return false;
        // median of three keys at hashed positions: fixed positions (first, middle, last) meet
        // structured rows (sorted runs, sawtooth) with a pivot near the segment's minimum at
        // every step, and the reference list overflows
        const uint32_t h0 = mix32(static_cast<uint32_t>(st) * 0x9e3779b1u + static_cast<uint32_t>(en) +
                                  static_cast<uint32_t>(guard) * 0x85ebca6bu);
        const uint32_t h1 = mix32(h0), h2 = mix32(h0 ^ 0x5bd1e995u);
        const uint32_t ul = static_cast<uint32_t>(len);
        const uint64_t pivot = median3(src[st + h0 % ul], src[st + h1 % ul], src[st + h2 % ul]);
        int nlt, neq;
        partition3(src, dst, st, en, pivot, nlt, neq);  // neq == 1: keys are unique
        const uint32_t where = (ef & SEG_IN_B) ? 0u : SEG_IN_B;
        // the segment now lives in dst as [left][pivot][right]; replace it by its parts
        if (lane == 0) {
            int c = s.count;
            const int mid = st + nlt;
            s.start[found] = mid;  // the pivot alone, already in place
            s.end[found] = static_cast<uint32_t>(mid + 1) | where | SEG_SORTED;
            if (nlt > 0) {
                s.start[c] = st;
                s.end[c] = static_cast<uint32_t>(mid) | where;
                ++c;
            }
            if (mid + 1 < en) {
                s.start[c] = mid + 1;
                s.end[c] = static_cast<uint32_t>(en) | where;
                ++c;
            }
        }
        s.count += (nlt > 0 ? 1 : 0) + (st + nlt + 1 < en ? 1 : 0);
        __syncwarp();
        if (r == st + nlt) {
            *out = pivot;
            return true;
        }
    }
    return false;
}

// Gathers the live keys of every segment into B[0, n) (position order).
__device__ __forceinline__ void seg_materialise_in_B(const SegRefs& s, const uint64_t* A, uint64_t* B) {
    const uint32_t lane = lane_id();
    for (int t = 0; t < s.count; ++t) {
        const uint32_t ef = s.end[t];
        if (ef & SEG_IN_B) continue;
        const int st = s.start[t];
        const int en = static_cast<int>(ef & SEG_END_MASK);
        for (int p = st + static_cast<int>(lane); p < en; p += 32) B[p] = A[p];
    }
    __syncwarp();
}

// Number of live keys <= limit over all segments.
__device__ __forceinline__ int seg_count_le(const SegRefs& s, const uint64_t* A, const uint64_t* B, uint64_t limit) {
    const uint32_t lane = lane_id();
    int c = 0;
    for (int t = 0; t < s.count; ++t) {
        const uint32_t ef = s.end[t];
        const uint64_t* src = (ef & SEG_IN_B) ? B : A;
        const int st = s.start[t];
        const int en = static_cast<int>(ef & SEG_END_MASK);
        for (int p = st + static_cast<int>(lane); p < en; p += 32) c += src[p] <= limit ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    return c;
}

// Ballot/popc compaction of the keys <= limit of src[0, n) into dst (any memory);
// returns how many were written (the order of src is kept).
__device__ __forceinline__ int compact_le(const uint64_t* src, int n, uint64_t limit, uint64_t* dst) {
    const uint32_t lane = lane_id();
    const uint32_t lt_mask = lanemask_lt();
    int w = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + static_cast<int>(lane);
        const uint64_t v = i < n ? src[i] : KEY_MAX;
        const bool keep = i < n && v <= limit;
        const uint32_t b = __ballot_sync(0xffffffffu, keep);
        if (keep) dst[w + __popc(b & lt_mask)] = v;
        w += __popc(b);
    }
    __syncwarp();
    return w;
}

__device__ __forceinline__ int count_le(const uint64_t* src, int n, uint64_t limit) {
    const uint32_t lane = lane_id();
    int c = 0;
    for (int i = static_cast<int>(lane); i < n; i += 32) c += src[i] <= limit ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    return c;
}

// Result of shrinking one row's candidate buffer.
struct CompactResult {
    int n;              // keys kept, now in A[0, n)
    uint64_t tau;       // every key dropped so far is > tau (the row's new threshold)
    uint64_t band;      // max(km-th key, ceiling(value of k-th key + window)): the unclamped threshold
    bool truncated;     // capacity truncation: kept fewer keys than the band asks for
    bool ok;            // false when the reference list overflowed (caller must give up)
};

// Quick multi-select on the row's buffer A[0, n) (B is the auxiliary array):
// finds the k-th and km-th smallest keys, sets the threshold to the band
//   tau = max(key_km, ceiling(value(key_k) + window))   (window > 0)
//   tau = key_km                                          (window == 0)
// clamped by tau_limit, keeps the keys <= tau, and if more than keep_max remain,
// keeps only the keep_trunc smallest (truncation). Requires n >= 1.
__device__ __forceinline__ CompactResult compact_row(uint64_t* A, uint64_t* B, int* seg_start, uint32_t* seg_end,
                                                     int n, int k, int km, float window, uint64_t tau_limit,
                                                     int keep_max, int keep_trunc) {
    CompactResult res{};
    res.ok = true;
    SegRefs s{seg_start, seg_end, 0};
    seg_init(s, n);
    const int kk = k < n ? k : n;
    const int kme = km < n ? km : n;
    uint64_t key_km = 0, key_k = 0;
    if (!seg_rank(s, A, B, kme - 1, &key_km)) res.ok = false;
    if (res.ok && kk != kme && !seg_rank(s, A, B, kk - 1, &key_k)) res.ok = false;
    if (kk == kme) key_k = key_km;
    if (!res.ok) return res;
    uint64_t band = key_km;
    if (window > 0.f) {
        const uint64_t wk = key_ceiling(key_val(key_k) + window);
        band = wk > band ? wk : band;
    }
    if (n < km) band = KEY_MAX;  // fewer keys than the row keeps: nothing may be dropped yet
    res.band = band;
    uint64_t tau = band < tau_limit ? band : tau_limit;
    int keep = seg_count_le(s, A, B, tau);
    if (keep > keep_max) {
        // too many keys inside the band: keep the keep_trunc smallest only
        uint64_t kt = 0;
        if (!seg_rank(s, A, B, keep_trunc - 1, &kt)) {
            res.ok = false;
            return res;
        }
        tau = kt;
        res.truncated = true;
    }
    seg_materialise_in_B(s, A, B);
    res.n = compact_le(B, n, tau, A);
    res.tau = tau;
    return res;
}

}  // namespace knn

namespace knn {

// Ascending bitonic sort of X[0, P) by one warp (P a power of two). Two stride levels of a
// merge step share one pass over shared memory: a lane loads four keys b, b + h, b + 2h,
// b + 3h, compares them at stride 2h and then h in registers and stores them back. Pair and
// quad positions come from shifts and masks of the lane's item index.
template <typename K>
__device__ __forceinline__ void bitonic_ce(K& a, K& b, bool up) {
    if ((a > b) == up) {
        const K t = a;
        a = b;
        b = t;
    }
}

template <typename K>
__device__ __forceinline__ void warp_bitonic_sort_smem(K* X, int P) {
    const int lane = static_cast<int>(lane_id());
    for (int lsz = 1; (1 << lsz) <= P; ++lsz) {
        const int size = 1 << lsz;
        int ls = lsz - 1;  // stride 2^ls
        for (; ls >= 1; ls -= 2) {
            const int h = 1 << (ls - 1);
            for (int q = lane; q < (P >> 2); q += 32) {
                const int b = ((q >> (ls - 1)) << (ls + 1)) | (q & (h - 1));
                const bool up = (b & size) == 0;
                K x0 = X[b], x1 = X[b + h], x2 = X[b + 2 * h], x3 = X[b + 3 * h];
                bitonic_ce(x0, x2, up);
                bitonic_ce(x1, x3, up);
                bitonic_ce(x0, x1, up);
                bitonic_ce(x2, x3, up);
                X[b] = x0;
                X[b + h] = x1;
                X[b + 2 * h] = x2;
                X[b + 3 * h] = x3;
            }
            __syncwarp();
        }
        if (ls == 0) {
            for (int i = lane; i < (P >> 1); i += 32) {
                const int lo = i << 1;
                const bool up = (lo & size) == 0;
                const K a = X[lo], b = X[lo + 1];
                if ((a > b) == up) {
                    X[lo] = b;
                    X[lo + 1] = a;
                }
            }
            __syncwarp();
        }
    }
}

// Ascending sort of X[0, n) by one warp for a list that is already nearly in order:
// odd-even transposition passes (each lane compares and swaps pairs i, i + 1 for i of one
// parity) until an even and an odd pass in a row swap nothing, which leaves every adjacent
// pair in order. A key displaced by r positions needs about r passes. Returns false when
// max_pass passes did not settle the list (it is then a permutation of the input, and the
// caller sorts it in full).
template <typename K>
__device__ __forceinline__ bool warp_oddeven_settle(K* X, int n, int max_pass) {
    const int lane = static_cast<int>(lane_id());
    int quiet = 0;
    for (int pass = 0; pass < max_pass; ++pass) {
        bool swapped = false;
        for (int i = (pass & 1) + 2 * lane; i + 1 < n; i += 64) {
            const K a = X[i], b = X[i + 1];
            if (a > b) {
                X[i] = b;
                X[i + 1] = a;
                swapped = true;
            }
        }
        __syncwarp();
        quiet = __any_sync(0xffffffffu, swapped) ? 0 : quiet + 1;
        if (quiet == 2) return true;
    }
    return false;
}

__host__ __device__ __forceinline__ int pow2_ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace knn

namespace knn {

// Values of ranks r1 <= r2 (0-based) among a[0, n) (32-bit, duplicates allowed), by a
// two-level sample select: 32 evenly spaced keys, sorted across the lanes, split the
// values into 33 buckets; a shared-memory histogram of the buckets locates the bucket
// of each rank, whose members are gathered into b and finished with a 32-lane sort
// (or the quick multi-select when a bucket holds more than 32). a is preserved; b and
// hist (at least 33 words) are scratch. Returns false only if the fallback overflows.
__device__ __forceinline__ bool two_ranks_sampled(const uint32_t* a, uint32_t* b, uint32_t* tmp, uint32_t* hist,
                                                  int n, int r1, int r2, uint32_t& v1, uint32_t& v2) {
    const uint32_t lane = lane_id();
    const uint32_t lt_mask = lanemask_lt();
    // 1. pivots
    uint32_t piv = a[(static_cast<int64_t>(lane) * n) >> 5];
    piv = warp_sort32(piv);
    for (int i = static_cast<int>(lane); i < 33; i += 32) hist[i] = 0u;
    __syncwarp();
    // 2. bucket histogram: bucket(x) = number of pivots <= x (0..32)
    const uint32_t p31 = __shfl_sync(0xffffffffu, piv, 31);
    for (int base = 0; base < n; base += 32) {
        const int i = base + static_cast<int>(lane);
        const uint32_t x = i < n ? a[i] : 0u;
        int lo = 0;  // number of pivots <= x, by binary search over the sorted lanes
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t pv = __shfl_sync(0xffffffffu, piv, lo + step - 1);
            if (pv <= x) lo += step;
        }
        if (lo == 31 && p31 <= x) lo = 32;
        if (i < n) atomicAdd(&hist[lo], 1u);
    }
    __syncwarp();
    // 3. exclusive prefix over the 33 buckets (lane j holds buckets j; lane 0 also bucket 32)
    const uint32_t h = hist[lane];
    uint32_t incl = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (static_cast<int>(lane) >= o) incl += y;
    }
    const uint32_t excl = incl - h;
    const uint32_t total31 = __shfl_sync(0xffffffffu, incl, 31);
    // 4. each rank: its bucket, the bucket's members, then an exact small select
    uint32_t out[2];
    const int rr[2] = {r1, r2};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int r = rr[q];
        int bkt;
        uint32_t base_cnt;
        if (static_cast<uint32_t>(r) >= total31) {
            bkt = 32;
            base_cnt = total31;
        } else {
            const uint32_t hit = __ballot_sync(0xffffffffu, excl <= static_cast<uint32_t>(r) &&
                                                                 static_cast<uint32_t>(r) < incl);
            bkt = __ffs(hit) - 1;
            base_cnt = __shfl_sync(0xffffffffu, excl, bkt);
        }
        // bucket bounds: [pivot bkt-1, pivot bkt)
        const uint32_t lo_v = bkt > 0 ? __shfl_sync(0xffffffffu, piv, bkt - 1) : 0u;
        const uint32_t hi_v = bkt < 32 ? __shfl_sync(0xffffffffu, piv, bkt < 32 ? bkt : 31) : 0xffffffffu;
        int w = 0;
        for (int base = 0; base < n; base += 32) {
            const int i = base + static_cast<int>(lane);
            const uint32_t x = i < n ? a[i] : 0u;
            const bool in = i < n && (bkt == 0 || x >= lo_v) && (bkt == 32 ? true : x < hi_v);
            const uint32_t bb = __ballot_sync(0xffffffffu, in);
            if (in) b[w + __popc(bb & lt_mask)] = x;
            w += __popc(bb);
        }
        __syncwarp();
        const int rel = r - static_cast<int>(base_cnt);
        if (w <= 32) {
            uint32_t v = static_cast<int>(lane) < w ? b[lane] : 0xffffffffu;
            v = warp_sort32(v);
            out[q] = __shfl_sync(0xffffffffu, v, rel);
        } else if (tmp != nullptr) {
            out[q] = warp_rank_select<uint32_t>(b, tmp, w, rel);
        } else {
            return false;  // a crowded bucket (ties) and no auxiliary array: caller takes the exact path
        }
        __syncwarp();
    }
    v1 = out[0];
    v2 = out[1];
    return true;
}

}  // namespace knn
