// Device-side helpers shared by the engine's kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace knn {

constexpr uint64_t KEY_MAX = ~0ull;
constexpr float F_INF = __builtin_huge_valf();

// Order-preserving map of a finite float (or +inf) to uint32: a < b  <=>  ord(a) < ord(b).
// -0.0 is folded onto +0.0 so that equal distances compare equal.
__host__ __device__ __forceinline__ uint32_t float_to_ord(float f) {
#ifdef __CUDA_ARCH__
    uint32_t u = __float_as_uint(f == 0.0f ? 0.0f : f);
#else
    float g = (f == 0.0f ? 0.0f : f);
    uint32_t u;
    __builtin_memcpy(&u, &g, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__host__ __device__ __forceinline__ float ord_to_float(uint32_t o) {
    uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    __builtin_memcpy(&f, &u, 4);
    return f;
#endif
}

// A selection key: (value, index) in lexicographic order as one unsigned 64-bit integer.
// Distinct indices make every key in a row unique, so "the k smallest keys" is unique.
__host__ __device__ __forceinline__ uint64_t make_key(float v, uint32_t j) {
    return (static_cast<uint64_t>(float_to_ord(v)) << 32) | j;
}
__host__ __device__ __forceinline__ float key_val(uint64_t k) { return ord_to_float(static_cast<uint32_t>(k >> 32)); }
__host__ __device__ __forceinline__ uint32_t key_idx(uint64_t k) { return static_cast<uint32_t>(k & 0xffffffffu); }
// Largest key whose value is v: every key with value <= v is <= this.
__host__ __device__ __forceinline__ uint64_t key_ceiling(float v) {
    return (static_cast<uint64_t>(float_to_ord(v)) << 32) | 0xffffffffu;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src) {
    uint32_t lo = __shfl_sync(0xffffffffu, static_cast<uint32_t>(v), src);
    uint32_t hi = __shfl_sync(0xffffffffu, static_cast<uint32_t>(v >> 32), src);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Streaming 16-byte load that does not allocate in L1 (each distance is read once).
__device__ __forceinline__ float4 ldg_stream_f4(const float* p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// Error-free transformation a + b = s + e (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

}  // namespace knn
