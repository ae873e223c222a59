// Double-float and FP32 arithmetic policies and the block-level helpers shared
// by the persistent PCG kernels (pcg_df.cu: Jacobi-scaled PCG; pcg_ml.cu: the
// same with the multilevel preconditioner).  Device code only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pgcp {
namespace dfa {

constexpr int RUN_THREADS = 256;

// ---------------------------------------------------------------- double-float

__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}

__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// acc + a * b (the lo * lo product, ~2^-48 relative, is dropped)
__device__ __forceinline__ float2 df_fma(float2 acc, float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float2 s = two_sum(acc.x, p);
    const float t = __fadd_rn(s.y, __fadd_rn(e, acc.y));
    return fast_two_sum(s.x, t);
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float2 s = two_sum(a.x, b.x);
    return fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}

__device__ __forceinline__ double df_to_d(float2 a) { return (double)a.x + (double)a.y; }

__device__ __forceinline__ float2 d_to_df(double d) {
    const float h = __double2float_rn(d);
    return make_float2(h, __double2float_rn(d - (double)h));
}

// Arithmetic policies: one scalar S (also the stored matrix value) and a
// row's (x, y) pair V.
// ArithDF: double-float scalars, V = float4 {x.hi, x.lo, y.hi, y.lo}.
// ArithF32: FP32 scalars, V = float2, FP32 accumulation.
struct ArithDF {
    using S = float2;
    using V = float4;
    static constexpr int bytes = 8;
    static __device__ __forceinline__ S zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ S fma(S acc, S a, S b) { return df_fma(acc, a, b); }
    static __device__ __forceinline__ S neg(S a) { return make_float2(-a.x, -a.y); }
    static __device__ __forceinline__ S cx(V v) { return make_float2(v.x, v.y); }
    static __device__ __forceinline__ S cy(V v) { return make_float2(v.z, v.w); }
    static __device__ __forceinline__ V pack(S a, S b) { return make_float4(a.x, a.y, b.x, b.y); }
    static __device__ __forceinline__ V vzero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    static __device__ __forceinline__ S from_d(double d) { return d_to_df(d); }
    static __device__ __forceinline__ double to_d(S a) { return df_to_d(a); }
    static __device__ __forceinline__ float2 as_df(S a) { return a; }
    static __device__ __forceinline__ float lead(S a) { return a.x; }
};
struct ArithF32 {
    using S = float;
    using V = float2;
    static constexpr int bytes = 4;
    static __device__ __forceinline__ S zero() { return 0.f; }
    static __device__ __forceinline__ S fma(S acc, S a, S b) { return fmaf(a, b, acc); }
    static __device__ __forceinline__ S neg(S a) { return -a; }
    static __device__ __forceinline__ S cx(V v) { return v.x; }
    static __device__ __forceinline__ S cy(V v) { return v.y; }
    static __device__ __forceinline__ V pack(S a, S b) { return make_float2(a, b); }
    static __device__ __forceinline__ V vzero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ S from_d(double d) { return __double2float_rn(d); }
    static __device__ __forceinline__ double to_d(S a) { return (double)a; }
    static __device__ __forceinline__ float2 as_df(S a) { return make_float2(a, 0.f); }
    static __device__ __forceinline__ float lead(S a) { return a; }
};

// Sum NV double-float values over the block on the FP32 pipe; thread 0 gets
// the totals as doubles.  red: NV * (warps) float2 of shared memory.
template <int NV>
__device__ __forceinline__ void block_sum_df(float2* v, float2* red, double* out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float2 t;
            t.x = __shfl_xor_sync(0xffffffffu, v[i].x, o);
            t.y = __shfl_xor_sync(0xffffffffu, v[i].y, o);
            v[i] = df_add(v[i], t);
        }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = RUN_THREADS / 32;
    __syncthreads();   // red is free (its previous readers are done)
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) red[NV * warp + i] = v[i];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            float2 t = lane < NW ? red[NV * lane + i] : make_float2(0.f, 0.f);
#pragma unroll
            for (int o = NW / 2; o > 0; o >>= 1) {
                float2 u;
                u.x = __shfl_xor_sync(0xffffffffu, t.x, o);
                u.y = __shfl_xor_sync(0xffffffffu, t.y, o);
                t = df_add(t, u);
            }
            if (lane == 0) out[i] = df_to_d(t);
        }
    }
}

__device__ __forceinline__ void prefetch_l2(const void* ptr) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

// One stored entry of the SpMV: w += v * r_c (or the cross form).
template <typename A>
__device__ __forceinline__ void spmv_entry(int32_t c, typename A::S v, const typename A::V* r, typename A::S& w0,
                                           typename A::S& w1) {
    const bool cross = c < 0;
    const typename A::V rc = r[cross ? ~c : c];
    const typename A::S a0 = cross ? A::cy(rc) : A::cx(rc);
    const typename A::S a1 = cross ? A::cx(rc) : A::cy(rc);
    const typename A::S v0 = cross ? A::neg(v) : v;
    w0 = A::fma(w0, v0, a0);
    w1 = A::fma(w1, v, a1);
}


}  // namespace dfa
}  // namespace pgcp
