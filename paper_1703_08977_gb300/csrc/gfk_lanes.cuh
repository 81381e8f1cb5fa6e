// FP32 arithmetic of the mixed-precision walk, written once for one walker
// (`float`) and for two walkers at a time (the two lanes of a `float2`).
//
// sm_100-class GPUs (GB300 included) execute FP32 additions, multiplications
// and fused multiply-adds on float pairs as single packed instructions
// (FADD2 / FMUL2 / FFMA2: one issue slot, two results).  The walk kernel is
// bound by instruction issue, and each thread advances two (or four) walkers
// that run exactly the same arithmetic, so evaluating them pairwise halves
// the issue cost of everything below that is not a special function.
//
// Every operation is written out with its rounding (round to nearest; no
// multiply-add contraction is left to the compiler), so one walker gets bit
// for bit the same result whether it is evaluated alone or in either lane of
// a pair: in any launch shape (1, 2 or 4 walkers per thread), in the
// initialisation kernel, and in the adjoint's recompute of its positions.
// Special functions (reciprocal square root, reciprocal, base-2 logarithm and
// exponential, sine, cosine, square root) have no packed form and run per
// lane on the special-function unit.
//
// This header holds the lane arithmetic; gfk_eval_f32.cuh writes the trial
// evaluation with it, and gfk_device.cuh the Box-Muller normals and the move.
#pragma once

#include <cuda_runtime.h>

namespace gfk {

// ---------------------------------------------------------------------------
// Lane arithmetic
// ---------------------------------------------------------------------------
template <typename L> struct LaneCount;
template <> struct LaneCount<float> { static constexpr int value = 1; };
template <> struct LaneCount<float2> { static constexpr int value = 2; };

__device__ __forceinline__ float lsplat(float v, float) { return v; }
__device__ __forceinline__ float2 lsplat(float v, float2) { return make_float2(v, v); }
template <typename L>
__device__ __forceinline__ L splat(float v) { return lsplat(v, L()); }

// Both forms are written as PTX instructions with an explicit .rn rounding,
// which the assembler never merges into multiply-adds (a product feeding an
// addition in one form and fused with it in the other would give the two
// forms different last bits; measured on the compiler's own intrinsics, which
// did not keep that guarantee for the one-walker form inside this code).
__device__ __forceinline__ float ladd(float a, float b) {
    float r;
    asm("add.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float lsub(float a, float b) {
    float r;
    asm("sub.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float lmul(float a, float b) {
    float r;
    asm("mul.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float lfma(float a, float b, float c) {
    float r;
    asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float lneg(float a) { return -a; }

#define GFK_F32X2_BINARY(NAME, OP)                                                      \
    __device__ __forceinline__ float2 NAME(float2 a, float2 b) {                        \
        float2 r;                                                                       \
        asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\t"                     \
            "mov.b64 rb, {%4, %5};\n\t" OP " rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"  \
            : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));            \
        return r;                                                                       \
    }
GFK_F32X2_BINARY(ladd, "add.rn.f32x2")
GFK_F32X2_BINARY(lsub, "sub.rn.f32x2")
GFK_F32X2_BINARY(lmul, "mul.rn.f32x2")
#undef GFK_F32X2_BINARY
__device__ __forceinline__ float2 lfma(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
__device__ __forceinline__ float2 lneg(float2 a) { return make_float2(-a.x, -a.y); }

// lane j (compile-time) of a value, and a value from its lanes
template <int J> __device__ __forceinline__ float lane(float a) { return a; }
template <int J> __device__ __forceinline__ float lane(float2 a) { return J == 0 ? a.x : a.y; }
__device__ __forceinline__ float lane_at(float a, int) { return a; }
__device__ __forceinline__ float lane_at(float2 a, int j) { return j == 0 ? a.x : a.y; }
__device__ __forceinline__ void set_lane(float& a, int, float v) { a = v; }
__device__ __forceinline__ void set_lane(float2& a, int j, float v) {
    if (j == 0) a.x = v;
    else a.y = v;
}

// per-lane special functions and comparisons
__device__ __forceinline__ float rsqrt_approx(float s) {
    float y;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(s));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lrsqrt(float a) { return rsqrt_approx(a); }
__device__ __forceinline__ float2 lrsqrt(float2 a) {
    return make_float2(rsqrt_approx(a.x), rsqrt_approx(a.y));
}
__device__ __forceinline__ float lrcp(float a) { return rcp_approx(a); }
__device__ __forceinline__ float2 lrcp(float2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
__device__ __forceinline__ float lex2(float a) { return ex2_approx_ftz(a); }
__device__ __forceinline__ float2 lex2(float2 a) {
    return make_float2(ex2_approx_ftz(a.x), ex2_approx_ftz(a.y));
}
__device__ __forceinline__ float lmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float2 lmin(float2 a, float2 b) {
    return make_float2(fminf(a.x, b.x), fminf(a.y, b.y));
}
__device__ __forceinline__ float lmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float2 lmax(float2 a, float2 b) {
    return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y));
}

// e^x as 2^(x log2 e): one rounded product, then the hardware base-2
// exponential (flush-to-zero: results below 2^-126 are 0, which the orbital
// exponentials, scaled by their largest term, never need)
template <typename L>
__device__ __forceinline__ L lexp(L x) {
    return lex2(lmul(x, splat<L>(1.4426950408889634f)));
}

// Distance and inverse distance from a squared distance: one hardware
// reciprocal square root, then the product.
template <typename L>
__device__ __forceinline__ void lradius(L s, L& r, L& i) {
    i = lrsqrt(s);
    r = lmul(s, i);
}

}  // namespace gfk
