// Forward-mode dual numbers: a value and N tangents, for the trial function's
// derivatives in the adjoint (gradient) kernels.  Every operation propagates
// the tangents by the chain rule; comparisons look at the value only.
#pragma once

#include <cuda_runtime.h>

namespace gfk {

// keep the math library's scalar overloads visible next to the dual ones
using ::fmax;
using ::fmin;

template <int N, typename T>
struct Dual {
    T v;
    T d[N];
    __device__ __forceinline__ Dual() {}
    __device__ __forceinline__ Dual(T x) : v(x) {
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] = T(0);
    }
    template <typename U>
    __device__ __forceinline__ explicit Dual(U x) : Dual(T(x)) {}
    __device__ __forceinline__ static Dual seed(T x, int k) {
        Dual r(x);
        if (k >= 0 && k < N) r.d[k] = T(1);
        return r;
    }
};

#define GFK_DUAL template <int N, typename T> __device__ __forceinline__

GFK_DUAL Dual<N, T> operator+(const Dual<N, T>& a, const Dual<N, T>& b) {
    Dual<N, T> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
GFK_DUAL Dual<N, T> operator-(const Dual<N, T>& a, const Dual<N, T>& b) {
    Dual<N, T> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
GFK_DUAL Dual<N, T> operator-(const Dual<N, T>& a) {
    Dual<N, T> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
}
GFK_DUAL Dual<N, T> operator*(const Dual<N, T>& a, const Dual<N, T>& b) {
    Dual<N, T> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
GFK_DUAL Dual<N, T> operator/(const Dual<N, T>& a, const Dual<N, T>& b) {
    Dual<N, T> r;
    const T ib = T(1) / b.v;
    r.v = a.v * ib;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
GFK_DUAL Dual<N, T> operator+(const Dual<N, T>& a, T b) { Dual<N, T> r = a; r.v += b; return r; }
GFK_DUAL Dual<N, T> operator+(T a, const Dual<N, T>& b) { return b + a; }
GFK_DUAL Dual<N, T> operator-(const Dual<N, T>& a, T b) { Dual<N, T> r = a; r.v -= b; return r; }
GFK_DUAL Dual<N, T> operator-(T a, const Dual<N, T>& b) { return -(b - a); }
GFK_DUAL Dual<N, T> operator*(const Dual<N, T>& a, T b) {
    Dual<N, T> r;
    r.v = a.v * b;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
    return r;
}
GFK_DUAL Dual<N, T> operator*(T a, const Dual<N, T>& b) { return b * a; }
GFK_DUAL Dual<N, T>& operator+=(Dual<N, T>& a, const Dual<N, T>& b) { a = a + b; return a; }
GFK_DUAL Dual<N, T>& operator-=(Dual<N, T>& a, const Dual<N, T>& b) { a = a - b; return a; }

GFK_DUAL bool operator<(const Dual<N, T>& a, const Dual<N, T>& b) { return a.v < b.v; }
GFK_DUAL bool operator>(const Dual<N, T>& a, const Dual<N, T>& b) { return a.v > b.v; }
GFK_DUAL bool operator<(const Dual<N, T>& a, T b) { return a.v < b; }
GFK_DUAL bool operator>(const Dual<N, T>& a, T b) { return a.v > b; }

// sqrt(s) and 1/sqrt(s): d sqrt = ds / (2 sqrt)
template <int N, typename T>
__device__ __forceinline__ void radius(const Dual<N, T>& s, Dual<N, T>& r, Dual<N, T>& i) {
    const T rv = sqrt(s.v);
    const T iv = T(1) / rv;
    r.v = rv;
    i.v = iv;
    const T half_i = T(0.5) * iv;             // d r / d s
    const T di = -half_i * iv * iv;           // d (1/r) / d s = -1 / (2 r^3)
#pragma unroll
    for (int k = 0; k < N; ++k) {
        r.d[k] = half_i * s.d[k];
        i.d[k] = di * s.d[k];
    }
}
GFK_DUAL Dual<N, T> rcp(const Dual<N, T>& a) {
    Dual<N, T> r;
    r.v = T(1) / a.v;
    const T m = -r.v * r.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = m * a.d[i];
    return r;
}
GFK_DUAL Dual<N, T> expn(const Dual<N, T>& a) {
    Dual<N, T> r;
    r.v = exp(a.v);
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = r.v * a.d[i];
    return r;
}
GFK_DUAL Dual<N, T> fmin(const Dual<N, T>& a, const Dual<N, T>& b) { return b.v < a.v ? b : a; }
GFK_DUAL Dual<N, T> fmax(const Dual<N, T>& a, const Dual<N, T>& b) { return b.v > a.v ? b : a; }
GFK_DUAL bool finite_(const Dual<N, T>& a) { return isfinite(a.v); }

#undef GFK_DUAL

}  // namespace gfk
