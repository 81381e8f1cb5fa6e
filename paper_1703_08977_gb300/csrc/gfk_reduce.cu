// Deferred population reduction (space averaging over the replications) and
// small output kernels.
//
// reduce_rows_kernel: for one instance and one step, merges the instance's
// block records {c_b, W_b, P_b, Q_b, R_b, n_b} into
//   C = max_b c_b,  W = sum_b W_b e^{c_b - C},  P = sum_b P_b e^{c_b - C},
//   Q = sum_b Q_b e^{2 (c_b - C)},  R = sum_b R_b e^{c_b - C},  n = sum_b n_b.
// W and P (the energy's denominator and numerator: Eq. 4's z(t) and the
// space-averaged energy) are carried as unevaluated double-doubles on both
// paths -- a Neumaier-compensated sum per thread, TwoSum across the threads
// of a warp and across warps -- so E = P / W is the quotient of sums correct
// to O(2^-100) relative, independent of the number of blocks and of their
// order.  Q and R (effective sample size, variance) are plain FP64 sums;
// n is an integer count, exact in FP64.  The shifts c_b are integer-valued, so
// the factors e^{c_b - C} for C - c_b < kExpTable come from a table the block
// fills once with the same exp calls (the FP64 exponential per record was what
// bounded this kernel); larger or non-integer gaps call exp directly.
// finalize_kernel turns merged rows into E(t) = P/W, ln z(t) = C + ln W - ln N
// and ESS = W^2/Q (Eq. 4's z(t) and the space-averaged energy).
#include <cuda_runtime.h>

#include "gfk_device.cuh"
#include "gfk_types.h"

namespace gfk {

struct DD { double hi, lo; };

__device__ __forceinline__ DD dd_add(DD a, DD b) {
    double s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __dadd_rn(e, __dadd_rn(a.lo, b.lo));
    double hi = __dadd_rn(s, e);
    double lo = __dsub_rn(e, __dsub_rn(hi, s));
    DD r = {hi, lo};
    return r;
}

__device__ __forceinline__ DD dd_shfl_xor(DD v, int o) {
    DD r;
    r.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    r.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    return r;
}

constexpr int kReduceThreads = 256;
constexpr int kExpTable = 64;   // e^{-k}, k = 0 .. kExpTable - 1

__global__ void __launch_bounds__(kReduceThreads)
reduce_rows_kernel(const PartialRec* __restrict__ part, int nblk, BlockMap bm,
                   SeriesRow* __restrict__ series, int64_t series_cap, int64_t row_base) {
    __shared__ double s_max[kReduceThreads / 32];
    __shared__ DD s_acc[5][kReduceThreads / 32];
    __shared__ double s_exp[kExpTable];
    if (threadIdx.x < kExpTable) s_exp[threadIdx.x] = exp(-(double)threadIdx.x);
    const int row = blockIdx.x;
    const int inst = blockIdx.y;
    const int b0 = bm.begin[inst], b1 = bm.begin[inst + 1];
    const PartialRec* rp = part + (int64_t)row * nblk;
    // debug build: the row's records of this instance must lie in the buffer
    // (uniform over the block, so every thread returns together)
    if (b1 > b0 && !(GFK_DBG_OK(rp + b0, sizeof(PartialRec), kDbgRecord) &&
                     GFK_DBG_OK(rp + b1 - 1, sizeof(PartialRec), kDbgRecord)))
        return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    double m = -INFINITY;
    for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x)
        if (rp[b].n > 0.0) m = fmax(m, rp[b].c);
    m = warp_max(m);
    if (lane == 0) s_max[warp] = m;
    __syncthreads();
    double C = s_max[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) C = fmax(C, s_max[w]);
    if (!isfinite(C)) C = 0.0;

    // per-thread Neumaier sums for W and P, plain sums for Q, R, n
    double sW = 0.0, cW = 0.0, sP = 0.0, cP = 0.0, sQ = 0.0, sR = 0.0, sN = 0.0;
    for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
        const PartialRec r = rp[b];
        if (!(r.n > 0.0)) continue;
        const double k = C - r.c;
        double f;
        if (k >= 0.0 && k < (double)kExpTable && (double)(int)k == k) f = s_exp[(int)k];
        else f = exp(-k);
        const double w = r.W * f, p = r.P * f;
        double t = sW + w;
        cW += fabs(sW) >= fabs(w) ? (sW - t) + w : (w - t) + sW;
        sW = t;
        t = sP + p;
        cP += fabs(sP) >= fabs(p) ? (sP - t) + p : (p - t) + sP;
        sP = t;
        sQ += r.Q * f * f;
        sR += r.R * f;
        sN += r.n;
    }
    DD acc[5] = {{sW, cW}, {sP, cP}, {sQ, 0.0}, {sR, 0.0}, {sN, 0.0}};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        if (k < 2) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[k] = dd_add(acc[k], dd_shfl_xor(acc[k], o));
        } else {
            acc[k].hi = warp_sum(acc[k].hi);
        }
        if (lane == 0) s_acc[k][warp] = acc[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        DD tot[5];
        for (int k = 0; k < 5; ++k) {
            tot[k] = s_acc[k][0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                if (k < 2) tot[k] = dd_add(tot[k], s_acc[k][w]);
                else tot[k].hi += s_acc[k][w].hi;
            }
        }
        SeriesRow out;
        out.c = C;
        out.W = tot[0].hi + tot[0].lo;
        out.P = tot[1].hi + tot[1].lo;
        out.Q = tot[2].hi;
        out.R = tot[3].hi;
        out.n = tot[4].hi;
        SeriesRow* dst = series + (int64_t)inst * series_cap + row_base + row;
        if (GFK_DBG_OK(dst, sizeof(SeriesRow), kDbgSeries)) *dst = out;
    }
}

__global__ void finalize_kernel(const SeriesRow* __restrict__ rows, int64_t n, double n0,
                                double* __restrict__ e, double* __restrict__ lnz,
                                double* __restrict__ ess) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const SeriesRow r = rows[i];
    if (r.W > 0.0) {
        e[i] = r.P / r.W;
        lnz[i] = r.c + log(r.W) - log(n0);
        ess[i] = r.W * r.W / r.Q;
    } else {
        e[i] = NAN;
        lnz[i] = -INFINITY;
        ess[i] = 0.0;
    }
}

// Walkers of one instance to walker-major FP64 (x6, logw, alive).
__global__ void export_fp64_kernel(StateF64 st, int64_t off, int64_t n, double* __restrict__ x6,
                                   double* __restrict__ logw, uint8_t* __restrict__ alive) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t slot = off + i;
    if (!(GFK_DBG_OK(st.x + slot, sizeof(double), kDbgState) &&
          GFK_DBG_OK(st.x + 5 * st.stride + slot, sizeof(double), kDbgState) &&
          GFK_DBG_OK(st.logw + slot, sizeof(double), kDbgState) &&
          GFK_DBG_OK(st.sgn + slot, 1, kDbgState) &&
          GFK_DBG_OK(x6 + 6 * i, 6 * sizeof(double), kDbgSeries) &&
          GFK_DBG_OK(logw + i, sizeof(double), kDbgSeries) && GFK_DBG_OK(alive + i, 1, kDbgSeries)))
        return;
#pragma unroll
    for (int d = 0; d < 6; ++d) x6[6 * i + d] = st.x[d * st.stride + slot];
    const int sg = st.sgn[slot];
    logw[i] = sg != 0 ? st.logw[slot] : -INFINITY;
    alive[i] = sg != 0 ? 1 : 0;
}

__global__ void export_mixed_kernel(StateMixed st, int64_t off, int64_t n, double* __restrict__ x6,
                                    double* __restrict__ logw, uint8_t* __restrict__ alive) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t slot = off + i;
    if (!(GFK_DBG_OK(st.p0 + slot, sizeof(float4), kDbgState) &&
          GFK_DBG_OK(st.p1 + slot, sizeof(float4), kDbgState) &&
          GFK_DBG_OK(st.sgn + slot, 1, kDbgState) &&
          GFK_DBG_OK(x6 + 6 * i, 6 * sizeof(double), kDbgSeries) &&
          GFK_DBG_OK(logw + i, sizeof(double), kDbgSeries) && GFK_DBG_OK(alive + i, 1, kDbgSeries)))
        return;
    const float4 a = st.p0[slot];
    const float4 b = st.p1[slot];
    x6[6 * i + 0] = a.x; x6[6 * i + 1] = a.y; x6[6 * i + 2] = a.z;
    x6[6 * i + 3] = a.w; x6[6 * i + 4] = b.x; x6[6 * i + 5] = b.y;
    const long long lo = (unsigned)__float_as_int(b.z);
    const long long hi = (long long)__float_as_int(b.w);
    const int sg = st.sgn[slot];
    logw[i] = sg != 0 ? __longlong_as_double((hi << 32) | lo) : -INFINITY;
    alive[i] = sg != 0 ? 1 : 0;
}

cudaError_t launch_reduce_rows(const PartialRec* part, int nblk, const BlockMap& bm, int rows,
                               SeriesRow* series, int64_t series_cap, int64_t row_base,
                               cudaStream_t stream) {
    dim3 grid(rows, bm.n_inst);
    reduce_rows_kernel<<<grid, kReduceThreads, 0, stream>>>(part, nblk, bm, series, series_cap,
                                                            row_base);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const SeriesRow* rows, int64_t n, double n0, double* e, double* lnz,
                            double* ess, cudaStream_t stream) {
    const int th = 256;
    const int nb = (int)((n + th - 1) / th);
    finalize_kernel<<<nb, th, 0, stream>>>(rows, n, n0, e, lnz, ess);
    return cudaGetLastError();
}

cudaError_t launch_export(bool mixed, const StateF64& s64, const StateMixed& smx, int64_t off,
                          int64_t n, double* x6, double* logw, uint8_t* alive,
                          cudaStream_t stream) {
    const int th = 256;
    const int nb = (int)((n + th - 1) / th);
    if (mixed) export_mixed_kernel<<<nb, th, 0, stream>>>(smx, off, n, x6, logw, alive);
    else export_fp64_kernel<<<nb, th, 0, stream>>>(s64, off, n, x6, logw, alive);
    return cudaGetLastError();
}

}  // namespace gfk
