// Instruction-throughput microbenchmarks: the ALU denominators of the walk's
// roofline, measured on the device at hand (a measurement utility; the paper
// has no counterpart).
//
// Each kernel runs kChains independent dependency chains per thread of one
// instruction (inline PTX, so the compiler keeps exactly that instruction),
// on enough blocks to fill every SM several times over.  The rate reported is
// lane operations per second: threads x chains x iterations / elapsed time.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "gfk_device.cuh"
#include "gfk_mixed_consts.h"
#include "gfk_trial_parse.h"
#include "gfk_types.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;
constexpr int kThreads = 256;

template <int OP>
__global__ void __launch_bounds__(kThreads) peak_kernel(unsigned* __restrict__ sink, unsigned seed) {
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned u[kChains];
    float f[kChains];
    double d[kChains];
    unsigned long long f2[kChains];      // packed float pairs (GFK_PEAK_FFMA2)
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        u[j] = t * 2654435761u + seed + j;
        f[j] = 1.0f + (float)(u[j] & 1023) * 1e-4f;
        d[j] = (double)f[j];
        f2[j] = ((unsigned long long)__float_as_uint(f[j]) << 32) | __float_as_uint(f[j] + 0.5f);
    }
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) {
            if (OP == GFK_PEAK_FFMA) {
                asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[j]) : "f"(0.9999f), "f"(1e-4f));
            } else if (OP == GFK_PEAK_DFMA) {
                asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(d[j]) : "d"(0.9999), "d"(1e-4));
            } else if (OP == GFK_PEAK_IMAD) {
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(u[j]) : "r"(0xD2511F53u), "r"(7u));
            } else if (OP == GFK_PEAK_IMAD_HI) {
                asm volatile("mad.hi.u32 %0, %0, %1, %0;" : "+r"(u[j]) : "r"(0xCD9E8D57u));
            } else if (OP == GFK_PEAK_IMAD_WIDE) {
                unsigned hi;
                asm volatile("{ .reg .u64 w; mad.wide.u32 w, %0, %2, 12345; mov.b64 {%0, %1}, w; }"
                             : "+r"(u[j]), "=r"(hi) : "r"(0xD2511F53u));
                u[j] ^= hi;
            } else if (OP == GFK_PEAK_LOP3) {
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(u[j]) : "r"(0x9E3779B9u), "r"(i));
            } else if (OP == GFK_PEAK_EX2) {
                asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(f[j]));
            } else if (OP == GFK_PEAK_RSQ) {
                asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(f[j]));
            } else if (OP == GFK_PEAK_LG2) {
                asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+f"(f[j]));
            } else if (OP == GFK_PEAK_SIN) {
                asm volatile("sin.approx.ftz.f32 %0, %0;" : "+f"(f[j]));
            } else if (OP == GFK_PEAK_I2F) {
                asm volatile("{ .reg .f32 v; cvt.rn.f32.u32 v, %0; mov.b32 %0, v; }" : "+r"(u[j]));
            } else if (OP == GFK_PEAK_F2F) {
                asm volatile("{ .reg .f64 v; cvt.f64.f32 v, %0; cvt.rn.f32.f64 %0, v; }" : "+f"(f[j]));
            } else if (OP == GFK_PEAK_FFMA2) {
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;"
                             : "+l"(f2[j]) : "l"(0x3F7FF9723F7FF972ull), "l"(0x38D1B71738D1B717ull));
            }
        }
    }
    unsigned acc = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        acc ^= u[j] ^ __float_as_uint(f[j]) ^ (unsigned)__double_as_longlong(d[j]) ^
               (unsigned)(f2[j] ^ (f2[j] >> 32));
    if (acc == 0x9E3779B9u) sink[0] = acc;   // practically never; keeps the chains live
}

template <int OP>
cudaError_t time_op(int blocks, unsigned* sink, cudaStream_t s, float* best_ms) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) { cudaEventDestroy(a); return e; }
    *best_ms = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(a, s);
        if (e == cudaSuccess) { peak_kernel<OP><<<blocks, kThreads, 0, s>>>(sink, rep); e = cudaGetLastError(); }
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0 && ms < *best_ms) *best_ms = ms;   // rep 0 warms up
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

}  // namespace

extern "C" gfk_status gfk_measure_peak(int32_t op, void* cuda_stream, double* lane_ops_per_s) {
    if (!lane_ops_per_s || op < 0 || op >= GFK_PEAK_COUNT) return GFK_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GFK_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GFK_ECUDA;
    const int blocks = sms * 32;   // 8 resident blocks of 256 threads per SM, 4 waves
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned* sink = nullptr;
    // 4 bytes the kernels may write; taken from the stream-ordered pool and
    // returned at the end of the call
    if (cudaMallocAsync((void**)&sink, sizeof(unsigned), s) != cudaSuccess) return GFK_ENOMEM;
    float ms = 0.f;
    cudaError_t e = cudaSuccess;
    switch (op) {
        case GFK_PEAK_FFMA: e = time_op<GFK_PEAK_FFMA>(blocks, sink, s, &ms); break;
        case GFK_PEAK_DFMA: e = time_op<GFK_PEAK_DFMA>(blocks, sink, s, &ms); break;
        case GFK_PEAK_IMAD: e = time_op<GFK_PEAK_IMAD>(blocks, sink, s, &ms); break;
        case GFK_PEAK_IMAD_HI: e = time_op<GFK_PEAK_IMAD_HI>(blocks, sink, s, &ms); break;
        case GFK_PEAK_IMAD_WIDE: e = time_op<GFK_PEAK_IMAD_WIDE>(blocks, sink, s, &ms); break;
        case GFK_PEAK_LOP3: e = time_op<GFK_PEAK_LOP3>(blocks, sink, s, &ms); break;
        case GFK_PEAK_EX2: e = time_op<GFK_PEAK_EX2>(blocks, sink, s, &ms); break;
        case GFK_PEAK_RSQ: e = time_op<GFK_PEAK_RSQ>(blocks, sink, s, &ms); break;
        case GFK_PEAK_LG2: e = time_op<GFK_PEAK_LG2>(blocks, sink, s, &ms); break;
        case GFK_PEAK_SIN: e = time_op<GFK_PEAK_SIN>(blocks, sink, s, &ms); break;
        case GFK_PEAK_I2F: e = time_op<GFK_PEAK_I2F>(blocks, sink, s, &ms); break;
        case GFK_PEAK_F2F: e = time_op<GFK_PEAK_F2F>(blocks, sink, s, &ms); break;
        case GFK_PEAK_FFMA2: e = time_op<GFK_PEAK_FFMA2>(blocks, sink, s, &ms); break;
        default: e = cudaErrorInvalidValue; break;
    }
    cudaFreeAsync(sink, s);
    if (e != cudaSuccess) return GFK_ECUDA;
    const double ops = (double)blocks * kThreads * kChains * kIters *
                       (op == GFK_PEAK_F2F || op == GFK_PEAK_FFMA2 ? 2 : 1);
    *lane_ops_per_s = ops / (ms * 1e-3);
    return GFK_OK;
}

// ---------------------------------------------------------------------------
// gfk_normal_moments: the FP32 Box-Muller generator against FP64, summed over
// every radius word (2^32) and every angle of the 1024-point grid.  One FP64
// partial per thread and quantity, one atomic add per block and quantity.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNumMoments = 6;

__device__ __forceinline__ float radius2_variant(uint32_t w, int method, float r2_fix) {
    constexpr float kInv32 = 1.0f / 4294967296.0f;
    constexpr float kHalfInv32 = 0.5f / 4294967296.0f;
    const float ua = fmaf((float)w, kInv32, kHalfInv32);
    if (method == 0) return gfk::radius2_f32(w, r2_fix);
    if (method == 1) {
        float l2;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(ua));
        return fmaxf(-1.3862943611198906f * l2, 0.0f);
    }
    return fmaxf(-2.0f * logf(ua), 0.0f);
}

__device__ __forceinline__ void block_add(double v, double* s_part, double* out) {
    v = gfk::warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) b += s_part[k];
        atomicAdd(out, b);
    }
}

__global__ void normal_moments_kernel(int method, float r2_fix, double* __restrict__ out) {
    __shared__ double s_part[8];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t first = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e_r2 = 0.0, e_rho2 = 0.0;
    for (uint64_t i = first; i < (1ull << 32); i += stride) {
        const uint32_t w = (uint32_t)i;
        const double exact = -2.0 * log(((double)w + 0.5) * (1.0 / 4294967296.0));
        const float r2 = radius2_variant(w, method, r2_fix);
        const double rho = (double)gfk::radius_f32(r2);
        e_r2 += (double)r2 - exact;
        e_rho2 += rho * rho - exact;
    }
    double c2 = 0.0, s2 = 0.0, c1 = 0.0, s1 = 0.0;
    for (uint64_t k = first; k < 1024u; k += stride) {
        const float2 cs = gfk::angle_cs_entry((uint32_t)k);   // the walk's angle table entry
        const float c = cs.x, s = cs.y;
        c2 += (double)c * (double)c - 0.5;
        s2 += (double)s * (double)s - 0.5;
        c1 += (double)c;
        s1 += (double)s;
    }
    const double v[kNumMoments] = {e_r2, e_rho2, c2, s2, c1, s1};
    for (int q = 0; q < kNumMoments; ++q) block_add(v[q], s_part, out + q);
}

}  // namespace

extern "C" gfk_status gfk_normal_moments(int32_t method, void* cuda_stream, double* moments) {
    if (!moments || method < 0 || method > 2) return GFK_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GFK_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GFK_ECUDA;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    double* d = nullptr;
    if (cudaMalloc(&d, sizeof(double) * kNumMoments) != cudaSuccess) {
        (void)cudaGetLastError();
        return GFK_ENOMEM;
    }
    double h[kNumMoments] = {0, 0, 0, 0, 0, 0};
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(double) * kNumMoments, stream);
    if (e == cudaSuccess) {
        // the kernels' radius constant for a variance of exactly 1
        const float r2_fix = (float)gfk::gaussian_r2_fix(0.0);
        normal_moments_kernel<<<sms * 8, 256, 0, stream>>>(method, r2_fix, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFree(d);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return GFK_ECUDA;
    }
    const double n_radius = 4294967296.0, n_angle = 1024.0;
    moments[0] = h[0] / n_radius;
    moments[1] = h[1] / n_radius;
    for (int q = 2; q < kNumMoments; ++q) moments[q] = h[q] / n_angle;
    return GFK_OK;
}

// ---------------------------------------------------------------------------
// gfk_eval_f32: the mixed walk's FP32 trial evaluation at given positions, one
// walker at a time (float lanes) or two at a time (float2 lanes), through the
// per-block dispatch the walk kernels use (eval_lanes, KIND 2).
// ---------------------------------------------------------------------------
namespace {

template <int W>
__global__ void eval_f32_kernel(gfk::TrialDev<float> t, int64_t n, const float* __restrict__ x,
                                float* __restrict__ b, float* __restrict__ el,
                                int* __restrict__ sign) {
    using L = typename std::conditional<W == 1, float, float2>::type;
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * W;
    if (i0 >= n) return;
    L xl[6];
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const int64_t i = i0 + j < n ? i0 + j : i0;    // an odd last walker pairs with itself
#pragma unroll
        for (int d = 0; d < 6; ++d) gfk::set_lane(xl[d], j, x[6 * i + d]);
    }
    gfk::EvalLanes<L> ev;
    gfk::eval_lanes<2, L>(t, xl, ev);
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const int64_t i = i0 + j;
        if (i >= n) break;
#pragma unroll
        for (int d = 0; d < 6; ++d) b[6 * i + d] = gfk::lane_at(ev.b[d], j);
        el[i] = gfk::lane_at(ev.el, j);
        sign[i] = ev.sign[j];
    }
}

}  // namespace

extern "C" gfk_status gfk_eval_f32(int32_t trial_kind, const double* params, int32_t n_params,
                                   int32_t ee_on, int64_t n, const float* host_x, int32_t lanes,
                                   float* host_b, float* host_el, int32_t* host_sign,
                                   void* cuda_stream) {
    if (!host_x || n < 1 || n > (1ll << 26) || (lanes != 1 && lanes != 2)) return GFK_EINVAL;
    if (ee_on != 0 && ee_on != 1) return GFK_EINVAL;
    gfk::TrialHost th;
    if (!gfk::parse_trial_params(trial_kind, params, n_params, &th)) return GFK_EINVAL;
    gfk::TrialDev<float> t;
    gfk::load_trial<float>(th, ee_on, t);
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const size_t nb = (size_t)n;
    char* d = nullptr;
    const size_t bytes = nb * (6 + 6 + 1) * sizeof(float) + nb * sizeof(int);
    if (cudaMallocAsync((void**)&d, bytes, stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return GFK_ENOMEM;
    }
    float* dx = (float*)d;
    float* db = dx + 6 * nb;
    float* del = db + 6 * nb;
    int* dsg = (int*)(del + nb);
    cudaError_t e = cudaMemcpyAsync(dx, host_x, nb * 6 * sizeof(float), cudaMemcpyHostToDevice,
                                    stream);
    const int th_per_block = 128;
    const int64_t threads = (n + lanes - 1) / lanes;
    const int blocks = (int)((threads + th_per_block - 1) / th_per_block);
    if (e == cudaSuccess) {
        if (lanes == 1) eval_f32_kernel<1><<<blocks, th_per_block, 0, stream>>>(t, n, dx, db, del, dsg);
        else eval_f32_kernel<2><<<blocks, th_per_block, 0, stream>>>(t, n, dx, db, del, dsg);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && host_b)
        e = cudaMemcpyAsync(host_b, db, nb * 6 * sizeof(float), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess && host_el)
        e = cudaMemcpyAsync(host_el, del, nb * sizeof(float), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess && host_sign)
        e = cudaMemcpyAsync(host_sign, dsg, nb * sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFreeAsync(d, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return GFK_ECUDA;
    }
    return GFK_OK;
}
