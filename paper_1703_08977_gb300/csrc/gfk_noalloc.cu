// gfk_propagate_noalloc: the mixed-precision walk without any allocation.
//
// Some callers cannot let a library call cudaMalloc: frameworks that own all
// device memory through their own caching allocator or a fixed arena carved
// out at start-up, and services whose memory budget is fixed for the life of
// the process (cudaMalloc synchronises the device, can fail mid-run and
// fragments memory).  This entry point serves them.  The caller passes every
// input and output buffer; the only other device memory used is the
// file-scope array below, which the CUDA runtime creates when the library is
// loaded and every GPU that loads the library holds until the process exits.
//
// The array holds the instance record and the per-(move, block) population
// records of one chunk of moves (the scratch the walk kernel writes and the
// merge kernel reads).  Every call shares it, and it keeps the last call's
// contents: each call rewrites the instance record (with a one-thread kernel
// that receives it as a launch argument, so no host buffer has to outlive the
// call) and every record it later reads, so nothing in it has to start at
// zero.  Calls whose work overlaps on the GPU (two streams, or two host
// threads) race on it.
//
// The kernels launched are the library's own mixed init / walk / merge
// kernels; only the memory they are given differs from gfk_propagate.  The
// moves of a call are walked in chunks whose lengths are multiples of the
// walk's 64-move fold window (except the last), so the FP32 log-weight
// increments are folded after the same moves as in gfk_propagate and the
// results equal gfk_propagate's bit for bit for the same sequence of calls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "gfk_launch.h"
#include "gfk_mixed_consts.h"
#include "gfk_trial_parse.h"
#include "gfk_types.h"


using namespace gfk;

namespace {

// The scratch.  Layout: [0, 4096) the InstDev record; [4096, 12288) the
// Box-Muller angle table (kAngleGrid float2); [12288, end) PartialRec records
// of one chunk, [move][block].
constexpr size_t kInstBytes = 4096;
constexpr size_t kHeaderBytes = kInstBytes + sizeof(float2) * kAngleGrid;
static_assert(sizeof(InstDev) <= kInstBytes, "instance record must fit the header");
static __device__ __align__(256) unsigned char g_noalloc_scratch[GFK_NOALLOC_SCRATCH_BYTES];

constexpr int kThreads = 256;   // launch shape of this entry point
constexpr int kWpt = 2;
// GFK_NOALLOC_MAX_WALKERS walkers need one fold window of records per chunk
static_assert((GFK_NOALLOC_SCRATCH_BYTES - kHeaderBytes) / sizeof(PartialRec) >=
                  (size_t)kRing * (GFK_NOALLOC_MAX_WALKERS / (kThreads * kWpt)),
              "the scratch must hold 64 moves of block records at the largest population");

// Writes the instance record into the scratch (one thread; the record arrives
// as a launch argument).
__global__ void put_instance_kernel(InstDev rec, InstDev* dst) { *dst = rec; }

// Device address of the scratch, looked up once per device with that device
// current (in host code the symbol itself is only a host-side stand-in).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

gfk_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return GFK_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return GFK_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = (unsigned char*)g_addr[dev];
    return GFK_OK;
}

}  // namespace

extern "C" gfk_status gfk_propagate_noalloc(const gfk_instance_desc* desc, int32_t trial_kind,
                                            const double* params, int32_t n_params,
                                            void* dev_p0, void* dev_p1, int8_t* dev_sgn,
                                            int32_t init, int64_t step0, int64_t n_steps,
                                            double* dev_rows, unsigned long long* dev_counters,
                                            void* cuda_stream) {
    if (!desc || !dev_p0 || !dev_p1 || !dev_sgn || !dev_rows || !dev_counters) return GFK_EINVAL;
    const gfk_instance_desc& d = *desc;
    if (d.prec != GFK_PREC_MIXED) return GFK_EINVAL;
    if (d.state < GFK_1S || d.state > GFK_PZ) return GFK_EINVAL;
    if (d.n_walkers < 1 || d.n_walkers > GFK_NOALLOC_MAX_WALKERS) return GFK_EINVAL;
    if (!(d.dt > 0.0) || !std::isfinite(d.dt) || !std::isfinite(d.e_trial)) return GFK_EINVAL;
    if (!(d.init_sigma > 0.0) || !std::isfinite(d.init_sigma)) return GFK_EINVAL;
    if (d.ee_on != 0 && d.ee_on != 1) return GFK_EINVAL;
    if ((uint64_t)d.walker_id0 + (uint64_t)d.n_walkers > (1ull << 32)) return GFK_EINVAL;
    if (d.noise != GFK_NOISE_GAUSSIAN && d.noise != GFK_NOISE_BERNOULLI) return GFK_EINVAL;
    if (n_steps < 0 || step0 < 0 || (init && step0 != 0)) return GFK_EINVAL;
    if (step0 + n_steps > 0xffffffffll) return GFK_EINVAL;
    if (((uintptr_t)dev_p0 | (uintptr_t)dev_p1) & 15u) return GFK_EINVAL;
    TrialHost trial;
    if (!parse_trial_params(trial_kind, params, n_params, &trial)) return GFK_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GFK_ECUDA;
    unsigned char* scratch = nullptr;
    gfk_status st = scratch_address(dev, &scratch);
    if (st != GFK_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // instance record
    InstDev inst;
    std::memset(&inst, 0, sizeof(inst));
    inst.n = d.n_walkers;
    inst.off = 0;
    inst.dt = d.dt;
    inst.sqrt_dt = std::sqrt(d.dt);
    inst.e_trial = d.e_trial;
    inst.sigma = d.init_sigma;
    inst.k0 = (uint32_t)(d.seed & 0xffffffffull);
    inst.k1 = (uint32_t)(d.seed >> 32);
    inst.stream = d.rng_stream;
    inst.id0 = d.walker_id0;
    inst.ee_on = d.ee_on ? 1 : 0;
    inst.noise = d.noise;
    const MixedConsts mc = mixed_consts(d.dt, d.e_trial, d.noise);
    inst.dt_f32 = mc.dt;
    inst.sdt_f32 = mc.sdt;
    inst.sdt_lo = mc.sdt_lo;
    inst.r2_fix = mc.r2_fix;
    inst.et_f32 = mc.et;
    inst.dt_log2e = mc.dt_log2e;
    inst.et_fix = mc.et_fix;
    inst.trial = trial;
    inst.angle_cs = (const float2*)(scratch + kInstBytes);
    InstDev* d_inst = (InstDev*)scratch;
    PartialRec* part = (PartialRec*)(scratch + kHeaderBytes);

    BlockMap bm;
    std::memset(&bm, 0, sizeof(bm));
    bm.n_inst = 1;
    bm.wpt = kWpt;
    const int64_t per_block = (int64_t)kThreads * kWpt;
    const int nblk = (int)((d.n_walkers + per_block - 1) / per_block);
    bm.begin[0] = 0;
    bm.begin[1] = nblk;
    // chunk length: as many moves as the records fit, up to 1024, rounded down
    // to a multiple of the fold window (at GFK_NOALLOC_MAX_WALKERS: 64 moves)
    const int64_t rec_cap = (int64_t)((GFK_NOALLOC_SCRATCH_BYTES - kHeaderBytes) / sizeof(PartialRec));
    int64_t rows_fit = rec_cap / nblk;
    rows_fit = rows_fit > 1024 ? 1024 : (rows_fit / kRing) * kRing;
    if (rows_fit < kRing) return GFK_EINVAL;   // cannot happen up to GFK_NOALLOC_MAX_WALKERS

    // debug build: the scratch and the caller's buffers join the checked ranges
    debug_register(scratch, GFK_NOALLOC_SCRATCH_BYTES);
    debug_register(dev_p0, sizeof(float4) * (size_t)d.n_walkers);
    debug_register(dev_p1, sizeof(float4) * (size_t)d.n_walkers);
    debug_register(dev_sgn, (size_t)d.n_walkers);
    debug_register(dev_rows, sizeof(SeriesRow) * (size_t)(n_steps + (init ? 1 : 0)));

    StateMixed sm{};
    sm.p0 = (float4*)dev_p0;
    sm.p1 = (float4*)dev_p1;
    sm.sgn = dev_sgn;
    SeriesRow* rows = (SeriesRow*)dev_rows;
    const int64_t n_rows = n_steps + (init ? 1 : 0);
    const int kind = trial.kind;

#define NA_CK(call)                                  \
    do {                                             \
        if ((call) != cudaSuccess) {                 \
            (void)cudaGetLastError();                \
            return GFK_ECUDA;                        \
        }                                            \
    } while (0)
    put_instance_kernel<<<1, 1, 0, stream>>>(inst, d_inst);
    NA_CK(cudaGetLastError());
    if (d.noise == GFK_NOISE_GAUSSIAN)
        NA_CK(fill_angle_table((float2*)(scratch + kInstBytes), stream));
    if (init) {
        NA_CK(cudaMemsetAsync(dev_counters, 0, sizeof(unsigned long long) * kNumCounters, stream));
        NA_CK(launch_init_mixed(kind, kThreads, nblk, d_inst, bm, sm, part, dev_counters, stream));
        NA_CK(launch_reduce_rows(part, nblk, bm, 1, rows, n_rows, 0, stream));
    }
    int64_t done = 0;
    while (done < n_steps) {
        const int chunk = (int)((n_steps - done) < rows_fit ? (n_steps - done) : rows_fit);
        NA_CK(launch_walk_mixed(mixed_walk_kind(kind, &trial, 1), d.noise, kWpt, kThreads, nblk,
                                0, nblk, d_inst, bm, sm,
                                (uint32_t)(step0 + done), chunk, part, dev_counters, &trial,
                                inst.ee_on, stream));
        NA_CK(launch_reduce_rows(part, nblk, bm, chunk, rows, n_rows, (init ? 1 : 0) + done,
                                 stream));
        done += chunk;
    }
#undef NA_CK
    return GFK_OK;
}
