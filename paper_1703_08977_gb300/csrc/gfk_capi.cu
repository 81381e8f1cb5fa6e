// C ABI of the GFK walker library (declared in include/gfk.h): argument
// checking, device memory, launch shapes and the order of kernel launches.
// All arithmetic of the walk runs in the kernels of gfk_fp64.cu, gfk_mixed.cu
// and gfk_reduce.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gfk_launch.h"
#include "gfk_mixed_consts.h"
#include "gfk_trial_parse.h"
#include "gfk_types.h"

using namespace gfk;

struct gfk_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int prec = GFK_PREC_FP64;
    int noise = GFK_NOISE_GAUSSIAN;     // shared by every instance
    int n_inst = 0;
    std::vector<gfk_instance_desc> desc;
    std::vector<TrialHost> trial;
    std::vector<int> has_trial;
    std::vector<int64_t> off;     // first slot per instance
    int64_t n_slots = 0;
    InstDev* d_inst = nullptr;
    float2* d_angle_cs = nullptr;   // mixed path: the Box-Muller angle table
    // state
    StateF64 s64{};
    StateMixed smx{};
    // per-step block records for one chunk, double-buffered: chunk c writes
    // part_buf[c % 2] while the merge of chunk c - 1 reads the other buffer on
    // merge_stream (part == part_buf[0], one allocation)
    PartialRec* part = nullptr;
    PartialRec* part_buf[2] = {nullptr, nullptr};
    int64_t part_records = 0;     // capacity in records of each buffer
    // low priority: fills the walks' idle tails.  The ordering by priority
    // holds fully under graph replay (graph_stream and the auxiliary streams
    // have the highest priority); without graphs the first launch of a chunk
    // runs on the caller's stream, whose priority is usually the default
    // (lowest) one, so a merge then competes with it on equal terms
    cudaStream_t merge_stream = nullptr;
    cudaEvent_t ev_walked[2] = {nullptr, nullptr}, ev_merged[2] = {nullptr, nullptr};
    // the specialised launches of one chunk (launch_mixed_walks) after the first
    // run concurrently on these, forked from and joined to the context's stream
    static constexpr int kAuxStreams = 3;
    cudaStream_t aux_stream[kAuxStreams] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_aux[kAuxStreams] = {nullptr, nullptr, nullptr};
    // merged per-step sums, [inst][series_cap]
    SeriesRow* series = nullptr;
    int64_t series_cap = 0;
    unsigned long long* counters = nullptr;
    // output staging for gfk_energy / gfk_get_walkers, grown on demand
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // gfk_grad's working memory (checkpoints, segment, state copy), kept
    // between calls and grown on demand
    void* grad_ws = nullptr;
    size_t grad_ws_bytes = 0;
    // launch shape
    int threads = 128;
    int wpt = 1;
    int64_t part_budget_bytes = 256ll << 20;
    // CUDA-graph replay of gfk_propagate (gfk_set_graph)
    bool use_graph = false;
    struct GraphEntry {
        int64_t step0, n_steps, nblk;
        int init, threads, wpt;
        uint64_t trial_hash;            // single-instance walks take the trial as an argument
        int64_t kernels;                // kernels the graph launches
        const void* series;
        const void* part;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
    // graphs are captured and launched on a private stream, ordered against
    // the caller's stream by events (the legacy default stream cannot capture)
    cudaStream_t graph_stream = nullptr;
    cudaEvent_t graph_fork = nullptr, graph_join = nullptr;
    // kernel timing (gfk_profile)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;     // pairs: [2k] start, [2k+1] stop
    int64_t ev_used = 0;                  // pairs recorded since the last read
    int64_t prof_launches = 0;
    int64_t kernels = 0;                 // kernels queued by gfk_propagate (gfk_kernel_count)
    double prof_ms = 0.0;
    double prof_walker_steps = 0.0;
    // progress
    bool initialized = false;
    bool params_dirty = true;
    int64_t steps = 0;
    std::string last_error;
};

namespace {

// An NVTX range around one C-ABI call (header-only NVTX: a no-op unless a
// profiler that records NVTX ranges is attached), so that timelines show
// create / propagate / energy / grad around the kernels they launch.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

int g_fault_alloc_countdown = -1;   // GFK_FAULT_ALLOC=n: the n-th allocation fails

void read_fault_env() {
    static bool done = false;
    if (done) return;
    done = true;
    const char* v = std::getenv("GFK_FAULT_ALLOC");
    if (v && *v) g_fault_alloc_countdown = std::atoi(v);
}

gfk_status cuda_fail(gfk_ctx* ctx, cudaError_t e, const char* what) {
    if (ctx) {
        ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
    }
    (void)cudaGetLastError();   // clear it, so the next launch check does not see it again
    return GFK_ECUDA;
}

#define GFK_CK(ctx, call)                                    \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// Device allocation with the host-side fault-injection hook.
gfk_status dev_alloc(gfk_ctx* ctx, void** p, size_t bytes) {
    read_fault_env();
    *p = nullptr;
    if (g_fault_alloc_countdown > 0 && --g_fault_alloc_countdown == 0) {
        ctx->last_error = "allocation failure injected by GFK_FAULT_ALLOC";
        return GFK_ENOMEM;
    }
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        ctx->last_error = "cudaMalloc: out of device memory";
        return GFK_ENOMEM;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    debug_register(*p, bytes);
    return GFK_OK;
}

void dev_free(void* p) {
    if (!p) return;
    debug_unregister(p);
    cudaFree(p);
}

// Grows a device buffer of the context to at least `bytes` (its contents are
// not kept); the stream is synchronised first, as work queued on it may still
// use the old buffer.
gfk_status ensure_buffer(gfk_ctx* ctx, void** buf, size_t* cap, size_t bytes) {
    if (bytes <= *cap) return GFK_OK;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    dev_free(*buf);
    *buf = nullptr;
    *cap = 0;
    gfk_status st = dev_alloc(ctx, buf, bytes);
    if (st == GFK_OK) *cap = bytes;
    return st;
}

gfk_status ensure_scratch(gfk_ctx* ctx, size_t bytes) {
    return ensure_buffer(ctx, &ctx->scratch, &ctx->scratch_bytes, bytes);
}

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; prev = -1; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool finite_d(double v) { return std::isfinite(v); }

gfk_status parse_trial(int kind, const double* p, int np, TrialHost* t) {
    return parse_trial_params(kind, p, np, t) ? GFK_OK : GFK_EINVAL;
}

int64_t blocks_for(int64_t n, int threads, int wpt) {
    const int64_t per = (int64_t)threads * wpt;
    return (n + per - 1) / per;
}

BlockMap make_block_map(const gfk_ctx* ctx, int64_t* nblk_total) {
    BlockMap bm;
    std::memset(&bm, 0, sizeof(bm));
    bm.n_inst = ctx->n_inst;
    bm.wpt = ctx->wpt;
    int64_t b = 0;
    for (int i = 0; i < ctx->n_inst; ++i) {
        bm.begin[i] = (int32_t)b;
        b += blocks_for(ctx->desc[i].n_walkers, ctx->threads, ctx->wpt);
    }
    bm.begin[ctx->n_inst] = (int32_t)b;
    *nblk_total = b;
    return bm;
}

int launch_kind(const gfk_ctx* ctx) {
    int k = ctx->trial[0].kind;
    for (int i = 1; i < ctx->n_inst; ++i)
        if (ctx->trial[i].kind != k) return 2;
    return k;
}

// The kind the mixed walk kernels are launched with (gfk_launch.h).
int mixed_kind(const gfk_ctx* ctx) {
    return mixed_walk_kind(launch_kind(ctx), ctx->trial.data(), ctx->n_inst);
}

// Launches of one chunk of the mixed walk.  A context of several instances is
// split into runs of consecutive instances that share the specialised kernel
// kind, one launch each, provided every run has at least kMinSegmentBlocks
// blocks to fill the GPU; otherwise one launch covers all instances.  A launch
// whose instances all have the same trial function (and e-e switch) takes that
// function as a launch argument.
struct WalkSegment {
    int kind, i0, i1;
};

bool same_trials(const gfk_ctx* ctx, int i0, int i1) {
    for (int i = i0 + 1; i < i1; ++i)
        if (std::memcmp(&ctx->trial[i], &ctx->trial[i0], sizeof(TrialHost)) != 0 ||
            ctx->desc[i].ee_on != ctx->desc[i0].ee_on)
            return false;
    return true;
}
constexpr int64_t kMinSegmentBlocks = 1024;

std::vector<WalkSegment> walk_segments(const gfk_ctx* ctx, const BlockMap& bm) {
    std::vector<WalkSegment> v;
    if (ctx->n_inst > 1) {
        for (int i = 0; i < ctx->n_inst; ++i) {
            const int k = mixed_walk_kind(ctx->trial[i].kind, &ctx->trial[i], 1);
            if (!v.empty() && v.back().kind == k) v.back().i1 = i + 1;
            else v.push_back({k, i, i + 1});
        }
        bool big = v.size() > 1;
        for (const WalkSegment& g : v)
            if (bm.begin[g.i1] - bm.begin[g.i0] < kMinSegmentBlocks) big = false;
        if (big) return v;
        v.clear();
    }
    v.push_back({mixed_kind(ctx), 0, ctx->n_inst});
    return v;
}

// The launches of one chunk touch disjoint blocks, walker slots and record
// columns, so launches 2, 3, ... run on the auxiliary streams, concurrently
// with the first (no launch then waits for another's last partial wave).
// Every auxiliary stream that was forked is joined back to the context's
// stream before this returns, also when a launch fails (a capture would
// otherwise end with unjoined work); the first error is returned.
cudaError_t launch_mixed_walks(gfk_ctx* ctx, const BlockMap& bm, int64_t nblk, uint32_t step0,
                               int chunk, PartialRec* part) {
    const std::vector<WalkSegment> segs = walk_segments(ctx, bm);
    const bool fork = segs.size() > 1 && ctx->aux_stream[0] != nullptr;
    const int n_aux = fork ? (int)std::min<size_t>(segs.size() - 1, gfk_ctx::kAuxStreams) : 0;
    cudaError_t e = cudaSuccess;
    int n_forked = 0;
    if (fork) {
        e = cudaEventRecord(ctx->ev_fork, ctx->stream);
        for (int j = 0; j < n_aux && e == cudaSuccess; ++j) {
            e = cudaStreamWaitEvent(ctx->aux_stream[j], ctx->ev_fork, 0);
            if (e == cudaSuccess) ++n_forked;
        }
    }
    for (size_t k = 0; k < segs.size() && e == cudaSuccess; ++k) {
        const WalkSegment& g = segs[k];
        const bool one = same_trials(ctx, g.i0, g.i1);
        cudaStream_t s = (fork && k > 0) ? ctx->aux_stream[(k - 1) % gfk_ctx::kAuxStreams]
                                         : ctx->stream;
        e = launch_walk_mixed(
            g.kind, ctx->noise, ctx->wpt, ctx->threads, (int)nblk, bm.begin[g.i0],
            bm.begin[g.i1] - bm.begin[g.i0], ctx->d_inst, bm, ctx->smx, step0, chunk, part,
            ctx->counters, one ? &ctx->trial[g.i0] : nullptr, ctx->desc[g.i0].ee_on, s);
    }
    for (int j = 0; j < n_forked; ++j) {
        cudaError_t ej = cudaEventRecord(ctx->ev_aux[j], ctx->aux_stream[j]);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(ctx->stream, ctx->ev_aux[j], 0);
        if (e == cudaSuccess) e = ej;
    }
    return e;
}

cudaError_t prepare_mixed_walks(const gfk_ctx* ctx, const BlockMap& bm) {
    for (const WalkSegment& g : walk_segments(ctx, bm)) {
        const cudaError_t e = prepare_walk_mixed(g.kind, ctx->noise, ctx->wpt, ctx->threads,
                                                 same_trials(ctx, g.i0, g.i1));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

gfk_status upload_instances(gfk_ctx* ctx) {
    std::vector<InstDev> h(ctx->n_inst);
    for (int i = 0; i < ctx->n_inst; ++i) {
        const gfk_instance_desc& d = ctx->desc[i];
        InstDev& v = h[i];
        std::memset(&v, 0, sizeof(v));
        v.n = d.n_walkers;
        v.off = ctx->off[i];
        v.dt = d.dt;
        v.sqrt_dt = std::sqrt(d.dt);
        v.e_trial = d.e_trial;
        v.sigma = d.init_sigma;
        v.k0 = (uint32_t)(d.seed & 0xffffffffull);
        v.k1 = (uint32_t)(d.seed >> 32);
        v.stream = d.rng_stream;
        v.id0 = d.walker_id0;
        v.ee_on = d.ee_on ? 1 : 0;
        v.noise = d.noise;
        const MixedConsts mc = mixed_consts(d.dt, d.e_trial, d.noise);
        v.dt_f32 = mc.dt;
        v.sdt_f32 = mc.sdt;
        v.sdt_lo = mc.sdt_lo;
        v.r2_fix = mc.r2_fix;
        v.et_f32 = mc.et;
        v.dt_log2e = mc.dt_log2e;
        v.et_fix = mc.et_fix;
        v.angle_cs = ctx->d_angle_cs;
        v.trial = ctx->trial[i];
    }
    GFK_CK(ctx, cudaMemcpyAsync(ctx->d_inst, h.data(), sizeof(InstDev) * ctx->n_inst,
                                cudaMemcpyHostToDevice, ctx->stream));
    // the host vector dies at return: wait for the copy
    GFK_CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->params_dirty = false;
    return GFK_OK;
}

// Ensures room for `rows` chunk rows of block records in each of the two
// buffers, and the merge stream and its events; returns the rows that fit.
gfk_status ensure_partials(gfk_ctx* ctx, int64_t nblk, int64_t* rows_fit) {
    int64_t rows = ctx->part_budget_bytes / (int64_t)(nblk * sizeof(PartialRec));
    rows = std::max<int64_t>(kRing, std::min<int64_t>(rows, 1024));
    rows = (rows / kRing) * kRing;
    const int64_t need = rows * nblk;
    if (need > ctx->part_records) {
        // the old buffers may still be read by queued kernels (the caller's
        // stream waits for every merge it queued)
        GFK_CK(ctx, cudaStreamSynchronize(ctx->stream));
        dev_free(ctx->part);
        ctx->part = ctx->part_buf[0] = ctx->part_buf[1] = nullptr;
        ctx->part_records = 0;
        void* p = nullptr;
        gfk_status st = dev_alloc(ctx, &p, 2 * sizeof(PartialRec) * (size_t)need);
        if (st != GFK_OK) return st;
        ctx->part = ctx->part_buf[0] = (PartialRec*)p;
        ctx->part_buf[1] = ctx->part + need;
        ctx->part_records = need;
    }
    if (!ctx->merge_stream) {
        int least = 0, greatest = 0;
        GFK_CK(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest));
        GFK_CK(ctx, cudaStreamCreateWithPriority(&ctx->merge_stream, cudaStreamNonBlocking, least));
        for (int b = 0; b < 2; ++b) {
            GFK_CK(ctx, cudaEventCreateWithFlags(&ctx->ev_walked[b], cudaEventDisableTiming));
            GFK_CK(ctx, cudaEventCreateWithFlags(&ctx->ev_merged[b], cudaEventDisableTiming));
        }
        GFK_CK(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
        for (int j = 0; j < gfk_ctx::kAuxStreams; ++j) {
            GFK_CK(ctx, cudaStreamCreateWithPriority(&ctx->aux_stream[j], cudaStreamNonBlocking,
                                                     greatest));
            GFK_CK(ctx, cudaEventCreateWithFlags(&ctx->ev_aux[j], cudaEventDisableTiming));
        }
    }
    *rows_fit = rows;
    return GFK_OK;
}

gfk_status ensure_series(gfk_ctx* ctx, int64_t rows_needed) {
    if (rows_needed <= ctx->series_cap) return GFK_OK;
    int64_t cap = std::max<int64_t>(rows_needed, std::max<int64_t>(2 * ctx->series_cap, 1024));
    void* p = nullptr;
    gfk_status st = dev_alloc(ctx, &p, sizeof(SeriesRow) * (size_t)cap * ctx->n_inst);
    if (st != GFK_OK) return st;
    SeriesRow* ns = (SeriesRow*)p;
    if (ctx->series && ctx->series_cap > 0) {
        for (int i = 0; i < ctx->n_inst; ++i) {
            cudaError_t e = cudaMemcpyAsync(ns + (int64_t)i * cap, ctx->series + (int64_t)i * ctx->series_cap,
                                            sizeof(SeriesRow) * ctx->series_cap,
                                            cudaMemcpyDeviceToDevice, ctx->stream);
            if (e != cudaSuccess) { dev_free(ns); return cuda_fail(ctx, e, "cudaMemcpyAsync(series)"); }
        }
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) { dev_free(ns); return cuda_fail(ctx, e, "cudaStreamSynchronize"); }
        dev_free(ctx->series);
    }
    ctx->series = ns;
    ctx->series_cap = cap;
    return GFK_OK;
}

// Buffers and the instance table for a population that is about to start.
gfk_status prepare_population(gfk_ctx* ctx) {
    for (int i = 0; i < ctx->n_inst; ++i)
        if (!ctx->has_trial[i]) return GFK_ESTATE;
    if (ctx->params_dirty) {
        gfk_status st = upload_instances(ctx);
        if (st != GFK_OK) return st;
    }
    return ensure_series(ctx, 1);
}

// Queues the initial population (positions, signs, log-weights) and its sums.
gfk_status enqueue_init(gfk_ctx* ctx, const BlockMap& bm, int64_t nblk) {
    GFK_CK(ctx, cudaMemsetAsync(ctx->counters, 0, sizeof(unsigned long long) * kNumCounters * ctx->n_inst,
                                ctx->stream));
    const int kind = launch_kind(ctx);
    if (ctx->prec == GFK_PREC_FP64) {
        GFK_CK(ctx, launch_init_fp64(kind, ctx->threads, (int)nblk, ctx->d_inst, bm, ctx->s64,
                                     ctx->part, ctx->counters, ctx->stream));
    } else {
        GFK_CK(ctx, launch_init_mixed(kind, ctx->threads, (int)nblk, ctx->d_inst, bm, ctx->smx,
                                      ctx->part, ctx->counters, ctx->stream));
    }
    GFK_CK(ctx, launch_reduce_rows(ctx->part, (int)nblk, bm, 1, ctx->series, ctx->series_cap, 0,
                                   ctx->stream));
    ctx->kernels += 2;                                  // the init and its merge
    return GFK_OK;
}

gfk_status profile_pair(gfk_ctx* ctx, cudaEvent_t* a, cudaEvent_t* b);

// Queues n_steps moves from global step step_begin in chunks of rows_fit.
// Chunk c's walk writes records buffer c % 2 on the context's stream; its
// merge runs on the low-priority merge stream, so that its blocks take the
// slots the next walk leaves idle in its last partial wave.  The walk of
// chunk c waits for the merge of chunk c - 2 (the same buffer), and the
// context's stream waits for every merge queued before this returns, on
// success and on failure alike (in a graph capture these waits join the merge
// stream into the graph).
gfk_status enqueue_moves(gfk_ctx* ctx, const BlockMap& bm, int64_t nblk, int64_t rows_fit,
                         int64_t step_begin, int64_t n_steps, bool events) {
    const int kind = launch_kind(ctx);
    int64_t walkers = 0;
    for (int i = 0; i < ctx->n_inst; ++i) walkers += ctx->desc[i].n_walkers;
    int64_t done = 0;
    int64_t c = 0;                                      // chunk index
    bool merged_any[2] = {false, false};
    gfk_status st = GFK_OK;
#define EM_CK(call)                                                    \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) { st = cuda_fail(ctx, e_, #call); goto join; } \
    } while (0)
    while (done < n_steps) {
        const int chunk = (int)std::min<int64_t>(n_steps - done, rows_fit);
        const uint32_t step0 = (uint32_t)(step_begin + done);
        const int b = (int)(c & 1);
        PartialRec* const part = ctx->part_buf[b];
        if (c >= 2) EM_CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_merged[b], 0));
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (events) {
            st = profile_pair(ctx, &ev0, &ev1);
            if (st != GFK_OK) goto join;
        }
        if (ev0) EM_CK(cudaEventRecord(ev0, ctx->stream));
        if (ctx->prec == GFK_PREC_FP64) {
            EM_CK(launch_walk_fp64(kind, ctx->noise, ctx->threads, (int)nblk, ctx->d_inst,
                                   bm, ctx->s64, step0, chunk, part, ctx->counters, ctx->stream));
        } else {
            EM_CK(launch_mixed_walks(ctx, bm, nblk, step0, chunk, part));
            ctx->kernels += (int64_t)walk_segments(ctx, bm).size() - 1;   // + 1 below
        }
        if (ev1) {
            EM_CK(cudaEventRecord(ev1, ctx->stream));
            ctx->prof_launches += 1;
            ctx->prof_walker_steps += (double)walkers * chunk;
        }
        ctx->kernels += 2;                              // the walk and the merge
        EM_CK(cudaEventRecord(ctx->ev_walked[b], ctx->stream));
        EM_CK(cudaStreamWaitEvent(ctx->merge_stream, ctx->ev_walked[b], 0));
        merged_any[b] = true;
        EM_CK(launch_reduce_rows(part, (int)nblk, bm, chunk, ctx->series,
                                 ctx->series_cap, step_begin + done + 1,
                                 ctx->merge_stream));
        EM_CK(cudaEventRecord(ctx->ev_merged[b], ctx->merge_stream));
        done += chunk;
        ++c;
    }
#undef EM_CK
join:
    // the merge stream's work (including whatever a failed step left queued on
    // it) is ordered before anything later on the context's stream
    for (int b = 0; b < 2; ++b) {
        if (!merged_any[b]) continue;
        cudaError_t e = cudaEventRecord(ctx->ev_merged[b], ctx->merge_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_merged[b], 0);
        if (e != cudaSuccess && st == GFK_OK) st = cuda_fail(ctx, e, "join of the merge stream");
    }
    return st;
}

gfk_status check_inst(gfk_ctx* ctx, int32_t inst) {
    if (!ctx) return GFK_EINVAL;
    if (inst < 0 || inst >= ctx->n_inst) return GFK_EINVAL;
    return GFK_OK;
}

void free_all(gfk_ctx* ctx) {
    dev_free(ctx->d_inst);
    dev_free(ctx->d_angle_cs);
    dev_free(ctx->s64.x);
    dev_free(ctx->s64.logw);
    dev_free(ctx->smx.p0);
    dev_free(ctx->smx.p1);
    dev_free(ctx->s64.sgn);
    dev_free(ctx->smx.sgn);
    dev_free(ctx->part);
    dev_free(ctx->scratch);
    dev_free(ctx->grad_ws);
    dev_free(ctx->series);
    dev_free(ctx->counters);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    ctx->ev_pool.clear();
    for (auto& gph : ctx->graphs) cudaGraphExecDestroy(gph.exec);
    ctx->graphs.clear();
    for (int b = 0; b < 2; ++b) {
        if (ctx->ev_walked[b]) cudaEventDestroy(ctx->ev_walked[b]);
        if (ctx->ev_merged[b]) cudaEventDestroy(ctx->ev_merged[b]);
        ctx->ev_walked[b] = ctx->ev_merged[b] = nullptr;
    }
    if (ctx->merge_stream) cudaStreamDestroy(ctx->merge_stream);
    ctx->merge_stream = nullptr;
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    ctx->ev_fork = nullptr;
    for (int j = 0; j < gfk_ctx::kAuxStreams; ++j) {
        if (ctx->aux_stream[j]) cudaStreamDestroy(ctx->aux_stream[j]);
        if (ctx->ev_aux[j]) cudaEventDestroy(ctx->ev_aux[j]);
        ctx->aux_stream[j] = nullptr;
        ctx->ev_aux[j] = nullptr;
    }
    if (ctx->graph_fork) cudaEventDestroy(ctx->graph_fork);
    if (ctx->graph_join) cudaEventDestroy(ctx->graph_join);
    if (ctx->graph_stream) cudaStreamDestroy(ctx->graph_stream);
    ctx->graph_fork = ctx->graph_join = nullptr;
    ctx->graph_stream = nullptr;
}

// Harvests recorded event pairs into the running tallies.
gfk_status profile_harvest(gfk_ctx* ctx) {
    if (ctx->ev_used == 0) return GFK_OK;
    GFK_CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int64_t k = 0; k < ctx->ev_used; ++k) {
        float ms = 0.f;
        GFK_CK(ctx, cudaEventElapsedTime(&ms, ctx->ev_pool[2 * k], ctx->ev_pool[2 * k + 1]));
        ctx->prof_ms += ms;
    }
    ctx->ev_used = 0;
    return GFK_OK;
}

// Event pair for the next walk launch (NULLs when profiling is off).
gfk_status profile_pair(gfk_ctx* ctx, cudaEvent_t* a, cudaEvent_t* b) {
    *a = *b = nullptr;
    if (!ctx->profiling) return GFK_OK;
    if (ctx->ev_used >= 4096) {
        gfk_status st = profile_harvest(ctx);
        if (st != GFK_OK) return st;
    }
    while ((int64_t)ctx->ev_pool.size() < 2 * (ctx->ev_used + 1)) {
        cudaEvent_t e;
        GFK_CK(ctx, cudaEventCreate(&e));
        ctx->ev_pool.push_back(e);
    }
    *a = ctx->ev_pool[2 * ctx->ev_used];
    *b = ctx->ev_pool[2 * ctx->ev_used + 1];
    ++ctx->ev_used;
    return GFK_OK;
}

// Checkpoint blob header.
struct BlobHeader {
    char magic[8];
    int32_t version, n_inst, prec, initialized;
    int64_t n_slots, steps, series_rows;
    uint64_t desc_hash;
};

uint64_t fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char* c = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
    return h;
}

uint64_t desc_hash(const gfk_ctx* ctx) {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < ctx->n_inst; ++i) {
        const gfk_instance_desc& d = ctx->desc[i];
        h = fnv1a(&d.state, sizeof(d.state), h);
        h = fnv1a(&d.prec, sizeof(d.prec), h);
        h = fnv1a(&d.n_walkers, sizeof(d.n_walkers), h);
        h = fnv1a(&d.dt, sizeof(d.dt), h);
        h = fnv1a(&d.e_trial, sizeof(d.e_trial), h);
        h = fnv1a(&d.seed, sizeof(d.seed), h);
        h = fnv1a(&d.rng_stream, sizeof(d.rng_stream), h);
        h = fnv1a(&d.ee_on, sizeof(d.ee_on), h);
        h = fnv1a(&d.init_sigma, sizeof(d.init_sigma), h);
        h = fnv1a(&d.walker_id0, sizeof(d.walker_id0), h);
        h = fnv1a(&d.noise, sizeof(d.noise), h);
        h = fnv1a(&ctx->trial[i], sizeof(TrialHost), h);
    }
    return h;
}

size_t state_bytes(const gfk_ctx* ctx) {
    if (ctx->prec == GFK_PREC_FP64) return (size_t)ctx->n_slots * (7 * sizeof(double) + 1);
    return (size_t)ctx->n_slots * (2 * sizeof(float4) + 1);
}

}  // namespace

extern "C" {

const char* gfk_status_string(gfk_status s) {
    switch (s) {
        case GFK_OK: return "ok";
        case GFK_EINVAL: return "invalid argument";
        case GFK_ENOMEM: return "out of memory";
        case GFK_ECUDA: return "CUDA error";
        case GFK_ESTATE: return "call not valid in the current state";
        case GFK_ENONFINITE: return "walkers killed for non-finite drift or local energy";
        case GFK_EOVERFLOW: return "caller buffer too small";
        case GFK_ETIMEOUT: return "timeout";
    }
    return "unknown status";
}

const char* gfk_last_error(gfk_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

gfk_status gfk_create(const gfk_instance_desc* inst, int32_t n_inst, void* cuda_stream,
                      gfk_ctx** out) {
    NvtxRange nvtx_("gfk_create");
    if (!out) return GFK_EINVAL;
    *out = nullptr;
    if (!inst || n_inst < 1 || n_inst > GFK_MAX_INSTANCES) return GFK_EINVAL;
    int64_t total = 0;
    for (int i = 0; i < n_inst; ++i) {
        const gfk_instance_desc& d = inst[i];
        if (d.state < GFK_1S || d.state > GFK_PZ) return GFK_EINVAL;
        if (d.prec != GFK_PREC_FP64 && d.prec != GFK_PREC_MIXED) return GFK_EINVAL;
        if (d.prec != inst[0].prec) return GFK_EINVAL;
        if (d.n_walkers < 1 || d.n_walkers > 0x7fffffffll) return GFK_EINVAL;
        if (!(d.dt > 0.0) || !finite_d(d.dt)) return GFK_EINVAL;
        if (!finite_d(d.e_trial)) return GFK_EINVAL;
        if (!(d.init_sigma > 0.0) || !finite_d(d.init_sigma)) return GFK_EINVAL;
        if (d.ee_on != 0 && d.ee_on != 1) return GFK_EINVAL;
        if ((uint64_t)d.walker_id0 + (uint64_t)d.n_walkers > (1ull << 32)) return GFK_EINVAL;
        if (d.noise != GFK_NOISE_GAUSSIAN && d.noise != GFK_NOISE_BERNOULLI) return GFK_EINVAL;
        if (d.noise != inst[0].noise) return GFK_EINVAL;
        total += (d.n_walkers + 31) / 32 * 32;
    }
    if (total > (1ll << 34)) return GFK_EINVAL;

    gfk_ctx* ctx = new (std::nothrow) gfk_ctx();
    if (!ctx) return GFK_ENOMEM;
    ctx->n_inst = n_inst;
    ctx->prec = inst[0].prec;
    ctx->noise = inst[0].noise;
    ctx->desc.assign(inst, inst + n_inst);
    ctx->trial.assign(n_inst, TrialHost());
    ctx->has_trial.assign(n_inst, 0);
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->threads = 128;
    ctx->wpt = ctx->prec == GFK_PREC_FP64 ? 1 : 2;
    int64_t o = 0;
    for (int i = 0; i < n_inst; ++i) {
        ctx->off.push_back(o);
        o += (inst[i].n_walkers + 31) / 32 * 32;
    }
    ctx->n_slots = o;

    gfk_status st = GFK_OK;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) {
        st = cuda_fail(ctx, e, "cudaGetDevice");
        delete ctx;
        return st;
    }
    void* p = nullptr;
#define ALLOC(field, type, bytes)                      \
    do {                                               \
        st = dev_alloc(ctx, &p, (bytes));              \
        if (st != GFK_OK) goto fail;                   \
        field = (type)p;                               \
    } while (0)
    ALLOC(ctx->d_inst, InstDev*, sizeof(InstDev) * n_inst);
    ALLOC(ctx->counters, unsigned long long*, sizeof(unsigned long long) * kNumCounters * n_inst);
    if (ctx->prec == GFK_PREC_FP64) {
        ALLOC(ctx->s64.x, double*, sizeof(double) * 6 * ctx->n_slots);
        ALLOC(ctx->s64.logw, double*, sizeof(double) * ctx->n_slots);
        ALLOC(ctx->s64.sgn, int8_t*, ctx->n_slots);
        ctx->s64.stride = ctx->n_slots;
    } else {
        ALLOC(ctx->smx.p0, float4*, sizeof(float4) * ctx->n_slots);
        ALLOC(ctx->smx.p1, float4*, sizeof(float4) * ctx->n_slots);
        ALLOC(ctx->smx.sgn, int8_t*, ctx->n_slots);
        ALLOC(ctx->d_angle_cs, float2*, sizeof(float2) * kAngleGrid);
    }
#undef ALLOC
    e = cudaMemsetAsync(ctx->counters, 0, sizeof(unsigned long long) * kNumCounters * n_inst, ctx->stream);
    if (e != cudaSuccess) { st = cuda_fail(ctx, e, "cudaMemsetAsync"); goto fail; }
    if (ctx->d_angle_cs) {
        e = fill_angle_table(ctx->d_angle_cs, ctx->stream);
        if (e != cudaSuccess) { st = cuda_fail(ctx, e, "fill_angle_table"); goto fail; }
    }
    *out = ctx;
    return GFK_OK;
fail:
    free_all(ctx);
    delete ctx;
    return st;
}

gfk_status gfk_set_trial(gfk_ctx* ctx, int32_t inst, int32_t trial_kind, const double* params,
                         int32_t n_params) {
    gfk_status st = check_inst(ctx, inst);
    if (st != GFK_OK) return st;
    if (ctx->initialized) return GFK_ESTATE;
    TrialHost t;
    st = parse_trial(trial_kind, params, n_params, &t);
    if (st != GFK_OK) return st;
    ctx->trial[inst] = t;
    ctx->has_trial[inst] = 1;
    ctx->params_dirty = true;
    return GFK_OK;
}

gfk_status gfk_set_launch(gfk_ctx* ctx, int32_t threads_per_block, int32_t walkers_per_thread) {
    if (!ctx) return GFK_EINVAL;
    if (threads_per_block != 64 && threads_per_block != 128 && threads_per_block != 256 &&
        threads_per_block != 512)
        return GFK_EINVAL;
    if (walkers_per_thread != 1 && walkers_per_thread != 2 && walkers_per_thread != 4)
        return GFK_EINVAL;
    if (ctx->prec == GFK_PREC_FP64 && walkers_per_thread != 1) return GFK_EINVAL;
    if (walkers_per_thread == 4 && threads_per_block > kMaxThreadsWpt4) return GFK_EINVAL;
    ctx->threads = threads_per_block;
    ctx->wpt = walkers_per_thread;
    return GFK_OK;
}

gfk_status gfk_propagate(gfk_ctx* ctx, int64_t n_steps) {
    NvtxRange nvtx_("gfk_propagate");
    if (!ctx || n_steps < 0) return GFK_EINVAL;
    DeviceGuard g(ctx->device);
    if (!g.ok) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
    const bool init = !ctx->initialized;
    if (ctx->steps + n_steps > 0xffffffffll) return GFK_EINVAL;
    gfk_status st = GFK_OK;
    if (init) {
        st = prepare_population(ctx);
        if (st != GFK_OK) return st;
    }
    st = ensure_series(ctx, ctx->steps + n_steps + 1);
    if (st != GFK_OK) return st;
    int64_t nblk = 0;
    BlockMap bm = make_block_map(ctx, &nblk);
    if (nblk > 0x7fffffffll) return GFK_EINVAL;
    int64_t rows_fit = 0;
    st = ensure_partials(ctx, nblk, &rows_fit);
    if (st != GFK_OK) return st;
    const int64_t step_begin = init ? 0 : ctx->steps;

    if (ctx->use_graph && !ctx->profiling && (init || n_steps > 0)) {
        // replay a captured graph of this exact launch sequence, or capture one,
        // on the private stream, after everything queued so far on the caller's
        if (!ctx->graph_stream) {
            // the highest priority: the walks captured on it run ahead of the
            // merges captured on merge_stream (lowest), which take the slots a
            // walk leaves idle (the graph is instantiated with node priorities)
            int least = 0, greatest = 0;
            GFK_CK(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest));
            GFK_CK(ctx, cudaStreamCreateWithPriority(&ctx->graph_stream, cudaStreamNonBlocking,
                                                     greatest));
            GFK_CK(ctx, cudaEventCreateWithFlags(&ctx->graph_fork, cudaEventDisableTiming));
            GFK_CK(ctx, cudaEventCreateWithFlags(&ctx->graph_join, cudaEventDisableTiming));
        }
        cudaStream_t user = ctx->stream;
        GFK_CK(ctx, cudaEventRecord(ctx->graph_fork, user));
        GFK_CK(ctx, cudaStreamWaitEvent(ctx->graph_stream, ctx->graph_fork, 0));
        gfk_ctx::GraphEntry* hit = nullptr;
        const uint64_t th = fnv1a(ctx->trial.data(), sizeof(TrialHost) * ctx->trial.size());
        for (auto& e : ctx->graphs)
            if (e.step0 == step_begin && e.n_steps == n_steps && e.nblk == nblk &&
                e.init == (init ? 1 : 0) && e.threads == ctx->threads && e.wpt == ctx->wpt &&
                e.trial_hash == th && e.series == ctx->series && e.part == ctx->part) {
                hit = &e;
                break;
            }
        if (!hit) {
            if (ctx->prec == GFK_PREC_MIXED) GFK_CK(ctx, prepare_mixed_walks(ctx, bm));
            GFK_CK(ctx, cudaStreamBeginCapture(ctx->graph_stream, cudaStreamCaptureModeThreadLocal));
            ctx->stream = ctx->graph_stream;          // the enqueue helpers use ctx->stream
            const int64_t k_before = ctx->kernels;     // captured, not yet run
            gfk_status cs = GFK_OK;
            if (init) cs = enqueue_init(ctx, bm, nblk);
            if (cs == GFK_OK) cs = enqueue_moves(ctx, bm, nblk, rows_fit, step_begin, n_steps, false);
            ctx->stream = user;
            const int64_t k_graph = ctx->kernels - k_before;
            ctx->kernels = k_before;
            cudaGraph_t graph = nullptr;
            cudaError_t ce = cudaStreamEndCapture(ctx->graph_stream, &graph);
            if (cs != GFK_OK) {
                if (graph) cudaGraphDestroy(graph);
                return cs;
            }
            if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamEndCapture");
            cudaGraphExec_t exec = nullptr;
            ce = cudaGraphInstantiateWithFlags(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaGraphInstantiate");
            if (ctx->graphs.size() >= 8) {
                cudaGraphExecDestroy(ctx->graphs.front().exec);
                ctx->graphs.erase(ctx->graphs.begin());
            }
            ctx->graphs.push_back({step_begin, n_steps, nblk, init ? 1 : 0, ctx->threads, ctx->wpt,
                                   th, k_graph, ctx->series, ctx->part, exec});
            hit = &ctx->graphs.back();
        }
        GFK_CK(ctx, cudaGraphLaunch(hit->exec, ctx->graph_stream));
        ctx->kernels += hit->kernels;
        GFK_CK(ctx, cudaEventRecord(ctx->graph_join, ctx->graph_stream));
        GFK_CK(ctx, cudaStreamWaitEvent(user, ctx->graph_join, 0));
    } else {
        if (init) {
            st = enqueue_init(ctx, bm, nblk);
            if (st != GFK_OK) return st;
        }
        st = enqueue_moves(ctx, bm, nblk, rows_fit, step_begin, n_steps, ctx->profiling);
        if (st != GFK_OK) return st;
    }
    ctx->initialized = true;
    ctx->steps = step_begin + n_steps;
    return GFK_OK;
}

gfk_status gfk_set_graph(gfk_ctx* ctx, int32_t enable) {
    if (!ctx) return GFK_EINVAL;
    ctx->use_graph = enable != 0;
    return GFK_OK;
}

gfk_status gfk_autotune(gfk_ctx* ctx, int64_t probe_steps, int32_t* best_threads,
                        int32_t* best_wpt, double* best_rate) {
    NvtxRange nvtx_("gfk_autotune");
    if (!ctx || probe_steps < 1 || probe_steps > 4096) return GFK_EINVAL;
    DeviceGuard g(ctx->device);
    if (!ctx->initialized) {
        // start the population so the probe walks representative walkers
        gfk_status st = gfk_propagate(ctx, 0);
        if (st != GFK_OK) return st;
    }
    // keep a copy of everything the probe launches change
    const size_t sb = state_bytes(ctx);
    const size_t cb = sizeof(unsigned long long) * kNumCounters * ctx->n_inst;
    void* saved = nullptr;
    gfk_status st = dev_alloc(ctx, &saved, sb + cb);
    if (st != GFK_OK) return st;
    char* sp = (char*)saved;
    const int64_t ns = ctx->n_slots;
    auto copy_state = [&](bool save) -> cudaError_t {
        cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
        size_t o = 0;
        cudaError_t e;
        auto cp = [&](void* dev, size_t n) {
            e = save ? cudaMemcpyAsync(sp + o, dev, n, k, ctx->stream)
                     : cudaMemcpyAsync(dev, sp + o, n, k, ctx->stream);
            o += n;
            return e;
        };
        if (ctx->prec == GFK_PREC_FP64) {
            if ((e = cp(ctx->s64.x, sizeof(double) * 6 * ns)) != cudaSuccess) return e;
            if ((e = cp(ctx->s64.logw, sizeof(double) * ns)) != cudaSuccess) return e;
            if ((e = cp(ctx->s64.sgn, (size_t)ns)) != cudaSuccess) return e;
        } else {
            if ((e = cp(ctx->smx.p0, sizeof(float4) * ns)) != cudaSuccess) return e;
            if ((e = cp(ctx->smx.p1, sizeof(float4) * ns)) != cudaSuccess) return e;
            if ((e = cp(ctx->smx.sgn, (size_t)ns)) != cudaSuccess) return e;
        }
        return cp(ctx->counters, cb);
    };
    cudaError_t e = copy_state(true);
    const int thr[4] = {64, 128, 256, 512};
    const int wp[3] = {1, 2, 4};
    const int n_wp = ctx->prec == GFK_PREC_FP64 ? 1 : 3;
    int bt = ctx->threads, bw = ctx->wpt;
    double best = -1.0;
    int64_t walkers = 0;
    for (int i = 0; i < ctx->n_inst; ++i) walkers += ctx->desc[i].n_walkers;
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    const int kind = launch_kind(ctx);
    for (int ti = 0; ti < 4 && e == cudaSuccess && st == GFK_OK; ++ti) {
        for (int wi = 0; wi < n_wp && e == cudaSuccess && st == GFK_OK; ++wi) {
            if (wp[wi] == 4 && thr[ti] > kMaxThreadsWpt4) continue;   // not a compiled shape
            const int save_t = ctx->threads, save_w = ctx->wpt;
            ctx->threads = thr[ti];
            ctx->wpt = wp[wi];
            int64_t nblk = 0;
            BlockMap bm = make_block_map(ctx, &nblk);
            int64_t rows_fit = 0;
            st = ensure_partials(ctx, nblk, &rows_fit);
            const int chunk = (int)std::min<int64_t>(probe_steps, rows_fit);
            // the merge of the chunk's block records is timed too (its cost grows
            // with the number of blocks); it writes rows past the last real one,
            // which the next gfk_propagate overwrites
            if (st == GFK_OK) st = ensure_series(ctx, ctx->steps + 1 + chunk);
            float best_ms = 1e30f;
            for (int rep = 0; rep < 2 && st == GFK_OK && e == cudaSuccess; ++rep) {
                e = cudaEventRecord(a, ctx->stream);
                if (e != cudaSuccess) break;
                if (ctx->prec == GFK_PREC_FP64)
                    e = launch_walk_fp64(kind, ctx->noise, ctx->threads, (int)nblk, ctx->d_inst,
                                         bm, ctx->s64, (uint32_t)ctx->steps, chunk, ctx->part, ctx->counters,
                                         ctx->stream);
                else
                    e = launch_mixed_walks(ctx, bm, nblk, (uint32_t)ctx->steps, chunk, ctx->part);
                if (e == cudaSuccess)
                    e = launch_reduce_rows(ctx->part, (int)nblk, bm, chunk, ctx->series,
                                           ctx->series_cap, ctx->steps + 1, ctx->stream);
                if (e == cudaSuccess) e = cudaEventRecord(b, ctx->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(b);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                if (e == cudaSuccess && rep > 0 && ms < best_ms) best_ms = ms;  // rep 0 warms up
                if (e == cudaSuccess) e = copy_state(false);   // same start for every candidate
            }
            ctx->threads = save_t;
            ctx->wpt = save_w;
            const double rate = (double)walkers * chunk / (best_ms * 1e-3);
            if (e == cudaSuccess && st == GFK_OK && rate > best) {
                best = rate;
                bt = thr[ti];
                bw = wp[wi];
            }
        }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
    dev_free(saved);
    if (st != GFK_OK) return st;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gfk_autotune");
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "gfk_autotune");
    ctx->threads = bt;
    ctx->wpt = bw;
    if (best_threads) *best_threads = bt;
    if (best_wpt) *best_wpt = bw;
    if (best_rate) *best_rate = best;
    return GFK_OK;
}

gfk_status gfk_steps(gfk_ctx* ctx, int64_t* n_steps) {
    if (!ctx || !n_steps) return GFK_EINVAL;
    *n_steps = ctx->steps;
    return GFK_OK;
}

gfk_status gfk_sums(gfk_ctx* ctx, int32_t inst, double* host_rows, int64_t cap) {
    gfk_status st = check_inst(ctx, inst);
    if (st != GFK_OK) return st;
    if (!host_rows) return GFK_EINVAL;
    if (!ctx->initialized) return GFK_ESTATE;
    const int64_t n = ctx->steps + 1;
    if (cap < n) return GFK_EOVERFLOW;
    DeviceGuard g(ctx->device);
    GFK_CK(ctx, cudaMemcpyAsync(host_rows, ctx->series + (int64_t)inst * ctx->series_cap,
                                sizeof(SeriesRow) * n, cudaMemcpyDeviceToHost, ctx->stream));
    GFK_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return GFK_OK;
}

gfk_status gfk_energy(gfk_ctx* ctx, int32_t inst, double* e_mixed, double* ln_z, double* ess,
                      int64_t cap, double* e_final) {
    NvtxRange nvtx_("gfk_energy");
    gfk_status st = check_inst(ctx, inst);
    if (st != GFK_OK) return st;
    if (!ctx->initialized) return GFK_ESTATE;
    const int64_t n = ctx->steps + 1;
    if ((e_mixed || ln_z || ess) && cap < n) return GFK_EOVERFLOW;
    DeviceGuard g(ctx->device);
    st = ensure_scratch(ctx, sizeof(double) * 3 * n);
    if (st != GFK_OK) return st;
    double* d = (double*)ctx->scratch;
    cudaError_t e = launch_finalize(ctx->series + (int64_t)inst * ctx->series_cap, n,
                                    (double)ctx->desc[inst].n_walkers, d, d + n, d + 2 * n,
                                    ctx->stream);
    std::vector<double> h(3 * n);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, ctx->stream);
    unsigned long long cnt[kNumCounters] = {0, 0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cnt, ctx->counters + (int64_t)inst * kNumCounters, sizeof(cnt),
                            cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gfk_energy");
    if (e_mixed) std::memcpy(e_mixed, h.data(), sizeof(double) * n);
    if (ln_z) std::memcpy(ln_z, h.data() + n, sizeof(double) * n);
    if (ess) std::memcpy(ess, h.data() + 2 * n, sizeof(double) * n);
    if (e_final) *e_final = h[n - 1];
    return cnt[0] > 0 ? GFK_ENONFINITE : GFK_OK;
}

gfk_status gfk_get_walkers(gfk_ctx* ctx, int32_t inst, double* x6, double* logw, uint8_t* alive) {
    NvtxRange nvtx_("gfk_get_walkers");
    gfk_status st = check_inst(ctx, inst);
    if (st != GFK_OK) return st;
    if (!ctx->initialized) return GFK_ESTATE;
    DeviceGuard g(ctx->device);
    const int64_t n = ctx->desc[inst].n_walkers;
    st = ensure_scratch(ctx, (size_t)n * (7 * sizeof(double) + 1));
    if (st != GFK_OK) return st;
    double* dx = (double*)ctx->scratch;
    double* dl = dx + 6 * n;
    uint8_t* da = (uint8_t*)(dl + n);
    cudaError_t e = launch_export(ctx->prec == GFK_PREC_MIXED, ctx->s64, ctx->smx, ctx->off[inst], n,
                                  dx, dl, da, ctx->stream);
    if (e == cudaSuccess && x6)
        e = cudaMemcpyAsync(x6, dx, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && logw)
        e = cudaMemcpyAsync(logw, dl, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && alive)
        e = cudaMemcpyAsync(alive, da, (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gfk_get_walkers");
    return GFK_OK;
}

gfk_status gfk_counters(gfk_ctx* ctx, int32_t inst, int64_t* host_counts3) {
    gfk_status st = check_inst(ctx, inst);
    if (st != GFK_OK) return st;
    if (!host_counts3) return GFK_EINVAL;
    DeviceGuard g(ctx->device);
    unsigned long long cnt[kNumCounters];
    GFK_CK(ctx, cudaMemcpyAsync(cnt, ctx->counters + (int64_t)inst * kNumCounters, sizeof(cnt),
                                cudaMemcpyDeviceToHost, ctx->stream));
    GFK_CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int j = 0; j < kNumCounters; ++j) host_counts3[j] = (int64_t)cnt[j];
    return GFK_OK;
}

gfk_status gfk_checkpoint_size(gfk_ctx* ctx, int64_t* bytes) {
    if (!ctx || !bytes) return GFK_EINVAL;
    const int64_t rows = ctx->initialized ? ctx->steps + 1 : 0;
    *bytes = (int64_t)(sizeof(BlobHeader) + state_bytes(ctx) +
                       sizeof(SeriesRow) * rows * ctx->n_inst +
                       sizeof(unsigned long long) * kNumCounters * ctx->n_inst);
    return GFK_OK;
}

gfk_status gfk_checkpoint(gfk_ctx* ctx, void* host_blob, int64_t bytes) {
    if (!ctx || !host_blob) return GFK_EINVAL;
    int64_t need = 0;
    gfk_checkpoint_size(ctx, &need);
    if (bytes < need) return GFK_EOVERFLOW;
    DeviceGuard g(ctx->device);
    BlobHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "GFKCKPT1", 8);
    h.version = 1;
    h.n_inst = ctx->n_inst;
    h.prec = ctx->prec;
    h.initialized = ctx->initialized ? 1 : 0;
    h.n_slots = ctx->n_slots;
    h.steps = ctx->steps;
    h.series_rows = ctx->initialized ? ctx->steps + 1 : 0;
    h.desc_hash = desc_hash(ctx);
    char* o = (char*)host_blob;
    std::memcpy(o, &h, sizeof(h));
    o += sizeof(h);
    const int64_t ns = ctx->n_slots;
    if (ctx->prec == GFK_PREC_FP64) {
        GFK_CK(ctx, cudaMemcpyAsync(o, ctx->s64.x, sizeof(double) * 6 * ns, cudaMemcpyDeviceToHost, ctx->stream));
        o += sizeof(double) * 6 * ns;
        GFK_CK(ctx, cudaMemcpyAsync(o, ctx->s64.logw, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->stream));
        o += sizeof(double) * ns;
        GFK_CK(ctx, cudaMemcpyAsync(o, ctx->s64.sgn, (size_t)ns, cudaMemcpyDeviceToHost, ctx->stream));
        o += ns;
    } else {
        GFK_CK(ctx, cudaMemcpyAsync(o, ctx->smx.p0, sizeof(float4) * ns, cudaMemcpyDeviceToHost, ctx->stream));
        o += sizeof(float4) * ns;
        GFK_CK(ctx, cudaMemcpyAsync(o, ctx->smx.p1, sizeof(float4) * ns, cudaMemcpyDeviceToHost, ctx->stream));
        o += sizeof(float4) * ns;
        GFK_CK(ctx, cudaMemcpyAsync(o, ctx->smx.sgn, (size_t)ns, cudaMemcpyDeviceToHost, ctx->stream));
        o += ns;
    }
    for (int i = 0; i < ctx->n_inst && h.series_rows > 0; ++i) {
        GFK_CK(ctx, cudaMemcpyAsync(o, ctx->series + (int64_t)i * ctx->series_cap,
                                    sizeof(SeriesRow) * h.series_rows, cudaMemcpyDeviceToHost, ctx->stream));
        o += sizeof(SeriesRow) * h.series_rows;
    }
    GFK_CK(ctx, cudaMemcpyAsync(o, ctx->counters, sizeof(unsigned long long) * kNumCounters * ctx->n_inst,
                                cudaMemcpyDeviceToHost, ctx->stream));
    GFK_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return GFK_OK;
}

gfk_status gfk_restore(gfk_ctx* ctx, const void* host_blob, int64_t bytes) {
    if (!ctx || !host_blob || bytes < (int64_t)sizeof(BlobHeader)) return GFK_EINVAL;
    BlobHeader h;
    std::memcpy(&h, host_blob, sizeof(h));
    if (std::memcmp(h.magic, "GFKCKPT1", 8) != 0 || h.version != 1 || h.n_inst != ctx->n_inst ||
        h.prec != ctx->prec || h.n_slots != ctx->n_slots || h.desc_hash != desc_hash(ctx))
        return GFK_EINVAL;
    for (int i = 0; i < ctx->n_inst; ++i)
        if (!ctx->has_trial[i]) return GFK_ESTATE;
    const int64_t need = (int64_t)(sizeof(BlobHeader) + state_bytes(ctx) +
                                   sizeof(SeriesRow) * h.series_rows * ctx->n_inst +
                                   sizeof(unsigned long long) * kNumCounters * ctx->n_inst);
    if (bytes < need || (h.initialized && h.series_rows != h.steps + 1)) return GFK_EINVAL;
    DeviceGuard g(ctx->device);
    if (ctx->params_dirty) {
        gfk_status st = upload_instances(ctx);
        if (st != GFK_OK) return st;
    }
    if (h.initialized) {
        gfk_status st = ensure_series(ctx, h.series_rows);
        if (st != GFK_OK) return st;
    }
    const char* o = (const char*)host_blob + sizeof(h);
    const int64_t ns = ctx->n_slots;
    if (ctx->prec == GFK_PREC_FP64) {
        GFK_CK(ctx, cudaMemcpyAsync(ctx->s64.x, o, sizeof(double) * 6 * ns, cudaMemcpyHostToDevice, ctx->stream));
        o += sizeof(double) * 6 * ns;
        GFK_CK(ctx, cudaMemcpyAsync(ctx->s64.logw, o, sizeof(double) * ns, cudaMemcpyHostToDevice, ctx->stream));
        o += sizeof(double) * ns;
        GFK_CK(ctx, cudaMemcpyAsync(ctx->s64.sgn, o, (size_t)ns, cudaMemcpyHostToDevice, ctx->stream));
        o += ns;
    } else {
        GFK_CK(ctx, cudaMemcpyAsync(ctx->smx.p0, o, sizeof(float4) * ns, cudaMemcpyHostToDevice, ctx->stream));
        o += sizeof(float4) * ns;
        GFK_CK(ctx, cudaMemcpyAsync(ctx->smx.p1, o, sizeof(float4) * ns, cudaMemcpyHostToDevice, ctx->stream));
        o += sizeof(float4) * ns;
        GFK_CK(ctx, cudaMemcpyAsync(ctx->smx.sgn, o, (size_t)ns, cudaMemcpyHostToDevice, ctx->stream));
        o += ns;
    }
    for (int i = 0; i < ctx->n_inst && h.series_rows > 0; ++i) {
        GFK_CK(ctx, cudaMemcpyAsync(ctx->series + (int64_t)i * ctx->series_cap, o,
                                    sizeof(SeriesRow) * h.series_rows, cudaMemcpyHostToDevice, ctx->stream));
        o += sizeof(SeriesRow) * h.series_rows;
    }
    GFK_CK(ctx, cudaMemcpyAsync(ctx->counters, o, sizeof(unsigned long long) * kNumCounters * ctx->n_inst,
                                cudaMemcpyHostToDevice, ctx->stream));
    GFK_CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->initialized = h.initialized != 0;
    ctx->steps = h.steps;
    return GFK_OK;
}

gfk_status gfk_grad(gfk_ctx* ctx, int32_t inst, int32_t loss_kind, int64_t n_steps,
                    int32_t ckpt_every, double* grad, int32_t n_params, double* loss) {
    NvtxRange nvtx_("gfk_grad");
    gfk_status st = check_inst(ctx, inst);
    if (st != GFK_OK) return st;
    if (loss_kind != 0 && loss_kind != 1) return GFK_EINVAL;
    if (n_steps < 1 || n_steps > 0x7fffffffll || ckpt_every < 0 || ckpt_every > 1024)
        return GFK_EINVAL;
    if (!grad || n_params != 7) return GFK_EINVAL;
    if (!ctx->has_trial[inst]) return GFK_ESTATE;
    if (ctx->trial[inst].kind != GFK_TRIAL_JASTROW_PRODUCT) return GFK_EINVAL;
    DeviceGuard g(ctx->device);
    if (ctx->params_dirty) {
        st = upload_instances(ctx);
        if (st != GFK_OK) return st;
    }
    const bool f64 = ctx->prec == GFK_PREC_FP64;
    const int64_t n = ctx->desc[inst].n_walkers;
    // ckpt_every 0: the mixed forward keeps the whole trajectory and the sweep
    // reads it in 64-move segments; the FP64 path checkpoints every 64 moves
    const bool keep_all = ckpt_every == 0 && !f64;
    const int S = (int)n_steps, K = ckpt_every == 0 ? kRing : ckpt_every;
    const int J = (S + K - 1) / K;
    const size_t tsz = f64 ? sizeof(double) : sizeof(float);
    const int words = f64 ? 6 : 8;                       // position words per walker
    // launch shape of the forward (one instance, slots from 0)
    gfk_ctx shape;
    shape.n_inst = 1;
    shape.threads = ctx->threads;
    shape.wpt = f64 ? 1 : ctx->wpt;
    shape.desc.push_back(ctx->desc[inst]);
    int64_t nblk = 0;
    BlockMap bm = make_block_map(&shape, &nblk);
    const int nblk_adj = (int)((n + 127) / 128);

    // one allocation, carved into the pieces below
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
    const size_t o_inst = take(sizeof(InstDev));
    const size_t o_state = take(f64 ? n * (7 * sizeof(double)) : n * 2 * sizeof(float4));
    const size_t o_sgn = take((size_t)n);
    // the mixed walk writes the checkpoints itself when they fall on its 64-move
    // folds, and then runs in launches of up to kGradChunk moves
    constexpr int kGradChunk = 1024;
    const bool ckpt_in_kernel = !f64 && K % kRing == 0;
    const int part_rows = ckpt_in_kernel ? std::min(S, kGradChunk) : K;
    const size_t o_part = take(sizeof(PartialRec) * (size_t)part_rows * nblk);
    const size_t o_cnt = take(sizeof(unsigned long long) * kNumCounters);
    const size_t o_ckpt = take(keep_all ? 0 : tsz * words * (size_t)n * J);
    // the reverse sweep's segment planes use an even walker stride (SegIO)
    const size_t n_even = (size_t)((n + 1) & ~(int64_t)1);
    const size_t o_seg = take(std::max(keep_all ? 0 : tsz * words * n_even * (K + 1),
                                       sizeof(double) * 7 * (size_t)n));
    // the whole trajectory: S + 1 planes of 6 floats per walker (SegIO layout)
    const size_t o_traj = take(keep_all ? sizeof(float) * 6 * n_even * ((size_t)S + 1) : 0);
    const size_t o_logw = take(sizeof(double) * (size_t)n);
    const size_t o_ew = take(sizeof(double) * 2 * (size_t)n);
    const size_t o_pmax = take(sizeof(double) * nblk_adj);
    const size_t o_psum = take(sizeof(double) * 3 * nblk_adj);
    const size_t o_pth = take(sizeof(double) * 7 * nblk_adj);
    const size_t o_term = take(64);
    const size_t o_grad = take(sizeof(double) * 8);
    st = ensure_buffer(ctx, &ctx->grad_ws, &ctx->grad_ws_bytes, off);
    if (st != GFK_OK) return st;
    char* base = (char*)ctx->grad_ws;
    InstDev* d_inst = (InstDev*)(base + o_inst);
    cudaError_t e = cudaMemcpyAsync(d_inst, ctx->d_inst + inst, sizeof(InstDev),
                                    cudaMemcpyDeviceToDevice, ctx->stream);
    // the copy's walkers start at slot 0
    const int64_t zero = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((char*)d_inst + offsetof(InstDev, off), &zero, sizeof(zero),
                            cudaMemcpyHostToDevice, ctx->stream);
    StateF64 s64{};
    StateMixed smx{};
    if (f64) {
        s64.x = (double*)(base + o_state);
        s64.logw = s64.x + 6 * n;
        s64.sgn = (int8_t*)(base + o_sgn);
        s64.stride = n;
    } else {
        smx.p0 = (float4*)(base + o_state);
        smx.p1 = smx.p0 + n;
        smx.sgn = (int8_t*)(base + o_sgn);
    }
    PartialRec* part = (PartialRec*)(base + o_part);
    unsigned long long* cnt = (unsigned long long*)(base + o_cnt);
    char* ckpt = base + o_ckpt;
    const int kind = GFK_TRIAL_JASTROW_PRODUCT;
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * kNumCounters, ctx->stream);
    // forward: the same init and walk kernels as gfk_propagate, checkpointing
    // the positions every K moves
    if (e == cudaSuccess)
        e = f64 ? launch_init_fp64(kind, shape.threads, (int)nblk, d_inst, bm, s64, part, cnt, ctx->stream)
                : launch_init_mixed(kind, shape.threads, (int)nblk, d_inst, bm, smx, part, cnt, ctx->stream);
    if (ckpt_in_kernel) {
        if (keep_all) {
            // every position, the initial ones included, from the walk kernel
            smx.traj = (float*)(base + o_traj);
            smx.traj_stride = (int64_t)n_even;
        } else {
            // checkpoint 0 is the initial state; the walk kernel writes 1 .. J - 1
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(ckpt, base + o_state, tsz * words * (size_t)n,
                                    cudaMemcpyDeviceToDevice, ctx->stream);
            smx.ckpt = (float4*)ckpt;
            smx.ckpt_slots = n;
            smx.ckpt_every = K;
            smx.ckpt_count = J;
        }
        for (int done = 0; done < S && e == cudaSuccess; done += kGradChunk) {
            const int steps = std::min(kGradChunk, S - done);
            e = launch_walk_mixed(mixed_walk_kind(kind, &ctx->trial[inst], 1), ctx->noise,
                                  shape.wpt, shape.threads, (int)nblk, 0, (int)nblk, d_inst, bm,
                                  smx, (uint32_t)done, steps, part, cnt, &ctx->trial[inst],
                                  ctx->desc[inst].ee_on, ctx->stream);
        }
        smx.ckpt = nullptr;
        smx.traj = nullptr;
    }
    for (int j = 0; j < J && !ckpt_in_kernel && e == cudaSuccess; ++j) {
        const size_t plane_bytes = tsz * words * (size_t)n;
        e = cudaMemcpyAsync(ckpt + plane_bytes * j, base + o_state, plane_bytes,
                            cudaMemcpyDeviceToDevice, ctx->stream);
        const int steps = std::min(K, S - j * K);
        if (e == cudaSuccess)
            e = f64 ? launch_walk_fp64(kind, ctx->noise, shape.threads, (int)nblk, d_inst, bm, s64,
                                       (uint32_t)(j * K), steps, part, cnt, ctx->stream)
                    : launch_walk_mixed(mixed_walk_kind(kind, &ctx->trial[inst], 1), ctx->noise,
                                        shape.wpt, shape.threads, (int)nblk, 0,
                                        (int)nblk,
                                        d_inst, bm, smx, (uint32_t)(j * K), steps, part, cnt,
                                        &ctx->trial[inst], ctx->desc[inst].ee_on, ctx->stream);
    }
    double* logw_final = (double*)(base + o_logw);
    if (e == cudaSuccess) {
        // final log-weights (-inf for dead walkers) through the export kernel
        double* x6 = (double*)(base + o_seg);
        uint8_t* alive = (uint8_t*)(base + o_ew);
        e = launch_export(!f64, s64, smx, 0, n, x6, logw_final, alive, ctx->stream);
    }
    double* grad_d = (double*)(base + o_grad);
    void* term = base + o_term;
    if (e == cudaSuccess) {
        if (f64)
            e = launch_adjoint_f64(d_inst, n, S, K, loss_kind, (const double*)ckpt,
                                   (double*)(base + o_seg), (const double*)(base + o_state),
                                   logw_final, (double*)(base + o_ew), (double*)(base + o_pmax),
                                   (double*)(base + o_psum), (double*)(base + o_pth), term, grad_d,
                                   ctx->stream);
        else
            e = launch_adjoint_f32(d_inst, n, S, K, loss_kind, (const float*)ckpt,
                                   (float*)(base + o_seg),
                                   keep_all ? (const float*)(base + o_traj) : nullptr,
                                   (const float*)(base + o_state),
                                   logw_final, (double*)(base + o_ew), (double*)(base + o_pmax),
                                   (double*)(base + o_psum), (double*)(base + o_pth), term, grad_d,
                                   ctx->stream);
    }
    double hg[7];
    double hterm[5];
    if (e == cudaSuccess) e = cudaMemcpyAsync(hg, grad_d, sizeof(hg), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hterm, term, sizeof(hterm), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gfk_grad");
    for (int k = 0; k < 7; ++k) grad[k] = hg[k];
    if (loss) *loss = hterm[4];
    return GFK_OK;
}

gfk_status gfk_profile(gfk_ctx* ctx, int32_t enable) {
    if (!ctx) return GFK_EINVAL;
    ctx->profiling = enable != 0;
    return GFK_OK;
}

gfk_status gfk_profile_read(gfk_ctx* ctx, double* walk_ms, int64_t* launches,
                            double* walker_steps, int32_t reset) {
    if (!ctx) return GFK_EINVAL;
    DeviceGuard g(ctx->device);
    gfk_status st = profile_harvest(ctx);
    if (st != GFK_OK) return st;
    if (walk_ms) *walk_ms = ctx->prof_ms;
    if (launches) *launches = ctx->prof_launches;
    if (walker_steps) *walker_steps = ctx->prof_walker_steps;
    if (reset) {
        ctx->prof_ms = 0.0;
        ctx->prof_launches = 0;
        ctx->prof_walker_steps = 0.0;
    }
    return GFK_OK;
}

gfk_status gfk_kernel_count(gfk_ctx* ctx, int64_t* count, int32_t reset) {
    if (!ctx || !count) return GFK_EINVAL;
    *count = ctx->kernels;
    if (reset) ctx->kernels = 0;
    return GFK_OK;
}

gfk_status gfk_reset(gfk_ctx* ctx) {
    if (!ctx) return GFK_EINVAL;
    ctx->initialized = false;
    ctx->steps = 0;
    return GFK_OK;
}

void gfk_destroy(gfk_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    delete ctx;
}

}  // extern "C"
