/*
 * gfk.h -- C ABI of the GB300 generalized Feynman-Kac (GFK) walker library.
 *
 * The library advances large populations of independent 6-D two-electron
 * walkers for helium by the importance-sampled diffusion of the GFK method
 * (Datta, Rejcek, Fry, "The He atom revisited", arXiv:1703.08977) and forms
 * the space-averaged energy after every step.  All arithmetic runs in CUDA
 * kernels for sm_103a; the calls below only validate, allocate and launch.
 *
 * Conventions shared by every call:
 *   - A walker's position is X = (x1, y1, z1, x2, y2, z2) in bohr.
 *   - Pointers named host_* or documented "host" are ordinary CPU memory; no
 *     call takes a device pointer unless it says so.
 *   - Every call returns a gfk_status; none aborts, traps or exits.  A CUDA
 *     failure returns GFK_ECUDA and gfk_last_error() gives CUDA's message.
 *   - A context is used from one host thread at a time.
 *   - Work is queued on the CUDA stream given to gfk_create (NULL = the
 *     legacy default stream).  Calls that return data to the host synchronise
 *     that stream; gfk_propagate does not.
 */
#ifndef GFK_H
#define GFK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gfk_ctx gfk_ctx;   /* opaque; owned by the library */

typedef enum {
    GFK_OK = 0,
    GFK_EINVAL = 1,       /* an argument is out of range or malformed            */
    GFK_ENOMEM = 2,       /* a device or host allocation failed                  */
    GFK_ECUDA = 3,        /* a CUDA call failed; see gfk_last_error()            */
    GFK_ESTATE = 4,       /* the call is not valid in the context's state        */
    GFK_ENONFINITE = 5,   /* outputs were written, but some walkers were killed
                             because their drift or local energy was not finite */
    GFK_EOVERFLOW = 6,    /* a caller buffer is too small                        */
    GFK_ETIMEOUT = 7      /* reserved: no call waits on a device-side flag       */
} gfk_status;

/* Symmetry of the state sought (the paper's three cases: the nodeless ground
 * state, the 2^3S state whose node r1 = r2 is exact, and a P_z state handled
 * by its necessary nodal condition).  Every state uses the same fixed-node
 * rule: a walker whose trial function changes sign, or becomes exactly zero,
 * is killed (its weight is zero from then on). */
typedef enum { GFK_1S = 0, GFK_2S3 = 1, GFK_PZ = 2 } gfk_state;

/* Arithmetic of the walk.
 * GFK_PREC_FP64:  every operation in FP64.
 * GFK_PREC_MIXED: positions, drift, local energy and random normals in FP32;
 *                 each walker's log-weight is an FP64 base plus an FP32
 *                 Kahan-compensated sum of increments folded into the base
 *                 every 64 steps; population sums go FP32 within a warp,
 *                 FP64 above it; across blocks the sums of weights W and of
 *                 weighted local energies P are double-doubles (Neumaier
 *                 sums per thread, TwoSum between threads), as on the FP64
 *                 path. */
typedef enum { GFK_PREC_FP64 = 0, GFK_PREC_MIXED = 1 } gfk_prec;

/* Increments of the walk, X <- X + b dt + sqrt(dt) xi.
 * GFK_NOISE_GAUSSIAN:  xi = six N(0,1) normals (the Brownian increment of the
 *   drifted diffusion written under Eq. 4) from Philox4x32-10 words by Box-Muller.
 * GFK_NOISE_BERNOULLI: xi = six signs +-1, the paper's own random walk (the
 *   construction of W(l) before the invariance principle: each coordinate moves
 *   by eps/sqrt(n) per time step 1/n, so dt = 1/n and the paper's step length
 *   1/scale is sqrt(dt)).  eps comes from the "Superduper" congruential generator
 *   S_i = (69069 S_{i-1} + 1) mod 2^32, eps_i = +1 if S_i > 2^31, else -1.  Each
 *   walker runs its own generator, seeded with word 0 of the Philox block
 *   (walker id, 0, rng_stream, 5); move `step` uses outputs 6 step + 1 ..
 *   6 step + 6 for x1, y1, z1, x2, y2, z2.  The initial positions are Gaussian
 *   in both modes.  The generator's period is 2^32 outputs. */
typedef enum { GFK_NOISE_GAUSSIAN = 0, GFK_NOISE_BERNOULLI = 1 } gfk_noise;

/* Trial-function families, psi = Phi(r1_vec, r2_vec) * exp(u(r12)) with the
 * Jastrow factor u(r) = a rho + sum_{k=1..4} c_k rho^(k+1), rho = r/(1+beta r).
 *
 * GFK_TRIAL_JASTROW_PRODUCT: Phi = exp(-Z r1 - Z r2).
 *   params = [Z, a, beta, c1, c2, c3, c4]   (3 to 7 values; missing c_k = 0)
 *   The benchmark ground-state function exp(-2 r1 - 2 r2) exp(r12/(2(1+0.5 r12)))
 *   is [2, 0.5, 0.5].
 * GFK_TRIAL_ORBITAL_PAIRS: Phi = sum_t s_t f_{A,t}(r1_vec) f_{B,t}(r2_vec) with
 *   orbitals f(r_vec) = (c0 + c1 r + cz z) exp(-alpha r).
 *   params = [a, beta, c1, c2, c3, c4, nterms,
 *             then for each term: s, alphaA, c0A, c1A, czA, alphaB, c0B, c1B, czB]
 *   (7 + 9 nterms values, 1 <= nterms <= GFK_MAX_TERMS).  This covers the
 *   paper's trial functions 3, 4, 5 ((r0 - r) e^{-alpha r} orbitals,
 *   antisymmetrised) and 7 ((z1 + z2) times a symmetric pair), and the
 *   triplet and P_z functions of the benchmark workloads. */
typedef enum { GFK_TRIAL_JASTROW_PRODUCT = 0, GFK_TRIAL_ORBITAL_PAIRS = 1 } gfk_trial_kind;

#define GFK_MAX_TERMS 4
#define GFK_MAX_PARAMS (7 + 9 * GFK_MAX_TERMS)
#define GFK_MAX_INSTANCES 64

/* One independent walk (an "instance"): the paper's statement of the problem
 * -- a symmetry, the trial energy E_T (the paper's lambda_0 of the trial
 * function), the time step dt, the number of replications N_rep and a seed.
 * Random numbers are Philox4x32-10 with counter (walker id, n, rng_stream,
 * tag) and key (seed low, seed high): move n takes the block with tag 0 (its
 * words 0-2 the Box-Muller radii, its word 3 three 10-bit angle indices on a
 * 1024-point grid), the initial position the block of n = 0 with tag 1
 * (Gaussian noise; see gfk_noise for the Bernoulli mode); the walker id is
 * walker_id0 + the walker's index.  The same (seed, rng_stream, walker id)
 * gives the same trajectory in any context and any launch configuration. */
typedef struct {
    int32_t  state;          /* gfk_state                                         */
    int32_t  prec;           /* gfk_prec; all instances of a context share it     */
    int64_t  n_walkers;      /* N_rep, 1 .. 2^31 - 1                              */
    double   dt;             /* time step (hartree^-1), > 0                       */
    double   e_trial;        /* E_T, hartree                                      */
    uint64_t seed;           /* Philox key                                        */
    uint32_t rng_stream;     /* third Philox counter word                         */
    int32_t  ee_on;          /* 1: V includes 1/r12; 0: drops it (test hook)      */
    double   init_sigma;     /* initial positions: each coordinate ~ N(0, sigma^2) */
    uint32_t walker_id0;     /* Philox id of walker 0 (walker k uses id0 + k): shards
                                of one population on several GPUs take disjoint
                                id ranges and together reproduce it exactly;
                                id0 + n_walkers must not exceed 2^32             */
    int32_t  noise;          /* gfk_noise; all instances of a context share it    */
} gfk_instance_desc;

/* Create a context holding n_inst instances (1 .. GFK_MAX_INSTANCES).
 * cuda_stream: a cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream)
 * or NULL.  The context allocates and owns all device memory it uses.
 * The current CUDA device at this call is the context's device.
 * Returns GFK_EINVAL for a bad descriptor, GFK_ENOMEM / GFK_ECUDA on failure;
 * *out is NULL unless GFK_OK. */
gfk_status gfk_create(const gfk_instance_desc* inst, int32_t n_inst, void* cuda_stream,
                      gfk_ctx** out);

/* Set instance inst's trial function (host params, copied): the importance
 * function phi_0 of the GFK split H = H0 + V_P ("Path Integral Theory"
 * section, before Eq. 4), whose drift grad(phi)/phi steers the walk and whose
 * local energy gives the weight of Eq. 4; the paper's trial-function list
 * (functions 3 to 7) and its variational tuning remark (parameters chosen to
 * minimise the variance of the local energy) are what the parameter vectors
 * of gfk_trial_kind cover.  Allowed before the first gfk_propagate, or after
 * gfk_reset.  GFK_ESTATE otherwise; GFK_EINVAL for a malformed parameter
 * vector. */
gfk_status gfk_set_trial(gfk_ctx* ctx, int32_t inst, int32_t trial_kind,
                         const double* params, int32_t n_params);

/* Choose the launch shape of the walk kernels: threads per block
 * (64, 128, 256 or 512) and walkers per thread (1, 2 or 4; 4 only with at
 * most 128 threads per block, GFK_EINVAL otherwise).  Results per
 * walker do not depend on it; population sums differ only by rounding order
 * (FP64 path) or by the FP32 rounding of the block shift (mixed path).
 * Allowed at any time between calls. */
gfk_status gfk_set_launch(gfk_ctx* ctx, int32_t threads_per_block, int32_t walkers_per_thread);

/* Replay gfk_propagate as a CUDA graph.  When enabled (and gfk_profile is
 * off), each gfk_propagate captures its launch sequence -- the initial
 * population if due, then the walk and merge kernels of every chunk -- into a
 * CUDA graph, keyed by start step, length and launch shape, and launches the
 * graph; a later call with the same key (for example after gfk_reset) replays
 * it without re-issuing the launches.  Up to 8 graphs are kept per context.
 * Results are identical to the non-graph path.  The walk over all instances
 * of a context is one launch per chunk: a batch of instances (several
 * states, time steps and walker counts) runs as one launch sequence. */
gfk_status gfk_set_graph(gfk_ctx* ctx, int32_t enable);

/* Choose the launch shape by measurement: for every threads-per-block in
 * {64, 128, 256, 512} and walkers-per-thread in {1, 2, 4} (FP64: 1; 4 with
 * at most 128 threads), time the
 * walk kernel and the merge of its block records on probe_steps moves
 * (1..4096) of this context's own population,
 * restoring the population and counters after each candidate, then keep the
 * fastest shape (as gfk_set_launch would).  Outputs may be NULL.  Initialises
 * the population first if needed.  Synchronises the stream; allocates a
 * temporary copy of the population. */
gfk_status gfk_autotune(gfk_ctx* ctx, int64_t probe_steps, int32_t* best_threads,
                        int32_t* best_walkers_per_thread, double* best_walker_steps_per_s);

/* Advance every instance by n_steps moves (asynchronous on the context's
 * stream: part of the work runs on the context's own internal streams -- the
 * merges of the block sums, concurrent launches of several instance groups,
 * CUDA-graph replays -- ordered after the work already queued on the
 * context's stream, which in turn waits for all of it before any later work
 * queued there).  The first call after gfk_create / gfk_reset initialises the
 * population (X0 = init_sigma * xi from the Philox blocks (id, 0, stream, 3/4),
 * log-weight 0) and records the step-0 population sums.  Each move is
 *   X <- X + b(X) dt + sqrt(dt) xi,   b = grad ln|psi|       (the SDE under Eq. 4)
 *   logw <- logw - (E_L(X) - E_T) dt, E_L = -Delta(psi)/(2 psi) + V
 * (the right-point Riemann sum of the Feynman-Kac exponent, Eq. 4), then the
 * fixed-node test, then the population sums of that step.
 * GFK_ESTATE if an instance has no trial function.  Step counts are
 * cumulative; a run interrupted and resumed at a multiple of 64 steps is
 * bitwise identical to an uninterrupted one. */
gfk_status gfk_propagate(gfk_ctx* ctx, int64_t n_steps);

/* Number of moves made so far (all instances move together). */
gfk_status gfk_steps(gfk_ctx* ctx, int64_t* n_steps);

/* Space-averaged estimators of instance inst for steps 0..S (S = gfk_steps),
 * written to host arrays of cap >= S + 1 doubles (any of them may be NULL):
 *   e_mixed[k] = sum_i w_i E_L(X_i) / sum_i w_i     after k moves
 *   ln_z[k]    = ln( sum_i w_i / N_rep )            (Eq. 4: lambda ~ E_T - ln z / t)
 *   ess[k]     = (sum_i w_i)^2 / sum_i w_i^2        (effective sample size)
 * and *e_final = e_mixed[S] (may be NULL).  Dead walkers have w = 0.
 * Synchronises the stream.  GFK_EOVERFLOW if cap < S + 1 (nothing written);
 * GFK_ENONFINITE (outputs written) if any walker was killed for a non-finite
 * drift or local energy. */
gfk_status gfk_energy(gfk_ctx* ctx, int32_t inst, double* e_mixed, double* ln_z,
                      double* ess, int64_t cap, double* e_final);

/* Raw population sums of instance inst, 6 doubles per step for steps 0..S:
 * { c, W, P, Q, R, n_alive } with W = sum e^{logw - c}, P = sum w E_L,
 * Q = sum w^2, R = sum w E_L^2 (w = e^{logw - c}).  host_rows holds cap rows.
 * Synchronises the stream.  GFK_EOVERFLOW if cap < S + 1. */
gfk_status gfk_sums(gfk_ctx* ctx, int32_t inst, double* host_rows, int64_t cap);

/* Copy instance inst's walkers to host memory: the N_rep independent
 * replications of the space average (the paths Y_m of the discretisation
 * section whose weights are averaged after the invariance principle), each
 * with its position and its Feynman-Kac log-weight -int (E_L - E_T) dt of
 * Eq. 4 (any pointer may be NULL):
 * x6 (n_walkers * 6 doubles, walker-major), logw (n_walkers doubles, -inf for
 * dead walkers), alive (n_walkers bytes).  Mixed-precision positions are
 * widened exactly from FP32.  Synchronises the stream.  GFK_ESTATE before the
 * population exists. */
gfk_status gfk_get_walkers(gfk_ctx* ctx, int32_t inst, double* x6, double* logw,
                           uint8_t* alive);

/* Per-instance event counters (host int64[3]): walkers killed for a non-finite
 * drift or local energy, walkers killed at the node, and moves that landed an
 * electron within 1e-10 (FP64) or 1e-5 (mixed) bohr of the nucleus or of the
 * other electron (a diagnostic only: nothing is changed). */
gfk_status gfk_counters(gfk_ctx* ctx, int32_t inst, int64_t* host_counts3);

/* Checkpoint: the whole walk state (population planes, step counter, per-step
 * sums, counters) as an opaque host blob of gfk_checkpoint_size bytes.
 * gfk_restore loads a blob written by a context created with the same
 * descriptors and trial functions; resuming from it is bitwise identical to
 * never having stopped (when the step count is a multiple of 64).
 * GFK_EINVAL if the blob does not match the context. */
gfk_status gfk_checkpoint_size(gfk_ctx* ctx, int64_t* bytes);
gfk_status gfk_checkpoint(gfk_ctx* ctx, void* host_blob, int64_t bytes);
gfk_status gfk_restore(gfk_ctx* ctx, const void* host_blob, int64_t bytes);

/* Gradient of a space-averaged loss with respect to the trial parameters,
 * through the walk (the pathwise derivative with the Philox noise held fixed).
 * Runs instance inst from a fresh population for n_steps moves (>= 1) in the
 * context's precision -- the same trajectories gfk_propagate produces --
 * keeping the positions every ckpt_every moves (1..1024), then sweeps the
 * adjoint of the Euler-Maruyama recursion backwards, recomputing each segment
 * from its checkpoint.  ckpt_every = 0 trades memory for that recompute: the
 * mixed path's forward keeps every position (the whole trajectory) and the
 * sweep reads it in 64-move segments, with nothing recomputed; the gradient is
 * bitwise the one of ckpt_every = 64 (the FP64 path runs ckpt_every = 64).
 * Loss 0: E = sum_i w_i E_L(X_i) / sum_i w_i at the last
 * move (the quantity of Eq. 4's space average); loss 1: the weighted variance
 * of E_L at the last move.  Only the Jastrow-product family is supported
 * (GFK_EINVAL otherwise); grad receives the derivatives with respect to all
 * seven parameters [Z, a, beta, c1, c2, c3, c4] (n_params must be 7), *loss
 * the loss (may be NULL).  Does not touch the context's population.
 * Synchronises the stream.  Needs working memory of about
 * n_walkers x (n_steps / ckpt_every + ckpt_every) x 48 bytes (FP64; 32 bytes
 * mixed), or n_walkers x (n_steps + 1) x 24 bytes for ckpt_every = 0 on the
 * mixed path (12.6 GB for 2^18 walkers and 2000 moves), which the context
 * allocates on the first call, keeps for later calls (growing it when one
 * needs more) and frees in gfk_destroy; GFK_ENOMEM when it cannot. */
gfk_status gfk_grad(gfk_ctx* ctx, int32_t inst, int32_t loss_kind, int64_t n_steps,
                    int32_t ckpt_every, double* grad, int32_t n_params, double* loss);

/* Kernel timing.  While enabled, CUDA events on the context's stream bracket
 * every walk-kernel launch.  gfk_profile_read synchronises the stream and
 * returns the summed device time of those launches (ms), their number and the
 * walker-steps they advanced (sum over launches of live-or-dead walkers x
 * steps), then clears the tallies if reset != 0.  Any pointer may be NULL. */
gfk_status gfk_profile(gfk_ctx* ctx, int32_t enable);
gfk_status gfk_profile_read(gfk_ctx* ctx, double* walk_ms, int64_t* launches,
                            double* walker_steps, int32_t reset);

/* Number of kernels gfk_propagate has queued on the context's stream since
 * gfk_create or the last reset of the count (reset != 0 clears it after
 * reading): for each initialisation its kernel and the merge of its sums, for
 * each chunk of moves the walk kernels (one per run of instances that share a
 * specialised kernel) and the merge, and for a CUDA-graph replay the kernels
 * the graph holds.  GFK_EINVAL for a NULL argument. */
gfk_status gfk_kernel_count(gfk_ctx* ctx, int64_t* count, int32_t reset);

/* Allocation-free variant of the mixed-precision walk (the paper has no
 * counterpart: this is a service to callers that cannot let a library call
 * cudaMalloc -- frameworks that own all device memory through their own
 * caching allocator or an arena reserved at start-up, and processes with a
 * fixed memory budget, for whom a cudaMalloc would synchronise the device,
 * could fail mid-run and fragments memory).
 *
 * Runs the same init / walk / merge kernels as gfk_propagate on one instance
 * (desc->prec must be GFK_PREC_MIXED), with a fixed launch shape of 256
 * threads x 2 walkers per thread, on memory the caller provides:
 *   dev_p0, dev_p1  device float4[n_walkers] each (16-byte aligned): the
 *                   walker planes p0 = (x1,y1,z1,x2), p1 = (y2,z2, log-weight as
 *                   two 32-bit halves); written when init != 0, read and
 *                   written otherwise
 *   dev_sgn         device int8[n_walkers]: sign of psi at the start, 0 = dead
 *   dev_rows        device double[(n_steps + (init ? 1 : 0)) * 6]: per-step sums
 *                   {c, W, P, Q, R, n_alive} as in gfk_sums; row 0 is the initial
 *                   population when init != 0
 *   dev_counters    device uint64[3]: the counters of gfk_counters; zeroed by
 *                   the call when init != 0, accumulated otherwise
 * step0 is the global step of the first move (0 when init != 0).  The call is
 * asynchronous on cuda_stream (NULL = legacy default stream).
 * The moves are walked in chunks of a multiple of 64 moves (64 at
 * GFK_NOALLOC_MAX_WALKERS, up to 1024 for smaller populations), so the FP32
 * log-weight increments are folded into the FP64 base after the same moves
 * as in gfk_propagate: walkers, per-step sums and counters equal those of a
 * context with launch shape (256, 2) given the same sequence of calls.
 * It allocates nothing.  Its only other device memory is a file-scope array of
 * GFK_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until
 * the process exits; the first call on each device looks up that array's
 * address (make this first call before any stream capture).  All calls share
 * the array, so calls that overlap on the GPU race; each call rewrites what it
 * reads.  Returns GFK_EINVAL for n_walkers above GFK_NOALLOC_MAX_WALKERS (the
 * most whose per-move records fit the array, 64 moves at a time) or any other
 * bad argument, GFK_ECUDA if a launch fails. */
#define GFK_NOALLOC_SCRATCH_BYTES (32u << 20)
#define GFK_NOALLOC_MAX_WALKERS (1ll << 22)
gfk_status gfk_propagate_noalloc(const gfk_instance_desc* desc, int32_t trial_kind,
                                 const double* params, int32_t n_params,
                                 void* dev_p0, void* dev_p1, int8_t* dev_sgn,
                                 int32_t init, int64_t step0, int64_t n_steps,
                                 double* dev_rows, unsigned long long* dev_counters,
                                 void* cuda_stream);

/* Forget the population: the next gfk_propagate re-initialises it (step 0). */
gfk_status gfk_reset(gfk_ctx* ctx);

/* Free the context and everything it allocated.  NULL is ignored. */
void gfk_destroy(gfk_ctx* ctx);

/* Static description of a status code. */
const char* gfk_status_string(gfk_status s);

/* The last CUDA error message recorded by ctx ("" if none). */
const char* gfk_last_error(gfk_ctx* ctx);

/* ------------------------------------------------------------------------
 * Diagnostics and measurement utilities.  None of these is a step of the
 * method: they measure the device (instruction rates), check the FP32
 * arithmetic of the mixed walk (moments of its normals, its trial evaluation
 * at given positions) and read the debug build's bounds checks.  The tests
 * and the benchmark use them; a user of the walk does not need them.
 * ------------------------------------------------------------------------ */

/* Instruction-throughput microbenchmarks (a measurement utility; the paper has
 * no counterpart): the denominators of the walk kernels' ALU roofline,
 * measured on the current device.  Each op runs independent chains of one
 * PTX instruction on every SM; *lane_ops_per_s receives thread-level
 * operations per second (one fma = one op; GFK_PEAK_IMAD_WIDE counts one
 * mad.wide plus one xor per op; GFK_PEAK_F2F counts each of the two
 * conversions of a float -> double -> float round trip; GFK_PEAK_FFMA2 counts
 * the two fused multiply-adds of one packed fma.rn.f32x2).  Takes about 10 ms;
 * synchronises cuda_stream; allocates 4 bytes from the stream-ordered pool. */
typedef enum {
    GFK_PEAK_FFMA = 0, GFK_PEAK_DFMA, GFK_PEAK_IMAD, GFK_PEAK_IMAD_HI, GFK_PEAK_IMAD_WIDE,
    GFK_PEAK_LOP3, GFK_PEAK_EX2, GFK_PEAK_RSQ, GFK_PEAK_LG2, GFK_PEAK_SIN, GFK_PEAK_I2F,
    GFK_PEAK_F2F, GFK_PEAK_FFMA2, GFK_PEAK_COUNT
} gfk_peak_op;
gfk_status gfk_measure_peak(int32_t op, void* cuda_stream, double* lane_ops_per_s);

/* Exhaustive moments of the FP32 Box-Muller normals of the GFK_PREC_MIXED walk
 * (Gaussian noise), against FP64.  Over all 2^32 radius words w, with
 * r2(w) the squared radius and rho = sqrt(r2) as the kernels compute them and
 * R2(w) = -2 ln((w + 1/2) 2^-32) in FP64:
 *   moments[0] = mean of r2 - R2,   moments[1] = mean of rho^2 - R2;
 * over the 1024 angles of the grid, with c, s the kernels' cosine and sine:
 *   moments[2] = mean c^2 - 1/2,    moments[3] = mean s^2 - 1/2,
 *   moments[4] = mean c,            moments[5] = mean s.
 * The normals' variances are (2 + moments[1]) (1/2 + moments[2]) and
 * (2 + moments[1]) (1/2 + moments[3]).  method selects r2: 0 the kernels'
 * (hardware log2 plus its mean-error correction), 1 the hardware log2 alone,
 * 2 the library logf.  Runs on the current device and on `cuda_stream`, which
 * it synchronises.  GFK_EINVAL for a bad method or a NULL output. */
gfk_status gfk_normal_moments(int32_t method, void* cuda_stream, double* moments);

/* The FP32 trial evaluation of the GFK_PREC_MIXED walk at caller-given
 * positions (a diagnostic: the same device code the walk kernels run).
 * host_x holds n walkers x 6 floats (walker-major).  lanes = 1 evaluates each
 * walker alone, lanes = 2 two at a time in the packed form of the walk
 * kernels with 2 or 4 walkers per thread (an odd last walker is paired with
 * itself); both give the same results bit for bit.  Outputs (host, any may be
 * NULL): host_b n x 6 drift components, host_el n local energies, host_sign n
 * signs of psi (0 where psi is exactly zero).  Runs on the current device and
 * on cuda_stream, which it synchronises; takes its device memory from the
 * stream-ordered pool.  GFK_EINVAL for a bad argument or parameter vector. */
gfk_status gfk_eval_f32(int32_t trial_kind, const double* params, int32_t n_params,
                        int32_t ee_on, int64_t n, const float* host_x, int32_t lanes,
                        float* host_b, float* host_el, int32_t* host_sign, void* cuda_stream);

/* Bounds checks of the debug build (the library compiled with -DGFK_DEBUG,
 * libgfk_debug.so; not a passage of the paper: a tool for changing the
 * library).  That build registers every device buffer it allocates, the
 * allocation-free entry point's scratch and the caller buffers passed to it,
 * and its kernels check each access to walker state, block records, per-step
 * series, exported walkers and the gradient's checkpoints, segments and
 * trajectory against those ranges.  A failed check skips the access (a load
 * reads zeros), sets a bit in a device status word and records the first
 * failing device address; no kernel traps.  Registration synchronises the
 * device, so the debug build is slow and is not for timing.
 *   *debug_build  1 in the debug build, 0 in the release build (which has no
 *                 checks and reports zeros)
 *   *flags        the bits that failed since the last clear: 1 walker state,
 *                 2 block record, 4 series row or exported walker, 8
 *                 checkpoint / segment / trajectory, 16 more live buffers than
 *                 the table holds (checks were off)
 *   *first_addr   the first failing address (0 if none)
 *   clear != 0    resets flags and address after reading them
 * Any pointer may be NULL.  Reads the current device's word (synchronous);
 * GFK_ECUDA if that fails. */
gfk_status gfk_debug_status(int32_t* debug_build, uint32_t* flags, uint64_t* first_addr,
                            int32_t clear);

#ifdef __cplusplus
}
#endif

#endif /* GFK_H */
