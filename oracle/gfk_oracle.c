/*
 * Oracle for the importance-sampled generalized Feynman-Kac (GFK) random walk
 * for helium (Datta, Rejcek, Fry, "The He atom revisited", arXiv:1703.08977).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct
 * FP64 CPU restatement of what the GPU path computes.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark load it.  It shares
 * no code, header, table or helper with the CUDA library: everything below is
 * written again from the paper and from the published definitions it cites.
 *
 * What it computes, in the paper's terms:
 *  - H = -Delta/2 + V on R^6 (two electrons, d = 3N, Sec. "Path Integral
 *    Theory", Eq. 1), V = -2/r1 - 2/r2 + 1/r12 (helium, Z_nuc = 2).
 *  - The GFK split H = H0 + V_P with V_P = V - lambda0 - Delta(phi)/(2 phi)
 *    (the text prints Delta(phi)/phi; the 1/2 is required for H0 phi = lambda0
 *    phi with H0 = -Delta/2 + V0).  So V_P = E_L - E_T with the local energy
 *    E_L = -Delta(psi)/(2 psi) + V and E_T = lambda0.
 *  - The drifted diffusion dY = grad(psi)/psi dt + dX (the SDE under Eq. 4),
 *    discretised by Euler-Maruyama with Gaussian increments.
 *  - The Feynman-Kac weight exp(-int V_P ds) of Eq. 4, by the right-point
 *    Riemann sum of the invariance-principle construction (the sum over
 *    l = 1..nt in the discretisation section): after each move the walker's
 *    log-weight decreases by (E_L(X_new) - E_T) dt.
 *  - Space averaging over N_rep independent replications (the law-of-large-
 *    numbers step after the invariance principle): after every step the
 *    population sums W = sum w, P = sum w E_L, Q = sum w^2, R = sum w E_L^2,
 *    giving E(t) = P/W and z(t) = W/N.
 *  - Fixed-node handling (the remarks on nodal structure in the
 *    introduction and before the trial-function list): a walker whose trial
 *    function changes sign (or becomes exactly zero) is killed.
 *
 * Random numbers: two noise modes.  Mode 0 (Gaussian increments): Philox4x32-10
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11) with Box-Muller normals.  Mode 1 (the paper's own scheme): Bernoulli
 * +-1 increments from the "Superduper" congruential generator, one generator
 * per walker (section "Bernoulli steps" below).  For mode 0 the counter is
 * (walker id, move index, instance id, tag), the key the two halves of the
 * 64-bit seed.  Move n (from global step n to n + 1) takes the one block
 * (walker, n, instance, 0); the initial position the block (walker, 0,
 * instance, 1).  A block's four words give six normals by the Box-Muller
 * transform (Box and Muller 1958), xi = sqrt(-2 ln u_a) (cos 2 pi u_b,
 * sin 2 pi u_b), three times: the radius uniforms u_a = (w_j + 1/2) 2^-32 from
 * words 0, 1, 2, and the angle uniforms u_b = (k_j + 1/2) / 1024 on an equally
 * spaced grid of 1024 angles, k_j = bits 10 j .. 10 j + 9 of word 3.  On such
 * a grid the angular moments cos^p and sin^p average to their continuous
 * values for every p below 1024, so the normals' moments that drive the walk
 * are those of the continuous transform.
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                            */
/* ------------------------------------------------------------------------ */

/* Round multipliers and Weyl key increments of Philox4x32 (Salmon et al.). */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {            /* the key is bumped before rounds 2..10 */
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on (0,1) from one 32-bit word: (w + 1/2) / 2^32. */
double orc_uniform(uint32_t w)
{
    return ((double)w + 0.5) * (1.0 / 4294967296.0);
}

/* Angle uniform from a 10-bit grid index: (k + 1/2) / 1024. */
double orc_angle_uniform(uint32_t k)
{
    return ((double)k + 0.5) * (1.0 / 1024.0);
}

/* Box-Muller pair from a radius word and an angle index:
 * xi_a = rho cos(2 pi u_b), xi_b = rho sin(2 pi u_b), rho = sqrt(-2 ln u_a). */
static void orc_box_muller(uint32_t wa, uint32_t kb, double* xa, double* xb)
{
    const double two_pi = 6.283185307179586476925286766559;
    double ua = orc_uniform(wa);
    double ub = orc_angle_uniform(kb);
    double rho = sqrt(-2.0 * log(ua));
    double ang = two_pi * ub;
    *xa = rho * cos(ang);
    *xb = rho * sin(ang);
}

/* Six standard normals from the four words of one Philox block: Box-Muller on
 * the radius words w0, w1, w2 with the angle indices of bits 0-9, 10-19 and
 * 20-29 of w3. */
static void orc_normals_from_block(const uint32_t w[4], double xi[6])
{
    for (int j = 0; j < 3; ++j)
        orc_box_muller(w[j], (w[3] >> (10 * j)) & 1023u, &xi[2 * j], &xi[2 * j + 1]);
}

/* The block (walker, n, inst, tag). */
static void orc_block(uint64_t seed, uint32_t walker, uint32_t n, uint32_t inst, uint32_t tag,
                      uint32_t words[4])
{
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { walker, n, inst, tag };
    orc_philox4x32_10(ctr, key, words);
}

/* The six normals of move `step` (from global step `step` to step + 1). */
void orc_move_normals(uint64_t seed, uint32_t walker, uint32_t step, uint32_t inst,
                      double xi[6])
{
    uint32_t words[4];
    orc_block(seed, walker, step, inst, 0u, words);
    orc_normals_from_block(words, xi);
}

/* The six normals of the initial position: the block (walker, 0, inst, 1). */
void orc_init_normals(uint64_t seed, uint32_t walker, uint32_t inst, double xi[6])
{
    uint32_t words[4];
    orc_block(seed, walker, 0u, inst, 1u, words);
    orc_normals_from_block(words, xi);
}

/* ------------------------------------------------------------------------ */
/* Bernoulli steps from the "Superduper" congruential generator             */
/* ------------------------------------------------------------------------ */
/*
 * The paper's own discretisation of the Brownian motion (the construction of
 * W(l) before the invariance principle, and the generator paragraph after the
 * space-averaging remarks): every coordinate moves by eps / sqrt(n) per time
 * step 1/n, with eps = +1 or -1 independently and with equal probability.  With
 * the time step written dt = 1/n the increment is sqrt(dt) eps, so this mode
 * replaces the Gaussian xi of the Euler-Maruyama move by eps and nothing else.
 *
 * eps comes from the congruential generator the paper calls "Superduper",
 * S_i = (69069 S_{i-1} + 1) mod 2^32, with eps_i = +1 if S_i > 2^31 and
 * eps_i = -1 otherwise (so S_i = 2^31 gives -1).
 *
 * The paper names one initial seed S_0 but not how the draws are shared among
 * paths.  Here every walker runs its own generator: its S_0 is word 0 of the
 * Philox block (walker, 0, inst, 5), and move `step` uses the outputs
 * S_{6 step + 1} .. S_{6 step + 6} for the coordinates x1, y1, z1, x2, y2, z2 in
 * that order.  The oracle steps each generator serially, one output at a time.
 */
#define ORC_SUPERDUPER_MULT 69069u

uint32_t orc_superduper_next(uint32_t s)
{
    /* unsigned 32-bit arithmetic wraps modulo 2^32 */
    return (uint32_t)(ORC_SUPERDUPER_MULT * s + 1u);
}

int orc_bernoulli_eps(uint32_t s)
{
    return s > 2147483648u ? 1 : -1;
}

uint32_t orc_superduper_seed(uint64_t seed, uint32_t walker, uint32_t inst)
{
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { walker, 0u, inst, 5u };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[0];
}

/* The six increments of one move: advances *state by six outputs. */
static void orc_bernoulli_step(uint32_t* state, double eps[6])
{
    for (int d = 0; d < 6; ++d) {
        *state = orc_superduper_next(*state);
        eps[d] = (double)orc_bernoulli_eps(*state);
    }
}

/* The six increments of move `step` of a walker, by stepping its generator
 * from S_0 through all earlier moves (cost proportional to step). */
void orc_move_bernoulli(uint64_t seed, uint32_t walker, uint32_t step, uint32_t inst,
                        double eps[6])
{
    uint32_t s = orc_superduper_seed(seed, walker, inst);
    for (uint32_t k = 0; k <= step; ++k) orc_bernoulli_step(&s, eps);
}

/* ------------------------------------------------------------------------ */
/* Trial functions                                                          */
/* ------------------------------------------------------------------------ */
/*
 * Every trial function here has the form psi = Phi(r1_vec, r2_vec) exp(u(r12))
 * with
 *   Phi = sum_t s_t f_{A,t}(r1_vec) f_{B,t}(r2_vec),
 *   f(r_vec) = (c0 + c1 r + cz z) exp(-alpha r)          (one-electron orbital)
 *   u(r) = a rho + sum_{k=1..4} c_k rho^(k+1),  rho = r / (1 + beta r)
 * Kind 0 ("Jastrow product", the ground-state form exp(-Z r1 - Z r2) times the
 * Pade-Jastrow factor) is the single term s = 1, f_A = f_B = exp(-Z r).
 * Kind 1 ("orbital pairs") covers the antisymmetrised 1s2s-like functions of
 * the trial-function list (functions 3, 4, 5), the P_z function 7 and the
 * excited-state trial functions of the benchmark workloads.
 *
 * Parameter vectors:
 *   kind 0: [Z, a, beta, c1, c2, c3, c4]            (c_k may be omitted: 0)
 *   kind 1: [a, beta, c1, c2, c3, c4, nterms,
 *            then per term s, alphaA, c0A, c1A, czA, alphaB, c0B, c1B, czB]
 */

#define ORC_MAX_TERMS 8

typedef struct {
    double s;
    double alpha[2], c0[2], c1[2], cz[2];   /* [0] = electron 1 (A), [1] = electron 2 (B) */
} orc_term;

typedef struct {
    double a, beta, ck[4];
    int nterms;
    orc_term term[ORC_MAX_TERMS];
} orc_trial;

/* Returns 0 on success, -1 on a malformed parameter vector. */
static int orc_trial_parse(int kind, const double* p, int np, orc_trial* t)
{
    memset(t, 0, sizeof(*t));
    if (kind == 0) {
        if (np < 3 || np > 7) return -1;
        double Z = p[0];
        t->a = p[1];
        t->beta = p[2];
        for (int k = 0; k < 4; ++k) t->ck[k] = (3 + k < np) ? p[3 + k] : 0.0;
        t->nterms = 1;
        t->term[0].s = 1.0;
        for (int e = 0; e < 2; ++e) {
            t->term[0].alpha[e] = Z;
            t->term[0].c0[e] = 1.0;
            t->term[0].c1[e] = 0.0;
            t->term[0].cz[e] = 0.0;
        }
        return 0;
    }
    if (kind == 1) {
        if (np < 7) return -1;
        t->a = p[0];
        t->beta = p[1];
        for (int k = 0; k < 4; ++k) t->ck[k] = p[2 + k];
        int nt = (int)p[6];
        if (nt < 1 || nt > ORC_MAX_TERMS || np != 7 + 9 * nt) return -1;
        t->nterms = nt;
        for (int i = 0; i < nt; ++i) {
            const double* q = p + 7 + 9 * i;
            t->term[i].s = q[0];
            t->term[i].alpha[0] = q[1]; t->term[i].c0[0] = q[2];
            t->term[i].c1[0] = q[3];    t->term[i].cz[0] = q[4];
            t->term[i].alpha[1] = q[5]; t->term[i].c0[1] = q[6];
            t->term[i].c1[1] = q[7];    t->term[i].cz[1] = q[8];
        }
        return 0;
    }
    return -1;
}

/* One-electron orbital f = (c0 + c1 r + cz z) e^{-alpha r} at r_vec:
 * value, gradient and Laplacian. */
static void orc_orbital(double alpha, double c0, double c1, double cz,
                        const double rv[3], double* f, double g[3], double* lap)
{
    double r = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
    double ex = exp(-alpha * r);
    double p = c0 + c1 * r + cz * rv[2];
    /* grad p = c1 r_vec / r + cz e_z ; grad e^{-alpha r} = -alpha (r_vec / r) e^{-alpha r} */
    double gp[3] = { c1 * rv[0] / r, c1 * rv[1] / r, c1 * rv[2] / r + cz };
    for (int d = 0; d < 3; ++d) g[d] = (gp[d] - alpha * p * rv[d] / r) * ex;
    /* lap(p e) = e lap p + 2 grad p . grad e + p lap e,
     * lap p = 2 c1 / r, grad p . r_hat = c1 + cz z / r, lap e = (alpha^2 - 2 alpha / r) e */
    double lap_p = 2.0 * c1 / r;
    double gp_dot_rhat = c1 + cz * rv[2] / r;
    *lap = (lap_p - 2.0 * alpha * gp_dot_rhat + p * (alpha * alpha - 2.0 * alpha / r)) * ex;
    *f = p * ex;
}

/* Jastrow factor u(r) = a rho + sum c_k rho^{k+1}, rho = r/(1+beta r):
 * u, du/dr, d2u/dr2. */
static void orc_jastrow(const orc_trial* t, double r, double* u, double* up, double* upp)
{
    double q = 1.0 + t->beta * r;
    double rho = r / q;
    double drho = 1.0 / (q * q);                  /* d rho / dr   */
    double d2rho = -2.0 * t->beta / (q * q * q);  /* d2 rho / dr2 */
    double val = t->a * rho;
    double d1 = t->a;                             /* du / d rho   */
    double d2 = 0.0;                              /* d2u / d rho2 */
    for (int k = 1; k <= 4; ++k) {
        double c = t->ck[k - 1];
        val += c * pow(rho, k + 1);
        d1 += c * (k + 1) * pow(rho, k);
        d2 += c * (k + 1) * k * pow(rho, k - 1);
    }
    *u = val;
    *up = d1 * drho;
    *upp = d2 * drho * drho + d1 * d2rho;
}

/*
 * Evaluate the trial function at X = (x1,y1,z1,x2,y2,z2).
 * Outputs: sign of psi (+1, -1 or 0), the drift b = grad ln|psi| (6),
 * the local energy E_L = -Delta(psi)/(2 psi) + V, and ln|psi|.
 * ee_on = 0 drops the 1/r12 repulsion from V (a test hook).
 * When psi = 0 the drift and E_L are set to NaN.
 */
static void orc_eval(const orc_trial* t, int ee_on, const double x[6],
                     int* sign, double b[6], double* el, double* lnpsi)
{
    const double* r1v = x;
    const double* r2v = x + 3;
    double Phi = 0.0, lapPhi = 0.0;
    double g1[3] = { 0, 0, 0 }, g2[3] = { 0, 0, 0 };
    for (int i = 0; i < t->nterms; ++i) {
        const orc_term* tm = &t->term[i];
        double fa, ga[3], la, fb, gb[3], lb;
        orc_orbital(tm->alpha[0], tm->c0[0], tm->c1[0], tm->cz[0], r1v, &fa, ga, &la);
        orc_orbital(tm->alpha[1], tm->c0[1], tm->c1[1], tm->cz[1], r2v, &fb, gb, &lb);
        Phi += tm->s * fa * fb;
        lapPhi += tm->s * (la * fb + fa * lb);
        for (int d = 0; d < 3; ++d) {
            g1[d] += tm->s * ga[d] * fb;
            g2[d] += tm->s * fa * gb[d];
        }
    }
    double r1 = sqrt(r1v[0] * r1v[0] + r1v[1] * r1v[1] + r1v[2] * r1v[2]);
    double r2 = sqrt(r2v[0] * r2v[0] + r2v[1] * r2v[1] + r2v[2] * r2v[2]);
    double d12[3] = { r1v[0] - r2v[0], r1v[1] - r2v[1], r1v[2] - r2v[2] };
    double r12 = sqrt(d12[0] * d12[0] + d12[1] * d12[1] + d12[2] * d12[2]);
    double u, up, upp;
    orc_jastrow(t, r12, &u, &up, &upp);

    if (!(Phi > 0.0 || Phi < 0.0)) {      /* exactly zero (or not a number) */
        *sign = 0;
        for (int d = 0; d < 6; ++d) b[d] = NAN;
        *el = NAN;
        *lnpsi = -INFINITY;
        return;
    }
    *sign = Phi > 0.0 ? 1 : -1;
    *lnpsi = log(fabs(Phi)) + u;

    /* grad_1 u = u' e12, grad_2 u = -u' e12 with e12 = (r1_vec - r2_vec)/r12 */
    double gu1[3], gu2[3];
    for (int d = 0; d < 3; ++d) {
        gu1[d] = up * d12[d] / r12;
        gu2[d] = -gu1[d];
    }
    double cross = 0.0;           /* grad Phi . grad u (both electrons) */
    for (int d = 0; d < 3; ++d) {
        b[d] = g1[d] / Phi + gu1[d];
        b[3 + d] = g2[d] / Phi + gu2[d];
        cross += g1[d] * gu1[d] + g2[d] * gu2[d];
    }
    double lap_u = 2.0 * (upp + 2.0 * up / r12);   /* Delta_1 u + Delta_2 u */
    double grad_u_sq = 2.0 * up * up;               /* |grad_1 u|^2 + |grad_2 u|^2 */
    /* Delta(Phi e^u) / (Phi e^u) */
    double lap_over_psi = lapPhi / Phi + 2.0 * cross / Phi + lap_u + grad_u_sq;
    double V = -2.0 / r1 - 2.0 / r2 + (ee_on ? 1.0 / r12 : 0.0);
    *el = -0.5 * lap_over_psi + V;
}

/* Public form of the evaluation for tests.  Returns 0, or -1 on bad params. */
int orc_trial_eval(int kind, const double* params, int n_params, int ee_on,
                   const double x[6], int* sign, double b[6], double* el,
                   double* lnpsi)
{
    orc_trial t;
    if (orc_trial_parse(kind, params, n_params, &t) != 0) return -1;
    orc_eval(&t, ee_on, x, sign, b, el, lnpsi);
    return 0;
}

/* The same evaluation at n points x[6 i .. 6 i + 5] (a loop over orc_eval,
 * for tests that evaluate whole populations).  Any output may be NULL.
 * Returns 0, or -1 on bad params. */
int orc_trial_eval_many(int kind, const double* params, int n_params, int ee_on,
                        int64_t n, const double* x, int* sign, double* b, double* el,
                        double* lnpsi)
{
    orc_trial t;
    if (orc_trial_parse(kind, params, n_params, &t) != 0) return -1;
    for (int64_t i = 0; i < n; ++i) {
        int s;
        double bi[6], e, lp;
        orc_eval(&t, ee_on, x + 6 * i, &s, bi, &e, &lp);
        if (sign) sign[i] = s;
        if (b) for (int d = 0; d < 6; ++d) b[6 * i + d] = bi[d];
        if (el) el[i] = e;
        if (lnpsi) lnpsi[i] = lp;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Compensated summation (Neumaier 1974)                                    */
/* ------------------------------------------------------------------------ */

typedef struct { double s, c; } orc_sum;

static void orc_sum_add(orc_sum* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

static double orc_sum_value(const orc_sum* a) { return a->s + a->c; }

/* Sum of an array in index order, compensated; exposed for tests. */
double orc_neumaier_sum(const double* v, int64_t n)
{
    orc_sum s = { 0.0, 0.0 };
    for (int64_t i = 0; i < n; ++i) orc_sum_add(&s, v[i]);
    return orc_sum_value(&s);
}

/* ------------------------------------------------------------------------ */
/* The GFK walk                                                             */
/* ------------------------------------------------------------------------ */

/* Population sums of one step, over alive walkers, in walker order, with the
 * weights shifted by c = max logw so that exp() cannot overflow:
 * row = { c, W, P, Q, R, n_alive } with W = sum e^{logw-c}, P = sum w E_L,
 * Q = sum w^2, R = sum w E_L^2. */
static void orc_population_sums(int64_t n, const double* logw, const double* el,
                                const uint8_t* alive, double row[6])
{
    double c = -INFINITY;
    int64_t n_alive = 0;
    for (int64_t i = 0; i < n; ++i)
        if (alive[i]) {
            if (logw[i] > c) c = logw[i];
            ++n_alive;
        }
    orc_sum W = { 0, 0 }, P = { 0, 0 }, Q = { 0, 0 }, R = { 0, 0 };
    if (n_alive > 0) {
        for (int64_t i = 0; i < n; ++i) {
            if (!alive[i]) continue;
            double w = exp(logw[i] - c);
            orc_sum_add(&W, w);
            orc_sum_add(&P, w * el[i]);
            orc_sum_add(&Q, w * w);
            orc_sum_add(&R, w * el[i] * el[i]);
        }
    } else {
        c = 0.0;
    }
    row[0] = c;
    row[1] = orc_sum_value(&W);
    row[2] = orc_sum_value(&P);
    row[3] = orc_sum_value(&Q);
    row[4] = orc_sum_value(&R);
    row[5] = (double)n_alive;
}

/*
 * Run the walk for n walkers with ids ids[0..n) (NULL: ids 0..n-1).
 * State arrays (x: 6n, logw, el, alive, sgn) are read and written.
 *  - do_init != 0: first initialise every walker (X0 = sigma * xi from the
 *    initial-position normals, logw = 0, alive = sign(psi(X0)) != 0 and finite) and write
 *    one stats row for the initial population (all weights 1).
 *  - then n_steps moves with global step counters step0 .. step0+n_steps-1,
 *    each followed by one stats row.
 * noise: 0 = Gaussian increments (Philox normals), 1 = Bernoulli increments
 *   from each walker's Superduper generator, whose state lcg[i] is set at
 *   initialisation and advanced by six outputs per move of an alive walker
 *   (lcg may be NULL for noise 0).
 * stats: (n_steps + (do_init ? 1 : 0)) rows of 6 doubles (see above), or NULL.
 * counters (may be NULL): [0] non-finite kills, [1] node kills,
 *   [2] coalescence events (r1, r2 or r12 below 1e-10 after a move).
 * Returns 0, or -1 on bad parameters.
 */
int orc_run(int kind, const double* params, int n_params, int ee_on,
            double dt, double e_trial, uint64_t seed, uint32_t inst, double sigma,
            int64_t n, const uint32_t* ids,
            double* x, double* logw, double* el, uint8_t* alive, int8_t* sgn,
            uint32_t step0, int64_t n_steps, int do_init,
            double* stats, int64_t* counters, int noise, uint32_t* lcg)
{
    orc_trial t;
    if (orc_trial_parse(kind, params, n_params, &t) != 0) return -1;
    if (n < 0 || n_steps < 0 || !(dt > 0.0)) return -1;
    if (noise != 0 && (noise != 1 || !lcg)) return -1;
    int64_t cnt[3] = { 0, 0, 0 };
    double sqrt_dt = sqrt(dt);
    int64_t row = 0;

    if (do_init) {
        for (int64_t i = 0; i < n; ++i) {
            uint32_t id = ids ? ids[i] : (uint32_t)i;
            double xi[6];
            orc_init_normals(seed, id, inst, xi);
            if (noise == 1) lcg[i] = orc_superduper_seed(seed, id, inst);
            double* xw = x + 6 * i;
            for (int d = 0; d < 6; ++d) xw[d] = sigma * xi[d];
            int s;
            double b[6], lp;
            orc_eval(&t, ee_on, xw, &s, b, &el[i], &lp);
            logw[i] = 0.0;
            int finite = isfinite(el[i]);
            for (int d = 0; d < 6; ++d) finite = finite && isfinite(b[d]);
            sgn[i] = (int8_t)s;
            alive[i] = (uint8_t)(s != 0 && finite);
            if (!alive[i]) {
                logw[i] = -INFINITY;
                if (s != 0) ++cnt[0]; else ++cnt[1];
            }
        }
        if (stats) orc_population_sums(n, logw, el, alive, stats + 6 * row);
        ++row;
    }

    for (int64_t k = 0; k < n_steps; ++k) {
        uint32_t step = step0 + (uint32_t)k;
        for (int64_t i = 0; i < n; ++i) {
            if (!alive[i]) continue;
            uint32_t id = ids ? ids[i] : (uint32_t)i;
            double* xw = x + 6 * i;
            /* drift at the current position */
            int s0;
            double b[6], e0, lp;
            orc_eval(&t, ee_on, xw, &s0, b, &e0, &lp);
            /* Euler-Maruyama move X <- X + b dt + sqrt(dt) xi; in the Bernoulli
             * mode xi is the walker's next six +-1 increments */
            double xi[6];
            if (noise == 1)
                orc_bernoulli_step(&lcg[i], xi);
            else
                orc_move_normals(seed, id, step, inst, xi);
            for (int d = 0; d < 6; ++d) xw[d] = xw[d] + b[d] * dt + sqrt_dt * xi[d];
            /* trial function at the new position */
            int s1;
            double b1[6], e1;
            orc_eval(&t, ee_on, xw, &s1, b1, &e1, &lp);
            double r1 = sqrt(xw[0] * xw[0] + xw[1] * xw[1] + xw[2] * xw[2]);
            double r2 = sqrt(xw[3] * xw[3] + xw[4] * xw[4] + xw[5] * xw[5]);
            double dx = xw[0] - xw[3], dy = xw[1] - xw[4], dz = xw[2] - xw[5];
            double r12 = sqrt(dx * dx + dy * dy + dz * dz);
            if (r1 < 1e-10 || r2 < 1e-10 || r12 < 1e-10) ++cnt[2];
            /* the order of the tests: a position that is not finite is a
             * non-finite kill; then a sign change (or psi = 0) is a node kill;
             * then a drift or local energy that is not finite */
            int xfinite = 1;
            for (int d = 0; d < 6; ++d) xfinite = xfinite && isfinite(xw[d]);
            if (xfinite && s1 != sgn[i]) {             /* node crossed (or psi = 0) */
                alive[i] = 0;
                logw[i] = -INFINITY;
                ++cnt[1];
                continue;
            }
            int finite = xfinite && isfinite(e1);
            for (int d = 0; d < 6; ++d) finite = finite && isfinite(b1[d]);
            if (!finite) {
                alive[i] = 0;
                logw[i] = -INFINITY;
                ++cnt[0];
                continue;
            }
            el[i] = e1;
            logw[i] = logw[i] - (e1 - e_trial) * dt;   /* right-point rule */
        }
        if (stats) orc_population_sums(n, logw, el, alive, stats + 6 * row);
        ++row;
    }
    if (counters)
        for (int j = 0; j < 3; ++j) counters[j] += cnt[j];
    return 0;
}
