// The FP32 trial evaluation of the mixed-precision walk in lanes (one walker
// in a float, or two in the lanes of a float2; gfk_lanes.cuh): drift,
// local energy and sign of the trial function, every operation written out
// with its rounding so that a walker's result is the same bit for bit in
// either form.  Included by gfk_device.cuh after the trial parameters
// (TrialDev) are defined.
#pragma once

#include "gfk_lanes.cuh"

namespace gfk {

// ---------------------------------------------------------------------------
// Trial evaluation in lanes (drift b = grad ln|psi|, local energy E_L, sign)
// ---------------------------------------------------------------------------
template <typename L>
struct EvalLanes {
    L b[6];
    L el;
    L rmin;                               // min(r1, r2, r12): the coalescence diagnostic
    int sign[LaneCount<L>::value];        // sign of psi per lane (0: exactly zero)
};

// No product is ever added to or subtracted from another value directly: the
// assembler fuses such a pair into a multiply-add in the packed form (with or
// without an explicit rounding modifier) but not always in the one-walker
// form, and the two forms would then differ in the last bit.  Every sum of a
// product is therefore an explicit multiply-add here, so there is nothing left
// to fuse, and a product only ever feeds a multiplication or a multiply-add's
// multiplicand or addend.

// u(r12) = a rho + sum c_k rho^{k+1}, rho = r/(1+beta r).  Returns u' and
// el + (ee - 2u')/r12 - u'' (the Jastrow factor's share of the local energy
// added to el), with (ee - 2 a rho')/r = [(ee - 2a)/r + ee beta (2 + beta r)] rho'
// (no 1/r12 cancellation) and the polynomial's share -2 h rho' / (1 + beta r),
// h = (du/drho - a)/rho:
//   (ee - 2u')/r12 = rho' [(ee - 2a)/r + ee beta (2 + beta r) - 2 h / (1 + beta r)].
template <typename L>
struct JastrowLanes { L up, el; };

template <typename L, typename TD, int POLY>
__device__ __forceinline__ JastrowLanes<L> jastrow_lanes(const TD& t, L r12, L i12, L el) {
    const L beta = splat<L>(t.beta);
    const L q = lfma(beta, r12, splat<L>(1.0f));
    const L iq = lrcp(q);
    const L drho = lmul(iq, iq);                                    // d rho / dr
    const L d2rho = lmul(lmul(splat<L>(t.m2beta), drho), iq);      // d2 rho / dr2
    // (ee - 2a)/r + ee beta (2 + beta r)
    const L jA = lfma(splat<L>(t.eem2a), i12,
                      lmul(splat<L>(t.eebeta), lfma(beta, r12, splat<L>(2.0f))));
    JastrowLanes<L> o;
    if (POLY != 0) {
        const L rho = lmul(r12, iq);
        // h = 2c1 + rho (3c2 + rho (4c3 + rho 5c4)), du/drho = a + rho h
        const L h = lfma(rho, lfma(rho, lfma(rho, splat<L>(t.c5), splat<L>(t.c4)),
                                   splat<L>(t.c3)),
                         splat<L>(t.c2));
        const L du = lfma(rho, h, splat<L>(t.a));
        const L d2u = lfma(rho, lfma(rho, lfma(rho, splat<L>(t.d20), splat<L>(t.d12)),
                                     splat<L>(t.d6)),
                           splat<L>(t.d2));
        o.up = lmul(du, drho);
        const L jF = lfma(lmul(splat<L>(-2.0f), h), iq, jA);
        el = lfma(jF, drho, el);                                   // + (ee - 2u')/r12
        el = lfma(lneg(lmul(d2u, drho)), drho, el);                // - u'' = - d2u rho'^2
        o.el = lfma(lneg(du), d2rho, el);                          //        - du rho''
    } else {                              // u = a rho: du/drho = a, d2u/drho2 = 0
        const L a = splat<L>(t.a);
        o.up = lmul(a, drho);
        el = lfma(jA, drho, el);
        o.el = lfma(lneg(a), d2rho, el);
    }
    return o;
}

// Squared distances |r1|^2, |r2|^2, |r1 - r2|^2 and the difference vector.
template <typename L>
__device__ __forceinline__ void pair_geometry(const L x[6], L& s1, L& s2, L& s12, L d[3]) {
    s1 = lfma(x[2], x[2], lfma(x[1], x[1], lmul(x[0], x[0])));
    s2 = lfma(x[5], x[5], lfma(x[4], x[4], lmul(x[3], x[3])));
    d[0] = lsub(x[0], x[3]);
    d[1] = lsub(x[1], x[4]);
    d[2] = lsub(x[2], x[5]);
    s12 = lfma(d[2], d[2], lfma(d[1], d[1], lmul(d[0], d[0])));
}

// Kind 0: psi = exp(-Z r1 - Z r2 + u(r12)) in the cusp-cancelled form
//   b_1 = -Z r1_hat + u' e12,  b_2 = -Z r2_hat - u' e12   (e12 = (r1 - r2)/r12)
//   E_L = (Z - 2)(1/r1 + 1/r2) - Z^2 + (ee - 2u')/r12 - u'' - u'^2
//         + Z u' (r1_hat - r2_hat) . e12.
template <typename L, typename TD, int POLY>
__device__ __forceinline__ void eval0_lanes(const TD& t, const L x[6], EvalLanes<L>& o) {
    L s1, s2, s12, d[3];
    pair_geometry(x, s1, s2, s12, d);
    L r1, r2, r12, i1, i2, i12;
    lradius(s1, r1, i1);
    lradius(s2, r2, i2);
    lradius(s12, r12, i12);
    const L e[3] = {lmul(d[0], i12), lmul(d[1], i12), lmul(d[2], i12)};
    const L el0 = lfma(splat<L>(t.Zm2), ladd(i1, i2), splat<L>(-t.Z2));
    const JastrowLanes<L> j = jastrow_lanes<L, TD, POLY>(t, r12, i12, el0);
    const L mZ = splat<L>(t.mZ);
    const L nup = lneg(j.up);
    L proj = splat<L>(0.0f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const L h1 = lmul(x[c], i1), h2 = lmul(x[3 + c], i2);
        o.b[c] = lfma(j.up, e[c], lmul(mZ, h1));
        o.b[3 + c] = lfma(nup, e[c], lmul(mZ, h2));
        // (r1_hat - r2_hat)_c = x1_c i1 - h2 as one multiply-add
        proj = lfma(lfma(x[c], i1, lneg(h2)), e[c], proj);
    }
    L el = lfma(nup, j.up, j.el);
    el = lfma(lmul(splat<L>(t.Z), j.up), proj, el);
    o.el = el;
    const L s = ladd(s1, s2);
#pragma unroll
    for (int k = 0; k < LaneCount<L>::value; ++k) o.sign[k] = isfinite(lane_at(s, k)) ? 1 : 0;
    o.rmin = lmin(lmin(r1, r2), r12);
}

// One term s_t f_A(r1) f_B(r2) of the orbital-pair trial function, orbitals
// f = p e^{-alpha r}, p = c0 + c1 r + cz z, with the largest exponent emax of
// the terms factored out: g = e^{arg - emax}, arg = -(alpha_A r1 + alpha_B r2).
// Per orbital (divided by its exponential):
//   grad f               = c1 r_hat + cz z_hat - alpha p r_hat
//   -lap f / 2 - 2 f / r = -c1/r + alpha (c1 + cz z / r) - alpha^2 p / 2 + (alpha - 2) p / r
// (the nuclear attraction folded into the kinetic term, so the 1/r
// singularities cancel exactly when the orbital meets the cusp).
// PLAIN: every orbital is c0 e^{-alpha r}, so the term is v = s c0A c0B g
// (the parameter product formed on the host), its gradients are
// -alpha_A v r1_hat and -alpha_B v r2_hat, and its kinetic part is
// v [((alpha_A - 2)/r1 - alpha_A^2/2) + ((alpha_B - 2)/r2 - alpha_B^2/2)].
template <typename L>
struct Kind1Lanes {
    L Phi, T, G1[3], G2[3];
};

template <typename L>
__device__ __forceinline__ L term_exponent(const TrialDev<float>& t, int k, L r1, L r2) {
    return lfma(splat<L>(t.mal[k][1]), r2, lmul(splat<L>(t.mal[k][0]), r1));
}

template <typename L, bool PLAIN>
__device__ __forceinline__ void kind1_term_lanes(const TrialDev<float>& t, int k, L arg, L r1,
                                                 L r2, const L ir[2], const L zz[2],
                                                 const L h1[3], const L h2[3], L emax,
                                                 Kind1Lanes<L>& acc) {
    const L g = lexp(lsub(arg, emax));
    if constexpr (PLAIN) {
        const L sc = splat<L>(t.sc[k]);
        const L v = lmul(sc, g);
        const L ga = lmul(splat<L>(t.mal[k][0]), v), gb = lmul(splat<L>(t.mal[k][1]), v);
        const L kin = ladd(lfma(splat<L>(t.km2[k][0]), ir[0], splat<L>(-t.hal2[k][0])),
                           lfma(splat<L>(t.km2[k][1]), ir[1], splat<L>(-t.hal2[k][1])));
        acc.Phi = lfma(sc, g, acc.Phi);
        acc.T = lfma(v, kin, acc.T);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            acc.G1[d] = lfma(ga, h1[d], acc.G1[d]);
            acc.G2[d] = lfma(gb, h2[d], acc.G2[d]);
        }
    } else {
        L p[2], K[2], gr[2][3];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const L* hh = e == 0 ? h1 : h2;
            const L al = splat<L>(t.al[k][e]), c1 = splat<L>(t.c1[k][e]);
            const L cz = splat<L>(t.cz[k][e]);
            const L rr = e == 0 ? r1 : r2;
            const L pe = lfma(cz, zz[e], lfma(c1, rr, splat<L>(t.c0[k][e])));
            const L radial = lfma(splat<L>(t.mal[k][e]), pe, c1);      // coefficient of r_hat
            gr[e][0] = lmul(radial, hh[0]);
            gr[e][1] = lmul(radial, hh[1]);
            gr[e][2] = lfma(radial, hh[2], cz);
            // -c1/r + alpha (c1 + cz z/r) - alpha^2 p / 2 + (alpha - 2) p / r
            const L a1 = lmul(al, lfma(lmul(cz, zz[e]), ir[e], c1));
            const L a2 = lfma(lneg(c1), ir[e], a1);
            const L a3 = lfma(splat<L>(-t.hal2[k][e]), pe, a2);
            K[e] = lfma(lmul(splat<L>(t.km2[k][e]), pe), ir[e], a3);
            p[e] = pe;
        }
        const L sg = lmul(splat<L>(t.s[k]), g);
        const L sp0 = lmul(sg, p[0]), sp1 = lmul(sg, p[1]);
        acc.Phi = lfma(sp0, p[1], acc.Phi);
        acc.T = lfma(K[0], sp1, lfma(sp0, K[1], acc.T));
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            acc.G1[d] = lfma(gr[0][d], sp1, acc.G1[d]);
            acc.G2[d] = lfma(sp0, gr[1][d], acc.G2[d]);
        }
    }
}

// Kind 1: psi = Phi exp(u(r12)), Phi = sum_t s_t f_A(r1) f_B(r2):
//   b_1 = grad_1 Phi / Phi + u' e12,  b_2 = grad_2 Phi / Phi - u' e12
//   E_L = T / Phi - u' (grad_1 Phi - grad_2 Phi) . e12 / Phi - u'' - u'^2
//         + (ee - 2u')/r12,   T = sum_t s_t [K_A p_B + p_A K_B] g_A g_B.
// UNROLL: the term loops run to NT (at most GFK_MAX_TERMS) with a uniform
// early exit (every parameter index a compile-time constant, for a trial held
// in the kernel's parameter bank); otherwise they run to t.nterms.  A trial of
// NT terms gets the same operations from any NT >= its term count.
template <typename L, bool UNROLL, bool PLAIN, int POLY, int NT = GFK_MAX_TERMS>
__device__ __forceinline__ void eval1_lanes(const TrialDev<float>& t, const L x[6],
                                            EvalLanes<L>& o) {
    L s1, s2, s12, d[3];
    pair_geometry(x, s1, s2, s12, d);
    L r1, r2, r12, i1, i2, i12;
    lradius(s1, r1, i1);
    lradius(s2, r2, i2);
    lradius(s12, r12, i12);
    const L e[3] = {lmul(d[0], i12), lmul(d[1], i12), lmul(d[2], i12)};
    const L h1[3] = {lmul(x[0], i1), lmul(x[1], i1), lmul(x[2], i1)};
    const L h2[3] = {lmul(x[3], i2), lmul(x[4], i2), lmul(x[5], i2)};
    const L ir[2] = {i1, i2};
    const L zz[2] = {x[2], x[5]};
    Kind1Lanes<L> acc;
    acc.Phi = acc.T = splat<L>(0.0f);
#pragma unroll
    for (int d = 0; d < 3; ++d) acc.G1[d] = acc.G2[d] = splat<L>(0.0f);
    if constexpr (UNROLL) {
        // every term's exponent once, then the largest of them
        L arg[NT];
        arg[0] = term_exponent(t, 0, r1, r2);
        L emax = arg[0];
#pragma unroll
        for (int k = 1; k < NT; ++k) {
            if (k >= t.nterms) break;
            arg[k] = term_exponent(t, k, r1, r2);
            emax = lmax(emax, arg[k]);
        }
        kind1_term_lanes<L, PLAIN>(t, 0, arg[0], r1, r2, ir, zz, h1, h2, emax, acc);
#pragma unroll
        for (int k = 1; k < NT; ++k) {
            if (k >= t.nterms) break;
            kind1_term_lanes<L, PLAIN>(t, k, arg[k], r1, r2, ir, zz, h1, h2, emax, acc);
        }
    } else {
        L emax = term_exponent(t, 0, r1, r2);
        for (int k = 1; k < t.nterms; ++k) emax = lmax(emax, term_exponent(t, k, r1, r2));
        for (int k = 0; k < t.nterms; ++k)
            kind1_term_lanes<L, PLAIN>(t, k, term_exponent(t, k, r1, r2), r1, r2, ir, zz, h1, h2,
                                       emax, acc);
    }
    const L iP = lrcp(acc.Phi);
    // u' first (the Jastrow factor's share of E_L is added once T / Phi is known)
    const JastrowLanes<L> j0 = jastrow_lanes<L, TrialDev<float>, POLY>(t, r12, i12,
                                                                        splat<L>(0.0f));
    const L up = j0.up, nup = lneg(up);
    L cross = splat<L>(0.0f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        o.b[c] = lfma(up, e[c], lmul(acc.G1[c], iP));
        o.b[3 + c] = lfma(nup, e[c], lmul(acc.G2[c], iP));
        cross = lfma(lsub(acc.G1[c], acc.G2[c]), e[c], cross);
    }
    // (T - u' (grad_1 Phi - grad_2 Phi) . e12) / Phi, then the Jastrow terms
    const JastrowLanes<L> j = jastrow_lanes<L, TrialDev<float>, POLY>(
        t, r12, i12, lmul(lfma(nup, cross, acc.T), iP));
    o.el = lfma(nup, up, j.el);
#pragma unroll
    for (int k = 0; k < LaneCount<L>::value; ++k) {
        const float ph = lane_at(acc.Phi, k);
        o.sign[k] = ph > 0.0f ? 1 : (ph < 0.0f ? -1 : 0);
    }
    o.rmin = lmin(lmin(r1, r2), r12);
}

// KIND 0 / 1 / 3 as for eval_trial (3: orbital pairs without prefactor terms);
// KIND 4 is KIND 1 for a two-term trial in the kernel's parameter bank (the
// term loops fixed at two: the same operations, fewer live registers);
// KIND 2 dispatches on t.kind.  POLY < 0 decides on the Jastrow polynomial at
// run time (one branch at the top).  An orbital-pair function whose orbitals
// all lack the prefactor terms (t.plain) is evaluated in the PLAIN form by
// every kernel, so its walkers do not depend on the kernel that runs them:
// KIND 3 always, KIND 1 and 2 by a block-uniform branch.  UNROLL (a trial in
// the kernel's parameter bank) is only used with KIND 1 for functions that
// have prefactor terms and with KIND 3 (the launcher's choice), so it needs
// no branch.
template <int KIND, typename L, bool UNROLL = false, int POLY = -1>
__device__ __forceinline__ void eval_lanes(const TrialDev<float>& t, const L x[6], EvalLanes<L>& o) {
    if constexpr (POLY < 0) {
        if (t.poly != 0) eval_lanes<KIND, L, UNROLL, 1>(t, x, o);
        else eval_lanes<KIND, L, UNROLL, 0>(t, x, o);
        return;
    } else {
        if (KIND == 0) {
            eval0_lanes<L, TrialDev<float>, POLY>(t, x, o);
        } else if (KIND == 3) {
            eval1_lanes<L, UNROLL, true, POLY>(t, x, o);
        } else if (KIND == 1 && UNROLL) {
            eval1_lanes<L, true, false, POLY>(t, x, o);
        } else if (KIND == 4) {
            eval1_lanes<L, true, false, POLY, 2>(t, x, o);
        } else if (KIND == 2 && t.kind == 0) {
            eval0_lanes<L, TrialDev<float>, POLY>(t, x, o);
        } else if (t.plain != 0) {
            eval1_lanes<L, false, true, POLY>(t, x, o);
        } else {
            eval1_lanes<L, false, false, POLY>(t, x, o);
        }
    }
}

// finite drift and local energy in every term (one test per lane: a sum is
// finite only if every term is)
template <typename L>
__device__ __forceinline__ L eval_check_sum(const EvalLanes<L>& o) {
    return ladd(ladd(ladd(o.b[0], o.b[1]), ladd(o.b[2], o.b[3])), ladd(ladd(o.b[4], o.b[5]), o.el));
}

}  // namespace gfk
