// Host-side parsing of a trial-function parameter vector (the layouts
// gfk_trial_kind documents in gfk.h) into the TrialHost record the kernels
// read.  Shared by gfk_set_trial and gfk_propagate_noalloc.
#pragma once

#include <cmath>
#include <cstring>

#include "gfk_types.h"

namespace gfk {

// Returns false for a malformed vector: a null pointer, a non-finite value, a
// wrong length or term count, Z <= 0, beta < 0 or a negative orbital exponent.
inline bool parse_trial_params(int kind, const double* p, int np, TrialHost* t) {
    std::memset(t, 0, sizeof(*t));
    if (!p) return false;
    for (int i = 0; i < np; ++i)
        if (!std::isfinite(p[i])) return false;
    t->kind = kind;
    if (kind == GFK_TRIAL_JASTROW_PRODUCT) {
        if (np < 3 || np > 7) return false;
        t->Z = p[0];
        t->a = p[1];
        t->beta = p[2];
        for (int k = 0; k < 4; ++k) t->ck[k] = (3 + k < np) ? p[3 + k] : 0.0;
        t->nterms = 1;
        return t->Z > 0.0 && t->beta >= 0.0;
    }
    if (kind == GFK_TRIAL_ORBITAL_PAIRS) {
        if (np < 7) return false;
        t->a = p[0];
        t->beta = p[1];
        for (int k = 0; k < 4; ++k) t->ck[k] = p[2 + k];
        if (!(p[6] >= 1.0 && p[6] <= (double)GFK_MAX_TERMS)) return false;
        const int nt = (int)p[6];
        if ((double)nt != p[6] || np != 7 + 9 * nt) return false;
        if (t->beta < 0.0) return false;
        t->nterms = nt;
        for (int i = 0; i < nt; ++i) {
            const double* q = p + 7 + 9 * i;
            t->s[i] = q[0];
            t->alpha[i][0] = q[1]; t->c0[i][0] = q[2]; t->c1[i][0] = q[3]; t->cz[i][0] = q[4];
            t->alpha[i][1] = q[5]; t->c0[i][1] = q[6]; t->c1[i][1] = q[7]; t->cz[i][1] = q[8];
            if (t->alpha[i][0] < 0.0 || t->alpha[i][1] < 0.0) return false;
        }
        return true;
    }
    return false;
}

}  // namespace gfk
