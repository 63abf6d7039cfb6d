/*
 * opcount.cpp -- counting build of the oracle (see opcount.h).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Built only by oracle/opcount.py for the test suite.
 * The oracle's sources are compiled here as C++ with every double counting its operations;
 * or_opcount_trace traces a list of impact points and returns the counters and the number of
 * interactions of the rays that hit.
 */
#define OR_OPCOUNT 1
#include "opcount.h"

#include "rtw_oracle.c"
#include "mlp_oracle.c"

#undef double

or_opcount g_or_opcount;

/* params: the or_make_object parameter vector (OR_NPARAM doubles); xy: n impact points; records
 * of every ray go to out (n x (pmax+1) x OR_NFIELD doubles, may be NULL); counts (5): additions,
 * multiplications, divisions, square roots, elementary functions.  Returns the number of
 * interactions of the rays that hit (pmax + 1 each), or -1 for invalid parameters. */
extern "C" int64_t or_opcount_trace(const double* params, const double* xy, int64_t n, int pmax, double* out,
                                    unsigned long long* counts)
{
    or_cdbl p[OR_NPARAM];
    for (int i = 0; i < OR_NPARAM; ++i) p[i] = params[i];
    or_object* o = (or_object*)malloc(sizeof(or_object));
    if (or_make_object(p, o) != 0) {
        free(o);
        return -1;
    }
    const int np = pmax + 1;
    or_cdbl* rec = (or_cdbl*)malloc(sizeof(or_cdbl) * (size_t)np * OR_NFIELD);
    g_or_opcount = or_opcount{0, 0, 0, 0, 0};
    int64_t inter = 0;
    for (int64_t k = 0; k < n; ++k) {
        const int hit = or_trace_ray(o, xy[2 * k], xy[2 * k + 1], pmax, rec, NULL);
        if (hit) inter += np;
        if (out)
            for (int64_t j = 0; j < (int64_t)np * OR_NFIELD; ++j) out[k * np * OR_NFIELD + j] = rec[j].v;
    }
    counts[0] = g_or_opcount.add;
    counts[1] = g_or_opcount.mul;
    counts[2] = g_or_opcount.div;
    counts[3] = g_or_opcount.sqrt;
    counts[4] = g_or_opcount.fn;
    free(rec);
    free(o);
    return inter;
}
