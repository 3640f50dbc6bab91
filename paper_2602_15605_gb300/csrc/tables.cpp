// tables.cpp -- host builder of the g(p) lookup tables (Sec. 3.1).
//
// g(p) = (2p)! / (2^{2p} (p!)^2) (Eq. gdef) obeys g(p) = (p - 1/2)/p g(p-1),
// g(0) = 1 (Eq. g_rec).  The paper runs this recurrence on ln g and
// exponentiates; here it runs directly on g in double-double arithmetic
// (Dekker 1971 two-product / Knuth two-sum), which needs no logarithms
// because g(p) ~ (pi p)^{-1/2} stays far inside the FP64 range, and each
// entry is rounded to FP64 once.  The second table fuses the paper's 1/g
// and (J+1)^{-1} tables: h(p) = 1 / ((2p + 1) g(p)), so that the
// J-dependent part of Eq. 000_sq_main, 1 / ((J+1) g(J/2)), is a single load.
//
// This file must be compiled without floating-point contraction
// (-ffp-contract=off): the error-free transformations below rely on every
// product and sum being rounded separately.
#include <cmath>
#include <vector>

#include "internal.h"

namespace {

struct dd {
    double hi, lo;
};

inline dd quick_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    return {s, e};
}

inline dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

inline dd two_prod(double a, double b) {
    double p = a * b;
    double e = std::fma(a, b, -p);
    return {p, e};
}

// x * y for a double y
inline dd mul(dd x, double y) {
    dd p = two_prod(x.hi, y);
    p.lo += x.lo * y;
    return quick_two_sum(p.hi, p.lo);
}

// x / y for a double y
inline dd div(dd x, double y) {
    double q1 = x.hi / y;
    dd p = two_prod(q1, y);               // q1 * y exactly
    dd r = two_sum(x.hi, -p.hi);          // x - q1 y
    r.lo += x.lo - p.lo;
    double q2 = (r.hi + r.lo) / y;
    return quick_two_sum(q1, q2);
}

// 1 / x
inline dd recip(dd x) {
    double q1 = 1.0 / x.hi;
    dd p = mul(x, q1);                    // x q1 ~ 1
    dd r = two_sum(1.0, -p.hi);
    r.lo -= p.lo;
    double q2 = (r.hi + r.lo) / x.hi;
    return quick_two_sum(q1, q2);
}

}  // namespace

namespace cpl {

void build_tables_host(int pmax, std::vector<double> &g, std::vector<double> &h) {
    g.assign((size_t)pmax + 1, 0.0);
    h.assign((size_t)pmax + 1, 0.0);
    dd gp = {1.0, 0.0};
    for (int p = 0; p <= pmax; ++p) {
        if (p > 0) gp = div(mul(gp, 2.0 * p - 1.0), 2.0 * p);  // (p - 1/2)/p = (2p-1)/(2p)
        g[p] = gp.hi + gp.lo;
        dd den = mul(gp, 2.0 * p + 1.0);
        dd inv = recip(den);
        h[p] = inv.hi + inv.lo;
    }
}

}  // namespace cpl
