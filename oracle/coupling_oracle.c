/*
 * coupling_oracle.c -- CPU FP64 oracle for the pseudo-C_ell mode-coupling
 * matrices of Kiddier & Gratton (arXiv 2602.15605).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check of __graft_entry__ and the CPU-baseline leg of bench.py may
 * build, load or call it.  It shares no code, header, table or constant with
 * the CUDA library, and it does not use the paper's lookup-table method at
 * all: every Wigner-3j value here comes from the classical Schulten-Gordon
 * three-term recursion in the first angular momentum (the S-G reference
 * method the paper benchmarks against, Sec. 1 and Sec. 4), normalised by the
 * orthogonality sum and given the sign of the stretched configuration.
 *
 * What is computed (Appendix A, Eqs. K_TT, Sig_TE and the EE / EB kernels):
 *
 *   M^X[l1][l2] = (2 l2 + 1) Xi_X(l1, l2),
 *   Xi_X(l1,l2) = 1/(4 pi) sum_{l3} (2 l3 + 1) W_{l3} S_X(l1, l2, l3)
 *
 *   S_TT   = (l1 l2 l3; 0 0 0)^2
 *   S_TE   = [L even] (l1 l2 l3; 0 0 0) (l1 l2 l3; -2 2 0)      (TB = TE)
 *   S_EE   = [L even] (l1 l2 l3; -2 2 0)^2                       (BB = EE)
 *   S_EEBB = [L odd]  (l1 l2 l3; -2 2 0)^2   (the paper's odd-parity "EB"
 *                                             kernel, EE <-> BB leakage)
 *   S_EB   = S_EE - S_EEBB                   (EB <-> EB block of the MASTER
 *                                             polarisation system)
 *
 * with L = l1 + l2 + l3 and l3 running over the triangle |l1-l2| .. l1+l2,
 * capped at the last supplied window entry and at an optional band limit
 * (Sec. 4.3: W is zero above L_cut, so the cap is exact).  Terms are summed
 * in ascending l3.  Alongside each element the oracle returns
 * S_abs = (2 l2 + 1)/(4 pi) sum |(2 l3 + 1) W_{l3} S_X|, the scale that the
 * per-element error metric divides by (signed spectra can cancel).
 *
 * The polarisation symbol (l1 l2 l3; -2 2 0) is evaluated as
 * (l3 l1 l2; 0 -2 2), its cyclic permutation (Eq. permutation), so that the
 * recursion variable l3 carries m = 0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Spectrum bits (order defines the output order of the requested set). */
#define ORC_TT   1u
#define ORC_TE   2u
#define ORC_EE   4u
#define ORC_EEBB 8u
#define ORC_EB   16u

/* A(j) of the Schulten-Gordon recursion for f(j) = (j j2 j3; m1 m2 m3). */
static double sg_A(double j, double j2, double j3, double m1)
{
    double a = (j * j - (j2 - j3) * (j2 - j3));
    double b = ((j2 + j3 + 1.0) * (j2 + j3 + 1.0) - j * j);
    double c = (j * j - m1 * m1);
    double p = a * b * c;
    return p > 0.0 ? sqrt(p) : 0.0;
}

/* B(j) of the Schulten-Gordon recursion. */
static double sg_B(double j, double j2, double j3, double m1, double m2, double m3)
{
    double w = 2.0 * j + 1.0;
    return -w * (j2 * (j2 + 1.0) * m1 - j3 * (j3 + 1.0) * m1 - j * (j + 1.0) * (m3 - m2));
}

/*
 * orc_threej_j1: all symbols f(j) = (j j2 j3; m1 m2 m3), m1 + m2 + m3 = 0,
 * for j = jmin .. jmax with jmin = max(|j2-j3|, |m1|), jmax = j2 + j3.
 *
 * The recursion  j A(j+1) f(j+1) + B(j) f(j) + (j+1) A(j) f(j-1) = 0  is run
 * downward from jmax (seed f(jmax) = 1, f(jmax+1) = 0) and, when jmin > 0,
 * upward from jmin (seed f(jmin) = 1, f(jmin-1) = 0).  Each sweep recurses
 * out of the end region where the solution grows, so both stay stable; the
 * upward solution is rescaled onto the downward one by least squares over
 * three points around the midpoint.  When jmin = 0 (j2 = j3, m1 = 0) the
 * j = 0 equation is empty, so the upward sweep takes its first two values
 * from the closed forms (0 j j; 0 m -m) = (-1)^(j-m) / sqrt(2j+1) and
 * (1 j j; 0 m -m) = (-1)^(j-m) m / sqrt(j(j+1)(2j+1)) (Edmonds 1957,
 * Table 2): f(1) / f(0) = m2 / sqrt(j2 (j2+1)).  (Carrying the downward sweep
 * down to j = 0 instead loses the small odd-j values: 5e-11 relative at
 * j2 = 9000.)  With all m zero the odd-j values vanish and the downward
 * sweep is carried all the way.  Finally sum_j (2j+1) f(j)^2 = 1 and
 * sign f(jmax) = (-1)^(j2 - j3 - m1).
 *
 * out must hold jmax - jmin + 1 doubles; out[k] = f(jmin + k).
 * Returns the count, 0 if the symbol set is empty, -1 on bad arguments.
 */
int orc_threej_j1(int j2, int j3, int m1, int m2, int m3, double *out, int out_len)
{
    if (j2 < 0 || j3 < 0 || m1 + m2 + m3 != 0) return -1;
    if (abs(m2) > j2 || abs(m3) > j3) return 0;
    int jmin = abs(j2 - j3);
    if (abs(m1) > jmin) jmin = abs(m1);
    int jmax = j2 + j3;
    if (jmax < jmin) return 0;
    int n = jmax - jmin + 1;
    if (out_len < n) return -1;
    const double J2 = j2, J3 = j3, M1 = m1, M2 = m2, M3 = m3;
    const double BIG = 1e150, SMALL = 1e-150;

    if (n == 1) {
        out[0] = 1.0;
    } else {
        /* downward sweep */
        const int seed2 = (jmin == 0 && m2 != 0);   /* upward sweep seeded by the two closed forms */
        int jstop = (jmin == 0 && !seed2) ? 0 : (jmin + jmax) / 2 - 1;
        if (jstop < jmin) jstop = jmin;
        for (int k = 0; k < n; k++) out[k] = 0.0;
        out[n - 1] = 1.0;
        double fp1 = 0.0;                    /* f(j+1) */
        for (int j = jmax; j > jstop; j--) {
            double fj = out[j - jmin];
            double Aj = sg_A(j, J2, J3, M1);
            double Ajp1 = sg_A(j + 1, J2, J3, M1);
            double fm1 = -(sg_B(j, J2, J3, M1, M2, M3) * fj + j * Ajp1 * fp1) / ((j + 1) * Aj);
            out[j - 1 - jmin] = fm1;
            fp1 = fj;
            if (fabs(fm1) > BIG) {
                for (int q = j - 1 - jmin; q < n; q++) out[q] *= SMALL;
                fp1 *= SMALL;
            }
        }
        if ((jmin > 0 || seed2) && jstop > jmin) {
            /* upward sweep from jmin to jstop + 2, into a scratch array */
            int nu = jstop + 2 - jmin + 1;
            double *up = (double *)malloc(sizeof(double) * (size_t)nu);
            if (!up) return -1;
            up[0] = 1.0;
            double fm1 = 0.0;                /* f(j-1) */
            int jfirst = jmin;
            if (seed2) {                     /* f(0) = 1, f(1) = m2 / sqrt(j2 (j2+1)) */
                up[1] = M2 / sqrt(J2 * (J2 + 1.0));
                fm1 = up[0];
                jfirst = 1;
            }
            for (int j = jfirst; j < jstop + 2; j++) {
                double fj = up[j - jmin];
                double Aj = sg_A(j, J2, J3, M1);
                double Ajp1 = sg_A(j + 1, J2, J3, M1);
                double fnext = -(sg_B(j, J2, J3, M1, M2, M3) * fj + (j + 1) * Aj * fm1) / (j * Ajp1);
                up[j + 1 - jmin] = fnext;
                fm1 = fj;
                if (fabs(fnext) > BIG) {
                    for (int q = 0; q <= j + 1 - jmin; q++) up[q] *= SMALL;
                    fm1 *= SMALL;
                }
            }
            /* match on j = jstop .. jstop + 2 (downward values exist there) */
            double num = 0.0, den = 0.0;
            for (int j = jstop; j <= jstop + 2; j++) {
                num += out[j - jmin] * up[j - jmin];
                den += up[j - jmin] * up[j - jmin];
            }
            double scale = den > 0.0 ? num / den : 0.0;
            for (int j = jmin; j < jstop; j++) out[j - jmin] = up[j - jmin] * scale;
            free(up);
        }
    }
    /* normalisation and sign */
    double norm = 0.0;
    for (int k = 0; k < n; k++) {
        double j = jmin + k;
        norm += (2.0 * j + 1.0) * out[k] * out[k];
    }
    double c = 1.0 / sqrt(norm);
    int sgn_exp = j2 - j3 - m1;
    double want = (sgn_exp % 2 == 0) ? 1.0 : -1.0;
    if ((out[n - 1] < 0.0) != (want < 0.0)) c = -c;
    for (int k = 0; k < n; k++) out[k] *= c;
    return n;
}

static int popcount5(unsigned s)
{
    int c = 0;
    for (int b = 0; b < 5; b++) c += (s >> b) & 1u;
    return c;
}

/*
 * orc_coupling_pairs: M and S_abs for an explicit list of (l1, l2) pairs.
 *
 *   l1s, l2s    [npairs]                     multipoles (>= 0)
 *   W_tt/tp/pp  [n_win][w_len] row-major     window power spectra; W_tt is
 *               used by TT, W_tp by TE, W_pp by EE, EEBB and EB.  A window
 *               not needed by the requested set may be NULL.
 *   band_limit  [n_win] or NULL              last l3 kept per window
 *   spectra     OR of ORC_* bits
 *   out, sabs   [n_win][nspec][npairs]       nspec = bits set in spectra,
 *                                            ordered by bit value
 *   nthreads    OpenMP threads (<= 0: library default)
 * Returns 0, or -1 on bad arguments / allocation failure.
 */
int orc_coupling_pairs(int npairs, const int *l1s, const int *l2s, int n_win,
                       const double *W_tt, const double *W_tp, const double *W_pp,
                       int w_len, const int *band_limit, unsigned spectra,
                       double *out, double *sabs, int nthreads)
{
    if (npairs < 0 || n_win < 1 || w_len < 1 || (spectra & ~31u) || !spectra) return -1;
    if ((spectra & ORC_TT) && !W_tt) return -1;
    if ((spectra & ORC_TE) && !W_tp) return -1;
    if ((spectra & (ORC_EE | ORC_EEBB | ORC_EB)) && !W_pp) return -1;
    int lmax_seen = 0;
    for (int q = 0; q < npairs; q++) {
        if (l1s[q] < 0 || l2s[q] < 0) return -1;
        if (l1s[q] > lmax_seen) lmax_seen = l1s[q];
        if (l2s[q] > lmax_seen) lmax_seen = l2s[q];
    }
    const int nspec = popcount5(spectra);
    const int want_pol = (spectra & (ORC_TE | ORC_EE | ORC_EEBB | ORC_EB)) != 0;
    const int buf_len = 2 * lmax_seen + 2;
    const double inv4pi = 1.0 / (4.0 * M_PI);
    int status = 0;

#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double *f00 = (double *)malloc(sizeof(double) * (size_t)buf_len);
        double *f22 = (double *)malloc(sizeof(double) * (size_t)buf_len);
        if (!f00 || !f22) {
#pragma omp atomic write
            status = -1;
        }
#pragma omp for schedule(dynamic, 8)
        for (int q = 0; q < npairs; q++) {
            if (!f00 || !f22) continue;
            const int l1 = l1s[q], l2 = l2s[q];
            const int lo = abs(l1 - l2), hi = l1 + l2;
            /* (l3 l1 l2; 0 0 0) for l3 = lo..hi */
            int n00 = orc_threej_j1(l1, l2, 0, 0, 0, f00, buf_len);
            /* (l3 l1 l2; 0 -2 2) = (l1 l2 l3; -2 2 0); zero unless l1, l2 >= 2 */
            int n22 = 0;
            if (want_pol && l1 >= 2 && l2 >= 2)
                n22 = orc_threej_j1(l1, l2, 0, -2, 2, f22, buf_len);
            const double pref = 2.0 * l2 + 1.0;
            for (int w = 0; w < n_win; w++) {
                int top = hi;
                if (top > w_len - 1) top = w_len - 1;
                if (band_limit && band_limit[w] < top) top = band_limit[w];
                int si = 0;
                for (unsigned bit = 1; bit <= ORC_EB; bit <<= 1) {
                    if (!(spectra & bit)) continue;
                    const double *W = (bit == ORC_TT) ? W_tt : (bit == ORC_TE) ? W_tp : W_pp;
                    W += (size_t)w * (size_t)w_len;
                    double acc = 0.0, aabs = 0.0;
                    for (int l3 = lo; l3 <= top; l3++) {
                        const int k = l3 - lo;
                        const int even = ((l1 + l2 + l3) % 2) == 0;
                        double s = 0.0;
                        if (bit == ORC_TT) {
                            s = (n00 > 0) ? f00[k] * f00[k] : 0.0;
                        } else if (n22 > 0) {
                            const double p = f22[k];
                            if (bit == ORC_TE)        s = even ? f00[k] * p : 0.0;
                            else if (bit == ORC_EE)   s = even ? p * p : 0.0;
                            else if (bit == ORC_EEBB) s = !even ? p * p : 0.0;
                            else                      s = even ? p * p : -p * p;
                        }
                        const double wt = 2.0 * l3 + 1.0;
                        const double term = wt * W[l3] * s;
                        acc += term;
                        aabs += fabs(term);
                    }
                    const size_t o = ((size_t)w * nspec + si) * (size_t)npairs + q;
                    out[o] = pref * inv4pi * acc;
                    if (sabs) sabs[o] = pref * inv4pi * aabs;
                    si++;
                }
            }
        }
        free(f00);
        free(f22);
    }
    return status;
}
