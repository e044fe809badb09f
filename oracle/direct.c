/*
 * Oracle: direct O(N^2) FP64 evaluation of the discretised oscillatory
 * integral transform g = K f, K_ij = alpha(x_i, xi_j) exp(2 pi i Phi(x_i, xi_j)).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may use it.  It shares no code with the CUDA path.
 *
 * Definition followed: Sec. 4 (the potential g(x) = sum_xi K(x,xi) f(xi)) and
 * the discretisation of Sec. 5, Eq. (1D-FIO)/(1D-xandxi): x_i = i/N and
 * xi_j = j - N/2 (the paper's 1-based x_i = (i-1)/N, xi_j = j-1-N/2 written
 * 0-based).  No quadrature weight.
 *
 * Phase kinds (the same numbering is used by the product's built-in kernels):
 *   0 DFT:   Phi = x xi                                   (closed-form pin)
 *   1 FIO:   Phi = x xi + c(x)|xi|,  c(x) = (2 + s sin 2 pi x)/16   (Sec. 5, Eq. 1D-FIO-kernal)
 *   2 FIOPW: Phi = x xi + c(x)|xi| for x < 1/2, x xi - c(x)|xi|/2 for x >= 1/2
 *   3 ONES:  Phi = 0                                      (structural pin)
 *   4 SEP:   Phi = p(x) + q(xi), p = 0.3 sin 2 pi x, q = xi^2/(4N)  (structural pin)
 * Amplitude: amp = 0 -> alpha = 1;  amp = 1 -> alpha = 1 + 0.25 sin(2 pi x) cos(2 pi xi / N).
 *
 * Accuracy: the x*xi part of the phase is reduced mod 1 exactly in integer
 * arithmetic (N is a power of two, so i*(j-N/2) mod N divided by N is exact);
 * the remaining part is reduced by subtracting the nearest integer; sums over j
 * are Neumaier-compensated.
 */
#include <math.h>
#include <stdint.h>

#define TWO_PI 6.283185307179586476925286766559

static int64_t mod_pos(int64_t a, int64_t n) { int64_t r = a % n; return r < 0 ? r + n : r; }

/* fractional phase of Phi(x_i, xi_j), in (-1, 2) */
static double phase_frac(int kind, double s, int64_t N, int64_t i, int64_t j)
{
    int64_t xi = j - N / 2;
    double x = (double)i / (double)N;
    double axi = (double)(xi < 0 ? -xi : xi);
    double t1 = 0.0, t2 = 0.0;
    if (kind == 0 || kind == 1 || kind == 2)
        t1 = (double)mod_pos(i * xi, N) / (double)N;
    if (kind == 1) {
        t2 = (2.0 + s * sin(TWO_PI * x)) / 16.0 * axi;
    } else if (kind == 2) {
        double c = (2.0 + s * sin(TWO_PI * x)) / 16.0;
        t2 = (2 * i < N) ? c * axi : -0.5 * c * axi;
    } else if (kind == 4) {
        double q = (double)mod_pos(xi * xi, 4 * N) / (double)(4 * N);
        t2 = 0.3 * sin(TWO_PI * x) + q;
    }
    t2 -= nearbyint(t2);
    return t1 + t2;
}

static double amplitude(int amp, int64_t N, int64_t i, int64_t j)
{
    if (!amp) return 1.0;
    double x = (double)i / (double)N;
    double xi = (double)(j - N / 2);
    return 1.0 + 0.25 * sin(TWO_PI * x) * cos(TWO_PI * xi / (double)N);
}

/* Neumaier compensated accumulation */
static inline void nsum(double* s, double* c, double v)
{
    double t = *s + v;
    if (fabs(*s) >= fabs(v)) *c += (*s - t) + v; else *c += (v - t) + *s;
    *s = t;
}

/* g[r][c] = sum_j K(rows[r], j) f[j][c]; f, g complex interleaved (re, im),
 * f is [N][m] with the m right-hand sides innermost, g is [nrows][m]. */
void oracle_direct(int kind, double s, int amp, int64_t N, const int64_t* rows,
                   int64_t nrows, const double* f, int64_t m, double* g)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        double sr[m > 0 ? m : 1], si[m > 0 ? m : 1], cr[m > 0 ? m : 1], ci[m > 0 ? m : 1];
        for (int64_t c = 0; c < m; ++c) sr[c] = si[c] = cr[c] = ci[c] = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double th = TWO_PI * phase_frac(kind, s, N, i, j);
            double a = amplitude(amp, N, i, j);
            double kr = a * cos(th), ki = a * sin(th);
            const double* fj = f + 2 * j * m;
            for (int64_t c = 0; c < m; ++c) {
                double fr = fj[2 * c], fi = fj[2 * c + 1];
                nsum(&sr[c], &cr[c], kr * fr);
                nsum(&sr[c], &cr[c], -ki * fi);
                nsum(&si[c], &ci[c], kr * fi);
                nsum(&si[c], &ci[c], ki * fr);
            }
        }
        for (int64_t c = 0; c < m; ++c) {
            g[2 * (r * m + c)] = sr[c] + cr[c];
            g[2 * (r * m + c) + 1] = si[c] + ci[c];
        }
    }
}

/* The same definition evaluated in long double throughout (phase, sin/cos,
 * products and plain summation): a brute-force cross-check for small N. */
void oracle_direct_ld(int kind, double s, int amp, int64_t N, const int64_t* rows,
                      int64_t nrows, const double* f, int64_t m, double* g)
{
    const long double two_pi = 6.283185307179586476925286766559L;
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        for (int64_t c = 0; c < m; ++c) {
            long double ar = 0.0L, ai = 0.0L;
            for (int64_t j = 0; j < N; ++j) {
                int64_t xi = j - N / 2;
                long double x = (long double)i / (long double)N;
                long double axi = (long double)(xi < 0 ? -xi : xi);
                long double ph = 0.0L;
                if (kind == 0 || kind == 1 || kind == 2) ph = x * (long double)xi;
                if (kind == 1) ph += (2.0L + (long double)s * sinl(two_pi * x)) / 16.0L * axi;
                if (kind == 2) {
                    long double cc = (2.0L + (long double)s * sinl(two_pi * x)) / 16.0L;
                    ph += (2 * i < N) ? cc * axi : -0.5L * cc * axi;
                }
                if (kind == 4) ph = 0.3L * sinl(two_pi * x) + (long double)xi * (long double)xi / (4.0L * (long double)N);
                long double a = 1.0L;
                if (amp) a = 1.0L + 0.25L * sinl(two_pi * x) * cosl(two_pi * (long double)xi / (long double)N);
                long double kr = a * cosl(two_pi * ph), ki = a * sinl(two_pi * ph);
                long double fr = f[2 * (j * m + c)], fi = f[2 * (j * m + c) + 1];
                ar += kr * fr - ki * fi;
                ai += kr * fi + ki * fr;
            }
            g[2 * (r * m + c)] = (double)ar;
            g[2 * (r * m + c) + 1] = (double)ai;
        }
    }
}

/* Entries K(rows[r], cols[c]) (complex interleaved), for structural tests. */
void oracle_entries(int kind, double s, int amp, int64_t N, const int64_t* rows, int64_t nrows,
                    const int64_t* cols, int64_t ncols, double* out)
{
    for (int64_t r = 0; r < nrows; ++r)
        for (int64_t c = 0; c < ncols; ++c) {
            double th = TWO_PI * phase_frac(kind, s, N, rows[r], cols[c]);
            double a = amplitude(amp, N, rows[r], cols[c]);
            out[2 * (r * ncols + c)] = a * cos(th);
            out[2 * (r * ncols + c) + 1] = a * sin(th);
        }
}

/* out[k] = exp(sign * 2 pi i Phi(x_{ii[k]}, xi_{jj[k]})) for index pairs (ii[k], jj[k]) */
void oracle_expphase(int kind, double s, int64_t N, const int64_t* ii, const int64_t* jj,
                     int64_t n, int sign, double* out)
{
    for (int64_t k = 0; k < n; ++k) {
        double th = TWO_PI * phase_frac(kind, s, N, ii[k], jj[k]);
        out[2 * k] = cos(th);
        out[2 * k + 1] = (sign < 0 ? -1.0 : 1.0) * sin(th);
    }
}

/* out[k] = alpha(x_{ii[k]}, xi_{jj[k]}) (real amplitudes of the built-in kinds) */
void oracle_amplitude(int amp, int64_t N, const int64_t* ii, const int64_t* jj, int64_t n, double* out)
{
    for (int64_t k = 0; k < n; ++k) out[k] = amplitude(amp, N, ii[k], jj[k]);
}

/* the host threads of the oracle's parallel loops from now on, for calls made from this thread
   (a launcher that pins each process to one thread still lets the timed baseline use all cores) */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
