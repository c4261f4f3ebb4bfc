/*
 * pt_oracle.c -- FP64 CPU oracle for the transit-model hot path of
 * Parviainen (2015), "PyTransit: fast and easy exoplanet transit modelling
 * in Python".
 *
 * TEST INFRASTRUCTURE.  This is the plain, slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * Everything is FP64.  Each function names the passage it follows:
 *   - Sec. 2.2.1, Eq. (ma_model): quadratic Mandel-Agol flux from
 *     lambda_e, lambda_d, eta_d.  Those three functions are not printed in
 *     the paper; they are restated here from Mandel & Agol (2002), Table 1
 *     and the equations it references (the paper defers to that source).
 *   - Sec. 2.1.1 Eqs. (gimenez_flux, gimenez_alpha, gimenez), Sec. 2.1.2
 *     Eq. (ld_general), Sec. 2.1.3 (C_n), Sec. 2.1.4 (A_{n,j} and the Jacobi
 *     recursion): the Gimenez series model.
 *   - Sec. 3.2: exposure supersampling.
 *   - Sec. 2.2.3: interpolation tables of the Mandel-Agol terms.
 *   - Sec. 3.3: the Gimenez model interpolated in z.
 *   - Sec. 3.5: per-passband radius ratios through the k^2 / k_hat^2 scaling.
 *   - Sec. 1: circular orbits and eccentric orbits solved with Newton's
 *     method (the paper names the solver but prints no formula).
 *   - Carlson (1995, Numer. Algorithms 10, 13): symmetric elliptic integrals
 *     by the duplication theorem, iterated until the arguments agree to
 *     1e-10 relative, where the remainder is below FP64 resolution.
 *
 * Readings of points where the paper is silent (all listed in the design
 * notes of the repository):
 *   - Pi(n,k) = int_0^{pi/2} dtheta / ((1 - n sin^2) sqrt(1 - k^2 sin^2)).
 *   - lambda_d as in Mandel & Agol, with the +2/3 Theta(k - z) term added in
 *     the flux (Eq. ma_model omits it); eps_d in Eq. (ma_model) is eta_d.
 *   - G_j(p,q;x) = 2F1(-j, p+j; q; x); the series keeps j = 0 .. n_j-1.
 *   - t0 is the time of inferior conjunction (true anomaly pi/2 - omega);
 *     a point behind the star gets z = PTO_Z_BEHIND.
 *   - Supersamples sit at t + t_exp ((s + 1/2)/n_ss - 1/2), unweighted mean.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PTO_PI 3.14159265358979323846

/* Threads of an OpenMP loop: n_threads if positive, else the default. */
#ifdef _OPENMP
static int pto_nthreads(int n_threads) { return n_threads > 0 ? n_threads : omp_get_max_threads(); }
#endif
#define PTO_Z_BEHIND 1.0e30
#define PTO_CARLSON_TOL 1e-10

/* ------------------------------------------------------------------------
 * Carlson symmetric elliptic integrals (Carlson 1995), duplication theorem:
 *   R_F(x,y,z)   = R_F(x',y',z'),                     x' = (x + lam)/4
 *   R_D(x,y,z)   = R_D(x',y',z')/4 + 3 / (sqrt(z) (z + lam))
 *   R_J(x,y,z,p) = R_J(x',y',z',p')/4 + 6 R_C(d^2, d^2 + (p-x)(p-y)(p-z))
 * with lam = sqrt(xy) + sqrt(yz) + sqrt(zx), d = prod (sqrt p + sqrt x_i).
 * Iterate until all arguments agree with their (weighted) mean A to 1e-10;
 * then R(A,...,A) = A^(-1/2) (R_F) or A^(-3/2) (R_D, R_J), whose error is
 * second order in the spread (~1e-20).
 * ---------------------------------------------------------------------- */
double pto_rc(double x, double y)
{
    /* R_C(x,y) = (1/2) int_0^inf (t+x)^(-1/2) (t+y)^(-1) dt, x >= 0, y > 0 */
    if (y > x) return atan(sqrt((y - x) / x)) / sqrt(y - x);
    if (y < x) return atanh(sqrt((x - y) / x)) / sqrt(x - y);
    return 1.0 / sqrt(x);
}

static double max4(double a, double b, double c, double d)
{
    return fmax(fmax(a, b), fmax(c, d));
}

double pto_rf(double x, double y, double z)
{
    for (int it = 0; it < 200; ++it) {
        double A = (x + y + z) / 3.0;
        double dev = max4(fabs(x - A), fabs(y - A), fabs(z - A), 0.0);
        if (dev <= PTO_CARLSON_TOL * A) return 1.0 / sqrt(A);
        double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
        double lam = sx * sy + sy * sz + sz * sx;
        x = 0.25 * (x + lam);
        y = 0.25 * (y + lam);
        z = 0.25 * (z + lam);
    }
    return NAN;
}

double pto_rd(double x, double y, double z)
{
    double sum = 0.0, fac = 1.0;
    for (int it = 0; it < 200; ++it) {
        double A = (x + y + 3.0 * z) / 5.0;
        double dev = max4(fabs(x - A), fabs(y - A), fabs(z - A), 0.0);
        if (dev <= PTO_CARLSON_TOL * A) return sum + fac / (A * sqrt(A));
        double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
        double lam = sx * sy + sy * sz + sz * sx;
        sum += fac * 3.0 / (sz * (z + lam));
        fac *= 0.25;
        x = 0.25 * (x + lam);
        y = 0.25 * (y + lam);
        z = 0.25 * (z + lam);
    }
    return NAN;
}

double pto_rj(double x, double y, double z, double p)
{
    double sum = 0.0, fac = 1.0;
    for (int it = 0; it < 200; ++it) {
        double A = (x + y + z + 2.0 * p) / 5.0;
        double dev = max4(fabs(x - A), fabs(y - A), fabs(z - A), fabs(p - A));
        if (dev <= PTO_CARLSON_TOL * A) return sum + fac / (A * sqrt(A));
        double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z), sp = sqrt(p);
        double lam = sx * sy + sy * sz + sz * sx;
        double d = (sp + sx) * (sp + sy) * (sp + sz);
        sum += fac * 6.0 * pto_rc(d * d, d * d + (p - x) * (p - y) * (p - z));
        fac *= 0.25;
        x = 0.25 * (x + lam);
        y = 0.25 * (y + lam);
        z = 0.25 * (z + lam);
        p = 0.25 * (p + lam);
    }
    return NAN;
}

/* Complete elliptic integrals of parameter m = k^2, passed together with its
 * complement mc = 1 - m (callers form mc from factored geometry so that it
 * keeps full relative precision near m -> 1). */
double pto_ellk(double mc) { return pto_rf(0.0, mc, 1.0); }

double pto_elle(double m, double mc)
{
    return pto_rf(0.0, mc, 1.0) - m / 3.0 * pto_rd(0.0, mc, 1.0);
}

/* Pi(n | m) = int_0^{pi/2} dth / ((1 - n sin^2 th) sqrt(1 - m sin^2 th)),
 * for n < 1, written through rho = 1 - n > 0 as
 *   int (cos^2 + sin^2) / ((cos^2 + rho sin^2) sqrt(cos^2 + mc sin^2))
 * and each half as a positive R_J (cot^2 substitution, then the
 * complementary angle and homogeneity for the cos^2 half):
 *   = R_J(0, 1/mc, 1, 1/rho) / (3 rho sqrt(mc)) + R_J(0, mc, 1, rho) / 3.
 * Both terms are positive, so there is no cancellation when n -> -inf
 * (the z -> k neighbourhood of Mandel & Agol's lambda_1 and lambda_2). */
double pto_ellpi(double n, double mc)
{
    double rho = 1.0 - n;
    return pto_rj(0.0, 1.0 / mc, 1.0, 1.0 / rho) / (3.0 * rho * sqrt(mc)) +
           pto_rj(0.0, mc, 1.0, rho) / 3.0;
}

/* ------------------------------------------------------------------------
 * Mandel & Agol (2002) quadratic-law terms (Sec. 2.2.1, Eq. ma_model).
 * ---------------------------------------------------------------------- */

/* Geometry of the partial overlap: the triangle with sides 1 (star radius),
 * p (planet radius) and z (centre distance).  kap1 and kap0 are its angles
 * at the star and planet centres (half-angles of the chord through the two
 * intersection points).  The law of cosines gives their cosines and the
 * triangle area A their sines (sin kap1 = 2A/z, sin kap0 = 2A/(pz)); A comes
 * from Heron's formula in the factored form
 *   16 A^2 = (1 - (z-p)^2) ((z+p)^2 - 1) = 4 z^2 - (1 + z^2 - p^2)^2,
 * and atan2 keeps full precision at the contact points z = 1 -+ p, where an
 * acos of the rounded cosine would lose half the digits. */
static void overlap_geometry(double p, double z, double *kap0, double *kap1, double *four_a)
{
    double d = (z - 1.0) + p;                         /* z + p - 1 */
    double oma = (1.0 - z + p) * (1.0 + z - p);       /* 1 - (z-p)^2 */
    double bm1 = d * (1.0 + z + p);                   /* (z+p)^2 - 1 */
    double fa = sqrt(fmax(0.0, oma * bm1));
    *four_a = fa;
    *kap1 = atan2(fa, 1.0 - p * p + z * z);
    *kap0 = atan2(fa, p * p + z * z - 1.0);
}

/* lambda_e: fraction of a uniform unit disk covered by a disk of radius p at
 * centre distance z (the lens area over pi):
 *   (p^2 kap0 + kap1 - sqrt(4 z^2 - (1 + z^2 - p^2)^2) / 2) / pi. */
double pto_lambda_e(double p, double z)
{
    z = fabs(z);
    if (p <= 0.0 || z >= 1.0 + p) return 0.0;
    if (p >= 1.0 && z <= p - 1.0) return 1.0;
    if ((z - 1.0) + p <= 0.0) return p * p;
    double kap0, kap1, fa;
    overlap_geometry(p, z, &kap0, &kap1, &fa);
    return (p * p * kap0 + kap1 - 0.5 * fa) / PTO_PI;
}

/* out[0] = lambda_e, out[1] = lambda_d (without the 2/3 Theta(p-z) term),
 * out[2] = eta_d.  Case numbers are those of Mandel & Agol (2002) Table 1;
 * equality tests are exact, as in that table. */
void pto_ma_terms(double p, double z, double *out)
{
    const double pi = PTO_PI;
    z = fabs(z);
    out[0] = out[1] = out[2] = 0.0;
    if (p <= 0.0 || z >= 1.0 + p) return;              /* case 1 */
    if (p >= 1.0 && z <= p - 1.0) {                    /* case 11: star covered */
        out[0] = 1.0; out[1] = 0.0; out[2] = 0.5;
        return;
    }
    out[0] = pto_lambda_e(p, z);

    /* q and the Pi parameters are formed from differences taken once, so
     * that they keep their relative precision as z -> p (a -> 0):
     * q = p^2 - z^2 = (p - z)(p + z), a - b = -4zp, a - 1 = -(1 - a). */
    double a = (z - p) * (z - p), b = (z + p) * (z + p), q = (p - z) * (p + z);
    /* d = z + p - 1 decides inside (d < 0), contact with the limb (d == 0)
     * and partial (d > 0); 1 - b and b - 1 are formed from it so that the
     * branch and the sign of the elliptic parameter always agree. */
    double d = (z - 1.0) + p;
    double oma = (1.0 - z + p) * (1.0 + z - p);   /* 1 - a */
    double omb = -d * (1.0 + z + p);              /* 1 - b */
    double bm1 = d * (1.0 + z + p);               /* b - 1 */
    double eta2 = 0.5 * p * p * (p * p + 2.0 * z * z);
    double ld, ed;

    if (z == 0.0) {                                    /* case 10: lambda_6 */
        ld = -2.0 / 3.0 * pow(1.0 - p * p, 1.5);
        ed = eta2;
    } else if (p == 0.5 && z == 0.5) {                 /* case 6 */
        ld = 1.0 / 3.0 - 4.0 / (9.0 * pi);
        ed = 3.0 / 32.0;
    } else if (z == p) {
        if (p < 0.5) {                                 /* case 5: lambda_4, modulus 2p */
            double m = 4.0 * p * p, mc = (1.0 - 2.0 * p) * (1.0 + 2.0 * p);
            ld = 1.0 / 3.0 + 2.0 / (9.0 * pi) *
                 (4.0 * (2.0 * p * p - 1.0) * pto_elle(m, mc) + (1.0 - 4.0 * p * p) * pto_ellk(mc));
            ed = eta2;
        } else {                                       /* case 7: lambda_3, modulus 1/(2p) */
            double m = 1.0 / (4.0 * p * p), mc = (2.0 * p - 1.0) * (2.0 * p + 1.0) / (4.0 * p * p);
            ld = 1.0 / 3.0 + 16.0 * p / (9.0 * pi) * (2.0 * p * p - 1.0) * pto_elle(m, mc) -
                 (1.0 - 4.0 * p * p) * (3.0 - 8.0 * p * p) / (9.0 * pi * p) * pto_ellk(mc);
            double kap0, kap1, fa;
            overlap_geometry(p, z, &kap0, &kap1, &fa);
            ed = (kap1 + 2.0 * eta2 * kap0 - 0.25 * (1.0 + 5.0 * p * p + z * z) * fa) / (2.0 * pi);
        }
    } else if (d == 0.0) {                             /* case 4: lambda_5, z = 1 - p */
        ld = 2.0 / (3.0 * pi) * acos(1.0 - 2.0 * p) -
             4.0 / (9.0 * pi) * (3.0 + 2.0 * p - 8.0 * p * p) * sqrt(p * (1.0 - p)) -
             (p > 0.5 ? 2.0 / 3.0 : 0.0);
        ed = eta2;
    } else if (d < 0.0) {                              /* cases 3, 9: lambda_2 */
        double m = 4.0 * z * p / oma, mc = omb / oma;
        double K = pto_ellk(mc), E = pto_elle(m, mc), P = pto_ellpi(-4.0 * z * p / a, mc);
        ld = 2.0 / (9.0 * pi * sqrt(oma)) *
             ((1.0 - 5.0 * z * z + p * p + q * q) * K + oma * (z * z + 7.0 * p * p - 4.0) * E - 3.0 * q / a * P);
        ed = eta2;
    } else {                                           /* cases 2, 8: lambda_1, eta_1 */
        double m = oma / (4.0 * z * p), mc = bm1 / (4.0 * z * p);
        double K = pto_ellk(mc), E = pto_elle(m, mc), P = pto_ellpi(-oma / a, mc);
        ld = 1.0 / (9.0 * pi * sqrt(p * z)) *
             (((1.0 - b) * (2.0 * b + a - 3.0) - 3.0 * q * (b - 2.0)) * K +
              4.0 * p * z * (z * z + 7.0 * p * p - 4.0) * E - 3.0 * q / a * P);
        double kap0, kap1, fa;     /* fa = 4A = sqrt((1 - a)(b - 1)) */
        overlap_geometry(p, z, &kap0, &kap1, &fa);
        ed = (kap1 + 2.0 * eta2 * kap0 - 0.25 * (1.0 + 5.0 * p * p + z * z) * fa) / (2.0 * pi);
    }
    out[1] = ld;
    out[2] = ed;
}

/* Eq. (ma_model) with a = u1, b = u2, c = u1 + 2 u2, eps_d read as eta_d and
 * Mandel & Agol's 2/3 Theta(p - z) term restored. */
double pto_flux_quad(double p, double z, double u1, double u2)
{
    double t[3];
    pto_ma_terms(p, z, t);
    double c = u1 + 2.0 * u2;
    double th = (p > fabs(z)) ? 2.0 / 3.0 : 0.0;
    if (t[0] == 0.0 && t[1] == 0.0 && t[2] == 0.0) return 1.0;
    return 1.0 - ((1.0 - c) * t[0] + c * (t[1] + th) + u2 * t[2]) / (1.0 - u1 / 3.0 - u2 / 6.0);
}

/* ------------------------------------------------------------------------
 * Interpolated Mandel-Agol terms (Sec. 2.2.3).  lambda_e, lambda_d + 2/3
 * Theta(p - z) (continuous in z, unlike lambda_d alone) and eta_d are
 * tabulated on the grid
 *   k_i = k_lo + i (k_hi - k_lo) / (n_k - 1),   i = 0 .. n_k - 1,
 *   z_j = j (1 + k_hi) / (n_z - 1),             j = 0 .. n_z - 1,
 * i.e. z spans [0, 1 + k] for every k of the table, and read back by
 * bilinear interpolation (linear in k, then in z).  Readings: out of transit
 * (z >= 1 + k) the terms are zero, as for the exact model; k outside
 * [k_lo, k_hi] is clamped to the table's range.
 * ---------------------------------------------------------------------- */
void pto_ma_table(double k_lo, double k_hi, int n_k, int n_z, double *tab /* [n_k][n_z][3] */)
{
    for (int i = 0; i < n_k; ++i) {
        double k = k_lo + i * (k_hi - k_lo) / (n_k - 1);
        for (int j = 0; j < n_z; ++j) {
            double z = j * (1.0 + k_hi) / (n_z - 1);
            double t[3];
            pto_ma_terms(k, z, t);
            if (k > z) t[1] += 2.0 / 3.0;
            for (int c = 0; c < 3; ++c) tab[((size_t)i * n_z + j) * 3 + c] = t[c];
        }
    }
}

void pto_ma_interp(const double *tab, double k_lo, double k_hi, int n_k, int n_z, double k, double z,
                   double *out /* [3] */)
{
    out[0] = out[1] = out[2] = 0.0;
    if (!(z < 1.0 + k)) return;
    double fk = (k - k_lo) / ((k_hi - k_lo) / (n_k - 1));
    if (fk < 0.0) fk = 0.0;
    if (fk > n_k - 1) fk = n_k - 1;
    int ik = (int)floor(fk);
    if (ik > n_k - 2) ik = n_k - 2;
    double wk = fk - ik;
    double fz = z / ((1.0 + k_hi) / (n_z - 1));
    if (fz < 0.0) fz = 0.0;
    if (fz > n_z - 1) fz = n_z - 1;
    int iz = (int)floor(fz);
    if (iz > n_z - 2) iz = n_z - 2;
    double wz = fz - iz;
    for (int c = 0; c < 3; ++c) {
        double a = tab[((size_t)ik * n_z + iz) * 3 + c], b = tab[((size_t)ik * n_z + iz + 1) * 3 + c];
        double d = tab[((size_t)(ik + 1) * n_z + iz) * 3 + c], e = tab[((size_t)(ik + 1) * n_z + iz + 1) * 3 + c];
        out[c] = (1.0 - wk) * ((1.0 - wz) * a + wz * b) + wk * ((1.0 - wz) * d + wz * e);
    }
}

/* Eq. (ma_model) from interpolated terms (the Theta term is in out[1]). */
double pto_flux_quad_interp(const double *tab, double k_lo, double k_hi, int n_k, int n_z, double p, double z,
                            double u1, double u2)
{
    double t[3];
    pto_ma_interp(tab, k_lo, k_hi, n_k, n_z, p, z, t);
    if (t[0] == 0.0 && t[1] == 0.0 && t[2] == 0.0) return 1.0;
    double c = u1 + 2.0 * u2;
    return 1.0 - ((1.0 - c) * t[0] + c * t[1] + u2 * t[2]) / (1.0 - u1 / 3.0 - u2 / 6.0);
}

/* ------------------------------------------------------------------------
 * Gimenez (2006) series, Sec. 2.1.
 * ---------------------------------------------------------------------- */

/* G_j(p,q;x) = 2F1(-j, p+j; q; x) for j = 0..n-1 by the Jacobi three-term
 * recurrence (Sec. 2.1.4).  With s = 2j + p:
 *   2(j+p)(s-1)(q+j) G_{j+1} =
 *       s[(s+1)(s-1)(1-2x) + (q-1)^2 - (p-q)^2] G_j - 2j(j+p-q)(s+1) G_{j-1},
 * the standard recurrence of P_j^{(q-1,p-q)}(1-2x) rescaled by j!/(q)_j. */
void pto_jacobi_g(int n, double p, double q, double x, double *g)
{
    if (n <= 0) return;
    g[0] = 1.0;
    if (n == 1) return;
    g[1] = 1.0 - (p + 1.0) * x / q;
    for (int j = 1; j + 1 < n; ++j) {
        double s = 2.0 * j + p;
        double j1 = s * ((s + 1.0) * (s - 1.0) + (q - 1.0) * (q - 1.0) - (p - q) * (p - q));
        double j2 = -2.0 * s * (s + 1.0) * (s - 1.0);
        double j3 = -2.0 * j * (j + p - q) * (s + 1.0);
        double j4 = 2.0 * (j + p) * (s - 1.0) * (q + j);
        g[j + 1] = ((j1 + j2 * x) * g[j] + j3 * g[j - 1]) / j4;
    }
}

/* Eq. (gimemez_a): A_{n,j} = (-1)^j (2j+nu+2) Gamma(nu+j+1) / (nu Gamma(nu+1) Gamma(j+2)). */
double pto_gimenez_a(int n, int j)
{
    double nu = 0.5 * (n + 2);
    double sgn = (j % 2) ? -1.0 : 1.0;
    return sgn * (2.0 * j + nu + 2.0) / nu * exp(lgamma(nu + j + 1.0) - lgamma(nu + 1.0) - lgamma(j + 2.0));
}

/* Eq. (gimenez): alpha_n(b,c) for n = 0..N with b = k/(1+k), c = z/(1+k),
 * series truncated to n_j terms. */
void pto_gimenez_alpha(int N, int n_j, double k, double z, double *alpha)
{
    z = fabs(z);
    for (int n = 0; n <= N; ++n) alpha[n] = 0.0;
    if (k <= 0.0 || z >= 1.0 + k || n_j <= 0) return;
    double b = k / (1.0 + k), c = z / (1.0 + k);
    double *g1 = (double *)malloc(sizeof(double) * (size_t)n_j);
    double *g2 = (double *)malloc(sizeof(double) * (size_t)n_j);
    for (int n = 0; n <= N; ++n) {
        double nu = 0.5 * (n + 2);
        pto_jacobi_g(n_j, nu + 2.0, nu + 1.0, 1.0 - b, g1);
        pto_jacobi_g(n_j, nu + 2.0, 1.0, c * c, g2);
        double s = 0.0;
        for (int j = 0; j < n_j; ++j) s += pto_gimenez_a(n, j) * g1[j] * g1[j] * g2[j];
        alpha[n] = b * b * pow(1.0 - c * c, nu + 1.0) * s;
    }
    free(g1);
    free(g2);
}

/* Eqs. (gimenez_flux, gimenez_alpha) with the C_n of Sec. 2.1.3;
 * u[0..N-1] holds u_1..u_N of Eq. (ld_general). */
double pto_flux_gimenez(int N, int n_j, double k, double z, const double *u)
{
    double alpha[64];
    if (N > 63) return NAN;
    pto_gimenez_alpha(N, n_j, k, z, alpha);
    double su = 0.0, sd = 0.0;
    for (int n = 1; n <= N; ++n) {
        su += u[n - 1];
        sd += n * u[n - 1] / (n + 2.0);
    }
    double D = 1.0 - sd;
    double a = (1.0 - su) / D * alpha[0];
    for (int n = 1; n <= N; ++n) a += u[n - 1] / D * alpha[n];
    return 1.0 - a;
}

/* ------------------------------------------------------------------------
 * The occulted flux from its definition (the quantity both models compute,
 * Sec. 2.1.1 Eq. gimenez_flux and Sec. 2.2.1: the light of the limb-darkened
 * stellar disk of unit radius blocked by an opaque disk of radius k whose
 * centre is z away), written as a 1-D integral over rings of radius r:
 *   blocked = int_0^1 w(r) r theta(r) dr,
 * theta(r) = the angle of the ring that lies inside the planet's disk:
 *   2 pi if r <= k - z;  0 if r >= z + k or r <= z - k;
 *   2 acos((r^2 + z^2 - k^2) / (2 r z)) otherwise.
 * With w = mu^n (mu = sqrt(1 - r^2)) this is pi alpha_n (the mu^n-weighted
 * covered area of Eq. gimenez_alpha); with w = I(mu) of Eq. ld_general it
 * gives f = 1 - blocked / F_tot, F_tot = int_0^1 I 2 pi r dr.  The series of
 * Eq. gimenez converges to these values as N_J grows, so they measure its
 * truncation error (the quantity of the paper's Fig. 1).
 *
 * Quadrature: tanh-sinh (Takahasi & Mori 1974) on each piece between the
 * kinks |z - k|, z + k and 1, where the integrands have square-root end
 * point behaviour; the step is halved until two levels agree to 1e-15.  The
 * distance of a node to the nearer end is formed directly, so nodes that
 * crowd an end point keep their accuracy.
 * ---------------------------------------------------------------------- */
typedef struct ring_weight {
    int N;             /* mu^N (u == NULL) or the general law with N coefficients */
    const double *u;   /* u_1..u_N of Eq. ld_general, or NULL */
    double k, z;
} ring_weight;

/* 2 acos(c) for the ring at radius r, with 1 - c and 1 + c in factored form. */
static double ring_theta(double r, double k, double z)
{
    if (r <= k - z) return 2.0 * PTO_PI;
    if (r >= z + k || r <= z - k) return 0.0;
    double omc = (k - r + z) * (k + r - z) / (2.0 * r * z);
    double opc = (r + z - k) * (r + z + k) / (2.0 * r * z);
    if (omc < 0.0) omc = 0.0;
    if (opc < 0.0) opc = 0.0;
    return 4.0 * atan2(sqrt(omc), sqrt(opc));
}

/* w(r) r theta(r); one_m_r = 1 - r, supplied separately for accuracy near r = 1. */
static double ring_integrand(const ring_weight *W, double r, double one_m_r, int with_theta)
{
    double mu2 = one_m_r * (1.0 + r);
    double mu = sqrt(mu2 > 0.0 ? mu2 : 0.0);
    double w;
    if (!W->u) {
        w = pow(mu, (double)W->N);
    } else {
        w = 1.0;
        double mun = 1.0;
        for (int n = 1; n <= W->N; ++n) {
            mun *= mu;
            w -= W->u[n - 1] * (1.0 - mun);
        }
    }
    double th = with_theta ? ring_theta(r, W->k, W->z) : 2.0 * PTO_PI;
    return w * r * th;
}

static double tanh_sinh(const ring_weight *W, double a, double b, int with_theta)
{
    const double T = 4.0;
    double half = 0.5 * (b - a), mid = 0.5 * (a + b);
    double h = 0.5, sum = 0.0, prev = 0.0;
    for (int level = 0; level <= 12; ++level) {
        /* level 0 takes every node k h; later levels only the new odd nodes */
        double step = (level == 0) ? h : 2.0 * h;
        double start = (level == 0) ? 0.0 : h;
        double add = 0.0;
        for (double t = start; t <= T; t += step) {
            double u = 0.5 * PTO_PI * sinh(t);
            double cu = cosh(u);
            double wgt = 0.5 * PTO_PI * cosh(t) / (cu * cu);
            double dist = (b - a) / (1.0 + exp(2.0 * u));   /* distance to the nearer end */
            for (int side = (t == 0.0) ? 1 : 0; side < 2; ++side) {
                double r, omr;
                if (side == 0) {          /* node near a */
                    r = a + dist;
                    omr = 1.0 - r;
                } else {                  /* node near b (t = 0: the midpoint) */
                    r = (t == 0.0) ? mid : b - dist;
                    omr = (b == 1.0 && t != 0.0) ? dist : 1.0 - r;
                }
                add += wgt * ring_integrand(W, r, omr, with_theta);
            }
        }
        sum = (level == 0) ? add : sum + add;
        double val = half * h * sum;
        if (level >= 3 && fabs(val - prev) <= 1e-15 * (fabs(val) + 1e-300)) return val;
        prev = val;
        h *= 0.5;
    }
    return prev;
}

static double ring_blocked(const ring_weight *W)
{
    double k = W->k, z = fabs(W->z);
    ring_weight V = *W;
    V.z = z;
    double pts[4];
    int np = 0;
    pts[np++] = 0.0;
    double c1 = fabs(z - k), c2 = z + k;
    if (c1 > 0.0 && c1 < 1.0) pts[np++] = c1;
    if (c2 > 0.0 && c2 < 1.0 && c2 != c1) pts[np++] = c2;
    pts[np++] = 1.0;
    if (np == 4 && pts[1] > pts[2]) {
        double s = pts[1];
        pts[1] = pts[2];
        pts[2] = s;
    }
    double tot = 0.0;
    for (int i = 0; i + 1 < np; ++i)
        if (pts[i + 1] > pts[i]) tot += tanh_sinh(&V, pts[i], pts[i + 1], 1);
    return tot;
}

/* alpha_n(k, z) = (1/pi) x (mu^n-weighted area covered), from the definition. */
double pto_ring_alpha(int n, double k, double z)
{
    if (k <= 0.0 || fabs(z) >= 1.0 + k) return 0.0;
    ring_weight W = {n, NULL, k, z};
    return ring_blocked(&W) / PTO_PI;
}

/* f(k, z) for the general law u_1..u_N (Eq. ld_general), from the definition:
 * 1 - blocked light / total light, both integrated over rings. */
double pto_ring_flux(int N, const double *u, double k, double z)
{
    if (k <= 0.0 || fabs(z) >= 1.0 + k) return 1.0;
    ring_weight W = {N, u, k, z};
    double tot = tanh_sinh(&W, 0.0, 1.0, 0);
    return 1.0 - ring_blocked(&W) / tot;
}

/* ------------------------------------------------------------------------
 * Orbits (Sec. 1: circular orbits; eccentric orbits by Newton's method).
 * ---------------------------------------------------------------------- */

/* Circular orbit: phase phi = 2 pi (t - t0)/P from conjunction,
 * z = a sqrt(sin^2 phi + cos^2 i cos^2 phi); behind the star if cos phi <= 0. */
double pto_z_circ(double t, double t0, double P, double a, double inc)
{
    double x = (t - t0) / P;
    x -= rint(x);
    double ph = 2.0 * PTO_PI * x;
    double cp = cos(ph), sp = sin(ph), ci = cos(inc);
    if (cp <= 0.0) return PTO_Z_BEHIND;
    return a * sqrt(sp * sp + ci * ci * cp * cp);
}

/* Kepler's equation E - e sin E = M by Newton's method; returns iterations
 * used, or -1 if |dE| did not fall below tol within max_iter.  M is first
 * reduced to [0, 2 pi); the start E = M (e < 0.8) or E = pi (the inflection
 * point of E - e sin E, from which Newton's iterates are monotone) follows
 * the usual practice.  The returned E is shifted back by the same multiple
 * of 2 pi. */
int pto_kepler_newton(double M, double e, int max_iter, double tol, double *E_out)
{
    double shift = 2.0 * PTO_PI * floor(M / (2.0 * PTO_PI));
    double Mr = M - shift;
    double E = (e < 0.8) ? Mr : PTO_PI;
    for (int it = 1; it <= max_iter; ++it) {
        double d = (E - e * sin(E) - Mr) / (1.0 - e * cos(E));
        E -= d;
        if (fabs(d) < tol) {
            *E_out = E + shift;
            return it;
        }
    }
    *E_out = E + shift;
    return -1;
}

/* Eccentric orbit: mean anomaly M = M_tr + 2 pi (t - t0)/P where M_tr is the
 * mean anomaly at true anomaly f_tr = pi/2 - omega; Newton for E; true anomaly
 * f; r = a (1 - e cos E); z = r sqrt(cos^2(w+f) + sin^2(w+f) cos^2 i);
 * behind the star if sin(w+f) <= 0.  *status is set to -1 on non-convergence. */
double pto_z_ecc(double t, double t0, double P, double a, double inc, double e, double w,
                 int max_iter, double tol, int *status)
{
    double ftr = 0.5 * PTO_PI - w;
    double Etr = 2.0 * atan2(sqrt(1.0 - e) * sin(0.5 * ftr), sqrt(1.0 + e) * cos(0.5 * ftr));
    double Mtr = Etr - e * sin(Etr);
    double x = (t - t0) / P;
    x -= rint(x);
    double M = Mtr + 2.0 * PTO_PI * x;
    double E;
    int it = pto_kepler_newton(M, e, max_iter, tol, &E);
    if (status) *status = (it < 0) ? -1 : 0;
    double f = 2.0 * atan2(sqrt(1.0 + e) * sin(0.5 * E), sqrt(1.0 - e) * cos(0.5 * E));
    double r = a * (1.0 - e * cos(E));
    double s = sin(w + f), c = cos(w + f), ci = cos(inc);
    if (s <= 0.0) return PTO_Z_BEHIND;
    return r * sqrt(c * c + s * s * ci * ci);
}

/* Impact parameter to inclination (Winn 2010 convention):
 * b = a cos i (1 - e^2) / (1 + e sin w). */
double pto_inc_from_b(double b, double a, double e, double w)
{
    return acos(b / a * (1.0 + e * sin(w)) / (1.0 - e * e));
}

/* ------------------------------------------------------------------------
 * Batched drivers: flux cube [v][b][t] with supersampling (Sec. 3.2) and the
 * multi-passband evaluation of Secs. 2.1.3 and 2.2.2 (here simply evaluated
 * per passband: the oracle does no factoring of its own).
 * e == NULL selects the circular orbit.  k is [v] or, if k_per_band, [v][b].
 * ---------------------------------------------------------------------- */
static double orbit_z(const double *t0, const double *P, const double *a, const double *inc,
                      const double *e, const double *w, int v, double tt, int *bad)
{
    if (!e) return pto_z_circ(tt, t0[v], P[v], a[v], inc[v]);
    int st = 0;
    double z = pto_z_ecc(tt, t0[v], P[v], a[v], inc[v], e[v], w[v], 50, 1e-14, &st);
    if (st) *bad = 1;
    return z;
}

int pto_z_batch(const double *t, int n_t, const double *t0, const double *P, const double *a,
                const double *inc, const double *e, const double *w, int n_v, int n_ss, double t_exp,
                double *z /* [v][t*n_ss + s] */)
{
    int nbad = 0;
    for (int v = 0; v < n_v; ++v)
        for (int i = 0; i < n_t; ++i)
            for (int s = 0; s < n_ss; ++s) {
                double tt = t[i] + t_exp * ((s + 0.5) / n_ss - 0.5);
                int bad = 0;
                z[((size_t)v * n_t + i) * n_ss + s] = orbit_z(t0, P, a, inc, e, w, v, tt, &bad);
                nbad += bad;
            }
    return nbad;
}

int pto_lc_ma(const double *t, int n_t, const double *t0, const double *P, const double *a,
              const double *inc, const double *e, const double *w, int n_v, const double *k,
              int k_per_band, const double *ld /* [v][b][2] */, int n_b, int n_ss, double t_exp,
              double *flux /* [v][b][t] */, int n_threads)
{
    int nbad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nbad) num_threads(pto_nthreads(n_threads))
#endif
    for (int v = 0; v < n_v; ++v) {
        for (int i = 0; i < n_t; ++i) {
            for (int b = 0; b < n_b; ++b) flux[((size_t)v * n_b + b) * n_t + i] = 0.0;
            for (int s = 0; s < n_ss; ++s) {
                double tt = t[i] + t_exp * ((s + 0.5) / n_ss - 0.5);
                int bad = 0;
                double z = orbit_z(t0, P, a, inc, e, w, v, tt, &bad);
                nbad += bad;
                for (int b = 0; b < n_b; ++b) {
                    double kk = k_per_band ? k[(size_t)v * n_b + b] : k[v];
                    const double *u = ld + ((size_t)v * n_b + b) * 2;
                    flux[((size_t)v * n_b + b) * n_t + i] += pto_flux_quad(kk, z, u[0], u[1]);
                }
            }
            for (int b = 0; b < n_b; ++b) flux[((size_t)v * n_b + b) * n_t + i] /= n_ss;
        }
    }
    return nbad;
}

/* Per-passband radius ratios through the approximation of Sec. 3.5: the
 * model is evaluated once with the mean radius ratio k_hat of the vector's
 * passbands, and each passband's transit depth 1 - f is scaled by
 * k_b^2 / k_hat^2.  Reading: the factor multiplies the depth (the flux
 * deficit), k_hat is the arithmetic mean over the passbands. */
int pto_lc_ma_khat(const double *t, int n_t, const double *t0, const double *P, const double *a,
                   const double *inc, const double *e, const double *w, int n_v, const double *k /* [v][b] */,
                   const double *ld /* [v][b][2] */, int n_b, int n_ss, double t_exp, double *flux /* [v][b][t] */,
                   int n_threads)
{
    int nbad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nbad) num_threads(pto_nthreads(n_threads))
#endif
    for (int v = 0; v < n_v; ++v) {
        double kh = 0.0;
        for (int b = 0; b < n_b; ++b) kh += k[(size_t)v * n_b + b];
        kh /= n_b;
        for (int i = 0; i < n_t; ++i) {
            for (int b = 0; b < n_b; ++b) flux[((size_t)v * n_b + b) * n_t + i] = 0.0;
            for (int s = 0; s < n_ss; ++s) {
                double tt = t[i] + t_exp * ((s + 0.5) / n_ss - 0.5);
                int bad = 0;
                double z = orbit_z(t0, P, a, inc, e, w, v, tt, &bad);
                nbad += bad;
                for (int b = 0; b < n_b; ++b) {
                    const double *u = ld + ((size_t)v * n_b + b) * 2;
                    flux[((size_t)v * n_b + b) * n_t + i] += pto_flux_quad(kh, z, u[0], u[1]);
                }
            }
            for (int b = 0; b < n_b; ++b) {
                double kb = k[(size_t)v * n_b + b];
                double f = flux[((size_t)v * n_b + b) * n_t + i] / n_ss;
                flux[((size_t)v * n_b + b) * n_t + i] = 1.0 - (kb * kb) / (kh * kh) * (1.0 - f);
            }
        }
    }
    return nbad;
}

/* pto_lc_ma with the terms read from an interpolation table (Sec. 2.2.3). */
int pto_lc_ma_interp(const double *tab, double k_lo, double k_hi, int n_k, int n_z, const double *t, int n_t,
                     const double *t0, const double *P, const double *a, const double *inc, const double *e,
                     const double *w, int n_v, const double *k, int k_per_band, const double *ld /* [v][b][2] */,
                     int n_b, int n_ss, double t_exp, double *flux /* [v][b][t] */, int n_threads)
{
    int nbad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nbad) num_threads(pto_nthreads(n_threads))
#endif
    for (int v = 0; v < n_v; ++v) {
        for (int i = 0; i < n_t; ++i) {
            for (int b = 0; b < n_b; ++b) flux[((size_t)v * n_b + b) * n_t + i] = 0.0;
            for (int s = 0; s < n_ss; ++s) {
                double tt = t[i] + t_exp * ((s + 0.5) / n_ss - 0.5);
                int bad = 0;
                double z = orbit_z(t0, P, a, inc, e, w, v, tt, &bad);
                nbad += bad;
                for (int b = 0; b < n_b; ++b) {
                    double kk = k_per_band ? k[(size_t)v * n_b + b] : k[v];
                    const double *u = ld + ((size_t)v * n_b + b) * 2;
                    flux[((size_t)v * n_b + b) * n_t + i] +=
                        pto_flux_quad_interp(tab, k_lo, k_hi, n_k, n_z, kk, z, u[0], u[1]);
                }
            }
            for (int b = 0; b < n_b; ++b) flux[((size_t)v * n_b + b) * n_t + i] /= n_ss;
        }
    }
    return nbad;
}

int pto_lc_gimenez(const double *t, int n_t, const double *t0, const double *P, const double *a,
                   const double *inc, const double *e, const double *w, int n_v, const double *k,
                   int k_per_band, const double *ld /* [v][b][N] */, int N, int n_b, int n_j, int n_ss,
                   double t_exp, double *flux /* [v][b][t] */, int n_threads)
{
    int nbad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nbad) num_threads(pto_nthreads(n_threads))
#endif
    for (int v = 0; v < n_v; ++v) {
        for (int i = 0; i < n_t; ++i) {
            for (int b = 0; b < n_b; ++b) flux[((size_t)v * n_b + b) * n_t + i] = 0.0;
            for (int s = 0; s < n_ss; ++s) {
                double tt = t[i] + t_exp * ((s + 0.5) / n_ss - 0.5);
                int bad = 0;
                double z = orbit_z(t0, P, a, inc, e, w, v, tt, &bad);
                nbad += bad;
                for (int b = 0; b < n_b; ++b) {
                    double kk = k_per_band ? k[(size_t)v * n_b + b] : k[v];
                    const double *u = ld + ((size_t)v * n_b + b) * N;
                    flux[((size_t)v * n_b + b) * n_t + i] += pto_flux_gimenez(N, n_j, kk, z, u);
                }
            }
            for (int b = 0; b < n_b; ++b) flux[((size_t)v * n_b + b) * n_t + i] /= n_ss;
        }
    }
    return nbad;
}

/* ------------------------------------------------------------------------
 * Gimenez model interpolated in z (Sec. 3.3).  The series is evaluated on
 * n_in points over z in [0, zb], zb = max(1 - k, 0), and n_edge points over
 * (zb, 1 + k]; light-curve points are read from these values by linear
 * interpolation.  The tabulated values are alpha_0 .. alpha_N (free of limb
 * darkening), so one table serves every passband; the flux is linear in the
 * alpha_n, so this is the same as interpolating each passband's flux.
 * Readings: linear interpolation; nodes
 *   z_i = i zb / (n_in - 1),                 i = 0 .. n_in - 1,
 *   z_{n_in + j} = zb + (j + 1)(1 + k - zb) / n_edge,   j = 0 .. n_edge - 1;
 * out of transit (z >= 1 + k) alpha = 0.
 * ---------------------------------------------------------------------- */
static double zi_node(int i, int n_in, int n_edge, double k)
{
    double zb = (1.0 - k > 0.0) ? 1.0 - k : 0.0;
    if (i < n_in) return i * zb / (n_in - 1);
    return zb + (i - n_in + 1) * (1.0 + k - zb) / n_edge;
}

void pto_gimenez_zi_table(int N, int n_j, double k, int n_in, int n_edge, double *tab /* [n_in+n_edge][N+1] */)
{
    for (int i = 0; i < n_in + n_edge; ++i)
        pto_gimenez_alpha(N, n_j, k, zi_node(i, n_in, n_edge, k), tab + (size_t)i * (N + 1));
}

void pto_gimenez_zi_alpha(int N, int n_in, int n_edge, double k, const double *tab, double z, double *alpha)
{
    z = fabs(z);
    for (int n = 0; n <= N; ++n) alpha[n] = 0.0;
    if (!(z < 1.0 + k)) return;
    double zb = (1.0 - k > 0.0) ? 1.0 - k : 0.0;
    int i0;
    double w;
    if (z <= zb && zb > 0.0) {
        double f = z / (zb / (n_in - 1));
        i0 = (int)floor(f);
        if (i0 > n_in - 2) i0 = n_in - 2;
        w = f - i0;
    } else if (z <= zb) {   /* k >= 1: the first region is the single point z = 0 */
        i0 = 0;
        w = 0.0;
    } else {
        double f = (z - zb) / ((1.0 + k - zb) / n_edge);   /* 0 at node n_in - 1 */
        int c = (int)floor(f);
        if (c > n_edge - 1) c = n_edge - 1;
        i0 = n_in - 1 + c;
        w = f - c;
    }
    for (int n = 0; n <= N; ++n)
        alpha[n] = (1.0 - w) * tab[(size_t)i0 * (N + 1) + n] + w * tab[(size_t)(i0 + 1) * (N + 1) + n];
}

int pto_lc_gimenez_zi(const double *t, int n_t, const double *t0, const double *P, const double *a,
                      const double *inc, const double *e, const double *w, int n_v, const double *k,
                      int k_per_band, const double *ld /* [v][b][N] */, int N, int n_b, int n_j, int n_in,
                      int n_edge, int n_ss, double t_exp, double *flux /* [v][b][t] */, int n_threads)
{
    int nbad = 0;
    int nz = n_in + n_edge;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nbad) num_threads(pto_nthreads(n_threads))
#endif
    for (int v = 0; v < n_v; ++v) {
        double *tab = (double *)malloc(sizeof(double) * (size_t)nz * (N + 1) * n_b);
        double alpha[64];
        for (int b = 0; b < n_b; ++b) {
            double kk = k_per_band ? k[(size_t)v * n_b + b] : k[v];
            if (b == 0 || k_per_band)
                pto_gimenez_zi_table(N, n_j, kk, n_in, n_edge, tab + (size_t)b * nz * (N + 1));
        }
        for (int i = 0; i < n_t; ++i) {
            for (int b = 0; b < n_b; ++b) flux[((size_t)v * n_b + b) * n_t + i] = 0.0;
            for (int s = 0; s < n_ss; ++s) {
                double tt = t[i] + t_exp * ((s + 0.5) / n_ss - 0.5);
                int bad = 0;
                double z = orbit_z(t0, P, a, inc, e, w, v, tt, &bad);
                nbad += bad;
                for (int b = 0; b < n_b; ++b) {
                    double kk = k_per_band ? k[(size_t)v * n_b + b] : k[v];
                    const double *tb = tab + (size_t)(k_per_band ? b : 0) * nz * (N + 1);
                    pto_gimenez_zi_alpha(N, n_in, n_edge, kk, tb, z, alpha);
                    const double *u = ld + ((size_t)v * n_b + b) * N;
                    double su = 0.0, sd = 0.0;
                    for (int n = 1; n <= N; ++n) {
                        su += u[n - 1];
                        sd += n * u[n - 1] / (n + 2.0);
                    }
                    double D = 1.0 - sd;
                    double al = (1.0 - su) / D * alpha[0];
                    for (int n = 1; n <= N; ++n) al += u[n - 1] / D * alpha[n];
                    flux[((size_t)v * n_b + b) * n_t + i] += 1.0 - al;
                }
            }
            for (int b = 0; b < n_b; ++b) flux[((size_t)v * n_b + b) * n_t + i] /= n_ss;
        }
        free(tab);
    }
    return nbad;
}


/* Sum of squared residuals per (vector, passband): sum_t w (y - f)^2, the
 * likelihood reduction the paper moves onto the device (Sec. 3.4).
 * y and wt are [b][t]; wt == NULL means unit weights. */
void pto_ssr(const double *flux, const double *y, const double *wt, int n_v, int n_b, int n_t,
             double *ssr)
{
    for (int v = 0; v < n_v; ++v)
        for (int b = 0; b < n_b; ++b) {
            double s = 0.0;
            for (int i = 0; i < n_t; ++i) {
                double r = y[(size_t)b * n_t + i] - flux[((size_t)v * n_b + b) * n_t + i];
                s += (wt ? wt[(size_t)b * n_t + i] : 1.0) * r * r;
            }
            ssr[(size_t)v * n_b + b] = s;
        }
}

/* pto_ma_terms at n points (k[i], z[i]); out is [n][3].  OpenMP over points. */
void pto_ma_terms_batch(long n, const double *k, const double *z, double *out, int n_threads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(pto_nthreads(n_threads))
#endif
    for (long i = 0; i < n; ++i) pto_ma_terms(k[i], z[i], out + 3 * i);
}

int pto_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}


/* ------------------------------------------------------------------------
 * Gradients (the adjoint's reference).  The paper evaluates no gradients; it
 * cites analytic derivatives of the quadratic model (Pal 2008).  Here they
 * follow from the definition of the occulted flux:
 *   I_g(p, z) = int int_{overlap} g(r) dA,  g in {1, mu, mu^2},  mu = sqrt(1 - r^2),
 *   pi lambda_e = I_1,  pi (lambda_d + 2/3 Theta(p - z)) = I_mu,  pi eta_d = I_1 - I_mu2,
 *   F = 1 - [(1 - u1 - u2) I_1 + (u1 + 2 u2) I_mu - u2 I_mu2] / (pi (1 - u1/3 - u2/6)).
 * Only the planet's edge inside the star moves with p or z (Reynolds
 * transport): with the edge point (z + p cos phi, p sin phi),
 *   dI_g/dp = p int_arc g dphi,   dI_g/dz = p int_arc g cos(phi) dphi,
 * where the arc is the full circle inside the star, or the part of it within
 * kap0 of the direction towards the star centre.  For g = mu the arc
 * integrals are complete elliptic integrals (with m1 = (1-a)/(4zp) on the
 * partial arc, m2 = 4zp/(1-a) on the full circle, a = (z-p)^2).
 * ---------------------------------------------------------------------- */

/* S(m) = int_0^{pi/2} sin^2 cos^2 / sqrt(1 - m sin^2) dth: binomial series of
 * (1 - m s^2)^(-1/2) term by term below m = 1/2 (60 terms, < 1e-20), and
 * ((2-m) E - 2 (1-m) K) / (3 m^2) above, where that difference has no
 * cancellation to speak of. */
static double s2c2_int(double m)
{
    if (m < 0.5) {
        double w[64];   /* w_j = int_0^{pi/2} sin^(2j) = (pi/2) C(2j,j)/4^j */
        w[0] = 0.5 * PTO_PI;
        for (int j = 1; j < 64; ++j) w[j] = w[j - 1] * (2.0 * j - 1.0) / (2.0 * j);
        double c = 1.0, mn = 1.0, s = 0.0;   /* c_n = C(2n,n)/4^n */
        for (int n = 0; n < 60; ++n) {
            s += c * mn * (w[n + 1] - w[n + 2]);
            c *= (2.0 * n + 1.0) / (2.0 * n + 2.0);
            mn *= m;
        }
        return s;
    }
    double mc = 1.0 - m;
    return ((2.0 - m) * pto_elle(m, mc) - 2.0 * mc * pto_ellk(mc)) / (3.0 * m * m);
}

/* d[0..5] = dI_1/dp, dI_1/dz, dI_mu/dp, dI_mu/dz, dI_mu2/dp, dI_mu2/dz. */
void pto_overlap_derivs(double p, double z, double *d)
{
    for (int i = 0; i < 6; ++i) d[i] = 0.0;
    z = fabs(z);
    if (p <= 0.0 || z >= 1.0 + p) return;
    if (p >= 1.0 && z <= p - 1.0) return;        /* star covered: nothing moves */
    double a = (z - p) * (z - p);
    double oma = (1.0 - z + p) * (1.0 + z - p);
    double dd = (z - 1.0) + p;
    double al = 1.0 - z * z - p * p;              /* mu^2 = al + 2 z p cos(psi) on the edge */
    if (dd < 0.0) {                               /* full circle inside the star */
        double m = 4.0 * z * p / oma;
        d[0] = 2.0 * PTO_PI * p;
        d[1] = 0.0;
        d[2] = 4.0 * p * sqrt(oma) * pto_elle(m, 1.0 - m);
        d[3] = -p * 4.0 * sqrt(oma) * m * s2c2_int(m);
        d[4] = p * al * 2.0 * PTO_PI;
        d[5] = -p * 2.0 * z * p * PTO_PI;
        return;
    }
    double fa = sqrt(fmax(0.0, oma * dd * (1.0 + z + p)));
    double kap0 = atan2(fa, p * p + z * z - 1.0);
    double sk = fa / (2.0 * p * z), ck = (p * p + z * z - 1.0) / (2.0 * p * z);
    double m1 = oma / (4.0 * z * p), mc1 = dd * (1.0 + z + p) / (4.0 * z * p);
    double K = pto_ellk(mc1), E = pto_elle(m1, mc1);
    double icos = -2.0 * sk, icos2 = kap0 + sk * ck;   /* arc integrals of cos, cos^2 */
    d[0] = 2.0 * p * kap0;
    d[1] = p * icos;
    d[2] = 8.0 * p * sqrt(z * p) * (E - mc1 * K);
    d[3] = -p * (4.0 / 3.0) * sqrt(4.0 * z * p) * ((2.0 * m1 - 1.0) * E + mc1 * K);
    d[4] = p * (al * 2.0 * kap0 - 2.0 * z * p * icos);
    d[5] = p * (al * icos - 2.0 * z * p * icos2);
}

/* Flux at time t for theta = (t0, P, a, b, e, w, k, u1, u2): the plain
 * composition of the orbit (inclination from b) and Eq. (ma_model),
 * supersampled.  Used as the function the gradient is checked against. */
double pto_flux_theta(double t, const double *th, int n_ss, double t_exp)
{
    double inc = pto_inc_from_b(th[3], th[2], th[4], th[5]);
    double f = 0.0;
    for (int s = 0; s < n_ss; ++s) {
        double tt = t + t_exp * ((s + 0.5) / n_ss - 0.5);
        int st;
        double z = pto_z_ecc(tt, th[0], th[1], th[2], inc, th[4], th[5], 60, 1e-15, &st);
        f += pto_flux_quad(th[6], z, th[7], th[8]);
    }
    return f / n_ss;
}

/* Flux and its gradient with respect to theta at one time (chain rule
 * through z, Kepler's equation and the conjunction anchor), FP64. */
double pto_flux_grad(double t, const double *th, int n_ss, double t_exp, double *g)
{
    const double t0 = th[0], P = th[1], A = th[2], b = th[3], e = th[4], w = th[5];
    const double k = th[6], u1 = th[7], u2 = th[8];
    for (int i = 0; i < 9; ++i) g[i] = 0.0;
    double se = sqrt(1.0 - e * e);
    double sw = sin(w), cw = cos(w);
    double ci = b * (1.0 + e * sw) / (A * (1.0 - e * e));          /* cos i */
    double dci[9] = {0};
    dci[2] = -ci / A;
    dci[3] = (1.0 + e * sw) / (A * (1.0 - e * e));
    dci[4] = b / A * (sw * (1.0 - e * e) + 2.0 * e * (1.0 + e * sw)) / ((1.0 - e * e) * (1.0 - e * e));
    dci[5] = b / A * e * cw / (1.0 - e * e);
    /* conjunction anchor and its derivatives: f_tr = pi/2 - w */
    double ftr = 0.5 * PTO_PI - w;
    double Etr = 2.0 * atan2(sqrt(1.0 - e) * sin(0.5 * ftr), sqrt(1.0 + e) * cos(0.5 * ftr));
    double Mtr = Etr - e * sin(Etr);
    double ecEt = 1.0 - e * cos(Etr);
    double dMtr_dw = -ecEt * ecEt / se;                            /* -dM/df at f_tr */
    double dMtr_de = -ecEt * sin(Etr) / (1.0 - e * e) - sin(Etr);  /* dM/de at fixed f */
    double c0 = 1.0 - u1 - u2, c2 = u1 + 2.0 * u2, D = 1.0 - u1 / 3.0 - u2 / 6.0;
    double fsum = 0.0;
    for (int s = 0; s < n_ss; ++s) {
        double tt = t + t_exp * ((s + 0.5) / n_ss - 0.5);
        double x = (tt - t0) / P;
        double M = Mtr + 2.0 * PTO_PI * (x - rint(x));
        double E;
        pto_kepler_newton(M, e, 60, 1e-15, &E);
        double sE = sin(E), cE = cos(E);
        double X = A * (cE - e), Y = A * se * sE;
        double U = X * cw - Y * sw, V = X * sw + Y * cw;
        if (V <= 0.0) { fsum += 1.0; continue; }
        double z = sqrt(U * U + V * V * ci * ci);
        double I[3], T[3], dI[6];
        pto_ma_terms(k, z, T);
        if (T[0] == 0.0 && T[1] == 0.0 && T[2] == 0.0) { fsum += 1.0; continue; }
        I[0] = PTO_PI * T[0];
        I[1] = PTO_PI * (T[1] + ((k > z) ? 2.0 / 3.0 : 0.0));
        I[2] = PTO_PI * (T[0] - T[2]);
        double N = c0 * I[0] + c2 * I[1] - u2 * I[2];
        fsum += 1.0 - N / (PTO_PI * D);
        pto_overlap_derivs(k, z, dI);
        double dFdk = -(c0 * dI[0] + c2 * dI[2] - u2 * dI[4]) / (PTO_PI * D);
        double dFdz = -(c0 * dI[1] + c2 * dI[3] - u2 * dI[5]) / (PTO_PI * D);
        /* dM/dtheta, then dE = (dM + sin E de) / (1 - e cos E) */
        double dM[9] = {0}, de[9] = {0}, da[9] = {0}, dw[9] = {0};
        dM[0] = -2.0 * PTO_PI / P;
        dM[1] = -2.0 * PTO_PI * (tt - t0) / (P * P);
        dM[4] = dMtr_de;
        dM[5] = dMtr_dw;
        de[4] = 1.0;
        da[2] = 1.0;
        dw[5] = 1.0;
        double gz[9];
        for (int i = 0; i < 6; ++i) {
            double dE = (dM[i] + sE * de[i]) / (1.0 - e * cE);
            double dX = da[i] * (cE - e) - A * sE * dE - A * de[i];
            double dY = da[i] * se * sE + A * se * cE * dE - A * e * sE / se * de[i];
            double dU = dX * cw - dY * sw - V * dw[i];
            double dV = dX * sw + dY * cw + U * dw[i];
            gz[i] = (U * dU + V * ci * ci * dV + V * V * ci * dci[i]) / z;
        }
        for (int i = 0; i < 6; ++i) g[i] += dFdz * gz[i];
        g[6] += dFdk;
        g[7] += -((I[1] - I[0]) / (PTO_PI * D) + N / (3.0 * PTO_PI * D * D));
        g[8] += -((-I[0] + 2.0 * I[1] - I[2]) / (PTO_PI * D) + N / (6.0 * PTO_PI * D * D));
    }
    for (int i = 0; i < 9; ++i) g[i] /= n_ss;
    return fsum / n_ss;
}

/* SSR = sum_t wt (y - f)^2 and its gradient for n_v parameter vectors
 * (th is [n_v][9]); y, wt are [n_t] (wt NULL: unit weights). */
void pto_ssr_grad(const double *t, int n_t, const double *th, int n_v, int n_ss, double t_exp,
                  const double *y, const double *wt, double *ssr, double *grad, int n_threads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(pto_nthreads(n_threads))
#endif
    for (int v = 0; v < n_v; ++v) {
        double s = 0.0, G[9] = {0}, g[9];
        for (int i = 0; i < n_t; ++i) {
            double f = pto_flux_grad(t[i], th + (size_t)v * 9, n_ss, t_exp, g);
            double wi = wt ? wt[i] : 1.0;
            double r = f - y[i];
            s += wi * r * r;
            for (int j = 0; j < 9; ++j) G[j] += 2.0 * wi * r * g[j];
        }
        ssr[v] = s;
        for (int j = 0; j < 9; ++j) grad[(size_t)v * 9 + j] = G[j];
    }
}


/* ------------------------------------------------------------------------
 * Surrogate network (not in the paper; its analogue there is the
 * interpolation tables of Sec. 2.2.3): a multilayer perceptron
 * 2 -> 128 -> 128 -> 128 -> 2 with SiLU activations, silu(x) = x / (1 + e^-x).
 * Parameters, flattened in this order (FP64 here):
 *   W1[128][2], b1[128], W2[128][128], b2[128], W3[128][128], b3[128],
 *   W4[2][128], b4[2]                                  (33,666 values)
 * Loss: L = (1/n) sum_i sum_o (y_io - t_io)^2.
 * ---------------------------------------------------------------------- */
#define PTO_H 128
#define PTO_NPAR (PTO_H * 2 + PTO_H + PTO_H * PTO_H + PTO_H + PTO_H * PTO_H + PTO_H + 2 * PTO_H + 2)

int pto_mlp_nparams(void) { return PTO_NPAR; }

static double silu(double x) { return x / (1.0 + exp(-x)); }

static double dsilu(double x)
{
    double s = 1.0 / (1.0 + exp(-x));
    return s * (1.0 + x * (1.0 - s));
}

/* forward for one input; z[3][H] and h[3][H] keep pre-activations and
 * activations of the hidden layers (for the backward pass) */
static void mlp_fwd(const double *p, const double *x, double *y, double z[3][PTO_H], double h[3][PTO_H])
{
    const double *W1 = p, *b1 = W1 + 2 * PTO_H, *W2 = b1 + PTO_H, *b2 = W2 + PTO_H * PTO_H;
    const double *W3 = b2 + PTO_H, *b3 = W3 + PTO_H * PTO_H, *W4 = b3 + PTO_H, *b4 = W4 + 2 * PTO_H;
    for (int j = 0; j < PTO_H; ++j) {
        z[0][j] = W1[2 * j] * x[0] + W1[2 * j + 1] * x[1] + b1[j];
        h[0][j] = silu(z[0][j]);
    }
    const double *Ws[2] = {W2, W3}, *bs[2] = {b2, b3};
    for (int l = 1; l < 3; ++l) {
        for (int j = 0; j < PTO_H; ++j) {
            double a = bs[l - 1][j];
            for (int i = 0; i < PTO_H; ++i) a += Ws[l - 1][j * PTO_H + i] * h[l - 1][i];
            z[l][j] = a;
            h[l][j] = silu(a);
        }
    }
    for (int o = 0; o < 2; ++o) {
        double a = b4[o];
        for (int i = 0; i < PTO_H; ++i) a += W4[o * PTO_H + i] * h[2][i];
        y[o] = a;
    }
}

void pto_mlp_forward(const double *p, const double *X, int n, double *Y)
{
    double z[3][PTO_H], h[3][PTO_H];
    for (int i = 0; i < n; ++i) mlp_fwd(p, X + 2 * i, Y + 2 * i, z, h);
}

/* loss and its gradient with respect to every parameter (backpropagation) */
double pto_mlp_loss_grad(const double *p, const double *X, const double *T, int n, double *g)
{
    const double *W2 = p + 3 * PTO_H, *W3 = W2 + PTO_H * PTO_H + PTO_H, *W4 = W3 + PTO_H * PTO_H + PTO_H;
    double *gW1 = g, *gb1 = gW1 + 2 * PTO_H, *gW2 = gb1 + PTO_H, *gb2 = gW2 + PTO_H * PTO_H;
    double *gW3 = gb2 + PTO_H, *gb3 = gW3 + PTO_H * PTO_H, *gW4 = gb3 + PTO_H, *gb4 = gW4 + 2 * PTO_H;
    for (int i = 0; i < PTO_NPAR; ++i) g[i] = 0.0;
    double loss = 0.0;
    double z[3][PTO_H], h[3][PTO_H], y[2], dz[PTO_H], dh[PTO_H];
    for (int s = 0; s < n; ++s) {
        const double *x = X + 2 * s;
        mlp_fwd(p, x, y, z, h);
        double dy[2];
        for (int o = 0; o < 2; ++o) {
            double r = y[o] - T[2 * s + o];
            loss += r * r;
            dy[o] = 2.0 * r / n;
        }
        for (int o = 0; o < 2; ++o) {
            gb4[o] += dy[o];
            for (int i = 0; i < PTO_H; ++i) gW4[o * PTO_H + i] += dy[o] * h[2][i];
        }
        for (int i = 0; i < PTO_H; ++i) dh[i] = W4[i] * dy[0] + W4[PTO_H + i] * dy[1];
        const double *Ws[2] = {W2, W3};
        double *gWs[2] = {gW2, gW3}, *gbs[2] = {gb2, gb3};
        for (int l = 2; l >= 1; --l) {
            for (int j = 0; j < PTO_H; ++j) dz[j] = dh[j] * dsilu(z[l][j]);
            for (int j = 0; j < PTO_H; ++j) {
                gbs[l - 1][j] += dz[j];
                for (int i = 0; i < PTO_H; ++i) gWs[l - 1][j * PTO_H + i] += dz[j] * h[l - 1][i];
            }
            for (int i = 0; i < PTO_H; ++i) {
                double a = 0.0;
                for (int j = 0; j < PTO_H; ++j) a += Ws[l - 1][j * PTO_H + i] * dz[j];
                dh[i] = a;
            }
        }
        for (int j = 0; j < PTO_H; ++j) {
            double d = dh[j] * dsilu(z[0][j]);
            gb1[j] += d;
            gW1[2 * j] += d * x[0];
            gW1[2 * j + 1] += d * x[1];
        }
    }
    return loss / n;
}
