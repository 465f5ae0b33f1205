/*
 * afmm_oracle.c -- plain, slow, FP64 CPU oracle for the cylindrical-coordinate FMM
 * of Carley, "A Fast Multipole Method for axisymmetric domains" (arXiv 2301.01179).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file: only the test suite, the smoke check and the benchmark's CPU-baseline leg use
 * it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Every routine follows the paper's definitions and steps, in the paper's notation:
 *   - modal Green's function G^(n) = Q_{n-1/2}(chi) / (2 pi sqrt(r r1))   (Eq. analysis:gfunc,
 *     Appendix A Eq. gfunc:basic), chi = (r^2 + r1^2 + x^2) / (2 r r1);
 *   - Q_{-1/2}, Q_{1/2} from complete elliptic integrals K, E of modulus mu = sqrt(2/(1+chi))
 *     (Eq. gfunc:Q0), K and E by Carlson's symmetric integrals R_F, R_D (Carlson 1995);
 *   - the Legendre three-term recursion (Eq. gfunc:recursion): forward from the elliptic
 *     start values when the forward direction is stable, otherwise Miller's backward
 *     recursion from arbitrary start values, scaled with the known Q_{-1/2};
 *   - derivative (Taylor) coefficients gbar^(n)_{i,j,k} (Eq. gfunc:gnbar) from the
 *     x-recursion (Eq. gfunc:derivatives:x), the closed r-, r1- and mixed forms (these and
 *     their Legendre start values in binary128, see the reading there), and the
 *     Laplace-equation recursion (Eq. gfunc:laplace:recursion) with the x-derivative term
 *     that the printed formula leaves out (derived from Eq. gfunc:laplace);
 *   - the direct modal sum (Eq. analysis:sum), its field gradient, and the uniform
 *     quadtree FMM of Algorithm 1: moments (Eq. analysis:moments), upward shift
 *     (Eq. analysis:shift), S2L in its FO/BO/FI/BI forms (Eq. analysis:s2l, Sec. 2.2),
 *     local shift (Eq. analysis:l2l), local evaluation (Eq. analysis:local) plus direct
 *     near-neighbour sums.
 * Readings where the paper is silent or inexact (Legendre switch and Miller start, the
 * domain square, depth from a leaf size, treatment of coincident points) are marked
 * "Reading:" where they are used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

/* Legendre-recursion rules.  ORC_RULE_PAPER is the paper's literal rule (forward for
 * chi < 1.008, Miller from n = N + 80).  ORC_RULE_SAFE (default) is the reading used for
 * the 1e-10 target: forward only where its error growth, about exp(2 N acosh chi), stays
 * below e^4, otherwise Miller started far enough above N that the start error,
 * about exp(-2 (L - N) acosh chi), is below e^-60. */
#define ORC_RULE_SAFE 0
#define ORC_RULE_PAPER 1

/* ------------------------------------------------------------------------------------ */
/* Carlson's symmetric elliptic integrals by the duplication theorem (Carlson 1995).     */
/* ------------------------------------------------------------------------------------ */

double orc_carlson_rf(double x, double y, double z)
{
    for (int m = 0; m < 200; ++m) {
        double A = (x + y + z) / 3.0;
        double X = 1.0 - x / A, Y = 1.0 - y / A, Z = 1.0 - z / A;
        double dev = fmax(fabs(X), fmax(fabs(Y), fabs(Z)));
        if (dev < 1e-3) {
            double E2 = X * Y - Z * Z, E3 = X * Y * Z;
            double s = 1.0 - E2 / 10.0 + E3 / 14.0 + E2 * E2 / 24.0 - 3.0 * E2 * E3 / 44.0;
            return s / sqrt(A);
        }
        double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
        double lam = sx * sy + sy * sz + sz * sx;
        x = 0.25 * (x + lam);
        y = 0.25 * (y + lam);
        z = 0.25 * (z + lam);
    }
    return NAN;
}

double orc_carlson_rd(double x, double y, double z)
{
    double sum = 0.0, fac = 1.0;
    for (int m = 0; m < 200; ++m) {
        double A = (x + y + 3.0 * z) / 5.0;
        double X = 1.0 - x / A, Y = 1.0 - y / A, Z = 1.0 - z / A;
        double dev = fmax(fabs(X), fmax(fabs(Y), fabs(Z)));
        if (dev < 1e-3) {
            double XY = X * Y, Z2 = Z * Z;
            double E2 = XY - 6.0 * Z2;
            double E3 = (3.0 * XY - 8.0 * Z2) * Z;
            double E4 = 3.0 * (XY - Z2) * Z2;
            double E5 = XY * Z2 * Z;
            double s = 1.0 - 3.0 * E2 / 14.0 + E3 / 6.0 + 9.0 * E2 * E2 / 88.0 - 3.0 * E4 / 22.0
                     - 9.0 * E2 * E3 / 52.0 + 3.0 * E5 / 26.0;
            return 3.0 * sum + fac * s / (A * sqrt(A));
        }
        double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
        double lam = sx * sy + sy * sz + sz * sx;
        sum += fac / (sz * (z + lam));
        fac *= 0.25;
        x = 0.25 * (x + lam);
        y = 0.25 * (y + lam);
        z = 0.25 * (z + lam);
    }
    return NAN;
}

/* Complete elliptic integrals of modulus k (K(k) = int_0^{pi/2} (1 - k^2 sin^2)^{-1/2}),
 * given k^2 and the complementary k'^2 = 1 - k^2 (both passed so that neither is formed
 * by cancellation):  K = R_F(0, k'^2, 1),  E = R_F(0, k'^2, 1) - k^2/3 R_D(0, k'^2, 1). */
void orc_ellip_ke(double k2, double kp2, double *K, double *E)
{
    double rf = orc_carlson_rf(0.0, kp2, 1.0);
    *K = rf;
    if (E) *E = rf - k2 / 3.0 * orc_carlson_rd(0.0, kp2, 1.0);
}

/* ------------------------------------------------------------------------------------ */
/* Legendre functions Q_{n-1/2}(chi), n = 0..N  (Eqs. gfunc:recursion, gfunc:Q0).        */
/* chi is passed as t = chi - 1 together with k^2 = mu^2 = 2/(1+chi) and                  */
/* k'^2 = (chi-1)/(chi+1), each formed without cancellation by the caller.                */
/* Returns 0 when the forward recursion was used and 1 for Miller's backward recursion.   */
/* ------------------------------------------------------------------------------------ */

int orc_legendre_q(double t, double k2, double kp2, int N, int rule, double *Q)
{
    double chi = 1.0 + t;
    double mu = sqrt(k2);
    double a = log1p(t + sqrt(t * (t + 2.0))); /* acosh(chi) */
    int Nr = N < 2 ? 2 : N;
    int forward, L;
    if (rule == ORC_RULE_PAPER) {
        forward = chi < 1.008;
        L = N + 80;
    } else {
        forward = 2.0 * Nr * a <= 4.0;
        double extra = ceil(30.0 / a) + 10.0;
        if (extra > 100000.0) extra = 100000.0;
        L = N + (int)extra;
    }
    if (forward) {
        double K, E;
        orc_ellip_ke(k2, kp2, &K, &E);
        Q[0] = mu * K;
        /* chi = 1 + t is kept split as (1, t): rounding 1 + t near chi = 1 would move the
         * recursion coefficient by an absolute 1e-16 and cost about n^2 * 1e-16. */
        if (N >= 1) Q[1] = mu * ((K - 2.0 * E) + t * (K - E));
        for (int n = 2; n <= N; ++n)
            Q[n] = (4.0 * (n - 1) * (Q[n - 1] + t * Q[n - 1]) - (2.0 * n - 3.0) * Q[n - 2]) / (2.0 * n - 1.0);
        return 0;
    }
    /* Miller: arbitrary start q_L = 0, q_{L-1} = 1, recursion downward to n = 0,
     * then scale so that q_0 equals the known Q_{-1/2} = mu K(mu). */
    double q_hi = 0.0, q_lo = 1.0; /* q_{n}, q_{n-1} at the top of each step */
    if (L - 1 <= N) Q[L - 1] = q_lo;
    for (int n = L; n >= 2; --n) {
        double q_new = (4.0 * (n - 1) * (q_lo + t * q_lo) - (2.0 * n - 1.0) * q_hi) / (2.0 * n - 3.0);
        q_hi = q_lo;
        q_lo = q_new;
        if (n - 2 <= N) Q[n - 2] = q_new;
        if (fabs(q_new) > 1e200) { /* rescale everything held so far */
            q_hi *= 1e-200;
            q_lo *= 1e-200;
            int top = (L - 1 <= N) ? L - 1 : N;
            for (int m = n - 2; m <= top; ++m)
                if (m >= 0) Q[m] *= 1e-200;
        }
    }
    double K;
    orc_ellip_ke(k2, kp2, &K, NULL);
    double s = mu * K / Q[0];
    for (int n = 0; n <= N; ++n) Q[n] *= s;
    return 1;
}

/* Geometry of one (field, source) pair: rho_-^2, rho_+^2 and the quantities of
 * Eq. gfunc:Q0, formed from rho_-^2 so that chi - 1 keeps full relative accuracy. */
typedef struct {
    double rm2, rp2, t, k2, kp2;
} orc_pair;

static void orc_pair_geom(double r, double r1, double x, orc_pair *p)
{
    double dr = r - r1, sr = r + r1;
    p->rm2 = dr * dr + x * x;
    p->rp2 = sr * sr + x * x;
    p->kp2 = p->rm2 / p->rp2;
    p->k2 = 4.0 * r * r1 / p->rp2;
    p->t = p->rm2 / (2.0 * r * r1);
}

static int g_rule = ORC_RULE_SAFE;
void orc_set_rule(int rule) { g_rule = rule; }

/* G^(n)(r, r1, x), n = 0..N  (Eq. analysis:gfunc).  Reading: a coincident pair
 * (rho_- = 0, a logarithmic singularity) contributes nothing; it returns zeros. */
void orc_green(double r, double r1, double x, int N, double *G)
{
    orc_pair p;
    orc_pair_geom(r, r1, x, &p);
    if (p.rm2 == 0.0) {
        for (int n = 0; n <= N; ++n) G[n] = 0.0;
        return;
    }
    orc_legendre_q(p.t, p.k2, p.kp2, N, g_rule, G);
    double c = 1.0 / (2.0 * ORC_PI * sqrt(r * r1));
    for (int n = 0; n <= N; ++n) G[n] *= c;
}

/* G^(n) and its first derivatives d/dr (field radius) and d/dx (x = z - z1), n = 0..N,
 * from the closed forms for gbar_{1,0,0} and gbar_{0,0,1} (Appendix A) with
 * G^(-1) = G^(1).  Gw must hold max(N,1)+1 doubles of workspace. */
void orc_green_grad(double r, double r1, double x, int N, double *G, double *Gr, double *Gx, double *Gw)
{
    orc_pair p;
    orc_pair_geom(r, r1, x, &p);
    int Nw = N < 1 ? 1 : N;
    if (p.rm2 == 0.0) {
        for (int n = 0; n <= N; ++n) G[n] = Gr[n] = Gx[n] = 0.0;
        return;
    }
    orc_legendre_q(p.t, p.k2, p.kp2, Nw, g_rule, Gw);
    double c = 1.0 / (2.0 * ORC_PI * sqrt(r * r1));
    for (int n = 0; n <= Nw; ++n) Gw[n] *= c;
    /* Reading: the factor r^2 - r1^2 - x^2 of the Appendix A first-derivative forms is
     * evaluated as (r - r1)(r + r1) - x^2; forming r^2 - r1^2 directly cancels
     * catastrophically when r1 -> r (near-coincident pairs). */
    double w = (r - r1) * (r + r1) - x * x;
    for (int n = 0; n <= N; ++n) {
        double g = Gw[n], gm = (n == 0) ? Gw[1] : Gw[n - 1];
        double nu = n - 0.5;
        double bracket = (g + gm) / p.rp2 + (g - gm) / p.rm2;
        G[n] = g;
        Gx[n] = nu * x * bracket;
        Gr[n] = -g / (2.0 * r) + nu * w / (2.0 * r) * bracket;
    }
}

/* ------------------------------------------------------------------------------------ */
/* binary128 copies of the steps that feed the Taylor coefficients (Appendix A).          */
/* Reading: the paper gives no precision.  The x-recursion (Eq. gfunc:derivatives:x) and  */
/* the closed first-derivative forms couple G^(n) with G^(n-1) through their difference,  */
/* which cancels as chi -> 1; the Laplace recursion then carries those errors into the    */
/* high mixed coefficients.  At the paper's own sizes (modes 0..17) FP64 loses nothing    */
/* visible, but at modes 0..32 and beyond the FP64 coefficients of axially adjacent boxes */
/* on fine levels lose up to ten digits (measured against an 80-bit run).  So the oracle  */
/* forms the Legendre start values, the Taylor vectors of the rational factors and the    */
/* four base columns gbar_{0,0,k}, gbar_{1,0,k}, gbar_{0,1,k}, gbar_{1,1,k} in binary128  */
/* (_Float128: + - * / only, from the compiler), rounds them to FP64, and runs the        */
/* Laplace recursion (which is stable given accurate base columns) in FP64.               */
/* ------------------------------------------------------------------------------------ */
typedef _Float128 orc_q;

static orc_q q_abs(orc_q a) { return a < 0 ? -a : a; }
static orc_q q_max(orc_q a, orc_q b) { return a > b ? a : b; }

/* square root: Newton's iteration from the FP64 root (three steps reach full precision) */
static orc_q q_sqrt(orc_q a)
{
    if (!(a > 0)) return 0;
    orc_q s = (orc_q)sqrt((double)a);
    for (int it = 0; it < 3; ++it) s = (s + a / s) / 2;
    return s;
}

/* pi as the sum of its two nearest FP64 parts (about 107 bits) */
static orc_q q_pi(void) { return (orc_q)3.141592653589793 + (orc_q)1.2246467991473532e-16; }

/* Carlson R_F and R_D as above; the series is used once the deviation is below 3e-6, where
 * its first neglected term (about dev^6) is below the binary128 rounding. */
static orc_q q_carlson_rf(orc_q x, orc_q y, orc_q z)
{
    for (int m = 0; m < 200; ++m) {
        orc_q A = (x + y + z) / 3;
        orc_q X = 1 - x / A, Y = 1 - y / A, Z = 1 - z / A;
        orc_q dev = q_max(q_abs(X), q_max(q_abs(Y), q_abs(Z)));
        if (dev < (orc_q)3e-6) {
            orc_q E2 = X * Y - Z * Z, E3 = X * Y * Z;
            orc_q s = 1 - E2 / 10 + E3 / 14 + E2 * E2 / 24 - 3 * E2 * E3 / 44;
            return s / q_sqrt(A);
        }
        orc_q sx = q_sqrt(x), sy = q_sqrt(y), sz = q_sqrt(z);
        orc_q lam = sx * sy + sy * sz + sz * sx;
        x = (x + lam) / 4;
        y = (y + lam) / 4;
        z = (z + lam) / 4;
    }
    return 0;
}

static orc_q q_carlson_rd(orc_q x, orc_q y, orc_q z)
{
    orc_q sum = 0, fac = 1;
    for (int m = 0; m < 200; ++m) {
        orc_q A = (x + y + 3 * z) / 5;
        orc_q X = 1 - x / A, Y = 1 - y / A, Z = 1 - z / A;
        orc_q dev = q_max(q_abs(X), q_max(q_abs(Y), q_abs(Z)));
        if (dev < (orc_q)3e-6) {
            orc_q XY = X * Y, Z2 = Z * Z;
            orc_q E2 = XY - 6 * Z2;
            orc_q E3 = (3 * XY - 8 * Z2) * Z;
            orc_q E4 = 3 * (XY - Z2) * Z2;
            orc_q E5 = XY * Z2 * Z;
            orc_q s = 1 - 3 * E2 / 14 + E3 / 6 + 9 * E2 * E2 / 88 - 3 * E4 / 22 - 9 * E2 * E3 / 52 + 3 * E5 / 26;
            return 3 * sum + fac * s / (A * q_sqrt(A));
        }
        orc_q sx = q_sqrt(x), sy = q_sqrt(y), sz = q_sqrt(z);
        orc_q lam = sx * sy + sy * sz + sz * sx;
        sum += fac / (sz * (z + lam));
        fac /= 4;
        x = (x + lam) / 4;
        y = (y + lam) / 4;
        z = (z + lam) / 4;
    }
    return 0;
}

/* G^(n)(r, r1, x), n = 0..N, in binary128: the same geometry (from rho_-^2), start values
 * (Eq. gfunc:Q0) and forward or Miller recursion (Eq. gfunc:recursion) as orc_green with
 * ORC_RULE_SAFE, whose Miller start error (about e^-60) is below what the Taylor
 * coefficients need.  The forward/backward decision is taken in FP64. */
static void q_green(double r_, double r1_, double x_, int N, orc_q *G)
{
    orc_q r = r_, r1 = r1_, x = x_;
    orc_q dr = r - r1, sr = r + r1;
    orc_q rm2 = dr * dr + x * x, rp2 = sr * sr + x * x;
    if (rm2 == 0) {
        for (int n = 0; n <= N; ++n) G[n] = 0;
        return;
    }
    orc_q kp2 = rm2 / rp2, k2 = 4 * r * r1 / rp2, t = rm2 / (2 * r * r1);
    orc_q mu = q_sqrt(k2);
    double td = (double)t;
    double a = log1p(td + sqrt(td * (td + 2.0))); /* acosh(chi) */
    int Nr = N < 2 ? 2 : N;
    int forward = 2.0 * Nr * a <= 4.0;
    double extra = ceil(30.0 / a) + 10.0;
    if (extra > 100000.0) extra = 100000.0;
    int L = N + (int)extra;
    orc_q rf = q_carlson_rf(0, kp2, 1);
    if (forward) {
        orc_q K = rf, E = rf - k2 / 3 * q_carlson_rd(0, kp2, 1);
        G[0] = mu * K;
        if (N >= 1) G[1] = mu * ((K - 2 * E) + t * (K - E));
        for (int n = 2; n <= N; ++n)
            G[n] = (4 * (orc_q)(n - 1) * (G[n - 1] + t * G[n - 1]) - (orc_q)(2 * n - 3) * G[n - 2]) / (orc_q)(2 * n - 1);
    } else {
        orc_q q_hi = 0, q_lo = 1;
        if (L - 1 <= N) G[L - 1] = q_lo;
        for (int n = L; n >= 2; --n) {
            orc_q q_new = (4 * (orc_q)(n - 1) * (q_lo + t * q_lo) - (orc_q)(2 * n - 1) * q_hi) / (orc_q)(2 * n - 3);
            q_hi = q_lo;
            q_lo = q_new;
            if (n - 2 <= N) G[n - 2] = q_new;
            if (q_abs(q_new) > (orc_q)1e200) {
                q_hi /= (orc_q)1e200;
                q_lo /= (orc_q)1e200;
                int top = (L - 1 <= N) ? L - 1 : N;
                for (int m = n - 2; m <= top; ++m)
                    if (m >= 0) G[m] /= (orc_q)1e200;
            }
        }
        orc_q s = mu * rf / G[0];
        for (int n = 0; n <= N; ++n) G[n] *= s;
    }
    orc_q c = 1 / (2 * q_pi() * q_sqrt(r * r1));
    for (int n = 0; n <= N; ++n) G[n] *= c;
}

/* Taylor coefficients (in x about x0) of 1/(a^2 + x^2) and of (c - x^2) w(x), binary128 */
static void q_taylor_inv(orc_q a, orc_q x0, int P, orc_q *v)
{
    orc_q u0 = a * a + x0 * x0;
    v[0] = 1 / u0;
    if (P >= 1) v[1] = -2 * x0 * v[0] / u0;
    for (int q = 2; q <= P; ++q) v[q] = -(2 * x0 * v[q - 1] + v[q - 2]) / u0;
}

static void q_taylor_cmx2(orc_q c, orc_q x0, int P, const orc_q *w, orc_q *out)
{
    for (int q = 0; q <= P; ++q) {
        orc_q s = (c - x0 * x0) * w[q];
        if (q >= 1) s -= 2 * x0 * w[q - 1];
        if (q >= 2) s -= w[q - 2];
        out[q] = s;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Taylor coefficients gbar^(n)_{i,j,k}(r, r1, x), i+j+k <= P, n = 0..N (Appendix A).      */
/* Output layout: g[((n*(P+1) + i)*(P+1) + j)*(P+1) + k] (dense cube; entries with          */
/* i+j+k > P are left at zero).                                                          */
/* ------------------------------------------------------------------------------------ */

#define GIDX(n, i, j, k) ((((size_t)(n) * (P + 1) + (i)) * (P + 1) + (j)) * (P + 1) + (k))

int orc_gbar(double r, double r1, double x, int N, int P, double *g)
{
    int Nw = N < 1 ? 1 : N; /* mode 1 is needed for n = 0 via G^(-1) = G^(1) */
    size_t cube = (size_t)(P + 1) * (P + 1) * (P + 1);
    size_t Q = (size_t)P + 1;
    double *gw = (double *)calloc((size_t)(Nw + 1) * cube, sizeof(double));
    orc_q *vq = (orc_q *)malloc(sizeof(orc_q) * (P + 2) * 12);
    /* base columns in binary128: [Nw+1][P+1] each */
    orc_q *b00 = (orc_q *)calloc((size_t)(Nw + 1) * Q * 4, sizeof(orc_q));
    if (!gw || !vq || !b00) {
        free(gw);
        free(vq);
        free(b00);
        return -1;
    }
    orc_q *b10 = b00 + (size_t)(Nw + 1) * Q, *b01 = b10 + (size_t)(Nw + 1) * Q, *b11 = b01 + (size_t)(Nw + 1) * Q;
    orc_q *vp = vq, *vm = vp + (P + 2);
    orc_q *fxp = vm + (P + 2), *fxm = fxp + (P + 2);      /* x / rho_pm^2 */
    orc_q *hp = fxm + (P + 2), *hm = hp + (P + 2);        /* (r^2-r1^2-x^2)/rho_pm^2 */
    orc_q *hp1 = hm + (P + 2), *hm1 = hp1 + (P + 2);      /* (r1^2-r^2-x^2)/rho_pm^2 */
    orc_q *dhp = hm1 + (P + 2), *dhm = dhp + (P + 2);     /* d/dr1 of hp, hm */
    orc_q *tmp = dhm + (P + 2), *tmp2 = tmp + (P + 2);
    const orc_q rq = r, r1q = r1, xq = x;

    q_taylor_inv(rq + r1q, xq, P, vp);
    q_taylor_inv(rq - r1q, xq, P, vm);
    for (int q = 0; q <= P; ++q) {
        fxp[q] = xq * vp[q] + (q >= 1 ? vp[q - 1] : 0);
        fxm[q] = xq * vm[q] + (q >= 1 ? vm[q - 1] : 0);
    }
    orc_q c = (rq - r1q) * (rq + r1q);
    q_taylor_cmx2(c, xq, P, vp, hp);
    q_taylor_cmx2(c, xq, P, vm, hm);
    q_taylor_cmx2(-c, xq, P, vp, hp1);
    q_taylor_cmx2(-c, xq, P, vm, hm1);
    /* d/dr1 [(c - x^2)/((r+s r1)^2 + x^2)] = -2 r1 v - 2 s (r + s r1) (c - x^2) v^2, s = +-1 */
    for (int sgn = 0; sgn < 2; ++sgn) {
        const orc_q *v = sgn == 0 ? vp : vm;
        orc_q s = sgn == 0 ? 1 : -1;
        orc_q a = rq + s * r1q;
        for (int q = 0; q <= P; ++q) {
            orc_q acc = 0;
            for (int p = 0; p <= q; ++p) acc += v[p] * v[q - p];
            tmp[q] = acc;
        }
        q_taylor_cmx2(c, xq, P, tmp, tmp2);
        orc_q *d = sgn == 0 ? dhp : dhm;
        for (int q = 0; q <= P; ++q) d[q] = -2 * r1q * v[q] - 2 * s * a * tmp2[q];
    }

    /* gbar_{0,0,0} = G^(n) */
    {
        orc_q *G0 = (orc_q *)malloc(sizeof(orc_q) * (Nw + 1));
        q_green(r, r1, x, Nw, G0);
        for (int n = 0; n <= Nw; ++n) b00[(size_t)n * Q] = G0[n];
        free(G0);
    }
#define B(arr, n, k) arr[(size_t)(n) * Q + (k)]
#define BM(arr, n, k) arr[(size_t)((n) == 0 ? 1 : (n) - 1) * Q + (k)]
    /* x-derivatives, Eq. gfunc:derivatives:x (coupled in n; G^(-1) = G^(1)) */
    for (int k = 0; k < P; ++k) {
        for (int n = 0; n <= Nw; ++n) {
            orc_q nu = (orc_q)n - (orc_q)0.5, acc = 0;
            for (int q = 0; q <= k; ++q) {
                orc_q gp = B(b00, n, k - q), gm = BM(b00, n, k - q);
                acc += (gp + gm) * fxp[q] + (gp - gm) * fxm[q];
            }
            B(b00, n, k + 1) = nu / (k + 1) * acc;
        }
    }
    /* r-derivatives gbar_{1,0,k} and (by exchanging r and r1) gbar_{0,1,k} */
    for (int k = 0; k + 1 <= P; ++k) {
        for (int n = 0; n <= Nw; ++n) {
            orc_q nu = (orc_q)n - (orc_q)0.5, a1 = 0, a2 = 0;
            for (int q = 0; q <= k; ++q) {
                orc_q gp = B(b00, n, k - q), gm = BM(b00, n, k - q);
                a1 += (gp + gm) * hp[q] + (gp - gm) * hm[q];
                a2 += (gp + gm) * hp1[q] + (gp - gm) * hm1[q];
            }
            B(b10, n, k) = -B(b00, n, k) / (2 * rq) + nu / (2 * rq) * a1;
            B(b01, n, k) = -B(b00, n, k) / (2 * r1q) + nu / (2 * r1q) * a2;
        }
    }
    /* mixed gbar_{1,1,k} */
    for (int k = 0; k + 2 <= P; ++k) {
        for (int n = 0; n <= Nw; ++n) {
            orc_q nu = (orc_q)n - (orc_q)0.5, acc = 0;
            for (int q = 0; q <= k; ++q) {
                orc_q g0p = B(b00, n, k - q), g0m = BM(b00, n, k - q);
                orc_q g1p = B(b01, n, k - q), g1m = BM(b01, n, k - q);
                acc += (g0p + g0m) * dhp[q] + (g1p + g1m) * hp[q] + (g0p - g0m) * dhm[q] + (g1p - g1m) * hm[q];
            }
            B(b11, n, k) = -B(b01, n, k) / (2 * rq) + nu / (2 * rq) * acc;
        }
    }
#undef B
#undef BM
#define GW(n, i, j, k) gw[GIDX(n, i, j, k)]
    /* the base columns, rounded to FP64, start the Laplace recursions */
    for (int n = 0; n <= Nw; ++n)
        for (int k = 0; k <= P; ++k) {
            GW(n, 0, 0, k) = (double)b00[(size_t)n * Q + k];
            if (k + 1 <= P) GW(n, 1, 0, k) = (double)b10[(size_t)n * Q + k];
            if (k + 1 <= P) GW(n, 0, 1, k) = (double)b01[(size_t)n * Q + k];
            if (k + 2 <= P) GW(n, 1, 1, k) = (double)b11[(size_t)n * Q + k];
        }
    free(b00);
    free(vq);
    /* Reading of Eq. gfunc:laplace:recursion: the Laplace equation (Eq. gfunc:laplace)
     * expanded in powers of the radial offset gives the printed sum plus the term
     * -(k+1)(k+2)/((i+1)(i+2)) gbar_{i,j,k+2} from d^2G/dx^2, which the printed formula
     * omits.  The same relation in r1 (source Laplace equation) raises j. */
    for (int n = 0; n <= Nw; ++n) {
        double n2 = (double)n * n;
        for (int i = 0; i <= 1; ++i) {
            for (int j = 0; i + j + 2 <= P; ++j) {
                for (int k = 0; i + j + 2 + k <= P; ++k) {
                    double acc = 0.0, rp = 1.0 / r1;
                    for (int u = 0; u <= j; ++u) {
                        double sg = (u & 1) ? -1.0 : 1.0;
                        acc += sg * rp * ((u + 1) * n2 / r1 * GW(n, i, j - u, k) - (j - u + 1) * GW(n, i, j - u + 1, k));
                        rp /= r1;
                    }
                    acc /= (double)(j + 1) * (j + 2);
                    acc -= (double)(k + 1) * (k + 2) / ((double)(j + 1) * (j + 2)) * GW(n, i, j, k + 2);
                    GW(n, i, j + 2, k) = acc;
                }
            }
        }
        for (int i = 0; i + 2 <= P; ++i) {
            for (int j = 0; i + 2 + j <= P; ++j) {
                for (int k = 0; i + 2 + j + k <= P; ++k) {
                    double acc = 0.0, rp = 1.0 / r;
                    for (int u = 0; u <= i; ++u) {
                        double sg = (u & 1) ? -1.0 : 1.0;
                        acc += sg * rp * ((u + 1) * n2 / r * GW(n, i - u, j, k) - (i - u + 1) * GW(n, i - u + 1, j, k));
                        rp /= r;
                    }
                    acc /= (double)(i + 1) * (i + 2);
                    acc -= (double)(k + 1) * (k + 2) / ((double)(i + 1) * (i + 2)) * GW(n, i, j, k + 2);
                    GW(n, i + 2, j, k) = acc;
                }
            }
        }
    }
#undef GW
    memcpy(g, gw, (size_t)(N + 1) * cube * sizeof(double));
    free(gw);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Direct modal sum (Eq. analysis:sum) and its field gradient.                            */
/* Amplitudes and outputs are mode-major planes: q[n*ns + i], phi[n*nf + j].              */
/* Summation over sources is compensated (Neumaier) so the reference is accurate to a     */
/* few ulps of each result whatever the source order.                                     */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    double s, c;
} orc_ksum;
static inline void orc_kadd(orc_ksum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}

void orc_direct(int64_t ns, const double *sr, const double *sz, int64_t nf, const double *tr, const double *tz,
                int nmodes, const double *q_re, const double *q_im, double *phi_re, double *phi_im,
                double *dr_re, double *dr_im, double *dz_re, double *dz_im, int nthreads)
{
    int N = nmodes - 1;
    int grad = dr_re != NULL;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        int Nw = N < 1 ? 1 : N;
        double *G = (double *)malloc(sizeof(double) * (Nw + 1) * 4);
        double *Gr = G + (Nw + 1), *Gx = Gr + (Nw + 1), *Gw = Gx + (Nw + 1);
        orc_ksum *acc = (orc_ksum *)malloc(sizeof(orc_ksum) * nmodes * 6);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t j = 0; j < nf; ++j) {
            memset(acc, 0, sizeof(orc_ksum) * nmodes * 6);
            for (int64_t i = 0; i < ns; ++i) {
                double x = tz[j] - sz[i];
                if (grad)
                    orc_green_grad(tr[j], sr[i], x, N, G, Gr, Gx, Gw);
                else
                    orc_green(tr[j], sr[i], x, N, G);
                for (int n = 0; n < nmodes; ++n) {
                    double a = q_re[(size_t)n * ns + i], b = q_im[(size_t)n * ns + i];
                    orc_kadd(&acc[6 * n + 0], a * G[n]);
                    orc_kadd(&acc[6 * n + 1], b * G[n]);
                    if (grad) {
                        orc_kadd(&acc[6 * n + 2], a * Gr[n]);
                        orc_kadd(&acc[6 * n + 3], b * Gr[n]);
                        orc_kadd(&acc[6 * n + 4], a * Gx[n]);
                        orc_kadd(&acc[6 * n + 5], b * Gx[n]);
                    }
                }
            }
            for (int n = 0; n < nmodes; ++n) {
                size_t o = (size_t)n * nf + j;
                if (phi_re) phi_re[o] = acc[6 * n + 0].s + acc[6 * n + 0].c;
                if (phi_im) phi_im[o] = acc[6 * n + 1].s + acc[6 * n + 1].c;
                if (grad) {
                    dr_re[o] = acc[6 * n + 2].s + acc[6 * n + 2].c;
                    dr_im[o] = acc[6 * n + 3].s + acc[6 * n + 3].c;
                    dz_re[o] = acc[6 * n + 4].s + acc[6 * n + 4].c;
                    dz_im[o] = acc[6 * n + 5].s + acc[6 * n + 5].c;
                }
            }
        }
        free(G);
        free(acc);
    }
}

/* Adjoint of the direct sum for a real loss L(Phi): given gphi = dL/dRe(Phi) + i dL/dIm(Phi)
 * at the field points, returns gq = dL/dRe(q) + i dL/dIm(q) and dL/dr_i, dL/dz_i of the
 * source positions.  G is real, symmetric in r <-> r1 and even in x (Sec. 2.2), so the
 * adjoint is the same sum with the roles of sources and field points exchanged:
 *   A_i = sum_j G(r_i, r_j, z_i - z_j) gphi_j                       -> gq_i = A_i
 *   B_i, C_i = the r- and z-gradient of that sum at the source point
 *   dL/dr_i = sum_n Re(q_i conj(B_i)),  dL/dz_i = sum_n Re(q_i conj(C_i)). */
void orc_adjoint_direct(int64_t ns, const double *sr, const double *sz, int64_t nf, const double *tr,
                        const double *tz, int nmodes, const double *q_re, const double *q_im,
                        const double *gphi_re, const double *gphi_im, double *gq_re, double *gq_im,
                        double *g_r, double *g_z, int nthreads)
{
    size_t m = (size_t)nmodes * ns;
    double *B = (double *)malloc(sizeof(double) * m * 4);
    orc_direct(nf, tr, tz, ns, sr, sz, nmodes, gphi_re, gphi_im, gq_re, gq_im, B, B + m, B + 2 * m, B + 3 * m,
               nthreads);
    for (int64_t i = 0; i < ns; ++i) {
        double ar = 0.0, az = 0.0;
        for (int n = 0; n < nmodes; ++n) {
            size_t o = (size_t)n * ns + i;
            ar += q_re[o] * B[o] + q_im[o] * B[m + o];
            az += q_re[o] * B[2 * m + o] + q_im[o] * B[3 * m + o];
        }
        g_r[i] = ar;
        g_z[i] = az;
    }
    free(B);
}

/* ------------------------------------------------------------------------------------ */
/* Uniform quadtree (Sec. 2.1, Algorithm 1).                                             */
/* Reading of the domain: the paper subdivides the square 0 <= r, z <= r_max.  Here the  */
/* square is anchored at (min r, min z) over sources and field points, with side          */
/* L = max(r extent, z extent); a point on the upper edge belongs to the last box.        */
/* Reading of the depth: the smallest d >= 2 for which the mean number of sources in the  */
/* non-empty leaves is at most leaf_size (capped at 16).                                  */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int d;
    double r0, z0, L;
} orc_tree;

static int orc_box_coord(double v, double v0, double L, int level)
{
    double s = (double)(1 << level) / L;
    double f = floor((v - v0) * s);
    int i = (int)f;
    int nmax = (1 << level) - 1;
    if (f < 0.0) i = 0;
    if (i > nmax) i = nmax;
    return i;
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y);
}

int orc_tree_setup(int64_t ns, const double *sr, const double *sz, int64_t nf, const double *tr, const double *tz,
                   int leaf_size, int depth_override, int *d_out, double *geom_out)
{
    double rmin = INFINITY, rmax = -INFINITY, zmin = INFINITY, zmax = -INFINITY;
    for (int64_t i = 0; i < ns; ++i) {
        rmin = fmin(rmin, sr[i]); rmax = fmax(rmax, sr[i]);
        zmin = fmin(zmin, sz[i]); zmax = fmax(zmax, sz[i]);
    }
    for (int64_t j = 0; j < nf; ++j) {
        rmin = fmin(rmin, tr[j]); rmax = fmax(rmax, tr[j]);
        zmin = fmin(zmin, tz[j]); zmax = fmax(zmax, tz[j]);
    }
    double L = fmax(rmax - rmin, zmax - zmin);
    if (!(L > 0.0)) L = 1.0;
    geom_out[0] = rmin;
    geom_out[1] = zmin;
    geom_out[2] = L;
    int d = depth_override;
    if (d <= 0 && ns == 0) d = 2;
    if (d <= 0) {
        const int D = 16;
        uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (ns > 0 ? ns : 1));
        d = D;
        for (int dd = 2; dd <= D; ++dd) {
            /* number of non-empty leaves at depth dd: distinct (ir, iz) among the sources */
            for (int64_t i = 0; i < ns; ++i) {
                uint64_t a = (uint64_t)orc_box_coord(sr[i], rmin, L, dd);
                uint64_t b = (uint64_t)orc_box_coord(sz[i], zmin, L, dd);
                key[i] = (a << 32) | b;
            }
            qsort(key, (size_t)ns, sizeof(uint64_t), cmp_u64);
            int64_t cnt = 0;
            for (int64_t i = 0; i < ns; ++i)
                if (i == 0 || key[i] != key[i - 1]) ++cnt;
            if (cnt > 0 && (double)ns <= (double)leaf_size * (double)cnt) { d = dd; break; }
        }
        free(key);
    }
    *d_out = d;
    return 0;
}

/* moment / local coefficient index for i + j <= M (row i holds M+1-i entries) */
static inline int cidx(int i, int j, int M) { return i * (M + 1) - i * (i - 1) / 2 + j; }

static double binom_slow(int n, int k)
{
    double b = 1.0;
    for (int t = 1; t <= k; ++t) b = b * (n - k + t) / t;
    return b;
}

/* binomial coefficients C(n, k), n <= 127, tabulated once */
static double g_binom[128][128];
static int g_binom_ready = 0;
static inline double binom(int n, int k)
{
    return g_binom[n][k];
}
static void binom_init(void)
{
    if (g_binom_ready) return;
    for (int n = 0; n < 128; ++n)
        for (int k = 0; k < 128; ++k) g_binom[n][k] = k <= n ? binom_slow(n, k) : 0.0;
    g_binom_ready = 1;
}

/* One S2L application (Eq. analysis:s2l and its three variants, Sec. 2.2).
 * E is the expansion gbar(r_big, r_small, |x|) for one mode, dense cube with side P+1.
 * inward = 0: field box at the larger radius (FO/BO), uses E_{k,i,j+l};
 * inward = 1: field box at the smaller radius (FI/BI), uses E_{i,k,j+l};
 * backward = 0: sign (-1)^j (x >= 0);  backward = 1: sign (-1)^l (x < 0). */
static void orc_s2l(const double *E, int P, int M, int inward, int backward, const double *S_re,
                    const double *S_im, double *F_re, double *F_im)
{
    for (int k = 0; k <= M; ++k)
        for (int l = 0; k + l <= M; ++l) {
            double ar = 0.0, ai = 0.0;
            for (int i = 0; i <= M; ++i)
                for (int j = 0; i + j <= M; ++j) {
                    int e = backward ? l : j;
                    double sg = (e & 1) ? -1.0 : 1.0;
                    double g = inward ? E[((size_t)i * (P + 1) + k) * (P + 1) + (j + l)]
                                      : E[((size_t)k * (P + 1) + i) * (P + 1) + (j + l)];
                    double w = sg * binom(j + l, j) * g;
                    ar += w * S_re[cidx(i, j, M)];
                    ai += w * S_im[cidx(i, j, M)];
                }
            F_re[cidx(k, l, M)] += ar;
            F_im[cidx(k, l, M)] += ai;
        }
}

static int in_s2l_list(int ti, int tj, int si, int sj)
{
    int pi = ti >> 1, pj = tj >> 1, qi = si >> 1, qj = sj >> 1;
    if (abs(pi - qi) > 1 || abs(pj - qj) > 1) return 0;
    int di = abs(si - ti), dj = abs(sj - tj);
    return (di > 1 || dj > 1);
}

/* The uniform FMM of Algorithm 1, FP64, with optional field gradient at the targets.
 * Boxes at level l are (ir, iz), 0 <= ir, iz < 2^l, index ir * 2^l + iz; centres at
 * r0 + (ir + 1/2) L / 2^l, z0 + (iz + 1/2) L / 2^l.  Moments and local expansions are
 * truncated at total degree M (i + j <= M, k + l <= M), so S2L needs gbar to order 2M. */
int orc_fmm(int64_t ns, const double *sr, const double *sz, int64_t nf, const double *tr, const double *tz,
            int nmodes, const double *q_re, const double *q_im, int M, int d, const double *geom,
            double *phi_re, double *phi_im, double *dr_re, double *dr_im, double *dz_re, double *dz_im)
{
    if (d < 2 || M > 60) return -1;
    binom_init();
    int N = nmodes - 1;
    int P = 2 * M;
    int nc = (M + 1) * (M + 2) / 2;
    double r0 = geom[0], z0 = geom[1], L = geom[2];
    int grad = dr_re != NULL;
    /* per-level moment and local arrays: [box][mode][coef] */
    double **mom_re = (double **)calloc(d + 1, sizeof(double *));
    double **mom_im = (double **)calloc(d + 1, sizeof(double *));
    double **loc_re = (double **)calloc(d + 1, sizeof(double *));
    double **loc_im = (double **)calloc(d + 1, sizeof(double *));
    for (int l = 1; l <= d; ++l) {
        size_t sz_ = (size_t)(1u << (2 * l)) * nmodes * nc;
        mom_re[l] = (double *)calloc(sz_, sizeof(double));
        mom_im[l] = (double *)calloc(sz_, sizeof(double));
        loc_re[l] = (double *)calloc(sz_, sizeof(double));
        loc_im[l] = (double *)calloc(sz_, sizeof(double));
        if (!mom_re[l] || !mom_im[l] || !loc_re[l] || !loc_im[l]) return -2;
    }
#define BOXOFF(l, b, n) ((((size_t)(b)) * nmodes + (n)) * nc)
    int nside = 1 << d;
    double hd = L / nside;
    /* leaf moments, Eq. analysis:moments.  Modes are independent, so they run on
     * separate threads; each moment still sums its sources in source order. */
#pragma omp parallel for schedule(dynamic, 1)
    for (int n = 0; n < nmodes; ++n) {
        double pw_r[61], pw_z[61];
        for (int64_t q = 0; q < ns; ++q) {
            int ir = orc_box_coord(sr[q], r0, L, d), iz = orc_box_coord(sz[q], z0, L, d);
            int b = ir * nside + iz;
            double cr = r0 + (ir + 0.5) * hd, cz = z0 + (iz + 0.5) * hd;
            double dr = sr[q] - cr, dz = sz[q] - cz;
            pw_r[0] = pw_z[0] = 1.0;
            for (int i = 1; i <= M; ++i) {
                pw_r[i] = pw_r[i - 1] * dr;
                pw_z[i] = pw_z[i - 1] * dz;
            }
            double a = q_re[(size_t)n * ns + q], bb = q_im[(size_t)n * ns + q];
            for (int i = 0; i <= M; ++i)
                for (int j = 0; i + j <= M; ++j) {
                    double w = pw_r[i] * pw_z[j];
                    mom_re[d][BOXOFF(d, b, n) + cidx(i, j, M)] += a * w;
                    mom_im[d][BOXOFF(d, b, n) + cidx(i, j, M)] += bb * w;
                }
        }
    }
    /* upward pass, Eq. analysis:shift, Delta = parent centre - child centre (one thread
     * per mode; each parent sums its children in the same order for every mode) */
    for (int l = d - 1; l >= 2; --l) {
        int ns_c = 1 << (l + 1);
        double hc = L / ns_c;
#pragma omp parallel for schedule(dynamic, 1)
        for (int n = 0; n < nmodes; ++n)
        for (int ci = 0; ci < ns_c; ++ci)
            for (int cj = 0; cj < ns_c; ++cj) {
                int pi = ci >> 1, pj = cj >> 1;
                int cb = ci * ns_c + cj, pb = pi * (ns_c >> 1) + pj;
                double Dr = (pi + 0.5) * 2.0 * hc - (ci + 0.5) * hc;
                double Dz = (pj + 0.5) * 2.0 * hc - (cj + 0.5) * hc;
                {
                    const double *cre = &mom_re[l + 1][BOXOFF(l + 1, cb, n)];
                    const double *cim = &mom_im[l + 1][BOXOFF(l + 1, cb, n)];
                    double *pre = &mom_re[l][BOXOFF(l, pb, n)];
                    double *pim = &mom_im[l][BOXOFF(l, pb, n)];
                    for (int i = 0; i <= M; ++i)
                        for (int j = 0; i + j <= M; ++j) {
                            double ar = 0.0, ai = 0.0;
                            for (int q = 0; q <= i; ++q)
                                for (int u = 0; u <= j; ++u) {
                                    double w = binom(i, q) * binom(j, u) * pow(-Dr, q) * pow(-Dz, u);
                                    ar += w * cre[cidx(i - q, j - u, M)];
                                    ai += w * cim[cidx(i - q, j - u, M)];
                                }
                            pre[cidx(i, j, M)] += ar;
                            pim[cidx(i, j, M)] += ai;
                        }
                }
            }
    }
    /* downward pass */
    size_t cube = (size_t)(P + 1) * (P + 1) * (P + 1);
    double *E = (double *)malloc(sizeof(double) * cube * nmodes * 16);
    if (!E) return -2;
    for (int l = 2; l <= d; ++l) {
        int nl = 1 << l;
        double h = L / nl;
        /* local shift from the parent, Eq. analysis:l2l (level-1 locals are zero) */
        if (l > 2) {
            /* each child box is written by one thread */
#pragma omp parallel for schedule(dynamic, 1)
            for (int ci = 0; ci < nl; ++ci)
                for (int cj = 0; cj < nl; ++cj) {
                    int pi = ci >> 1, pj = cj >> 1;
                    int cb = ci * nl + cj, pb = pi * (nl >> 1) + pj;
                    double Dr = (pi + 0.5) * 2.0 * h - (ci + 0.5) * h;
                    double Dz = (pj + 0.5) * 2.0 * h - (cj + 0.5) * h;
                    for (int n = 0; n < nmodes; ++n) {
                        const double *pre = &loc_re[l - 1][BOXOFF(l - 1, pb, n)];
                        const double *pim = &loc_im[l - 1][BOXOFF(l - 1, pb, n)];
                        double *cre = &loc_re[l][BOXOFF(l, cb, n)];
                        double *cim = &loc_im[l][BOXOFF(l, cb, n)];
                        for (int i = 0; i <= M; ++i)
                            for (int j = 0; i + j <= M; ++j) {
                                double ar = 0.0, ai = 0.0;
                                for (int q = 0; i + q <= M; ++q)
                                    for (int u = 0; i + q + j + u <= M; ++u) {
                                        double w = binom(i + q, q) * binom(j + u, u) * pow(-Dr, q) * pow(-Dz, u);
                                        ar += w * pre[cidx(i + q, j + u, M)];
                                        ai += w * pim[cidx(i + q, j + u, M)];
                                    }
                                cre[cidx(i, j, M)] += ar;
                                cim[cidx(i, j, M)] += ai;
                            }
                    }
                }
        }
        /* per radial station: the twelve Green's-function expansions (offsets dr, dz in
         * 0..3, not both <= 1) at r_small = station centre, r_big = r_small + dr h, x = dz h,
         * then FO/BO from sources in the station and FI/BI into locals in the station. */
        for (int si = 0; si < nl; ++si) {
            double rs = r0 + (si + 0.5) * h;
            int have[4][4];
            int gfail = 0;
            /* the twelve expansions of the station are independent: one thread each */
#pragma omp parallel for schedule(dynamic, 1) reduction(|: gfail)
            for (int ab = 0; ab < 16; ++ab) {
                int a = ab / 4, b = ab % 4;
                have[a][b] = 0;
                if (a <= 1 && b <= 1) continue;
                if (si + a >= nl) continue;
                double rb = r0 + (si + a + 0.5) * h;
                double *Eab = E + (size_t)(a * 4 + b) * cube * nmodes;
                if (orc_gbar(rb, rs, b * h, N, P, Eab) != 0) gfail = 1;
                have[a][b] = 1;
            }
            if (gfail) return -2;
            /* the S2L applications of one mode touch only that mode's moments and locals:
             * one thread per mode, the same application order within each mode */
#pragma omp parallel for schedule(dynamic, 1)
            for (int n = 0; n < nmodes; ++n)
            for (int sj = 0; sj < nl; ++sj) {
                for (int a = 0; a < 4; ++a)
                    for (int b = 0; b < 4; ++b) {
                        if (!have[a][b]) continue;
                        const double *Eab = E + (size_t)(a * 4 + b) * cube * nmodes;
                        /* FO / BO: source box (si, sj) -> field box (si + a, sj +- b) */
                        for (int dir = 0; dir < 2; ++dir) {
                            if (b == 0 && dir == 1) continue;
                            int ti = si + a, tj = dir == 0 ? sj + b : sj - b;
                            if (tj < 0 || tj >= nl) continue;
                            if (!in_s2l_list(ti, tj, si, sj)) continue;
                            int tb = ti * nl + tj, sb = si * nl + sj;
                            orc_s2l(Eab + (size_t)n * cube, P, M, 0, dir, &mom_re[l][BOXOFF(l, sb, n)],
                                    &mom_im[l][BOXOFF(l, sb, n)], &loc_re[l][BOXOFF(l, tb, n)],
                                    &loc_im[l][BOXOFF(l, tb, n)]);
                        }
                        /* FI / BI: source box (si + a, sj -+ b) -> field box (si, sj), a >= 1 */
                        if (a == 0) continue;
                        for (int dir = 0; dir < 2; ++dir) {
                            if (b == 0 && dir == 1) continue;
                            int ti = si, tj = sj;
                            int ui = si + a, uj = dir == 0 ? sj - b : sj + b;
                            if (uj < 0 || uj >= nl) continue;
                            if (!in_s2l_list(ti, tj, ui, uj)) continue;
                            int tb = ti * nl + tj, sb = ui * nl + uj;
                            orc_s2l(Eab + (size_t)n * cube, P, M, 1, dir, &mom_re[l][BOXOFF(l, sb, n)],
                                    &mom_im[l][BOXOFF(l, sb, n)], &loc_re[l][BOXOFF(l, tb, n)],
                                    &loc_im[l][BOXOFF(l, tb, n)]);
                        }
                    }
            }
        }
    }
    free(E);
    /* leaf evaluation: local expansion (Eq. analysis:local) + direct sums over the 3x3
     * neighbour leaves (the D list) */
    int Nw = N < 1 ? 1 : N;
    /* bucket sources by leaf (stable, original order inside a leaf) */
    int64_t nleaf = (int64_t)nside * nside;
    int64_t *cnt = (int64_t *)calloc(nleaf + 1, sizeof(int64_t));
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (ns > 0 ? ns : 1));
    int *sleaf = (int *)malloc(sizeof(int) * (ns > 0 ? ns : 1));
    for (int64_t q = 0; q < ns; ++q) {
        int ir = orc_box_coord(sr[q], r0, L, d), iz = orc_box_coord(sz[q], z0, L, d);
        sleaf[q] = ir * nside + iz;
        cnt[sleaf[q] + 1]++;
    }
    for (int64_t b = 0; b < nleaf; ++b) cnt[b + 1] += cnt[b];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (nleaf + 1));
        memcpy(fill, cnt, sizeof(int64_t) * (nleaf + 1));
        for (int64_t q = 0; q < ns; ++q) ord[fill[sleaf[q]]++] = q;
        free(fill);
    }
    /* field points are independent: one thread per point, private buffers */
#pragma omp parallel
    {
    double pw_r[61], pw_z[61];
    double *G = (double *)malloc(sizeof(double) * (Nw + 1) * 4);
    double *Gr = G + (Nw + 1), *Gx = Gr + (Nw + 1), *Gw = Gx + (Nw + 1);
    double *acc = (double *)malloc(sizeof(double) * nmodes * 6);
#pragma omp for schedule(dynamic, 16)
    for (int64_t j = 0; j < nf; ++j) {
        int ir = orc_box_coord(tr[j], r0, L, d), iz = orc_box_coord(tz[j], z0, L, d);
        int b = ir * nside + iz;
        double cr = r0 + (ir + 0.5) * hd, cz = z0 + (iz + 0.5) * hd;
        double dr = tr[j] - cr, dz = tz[j] - cz;
        pw_r[0] = pw_z[0] = 1.0;
        for (int i = 1; i <= M; ++i) {
            pw_r[i] = pw_r[i - 1] * dr;
            pw_z[i] = pw_z[i - 1] * dz;
        }
        memset(acc, 0, sizeof(double) * nmodes * 6);
        for (int n = 0; n < nmodes; ++n) {
            const double *Fr = &loc_re[d][BOXOFF(d, b, n)], *Fi = &loc_im[d][BOXOFF(d, b, n)];
            for (int k = 0; k <= M; ++k)
                for (int l = 0; k + l <= M; ++l) {
                    double w = pw_r[k] * pw_z[l];
                    acc[6 * n + 0] += Fr[cidx(k, l, M)] * w;
                    acc[6 * n + 1] += Fi[cidx(k, l, M)] * w;
                    if (grad) {
                        if (k >= 1) {
                            double wr = k * pw_r[k - 1] * pw_z[l];
                            acc[6 * n + 2] += Fr[cidx(k, l, M)] * wr;
                            acc[6 * n + 3] += Fi[cidx(k, l, M)] * wr;
                        }
                        if (l >= 1) {
                            double wz = l * pw_r[k] * pw_z[l - 1];
                            acc[6 * n + 4] += Fr[cidx(k, l, M)] * wz;
                            acc[6 * n + 5] += Fi[cidx(k, l, M)] * wz;
                        }
                    }
                }
        }
        for (int a = -1; a <= 1; ++a)
            for (int c = -1; c <= 1; ++c) {
                int ni = ir + a, nj = iz + c;
                if (ni < 0 || nj < 0 || ni >= nside || nj >= nside) continue;
                int nb = ni * nside + nj;
                for (int64_t t = cnt[nb]; t < cnt[nb + 1]; ++t) {
                    int64_t q = ord[t];
                    double x = tz[j] - sz[q];
                    if (grad)
                        orc_green_grad(tr[j], sr[q], x, N, G, Gr, Gx, Gw);
                    else
                        orc_green(tr[j], sr[q], x, N, G);
                    for (int n = 0; n < nmodes; ++n) {
                        double qa = q_re[(size_t)n * ns + q], qb = q_im[(size_t)n * ns + q];
                        acc[6 * n + 0] += qa * G[n];
                        acc[6 * n + 1] += qb * G[n];
                        if (grad) {
                            acc[6 * n + 2] += qa * Gr[n];
                            acc[6 * n + 3] += qb * Gr[n];
                            acc[6 * n + 4] += qa * Gx[n];
                            acc[6 * n + 5] += qb * Gx[n];
                        }
                    }
                }
            }
        for (int n = 0; n < nmodes; ++n) {
            size_t o = (size_t)n * nf + j;
            if (phi_re) phi_re[o] = acc[6 * n + 0];
            if (phi_im) phi_im[o] = acc[6 * n + 1];
            if (grad) {
                dr_re[o] = acc[6 * n + 2];
                dr_im[o] = acc[6 * n + 3];
                dz_re[o] = acc[6 * n + 4];
                dz_im[o] = acc[6 * n + 5];
            }
        }
    }
    free(acc);
    free(G);
    }
    free(cnt);
    free(ord);
    free(sleaf);
    for (int l = 1; l <= d; ++l) {
        free(mom_re[l]);
        free(mom_im[l]);
        free(loc_re[l]);
        free(loc_im[l]);
    }
    free(mom_re);
    free(mom_im);
    free(loc_re);
    free(loc_im);
#undef BOXOFF
    return 0;
}

/* Adjoint of the FMM: the transposed FMM on the same tree (sources and field points
 * exchanged, strengths gphi), giving potential A and gradient B, C at the sources. */
int orc_adjoint_fmm(int64_t ns, const double *sr, const double *sz, int64_t nf, const double *tr,
                    const double *tz, int nmodes, const double *q_re, const double *q_im, const double *gphi_re,
                    const double *gphi_im, int M, int d, const double *geom, double *gq_re, double *gq_im,
                    double *g_r, double *g_z)
{
    size_t m = (size_t)nmodes * ns;
    double *B = (double *)malloc(sizeof(double) * m * 4);
    int rc = orc_fmm(nf, tr, tz, ns, sr, sz, nmodes, gphi_re, gphi_im, M, d, geom, gq_re, gq_im, B, B + m,
                     B + 2 * m, B + 3 * m);
    for (int64_t i = 0; i < ns; ++i) {
        double ar = 0.0, az = 0.0;
        for (int n = 0; n < nmodes; ++n) {
            size_t o = (size_t)n * ns + i;
            ar += q_re[o] * B[o] + q_im[o] * B[m + o];
            az += q_re[o] * B[2 * m + o] + q_im[o] * B[3 * m + o];
        }
        g_r[i] = ar;
        g_z[i] = az;
    }
    free(B);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* The uniform FMM at selected field points only, for checks at sizes where the full     */
/* oracle FMM does not fit in memory or time.                                            */
/* Reading: both truncations are by total degree (i + j <= M, k + l <= M), so the upward  */
/* and downward shifts (Eqs. analysis:shift, analysis:l2l) re-expand polynomials exactly. */
/* The FMM field at a point of leaf b therefore equals, up to rounding, the sum over the  */
/* levels l = 2..d of the level-l ancestor's local expansion built from that level's S2L  */
/* alone (Eq. analysis:s2l over the interaction list, from the source boxes' moments      */
/* about their level-l centres, Eq. analysis:moments) and evaluated at the point          */
/* (Eq. analysis:local), plus the direct sum over the 3x3 neighbour leaves.  The tests    */
/* check that this equals orc_fmm at every point where both run.                          */
/* samples[s] indexes the field points; outputs are [nmodes][nsamp].                      */
/* ------------------------------------------------------------------------------------ */

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y);
}

int orc_fmm_sampled(int64_t ns, const double *sr, const double *sz, int64_t nf, const double *tr,
                    const double *tz, int nmodes, const double *q_re, const double *q_im, int M, int d,
                    const double *geom, int64_t nsamp, const int64_t *samples, double *phi_re,
                    double *phi_im, double *dr_re, double *dr_im, double *dz_re, double *dz_im)
{
    if (d < 2 || M > 60 || nsamp < 0) return -1;
    for (int64_t s = 0; s < nsamp; ++s)
        if (samples[s] < 0 || samples[s] >= nf) return -1;
    binom_init();
    int N = nmodes - 1;
    int P = 2 * M;
    int nc = (M + 1) * (M + 2) / 2;
    int grad = dr_re != NULL;
    double r0 = geom[0], z0 = geom[1], L = geom[2];
    int nside = 1 << d;
    size_t cube = (size_t)(P + 1) * (P + 1) * (P + 1);
    /* bucket sources by leaf (stable, original order inside a leaf) */
    int64_t nleaf = (int64_t)nside * nside;
    int64_t *cnt = (int64_t *)calloc(nleaf + 1, sizeof(int64_t));
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (ns > 0 ? ns : 1));
    int *sleaf = (int *)malloc(sizeof(int) * (ns > 0 ? ns : 1));
    if (!cnt || !ord || !sleaf) return -2;
    for (int64_t q = 0; q < ns; ++q) {
        int ir = orc_box_coord(sr[q], r0, L, d), iz = orc_box_coord(sz[q], z0, L, d);
        sleaf[q] = ir * nside + iz;
        cnt[sleaf[q] + 1]++;
    }
    for (int64_t b = 0; b < nleaf; ++b) cnt[b + 1] += cnt[b];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (nleaf + 1));
        memcpy(fill, cnt, sizeof(int64_t) * (nleaf + 1));
        for (int64_t q = 0; q < ns; ++q) ord[fill[sleaf[q]]++] = q;
        free(fill);
    }
    /* per level: the source boxes of the samples' interaction lists and their moments */
    int64_t *nbx = (int64_t *)calloc(d + 1, sizeof(int64_t));
    int64_t **bx = (int64_t **)calloc(d + 1, sizeof(int64_t *));
    double **bm_re = (double **)calloc(d + 1, sizeof(double *));
    double **bm_im = (double **)calloc(d + 1, sizeof(double *));
    for (int l = 2; l <= d; ++l) {
        int nl = 1 << l, sh = d - l;
        int64_t *lst = (int64_t *)malloc(sizeof(int64_t) * (nsamp * 36 + 1));
        int64_t m = 0;
        for (int64_t s = 0; s < nsamp; ++s) {
            int64_t j = samples[s];
            int ti = orc_box_coord(tr[j], r0, L, d) >> sh, tj = orc_box_coord(tz[j], z0, L, d) >> sh;
            for (int ui = 2 * (ti / 2) - 2; ui <= 2 * (ti / 2) + 3; ++ui)
                for (int uj = 2 * (tj / 2) - 2; uj <= 2 * (tj / 2) + 3; ++uj) {
                    if (ui < 0 || uj < 0 || ui >= nl || uj >= nl) continue;
                    if (!in_s2l_list(ti, tj, ui, uj)) continue;
                    lst[m++] = (int64_t)ui * nl + uj;
                }
        }
        qsort(lst, (size_t)m, sizeof(int64_t), cmp_i64);
        int64_t u = 0;
        for (int64_t t = 0; t < m; ++t)
            if (t == 0 || lst[t] != lst[t - 1]) lst[u++] = lst[t];
        nbx[l] = u;
        bx[l] = lst;
        bm_re[l] = (double *)calloc((size_t)(u > 0 ? u : 1) * nmodes * nc, sizeof(double));
        bm_im[l] = (double *)calloc((size_t)(u > 0 ? u : 1) * nmodes * nc, sizeof(double));
        if (!bm_re[l] || !bm_im[l]) return -2;
        double h = L / nl;
        /* moments of each listed box about its level-l centre, one thread per (box, mode) */
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
        for (int64_t t = 0; t < u; ++t)
            for (int n = 0; n < nmodes; ++n) {
                int bi = (int)(bx[l][t] / nl), bj = (int)(bx[l][t] % nl);
                double cr = r0 + (bi + 0.5) * h, cz = z0 + (bj + 0.5) * h;
                double *mre = bm_re[l] + ((size_t)t * nmodes + n) * nc;
                double *mim = bm_im[l] + ((size_t)t * nmodes + n) * nc;
                double pw_r[61], pw_z[61];
                for (int ir = bi << sh; ir < (bi + 1) << sh; ++ir) {
                    int64_t lo = cnt[(int64_t)ir * nside + ((int64_t)bj << sh)];
                    int64_t hi = cnt[(int64_t)ir * nside + ((int64_t)(bj + 1) << sh)];
                    for (int64_t k = lo; k < hi; ++k) {
                        int64_t q = ord[k];
                        double dr = sr[q] - cr, dz = sz[q] - cz;
                        pw_r[0] = pw_z[0] = 1.0;
                        for (int i = 1; i <= M; ++i) {
                            pw_r[i] = pw_r[i - 1] * dr;
                            pw_z[i] = pw_z[i - 1] * dz;
                        }
                        double a = q_re[(size_t)n * ns + q], bb = q_im[(size_t)n * ns + q];
                        for (int i = 0; i <= M; ++i)
                            for (int jj = 0; i + jj <= M; ++jj) {
                                double w = pw_r[i] * pw_z[jj];
                                mre[cidx(i, jj, M)] += a * w;
                                mim[cidx(i, jj, M)] += bb * w;
                            }
                    }
                }
            }
    }
    /* per (sample, level): S2L of that level into the ancestor's local expansion, evaluated
     * at the sample; level d + 1 stands for the near-field sum over the 3x3 leaves */
    int nlev = d + 2;
    double *res = (double *)calloc((size_t)(nsamp > 0 ? nsamp : 1) * nlev * nmodes * 6, sizeof(double));
    if (!res) return -2;
    int fail = 0;
#pragma omp parallel reduction(|: fail)
    {
        double *E = (double *)malloc(sizeof(double) * cube * nmodes);
        double *F = (double *)malloc(sizeof(double) * 2 * (size_t)nmodes * nc);
        int Nw = N < 1 ? 1 : N;
        double *G = (double *)malloc(sizeof(double) * (Nw + 1) * 4);
        double *Gr = G + (Nw + 1), *Gx = Gr + (Nw + 1), *Gw = Gx + (Nw + 1);
        if (!E || !F || !G) fail = 1;
#pragma omp for schedule(dynamic, 1) collapse(2)
        for (int64_t s = 0; s < nsamp; ++s)
            for (int l = 2; l <= d + 1; ++l) {
                if (fail) continue;
                int64_t j = samples[s];
                double *acc = res + ((size_t)s * nlev + l) * nmodes * 6;
                int ir = orc_box_coord(tr[j], r0, L, d), iz = orc_box_coord(tz[j], z0, L, d);
                if (l == d + 1) {
                    for (int a = -1; a <= 1; ++a)
                        for (int c = -1; c <= 1; ++c) {
                            int ni = ir + a, nj = iz + c;
                            if (ni < 0 || nj < 0 || ni >= nside || nj >= nside) continue;
                            int64_t nb = (int64_t)ni * nside + nj;
                            for (int64_t t = cnt[nb]; t < cnt[nb + 1]; ++t) {
                                int64_t q = ord[t];
                                double x = tz[j] - sz[q];
                                if (grad)
                                    orc_green_grad(tr[j], sr[q], x, N, G, Gr, Gx, Gw);
                                else
                                    orc_green(tr[j], sr[q], x, N, G);
                                for (int n = 0; n < nmodes; ++n) {
                                    double qa = q_re[(size_t)n * ns + q], qb = q_im[(size_t)n * ns + q];
                                    acc[6 * n + 0] += qa * G[n];
                                    acc[6 * n + 1] += qb * G[n];
                                    if (grad) {
                                        acc[6 * n + 2] += qa * Gr[n];
                                        acc[6 * n + 3] += qb * Gr[n];
                                        acc[6 * n + 4] += qa * Gx[n];
                                        acc[6 * n + 5] += qb * Gx[n];
                                    }
                                }
                            }
                        }
                    continue;
                }
                int nl = 1 << l, sh = d - l;
                double h = L / nl;
                int ti = ir >> sh, tj = iz >> sh;
                memset(F, 0, sizeof(double) * 2 * (size_t)nmodes * nc);
                for (int ui = 2 * (ti / 2) - 2; ui <= 2 * (ti / 2) + 3; ++ui)
                    for (int uj = 2 * (tj / 2) - 2; uj <= 2 * (tj / 2) + 3; ++uj) {
                        if (ui < 0 || uj < 0 || ui >= nl || uj >= nl) continue;
                        if (!in_s2l_list(ti, tj, ui, uj)) continue;
                        int64_t key = (int64_t)ui * nl + uj;
                        int64_t *hit = (int64_t *)bsearch(&key, bx[l], (size_t)nbx[l], sizeof(int64_t), cmp_i64);
                        int64_t t = hit - bx[l];
                        /* the field box at the larger radius: FO/BO with E_{k,i,j+l}; at the
                         * smaller radius: FI/BI with E_{i,k,j+l}; field box below: backward */
                        int inward = ti < ui, backward = tj < uj;
                        int lo = ti < ui ? ti : ui, hi = ti < ui ? ui : ti;
                        int b = abs(tj - uj);
                        double rb = r0 + (hi + 0.5) * h, rs = r0 + (lo + 0.5) * h;
                        if (orc_gbar(rb, rs, b * h, N, P, E) != 0) {
                            fail = 1;
                            continue;
                        }
                        for (int n = 0; n < nmodes; ++n)
                            orc_s2l(E + (size_t)n * cube, P, M, inward, backward,
                                    bm_re[l] + ((size_t)t * nmodes + n) * nc, bm_im[l] + ((size_t)t * nmodes + n) * nc,
                                    F + (size_t)n * nc, F + (size_t)(nmodes + n) * nc);
                    }
                double dr = tr[j] - (r0 + (ti + 0.5) * h), dz = tz[j] - (z0 + (tj + 0.5) * h);
                double pw_r[61], pw_z[61];
                pw_r[0] = pw_z[0] = 1.0;
                for (int i = 1; i <= M; ++i) {
                    pw_r[i] = pw_r[i - 1] * dr;
                    pw_z[i] = pw_z[i - 1] * dz;
                }
                for (int n = 0; n < nmodes; ++n) {
                    const double *Fr = F + (size_t)n * nc, *Fi = F + (size_t)(nmodes + n) * nc;
                    for (int k = 0; k <= M; ++k)
                        for (int ll = 0; k + ll <= M; ++ll) {
                            double w = pw_r[k] * pw_z[ll];
                            acc[6 * n + 0] += Fr[cidx(k, ll, M)] * w;
                            acc[6 * n + 1] += Fi[cidx(k, ll, M)] * w;
                            if (grad) {
                                if (k >= 1) {
                                    double wr = k * pw_r[k - 1] * pw_z[ll];
                                    acc[6 * n + 2] += Fr[cidx(k, ll, M)] * wr;
                                    acc[6 * n + 3] += Fi[cidx(k, ll, M)] * wr;
                                }
                                if (ll >= 1) {
                                    double wz = ll * pw_r[k] * pw_z[ll - 1];
                                    acc[6 * n + 4] += Fr[cidx(k, ll, M)] * wz;
                                    acc[6 * n + 5] += Fi[cidx(k, ll, M)] * wz;
                                }
                            }
                        }
                }
            }
        free(E);
        free(F);
        free(G);
    }
    /* the levels' contributions in level order, then the near field */
    for (int64_t s = 0; s < nsamp; ++s)
        for (int n = 0; n < nmodes; ++n) {
            double v[6] = {0, 0, 0, 0, 0, 0};
            for (int l = 2; l <= d + 1; ++l)
                for (int c = 0; c < 6; ++c) v[c] += res[((size_t)s * nlev + l) * nmodes * 6 + 6 * n + c];
            size_t o = (size_t)n * nsamp + s;
            if (phi_re) phi_re[o] = v[0];
            if (phi_im) phi_im[o] = v[1];
            if (grad) {
                dr_re[o] = v[2];
                dr_im[o] = v[3];
                dz_re[o] = v[4];
                dz_im[o] = v[5];
            }
        }
    free(res);
    for (int l = 2; l <= d; ++l) {
        free(bx[l]);
        free(bm_re[l]);
        free(bm_im[l]);
    }
    free(nbx);
    free(bx);
    free(bm_re);
    free(bm_im);
    free(cnt);
    free(ord);
    free(sleaf);
    return fail ? -2 : 0;
}

/* Adjoint of the FMM at selected sources: the sampled FMM of the transposed problem
 * (field points as sources with strengths gphi, evaluated at the sources samples[s]),
 * then gq = A, dL/dr = sum_n Re(q conj B), dL/dz = sum_n Re(q conj C) there.
 * Outputs gq [nmodes][nsamp], g_r, g_z [nsamp]. */
int orc_adjoint_fmm_sampled(int64_t ns, const double *sr, const double *sz, int64_t nf, const double *tr,
                            const double *tz, int nmodes, const double *q_re, const double *q_im,
                            const double *gphi_re, const double *gphi_im, int M, int d, const double *geom,
                            int64_t nsamp, const int64_t *samples, double *gq_re, double *gq_im, double *g_r,
                            double *g_z)
{
    size_t m = (size_t)nmodes * (nsamp > 0 ? nsamp : 1);
    double *B = (double *)malloc(sizeof(double) * m * 4);
    if (!B) return -2;
    int rc = orc_fmm_sampled(nf, tr, tz, ns, sr, sz, nmodes, gphi_re, gphi_im, M, d, geom, nsamp, samples, gq_re,
                             gq_im, B, B + m, B + 2 * m, B + 3 * m);
    for (int64_t s = 0; s < nsamp; ++s) {
        int64_t i = samples[s];
        double ar = 0.0, az = 0.0;
        for (int n = 0; n < nmodes; ++n) {
            size_t o = (size_t)n * ns + i, u = (size_t)n * nsamp + s;
            ar += q_re[o] * B[u] + q_im[o] * B[m + u];
            az += q_re[o] * B[2 * m + u] + q_im[o] * B[3 * m + u];
        }
        g_r[s] = ar;
        g_z[s] = az;
    }
    free(B);
    return rc;
}

/* Counts of the uniform tree's work, from the definitions of Sec. 2.2: a box of level l
 * is present when it holds a source or a field point; out[0] = (field point, source)
 * pairs of the near field (3x3 neighbour leaves), out[1] = (field box, source box) pairs
 * of the interaction lists of levels 2..d with both boxes present, out[2] = the
 * (field point, source) pairs those box pairs stand for.  Every pair of points is then
 * counted exactly once: out[0] + out[2] = ns nf. */
int orc_tree_counts(int64_t ns, const double *sr, const double *sz, int64_t nf, const double *tr,
                    const double *tz, int d, const double *geom, int64_t *out)
{
    if (d < 2 || d > 14) return -1;
    double r0 = geom[0], z0 = geom[1], L = geom[2];
    out[0] = out[1] = out[2] = 0;
    for (int l = 2; l <= d; ++l) {
        int nl = 1 << l;
        int64_t nb = (int64_t)nl * nl;
        int64_t *cs = (int64_t *)calloc(nb, sizeof(int64_t));
        int64_t *ct = (int64_t *)calloc(nb, sizeof(int64_t));
        if (!cs || !ct) return -2;
        for (int64_t q = 0; q < ns; ++q)
            cs[(int64_t)orc_box_coord(sr[q], r0, L, l) * nl + orc_box_coord(sz[q], z0, L, l)]++;
        for (int64_t j = 0; j < nf; ++j)
            ct[(int64_t)orc_box_coord(tr[j], r0, L, l) * nl + orc_box_coord(tz[j], z0, L, l)]++;
        for (int ti = 0; ti < nl; ++ti)
            for (int tj = 0; tj < nl; ++tj) {
                int64_t tb = (int64_t)ti * nl + tj;
                if (cs[tb] + ct[tb] == 0) continue;
                for (int ui = 2 * (ti / 2) - 2; ui <= 2 * (ti / 2) + 3; ++ui)
                    for (int uj = 2 * (tj / 2) - 2; uj <= 2 * (tj / 2) + 3; ++uj) {
                        if (ui < 0 || uj < 0 || ui >= nl || uj >= nl) continue;
                        int64_t ub = (int64_t)ui * nl + uj;
                        if (cs[ub] + ct[ub] == 0 || !in_s2l_list(ti, tj, ui, uj)) continue;
                        out[1] += 1;
                        out[2] += ct[tb] * cs[ub];
                    }
                if (l == d)
                    for (int a = -1; a <= 1; ++a)
                        for (int c = -1; c <= 1; ++c) {
                            int ni = ti + a, nj = tj + c;
                            if (ni < 0 || nj < 0 || ni >= nl || nj >= nl) continue;
                            out[0] += ct[tb] * cs[(int64_t)ni * nl + nj];
                        }
            }
        free(cs);
        free(ct);
    }
    return 0;
}

/* ---- Fourier analysis and synthesis in the azimuth (Sec. 2, Eqs. analysis:source and
 * analysis:phi).  s(theta) = sum_{n=-N..N} S^(n) e^{i n theta} with S^(-n) = conj(S^(n)) for a
 * real density, and phi(theta) = sum_n Phi^(n) e^{i n theta}.  Reading: the paper's
 * intermediate step writes e^{-i n theta}; substituting u = theta_1 - theta in the ring
 * integral gives the final e^{+i n theta} of Eq. analysis:phi, which is used.
 * Analysis from K equispaced samples theta_k = 2 pi k / K (exact for K >= 2N + 1):
 *   S^(n) = (1/K) sum_k s(theta_k) e^{-i n theta_k},  n = 0..n_modes-1.
 * Synthesis at the same angles:  phi(theta_k) = Re Phi^(0) + 2 sum_{n>=1} Re(Phi^(n) e^{i n theta_k}).
 * Layouts: samples [K][npts] (angle-major), coefficients [n_modes][npts].  Sums are plain
 * Neumaier-compensated loops over k (analysis) and n (synthesis). */
static void neumaier(double *s, double *c, double v)
{
    double t = *s + v;
    if (fabs(*s) >= fabs(v))
        *c += (*s - t) + v;
    else
        *c += (v - t) + *s;
    *s = t;
}

void orc_fourier_analysis(int64_t npts, int K, const double *samples, int n_modes, double *S_re, double *S_im)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npts; ++p)
        for (int n = 0; n < n_modes; ++n) {
            double ar = 0, cr = 0, ai = 0, ci = 0;
            for (int k = 0; k < K; ++k) {
                /* angle n theta_k reduced exactly: (n k mod K) / K of a turn */
                double th = 2.0 * ORC_PI * (double)(((int64_t)n * k) % K) / (double)K;
                double v = samples[(size_t)k * npts + p];
                neumaier(&ar, &cr, v * cos(th));
                neumaier(&ai, &ci, -v * sin(th));
            }
            S_re[(size_t)n * npts + p] = (ar + cr) / K;
            S_im[(size_t)n * npts + p] = (ai + ci) / K;
        }
}

void orc_fourier_synthesis(int64_t npts, int n_modes, const double *P_re, const double *P_im, int K, double *phi)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npts; ++p)
        for (int k = 0; k < K; ++k) {
            double a = P_re[p], c = 0;
            for (int n = 1; n < n_modes; ++n) {
                double th = 2.0 * ORC_PI * (double)(((int64_t)n * k) % K) / (double)K;
                neumaier(&a, &c, 2.0 * (P_re[(size_t)n * npts + p] * cos(th) - P_im[(size_t)n * npts + p] * sin(th)));
            }
            phi[(size_t)k * npts + p] = a + c;
        }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
