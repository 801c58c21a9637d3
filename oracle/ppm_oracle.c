/*
 * ppm_oracle.c -- FP64 CPU oracle of the energy-resolved pulse-profile
 * forward model and Poisson likelihood of Zhou & Huang, "GPU-accelerated
 * X-ray pulse profile modeling" (arXiv 2510.07764).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * reference that the CUDA path is checked against.  It is called only by the
 * test-suite, by the smoke check and by the CPU-baseline leg of the
 * benchmark; the library's product path never links, loads or calls it.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Everything is double precision, single threaded, in the order of the
 * paper's computation recipe (Sect. 2.8):
 *   light bending + time delay integrals  .... Sect. 2.3, Eqs. salmi_lf,
 *                                              salmi_td, rho, tot_time_delay
 *   lens-table generation ................... Sect. 2.8.2
 *   star shape, slope, gravity .............. Sect. 2.1-2.2, Eqs. def_f,
 *                                              Rtheta, Omega_c_def, area_oblate
 *   Doppler / aberration .................... Sect. 2.4, App. A
 *   per-ring pseudo-patch template .......... Sect. 2.8.3 (steps 1-5)
 *   invisible-segment fill .................. Sect. 2.8.3
 *   shift-and-add ........................... Sect. 2.8.3, Eq. add_Ft
 *   flux formula ............................ Sect. 2.5, App. C
 *   mixed-order atmosphere interpolation .... Sect. 4
 *   ISM, response ........................... Sect. 2.7, 2.8.4
 *   Poisson log-likelihood .................. Sect. 5 (Eq. chi2_def context), Sect. 6
 *
 * Where the paper is silent the reading is stated next to the code.
 * Compile with -ffp-contract=off so x86 and Arm builds round identically.
 *
 * Forward-mode derivatives.  Everything downstream of the parameters is
 * written in the type `real`.  The ordinary build has real = double.  The
 * tangent build (ppm_oracle_tangent.c: ORC_CSTEP defined, then this file
 * included) has real = double complex and seeds a parameter p as
 * p + i h v_p with h ~ 1e-20 |p|: the imaginary parts then carry h times
 * the directional derivative along v, exactly to rounding, because every
 * product of two imaginary parts (order h^2) vanishes against the real parts
 * (the complex-step method of Squire & Trapp 1998; Martins, Sturdza & Alonso
 * 2003).  Elementary functions take their first-order expansion
 * f(a + ib) = f(a) + i b f'(a); branches, comparisons, floors and clamps act
 * on the real part only, so the derivative is that of the same
 * piecewise-smooth function the ordinary build evaluates.  The lens tables
 * and the quadrature do not depend on the parameters and stay double.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef ORC_CSTEP
#include <complex.h>
#undef I /* the imaginary unit macro; this file names intensities I */
typedef double complex real;
static double RE(real x) { return creal(x); }
static double IM(real x) { return cimag(x); }
static real mk(double a, double b) { return CMPLX(a, b); }
static real r_sqrt(real x)
{
    double a = creal(x), s = sqrt(a);
    return mk(s, s > 0.0 ? cimag(x) * 0.5 / s : 0.0);
}
static real r_sin(real x) { return mk(sin(creal(x)), cimag(x) * cos(creal(x))); }
static real r_cos(real x) { return mk(cos(creal(x)), -cimag(x) * sin(creal(x))); }
static real r_acos(real x)
{
    double a = creal(x);
    return mk(acos(a), -cimag(x) / sqrt(1.0 - a * a));
}
static real r_log(real x) { return mk(log(creal(x)), cimag(x) / creal(x)); }
static real r_log10(real x) { return mk(log10(creal(x)), cimag(x) / (creal(x) * log(10.0))); }
static real r_exp(real x)
{
    double e = exp(creal(x));
    return mk(e, cimag(x) * e);
}
static real r_expm1(real x) { return mk(expm1(creal(x)), cimag(x) * exp(creal(x))); }
static real r_pow(double base, real x)
{
    double v = pow(base, creal(x));
    return mk(v, cimag(x) * v * log(base));
}
static real r_fabs(real x) { return creal(x) < 0.0 ? -x : x; }
#else
typedef double real;
#define RE(x) (x)
#define IM(x) (0.0)
#define r_sqrt sqrt
#define r_sin sin
#define r_cos cos
#define r_acos acos
#define r_log log
#define r_log10 log10
#define r_exp exp
#define r_expm1 expm1
#define r_pow pow
#define r_fabs fabs
#endif

/* ---- physical constants (CODATA 2018, IAU 2015 nominal GM_sun) ---- */
#define ORC_PI 3.14159265358979323846
static const double GM_SUN = 1.32712440018e20;      /* m^3 s^-2 */
static const double C_MS = 299792458.0;             /* m s^-1 */
static const double C_CMS = 29979245800.0;          /* cm s^-1 */
static const double H_KEVS = 4.135667696e-18;       /* keV s */
static const double KB_KEVK = 8.617333262e-8;       /* keV K^-1 */
static const double KPC_M = 3.0856775814913673e19;  /* m */

/* =====================================================================
 * Adaptive Gauss-Kronrod (7,15) quadrature
 * ===================================================================== */
typedef double (*orc_fn)(double x, const void *ctx);

static const double XGK[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.0};
static const double WGK[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double WG7[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

static void gk15(orc_fn f, const void *ctx, double a, double b, double *res, double *err)
{
    double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double fc = f(c, ctx);
    double rk = fc * WGK[7], rg = fc * WG7[3];
    for (int j = 0; j < 7; j++) {
        double dx = h * XGK[j];
        double f1 = f(c - dx, ctx), f2 = f(c + dx, ctx);
        rk += WGK[j] * (f1 + f2);
        if (j % 2 == 1) rg += WG7[j / 2] * (f1 + f2);
    }
    *res = rk * h;
    *err = fabs((rk - rg) * h);
}

static double adapt(orc_fn f, const void *ctx, double a, double b, double whole,
                    double tol, int depth)
{
    double r, e;
    gk15(f, ctx, a, b, &r, &e);
    if (e <= tol || depth >= 48 || (b - a) < 1e-15 * (1.0 + fabs(a))) return r;
    double m = 0.5 * (a + b);
    return adapt(f, ctx, a, m, whole, 0.5 * tol, depth + 1) +
           adapt(f, ctx, m, b, whole, 0.5 * tol, depth + 1);
}

/* integral over [a, b] to ~1e-14 relative */
static double integrate(orc_fn f, const void *ctx, double a, double b)
{
    double r, e;
    gk15(f, ctx, a, b, &r, &e);
    double tol = 1e-14 * fabs(r) + 1e-300;
    if (e <= tol) return r;
    double m = 0.5 * (a + b);
    return adapt(f, ctx, a, m, r, 0.5 * tol, 1) + adapt(f, ctx, m, b, r, 0.5 * tol, 1);
}

/* =====================================================================
 * Light bending and time delay (Sect. 2.3, 2.8.2)
 * ===================================================================== */
typedef struct { double u, c2, s2; } bend_ctx;

/* q(x) = [2 - x^2 - u (1-x^2)^2 / (1-u)] sin^2(alpha)   (Eq. under salmi_lf) */
static double bend_q(double x, const bend_ctx *b)
{
    double y = 1.0 - x * x;
    return (2.0 - x * x - b->u * y * y / (1.0 - b->u)) * b->s2;
}

static double psi_integrand(double x, const void *p)
{
    const bend_ctx *b = (const bend_ctx *)p;
    return x / sqrt(b->c2 + x * x * bend_q(x, b));
}

static double td_integrand(double x, const void *p)
{
    const bend_ctx *b = (const bend_ctx *)p;
    double w = sqrt(b->c2 + x * x * bend_q(x, b));
    return x / (w * (1.0 + w));
}

/* integrate on [0,1] with extra break points near x ~ |cos alpha| where the
 * integrand turns over for near-grazing rays */
static double bend_integral(orc_fn f, const bend_ctx *b)
{
    double c = sqrt(b->c2);
    double brk[4];
    int nb = 0;
    brk[nb++] = 0.0;
    if (c > 0.0 && c < 0.1) {
        brk[nb++] = c;
        if (10.0 * c < 0.5) brk[nb++] = 10.0 * c;
    }
    brk[nb++] = 1.0;
    double s = 0.0;
    for (int i = 0; i + 1 < nb; i++) s += integrate(f, b, brk[i], brk[i + 1]);
    return s;
}

/* Eq. salmi_lf: bending angle psi(u, alpha) of an outgoing ray, alpha <= pi/2 */
double orc_psi_out(double u, double alpha)
{
    double s = sin(alpha), c = cos(alpha);
    if (s == 0.0) return 0.0;
    bend_ctx b = {u, c * c, s * s};
    return 2.0 * s / sqrt(1.0 - u) * bend_integral(psi_integrand, &b);
}

/* Eq. salmi_td: c Delta t_p / R of an outgoing ray, alpha <= pi/2 */
double orc_td_out(double u, double alpha)
{
    double s = sin(alpha), c = cos(alpha);
    if (s == 0.0) return 0.0;
    bend_ctx b = {u, c * c, s * s};
    return 2.0 * s * s / (1.0 - u) * bend_integral(td_integrand, &b);
}

/* Eq. rho: periastron radius / R of an inward ray (alpha > pi/2).
 * Returns NaN when the arccos argument exceeds 1 (ray captured; reading). */
double orc_rho(double u, double alpha)
{
    double s = sin(alpha);
    double k = sqrt(3.0 * (1.0 - u));
    double arg = 3.0 * u * k / (2.0 * s);
    if (!(arg <= 1.0)) return NAN;
    return -2.0 * s / k * cos((acos(arg) + 2.0 * ORC_PI) / 3.0);
}

/* psi(u, alpha) for any alpha: inward rays use 2 psi(u/rho, pi/2) - psi(u, pi-alpha) */
double orc_psi(double u, double alpha)
{
    if (alpha <= 0.5 * ORC_PI) return orc_psi_out(u, alpha);
    double rho = orc_rho(u, alpha);
    if (isnan(rho)) return NAN;
    return 2.0 * orc_psi_out(u / rho, 0.5 * ORC_PI) - orc_psi_out(u, ORC_PI - alpha);
}

/* c Delta t / R for any alpha.  Inward rays (reading of Eq. tot_time_delay):
 * the periastron leg Delta t_p(u_p, pi/2) is measured in units of R_p = rho R,
 * and the radial-delay difference 2[delta t(R_p) - delta t(R)] is folded into
 * the table so that the run-time delay is (R/c) TD + delta t(R) for every ray:
 *   TD = 2 rho TDp(u/rho, pi/2) - TDp(u, pi - alpha)
 *        + 2 [(1 - rho) + u ln((1 - u) / (rho - u))].                        */
double orc_td(double u, double alpha)
{
    if (alpha <= 0.5 * ORC_PI) return orc_td_out(u, alpha);
    double rho = orc_rho(u, alpha);
    if (isnan(rho)) return NAN;
    return 2.0 * rho * orc_td_out(u / rho, 0.5 * ORC_PI) - orc_td_out(u, ORC_PI - alpha) +
           2.0 * ((1.0 - rho) + u * log((1.0 - u) / (rho - u)));
}

/* =====================================================================
 * Lens tables C_alpha, LF on (u, cos psi) and TD on (u, cos alpha)
 * (Sect. 2.8.2)
 * ===================================================================== */
typedef struct {
    double u_min, u_max; int n_u;
    double cpsi_min, cpsi_max; int n_cpsi;
    double calpha_min, calpha_max; int n_calpha;
    double dalpha;
} orc_lens_spec;

typedef struct {
    orc_lens_spec spec;
    const double *Ca;  /* [n_u][n_cpsi] cos alpha, NaN = not reached */
    const double *LF;  /* [n_u][n_cpsi] d cos alpha / d cos psi */
    const double *TD;  /* [n_u][n_calpha] c Delta t / R, NaN = captured */
} orc_lens;

/* Linspace(x_min, x_max, n)[i] */
static double linspace_at(double lo, double hi, int n, int i)
{
    return lo + (hi - lo) * (double)i / (double)(n - 1);
}

/* Build the three tables.  For each u: march alpha = 0, dalpha, 2 dalpha, ...
 * appending (alpha, psi) until psi > arccos(cpsi_min); the march also stops
 * (reading) when the ray is captured or psi would pass pi.  Convert to
 * (cos psi, cos alpha); d cos alpha / d cos psi by central differences on the
 * list (one-sided at the two ends, reading); linear interpolation of both
 * lists onto the cos psi grid (reading); grid points beyond the march are NaN.
 * TD is evaluated directly at every (u, cos alpha) grid point.
 * Returns the longest march length, or -1 on bad input. */
int orc_lens_build(const orc_lens_spec *sp, double *Ca, double *LF, double *TD)
{
    if (sp->n_u < 2 || sp->n_cpsi < 2 || sp->n_calpha < 2 || !(sp->dalpha > 0.0)) return -1;
    int cap = (int)(ORC_PI / sp->dalpha) + 4;
    double *lp = (double *)malloc(sizeof(double) * cap);
    double *la = (double *)malloc(sizeof(double) * cap);
    double *ld = (double *)malloc(sizeof(double) * cap);
    double psi_stop = acos(sp->cpsi_min);
    int longest = 0;
    for (int iu = 0; iu < sp->n_u; iu++) {
        double u = linspace_at(sp->u_min, sp->u_max, sp->n_u, iu);
        int n = 0;
        for (int j = 0; j < cap; j++) {
            double alpha = j * sp->dalpha;
            if (alpha > ORC_PI) break;
            double psi = orc_psi(u, alpha);
            if (isnan(psi) || psi > ORC_PI) break;
            lp[n] = cos(psi);
            la[n] = cos(alpha);
            n++;
            if (psi > psi_stop) break;
        }
        if (n > longest) longest = n;
        for (int j = 0; j < n; j++) {
            int a = j > 0 ? j - 1 : j, b = j < n - 1 ? j + 1 : j;
            ld[j] = (b > a) ? (la[b] - la[a]) / (lp[b] - lp[a]) : NAN;
        }
        for (int ic = 0; ic < sp->n_cpsi; ic++) {
            double cp = linspace_at(sp->cpsi_min, sp->cpsi_max, sp->n_cpsi, ic);
            double *ca = &Ca[(size_t)iu * sp->n_cpsi + ic];
            double *lf = &LF[(size_t)iu * sp->n_cpsi + ic];
            if (n < 2 || cp < lp[n - 1]) { *ca = NAN; *lf = NAN; continue; }
            /* lp is decreasing: find j with lp[j] >= cp >= lp[j+1] */
            int lo = 0, hi = n - 1;
            while (hi - lo > 1) {
                int mid = (lo + hi) / 2;
                if (lp[mid] >= cp) lo = mid; else hi = mid;
            }
            double w = (cp - lp[lo]) / (lp[hi] - lp[lo]);
            *ca = la[lo] + w * (la[hi] - la[lo]);
            *lf = ld[lo] + w * (ld[hi] - ld[lo]);
        }
        for (int ia = 0; ia < sp->n_calpha; ia++) {
            double ca = linspace_at(sp->calpha_min, sp->calpha_max, sp->n_calpha, ia);
            TD[(size_t)iu * sp->n_calpha + ia] = orc_td(u, acos(ca));
        }
    }
    free(lp); free(la); free(ld);
    return longest;
}

/* Bilinear lookup of C_alpha and LF at (u, cos psi) (reading: bilinear).
 * Returns 1 if all four corners are valid, 0 otherwise (point invisible). */
int orc_lens_lookup(const orc_lens *L, real u, real cpsi, real *ca, real *lf)
{
    const orc_lens_spec *s = &L->spec;
    real fu = (u - s->u_min) / (s->u_max - s->u_min) * (s->n_u - 1);
    real fc = (cpsi - s->cpsi_min) / (s->cpsi_max - s->cpsi_min) * (s->n_cpsi - 1);
    int iu = (int)floor(RE(fu)), ic = (int)floor(RE(fc));
    if (iu < 0) iu = 0;
    if (iu > s->n_u - 2) iu = s->n_u - 2;
    if (ic < 0) ic = 0;
    if (ic > s->n_cpsi - 2) ic = s->n_cpsi - 2;
    real tu = fu - iu, tc = fc - ic;
    size_t k00 = (size_t)iu * s->n_cpsi + ic, k10 = k00 + s->n_cpsi;
    double a00 = L->Ca[k00], a01 = L->Ca[k00 + 1], a10 = L->Ca[k10], a11 = L->Ca[k10 + 1];
    double d00 = L->LF[k00], d01 = L->LF[k00 + 1], d10 = L->LF[k10], d11 = L->LF[k10 + 1];
    if (isnan(a00) || isnan(a01) || isnan(a10) || isnan(a11)) return 0;
    *ca = (1.0 - tu) * ((1.0 - tc) * a00 + tc * a01) + tu * ((1.0 - tc) * a10 + tc * a11);
    *lf = (1.0 - tu) * ((1.0 - tc) * d00 + tc * d01) + tu * ((1.0 - tc) * d10 + tc * d11);
    return 1;
}

/* Bilinear lookup of TD at (u, cos alpha); cos alpha is clamped to the grid. */
real orc_td_lookup(const orc_lens *L, real u, real calpha)
{
    const orc_lens_spec *s = &L->spec;
    if (RE(calpha) < s->calpha_min) calpha = s->calpha_min;
    if (RE(calpha) > s->calpha_max) calpha = s->calpha_max;
    real fu = (u - s->u_min) / (s->u_max - s->u_min) * (s->n_u - 1);
    real fc = (calpha - s->calpha_min) / (s->calpha_max - s->calpha_min) * (s->n_calpha - 1);
    int iu = (int)floor(RE(fu)), ic = (int)floor(RE(fc));
    if (iu < 0) iu = 0;
    if (iu > s->n_u - 2) iu = s->n_u - 2;
    if (ic < 0) ic = 0;
    if (ic > s->n_calpha - 2) ic = s->n_calpha - 2;
    real tu = fu - iu, tc = fc - ic;
    size_t k00 = (size_t)iu * s->n_calpha + ic, k10 = k00 + s->n_calpha;
    return (1.0 - tu) * ((1.0 - tc) * L->TD[k00] + tc * L->TD[k00 + 1]) +
           tu * ((1.0 - tc) * L->TD[k10] + tc * L->TD[k10 + 1]);
}

/* =====================================================================
 * Atmosphere table and mixed-order interpolation (Sect. 4)
 * ===================================================================== */
typedef struct {
    int nT, ng, nmu, nE, n_protect;
    const double *logT, *logg, *mu, *lnE;  /* node positions */
    const float *I;                         /* [nT][ng][nmu][nE], linear intensity */
    int strategy;                           /* ORC_INTERP_* below */
} orc_atm;

/* Interpolation strategies of Sect. 4 (the four compared on the paper's two
 * interpolation tests):
 *   D  the method's mixed scheme: linear in logT and logg; cubic Lagrange in
 *      mu and ln E, linear where the centred stencil would leave the grid
 *      and on the protected small-mu intervals;
 *   A  cubic Lagrange in all four axes, the four-node stencil shifted to stay
 *      inside the grid at the edges (one-sided);
 *   B  as A, negative interpolants clipped to zero;
 *   C  cubic in all four axes with the linear treatment of D at the table
 *      edges and on the protected small-mu intervals. */
enum { ORC_INTERP_D = 0, ORC_INTERP_A = 1, ORC_INTERP_B = 2, ORC_INTERP_C = 3 };
/* per-axis rules */
enum { AX_LINEAR = 0, AX_CUBIC = 1, AX_CUBIC_ONESIDED = 2 };

/* interval index i with x[i] <= q < x[i+1] after clamping q to [x0, x_{n-1}] */
static int find_interval(const double *x, int n, real *q)
{
    if (RE(*q) <= x[0]) { *q = x[0]; return 0; }
    if (RE(*q) >= x[n - 1]) { *q = x[n - 1]; return n - 2; }
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (x[mid] <= RE(*q)) lo = mid; else hi = mid;
    }
    return lo;
}

/* Interpolation weights along one axis.  Writes node indices idx[] and
 * weights w[] (n_taps = 2 or 4).  AX_CUBIC: Lagrange on the four nodes
 * i-1..i+2 around interval i (actual node positions); falls back to linear
 * on (i, i+1) when the interval lies in the protected zone (i < n_protect-1)
 * or when the four-node stencil would leave the grid.  AX_CUBIC_ONESIDED:
 * Lagrange on the four nodes s..s+3 with s = i-1 moved into [0, n-4]. */
static int axis_weights(const double *x, int n, real q, int rule, int n_protect,
                        int *idx, real *w)
{
    int i = find_interval(x, n, &q);
    int s0 = -1;
    if (rule == AX_CUBIC && i >= 1 && i + 2 <= n - 1 && i >= n_protect - 1) s0 = i - 1;
    if (rule == AX_CUBIC_ONESIDED && n >= 4) s0 = i - 1 < 0 ? 0 : (i - 1 > n - 4 ? n - 4 : i - 1);
    if (s0 >= 0) {
        for (int a = 0; a < 4; a++) {
            int ka = s0 + a;
            real l = 1.0;
            for (int b = 0; b < 4; b++) {
                if (b == a) continue;
                int kb = s0 + b;
                l *= (q - x[kb]) / (x[ka] - x[kb]);
            }
            idx[a] = ka;
            w[a] = l;
        }
        return 4;
    }
    real t = (q - x[i]) / (x[i + 1] - x[i]);
    idx[0] = i; w[0] = 1.0 - t;
    idx[1] = i + 1; w[1] = t;
    return 2;
}

/* I(E', mu; logT, logg): linear in logT and logg, cubic (mixed) in mu and ln E.
 * Out-of-range queries clamp to the edge node; negative interpolants are kept. */
real orc_atm_interp(const orc_atm *A, real logT, real logg, real mu, real E_keV)
{
    int iT[4], ig[4], im[4], ie[4];
    real wT[4], wg[4], wm[4], we[4];
    const int st = A->strategy;
    const int cubic_all = st == ORC_INTERP_A || st == ORC_INTERP_B;
    const int rTg = cubic_all ? AX_CUBIC_ONESIDED : (st == ORC_INTERP_C ? AX_CUBIC : AX_LINEAR);
    const int rmE = cubic_all ? AX_CUBIC_ONESIDED : AX_CUBIC;
    const int prot = cubic_all ? 0 : A->n_protect;
    int nT = axis_weights(A->logT, A->nT, logT, rTg, 0, iT, wT);
    int ng = axis_weights(A->logg, A->ng, logg, rTg, 0, ig, wg);
    int nm = axis_weights(A->mu, A->nmu, mu, rmE, prot, im, wm);
    int ne = axis_weights(A->lnE, A->nE, r_log(E_keV), rmE, 0, ie, we);
    real v = 0.0;
    for (int a = 0; a < nT; a++)
        for (int b = 0; b < ng; b++)
            for (int c = 0; c < nm; c++)
                for (int d = 0; d < ne; d++) {
                    size_t k = (((size_t)iT[a] * A->ng + ig[b]) * A->nmu + im[c]) * A->nE + ie[d];
                    v += wT[a] * wg[b] * wm[c] * we[d] * (double)A->I[k];
                }
    if (st == ORC_INTERP_B && RE(v) < 0.0) v = 0.0;
    return v;
}

/* comoving blackbody specific intensity 2 E^3 / (h^3 c^2) / (e^{E/kT} - 1)
 * in keV cm^-2 s^-1 keV^-1 sr^-1 (App. C) */
real orc_bb_intensity(real E_keV, real kT_keV)
{
    return 2.0 * E_keV * E_keV * E_keV / (H_KEVS * H_KEVS * H_KEVS * C_CMS * C_CMS) /
           r_expm1(E_keV / kT_keV);
}

/* =====================================================================
 * Star, rings, elements (Sect. 2.1, 2.2, 2.4, 2.6)
 * ===================================================================== */
typedef struct {
    real mass_msun, radius_km, spin_hz, incl_rad, dist_kpc, nh_1e20;
    real colat[2], azim[2], zeta[2], logT[2], mask_colat[2], mask_azim[2], mask_zeta[2];
    int n_spots, oblate, emission, n_theta, n_phi, n_phase, n_fp;
    int grid;  /* 0: spot-bounding grid; 1: HEALPix whole-surface mesh, N_side = n_theta */
    int phase_sub;  /* sub-samples per output phase bin (reading: 1 = point samples) */
    /* full-surface temperature map (Sect. 2.6): log10 T_eff per HEALPix pixel
     * in ring order (grid 1 only), or NULL; a pixel with a non-finite or
     * non-positive value emits nothing.  With a map the spot parameters are
     * not used: every mesh pixel is a candidate and carries its own T. */
    const double *logT_map;
} orc_inst;

typedef struct {
    real GM, Rs, Re, nu, Obar, x, o2, g0, sini, cosi, D;
    int oblate;
} orc_star;

static void star_init(const orc_inst *in, orc_star *s)
{
    s->GM = in->mass_msun * GM_SUN;
    s->Rs = 2.0 * s->GM / (C_MS * C_MS);
    s->Re = in->radius_km * 1e3;
    s->nu = in->spin_hz;
    s->Obar = 2.0 * ORC_PI * s->nu * r_sqrt(s->Re * s->Re * s->Re / s->GM);  /* Eq. Omega_c_def */
    s->x = s->GM / (C_MS * C_MS * s->Re);
    s->oblate = in->oblate;
    /* Eq. Rtheta; the S+D mode is the spherical star o2 = 0 */
    s->o2 = in->oblate ? s->Obar * s->Obar * (-0.788 + 1.030 * s->x) : 0.0;
    s->g0 = s->GM / (s->Re * s->Re) / r_sqrt(1.0 - s->Rs / s->Re);
    s->sini = r_sin(in->incl_rad);
    s->cosi = r_cos(in->incl_rad);
    s->D = in->dist_kpc * KPC_M;
}

typedef struct {
    real theta, dcos, R, u, f, cos_eta, sin_eta, logg, beta, gamma;
} orc_ring;

/* Ring quantities at colatitude theta (Eqs. Rtheta, def_f, the g(theta)
 * polynomial of Sect. 2.2, beta/gamma of Sect. 2.4).  Readings: R and u are
 * the local R(theta), u(theta) (Omega_bar and x use R_e); dR/dtheta =
 * -2 o2 R_e cos(theta) sin(theta); in the S+D mode g = g0. */
static void ring_geom(const orc_star *s, real theta, real dcos, orc_ring *r)
{
    real ct = r_cos(theta), st = r_sin(theta);
    r->theta = theta;
    r->dcos = dcos;
    r->R = s->Re * (1.0 + s->o2 * ct * ct);
    r->u = s->Rs / r->R;
    real dRdth = -2.0 * s->o2 * s->Re * ct * st;
    r->f = dRdth / (r->R * r_sqrt(1.0 - r->u));
    r->cos_eta = 1.0 / r_sqrt(1.0 + r->f * r->f);
    r->sin_eta = r->f / r_sqrt(1.0 + r->f * r->f);
    real g = s->g0;
    if (s->oblate) {
        real O2 = s->Obar * s->Obar, O4 = O2 * O2, O6 = O4 * O2, x = s->x;
        real c2 = ct * ct, s2 = st * st;
        real ratio = 1.0
            + s2 * (O2 * (-0.791 + 0.776 * x) + O4 * (-1.315 * x + 2.431 * x * x) + O6 * (-1.172 * x))
            + c2 * (O2 * (1.138 - 1.431 * x) + O4 * (0.653 * x - 2.864 * x * x) + O6 * (0.975 * x)
                    - O4 * (13.47 * x - 27.13 * x * x))
            + r_fabs(ct) * O4 * (13.47 * x - 27.13 * x * x);
        g = s->g0 * ratio;
    }
    r->logg = r_log10(g * 100.0); /* m s^-2 -> cm s^-2 */
    r->beta = 2.0 * ORC_PI * s->nu * r->R * st / (C_MS * r_sqrt(1.0 - r->u));
    r->gamma = 1.0 / r_sqrt(1.0 - r->beta * r->beta);
}

/* Element grid of one spot (reading): n_theta rings uniform in theta over
 * [max(0, theta_c - zeta), min(pi, theta_c + zeta)]; each ring holds n_phi
 * elements uniform over the emitter's azimuth span phi_c +- Delta_i; an
 * element is active unless its centre lies inside the spot's masking cap. */
static void ring_of_spot(const orc_inst *in, int spot, int r, real *theta,
                         real *dcos, real *half)
{
    real tc = in->colat[spot], z = in->zeta[spot];
    real lo = RE(tc - z) > 0.0 ? tc - z : 0.0;
    real hi = RE(tc + z) < ORC_PI ? tc + z : ORC_PI;
    real dth = (hi - lo) / in->n_theta;
    real e0 = lo + r * dth, e1 = lo + (r + 1) * dth;
    *theta = lo + (r + 0.5) * dth;
    *dcos = r_cos(e0) - r_cos(e1);
    real num = r_cos(z) - r_cos(*theta) * r_cos(tc);
    real den = r_sin(*theta) * r_sin(tc);
    if (RE(den) <= 0.0) {
        *half = RE(num) <= 0.0 ? ORC_PI : 0.0;
    } else {
        /* a clamped half-width is a constant (pi: the ring encircles the
         * pole inside the cap; 0: it misses the cap) and has no derivative */
        real a = num / den;
        if (RE(a) <= -1.0) *half = ORC_PI;
        else if (RE(a) >= 1.0) *half = 0.0;
        else *half = r_acos(a);
    }
}

/* a decision only: evaluated on the real parts */
static int element_active(const orc_inst *in, int spot, real theta_r, real phi_r)
{
    double mz = RE(in->mask_zeta[spot]);
    if (!(mz > 0.0)) return 1;
    double theta = RE(theta_r), phi = RE(phi_r);
    double cd = cos(theta) * cos(RE(in->mask_colat[spot])) +
                sin(theta) * sin(RE(in->mask_colat[spot])) * cos(phi - RE(in->mask_azim[spot]));
    return !(cd > cos(mz));
}

/* One ring of a spot's elements: colatitude, the cos(theta) width and the
 * azimuth step whose product is the element's solid angle, the first element
 * azimuth, the element count, and whether element membership needs the
 * emitter-cap test (the HEALPix mesh is not aligned with the spot).
 *
 * grid 0 (reading of the element grid): ring_of_spot above.
 * grid 1 (Sect. 2.6, the HEALPix scheme of Gorski et al. 2005 with
 * N = N_side): ring i = 1 .. 4N-1 has
 *   z = 1 - i^2/(3N^2) and 4i pixels                (i < N),
 *   z = 4/3 - 2i/(3N) and 4N pixels                 (N <= i <= 3N),
 *   z = -(1 - (4N-i)^2/(3N^2)) and 4(4N-i) pixels   (i > 3N);
 * pixel j = 1 .. n of a polar ring sits at phi = (pi/2)(j - 1/2)/i' (i' = i
 * or 4N-i), of an equatorial ring at phi = (pi/2N)(j - s/2) with
 * s = (i - N + 1) mod 2; every pixel has solid angle pi / (3 N^2).  A pixel
 * belongs to the spot when its centre is within zeta of the spot centre
 * and outside the mask (Sect. 2.6: the spot is selected on the mesh). */
typedef struct {
    real theta, dcos, dphi, phi0, half;
    int n_el, cap_test, ok;
} orc_ringdef;

static int ring_count(const orc_inst *in)
{
    return in->grid == 1 ? 4 * in->n_theta - 1 : in->n_theta;
}

static void ring_def(const orc_inst *in, int spot, int r, orc_ringdef *d)
{
    if (in->grid != 1) {
        ring_of_spot(in, spot, r, &d->theta, &d->dcos, &d->half);
        d->dphi = 2.0 * d->half / in->n_phi;
        d->phi0 = 0.0;
        d->n_el = in->n_phi;
        d->cap_test = 0;
        d->ok = RE(d->half) > 0.0;
        return;
    }
    const int N = in->n_theta, i = r + 1;
    const double NN = (double)N;
    double z, phi0;
    int n;
    if (i < N || i > 3 * N) {
        const int ip = i < N ? i : 4 * N - i;
        const double zz = 1.0 - (double)ip * ip / (3.0 * NN * NN);
        z = i < N ? zz : -zz;
        n = 4 * ip;
        phi0 = 0.25 * ORC_PI / ip;
    } else {
        z = 4.0 / 3.0 - 2.0 * i / (3.0 * NN);
        n = 4 * N;
        const int sh = (i - N + 1) % 2;
        phi0 = 0.5 * ORC_PI / NN * (1.0 - 0.5 * sh);
    }
    d->theta = acos(z);
    d->n_el = n;
    d->dphi = 2.0 * ORC_PI / n;
    d->dcos = (ORC_PI / (3.0 * NN * NN)) / d->dphi;
    d->phi0 = phi0;
    d->half = ORC_PI;
    d->cap_test = 1;
    /* rings that cannot reach the cap are skipped (a decision only) */
    d->ok = in->logT_map != NULL ||
            fabs(RE(d->theta) - RE(in->colat[spot])) <= RE(in->zeta[spot]) + 1e-12;
}

/* pixels of the HEALPix rings before ring r (0-based), i.e. the ring-order
 * index of the ring's first pixel */
static size_t ring_first_pixel(const orc_inst *in, int r)
{
    const int N = in->n_theta;
    size_t n = 0;
    for (int k = 1; k <= r; k++) n += (size_t)(k < N ? 4 * k : (k > 3 * N ? 4 * (4 * N - k) : 4 * N));
    return n;
}

/* azimuth of element m of a ring */
static real ring_phi(const orc_inst *in, int spot, const orc_ringdef *d, int m)
{
    if (in->grid != 1) return in->azim[spot] - d->half + (m + 0.5) * d->dphi;
    return d->phi0 + m * d->dphi;
}

/* emitter-cap membership of a mesh element (a decision only, real parts) */
static int inside_cap(const orc_inst *in, int spot, real theta_r, real phi_r)
{
    double th = RE(theta_r), ph = RE(phi_r), tc = RE(in->colat[spot]);
    double cd = cos(th) * cos(tc) + sin(th) * sin(tc) * cos(ph - RE(in->azim[spot]));
    return cd >= cos(RE(in->zeta[spot]));
}

/* =====================================================================
 * Per-ring pseudo-patch template (Sect. 2.8.3, steps 1-5, and the
 * invisible-segment fill).  Arrays have n_fp + 1 entries.
 * Returns 1 if the ring contributes, 0 if it is invisible at i_fp = 0
 * (whole ring skipped), -1 if u lies outside the lens table.
 * ===================================================================== */
/* radial delay of emission radius R relative to R_e (Eq. delta_t_oblate) */
static real oblate_delay(const orc_star *s, const orc_ring *rg)
{
    return (s->Re - rg->R + s->Rs * r_log((s->Re - s->Rs) / (rg->R - s->Rs))) / C_MS;
}

static int ring_template(const orc_star *s, const orc_ring *rg, real dphi,
                         const orc_lens *L, int n_fp, real *F, real *z,
                         real *phio, real *mu)
{
    const orc_lens_spec *ls = &L->spec;
    if (RE(rg->u) < ls->u_min || RE(rg->u) > ls->u_max) return -1;
    real st = r_sin(rg->theta), ct = r_cos(rg->theta);
    real sq = r_sqrt(1.0 - rg->u);
    /* area element R^2 sqrt(1+f^2) dcos(theta) dphi / D^2 (Eq. area_oblate) */
    real area = rg->R * rg->R * r_sqrt(1.0 + rg->f * rg->f) * rg->dcos * dphi / (s->D * s->D);
    real dt_obl = oblate_delay(s, rg);
    int inv_min = n_fp, inv_max = 0;
    int vis0 = 0;
    for (int i = 0; i <= n_fp; i++) {
        if (i == n_fp) {
            /* i_fp = N_fp is the same surface point as i_fp = 0 (reading:
             * exact periodicity, phi_o[N_fp] = phi_o[0] + 1) */
            if (vis0) {
                F[i] = F[0]; z[i] = z[0]; mu[i] = mu[0]; phio[i] = phio[0] + 1.0;
            } else {
                F[i] = 0.0; mu[i] = 0.0; z[i] = 0.0; phio[i] = 0.0;
            }
            break;
        }
        double phi = 2.0 * ORC_PI * (double)i / (double)n_fp;
        double cphi = cos(phi), sphi = sin(phi);
        /* step 2: cos psi */
        real cpsi = s->sini * st * cphi + s->cosi * ct;
        int visible = 0;
        real ca, lf;
        /* step 3: lens lookup; points beyond the cos psi grid are invisible */
        if (RE(cpsi) >= ls->cpsi_min && orc_lens_lookup(L, rg->u, cpsi, &ca, &lf)) {
            real one_ca2 = 1.0 - ca * ca, one_cp2 = 1.0 - cpsi * cpsi;
            real sa = r_sqrt(RE(one_ca2) > 0.0 ? one_ca2 : 0.0);
            real sp = r_sqrt(RE(one_cp2) > 0.0 ? one_cp2 : 0.0);
            /* sin(alpha)/sin(psi); limit sqrt(LF) as psi -> 0 (reading) */
            real ratio = RE(sp) > 1e-12 ? sa / sp : r_sqrt(lf);
            /* step 4: Eq. sigma_relation */
            real csig = ca * rg->cos_eta +
                        ratio * rg->sin_eta * (s->cosi * st - s->sini * ct * cphi);
            /* step 5 */
            if (RE(csig) >= 0.0) {
                visible = 1;
                real cxi = -ratio * s->sini * sphi;            /* Table tab:angles */
                real delta = 1.0 / (rg->gamma * (1.0 - rg->beta * cxi));
                real m = delta * csig;                          /* mu = cos sigma' */
                F[i] = sq * delta * delta * delta * m * lf * rg->gamma * area;
                z[i] = 1.0 / (delta * sq);
                real dt = rg->R / C_MS * orc_td_lookup(L, rg->u, ca) + dt_obl;
                phio[i] = (double)i / (double)n_fp + s->nu * dt;
                mu[i] = m;
            }
        }
        if (i == 0) vis0 = visible;
        if (!visible) {
            if (i < inv_min) inv_min = i;
            if (i > inv_max) inv_max = i;
            F[i] = 0.0; mu[i] = 0.0; z[i] = 0.0; phio[i] = 0.0;
        }
    }
    if (!vis0) return 0;
    if (inv_min <= inv_max) {
        int a = inv_min - 1, b = inv_max + 1;
        for (int i = inv_min; i <= inv_max; i++) {
            double t = (double)(i - a) / (double)(b - a);
            F[i] = 0.0;
            mu[i] = 0.0;
            z[i] = z[a] + (z[b] - z[a]) * t;
            phio[i] = phio[a] + (phio[b] - phio[a]) * t;
        }
    }
    return 1;
}

/* =====================================================================
 * Forward profile F_t (Sect. 2.8.3 shift-and-add, Eq. add_Ft)
 * ===================================================================== */

/* floor-mod into [0, 1) */
static real frac1(real x) { return x - floor(RE(x)); }

/* Linear interpolation of the template at phase phip (reading: linear,
 * binary search on the monotone phi_o). */
static void template_at(const real *phio, const real *F, const real *z,
                        const real *mu, int n_fp, real phip,
                        real *Fp, real *zp, real *mup)
{
    int lo = 0, hi = n_fp;
    if (RE(phip) <= RE(phio[0])) hi = 1;
    else if (RE(phip) >= RE(phio[n_fp])) lo = n_fp - 1;
    else {
        while (hi - lo > 1) {
            int mid = (lo + hi) / 2;
            if (RE(phio[mid]) <= RE(phip)) lo = mid; else hi = mid;
        }
    }
    real w = (phip - phio[lo]) / (phio[lo + 1] - phio[lo]);
    if (RE(w) < 0.0) w = 0.0;
    if (RE(w) > 1.0) w = 1.0;
    *Fp = F[lo] + (F[lo + 1] - F[lo]) * w;
    *zp = z[lo] + (z[lo + 1] - z[lo]) * w;
    *mup = mu[lo] + (mu[lo + 1] - mu[lo]) * w;
}

/* Status codes of the oracle */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ERANGE = 2 };

/* Reading (the paper is silent on non-finite inputs): a NaN or infinite
 * parameter the instance uses lies outside every table and is a range error.
 * An infinite distance is not: it is a valid limit (zero flux).  Spot and
 * mask parameters count only without a temperature map; a mask radius <= 0
 * (-inf included) means no mask, and a mask needs finite geometry. */
static int params_finite(const orc_inst *in)
{
    const double g[] = {RE(in->mass_msun), RE(in->radius_km), RE(in->spin_hz),
                        RE(in->incl_rad), RE(in->nh_1e20)};
    for (int i = 0; i < 5; i++)
        if (!isfinite(g[i])) return 0;
    if (isnan(RE(in->dist_kpc))) return 0;
    if (in->logT_map) return 1;
    for (int sp = 0; sp < in->n_spots; sp++) {
        const double mz = RE(in->mask_zeta[sp]);
        if (!isfinite(RE(in->colat[sp])) || !isfinite(RE(in->azim[sp])) ||
            !isfinite(RE(in->zeta[sp])) || !isfinite(RE(in->logT[sp])) || isnan(mz))
            return 0;
        if (mz > 0.0 && !(isfinite(mz) && isfinite(RE(in->mask_colat[sp])) &&
                          isfinite(RE(in->mask_azim[sp]))))
            return 0;
    }
    return 1;
}

/* Shift-and-add of Sect. 2.8.3 (Eq. add_Ft) with the flux of Sect. 2.5 /
 * App. C and the atmosphere interpolation of Sect. 4:
 * F_t[j][k] for the selected output phases jsel (indices into
 * phi_out = j / n_phase) and energies ksel (indices into E_keV); NULL
 * selects all.  ring_stride > 1 evaluates every ring_stride-th ring only
 * (used to time a bounded sample).  Ft has n_j * n_k entries, row-major. */
int orc_profile(const orc_inst *in, const orc_lens *L, const orc_atm *A,
                const double *E_keV, int nE, const int *jsel, int nj,
                const int *ksel, int nk, int ring_stride, real *Ft)
{
    if (in->n_spots < 1 || in->n_spots > 2 || in->n_theta < 1 || in->n_phi < 1 ||
        in->n_phase < 1 || in->n_fp < 2 || nE < 1 || in->grid < 0 || in->grid > 1 ||
        in->phase_sub < 1)
        return ORC_EINVAL;
    const int S = in->phase_sub;
    if (in->emission == 1 && A == NULL) return ORC_EINVAL;
    const int use_map = in->logT_map != NULL;
    if (use_map && in->grid != 1) return ORC_EINVAL;
    if (!params_finite(in)) return ORC_ERANGE;
    if (ring_stride < 1) ring_stride = 1;
    int NJ = jsel ? nj : in->n_phase;
    int NK = ksel ? nk : nE;
    for (size_t q = 0; q < (size_t)NJ * NK; q++) Ft[q] = 0.0;
    orc_star s;
    star_init(in, &s);
    int n_fp = in->n_fp;
    real *F = (real *)malloc(sizeof(real) * (n_fp + 1));
    real *z = (real *)malloc(sizeof(real) * (n_fp + 1));
    real *ph = (real *)malloc(sizeof(real) * (n_fp + 1));
    real *mu = (real *)malloc(sizeof(real) * (n_fp + 1));
    int status = ORC_OK;
    for (int sp = 0; sp < (use_map ? 1 : in->n_spots) && status == ORC_OK; sp++) {
        real logT = use_map ? 6.0 : in->logT[sp];   /* a map sets it per pixel */
        real kT = KB_KEVK * r_pow(10.0, logT);
        if (!use_map && in->emission == 1 &&
            (RE(logT) < A->logT[0] || RE(logT) > A->logT[A->nT - 1])) {
            status = ORC_ERANGE;
            break;
        }
        for (int r = 0; r < ring_count(in); r += ring_stride) {
            orc_ringdef rd;
            ring_def(in, sp, r, &rd);
            if (!rd.ok) continue;
            const real theta = rd.theta;
            orc_ring rg;
            ring_geom(&s, theta, rd.dcos, &rg);
            if (in->emission == 1 &&
                (RE(rg.logg) < A->logg[0] || RE(rg.logg) > A->logg[A->ng - 1])) {
                status = ORC_ERANGE;
                break;
            }
            const real dphi = rd.dphi;
            int tv = ring_template(&s, &rg, dphi, L, n_fp, F, z, ph, mu);
            if (tv < 0) { status = ORC_ERANGE; break; }
            if (tv == 0) continue;
            const size_t pix0 = use_map ? ring_first_pixel(in, r) : 0;
            for (int m = 0; m < rd.n_el && status == ORC_OK; m++) {
                real phia = ring_phi(in, sp, &rd, m);
                if (use_map) {
                    const double lt = in->logT_map[pix0 + m];
                    if (!(isfinite(lt) && lt > 0.0)) continue;  /* dark pixel */
                    if (in->emission == 1 && (lt < A->logT[0] || lt > A->logT[A->nT - 1])) {
                        status = ORC_ERANGE;
                        break;
                    }
                    logT = lt;
                    kT = KB_KEVK * r_pow(10.0, logT);
                } else {
                    if (rd.cap_test && !inside_cap(in, sp, theta, phia)) continue;
                    if (!element_active(in, sp, theta, phia)) continue;
                }
                real sm = phia / (2.0 * ORC_PI);
                for (int jj = 0; jj < NJ; jj++) {
                    int j = jsel ? jsel[jj] : jj;
                    /* reading: phase bin j is centred on j / n_phase; with
                     * phase_sub = S its value is the mean of S point samples
                     * at the centres of its S equal sub-intervals */
                    for (int q = 0; q < S; q++) {
                        double phi_out = S == 1 ? (double)j / (double)in->n_phase
                                                : ((double)j + ((q + 0.5) / S - 0.5)) /
                                                      (double)in->n_phase;
                        real phip = frac1(phi_out + sm + 1.0 - ph[0]) + ph[0];
                        real Fp, zp, mup;
                        template_at(ph, F, z, mu, n_fp, phip, &Fp, &zp, &mup);
                        if (RE(Fp) == 0.0) continue;
                        for (int kk = 0; kk < NK; kk++) {
                            int k = ksel ? ksel[kk] : kk;
                            double E = E_keV[k];
                            real Ep = zp * E;
                            real I = (in->emission == 1)
                                           ? orc_atm_interp(A, logT, rg.logg, mup, Ep)
                                           : orc_bb_intensity(Ep, kT);
                            Ft[(size_t)jj * NK + kk] += Fp * I / E / (double)S;
                        }
                    }
                }
            }
        }
    }
    free(F); free(z); free(ph); free(mu);
    return status;
}

/* Ring quantities (Sect. 2.1-2.2, 2.4; Eq. delta_t_oblate) and template
 * (Sect. 2.8.3) for tests: fills info[0..14] =
 * {theta, dcos, half_width, R, u, f, cos_eta, sin_eta, logg, beta, gamma,
 *  dphi, n_active, status, dt_obl} and the four template arrays. */
int orc_ring_template(const orc_inst *in, const orc_lens *L, int spot, int r,
                      double *info, double *F, double *z, double *phio, double *mu)
{
    orc_star s;
    star_init(in, &s);
    orc_ringdef rd;
    ring_def(in, spot, r, &rd);
    const real theta = rd.theta, dphi = rd.dphi;
    const real half = rd.half;
    orc_ring rg;
    ring_geom(&s, theta, rd.dcos, &rg);
    int nact = 0;
    for (int m = 0; m < rd.n_el; m++) {
        const real phia = ring_phi(in, spot, &rd, m);
        nact += (!rd.cap_test || inside_cap(in, spot, theta, phia)) &&
                element_active(in, spot, theta, phia);
    }
    int n = in->n_fp + 1;
    real *t = (real *)malloc(sizeof(real) * 4 * n);
    int st = rd.ok ? ring_template(&s, &rg, dphi, L, in->n_fp, t, t + n, t + 2 * n, t + 3 * n)
                   : 0;
    for (int i = 0; i < n && rd.ok; i++) {
        F[i] = RE(t[i]); z[i] = RE(t[n + i]); phio[i] = RE(t[2 * n + i]); mu[i] = RE(t[3 * n + i]);
    }
    free(t);
    double v[15] = {RE(rg.theta), RE(rg.dcos), RE(half), RE(rg.R), RE(rg.u), RE(rg.f),
                    RE(rg.cos_eta), RE(rg.sin_eta), RE(rg.logg), RE(rg.beta), RE(rg.gamma),
                    RE(dphi), (double)nact, (double)st, RE(oblate_delay(&s, &rg))};
    memcpy(info, v, sizeof(v));
    return st;
}

/* =====================================================================
 * ISM, response and Poisson likelihood (Sect. 2.7, 2.8.4, 6)
 * ===================================================================== */

/* C[j][c] = sum_k Ft[j][k] ATT_k R[k][c], ATT_k = exp(-N_H sigma_k)
 * (ISM attenuation of Sect. 2.7, response contraction of Sect. 2.8.4) */
void orc_counts(const real *Ft, int n_phase, int nE, const float *R, int nc,
                const float *sigma, real nh_1e20, real *C)
{
    real nh = nh_1e20 * 1e20;
    for (int j = 0; j < n_phase; j++)
        for (int c = 0; c < nc; c++) {
            real s = 0.0;
            for (int k = 0; k < nE; k++)
                s += Ft[(size_t)j * nE + k] * r_exp(-nh * (double)sigma[k]) * (double)R[(size_t)k * nc + c];
            C[(size_t)j * nc + c] = s;
        }
}

/* logL = sum d ln(lambda) - lambda - ln Gamma(d + 1), lambda = tau C + b.
 * (reading: the Poisson log-likelihood; lambda = 0 gives 0 for d = 0 and
 * -inf for d > 0). */
static real loglike_sum(const real *C, int n, const int *d, const float *bkg, double tau)
{
    real s = 0.0;
    for (int i = 0; i < n; i++) {
        real lam = tau * C[i] + (bkg ? (double)bkg[i] : 0.0);
        if (RE(lam) <= 0.0) {
            if (d[i] > 0) return -INFINITY;
            continue;
        }
        s += (double)d[i] * r_log(lam) - lam - lgamma((double)d[i] + 1.0);
    }
    return s;
}

#ifndef ORC_CSTEP
double orc_loglike(const double *C, int n, const int *d, const float *bkg, double tau)
{
    return loglike_sum(C, n, d, bkg, tau);
}
#endif

/* The whole chain for one instance: profile, attenuation and response,
 * likelihood.  out[0] = logL; out[1] = its imaginary part (the tangent
 * build's h times the directional derivative; 0 in the ordinary build).
 * Returns the orc_profile status. */
int orc_loglike_full(const orc_inst *in, const orc_lens *L, const orc_atm *A,
                     const double *E_keV, int nE, const float *R, int nc,
                     const float *sigma, const int *d, const float *bkg, double tau,
                     double *out)
{
    real *Ft = (real *)malloc(sizeof(real) * (size_t)in->n_phase * nE);
    real *C = (real *)malloc(sizeof(real) * (size_t)in->n_phase * nc);
    int st = orc_profile(in, L, A, E_keV, nE, NULL, 0, NULL, 0, 1, Ft);
    if (st == ORC_OK) {
        orc_counts(Ft, in->n_phase, nE, R, nc, sigma, in->nh_1e20, C);
        real ll = loglike_sum(C, in->n_phase * nc, d, bkg, tau);
        out[0] = RE(ll);
        out[1] = IM(ll);
    }
    free(Ft);
    free(C);
    return st;
}
