/*
 * FP64 CPU oracle for the Schwarzschild orbit-library hot path
 * (arxiv 2607.00117, "SchwarMAX").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * Everything is plain IEEE double arithmetic in the order the formulas are
 * written, compiled with -ffp-contract=off.  Each function cites the passage
 * of the paper it follows.  Units: kpc, km/s, Msun; G = 4.300917e-6
 * kpc (km/s)^2 / Msun (the paper does not state its units; this is the usual
 * galactic-dynamics choice).  One time unit is kpc/(km/s) = 977.79 Myr.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_G 4.300917e-6
#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------------- */
/* Potential description (bar-frame, static).                               */
/* ---------------------------------------------------------------------- */
typedef struct {
    double disc_M, disc_a, disc_b;      /* Miyamoto-Nagai: M_d, R_d, H_d (Sec. 3.2.2) */
    double halo_Mdm, halo_rs;           /* NFW characteristic mass M_DM and R_s (Sec. 3.2.1) */
    double bar_M, bar_L, bar_a, bar_b;  /* needle-convolved MN: mass, half-length L, a, b (Eq. Rn_to_In) */
    int32_t test_kind;                  /* 0 none, 1 point mass, 2 Plummer sphere */
    int32_t bar_kind;                   /* 0 needle-convolved MN (Long-Murali); 1 the paper's T3 + V4 bar */
    double test_M, test_a;
} orc_pot;

enum { ORC_DISC = 1, ORC_HALO = 2, ORC_BAR = 4, ORC_TEST = 8 };

/* NFW re-parameterisation (Sec. 3.2.1): R_vir = (3 M_vir / (4 pi 200 rho_crit))^(1/3),
 * c = R_vir / R_s, and M_DM = 4 pi rho_0 R_s^3 equals M_vir / [ln(1+c) - c/(1+c)]
 * because the enclosed-mass formula evaluated at R = R_vir must give M_vir.
 * rho_crit = 3 H0^2 / (8 pi G); H0 is given in km/s/Mpc. */
void orc_nfw_from_m200(double M200, double c, double H0_kms_mpc, double* Mdm, double* rs)
{
    double H = H0_kms_mpc / 1000.0;              /* km/s/kpc */
    double rho_crit = 3.0 * H * H / (8.0 * ORC_PI * ORC_G);
    double Rvir = cbrt(3.0 * M200 / (4.0 * ORC_PI * 200.0 * rho_crit));
    *rs = Rvir / c;
    *Mdm = M200 / (log(1.0 + c) - c / (1.0 + c));
}

/* NFW enclosed mass M(<R) (Sec. 3.2.1, first line of the re-parameterisation). */
double orc_nfw_enclosed(double Mdm, double rs, double R)
{
    return Mdm * (log((rs + R) / rs) - R / (rs + R));
}

/* ---- Miyamoto-Nagai (Sec. 3.2.2): Phi = -G M / calR, calR^2 = R^2 + (a + zeta)^2,
 *      zeta = sqrt(z^2 + b^2).  Force a = -grad Phi. */
static void mn_phi_acc(double M, double a, double b, const double x[3], double* phi, double acc[3])
{
    double zeta = sqrt(x[2] * x[2] + b * b);
    double az = a + zeta;
    double D2 = x[0] * x[0] + x[1] * x[1] + az * az;
    double D = sqrt(D2);
    double D3 = D2 * D;
    *phi = -ORC_G * M / D;
    acc[0] = -ORC_G * M * x[0] / D3;
    acc[1] = -ORC_G * M * x[1] / D3;
    acc[2] = -ORC_G * M * x[2] * az / (zeta * D3);
}

/* Paper's MN density, Sec. 3.2.2 (printed beside the potential). */
static double mn_rho(double M, double a, double b, const double x[3])
{
    double zeta = sqrt(x[2] * x[2] + b * b);
    double R2 = x[0] * x[0] + x[1] * x[1];
    double calR2 = R2 + (a + zeta) * (a + zeta);
    double calR = sqrt(calR2);
    double num = a * calR2 + 3.0 * zeta * (zeta + a) * (zeta + a);
    return (b * b * M / (4.0 * ORC_PI)) * num / (pow(calR, 5.0) * zeta * zeta * zeta);
}

/* ---- NFW (Sec. 3.2.1): Phi = -G M_DM ln(1 + r/R_s) / r.
 *      dPhi/dr = G M_DM [ln(1+r/R_s) - (r/R_s)/(1+r/R_s)] / r^2. */
static void nfw_phi_acc(double Mdm, double rs, const double x[3], double* phi, double acc[3])
{
    double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    if (r == 0.0) {
        /* limits: Phi(0) = -G M_DM / R_s, force is finite in magnitude but
         * without direction at the exact centre */
        *phi = -ORC_G * Mdm / rs;
        acc[0] = acc[1] = acc[2] = 0.0;
        return;
    }
    double s = r / rs;
    double L = log1p(s);
    *phi = -ORC_G * Mdm * L / r;
    /* m(s) = ln(1+s) - s/(1+s); below s = 1e-3 the difference cancels, so use
     * its Taylor series sum_{k>=2} (-1)^k (k-1) s^k / k (truncation < s^8). */
    double m;
    if (s < 1e-3) {
        m = 0.0;
        for (int k = 7; k >= 2; --k) m = m * s + ((k % 2) ? -1.0 : 1.0) * (k - 1.0) / k;
        m *= s * s;
    } else {
        m = L - s / (1.0 + s);
    }
    double dphidr = ORC_G * Mdm * m / (r * r);
    acc[0] = -dphidr * x[0] / r;
    acc[1] = -dphidr * x[1] / r;
    acc[2] = -dphidr * x[2] / r;
}

static double nfw_rho(double Mdm, double rs, const double x[3])
{
    double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    double s = r / rs;
    return Mdm / (4.0 * ORC_PI * rs * rs * rs) / (s * (1.0 + s) * (1.0 + s));
}

/* ---- Needle-convolved MN bar, n = 1 and eta = 0 of Eq. (Rn_to_In):
 *   calR^-1 -> I_1 = (1/2L) int_{x-L}^{x+L} dx' / sqrt(x'^2 + y^2 + Z^2),  Z = a + zeta,
 *   which integrates to (1/2L) ln[(x + L + T+)/(x - L + T-)],
 *   T+- = sqrt((x +- L)^2 + y^2 + Z^2).  Phi = -G M I_1 (the Long-Murali bar).
 * Gradient: d/dx ln(x -+ L + T-+) = 1/T-+, d/dy ln(...) = y / (T (x -+ L + T)),
 *           d/dZ ln(...) = Z / (T (x -+ L + T)),  dZ/dz = z / zeta. */
static void bar_phi_acc(double M, double L, double a, double b, const double x[3], double* phi, double acc[3])
{
    double zeta = sqrt(x[2] * x[2] + b * b);
    double Z = a + zeta;
    double q2 = x[1] * x[1] + Z * Z;
    double Tp = sqrt((x[0] + L) * (x[0] + L) + q2);
    double Tm = sqrt((x[0] - L) * (x[0] - L) + q2);
    double up = x[0] + L + Tp;
    double um = x[0] - L + Tm;
    double k = ORC_G * M / (2.0 * L);
    *phi = k * log(um / up);
    double Kf = 1.0 / (Tm * um) - 1.0 / (Tp * up);
    acc[0] = -k * (1.0 / Tm - 1.0 / Tp);
    acc[1] = -k * x[1] * Kf;
    acc[2] = -k * Z * (x[2] / zeta) * Kf;
}

/* Bar density by the definition behind Eq. (Rn_to_In): the same needle
 * convolution applied to the parent MN density, evaluated here by
 * composite Gauss-Legendre quadrature along the needle (used only by the
 * Poisson pin).  f(x) = 1/(2L) on |x| < L for eta = 0. */
static double bar_rho(double M, double L, double a, double b, const double x[3], int nodes)
{
    /* 8-point Gauss-Legendre on each of `nodes` sub-intervals of [-L, L] */
    static const double gx[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                                 -0.1834346424956498, 0.1834346424956498, 0.5255324099163290,
                                 0.7966664774136267, 0.9602898564975363};
    static const double gw[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                                 0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                                 0.2223810344533745, 0.1012285362903763};
    double h = 2.0 * L / nodes, sum = 0.0;
    for (int k = 0; k < nodes; ++k) {
        double lo = -L + k * h, mid = lo + 0.5 * h;
        for (int j = 0; j < 8; ++j) {
            double s = mid + 0.5 * h * gx[j];           /* needle offset x - x' */
            double p[3] = {x[0] - s, x[1], x[2]};
            sum += 0.5 * h * gw[j] * mn_rho(M, a, b, p) / (2.0 * L);
        }
    }
    return sum;
}

/* ---- Test potentials (fixtures, not in the paper). */
static void kepler_phi_acc(double M, const double x[3], double* phi, double acc[3])
{
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double r = sqrt(r2);
    *phi = -ORC_G * M / r;
    double f = -ORC_G * M / (r2 * r);
    acc[0] = f * x[0]; acc[1] = f * x[1]; acc[2] = f * x[2];
}

static void plummer_phi_acc(double M, double a, const double x[3], double* phi, double acc[3])
{
    double s2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2] + a * a;
    double s = sqrt(s2);
    *phi = -ORC_G * M / s;
    double f = -ORC_G * M / (s2 * s);
    acc[0] = f * x[0]; acc[1] = f * x[1]; acc[2] = f * x[2];
}

static double plummer_rho(double M, double a, const double x[3])
{
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    return 3.0 * M / (4.0 * ORC_PI * a * a * a) * pow(1.0 + r2 / (a * a), -2.5);
}

/* Static potential and acceleration of the selected components at a
 * bar-frame position. */
/* ---- The paper's bar (Sec. 2.1.2, App. A): Dehnen & Aly (2023) T3 long bar
 * (eta = 1, a = L_b/5, b = the disc's height b_d, L = L_b) plus V4 bulge (eta = 0,
 * a = b = 0.5, L = 0.1 kpc), each of mass M_b/2, every R^-n of the parent pair
 * replaced by the needle integral I_n (Eq. Rn_to_In).  The integrals and their x
 * derivatives, d I_n/dx = -n int f(x - x') x' S^-(n+2) dx', are taken by 48-point
 * Gauss-Legendre quadrature on the pieces between x - L, 0, x and x + L; y and Z
 * derivatives use d I_n/dy = -n y I_(n+2) and d I_n/dZ = -n Z I_(n+2). */
#define DA_NQ 48
#define DA_NMAX 13
static double da_gx[DA_NQ], da_gw[DA_NQ];
/* built once, before first use, by pthread_once (callers run inside OpenMP loops) */
static pthread_once_t da_once = PTHREAD_ONCE_INIT;

static void da_nodes(void)
{
    /* Gauss-Legendre nodes by Newton's method on P_48 (Golub-Welsch-free textbook form) */
    for (int i = 0; i < DA_NQ; ++i) {
        double t = cos(ORC_PI * (i + 0.75) / (DA_NQ + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= DA_NQ; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = DA_NQ * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        da_gx[i] = t;
        da_gw[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

/* I[n] = I_n and Ix[n] = d I_n / dx for odd n = 1..nmax at (x, q^2 = y^2 + Z^2) */
static void da_integrals(double x, double q2, double L, double eta, int nmax, double* I, double* Ix)
{
    for (int n = 0; n <= nmax + 2; ++n) { I[n] = 0.0; Ix[n] = 0.0; }
    double lo = x - L, hi = x + L;
    double c1 = 0.0 < lo ? lo : (0.0 > x ? x : 0.0);
    double c2 = 0.0 < x ? x : (0.0 > hi ? hi : 0.0);
    double ends[5] = {lo, c1, x, c2, hi};
    for (int pc = 0; pc < 4; ++pc) {
        double a = ends[pc], b = ends[pc + 1], half = 0.5 * (b - a), mid = 0.5 * (a + b);
        if (half <= 0.0) continue;
        for (int k = 0; k < DA_NQ; ++k) {
            double t = mid + half * da_gx[k];
            double u = fabs(x - t);
            double f = (1.0 + eta * (1.0 - 2.0 * u / L)) / (2.0 * L);
            double s2 = t * t + q2, inv_s = 1.0 / sqrt(s2), inv_s2 = 1.0 / s2;
            double w = half * da_gw[k] * f, pw = inv_s;       /* S^-n, n = 1, 3, ... */
            for (int n = 1; n <= nmax + 2; n += 2) {
                I[n] += w * pw;
                Ix[n] += -n * w * t * pw * inv_s2;
                pw *= inv_s2;
            }
        }
    }
}

/* one barred component: family 0 = T3, 1 = V4 */
static void da_component(int family, double M, double a, double b, double L, double eta, const double x[3],
                         double* phi, double acc[3])
{
    pthread_once(&da_once, da_nodes);
    double z = x[2], zeta = sqrt(z * z + b * b), Z = a + zeta, dzeta = z / zeta;
    double c[DA_NMAX + 1] = {0}, dc[DA_NMAX + 1] = {0};   /* c_n and dc_n/dzeta (Z = a + zeta) */
    int nmax;
    if (family == 0) {
        nmax = 5;
        c[1] = 1.0;
        c[3] = a * (Z - a / 3.0);             dc[3] = a;
        c[5] = a * a * Z * Z;                 dc[5] = 2.0 * a * a * Z;
    } else {
        nmax = 9;
        c[1] = 1.0;
        c[3] = a * (Z - 2.0 * a / 5.0) + b * b / 2.0;                      dc[3] = a;
        c[5] = 3.0 * a * (a * Z * (2.0 * Z - a) / 5.0 + b * b / 2.0 * (Z - a / 5.0));
        dc[5] = 3.0 * a * (a * (4.0 * Z - a) / 5.0 + b * b / 2.0);
        c[7] = a * a * Z * Z * (a * Z + 3.0 * b * b);                       dc[7] = a * a * (3.0 * a * Z * Z + 6.0 * b * b * Z);
        c[9] = 7.0 * a * a * a * b * b * Z * Z * Z * Z / (2.0 * zeta);
        dc[9] = 3.5 * a * a * a * b * b * (4.0 * Z * Z * Z / zeta - Z * Z * Z * Z / (zeta * zeta));
    }
    double I[DA_NMAX + 3], Ix[DA_NMAX + 3];
    da_integrals(x[0], x[1] * x[1] + Z * Z, L, eta, nmax, I, Ix);
    double ph = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int n = 1; n <= nmax; n += 2) {
        ph += c[n] * I[n];
        gx += c[n] * Ix[n];
        gy += c[n] * (-n * x[1] * I[n + 2]);
        gz += (dc[n] * I[n] + c[n] * (-n * Z * I[n + 2])) * dzeta;
    }
    *phi = -ORC_G * M * ph;
    acc[0] = ORC_G * M * gx;                 /* a = -grad Phi = G M grad(sum c_n I_n) */
    acc[1] = ORC_G * M * gy;
    acc[2] = ORC_G * M * gz;
}

/* density of one barred component: M sum_n d_n I_n with the parent's density coefficients */
static double da_component_rho(int family, double M, double a, double b, double L, double eta, const double x[3])
{
    pthread_once(&da_once, da_nodes);
    double z = x[2], zeta = sqrt(z * z + b * b), Z = a + zeta;
    double d[DA_NMAX + 1] = {0};
    int nmax;
    if (family == 0) {
        double k = b * b / (4.0 * ORC_PI);
        nmax = 9;
        d[5] = 3.0 * k;
        d[7] = k * 5.0 * a * Z * Z * (3.0 * zeta * zeta - 2.0 * a * zeta + a * a) / (zeta * zeta * zeta);
        d[9] = k * 35.0 * a * a * Z * Z * Z * Z / (zeta * zeta);
    } else {
        double k = 3.0 * b * b * b * b / (8.0 * ORC_PI), z2 = zeta * zeta;
        nmax = 13;
        d[7] = 5.0 * k;
        d[9] = k * 7.0 * a * Z * Z *
               (5.0 * z2 * z2 - 4.0 * a * z2 * zeta + 3.0 * a * a * z2 - 2.0 * a * a * a * zeta + a * a * a * a) /
               (z2 * z2 * zeta);
        d[11] = k * 63.0 * a * a * Z * Z * Z * Z * (2.0 * z2 - 2.0 * a * zeta + a * a) / (z2 * z2);
        d[13] = k * 231.0 * a * a * a * Z * Z * Z * Z * Z * Z / (z2 * zeta);
    }
    double I[DA_NMAX + 3], Ix[DA_NMAX + 3];
    da_integrals(x[0], x[1] * x[1] + Z * Z, L, eta, nmax, I, Ix);
    double r = 0.0;
    for (int n = 5; n <= nmax; n += 2) r += d[n] * I[n];
    return M * r;
}

static double paper_bar_rho(const orc_pot* p, const double x[3])
{
    return da_component_rho(0, 0.5 * p->bar_M, p->bar_L / 5.0, p->disc_b, p->bar_L, 1.0, x) +
           da_component_rho(1, 0.5 * p->bar_M, 0.5, 0.5, 0.1, 0.0, x);
}

static void paper_bar_phi_acc(const orc_pot* p, const double x[3], double* phi, double acc[3])
{
    double ph1, a1[3], ph2, a2[3];
    da_component(0, 0.5 * p->bar_M, p->bar_L / 5.0, p->disc_b, p->bar_L, 1.0, x, &ph1, a1);
    da_component(1, 0.5 * p->bar_M, 0.5, 0.5, 0.1, 0.0, x, &ph2, a2);
    *phi = ph1 + ph2;
    for (int k = 0; k < 3; ++k) acc[k] = a1[k] + a2[k];
}

static void pot_static(const orc_pot* p, int mask, const double x[3], double* phi, double acc[3])
{
    double ph, ac[3];
    *phi = 0.0; acc[0] = acc[1] = acc[2] = 0.0;
    if ((mask & ORC_DISC) && p->disc_M != 0.0) {
        mn_phi_acc(p->disc_M, p->disc_a, p->disc_b, x, &ph, ac);
        *phi += ph; acc[0] += ac[0]; acc[1] += ac[1]; acc[2] += ac[2];
    }
    if ((mask & ORC_HALO) && p->halo_Mdm != 0.0) {
        nfw_phi_acc(p->halo_Mdm, p->halo_rs, x, &ph, ac);
        *phi += ph; acc[0] += ac[0]; acc[1] += ac[1]; acc[2] += ac[2];
    }
    if ((mask & ORC_BAR) && p->bar_M != 0.0) {
        if (p->bar_kind == 1) paper_bar_phi_acc(p, x, &ph, ac);
        else bar_phi_acc(p->bar_M, p->bar_L, p->bar_a, p->bar_b, x, &ph, ac);
        *phi += ph; acc[0] += ac[0]; acc[1] += ac[1]; acc[2] += ac[2];
    }
    if ((mask & ORC_TEST) && p->test_kind == 1) {
        kepler_phi_acc(p->test_M, x, &ph, ac);
        *phi += ph; acc[0] += ac[0]; acc[1] += ac[1]; acc[2] += ac[2];
    }
    if ((mask & ORC_TEST) && p->test_kind == 2) {
        plummer_phi_acc(p->test_M, p->test_a, x, &ph, ac);
        *phi += ph; acc[0] += ac[0]; acc[1] += ac[1]; acc[2] += ac[2];
    }
}

/* Vectorised entry points used by the pins. */
void orc_potential_eval(const orc_pot* p, int mask, int64_t n, const double* xyz, double* phi, double* acc)
{
    for (int64_t i = 0; i < n; ++i) pot_static(p, mask, xyz + 3 * i, phi + i, acc + 3 * i);
}

void orc_density_eval(const orc_pot* p, int mask, int64_t n, const double* xyz, double* rho, int bar_nodes)
{
    for (int64_t i = 0; i < n; ++i) {
        const double* x = xyz + 3 * i;
        double r = 0.0;
        if ((mask & ORC_DISC) && p->disc_M != 0.0) r += mn_rho(p->disc_M, p->disc_a, p->disc_b, x);
        if ((mask & ORC_HALO) && p->halo_Mdm != 0.0) r += nfw_rho(p->halo_Mdm, p->halo_rs, x);
        if ((mask & ORC_BAR) && p->bar_M != 0.0)
            r += p->bar_kind == 1 ? paper_bar_rho(p, x) : bar_rho(p->bar_M, p->bar_L, p->bar_a, p->bar_b, x, bar_nodes);
        if ((mask & ORC_TEST) && p->test_kind == 2) r += plummer_rho(p->test_M, p->test_a, x);
        rho[i] = r;
    }
}

/* ---------------------------------------------------------------------- */
/* Time-dependent field of the rotating bar (Sec. 2.2.2).                   */
/* The bar's major axis lies along the rotating x axis, which makes angle    */
/* theta = Omega_p t with the inertial x axis.  The axisymmetric parts are   */
/* evaluated directly; the bar is evaluated at R_z(-theta) x and its force   */
/* rotated back by R_z(theta).                                              */
/* ---------------------------------------------------------------------- */
static void field_inertial(const orc_pot* p, double omega, double t, const double x[3], double* phi, double acc[3])
{
    double th = omega * t;
    double c = cos(th), s = sin(th);
    double xb[3] = {c * x[0] + s * x[1], -s * x[0] + c * x[1], x[2]};
    double ph_axi, a_axi[3], ph_bar, a_bar[3];
    pot_static(p, ORC_DISC | ORC_HALO | ORC_TEST, x, &ph_axi, a_axi);
    pot_static(p, ORC_BAR, xb, &ph_bar, a_bar);
    *phi = ph_axi + ph_bar;
    acc[0] = a_axi[0] + (c * a_bar[0] - s * a_bar[1]);
    acc[1] = a_axi[1] + (s * a_bar[0] + c * a_bar[1]);
    acc[2] = a_axi[2] + a_bar[2];
}

/* Jacobi energy E_J = |v|^2/2 + Phi(x, t) - Omega_p (x v_y - y v_x)
 * (Sec. 2.2.2: the only integral of motion with figure rotation). */
static double jacobi(const orc_pot* p, double omega, double t, const double x[3], const double v[3])
{
    double phi, acc[3];
    field_inertial(p, omega, t, x, &phi, acc);
    return 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) + phi - omega * (x[0] * v[1] - x[1] * v[0]);
}

double orc_jacobi(const orc_pot* p, double omega, double t, const double* state6)
{
    return jacobi(p, omega, t, state6, state6 + 3);
}

/* One kick-drift-kick leapfrog step of size dt from t_n = n dt to t_{n+1}.
 * acc holds a(x, t_n) on entry and a(x, t_{n+1}) on exit.  Times are always
 * formed as (step index) * dt, never accumulated. */
static void kdk_step(const orc_pot* p, double omega, double dt, int64_t n, double x[3], double v[3], double acc[3])
{
    double phi;
    v[0] += 0.5 * dt * acc[0]; v[1] += 0.5 * dt * acc[1]; v[2] += 0.5 * dt * acc[2];
    x[0] += dt * v[0]; x[1] += dt * v[1]; x[2] += dt * v[2];
    field_inertial(p, omega, (double)(n + 1) * dt, x, &phi, acc);
    v[0] += 0.5 * dt * acc[0]; v[1] += 0.5 * dt * acc[1]; v[2] += 0.5 * dt * acc[2];
}

/* Full trajectory: out[(n)*6 + k] for n = 0..nsteps (inertial x, v). */
void orc_trajectory(const orc_pot* p, double omega, double dt, int64_t nsteps, const double* ic, double* out)
{
    double x[3] = {ic[0], ic[1], ic[2]}, v[3] = {ic[3], ic[4], ic[5]}, acc[3], phi;
    field_inertial(p, omega, 0.0, x, &phi, acc);
    memcpy(out, ic, 6 * sizeof(double));
    for (int64_t n = 0; n < nsteps; ++n) {
        kdk_step(p, omega, dt, n, x, v, acc);
        double* o = out + 6 * (n + 1);
        o[0] = x[0]; o[1] = x[1]; o[2] = x[2]; o[3] = v[0]; o[4] = v[1]; o[5] = v[2];
    }
}

/* Jacobi drift of a batch of orbits: max_n |E_J(t_n) - E_J(0)| / |E_J(0)|
 * over n = 1..nsteps (Sec. 2.2.2 quality cut). */
void orc_drift(const orc_pot* p, double omega, double dt, int64_t nsteps, int64_t n_orb, const double* ics, double* drift)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n_orb; ++i) {
        const double* ic = ics + 6 * i;
        double x[3] = {ic[0], ic[1], ic[2]}, v[3] = {ic[3], ic[4], ic[5]}, acc[3], phi;
        field_inertial(p, omega, 0.0, x, &phi, acc);
        double e0 = jacobi(p, omega, 0.0, x, v), worst = 0.0;
        for (int64_t n = 0; n < nsteps; ++n) {
            kdk_step(p, omega, dt, n, x, v, acc);
            double e = jacobi(p, omega, (double)(n + 1) * dt, x, v);
            double d = fabs(e - e0) / fabs(e0);
            if (isnan(d) || d > worst) worst = d;   /* a NaN, once seen, is kept */
        }
        drift[i] = worst;
    }
}

/* ---------------------------------------------------------------------- */
/* Observables (Sec. 2.2.3-2.2.4).                                          */
/* ---------------------------------------------------------------------- */
typedef struct {
    /* Euler angles, z-x-z convention: R = Rz(gamma) Rx(beta) Rz(alpha) */
    double alpha, beta, gamma;
    /* regular sky pixels, half-open [x0 + i dx, x0 + (i+1) dx) */
    int32_t nx, ny; double x0, y0, dx, dy;
    /* line-of-sight velocity bins (histogram mode) */
    int32_t nv, pad0; double v0, dv;
    /* cylindrical density cells in the bar frame: R in [0,Rmax), phi in [0,2pi), z in [zmin,zmax) */
    int32_t nR, nphi, nz, pad1; double Rmax, zmin, zmax;
    /* 1: Gauss-Hermite rows (h1..h4) instead of the velocity histogram */
    int32_t gh, mirror4;
} orc_obs;

/* Rotation matrix R(alpha, beta, gamma) = Rz(gamma) Rx(beta) Rz(alpha) with
 * Rz(t) = [[c,-s,0],[s,c,0],[0,0,1]], Rx(t) = [[1,0,0],[0,c,-s],[0,s,c]]. */
void orc_euler_matrix(double alpha, double beta, double gamma, double R[9])
{
    double Rzg[9] = {cos(gamma), -sin(gamma), 0, sin(gamma), cos(gamma), 0, 0, 0, 1};
    double Rxb[9] = {1, 0, 0, 0, cos(beta), -sin(beta), 0, sin(beta), cos(beta)};
    double Rza[9] = {cos(alpha), -sin(alpha), 0, sin(alpha), cos(alpha), 0, 0, 0, 1};
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Rxb[3 * i + k] * Rza[3 * k + j];
            T[3 * i + j] = s;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Rzg[3 * i + k] * T[3 * k + j];
            R[3 * i + j] = s;
        }
}

int64_t orc_n_rows(const orc_obs* o)
{
    int64_t nd = (int64_t)o->nR * o->nphi * o->nz;
    int64_t np = (int64_t)o->nx * o->ny;
    return nd + np + (o->gh ? 4 * np : np * o->nv);
}

/* floor((u - lo)/w) if it lies in [0, n), else -1 */
static int bin_index(double u, double lo, double w, int n)
{
    double f = floor((u - lo) / w);
    if (!(f >= 0.0) || f >= (double)n) return -1;
    return (int)f;
}

/* Modified Hermite polynomials of Gerhard (1993) / van der Marel & Franx
 * (1993), orthonormal under exp(-w^2)/sqrt(pi). */
static double hermite(int m, double w)
{
    switch (m) {
    case 0: return 1.0;
    case 1: return sqrt(2.0) * w;
    case 2: return (2.0 * w * w - 1.0) / sqrt(2.0);
    case 3: return (2.0 * sqrt(2.0) * w * w * w - 3.0 * sqrt(2.0) * w) / sqrt(6.0);
    default: return (4.0 * w * w * w * w - 12.0 * w * w + 3.0) / sqrt(24.0);
    }
}

/* Contribution of one sample (bar-frame position xb and inertial velocity in
 * bar axes vb) to an orbit's column, for each of the four mirror copies of
 * Table 1.  `col` is indexed by row; mass rows get +wt per copy (wt = 1 for
 * the fixed-step integrator: integer counts held exactly in double), GH rows
 * get wt 2 sqrt(pi) alpha(w) H_m(w) (mass-weighted linearisation of the GH
 * moments, Eq. GH and the Rix et al. 1997 estimator the paper cites).
 * gh_v0s: per pixel (v0, s). */
static void bin_sample(const orc_obs* o, const double R[9], const double* gh_v0s,
                       const double xb[3], const double vb[3], double wt, double* col)
{
    static const double sx[4] = {1, 1, -1, -1}, sz[4] = {1, -1, 1, -1};
    int64_t nd = (int64_t)o->nR * o->nphi * o->nz;
    int64_t np = (int64_t)o->nx * o->ny;
    int ncopy = o->mirror4 ? 4 : 1;
    for (int c = 0; c < ncopy; ++c) {
        double p[3] = {sx[c] * xb[0], sx[c] * xb[1], sz[c] * xb[2]};
        double u[3] = {sx[c] * vb[0], sx[c] * vb[1], sz[c] * vb[2]};
        /* 3-D density cell (Sec. 2.2.4, uniform in R, phi, z) */
        double Rc = sqrt(p[0] * p[0] + p[1] * p[1]);
        double ph = atan2(p[1], p[0]);
        if (ph < 0.0) ph += 2.0 * ORC_PI;
        int iR = bin_index(Rc, 0.0, o->Rmax / o->nR, o->nR);
        int iphi = bin_index(ph, 0.0, 2.0 * ORC_PI / o->nphi, o->nphi + 1);
        if (iphi == o->nphi) iphi = 0;   /* phi rounded up to exactly 2 pi */
        int iz = bin_index(p[2], o->zmin, (o->zmax - o->zmin) / o->nz, o->nz);
        if (iR >= 0 && iphi >= 0 && iz >= 0) col[((int64_t)iR * o->nphi + iphi) * o->nz + iz] += wt;
        /* sky projection (Eq. Euler): X = x', Y = y', v_los = v'_z */
        double X = R[0] * p[0] + R[1] * p[1] + R[2] * p[2];
        double Y = R[3] * p[0] + R[4] * p[1] + R[5] * p[2];
        double V = R[6] * u[0] + R[7] * u[1] + R[8] * u[2];
        int ix = bin_index(X, o->x0, o->dx, o->nx);
        int iy = bin_index(Y, o->y0, o->dy, o->ny);
        if (ix < 0 || iy < 0) continue;
        int64_t pix = (int64_t)iy * o->nx + ix;
        col[nd + pix] += wt;
        if (o->gh) {
            double v0 = gh_v0s[2 * pix], s = gh_v0s[2 * pix + 1];
            double w = (V - v0) / s;
            double al = exp(-0.5 * w * w) / sqrt(2.0 * ORC_PI);
            for (int m = 1; m <= 4; ++m) col[nd + np + 4 * pix + (m - 1)] += wt * 2.0 * sqrt(ORC_PI) * al * hermite(m, w);
        } else {
            int iv = bin_index(V, o->v0, o->dv, o->nv);
            if (iv >= 0) col[nd + np + pix * o->nv + iv] += wt;
        }
    }
}

/* Integrate one orbit and fill its column (length n_rows, zeroed here) with
 * sample weights 1/(ncopy * nsteps) (Sec. 2.2.4: delta t / t_total with a
 * fixed step).  Samples are taken at t_1..t_nsteps.  Returns the status:
 * 0 ok, 1 Jacobi drift > 0.1 (Sec. 2.2.2 quality cut), 2 non-finite state;
 * a rejected orbit gets an all-zero column. */
static int orbit_column(const orc_pot* p, double omega, double dt, int64_t nsteps, const double* ic,
                        const orc_obs* o, const double R[9], const double* gh_v0s, double* col, double* drift_out)
{
    int64_t M = orc_n_rows(o);
    memset(col, 0, M * sizeof(double));
    double x[3] = {ic[0], ic[1], ic[2]}, v[3] = {ic[3], ic[4], ic[5]}, acc[3], phi;
    field_inertial(p, omega, 0.0, x, &phi, acc);
    double e0 = jacobi(p, omega, 0.0, x, v), worst = 0.0;
    for (int64_t n = 0; n < nsteps; ++n) {
        kdk_step(p, omega, dt, n, x, v, acc);
        double t = (double)(n + 1) * dt;
        double e = jacobi(p, omega, t, x, v);
        double d = fabs(e - e0) / fabs(e0);
        if (isnan(d) || d > worst) worst = d;
        double th = omega * t, c = cos(th), s = sin(th);
        double xb[3] = {c * x[0] + s * x[1], -s * x[0] + c * x[1], x[2]};
        double vb[3] = {c * v[0] + s * v[1], -s * v[0] + c * v[1], v[2]};
        if (!isfinite(xb[0] + xb[1] + xb[2] + vb[0] + vb[1] + vb[2])) { worst = NAN; break; }
        bin_sample(o, R, gh_v0s, xb, vb, 1.0, col);
    }
    if (drift_out) *drift_out = worst;
    int status = isnan(worst) ? 2 : (worst > 0.1 ? 1 : 0);
    double norm = 1.0 / ((double)(o->mirror4 ? 4 : 1) * (double)nsteps);
    for (int64_t r = 0; r < M; ++r) col[r] = status ? 0.0 : col[r] * norm;
    return status;
}

/* Orbit matrix, orbit-major: U[i * n_rows + row]. */
void orc_build_matrix(const orc_pot* p, double omega, double dt, int64_t nsteps, int64_t n_orb, const double* ics,
                      const orc_obs* o, const double* gh_v0s, double* U, double* drift, int32_t* status)
{
    double R[9];
    orc_euler_matrix(o->alpha, o->beta, o->gamma, R);
    int64_t M = orc_n_rows(o);
#pragma omp parallel for schedule(dynamic, 2)
    for (int64_t i = 0; i < n_orb; ++i) {
        double d;
        int st = orbit_column(p, omega, dt, nsteps, ics + 6 * i, o, R, gh_v0s, U + i * M, &d);
        if (drift) drift[i] = d;
        if (status) status[i] = st;
    }
}

/* y = U w without storing U (for mock data at large N). */
void orc_apply_matrix(const orc_pot* p, double omega, double dt, int64_t nsteps, int64_t n_orb, const double* ics,
                      const orc_obs* o, const double* gh_v0s, const double* w, double* y)
{
    double R[9];
    orc_euler_matrix(o->alpha, o->beta, o->gamma, R);
    int64_t M = orc_n_rows(o);
    memset(y, 0, M * sizeof(double));
#pragma omp parallel
    {
        double* col = (double*)malloc(M * sizeof(double));
        double* acc = (double*)calloc(M, sizeof(double));
#pragma omp for schedule(dynamic, 2)
        for (int64_t i = 0; i < n_orb; ++i) {
            orbit_column(p, omega, dt, nsteps, ics + 6 * i, o, R, gh_v0s, col, NULL);
            for (int64_t r = 0; r < M; ++r) acc[r] += w[i] * col[r];
        }
#pragma omp critical
        for (int64_t r = 0; r < M; ++r) y[r] += acc[r];
        free(col);
        free(acc);
    }
}

/* Mass-weighted line-of-sight moments per pixel for orbit weights w:
 * out[3 p + k] = sum_i w_i (1/(ncopy S)) sum_{copies in p} V^k, k = 0, 1, 2.
 * Used to fix each pixel's reference Gaussian (v0, s) for the GH rows the way
 * Sec. 3.1 fixes them (mean and dispersion of the LOSVD). */
void orc_pixel_moments(const orc_pot* p, double omega, double dt, int64_t nsteps, int64_t n_orb, const double* ics,
                       const orc_obs* o, const double* w, double* out)
{
    double R[9];
    orc_euler_matrix(o->alpha, o->beta, o->gamma, R);
    int64_t np = (int64_t)o->nx * o->ny;
    int ncopy = o->mirror4 ? 4 : 1;
    double norm = 1.0 / ((double)ncopy * (double)nsteps);
    static const double sx[4] = {1, 1, -1, -1}, sz[4] = {1, -1, 1, -1};
    memset(out, 0, 3 * np * sizeof(double));
#pragma omp parallel
    {
        double* acc = (double*)calloc(3 * np, sizeof(double));
        double* mine = (double*)calloc(3 * np, sizeof(double));
#pragma omp for schedule(dynamic, 2)
        for (int64_t i = 0; i < n_orb; ++i) {
            const double* ic = ics + 6 * i;
            double x[3] = {ic[0], ic[1], ic[2]}, v[3] = {ic[3], ic[4], ic[5]}, a[3], phi;
            memset(mine, 0, 3 * np * sizeof(double));
            field_inertial(p, omega, 0.0, x, &phi, a);
            double e0 = jacobi(p, omega, 0.0, x, v), worst = 0.0;
            for (int64_t n = 0; n < nsteps; ++n) {
                kdk_step(p, omega, dt, n, x, v, a);
                double t = (double)(n + 1) * dt;
                double d = fabs(jacobi(p, omega, t, x, v) - e0) / fabs(e0);
                if (isnan(d) || d > worst) worst = d;
                double th = omega * t, c = cos(th), s = sin(th);
                double xb[3] = {c * x[0] + s * x[1], -s * x[0] + c * x[1], x[2]};
                double vb[3] = {c * v[0] + s * v[1], -s * v[0] + c * v[1], v[2]};
                for (int cc = 0; cc < ncopy; ++cc) {
                    double q[3] = {sx[cc] * xb[0], sx[cc] * xb[1], sz[cc] * xb[2]};
                    double u[3] = {sx[cc] * vb[0], sx[cc] * vb[1], sz[cc] * vb[2]};
                    double X = R[0] * q[0] + R[1] * q[1] + R[2] * q[2];
                    double Y = R[3] * q[0] + R[4] * q[1] + R[5] * q[2];
                    double V = R[6] * u[0] + R[7] * u[1] + R[8] * u[2];
                    int ix = bin_index(X, o->x0, o->dx, o->nx), iy = bin_index(Y, o->y0, o->dy, o->ny);
                    if (ix < 0 || iy < 0) continue;
                    int64_t pix = (int64_t)iy * o->nx + ix;
                    mine[3 * pix] += 1.0; mine[3 * pix + 1] += V; mine[3 * pix + 2] += V * V;
                }
            }
            if (!(worst > 0.1) && !isnan(worst))
                for (int64_t k = 0; k < 3 * np; ++k) acc[k] += w[i] * norm * mine[k];
        }
#pragma omp critical
        for (int64_t k = 0; k < 3 * np; ++k) out[k] += acc[k];
        free(acc);
        free(mine);
    }
}

/* ---------------------------------------------------------------------- */
/* The paper's own integrator (Sec. 2.2.2): the third-order adaptive        */
/* Runge-Kutta pair of Bogacki & Shampine (1989) with a relative tolerance  */
/* (1e-4 in the paper), run for a fixed number of accepted steps in the     */
/* frame that rotates with the bar (the bar at rest along x); the total     */
/* time then differs from orbit to orbit.  Each sample is weighted by the   */
/* step that produced it over the orbit's total time (Sec. 2.2.4).          */
/* ---------------------------------------------------------------------- */
typedef struct {
    double rtol;              /* relative tolerance on |x| and on |v| */
    double h0;                /* first trial step */
    double safety, fac_min, fac_max;   /* step-size controller */
    int32_t fixed;            /* 1: every step accepted with h = h0 (no control) */
    int32_t max_reject;       /* consecutive rejected steps that end the orbit */
} orc_bs3_opts;

/* Equations of motion in the frame rotating at omega about z (bar static):
 * dx/dt = v, dv/dt = -grad Phi(x) - 2 Omega x v - Omega x (Omega x x)
 *                  = a(x) + 2 omega (v_y, -v_x, 0) + omega^2 (x, y, 0). */
static void rot_rhs(const orc_pot* p, double omega, const double y[6], double f[6])
{
    double phi, a[3];
    pot_static(p, ORC_DISC | ORC_HALO | ORC_BAR | ORC_TEST, y, &phi, a);
    f[0] = y[3];
    f[1] = y[4];
    f[2] = y[5];
    f[3] = a[0] + 2.0 * omega * y[4] + omega * omega * y[0];
    f[4] = a[1] - 2.0 * omega * y[3] + omega * omega * y[1];
    f[5] = a[2];
}

/* One Bogacki-Shampine step of size h from y, where k1 = f(y).  Stages at
 * h/2 and 3h/4; third-order solution y_new = y + h (2 k1 + 3 k2 + 4 k3)/9;
 * k4 = f(y_new) (reused as the next step's k1); the embedded second-order
 * solution z = y + h (7 k1/24 + k2/4 + k3/3 + k4/8); err = y_new - z. */
static void bs3_step(const orc_pot* p, double omega, double h, const double y[6], const double k1[6],
                     double y_new[6], double k4[6], double err[6])
{
    double k2[6], k3[6], t[6];
    for (int i = 0; i < 6; ++i) t[i] = y[i] + 0.5 * h * k1[i];
    rot_rhs(p, omega, t, k2);
    for (int i = 0; i < 6; ++i) t[i] = y[i] + 0.75 * h * k2[i];
    rot_rhs(p, omega, t, k3);
    for (int i = 0; i < 6; ++i) y_new[i] = y[i] + h * (2.0 * k1[i] + 3.0 * k2[i] + 4.0 * k3[i]) / 9.0;
    rot_rhs(p, omega, y_new, k4);
    for (int i = 0; i < 6; ++i) {
        double z = y[i] + h * (7.0 * k1[i] / 24.0 + k2[i] / 4.0 + k3[i] / 3.0 + k4[i] / 8.0);
        err[i] = y_new[i] - z;
    }
}

static double norm3(const double* a) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* Error ratio of a step: the position and velocity parts of err each against
 * rtol times the larger of their magnitudes before and after the step. */
static double bs3_ratio(double rtol, const double y[6], const double yn[6], const double err[6])
{
    double sx = rtol * fmax(norm3(y), norm3(yn)), sv = rtol * fmax(norm3(y + 3), norm3(yn + 3));
    return fmax(norm3(err) / fmax(sx, 1e-300), norm3(err + 3) / fmax(sv, 1e-300));
}

/* Inertial initial condition at t = 0 (bar frame = inertial frame then) ->
 * rotating-frame state: v_rot = v - Omega z^ x x. */
static void to_rotating(double omega, const double* ic, double y[6])
{
    y[0] = ic[0]; y[1] = ic[1]; y[2] = ic[2];
    y[3] = ic[3] + omega * ic[1];
    y[4] = ic[4] - omega * ic[0];
    y[5] = ic[5];
}

/* Jacobi energy in the rotating frame: |v_rot|^2/2 + Phi(x) - omega^2 (x^2 + y^2)/2
 * (equal to the inertial-frame form |v|^2/2 + Phi - omega (x v_y - y v_x)). */
static double jacobi_rot(const orc_pot* p, double omega, const double y[6])
{
    double phi, a[3];
    pot_static(p, ORC_DISC | ORC_HALO | ORC_BAR | ORC_TEST, y, &phi, a);
    return 0.5 * (y[3] * y[3] + y[4] * y[4] + y[5] * y[5]) + phi - 0.5 * omega * omega * (y[0] * y[0] + y[1] * y[1]);
}

/* Advance one accepted step: on entry y, k1 = f(y) and *h the trial step; on
 * exit y, k1 for the new state, *h_used the step taken and *h the next trial
 * step.  Returns the rejected trials, or -1 after max_reject of them in a row
 * or a non-finite state. */
static int bs3_advance(const orc_pot* p, double omega, const orc_bs3_opts* o, double y[6], double k1[6], double* h,
                       double* h_used)
{
    double yn[6], k4[6], err[6];
    int rejected = 0;
    for (;;) {
        double hh = o->fixed ? o->h0 : *h;
        bs3_step(p, omega, hh, y, k1, yn, k4, err);
        double r = o->fixed ? 0.0 : bs3_ratio(o->rtol, y, yn, err);
        int finite = 1;
        for (int i = 0; i < 6; ++i) finite &= isfinite(yn[i]);
        if (!finite || isnan(r)) return -1;
        double grow = r > 0.0 ? o->safety * pow(r, -1.0 / 3.0) : o->fac_max;
        grow = fmin(o->fac_max, fmax(o->fac_min, grow));
        if (r <= 1.0) {
            memcpy(y, yn, sizeof yn);
            memcpy(k1, k4, sizeof k4);
            *h_used = hh;
            *h = hh * grow;
            return rejected;
        }
        *h = hh * grow;
        if (++rejected >= o->max_reject) return -1;
    }
}

/* nsteps accepted steps from an inertial initial condition.  ts[n] (n = 0..nsteps)
 * the times and ys[6 n + k] the rotating-frame states (both nullable).  Returns the
 * total number of rejected trial steps, or -1 if the orbit had to be abandoned. */
int64_t orc_bs3_trajectory(const orc_pot* p, double omega, const orc_bs3_opts* o, int64_t nsteps, const double* ic,
                           double* ts, double* ys)
{
    double y[6], k1[6], h = o->h0, t = 0.0;
    int64_t rej = 0;
    to_rotating(omega, ic, y);
    rot_rhs(p, omega, y, k1);
    if (ts) ts[0] = 0.0;
    if (ys) memcpy(ys, y, sizeof y);
    for (int64_t n = 0; n < nsteps; ++n) {
        double hu;
        int r = bs3_advance(p, omega, o, y, k1, &h, &hu);
        if (r < 0) return -1;
        rej += r;
        t += hu;
        if (ts) ts[n + 1] = t;
        if (ys) memcpy(ys + 6 * (n + 1), y, sizeof y);
    }
    return rej;
}

/* One orbit's column from the adaptive integrator: the sample after accepted
 * step n (n = 1..nsteps) has weight h_n / t_total (Sec. 2.2.4) shared by its
 * mirror copies; its bar-frame position is the state's x and its velocity the
 * inertial one in bar axes, v_rot + Omega z^ x x (Sec. 2.2.2: velocities are
 * taken back to the inertial frame for the comparison with data).  Status as
 * in orbit_column; 2 also when the step control gave up. */
static int orbit_column_bs3(const orc_pot* p, double omega, const orc_bs3_opts* opt, int64_t nsteps,
                            const double* ic, const orc_obs* o, const double R[9], const double* gh_v0s, double* col,
                            double* drift_out)
{
    int64_t M = orc_n_rows(o);
    memset(col, 0, M * sizeof(double));
    double y[6], k1[6], h = opt->h0, total = 0.0;
    to_rotating(omega, ic, y);
    rot_rhs(p, omega, y, k1);
    double e0 = jacobi_rot(p, omega, y), worst = 0.0;
    for (int64_t n = 0; n < nsteps; ++n) {
        double hu;
        if (bs3_advance(p, omega, opt, y, k1, &h, &hu) < 0) { worst = NAN; break; }
        total += hu;
        double d = fabs(jacobi_rot(p, omega, y) - e0) / fabs(e0);
        if (isnan(d) || d > worst) worst = d;
        double vb[3] = {y[3] - omega * y[1], y[4] + omega * y[0], y[5]};
        bin_sample(o, R, gh_v0s, y, vb, hu, col);
    }
    if (drift_out) *drift_out = worst;
    int status = isnan(worst) ? 2 : (worst > 0.1 ? 1 : 0);
    double norm = 1.0 / ((double)(o->mirror4 ? 4 : 1) * total);
    for (int64_t r = 0; r < M; ++r) col[r] = status ? 0.0 : col[r] * norm;
    return status;
}

/* Orbit matrix from the adaptive integrator, orbit-major as orc_build_matrix. */
void orc_build_matrix_bs3(const orc_pot* p, double omega, const orc_bs3_opts* opt, int64_t nsteps, int64_t n_orb,
                          const double* ics, const orc_obs* o, const double* gh_v0s, double* U, double* drift,
                          int32_t* status)
{
    double R[9];
    orc_euler_matrix(o->alpha, o->beta, o->gamma, R);
    int64_t M = orc_n_rows(o);
#pragma omp parallel for schedule(dynamic, 2)
    for (int64_t i = 0; i < n_orb; ++i) {
        double d;
        int st = orbit_column_bs3(p, omega, opt, nsteps, ics + 6 * i, o, R, gh_v0s, U + i * M, &d);
        if (drift) drift[i] = d;
        if (status) status[i] = st;
    }
}

/* One step from a rotating-frame state (for the order pins): y_new and err. */
void orc_bs3_single_step(const orc_pot* p, double omega, double h, const double* y, double* y_new, double* err)
{
    double k1[6], k4[6];
    rot_rhs(p, omega, y, k1);
    bs3_step(p, omega, h, y, k1, y_new, k4, err);
}

/* Jacobi energy of a rotating-frame state. */
double orc_jacobi_rot(const orc_pot* p, double omega, const double* y)
{
    return jacobi_rot(p, omega, y);
}

/* Per-sample Gauss-Hermite row weights 2 sqrt(pi) alpha(w) H_m(w), m = 0..4. */
void orc_gh_weights(double w, double* out)
{
    double al = exp(-0.5 * w * w) / sqrt(2.0 * ORC_PI);
    for (int m = 0; m <= 4; ++m) out[m] = 2.0 * sqrt(ORC_PI) * al * hermite(m, w);
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
