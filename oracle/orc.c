/*
 * FP64 CPU oracle for the SFF-PIC step (arXiv 2310.11393).  TEST INFRASTRUCTURE:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 *
 * One time step, in the order of Sec. 2 (text after Eq. "scatt_field"):
 *   1. interpolate the grid-held scattered field E_s, B_s to each macro-electron
 *      with order-2 (quadratic B-spline) shapes on the Yee stagger (order 2:
 *      Sec. 3.1, "default interpolation order is 2");
 *   2. add the closed-form incident field E_inc, B_inc evaluated at the particle
 *      position and time (Sec. 2: "added to the incident field at the position of
 *      the macroparticle");
 *   3. relativistic Boris push of the Lorentz force in Eq. (vlasov);
 *   4. Esirkepov charge-conserving current deposition of the straight move;
 *   5. Yee update (Eqs. MAmper, MFaraday) of the scattered field only, driven by J.
 * The magnetic field is kept at integer times and advanced in two half steps
 * around the electric update; this is the leapfrog with the magnetic field
 * time-centred for the gather.
 *
 * Readings of the paper taken here (the paper is silent on them):
 *   - open boxes use first-order Mur conditions on the tangential E of every face;
 *   - particles closer than `remove_margin` cells to a face are removed after their
 *     deposit, and their momenta are kept as exit records;
 *   - immobile ions: rho_ion = -rho_e at creation (so div E = rho holds at t = 0
 *     with E = 0 and no Poisson solve is needed);
 *   - LP closed form: the printed expansion (Sec. 4.1) with (x^2/r^2) sin^2(theta)
 *     written as xi^2/R^2 and (x/r) sin(theta) as xi/R so that it holds on the axis;
 *   - RP: the paper cites April (2010) without formulas; the field is generated by
 *     the electric Hertz vector Psi z^ with the same Psi (Eq. phasor):
 *     E = grad(d_z Psi) - d_tt Psi z^, B = d_t curl(Psi z^);
 *   - |R~| < 0.2 (the ring R~ = 0 where the printed terms cancel): Psi is expanded
 *     in powers of u = R~^2 about u = 0 and the same component rules are applied.
 */
#include "orc.h"
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_RING_SWITCH 0.2

/* ------------------------------------------------------------------------------
 * SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state advances by the golden
 * gamma, output is the variant-13 finaliser.  The k-th output of the stream that
 * starts at `seed` is mix(seed + (k+1) * gamma).
 * ------------------------------------------------------------------------------ */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ==============================================================================
 * Incident fields
 * ============================================================================== */

/* Eq. (poisson_dstr): g^(n)(tau) = e^{i phi0} Gamma(s+n+1)/Gamma(s+1) (i k a/s)^n (1 - i tau/s)^{-(s+n+1)}, k = 1 */
static cplx g_n(int n, cplx tau, double a, double s, double phi0)
{
    double gratio = 1.0;
    cplx ias_n = 1.0;
    for (int k = 1; k <= n; k++) {
        gratio *= (s + k);
        ias_n *= I * a / s;
    }
    return cexp(I * phi0) * gratio * ias_n * cpow(1.0 - I * tau / s, -(s + n + 1));
}

/* Series about the ring u = R~^2 = 0.  Psi = (Psi0/a) Phi(u, tau) with
 *   Phi = [g(tau0 + a R) - g(tau0 - a R)] / R = 2 sum_j c_{2j+1} u^j,
 *   c_k = g^(k)(tau0)/k!,  tau0 = tau + i a,
 * (g^(k) of Eq. poisson_dstr is the k-th derivative of g with respect to tau/a).
 * Returns Phi_u, Phi_uu, Phi_uD, Phi_DD where D = a d/dtau. */
static void phi_series(double a, double s, double phi0, cplx u, double tau, cplx out[4])
{
    cplx tau0 = tau + I * a;
    cplx w0 = 1.0 - I * tau0 / s;
    cplx q = I * a / (s * w0);                  /* (i a/s)^k (1 - i tau0/s)^{-k} = q^k */
    cplx base = cexp(I * phi0) * cpow(w0, -(s + 1));
    cplx Su = 0, Suu = 0, SuD = 0, SDD = 0;
    cplx pj = 1.0, pjm1 = 0.0, pjm2 = 0.0;      /* u^j, u^(j-1), u^(j-2) (0 when negative) */
    int small = 0;
    for (int j = 0; j < 600; j++) {
        /* c_k for k = 2j+1, 2j+2, 2j+3: binomial(s+k, k) q^k g(tau0) */
        cplx ck[3];
        for (int m = 0; m < 3; m++) {
            int k = 2 * j + 1 + m;
            double lb = lgamma(s + k + 1) - lgamma(s + 1) - lgamma((double)k + 1);
            ck[m] = base * exp(lb) * cpow(q, k);
        }
        cplx a1 = 2.0 * j * ck[0] * pjm1;                      /* Phi_u  : 2 j c_{2j+1} u^{j-1} */
        cplx a2 = 2.0 * j * (j - 1) * ck[0] * pjm2;            /* Phi_uu : 2 j (j-1) c_{2j+1} u^{j-2} */
        cplx a3 = 2.0 * j * (2 * j + 2) * ck[1] * pjm1;        /* Phi_uD : 2 j (2j+2) c_{2j+2} u^{j-1} */
        cplx a4 = 2.0 * (2 * j + 2) * (2 * j + 3) * ck[2] * pj; /* Phi_DD : 2 (2j+2)(2j+3) c_{2j+3} u^j */
        Su += a1; Suu += a2; SuD += a3; SDD += a4;
        double mag = cabs(a1) + cabs(a2) + cabs(a3) + cabs(a4);
        double tot = cabs(Su) + cabs(Suu) + cabs(SuD) + cabs(SDD);
        if (j > 4 && mag <= 1e-18 * tot) {
            if (++small >= 2) break;
        } else {
            small = 0;
        }
        pjm2 = pjm1; pjm1 = pj; pj *= u;
    }
    out[0] = Su; out[1] = Suu; out[2] = SuD; out[3] = SDD;
}

/* Component rules applied to Psi = (Psi0/a) Phi(u, tau): d_x u = 2 xi/a, d_z u = 2(zeta+i)/a,
 * d_t = D/a.  LP: Eq. (components).  RP: Hertz vector Psi z^. */
static void fields_from_phi(int beam, double kscale, double xi, double eta, double zeta,
                            const cplx P[4], cplx E[3], cplx B[3])
{
    cplx zi = zeta + I;
    cplx Pu = P[0], Puu = P[1], PuD = P[2], PDD = P[3];
    if (beam == ORC_BEAM_LP) {
        E[0] = kscale * (2.0 * Pu + 4.0 * xi * xi * Puu - PDD + 2.0 * zi * PuD);   /* d_xx - d_tt + d_tz */
        E[1] = kscale * (4.0 * xi * eta * Puu);                                     /* d_xy */
        E[2] = kscale * (4.0 * xi * zi * Puu - 2.0 * xi * PuD);                     /* d_zx - d_tx */
        B[0] = kscale * (4.0 * xi * eta * Puu);                                     /* d_xy */
        B[1] = kscale * (2.0 * Pu + 4.0 * eta * eta * Puu - PDD + 2.0 * zi * PuD);  /* d_yy - d_tt + d_tz */
        B[2] = kscale * (4.0 * eta * zi * Puu - 2.0 * eta * PuD);                   /* d_zy - d_ty */
    } else {
        E[0] = kscale * (4.0 * xi * zi * Puu);                                      /* d_xz */
        E[1] = kscale * (4.0 * eta * zi * Puu);                                     /* d_yz */
        E[2] = kscale * (2.0 * Pu + 4.0 * zi * zi * Puu - PDD);                     /* d_zz - d_tt */
        B[0] = kscale * (2.0 * eta * PuD);                                          /* d_ty */
        B[1] = -kscale * (2.0 * xi * PuD);                                          /* -d_tx */
        B[2] = 0;
    }
}

/* Closed forms in the paper's notation (Sec. 4.1): R = R~/a = sqrt(rho^2 + (zeta+i)^2),
 * tau_pm = tau + a(+-R + i), G^(n)_pm = g^(n)(tau_+) +- g^(n)(tau_-),
 * cos(theta) = (zeta+i)/R, sin(theta) = rho/R. */
static void beam_closed(int beam, double a, double s, double psi0, double phi0,
                        double xi, double eta, double zeta, double tau, cplx R, cplx E[3], cplx B[3])
{
    cplx taup = tau + a * (R + I);
    cplx taum = tau + a * (-R + I);
    cplx g0p = g_n(0, taup, a, s, phi0), g0m = g_n(0, taum, a, s, phi0);
    cplx g1p = g_n(1, taup, a, s, phi0), g1m = g_n(1, taum, a, s, phi0);
    cplx g2p = g_n(2, taup, a, s, phi0), g2m = g_n(2, taum, a, s, phi0);
    cplx G0m = g0p - g0m;
    cplx G1p = g1p + g1m, G1m = g1p - g1m;
    cplx G2p = g2p + g2m, G2m = g2p - g2m;
    cplx cth = (zeta + I) / R;
    cplx R2 = R * R;
    double k = psi0 / (a * a * a);
    /* bracket shared by the sin^2(theta) terms, divided by R */
    cplx T1 = (3.0 * G0m / R2 - 3.0 * G1p / R + G2m) / R;
    if (beam == ORC_BEAM_LP) {
        cplx A = (G0m / R2 + G1m * cth / R - G1p / R + G2m - G2p * cth) / R;
        cplx Qb = 3.0 * G0m * cth / R2 + G1m / R - 3.0 * G1p * cth / R + G2m * cth - G2p;
        E[0] = k * (xi * xi / R2 * T1 - A);
        E[1] = k * (xi * eta / R2 * T1);
        E[2] = k * (xi / R2 * Qb);
        B[0] = k * (xi * eta / R2 * T1);
        B[1] = k * (eta * eta / R2 * T1 - A);
        B[2] = k * (eta / R2 * Qb);
    } else {
        /* Hertz vector Psi z^: 4 Phi_uu = T1/R^2, 2 Phi_u = G1+/R^2 - G0-/R^3,
         * Phi_DD = G2-/R, 2 Phi_uD = G2+/R^2 - G1-/R^3 */
        cplx zi = zeta + I;
        cplx PuD2 = G2p / R2 - G1m / (R2 * R);
        E[0] = k * (xi * zi * T1 / R2);
        E[1] = k * (eta * zi * T1 / R2);
        E[2] = k * ((G1p / R2 - G0m / (R2 * R)) + zi * zi * T1 / R2 - G2m / R);
        B[0] = k * (eta * PuD2);
        B[1] = -k * (xi * PuD2);
        B[2] = 0;
    }
}

void orc_beam_complex(int beam, double a, double s, double psi0, double phi0,
                      double X, double Y, double Z, double tau, int branch,
                      double Ere[3], double Eim[3], double Bre[3], double Bim[3])
{
    double xi = X / a, eta = Y / a, zeta = Z / a;
    cplx u = xi * xi + eta * eta + (zeta + I) * (zeta + I);
    cplx R = csqrt(u);
    cplx E[3], B[3];
    int use_series = (branch == 2) || (branch == 0 && cabs(R) < ORC_RING_SWITCH);
    if (use_series) {
        cplx P[4];
        phi_series(a, s, phi0, u, tau, P);
        fields_from_phi(beam, psi0 / (a * a * a), xi, eta, zeta, P, E, B);
    } else {
        beam_closed(beam, a, s, psi0, phi0, xi, eta, zeta, tau, R, E, B);
    }
    for (int c = 0; c < 3; c++) {
        Ere[c] = creal(E[c]); Eim[c] = cimag(E[c]);
        Bre[c] = creal(B[c]); Bim[c] = cimag(B[c]);
    }
}

void orc_lp_field(double a, double s, double psi0, double phi0,
                  double X, double Y, double Z, double tau, int branch, double E[3], double B[3])
{
    double Ei[3], Bi[3];
    orc_beam_complex(ORC_BEAM_LP, a, s, psi0, phi0, X, Y, Z, tau, branch, E, Ei, B, Bi);
}

void orc_rp_field(double a, double s, double psi0, double phi0,
                  double X, double Y, double Z, double tau, int branch, double E[3], double B[3])
{
    double Ei[3], Bi[3];
    orc_beam_complex(ORC_BEAM_RP, a, s, psi0, phi0, X, Y, Z, tau, branch, E, Ei, B, Bi);
}

/* Plane wave travelling toward +x, polarised along y (the 1D solution of Sec. 3.1,
 * with the propagation axis named x): E_y = B_z = a0 sin(xi - xi_c + phi0) env(xi),
 * xi = t - (x - x_ref).  Envelope: Gaussian 2^{-4(xi - t_c)^2/FWHM^2} (Sec. 3.1) or
 * sin^2(pi xi / (2 FWHM)) on [0, 2 FWHM] whose field FWHM is FWHM. */
static double plane_wave(const orc_config* c, double x, double t)
{
    double xi = t - (x - c->focus[0]);
    double T = c->duration;
    double env, xic;
    if (c->envelope == ORC_ENV_GAUSS) {
        xic = c->t_focus;
        env = pow(2.0, -4.0 * (xi - xic) * (xi - xic) / (T * T));
    } else {
        xic = T;
        if (xi <= 0.0 || xi >= 2.0 * T) return 0.0;
        double sn = sin(M_PI * xi / (2.0 * T));
        env = sn * sn;
    }
    return c->a0 * sin(xi - xic + c->phi0) * env;
}

/* 2D paraxial Gaussian beam of Sec. 3.2, Eq. (gauss2D), focus at the origin of (X, Z),
 * propagation +Z, polarisation X (the paper's x, z), k = omega = 1:
 *   w(Z) = w0 sqrt(1 + (Z/zR)^2), zR = w0^2/2, 1/R(Z) = Z/(Z^2 + zR^2), eta = atan(Z/zR)/2,
 *   E_x = E0 sqrt(w0/w) exp(-X^2/w^2) cos(Z - t + X^2/(2R) - eta + phi0) env,  B_y = E_x,
 *   E_z = E0 sqrt(w0/w) exp(-X^2/w^2) [2 (X/w^2) sin(same phase) - (X/R) cos(same phase)] env,
 *   env = 2^{-4 (t - t0 - Z)^2 / FWHM_T^2}.
 * E_z is the longitudinal field to first order in 1/(k w0), the one that makes div E vanish
 * to that order at every Z (E_z = Re[i dA/dX e^{i(Z-t)}] for E_x = Re[A e^{i(Z-t)}]).  At
 * the focus (1/R = 0) it is the printed form, with the printed factor X/w(Z) read as
 * X/w(Z)^2; the printed form omits the curvature term -(X/R) cos, of the same order. */
static void gauss2d_field(const orc_config* c, double Z, double X, double t, double Ep[3], double Bp[3])
{
    const double w0 = c->w0, zR = 0.5 * w0 * w0;
    const double w = w0 * sqrt(1.0 + (Z / zR) * (Z / zR));
    const double invR = Z / (Z * Z + zR * zR);
    const double eta = 0.5 * atan(Z / zR);
    const double xi = t - c->t_focus - Z;
    const double env = pow(2.0, -4.0 * xi * xi / (c->duration * c->duration));
    const double amp = c->a0 * sqrt(w0 / w) * exp(-X * X / (w * w)) * env;
    const double ph = Z - t + 0.5 * X * X * invR - eta + c->phi0;
    Ep[0] = amp * cos(ph);
    Ep[1] = 0.0;
    Ep[2] = amp * (2.0 * X / (w * w) * sin(ph) - X * invR * cos(ph));
    Bp[0] = 0.0;
    Bp[1] = Ep[0];
    Bp[2] = 0.0;
}

void orc_incident(const orc_config* c, const double x[3], double t, double E[3], double B[3])
{
    for (int d = 0; d < 3; d++) { E[d] = 0; B[d] = 0; }
    switch (c->beam) {
    case ORC_BEAM_PLANE: {
        double f = plane_wave(c, x[0], t);
        E[1] = f; B[2] = f;
        break;
    }
    case ORC_BEAM_LP:
    case ORC_BEAM_RP: {
        /* beam frame: paper z = grid x (propagation), paper x = grid y (polarisation), paper y = grid z */
        double Z = x[0] - c->focus[0];
        double X = (c->dim >= 2) ? x[1] - c->focus[1] : 0.0;
        double Y = (c->dim >= 3) ? x[2] - c->focus[2] : 0.0;
        double Ep[3], Bp[3];
        if (c->beam == ORC_BEAM_LP) orc_lp_field(c->a, c->s, c->psi0, c->phi0, X, Y, Z, t - c->t_focus, 0, Ep, Bp);
        else orc_rp_field(c->a, c->s, c->psi0, c->phi0, X, Y, Z, t - c->t_focus, 0, Ep, Bp);
        E[0] = Ep[2]; E[1] = Ep[0]; E[2] = Ep[1];
        B[0] = Bp[2]; B[1] = Bp[0]; B[2] = Bp[1];
        break;
    }
    case ORC_BEAM_UNIFORM:
        for (int d = 0; d < 3; d++) { E[d] = c->e_unif[d]; B[d] = c->b_unif[d]; }
        break;
    case ORC_BEAM_GAUSS2D: {
        /* same frame as the 2D slice of LP/RP: paper z = grid x, paper x = grid y */
        double Ep[3], Bp[3];
        gauss2d_field(c, x[0] - c->focus[0], (c->dim >= 2) ? x[1] - c->focus[1] : 0.0, t, Ep, Bp);
        E[0] = Ep[2]; E[1] = Ep[0]; E[2] = Ep[1];
        B[0] = Bp[2]; B[1] = Bp[0]; B[2] = Bp[1];
        break;
    }
    default:
        break;
    }
}

/* ==============================================================================
 * Pulse parameters (Sec. 4.1)
 * ============================================================================== */
double orc_a_from_w0(double w0)
{
    /* k^2 w0^2 = 2 (sqrt(1 + (k a)^2) - 1), k = 1 */
    double h = 1.0 + 0.5 * w0 * w0;
    return sqrt(h * h - 1.0);
}

/* modulus of the on-axis focal complex field: LP -> E_x, RP -> E_z (the only on-axis component) */
static double focal_env(int beam, double a, double s, double tau)
{
    double Er[3], Ei[3], Br[3], Bi[3];
    orc_beam_complex(beam, a, s, 1.0, 0.0, 0.0, 0.0, 0.0, tau, 0, Er, Ei, Br, Bi);
    int c = (beam == ORC_BEAM_LP) ? 0 : 2;
    return hypot(Er[c], Ei[c]);
}

static double focal_peak(int beam, double a, double s, double* tpk)
{
    /* coarse scan, then golden-section refinement of the maximum */
    int n = 400;
    double lo = -2.0 * s, hi = 2.0 * s, best = -1, tb = 0;
    for (int i = 0; i <= n; i++) {
        double t = lo + (hi - lo) * i / n;
        double v = focal_env(beam, a, s, t);
        if (v > best) { best = v; tb = t; }
    }
    double h = (hi - lo) / n;
    double l = tb - h, r = tb + h;
    const double gr = 0.5 * (sqrt(5.0) - 1.0);
    double c1 = r - gr * (r - l), c2 = l + gr * (r - l);
    double f1 = focal_env(beam, a, s, c1), f2 = focal_env(beam, a, s, c2);
    for (int it = 0; it < 200 && (r - l) > 1e-13 * (1.0 + fabs(tb)); it++) {
        if (f1 > f2) { r = c2; c2 = c1; f2 = f1; c1 = r - gr * (r - l); f1 = focal_env(beam, a, s, c1); }
        else { l = c1; c1 = c2; f1 = f2; c2 = l + gr * (r - l); f2 = focal_env(beam, a, s, c2); }
    }
    *tpk = 0.5 * (l + r);
    return focal_env(beam, a, s, *tpk);
}

static double half_crossing(int beam, double a, double s, double tpk, double half, double dir)
{
    double l = tpk, r = tpk + dir * 60.0 * s;
    for (int it = 0; it < 300; it++) {
        double m = 0.5 * (l + r);
        if (focal_env(beam, a, s, m) > half) l = m; else r = m;
        if (fabs(r - l) < 1e-13 * (1.0 + fabs(m))) break;
    }
    return 0.5 * (l + r);
}

double orc_focal_fwhm(int beam, double a, double s)
{
    double tpk;
    double pk = focal_peak(beam, a, s, &tpk);
    double tr = half_crossing(beam, a, s, tpk, 0.5 * pk, +1.0);
    double tl = half_crossing(beam, a, s, tpk, 0.5 * pk, -1.0);
    return tr - tl;
}

double orc_s_from_duration(int beam, double a, double duration)
{
    double lo = 1.0, hi = 1.0e4;
    for (int it = 0; it < 200; it++) {
        double m = 0.5 * (lo + hi);
        if (orc_focal_fwhm(beam, a, m) < duration) lo = m; else hi = m;
        if (hi - lo < 1e-12 * m) break;
    }
    return 0.5 * (lo + hi);
}

double orc_psi0_from_a0(int beam, double a, double s, double a0)
{
    double tpk;
    return a0 / focal_peak(beam, a, s, &tpk);
}

/* ==============================================================================
 * Simulation
 * ============================================================================== */
struct orc_sim {
    orc_config c;
    int res[3];        /* axis resolved? */
    int ext[3];        /* array extent per axis */
    int64_t nnode;
    double* F[9];      /* Ex Ey Ez Bx By Bz Jx Jy Jz */
    double* Finc[6];   /* incident E, B on the Yee nodes at t^n (incident_grid runs only) */
    double* rho_ion;
    int64_t np, cap;
    double *px, *pu, *pw;
    int64_t* pid;
    int64_t nexit, capexit;
    double *eu, *ew;
    int64_t *eid, *estep;
    int64_t step;
};

static inline int64_t IX(const orc_sim* s, int i, int j, int k)
{
    return (int64_t)i + (int64_t)s->ext[0] * ((int64_t)j + (int64_t)s->ext[1] * k);
}

static inline int periodic(const orc_sim* s) { return s->c.field_bc == ORC_BC_PERIODIC; }

static inline int wrapi(const orc_sim* s, int d, int i)
{
    if (periodic(s) && s->res[d]) {
        int N = s->c.n[d];
        i %= N;
        if (i < 0) i += N;
    }
    return i;
}

/* field component value at an integer index triple, periodic axes wrapped */
static inline double* ref(orc_sim* s, int comp, const int idx[3])
{
    return &s->F[comp][IX(s, wrapi(s, 0, idx[0]), wrapi(s, 1, idx[1]), wrapi(s, 2, idx[2]))];
}
static inline double val(const orc_sim* s, int comp, const int idx[3])
{
    return s->F[comp][IX(s, wrapi(s, 0, idx[0]), wrapi(s, 1, idx[1]), wrapi(s, 2, idx[2]))];
}

/* Yee stagger: E_c and J_c are at half-integer positions along axis c; B_c along the two others */
static inline int staggered(int comp, int d)
{
    int c = comp % 3;
    if (comp < 3 || comp >= 6) return d == c;
    return d != c;
}

/* number of stored points of a component along an axis */
static int npts(const orc_sim* s, int comp, int d)
{
    if (!s->res[d]) return 1;
    if (periodic(s)) return s->c.n[d];
    return staggered(comp, d) ? s->c.n[d] : s->c.n[d] + 1;
}

static void ensure_cap(orc_sim* s, int64_t n)
{
    if (n <= s->cap) return;
    int64_t cap = n;
    s->px = realloc(s->px, sizeof(double) * 3 * cap);
    s->pu = realloc(s->pu, sizeof(double) * 3 * cap);
    s->pw = realloc(s->pw, sizeof(double) * cap);
    s->pid = realloc(s->pid, sizeof(int64_t) * cap);
    s->cap = cap;
}

/* quadratic B-spline weights for offset delta in [-1/2, 1/2] from the nearest node */
static void shape2(double delta, double w[3])
{
    w[0] = 0.5 * (0.5 - delta) * (0.5 - delta);
    w[1] = 0.75 - delta * delta;
    w[2] = 0.5 * (0.5 + delta) * (0.5 + delta);
}

void orc_charge_density(const orc_sim* s, double* out)
{
    memset(out, 0, sizeof(double) * s->nnode);
    for (int64_t p = 0; p < s->np; p++) {
        int lo[3], na[3];
        double w[3][3];
        for (int d = 0; d < 3; d++) {
            if (s->res[d]) {
                double X = s->px[3 * p + d] / s->c.dx;
                int i = (int)floor(X + 0.5);
                shape2(X - i, w[d]);
                lo[d] = i - 1; na[d] = 3;
            } else {
                lo[d] = 0; na[d] = 1; w[d][0] = 1.0;
            }
        }
        for (int c = 0; c < na[2]; c++)
            for (int b = 0; b < na[1]; b++)
                for (int a = 0; a < na[0]; a++) {
                    int i = wrapi(s, 0, lo[0] + a), j = wrapi(s, 1, lo[1] + b), k = wrapi(s, 2, lo[2] + c);
                    out[IX(s, i, j, k)] += -1.0 * s->pw[p] * w[0][a] * w[1][b] * w[2][c];
                }
    }
}

/* density profile along x at position x (code units): Sec. 3.1's super-Gaussian
 * n(x)/n0 = 2^-|2 (x - x0)/FWHM|^p beyond the cut (0 before it), or 1 (the paper's p = 12 is
 * even; the modulus keeps odd orders meaningful) */
static double profile_factor(const orc_config* c, double x)
{
    if (c->profile != ORC_PROFILE_SUPERGAUSS) return 1.0;
    if (x <= c->prof_cut) return 0.0;
    return pow(2.0, -pow(fabs(2.0 * (x - c->prof_x0) / c->prof_fwhm), (double)c->prof_order));
}

orc_sim* orc_create(const orc_config* cfg)
{
    orc_sim* s = calloc(1, sizeof(orc_sim));
    s->c = *cfg;
    if (s->c.remove_margin <= 0) s->c.remove_margin = 3;
    s->nnode = 1;
    for (int d = 0; d < 3; d++) {
        s->res[d] = d < cfg->dim;
        s->ext[d] = s->res[d] ? cfg->n[d] + 1 : 1;
        s->nnode *= s->ext[d];
    }
    for (int c = 0; c < 9; c++) s->F[c] = calloc(s->nnode, sizeof(double));
    for (int c = 0; c < 6; c++) s->Finc[c] = cfg->incident_grid ? calloc(s->nnode, sizeof(double)) : NULL;
    s->rho_ion = calloc(s->nnode, sizeof(double));

    /* seeded slab: slab cells in x-fastest order, ppc particles per cell; particle p
     * draws outputs 3p, 3p+1, 3p+2 of SplitMix64(seed); offset = top 24 bits / 2^24 */
    int64_t ns[3] = {1, 1, 1}, np = 0;
    if (cfg->ppc > 0) {
        np = cfg->ppc;
        for (int d = 0; d < cfg->dim; d++) {
            ns[d] = cfg->slab_hi[d] - cfg->slab_lo[d];
            if (ns[d] < 0) ns[d] = 0;
            np *= ns[d];
        }
    }
    ensure_cap(s, np > 0 ? np : 1);
    int64_t p = 0;
    for (int64_t cz = 0; cz < ns[2]; cz++)
        for (int64_t cy = 0; cy < ns[1]; cy++)
            for (int64_t cx = 0; cx < ns[0]; cx++)
                for (int k = 0; k < cfg->ppc; k++, p++) {
                    int64_t cell[3] = {cx, cy, cz};
                    for (int d = 0; d < 3; d++) {
                        if (d < cfg->dim) {
                            uint64_t r = orc_splitmix64(cfg->seed, 3 * (uint64_t)p + d);
                            double off = (double)(r >> 40) * (1.0 / 16777216.0);
                            s->px[3 * p + d] = ((double)(cfg->slab_lo[d] + cell[d]) + off) * cfg->dx;
                        } else {
                            s->px[3 * p + d] = 0.0;
                        }
                        s->pu[3 * p + d] = 0.0;
                    }
                    s->pw[p] = cfg->n_e / cfg->ppc * profile_factor(cfg, s->px[3 * p]);
                    s->pid[p] = p;
                }
    s->np = np;
    orc_charge_density(s, s->rho_ion);
    for (int64_t i = 0; i < s->nnode; i++) s->rho_ion[i] = -s->rho_ion[i];
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    for (int c = 0; c < 9; c++) free(s->F[c]);
    for (int c = 0; c < 6; c++) free(s->Finc[c]);
    free(s->rho_ion);
    free(s->px); free(s->pu); free(s->pw); free(s->pid);
    free(s->eu); free(s->ew); free(s->eid); free(s->estep);
    free(s);
}

int64_t orc_num_particles(const orc_sim* s) { return s->np; }
int64_t orc_num_exits(const orc_sim* s) { return s->nexit; }
int64_t orc_step_index(const orc_sim* s) { return s->step; }
void orc_extents(const orc_sim* s, int ext[3]) { for (int d = 0; d < 3; d++) ext[d] = s->ext[d]; }

void orc_set_particles(orc_sim* s, int64_t n, const double* x, const double* u, const double* w, const int64_t* id)
{
    ensure_cap(s, n > 0 ? n : 1);
    memcpy(s->px, x, sizeof(double) * 3 * n);
    memcpy(s->pu, u, sizeof(double) * 3 * n);
    memcpy(s->pw, w, sizeof(double) * n);
    memcpy(s->pid, id, sizeof(int64_t) * n);
    s->np = n;
    if (s->step == 0) {
        orc_charge_density(s, s->rho_ion);
        for (int64_t i = 0; i < s->nnode; i++) s->rho_ion[i] = -s->rho_ion[i];
    }
}

void orc_get_particles(const orc_sim* s, double* x, double* u, double* w, int64_t* id)
{
    memcpy(x, s->px, sizeof(double) * 3 * s->np);
    memcpy(u, s->pu, sizeof(double) * 3 * s->np);
    memcpy(w, s->pw, sizeof(double) * s->np);
    memcpy(id, s->pid, sizeof(int64_t) * s->np);
}

void orc_get_exits(const orc_sim* s, double* u, double* w, int64_t* id, int64_t* step)
{
    memcpy(u, s->eu, sizeof(double) * 3 * s->nexit);
    memcpy(w, s->ew, sizeof(double) * s->nexit);
    memcpy(id, s->eid, sizeof(int64_t) * s->nexit);
    memcpy(step, s->estep, sizeof(int64_t) * s->nexit);
}

void orc_get_fields(const orc_sim* s, double* out)
{
    for (int c = 0; c < 9; c++) memcpy(out + c * s->nnode, s->F[c], sizeof(double) * s->nnode);
}

void orc_set_fields(orc_sim* s, const double* in)
{
    for (int c = 0; c < 9; c++) memcpy(s->F[c], in + c * s->nnode, sizeof(double) * s->nnode);
}

/* ---- gather -------------------------------------------------------------------- */
static double gather_from(const orc_sim* s, const double* arr, int comp, const double X[3]);

static double gather(const orc_sim* s, int comp, const double X[3]) { return gather_from(s, s->F[comp], comp, X); }

static double gather_from(const orc_sim* s, const double* arr, int comp, const double X[3])
{
    int lo[3], na[3];
    double w[3][3];
    for (int d = 0; d < 3; d++) {
        if (s->res[d]) {
            double Y = X[d] - (staggered(comp, d) ? 0.5 : 0.0);
            int i = (int)floor(Y + 0.5);
            shape2(Y - i, w[d]);
            lo[d] = i - 1; na[d] = 3;
        } else {
            lo[d] = 0; na[d] = 1; w[d][0] = 1.0;
        }
    }
    double v = 0.0;
    for (int c = 0; c < na[2]; c++)
        for (int b = 0; b < na[1]; b++)
            for (int a = 0; a < na[0]; a++) {
                int idx[3] = {lo[0] + a, lo[1] + b, lo[2] + c};
                v += w[0][a] * w[1][b] * w[2][c] *
                     arr[IX(s, wrapi(s, 0, idx[0]), wrapi(s, 1, idx[1]), wrapi(s, 2, idx[2]))];
            }
    return v;
}

/* ---- Esirkepov deposition (order-2 shapes, straight move xo -> xn) ---------------- */
static void deposit(orc_sim* s, const double xo[3], const double xn[3], const double v[3], double w)
{
    const double q = -1.0;
    const double dx = s->c.dx, dt = s->c.dt;
    double S0[3][5], DS[3][5];
    int i0[3], lo[3], hi[3];
    for (int d = 0; d < 3; d++) {
        for (int m = 0; m < 5; m++) { S0[d][m] = 0; DS[d][m] = 0; }
        if (s->res[d]) {
            double X0 = xo[d] / dx, X1 = xn[d] / dx;
            i0[d] = (int)floor(X0 + 0.5);
            int i1 = (int)floor(X1 + 0.5);
            int sh = i1 - i0[d];
            double w0[3], w1[3], S1[5] = {0, 0, 0, 0, 0};
            shape2(X0 - i0[d], w0);
            shape2(X1 - i1, w1);
            for (int m = 0; m < 3; m++) { S0[d][1 + m] = w0[m]; S1[1 + sh + m] = w1[m]; }
            for (int m = 0; m < 5; m++) DS[d][m] = S1[m] - S0[d][m];
            lo[d] = 0; hi[d] = 5;
        } else {
            i0[d] = 0; /* only stencil slot 2, i.e. node index i0 - 2 + 2 = 0 */
            S0[d][2] = 1.0;
            lo[d] = 2; hi[d] = 3;
        }
    }
    const double third = 1.0 / 3.0;
    /* W_x, W_y, W_z of Esirkepov (2001) on the 5x5x5 stencil */
    for (int c = lo[2]; c < hi[2]; c++)
        for (int b = lo[1]; b < hi[1]; b++) {
            double acc = 0.0;
            for (int a = lo[0]; a < hi[0]; a++) {
                double Wx = DS[0][a] * (S0[1][b] * S0[2][c] + 0.5 * DS[1][b] * S0[2][c]
                                        + 0.5 * S0[1][b] * DS[2][c] + third * DS[1][b] * DS[2][c]);
                int idx[3] = {i0[0] - 2 + a, i0[1] - 2 + b, i0[2] - 2 + c};
                if (s->res[0]) {
                    acc += -q * w * (dx / dt) * Wx;
                    *ref(s, 6, idx) += acc;
                } else {
                    double Wb = S0[1][b] * S0[2][c] + 0.5 * DS[1][b] * S0[2][c]
                              + 0.5 * S0[1][b] * DS[2][c] + third * DS[1][b] * DS[2][c];
                    *ref(s, 6, idx) += q * w * v[0] * Wb;
                }
            }
        }
    for (int c = lo[2]; c < hi[2]; c++)
        for (int a = lo[0]; a < hi[0]; a++) {
            double acc = 0.0;
            for (int b = lo[1]; b < hi[1]; b++) {
                double Wb = S0[0][a] * S0[2][c] + 0.5 * DS[0][a] * S0[2][c]
                          + 0.5 * S0[0][a] * DS[2][c] + third * DS[0][a] * DS[2][c];
                int idx[3] = {i0[0] - 2 + a, i0[1] - 2 + b, i0[2] - 2 + c};
                if (s->res[1]) {
                    acc += -q * w * (dx / dt) * DS[1][b] * Wb;
                    *ref(s, 7, idx) += acc;
                } else {
                    *ref(s, 7, idx) += q * w * v[1] * Wb;
                }
            }
        }
    for (int b = lo[1]; b < hi[1]; b++)
        for (int a = lo[0]; a < hi[0]; a++) {
            double acc = 0.0;
            for (int c = lo[2]; c < hi[2]; c++) {
                double Wb = S0[0][a] * S0[1][b] + 0.5 * DS[0][a] * S0[1][b]
                          + 0.5 * S0[0][a] * DS[1][b] + third * DS[0][a] * DS[1][b];
                int idx[3] = {i0[0] - 2 + a, i0[1] - 2 + b, i0[2] - 2 + c};
                if (s->res[2]) {
                    acc += -q * w * (dx / dt) * DS[2][c] * Wb;
                    *ref(s, 8, idx) += acc;
                } else {
                    *ref(s, 8, idx) += q * w * v[2] * Wb;
                }
            }
        }
}

/* ---- Yee ------------------------------------------------------------------------ */
/* forward / backward difference of a component along axis d (0 on unresolved axes) */
static inline double dfw(const orc_sim* s, int comp, const int idx[3], int d)
{
    if (!s->res[d]) return 0.0;
    int nb[3] = {idx[0], idx[1], idx[2]};
    nb[d] += 1;
    return (val(s, comp, nb) - val(s, comp, idx)) / s->c.dx;
}
static inline double dbw(const orc_sim* s, int comp, const int idx[3], int d)
{
    if (!s->res[d]) return 0.0;
    int nb[3] = {idx[0], idx[1], idx[2]};
    nb[d] -= 1;
    return (val(s, comp, idx) - val(s, comp, nb)) / s->c.dx;
}

/* B -= h curl E at every B point (Eq. MFaraday) */
static void faraday(orc_sim* s, double h)
{
    for (int c = 0; c < 3; c++) {
        int comp = 3 + c;
        int a1 = (c + 1) % 3, a2 = (c + 2) % 3;   /* (curl E)_c = d_{a1} E_{a2} - d_{a2} E_{a1} */
        int n0 = npts(s, comp, 0), n1 = npts(s, comp, 1), n2 = npts(s, comp, 2);
        for (int k = 0; k < n2; k++)
            for (int j = 0; j < n1; j++)
                for (int i = 0; i < n0; i++) {
                    int idx[3] = {i, j, k};
                    double curl = dfw(s, a2, idx, a1) - dfw(s, a1, idx, a2);
                    s->F[comp][IX(s, i, j, k)] -= h * curl;
                }
    }
}

/* is E component c at idx on a boundary face?  returns the bitmask of boundary axes */
static int boundary_axes(const orc_sim* s, int c, const int idx[3])
{
    if (periodic(s)) return 0;
    int m = 0;
    for (int d = 0; d < 3; d++)
        if (s->res[d] && d != c && (idx[d] == 0 || idx[d] == s->c.n[d])) m |= 1 << d;
    return m;
}

/* E += dt (curl B - J) at interior E points (Eq. MAmper) */
static void ampere(orc_sim* s)
{
    double dt = s->c.dt;
    for (int c = 0; c < 3; c++) {
        int a1 = (c + 1) % 3, a2 = (c + 2) % 3;   /* (curl B)_c = d_{a1} B_{a2} - d_{a2} B_{a1} */
        int n0 = npts(s, c, 0), n1 = npts(s, c, 1), n2 = npts(s, c, 2);
        for (int k = 0; k < n2; k++)
            for (int j = 0; j < n1; j++)
                for (int i = 0; i < n0; i++) {
                    int idx[3] = {i, j, k};
                    if (boundary_axes(s, c, idx)) continue;
                    double curl = dbw(s, 3 + a2, idx, a1) - dbw(s, 3 + a1, idx, a2);
                    int64_t o = IX(s, i, j, k);
                    s->F[c][o] += dt * (curl - s->F[6 + c][o]);
                }
    }
}

/* first-order Mur on the tangential E of every face:
 *   E^{n+1}(0) = E^n(1) + (dt - dx)/(dt + dx) (E^{n+1}(1) - E^n(0)),
 * applied along the lowest boundary axis of the point, points on fewer boundary
 * axes first (their inward neighbour is then already advanced).  In the total-field
 * mode the condition acts on E - E_inc at x = 0 so that the plane wave enters. */
static void mur(orc_sim* s, double* const Eold[3])
{
    double km = (s->c.dt - s->c.dx) / (s->c.dt + s->c.dx);
    double tn = s->step * s->c.dt, tn1 = (s->step + 1) * s->c.dt;
    for (int nb = 1; nb <= 3; nb++)
        for (int c = 0; c < 3; c++) {
            int n0 = npts(s, c, 0), n1 = npts(s, c, 1), n2 = npts(s, c, 2);
            for (int k = 0; k < n2; k++)
                for (int j = 0; j < n1; j++)
                    for (int i = 0; i < n0; i++) {
                        int idx[3] = {i, j, k};
                        int m = boundary_axes(s, c, idx);
                        if (!m || __builtin_popcount(m) != nb) continue;
                        int a = __builtin_ctz(m);
                        int nbr[3] = {i, j, k};
                        nbr[a] += (idx[a] == 0) ? 1 : -1;
                        int64_t o = IX(s, i, j, k), on = IX(s, nbr[0], nbr[1], nbr[2]);
                        double inc_o_n = 0, inc_o_n1 = 0, inc_b_n = 0, inc_b_n1 = 0;
                        if (s->c.tf_mode && a == 0 && idx[0] == 0) {
                            double xo[3] = {0, 0, 0}, xb[3] = {0, 0, 0}, Ei[3], Bi[3];
                            for (int d = 0; d < 3; d++) {
                                xo[d] = (idx[d] + (staggered(c, d) ? 0.5 : 0.0)) * s->c.dx;
                                xb[d] = (nbr[d] + (staggered(c, d) ? 0.5 : 0.0)) * s->c.dx;
                            }
                            orc_incident(&s->c, xo, tn, Ei, Bi); inc_o_n = Ei[c];
                            orc_incident(&s->c, xo, tn1, Ei, Bi); inc_o_n1 = Ei[c];
                            orc_incident(&s->c, xb, tn, Ei, Bi); inc_b_n = Ei[c];
                            orc_incident(&s->c, xb, tn1, Ei, Bi); inc_b_n1 = Ei[c];
                        }
                        double Sb_n = Eold[c][on] - inc_b_n, Sb_n1 = s->F[c][on] - inc_b_n1;
                        double So_n = Eold[c][o] - inc_o_n;
                        s->F[c][o] = inc_o_n1 + Sb_n + km * (Sb_n1 - So_n);
                    }
        }
}

static void yee(orc_sim* s)
{
    double* Eold[3];
    for (int c = 0; c < 3; c++) {
        Eold[c] = malloc(sizeof(double) * s->nnode);
        memcpy(Eold[c], s->F[c], sizeof(double) * s->nnode);
    }
    faraday(s, 0.5 * s->c.dt);   /* B^n -> B^{n+1/2} */
    ampere(s);                   /* E^n -> E^{n+1} with J^{n+1/2} */
    mur(s, Eold);
    faraday(s, 0.5 * s->c.dt);   /* B^{n+1/2} -> B^{n+1} */
    for (int c = 0; c < 3; c++) free(Eold[c]);
}

/* ---- the step ------------------------------------------------------------------ */
static void add_exit(orc_sim* s, const double u[3], double w, int64_t id)
{
    if (s->nexit == s->capexit) {
        s->capexit = s->capexit ? 2 * s->capexit : 1024;
        s->eu = realloc(s->eu, sizeof(double) * 3 * s->capexit);
        s->ew = realloc(s->ew, sizeof(double) * s->capexit);
        s->eid = realloc(s->eid, sizeof(int64_t) * s->capexit);
        s->estep = realloc(s->estep, sizeof(int64_t) * s->capexit);
    }
    for (int d = 0; d < 3; d++) s->eu[3 * s->nexit + d] = u[d];
    s->ew[s->nexit] = w;
    s->eid[s->nexit] = id;
    s->estep[s->nexit] = s->step;
    s->nexit++;
}

/* ---- momentum updates (h = q dt / 2m, m = 1, c = 1) -------------------------------
 * All three take u^{n-1/2} and the fields at x^n to u^{n+1/2}.  a x b: cross product. */
static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Boris: half electric kick, rotation about B by the angle 2 atan(|h B|/gamma^-), half kick. */
static void push_boris(double u[3], const double E[3], const double B[3], double h)
{
    double um[3], tv[3], sv[3], c1[3], up[3], c2[3];
    for (int c = 0; c < 3; c++) um[c] = u[c] + h * E[c];
    const double gm = sqrt(1.0 + dot3(um, um));
    for (int c = 0; c < 3; c++) tv[c] = h / gm * B[c];
    const double t2 = dot3(tv, tv);
    for (int c = 0; c < 3; c++) sv[c] = 2.0 * tv[c] / (1.0 + t2);
    cross3(um, tv, c1);
    for (int c = 0; c < 3; c++) up[c] = um[c] + c1[c];
    cross3(up, sv, c2);
    for (int c = 0; c < 3; c++) u[c] = um[c] + c2[c] + h * E[c];
}

/* gamma of the rotation in the Vay and Higuera-Cary schemes: the positive root of
 * g^4 - sigma g^2 - (tau^2 + (w.tau)^2) = 0, sigma = 1 + w^2 - tau^2, for the vector w the
 * rotation acts on and tau = h B */
static double implicit_gamma(const double w[3], const double tau[3])
{
    const double t2 = dot3(tau, tau), ws = dot3(w, tau);
    const double sigma = 1.0 + dot3(w, w) - t2;
    return sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (t2 + ws * ws))));
}

/* the solution v of v - v x t = w (implicit midpoint rotation): s (w + (w.t) t + w x t),
 * s = 1/(1 + t^2) */
static void midpoint_rotation(const double w[3], const double t[3], double v[3])
{
    double c[3];
    cross3(w, t, c);
    const double wt = dot3(w, t), s = 1.0 / (1.0 + dot3(t, t));
    for (int k = 0; k < 3; k++) v[k] = s * (w[k] + wt * t[k] + c[k]);
}

/* Vay (2008): a full kick of E + v x B with the old velocity to the half step, a second
 * electric half kick, then u^{n+1/2} from the implicit midpoint rotation with the gamma of
 * the new momentum. */
static void push_vay(double u[3], const double E[3], const double B[3], double h)
{
    const double g0 = sqrt(1.0 + dot3(u, u));
    double v[3], vxb[3], w[3], tau[3], t[3];
    for (int c = 0; c < 3; c++) v[c] = u[c] / g0;
    cross3(v, B, vxb);
    for (int c = 0; c < 3; c++) w[c] = u[c] + h * (E[c] + vxb[c]) + h * E[c];
    for (int c = 0; c < 3; c++) tau[c] = h * B[c];
    const double g1 = implicit_gamma(w, tau);
    for (int c = 0; c < 3; c++) t[c] = tau[c] / g1;
    midpoint_rotation(w, t, u);
}

/* Higuera-Cary (2017): electric half kick to u^-, the implicit midpoint rotation with the
 * gamma of the mid-rotation momentum ubar (u^+ = 2 ubar - u^-), electric half kick. */
static void push_higuera_cary(double u[3], const double E[3], const double B[3], double h)
{
    double um[3], tau[3], t[3], ub[3];
    for (int c = 0; c < 3; c++) um[c] = u[c] + h * E[c];
    for (int c = 0; c < 3; c++) tau[c] = h * B[c];
    const double gb = implicit_gamma(um, tau);
    for (int c = 0; c < 3; c++) t[c] = tau[c] / gb;
    midpoint_rotation(um, t, ub);
    for (int c = 0; c < 3; c++) u[c] = 2.0 * ub[c] - um[c] + h * E[c];
}

/* incident E, B of every component on its own Yee nodes at time t */
static void incident_on_nodes(orc_sim* s, double t)
{
    for (int comp = 0; comp < 6; comp++)
        for (int k = 0; k < s->ext[2]; k++)
            for (int j = 0; j < s->ext[1]; j++)
                for (int i = 0; i < s->ext[0]; i++) {
                    int idx[3] = {i, j, k};
                    double xp[3], Ei[3], Bi[3];
                    for (int d = 0; d < 3; d++)
                        xp[d] = s->res[d] ? (idx[d] + (staggered(comp, d) ? 0.5 : 0.0)) * s->c.dx : 0.0;
                    orc_incident(&s->c, xp, t, Ei, Bi);
                    s->Finc[comp][IX(s, i, j, k)] = comp < 3 ? Ei[comp] : Bi[comp - 3];
                }
}

/* First part of a step (Sec. 2 cycle): J cleared, then for every electron the gather, the
 * incident field at its position, the momentum update, the move and its Esirkepov current;
 * electrons that leave are recorded as exits. */
void orc_step_particles(orc_sim* s)
{
    const double dt = s->c.dt, dx = s->c.dx;
    const double q = -1.0;
    double t = s->step * dt;
    int64_t keep = 0;
    /* J of this step; it stays readable after the step as J^{n+1/2} */
    for (int c = 6; c < 9; c++) memset(s->F[c], 0, sizeof(double) * s->nnode);
    const int inc_grid = s->c.incident_grid && s->c.beam != ORC_BEAM_NONE && !s->c.tf_mode;
    if (inc_grid) incident_on_nodes(s, t);
    for (int64_t p = 0; p < s->np; p++) {
        double* x = &s->px[3 * p];
        double* u = &s->pu[3 * p];
        double X[3] = {x[0] / dx, x[1] / dx, x[2] / dx};
        double E[3], B[3];
        for (int c = 0; c < 3; c++) { E[c] = gather(s, c, X); B[c] = gather(s, 3 + c, X); }
        if (inc_grid) {
            for (int c = 0; c < 3; c++) {
                E[c] += gather_from(s, s->Finc[c], c, X);
                B[c] += gather_from(s, s->Finc[3 + c], 3 + c, X);
            }
        } else if (s->c.beam != ORC_BEAM_NONE && !s->c.tf_mode) {
            double Ei[3], Bi[3];
            orc_incident(&s->c, x, t, Ei, Bi);
            for (int c = 0; c < 3; c++) { E[c] += Ei[c]; B[c] += Bi[c]; }
        }
        /* momentum update of the Lorentz force (charge q, mass 1) */
        const double h = 0.5 * q * dt;
        if (s->c.pusher == ORC_PUSHER_VAY) push_vay(u, E, B, h);
        else if (s->c.pusher == ORC_PUSHER_HC) push_higuera_cary(u, E, B, h);
        else push_boris(u, E, B, h);
        double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double v[3] = {u[0] / g, u[1] / g, u[2] / g};
        double xn[3] = {x[0], x[1], x[2]};
        for (int d = 0; d < s->c.dim; d++) xn[d] = x[d] + dt * v[d];
        deposit(s, x, xn, v, s->pw[p]);
        int out = 0;
        for (int d = 0; d < s->c.dim; d++) {
            if (periodic(s)) {
                double L = s->c.n[d] * dx;
                xn[d] = fmod(xn[d], L);
                if (xn[d] < 0) xn[d] += L;
            } else {
                double Xn = xn[d] / dx;
                if (Xn < s->c.remove_margin || Xn >= s->c.n[d] - s->c.remove_margin) out = 1;
            }
        }
        if (out) {
            add_exit(s, u, s->pw[p], s->pid[p]);
            continue;
        }
        for (int d = 0; d < 3; d++) {
            s->px[3 * keep + d] = xn[d];
            s->pu[3 * keep + d] = u[d];
        }
        s->pw[keep] = s->pw[p];
        s->pid[keep] = s->pid[p];
        keep++;
    }
    s->np = keep;
}

/* Second part of a step: the Yee update of the scattered field driven by that J, then the
 * step counter. */
void orc_step_fields(orc_sim* s)
{
    yee(s);
    s->step++;
}

void orc_step(orc_sim* s, int nsteps)
{
    for (int it = 0; it < nsteps; it++) {
        orc_step_particles(s);
        orc_step_fields(s);
    }
}

/* ---- diagnostics ---------------------------------------------------------------- */
/* Total energies of Sec. 3.1 (the curves Eqs. L2_t / L2_t_cross compare), in the units of
 * Table tab:units (energy density in n_c m c^2): EM = sum over the Yee points of
 * (E^2 + B^2)/2 times the cell volume, for the scattered field and for scattered +
 * incident field at the same points and time; kinetic = sum over electrons of
 * w (gamma - 1) times the cell volume (w is the density one macro-electron carries), for
 * the electrons in the box and for those that left it. */
void orc_energies(const orc_sim* s, double out[4])
{
    double vol = 1.0;
    for (int d = 0; d < s->c.dim; d++) vol *= s->c.dx;
    double t = s->step * s->c.dt;
    double em_s = 0.0, em_t = 0.0;
    for (int comp = 0; comp < 6; comp++) {
        int n0 = npts(s, comp, 0), n1 = npts(s, comp, 1), n2 = npts(s, comp, 2);
        for (int k = 0; k < n2; k++)
            for (int j = 0; j < n1; j++)
                for (int i = 0; i < n0; i++) {
                    int idx[3] = {i, j, k};
                    double f = s->F[comp][IX(s, i, j, k)];
                    em_s += 0.5 * f * f * vol;
                    double inc = 0.0;
                    if (s->c.beam != ORC_BEAM_NONE && !s->c.tf_mode) {
                        double xp[3], Ei[3], Bi[3];
                        for (int d = 0; d < 3; d++)
                            xp[d] = s->res[d] ? (idx[d] + (staggered(comp, d) ? 0.5 : 0.0)) * s->c.dx : 0.0;
                        orc_incident(&s->c, xp, t, Ei, Bi);
                        inc = comp < 3 ? Ei[comp] : Bi[comp - 3];
                    }
                    em_t += 0.5 * (f + inc) * (f + inc) * vol;
                }
    }
    double kin = 0.0, kex = 0.0;
    for (int64_t p = 0; p < s->np; p++) {
        const double* u = &s->pu[3 * p];
        kin += s->pw[p] * (sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) - 1.0) * vol;
    }
    for (int64_t p = 0; p < s->nexit; p++) {
        const double* u = &s->eu[3 * p];
        kex += s->ew[p] * (sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) - 1.0) * vol;
    }
    out[0] = em_s; out[1] = em_t; out[2] = kin; out[3] = kex;
}

double orc_gauss_residual(const orc_sim* s)
{
    double* rho = malloc(sizeof(double) * s->nnode);
    orc_charge_density(s, rho);
    double worst = 0.0;
    int n0 = npts(s, 3, 0), n1 = npts(s, 4, 1), n2 = npts(s, 5, 2); /* primal extents along each axis */
    for (int k = 0; k < n2; k++)
        for (int j = 0; j < n1; j++)
            for (int i = 0; i < n0; i++) {
                int idx[3] = {i, j, k};
                int interior = 1;
                if (!periodic(s))
                    for (int d = 0; d < s->c.dim; d++)
                        if (idx[d] == 0 || idx[d] == s->c.n[d]) interior = 0;
                if (!interior) continue;
                double div = 0.0;
                for (int d = 0; d < s->c.dim; d++) div += dbw(s, d, idx, d);
                int64_t o = IX(s, i, j, k);
                double r = fabs(div - (rho[o] + s->rho_ion[o]));
                if (r > worst) worst = r;
            }
    free(rho);
    return worst;
}
