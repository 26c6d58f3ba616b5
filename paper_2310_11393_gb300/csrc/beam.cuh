// Incident fields evaluated at a particle (Sec. 2: the incident field is added "at the
// position of the macroparticle"), device side.
//
// Plane wave (Sec. 3.1, propagation axis named x): E_y = B_z = a0 sin(xi - xi_c + phi0) env(xi),
// xi = t - (x - x_ref); envelope 2^{-4(xi - t_c)^2/FWHM^2} or sin^2(pi xi/(2 FWHM)) on [0, 2 FWHM].
//
// Tightly focused pulses (Sec. 4.1).  With the focus at the origin, propagation along
// +z, rho = r/a, zeta = z/a, R = sqrt(rho^2 + (zeta+i)^2) and u = R^2, Eq. (phasor) is
// Psi = (Psi0/a) Phi(u, tau) with Phi = [g(tau_+) - g(tau_-)]/R, tau_pm = tau + a(+-R + i),
// g from Eq. (poisson_dstr).  Every field is Psi0/a^3 times the real part of a
// polynomial in (xi, eta, zeta+i) times four complex numbers
//     Phi_u  = (G1+/R^2 - G0-/R^3)/2,             Phi_uu = (G2-/R^3 - 3G1+/R^4 + 3G0-/R^5)/4,
//     Phi_uD = (G2+/R^2 - G1-/R^3)/2,             Phi_DD = G2-/R,          (D = a d/dtau)
// obtained from the component rules: Eq. (components) for LP, and the Hertz vector
// Psi z^ (E = grad d_z Psi - d_tt Psi z^, B = d_t curl Psi z^) for RP.  This is the
// paper's expansion regrouped (sin^2(theta)/R^3 = rho^2/R^5 etc.), so nothing divides by r.
//
// Precision: the phase-critical differences t - z and t + z are formed in double once per
// reference cell and carried as hi + lo pairs (see PhaseRef), so the particle loop has no
// double-precision arithmetic and no cancellation beyond the final rounding; the choice of
// the square-root branch (Re(R conj(zeta+i)) >= 0, allowed because Phi is even in R)
// and aR - (z+ia) = a rho^2/(R + zeta + i) remove the remaining cancellations.  Near the
// ring u = 0, where the terms above cancel, Phi is summed as its power series in u:
//     Phi = 2 sum_j c_{2j+1} u^j,  c_k = g^(k)(tau0)/k!,  tau0 = tau + i a,
//     c_{k+1} = c_k q (s+k+1)/(k+1),  q = i a/(s - i tau0).
#pragma once

#include "sff_common.cuh"

namespace sff {

// Incident-field constants (host side, at set-up) from the descriptor's double values.
template <typename R>
inline BeamC<R> make_beam_consts(const SimDev& S)
{
    BeamC<R> b;
    b.beam = S.beam;
    b.envelope = S.envelope;
    b.a = R(S.a);
    b.inv_a = R(S.a > 0 ? 1.0 / S.a : 0.0);
    b.two_a = R(2.0 * S.a);
    b.s = R(S.s);
    b.inv_s = R(S.s > 0 ? 1.0 / S.s : 0.0);
    b.sp1 = R(S.s + 1.0);
    b.sp2 = R(S.s + 2.0);
    b.k = R(S.a > 0 ? S.psi0 / (S.a * S.a * S.a) : 0.0);
    b.phi0 = R(S.phi0);
    // ring series below |R| = delta: in FP32 from 0.5 (the closed form's 1/R^5 terms cancel more
    // the closer to the ring, amplifying its single-precision error; the series in FP32 stays
    // within 2e-7 of the field amplitude up to |R| = 0.5)
    const double delta = sizeof(R) == 4 ? 0.5 : 0.2;
    b.ring2 = R(delta * delta * delta * delta);
    b.a0 = R(S.a0);
    b.dur = R(S.duration);
    b.inv_dur = R(S.duration > 0 ? 1.0 / S.duration : 0.0);
    b.t_c = R(S.t_focus);
    b.dxr = R(S.dx);
    for (int d = 0; d < 3; ++d) {
        b.eu[d] = R(S.e_unif[d]);
        b.bu[d] = R(S.b_unif[d]);
        b.frf[d] = R(S.frf[d]);
    }
    b.gw0 = R(S.w0);
    b.ginv_zr = R(S.w0 > 0 ? 2.0 / (S.w0 * S.w0) : 0.0);
    b.ginv_w02 = R(S.w0 > 0 ? 1.0 / (S.w0 * S.w0) : 0.0);
    b.cph = R(std::remainder(S.phi0 - S.t_focus, 6.283185307179586));
    b.hq = R(-0.5 * S.dt);
    b.dtdx = R(S.dt * S.inv_dx);
    b.jfac = R(S.dx / S.dt);
    return b;
}

// log|w|, w = 1 - i tau/s (decides whether the term matters at all)
template <typename R>
__device__ __forceinline__ R log_abs_w(const BeamC<R>& b, Cx<R> tau)
{
    const R ti = tau.y * b.inv_s, tr = tau.x * b.inv_s;
    return R(0.5) * m_log1p(ti * (R(2) + ti) + tr * tr);
}

// |w|^{-(s+1)} below e^{-36}: the term is below ~1e-11 of the peak field even after the
// largest 1/R^5 and polynomial factors the closed form applies, so it is dropped
template <typename R>
__device__ __forceinline__ bool negligible(const BeamC<R>& b, R lnw)
{
    return b.sp1 * lnw > R(36);
}

__device__ __forceinline__ float m_exp_mag(float x) { return __expf(x); }   // error matters only near x = 0
__device__ __forceinline__ double m_exp_mag(double x) { return exp(x); }

// sin and cos of a phase of a few tens of radians: Cody-Waite reduction by 2 pi (2 pi split
// into its float value and the float of the remainder; k <= 2^4 keeps k c1 within the
// fused multiply-add's exact range) to |r| <= pi, then the SFU pair, whose absolute error
// on [-pi, pi] is below 1e-6: the carrier phase keeps ~5e-7 absolute accuracy.
__device__ __forceinline__ void sincos_phase(float x, float* s, float* c)
{
    const float k = rintf(x * 0.159154937f);
    float r = fmaf(-k, 6.28318548f, x);
    r = fmaf(-k, -1.74845553e-7f, r);
    __sincosf(r, s, c);
}
__device__ __forceinline__ void sincos_phase(double x, double* s, double* c) { sincos(x, s, c); }

// e^{i phi0} w^{-(s+1)}, w = 1 - i tau/s, and g^(1), g^(2) (Eq. poisson_dstr), given log|w|
template <typename R>
__device__ __forceinline__ void poisson3(const BeamC<R>& b, Cx<R> tau, R lnw, Cx<R>& g0, Cx<R>& g1, Cx<R>& g2)
{
    const Cx<R> w = {R(1) + tau.y * b.inv_s, -tau.x * b.inv_s};
    const R th = m_atan2(w.y, w.x);
    const R mag = m_exp_mag(-b.sp1 * lnw);
    R sn, cs;
    sincos_phase(b.phi0 - b.sp1 * th, &sn, &cs);
    g0 = {mag * cs, mag * sn};
    // q = i a/(s w)
    const R den = R(1) / (b.s * (w.x * w.x + w.y * w.y));
    const Cx<R> q = {b.a * w.y * den, b.a * w.x * den};
    g1 = b.sp1 * (g0 * q);
    g2 = b.sp2 * (g1 * q);
}

// Phi_u, Phi_uu, Phi_uD, Phi_DD by the power series about the ring
template <typename R>
__device__ __noinline__ void phi_series(const BeamC<R>& b, Cx<R> u, R trel, Cx<R> P[4])
{
    const Cx<R> w0 = {R(1) + b.a * b.inv_s, -trel * b.inv_s};      // 1 - i(trel + i a)/s
    R lnw = R(0.5) * m_log1p((w0.x * w0.x + w0.y * w0.y) - R(1));
    if (negligible(b, lnw)) {
        P[0] = P[1] = P[2] = P[3] = Cx<R>{R(0), R(0)};
        return;
    }
    R th = m_atan2(w0.y, w0.x);
    R mag = m_exp(-b.sp1 * lnw);
    R sn, cs;
    m_sincos(b.phi0 - b.sp1 * th, &sn, &cs);
    const Cx<R> c0 = {mag * cs, mag * sn};
    const R den = R(1) / (b.s * (w0.x * w0.x + w0.y * w0.y));
    const Cx<R> q = {b.a * w0.y * den, b.a * w0.x * den};
    Cx<R> ck = b.sp1 * (c0 * q);                          // c_1
    Cx<R> ck1 = (R(0.5) * (b.s + R(2))) * (ck * q);       // c_2
    Cx<R> ck2 = ((b.s + R(3)) / R(3)) * (ck1 * q);        // c_3
    Cx<R> pj = {R(1), R(0)}, pjm1 = {R(0), R(0)}, pjm2 = {R(0), R(0)};
    Cx<R> Su = {0, 0}, Suu = {0, 0}, SuD = {0, 0}, SDD = {0, 0};
    const R tol = sizeof(R) == 4 ? R(1e-9) : R(1e-18);
    int small = 0;
    for (int j = 0; j < 96; ++j) {
        const R rj = R(j);
        const Cx<R> a1 = (R(2) * rj) * (ck * pjm1);
        const Cx<R> a2 = (R(2) * rj * (rj - R(1))) * (ck * pjm2);
        const Cx<R> a3 = (R(2) * rj * (R(2) * rj + R(2))) * (ck1 * pjm1);
        const Cx<R> a4 = (R(2) * (R(2) * rj + R(2)) * (R(2) * rj + R(3))) * (ck2 * pj);
        Su = Su + a1;
        Suu = Suu + a2;
        SuD = SuD + a3;
        SDD = SDD + a4;
        const R mag_t = m_abs(a1.x) + m_abs(a1.y) + m_abs(a2.x) + m_abs(a2.y) + m_abs(a3.x) + m_abs(a3.y) +
                        m_abs(a4.x) + m_abs(a4.y);
        const R mag_s = m_abs(Su.x) + m_abs(Su.y) + m_abs(Suu.x) + m_abs(Suu.y) + m_abs(SuD.x) + m_abs(SuD.y) +
                        m_abs(SDD.x) + m_abs(SDD.y);
        if (j > 3 && mag_t <= tol * mag_s) {
            if (++small >= 2) break;
        } else {
            small = 0;
        }
        // advance c_{2j+3} -> c_{2j+4} -> c_{2j+5}
        const R kk = R(2 * j + 3);
        const Cx<R> c4 = ((b.s + kk + R(1)) / (kk + R(1))) * (ck2 * q);
        const Cx<R> c5 = ((b.s + kk + R(2)) / (kk + R(2))) * (c4 * q);
        ck = ck2;
        ck1 = c4;
        ck2 = c5;
        pjm2 = pjm1;
        pjm1 = pj;
        pj = pj * u;
    }
    P[0] = Su;
    P[1] = Suu;
    P[2] = SuD;
    P[3] = SDD;
}

// LP / RP field in the beam frame (paper x, y, z), E and B real parts.
//   xi = x/a, eta = y/a, zeta = z/a;  tmz = t_rel - z, tpz = t_rel + z (formed in double);
//   trel = t - t_focus.
template <typename R>
__device__ __forceinline__ void focused_field(const BeamC<R>& b, R xi, R eta, R zeta, R tmz, R tpz, R trel, R E[3],
                                              R B[3])
{
    const R rho2 = xi * xi + eta * eta;
    const Cx<R> u = {rho2 + zeta * zeta - R(1), R(2) * zeta};
    Cx<R> P[4];
    if (u.x * u.x + u.y * u.y < b.ring2) {
        phi_series(b, u, trel, P);
    } else {
        Cx<R> Rr = csqrt_(u);
        if (Rr.x * zeta + Rr.y < R(0)) Rr = -Rr;      // Re(R conj(zeta + i)) >= 0
        const Cx<R> den = {Rr.x + zeta, Rr.y + R(1)};
        const Cx<R> qq = (b.a * rho2) * cinv(den);     // a R - (z + i a)
        const Cx<R> taum = {tmz - qq.x, -qq.y};
        const Cx<R> taup = {tpz + qq.x, b.two_a + qq.y};
        const R lnm = log_abs_w(b, taum), lnp = log_abs_w(b, taup);
        const bool use_m = !negligible(b, lnm), use_p = !negligible(b, lnp);
        if (!use_m && !use_p) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                E[d] = R(0);
                B[d] = R(0);
            }
            return;
        }
        Cx<R> g0m = {0, 0}, g1m = {0, 0}, g2m = {0, 0}, g0p = {0, 0}, g1p = {0, 0}, g2p = {0, 0};
        if (use_m) poisson3(b, taum, lnm, g0m, g1m, g2m);
        if (use_p) poisson3(b, taup, lnp, g0p, g1p, g2p);
        const Cx<R> G0m = g0p - g0m, G1p = g1p + g1m, G1m = g1p - g1m, G2p = g2p + g2m, G2m = g2p - g2m;
        const Cx<R> iR = cinv(Rr);
        const Cx<R> iR2 = iR * iR;
        const Cx<R> iR3 = iR2 * iR;
        P[0] = R(0.5) * (G1p * iR2 - G0m * iR3);
        P[1] = R(0.25) * ((G2m * iR3) - R(3) * ((G1p * iR2) * iR2) + R(3) * ((G0m * iR3) * iR2));
        P[2] = R(0.5) * (G2p * iR2 - G1m * iR3);
        P[3] = G2m * iR;
    }
    const Cx<R> Pu = P[0], Puu = P[1], PuD = P[2], PDD = P[3];
    const R k = b.k;
    // real parts of the combinations
    const R zPuu = zeta * Puu.x - Puu.y;              // Re((zeta+i) Phi_uu)
    const R zPuD = zeta * PuD.x - PuD.y;              // Re((zeta+i) Phi_uD)
    const R base = R(2) * Pu.x - PDD.x;               // Re(2 Phi_u - Phi_DD)
    if (b.beam == BEAM_LP) {
        E[0] = k * (base + R(2) * zPuD + R(4) * xi * xi * Puu.x);
        E[1] = k * (R(4) * xi * eta * Puu.x);
        E[2] = k * (R(4) * xi * zPuu - R(2) * xi * PuD.x);
        B[0] = E[1];
        B[1] = k * (base + R(2) * zPuD + R(4) * eta * eta * Puu.x);
        B[2] = k * (R(4) * eta * zPuu - R(2) * eta * PuD.x);
    } else {
        // Re((zeta+i)^2 Phi_uu) = (zeta^2 - 1) Re Phi_uu - 2 zeta Im Phi_uu
        const R z2Puu = (zeta * zeta - R(1)) * Puu.x - R(2) * zeta * Puu.y;
        E[0] = k * (R(4) * xi * zPuu);
        E[1] = k * (R(4) * eta * zPuu);
        E[2] = k * (base + R(4) * z2Puu);
        B[0] = k * (R(2) * eta * PuD.x);
        B[1] = -k * (R(2) * xi * PuD.x);
        B[2] = R(0);
    }
}

// Phase-critical x-differences, formed once per reference cell x0 in double precision and
// carried as unevaluated sums hi + lo of two R numbers.  For a particle at cell x0 + lx with
// offset o, x - x(x0) = lx dx_h + (o dx + lx dx_l), where dx_h keeps 12 significant bits so
// that lx dx_h is exact; then t - z = ((A_h - lx dx_h) + A_l) - (o dx + lx dx_l) has no
// cancellation beyond the final rounding, without any double-precision work per particle.
template <typename R>
struct PhaseRef {
    int x0;
    R ah, al;      // LP/RP: t_rel - Z(x0);  plane: xi(x0) - xi_c + phi0 (carrier phase)
    R bh, bl;      // LP/RP: t_rel + Z(x0);  plane: xi(x0) = t - (x(x0) - x_ref)
    R zh, zl;      // Z(x0) = x(x0) - focus_x
    R dxh, dxl, dxr;
    R trel;
};

template <typename R>
__device__ __forceinline__ void split_hl(double v, R& h, R& l)
{
    h = R(v);
    l = R(v - (double)h);
}

template <typename R>
__device__ __forceinline__ PhaseRef<R> phase_ref(const SimDev& S, double t, int x0)
{
    PhaseRef<R> p;
    p.x0 = x0;
    const double Z0 = (double)x0 * S.dx - S.focus[0];
    double A, Bv;
    if (S.beam == BEAM_PLANE) {
        const double xi0 = t - Z0;
        A = xi0 - (S.envelope == 1 ? S.t_focus : S.duration) + S.phi0;
        Bv = xi0;
        p.trel = R(0);
    } else {
        const double trel = t - S.t_focus;
        A = trel - Z0;
        Bv = trel + Z0;
        p.trel = R(trel);
    }
    split_hl(A, p.ah, p.al);
    split_hl(Bv, p.bh, p.bl);
    split_hl(Z0, p.zh, p.zl);
    const double dh = (double)__int_as_float(__float_as_int((float)S.dx) & (int)0xFFFFF000);
    p.dxh = R(dh);
    p.dxl = R(S.dx - dh);
    p.dxr = R(S.dx);
    return p;
}

// Incident E, B (grid axes) at a particle in cell c with offsets o, at the time of `pr`.
template <int D, typename R>
__device__ __forceinline__ void incident_at(const SimDev& S, const BeamC<R>& b, const PhaseRef<R>& pr, const int c[3],
                                            const R o[3], R E[3], R B[3])
{
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        E[d] = R(0);
        B[d] = R(0);
    }
    if (b.beam == BEAM_PLANE || b.beam == BEAM_LP || b.beam == BEAM_RP) {
        const R lx = R(c[0] - pr.x0);
        const R sh = lx * pr.dxh;                       // exact
        const R sl = o[0] * pr.dxr + lx * pr.dxl;
        if (b.beam == BEAM_PLANE) {
            const R xi = ((pr.bh - sh) + pr.bl) - sl;
            const R arg = ((pr.ah - sh) + pr.al) - sl;
            R env;
            if (b.envelope == 1) {
                const R v = (xi - b.t_c) * b.inv_dur;
                env = m_exp2(R(-4) * v * v);
            } else {
                if (xi <= R(0) || xi >= R(2) * b.dur) return;
                const R sn = m_sinpi(xi * R(0.5) * b.inv_dur);
                env = sn * sn;
            }
            const R f = b.a0 * m_sin(arg) * env;
            E[1] = f;
            B[2] = f;
            return;
        }
        // beam frame: paper z = grid x, paper x = grid y, paper y = grid z
        const R tmz = ((pr.ah - sh) + pr.al) - sl;
        const R tpz = ((pr.bh + sh) + pr.bl) + sl;
        const R inv_a = b.inv_a;
        const R zeta = ((pr.zh + sh) + (pr.zl + sl)) * inv_a;
        R xi = R(0), eta = R(0);
        if constexpr (D >= 2) xi = ((R)(c[1] - S.icf[1]) + (o[1] - b.frf[1])) * (b.dxr * inv_a);
        if constexpr (D >= 3) eta = ((R)(c[2] - S.icf[2]) + (o[2] - b.frf[2])) * (b.dxr * inv_a);
        R Ep[3], Bp[3];
        focused_field<R>(b, xi, eta, zeta, tmz, tpz, pr.trel, Ep, Bp);
        E[0] = Ep[2];
        E[1] = Ep[0];
        E[2] = Ep[1];
        B[0] = Bp[2];
        B[1] = Bp[0];
        B[2] = Bp[1];
    } else if (b.beam == BEAM_GAUSS2D) {
        // 2D paraxial Gaussian beam (Sec. 3.2), beam frame Z = grid x - focus, X = grid y - focus:
        // the envelope argument t - t0 - Z and the carrier Z - t = -(t - t0 - Z) - t0 come
        // from the tile's float-float phase reference
        const R lx = R(c[0] - pr.x0);
        const R sh = lx * pr.dxh;
        const R sl = o[0] * pr.dxr + lx * pr.dxl;
        const R xi = ((pr.ah - sh) + pr.al) - sl;                 // t - t0 - Z
        const R ev = R(4) * xi * xi * b.inv_dur * b.inv_dur;
        if (ev > R(40)) return;                                   // envelope below 2^-40
        const R Z = (pr.zh + sh) + (pr.zl + sl);
        R X = R(0);
        if constexpr (D >= 2) X = ((R)(c[1] - S.icf[1]) + (o[1] - b.frf[1])) * b.dxr;
        const R zz = Z * b.ginv_zr;
        const R q1 = R(1) + zz * zz;                              // (w/w0)^2
        const R iw2 = b.ginv_w02 / q1;                            // 1/w^2
        const R invR = zz * b.ginv_zr / q1;                       // Z/(Z^2 + zR^2)
        const R eta = R(0.5) * m_atan(zz);
        const R amp = b.a0 * m_rsqrt(m_sqrt(q1)) * m_exp(-X * X * iw2) * m_exp2(-ev);
        const R ph = (b.cph - xi) + (R(0.5) * X * X * invR - eta);
        R sn, cs;
        sincos_phase(ph, &sn, &cs);
        E[1] = amp * cs;                                          // paper E_x
        B[2] = E[1];                                              // paper B_y
        E[0] = amp * (R(2) * X * iw2 * sn - X * invR * cs);       // paper E_z
    } else if (b.beam == BEAM_UNIFORM) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            E[d] = b.eu[d];
            B[d] = b.bu[d];
        }
    }
}

}  // namespace sff
