// Device cell models of the ten Tusscher family (Sec. 3.1):
//   - ten Tusscher & Panfilov 2006 human ventricular myocyte (TP06), with the
//     endo / M / epi variants of its I_to and I_Ks;
//   - Stewart et al. 2009 human Purkinje cell, which adds I_f and I_sus to the
//     same scaffold and changes I_Na, I_K1, I_to, I_Kr and I_Ks.
// One step: currents and rates at (V^n, s^n); gates and Rbar by Rush-Larsen;
// [Na]i, [K]i by forward Euler (or AB2, see Rates), accumulated in FP64 (plain path) or as a
// two-float compensated sum (mixed path); the three calcium
// compartments by forward Euler on the buffered total, applied as an
// increment of the free concentration (Sec. 3.2).
//
// Storage of a region (see DevRegion): compute-type slots
//   0 Ca_i, 1 Ca_SS, 2 m, 3 h, 4 j, 5 xr1, 6 xr2, 7 xs, 8 r, 9 s, 10 d, 11 f,
//   12 f2, 13 fCaSS, 14 Rbar, [15 y (Stewart)]
// and accumulator slots (FP64 / two-float) 0 Na_i, 1 K_i, 2 Ca_SR.
#pragma once
#include "cellmath.cuh"
#include "devtypes.h"

namespace ep {

constexpr int kTTnr = 15, kSTWnr = 16, kTTna = 3;

// Returns I_ion(V^n, s^n) in uA/uF and writes s^{n+1} (all but V).
template <class R, bool PURKINJE, bool AB2 = false>
__device__ __forceinline__ R tt_step(const CellIO<R> &io, const DevParams &P, R V, R dt, R i_stim,
                                     const Rates<R, AB2> &rt = Rates<R, AB2>{}) {
    const R *xi = io.xi;
    const double *ai = io.ai;
    const long long si = io.si;
    R *xo = io.xo;
    double *ao = io.ao;
    const long long so = io.so;
    const R Cai = xi[0], Cass = xi[si], m = xi[2 * si], h = xi[3 * si], jj = xi[4 * si];
    const R xr1 = xi[5 * si], xr2 = xi[6 * si], xs = xi[7 * si], r = xi[8 * si], s = xi[9 * si];
    const R d = xi[10 * si], f = xi[11 * si], f2 = xi[12 * si], fcass = xi[13 * si], rr = xi[14 * si];
    const Accum<R> Nai_a = Accum<R>::load(ai), Ki_a = Accum<R>::load(ai + si), Casr_a = Accum<R>::load(ai + 2 * si);
    const R Nai = Nai_a.value(), Ki = Ki_a.value(), Casr = Casr_a.value();

    // constants (model papers' parameter tables)
    const R RTF = R(8314.472 * 310.0 / 96485.3415), FRT = R(96485.3415 / (8314.472 * 310.0));
    const R Fc = R(96485.3415);
    const R Cm = R(0.185), Vc = R(0.016404), Vsr = R(0.001094), Vss = R(0.00005468);
    const R Nao = R(140.0), Cao = R(2.0);
    const R Ko = pick<R>(P.K_o, P.Ko_f);
    const R sqKo = pick<R>(P.sqrt_Ko, P.sqrt_Ko_f);

    const R ENa = RTF * flog(Nao / Nai);
    const R EK = RTF * flog(Ko / Ki);
    const R EKs = RTF * flog((Ko + R(0.03) * Nao) / (Ki + R(0.03) * Nai));
    const R ECa = R(0.5) * RTF * flog(Cao / Cai);

    // ---- membrane currents ----
    const R GNa = PURKINJE ? R(130.5744) : R(14.838);
    const R INa = GNa * m * m * m * h * jj * (V - ENa);
    const R xl = R(2) * (V - R(15)) * FRT;
    const R ICaL = R(3.980e-5) * d * f * f2 * fcass * R(2) * Fc * x_over_expm1(xl) *
                   (R(0.25) * Cass * fexp(xl) - Cao);
    R Gto, GKs, GKr;
    if (PURKINJE) {
        Gto = R(0.08184);
        GKs = R(0.2352);
        GKr = R(0.0918);
    } else {
        Gto = (P.variant == 2) ? R(0.073) : R(0.294);
        GKs = (P.variant == 1) ? R(0.098) : R(0.392);
        GKr = R(0.153);
    }
    GKs *= pick<R>(P.gks_scale, P.gks_f);
    GKr *= pick<R>(P.gkr_scale, P.gkr_f);
    const R Ito = Gto * r * s * (V - EK);
    const R IKr = GKr * sqKo * xr1 * xr2 * (V - EK);
    const R IKs = GKs * xs * xs * (V - EKs);
    R IK1;
    if (PURKINJE) {
        IK1 = R(0.065) * logistic(R(0.1) * (V + R(75.44))) * (V - R(8) - EK);
    } else {
        const R aK1 = R(0.1) * logistic(R(0.06) * (V - EK - R(200)));
        const R bK1 = (R(3) * fexp(R(0.0002) * (V - EK + R(100))) + fexp(R(0.1) * (V - EK - R(10)))) *
                      logistic(R(-0.5) * (V - EK));
        IK1 = R(5.405) * sqKo * (aK1 / (aK1 + bK1)) * (V - EK);
    }
    const R eg = fexp(R(0.35) * V * FRT), egm1 = fexp(R(-0.65) * V * FRT);
    const R INaCa = R(1000) * (eg * Nai * Nai * Nai * Cao - egm1 * Nao * Nao * Nao * Cai * R(2.5)) /
                    ((R(87.5 * 87.5 * 87.5) + Nao * Nao * Nao) * (R(1.38) + Cao) * (R(1) + R(0.1) * egm1));
    const R INaK = R(2.724) * Ko * Nai /
                   ((Ko + R(1)) * (Nai + R(40)) * (R(1) + R(0.1245) * fexp(R(-0.1) * V * FRT) + R(0.0353) * fexp(-V * FRT)));
    const R IpCa = R(0.1238) * Cai / (R(0.0005) + Cai);
    const R IpK = R(0.0146) * (V - EK) * logistic((R(25) - V) * R(1.0 / 5.98));
    const R IbNa = R(0.00029) * (V - ENa);
    const R IbCa = R(0.000592) * (V - ECa);
    R Iion = INa + IK1 + Ito + IKr + IKs + ICaL + INaCa + INaK + IpCa + IpK + IbNa + IbCa;
    R IfNa = R(0), IfK = R(0), Isus = R(0), y = R(0);
    if (PURKINJE) {
        y = xi[15 * si];
        IfNa = y * R(0.0145654) * (V - ENa);
        IfK = y * R(0.0234346) * (V - EK);
        Isus = R(0.0227) * logistic((R(5) - V) * R(1.0 / 17.0)) * (V - EK);
        Iion += IfNa + IfK + Isus;
    }

    // ---- calcium handling ----
    const R kcasr = R(2.5) - R(1.5) / (R(1) + (R(1.5) / Casr) * (R(1.5) / Casr));
    const R k1 = R(0.15) / kcasr, k2 = R(0.045) * kcasr;
    const R O = k1 * Cass * Cass * rr / (R(0.06) + k1 * Cass * Cass);
    const R Irel = R(0.102) * O * (Casr - Cass);
    const R Iup = R(0.006375) / (R(1) + (R(0.00025) / Cai) * (R(0.00025) / Cai));
    const R Ileak = R(0.00036) * (Casr - Cai);
    const R Ixfer = R(0.0038) * (Cass - Cai);
    const R dCai_tot = -(IbCa + IpCa - R(2) * INaCa) * (Cm / (R(2) * Vc * Fc)) + (Vsr / Vc) * (Ileak - Iup) + Ixfer;
    const R dCasr_tot = Iup - Irel - Ileak;
    const R dCass_tot = -ICaL * (Cm / (R(2) * Vss * Fc)) + (Vsr / Vss) * Irel - (Vc / Vss) * Ixfer;
    const R dNai = -(INa + IbNa + IfNa + R(3) * INaK + R(3) * INaCa) * (Cm / (Vc * Fc));
    const R dKi = -(IK1 + Ito + Isus + IfK + IKr + IKs - R(2) * INaK + IpK + i_stim) * (Cm / (Vc * Fc));

    // ---- gates (Rush-Larsen at V^n) ----
    R yinf, tau, al, be;
    {
        const R e = R(1) + fexp((R(-56.86) - V) * R(1.0 / 9.03));
        yinf = R(1) / (e * e);
        al = logistic((R(-60) - V) * R(0.2));
        be = R(0.1) * logistic((V + R(35)) * R(0.2)) + R(0.1) * logistic((V - R(50)) * R(0.005));
        xo[2 * so] = rush_larsen(m, yinf, al * be, dt);
    }
    {
        const R e = R(1) + fexp((V + R(71.55)) * R(1.0 / 7.43));
        const R hinf = R(1) / (e * e);
        R ah, bh, aj, bj;
        if (V >= R(-40)) {
            ah = R(0);
            bh = R(0.77) / (R(0.13) * (R(1) + fexp(-(V + R(10.66)) * R(1.0 / 11.1))));
            aj = R(0);
            bj = R(0.6) * fexp(R(0.057) * V) * logistic(R(-0.1) * (V + R(32)));
        } else {
            ah = R(0.057) * fexp(-(V + R(80)) * R(1.0 / 6.8));
            bh = R(2.7) * fexp(R(0.079) * V) + R(3.1e5) * fexp(R(0.3485) * V);
            aj = (R(-2.5428e4) * fexp(R(0.2444) * V) - R(6.948e-6) * fexp(R(-0.04391) * V)) * (V + R(37.78)) *
                 logistic(R(0.311) * (V + R(79.23)));
            bj = R(0.02424) * fexp(R(-0.01052) * V) * logistic(R(-0.1378) * (V + R(40.14)));
        }
        xo[3 * so] = rush_larsen_rate(h, hinf, ah + bh, dt);
        xo[4 * so] = rush_larsen_rate(jj, hinf, aj + bj, dt);
    }
    yinf = logistic((R(-26) - V) * R(1.0 / 7.0));
    al = R(450) * logistic((R(-45) - V) * R(0.1));
    be = R(6) * logistic((V + R(30)) * R(1.0 / 11.5));
    xo[5 * so] = rush_larsen(xr1, yinf, al * be, dt);
    yinf = logistic((V + R(88)) * R(1.0 / 24.0));
    al = R(3) * logistic((R(-60) - V) * R(0.05));
    be = R(1.12) * logistic((V - R(60)) * R(0.05));
    xo[6 * so] = rush_larsen(xr2, yinf, al * be, dt);
    yinf = logistic((R(-5) - V) * R(1.0 / 14.0));
    al = R(1400) / fsqrt(R(1) + fexp((R(5) - V) * R(1.0 / 6.0)));
    be = logistic((V - R(35)) * R(1.0 / 15.0));
    xo[7 * so] = rush_larsen(xs, yinf, al * be + R(80), dt);
    if (PURKINJE) {
        yinf = logistic((R(20) - V) * R(1.0 / 13.0));
        tau = R(10.45) * fexp(-(V + R(40)) * (V + R(40)) * R(1.0 / 1800.0)) + R(7.3);
        xo[8 * so] = rush_larsen(r, yinf, tau, dt);
        yinf = logistic((V + R(27)) * R(1.0 / 13.0));
        tau = R(85) * fexp(-(V + R(25)) * (V + R(25)) * R(1.0 / 320.0)) + R(5) * logistic((V - R(40)) * R(0.2)) + R(42);
        xo[9 * so] = rush_larsen(s, yinf, tau, dt);
    } else {
        yinf = logistic((R(20) - V) * R(1.0 / 6.0));
        tau = R(9.5) * fexp(-(V + R(40)) * (V + R(40)) * R(1.0 / 1800.0)) + R(0.8);
        xo[8 * so] = rush_larsen(r, yinf, tau, dt);
        if (P.variant == 2) {
            yinf = logistic((V + R(28)) * R(0.2));
            tau = R(1000) * fexp(-(V + R(67)) * (V + R(67)) * R(0.001)) + R(8);
        } else {
            yinf = logistic((V + R(20)) * R(0.2));
            tau = R(85) * fexp(-(V + R(45)) * (V + R(45)) * R(1.0 / 320.0)) + R(5) * logistic((V - R(20)) * R(0.2)) + R(3);
        }
        xo[9 * so] = rush_larsen(s, yinf, tau, dt);
    }
    yinf = logistic((R(-8) - V) * R(1.0 / 7.5));
    al = R(1.4) * logistic((R(-35) - V) * R(1.0 / 13.0)) + R(0.25);
    be = R(1.4) * logistic((V + R(5)) * R(0.2));
    xo[10 * so] = rush_larsen(d, yinf, al * be + logistic((R(50) - V) * R(0.05)), dt);
    yinf = logistic((V + R(20)) * R(1.0 / 7.0));
    tau = R(1102.5) * fexp(-(V + R(27)) * (V + R(27)) * R(1.0 / 225.0)) + R(200) * logistic((R(13) - V) * R(0.1)) +
          R(180) * logistic((V + R(30)) * R(0.1)) + R(20);
    xo[11 * so] = rush_larsen(f, yinf, tau, dt);
    yinf = R(0.67) * logistic((V + R(35)) * R(1.0 / 7.0)) + R(0.33);
    tau = R(562) * fexp(-(V + R(27)) * (V + R(27)) * R(1.0 / 240.0)) + R(31) * logistic((R(25) - V) * R(0.1)) +
          R(80) * logistic((V + R(30)) * R(0.1));
    xo[12 * so] = rush_larsen(f2, yinf, tau, dt);
    {
        const R cr = Cass * R(20);  // Ca_SS / 0.05
        const R den = R(1) / (R(1) + cr * cr);
        xo[13 * so] = rush_larsen(fcass, R(0.6) * den + R(0.4), R(80) * den + R(2), dt);
    }
    {
        const R rate = k2 * Cass + R(0.005);
        xo[14 * so] = rush_larsen_rate(rr, R(0.005) / rate, rate, dt);
    }
    if (PURKINJE) {
        yinf = logistic((V + R(80.6)) * R(1.0 / 6.8));
        tau = R(4000) / (fexp(R(-2.9) - R(0.04) * V) + fexp(R(3.6) + R(0.11) * V));
        xo[15 * so] = rush_larsen(y, yinf, tau, dt);
    }

    // ---- concentrations ----
    xo[0] = Cai + buffered_increment(Cai, dt * rt(3, dCai_tot), R(0.2), R(0.001));
    xo[so] = Cass + buffered_increment(Cass, dt * rt(5, dCass_tot), R(0.4), R(0.00025));
    Nai_a.store_add(ao, dt * rt(1, dNai));
    Ki_a.store_add(ao + so, dt * rt(2, dKi));
    Casr_a.store_add(ao + 2 * so, buffered_increment(Casr, dt * rt(4, dCasr_tot), R(10), R(0.3)));
    return Iion;
}

// Published resting states (model papers' initial-value tables).
template <class R, bool PURKINJE>
__device__ __forceinline__ void tt_init(const DevRegion &rg, long long i, R *V) {
    R *x = static_cast<R *>(rg.r) + i;
    double *a = rg.a + i;
    const long long st = rg.stride;
    if (!PURKINJE) {
        *V = R(-85.23);
        const R v[kTTnr] = {R(0.000126), R(0.00036), R(0.00172), R(0.7444), R(0.7045), R(0.00621), R(0.4712),
                            R(0.0095), R(2.42e-8), R(0.999998), R(3.373e-5), R(0.7888), R(0.9755), R(0.9953),
                            R(0.9073)};
        for (int k = 0; k < kTTnr; ++k) x[k * st] = v[k];
        Accum<R>::init(a, 8.604);
        Accum<R>::init(a + st, 136.89);
        Accum<R>::init(a + 2 * st, 3.64);
    } else {
        *V = R(-69.1865);
        const R v[kSTWnr] = {R(0.000101878), R(0.000446818), R(0.0417391), R(0.190678), R(0.238219),
                             R(0.00550281), R(0.313298), R(0.00953708), R(0.00103629), R(0.96589),
                             R(0.000287906), R(0.989144), R(0.995762), R(0.999934), R(0.991227), R(0.0457562)};
        for (int k = 0; k < kSTWnr; ++k) x[k * st] = v[k];
        Accum<R>::init(a, 8.80545);
        Accum<R>::init(a + st, 136.781894);
        Accum<R>::init(a + 2 * st, 3.10836);
    }
}

}  // namespace ep
