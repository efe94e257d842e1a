// Device cell model: Courtemanche, Ramirez & Nattel 1998 human atrial
// myocyte (Sec. 3.1, atria and 1D bundles). One step: currents at
// (V^n, s^n), the 15 gates by Rush-Larsen, the concentrations by forward
// Euler with the model's differential buffering factors; [Na]i, [K]i and the
// SR compartments (Ca_up, Ca_rel) accumulated in FP64 (plain path) or as
// two-float compensated sums (mixed path) (Sec. 3.2).
//
// Storage: compute-type slots 0 Ca_i, 1 m, 2 h, 3 j, 4 oa, 5 oi, 6 ua, 7 ui,
// 8 xr, 9 xs, 10 d, 11 f, 12 fCa, 13 u, 14 v, 15 w; accumulator slots 0 Na_i,
// 1 K_i, 2 Ca_up, 3 Ca_rel.
#pragma once
#include "cellmath.cuh"
#include "devtypes.h"

namespace ep {

constexpr int kCRNnr = 16, kCRNna = 4;

// x / (1 - exp(-x/k)) and x / (exp(x/k) - 1), both equal to k at x = 0.
template <class R>
__device__ __forceinline__ R lin_over_1mexp(R x, R k) {
    const R y = x / k;
    return y == R(0) ? k : k * y / (-fexpm1(-y));
}
template <class R>
__device__ __forceinline__ R lin_over_expm1(R x, R k) {
    const R y = x / k;
    return y == R(0) ? k : k * y / fexpm1(y);
}

template <class R, bool AB2 = false>
__device__ __forceinline__ R crn_step(const CellIO<R> &io, const DevParams &P, R V, R dt,
                                      const Rates<R, AB2> &rt = Rates<R, AB2>{}) {
    const R *xi = io.xi;
    const double *ai = io.ai;
    const long long si = io.si;
    R *xo = io.xo;
    double *ao = io.ao;
    const long long so = io.so;
    const R Cai = xi[0], m = xi[si], h = xi[2 * si], jj = xi[3 * si], oa = xi[4 * si], oi = xi[5 * si];
    const R ua = xi[6 * si], ui = xi[7 * si], xr = xi[8 * si], xs = xi[9 * si], d = xi[10 * si];
    const R f = xi[11 * si], fCa = xi[12 * si], u = xi[13 * si], vv = xi[14 * si], w = xi[15 * si];
    const Accum<R> Nai_a = Accum<R>::load(ai), Ki_a = Accum<R>::load(ai + si);
    const Accum<R> Caup_a = Accum<R>::load(ai + 2 * si), Carel_a = Accum<R>::load(ai + 3 * si);
    const R Nai = Nai_a.value(), Ki = Ki_a.value(), Caup = Caup_a.value(), Carel = Carel_a.value();

    const R Fc = R(96.4867);
    const R RTF = R(8.3143 * 310.0 / 96.4867), FRT = R(96.4867 / (8.3143 * 310.0));
    const R Cm = R(100), Vi = R(13668), Vup = R(1109.52), Vrel = R(96.48);
    const R Nao = R(140), Cao = R(1.8), Ko = pick<R>(P.K_o, P.Ko_f);

    const R ENa = RTF * flog(Nao / Nai);
    const R EK = RTF * flog(Ko / Ki);
    const R ECa = R(0.5) * RTF * flog(Cao / Cai);

    const R INa = R(7.8) * m * m * m * h * jj * (V - ENa);
    const R IK1 = R(0.09) * (V - EK) * logistic(R(0.07) * (V + R(80)));
    const R Ito = R(0.1652) * oa * oa * oa * oi * (V - EK);
    const R gKur = R(0.005) + R(0.05) * logistic(-(V - R(15)) * R(1.0 / 13.0));
    const R IKur = gKur * ua * ua * ua * ui * (V - EK);
    const R IKr = R(0.0294) * pick<R>(P.gkr_scale, P.gkr_f) * xr * (V - EK) * logistic((V + R(15)) * R(1.0 / 22.4));
    const R IKs = R(0.129) * pick<R>(P.gks_scale, P.gks_f) * xs * xs * (V - EK);
    const R ICaL = R(0.1238) * d * f * fCa * (V - R(65));
    const R sigma = (fexp(Nao * R(1.0 / 67.3)) - R(1)) * R(1.0 / 7.0);
    const R fNaK = R(1) / (R(1) + R(0.1245) * fexp(R(-0.1) * V * FRT) + R(0.0365) * sigma * fexp(-V * FRT));
    const R rN = R(10) / Nai;
    const R INaK = R(0.59933874) * fNaK / (R(1) + rN * fsqrt(rN)) * Ko / (Ko + R(1.5));
    const R egm1 = fexp(R(-0.65) * V * FRT);
    const R INaCa = R(1600) * (fexp(R(0.35) * V * FRT) * Nai * Nai * Nai * Cao - egm1 * Nao * Nao * Nao * Cai) /
                    ((R(87.5 * 87.5 * 87.5) + Nao * Nao * Nao) * (R(1.38) + Cao) * (R(1) + R(0.1) * egm1));
    const R IbCa = R(0.00113) * (V - ECa);
    const R IbNa = R(0.000674) * (V - ENa);
    const R IpCa = R(0.275) * Cai / (R(0.0005) + Cai);
    const R Iion = INa + IK1 + Ito + IKur + IKr + IKs + ICaL + INaK + INaCa + IbCa + IbNa + IpCa;

    const R Irel = R(30) * u * u * vv * w * (Carel - Cai);
    const R Itr = (Caup - Carel) * R(1.0 / 180.0);
    const R Iup = R(0.005) / (R(1) + R(0.00092) / Cai);
    const R Iupleak = R(0.005) * Caup * R(1.0 / 15.0);

    const R dNai = (R(-3) * INaK - R(3) * INaCa - IbNa - INa) * (Cm / (Vi * Fc));
    const R dKi = (R(2) * INaK - IK1 - Ito - IKur - IKr - IKs) * (Cm / (Vi * Fc));
    const R B1 = (R(2) * INaCa - IpCa - ICaL - IbCa) * (Cm / (R(2) * Vi * Fc)) + (Vup * (Iupleak - Iup) + Irel * Vrel) / Vi;
    const R B2 = R(1) + R(0.07 * 0.0005) / ((Cai + R(0.0005)) * (Cai + R(0.0005))) +
                 R(0.05 * 0.00238) / ((Cai + R(0.00238)) * (Cai + R(0.00238)));
    const R dCaup = Iup - Iupleak - Itr * (Vrel / Vup);
    const R dCarel = (Itr - Irel) / (R(1) + R(10 * 0.8) / ((Carel + R(0.8)) * (Carel + R(0.8))));

    // ---- gates ----
    R al, be;
    al = R(0.32) * lin_over_1mexp(V + R(47.13), R(10));
    be = R(0.08) * fexp(-V * R(1.0 / 11.0));
    R ab = al + be;
    xo[so] = rush_larsen_rate(m, al / ab, ab, dt);
    if (V >= R(-40)) {
        al = R(0);
        be = R(1) / (R(0.13) * (R(1) + fexp(-(V + R(10.66)) * R(1.0 / 11.1))));
    } else {
        al = R(0.135) * fexp(-(V + R(80)) * R(1.0 / 6.8));
        be = R(3.56) * fexp(R(0.079) * V) + R(3.1e5) * fexp(R(0.35) * V);
    }
    ab = al + be;
    xo[2 * so] = rush_larsen_rate(h, al / ab, ab, dt);
    if (V >= R(-40)) {
        al = R(0);
        be = R(0.3) * fexp(R(-2.535e-7) * V) * logistic(R(-0.1) * (V + R(32)));
    } else {
        al = (R(-127140) * fexp(R(0.2444) * V) - R(3.474e-5) * fexp(R(-0.04391) * V)) * (V + R(37.78)) *
             logistic(R(0.311) * (V + R(79.23)));
        be = R(0.1212) * fexp(R(-0.01052) * V) * logistic(R(-0.1378) * (V + R(40.14)));
    }
    ab = al + be;
    xo[3 * so] = rush_larsen_rate(jj, al / ab, ab, dt);
    // oa and ua share their rate functions
    al = R(0.65) / (fexp(-(V + R(10)) * R(1.0 / 8.5)) + fexp(-(V - R(30)) * R(1.0 / 59.0)));
    be = R(0.65) / (R(2.5) + fexp((V + R(82)) * R(1.0 / 17.0)));
    const R rate_a = (al + be) * R(3);
    xo[4 * so] = rush_larsen_rate(oa, logistic(-(V + R(20.47)) * R(1.0 / 17.54)), rate_a, dt);
    xo[6 * so] = rush_larsen_rate(ua, logistic(-(V + R(30.3)) * R(1.0 / 9.6)), rate_a, dt);
    al = R(1) / (R(18.53) + fexp((V + R(113.7)) * R(1.0 / 10.95)));
    be = R(1) / (R(35.56) + fexp(-(V + R(1.26)) * R(1.0 / 7.44)));
    xo[5 * so] = rush_larsen_rate(oi, logistic((V + R(43.1)) * R(1.0 / 5.3)), (al + be) * R(3), dt);
    al = R(1) / (R(21) + fexp(-(V - R(185)) * R(1.0 / 28.0)));
    be = fexp((V - R(158)) * R(1.0 / 16.0));
    xo[7 * so] = rush_larsen_rate(ui, logistic((V - R(99.45)) * R(1.0 / 27.48)), (al + be) * R(3), dt);
    al = R(0.0003) * lin_over_1mexp(V + R(14.1), R(5));
    be = R(7.3898e-5) * lin_over_expm1(V - R(3.3328), R(5.1237));
    xo[8 * so] = rush_larsen_rate(xr, logistic(-(V + R(14.1)) * R(1.0 / 6.5)), al + be, dt);
    al = R(4e-5) * lin_over_1mexp(V - R(19.9), R(17));
    be = R(3.5e-5) * lin_over_expm1(V - R(19.9), R(9));
    xo[9 * so] = rush_larsen_rate(xs, R(1) / fsqrt(R(1) + fexp(-(V - R(19.9)) * R(1.0 / 12.7))), (al + be) * R(2), dt);
    {
        const R yv = (V + R(10)) * R(1.0 / 6.24);
        const R g = yv == R(0) ? R(1) : -fexpm1(-yv) / yv;
        const R tau = g / (R(6.24 * 0.035) * (R(1) + fexp(-yv)));
        xo[10 * so] = rush_larsen(d, logistic(-(V + R(10)) * R(0.125)), tau, dt);
    }
    {
        const R tau = R(9) / (R(0.0197) * fexp(R(-0.0337 * 0.0337) * (V + R(10)) * (V + R(10))) + R(0.02));
        xo[11 * so] = rush_larsen(f, logistic((V + R(28)) * R(1.0 / 6.9)), tau, dt);
    }
    xo[12 * so] = rush_larsen(fCa, R(1) / (R(1) + Cai * R(1.0 / 0.00035)), R(2), dt);
    {
        const R Fn = R(1e-12) * Vrel * Irel - R(5e-13) / Fc * (R(0.5) * ICaL - R(0.2) * INaCa) * Cm;
        const R su = logistic(-(Fn - R(3.4175e-13)) * R(1.0 / 13.67e-16));
        xo[13 * so] = rush_larsen(u, su, R(8), dt);
        const R vinf = R(1) - logistic(-(Fn - R(6.835e-14)) * R(1.0 / 13.67e-16));
        xo[14 * so] = rush_larsen(vv, vinf, R(1.91) + R(2.09) * su, dt);
        const R yw = (V - R(7.9)) * R(0.2);
        const R g = yw == R(0) ? R(1) : -fexpm1(-yw) / yw;
        const R tau = R(6) * g / (R(5) * (R(1) + R(0.3) * fexp(-yw)));
        xo[15 * so] = rush_larsen(w, R(1) - logistic(-(V - R(40)) * R(1.0 / 17.0)), tau, dt);
    }

    // ---- concentrations ----
    xo[0] = Cai + dt * rt(3, B1 / B2);
    Nai_a.store_add(ao, dt * rt(1, dNai));
    Ki_a.store_add(ao + so, dt * rt(2, dKi));
    Caup_a.store_add(ao + 2 * so, dt * rt(4, dCaup));
    Carel_a.store_add(ao + 3 * so, dt * rt(5, dCarel));
    return Iion;
}

template <class R>
__device__ __forceinline__ void crn_init(const DevRegion &rg, long long i, R *V) {
    R *x = static_cast<R *>(rg.r) + i;
    double *a = rg.a + i;
    const long long st = rg.stride;
    *V = R(-81.18);
    const R v[kCRNnr] = {R(1.013e-4), R(2.908e-3), R(9.649e-1), R(9.775e-1), R(3.043e-2), R(9.992e-1),
                         R(4.966e-3), R(9.986e-1), R(3.296e-5), R(1.869e-2), R(1.367e-4), R(9.996e-1),
                         R(7.755e-1), R(0), R(1), R(9.992e-1)};
    for (int k = 0; k < kCRNnr; ++k) x[k * st] = v[k];
    Accum<R>::init(a, 11.17);
    Accum<R>::init(a + st, 139.0);
    Accum<R>::init(a + 2 * st, 1.488);
    Accum<R>::init(a + 3 * st, 1.488);
}

}  // namespace ep
