/*
 * Oracle (test infrastructure only): Courtemanche, Ramirez & Nattel 1998
 * human atrial myocyte model (Am J Physiol 275:H301), the atrial cell model
 * of Sec. 3.1. Rush-Larsen for the 15 gates, forward Euler for V and the five
 * concentrations, all at (V^n, s^n) (Sec. 3.2). Calcium buffering in the
 * model's differential form (the published B1/B2 factor).
 *
 * State: V, Na_i, K_i, Ca_i, Ca_up, Ca_rel, m, h, j, oa, oi, ua, ui, xr, xs,
 * d, f, fCa, u, v, w (21 variables).
 */
#include <math.h>
#include "oracle.h"

enum { V_, NAI, KI, CAI, CAUP, CAREL, M_, H_, J_, OA, OI, UA, UI, XR, XS, D_, F_, FCA, U_, VV, W_, NVAR };

static const char *names[NVAR] = {"V", "Na_i", "K_i", "Ca_i", "Ca_up", "Ca_rel", "m", "h", "j", "oa",
                                  "oi", "ua", "ui", "xr", "xs", "d", "f", "fCa", "u", "v", "w"};

static const double Rgas = 8.3143, Temp = 310.0, Fara = 96.4867;
static const double Cm = 100.0, Vi = 13668.0, Vup = 1109.52, Vrel = 96.48;
static const double Nao = 140.0, Cao = 1.8;
static const double gNa = 7.8, gK1 = 0.09, gto = 0.1652, gKr = 0.0294, gKs = 0.129, gCaL = 0.1238;
static const double gbCa = 0.00113, gbNa = 0.000674;
static const double INaKmax = 0.59933874, INaCamax = 1600.0, IpCamax = 0.275, Iupmax = 0.005;
static const double KQ10 = 3.0, gamma_ = 0.35, KmNai = 10.0, KmKo = 1.5, KmNa = 87.5, KmCa = 1.38;
static const double ksat = 0.1, krel = 30.0, Kup = 0.00092, Caupmax = 15.0;
static const double CMDNmax = 0.05, TRPNmax = 0.07, CSQNmax = 10.0;
static const double KmCMDN = 0.00238, KmTRPN = 0.0005, KmCSQN = 0.8;
static const double tau_tr = 180.0, tau_u = 8.0, tau_fCa = 2.0;

int orc_crn_nvar(void) { return NVAR; }
const char *orc_crn_varname(int v) { return (v >= 0 && v < NVAR) ? names[v] : 0; }

void orc_crn_init(double *s) {
    s[V_] = -81.18;  s[NAI] = 11.17;  s[KI] = 139.0;   s[CAI] = 1.013e-4;
    s[CAUP] = 1.488; s[CAREL] = 1.488; s[M_] = 2.908e-3; s[H_] = 9.649e-1;
    s[J_] = 9.775e-1; s[OA] = 3.043e-2; s[OI] = 9.992e-1; s[UA] = 4.966e-3;
    s[UI] = 9.986e-1; s[XR] = 3.296e-5; s[XS] = 1.869e-2; s[D_] = 1.367e-4;
    s[F_] = 9.996e-1; s[FCA] = 7.755e-1; s[U_] = 0.0; s[VV] = 1.0; s[W_] = 9.992e-1;
}

static double rush_larsen(double y, double yinf, double tau, double dt) {
    return yinf + (y - yinf) * exp(-dt / tau);
}

/* x / (1 - exp(-x/k)), continuous at x = 0 where it equals k */
static double x_over_1mexp(double x, double k) {
    double y = x / k;
    return (y == 0.0) ? k : k * y / (-expm1(-y));
}
/* x / (exp(x/k) - 1), continuous at x = 0 where it equals k */
static double x_over_expm1(double x, double k) {
    double y = x / k;
    return (y == 0.0) ? k : k * y / expm1(y);
}

double orc_crn_step(double *s, double dt, double i_stim, const orc_cellparams *p, orc_ab2 *ab) {
    (void)i_stim;
    const double V = s[V_], Nai = s[NAI], Ki = s[KI], Cai = s[CAI];
    const double Caup = s[CAUP], Carel = s[CAREL];
    const double RTF = Rgas * Temp / Fara;
    const double Ko = p->K_o;

    const double ENa = RTF * log(Nao / Nai);
    const double EK = RTF * log(Ko / Ki);
    const double ECa = 0.5 * RTF * log(Cao / Cai);

    const double INa = gNa * s[M_] * s[M_] * s[M_] * s[H_] * s[J_] * (V - ENa);
    const double IK1 = gK1 * (V - EK) / (1.0 + exp(0.07 * (V + 80.0)));
    const double Ito = gto * s[OA] * s[OA] * s[OA] * s[OI] * (V - EK);
    const double gKur = 0.005 + 0.05 / (1.0 + exp(-(V - 15.0) / 13.0));
    const double IKur = gKur * s[UA] * s[UA] * s[UA] * s[UI] * (V - EK);
    const double IKr = gKr * p->gkr_scale * s[XR] * (V - EK) / (1.0 + exp((V + 15.0) / 22.4));
    const double IKs = gKs * p->gks_scale * s[XS] * s[XS] * (V - EK);
    const double ICaL = gCaL * s[D_] * s[F_] * s[FCA] * (V - 65.0);
    const double sigma = (exp(Nao / 67.3) - 1.0) / 7.0;
    const double fNaK = 1.0 / (1.0 + 0.1245 * exp(-0.1 * V / RTF) + 0.0365 * sigma * exp(-V / RTF));
    const double INaK = INaKmax * fNaK / (1.0 + pow(KmNai / Nai, 1.5)) * Ko / (Ko + KmKo);
    const double INaCa = INaCamax * (exp(gamma_ * V / RTF) * Nai * Nai * Nai * Cao
                                     - exp((gamma_ - 1.0) * V / RTF) * Nao * Nao * Nao * Cai)
                         / ((KmNa * KmNa * KmNa + Nao * Nao * Nao) * (KmCa + Cao)
                            * (1.0 + ksat * exp((gamma_ - 1.0) * V / RTF)));
    const double IbCa = gbCa * (V - ECa);
    const double IbNa = gbNa * (V - ENa);
    const double IpCa = IpCamax * Cai / (0.0005 + Cai);
    const double Iion = INa + IK1 + Ito + IKur + IKr + IKs + ICaL + INaK + INaCa + IbCa + IbNa + IpCa;

    const double Irel = krel * s[U_] * s[U_] * s[VV] * s[W_] * (Carel - Cai);
    const double Itr = (Caup - Carel) / tau_tr;
    const double Iup = Iupmax / (1.0 + Kup / Cai);
    const double Iupleak = Iupmax * Caup / Caupmax;

    const double dNai = (-3.0 * INaK - 3.0 * INaCa - IbNa - INa) * Cm / (Vi * Fara);
    const double dKi = (2.0 * INaK - IK1 - Ito - IKur - IKr - IKs) * Cm / (Vi * Fara);
    const double B1 = (2.0 * INaCa - IpCa - ICaL - IbCa) * Cm / (2.0 * Vi * Fara)
                      + (Vup * (Iupleak - Iup) + Irel * Vrel) / Vi;
    const double B2 = 1.0 + TRPNmax * KmTRPN / ((Cai + KmTRPN) * (Cai + KmTRPN))
                      + CMDNmax * KmCMDN / ((Cai + KmCMDN) * (Cai + KmCMDN));
    const double dCai = B1 / B2;
    const double dCaup = Iup - Iupleak - Itr * Vrel / Vup;
    const double dCarel = (Itr - Irel) / (1.0 + CSQNmax * KmCSQN / ((Carel + KmCSQN) * (Carel + KmCSQN)));

    double ns[NVAR];
    double a, b, yinf, tau;
    /* m */
    a = 0.32 * x_over_1mexp(V + 47.13, 10.0);
    b = 0.08 * exp(-V / 11.0);
    ns[M_] = rush_larsen(s[M_], a / (a + b), 1.0 / (a + b), dt);
    /* h, j */
    if (V >= -40.0) {
        a = 0.0;
        b = 1.0 / (0.13 * (1.0 + exp(-(V + 10.66) / 11.1)));
    } else {
        a = 0.135 * exp(-(V + 80.0) / 6.8);
        b = 3.56 * exp(0.079 * V) + 3.1e5 * exp(0.35 * V);
    }
    ns[H_] = rush_larsen(s[H_], a / (a + b), 1.0 / (a + b), dt);
    if (V >= -40.0) {
        a = 0.0;
        b = 0.3 * exp(-2.535e-7 * V) / (1.0 + exp(-0.1 * (V + 32.0)));
    } else {
        a = (-127140.0 * exp(0.2444 * V) - 3.474e-5 * exp(-0.04391 * V)) * (V + 37.78)
            / (1.0 + exp(0.311 * (V + 79.23)));
        b = 0.1212 * exp(-0.01052 * V) / (1.0 + exp(-0.1378 * (V + 40.14)));
    }
    ns[J_] = rush_larsen(s[J_], a / (a + b), 1.0 / (a + b), dt);
    /* oa, oi */
    a = 0.65 / (exp(-(V + 10.0) / 8.5) + exp(-(V - 30.0) / 59.0));
    b = 0.65 / (2.5 + exp((V + 82.0) / 17.0));
    ns[OA] = rush_larsen(s[OA], 1.0 / (1.0 + exp(-(V + 20.47) / 17.54)), 1.0 / ((a + b) * KQ10), dt);
    a = 1.0 / (18.53 + exp((V + 113.7) / 10.95));
    b = 1.0 / (35.56 + exp(-(V + 1.26) / 7.44));
    ns[OI] = rush_larsen(s[OI], 1.0 / (1.0 + exp((V + 43.1) / 5.3)), 1.0 / ((a + b) * KQ10), dt);
    /* ua, ui */
    a = 0.65 / (exp(-(V + 10.0) / 8.5) + exp(-(V - 30.0) / 59.0));
    b = 0.65 / (2.5 + exp((V + 82.0) / 17.0));
    ns[UA] = rush_larsen(s[UA], 1.0 / (1.0 + exp(-(V + 30.3) / 9.6)), 1.0 / ((a + b) * KQ10), dt);
    a = 1.0 / (21.0 + exp(-(V - 185.0) / 28.0));
    b = exp((V - 158.0) / 16.0);
    ns[UI] = rush_larsen(s[UI], 1.0 / (1.0 + exp((V - 99.45) / 27.48)), 1.0 / ((a + b) * KQ10), dt);
    /* xr, xs */
    a = 0.0003 * x_over_1mexp(V + 14.1, 5.0);
    b = 7.3898e-5 * x_over_expm1(V - 3.3328, 5.1237);
    ns[XR] = rush_larsen(s[XR], 1.0 / (1.0 + exp(-(V + 14.1) / 6.5)), 1.0 / (a + b), dt);
    a = 4e-5 * x_over_1mexp(V - 19.9, 17.0);
    b = 3.5e-5 * x_over_expm1(V - 19.9, 9.0);
    ns[XS] = rush_larsen(s[XS], 1.0 / sqrt(1.0 + exp(-(V - 19.9) / 12.7)), 0.5 / (a + b), dt);
    /* d: tau = (1 - e^-y) / (0.035 (V+10) (1 + e^-y)), y = (V+10)/6.24 */
    {
        double y = (V + 10.0) / 6.24;
        double g = (y == 0.0) ? 1.0 : -expm1(-y) / y;
        tau = g / (6.24 * 0.035 * (1.0 + exp(-y)));
        ns[D_] = rush_larsen(s[D_], 1.0 / (1.0 + exp(-(V + 10.0) / 8.0)), tau, dt);
    }
    /* f, fCa */
    tau = 9.0 / (0.0197 * exp(-0.0337 * 0.0337 * (V + 10.0) * (V + 10.0)) + 0.02);
    ns[F_] = rush_larsen(s[F_], 1.0 / (1.0 + exp((V + 28.0) / 6.9)), tau, dt);
    ns[FCA] = rush_larsen(s[FCA], 1.0 / (1.0 + Cai / 0.00035), tau_fCa, dt);
    /* u, v, w: release gates driven by the flux signal Fn */
    const double Fn = 1e-12 * Vrel * Irel - 5e-13 / Fara * (0.5 * ICaL - 0.2 * INaCa) * Cm;
    const double su = 1.0 / (1.0 + exp(-(Fn - 3.4175e-13) / 13.67e-16));
    ns[U_] = rush_larsen(s[U_], su, tau_u, dt);
    yinf = 1.0 - 1.0 / (1.0 + exp(-(Fn - 6.835e-14) / 13.67e-16));
    ns[VV] = rush_larsen(s[VV], yinf, 1.91 + 2.09 * su, dt);
    {
        double y = (V - 7.9) / 5.0;
        double g = (y == 0.0) ? 1.0 : -expm1(-y) / y;
        tau = 6.0 * g / (5.0 * (1.0 + 0.3 * exp(-y)));
        ns[W_] = rush_larsen(s[W_], 1.0 - 1.0 / (1.0 + exp(-(V - 40.0) / 17.0)), tau, dt);
    }

    ns[NAI] = Nai + dt * orc_rate(ab, 1, dNai);
    ns[KI] = Ki + dt * orc_rate(ab, 2, dKi);
    ns[CAI] = Cai + dt * orc_rate(ab, 3, dCai);
    ns[CAUP] = Caup + dt * orc_rate(ab, 4, dCaup);
    ns[CAREL] = Carel + dt * orc_rate(ab, 5, dCarel);
    for (int k = 1; k < NVAR; ++k) s[k] = ns[k];
    return Iion;
}
