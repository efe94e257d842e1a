/*
 * Oracle (test infrastructure only): Stewart, Aslanidi, Noble, Noble, Boyett
 * & Zhang 2009 human Purkinje fibre cell model (Phil Trans R Soc A 367:2225),
 * the Purkinje cell model of Sec. 3.1. It extends the ten Tusscher-Panfilov
 * ventricular model with the hyperpolarisation-activated current I_f and the
 * sustained outward current I_sus and reparametrises I_Na, I_K1, I_to, I_Kr,
 * I_Ks. Rush-Larsen for the gates and Rbar, forward Euler for V and the
 * concentrations, all at (V^n, s^n) (Sec. 3.2); calcium buffering in the
 * rapid-buffering closed form, as for TP06.
 *
 * State: V, Ca_i, Ca_SR, Ca_SS, Na_i, K_i, m, h, j, xr1, xr2, xs, r, s, d, f,
 * f2, fCaSS, Rbar, y (20 variables).
 */
#include <math.h>
#include "oracle.h"

enum { V_, CAI, CASR, CASS, NAI, KI, M_, H_, J_, XR1, XR2, XS, R_, S_, D_, F_, F2, FCASS, RR, Y_, NVAR };

static const char *names[NVAR] = {"V", "Ca_i", "Ca_SR", "Ca_SS", "Na_i", "K_i", "m", "h", "j", "xr1",
                                  "xr2", "xs", "r", "s", "d", "f", "f2", "fCaSS", "Rbar", "y"};

static const double Rgas = 8314.472, Temp = 310.0, Fara = 96485.3415;
static const double Cm = 0.185, Vc = 0.016404, Vsr = 0.001094, Vss = 0.00005468;
static const double Nao = 140.0, Cao = 2.0;
static const double GNa = 130.5744, GK1 = 0.065, Gto = 0.08184, GKr = 0.0918, GKs = 0.2352;
static const double Gsus = 0.0227, GfNa = 0.0145654, GfK = 0.0234346, pKNa = 0.03, GCaL = 3.980e-5;
static const double kNaCa = 1000.0, gamma_ = 0.35, KmCa = 1.38, KmNai = 87.5, ksat = 0.1, alpha_ = 2.5;
static const double PNaK = 2.724, KmK = 1.0, KmNa = 40.0;
static const double GpK = 0.0146, GpCa = 0.1238, KpCa = 0.0005, GbNa = 0.00029, GbCa = 0.000592;
static const double Vmaxup = 0.006375, Kup = 0.00025, Vrel = 0.102, k1p = 0.15, k2p = 0.045;
static const double k3 = 0.060, k4 = 0.005, EC = 1.5, maxsr = 2.5, minsr = 1.0;
static const double Vleak = 0.00036, Vxfer = 0.0038;
static const double Bufc = 0.2, Kbufc = 0.001, Bufsr = 10.0, Kbufsr = 0.3, Bufss = 0.4, Kbufss = 0.00025;

int orc_stewart_nvar(void) { return NVAR; }
const char *orc_stewart_varname(int v) { return (v >= 0 && v < NVAR) ? names[v] : 0; }

void orc_stewart_init(double *s) {
    s[V_] = -69.1865;  s[KI] = 136.781894; s[NAI] = 8.80545;   s[CAI] = 0.000101878;
    s[CASS] = 0.000446818; s[CASR] = 3.10836; s[RR] = 0.991227; s[Y_] = 0.0457562;
    s[XR1] = 0.00550281; s[XR2] = 0.313298; s[XS] = 0.00953708; s[M_] = 0.0417391;
    s[H_] = 0.190678;  s[J_] = 0.238219;   s[D_] = 0.000287906; s[F_] = 0.989144;
    s[F2] = 0.995762;  s[FCASS] = 0.999934; s[S_] = 0.96589;    s[R_] = 0.00103629;
}

static double sq(double x) { return x * x; }
static double buffered_total(double ca, double B, double K) { return ca + B * ca / (ca + K); }
static double buffered_free(double tot, double B, double K) {
    double b = B + K - tot;
    return 0.5 * (-b + sqrt(b * b + 4.0 * K * tot));
}
static double rush_larsen(double y, double yinf, double tau, double dt) {
    return yinf + (y - yinf) * exp(-dt / tau);
}

double orc_stewart_step(double *s, double dt, double i_stim, const orc_cellparams *p, orc_ab2 *ab) {
    const double V = s[V_], Cai = s[CAI], Casr = s[CASR], Cass = s[CASS];
    const double Nai = s[NAI], Ki = s[KI];
    const double RTF = Rgas * Temp / Fara;
    const double Ko = p->K_o;

    const double ENa = RTF * log(Nao / Nai);
    const double EK = RTF * log(Ko / Ki);
    const double EKs = RTF * log((Ko + pKNa * Nao) / (Ki + pKNa * Nai));
    const double ECa = 0.5 * RTF * log(Cao / Cai);

    const double INa = GNa * s[M_] * s[M_] * s[M_] * s[H_] * s[J_] * (V - ENa);
    const double xl = 2.0 * (V - 15.0) / RTF;
    const double xl_over = (xl == 0.0) ? 1.0 : xl / expm1(xl);
    const double ICaL = GCaL * s[D_] * s[F_] * s[F2] * s[FCASS] * 2.0 * Fara * xl_over
                        * (0.25 * Cass * exp(xl) - Cao);
    const double Ito = Gto * s[R_] * s[S_] * (V - EK);
    const double Isus = Gsus * (1.0 / (1.0 + exp((5.0 - V) / 17.0))) * (V - EK);
    const double IKr = GKr * p->gkr_scale * sqrt(Ko / 5.4) * s[XR1] * s[XR2] * (V - EK);
    const double IKs = GKs * p->gks_scale * s[XS] * s[XS] * (V - EKs);
    const double IK1 = GK1 * (1.0 / (1.0 + exp(0.1 * (V + 75.44)))) * (V - 8.0 - EK);
    const double IfNa = s[Y_] * GfNa * (V - ENa);
    const double IfK = s[Y_] * GfK * (V - EK);
    const double INaCa = kNaCa * (exp(gamma_ * V / RTF) * Nai * Nai * Nai * Cao
                                  - exp((gamma_ - 1.0) * V / RTF) * Nao * Nao * Nao * Cai * alpha_)
                         / ((KmNai * KmNai * KmNai + Nao * Nao * Nao) * (KmCa + Cao)
                            * (1.0 + ksat * exp((gamma_ - 1.0) * V / RTF)));
    const double INaK = PNaK * Ko * Nai / ((Ko + KmK) * (Nai + KmNa)
                        * (1.0 + 0.1245 * exp(-0.1 * V / RTF) + 0.0353 * exp(-V / RTF)));
    const double IpCa = GpCa * Cai / (KpCa + Cai);
    const double IpK = GpK * (V - EK) / (1.0 + exp((25.0 - V) / 5.98));
    const double IbNa = GbNa * (V - ENa);
    const double IbCa = GbCa * (V - ECa);
    const double Iion = INa + IK1 + Ito + Isus + IKr + IKs + ICaL + INaCa + INaK + IpCa + IpK
                        + IbNa + IbCa + IfNa + IfK;

    const double kcasr = maxsr - (maxsr - minsr) / (1.0 + sq(EC / Casr));
    const double k1 = k1p / kcasr, k2 = k2p * kcasr;
    const double O = k1 * Cass * Cass * s[RR] / (k3 + k1 * Cass * Cass);
    const double Irel = Vrel * O * (Casr - Cass);
    const double Iup = Vmaxup / (1.0 + Kup * Kup / (Cai * Cai));
    const double Ileak = Vleak * (Casr - Cai);
    const double Ixfer = Vxfer * (Cass - Cai);

    const double dCai_tot = -(IbCa + IpCa - 2.0 * INaCa) * Cm / (2.0 * Vc * Fara)
                            + (Vsr / Vc) * (Ileak - Iup) + Ixfer;
    const double dCasr_tot = Iup - Irel - Ileak;
    const double dCass_tot = -ICaL * Cm / (2.0 * Vss * Fara) + (Vsr / Vss) * Irel - (Vc / Vss) * Ixfer;
    const double dNai = -(INa + IbNa + IfNa + 3.0 * INaK + 3.0 * INaCa) * Cm / (Vc * Fara);
    const double dKi = -(IK1 + Ito + Isus + IfK + IKr + IKs - 2.0 * INaK + IpK + i_stim) * Cm / (Vc * Fara);

    double ns[NVAR];
    double yinf, tau, a, b, c;
    yinf = 1.0 / sq(1.0 + exp((-56.86 - V) / 9.03));
    a = 1.0 / (1.0 + exp((-60.0 - V) / 5.0));
    b = 0.1 / (1.0 + exp((V + 35.0) / 5.0)) + 0.10 / (1.0 + exp((V - 50.0) / 200.0));
    ns[M_] = rush_larsen(s[M_], yinf, a * b, dt);
    const double hinf = 1.0 / sq(1.0 + exp((V + 71.55) / 7.43));
    if (V >= -40.0) {
        a = 0.0;
        b = 0.77 / (0.13 * (1.0 + exp(-(V + 10.66) / 11.1)));
    } else {
        a = 0.057 * exp(-(V + 80.0) / 6.8);
        b = 2.7 * exp(0.079 * V) + 3.1e5 * exp(0.3485 * V);
    }
    ns[H_] = rush_larsen(s[H_], hinf, 1.0 / (a + b), dt);
    if (V >= -40.0) {
        a = 0.0;
        b = 0.6 * exp(0.057 * V) / (1.0 + exp(-0.1 * (V + 32.0)));
    } else {
        a = (-2.5428e4 * exp(0.2444 * V) - 6.948e-6 * exp(-0.04391 * V)) * (V + 37.78)
            / (1.0 + exp(0.311 * (V + 79.23)));
        b = 0.02424 * exp(-0.01052 * V) / (1.0 + exp(-0.1378 * (V + 40.14)));
    }
    ns[J_] = rush_larsen(s[J_], hinf, 1.0 / (a + b), dt);
    yinf = 1.0 / (1.0 + exp((-26.0 - V) / 7.0));
    a = 450.0 / (1.0 + exp((-45.0 - V) / 10.0));
    b = 6.0 / (1.0 + exp((V + 30.0) / 11.5));
    ns[XR1] = rush_larsen(s[XR1], yinf, a * b, dt);
    yinf = 1.0 / (1.0 + exp((V + 88.0) / 24.0));
    a = 3.0 / (1.0 + exp((-60.0 - V) / 20.0));
    b = 1.12 / (1.0 + exp((V - 60.0) / 20.0));
    ns[XR2] = rush_larsen(s[XR2], yinf, a * b, dt);
    yinf = 1.0 / (1.0 + exp((-5.0 - V) / 14.0));
    a = 1400.0 / sqrt(1.0 + exp((5.0 - V) / 6.0));
    b = 1.0 / (1.0 + exp((V - 35.0) / 15.0));
    ns[XS] = rush_larsen(s[XS], yinf, a * b + 80.0, dt);
    /* I_to gates, Purkinje kinetics */
    yinf = 1.0 / (1.0 + exp((20.0 - V) / 13.0));
    tau = 10.45 * exp(-sq(V + 40.0) / 1800.0) + 7.3;
    ns[R_] = rush_larsen(s[R_], yinf, tau, dt);
    yinf = 1.0 / (1.0 + exp((V + 27.0) / 13.0));
    tau = 85.0 * exp(-sq(V + 25.0) / 320.0) + 5.0 / (1.0 + exp((V - 40.0) / 5.0)) + 42.0;
    ns[S_] = rush_larsen(s[S_], yinf, tau, dt);
    yinf = 1.0 / (1.0 + exp((-8.0 - V) / 7.5));
    a = 1.4 / (1.0 + exp((-35.0 - V) / 13.0)) + 0.25;
    b = 1.4 / (1.0 + exp((V + 5.0) / 5.0));
    c = 1.0 / (1.0 + exp((50.0 - V) / 20.0));
    ns[D_] = rush_larsen(s[D_], yinf, a * b + c, dt);
    yinf = 1.0 / (1.0 + exp((V + 20.0) / 7.0));
    tau = 1102.5 * exp(-sq(V + 27.0) / 225.0) + 200.0 / (1.0 + exp((13.0 - V) / 10.0))
          + 180.0 / (1.0 + exp((V + 30.0) / 10.0)) + 20.0;
    ns[F_] = rush_larsen(s[F_], yinf, tau, dt);
    yinf = 0.67 / (1.0 + exp((V + 35.0) / 7.0)) + 0.33;
    tau = 562.0 * exp(-sq(V + 27.0) / 240.0) + 31.0 / (1.0 + exp((25.0 - V) / 10.0))
          + 80.0 / (1.0 + exp((V + 30.0) / 10.0));
    ns[F2] = rush_larsen(s[F2], yinf, tau, dt);
    yinf = 0.6 / (1.0 + sq(Cass / 0.05)) + 0.4;
    tau = 80.0 / (1.0 + sq(Cass / 0.05)) + 2.0;
    ns[FCASS] = rush_larsen(s[FCASS], yinf, tau, dt);
    ns[RR] = rush_larsen(s[RR], k4 / (k2 * Cass + k4), 1.0 / (k2 * Cass + k4), dt);
    /* I_f gate */
    yinf = 1.0 / (1.0 + exp((V + 80.6) / 6.8));
    tau = 4000.0 / (exp(-2.9 - 0.04 * V) + exp(3.6 + 0.11 * V));
    ns[Y_] = rush_larsen(s[Y_], yinf, tau, dt);

    ns[NAI] = Nai + dt * orc_rate(ab, 1, dNai);
    ns[KI] = Ki + dt * orc_rate(ab, 2, dKi);
    ns[CAI] = buffered_free(buffered_total(Cai, Bufc, Kbufc) + dt * orc_rate(ab, 3, dCai_tot), Bufc, Kbufc);
    ns[CASR] = buffered_free(buffered_total(Casr, Bufsr, Kbufsr) + dt * orc_rate(ab, 4, dCasr_tot), Bufsr, Kbufsr);
    ns[CASS] = buffered_free(buffered_total(Cass, Bufss, Kbufss) + dt * orc_rate(ab, 5, dCass_tot), Bufss, Kbufss);
    for (int k = 1; k < NVAR; ++k) s[k] = ns[k];
    return Iion;
}
