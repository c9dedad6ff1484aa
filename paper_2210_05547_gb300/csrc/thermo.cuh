// Per-point thermochemistry closure (Sec. 2.2), FP64, shared by the host set-up code and the
// kernels of this library. All quantities SI unless stated.
#pragma once

#include <math.h>

#include "internal.h"

namespace hyp {

constexpr double R_U = 1.380649e-23 * 6.02214076e23;   // N_A k_B, J/(mol K)
constexpr double P_STD = 1.0e5;
constexpr double T_LO = 50.0;
constexpr double T_HI = 100000.0;
constexpr int NEWTON_MAXIT = 60;
constexpr double NEWTON_RTOL = 1.0e-11;
constexpr double SUTH_C1 = 1.458e-6;   // Eq. (24)
constexpr double SUTH_TS = 110.4;      // Eq. (24)

// Species modal sums at temperature T: energies (J/kg), heat capacities, and the electronic
// partition function / mean level used by the entropy.
struct SpeciesState {
    double e[NSP];      // internal energy including formation, J/kg
    double cv[NSP];     // J/(kg K)
    double qel[NSP];    // electronic partition function
    double m1[NSP];     // Boltzmann mean of theta_el
    double xv[NSP];     // theta_v / T (molecules)
    double em1[NSP];    // expm1(theta_v / T) (molecules)
};

__host__ __device__ inline void species_state(const GasDev& g, double T, SpeciesState& s) {
    const double invT = 1.0 / T;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        double q = 0.0, m1 = 0.0, m2 = 0.0;
        for (int l = 0; l < g.nlev[i]; ++l) {
            const double th = g.lev_th[i][l];
            const double w = g.lev_g[i][l] * exp(-th * invT);
            q += w;
            m1 += w * th;
            m2 += w * th * th;
        }
        m1 /= q;
        m2 /= q;
        double eo = 1.5 * T + m1;
        double cvo = 1.5 + (m2 - m1 * m1) * invT * invT;
        double xv = 0.0, em1 = 0.0;
        if (g.linear[i]) {
            xv = g.theta_v[i] * invT;
            em1 = expm1(xv);
            eo += T + g.theta_v[i] / em1;
            cvo += 1.0 + xv * xv * (em1 + 1.0) / (em1 * em1);
        }
        s.e[i] = g.e0[i] + g.Rs[i] * eo;
        s.cv[i] = g.Rs[i] * cvo;
        s.qel[i] = q;
        s.m1[i] = m1;
        s.xv[i] = xv;
        s.em1[i] = em1;
    }
}

__host__ __device__ inline double mixture_energy(const GasDev& g, double T, const double* Y) {
    SpeciesState s;
    species_state(g, T, s);
    double e = 0.0;
#pragma unroll
    for (int i = 0; i < NSP; ++i) e += Y[i] * s.e[i];
    return e;
}

// Safeguarded Newton for sum_s Y_s e_s(T) = e, same stopping rule for every caller.
__host__ __device__ inline double temperature_from_energy(const GasDev& g, double e,
                                                          const double* Y, double T0,
                                                          unsigned& status, SpeciesState& s) {
    double T = fmin(fmax(T0, T_LO), T_HI);
    double lo = T_LO, hi = T_HI;
    bool converged = false;
    for (int it = 0; it < NEWTON_MAXIT; ++it) {
        species_state(g, T, s);
        double f = -e, cv = 0.0;
#pragma unroll
        for (int i = 0; i < NSP; ++i) {
            f += Y[i] * s.e[i];
            cv += Y[i] * s.cv[i];
        }
        if (f > 0.0) hi = T; else lo = T;
        double Tn = T - f / cv;
        if (fabs(Tn - T) <= NEWTON_RTOL * T) {
            T = Tn;
            converged = true;
            break;
        }
        if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
        T = Tn;
    }
    if (!converged) {
        const double elo = mixture_energy(g, T_LO, Y);
        const double ehi = mixture_energy(g, T_HI, Y);
        if (e <= elo) {
            T = T_LO;
            status |= HYP_STATUS_T_CLAMPED;
        } else if (e >= ehi) {
            T = T_HI;
            status |= HYP_STATUS_T_CLAMPED;
        } else {
            status |= HYP_STATUS_NOT_CONVERGED;
        }
    }
    species_state(g, T, s);
    return T;
}

struct ClosureOut {
    double T, p, cv, Rmix, a;
    double h[NSP];      // J/kg
    double wdot[NSP];   // kg/(m^3 s)
    double X[NSP];
    double D[NSP];      // m^2/s
    double mu, k;
    unsigned status;
};

// Full closure (SI). reactions: evaluate w_s; transport: evaluate mu, k, D_s.
__host__ __device__ inline void closure_si(const GasDev& g, double rho, double e, const double* Y,
                                           double T0, bool reactions, bool diffusion,
                                           ClosureOut& o) {
    SpeciesState s;
    o.status = rho > 0.0 ? 0u : HYP_STATUS_NONPHYSICAL;
    const double T = temperature_from_energy(g, e, Y, T0, o.status, s);
    double ym = 0.0, cv = 0.0;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        ym += Y[i] * g.invM[i];
        cv += Y[i] * s.cv[i];
    }
    const double Rmix = R_U * ym;
    const double p = rho * Rmix * T;
    o.T = T;
    o.p = p;
    o.cv = cv;
    o.Rmix = Rmix;
    o.a = sqrt((cv + Rmix) / cv * p / rho);
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        o.h[i] = s.e[i] + g.Rs[i] * T;
        o.X[i] = Y[i] * g.invM[i] / ym;
    }
    const double lnT = log(T);
    const double invT = 1.0 / T;

    // ---- kinetics (Eqs. 14, 15) ----
#pragma unroll
    for (int i = 0; i < NSP; ++i) o.wdot[i] = 0.0;
    if (reactions) {
        double grt[NSP];      // G_s / (R_u T) at p_std
#pragma unroll
        for (int i = 0; i < NSP; ++i) {
            double S = g.s0[i] + 2.5 * lnT + log(s.qel[i]) + s.m1[i] * invT;
            if (g.linear[i]) S += lnT + s.xv[i] / s.em1[i] - log(-expm1(-s.xv[i]));
            grt[i] = o.h[i] / (g.Rs[i] * T) - S;
        }
        const double ln_pref = log(P_STD / (R_U * T));
        double Ef[MAXG], Eb[MAXG];
        for (int k = 0; k < g.ngroup; ++k) {
            double lnkc = g.g_dnu[k] * ln_pref;
#pragma unroll
            for (int i = 0; i < NSP; ++i) lnkc -= g.g_nu[k][i] * grt[i];
            const double base = g.g_n[k] * lnT - g.g_Ta[k] * invT;
            Ef[k] = exp(base);
            Eb[k] = exp(base - lnkc);
        }
        double conc[NSP];
#pragma unroll
        for (int i = 0; i < NSP; ++i) conc[i] = rho * Y[i] * g.invM[i];
        double molar[NSP];
#pragma unroll
        for (int i = 0; i < NSP; ++i) molar[i] = 0.0;
        for (int r = 0; r < g.nr; ++r) {
            double fwd = 1.0, bwd = 1.0;
#pragma unroll
            for (int i = 0; i < NSP; ++i) {
                for (int q = 0; q < g.nu_f[r][i]; ++q) fwd *= conc[i];
                for (int q = 0; q < g.nu_b[r][i]; ++q) bwd *= conc[i];
            }
            const int k = g.group[r];
            const double R = g.C[r] * Ef[k] * fwd - g.C[r] * Eb[k] * bwd;
#pragma unroll
            for (int i = 0; i < NSP; ++i) molar[i] += (g.nu_b[r][i] - g.nu_f[r][i]) * R;
        }
#pragma unroll
        for (int i = 0; i < NSP; ++i) o.wdot[i] = g.M[i] * molar[i];
    }

    // ---- transport ----
    double mu_s[NSP], sq[NSP], k_s[NSP];
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        mu_s[i] = 0.1 * exp((g.blA[i] * lnT + g.blB[i]) * lnT + g.blC[i]);
        sq[i] = sqrt(mu_s[i]);
        const double cv_tr = 1.5 * g.Rs[i];
        k_s[i] = mu_s[i] * (2.5 * cv_tr + (s.cv[i] - cv_tr));
    }
    double mu = 0.0, kk = 0.0;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        double phi = 0.0;
#pragma unroll
        for (int r = 0; r < NSP; ++r) {
            const double t = 1.0 + sq[i] / sq[r] * g.wilke_q[i][r];
            phi += o.X[r] * t * t * g.wilke_d[i][r];
        }
        mu += o.X[i] * mu_s[i] / phi;
        kk += o.X[i] * k_s[i] / phi;
    }
    o.mu = mu;
    o.k = kk;
#pragma unroll
    for (int i = 0; i < NSP; ++i) o.D[i] = 0.0;
    if (diffusion) {
        // Neufeld-Janzen-Aziz fit of Omega^(1,1)* per distinct well depth
        double om[MAXEPS];
        for (int q = 0; q < g.neps; ++q) {
            const double lts = lnT - g.ln_eps[q];
            const double ts = exp(lts);
            om[q] = 1.06036 * exp(-0.15610 * lts) + 0.19300 * exp(-0.47635 * ts) +
                    1.03587 * exp(-1.52996 * ts) + 1.76474 * exp(-3.89411 * ts);
        }
        const double c = p / (T * sqrt(T));
#pragma unroll
        for (int i = 0; i < NSP; ++i) {
            double den = 0.0;
#pragma unroll
            for (int r = 0; r < NSP; ++r)
                if (r != i) den += o.X[r] * (c * om[g.eps_group[i][r]] * g.dinv[i][r]);
            o.D[i] = den != 0.0 ? (1.0 - o.X[i]) / den : 0.0;
        }
    }
}

}  // namespace hyp
