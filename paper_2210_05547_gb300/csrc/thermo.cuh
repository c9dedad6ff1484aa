// Per-point thermochemistry closure (Sec. 2.2), FP64, shared by the host set-up code and the
// kernels of this library. All quantities SI unless stated.
//
// On GB300 the FP64 pipe (two FMAs per clock per SM) bounds this code, so it avoids FP64 work
// that cannot change a result: electronic levels whose Boltzmann factor is below e^-45 of the
// ground level are not evaluated (relative contribution under 1e-19), the equilibrium constants
// come from molar partition functions instead of logarithms of Gibbs energies, reactions sharing
// (n, T_a, net stoichiometry) share their exponentials, and collision-integral terms below e^-40
// of the fit are skipped.
#pragma once

#include <math.h>

#include "internal.h"
#ifdef __CUDACC__
#include "fp32.cuh"
#include "fp64_fast.cuh"
#endif

namespace hyp {

constexpr double R_U = 1.380649e-23 * 6.02214076e23;   // N_A k_B, J/(mol K)
constexpr double P_STD = 1.0e5;
constexpr double T_LO = 50.0;
constexpr double T_HI = 100000.0;
constexpr int NEWTON_MAXIT = 60;
// Stop after a Newton step of at most 1e-8 T: the error left after that step is of order
// (dT/T)^2 ~ 1e-16 relative.
constexpr double NEWTON_RTOL = 1.0e-8;
constexpr double NEWTON_RTOL_MIXED = 1.0e-6;   // binary32 modal sums (temperature_from_energy)
constexpr double SUTH_C1 = 1.458e-6;   // Eq. (24)
constexpr double SUTH_TS = 110.4;      // Eq. (24)
constexpr double LEVEL_CUT = 45.0;     // skip electronic levels with theta / T above this
constexpr double OMEGA_CUT = 40.0;     // skip collision-integral exponentials below e^-40
// Neufeld-Janzen-Aziz fit of the reduced diffusion collision integral Omega^(1,1)*
constexpr double NJA_A = 1.06036, NJA_B = 0.15610, NJA_C = 0.19300, NJA_D = 0.47635;
constexpr double NJA_E = 1.03587, NJA_F = 1.52996, NJA_G = 1.76474, NJA_H = 3.89411;

// Binary64 exponential, quotient and reciprocal of the closure: on the device the forms of
// fp64_fast.cuh (Tang's table-driven exp, Newton-refined binary32 reciprocals; within 2 ulp, on
// about half the FP64-pipe instructions of CUDA's), on the host the C library.
__host__ __device__ __forceinline__ double cl_exp(double x) {
#ifdef __CUDA_ARCH__
    return tang_exp(x);
#else
    return exp(x);
#endif
}

__host__ __device__ __forceinline__ double cl_div(double a, double b) {
#ifdef __CUDA_ARCH__
    return fast_div(a, b);
#else
    return a / b;
#endif
}

__host__ __device__ __forceinline__ double cl_rcp(double b) {
#ifdef __CUDA_ARCH__
    return fast_rcp(b);
#else
    return 1.0 / b;
#endif
}

// Natural logarithm: on the device Tang's table-driven form for x >= 2 (fp64_fast.cuh; within
// 1 ulp, 11 FP64 instructions against CUDA's ~28), CUDA's log below; on the host the C library.
__host__ __device__ __forceinline__ double cl_log(double x) {
#ifdef __CUDA_ARCH__
    return table_log(x);
#else
    return log(x);
#endif
}

// 1 / (e^x - 1) for x > 0: from the exponential where e^x - 1 loses at most a bit (x >= 1),
// from expm1 below.
__host__ __device__ __forceinline__ double cl_inv_expm1(double x) {
    return x >= 1.0 ? cl_rcp(cl_exp(x) - 1.0) : 1.0 / expm1(x);
}

// Species modal sums at temperature T: energies (J/kg), heat capacities and their temperature
// derivative, and the electronic partition function / vibrational factor used by the equilibrium
// constants, with what a first-order shift in T needs.
struct SpeciesState {
    double e[NSP];      // internal energy including formation, J/kg
    double cv[NSP];     // J/(kg K)
    double cvp[NSP];    // d c_v / dT
    double qel[NSP];    // electronic partition function
    double m1[NSP];     // Boltzmann mean of theta_el (d ln q_el / dT = m1 / T^2)
    double iem1[NSP];   // 1 / expm1(theta_v / T) (molecules): q_vib = 1 + iem1
    double xv[NSP];     // theta_v / T
};

__host__ __device__ __forceinline__ void species_state(const GasDev& g, double T, SpeciesState& s) {
    const double invT = cl_rcp(T);
    const double invT2 = invT * invT;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        double q = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
        for (int l = 0; l < g.nlev[i]; ++l) {
            const double th = g.lev_th[i][l];
            const double x = th * invT;
            if (x > LEVEL_CUT) break;
            const double w = th == 0.0 ? g.lev_g[i][l] : g.lev_g[i][l] * cl_exp(-x);
            const double wt = w * th;
            q += w;
            m1 += wt;
            m2 += wt * th;
            m3 += wt * th * th;
        }
        const double iq = cl_rcp(q);
        m1 *= iq;
        m2 *= iq;
        m3 *= iq;
        const double var = m2 - m1 * m1;
        double eo = 1.5 * T + m1;
        double cvo = 1.5 + var * invT2;
        // d/dT of var / T^2 with d m1/dT = var / T^2, d m2/dT = (m3 - m1 m2) / T^2
        double cvpo = ((m3 - m1 * m2) - 2.0 * m1 * var) * invT2 * invT2 - 2.0 * var * invT2 * invT;
        double r = 0.0, xv = 0.0;
        if (g.linear[i]) {
            xv = g.theta_v[i] * invT;
            r = cl_inv_expm1(xv);
            const double b = (1.0 + r) * r;                  // e^x / (e^x - 1)^2
            eo += T + g.theta_v[i] * r;
            cvo += 1.0 + xv * xv * b;
            // d/dT [x^2 e^x / (e^x - 1)^2] = -(x / T) x b (2 - x - 2 x r)
            cvpo -= xv * invT * xv * b * (2.0 - xv - 2.0 * xv * r);
        }
        s.e[i] = g.e0[i] + g.Rs[i] * eo;
        s.cv[i] = g.Rs[i] * cvo;
        s.cvp[i] = g.Rs[i] * cvpo;
        s.qel[i] = q;
        s.m1[i] = m1;
        s.iem1[i] = r;
        s.xv[i] = xv;
    }
}

// First-order shift of a species state from T to T + dT (used after a Newton step of at most
// 1e-8 T, where the neglected second-order terms are below 1e-16 relative).
__host__ __device__ __forceinline__ void species_shift(const GasDev& g, double T, double dT, SpeciesState& s) {
    const double invT = cl_rcp(T);
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        s.e[i] += s.cv[i] * dT;
        s.cv[i] += s.cvp[i] * dT;
        s.qel[i] += s.qel[i] * s.m1[i] * invT * invT * dT;
        if (g.linear[i]) {
            const double r = s.iem1[i];
            s.iem1[i] = r + s.xv[i] * invT * (1.0 + r) * r * dT;   // d/dT 1/(e^x - 1)
            s.xv[i] -= s.xv[i] * invT * dT;
        }
    }
}

#ifdef __CUDACC__
// The species modal sums of species_state for the mixed-precision closure (HYP_MIXED), split by
// what each term contributes to the energy. In binary64: the vibrational factor
// r = 1 / (e^x - 1) (theta_v r reaches ~T at high temperature) and the Boltzmann factors of the
// populated electronic levels (theta / T < LEVEL_HOT_F64: the fine-structure levels of O and NO
// at any temperature, the excited levels once they hold more than ~1e-4 of the population), with
// the partition function q_el and the mean level energy m1 summed over them in binary64. In
// binary32: the weakly populated levels (a level's energy share is at most (g_l / g_0) 9 e^-9 <=
// 6.7e-3 of T, so its binary32 rounding, ~1e-6 relative with that of theta / T, moves e_s by
// < 1e-8 R_s T), the second and third level moments and the heat capacities with their
// temperature derivative. A fully binary32 electronic sum was measured to move the inverted
// temperature by up to 5e-8 relative, which the exponents T_a / T ~ 50 of the dissociation rates
// carry into the species source terms at ~1e-6 of their scale. The energy is assembled in
// binary64 from its formation, translational-rotational (exact multiples of T), vibrational and
// electronic parts. Every binary32 multiply and add is explicit, as in transport_f32.
constexpr float LEVEL_HOT_F64 = 9.0f;

__device__ __forceinline__ void species_state_f32(const GasDev& g, double T, SpeciesState& s) {
    const double invT = cl_rcp(T);
    const float iT = f32_of(invT);
    const float iT2 = __fmul_rn(iT, iT);
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        double qd = 0.0, s1d = 0.0;                     // binary64 sums: populated levels
        float qc = 0.0f, s1c = 0.0f, s2 = 0.0f, s3 = 0.0f;
        for (int l = 0; l < g.nlev[i]; ++l) {
            const float th = f32_of(g.lev_th[i][l]);
            const float x = __fmul_rn(th, iT);
            if (x > (float)LEVEL_CUT) break;
            float w;
            if (x < LEVEL_HOT_F64) {
                const double wd = th == 0.0f ? g.lev_g[i][l]
                                             : g.lev_g[i][l] * cl_exp(-(g.lev_th[i][l] * invT));
                qd += wd;
                s1d = fma(wd, g.lev_th[i][l], s1d);
                w = f32_of(wd);
            } else {
                w = __fmul_rn(f32_of(g.lev_g[i][l]), expf(-x));
                qc = __fadd_rn(qc, w);
                s1c = fmaf(w, th, s1c);
            }
            const float wt2 = __fmul_rn(__fmul_rn(w, th), th);
            s2 = __fadd_rn(s2, wt2);
            s3 = fmaf(wt2, th, s3);
        }
        qd += f64_of(qc);
        // with no populated excited level (N2, and N and O2 below a few thousand K) the mean level
        // energy is the weak levels' alone, below 3e-3 T: binary32 suffices
        const double m1d = s1d == 0.0 ? f64_of(__fdiv_rn(s1c, f32_of(qd)))
                                      : cl_div(s1d + f64_of(s1c), qd);
        const float iq = __frcp_rn(f32_of(qd));
        const float m1 = f32_of(m1d);
        const float m2 = __fmul_rn(s2, iq);
        const float m3 = __fmul_rn(s3, iq);
        const float var = fmaf(-m1, m1, m2);
        double ev = m1d;                                 // electronic + vibrational energy, K
        float cvo = fmaf(var, iT2, 1.5f);
        float cvpo = __fmul_rn(__fmul_rn(fmaf(-2.0f * m1, var, fmaf(-m1, m2, m3)), iT2), iT2);
        cvpo = fmaf(__fmul_rn(-2.0f * var, iT2), iT, cvpo);
        if (g.linear[i]) {
            const double xd = g.theta_v[i] * invT;
            const double rd = cl_inv_expm1(xd);
            ev = fma(g.theta_v[i], rd, ev);
            const float xv = f32_of(xd);
            const float r = f32_of(rd);
            const float b = __fmul_rn(__fadd_rn(1.0f, r), r);
            const float xb = __fmul_rn(__fmul_rn(xv, xv), b);
            cvo = __fadd_rn(cvo, __fadd_rn(1.0f, xb));
            // d/dT [x^2 e^x / (e^x - 1)^2] = -(x / T) x b (2 - x - 2 x r)
            const float t = __fsub_rn(__fsub_rn(2.0f, xv), __fmul_rn(2.0f * xv, r));
            cvpo = fmaf(-__fmul_rn(xb, iT), t, cvpo);
            s.iem1[i] = rd;
            s.xv[i] = xd;
        } else {
            s.iem1[i] = 0.0;
            s.xv[i] = 0.0;
        }
        const double ctr = g.linear[i] ? 2.5 : 1.5;     // translation (+ rotation), per R_s
        s.e[i] = fma(g.Rs[i], fma(ctr, T, ev), g.e0[i]);
        s.cv[i] = f64_of(__fmul_rn(g.f_Rs[i], cvo));
        s.cvp[i] = f64_of(__fmul_rn(g.f_Rs[i], cvpo));
        s.qel[i] = qd;
        s.m1[i] = m1d;
    }
}
#endif

__host__ __device__ __forceinline__ double mixture_energy(const GasDev& g, double T, const double* Y) {
    SpeciesState s;
    species_state(g, T, s);
    double e = 0.0;
#pragma unroll
    for (int i = 0; i < NSP; ++i) e += Y[i] * s.e[i];
    return e;
}

// Starting temperature for the inversion of e = sum_s Y_s e_s(T) from the tabulated species
// energies: bisection over the table's temperatures for the bracketing interval, then the cubic
// Hermite model of e(T) on it (values and heat capacities at its ends) inverted by three Newton
// steps. Only the starting point of the safeguarded Newton iteration below: the temperature it
// returns does not depend on it beyond the iteration's tolerance.
__host__ __device__ __forceinline__ double temperature_guess(const GasDev& g, double e, const double* Y) {
    const double* et = g.etab;       // device only: [e | c_v][species][ETAB_N]
    auto emix = [&](int k) {
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < NSP; ++i) s += Y[i] * et[i * ETAB_N + k];
        return s;
    };
    int lo = 0, hi = ETAB_N - 1;
    if (!(e > emix(lo))) return T_LO;
    if (!(e < emix(hi))) return T_HI;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (emix(mid) <= e) lo = mid; else hi = mid;
    }
    const double Ta = cl_exp(g.etab_lnT0 + lo * g.etab_dlnT), Tb = cl_exp(g.etab_lnT0 + hi * g.etab_dlnT);
    const double ea = emix(lo), eb = emix(hi);
    double ca = 0.0, cb = 0.0;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        ca += Y[i] * et[(NSP + i) * ETAB_N + lo];
        cb += Y[i] * et[(NSP + i) * ETAB_N + hi];
    }
    const double h = Tb - Ta;
    double t = cl_div(e - ea, eb - ea);              // linear start
    for (int it = 0; it < 3; ++it) {
        const double t2 = t * t, t3 = t2 * t;
        const double h00 = 2 * t3 - 3 * t2 + 1, h10 = t3 - 2 * t2 + t;
        const double h01 = -2 * t3 + 3 * t2, h11 = t3 - t2;
        const double f = h00 * ea + h10 * h * ca + h01 * eb + h11 * h * cb - e;
        const double df = (6 * t2 - 6 * t) * ea + (3 * t2 - 4 * t + 1) * h * ca +
                          (-6 * t2 + 6 * t) * eb + (3 * t2 - 2 * t) * h * cb;
        if (df > 0.0) t -= cl_div(f, df);
        t = fmin(fmax(t, 0.0), 1.0);
    }
    return Ta + t * h;
}

#ifdef __CUDACC__
// The first-order shift of species_shift for the mixed-precision closure. The step is below
// 1e-6 T (NEWTON_RTOL_MIXED), so the corrections of the partition function and vibrational
// factor are at most 45 x 1e-6 of the value. They are formed in binary32, whose rounding stays
// below 1e-11 of the value, and added in binary64. The energies and heat capacities take their
// binary64 FMA. theta_v / T is not carried on, since nothing reads it after the shift.
__device__ __forceinline__ void species_shift_f32(const GasDev& g, double T, double dT,
                                                  SpeciesState& s) {
    const float iT = __frcp_rn(f32_of(T));
    const float dTf = f32_of(dT);
    const float idT = __fmul_rn(iT, dTf);
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        s.e[i] = fma(s.cv[i], dT, s.e[i]);
        s.cv[i] = fma(s.cvp[i], dT, s.cv[i]);
        s.qel[i] += f64_of(__fmul_rn(__fmul_rn(f32_of(s.qel[i]), f32_of(s.m1[i])), __fmul_rn(iT, idT)));
        if (g.linear[i]) {
            const float r = f32_of(s.iem1[i]);
            s.iem1[i] += f64_of(__fmul_rn(__fmul_rn(f32_of(s.xv[i]), idT), __fmul_rn(__fadd_rn(1.0f, r), r)));
        }
    }
}
#endif

// Safeguarded Newton for sum_s Y_s e_s(T) = e; s holds the species state at the returned T.
// MIXED (device only): the electronic modal sums in binary32 (species_state_f32). Their rounding
// moves sum_s Y_s e_s(T) by up to ~1e-8 c_v T, so successive Newton steps need not fall below
// 1e-8 T; the iteration stops at 1e-6 T instead, where the step's own error, (dT/T)^2 relative,
// and that of the first-order shift are ~1e-12, far below the binary32 part.
template <bool MIXED = false>
__host__ __device__ __forceinline__ double temperature_from_energy(const GasDev& g, double e,
                                                          const double* Y, double T0,
                                                          unsigned& status, SpeciesState& s) {
    double T = fmin(fmax(T0, T_LO), T_HI);
    double lo = T_LO, hi = T_HI;
    for (int it = 0; it < NEWTON_MAXIT; ++it) {
#ifdef __CUDA_ARCH__
        if constexpr (MIXED) species_state_f32(g, T, s);
        else
#endif
            species_state(g, T, s);
        double f = -e, cv = 0.0;
#pragma unroll
        for (int i = 0; i < NSP; ++i) {
            f += Y[i] * s.e[i];
            cv += Y[i] * s.cv[i];
        }
        if (f > 0.0) hi = T; else lo = T;
        double Tn = T - cl_div(f, cv);
        if (fabs(Tn - T) <= (MIXED ? NEWTON_RTOL_MIXED : NEWTON_RTOL) * T) {
#ifdef __CUDA_ARCH__
            if constexpr (MIXED) species_shift_f32(g, T, Tn - T, s);
            else
#endif
                species_shift(g, T, Tn - T, s);
            return Tn;
        }
        if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
        T = Tn;
    }
    {
        // the energy lies outside the temperature range (T clamped to its end) or the iteration
        // failed; the mixture energies at the ends come from the species energies there, which
        // the gas model holds (full species evaluations inlined here would only add code)
        double elo = 0.0, ehi = 0.0;
#pragma unroll
        for (int i = 0; i < NSP; ++i) {
            elo += Y[i] * g.e_lo[i];
            ehi += Y[i] * g.e_hi[i];
        }
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
    double es[NSP];     // species energies at T (J/kg), kept as the next Newton predictor
    double cvs[NSP];    // species heat capacities at T
    double cvps[NSP];   // their temperature derivatives
    double mu, k;
    unsigned status;
};

#ifdef __CUDACC__
// Transport and diffusion in binary32 for the mixed-precision closure (HYP_MIXED): the same
// Blottner, Eucken, Wilke and Chapman-Enskog formulas as the FP64 code in closure_si, on binary32
// copies of the constants. Inputs and outputs cross with the integer conversions of fp32.cuh.
__device__ __forceinline__ void transport_f32(const GasDev& g, double T, double lnT, double p,
                                     const SpeciesState& s, bool diffusion, ClosureOut& o) {
    // every binary32 multiply and add is explicit (fmaf where a fused operation is meant,
    // __fmul_rn / __fadd_rn / __fdiv_rn elsewhere): no contraction is left to the compiler, so
    // the result does not depend on the kernel this body is compiled into
    const float lnTf = f32_of(lnT);
    float Xf[NSP], mu_s[NSP], a[NSP], b[NSP], k_s[NSP];
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        Xf[i] = f32_of(o.X[i]);
        mu_s[i] = __fmul_rn(0.1f, expf(fmaf(fmaf(g.f_blA[i], lnTf, g.f_blB[i]), lnTf, g.f_blC[i])));
        const float ir = rsqrtf(mu_s[i]);
        a[i] = __fmul_rn(__fmul_rn(mu_s[i], ir), g.f_iMq[i]);
        b[i] = __fmul_rn(g.f_Mq[i], ir);
        const float cv_tr = __fmul_rn(1.5f, g.f_Rs[i]);
        k_s[i] = __fmul_rn(mu_s[i], fmaf(2.5f, cv_tr, __fsub_rn(f32_of(s.cv[i]), cv_tr)));
    }
    float mu = 0.0f, kk = 0.0f;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        if (HAS_CHARGE && !g.heavy[i]) continue;      // the electron is not in the mixing rule
        float phi = 0.0f;
#pragma unroll
        for (int r = 0; r < NSP; ++r) {
            if (HAS_CHARGE && !g.heavy[r]) continue;
            if (r == i) {
                phi = __fadd_rn(phi, Xf[i]);    // (1 + a_i b_i)^2 d_ii = 1
                continue;
            }
            const float t = fmaf(a[i], b[r], 1.0f);
            phi = fmaf(__fmul_rn(__fmul_rn(Xf[r], t), t), g.f_wilke_d[i][r], phi);
        }
        const float w = __fdiv_rn(Xf[i], phi);
        mu = fmaf(w, mu_s[i], mu);
        kk = fmaf(w, k_s[i], kk);
    }
    o.mu = f64_of(mu);
    o.k = f64_of(kk);
#pragma unroll
    for (int i = 0; i < NSP; ++i) o.D[i] = 0.0;
    if (!diffusion) return;
    float den[NSP];
#pragma unroll
    for (int i = 0; i < NSP; ++i) den[i] = 0.0f;
    const float Tf = f32_of(T);
    const float TmB = expf(__fmul_rn(-(float)NJA_B, lnTf));
    const float c = __fdiv_rn(f32_of(p), __fmul_rn(Tf, sqrtf(Tf)));
    for (int q = 0; q < g.neps; ++q) {
        const float ts = __fmul_rn(Tf, g.f_eps_inv[q]);
        float om = __fmul_rn(__fmul_rn((float)NJA_A, TmB), g.f_eps_powB[q]);
        const float xd = __fmul_rn((float)NJA_D, ts), xf = __fmul_rn((float)NJA_F, ts);
        const float xh = __fmul_rn((float)NJA_H, ts);
        if (xd < (float)OMEGA_CUT) om = fmaf((float)NJA_C, expf(-xd), om);
        if (xf < (float)OMEGA_CUT) om = fmaf((float)NJA_E, expf(-xf), om);
        if (xh < (float)OMEGA_CUT) om = fmaf((float)NJA_G, expf(-xh), om);
        const float com = __fmul_rn(c, om);
        for (int pr = g.pstart[q]; pr < g.pstart[q + 1]; ++pr) {
            const int i = g.pair_i[pr], r = g.pair_r[pr];
            const float inv_d = __fmul_rn(com, g.f_pair_dinv[pr]);
            den[i] = fmaf(Xf[r], inv_d, den[i]);
            den[r] = fmaf(Xf[i], inv_d, den[r]);
        }
    }
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        o.D[i] = den[i] != 0.0f ? f64_of(__fdiv_rn(__fsub_rn(1.0f, Xf[i]), den[i])) : 0.0;
        if (HAS_CHARGE) o.D[i] = __dmul_rn(o.D[i], g.dfac[i]);   // ambipolar ions, no electron coefficient
    }
}
#endif

// Transport and diffusion in FP64: Blottner species viscosities, Eucken conductivities, Wilke's
// mixing rule and the averaged diffusion coefficients of Eq. (19).
__host__ __device__ __forceinline__ void transport_f64(const GasDev& g, double T, double lnT, double p,
                                              const SpeciesState& s, bool diffusion,
                                              ClosureOut& o) {
    // ---- transport: Blottner, Eucken, Wilke ----
    // sqrt(mu_i / mu_r) (M_r / M_i)^(1/4) = a_i b_r with a_i = sqrt(mu_i) M_i^(-1/4),
    // b_r = M_r^(1/4) / sqrt(mu_r)
    double mu_s[NSP], a[NSP], b[NSP], k_s[NSP];
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        mu_s[i] = 0.1 * cl_exp((g.blA[i] * lnT + g.blB[i]) * lnT + g.blC[i]);
        const double rs = rsqrt(mu_s[i]);           // 1 / sqrt(mu_i): one FP64 sequence for both
        a[i] = mu_s[i] * rs * g.iMq[i];
        b[i] = g.Mq[i] * rs;
        const double cv_tr = 1.5 * g.Rs[i];
        k_s[i] = mu_s[i] * (2.5 * cv_tr + (s.cv[i] - cv_tr));
    }
    double mu = 0.0, kk = 0.0;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        if (HAS_CHARGE && !g.heavy[i]) continue;      // the electron is not in the mixing rule
        double phi = 0.0;
#pragma unroll
        for (int r = 0; r < NSP; ++r) {
            if (HAS_CHARGE && !g.heavy[r]) continue;
            if (r == i) {
                phi += o.X[i];          // (1 + a_i b_i)^2 d_ii = 2^2 / sqrt(16) = 1
                continue;
            }
            const double t = 1.0 + a[i] * b[r];
            phi += o.X[r] * t * t * g.wilke_d[i][r];
        }
        const double w = cl_div(o.X[i], phi);
        mu += w * mu_s[i];
        kk += w * k_s[i];
    }
    o.mu = mu;
    o.k = kk;

    // ---- averaged diffusion coefficients (Eq. 19) from Chapman-Enskog binary coefficients ----
#pragma unroll
    for (int i = 0; i < NSP; ++i) o.D[i] = 0.0;
    if (diffusion) {
        double den[NSP];
#pragma unroll
        for (int i = 0; i < NSP; ++i) den[i] = 0.0;
        const double TmB = cl_exp(-NJA_B * lnT);            // T^-B, shared by every well depth
        const double rT = rsqrt(T);
        const double c = p * (rT * (rT * rT));              // 1/D_sr = c Omega dinv_sr
        for (int q = 0; q < g.neps; ++q) {
            const double ts = T * g.eps_inv[q];
            double om = NJA_A * TmB * g.eps_powB[q];
            if (NJA_D * ts < OMEGA_CUT) om += NJA_C * cl_exp(-NJA_D * ts);
            if (NJA_F * ts < OMEGA_CUT) om += NJA_E * cl_exp(-NJA_F * ts);
            if (NJA_H * ts < OMEGA_CUT) om += NJA_G * cl_exp(-NJA_H * ts);
            const double com = c * om;
            for (int pr = g.pstart[q]; pr < g.pstart[q + 1]; ++pr) {
                const int i = g.pair_i[pr], r = g.pair_r[pr];
                const double inv_d = com * g.pair_dinv[pr];
                den[i] += o.X[r] * inv_d;
                den[r] += o.X[i] * inv_d;
            }
        }
#pragma unroll
        for (int i = 0; i < NSP; ++i) {
            o.D[i] = den[i] != 0.0 ? cl_div(1.0 - o.X[i], den[i]) : 0.0;
            if (HAS_CHARGE) o.D[i] *= g.dfac[i];   // ambipolar ions, no electron coefficient
        }
    }
}

// Full closure (SI). reactions: evaluate w_s; diffusion: evaluate D_s. MIXED (device only): the
// species modal sums (electronic and vibrational parts of e_s, c_v,s, the partition-function
// factors), the forward rate exponentials, transport and diffusion in binary32; the Newton
// iteration for T, the assembly of e_s, the equilibrium constants and backward rates stay FP64.
// MODES32 (with MIXED): the split modal sums of species_state_f32. Its binary64-or-binary32
// choice per electronic level follows T, so it stays uniform across a warp where neighbouring
// cells have similar temperatures (the right-hand side); the sweep of independent states
// (hyp_thermo_eval), whose temperatures differ from lane to lane, keeps the binary64 sums.
template <bool MIXED, bool MODES32 = MIXED>
__host__ __device__ __forceinline__ void closure_si_p(const GasDev& g, double rho, double e,
                                             const double* Y, double T0, bool reactions,
                                             bool diffusion, ClosureOut& o) {
    SpeciesState s;
    o.status = rho > 0.0 ? 0u : HYP_STATUS_NONPHYSICAL;
    const double T = temperature_from_energy<MIXED && MODES32>(g, e, Y, T0, o.status, s);
    double ym = 0.0, cv = 0.0;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        ym += Y[i] * g.invM[i];
        cv += Y[i] * s.cv[i];
    }
    const double Rmix = R_U * ym;
    const double p = rho * Rmix * T;
    const double iym = cl_rcp(ym);
    o.T = T;
    o.p = p;
    o.cv = cv;
    o.Rmix = Rmix;
    o.a = sqrt(cl_div((cv + Rmix) * p, cv * rho));
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        o.h[i] = s.e[i] + g.Rs[i] * T;
        o.X[i] = Y[i] * g.invM[i] * iym;
        o.es[i] = s.e[i];
        o.cvs[i] = s.cv[i];
        o.cvps[i] = s.cvp[i];
    }
    const double lnT = cl_log(T);
    const double invT = cl_rcp(T);

    // ---- kinetics (Eqs. 14, 15) ----
    // K_c = exp(-sum_s nu_s G_s/(R T)) (p_std/(R T))^dnu with G_s/(R T) = E0_s/(R T) - ln q_s, so
    // K_c = exp(-theta_d/T) prod_s r_s^nu_s with the molar partition functions
    // r_s = A_s T^(3/2) q_rot q_vib q_el, and k_b = C T^n exp(-(T_a - theta_d)/T) / prod r_s^nu_s.
#pragma unroll
    for (int i = 0; i < NSP; ++i) o.wdot[i] = 0.0;
    if (reactions) {
        const double T15 = T * T * rsqrt(T);
        double r[NSP];
#pragma unroll
        for (int i = 0; i < NSP; ++i) {
            double q = g.A_tr[i] * T15 * s.qel[i];
            if (g.linear[i]) q *= T * g.inv_sr[i] * (1.0 + s.iem1[i]);
            r[i] = q;
        }
        double conc[NSP], molar[NSP];
#pragma unroll
        for (int i = 0; i < NSP; ++i) {
            conc[i] = rho * Y[i] * g.invM[i];
            molar[i] = 0.0;
        }
        for (int k = 0; k < g.ngroup; ++k) {
            double num = 1.0, den = 1.0, fwd = 1.0, bwd = 1.0;
#pragma unroll
            for (int i = 0; i < NSP; ++i) {
                const int nu = g.g_nu[k][i];
                for (int q = 0; q < nu; ++q) num *= r[i];
                for (int q = 0; q < -nu; ++q) den *= r[i];
                for (int q = 0; q < g.g_rf[k][i]; ++q) fwd *= conc[i];
                for (int q = 0; q < g.g_rb[k][i]; ++q) bwd *= conc[i];
            }
            // the group's reactions differ only in the collider, a species present on both sides:
            // R_group = (sum_r C_r [M_r]) (k_f prod [reactants] - k_b prod [products]) / C factors
            double w = 0.0;
            for (int rx = g.gstart[k]; rx < g.gstart[k + 1]; ++rx)
                w += g.C[rx] * (g.spec[rx] >= 0 ? conc[g.spec[rx]] : 1.0);
            const double base = g.g_n[k] * lnT;
            double Ef;
#ifdef __CUDA_ARCH__
            if (MIXED) Ef = f64_of(expf(f32_of(base - g.g_Ta[k] * invT)));
            else
#endif
                Ef = cl_exp(base - g.g_Ta[k] * invT);
            const double Eb = cl_exp(base - (g.g_Ta[k] - g.g_theta_d[k]) * invT) * cl_div(den, num);
            const double Rg = w * (Ef * fwd - Eb * bwd);
#pragma unroll
            for (int i = 0; i < NSP; ++i)
                if (g.g_nu[k][i] != 0) molar[i] += g.g_nud[k][i] * Rg;   // the group's species only
        }
#pragma unroll
        for (int i = 0; i < NSP; ++i) o.wdot[i] = g.M[i] * molar[i];
    }

    if constexpr (MIXED) {
#ifdef __CUDA_ARCH__
        transport_f32(g, T, lnT, p, s, diffusion, o);
#endif
    } else {
        transport_f64(g, T, lnT, p, s, diffusion, o);
    }
}

__host__ __device__ __forceinline__ void closure_si(const GasDev& g, double rho, double e, const double* Y,
                                           double T0, bool reactions, bool diffusion,
                                           ClosureOut& o) {
    closure_si_p<false>(g, rho, e, Y, T0, reactions, diffusion, o);
}

// ---- thermally perfect gas (HYP_GAS_TPG; Eqs. 22-25) ----
// c_p(T) = c_p0 (1 + g1 s(Theta/T)) with g1 = (gamma_inf - 1)/gamma_inf and the harmonic-oscillator
// shape s(x) = x^2 e^x / (e^x - 1)^2 (the reading of Eq. 23); its integral from 0 gives
// h(T) = c_p0 (T + g1 Theta / (e^(Theta/T) - 1)); e = h - R T with the freestream gas constant.
constexpr double TPG_THETA = 3055.0;   // K (Eq. 23)
constexpr double KEYES_C2 = 2.646e-3, KEYES_C3 = 245.4, KEYES_C4 = 12.0;   // Eq. (25), SI

__host__ __device__ __forceinline__ double tpg_shape(double x) {
    const double d = -expm1(-x);
    return x * x * exp(-x) / (d * d);
}

__host__ __device__ __forceinline__ double keyes(double T) {
    return KEYES_C2 * sqrt(T) / (1.0 + (KEYES_C3 / T) * exp(-KEYES_C4 * 2.302585092994045684 / T));
}

struct TpgModel {
    double cp0, g1, theta, R;
    __host__ __device__ double cp(double T) const { return cp0 * (1.0 + g1 * tpg_shape(theta / T)); }
    __host__ __device__ double energy(double T) const {
        const double x = theta / T;
        return cp0 * (T + g1 * theta * exp(-x) / -expm1(-x)) - R * T;
    }
    // Newton on e(T) = e (de/dT = c_p - R > 0), from T0; T in K.
    __host__ __device__ double temperature(double e, double T0, unsigned& status) const {
        double T = fmin(fmax(T0, T_LO), T_HI);
        for (int it = 0; it < NEWTON_MAXIT; ++it) {
            const double dT = (energy(T) - e) / (cp(T) - R);
            T -= dT;
            if (!(T > T_LO)) {
                T = T_LO;
                status |= HYP_STATUS_T_CLAMPED;
                return T;
            }
            if (fabs(dT) <= 1e-14 * T) return T;
        }
        status |= HYP_STATUS_NOT_CONVERGED;
        return T;
    }
};

// ---- Stefan-Maxwell diffusion (Eq. 17) at one face ----
// Flux form of the Stefan-Maxwell relations, regular for vanishing mole fractions:
//     sum_{i != s} (X_s J_i / M_i - X_i J_s / M_s) / D_si = (rho / Mbar) grad X_s,  s >= 1,
// with the first (omitted, most abundant) species' equation replaced by sum_s J_s = 0, solved by
// Gaussian elimination with partial pivoting (5 x 5, in registers). Tsi, psi: SI temperature and
// pressure for the binary coefficients (Chapman-Enskog, the collision-integral fit of the
// closure); dscale converts 1/D_si (SI) to the nondimensional 1/(D_si rho_inf / (mu_inf Re)).
// rho, dX and the returned J are nondimensional.
__device__ __forceinline__ void stefan_maxwell_face(const GasDev& g, double Tsi, double psi, double dscale,
                                           double rho, const double* Yf, const double* dX,
                                           double* J) {
    double inv[NSP], X[NSP], ym = 0.0;
#pragma unroll
    for (int s = 0; s < NSP; ++s) {
        inv[s] = Yf[s] * g.invM[s];
        ym += inv[s];
    }
    const double Mbar = 1.0 / ym;
#pragma unroll
    for (int s = 0; s < NSP; ++s) X[s] = inv[s] * Mbar;
    double a[NSP][NSP], b[NSP];
#pragma unroll
    for (int r = 0; r < NSP; ++r) {
#pragma unroll
        for (int c = 0; c < NSP; ++c) a[r][c] = 0.0;
        b[r] = r == 0 ? 0.0 : rho * ym * dX[r];
    }
    const double lnT = cl_log(Tsi);
    const double TmB = cl_exp(-NJA_B * lnT);
    const double cc = psi / (Tsi * sqrt(Tsi)) * dscale;
    for (int q = 0; q < g.neps; ++q) {
        const double ts = Tsi * g.eps_inv[q];
        double om = NJA_A * TmB * g.eps_powB[q];
        if (NJA_D * ts < OMEGA_CUT) om += NJA_C * cl_exp(-NJA_D * ts);
        if (NJA_F * ts < OMEGA_CUT) om += NJA_E * cl_exp(-NJA_F * ts);
        if (NJA_H * ts < OMEGA_CUT) om += NJA_G * cl_exp(-NJA_H * ts);
        for (int pr = g.pstart[q]; pr < g.pstart[q + 1]; ++pr) {
            const int i = g.pair_i[pr], r = g.pair_r[pr];
            const double w = cc * om * g.pair_dinv[pr];          // nondimensional 1 / D_ir
#pragma unroll
            for (int s = 1; s < NSP; ++s) {
                if (s == i) {
                    a[s][r] += X[i] * w * g.invM[r];
                    a[s][s] -= X[r] * w * g.invM[i];
                }
                if (s == r) {
                    a[s][i] += X[r] * w * g.invM[i];
                    a[s][s] -= X[i] * w * g.invM[r];
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < NSP; ++c) a[0][c] = 1.0;
    // elimination with partial pivoting (all indices static after unrolling)
#pragma unroll
    for (int k = 0; k < NSP; ++k) {
        int p = k;
        double best = fabs(a[k][k]);
#pragma unroll
        for (int r = k + 1; r < NSP; ++r) {
            if (fabs(a[r][k]) > best) {
                best = fabs(a[r][k]);
                p = r;
            }
        }
#pragma unroll
        for (int r = k + 1; r < NSP; ++r) {
            if (r == p) {
#pragma unroll
                for (int c = 0; c < NSP; ++c) {
                    const double t = a[k][c];
                    a[k][c] = a[r][c];
                    a[r][c] = t;
                }
                const double t = b[k];
                b[k] = b[r];
                b[r] = t;
            }
        }
        const double ip = 1.0 / a[k][k];
#pragma unroll
        for (int r = k + 1; r < NSP; ++r) {
            const double f = a[r][k] * ip;
#pragma unroll
            for (int c = k + 1; c < NSP; ++c) a[r][c] -= f * a[k][c];
            b[r] -= f * b[k];
        }
    }
#pragma unroll
    for (int k = NSP - 1; k >= 0; --k) {
        double t = b[k];
#pragma unroll
        for (int c = k + 1; c < NSP; ++c) t -= a[k][c] * J[c];
        J[k] = t / a[k][k];
    }
}

// ---- local thermodynamic equilibrium (HYP_GAS_LTE; Sec. 2.2.2, special cases) ----
// The composition is the one of minimum Gibbs energy for the element content of the air. At that
// minimum the chemical potential of each species is the sum of its atoms' element potentials
// lambda_e (units of R T); with the molar partition function r_s of the closure (translation per
// unit volume, rotation, vibration, electronic levels) and the ground-state energy R theta0_s,
// the ideal-gas chemical potential gives
//     c_s = exp(a_s . lambda - gam_s),   gam_s = theta0_s / T - ln r_s        (mol/m^3),
// and lambda follows from the element totals sum_s a_es c_s = b_e (Newton on ln of the sums).
constexpr int EQ_MAXIT = 100;
constexpr double EQ_TOL = 1.0e-11;        // element-potential step that ends the iteration
constexpr double EQ_MAX_STEP = 25.0;      // largest change of an element potential in one step

__host__ __device__ __forceinline__ void lte_gammas(const GasDev& g, double T, double lnT,
                                           const SpeciesState& s, double* gam) {
    const double invT = 1.0 / T;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        double lr = g.lnA_tr[i] + 1.5 * lnT + log(s.qel[i]);
        if (g.linear[i]) lr += lnT + g.ln_isr[i] + log1p(s.iem1[i]);
        gam[i] = g.theta0[i] * invT - lr;
    }
}

// Element potentials for element totals b (mol/m^3, lnb = ln b). warm: start from lam; else from
// the smallest value at which one species made of that element alone would hold all of it (an
// upper bound of the solution). c receives the concentrations at the returned lam.
__host__ __device__ __forceinline__ bool lte_solve(const GasDev& g, const double* gam, const double* b,
                                          const double* lnb, bool warm, double* lam, double* c) {
    if (!warm) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            double best = HUGE_VAL;
#pragma unroll
            for (int i = 0; i < NSP; ++i) {
                const double a = g.atoms[i][e], o = g.atoms[i][1 - e];
                if (a > 0.0 && o == 0.0) best = fmin(best, (lnb[e] - log(a) + gam[i]) / a);
            }
            lam[e] = best;
        }
    }
    for (int it = 0; it < EQ_MAXIT; ++it) {
        double S0 = 0.0, S1 = 0.0, J00 = 0.0, J01 = 0.0, J11 = 0.0;
#pragma unroll
        for (int i = 0; i < NSP; ++i) {
            const double a0 = g.atoms[i][0], a1 = g.atoms[i][1];
            const double ci = cl_exp(a0 * lam[0] + a1 * lam[1] - gam[i]);
            S0 += a0 * ci;
            S1 += a1 * ci;
            J00 += a0 * a0 * ci;
            J01 += a0 * a1 * ci;
            J11 += a1 * a1 * ci;
        }
        // rows of the Jacobian of ln S_e: (sum_s a_es a_js c_s) / S_e
        const double F0 = log(S0) - lnb[0], F1 = log(S1) - lnb[1];
        const double j00 = J00 / S0, j01 = J01 / S0, j10 = J01 / S1, j11 = J11 / S1;
        const double idet = 1.0 / (j00 * j11 - j01 * j10);
        double d0 = -(F0 * j11 - F1 * j01) * idet;
        double d1 = -(F1 * j00 - F0 * j10) * idet;
        d0 = fmin(fmax(d0, -EQ_MAX_STEP), EQ_MAX_STEP);
        d1 = fmin(fmax(d1, -EQ_MAX_STEP), EQ_MAX_STEP);
        lam[0] += d0;
        lam[1] += d1;
        if (fmax(fabs(d0), fabs(d1)) <= EQ_TOL) {
#pragma unroll
            for (int i = 0; i < NSP; ++i)
                c[i] = cl_exp(g.atoms[i][0] * lam[0] + g.atoms[i][1] * lam[1] - gam[i]);
            return true;
        }
    }
#pragma unroll
    for (int i = 0; i < NSP; ++i) c[i] = cl_exp(g.atoms[i][0] * lam[0] + g.atoms[i][1] * lam[1] - gam[i]);
    return false;
}

// Equilibrium at (T, rho): species state, concentrations and the temperature derivatives along
// the equilibrium at fixed density, d ln c_s/dT = a_s . lambda'_rho + eps_s with eps_s =
// E_s / (R T^2) (E_s the molar internal energy) and sum_s a_es c_s d ln c_s/dT = 0.
struct LteState {
    SpeciesState s;
    double c[NSP];       // mol/m^3
    double lam[2];
    double eps[NSP];     // E_s / (R T^2)
    double dlnc[NSP];    // d ln c_s / dT at fixed density
    double H[3];         // sum_s c_s a_s a_s^T: (0,0), (0,1), (1,1)
    double e, cv_eq;     // J/kg, de/dT at fixed density
    bool ok;
};

__host__ __device__ __forceinline__ void lte_at(const GasDev& g, double T, double rho, const double* b,
                                       const double* lnb, bool warm, LteState& q) {
    species_state(g, T, q.s);
    // CUDA's log in the equilibrium closure: its element-potential solve carries the rounding of
    // ln q into the composition, and the table-driven log moved the stepped LTE parity check from
    // 0.73 to 1.04 of its bound (a different rounding, not a larger error)
    const double lnT = log(T);
    double gam[NSP];
    lte_gammas(g, T, lnT, q.s, gam);
    q.ok = lte_solve(g, gam, b, lnb, warm, q.lam, q.c);
    const double iRT2 = 1.0 / (R_U * T * T);
    double H00 = 0.0, H01 = 0.0, H11 = 0.0, r0 = 0.0, r1 = 0.0;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        const double a0 = g.atoms[i][0], a1 = g.atoms[i][1], ci = q.c[i];
        q.eps[i] = g.M[i] * q.s.e[i] * iRT2;
        H00 += a0 * a0 * ci;
        H01 += a0 * a1 * ci;
        H11 += a1 * a1 * ci;
        r0 -= a0 * ci * q.eps[i];
        r1 -= a1 * ci * q.eps[i];
    }
    q.H[0] = H00;
    q.H[1] = H01;
    q.H[2] = H11;
    const double idet = 1.0 / (H00 * H11 - H01 * H01);
    const double l0 = (r0 * H11 - r1 * H01) * idet, l1 = (r1 * H00 - r0 * H01) * idet;
    double ce = 0.0, ccv = 0.0, cedl = 0.0;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        q.dlnc[i] = g.atoms[i][0] * l0 + g.atoms[i][1] * l1 + q.eps[i];
        const double Ei = g.M[i] * q.s.e[i];
        ce += q.c[i] * Ei;
        ccv += q.c[i] * g.M[i] * q.s.cv[i];
        cedl += q.c[i] * Ei * q.dlnc[i];
    }
    const double irho = 1.0 / rho;
    q.e = ce * irho;
    q.cv_eq = (ccv + cedl) * irho;
}

// Closure in local thermodynamic equilibrium at (rho, e) (SI), from the temperature T0. T from
// the safeguarded Newton iteration of temperature_from_energy on the equilibrium energy at fixed
// density, which also bisects when the iteration does not contract; then the equilibrium composition at T, p = rho R_mix T, the frozen transport of that
// composition and the equilibrium conductivity k = k_frozen + k_reactive,
//     k_reactive = (rho / M_mix) sum_s M_s D_s (dX_s/dT)_p (h_s - h),   h = sum_s Y_s h_s,
// the heat carried by the algebraic diffusion of Eq. (18) when the mole fractions follow the
// equilibrium at the local pressure. (dX_s/dT)_p: at fixed pressure the element totals scale by
// a common factor s' (d ln c_s/dT = d ln c_s/dT|_rho + s' a_s . H^-1 b) fixed by
// sum_s c_s d ln c_s/dT = -c_tot / T; X_s' = X_s (d ln c_s/dT + 1/T). Yout receives the mass
// fractions, o.X the mole fractions, o.D the averaged diffusion coefficients of the composition,
// o.k the equilibrium conductivity; o.h and o.wdot are zero. lam (nullable, two values): the
// element potentials of an earlier evaluation near this state, where the first solve starts when
// they are finite (otherwise from the bound above); on return the potentials at the result.
// cv_eq (nullable) receives de/dT along the equilibrium at fixed density at the result.
template <bool MIXED>
__host__ __device__ __forceinline__ void lte_closure(const GasDev& g, double rho, double e, double T0,
                                            double* Yout, double& k_reactive, ClosureOut& o,
                                            double* lam = nullptr, double* cv_eq = nullptr) {
    o.status = rho > 0.0 ? 0u : HYP_STATUS_NONPHYSICAL;
    const double b[2] = {rho * g.elem_b[0], rho * g.elem_b[1]};
    const double lnb[2] = {log(b[0]), log(b[1])};
    LteState q;
    double T = fmin(fmax(T0, T_LO), T_HI);
    double lo = T_LO, hi = T_HI, dx_old = T_HI - T_LO;
    bool warm = false, conv = false;
    if (lam && isfinite(lam[0]) && isfinite(lam[1])) {
        q.lam[0] = lam[0];
        q.lam[1] = lam[1];
        warm = true;
    }
    for (int it = 0; it < NEWTON_MAXIT; ++it) {
        lte_at(g, T, rho, b, lnb, warm, q);
        warm = true;
        if (!q.ok) o.status |= HYP_STATUS_NOT_CONVERGED;
        const double f = q.e - e;
        if (f > 0.0) hi = T; else lo = T;
        double Tn = T - f / q.cv_eq;
        if (fabs(Tn - T) <= NEWTON_RTOL * T) {
            T = Tn;
            conv = true;
            break;
        }
        // e_eq(T) is S-shaped (c_v,eq peaks where a molecule dissociates): bisect when the step
        // leaves the bracket or the iteration does not contract, |f| > |dx_old c_v,eq| / 2
        if (!(Tn > lo && Tn < hi) || fabs(2.0 * f) > fabs(dx_old * q.cv_eq)) Tn = 0.5 * (lo + hi);
        dx_old = fabs(Tn - T);
        T = Tn;
    }
    if (!conv) {
        LteState qe;
        lte_at(g, T_LO, rho, b, lnb, false, qe);
        if (e <= qe.e) {
            T = T_LO;
            o.status |= HYP_STATUS_T_CLAMPED;
        } else {
            lte_at(g, T_HI, rho, b, lnb, false, qe);
            if (e >= qe.e) {
                T = T_HI;
                o.status |= HYP_STATUS_T_CLAMPED;
            } else {
                o.status |= HYP_STATUS_NOT_CONVERGED;
            }
        }
        warm = false;
    }
    lte_at(g, T, rho, b, lnb, warm, q);
    if (!q.ok) o.status |= HYP_STATUS_NOT_CONVERGED;

    double ctot = 0.0, cv = 0.0;
#pragma unroll
    for (int i = 0; i < NSP; ++i) ctot += q.c[i];
    const double irho = 1.0 / rho, ict = 1.0 / ctot;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        Yout[i] = q.c[i] * g.M[i] * irho;
        o.X[i] = q.c[i] * ict;
        cv += Yout[i] * q.s.cv[i];
        o.h[i] = 0.0;
        o.wdot[i] = 0.0;
        o.es[i] = q.s.e[i];
        o.cvs[i] = q.s.cv[i];
        o.cvps[i] = q.s.cvp[i];
    }
    const double Rmix = R_U * ctot * irho;
    const double p = rho * Rmix * T;
    o.T = T;
    o.p = p;
    o.cv = cv;
    o.Rmix = Rmix;
    o.a = sqrt((cv + Rmix) / cv * p * irho);
    const double lnT = log(T);
    if constexpr (MIXED) {
#ifdef __CUDA_ARCH__
        transport_f32(g, T, lnT, p, q.s, true, o);
#endif
    } else {
        transport_f64(g, T, lnT, p, q.s, true, o);
    }

    // (dX_s/dT)_p with u = H^-1 b
    const double idet = 1.0 / (q.H[0] * q.H[2] - q.H[1] * q.H[1]);
    const double u0 = (b[0] * q.H[2] - b[1] * q.H[1]) * idet;
    const double u1 = (b[1] * q.H[0] - b[0] * q.H[1]) * idet;
    double cdl = 0.0;
#pragma unroll
    for (int i = 0; i < NSP; ++i) cdl += q.c[i] * q.dlnc[i];
    const double sp = (-ctot / T - cdl) / (b[0] * u0 + b[1] * u1);
    double h = 0.0;
    double hs[NSP];
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        hs[i] = q.s.e[i] + g.Rs[i] * T;
        h += Yout[i] * hs[i];
    }
    double kr = 0.0;
    const double invT = 1.0 / T;
#pragma unroll
    for (int i = 0; i < NSP; ++i) {
        const double dlp = q.dlnc[i] + sp * (g.atoms[i][0] * u0 + g.atoms[i][1] * u1);
        const double dX = o.X[i] * (dlp + invT);
        kr += g.M[i] * o.D[i] * dX * (hs[i] - h);
    }
    k_reactive = ctot * kr;
    o.k += k_reactive;
    if (lam) {
        lam[0] = q.lam[0];
        lam[1] = q.lam[1];
    }
    if (cv_eq) *cv_eq = q.cv_eq;
}

}  // namespace hyp
