// Internal declarations of the GB300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/hyp.h"

// Species count the kernels are compiled for: the library is built once for five-species air
// (libhyp.so) and once for eleven-species air with ions and electrons (libhyp11.so).
#ifndef HYP_NSP
#define HYP_NSP 5
#endif
#define NSP HYP_NSP
#define MAXR 64                // elementary reactions
#define MAXG 24                // reaction groups sharing (n, T_a, net stoichiometry)
#define MAXLEV 6               // electronic levels per species
#define MAXEPS 16              // distinct Lennard-Jones well depths of species pairs
#define ETAB_N 64              // temperatures of the species-energy table (start of the T inversion)
#define LINE_BLOCK 128         // threads per block of the line-operator kernel

namespace hyp {

static_assert(NSP <= HYP_MAX_SPECIES, "species count above the C ABI's capacity");
// Only the eleven-species build accepts charged species (ions, the electron): in the five-species
// build the mixing rules, diffusion and fluxes compile without the charge handling.
constexpr bool HAS_CHARGE = NSP > 5;

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t err, const char* what);

#define HYP_CUDA(call)                                         \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) return ::hyp::cuda_fail(_e, #call); \
    } while (0)

// Gas model as seen by the kernels: a plain struct passed by value as a kernel parameter.
struct GasDev {
    int kind;                    // hyp_gas_kind
    int nr, ngroup, neps, npair;
    // species thermodynamics (rigid rotor / harmonic oscillator, Sec. 2.2.1)
    double M[NSP], invM[NSP], Rs[NSP];
    double e0[NSP];              // (hf298 - H_sens(298.15)) / M, J/kg: internal energy at 0 K
    int linear[NSP];
    double theta_v[NSP];
    int nlev[NSP];               // electronic levels, ascending theta (ground level first)
    double lev_g[NSP][MAXLEV], lev_th[NSP][MAXLEV];
    double A_tr[NSP];            // (2 pi m k / h^2)^(3/2) / N_A: molar translational factor
    double inv_sr[NSP];          // 1 / (sigma theta_r) for linear molecules
    // transport
    double blA[NSP], blB[NSP], blC[NSP];
    double Mq[NSP], iMq[NSP];    // M_s^(1/4) and its reciprocal (Wilke's rule)
    double wilke_d[NSP][NSP];    // 1 / sqrt(8 (1 + M_s / M_r))
    // unordered species pairs grouped by their Lennard-Jones well depth
    int pstart[MAXEPS + 1];
    int pair_i[NSP * (NSP - 1) / 2], pair_r[NSP * (NSP - 1) / 2];
    double pair_dinv[NSP * (NSP - 1) / 2];   // pi sigma^2 / ((3/16) sqrt(2 pi k^3 / m_sr))
    double eps_inv[MAXEPS];      // 1 / sqrt(eps_s eps_r)
    double eps_powB[MAXEPS];     // sqrt(eps_s eps_r)^B of the collision-integral fit
    // binary32 copies of the transport constants for the mixed-precision closure (HYP_MIXED)
    float f_blA[NSP], f_blB[NSP], f_blC[NSP], f_Mq[NSP], f_iMq[NSP], f_Rs[NSP];
    float f_wilke_d[NSP][NSP];
    float f_pair_dinv[NSP * (NSP - 1) / 2];
    float f_eps_inv[MAXEPS], f_eps_powB[MAXEPS];
    // species energies e_s and heat capacities c_v,s (J/kg, J/(kg K)) at ETAB_N temperatures
    // spaced evenly in ln T from 50 K to 1e5 K: a starting temperature for the inversion when no
    // earlier temperature is known. A device array [e | c_v][species][ETAB_N] in global memory
    // (the bisection reads it at a different temperature in every lane, which the constant cache
    // would serialise); null until an evaluation that needs it (hyp_thermo_eval, hyp_lte_eval).
    double etab_lnT0, etab_dlnT;
    const double* etab;
    // kinetics (Eqs. 13-15): elementary reactions with explicit colliders, sorted by group
    int gstart[MAXG + 1];        // reactions of group k: [gstart[k], gstart[k+1])
    double C[MAXR];              // SI pre-exponential factor
    int spec[MAXR];              // species on both sides of the reaction (collider), -1 if none
    signed char g_rf[MAXG][NSP], g_rb[MAXG][NSP];   // group reactants / products without collider
    double g_n[MAXG], g_Ta[MAXG];
    double g_theta_d[MAXG];      // sum_s nu_s E0_s / R_u (K): 0 K reaction energy of the group
    signed char g_nu[MAXG][NSP]; // net stoichiometry nu'' - nu' of the group
    double g_nud[MAXG][NSP];     // the same, as doubles
    // nondimensionalisation (Eqs. 7, 11)
    double rho_inf, a_inf, T_inf, p_inf, mu_inf, k_inf, cp_inf, gamma_inf, R_inf, T_ref, L_ref,
        Re, Pr;
    double prandtl_cpg;
    double mach;
    double Y_inf[NSP];
    double tpg_cp0, tpg_theta;   // thermally perfect gas (Eq. 23): c_p0 (J/(kg K)) and Theta (K)
    // local thermodynamic equilibrium (HYP_GAS_LTE): atoms of N and O per particle, element
    // content of the freestream air (mol/kg), and the partition-function constants of
    // c_s = exp(a_s . lambda - theta0_s / T + ln r_s)
    // charged species (eleven-species build): charge per species, 1 for the species in the mixing
    // rules and binary pairs (all but the electron), the factor on the averaged diffusion
    // coefficient (2: ambipolar ions, 1 neutrals, 0 the electron), the electron's index or -1
    int charge[NSP], heavy[NSP];
    double dfac[NSP];
    int ie;
    double atoms[NSP][2];
    double elem_b[2];
    double lnA_tr[NSP];          // ln A_tr
    double ln_isr[NSP];          // ln(1 / (sigma theta_r)) for linear molecules
    double theta0[NSP];          // E0_s / R_u (K): ground-state energy incl. formation
    double e_lo[NSP], e_hi[NSP]; // species energies at the ends of the inversion's range
};

}  // namespace hyp

struct hyp_gas {
    hyp::GasDev dev;
    std::vector<std::string> names;
    std::vector<double> etab_host;   // the table behind GasDev::etab
    double* etab_dev = nullptr;      // its device copy, made on first use (gas.cu)
    std::mutex etab_mu;
};

namespace hyp {

// One compact line operator (Sec. 3.1): tridiagonal left-hand side with precomputed Thomas
// factors, interior right-hand-side weights and explicit closure rows.
struct LineOp {
    int m, n_in;                 // output and input points along the line
    int dir;                     // 0 centre->face, 1 face->centre
    int kind;                    // 0 interpolation, 1 first derivative
    int wall;                    // 1: known value at position 0 enters the closure rows
    int first_interior, last_interior;
    double wi[4];                // interior weights on inputs at offsets -3/2, -1/2, +1/2, +3/2
    const double* lower;         // device: sub-diagonal of each row
    const double* cprime;        // device: Thomas c'
    const double* minv;          // device: Thomas 1 / pivot
    const double* wa;            // device, interior rows: weight of (f_{+1/2} +/- f_{-1/2}) / pivot
    const double* wb;            // device, interior rows: weight of (f_{+3/2} +/- f_{-3/2}) / pivot
    const double* lm;            // device: sub-diagonal / pivot
    // Interior rows rc..last_interior have bitwise-constant factors (the Thomas recurrence of the
    // Toeplitz interior reaches its fixed point within about 20 rows): wa, wb, lm, cprime there.
    int rc;
    double wac, wbc, lmc, cpc;
    float wac_f, wbc_f, lmc_f, cpc_f;   // the same in binary32 (HYP_MIXED jobs)
    float wac_l, wbc_l, lmc_l, cpc_l;   // their remainders: (x_f, x_l) is x as a double word
    int ncl;                     // closure rows (<= 4)
    int crow[4], cstart[4], cnum[4];
    double cw[4][5];
    double gw[4];                // weight of the wall value
};

struct LineJob {
    const LineOp* op;            // device pointer
    const double* in;            // input field, or an element offset into the state when in_state
    int in_state;
    double* out;
    double* tmp;                 // forward-sweep storage, same layout as out, distinct from it
    long long in_ls, in_es, out_ls, out_es;
    int nlines;
    int nseg;                    // segments per line (power of two dividing the block size)
    double wall_value;
    double scale;                // +1 or -1
    const double* metric;        // per output element along the line, nullable
    const float* metric_f;       // binary32 copy of metric (HYP_MIXED jobs)
    int f32ok;                   // under HYP_MIXED the constant-factor rows may run in binary32
    // three-dimensional grids: lines grouped by plane, line L starting at
    // (L / lpp) * plane stride + (L % lpp) * line stride (lpp = 0: one group)
    int lpp;
    long long in_ps, out_ps;
    const double* wall_arr;      // per-line wall values (line index), replacing wall_value
};

cudaError_t launch_lines(const LineJob* d_jobs, int njobs, int max_blocks, const double* U,
                         cudaStream_t s, int mixed = 0);

}  // namespace hyp
