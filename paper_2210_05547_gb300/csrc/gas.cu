// Gas model loading (Sec. 2.2 closure data) and the pointwise thermochemistry kernels.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"
#include "thermo.cuh"

namespace hyp {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t err, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(err);
    return err == cudaErrorMemoryAllocation ? HYP_ERR_OOM : HYP_ERR_CUDA;
}

namespace table {

constexpr double K_B = 1.380649e-23;
constexpr double N_A = 6.02214076e23;
constexpr double H_P = 6.62607015e-34;
constexpr double PI = 3.14159265358979323846;

struct SpeciesRow {
    std::string name;
    double M, hf, theta_v, theta_r, sym, bA, bB, bC, lj_s, lj_e;
    int linear, nN, nO, charge = 0;
    std::vector<std::pair<double, double>> levels;
};

struct ReactionRow {
    double C_cgs, n, Ta;
    std::vector<std::string> lhs, rhs;
};

int parse_table(const char* path, std::vector<SpeciesRow>& sp, std::vector<ReactionRow>& rx) {
    std::ifstream in(path);
    if (!in) return fail(HYP_ERR_IO, std::string("cannot open gas table ") + path);
    std::string line;
    while (std::getline(in, line)) {
        auto hash = line.find('#');
        if (hash != std::string::npos) line = line.substr(0, hash);
        std::istringstream ss(line);
        std::string key;
        if (!(ss >> key)) continue;
        if (key == "SPECIES") {
            SpeciesRow r;
            if (!(ss >> r.name >> r.M >> r.hf >> r.linear >> r.theta_v >> r.theta_r >> r.sym >>
                  r.bA >> r.bB >> r.bC >> r.lj_s >> r.lj_e >> r.nN >> r.nO))
                return fail(HYP_ERR_IO, "bad SPECIES line: " + line);
            int ch;
            if (ss >> ch) r.charge = ch;              // optional last column
            sp.push_back(r);
        } else if (key == "LEVEL") {
            std::string name;
            double gdeg, th;
            if (!(ss >> name >> gdeg >> th)) return fail(HYP_ERR_IO, "bad LEVEL line: " + line);
            bool found = false;
            for (auto& r : sp)
                if (r.name == name) {
                    r.levels.push_back({gdeg, th});
                    found = true;
                }
            if (!found) return fail(HYP_ERR_IO, "LEVEL for unknown species " + name);
        } else if (key == "REACTION") {
            ReactionRow r;
            std::string colon, tok;
            if (!(ss >> r.C_cgs >> r.n >> r.Ta >> colon) || colon != ":")
                return fail(HYP_ERR_IO, "bad REACTION line: " + line);
            bool right = false;
            while (ss >> tok) {
                if (tok == "=>") {
                    right = true;
                    continue;
                }
                (right ? r.rhs : r.lhs).push_back(tok);
            }
            if (!right || r.lhs.empty() || r.rhs.empty())
                return fail(HYP_ERR_IO, "bad REACTION line: " + line);
            rx.push_back(r);
        } else {
            return fail(HYP_ERR_IO, "unknown keyword " + key);
        }
    }
    return HYP_OK;
}

// Sensible molar enthalpy / R_u from 0 K (used once, at 298.15 K, for the formation offset).
double h_sens_over_r(const SpeciesRow& r, double T) {
    double q = 0.0, m1 = 0.0;
    for (auto& l : r.levels) {
        double w = l.first * exp(-l.second / T);
        q += w;
        m1 += w * l.second;
    }
    double h = 2.5 * T + m1 / q;
    if (r.linear) h += T + r.theta_v / expm1(r.theta_v / T);
    return h;
}

}  // namespace table
}  // namespace hyp

using namespace hyp;
using namespace hyp::table;

extern "C" int hyp_gas_model_load(const char* path, int kind, const hyp_freestream* fs,
                                  hyp_gas** out) {
    if (!path || !fs || !out) return fail(HYP_ERR_ARG, "null argument");
    if (kind < HYP_GAS_CNEQ || kind > HYP_GAS_LTE) return fail(HYP_ERR_ARG, "unknown gas kind");
    std::vector<SpeciesRow> sp;
    std::vector<ReactionRow> rx;
    int rc = parse_table(path, sp, rx);
    if (rc) return rc;
    if ((int)sp.size() != NSP)
        return fail(HYP_ERR_IO, "gas table must list " + std::to_string(NSP) +
                                    " species (the species count this library is built for)");
    if ((int)rx.size() > MAXR) return fail(HYP_ERR_IO, "too many reactions");
    hyp_gas* g = new hyp_gas();
    GasDev& d = g->dev;
    memset(&d, 0, sizeof(d));
    d.kind = kind;
    for (int i = 0; i < NSP; ++i) {
        const SpeciesRow& r = sp[i];
        g->names.push_back(r.name);
        if ((int)r.levels.size() > MAXLEV || r.levels.empty()) {
            delete g;
            return fail(HYP_ERR_IO, "species " + r.name + ": 1 to 6 electronic levels required");
        }
        d.M[i] = r.M;
        d.invM[i] = 1.0 / r.M;
        d.Rs[i] = R_U / r.M;
        d.e0[i] = (r.hf - R_U * h_sens_over_r(r, 298.15)) / r.M;
        d.linear[i] = r.linear;
        d.theta_v[i] = r.theta_v;
        std::vector<std::pair<double, double>> lev = r.levels;   // (g, theta), ascending theta
        std::stable_sort(lev.begin(), lev.end(),
                         [](const std::pair<double, double>& a, const std::pair<double, double>& b) {
                             return a.second < b.second;
                         });
        d.nlev[i] = (int)lev.size();
        for (size_t l = 0; l < lev.size(); ++l) {
            d.lev_g[i][l] = lev[l].first;
            d.lev_th[i][l] = lev[l].second;
        }
        const double m = r.M / N_A;
        d.A_tr[i] = pow(2.0 * PI * m * K_B / (H_P * H_P), 1.5) / N_A;
        d.inv_sr[i] = r.linear ? 1.0 / (r.sym * r.theta_r) : 0.0;
        d.lnA_tr[i] = log(d.A_tr[i]);
        d.ln_isr[i] = r.linear ? -log(r.sym * r.theta_r) : 0.0;
        d.theta0[i] = r.hf / R_U - h_sens_over_r(r, 298.15);
        d.atoms[i][0] = r.nN;
        d.atoms[i][1] = r.nO;
        d.charge[i] = r.charge;
        d.heavy[i] = r.charge >= 0;
        d.dfac[i] = r.charge > 0 ? 2.0 : (r.charge < 0 ? 0.0 : 1.0);
        d.blA[i] = r.bA;
        d.blB[i] = r.bB;
        d.blC[i] = r.bC;
    }
    d.ie = -1;
    for (int i = 0; i < NSP; ++i) {
        if (sp[i].charge != 0 && !HAS_CHARGE) {
            delete g;
            return fail(HYP_ERR_IO, "charged species need the eleven-species build (libhyp11)");
        }
        if (sp[i].charge < 0) {
            if (d.ie >= 0 || sp[i].charge != -1 || i == 0) {
                delete g;
                return fail(HYP_ERR_IO, "one electron species (charge -1, not the first) at most");
            }
            d.ie = i;
        }
        if (sp[i].charge > 1) {
            delete g;
            return fail(HYP_ERR_IO, "ions must be singly charged");
        }
    }
    bool charged = false;
    for (int i = 0; i < NSP; ++i) charged = charged || sp[i].charge != 0;
    if (kind == HYP_GAS_LTE && charged) {
        delete g;
        return fail(HYP_ERR_ARG, "LTE conserves N and O only: no charged species");
    }
    for (int i = 0; i < NSP; ++i)
        for (int j = 0; j < NSP; ++j) {
            d.Mq[i] = pow(sp[i].M, 0.25);
            d.iMq[i] = 1.0 / d.Mq[i];
            d.wilke_d[i][j] = 1.0 / sqrt(8.0 * (1.0 + sp[i].M / sp[j].M));
        }
    // unordered pairs grouped by well depth: one collision integral per distinct depth
    {
        std::vector<double> eps_list;
        std::vector<std::vector<int>> members;
        for (int i = 0; i < NSP; ++i)
            for (int j = i + 1; j < NSP; ++j) {
                if (!d.heavy[i] || !d.heavy[j]) continue;     // no binary pairs with the electron
                const double eps = sp[i].lj_e * sp[j].lj_e;
                int q = -1;
                for (size_t k = 0; k < eps_list.size(); ++k)
                    if (eps_list[k] == eps) q = (int)k;
                if (q < 0) {
                    if ((int)eps_list.size() == MAXEPS) {
                        delete g;
                        return fail(HYP_ERR_IO, "too many distinct well depths");
                    }
                    eps_list.push_back(eps);
                    members.emplace_back();
                    q = (int)eps_list.size() - 1;
                }
                members[q].push_back(i * NSP + j);
            }
        d.neps = (int)eps_list.size();
        int np = 0;
        for (int q = 0; q < d.neps; ++q) {
            d.pstart[q] = np;
            d.eps_inv[q] = 1.0 / sqrt(eps_list[q]);
            d.eps_powB[q] = pow(sqrt(eps_list[q]), 0.15610);
            for (int code : members[q]) {
                const int i = code / NSP, j = code % NSP;
                const SpeciesRow &a = sp[i], &b = sp[j];
                const double m_sr = (a.M * b.M / (a.M + b.M)) / N_A;
                const double sig = 0.5 * (a.lj_s + b.lj_s) * 1.0e-10;
                d.pair_i[np] = i;
                d.pair_r[np] = j;
                d.pair_dinv[np] = PI * sig * sig / (3.0 / 16.0 * sqrt(2.0 * PI * K_B * K_B * K_B / m_sr));
                ++np;
            }
        }
        d.pstart[d.neps] = np;
        d.npair = np;
    }
    // reactions, grouped by (n, T_a, net stoichiometry): one k_f exponential and one K_c per group;
    // stored sorted by group
    {
        const int nr = (int)rx.size();
        std::vector<int> grp(nr), order_f(nr * NSP, 0), order_b(nr * NSP, 0);
        std::vector<double> Cs(nr);
        for (int r = 0; r < nr; ++r) {
            int order = 0;
            for (int side = 0; side < 2; ++side)
                for (auto& nm : side == 0 ? rx[r].lhs : rx[r].rhs) {
                    int idx = -1;
                    for (int i = 0; i < NSP; ++i)
                        if (sp[i].name == nm) idx = i;
                    if (idx < 0) {
                        delete g;
                        return fail(HYP_ERR_IO, "reaction uses unknown species " + nm);
                    }
                    (side == 0 ? order_f : order_b)[r * NSP + idx] += 1;
                    if (side == 0) ++order;
                }
            Cs[r] = rx[r].C_cgs * pow(1.0e-6, order - 1);
            int k = -1;
            for (int q = 0; q < d.ngroup; ++q) {
                bool same = d.g_n[q] == rx[r].n && d.g_Ta[q] == rx[r].Ta;
                for (int i = 0; i < NSP; ++i)
                    same = same && d.g_nu[q][i] == order_b[r * NSP + i] - order_f[r * NSP + i];
                if (same) k = q;
            }
            if (k < 0) {
                if (d.ngroup == MAXG) {
                    delete g;
                    return fail(HYP_ERR_IO, "too many reaction groups");
                }
                k = d.ngroup++;
                d.g_n[k] = rx[r].n;
                d.g_Ta[k] = rx[r].Ta;
                double theta_d = 0.0;
                for (int i = 0; i < NSP; ++i) {
                    const int nu = order_b[r * NSP + i] - order_f[r * NSP + i];
                    d.g_nu[k][i] = (signed char)nu;
                    d.g_nud[k][i] = nu;
                    // E0 / R_u of species i: formation enthalpy minus the sensible part at 298.15 K
                    theta_d += nu * (sp[i].hf / R_U - h_sens_over_r(sp[i], 298.15));
                }
                d.g_theta_d[k] = theta_d;
            }
            grp[r] = k;
        }
        d.nr = nr;
        int pos = 0;
        for (int k = 0; k < d.ngroup; ++k) {
            d.gstart[k] = pos;
            bool first = true;
            for (int r = 0; r < nr; ++r)
                if (grp[r] == k) {
                    // the collider: first species on both sides; the rest must match the group's
                    int spec = -1;
                    for (int i = 0; i < NSP && spec < 0; ++i)
                        if (order_f[r * NSP + i] > 0 && order_b[r * NSP + i] > 0) spec = i;
                    for (int i = 0; i < NSP; ++i) {
                        const int rf = order_f[r * NSP + i] - (i == spec);
                        const int rb = order_b[r * NSP + i] - (i == spec);
                        if (first) {
                            d.g_rf[k][i] = (signed char)rf;
                            d.g_rb[k][i] = (signed char)rb;
                        } else if (d.g_rf[k][i] != rf || d.g_rb[k][i] != rb) {
                            delete g;
                            return fail(HYP_ERR_IO, "reactions of one rate group must differ only in their collider");
                        }
                    }
                    first = false;
                    d.C[pos] = Cs[r];
                    d.spec[pos] = spec;
                    ++pos;
                }
        }
        d.gstart[d.ngroup] = pos;
    }
    // freestream scales (Eqs. 7, 11)
    double Y[NSP], ym = 0.0, ysum = 0.0;
    for (int i = 0; i < NSP; ++i) {
        Y[i] = fs->Y_inf[i];
        d.Y_inf[i] = fs->Y_inf[i];
        ym += Y[i] * d.invM[i];
        ysum += Y[i];
    }
    if (!(fs->T_inf > 0 && fs->p_inf > 0 && fs->reynolds > 0 && fabs(ysum - 1.0) < 1e-12)) {
        delete g;
        return fail(HYP_ERR_ARG, "freestream needs T, p, Re > 0 and mass fractions summing to 1");
    }
    for (int e = 0; e < 2; ++e) {
        d.elem_b[e] = 0.0;
        bool pure = false;
        for (int i = 0; i < NSP; ++i) {
            d.elem_b[e] += d.atoms[i][e] * Y[i] * d.invM[i];
            pure = pure || (d.atoms[i][e] > 0 && d.atoms[i][1 - e] == 0);
        }
        if (kind == HYP_GAS_LTE && !(pure && d.elem_b[e] > 0.0)) {
            delete g;
            return fail(HYP_ERR_ARG, "LTE needs both elements in Y_inf and a species made of each "
                                     "element alone");
        }
    }
    {
        SpeciesState lo, hi;
        species_state(d, T_LO, lo);
        species_state(d, T_HI, hi);
        for (int i = 0; i < NSP; ++i) {
            d.e_lo[i] = lo.e[i];
            d.e_hi[i] = hi.e[i];
        }
    }
    SpeciesState s;
    species_state(d, fs->T_inf, s);
    double cv = 0.0;
    for (int i = 0; i < NSP; ++i) cv += Y[i] * s.cv[i];
    const double R = R_U * ym;
    d.R_inf = R;
    d.cp_inf = cv + R;
    d.gamma_inf = (cv + R) / cv;
    d.T_inf = fs->T_inf;
    d.p_inf = fs->p_inf;
    d.rho_inf = fs->p_inf / (R * fs->T_inf);
    d.a_inf = sqrt(d.gamma_inf * R * fs->T_inf);
    d.prandtl_cpg = fs->prandtl_cpg;
    d.mach = fs->mach;
    d.tpg_theta = TPG_THETA;
    d.tpg_cp0 = d.cp_inf / (1.0 + (d.gamma_inf - 1.0) / d.gamma_inf * tpg_shape(TPG_THETA / fs->T_inf));
    if (kind == HYP_GAS_CPG) {
        d.mu_inf = SUTH_C1 * pow(fs->T_inf, 1.5) / (fs->T_inf + SUTH_TS);
        d.k_inf = d.mu_inf * d.cp_inf / fs->prandtl_cpg;
    } else if (kind == HYP_GAS_TPG) {
        d.mu_inf = SUTH_C1 * pow(fs->T_inf, 1.5) / (fs->T_inf + SUTH_TS);
        d.k_inf = keyes(fs->T_inf);
    } else {
        ClosureOut o;
        const double e = mixture_energy(d, fs->T_inf, Y);
        closure_si(d, d.rho_inf, e, Y, fs->T_inf, false, false, o);
        d.mu_inf = o.mu;
        d.k_inf = o.k;
    }
    for (int i = 0; i < NSP; ++i) {
        d.f_blA[i] = (float)d.blA[i];
        d.f_blB[i] = (float)d.blB[i];
        d.f_blC[i] = (float)d.blC[i];
        d.f_Mq[i] = (float)d.Mq[i];
        d.f_iMq[i] = (float)d.iMq[i];
        d.f_Rs[i] = (float)d.Rs[i];
        for (int j = 0; j < NSP; ++j) d.f_wilke_d[i][j] = (float)d.wilke_d[i][j];
    }
    for (int q = 0; q < NSP * (NSP - 1) / 2; ++q) d.f_pair_dinv[q] = (float)d.pair_dinv[q];
    for (int q = 0; q < MAXEPS; ++q) {
        d.f_eps_inv[q] = (float)d.eps_inv[q];
        d.f_eps_powB[q] = (float)d.eps_powB[q];
    }
    d.etab_lnT0 = log(T_LO);
    d.etab_dlnT = (log(T_HI) - log(T_LO)) / (ETAB_N - 1);
    g->etab_host.assign(2 * NSP * ETAB_N, 0.0);
    for (int k = 0; k < ETAB_N; ++k) {
        SpeciesState st;
        species_state(d, exp(d.etab_lnT0 + k * d.etab_dlnT), st);
        for (int i = 0; i < NSP; ++i) {
            g->etab_host[i * ETAB_N + k] = st.e[i];
            g->etab_host[(NSP + i) * ETAB_N + k] = st.cv[i];
        }
    }
    d.etab = nullptr;
    d.Re = fs->reynolds;
    d.Pr = d.mu_inf * d.cp_inf / d.k_inf;
    d.T_ref = (d.gamma_inf - 1.0) * fs->T_inf;
    d.L_ref = d.Re * d.mu_inf / (d.rho_inf * d.a_inf);
    *out = g;
    return HYP_OK;
}

extern "C" int hyp_gas_scales(const hyp_gas* gas, int* n_species, double* sc) {
    if (!gas) return fail(HYP_ERR_ARG, "null gas");
    if (n_species) *n_species = NSP;
    if (sc) {
        const GasDev& d = gas->dev;
        const double v[13] = {d.rho_inf, d.a_inf, d.T_inf, d.p_inf, d.mu_inf, d.k_inf, d.cp_inf,
                              d.gamma_inf, d.R_inf, d.T_ref, d.L_ref, d.Re, d.Pr};
        memcpy(sc, v, sizeof(v));
    }
    return HYP_OK;
}

extern "C" void hyp_gas_free(hyp_gas* gas) {
    if (gas && gas->etab_dev) cudaFree(gas->etab_dev);
    delete gas;
}

extern "C" const char* hyp_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------------------------
// Pointwise kernels
// ---------------------------------------------------------------------------------------------

namespace gaskern {

template <bool MIXED>
__global__ void __launch_bounds__(128) k_thermo_eval(
    GasDev g, int64_t n, const double* __restrict__ rho, const double* __restrict__ e,
    const double* __restrict__ Y, double* __restrict__ T, double* __restrict__ p,
    double* __restrict__ wdot, double* __restrict__ mu, double* __restrict__ kk,
    double* __restrict__ D, uint8_t* __restrict__ status) {
    const bool reactions = g.kind == HYP_GAS_CNEQ;
    const bool diffusion = g.kind == HYP_GAS_CNEQ;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double y[NSP];
#pragma unroll
        for (int s = 0; s < NSP; ++s) y[s] = Y[s * n + i];
        ClosureOut o;
        // binary64 modal sums in both precisions: independent states (closure_si_p, MODES32)
        closure_si_p<MIXED, false>(g, rho[i], e[i], y, temperature_guess(g, e[i], y), reactions && wdot,
                            diffusion && D, o);
        if (T) T[i] = o.T;
        if (p) p[i] = o.p;
        if (mu) mu[i] = o.mu;
        if (kk) kk[i] = o.k;
        if (wdot)
#pragma unroll
            for (int s = 0; s < NSP; ++s) wdot[s * n + i] = o.wdot[s];
        if (D)
#pragma unroll
            for (int s = 0; s < NSP; ++s) D[s * n + i] = o.D[s];
        if (status) status[i] = (uint8_t)o.status;
    }
}

template <bool MIXED>
__global__ void __launch_bounds__(128) k_lte_eval(
    GasDev g, int64_t n, const double* __restrict__ rho, const double* __restrict__ e,
    double* __restrict__ T, double* __restrict__ p, double* __restrict__ Y,
    double* __restrict__ mu, double* __restrict__ kk, double* __restrict__ kr,
    uint8_t* __restrict__ status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        ClosureOut o;
        double y[NSP], k_r;
        lte_closure<MIXED>(g, rho[i], e[i], temperature_guess(g, e[i], g.Y_inf), y, k_r, o);
        if (T) T[i] = o.T;
        if (p) p[i] = o.p;
        if (mu) mu[i] = o.mu;
        if (kk) kk[i] = o.k;
        if (kr) kr[i] = k_r;
        if (Y)
#pragma unroll
            for (int s = 0; s < NSP; ++s) Y[s * n + i] = y[s];
        if (status) status[i] = (uint8_t)o.status;
    }
}

__global__ void k_thermo_energy(GasDev g, int64_t n, const double* __restrict__ T,
                                const double* __restrict__ Y, double* __restrict__ e) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double y[NSP];
#pragma unroll
        for (int s = 0; s < NSP; ++s) y[s] = Y[s * n + i];
        e[i] = mixture_energy(g, T[i], y);
    }
}

// The device copy of the starting-temperature table (GasDev::etab), made by the first evaluation
// that needs it: loading a gas model stays a host-only step.
int gas_etab(const hyp_gas* cgas) {
    hyp_gas* gas = const_cast<hyp_gas*>(cgas);
    std::lock_guard<std::mutex> lock(gas->etab_mu);
    if (gas->etab_dev) return HYP_OK;
    const size_t bytes = sizeof(double) * gas->etab_host.size();
    double* p = nullptr;
    HYP_CUDA(cudaMalloc(&p, bytes));
    const cudaError_t err = cudaMemcpy(p, gas->etab_host.data(), bytes, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        cudaFree(p);
        HYP_CUDA(err);
    }
    gas->etab_dev = p;
    gas->dev.etab = p;
    return HYP_OK;
}

int grid_for(int64_t n, int block) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (n + block - 1) / block;
    int64_t cap = (int64_t)sms * 16;
    return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace gaskern
using namespace gaskern;

extern "C" int hyp_thermo_eval(const hyp_gas* gas, int64_t n, const double* rho, const double* e,
                               const double* Y, double* T, double* p, double* wdot, double* mu,
                               double* k, double* D, uint8_t* status, int precision,
                               void* stream) {
    if (!gas || n < 0) return fail(HYP_ERR_ARG, "null gas or negative n");
    if (precision != HYP_FP64 && precision != HYP_MIXED) return fail(HYP_ERR_ARG, "unknown precision");
    if (gas->dev.kind == HYP_GAS_LTE)
        return fail(HYP_ERR_ARG, "an LTE gas has no independent composition: use hyp_lte_eval");
    if (n == 0) return HYP_OK;
    if (!rho || !e || !Y) return fail(HYP_ERR_ARG, "null input");
    if (const int rc = gas_etab(gas)) return rc;
    const int block = 128;
    if (precision == HYP_MIXED)
        k_thermo_eval<true><<<grid_for(n, block), block, 0, (cudaStream_t)stream>>>(
            gas->dev, n, rho, e, Y, T, p, wdot, mu, k, D, status);
    else
        k_thermo_eval<false><<<grid_for(n, block), block, 0, (cudaStream_t)stream>>>(
            gas->dev, n, rho, e, Y, T, p, wdot, mu, k, D, status);
    HYP_CUDA(cudaGetLastError());
    return HYP_OK;
}

extern "C" int hyp_thermo_energy(const hyp_gas* gas, int64_t n, const double* T, const double* Y,
                                 double* e, void* stream) {
    if (!gas || n < 0) return fail(HYP_ERR_ARG, "null gas or negative n");
    if (n == 0) return HYP_OK;
    if (!T || !Y || !e) return fail(HYP_ERR_ARG, "null pointer");
    const int block = 256;
    k_thermo_energy<<<grid_for(n, block), block, 0, (cudaStream_t)stream>>>(gas->dev, n, T, Y, e);
    HYP_CUDA(cudaGetLastError());
    return HYP_OK;
}

extern "C" int hyp_lte_eval(const hyp_gas* gas, int64_t n, const double* rho, const double* e,
                            double* T, double* p, double* Y, double* mu, double* k,
                            double* k_reactive, uint8_t* status, int precision, void* stream) {
    if (!gas || n < 0) return fail(HYP_ERR_ARG, "null gas or negative n");
    if (gas->dev.kind != HYP_GAS_LTE) return fail(HYP_ERR_ARG, "hyp_lte_eval needs an LTE gas");
    if (precision != HYP_FP64 && precision != HYP_MIXED) return fail(HYP_ERR_ARG, "unknown precision");
    if (n == 0) return HYP_OK;
    if (!rho || !e) return fail(HYP_ERR_ARG, "null input");
    if (const int rc = gas_etab(gas)) return rc;
    const int block = 128;
    if (precision == HYP_MIXED)
        k_lte_eval<true><<<grid_for(n, block), block, 0, (cudaStream_t)stream>>>(
            gas->dev, n, rho, e, T, p, Y, mu, k, k_reactive, status);
    else
        k_lte_eval<false><<<grid_for(n, block), block, 0, (cudaStream_t)stream>>>(
            gas->dev, n, rho, e, T, p, Y, mu, k, k_reactive, status);
    HYP_CUDA(cudaGetLastError());
    return HYP_OK;
}
