// Right-hand side of the reacting Navier-Stokes equations on the staggered grid (Eqs. 1-11, 26;
// Secs. 3.1-3.3) and the two-register RK3 stage update, plus the grid / state set-up.
//
// Device data of a grid: metrics, sponge strength and reference state in state layout, a
// Dirichlet mask, the compact operators, and one block of scratch fields (cell centres, x-faces,
// y-faces and corners). The right-hand side is a fixed sequence of launches: batched line
// operators (lines.cu) alternate with pointwise kernels defined here.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "grid.h"
#include "internal.h"
#include "pointwise.cuh"
#include "thermo.cuh"

using namespace hyp;


namespace {

// ---------------------------------------------------------------------------------------------
// Host: grid maps, oblique shock, reference profile
// ---------------------------------------------------------------------------------------------

__host__ __device__ void y_map(const hyp_grid_desc& d, double eta, double& y, double& dyde) {
    const double s = eta / d.ny;
    const double L = d.y1 - d.y0, q = d.y_param;
    if (d.y_stretch == 1) {
        y = d.y0 + L * (1.0 - tanh(q * (1.0 - s)) / tanh(q));
        const double ch = cosh(q * (1.0 - s));
        dyde = L * q / (ch * ch) / tanh(q) / d.ny;
    } else if (d.y_stretch == 2) {
        y = d.y0 + L * ((1.0 - q) * s * s * s + q * s);
        dyde = L * (3.0 * (1.0 - q) * s * s + q) / d.ny;
    } else {
        y = d.y0 + L * s;
        dyde = L / d.ny;
    }
}

struct Shock {
    double beta, p21, r21, T21, M2;
};

// Weak oblique shock for deflection theta: theta-beta-M relation by bisection on the rising
// branch, then the Rankine-Hugoniot jumps of a perfect gas.
Shock oblique_shock(double M1, double theta, double gam) {
    auto defl = [&](double b) {
        return atan(2.0 / tan(b) * (M1 * M1 * sin(b) * sin(b) - 1.0) /
                    (M1 * M1 * (gam + cos(2.0 * b)) + 2.0));
    };
    double lo = asin(1.0 / M1) + 1e-12, hi = lo;
    const double step = 1.0e-3;
    while (defl(hi + step) > defl(hi)) hi += step;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (defl(mid) < theta) lo = mid; else hi = mid;
    }
    Shock s;
    s.beta = 0.5 * (lo + hi);
    const double mn1 = M1 * sin(s.beta);
    s.p21 = 1.0 + 2.0 * gam / (gam + 1.0) * (mn1 * mn1 - 1.0);
    s.r21 = (gam + 1.0) * mn1 * mn1 / ((gam - 1.0) * mn1 * mn1 + 2.0);
    s.T21 = s.p21 / s.r21;
    const double mn2 =
        sqrt((1.0 + 0.5 * (gam - 1.0) * mn1 * mn1) / (gam * mn1 * mn1 - 0.5 * (gam - 1.0)));
    s.M2 = mn2 / sin(s.beta - theta);
    return s;
}

struct Profile {
    hyp_case c;
    double y0;
    int iN2, iO2, iNO, iN, iO;
    bool shock;
    Shock sh;
    double theta;
    double Yinf[NSP];

    // Boundary-layer profile below an edge state: u/u_e = erf(2 y / delta(x)), Crocco-Busemann T.
    __host__ __device__ void edge(const GasDev& g, double x, double y, double Te, double pe, double ue, double ve, double Me,
              double& T, double& p, double& u, double& v, double& f) const {
        if (c.wall) {
            const double delta = c.delta_coef * sqrt(x / (g.Re * g.mach));
            f = erf(2.0 * (y - y0) / delta);
            const double Tr = Te * (1.0 + RECOVERY * 0.5 * (g.gamma_inf - 1.0) * Me * Me);
            T = c.T_wall + (Tr - c.T_wall) * f - (Tr - Te) * f * f;
        } else {
            f = 1.0;
            T = Te;
        }
        p = pe;
        u = ue * f;
        v = ve * f;
    }

    // primitive reference state: T [K], p [Pa], u, v nondimensional, Y
    __host__ __device__ void at(const GasDev& g, double x, double y, double& T, double& p, double& u, double& v, double* Y) const {
        double f;
        edge(g, x, y, g.T_inf, g.p_inf, g.mach, 0.0, g.mach, T, p, u, v, f);
        if (shock) {
            const double V2 = sh.M2 * sqrt(sh.T21);
            double T2, p2, u2, v2, f2;
            edge(g, x, y, g.T_inf * sh.T21, g.p_inf * sh.p21, V2 * cos(theta), -V2 * sin(theta),
                 sh.M2, T2, p2, u2, v2, f2);
            const double ys = (c.shock_x - x) * tan(sh.beta);
            const double H = 0.5 * (1.0 + tanh((y - ys) / c.shock_width));
            T = (1.0 - H) * T + H * T2;
            p = (1.0 - H) * p + H * p2;
            u = (1.0 - H) * u + H * u2;
            v = (1.0 - H) * v + H * v2;
        }
        for (int s = 0; s < NSP; ++s) Y[s] = Yinf[s];
        const bool seed = c.wall && (g.kind == HYP_GAS_CNEQ || g.kind == HYP_GAS_FROZEN) && iN2 >= 0 && iO2 >= 0 && iNO >= 0 &&
                          iN >= 0 && iO >= 0;
        if (seed) {
            const double m = c.minor_species * 4.0 * f * (1.0 - f);
            Y[iN2] = Yinf[iN2] * (1.0 - m);
            Y[iO2] = Yinf[iO2] * (1.0 - m);
            Y[iNO] = 0.5 * m;
            Y[iN] = 0.2 * m;
            Y[iO] = 0.3 * m;
        }
    }

    // nondimensional rho, rho_s (all species), rho*E
    __host__ __device__ void conserved(const GasDev& g, double T, double p, double u, double v, const double* Y, double& rho,
                   double* rhoY, double& rhoE) const {
        double rho_si, e_nd;
        if (g.kind == HYP_GAS_TPG) {
            const TpgModel m{g.tpg_cp0, (g.gamma_inf - 1.0) / g.gamma_inf, g.tpg_theta, g.R_inf};
            rho_si = p / (g.R_inf * T);
            e_nd = m.energy(T) / (g.a_inf * g.a_inf);
        } else if (g.kind == HYP_GAS_CPG) {
            rho_si = p / (g.R_inf * T);
            e_nd = (T / g.T_ref) / g.gamma_inf;
        } else if (g.kind == HYP_GAS_LTE) {
            // density from T and p with the gas constant of Y, then the equilibrium composition
            // and energy at that (T, rho)
            double ym = 0.0;
            for (int s = 0; s < NSP; ++s) ym += Y[s] * g.invM[s];
            rho_si = p / (R_U * ym * T);
            const double b[2] = {rho_si * g.elem_b[0], rho_si * g.elem_b[1]};
            const double lnb[2] = {log(b[0]), log(b[1])};
            LteState q;
            lte_at(g, T, rho_si, b, lnb, false, q);
            e_nd = q.e / (g.a_inf * g.a_inf);
            rho = rho_si / g.rho_inf;
            for (int s = 0; s < NSP; ++s) rhoY[s] = rho * (q.c[s] * g.M[s] / rho_si);
            rhoE = rho * (e_nd + 0.5 * (u * u + v * v));
            return;
        } else {
            double ym = 0.0;
            for (int s = 0; s < NSP; ++s) ym += Y[s] * g.invM[s];
            rho_si = p / (R_U * ym * T);
            e_nd = mixture_energy(g, T, Y) / (g.a_inf * g.a_inf);
        }
        rho = rho_si / g.rho_inf;
        for (int s = 0; s < NSP; ++s) rhoY[s] = rho * Y[s];
        rhoE = rho * (e_nd + 0.5 * (u * u + v * v));
    }
};

// Sponge strength of Eq. (26) at (x, y): cubic ramps over the inflow, outflow and top zones.
__host__ __device__ inline double sponge_at(const hyp_grid_desc& d, const hyp_case& c, double x,
                                            double y) {
    double sg = 0.0;
    if (c.sponge_in > 0) {
        const double r = fmin(fmax((d.x0 + c.sponge_in - x) / c.sponge_in, 0.0), 1.0);
        sg += r * r * r;
    }
    if (c.sponge_out > 0) {
        const double r = fmin(fmax((x - (d.x1 - c.sponge_out)) / c.sponge_out, 0.0), 1.0);
        sg += r * r * r;
    }
    if (c.sponge_top_cells > 0) {
        double ytop, dy;
        y_map(d, (double)(d.ny - c.sponge_top_cells), ytop, dy);
        const double r = fmin(fmax((y - ytop) / (d.y1 - ytop), 0.0), 1.0);
        sg += r * r * r;
    }
    return c.sponge_sigma * sg;
}

// Reference state Q_ref (Eq. 26), sponge strength and the Dirichlet mask at every state entry:
// one thread per cell centre, x-face and y-face.
__global__ void k_reference(GasDev g, Profile P, hyp_grid_desc d, long long off_xf, long long off_yf,
                            double* __restrict__ Uref, double* __restrict__ sig,
                            uint8_t* __restrict__ mask) {
    const int nx = d.nx, ny = d.ny;
    const long long nc = (long long)nx * ny, nxf = (long long)(nx + 1) * ny;
    const long long n = nc + nxf + (long long)nx * (ny + 1);
    const double dx = (d.x1 - d.x0) / nx;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        int node, i, j;
        if (k < nc) {
            node = 0; j = (int)(k / nx); i = (int)(k - (long long)j * nx);
        } else if (k < nc + nxf) {
            node = 1; const long long q = k - nc; j = (int)(q / (nx + 1)); i = (int)(q - (long long)j * (nx + 1));
        } else {
            node = 2; const long long q = k - nc - nxf; j = (int)(q / nx); i = (int)(q - (long long)j * nx);
        }
        const double x = d.x0 + dx * (node == 1 ? (double)i : i + 0.5);
        double y, dy;
        y_map(d, node == 2 ? (double)j : j + 0.5, y, dy);
        double T, p, u, v, Y[NSP], rho, rY[NSP], rE;
        P.at(g, x, y, T, p, u, v, Y);
        P.conserved(g, T, p, u, v, Y, rho, rY, rE);
        const double sg = sponge_at(d, P.c, x, y);
        if (node == 0) {
            Uref[k] = rho;
            sig[k] = sg;
            mask[k] = 0;
            for (int sp = 1; sp < NSP; ++sp) {
                Uref[sp * nc + k] = rY[sp];
                sig[sp * nc + k] = sg;
                mask[sp * nc + k] = 0;
            }
            Uref[NSP * nc + k] = rE;
            sig[NSP * nc + k] = sg;
            mask[NSP * nc + k] = 0;
        } else if (node == 1) {
            const long long e = off_xf + (k - nc);
            Uref[e] = rho * u;
            sig[e] = sg;
            mask[e] = (i == 0 || i == nx) ? 1 : 0;
        } else {
            const long long e = off_yf + (k - nc - nxf);
            Uref[e] = rho * v;
            sig[e] = sg;
            mask[e] = (j == 0 || j == ny) ? 1 : 0;
        }
    }
}

// Initial state: the reference with the seeded multiplicative noise on every entry not held.
__global__ void k_initial(long long n, const double* __restrict__ Uref, const uint8_t* __restrict__ mask,
                          const double* __restrict__ noise, double amp, double* __restrict__ U) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        U[k] = (noise && !mask[k]) ? Uref[k] * (1.0 + amp * noise[k]) : Uref[k];
}

// ---------------------------------------------------------------------------------------------
// Host: compact operators
// ---------------------------------------------------------------------------------------------

void lagrange(const double* nodes, int n, double x, bool deriv, double* w) {
    for (int k = 0; k < n; ++k) {
        double den = 1.0;
        for (int m = 0; m < n; ++m)
            if (m != k) den *= nodes[k] - nodes[m];
        double num;
        if (!deriv) {
            num = 1.0;
            for (int m = 0; m < n; ++m)
                if (m != k) num *= x - nodes[m];
        } else {
            num = 0.0;
            for (int skip = 0; skip < n; ++skip) {
                if (skip == k) continue;
                double t = 1.0;
                for (int m = 0; m < n; ++m)
                    if (m != k && m != skip) t *= x - nodes[m];
                num += t;
            }
        }
        w[k] = num / den;
    }
}

// Build one operator: kind 0 interpolation / 1 derivative; dir 0 centre->face / 1 face->centre.
LineOp make_op(int kind, int dir, int n, int wall, std::vector<double>& data) {
    LineOp op;
    memset(&op, 0, sizeof(op));
    op.kind = kind;
    op.dir = dir;
    op.wall = wall;
    double alpha, a, b;
    if (kind == 0) { alpha = 3.0 / 10.0; a = 3.0 / 2.0; b = 1.0 / 10.0; }
    else { alpha = 9.0 / 62.0; a = 63.0 / 62.0; b = 17.0 / 62.0; }
    if (kind == 0) {
        op.wi[0] = b / 2.0; op.wi[1] = a / 2.0; op.wi[2] = a / 2.0; op.wi[3] = b / 2.0;
    } else {
        op.wi[0] = -b / 3.0; op.wi[1] = -a; op.wi[2] = a; op.wi[3] = b / 3.0;
    }
    std::vector<double> in_pos, out_pos;
    if (dir == 0) {
        op.m = n + 1;
        op.n_in = n;
        for (int k = 0; k < n; ++k) in_pos.push_back(k + 0.5);
        for (int i = 0; i <= n; ++i) out_pos.push_back(i);
        op.first_interior = 2;
        op.last_interior = n - 2;
    } else {
        op.m = n;
        op.n_in = n + 1;
        for (int i = 0; i <= n; ++i) in_pos.push_back(i);
        for (int k = 0; k < n; ++k) out_pos.push_back(k + 0.5);
        op.first_interior = 1;
        op.last_interior = n - 2;
    }
    const int m = op.m;
    std::vector<double> lower(m, 0.0), upper(m, 0.0);
    for (int r = 0; r < m; ++r) {
        const bool interior = r >= op.first_interior && r <= op.last_interior;
        if (interior) {
            if (r > 0) lower[r] = alpha;
            if (r < m - 1) upper[r] = alpha;
            continue;
        }
        const int c = op.ncl++;
        op.crow[c] = r;
        const bool left = r < op.first_interior;
        double nodes[5], w[5];
        if (left && wall) {
            nodes[0] = 0.0;
            for (int k = 0; k < 4; ++k) nodes[k + 1] = in_pos[k];
            lagrange(nodes, 5, out_pos[r], kind == 1, w);
            op.gw[c] = w[0];
            op.cstart[c] = 0;
            op.cnum[c] = 4;
            for (int k = 0; k < 4; ++k) op.cw[c][k] = w[k + 1];
        } else {
            const int start = left ? 0 : (int)in_pos.size() - 5;
            for (int k = 0; k < 5; ++k) nodes[k] = in_pos[start + k];
            lagrange(nodes, 5, out_pos[r], kind == 1, w);
            op.gw[c] = 0.0;
            op.cstart[c] = start;
            op.cnum[c] = 5;
            for (int k = 0; k < 5; ++k) op.cw[c][k] = w[k];
        }
    }
    // Thomas factors of the unit-diagonal tridiagonal matrix
    std::vector<double> cp(m), mi(m);
    for (int r = 0; r < m; ++r) {
        const double piv = 1.0 - (r > 0 ? lower[r] * cp[r - 1] : 0.0);
        mi[r] = 1.0 / piv;
        cp[r] = upper[r] * mi[r];
    }
    // interior weights folded with the pivot: d_r = wa_r (f1 +/- f0) + wb_r (f3 +/- f_-1) - lm_r d_{r-1}
    std::vector<double> wa(m), wb(m), lm(m);
    for (int r = 0; r < m; ++r) {
        wa[r] = (kind == 0 ? op.wi[1] : op.wi[2]) * mi[r];
        wb[r] = (kind == 0 ? op.wi[0] : op.wi[3]) * mi[r];
        lm[r] = lower[r] * mi[r];
    }
    // first row of the constant tail of the interior factors
    const int li = op.last_interior;
    op.rc = li + 1;
    if (li >= op.first_interior) {
        int r = li;
        while (r - 1 >= op.first_interior && wa[r - 1] == wa[li] && wb[r - 1] == wb[li] &&
               lm[r - 1] == lm[li] && cp[r - 1] == cp[li])
            --r;
        op.rc = r;
        op.wac = wa[li];
        op.wbc = wb[li];
        op.lmc = lm[li];
        op.cpc = cp[li];
        op.wac_f = (float)op.wac;
        op.wbc_f = (float)op.wbc;
        op.lmc_f = (float)op.lmc;
        op.cpc_f = (float)op.cpc;
        op.wac_l = (float)(op.wac - (double)op.wac_f);
        op.wbc_l = (float)(op.wbc - (double)op.wbc_f);
        op.lmc_l = (float)(op.lmc - (double)op.lmc_f);
        op.cpc_l = (float)(op.cpc - (double)op.cpc_f);
    }
    // store offsets into data (fixed up to device pointers later)
    const size_t base = data.size();
    for (auto* v : {&lower, &cp, &mi, &wa, &wb, &lm}) data.insert(data.end(), v->begin(), v->end());
    op.lower = (const double*)(base);
    op.cprime = (const double*)(base + m);
    op.minv = (const double*)(base + 2 * m);
    op.wa = (const double*)(base + 3 * m);
    op.wb = (const double*)(base + 4 * m);
    op.lm = (const double*)(base + 5 * m);
    return op;
}

enum OpId { OX_ICF, OX_DCF, OX_IFC, OX_DFC, OY_ICF, OY_DCF, OY_IFC, OY_DFC, OY_ICFW, OY_DCFW, NOPS };

// ---------------------------------------------------------------------------------------------
// Pointwise kernels
// ---------------------------------------------------------------------------------------------

// Single-grid kernels: grid-stride loops over the bodies of pointwise.cuh.
#define GRID_RANGE(n) (long long)blockIdx.x * blockDim.x, (long long)(n), (long long)gridDim.x * blockDim.x

// The scales, grid view and scratch pointers are copied to shared memory first, as the batched
// executor's kernel holds them, so that both pass the shared closure_point the same kinds of
// pointers.
template <bool MIXED, bool LTE>
__global__ void __launch_bounds__(128, CLOSURE_MIN_BLOCKS) k_closure(const __grid_constant__ GasDev g,
                                                    const Scales sc, const GridView v,
                                                    const double* __restrict__ U, const Scratch s) {
    __shared__ Scales sh_sc;
    __shared__ GridView sh_v;
    __shared__ Scratch sh_s;
    if (threadIdx.x == 0) {
        sh_sc = sc;
        sh_v = v;
        sh_s = s;
    }
    __syncthreads();
    closure_body<MIXED, LTE>(g, sh_sc, sh_v, U, sh_s, GRID_RANGE((long long)v.nx * v.ny));
}

// the closure kernel for the gas kind and precision
static void launch_closure(const GasDev& g, const Scales& sc, const GridView& v, const double* U,
                           const Scratch& S, bool mixed, int blocks, cudaStream_t s) {
    if (g.kind == HYP_GAS_LTE) {
        if (mixed) k_closure<true, true><<<blocks, 128, 0, s>>>(g, sc, v, U, S);
        else k_closure<false, true><<<blocks, 128, 0, s>>>(g, sc, v, U, S);
    } else {
        if (mixed) k_closure<true, false><<<blocks, 128, 0, s>>>(g, sc, v, U, S);
        else k_closure<false, false><<<blocks, 128, 0, s>>>(g, sc, v, U, S);
    }
}

__global__ void k_face_vel(GridView v, const double* __restrict__ U, Scratch s) {
    face_vel_body(v, U, s, GRID_RANGE((long long)v.ny * (v.nx + 1) + (long long)(v.ny + 1) * v.nx));
}

__global__ void k_ad_prep(GridView v, Scratch s) {
    ad_prep_body(s, GRID_RANGE((long long)v.nx * v.ny));
}

__global__ void k_ad_raw(int cneq, GridView v, const double* __restrict__ U, Scratch s) {
    ad_raw_body(cneq != 0, v, U, s, GRID_RANGE((long long)v.nx * v.ny));
}

template <bool MIXED>
__global__ void k_gauss(GridView v, Scratch s, int dir) {
    gauss_body<MIXED>(v, s, dir, GRID_RANGE((MIXED ? 1LL : (long long)AD_FIELDS) * v.nx * v.ny));
}

__global__ void k_ad_combine(GridView v, Scratch s) {
    ad_combine_body(s, GRID_RANGE((long long)v.nx * v.ny));
}

__global__ void k_stress_c(GridView v, Scratch s) {
    stress_c_body(s, GRID_RANGE((long long)v.nx * v.ny));
}

__global__ void k_stress_cn(GridView v, Scratch s) {
    stress_cn_body(s, GRID_RANGE((long long)(v.nx + 1) * (v.ny + 1)));
}

template <bool SMK>
__global__ void k_flux(GasDev g, Scales sc, GridView v, const double* __restrict__ U, Scratch s,
                       int dir) {
    flux_body<SMK>(g, sc, v, U, s, dir, GRID_RANGE(dir == 0 ? (long long)v.ny * (v.nx + 1) : (long long)(v.ny + 1) * v.nx));
}

__global__ void k_assemble(long long n, AssembleArgs a) { assemble_body(a, GRID_RANGE(n)); }

__global__ void k_filter(int nx, int ny, long long nstate, const double* __restrict__ in,
                         double* __restrict__ out, int dir, double sigma) {
    filter_body(nx, ny, in, out, dir, sigma, GRID_RANGE(nstate));
}

__global__ void k_fill(double* p, long long n, double val) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = val;
}

int blocks_for(long long n, int block) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long b = (n + block - 1) / block;
    long long cap = (long long)sms * 8;
    if (b < 1) b = 1;
    return (int)std::min(b, cap);
}

// ---------------------------------------------------------------------------------------------
// Host: job plans
// ---------------------------------------------------------------------------------------------

struct PlanBuilder {
    const hyp_grid* G;
    const LineOp* dops;   // device operator array
    const LineOp* hops;   // host copies (line lengths)
    std::vector<LineJob> jobs;
    std::vector<long long> out_size;
    int ph_start[PH_COUNT], ph_count[PH_COUNT], ph_blocks[PH_COUNT];
    int cur = -1;

    void begin(int ph) {
        cur = ph;
        ph_start[ph] = (int)jobs.size();
        ph_count[ph] = 0;
        ph_blocks[ph] = 0;
    }
    void add(OpId op, const double* in, Node tin, double* out, Node tout, const double* metric,
             double scale = 1.0, double wall_value = 0.0, int in_state = 0) {
        const Dims& d = G->d;
        const bool alongx = op <= OX_DFC;
        LineJob j;
        memset(&j, 0, sizeof(j));
        j.op = dops + op;
        j.in = in;
        j.in_state = in_state;
        j.out = out;
        if (alongx) {
            j.in_ls = d.pitch(tin);
            j.in_es = 1;
            j.out_ls = d.pitch(tout);
            j.out_es = 1;
            j.nlines = d.rows(tin);
        } else {
            j.in_ls = 1;
            j.in_es = d.pitch(tin);
            j.out_ls = 1;
            j.out_es = d.pitch(tout);
            j.nlines = d.pitch(tin);
        }
        j.nseg = hops[op].m;   // line length for now; replaced by the segment count in finish()
        j.wall_value = wall_value;
        j.scale = scale;
        j.metric = metric;
        jobs.push_back(j);
        out_size.push_back(d.size(tout));
        ph_count[cur]++;
    }
    // the last job added feeds only diffusive fluxes: binary32 allowed under HYP_MIXED
    void f32() { jobs.back().f32ok = 1; }
    // Segment counts (at most 260 points per segment, more segments when a phase has too few
    // threads to occupy the GPU), forward-sweep storage and block counts per phase. Returns the
    // tmp doubles needed by the largest phase.
    long long finish() {
        long long need = 0;
        long long face_need = 0;
        for (int k = ph_start[PH_FACE]; k < ph_start[PH_FACE] + ph_count[PH_FACE]; ++k)
            face_need += out_size[k];
        for (int ph = 0; ph < PH_COUNT; ++ph) {
            const int a = ph_start[ph], b = a + ph_count[ph];
            std::vector<int> nseg(ph_count[ph]);
            long long threads = 0;
            for (int k = a; k < b; ++k) {
                const int m = jobs[k].nseg;
                int ns = 1;
                while (ns < LINE_BLOCK / 2 && (m + ns - 1) / ns > 260) ns *= 2;
                nseg[k - a] = ns;
                threads += (long long)jobs[k].nlines * ns;
            }
            while (threads < 40960) {
                bool grew = false;
                threads = 0;
                for (int k = a; k < b; ++k) {
                    const int m = jobs[k].nseg;
                    if (nseg[k - a] < LINE_BLOCK / 2 && (m + 2 * nseg[k - a] - 1) / (2 * nseg[k - a]) >= 32) {
                        nseg[k - a] *= 2;
                        grew = true;
                    }
                    threads += (long long)jobs[k].nlines * nseg[k - a];
                }
                if (!grew) break;
            }
            // phases that run beside the face phase on the second stream take storage past it
            const bool beside_face = ph == PH_MU1 || ph == PH_MU2 || ph == PH_FACEB;
            long long off = beside_face ? face_need : 0;
            for (int k = a; k < b; ++k) {
                jobs[k].nseg = nseg[k - a];
                jobs[k].tmp = (double*)(size_t)off;   // relative; fixed up by the caller
                off += out_size[k];
                const int lpb = LINE_BLOCK / jobs[k].nseg;
                ph_blocks[ph] = std::max(ph_blocks[ph], (jobs[k].nlines + lpb - 1) / lpb);
            }
            need = std::max(need, off);
        }
        return need;
    }
};

// Event profile (hyp_grid_profile): a pair of CUDA events around a launch on stream s.
static int prof_begin(hyp_grid* G, int kid, cudaStream_t s) {
    EventProfile* P = G->prof;
    if (!P || !P->on) return -1;
    if (P->used + 2 > P->ev.size()) {
        for (int k = 0; k < 256; ++k) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            P->ev.push_back(e);
        }
        P->id.resize(P->ev.size() / 2);
    }
    const size_t slot = P->used;
    P->used += 2;
    P->id[slot / 2] = kid;
    cudaEventRecord(P->ev[slot], s);
    return (int)slot;
}

static void prof_end(hyp_grid* G, int slot, cudaStream_t s) {
    if (slot >= 0) cudaEventRecord(G->prof->ev[slot + 1], s);
}

#include "rhs3d.cuh"

}  // namespace

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------

static int check_desc(const hyp_grid_desc* d) {
    if (!d) return fail(HYP_ERR_ARG, "null grid descriptor");
    if (d->nx < 8 || d->ny < 8) return fail(HYP_ERR_ARG, "grid needs at least 8 cells per direction");
    if ((long long)d->nx * d->ny > (1LL << 28)) return fail(HYP_ERR_ARG, "grid too large");
    if (d->nz > 1 && (d->nz < 4 || (long long)(d->nx + 1) * (d->ny + 1) * d->nz > (1LL << 31)))
        return fail(HYP_ERR_ARG, "three-dimensional grids need 4 to 2^31 / ((nx+1)(ny+1)) z-cells");
    if (!(d->x1 > d->x0) || !(d->y1 > d->y0)) return fail(HYP_ERR_ARG, "empty domain");
    if (d->y_stretch < 0 || d->y_stretch > 2) return fail(HYP_ERR_ARG, "unknown y stretching");
    return HYP_OK;
}

extern "C" int hyp_state_size(const hyp_gas* gas, const hyp_grid_desc* desc, int64_t* n) {
    if (!gas || !n) return fail(HYP_ERR_ARG, "null argument");
    int rc = check_desc(desc);
    if (rc) return rc;
    const long long nc = (long long)desc->nx * desc->ny;
    *n = (NSP + 1) * nc + (long long)(desc->nx + 1) * desc->ny + (long long)desc->nx * (desc->ny + 1);
    if (desc->nz > 1) *n = *n * desc->nz + nc * desc->nz;        // planes, then rho w
    return HYP_OK;
}

static void free_streams(hyp_grid* G) {
    if (G->side) cudaStreamDestroy(G->side);
    for (int k = 0; k < 2; ++k) {
        if (G->fork[k]) cudaEventDestroy(G->fork[k]);
        if (G->join[k]) cudaEventDestroy(G->join[k]);
    }
}

static void free_grid(hyp_grid* G) {
    if (!G) return;
    if (G->g3) {
        free_grid3((Grid3*)G->g3);
        cudaFree(G->status);
        free_streams(G);
        delete G;
        return;
    }
    cudaFree(G->pool);
    cudaFree(G->mask);
    cudaFree(G->status);
    cudaFree(G->ops);
    cudaFree(G->opdata);
    cudaFree(G->jobs);
    cudaFree(G->linetmp);
    cudaFree(G->metf);
    free_streams(G);
    if (G->prof) {
        for (auto e : G->prof->ev) cudaEventDestroy(e);
        delete G->prof;
    }
    delete G;
}

extern "C" int hyp_state_init(const hyp_gas* gas, const hyp_grid_desc* desc, const hyp_case* cas,
                              double* U, double* dQ, void* stream, hyp_state** out) {
    if (!gas || !cas || !U || !dQ || !out) return fail(HYP_ERR_ARG, "null argument");
    int rc = check_desc(desc);
    if (rc) return rc;
    if (cas->flow == 1 && !(cas->shock_width > 0)) return fail(HYP_ERR_ARG, "shock_width must be > 0");
    if (cas->wall && !(cas->T_wall > 0)) return fail(HYP_ERR_ARG, "T_wall must be > 0");
    if (cas->sponge_top_cells < 0 || cas->sponge_top_cells >= desc->ny)
        return fail(HYP_ERR_ARG, "sponge_top_cells out of range");
    if (cas->diffusion_model == 1 && gas->dev.ie >= 0)
        return fail(HYP_ERR_ARG, "Stefan-Maxwell diffusion is not defined for charged mixtures");
    cudaStream_t s = (cudaStream_t)stream;
    const GasDev& g = gas->dev;
    hyp_grid* G = new hyp_grid();   // value-initialised: every pointer and count starts at zero
    G->d.nx = desc->nx;
    G->d.ny = desc->ny;
    G->cas = *cas;
    G->cas.noise = nullptr;
    G->gas = g;
    G->stream = s;
    if (desc->nz > 1) {
        cudaError_t e = cudaMalloc(&G->status, sizeof(unsigned));
        if (e != cudaSuccess) {
            delete G;
            return cuda_fail(e, "cudaMalloc(status)");
        }
        const int r3 = init3(gas, desc, cas, U, dQ, s, G);
        if (r3) {
            if (G->g3) free_grid3((Grid3*)G->g3);
            cudaFree(G->status);
            free_streams(G);
            delete G;
            return r3;
        }
        hyp_state* st = new hyp_state();
        st->grid = G;
        st->U = U;
        st->dQ = dQ;
        *out = st;
        return HYP_OK;
    }
    const Dims& d = G->d;
    const int nx = d.nx, ny = d.ny;
    const long long nc = d.size(NC), nxf = d.size(NXF), nyf = d.size(NYF), ncn = d.size(NCN);
    long long o = 0;
    for (int f = 0; f < NSP + 1; ++f) {
        G->off[f] = o;
        o += nc;
    }
    G->off[NSP + 1] = o;
    o += nxf;
    G->off[NSP + 2] = o;
    o += nyf;
    G->nstate = (int)o;
    const long long ns_ = o;
    G->Tw_nd = cas->T_wall / g.T_ref;

    // ---------------- host set-up: metrics, sponge, reference, initial state ----------------
    std::vector<double> xc(nx), xf(nx + 1), yc(ny), yf(ny + 1), xi_c(nx), xi_f(nx + 1),
        eta_c(ny), eta_f(ny + 1);
    const double dx = (desc->x1 - desc->x0) / nx;
    for (int i = 0; i <= nx; ++i) {
        xf[i] = desc->x0 + dx * i;
        xi_f[i] = 1.0 / dx;
    }
    for (int i = 0; i < nx; ++i) {
        xc[i] = desc->x0 + dx * (i + 0.5);
        xi_c[i] = 1.0 / dx;
    }
    for (int j = 0; j <= ny; ++j) {
        double y, dy;
        y_map(*desc, (double)j, y, dy);
        yf[j] = y;
        eta_f[j] = 1.0 / dy;
    }
    for (int j = 0; j < ny; ++j) {
        double y, dy;
        y_map(*desc, j + 0.5, y, dy);
        yc[j] = y;
        eta_c[j] = 1.0 / dy;
    }
    Profile P;
    P.c = *cas;
    P.c.noise = nullptr;
    P.y0 = desc->y0;
    P.iN2 = P.iO2 = P.iNO = P.iN = P.iO = -1;
    for (int sp = 0; sp < NSP; ++sp) {
        const std::string& nm = gas->names[sp];
        if (nm == "N2") P.iN2 = sp;
        if (nm == "O2") P.iO2 = sp;
        if (nm == "NO") P.iNO = sp;
        if (nm == "N") P.iN = sp;
        if (nm == "O") P.iO = sp;
        P.Yinf[sp] = 0.0;
    }
    P.shock = cas->flow == 1;
    P.theta = cas->shock_deflection_deg * 3.14159265358979323846 / 180.0;
    if (P.shock) P.sh = oblique_shock(g.mach, P.theta, g.gamma_inf);
    for (int sp = 0; sp < NSP; ++sp) P.Yinf[sp] = g.Y_inf[sp];
    // ---------------- device memory ----------------
    const long long n_c_fields = 13 + 9 * NSP + 13 + 2 * AD_FIELDS;
    const long long n_xf_fields = 2 + 6 * NSP + 8 + 3;
    const long long n_yf_fields = 2 + 6 * NSP + 8;
    const long long n_cn_fields = 8;
    const long long pool_n = n_c_fields * nc + n_xf_fields * nxf + n_yf_fields * nyf +
                             n_cn_fields * ncn + 6 * ns_ + (2 * nx + 1) + (2 * ny + 1) + 4;
    cudaError_t err = cudaMalloc(&G->pool, pool_n * sizeof(double));
    // cleared once: entries a kernel reads before any kernel writes them (fields of held boundary
    // rows, for instance) then read as zero on every grid, whatever the allocation held before
    if (err == cudaSuccess) err = cudaMemsetAsync(G->pool, 0, pool_n * sizeof(double), s);
    if (err != cudaSuccess) {
        free_grid(G);
        return cuda_fail(err, "cudaMalloc(grid pool)");
    }
    double* cur = G->pool;
    auto take = [&](long long n) {
        double* p = cur;
        cur += n;
        return p;
    };
    Scratch& S = G->s;
    double** cfields[] = {&S.ru_c, &S.rv_c, &S.T, &S.p, &S.H, &S.u_c, &S.v_c, &S.e, &S.a,
                          &S.mu_e, &S.K, &S.beta, &S.Tcache};
    for (double** f : cfields) *f = take(nc);
    for (int sp = 0; sp < NSP; ++sp) {
        S.esc[sp] = take(nc);
        S.cvsc[sp] = take(nc);
        S.cvpc[sp] = take(nc);
        S.Y[sp] = take(nc);
        S.X[sp] = take(nc);
        S.h[sp] = take(nc);
        S.Wd[sp] = take(nc);
        S.W[sp] = take(nc);
        S.G[sp] = take(nc);
    }
    double** c2[] = {&S.dudx, &S.dvdy, &S.tau_xx, &S.tau_yy, &S.Gxx, &S.Gyy, &S.mux_c, &S.mvy_c,
                     &S.dudy_c, &S.dvdx_c, &S.S, &S.div, &S.fsw};
    for (double** f : c2) *f = take(nc);
    for (int q = 0; q < AD_FIELDS; ++q) {
        S.raw[q] = take(nc);
        S.filt[q] = take(nc);
    }
    double** xfields[] = {&S.rho_xf, &S.u_xf, &S.Hx, &S.Kx, &S.txx_x, &S.v_x, &S.dTdx, &S.txy_x,
                          &S.FEx, &S.mu_xf, &S.dudy_t, &S.dvdx_t, &S.mux_f, &S.Tx, &S.px};
    for (double** f : xfields) *f = take(nxf);
    for (int sp = 0; sp < NSP; ++sp) {
        S.Yx[sp] = take(nxf);
        S.Gx[sp] = take(nxf);
        S.hx[sp] = take(nxf);
        S.dXdx[sp] = take(nxf);
        S.Fsx[sp] = take(nxf);
    }
    double** yfields[] = {&S.rho_yf, &S.v_yf, &S.Hy, &S.Ky, &S.tyy_y, &S.u_y, &S.dTdy, &S.txy_y,
                          &S.FEy, &S.mvy_f, &S.Ty, &S.py};
    for (double** f : yfields) *f = take(nyf);
    for (int sp = 0; sp < NSP; ++sp) {
        S.Yy[sp] = take(nyf);
        S.Gy[sp] = take(nyf);
        S.hy[sp] = take(nyf);
        S.dXdy[sp] = take(nyf);
        S.Fsy[sp] = take(nyf);
    }
    double** cnf[] = {&S.dudy_cn, &S.dvdx_cn, &S.u_cn, &S.v_cn, &S.rho_cn, &S.mu_cn, &S.tau_xy,
                      &S.Gxy};
    for (double** f : cnf) *f = take(ncn);
    S.DX = take(ns_);
    S.DY = take(ns_);
    S.SRC = take(ns_);
    S.R = take(ns_);
    G->Uref = take(ns_);
    G->sigma = take(ns_);
    G->xi_c = take(nx);
    G->xi_f = take(nx + 1);
    G->eta_c = take(ny);
    G->eta_f = take(ny + 1);
    if (cur - G->pool > pool_n) {
        free_grid(G);
        return fail(HYP_ERR_ARG, "internal: scratch pool too small");
    }
    err = cudaMalloc(&G->mask, ns_);
    if (err == cudaSuccess) err = cudaMalloc(&G->status, sizeof(unsigned));
    if (err != cudaSuccess) {
        free_grid(G);
        return cuda_fail(err, "cudaMalloc(grid)");
    }
    // operators
    std::vector<double> opdata;
    std::vector<LineOp> hops(NOPS);
    hops[OX_ICF] = make_op(0, 0, nx, 0, opdata);
    hops[OX_DCF] = make_op(1, 0, nx, 0, opdata);
    hops[OX_IFC] = make_op(0, 1, nx, 0, opdata);
    hops[OX_DFC] = make_op(1, 1, nx, 0, opdata);
    hops[OY_ICF] = make_op(0, 0, ny, 0, opdata);
    hops[OY_DCF] = make_op(1, 0, ny, 0, opdata);
    hops[OY_IFC] = make_op(0, 1, ny, 0, opdata);
    hops[OY_DFC] = make_op(1, 1, ny, 0, opdata);
    hops[OY_ICFW] = make_op(0, 0, ny, 1, opdata);
    hops[OY_DCFW] = make_op(1, 0, ny, 1, opdata);
    err = cudaMalloc(&G->opdata, opdata.size() * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&G->ops, NOPS * sizeof(LineOp));
    if (err != cudaSuccess) {
        free_grid(G);
        return cuda_fail(err, "cudaMalloc(operators)");
    }
    for (auto& op : hops) {
        op.lower = G->opdata + (size_t)op.lower;
        op.cprime = G->opdata + (size_t)op.cprime;
        op.minv = G->opdata + (size_t)op.minv;
        op.wa = G->opdata + (size_t)op.wa;
        op.wb = G->opdata + (size_t)op.wb;
        op.lm = G->opdata + (size_t)op.lm;
    }
    // plans
    PlanBuilder B;
    B.G = G;
    B.dops = G->ops;
    B.hops = hops.data();
    const bool wall = cas->wall != 0;
    const OpId y_icf_u = wall ? OY_ICFW : OY_ICF;
    const OpId y_dcf_u = wall ? OY_DCFW : OY_DCF;
    B.begin(PH_P3);
    B.add(OX_DFC, S.u_xf, NXF, S.dudx, NC, G->xi_c);
    B.add(OY_DFC, S.v_yf, NYF, S.dvdy, NC, G->eta_c);
    B.add(y_dcf_u, S.u_xf, NXF, S.dudy_cn, NCN, G->eta_f, 1.0, 0.0);
    B.add(OX_DCF, S.v_yf, NYF, S.dvdx_cn, NCN, G->xi_f);
    B.add(y_icf_u, S.u_xf, NXF, S.u_cn, NCN, nullptr, 1.0, 0.0);
    B.add(OX_ICF, S.v_yf, NYF, S.v_cn, NCN, nullptr);
    B.add(OY_ICF, S.rho_xf, NXF, S.rho_cn, NCN, nullptr);
    B.add(OX_IFC, S.mux_f, NXF, S.mux_c, NC, nullptr);
    B.add(OY_IFC, S.mvy_f, NYF, S.mvy_c, NC, nullptr);
    // (the velocity gradients feed the artificial-diffusivity sensors, whose fourth differences
    // would amplify binary32 rounding: they stay FP64 in every mode)
    B.begin(PH_AD1);
    B.add(OY_IFC, S.dudy_cn, NCN, S.dudy_t, NXF, nullptr);
    B.add(OY_IFC, S.dvdx_cn, NCN, S.dvdx_t, NXF, nullptr);
    B.begin(PH_AD2);
    B.add(OX_IFC, S.dudy_t, NXF, S.dudy_c, NC, nullptr);
    B.add(OX_IFC, S.dvdx_t, NXF, S.dvdx_c, NC, nullptr);
    B.begin(PH_MU1);
    B.add(OX_ICF, S.mu_e, NC, S.mu_xf, NXF, nullptr);
    B.f32();
    B.begin(PH_MU2);
    B.add(OY_ICF, S.mu_xf, NXF, S.mu_cn, NCN, nullptr);
    B.f32();
    B.begin(PH_FACE);
    for (int sp = 0; sp < NSP; ++sp) {
        B.add(OX_ICF, S.Y[sp], NC, S.Yx[sp], NXF, nullptr);
        B.add(OX_ICF, S.G[sp], NC, S.Gx[sp], NXF, nullptr);
        B.f32();
        B.add(OX_ICF, S.h[sp], NC, S.hx[sp], NXF, nullptr);
        B.f32();
        B.add(OX_DCF, S.X[sp], NC, S.dXdx[sp], NXF, G->xi_f);
        B.f32();
        B.add(OY_ICF, S.Y[sp], NC, S.Yy[sp], NYF, nullptr);
        B.add(OY_ICF, S.G[sp], NC, S.Gy[sp], NYF, nullptr);
        B.f32();
        B.add(OY_ICF, S.h[sp], NC, S.hy[sp], NYF, nullptr);
        B.f32();
        B.add(OY_DCF, S.X[sp], NC, S.dXdy[sp], NYF, G->eta_f);
        B.f32();
    }
    B.add(OX_ICF, S.H, NC, S.Hx, NXF, nullptr);
    B.add(OX_ICF, S.K, NC, S.Kx, NXF, nullptr);
    B.f32();
    B.add(OX_ICF, S.tau_xx, NC, S.txx_x, NXF, nullptr);
    B.f32();
    B.add(OX_ICF, S.v_c, NC, S.v_x, NXF, nullptr);
    B.f32();
    B.add(OX_DCF, S.T, NC, S.dTdx, NXF, G->xi_f);
    B.f32();
    B.add(OY_ICF, S.H, NC, S.Hy, NYF, nullptr);
    B.add(OY_ICF, S.K, NC, S.Ky, NYF, nullptr);
    B.f32();
    B.add(OY_ICF, S.tau_yy, NC, S.tyy_y, NYF, nullptr);
    B.f32();
    B.add(y_icf_u, S.u_c, NC, S.u_y, NYF, nullptr, 1.0, 0.0);
    B.f32();
    B.add(wall ? OY_DCFW : OY_DCF, S.T, NC, S.dTdy, NYF, G->eta_f, 1.0, G->Tw_nd);
    B.f32();
    if (G->view().sm) {
        // face temperature and pressure for the binary coefficients of Eq. (17)
        B.add(OX_ICF, S.T, NC, S.Tx, NXF, nullptr);
        B.f32();
        B.add(OX_ICF, S.p, NC, S.px, NXF, nullptr);
        B.f32();
        B.add(OY_ICF, S.T, NC, S.Ty, NYF, nullptr);
        B.f32();
        B.add(OY_ICF, S.p, NC, S.py, NYF, nullptr);
        B.f32();
    }
    B.begin(PH_FACEB);
    B.add(OY_IFC, S.tau_xy, NCN, S.txy_x, NXF, nullptr);
    B.f32();
    B.add(OX_IFC, S.tau_xy, NCN, S.txy_y, NYF, nullptr);
    B.f32();
    B.begin(PH_DIV);
    for (int sp = 1; sp < NSP; ++sp) {
        B.add(OX_DFC, S.Fsx[sp], NXF, S.DX + G->off[sp], NC, G->xi_c, -1.0);
        B.add(OY_DFC, S.Fsy[sp], NYF, S.DY + G->off[sp], NC, G->eta_c, -1.0);
    }
    B.add(OX_DFC, S.FEx, NXF, S.DX + G->off[NSP], NC, G->xi_c, -1.0);
    B.add(OY_DFC, S.FEy, NYF, S.DY + G->off[NSP], NC, G->eta_c, -1.0);
    B.add(OX_DCF, S.Gxx, NC, S.DX + G->off[NSP + 1], NXF, G->xi_f, -1.0);
    B.add(OY_DFC, S.Gxy, NCN, S.DY + G->off[NSP + 1], NXF, G->eta_c, -1.0);
    B.add(OX_DFC, S.Gxy, NCN, S.DX + G->off[NSP + 2], NYF, G->xi_c, -1.0);
    B.add(OY_DCF, S.Gyy, NC, S.DY + G->off[NSP + 2], NYF, G->eta_f, -1.0);
    // jobs reading the state: face momenta to centres, density to faces, continuity divergence
    B.begin(PH_P1);
    auto soff = [&](int f) { return (const double*)(size_t)G->off[f]; };
    B.add(OX_IFC, soff(NSP + 1), NXF, S.ru_c, NC, nullptr, 1.0, 0.0, 1);
    B.add(OY_IFC, soff(NSP + 2), NYF, S.rv_c, NC, nullptr, 1.0, 0.0, 1);
    B.add(OX_ICF, soff(0), NC, S.rho_xf, NXF, nullptr, 1.0, 0.0, 1);
    B.add(OY_ICF, soff(0), NC, S.rho_yf, NYF, nullptr, 1.0, 0.0, 1);
    B.add(OX_DFC, soff(NSP + 1), NXF, S.DX + G->off[0], NC, G->xi_c, -1.0, 0.0, 1);
    B.add(OY_DFC, soff(NSP + 2), NYF, S.DY + G->off[0], NC, G->eta_c, -1.0, 0.0, 1);
    const long long tmp_need = B.finish();
    memcpy(G->ph_start, B.ph_start, sizeof(B.ph_start));
    memcpy(G->ph_count, B.ph_count, sizeof(B.ph_count));
    memcpy(G->ph_blocks, B.ph_blocks, sizeof(B.ph_blocks));
    G->linetmp_n = tmp_need;
    err = cudaMalloc(&G->linetmp, tmp_need * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&G->jobs, B.jobs.size() * sizeof(LineJob));
    if (err != cudaSuccess) {
        free_grid(G);
        return cuda_fail(err, "cudaMalloc(jobs)");
    }
    if (err == cudaSuccess) err = cudaMalloc(&G->metf, (2 * (nx + ny) + 2) * sizeof(float));
    if (err != cudaSuccess) {
        free_grid(G);
        return cuda_fail(err, "cudaMalloc(metrics)");
    }
    std::vector<float> metf_h;
    for (const auto* v : {&xi_c, &xi_f, &eta_c, &eta_f})
        for (double x : *v) metf_h.push_back((float)x);
    const double* met_d[4] = {G->xi_c, G->xi_f, G->eta_c, G->eta_f};
    const long long met_off[4] = {0, nx, 2LL * nx + 1, 2LL * nx + 1 + ny};
    for (auto& j : B.jobs) {
        j.tmp = G->linetmp + (size_t)j.tmp;
        for (int k = 0; k < 4; ++k)
            if (j.metric == met_d[k]) j.metric_f = G->metf + met_off[k];
    }
    // uploads
#define UP(dst, src, bytes) HYP_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s))
    UP(G->opdata, opdata.data(), opdata.size() * sizeof(double));
    UP(G->ops, hops.data(), NOPS * sizeof(LineOp));
    UP(G->jobs, B.jobs.data(), B.jobs.size() * sizeof(LineJob));
    G->hjobs = B.jobs;
    UP(G->metf, metf_h.data(), metf_h.size() * sizeof(float));
    UP(G->xi_c, xi_c.data(), nx * sizeof(double));
    UP(G->xi_f, xi_f.data(), (nx + 1) * sizeof(double));
    UP(G->eta_c, eta_c.data(), ny * sizeof(double));
    UP(G->eta_f, eta_f.data(), (ny + 1) * sizeof(double));
    // reference state, sponge, mask and the initial state, computed on the device; the seeded
    // noise travels through the state-sized scratch vector
    k_reference<<<blocks_for(nc + nxf + nyf, 128), 128, 0, s>>>(g, P, *desc, G->off[NSP + 1],
                                                                 G->off[NSP + 2], G->Uref, G->sigma,
                                                                 G->mask);
    const bool noisy = cas->noise && cas->noise_amp > 0;
    if (noisy) UP(G->s.R, cas->noise, ns_ * sizeof(double));
    k_initial<<<blocks_for(ns_, 256), 256, 0, s>>>(ns_, G->Uref, G->mask, noisy ? G->s.R : nullptr,
                                                   cas->noise_amp, U);
    HYP_CUDA(cudaGetLastError());
#undef UP
    HYP_CUDA(cudaMemsetAsync(dQ, 0, ns_ * sizeof(double), s));
    HYP_CUDA(cudaMemsetAsync(G->s.SRC, 0, ns_ * sizeof(double), s));
    HYP_CUDA(cudaMemsetAsync(G->status, 0, sizeof(unsigned), s));
    k_fill<<<blocks_for(nc, 256), 256, 0, s>>>(G->s.Tcache, nc, 1000.0);
    HYP_CUDA(cudaStreamCreateWithFlags(&G->side, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
        HYP_CUDA(cudaEventCreateWithFlags(&G->fork[k], cudaEventDisableTiming));
        HYP_CUDA(cudaEventCreateWithFlags(&G->join[k], cudaEventDisableTiming));
    }
    {
        int dev = 0, sms = 0, per_sm = 0;
        HYP_CUDA(cudaGetDevice(&dev));
        HYP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const bool lte = gas->dev.kind == HYP_GAS_LTE;
        HYP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, lte ? k_closure<false, true> : k_closure<false, false>, 128, 0));
        G->closure_blocks = std::max(1, per_sm * sms);
        HYP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, lte ? k_closure<true, true> : k_closure<true, false>, 128, 0));
        G->closure_blocks_mixed = std::max(1, per_sm * sms);
    }
    HYP_CUDA(cudaGetLastError());
    // host vectors must outlive the async copies
    HYP_CUDA(cudaStreamSynchronize(s));
    hyp_state* st = new hyp_state();
    st->grid = G;
    st->U = U;
    st->dQ = dQ;
    *out = st;
    return HYP_OK;
}

extern "C" const hyp_grid* hyp_state_grid(const hyp_state* st) { return st ? st->grid : nullptr; }

extern "C" void hyp_state_free(hyp_state* st) {
    if (!st) return;
    free_grid(st->grid);
    delete st;
}

extern "C" int hyp_grid_reference(const hyp_grid* G, double* Uref, double* sigma) {
    if (!G) return fail(HYP_ERR_ARG, "null grid");
    HYP_CUDA(cudaStreamSynchronize(G->stream));
    if (Uref) HYP_CUDA(cudaMemcpy(Uref, G->Uref, G->nstate * sizeof(double), cudaMemcpyDeviceToHost));
    if (sigma) HYP_CUDA(cudaMemcpy(sigma, G->sigma, G->nstate * sizeof(double), cudaMemcpyDeviceToHost));
    return HYP_OK;
}

extern "C" int hyp_grid_status(const hyp_grid* G, uint32_t* flags, int clear) {
    if (!G || !flags) return fail(HYP_ERR_ARG, "null argument");
    HYP_CUDA(cudaStreamSynchronize(G->stream));
    unsigned v = 0;
    HYP_CUDA(cudaMemcpy(&v, G->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    *flags = v;
    if (clear) HYP_CUDA(cudaMemset(G->status, 0, sizeof(unsigned)));
    return HYP_OK;
}

#define TIMED_ON(st, kid, ...)                        \
    do {                                              \
        const int _slot = prof_begin(G, kid, st);     \
        __VA_ARGS__;                                  \
        prof_end(G, _slot, st);                       \
    } while (0)
#define TIMED(kid, ...) TIMED_ON(s, kid, __VA_ARGS__)

// The whole right-hand side; with rk != 0 the assemble step performs the stage update instead
// of writing dUdt.
static int run_rhs(const hyp_gas* gas, hyp_grid* G, const double* U, double* dUdt, int rk,
                   double A, double Bc, double dt, double* Urk, double* dQ, int precision,
                   cudaStream_t s) {
    const GasDev& g = gas->dev;
    const GridView v = G->view();
    Scratch& S = G->s;
    const Dims& d = G->d;
    const long long nc = d.size(NC);
    cudaError_t e1 = cudaSuccess;
    const bool mixed = precision == HYP_MIXED;
    const int mx = mixed ? 1 : 0;
    TIMED(KID_LINES_STATE, e1 = launch_lines(G->jobs + G->ph_start[PH_P1], G->ph_count[PH_P1],
                                             G->ph_blocks[PH_P1], U, s, mx));
    HYP_CUDA(e1);
    TIMED(KID_FACE_VEL, (k_face_vel<<<blocks_for(d.size(NXF) + d.size(NYF), 256), 256, 0, s>>>(v, U, S)));
    // fork: velocity gradients and the artificial-diffusivity line phases do not need the closure
    cudaStream_t s2 = G->side;
    HYP_CUDA(cudaEventRecord(G->fork[0], s));
    HYP_CUDA(cudaStreamWaitEvent(s2, G->fork[0], 0));
    const int cb = (int)std::min<long long>(mixed ? G->closure_blocks_mixed : G->closure_blocks,
                                            (nc + 127) / 128);
    const Scales sc = scales_of(g);
    TIMED(KID_CLOSURE, launch_closure(g, sc, v, U, S, mixed, cb, s));
    HYP_CUDA(cudaGetLastError());
    G->cache_valid = 1;
    TIMED_ON(s2, KID_LINES_VELGRAD, e1 = launch_lines(G->jobs + G->ph_start[PH_P3], G->ph_count[PH_P3],
                                                      G->ph_blocks[PH_P3], U, s2, mx));
    HYP_CUDA(e1);
    if (v.ad) {
        // the two small interpolation phases of the sensors' cross derivatives run in binary64 in
        // both precisions: with two jobs their lines cannot fill the GPU, and at that occupancy the
        // binary64 recurrence (one FMA per row on its chain) beats the double-word one
        TIMED_ON(s2, KID_LINES_AD, e1 = launch_lines(G->jobs + G->ph_start[PH_AD1], 2, G->ph_blocks[PH_AD1], U, s2, 0));
        HYP_CUDA(e1);
        TIMED_ON(s2, KID_LINES_AD, e1 = launch_lines(G->jobs + G->ph_start[PH_AD2], 2, G->ph_blocks[PH_AD2], U, s2, 0));
        HYP_CUDA(e1);
        TIMED_ON(s2, KID_AD_PREP, (k_ad_prep<<<blocks_for(nc, 256), 256, 0, s2>>>(v, S)));
    }
    HYP_CUDA(cudaEventRecord(G->join[0], s2));
    HYP_CUDA(cudaStreamWaitEvent(s, G->join[0], 0));
    if (v.ad) {
        TIMED(KID_AD_RAW, (k_ad_raw<<<blocks_for(nc, 256), 256, 0, s>>>(g.kind == HYP_GAS_CNEQ, v, U, S)));
        const int gg = blocks_for(mixed ? nc : AD_FIELDS * nc, 256);
        if (mixed) {
            TIMED(KID_AD_GAUSS, (k_gauss<true><<<gg, 256, 0, s>>>(v, S, 0)));
            TIMED(KID_AD_GAUSS, (k_gauss<true><<<gg, 256, 0, s>>>(v, S, 1)));
        } else {
            TIMED(KID_AD_GAUSS, (k_gauss<false><<<gg, 256, 0, s>>>(v, S, 0)));
            TIMED(KID_AD_GAUSS, (k_gauss<false><<<gg, 256, 0, s>>>(v, S, 1)));
        }
        TIMED(KID_AD_COMBINE, (k_ad_combine<<<blocks_for(nc, 256), 256, 0, s>>>(v, S)));
        HYP_CUDA(cudaGetLastError());
    }
    TIMED(KID_STRESS_C, (k_stress_c<<<blocks_for(nc, 256), 256, 0, s>>>(v, S)));
    // fork: viscosity to the corners, shear stress and its face interpolants beside the face phase
    HYP_CUDA(cudaEventRecord(G->fork[1], s));
    HYP_CUDA(cudaStreamWaitEvent(s2, G->fork[1], 0));
    TIMED_ON(s2, KID_LINES_MU, e1 = launch_lines(G->jobs + G->ph_start[PH_MU1], 1, G->ph_blocks[PH_MU1], U, s2, mx));
    HYP_CUDA(e1);
    TIMED_ON(s2, KID_LINES_MU, e1 = launch_lines(G->jobs + G->ph_start[PH_MU2], 1, G->ph_blocks[PH_MU2], U, s2, mx));
    HYP_CUDA(e1);
    TIMED_ON(s2, KID_STRESS_CN, (k_stress_cn<<<blocks_for(d.size(NCN), 256), 256, 0, s2>>>(v, S)));
    TIMED_ON(s2, KID_LINES_FACE, e1 = launch_lines(G->jobs + G->ph_start[PH_FACEB], G->ph_count[PH_FACEB],
                                                   G->ph_blocks[PH_FACEB], U, s2, mx));
    HYP_CUDA(e1);
    HYP_CUDA(cudaEventRecord(G->join[1], s2));
    TIMED(KID_LINES_FACE, e1 = launch_lines(G->jobs + G->ph_start[PH_FACE], G->ph_count[PH_FACE],
                                            G->ph_blocks[PH_FACE], U, s, mx));
    HYP_CUDA(e1);
    HYP_CUDA(cudaStreamWaitEvent(s, G->join[1], 0));
    if (v.sm) {
        TIMED(KID_FLUX, (k_flux<true><<<blocks_for(d.size(NXF), 128), 128, 0, s>>>(g, sc, v, U, S, 0)));
        TIMED(KID_FLUX, (k_flux<true><<<blocks_for(d.size(NYF), 128), 128, 0, s>>>(g, sc, v, U, S, 1)));
    } else {
        TIMED(KID_FLUX, (k_flux<false><<<blocks_for(d.size(NXF), 128), 128, 0, s>>>(g, sc, v, U, S, 0)));
        TIMED(KID_FLUX, (k_flux<false><<<blocks_for(d.size(NYF), 128), 128, 0, s>>>(g, sc, v, U, S, 1)));
    }
    TIMED(KID_LINES_DIV, e1 = launch_lines(G->jobs + G->ph_start[PH_DIV], G->ph_count[PH_DIV],
                                           G->ph_blocks[PH_DIV], U, s, mx));
    HYP_CUDA(e1);
    const AssembleArgs aa{S.DX, S.DY, S.SRC, G->sigma, G->Uref, G->mask,
                          rk ? Urk : (double*)U, dUdt, dQ, rk, A, Bc, dt};
    TIMED(KID_ASSEMBLE, (k_assemble<<<blocks_for(G->nstate, 256), 256, 0, s>>>(G->nstate, aa)));
    HYP_CUDA(cudaGetLastError());
    return HYP_OK;
}

extern "C" int hyp_rhs(const hyp_gas* gas, const hyp_grid* grid, const double* U, double* dUdt,
                       int precision, void* stream) {
    if (!gas || !grid || !U || !dUdt) return fail(HYP_ERR_ARG, "null argument");
    if (precision != HYP_FP64 && precision != HYP_MIXED) return fail(HYP_ERR_ARG, "unknown precision");
    if (U == dUdt) return fail(HYP_ERR_ARG, "U and dUdt must not alias");
    hyp_grid* G = const_cast<hyp_grid*>(grid);
    if (G->g3)
        return run_rhs3(gas, G, U, dUdt, 0, 0.0, 0.0, 0.0, nullptr, nullptr, precision,
                        (cudaStream_t)stream);
    return run_rhs(gas, G, U, dUdt, 0, 0.0, 0.0, 0.0, nullptr, nullptr, precision,
                   (cudaStream_t)stream);
}

extern "C" int hyp_grid_temperature(const hyp_grid* grid, int64_t n_T, double* T, void* stream) {
    if (!grid || !T) return fail(HYP_ERR_ARG, "null argument");
    const Grid3* g3 = static_cast<const Grid3*>(grid->g3);
    const int valid = g3 ? g3->cache_valid : grid->cache_valid;
    if (!valid) return fail(HYP_ERR_ARG, "no closure has been evaluated on this grid");
    const double* src = g3 ? g3->Tcache : grid->s.Tcache;
    const long long n = g3 ? g3->nc : (long long)grid->d.nx * grid->d.ny;
    if (n_T != n) return fail(HYP_ERR_ARG, "T must hold one double per cell centre");
    HYP_CUDA(cudaMemcpyAsync(T, src, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
    return HYP_OK;
}

// The state filter after the last RK stage: x pass into the scratch state vector, y pass back.
static int launch_filter(hyp_grid* G, double* U, cudaStream_t s) {
    const double sigma = G->cas.filter_sigma;
    const int blocks = blocks_for(G->nstate, 256);
    TIMED(KID_FILTER, (k_filter<<<blocks, 256, 0, s>>>(G->d.nx, G->d.ny, G->nstate, U, G->s.R, 0, sigma)));
    TIMED(KID_FILTER, (k_filter<<<blocks, 256, 0, s>>>(G->d.nx, G->d.ny, G->nstate, G->s.R, U, 1, sigma)));
    HYP_CUDA(cudaGetLastError());
    return HYP_OK;
}

// Coefficients of the other schemes of Sec. 3.1: TVD RK3 (Shu-Osher) weights of the start state
// and of the Euler update, and the (5,4) 2N-storage RK4 of Carpenter and Kennedy.
constexpr double TVD3_W[3] = {0.0, 3.0 / 4.0, 1.0 / 3.0};
constexpr double TVD3_S[3] = {1.0, 1.0 / 4.0, 2.0 / 3.0};
constexpr double CK4_A[5] = {0.0, -567301805773.0 / 1357537059087.0,
                             -2404267990393.0 / 2016746695238.0,
                             -3550918686646.0 / 2091501179385.0,
                             -1275806237668.0 / 842570457699.0};
constexpr double CK4_B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                             1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                             2277821191437.0 / 14882151754819.0};

extern "C" int hyp_rk_stage_scheme(hyp_state* st, int scheme, int stage, double dt, int precision,
                                   void* stream) {
    if (!st) return fail(HYP_ERR_ARG, "null state");
    if (scheme < HYP_RK3_2N || scheme > HYP_RK4_2N) return fail(HYP_ERR_ARG, "unknown scheme");
    const int nst = scheme == HYP_RK4_2N ? 5 : 3;
    if (stage < 0 || stage >= nst) return fail(HYP_ERR_ARG, "stage out of range for the scheme");
    if (precision != HYP_FP64 && precision != HYP_MIXED) return fail(HYP_ERR_ARG, "unknown precision");
    hyp_grid* G = st->grid;
    // the gas handle is not stored in the state: the grid keeps a copy of the device tables
    hyp_gas tmp;
    tmp.dev = G->gas;
    if (G->g3) {
        if (scheme != HYP_RK3_2N) return fail(HYP_ERR_ARG, "three-dimensional grids step the two-register RK3");
        return run_rhs3(&tmp, G, st->U, nullptr, 1, RK_A[stage], RK_B[stage], dt, st->U, st->dQ,
                        precision, (cudaStream_t)stream);
    }
    int mode = 1;
    double A = RK_A[stage < 3 ? stage : 0], B = RK_B[stage < 3 ? stage : 0];
    if (scheme == HYP_RK3_TVD) {
        mode = stage == 0 ? 3 : 2;
        A = TVD3_W[stage];
        B = TVD3_S[stage];
    } else if (scheme == HYP_RK4_2N) {
        A = CK4_A[stage];
        B = CK4_B[stage];
    }
    const int rc = run_rhs(&tmp, G, st->U, nullptr, mode, A, B, dt, st->U, st->dQ, precision,
                           (cudaStream_t)stream);
    if (rc || stage != nst - 1 || !(G->cas.filter_sigma > 0.0)) return rc;
    return launch_filter(G, st->U, (cudaStream_t)stream);
}

extern "C" int hyp_rk_stage(hyp_state* st, int stage, double dt, int precision, void* stream) {
    if (st && (stage < 0 || stage > 2)) return fail(HYP_ERR_ARG, "stage must be 0, 1 or 2");
    return hyp_rk_stage_scheme(st, HYP_RK3_2N, stage, dt, precision, stream);
}

// Wall heat flux q_w = -K dT/dy and wall shear stress tau_w = tau_xy on the wall row of the
// scratch left by the right-hand side just evaluated (the same face and corner values that enter
// the fluxes of Eq. 10 and Eq. 9).
__global__ void k_wall_out(GridView v, Scratch s, double* __restrict__ q_w,
                           double* __restrict__ tau_w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < v.nx) q_w[i] = -s.Ky[i] * s.dTdy[i];
    if (i <= v.nx) tau_w[i] = s.tau_xy[i];
}

extern "C" int hyp_wall_fluxes(const hyp_gas* gas, const hyp_grid* grid, const double* U,
                               double* q_w, double* tau_w, int precision, void* stream) {
    if (!gas || !grid || !U || !q_w || !tau_w) return fail(HYP_ERR_ARG, "null argument");
    if (precision != HYP_FP64 && precision != HYP_MIXED) return fail(HYP_ERR_ARG, "unknown precision");
    hyp_grid* G = const_cast<hyp_grid*>(grid);
    if (G->g3) return fail(HYP_ERR_ARG, "hyp_wall_fluxes takes two-dimensional grids");
    const GridView v = G->view();
    if (!v.wall) return fail(HYP_ERR_ARG, "the case has no wall");
    cudaStream_t s = (cudaStream_t)stream;
    const int rc = run_rhs(gas, G, U, G->s.R, 0, 0.0, 0.0, 0.0, nullptr, nullptr, precision, s);
    if (rc) return rc;
    k_wall_out<<<(v.nx + 1 + 127) / 128, 128, 0, s>>>(v, G->s, q_w, tau_w);
    HYP_CUDA(cudaGetLastError());
    return HYP_OK;
}

// The binary64 -> binary32 -> binary64 round trip of the mixed-precision path (fp32.cuh).
__global__ void k_round_f32(int64_t n, const double* __restrict__ x, float* __restrict__ y,
                            double* __restrict__ back) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float f = f32_of(x[i]);
        if (y) y[i] = f;
        if (back) back[i] = f64_of(f);
    }
}

extern "C" int hyp_round_f32(int64_t n, const double* x, float* y, double* back, void* stream) {
    if (n < 0 || (n > 0 && !x)) return fail(HYP_ERR_ARG, "null input or negative n");
    if (n == 0) return HYP_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_round_f32<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(n, x, y, back);
    HYP_CUDA(cudaGetLastError());
    return HYP_OK;
}

// The binary64 exponential, quotient and reciprocal of the closure (fp64_fast.cuh), one per
// element: fn 0 out = exp(a), 1 out = a / b, 2 out = 1 / b.
__global__ void k_fp64_fast(int fn, int64_t n, const double* __restrict__ a,
                            const double* __restrict__ b, double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (fn == 0) out[i] = tang_exp(a[i]);
        else if (fn == 1) out[i] = fast_div(a[i], b[i]);
        else if (fn == 2) out[i] = fast_rcp(b[i]);
        else out[i] = table_log(a[i]);
    }
}

extern "C" int hyp_fp64_fast(int fn, int64_t n, const double* a, const double* b, double* out,
                             void* stream) {
    if (fn < 0 || fn > 3 || n < 0) return fail(HYP_ERR_ARG, "unknown function or negative n");
    if (n > 0 && (!out || ((fn <= 1 || fn == 3) && !a) || ((fn == 1 || fn == 2) && !b)))
        return fail(HYP_ERR_ARG, "null argument");
    if (n == 0) return HYP_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_fp64_fast<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(fn, n, a, b, out);
    HYP_CUDA(cudaGetLastError());
    return HYP_OK;
}

extern "C" int hyp_profile_count(void) { return KID_COUNT; }

extern "C" const char* hyp_profile_name(int id) {
    return (id >= 0 && id < KID_COUNT) ? KERNEL_NAMES[id] : "";
}

extern "C" int hyp_grid_profile(const hyp_grid* grid, int enable) {
    if (!grid) return fail(HYP_ERR_ARG, "null grid");
    hyp_grid* G = const_cast<hyp_grid*>(grid);
    if (!G->prof) G->prof = new EventProfile();
    EventProfile* P = G->prof;
    if (enable) {
        HYP_CUDA(cudaStreamSynchronize(G->stream));
        P->used = 0;
        for (int k = 0; k < KID_COUNT; ++k) {
            P->ms[k] = 0.0;
            P->count[k] = 0;
        }
    }
    P->on = enable != 0;
    return HYP_OK;
}

extern "C" int hyp_grid_profile_read(const hyp_grid* grid, int n, double* ms, int64_t* launches) {
    if (!grid || n < 0) return fail(HYP_ERR_ARG, "bad argument");
    hyp_grid* G = const_cast<hyp_grid*>(grid);
    EventProfile* P = G->prof;
    if (P) {
        for (size_t slot = 0; slot < P->used; slot += 2) {
            HYP_CUDA(cudaEventSynchronize(P->ev[slot + 1]));
            float t = 0.0f;
            HYP_CUDA(cudaEventElapsedTime(&t, P->ev[slot], P->ev[slot + 1]));
            P->ms[P->id[slot / 2]] += t;
            P->count[P->id[slot / 2]] += 1;
        }
        P->used = 0;
    }
    for (int k = 0; k < n && k < KID_COUNT; ++k) {
        if (ms) ms[k] = P ? P->ms[k] : 0.0;
        if (launches) launches[k] = P ? P->count[k] : 0;
    }
    return HYP_OK;
}

// ---------------------------------------------------------------------------------------------
// hyp_rhs_noalloc: the right-hand side with all per-call scratch in one static device array.
//
// Some callers may not allocate device memory once they are running: real-time solver loops that
// forbid allocation after start-up, and hosts (simulation frameworks, language runtimes, plug-in
// hosts) that own all device memory through their own allocator and do not let a library call
// cudaMalloc behind their back. hyp_rhs never allocates either, but it keeps its scratch inside
// the grid handle, which the grid allocated when it was built; this variant instead takes every
// scratch field, the line-sweep storage and its launch plan from the file-scope array below, so a
// grid's scratch is not touched. The grid's read-only data (metrics, reference state, sponge,
// operators) are used as is, and the per-point status bits go to the grid's status word.
// ---------------------------------------------------------------------------------------------

#define HYP_NOALLOC_DOUBLES (3LL << 19)   // 1,572,864 doubles = 12 MiB per GPU
#define HYP_NOALLOC_MAX_JOBS 160
#define HYP_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_noalloc_scratch[HYP_NOALLOC_DOUBLES];
static double* g_noalloc_base[HYP_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

// Copy of a launch plan whose field pointers into the grid's scratch pool or line-sweep storage
// are moved to the same offsets in the static array (one thread per job).
__global__ void k_relocate_jobs(const LineJob* __restrict__ src, LineJob* __restrict__ dst, int n,
                                const double* pool, long long pool_n, const double* linetmp,
                                long long linetmp_n, double* base, double* tmp_base) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    auto relocate = [&](const double* p) -> double* {
        if (p >= pool && p < pool + pool_n) return base + (p - pool);
        if (p >= linetmp && p < linetmp + linetmp_n) return tmp_base + (p - linetmp);
        return const_cast<double*>(p);
    };
    LineJob j = src[k];
    if (!j.in_state) j.in = relocate(j.in);
    j.out = relocate(j.out);
    j.tmp = relocate(j.tmp);
    dst[k] = j;
}

// Device address of the static array on the current device, looked up once per device. The
// array's name in host code is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with the device current.
static int noalloc_base(double** base) {
    int dev = 0;
    HYP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= HYP_NOALLOC_MAX_DEVICES) return fail(HYP_ERR_ARG, "device index too large");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_base[dev]) {
        void* p = nullptr;
        HYP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_base[dev] = (double*)p;
    }
    *base = g_noalloc_base[dev];
    return HYP_OK;
}

extern "C" int hyp_rhs_noalloc(const hyp_gas* gas, const hyp_grid* grid, const double* U,
                               double* dUdt, void* stream) {
    if (!gas || !grid || !U || !dUdt) return fail(HYP_ERR_ARG, "null argument");
    if (U == dUdt) return fail(HYP_ERR_ARG, "U and dUdt must not alias");
    hyp_grid* G = const_cast<hyp_grid*>(grid);
    if (G->g3) return fail(HYP_ERR_ARG, "hyp_rhs_noalloc takes two-dimensional grids");
    cudaStream_t s = (cudaStream_t)stream;
    int njobs = 0;
    for (int ph = 0; ph < PH_COUNT; ++ph) njobs = std::max(njobs, G->ph_start[ph] + G->ph_count[ph]);
    const long long scratch_n = G->Uref - G->pool;    // scratch fields, DX, DY, SRC, R
    const long long jobs_n = ((long long)njobs * (long long)sizeof(LineJob) + 255) / 256 * 32;
    const long long need = scratch_n + G->linetmp_n + jobs_n;
    if (njobs > HYP_NOALLOC_MAX_JOBS || need > HYP_NOALLOC_DOUBLES)
        return fail(HYP_ERR_ARG, "grid too large for hyp_rhs_noalloc: needs " +
                                     std::to_string(need) + " doubles of scratch, the static array holds " +
                                     std::to_string((long long)HYP_NOALLOC_DOUBLES));
    double* base = nullptr;
    int rc = noalloc_base(&base);
    if (rc) return rc;
    double* tmp_base = base + scratch_n;
    LineJob* djobs = (LineJob*)(base + scratch_n + G->linetmp_n);
    auto relocate = [&](const double* p) -> double* {
        if (p >= G->pool && p < G->pool + scratch_n) return base + (p - G->pool);
        if (p >= G->linetmp && p < G->linetmp + G->linetmp_n) return tmp_base + (p - G->linetmp);
        return const_cast<double*>(p);
    };
    // the grid's launch plan, copied on the device with its scratch pointers moved into the
    // static array (no host buffer, no synchronisation)
    k_relocate_jobs<<<blocks_for(njobs, 64), 64, 0, s>>>(G->jobs, djobs, njobs, G->pool, scratch_n,
                                                         G->linetmp, G->linetmp_n, base, tmp_base);
    HYP_CUDA(cudaGetLastError());
    Scratch S = G->s;
    double** fields = reinterpret_cast<double**>(&S);
    for (size_t k = 0; k < sizeof(Scratch) / sizeof(double*); ++k) fields[k] = relocate(fields[k]);
    // every call starts from cleared scratch, as a newly built grid does (the array keeps the last
    // call's contents, possibly of another grid); the Newton iteration starts at 1000 K
    HYP_CUDA(cudaMemsetAsync(base, 0, (scratch_n + G->linetmp_n) * sizeof(double), s));
    const long long nc = G->d.size(NC);
    k_fill<<<blocks_for(nc, 256), 256, 0, s>>>(S.Tcache, nc, 1000.0);
    HYP_CUDA(cudaGetLastError());

    const GasDev& g = gas->dev;
    GridView v = G->view();
    v.predict = 0;
    const Dims& d = G->d;
    auto lines = [&](int ph, int count) {
        return launch_lines(djobs + G->ph_start[ph], count, G->ph_blocks[ph], U, s);
    };
    HYP_CUDA(lines(PH_P1, G->ph_count[PH_P1]));
    k_face_vel<<<blocks_for(d.size(NXF) + d.size(NYF), 256), 256, 0, s>>>(v, U, S);
    launch_closure(g, scales_of(g), v, U, S, false, (int)blocks_for(nc, 128), s);
    HYP_CUDA(cudaGetLastError());
    HYP_CUDA(lines(PH_P3, G->ph_count[PH_P3]));
    if (v.ad) {
        HYP_CUDA(lines(PH_AD1, 2));
        HYP_CUDA(lines(PH_AD2, 2));
        k_ad_prep<<<blocks_for(nc, 256), 256, 0, s>>>(v, S);
        k_ad_raw<<<blocks_for(nc, 256), 256, 0, s>>>(g.kind == HYP_GAS_CNEQ, v, U, S);
        const int gg = blocks_for(AD_FIELDS * nc, 256);
        k_gauss<false><<<gg, 256, 0, s>>>(v, S, 0);
        k_gauss<false><<<gg, 256, 0, s>>>(v, S, 1);
        k_ad_combine<<<blocks_for(nc, 256), 256, 0, s>>>(v, S);
        HYP_CUDA(cudaGetLastError());
    }
    k_stress_c<<<blocks_for(nc, 256), 256, 0, s>>>(v, S);
    HYP_CUDA(lines(PH_MU1, 1));
    HYP_CUDA(lines(PH_MU2, 1));
    k_stress_cn<<<blocks_for(d.size(NCN), 256), 256, 0, s>>>(v, S);
    HYP_CUDA(lines(PH_FACE, G->ph_count[PH_FACE]));
    HYP_CUDA(lines(PH_FACEB, G->ph_count[PH_FACEB]));
    if (v.sm) {
        k_flux<true><<<blocks_for(d.size(NXF), 128), 128, 0, s>>>(g, scales_of(g), v, U, S, 0);
        k_flux<true><<<blocks_for(d.size(NYF), 128), 128, 0, s>>>(g, scales_of(g), v, U, S, 1);
    } else {
        k_flux<false><<<blocks_for(d.size(NXF), 128), 128, 0, s>>>(g, scales_of(g), v, U, S, 0);
        k_flux<false><<<blocks_for(d.size(NYF), 128), 128, 0, s>>>(g, scales_of(g), v, U, S, 1);
    }
    HYP_CUDA(lines(PH_DIV, G->ph_count[PH_DIV]));
    const AssembleArgs aa{S.DX, S.DY, S.SRC, G->sigma, G->Uref, G->mask, (double*)U, dUdt,
                          nullptr, 0, 0.0, 0.0, 0.0};
    k_assemble<<<blocks_for(G->nstate, 256), 256, 0, s>>>(G->nstate, aa);
    HYP_CUDA(cudaGetLastError());
    return HYP_OK;
}
