// Grid data shared by the single-grid right-hand side (rhs.cu) and the batched executor
// (batch.cu): node layout, scratch fields, the kernel-side grid view, launch phases, and the grid
// and state handles of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

namespace hyp {

inline constexpr double RECOVERY = 0.85;
inline constexpr double DUCROS_EPS = 1.0e-32;
inline constexpr double RK_A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
inline constexpr double RK_B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
// nine-point truncated Gaussian filter weights (centre, +-1, +-2, +-3, +-4)
static __constant__ double c_gauss[5] = {3565.0 / 10368.0, 3091.0 / 12960.0, 1997.0 / 25920.0,
                                  149.0 / 12960.0, 107.0 / 103680.0};
// the same weights rounded to binary32 (the mixed path's filter)
static __constant__ float c_gauss_f[5] = {(float)(3565.0 / 10368.0), (float)(3091.0 / 12960.0),
                                          (float)(1997.0 / 25920.0), (float)(149.0 / 12960.0),
                                          (float)(107.0 / 103680.0)};

enum Node { NC = 0, NXF = 1, NYF = 2, NCN = 3 };

struct Dims {
    int nx, ny;
    int rows(Node t) const { return (t == NC || t == NXF) ? ny : ny + 1; }
    int pitch(Node t) const { return (t == NC || t == NYF) ? nx : nx + 1; }
    long long size(Node t) const { return (long long)rows(t) * pitch(t); }
};

// raw and filtered artificial diffusivities per cell: mu*, beta*, kappa* and D*_s per species
constexpr int AD_FIELDS = 3 + NSP;

struct Scratch {
    // cell centres
    double *ru_c, *rv_c, *T, *p, *H, *u_c, *v_c, *e, *a, *mu_e, *K, *beta, *Tcache;
    double *Y[NSP], *X[NSP], *h[NSP], *Wd[NSP], *W[NSP], *G[NSP];
    double *esc[NSP], *cvsc[NSP], *cvpc[NSP];   // species e, c_v, dc_v/dT at the cached T
    double *dudx, *dvdy, *tau_xx, *tau_yy, *Gxx, *Gyy, *mux_c, *mvy_c;
    double *dudy_c, *dvdx_c, *S, *div, *fsw, *raw[AD_FIELDS], *filt[AD_FIELDS];
    // x-faces
    double *rho_xf, *u_xf, *Yx[NSP], *Gx[NSP], *hx[NSP], *Hx, *Kx, *txx_x, *v_x, *dTdx,
        *dXdx[NSP], *txy_x, *Fsx[NSP], *FEx, *mu_xf, *dudy_t, *dvdx_t, *mux_f, *Tx, *px;
    // y-faces
    double *rho_yf, *v_yf, *Yy[NSP], *Gy[NSP], *hy[NSP], *Hy, *Ky, *tyy_y, *u_y, *dTdy,
        *dXdy[NSP], *txy_y, *Fsy[NSP], *FEy, *mvy_f, *Ty, *py;
    // corners
    double *dudy_cn, *dvdx_cn, *u_cn, *v_cn, *rho_cn, *mu_cn, *tau_xy, *Gxy;
    // state-sized
    double *DX, *DY, *SRC, *R;
};

// Kernel-side view of a grid (passed by value).
struct GridView {
    int nx, ny, wall, ad, nstate;
    int sm;                      // Stefan-Maxwell diffusion (Eq. 17) instead of Eq. (18)
    int predict;                 // Newton starts from a step off the cached species state
    long long off[NSP + 3];
    double Tw_nd;
    double C_mu, C_beta, C_kappa, C_D;
    const double *xi_c, *eta_c;
    unsigned* status;
};

enum Phase {
    PH_P1, PH_P3, PH_AD1, PH_AD2, PH_MU1, PH_MU2, PH_FACE, PH_FACEB, PH_DIV, PH_COUNT
};

// Launches of one right-hand side, as reported by the optional event profile.
enum KernelId {
    KID_LINES_STATE, KID_FACE_VEL, KID_CLOSURE, KID_LINES_VELGRAD, KID_LINES_AD, KID_AD_PREP,
    KID_AD_RAW, KID_AD_GAUSS, KID_AD_COMBINE, KID_STRESS_C, KID_LINES_MU, KID_STRESS_CN,
    KID_LINES_FACE, KID_FLUX, KID_LINES_DIV, KID_ASSEMBLE, KID_FILTER, KID_COUNT
};
inline constexpr const char* KERNEL_NAMES[KID_COUNT] = {
    "k_lines:state", "k_face_vel", "k_closure", "k_lines:velgrad", "k_lines:ad", "k_ad_prep",
    "k_ad_raw", "k_gauss", "k_ad_combine", "k_stress_c", "k_lines:mu", "k_stress_cn",
    "k_lines:face", "k_flux", "k_lines:div", "k_assemble", "k_filter"};

struct EventProfile {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> id;
    size_t used = 0;
    double ms[KID_COUNT] = {};
    long long count[KID_COUNT] = {};
};


// Freestream scales of a gas (Eqs. 7, 11) used by the pointwise kernels; the gas tables
// themselves do not depend on the freestream, so a batch of grids with different freestreams
// shares one table and carries these per grid.
struct Scales {
    int kind;
    double rho_inf, a_inf, T_ref, mu_inf, k_inf, L_ref, Re, Pr, gamma_inf;
    double R_inf, tpg_cp0, tpg_theta;   // thermally perfect gas (HYP_GAS_TPG)
};

inline Scales scales_of(const GasDev& g) {
    Scales sc;
    sc.kind = g.kind;
    sc.rho_inf = g.rho_inf;
    sc.a_inf = g.a_inf;
    sc.T_ref = g.T_ref;
    sc.mu_inf = g.mu_inf;
    sc.k_inf = g.k_inf;
    sc.L_ref = g.L_ref;
    sc.Re = g.Re;
    sc.Pr = g.Pr;
    sc.gamma_inf = g.gamma_inf;
    sc.R_inf = g.R_inf;
    sc.tpg_cp0 = g.tpg_cp0;
    sc.tpg_theta = g.tpg_theta;
    return sc;
}

}  // namespace hyp

using hyp::Dims;
using hyp::EventProfile;
using hyp::GasDev;
using hyp::GridView;
using hyp::LineJob;
using hyp::LineOp;
using hyp::PH_COUNT;
using hyp::Scratch;

struct hyp_grid {
    void* g3;                    // three-dimensional grids: their own data (rhs.cu), else null
    Dims d;
    hyp_case cas;
    GasDev gas;
    int nstate;
    long long off[NSP + 3];
    double *xi_c, *xi_f, *eta_c, *eta_f;
    float* metf;                 // binary32 copies of the four metric arrays, in that order
    double *Uref, *sigma;
    uint8_t* mask;
    unsigned* status;
    double* pool;
    Scratch s;
    LineOp* ops;
    double* opdata;
    LineJob* jobs;
    std::vector<LineJob> hjobs;  // host copy of the launch plan (the batched executor joins plans)
    int ph_start[PH_COUNT], ph_count[PH_COUNT], ph_blocks[PH_COUNT];
    double* linetmp;
    long long linetmp_n;
    cudaStream_t stream;
    double Tw_nd;
    EventProfile* prof;
    int cache_valid;             // the closure caches hold a previous evaluation
    cudaStream_t side;           // second stream for phases that do not wait on the closure
    cudaEvent_t fork[2], join[2];
    int closure_blocks;          // resident blocks of k_closure on this GPU
    int closure_blocks_mixed;    // the same for the mixed-precision closure
    GridView view() const {
        GridView v;
        v.nx = d.nx;
        v.ny = d.ny;
        v.wall = cas.wall;
        v.ad = cas.artificial_diffusivity;
        v.nstate = nstate;
        v.predict = cache_valid;
        for (int i = 0; i < NSP + 3; ++i) v.off[i] = off[i];
        v.Tw_nd = Tw_nd;
        v.C_mu = cas.C_mu;
        v.C_beta = cas.C_beta;
        v.C_kappa = cas.C_kappa;
        v.C_D = cas.C_D;
        v.sm = cas.diffusion_model == 1 && gas.kind == HYP_GAS_CNEQ;
        v.xi_c = xi_c;
        v.eta_c = eta_c;
        v.status = status;
        return v;
    }
};

struct hyp_state {
    hyp_grid* grid;
    double *U, *dQ;
};
