// Three-dimensional grids (hyp_grid_desc.nz > 1): the right-hand side of rhs.cu with a uniform,
// periodic third direction z and an optional jet from a circular orifice in the wall (the jet in
// hypersonic crossflow of Sec. 4, here with a spanwise-periodic domain). Included by rhs.cu
// inside its file-local namespace, so it shares the reference profile, grid map and operator
// construction of the two-dimensional path.
//
// Layout (x fastest): centres (nz, ny, nx) hold rho, rho_s (s >= 1), rho E; rho u on x-faces
// (nz, ny, nx+1); rho v on y-faces (nz, ny+1, nx); rho w on z-faces (nz, ny, nx), face k between
// centres k-1 and k. Shear stresses and cross momentum fluxes sit on edges: xy-edges
// (nz, ny+1, nx+1), xz-edges (the x-face array shape, at z-faces), yz-edges (the y-face shape).
//
// Every step follows the two-dimensional sequence, extended by the z terms: velocity gradients
// at centres and on the three edge families, the three-dimensional strain and vorticity in the
// artificial-diffusivity sensors (fourth differences and Gaussian filter periodic in z), stresses
// at centres and edges, species and energy fluxes on the three face families, divergences in
// three directions. Lines along x and y run through the segmented line kernel of the
// two-dimensional path (lines.cu; lines along y grouped by z-plane); lines along z are periodic:
// every row is interior, so the forward and backward recurrences run with the operator's
// constant factors around the ring, one thread per line, started W rows early from zero (W = 40
// for the interpolation, factor 1/3, and 26 for the derivative, factor 0.148: the dropped history
// is below 1e-19 of the values, and the result is the periodic solution to rounding). Each phase
// batches up to eight independent line jobs of one kind per launch; the velocity-gradient and
// artificial-diffusivity phases run on a second stream beside the closure, and the viscosity
// phase, the stresses and their face values there beside the other face values.
//
// Jet (reading; the paper gives a sonic jet of prescribed temperature ratio and momentum ratio
// J): inside the orifice the wall face holds the Dirichlet mass flux of a sonic jet at
// T_j = jet_T_ratio T_inf and p_j = J Ma^2 p_inf, blended to the no-slip wall by
// 1/2 (1 - tanh((r - r_j) / (jet_edge r_j))) (r: distance to the jet centre, the spanwise
// separation taken on the periodic domain); the wall temperature of the heat flux blends from
// T_wall to T_j the same way; u = w = 0 and no diffusion through the wall.

enum Shape3 : int { C3 = 0, XF3 = 1, YF3 = 2, XY3 = 3 };

struct Sh3 {
    int nx, ny, nz;
    __host__ __device__ int pitch(int t) const { return (t == C3 || t == YF3) ? nx : nx + 1; }
    __host__ __device__ int rows(int t) const { return (t == C3 || t == XF3) ? ny : ny + 1; }
    __host__ __device__ long long plane(int t) const { return (long long)pitch(t) * rows(t); }
    __host__ __device__ long long size(int t) const { return plane(t) * nz; }
};

// One batched line operation over a 3-D array.
struct Line3 {
    const LineOp* op;          // x or y operator (device); unused along z
    int axis, tin, tout;       // 0 x, 1 y, 2 z; array shapes of input and output
    const double* in;
    double* out;
    const double* metric;      // x, y: per output point along the line (nullable)
    double scale;              // z lines: includes the metric zeta
    double wall;               // y lines with a wall operator: wall value, or per line:
    const double* wall_arr;    //   wall value of line (k, i) at k * nx + i
    int kind, dir;             // z lines: 0 interpolation / 1 derivative; 0 c->f / 1 f->c
    double wa, wb, lm, cp;     // z lines: the operator's constant factors
    int job;                   // x, y lines: index of the segmented line job (Grid3::jobs)
    int f32;                   // feeds only diffusive fluxes: binary32 rows under HYP_MIXED
};


__device__ __forceinline__ double row3(int kind, double p0, double p1, double p2, double p3,
                                       double wa, double wb, double lm, double d) {
    if (kind == 0) return fma(-lm, d, fma(wa, p1 + p2, wb * (p0 + p3)));
    return fma(-lm, d, fma(wa, p2 - p1, wb * (p3 - p0)));
}

// Periodic lines along z: one thread per line, one job of the batch per blockIdx.y. The four
// stencil values slide through registers and the plane index wraps with a counter (one load per
// row, no integer division in the loop).
constexpr int BATCH3 = 8;      // line jobs per launch (x/y jobs: forward-sweep slots)
struct ZBatch {
    Line3 L[BATCH3];
};

struct ZRing {
    int n, W3, r0, b0;         // period, warm-up rows, first stencil row, first warm-up back row
    long long plane;
    __device__ ZRing(const Line3& L, const Sh3& sh) {
        plane = sh.plane(L.tin);
        n = sh.nz;
        W3 = L.kind == 0 ? 40 : 26;   // as the segmented solver: dropped history < 1e-19
        const int o = L.dir == 0 ? 2 : 1;          // first stencil row of output row t: t - o
        r0 = ((-W3 - o) % n + n) % n;
        b0 = (n - 1 + W3) % n;
    }
};

__device__ __forceinline__ void zline64(const Line3& L, const ZRing& z,
                                        const double* __restrict__ in, double* __restrict__ out) {
    const long long plane = z.plane;
    const int n = z.n, W3 = z.W3;
    int r = z.r0;
    auto next = [&]() {
        const double v = in[(long long)r * plane];
        r = r + 1 == n ? 0 : r + 1;
        return v;
    };
    double p0 = next(), p1 = next(), p2 = next();
    double d = 0.0;
    for (int t = -W3; t < 0; ++t) {      // warm-up: rows n - W3 .. n - 1 of the period
        const double p3 = next();
        d = row3(L.kind, p0, p1, p2, p3, L.wa, L.wb, L.lm, d);
        p0 = p1;
        p1 = p2;
        p2 = p3;
    }
    for (int t = 0; t < n; ++t) {
        const double p3 = next();
        d = row3(L.kind, p0, p1, p2, p3, L.wa, L.wb, L.lm, d);
        out[(long long)t * plane] = d;
        p0 = p1;
        p1 = p2;
        p2 = p3;
    }
    // back substitution: warm-up over rows W3 - 1 .. 0 of the next period, then the period
    int b = z.b0;
    double y = out[(long long)b * plane];
    for (int k = 1; k < W3; ++k) {
        b = b == 0 ? n - 1 : b - 1;
        y = out[(long long)b * plane] - L.cp * y;
    }
    for (int t = n - 1; t >= 0; --t) {
        y = out[(long long)t * plane] - L.cp * y;
        out[(long long)t * plane] = L.scale * y;
    }
}

__device__ __forceinline__ float* zslot(double* p) { return reinterpret_cast<float*>(p); }

// The same in binary32 (HYP_MIXED, lines feeding only diffusive fluxes): inputs rounded with the
// integer conversions of fp32.cuh, forward values kept as binary32 in the first half of their
// output slot, outputs widened back to binary64.
__device__ __forceinline__ void zline32(const Line3& L, const ZRing& z,
                                        const double* __restrict__ in, double* __restrict__ out) {
    const long long plane = z.plane;
    const int n = z.n, W3 = z.W3;
    const float wa = f32_of(L.wa), wb = f32_of(L.wb), lm = f32_of(L.lm), cp = f32_of(L.cp),
                sc = f32_of(L.scale);
    auto row = [&](float p0, float p1, float p2, float p3, float d) {
        if (L.kind == 0) return fmaf(-lm, d, fmaf(wa, p1 + p2, wb * (p0 + p3)));
        return fmaf(-lm, d, fmaf(wa, p2 - p1, wb * (p3 - p0)));
    };
    int r = z.r0;
    auto next = [&]() {
        const float v = f32_of(in[(long long)r * plane]);
        r = r + 1 == n ? 0 : r + 1;
        return v;
    };
    float p0 = next(), p1 = next(), p2 = next();
    float d = 0.0f;
    for (int t = -W3; t < 0; ++t) {
        const float p3 = next();
        d = row(p0, p1, p2, p3, d);
        p0 = p1;
        p1 = p2;
        p2 = p3;
    }
    for (int t = 0; t < n; ++t) {
        const float p3 = next();
        d = row(p0, p1, p2, p3, d);
        *zslot(out + (long long)t * plane) = d;
        p0 = p1;
        p1 = p2;
        p2 = p3;
    }
    int b = z.b0;
    float y = *zslot(out + (long long)b * plane);
    for (int k = 1; k < W3; ++k) {
        b = b == 0 ? n - 1 : b - 1;
        y = fmaf(-cp, y, *zslot(out + (long long)b * plane));
    }
    for (int t = n - 1; t >= 0; --t) {
        y = fmaf(-cp, y, *zslot(out + (long long)t * plane));
        out[(long long)t * plane] = f64_of(sc * y);
    }
}

__global__ void __launch_bounds__(128) k_line3z(ZBatch B, Sh3 sh, int mixed) {
    const Line3& L = B.L[blockIdx.y];
    const ZRing z(L, sh);
    const bool f32 = mixed && L.f32;      // uniform per block
    for (long long line = blockIdx.x * (long long)blockDim.x + threadIdx.x; line < z.plane;
         line += (long long)gridDim.x * blockDim.x) {
        if (f32) zline32(L, z, L.in + line, L.out + line);
        else zline64(L, z, L.in + line, L.out + line);
    }
}

struct Grid3 {
    Sh3 sh;
    double zeta;
    long long nc, nxf, nyf, nxy, nstate;
    long long off[NSP + 4];    // rho, rho_s (1..NSP-1), rho E, rho u, rho v, rho w
    double* pool;
    // centres (and z-faces, same shape)
    double *ru_c, *rv_c, *rw_c, *T, *p, *H, *u_c, *v_c, *w_c, *e, *a, *mu_e, *K, *beta, *Tcache;
    double *Y[NSP], *X[NSP], *h[NSP], *W[NSP], *Wd[NSP], *G[NSP];
    double *esc[NSP], *cvsc[NSP], *cvpc[NSP];   // species e, c_v, dc_v/dT at the cached T
    int cache_valid;                            // host: the caches hold an evaluation
    double *dudx, *dvdy, *dwdz, *tau_xx, *tau_yy, *tau_zz, *Gxx, *Gyy, *Gzz, *mux_c, *mvy_c, *mwz_c;
    double *S, *div, *fsw, *dudy_c, *dvdx_c, *dudz_c, *dwdx_c, *dvdz_c, *dwdy_c, *tc[4];
    double *raw[AD_FIELDS], *filt[AD_FIELDS];
    double *rho_zf, *w_zf, *mwz_f;
    double *Yz[NSP], *Gz[NSP], *hz[NSP], *dXdz[NSP], *Fsz[NSP];
    double *Hz, *Kz, *dTdz, *tzz_z, *u_z, *v_z, *txz_z, *tyz_z, *FEz;
    // x-faces and xz-edges
    double *rho_xf, *u_xf, *mux_f, *mu_xf, *Yx[NSP], *Gx[NSP], *hx[NSP], *dXdx[NSP], *Fsx[NSP];
    double *Hx, *Kx, *dTdx, *txx_x, *v_x, *w_x, *txy_x, *txz_x, *FEx;
    double *dudz_xz, *dwdx_xz, *u_xz, *w_xz, *rho_xz, *mu_xz, *tau_xz, *Gxz, *tx[2];
    // y-faces and yz-edges
    double *rho_yf, *v_yf, *mvy_f, *mu_yf, *Yy[NSP], *Gy[NSP], *hy[NSP], *dXdy[NSP], *Fsy[NSP];
    double *Hy, *Ky, *dTdy, *tyy_y, *u_y, *w_y, *txy_y, *tyz_y, *FEy;
    double *dvdz_yz, *dwdy_yz, *v_yz, *w_yz, *rho_yz, *mu_yz, *tau_yz, *Gyz;
    // xy-edges
    double *dudy_xy, *dvdx_xy, *u_xy, *v_xy, *rho_xy, *mu_xy, *tau_xy, *Gxy;
    // state-sized
    double *DX, *DY, *DZ, *SRC, *R;
    double *Uref, *sigma;
    uint8_t* mask;
    double *xi_c, *xi_f, *eta_c, *eta_f, *Tw;
    float* metf;               // binary32 copies of xi_c, xi_f, eta_c, eta_f (HYP_MIXED line jobs)
    LineOp* ops;
    double* opdata;
    Line3 zop[2][2];           // periodic z operators [kind][dir] (constants only)
    struct Plan3* plan;        // host: the line jobs of each phase
    LineJob* jobs;             // device: the x and y lines as segmented line jobs (lines.cu)
    double* ltmp;              // their forward-sweep storage (jobs run one after another)
};

// One launch of a phase: up to BATCH3 consecutive entries of its line list, all periodic z lines
// (k_line3z) or all x/y line jobs (k_lines, contiguous in Grid3::jobs).
struct Launch3 {
    int z;
    int first, count;
    int blocks;                // x/y: blocks per job, the largest of the batch
};

struct Phase3 {
    std::vector<Line3> lines;
    std::vector<Launch3> launches;
    int slot_base = 0;         // first forward-sweep buffer of its x/y jobs
};

// face: the face values that do not need the stresses; faceb: the stresses' face values, which
// run with mu on the second stream beside face (so their x/y jobs take other sweep buffers)
struct Plan3 {
    Phase3 p1, p3, ad1, ad2, mu, face, faceb, divs;
};

struct View3 {
    Sh3 sh;
    long long off[NSP + 4];
    int wall, ad, predict;
    double C_mu, C_beta, C_kappa, C_D, zeta;
    const double *xi_c, *eta_c;
    unsigned* status;
};

// ---- pointwise kernels ----
#define RANGE3(n) for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < (n); \
                       q += (long long)gridDim.x * blockDim.x)

__global__ void k_fv3(Grid3 g, View3 v, const double* __restrict__ U) {
    const long long a = g.nxf, b = a + g.nyf, c = b + g.nc;
    RANGE3(c) {
        if (q < a) {
            const double m = U[v.off[NSP + 1] + q], u = m / g.rho_xf[q];
            g.u_xf[q] = u;
            g.mux_f[q] = m * u;
        } else if (q < b) {
            const long long i = q - a;
            const double m = U[v.off[NSP + 2] + i], vv = m / g.rho_yf[i];
            g.v_yf[i] = vv;
            g.mvy_f[i] = m * vv;
        } else {
            const long long i = q - b;
            const double m = U[v.off[NSP + 3] + i], w = m / g.rho_zf[i];
            g.w_zf[i] = w;
            g.mwz_f[i] = m * w;
        }
    }
}

template <bool MIXED>
__global__ void __launch_bounds__(128) k_closure3(GasDev gd, Scales sc, Grid3 g, View3 v,
                                                  const double* __restrict__ U) {
    const bool cneq = sc.kind == HYP_GAS_CNEQ;
    RANGE3(g.nc) {
        const long long idx = q;
        const double rho = U[v.off[0] + idx];
        const double irho = 1.0 / rho;
        double Y[NSP];
        double rest = rho;
#pragma unroll
        for (int sp = 1; sp < NSP; ++sp) {
            const double r = U[v.off[sp] + idx];
            Y[sp] = r * irho;
            rest -= r;
        }
        Y[0] = rest * irho;
        const double rhoE = U[v.off[NSP] + idx];
        const double u = g.ru_c[idx] * irho, vv = g.rv_c[idx] * irho, w = g.rw_c[idx] * irho;
        const double e = rhoE * irho - 0.5 * (u * u + vv * vv + w * w);
        double T, p, mu, k, a;
        double h[NSP], wd[NSP], X[NSP], W[NSP], Wd[NSP];
        if (sc.kind == HYP_GAS_CPG) {
            T = sc.gamma_inf * e;
            p = rho * (sc.gamma_inf - 1.0) / sc.gamma_inf * T;
            const double Td = T * sc.T_ref;
            mu = SUTH_C1 * Td * sqrt(Td) / (Td + SUTH_TS) / sc.mu_inf;
            k = mu;
            a = sqrt(sc.gamma_inf * p / rho);
#pragma unroll
            for (int sp = 0; sp < NSP; ++sp) h[sp] = wd[sp] = X[sp] = W[sp] = Wd[sp] = 0.0;
        } else {
            const double e_si = e * sc.a_inf * sc.a_inf;
            double T0 = g.Tcache[idx];
            if (v.predict) {
                // second-order step from the cached species state with the new composition
                double ec = 0.0, cvc = 0.0, cvpc = 0.0;
#pragma unroll
                for (int sp = 0; sp < NSP; ++sp) {
                    ec += Y[sp] * g.esc[sp][idx];
                    cvc += Y[sp] * g.cvsc[sp][idx];
                    cvpc += Y[sp] * g.cvpc[sp][idx];
                }
                const double icv = 1.0 / cvc;
                const double d1 = (e_si - ec) * icv;
                T0 += d1 - 0.5 * cvpc * d1 * d1 * icv;
            }
            ClosureOut o;
            closure_si_p<MIXED>(gd, rho * sc.rho_inf, e_si, Y, T0, cneq, cneq, o);
            if (o.status) atomicOr(v.status, o.status);
            g.Tcache[idx] = o.T;
#pragma unroll
            for (int sp = 0; sp < NSP; ++sp) {
                g.esc[sp][idx] = o.es[sp];
                g.cvsc[sp][idx] = o.cvs[sp];
                g.cvpc[sp][idx] = o.cvps[sp];
            }
            T = o.T / sc.T_ref;
            p = o.p / (sc.rho_inf * sc.a_inf * sc.a_inf);
            mu = o.mu / sc.mu_inf;
            k = o.k / sc.k_inf;
            a = o.a / sc.a_inf;
            double ym = 0.0;
#pragma unroll
            for (int sp = 0; sp < NSP; ++sp) ym += Y[sp] * gd.invM[sp];
            const double wscale = sc.L_ref / (sc.rho_inf * sc.a_inf);
            const double inva2 = 1.0 / (sc.a_inf * sc.a_inf);
#pragma unroll
            for (int sp = 0; sp < NSP; ++sp) {
                h[sp] = o.h[sp] * inva2;
                wd[sp] = o.wdot[sp] * wscale;
                X[sp] = o.X[sp];
                W[sp] = cneq && (!HAS_CHARGE || gd.heavy[sp]) ? rho * gd.M[sp] * ym : 0.0;
                Wd[sp] = W[sp] * (o.D[sp] * sc.rho_inf / sc.mu_inf) / sc.Re;
            }
        }
        g.T[idx] = T;
        g.p[idx] = p;
        g.H[idx] = (rhoE + p) * irho;
        g.u_c[idx] = u;
        g.v_c[idx] = vv;
        g.w_c[idx] = w;
        g.e[idx] = e;
        g.a[idx] = a;
        g.mu_e[idx] = mu / sc.Re;
        g.K[idx] = k / (sc.Re * sc.Pr);
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp) {
            g.Y[sp][idx] = Y[sp];
            g.X[sp][idx] = X[sp];
            g.h[sp][idx] = h[sp];
            g.W[sp][idx] = W[sp];
            g.Wd[sp][idx] = Wd[sp];
            g.G[sp][idx] = Wd[sp];
        }
        g.beta[idx] = 0.0;
#pragma unroll
        for (int sp = 1; sp < NSP; ++sp) g.SRC[v.off[sp] + idx] = wd[sp];
    }
}

__global__ void k_adprep3(Grid3 g) {
    RANGE3(g.nc) {
        const double ux = g.dudx[q], vy = g.dvdy[q], wz = g.dwdz[q];
        const double uy = g.dudy_c[q], vx = g.dvdx_c[q], uz = g.dudz_c[q], wx = g.dwdx_c[q];
        const double vz = g.dvdz_c[q], wy = g.dwdy_c[q];
        const double sxy = uy + vx, sxz = uz + wx, syz = vz + wy;
        g.S[q] = sqrt(ux * ux + vy * vy + wz * wz + 0.5 * sxy * sxy + 0.5 * sxz * sxz + 0.5 * syz * syz);
        const double dv = ux + vy + wz;
        const double o1 = vx - uy, o2 = uz - wx, o3 = wy - vz;
        const double om2 = o1 * o1 + o2 * o2 + o3 * o3;
        g.div[q] = dv;
        g.fsw[q] = dv < 0.0 ? dv * dv / (dv * dv + om2 + DUCROS_EPS) : 0.0;
    }
}

__device__ __forceinline__ double d4_3(const double* f, const Sh3& s, int k, int j, int i, int axis) {
    const long long nx = s.nx, pl = (long long)s.nx * s.ny;
    if (axis == 0) {
        const int c = min(max(i, 2), s.nx - 3);
        const double* r = f + k * pl + j * nx + c;
        return r[-2] - 4.0 * r[-1] + 6.0 * r[0] - 4.0 * r[1] + r[2];
    }
    if (axis == 1) {
        const int c = min(max(j, 2), s.ny - 3);
        const double* r = f + k * pl + c * nx + i;
        return r[-2 * nx] - 4.0 * r[-nx] + 6.0 * r[0] - 4.0 * r[nx] + r[2 * nx];
    }
    const double* b = f + j * nx + i;
    auto at = [&](int kk) { return b[(long long)(((kk % s.nz) + s.nz) % s.nz) * pl]; };
    return at(k + 2) - 4.0 * at(k + 1) + 6.0 * at(k) - 4.0 * at(k - 1) + at(k - 2);
}

__global__ void k_adraw3(Grid3 g, View3 v, const double* __restrict__ U, int cneq) {
    const Sh3 s = g.sh;
    const double dz = 1.0 / v.zeta;
    RANGE3(g.nc) {
        const int i = (int)(q % s.nx);
        const long long t = q / s.nx;
        const int j = (int)(t % s.ny), k = (int)(t / s.ny);
        const double dx = 1.0 / v.xi_c[i], dy = 1.0 / v.eta_c[j];
        const double rho = U[v.off[0] + q];
        auto sens = [&](const double* f, int l) {
            const double fx = d4_3(f, s, k, j, i, 0), fy = d4_3(f, s, k, j, i, 1),
                         fz = d4_3(f, s, k, j, i, 2);
            return l == 2 ? fx * dx * dx + fy * dy * dy + fz * dz * dz : fx * dx + fy * dy + fz * dz;
        };
        g.raw[0][q] = v.C_mu * rho * fabs(sens(g.S, 2));
        g.raw[1][q] = v.C_beta * rho * g.fsw[q] * fabs(sens(g.div, 2));
        g.raw[2][q] = v.C_kappa * rho * g.a[q] / g.T[q] * fabs(sens(g.e, 1));
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp) g.raw[3 + sp][q] = cneq ? v.C_D * g.a[q] * fabs(sens(g.Y[sp], 1)) : 0.0;
    }
}

// Gaussian filter of the raw diffusivities along one axis (x, y clamped; z periodic):
// pass 0 raw -> filt (x), 1 filt -> raw (y), 2 raw -> filt (z). MIXED: in binary32 as gauss_body
// (pointwise.cuh) does for two-dimensional grids.
template <typename R, bool MIXED>
__device__ __forceinline__ R gauss3_load(const double* p) {
    if constexpr (MIXED) return f32_trunc(*p);
    else return *p;
}

__device__ __forceinline__ float gauss3_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double gauss3_fma(double a, double b, double c) { return fma(a, b, c); }

template <bool MIXED>
__global__ void k_gauss3(Grid3 g, int axis) {
    using R = typename std::conditional<MIXED, float, double>::type;
    const Sh3 s = g.sh;
    const long long n = g.nc, pl = (long long)s.nx * s.ny;
    const R* w;
    if constexpr (MIXED) w = c_gauss_f;
    else w = c_gauss;
    // FP64: one field value per thread (field-major index range, as gauss_body); binary32: every
    // field of a point per thread
    RANGE3(MIXED ? n : (long long)AD_FIELDS * n) {
        const int f0 = MIXED ? 0 : (int)(q / n);
        const long long idx = q - (long long)f0 * n;
        const int i = (int)(idx % s.nx);
        const long long t = idx / s.nx;
        const int j = (int)(t % s.ny), k = (int)(t / s.ny);
        long long nb[8];                                 // neighbours -4..-1, +1..+4 (indices)
#pragma unroll
        for (int d = 1; d <= 4; ++d) {
            if (axis == 0) {
                nb[d - 1] = idx - i + max(i - d, 0);
                nb[3 + d] = idx - i + min(i + d, s.nx - 1);
            } else if (axis == 1) {
                nb[d - 1] = idx + (long long)(max(j - d, 0) - j) * s.nx;
                nb[3 + d] = idx + (long long)(min(j + d, s.ny - 1) - j) * s.nx;
            } else {
                nb[d - 1] = idx + (long long)(((k - d) % s.nz + s.nz) % s.nz - k) * pl;
                nb[3 + d] = idx + (long long)((k + d) % s.nz - k) * pl;
            }
        }
        for (int f = f0; f < (MIXED ? AD_FIELDS : f0 + 1); ++f) {
            const double* __restrict__ in = axis == 1 ? g.filt[f] : g.raw[f];
            double* __restrict__ out = axis == 1 ? g.raw[f] : g.filt[f];
            R acc = w[0] * gauss3_load<R, MIXED>(in + idx);
#pragma unroll
            for (int d = 1; d <= 4; ++d)
                acc = gauss3_fma(w[d], gauss3_load<R, MIXED>(in + nb[d - 1]) +
                                           gauss3_load<R, MIXED>(in + nb[3 + d]), acc);
            if constexpr (MIXED) out[idx] = f64_of(acc);
            else out[idx] = acc;
        }
    }
}

__global__ void k_adcombine3(Grid3 g) {
    RANGE3(g.nc) {
        g.mu_e[q] += g.filt[0][q];
        g.beta[q] = g.filt[1][q];
        g.K[q] += g.filt[2][q];
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp) g.G[sp][q] = g.Wd[sp][q] + g.W[sp][q] * g.filt[3 + sp][q];
    }
}

__global__ void k_stress3(Grid3 g) {
    const long long a = g.nc, b = a + g.nxy, c = b + g.nxf, d = c + g.nyf;
    RANGE3(d) {
        if (q < a) {
            const double ux = g.dudx[q], vy = g.dvdy[q], wz = g.dwdz[q];
            const double dv = ux + vy + wz, mu = g.mu_e[q], be = g.beta[q];
            const double txx = mu * (2.0 * ux - 2.0 / 3.0 * dv) + be * dv;
            const double tyy = mu * (2.0 * vy - 2.0 / 3.0 * dv) + be * dv;
            const double tzz = mu * (2.0 * wz - 2.0 / 3.0 * dv) + be * dv;
            g.tau_xx[q] = txx;
            g.tau_yy[q] = tyy;
            g.tau_zz[q] = tzz;
            g.Gxx[q] = g.mux_c[q] + g.p[q] - txx;
            g.Gyy[q] = g.mvy_c[q] + g.p[q] - tyy;
            g.Gzz[q] = g.mwz_c[q] + g.p[q] - tzz;
        } else if (q < b) {
            const long long i = q - a;
            const double t = g.mu_xy[i] * (g.dudy_xy[i] + g.dvdx_xy[i]);
            g.tau_xy[i] = t;
            g.Gxy[i] = g.rho_xy[i] * g.u_xy[i] * g.v_xy[i] - t;
        } else if (q < c) {
            const long long i = q - b;
            const double t = g.mu_xz[i] * (g.dudz_xz[i] + g.dwdx_xz[i]);
            g.tau_xz[i] = t;
            g.Gxz[i] = g.rho_xz[i] * g.u_xz[i] * g.w_xz[i] - t;
        } else {
            const long long i = q - c;
            const double t = g.mu_yz[i] * (g.dvdz_yz[i] + g.dwdy_yz[i]);
            g.tau_yz[i] = t;
            g.Gyz[i] = g.rho_yz[i] * g.v_yz[i] * g.w_yz[i] - t;
        }
    }
}

// species and energy fluxes at x-faces, y-faces and z-faces
__global__ void __launch_bounds__(128) k_flux3(GasDev gd, Grid3 g, View3 v, const double* __restrict__ U) {
    const long long a = g.nxf, b = a + g.nyf, c = b + g.nc;
    RANGE3(c) {
        int dir;
        long long i;
        if (q < a) { dir = 0; i = q; }
        else if (q < b) { dir = 1; i = q - a; }
        else { dir = 2; i = q - b; }
        const double m = U[v.off[NSP + 1 + dir] + i];
        double* const* Yf = dir == 0 ? g.Yx : dir == 1 ? g.Yy : g.Yz;
        double* const* Gf = dir == 0 ? g.Gx : dir == 1 ? g.Gy : g.Gz;
        double* const* hf = dir == 0 ? g.hx : dir == 1 ? g.hy : g.hz;
        double* const* dX = dir == 0 ? g.dXdx : dir == 1 ? g.dXdy : g.dXdz;
        double* const* Fs = dir == 0 ? g.Fsx : dir == 1 ? g.Fsy : g.Fsz;
        const double Hf = (dir == 0 ? g.Hx : dir == 1 ? g.Hy : g.Hz)[i];
        const double Kf = (dir == 0 ? g.Kx : dir == 1 ? g.Ky : g.Kz)[i];
        const double dT = (dir == 0 ? g.dTdx : dir == 1 ? g.dTdy : g.dTdz)[i];
        const bool wallface = dir == 1 && v.wall && (i % ((long long)(g.sh.ny + 1) * g.sh.nx)) < g.sh.nx;
        double gg[NSP], J[NSP], sum = 0.0;
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp) {
            gg[sp] = Gf[sp][i] * dX[sp][i];
            sum += gg[sp];
        }
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp) J[sp] = wallface ? 0.0 : -(gg[sp] - Yf[sp][i] * sum);
        if (HAS_CHARGE && gd.ie >= 0 && !wallface) {
            double acc = 0.0;
#pragma unroll
            for (int sp = 0; sp < NSP; ++sp)
                if (gd.charge[sp] > 0) acc += J[sp] / gd.M[sp];
            double tot = 0.0;
#pragma unroll
            for (int sp = 1; sp < NSP; ++sp) {
                if (sp == gd.ie) J[sp] = gd.M[sp] * acc;
                tot += J[sp];
            }
            J[0] = -tot;
        }
        double qf = -Kf * dT;
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp) qf += hf[sp][i] * J[sp];
#pragma unroll
        for (int sp = 1; sp < NSP; ++sp) Fs[sp][i] = m * Yf[sp][i] + J[sp];
        double work;
        if (dir == 0) work = g.txx_x[i] * g.u_xf[i] + g.txy_x[i] * g.v_x[i] + g.txz_x[i] * g.w_x[i];
        else if (dir == 1) work = g.txy_y[i] * g.u_y[i] + g.tyy_y[i] * g.v_yf[i] + g.tyz_y[i] * g.w_y[i];
        else work = g.txz_z[i] * g.u_z[i] + g.tyz_z[i] * g.v_z[i] + g.tzz_z[i] * g.w_zf[i];
        (dir == 0 ? g.FEx : dir == 1 ? g.FEy : g.FEz)[i] = m * Hf + qf - work;
    }
}

struct Assemble3 {
    const double *DX, *DY, *DZ, *SRC, *sigma, *Uref;
    const uint8_t* mask;
    double *U, *out, *dQ;
    int rk;
    double A, B, dt;
};

__global__ void k_assemble3(Assemble3 a, long long n) {
    RANGE3(n) {
        const double u = a.U[q];
        double r = a.DX[q] + a.DY[q] + a.DZ[q] + a.SRC[q] - a.sigma[q] * (u - a.Uref[q]);
        if (a.mask[q]) r = 0.0;
        if (a.rk) {
            const double d = a.A * a.dQ[q] + a.dt * r;
            a.dQ[q] = d;
            a.U[q] = u + a.B * d;
        } else {
            a.out[q] = r;
        }
    }
}

// Jet of a three-dimensional case: orifice centre, radius, edge and the plume height of the
// initial state (two radii), and the sonic jet's T (K), p (Pa) and nondimensional v.
struct Jet3 {
    int on;
    double x, z, r, edge, height, Lz, T, p, v;
    __host__ __device__ double blend(double xx, double zz) const {
        double sz = fabs(zz - z);
        sz = fmin(sz, Lz - sz);
        const double rr = sqrt((xx - x) * (xx - x) + sz * sz);
        return 0.5 * (1.0 - tanh((rr - r) / (edge * r)));
    }
};

// Reference state Q_ref, sponge strength and Dirichlet mask at every entry of the 3-D state: the
// two-dimensional profile at (x, y), blended towards the jet inside its plume
// F = blend(x, z) exp(-((y - y0) / (height r))^2) (T, p -> T_j, p_j; u -> 0; v -> v_j).
__global__ void k_reference3(GasDev gd, Profile P, hyp_grid_desc d, Jet3 jet, Grid3 g) {
    const Sh3 s = g.sh;
    const double dx = (d.x1 - d.x0) / s.nx, dz = (d.z1 - d.z0) / s.nz;
    RANGE3(g.nstate) {
        int field, node, i, j, k;
        long long rem;
        if (q < (long long)(NSP + 1) * g.nc) {
            field = (int)(q / g.nc);
            rem = q - field * g.nc;
            node = 0;
        } else if (q < g.off[NSP + 2]) {
            field = NSP + 1;
            rem = q - g.off[NSP + 1];
            node = 1;
        } else if (q < g.off[NSP + 3]) {
            field = NSP + 2;
            rem = q - g.off[NSP + 2];
            node = 2;
        } else {
            field = NSP + 3;
            rem = q - g.off[NSP + 3];
            node = 0;
        }
        const int pitch = node == 1 ? s.nx + 1 : s.nx, rows = node == 2 ? s.ny + 1 : s.ny;
        k = (int)(rem / ((long long)pitch * rows));
        const long long w = rem - (long long)k * pitch * rows;
        j = (int)(w / pitch);
        i = (int)(w - (long long)j * pitch);
        const double x = d.x0 + dx * (node == 1 ? (double)i : i + 0.5);
        double y, dyde;
        y_map(d, node == 2 ? (double)j : j + 0.5, y, dyde);
        const double z = d.z0 + dz * (k + 0.5);
        const double sg = sponge_at(d, P.c, x, y);
        g.sigma[q] = sg;
        if (field == NSP + 3) {
            g.Uref[q] = 0.0;
            g.mask[q] = 0;
            continue;
        }
        double T, p, u, v, Y[NSP], rho, rY[NSP], rE;
        P.at(gd, x, y, T, p, u, v, Y);
        if (jet.on) {
            const double yh = (y - d.y0) / (jet.height * jet.r);
            const double F = jet.blend(x, z) * exp(-yh * yh);
            T = T + (jet.T - T) * F;
            p = p + (jet.p - p) * F;
            u = u * (1.0 - F);
            v = v + (jet.v - v) * F;
        }
        P.conserved(gd, T, p, u, v, Y, rho, rY, rE);
        double val;
        uint8_t m = 0;
        if (field == 0) val = rho;
        else if (field < NSP) val = rY[field];
        else if (field == NSP) val = rE;
        else if (field == NSP + 1) {
            val = rho * u;
            m = (i == 0 || i == s.nx) ? 1 : 0;
        } else {
            val = rho * v;
            m = (j == 0 || j == s.ny) ? 1 : 0;
        }
        g.Uref[q] = val;
        g.mask[q] = m;
    }
}

// ---- host: set-up and the right-hand side ----

void free_grid3(Grid3* g) {
    if (!g) return;
    delete g->plan;
    cudaFree(g->jobs);
    cudaFree(g->ltmp);
    cudaFree(g->metf);
    cudaFree(g->pool);
    cudaFree(g->mask);
    cudaFree(g->ops);
    cudaFree(g->opdata);
    delete g;
}

View3 view3(const hyp_grid* G, const Grid3* g) {
    View3 v;
    v.sh = g->sh;
    for (int i = 0; i < NSP + 4; ++i) v.off[i] = g->off[i];
    v.wall = G->cas.wall;
    v.ad = G->cas.artificial_diffusivity;
    v.predict = g->cache_valid;
    v.C_mu = G->cas.C_mu;
    v.C_beta = G->cas.C_beta;
    v.C_kappa = G->cas.C_kappa;
    v.C_D = G->cas.C_D;
    v.zeta = g->zeta;
    v.xi_c = g->xi_c;
    v.eta_c = g->eta_c;
    v.status = G->status;
    return v;
}

// The launches of one phase in order; `state`: the z lines' `in` is an element offset into U (the
// x and y jobs resolve theirs in the line kernel).
int launch3(const Grid3* g, const Phase3& ph, const double* U, bool state, int mixed,
            cudaStream_t s) {
    for (const Launch3& b : ph.launches) {
        if (b.z) {
            ZBatch zb;
            memset(&zb, 0, sizeof(zb));
            long long n = 0;
            for (int i = 0; i < b.count; ++i) {
                zb.L[i] = ph.lines[b.first + i];
                if (state) zb.L[i].in = U + (size_t)zb.L[i].in;
                n = std::max(n, g->sh.plane(zb.L[i].tin));
            }
            const int bx = (int)std::min<long long>((n + 127) / 128, 152LL * 64);
            k_line3z<<<dim3(bx, b.count), 128, 0, s>>>(zb, g->sh, mixed);
        } else {
            HYP_CUDA(launch_lines(g->jobs + ph.lines[b.first].job, b.count, b.blocks, U, s, mixed));
        }
    }
    HYP_CUDA(cudaGetLastError());
    return HYP_OK;
}

int blocks3(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 32)); }

int run_rhs3(const hyp_gas* gas, hyp_grid* G, const double* U, double* dUdt, int rk, double A,
             double Bc, double dt, double* Urk, double* dQ, int precision, cudaStream_t s) {
    Grid3* g = (Grid3*)G->g3;
    const View3 v = view3(G, g);
    const GasDev& gd = gas->dev;
    const Plan3& pl = *g->plan;
    const int mx = precision == HYP_MIXED ? 1 : 0;
    int rc = launch3(g, pl.p1, U, true, mx, s);
    if (rc) return rc;
    k_fv3<<<blocks3(g->nxf + g->nyf + g->nc), 256, 0, s>>>(*g, v, U);
    // fork: velocity gradients and the artificial-diffusivity line phases do not need the closure
    cudaStream_t s2 = G->side;
    HYP_CUDA(cudaEventRecord(G->fork[0], s));
    HYP_CUDA(cudaStreamWaitEvent(s2, G->fork[0], 0));
    const Scales sc = scales_of(gd);
    const int slot = prof_begin(G, KID_CLOSURE, s);     // the event profile's one 3-D entry
    if (precision == HYP_MIXED) k_closure3<true><<<blocks3(g->nc), 128, 0, s>>>(gd, sc, *g, v, U);
    else k_closure3<false><<<blocks3(g->nc), 128, 0, s>>>(gd, sc, *g, v, U);
    prof_end(G, slot, s);
    HYP_CUDA(cudaGetLastError());
    g->cache_valid = 1;
    if ((rc = launch3(g, pl.p3, U, false, mx, s2))) return rc;
    if (v.ad) {
        if ((rc = launch3(g, pl.ad1, U, false, mx, s2))) return rc;
        if ((rc = launch3(g, pl.ad2, U, false, mx, s2))) return rc;
        k_adprep3<<<blocks3(g->nc), 256, 0, s2>>>(*g);
        HYP_CUDA(cudaGetLastError());
    }
    HYP_CUDA(cudaEventRecord(G->join[0], s2));
    HYP_CUDA(cudaStreamWaitEvent(s, G->join[0], 0));
    if (v.ad) {
        k_adraw3<<<blocks3(g->nc), 256, 0, s>>>(*g, v, U, gd.kind == HYP_GAS_CNEQ);
        for (int ax = 0; ax < 3; ++ax) {
            if (mx) k_gauss3<true><<<blocks3(g->nc), 256, 0, s>>>(*g, ax);
            else k_gauss3<false><<<blocks3(AD_FIELDS * g->nc), 256, 0, s>>>(*g, ax);
        }
        k_adcombine3<<<blocks3(g->nc), 256, 0, s>>>(*g);
        HYP_CUDA(cudaGetLastError());
    }
    // fork: viscosities to faces and edges, the stresses and their face values beside the other
    // face values
    HYP_CUDA(cudaEventRecord(G->fork[1], s));
    HYP_CUDA(cudaStreamWaitEvent(s2, G->fork[1], 0));
    if ((rc = launch3(g, pl.mu, U, false, mx, s2))) return rc;
    k_stress3<<<blocks3(g->nc + g->nxy + g->nxf + g->nyf), 256, 0, s2>>>(*g);
    HYP_CUDA(cudaGetLastError());
    if ((rc = launch3(g, pl.faceb, U, false, mx, s2))) return rc;
    HYP_CUDA(cudaEventRecord(G->join[1], s2));
    if ((rc = launch3(g, pl.face, U, false, mx, s))) return rc;
    HYP_CUDA(cudaStreamWaitEvent(s, G->join[1], 0));
    k_flux3<<<blocks3(g->nxf + g->nyf + g->nc), 128, 0, s>>>(gd, *g, v, U);
    HYP_CUDA(cudaGetLastError());
    if ((rc = launch3(g, pl.divs, U, false, mx, s))) return rc;
    Assemble3 a;
    a.DX = g->DX;
    a.DY = g->DY;
    a.DZ = g->DZ;
    a.SRC = g->SRC;
    a.sigma = g->sigma;
    a.Uref = g->Uref;
    a.mask = g->mask;
    a.U = rk ? Urk : const_cast<double*>(U);
    a.out = dUdt;
    a.dQ = dQ;
    a.rk = rk;
    a.A = A;
    a.B = Bc;
    a.dt = dt;
    k_assemble3<<<blocks3(g->nstate), 256, 0, s>>>(a, g->nstate);
    HYP_CUDA(cudaGetLastError());
    return HYP_OK;
}

// Build a three-dimensional grid: operators, plan, reference and initial state.
int init3(const hyp_gas* gas, const hyp_grid_desc* desc, const hyp_case* cas, double* U,
          double* dQ, cudaStream_t s, hyp_grid* G) {
    const GasDev& gd = gas->dev;
    if (!(gd.kind == HYP_GAS_CNEQ || gd.kind == HYP_GAS_FROZEN || gd.kind == HYP_GAS_CPG))
        return fail(HYP_ERR_ARG, "three-dimensional grids take the cneq, frozen or cpg gas");
    if (cas->diffusion_model != 0) return fail(HYP_ERR_ARG, "three-dimensional grids use the algebraic diffusion");
    if (cas->filter_sigma > 0) return fail(HYP_ERR_ARG, "three-dimensional grids have no state filter");
    if (!(desc->z1 > desc->z0)) return fail(HYP_ERR_ARG, "z1 must exceed z0");
    Grid3* g = new Grid3();
    G->g3 = g;
    g->plan = new Plan3();
    Plan3& pl = *g->plan;
    const int nx = desc->nx, ny = desc->ny, nz = desc->nz;
    g->sh = Sh3{nx, ny, nz};
    const Sh3& sh = g->sh;
    g->zeta = nz / (desc->z1 - desc->z0);
    g->nc = sh.size(C3);
    g->nxf = sh.size(XF3);
    g->nyf = sh.size(YF3);
    g->nxy = sh.size(XY3);
    long long o = 0;
    for (int f = 0; f <= NSP; ++f) {
        g->off[f] = o;
        o += g->nc;
    }
    g->off[NSP + 1] = o;
    o += g->nxf;
    g->off[NSP + 2] = o;
    o += g->nyf;
    g->off[NSP + 3] = o;
    o += g->nc;
    g->nstate = o;
    G->nstate = (int)o;
    const long long nc = g->nc, nxf = g->nxf, nyf = g->nyf, nxy = g->nxy;
    // ---------------- memory ----------------
    const long long n_c = 15 + 9 * NSP + 12 + 10 + 4 + 2 * AD_FIELDS + 3 + 5 * NSP + 9;
    const long long n_x = 4 + 5 * NSP + 9 + 8 + 2;
    const long long n_y = 4 + 5 * NSP + 9 + 8;
    const long long n_xy = 8;
    const long long pool_n = n_c * nc + n_x * nxf + n_y * nyf + n_xy * nxy + 7 * g->nstate +
                             2 * (nx + 1) + 2 * (ny + 1) + (long long)nz * nx + 16;
    cudaError_t err = cudaMalloc(&g->pool, pool_n * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&g->mask, g->nstate);
    if (err != cudaSuccess) {
        free_grid3(g);
        G->g3 = nullptr;
        return cuda_fail(err, "cudaMalloc(3-D grid)");
    }
    double* cur = g->pool;
    auto take = [&](long long n) {
        double* p = cur;
        cur += n;
        return p;
    };
    for (double** f : {&g->ru_c, &g->rv_c, &g->rw_c, &g->T, &g->p, &g->H, &g->u_c, &g->v_c, &g->w_c,
                       &g->e, &g->a, &g->mu_e, &g->K, &g->beta, &g->Tcache})
        *f = take(nc);
    for (int sp = 0; sp < NSP; ++sp)
        for (double** f : {&g->Y[sp], &g->X[sp], &g->h[sp], &g->W[sp], &g->Wd[sp], &g->G[sp],
                           &g->esc[sp], &g->cvsc[sp], &g->cvpc[sp]})
            *f = take(nc);
    for (double** f : {&g->dudx, &g->dvdy, &g->dwdz, &g->tau_xx, &g->tau_yy, &g->tau_zz, &g->Gxx,
                       &g->Gyy, &g->Gzz, &g->mux_c, &g->mvy_c, &g->mwz_c})
        *f = take(nc);
    for (double** f : {&g->S, &g->div, &g->fsw, &g->dudy_c, &g->dvdx_c, &g->dudz_c, &g->dwdx_c,
                       &g->dvdz_c, &g->dwdy_c, &g->rho_zf})
        *f = take(nc);
    for (int q = 0; q < 4; ++q) g->tc[q] = take(nc);
    for (int q = 0; q < AD_FIELDS; ++q) {
        g->raw[q] = take(nc);
        g->filt[q] = take(nc);
    }
    g->w_zf = take(nc);
    g->mwz_f = take(nc);
    for (int sp = 0; sp < NSP; ++sp)
        for (double** f : {&g->Yz[sp], &g->Gz[sp], &g->hz[sp], &g->dXdz[sp], &g->Fsz[sp]}) *f = take(nc);
    for (double** f : {&g->Hz, &g->Kz, &g->dTdz, &g->tzz_z, &g->u_z, &g->v_z, &g->txz_z, &g->tyz_z, &g->FEz})
        *f = take(nc);
    for (double** f : {&g->rho_xf, &g->u_xf, &g->mux_f, &g->mu_xf}) *f = take(nxf);
    for (int sp = 0; sp < NSP; ++sp)
        for (double** f : {&g->Yx[sp], &g->Gx[sp], &g->hx[sp], &g->dXdx[sp], &g->Fsx[sp]}) *f = take(nxf);
    for (double** f : {&g->Hx, &g->Kx, &g->dTdx, &g->txx_x, &g->v_x, &g->w_x, &g->txy_x, &g->txz_x, &g->FEx})
        *f = take(nxf);
    for (double** f : {&g->dudz_xz, &g->dwdx_xz, &g->u_xz, &g->w_xz, &g->rho_xz, &g->mu_xz,
                       &g->tau_xz, &g->Gxz, &g->tx[0], &g->tx[1]})
        *f = take(nxf);
    for (double** f : {&g->rho_yf, &g->v_yf, &g->mvy_f, &g->mu_yf}) *f = take(nyf);
    for (int sp = 0; sp < NSP; ++sp)
        for (double** f : {&g->Yy[sp], &g->Gy[sp], &g->hy[sp], &g->dXdy[sp], &g->Fsy[sp]}) *f = take(nyf);
    for (double** f : {&g->Hy, &g->Ky, &g->dTdy, &g->tyy_y, &g->u_y, &g->w_y, &g->txy_y, &g->tyz_y, &g->FEy})
        *f = take(nyf);
    for (double** f : {&g->dvdz_yz, &g->dwdy_yz, &g->v_yz, &g->w_yz, &g->rho_yz, &g->mu_yz,
                       &g->tau_yz, &g->Gyz})
        *f = take(nyf);
    for (double** f : {&g->dudy_xy, &g->dvdx_xy, &g->u_xy, &g->v_xy, &g->rho_xy, &g->mu_xy,
                       &g->tau_xy, &g->Gxy})
        *f = take(nxy);
    for (double** f : {&g->DX, &g->DY, &g->DZ, &g->SRC, &g->R, &g->Uref, &g->sigma}) *f = take(g->nstate);
    g->xi_c = take(nx);
    g->xi_f = take(nx + 1);
    g->eta_c = take(ny);
    g->eta_f = take(ny + 1);
    g->Tw = take((long long)nz * nx);
    if (cur - g->pool > pool_n) {
        free_grid3(g);
        G->g3 = nullptr;
        return fail(HYP_ERR_ARG, "internal: 3-D scratch pool too small");
    }
    // ---------------- operators ----------------
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
    err = cudaMalloc(&g->opdata, opdata.size() * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc(&g->ops, NOPS * sizeof(LineOp));
    if (err != cudaSuccess) {
        free_grid3(g);
        G->g3 = nullptr;
        return cuda_fail(err, "cudaMalloc(3-D operators)");
    }
    for (auto& op : hops) {
        op.lower = g->opdata + (size_t)op.lower;
        op.cprime = g->opdata + (size_t)op.cprime;
        op.minv = g->opdata + (size_t)op.minv;
        op.wa = g->opdata + (size_t)op.wa;
        op.wb = g->opdata + (size_t)op.wb;
        op.lm = g->opdata + (size_t)op.lm;
    }
    // periodic z operators: the fixed point of the Thomas recurrence of (alpha, 1, alpha)
    for (int kind = 0; kind < 2; ++kind)
        for (int dir = 0; dir < 2; ++dir) {
            const double alpha = kind == 0 ? 3.0 / 10.0 : 9.0 / 62.0;
            const double wa0 = kind == 0 ? 3.0 / 4.0 : 63.0 / 62.0;          // a/2 or a
            const double wb0 = kind == 0 ? 1.0 / 20.0 : 17.0 / 62.0 / 3.0;   // b/2 or b/3
            double cp = 0.0, mi = 1.0;
            for (int it = 0; it < 400; ++it) {
                mi = 1.0 / (1.0 - alpha * cp);
                cp = alpha * mi;
            }
            Line3& L = g->zop[kind][dir];
            memset(&L, 0, sizeof(L));
            L.axis = 2;
            L.kind = kind;
            L.dir = dir;
            L.wa = wa0 * mi;
            L.wb = wb0 * mi;
            L.lm = alpha * mi;
            L.cp = cp;
        }
    // ---------------- host geometry ----------------
    std::vector<double> xc(nx), xf(nx + 1), yc(ny), yf(ny + 1), xi_c(nx), xi_f(nx + 1), eta_c(ny),
        eta_f(ny + 1);
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
    // reference profile (the two-dimensional one, evaluated on the device at every node)
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
        P.Yinf[sp] = gd.Y_inf[sp];
    }
    P.shock = cas->flow == 1;
    P.theta = cas->shock_deflection_deg * 3.14159265358979323846 / 180.0;
    if (P.shock) P.sh = oblique_shock(gd.mach, P.theta, gd.gamma_inf);
    // jet: the sonic jet's state, the wall temperature of the heat flux on the wall faces
    Jet3 jet;
    memset(&jet, 0, sizeof(jet));
    std::vector<double> Tw((size_t)nz * nx, cas->T_wall / gd.T_ref);
    if (cas->jet) {
        jet.on = 1;
        jet.x = cas->jet_x;
        jet.z = cas->jet_z;
        jet.r = cas->jet_radius;
        jet.edge = cas->jet_edge;
        jet.height = 2.0;      // plume height of the initial state, in orifice radii
        jet.Lz = desc->z1 - desc->z0;
        jet.T = cas->jet_T_ratio * gd.T_inf;
        jet.p = cas->jet_J * gd.mach * gd.mach * gd.p_inf;
        jet.v = sqrt(gd.gamma_inf * gd.R_inf * jet.T) / gd.a_inf;
        if (!(jet.r > 0 && jet.edge > 0 && jet.T > 0 && jet.p > 0))
            return fail(HYP_ERR_ARG, "the jet needs a positive radius, edge, J and temperature ratio");
        const double dzc = (desc->z1 - desc->z0) / nz;
        for (int k = 0; k < nz; ++k)
            for (int i = 0; i < nx; ++i) {
                const double f = jet.blend(xc[i], desc->z0 + dzc * (k + 0.5));
                Tw[(size_t)k * nx + i] = (cas->T_wall + (jet.T - cas->T_wall) * f) / gd.T_ref;
            }
    }
    // ---------------- plans ----------------
    const bool wall = cas->wall != 0;
    Line3 base;
    memset(&base, 0, sizeof(base));
    base.scale = 1.0;
    auto xy = [&](int opid, int axis, const double* in, int tin, double* out, int tout,
                  const double* metric, double scale = 1.0, const double* wall_arr = nullptr) {
        Line3 L = base;
        L.op = g->ops + opid;
        L.axis = axis;
        L.in = in;
        L.tin = tin;
        L.out = out;
        L.tout = tout;
        L.metric = metric;
        L.scale = scale;
        L.wall = 0.0;
        L.wall_arr = wall_arr;
        return L;
    };
    auto zl = [&](int kind, int dir, const double* in, int t, double* out, double scale = 1.0) {
        Line3 L = g->zop[kind][dir];
        L.in = in;
        L.tin = L.tout = t;
        L.out = out;
        L.scale = scale;
        return L;
    };
    const int yicfw = wall ? OY_ICFW : OY_ICF, ydcfw = wall ? OY_DCFW : OY_DCF;
    const double ze = g->zeta;
    auto soff = [&](int f) { return (const double*)(size_t)g->off[f]; };
    // P1: state-reading jobs (`in` is an element offset into U)
    pl.p1.lines = {xy(OX_IFC, 0, soff(NSP + 1), XF3, g->ru_c, C3, nullptr),
             xy(OY_IFC, 1, soff(NSP + 2), YF3, g->rv_c, C3, nullptr),
             zl(0, 1, soff(NSP + 3), C3, g->rw_c),
             xy(OX_ICF, 0, soff(0), C3, g->rho_xf, XF3, nullptr),
             xy(OY_ICF, 1, soff(0), C3, g->rho_yf, YF3, nullptr),
             zl(0, 0, soff(0), C3, g->rho_zf),
             xy(OX_DFC, 0, soff(NSP + 1), XF3, g->DX + g->off[0], C3, g->xi_c, -1.0),
             xy(OY_DFC, 1, soff(NSP + 2), YF3, g->DY + g->off[0], C3, g->eta_c, -1.0),
             zl(1, 1, soff(NSP + 3), C3, g->DZ + g->off[0], -ze)};
    pl.p3.lines = {xy(OX_DFC, 0, g->u_xf, XF3, g->dudx, C3, g->xi_c),
             xy(OY_DFC, 1, g->v_yf, YF3, g->dvdy, C3, g->eta_c),
             zl(1, 1, g->w_zf, C3, g->dwdz, ze),
             xy(ydcfw, 1, g->u_xf, XF3, g->dudy_xy, XY3, g->eta_f),
             xy(OX_DCF, 0, g->v_yf, YF3, g->dvdx_xy, XY3, g->xi_f),
             xy(yicfw, 1, g->u_xf, XF3, g->u_xy, XY3, nullptr),
             xy(OX_ICF, 0, g->v_yf, YF3, g->v_xy, XY3, nullptr),
             xy(OY_ICF, 1, g->rho_xf, XF3, g->rho_xy, XY3, nullptr),
             zl(1, 0, g->u_xf, XF3, g->dudz_xz, ze),
             xy(OX_DCF, 0, g->w_zf, C3, g->dwdx_xz, XF3, g->xi_f),
             zl(0, 0, g->u_xf, XF3, g->u_xz),
             xy(OX_ICF, 0, g->w_zf, C3, g->w_xz, XF3, nullptr),
             zl(0, 0, g->rho_xf, XF3, g->rho_xz),
             zl(1, 0, g->v_yf, YF3, g->dvdz_yz, ze),
             xy(ydcfw, 1, g->w_zf, C3, g->dwdy_yz, YF3, g->eta_f),
             zl(0, 0, g->v_yf, YF3, g->v_yz),
             xy(yicfw, 1, g->w_zf, C3, g->w_yz, YF3, nullptr),
             zl(0, 0, g->rho_yf, YF3, g->rho_yz),
             xy(OX_IFC, 0, g->mux_f, XF3, g->mux_c, C3, nullptr),
             xy(OY_IFC, 1, g->mvy_f, YF3, g->mvy_c, C3, nullptr),
             zl(0, 1, g->mwz_f, C3, g->mwz_c)};
    // artificial diffusivity: edge derivatives to the centres (y then x; x then z; y then z)
    pl.ad1.lines = {xy(OY_IFC, 1, g->dudy_xy, XY3, g->tx[0], XF3, nullptr),
              xy(OY_IFC, 1, g->dvdx_xy, XY3, g->tx[1], XF3, nullptr),
              xy(OX_IFC, 0, g->dudz_xz, XF3, g->tc[0], C3, nullptr),
              xy(OX_IFC, 0, g->dwdx_xz, XF3, g->tc[1], C3, nullptr),
              xy(OY_IFC, 1, g->dvdz_yz, YF3, g->tc[2], C3, nullptr),
              xy(OY_IFC, 1, g->dwdy_yz, YF3, g->tc[3], C3, nullptr)};
    pl.ad2.lines = {xy(OX_IFC, 0, g->tx[0], XF3, g->dudy_c, C3, nullptr),
              xy(OX_IFC, 0, g->tx[1], XF3, g->dvdx_c, C3, nullptr),
              zl(0, 1, g->tc[0], C3, g->dudz_c),
              zl(0, 1, g->tc[1], C3, g->dwdx_c),
              zl(0, 1, g->tc[2], C3, g->dvdz_c),
              zl(0, 1, g->tc[3], C3, g->dwdy_c)};
    // under HYP_MIXED the jobs feeding only the diffusive fluxes (viscosities, diffusion and
    // conduction coefficients, gradients of X_s and T, stresses, the velocities of the viscous
    // work) run their rows in binary32; those feeding the convective fluxes stay FP64
    auto f = [](Line3 L) {
        L.f32 = 1;
        return L;
    };
    pl.mu.lines = {f(xy(OX_ICF, 0, g->mu_e, C3, g->mu_xf, XF3, nullptr)),
                   f(xy(OY_ICF, 1, g->mu_e, C3, g->mu_yf, YF3, nullptr))};
    // edge viscosities from the face ones (the jobs of a list run in order on one stream)
    pl.mu.lines.push_back(f(zl(0, 0, g->mu_xf, XF3, g->mu_xz)));
    pl.mu.lines.push_back(f(zl(0, 0, g->mu_yf, YF3, g->mu_yz)));
    pl.mu.lines.push_back(f(xy(OY_ICF, 1, g->mu_xf, XF3, g->mu_xy, XY3, nullptr)));
    std::vector<Line3>& F = pl.face.lines;
    std::vector<Line3>& FB = pl.faceb.lines;
    for (int sp = 0; sp < NSP; ++sp) {
        F.push_back(xy(OX_ICF, 0, g->Y[sp], C3, g->Yx[sp], XF3, nullptr));
        F.push_back(f(xy(OX_ICF, 0, g->G[sp], C3, g->Gx[sp], XF3, nullptr)));
        F.push_back(f(xy(OX_ICF, 0, g->h[sp], C3, g->hx[sp], XF3, nullptr)));
        F.push_back(f(xy(OX_DCF, 0, g->X[sp], C3, g->dXdx[sp], XF3, g->xi_f)));
        F.push_back(xy(OY_ICF, 1, g->Y[sp], C3, g->Yy[sp], YF3, nullptr));
        F.push_back(f(xy(OY_ICF, 1, g->G[sp], C3, g->Gy[sp], YF3, nullptr)));
        F.push_back(f(xy(OY_ICF, 1, g->h[sp], C3, g->hy[sp], YF3, nullptr)));
        F.push_back(f(xy(OY_DCF, 1, g->X[sp], C3, g->dXdy[sp], YF3, g->eta_f)));
        F.push_back(zl(0, 0, g->Y[sp], C3, g->Yz[sp]));
        F.push_back(f(zl(0, 0, g->G[sp], C3, g->Gz[sp])));
        F.push_back(f(zl(0, 0, g->h[sp], C3, g->hz[sp])));
        F.push_back(f(zl(1, 0, g->X[sp], C3, g->dXdz[sp], ze)));
    }
    F.push_back(xy(OX_ICF, 0, g->H, C3, g->Hx, XF3, nullptr));
    F.push_back(f(xy(OX_ICF, 0, g->K, C3, g->Kx, XF3, nullptr)));
    F.push_back(f(xy(OX_DCF, 0, g->T, C3, g->dTdx, XF3, g->xi_f)));
    FB.push_back(f(xy(OX_ICF, 0, g->tau_xx, C3, g->txx_x, XF3, nullptr)));
    F.push_back(f(xy(OX_ICF, 0, g->v_c, C3, g->v_x, XF3, nullptr)));
    F.push_back(f(xy(OX_ICF, 0, g->w_c, C3, g->w_x, XF3, nullptr)));
    FB.push_back(f(xy(OY_IFC, 1, g->tau_xy, XY3, g->txy_x, XF3, nullptr)));
    FB.push_back(f(zl(0, 1, g->tau_xz, XF3, g->txz_x)));
    F.push_back(xy(OY_ICF, 1, g->H, C3, g->Hy, YF3, nullptr));
    F.push_back(f(xy(OY_ICF, 1, g->K, C3, g->Ky, YF3, nullptr)));
    F.push_back(f(xy(ydcfw, 1, g->T, C3, g->dTdy, YF3, g->eta_f, 1.0, wall ? g->Tw : nullptr)));
    FB.push_back(f(xy(OY_ICF, 1, g->tau_yy, C3, g->tyy_y, YF3, nullptr)));
    F.push_back(f(xy(yicfw, 1, g->u_c, C3, g->u_y, YF3, nullptr)));
    F.push_back(f(xy(yicfw, 1, g->w_c, C3, g->w_y, YF3, nullptr)));
    FB.push_back(f(xy(OX_IFC, 0, g->tau_xy, XY3, g->txy_y, YF3, nullptr)));
    FB.push_back(f(zl(0, 1, g->tau_yz, YF3, g->tyz_y)));
    F.push_back(zl(0, 0, g->H, C3, g->Hz));
    F.push_back(f(zl(0, 0, g->K, C3, g->Kz)));
    F.push_back(f(zl(1, 0, g->T, C3, g->dTdz, ze)));
    FB.push_back(f(zl(0, 0, g->tau_zz, C3, g->tzz_z)));
    F.push_back(f(zl(0, 0, g->u_c, C3, g->u_z)));
    F.push_back(f(zl(0, 0, g->v_c, C3, g->v_z)));
    FB.push_back(f(xy(OX_IFC, 0, g->tau_xz, XF3, g->txz_z, C3, nullptr)));
    FB.push_back(f(xy(OY_IFC, 1, g->tau_yz, YF3, g->tyz_z, C3, nullptr)));
    std::vector<Line3>& D = pl.divs.lines;
    for (int sp = 1; sp < NSP; ++sp) {
        D.push_back(xy(OX_DFC, 0, g->Fsx[sp], XF3, g->DX + g->off[sp], C3, g->xi_c, -1.0));
        D.push_back(xy(OY_DFC, 1, g->Fsy[sp], YF3, g->DY + g->off[sp], C3, g->eta_c, -1.0));
        D.push_back(zl(1, 1, g->Fsz[sp], C3, g->DZ + g->off[sp], -ze));
    }
    D.push_back(xy(OX_DFC, 0, g->FEx, XF3, g->DX + g->off[NSP], C3, g->xi_c, -1.0));
    D.push_back(xy(OY_DFC, 1, g->FEy, YF3, g->DY + g->off[NSP], C3, g->eta_c, -1.0));
    D.push_back(zl(1, 1, g->FEz, C3, g->DZ + g->off[NSP], -ze));
    D.push_back(xy(OX_DCF, 0, g->Gxx, C3, g->DX + g->off[NSP + 1], XF3, g->xi_f, -1.0));
    D.push_back(xy(OY_DFC, 1, g->Gxy, XY3, g->DY + g->off[NSP + 1], XF3, g->eta_c, -1.0));
    D.push_back(zl(1, 1, g->Gxz, XF3, g->DZ + g->off[NSP + 1], -ze));
    D.push_back(xy(OX_DFC, 0, g->Gxy, XY3, g->DX + g->off[NSP + 2], YF3, g->xi_c, -1.0));
    D.push_back(xy(OY_DCF, 1, g->Gyy, C3, g->DY + g->off[NSP + 2], YF3, g->eta_f, -1.0));
    D.push_back(zl(1, 1, g->Gyz, YF3, g->DZ + g->off[NSP + 2], -ze));
    D.push_back(xy(OX_DFC, 0, g->Gxz, XF3, g->DX + g->off[NSP + 3], C3, g->xi_c, -1.0));
    D.push_back(xy(OY_DFC, 1, g->Gyz, YF3, g->DY + g->off[NSP + 3], C3, g->eta_c, -1.0));
    D.push_back(zl(1, 0, g->Gzz, C3, g->DZ + g->off[NSP + 3], -ze));
    // launches: the independent phases put their x/y lines before their z lines and batch each
    // kind; the viscosity phase keeps its order (its edge values come from its face values)
    Phase3* phases[] = {&pl.p1, &pl.p3, &pl.ad1, &pl.ad2, &pl.mu, &pl.face, &pl.faceb, &pl.divs};
    pl.mu.slot_base = pl.faceb.slot_base = BATCH3;
    for (Phase3* ph : phases) {
        std::vector<Line3>& V = ph->lines;
        if (ph != &pl.mu)
            std::stable_partition(V.begin(), V.end(), [](const Line3& L) { return L.axis != 2; });
        for (size_t i = 0; i < V.size();) {
            const int z = V[i].axis == 2;
            size_t e = i;
            while (e < V.size() && (V[e].axis == 2) == z && e - i < (size_t)BATCH3) ++e;
            ph->launches.push_back(Launch3{z, (int)i, (int)(e - i), 0});
            i = e;
        }
    }
    // x and y lines as segmented line jobs: plane groups for y; per launch, segments as in two
    // dimensions (lines split while the launch has fewer than 40960 threads); one forward-sweep
    // buffer per position in a launch
    {
        // binary32 copies of the metrics for the jobs that run binary32 rows
        err = cudaMalloc(&g->metf, (2 * (nx + ny) + 2) * sizeof(float));
        if (err != cudaSuccess) return cuda_fail(err, "cudaMalloc(3-D binary32 metrics)");
        const double* met_d[4] = {g->xi_c, g->xi_f, g->eta_c, g->eta_f};
        const long long met_off[4] = {0, nx, 2LL * nx + 1, 2LL * nx + 1 + ny};
        std::vector<LineJob> lj;
        std::vector<int> slot;
        long long tmp_n = 0;
        int slots = 1;
        for (Phase3* ph : phases)
            for (Launch3& b : ph->launches) {
                if (b.z) continue;
                const int j0 = (int)lj.size();
                std::vector<int> ns(b.count), m(b.count);
                long long threads = 0;
                for (int i = 0; i < b.count; ++i) {
                    Line3& L = ph->lines[b.first + i];
                    m[i] = hops[L.op - g->ops].m;
                    LineJob j;
                    memset(&j, 0, sizeof(j));
                    j.op = L.op;
                    j.in_state = ph == &pl.p1 ? 1 : 0;
                    j.in = L.in;
                    j.out = L.out;
                    j.scale = L.scale;
                    j.metric = L.metric;
                    j.wall_value = L.wall;
                    j.wall_arr = L.wall_arr;
                    j.f32ok = L.f32;
                    for (int k = 0; k < 4; ++k)
                        if (L.metric && L.metric == met_d[k]) j.metric_f = g->metf + met_off[k];
                    if (L.axis == 0) {
                        j.in_ls = sh.pitch(L.tin);
                        j.out_ls = sh.pitch(L.tout);
                        j.in_es = j.out_es = 1;
                        j.nlines = sh.rows(L.tin) * nz;
                    } else {
                        j.lpp = sh.pitch(L.tin);
                        j.in_ls = j.out_ls = 1;
                        j.in_es = sh.pitch(L.tin);
                        j.out_es = sh.pitch(L.tout);
                        j.in_ps = sh.plane(L.tin);
                        j.out_ps = sh.plane(L.tout);
                        j.nlines = sh.pitch(L.tin) * nz;
                    }
                    ns[i] = 1;
                    while (ns[i] < LINE_BLOCK / 2 && (m[i] + ns[i] - 1) / ns[i] > 260) ns[i] *= 2;
                    threads += (long long)j.nlines * ns[i];
                    tmp_n = std::max(tmp_n, sh.size(L.tout));
                    L.job = (int)lj.size();
                    lj.push_back(j);
                    slot.push_back(ph->slot_base + i);
                }
                while (threads < 40960) {
                    bool grew = false;
                    threads = 0;
                    for (int i = 0; i < b.count; ++i) {
                        if (ns[i] < LINE_BLOCK / 2 && (m[i] + 2 * ns[i] - 1) / (2 * ns[i]) >= 32) {
                            ns[i] *= 2;
                            grew = true;
                        }
                        threads += (long long)lj[j0 + i].nlines * ns[i];
                    }
                    if (!grew) break;
                }
                for (int i = 0; i < b.count; ++i) {
                    LineJob& j = lj[j0 + i];
                    j.nseg = ns[i];
                    const int lpb = LINE_BLOCK / ns[i];
                    b.blocks = std::max(b.blocks, (j.nlines + lpb - 1) / lpb);
                }
                slots = std::max(slots, ph->slot_base + b.count);
            }
        err = cudaMalloc(&g->ltmp, (size_t)slots * tmp_n * sizeof(double));
        if (err == cudaSuccess) err = cudaMalloc(&g->jobs, lj.size() * sizeof(LineJob));
        if (err != cudaSuccess) return cuda_fail(err, "cudaMalloc(3-D line jobs)");
        for (size_t k = 0; k < lj.size(); ++k) lj[k].tmp = g->ltmp + (size_t)slot[k] * tmp_n;
        HYP_CUDA(cudaMemcpyAsync(g->jobs, lj.data(), lj.size() * sizeof(LineJob), cudaMemcpyHostToDevice, s));
        HYP_CUDA(cudaStreamSynchronize(s));
    }
    // second stream and its events (phases that do not wait on the closure)
    HYP_CUDA(cudaStreamCreateWithFlags(&G->side, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
        HYP_CUDA(cudaEventCreateWithFlags(&G->fork[k], cudaEventDisableTiming));
        HYP_CUDA(cudaEventCreateWithFlags(&G->join[k], cudaEventDisableTiming));
    }
    // ---------------- uploads, reference, initial state ----------------
#define UP3(dst, src, bytes) HYP_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s))
    UP3(g->ops, hops.data(), NOPS * sizeof(LineOp));
    UP3(g->opdata, opdata.data(), opdata.size() * sizeof(double));
    UP3(g->xi_c, xi_c.data(), nx * sizeof(double));
    UP3(g->xi_f, xi_f.data(), (nx + 1) * sizeof(double));
    UP3(g->eta_c, eta_c.data(), ny * sizeof(double));
    UP3(g->eta_f, eta_f.data(), (ny + 1) * sizeof(double));
    std::vector<float> metf_h;
    for (const auto* v : {&xi_c, &xi_f, &eta_c, &eta_f})
        for (double x : *v) metf_h.push_back((float)x);
    UP3(g->metf, metf_h.data(), metf_h.size() * sizeof(float));
    UP3(g->Tw, Tw.data(), Tw.size() * sizeof(double));
    k_reference3<<<blocks3(g->nstate), 128, 0, s>>>(gd, P, *desc, jet, *g);
    const bool noisy = cas->noise && cas->noise_amp > 0;
    if (noisy) UP3(g->R, cas->noise, g->nstate * sizeof(double));
    k_initial<<<blocks3(g->nstate), 256, 0, s>>>(g->nstate, g->Uref, g->mask, noisy ? g->R : nullptr,
                                                 cas->noise_amp, U);
    HYP_CUDA(cudaGetLastError());
#undef UP3
    HYP_CUDA(cudaMemsetAsync(dQ, 0, g->nstate * sizeof(double), s));
    HYP_CUDA(cudaMemsetAsync(g->SRC, 0, g->nstate * sizeof(double), s));
    HYP_CUDA(cudaMemsetAsync(G->status, 0, sizeof(unsigned), s));
    k_fill<<<blocks3(nc), 256, 0, s>>>(g->Tcache, nc, 1000.0);
    HYP_CUDA(cudaGetLastError());
    HYP_CUDA(cudaStreamSynchronize(s));
    G->Uref = g->Uref;
    G->sigma = g->sigma;
    G->mask = nullptr;
    return HYP_OK;
}
