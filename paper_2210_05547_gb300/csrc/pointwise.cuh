// Pointwise steps of the right-hand side (Eqs. 5-11, 26; Secs. 2.2, 3.3) as device bodies over an
// index range. Each body processes indices lo + threadIdx.x, lo + threadIdx.x + stride, ... < hi
// of one grid: the single-grid kernels (rhs.cu) call it with a grid-stride range, the batched
// persistent kernels (batch.cu) with one tile of one grid at a time. Both run the same
// arithmetic, so a grid's results do not depend on what it is batched with.
#pragma once

#include "grid.h"
#include "thermo.cuh"

namespace hyp {

__device__ __forceinline__ void atomic_status(unsigned* st, unsigned bits) {
    if (bits) atomicOr(st, bits);
}

// Resident blocks of 128 threads per SM the closure kernels are compiled for: three (164-168
// registers; left to itself ptxas picks 128 registers and spills more for five-species air; for
// eleven-species air the cap of 168 spills, yet measured faster than two blocks at 255 registers:
// 74.3 against 67.4 Mpts*RHS/s).
#define CLOSURE_MIN_BLOCKS 3   // also for the mixed closure (4 and 2 blocks measured slower)

// Reciprocals of the freestream scales, computed once per thread by the caller of closure_point
// (the point loop multiplies by them).
struct ScaleInv {
    double iT_ref, imu_inf, ik_inf, ia_inf, iRe, iRePr, ip_ref, ia2, d_nd, wscale;
};

__device__ __forceinline__ ScaleInv scale_inv(const Scales& sc) {
    ScaleInv c;
    c.iT_ref = 1.0 / sc.T_ref;
    c.imu_inf = 1.0 / sc.mu_inf;
    c.ik_inf = 1.0 / sc.k_inf;
    c.ia_inf = 1.0 / sc.a_inf;
    c.iRe = 1.0 / sc.Re;
    c.iRePr = 1.0 / (sc.Re * sc.Pr);
    c.ip_ref = __ddiv_rn(__dmul_rn(c.ia_inf, c.ia_inf), sc.rho_inf);
    c.ia2 = __dmul_rn(c.ia_inf, c.ia_inf);
    c.d_nd = __dmul_rn(__dmul_rn(sc.rho_inf, c.imu_inf), c.iRe);   // D (SI) -> rho_inf D / (mu_inf Re)
    c.wscale = __ddiv_rn(__dmul_rn(sc.L_ref, c.ia_inf), sc.rho_inf);   // w (SI) -> nondimensional
    return c;
}

// (A) primitives and the closure at one cell centre (MIXED: binary32 transport, Sec. 2.2).
// LTE: the gas is in local thermodynamic equilibrium (its own instantiation, so that the other
// kinds' code keeps its registers); the species fields are passive and the closure ignores them.
// The point is a function of its own, not inlined: the single-grid kernel and the batched
// executor call this one compiled body, so a member's results do not depend on which of the
// two ran it (inlined into two different kernels, the compiler's fusion of multiplies and adds
// may differ between the copies by a rounding).
template <bool MIXED, bool LTE>
__device__ __noinline__ void closure_point(const GasDev& g, const Scales& sc, const ScaleInv& c,
                                           const GridView& v, const double* __restrict__ U,
                                           const Scratch& s, int idx) {
    const bool cpg = sc.kind == HYP_GAS_CPG;
    const bool tpg = sc.kind == HYP_GAS_TPG;
    const bool cneq = sc.kind == HYP_GAS_CNEQ;
    const double iT_ref = c.iT_ref, imu_inf = c.imu_inf, ik_inf = c.ik_inf, ia_inf = c.ia_inf;
    const double iRe = c.iRe, iRePr = c.iRePr, ip_ref = c.ip_ref, ia2 = c.ia2, d_nd = c.d_nd;
    const double wscale = c.wscale;
    {
        const double rho = U[v.off[0] + idx];
        const double irho = cl_rcp(rho);
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
        const double u = s.ru_c[idx] * irho;
        const double vv = s.rv_c[idx] * irho;
        const double e = rhoE * irho - 0.5 * (u * u + vv * vv);
        double T, p, mu, k, a;
        double h[NSP], wd[NSP], X[NSP], W[NSP], Wd[NSP];
        if constexpr (LTE) {
            ClosureOut o;
            double Yeq[NSP], kr;
            // the previous evaluation at this point seeds this one: the element potentials start
            // the first equilibrium solve, and the temperature starts a step (e - e_c) / c_v,eq
            // off the cached one (kept in the first species-energy cache arrays, which the
            // equilibrium closure does not otherwise use)
            const double e_si = e * sc.a_inf * sc.a_inf;
            double lam[2] = {NAN, NAN}, cv_eq = 0.0;
            double T0 = s.Tcache[idx];
            if (v.predict) {
                lam[0] = s.esc[0][idx];
                lam[1] = s.esc[1][idx];
                const double ec = s.esc[2][idx], cvc = s.esc[3][idx];
                if (cvc > 0.0 && isfinite(ec)) T0 += (e_si - ec) / cvc;
            }
            lte_closure<MIXED>(g, rho * sc.rho_inf, e_si, T0, Yeq, kr, o, lam, &cv_eq);
            atomic_status(v.status, o.status);
            s.Tcache[idx] = o.T;
            s.esc[0][idx] = lam[0];
            s.esc[1][idx] = lam[1];
            s.esc[2][idx] = e_si;
            s.esc[3][idx] = cv_eq;
            T = __dmul_rn(o.T, iT_ref);
            p = __dmul_rn(o.p, ip_ref);
            mu = __dmul_rn(o.mu, imu_inf);
            k = __dmul_rn(o.k, ik_inf);
            a = __dmul_rn(o.a, ia_inf);
#pragma unroll
            for (int sp = 0; sp < NSP; ++sp) {
                h[sp] = wd[sp] = W[sp] = Wd[sp] = 0.0;
                X[sp] = o.X[sp];
            }
        } else if (cpg) {
            T = sc.gamma_inf * e;
            p = rho * (sc.gamma_inf - 1.0) / sc.gamma_inf * T;
            const double Td = T * sc.T_ref;
            mu = SUTH_C1 * Td * sqrt(Td) / (Td + SUTH_TS) / sc.mu_inf;
            k = mu;
            a = sqrt(sc.gamma_inf * p / rho);
#pragma unroll
            for (int sp = 0; sp < NSP; ++sp) h[sp] = wd[sp] = X[sp] = W[sp] = Wd[sp] = 0.0;
        } else if (tpg) {
            // thermally perfect gas (Eqs. 22-25): Newton on e(T) from the cached temperature
            const TpgModel m{sc.tpg_cp0, (sc.gamma_inf - 1.0) / sc.gamma_inf, sc.tpg_theta, sc.R_inf};
            unsigned st = rho > 0.0 ? 0u : HYP_STATUS_NONPHYSICAL;
            const double T0 = v.predict ? s.Tcache[idx] : sc.gamma_inf * e * sc.T_ref;
            const double Tk = m.temperature(e * sc.a_inf * sc.a_inf, T0, st);
            atomic_status(v.status, st);
            s.Tcache[idx] = Tk;
            T = Tk / sc.T_ref;
            p = rho * (sc.gamma_inf - 1.0) / sc.gamma_inf * T;
            mu = SUTH_C1 * Tk * sqrt(Tk) / (Tk + SUTH_TS) / sc.mu_inf;
            k = keyes(Tk) / sc.k_inf;
            const double cp = m.cp(Tk);
            a = sqrt(cp / (cp - sc.R_inf) * p / rho);
#pragma unroll
            for (int sp = 0; sp < NSP; ++sp) h[sp] = wd[sp] = X[sp] = W[sp] = Wd[sp] = 0.0;
        } else {
            const double e_si = e * sc.a_inf * sc.a_inf;
            double T0 = s.Tcache[idx];
            if (v.predict) {
                // second-order step from the cached species state with the new composition:
                // e(Tc + d) ~ ec + cv d + cvp d^2 / 2 = e
                double ec = 0.0, cvc = 0.0, cvpc = 0.0;
#pragma unroll
                for (int sp = 0; sp < NSP; ++sp) {
                    ec += Y[sp] * s.esc[sp][idx];
                    cvc += Y[sp] * s.cvsc[sp][idx];
                    cvpc += Y[sp] * s.cvpc[sp][idx];
                }
                const double icv = cl_rcp(cvc);
                const double d1 = (e_si - ec) * icv;
                T0 += d1 - 0.5 * cvpc * d1 * d1 * icv;
            }
            ClosureOut o;
            closure_si_p<MIXED>(g, rho * sc.rho_inf, e_si, Y, T0, cneq, cneq && !v.sm, o);
            atomic_status(v.status, o.status);
            s.Tcache[idx] = o.T;
#pragma unroll
            for (int sp = 0; sp < NSP; ++sp) {
                s.esc[sp][idx] = o.es[sp];
                s.cvsc[sp][idx] = o.cvs[sp];
                s.cvpc[sp][idx] = o.cvps[sp];
            }
            T = __dmul_rn(o.T, iT_ref);
            p = __dmul_rn(o.p, ip_ref);
            mu = __dmul_rn(o.mu, imu_inf);
            k = __dmul_rn(o.k, ik_inf);
            a = __dmul_rn(o.a, ia_inf);
            double ym = 0.0;
#pragma unroll
            for (int sp = 0; sp < NSP; ++sp) ym += Y[sp] * g.invM[sp];
#pragma unroll
            for (int sp = 0; sp < NSP; ++sp) {
                h[sp] = __dmul_rn(o.h[sp], ia2);
                wd[sp] = __dmul_rn(o.wdot[sp], wscale);
                X[sp] = o.X[sp];
                // the electron's diffusive flux follows the ions (flux_point): no coefficient
                W[sp] = cneq && (!HAS_CHARGE || g.heavy[sp]) ? rho * g.M[sp] * ym : 0.0;
                Wd[sp] = cneq ? __dmul_rn(W[sp], __dmul_rn(o.D[sp], d_nd)) : 0.0;
            }
        }
        s.T[idx] = T;
        s.p[idx] = p;
        s.H[idx] = (rhoE + p) * irho;
        s.u_c[idx] = u;
        s.v_c[idx] = vv;
        s.e[idx] = e;
        s.a[idx] = a;
        s.mu_e[idx] = __dmul_rn(mu, iRe);
        s.K[idx] = __dmul_rn(k, iRePr);
        if (!v.ad) s.beta[idx] = 0.0;
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp) {
            s.Y[sp][idx] = Y[sp];
            s.X[sp][idx] = X[sp];
            s.h[sp][idx] = h[sp];
            s.Wd[sp][idx] = Wd[sp];
            s.W[sp][idx] = W[sp];
            if (!v.ad) s.G[sp][idx] = Wd[sp];
        }
#pragma unroll
        for (int sp = 1; sp < NSP; ++sp) s.SRC[v.off[sp] + idx] = wd[sp];
    }
}

// (A) over an index range of one grid
template <bool MIXED, bool LTE = false>
__device__ __forceinline__ void closure_body(const GasDev& g, const Scales& sc, const GridView& v,
                                             const double* __restrict__ U, const Scratch& s,
                                             long long lo, long long hi, long long stride) {
    const ScaleInv c = scale_inv(sc);
    for (long long li = lo + threadIdx.x; li < hi; li += stride)
        closure_point<MIXED, LTE>(g, sc, c, v, U, s, (int)li);
}

// (B) face velocities and the face products of the normal momentum fluxes;
// index range: the x-faces, then the y-faces
__device__ __forceinline__ void face_vel_body(const GridView& v, const double* __restrict__ U,
                                              const Scratch& s, long long lo, long long hi,
                                              long long stride) {
    const int nxf = v.ny * (v.nx + 1);
    for (long long li = lo + threadIdx.x; li < hi; li += stride) {
        const int i = (int)li;
        if (i < nxf) {
            const double m = U[v.off[NSP + 1] + i];
            const double u = cl_div(m, s.rho_xf[i]);
            s.u_xf[i] = u;
            s.mux_f[i] = m * u;
        } else {
            const int j = i - nxf;
            const double m = U[v.off[NSP + 2] + j];
            const double vv = cl_div(m, s.rho_yf[j]);
            s.v_yf[j] = vv;
            s.mvy_f[j] = m * vv;
        }
    }
}

// (D) artificial diffusivity: strain-rate magnitude, dilatation, Ducros switch
__device__ __forceinline__ void ad_prep_body(const Scratch& s, long long lo, long long hi,
                                             long long stride) {
    for (long long li = lo + threadIdx.x; li < hi; li += stride) {
        const int i = (int)li;
        const double ux = s.dudx[i], vy = s.dvdy[i], uy = s.dudy_c[i], vx = s.dvdx_c[i];
        const double sxy = uy + vx;
        s.S[i] = sqrt(ux * ux + vy * vy + 0.5 * sxy * sxy);
        const double dv = ux + vy;
        const double om = vx - uy;
        s.div[i] = dv;
        s.fsw[i] = dv < 0.0 ? cl_div(dv * dv, dv * dv + om * om + DUCROS_EPS) : 0.0;
    }
}

__device__ __forceinline__ double d4x(const double* f, int j, int i, int nx) {
    const int c = min(max(i, 2), nx - 3);
    const double* r = f + (long long)j * nx + c;
    return r[-2] - 4.0 * r[-1] + 6.0 * r[0] - 4.0 * r[1] + r[2];
}

__device__ __forceinline__ double d4y(const double* f, int j, int i, int nx, int ny) {
    const int c = min(max(j, 2), ny - 3);
    const double* r = f + (long long)c * nx + i;
    return r[-2 * nx] - 4.0 * r[-nx] + 6.0 * r[0] - 4.0 * r[nx] + r[2 * nx];
}

__device__ __forceinline__ void ad_raw_body(bool cneq, const GridView& v,
                                            const double* __restrict__ U, const Scratch& s,
                                            long long lo, long long hi, long long stride) {
    for (long long li = lo + threadIdx.x; li < hi; li += stride) {
        const int idx = (int)li;
        const int j = idx / v.nx, i = idx - j * v.nx;
        const double dx = cl_rcp(v.xi_c[i]), dy = cl_rcp(v.eta_c[j]);
        const double rho = U[v.off[0] + idx];
        s.raw[0][idx] = v.C_mu * rho *
                        fabs(d4x(s.S, j, i, v.nx) * dx * dx + d4y(s.S, j, i, v.nx, v.ny) * dy * dy);
        s.raw[1][idx] = v.C_beta * rho * s.fsw[idx] *
                        fabs(d4x(s.div, j, i, v.nx) * dx * dx + d4y(s.div, j, i, v.nx, v.ny) * dy * dy);
        s.raw[2][idx] = v.C_kappa * rho * cl_div(s.a[idx], s.T[idx]) *
                        fabs(d4x(s.e, j, i, v.nx) * dx + d4y(s.e, j, i, v.nx, v.ny) * dy);
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp)
            s.raw[3 + sp][idx] =
                cneq ? v.C_D * s.a[idx] *
                           fabs(d4x(s.Y[sp], j, i, v.nx) * dx + d4y(s.Y[sp], j, i, v.nx, v.ny) * dy)
                     : 0.0;
    }
}

// Gaussian filter of the eight raw diffusivities along x (dir 0) or y (dir 1); indices clamp.
// FP64: index range field f * nc + point, one field value per thread (the filter is bound by the
// FP64 pipe, nine operations a point; the threads' independent loads hide the latency).
// MIXED: in binary32 (truncated inputs, binary32 weights and sums, the result widened exactly)
// over the points, each thread filtering every field at its point, so the point's indices and
// clamped neighbours are computed once for the eight fields (integer work bounds the binary32
// form). The filtered fields are the artificial diffusivities, nonnegative and entering only the
// diffusive fluxes, where the few 2^-24 of relative error are immaterial.
template <bool MIXED>
__device__ __forceinline__ void gauss_body(const GridView& v, const Scratch& s, int dir,
                                           long long lo, long long hi, long long stride) {
    if constexpr (MIXED) {
        for (long long li = lo + threadIdx.x; li < hi; li += stride) {
            const int idx = (int)li;
            const int j = idx / v.nx, i = idx - j * v.nx;
            int nb[8];                                   // neighbours -4..-1, +1..+4, clamped
            if (dir == 0) {
#pragma unroll
                for (int d = 1; d <= 4; ++d) {
                    nb[d - 1] = j * v.nx + max(i - d, 0);
                    nb[3 + d] = j * v.nx + min(i + d, v.nx - 1);
                }
            } else {
#pragma unroll
                for (int d = 1; d <= 4; ++d) {
                    nb[d - 1] = max(j - d, 0) * v.nx + i;
                    nb[3 + d] = min(j + d, v.ny - 1) * v.nx + i;
                }
            }
#pragma unroll 2
            for (int f = 0; f < AD_FIELDS; ++f) {
                const double* __restrict__ in = dir == 0 ? s.raw[f] : s.filt[f];
                double* __restrict__ out = dir == 0 ? s.filt[f] : s.raw[f];
                float acc = __fmul_rn(c_gauss_f[0], f32_trunc(in[idx]));
#pragma unroll
                for (int d = 1; d <= 4; ++d)
                    acc = fmaf(c_gauss_f[d], __fadd_rn(f32_trunc(in[nb[d - 1]]), f32_trunc(in[nb[3 + d]])),
                               acc);
                out[idx] = f64_of(acc);
            }
        }
    } else {
        const long long n = (long long)v.nx * v.ny;
        for (long long li = lo + threadIdx.x; li < hi; li += stride) {
            const int f = (int)(li / n);
            const int idx = (int)(li - f * n);
            const double* __restrict__ in = dir == 0 ? s.raw[f] : s.filt[f];
            double* __restrict__ out = dir == 0 ? s.filt[f] : s.raw[f];
            const int j = idx / v.nx, i = idx - j * v.nx;
            double acc = c_gauss[0] * in[idx];
            if (dir == 0) {
                const double* r = in + (long long)j * v.nx;
#pragma unroll
                for (int d = 1; d <= 4; ++d)
                    acc += c_gauss[d] * (r[max(i - d, 0)] + r[min(i + d, v.nx - 1)]);
            } else {
#pragma unroll
                for (int d = 1; d <= 4; ++d)
                    acc += c_gauss[d] * (in[(long long)max(j - d, 0) * v.nx + i] +
                                         in[(long long)min(j + d, v.ny - 1) * v.nx + i]);
            }
            out[idx] = acc;
        }
    }
}

__device__ __forceinline__ void ad_combine_body(const Scratch& s, long long lo, long long hi,
                                                long long stride) {
    for (long long li = lo + threadIdx.x; li < hi; li += stride) {
        const int i = (int)li;
        s.mu_e[i] += s.raw[0][i];
        s.beta[i] = s.raw[1][i];
        s.K[i] += s.raw[2][i];
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp) s.G[sp][i] = s.Wd[sp][i] + s.W[sp][i] * s.raw[3 + sp][i];
    }
}

// (F, I) normal stresses and momentum fluxes at centres (Eqs. 5, 6, 9)
__device__ __forceinline__ void stress_c_body(const Scratch& s, long long lo, long long hi,
                                              long long stride) {
    for (long long li = lo + threadIdx.x; li < hi; li += stride) {
        const int i = (int)li;
        const double ux = s.dudx[i], vy = s.dvdy[i];
        const double dv = ux + vy;
        const double mu = s.mu_e[i], b = s.beta[i];
        const double txx = mu * (2.0 * ux - 2.0 / 3.0 * dv) + b * dv;
        const double tyy = mu * (2.0 * vy - 2.0 / 3.0 * dv) + b * dv;
        s.tau_xx[i] = txx;
        s.tau_yy[i] = tyy;
        // normal momentum fluxes: rho u u formed on the faces, interpolated to the centres
        s.Gxx[i] = s.mux_c[i] + s.p[i] - txx;
        s.Gyy[i] = s.mvy_c[i] + s.p[i] - tyy;
    }
}

// (F, I) shear stress and cross momentum flux at corners
__device__ __forceinline__ void stress_cn_body(const Scratch& s, long long lo, long long hi,
                                               long long stride) {
    for (long long li = lo + threadIdx.x; li < hi; li += stride) {
        const int i = (int)li;
        const double txy = s.mu_cn[i] * (s.dudy_cn[i] + s.dvdx_cn[i]);
        s.tau_xy[i] = txy;
        s.Gxy[i] = s.rho_cn[i] * s.u_cn[i] * s.v_cn[i] - txy;
    }
}

// (G, H) species and energy fluxes at the x-faces (dir 0) or y-faces (dir 1) of face index i;
// SMK: the kernel carries the Stefan-Maxwell solve (used by grids with v.sm)
template <bool SMK>
__device__ __forceinline__ void flux_point(const GasDev& gd, const Scales& sc, const GridView& v,
                                           const double* __restrict__ U, const Scratch& s, int dir,
                                           int i) {
    const double* __restrict__ mom = U + v.off[NSP + 1 + dir];
    double* const* Yf = dir == 0 ? s.Yx : s.Yy;
    double* const* Gf = dir == 0 ? s.Gx : s.Gy;
    double* const* hf = dir == 0 ? s.hx : s.hy;
    double* const* dX = dir == 0 ? s.dXdx : s.dXdy;
    double* const* Fs = dir == 0 ? s.Fsx : s.Fsy;
    const double* Hf = dir == 0 ? s.Hx : s.Hy;
    const double* Kf = dir == 0 ? s.Kx : s.Ky;
    const double* dT = dir == 0 ? s.dTdx : s.dTdy;
    const double* tn = dir == 0 ? s.txx_x : s.tyy_y;      // normal stress at the face
    const double* tsh = dir == 0 ? s.txy_x : s.txy_y;     // shear stress at the face
    const double* un = dir == 0 ? s.u_xf : s.v_yf;        // velocity normal to the face
    const double* ut = dir == 0 ? s.v_x : s.u_y;          // tangential velocity
    double* FE = dir == 0 ? s.FEx : s.FEy;
    const bool wallface = dir == 1 && v.wall && i < v.nx;
    double g[NSP], J[NSP], sum = 0.0;
#pragma unroll
    for (int sp = 0; sp < NSP; ++sp) {
        g[sp] = Gf[sp][i] * dX[sp][i];
        sum += g[sp];
    }
    double q = -Kf[i] * dT[i];
    const double m = mom[i];
    if (SMK && v.sm && !wallface) {
        // Stefan-Maxwell fluxes (Eq. 17); the algebraic part above carries only the artificial
        // diffusivity in this mode
        double Yl[NSP], dXl[NSP], Jsm[NSP];
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp) {
            Yl[sp] = Yf[sp][i];
            dXl[sp] = dX[sp][i];
        }
        const double* Tf = dir == 0 ? s.Tx : s.Ty;
        const double* pf = dir == 0 ? s.px : s.py;
        const double* rf = dir == 0 ? s.rho_xf : s.rho_yf;
        stefan_maxwell_face(gd, Tf[i] * sc.T_ref, pf[i] * sc.rho_inf * sc.a_inf * sc.a_inf,
                            sc.mu_inf * sc.Re / sc.rho_inf, rf[i], Yl, dXl, Jsm);
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp) J[sp] = Jsm[sp];
    } else {
#pragma unroll
        for (int sp = 0; sp < NSP; ++sp) J[sp] = 0.0;
    }
#pragma unroll
    for (int sp = 0; sp < NSP; ++sp) J[sp] = wallface ? 0.0 : J[sp] - (g[sp] - Yf[sp][i] * sum);
    if (HAS_CHARGE && gd.ie >= 0 && !wallface) {
        // zero conduction current: J_e = M_e sum_ions J_i / M_i; the omitted first species
        // takes J_0 = -sum_{s >= 1} J_s (the diffusive mass fluxes sum to zero)
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
#pragma unroll
    for (int sp = 0; sp < NSP; ++sp) q += hf[sp][i] * J[sp];
#pragma unroll
    for (int sp = 1; sp < NSP; ++sp) Fs[sp][i] = m * Yf[sp][i] + J[sp];
    // tau . u normal component: x-face tau_xx u + tau_xy v; y-face tau_xy u + tau_yy v
    const double work = dir == 0 ? tn[i] * un[i] + tsh[i] * ut[i] : tsh[i] * ut[i] + tn[i] * un[i];
    FE[i] = m * Hf[i] + q - work;
}

// Index range: the x-faces, then the y-faces (dir < 0), or the faces of one direction.
template <bool SMK>
__device__ __forceinline__ void flux_body(const GasDev& gd, const Scales& sc, const GridView& v,
                                          const double* __restrict__ U, const Scratch& s, int dir,
                                          long long lo, long long hi, long long stride) {
    const int nxf = v.ny * (v.nx + 1);
    for (long long li = lo + threadIdx.x; li < hi; li += stride) {
        const int i = (int)li;
        if (dir >= 0) flux_point<SMK>(gd, sc, v, U, s, dir, i);
        else if (i < nxf) flux_point<SMK>(gd, sc, v, U, s, 0, i);
        else flux_point<SMK>(gd, sc, v, U, s, 1, i - nxf);
    }
}

// (J) sum of divergences, sources and sponge; Dirichlet rows; optional RK stage update
// rk: 0 right-hand side only, 1 2N-storage stage (dQ <- A dQ + dt R, U <- U + B dQ),
// 2 TVD stage, 3 first TVD stage (also stores the start state)
struct AssembleArgs {
    const double *DX, *DY, *SRC, *sigma, *Uref;
    const uint8_t* mask;
    double *U, *out, *dQ;
    int rk;
    double A, B, dt;
};

__device__ __forceinline__ void assemble_body(const AssembleArgs& a, long long lo, long long hi,
                                              long long stride) {
    for (long long li = lo + threadIdx.x; li < hi; li += stride) {
        const long long i = li;
        const double u = a.U[i];
        double r = a.DX[i] + a.DY[i] + a.SRC[i] - a.sigma[i] * (u - a.Uref[i]);
        if (a.mask[i]) r = 0.0;
        if (a.rk >= 2) {
            // TVD RK3 stage: U <- A W + B (U + dt R) with W the step's start state, which the
            // first stage (rk == 3) stores in the second register
            const double w = a.rk == 3 ? u : a.dQ[i];
            if (a.rk == 3) a.dQ[i] = u;
            a.U[i] = a.A * w + a.B * (u + a.dt * r);
        } else if (a.rk) {
            const double q = a.A * a.dQ[i] + a.dt * r;
            a.dQ[i] = q;
            a.U[i] = u + a.B * q;
        } else {
            a.out[i] = r;
        }
    }
}

// Low-pass filter of the conserved state along x (dir 0) or y (dir 1) lines of every field:
// out_i = in_i - sigma (D_m in)_i with the binomial 2m-th difference of weights c_filter_w,
// m = min(5, distance to the nearer end of the line); end points copied.
// c_filter_w[m - 1][n + m] = (-1)^n C(2m, m + n) / 4^m (exact in binary64).
static __constant__ double c_filter_w[5][11] = {
    {-1.0 / 4, 2.0 / 4, -1.0 / 4},
    {1.0 / 16, -4.0 / 16, 6.0 / 16, -4.0 / 16, 1.0 / 16},
    {-1.0 / 64, 6.0 / 64, -15.0 / 64, 20.0 / 64, -15.0 / 64, 6.0 / 64, -1.0 / 64},
    {1.0 / 256, -8.0 / 256, 28.0 / 256, -56.0 / 256, 70.0 / 256, -56.0 / 256, 28.0 / 256,
     -8.0 / 256, 1.0 / 256},
    {-1.0 / 1024, 10.0 / 1024, -45.0 / 1024, 120.0 / 1024, -210.0 / 1024, 252.0 / 1024,
     -210.0 / 1024, 120.0 / 1024, -45.0 / 1024, 10.0 / 1024, -1.0 / 1024}};

__device__ __forceinline__ void filter_body(int nx, int ny, const double* __restrict__ in,
                                            double* __restrict__ out, int dir, double sigma,
                                            long long lo, long long hi, long long stride) {
    const long long nc = (long long)nx * ny;
    const long long nxf = (long long)(nx + 1) * ny;
    for (long long idx = lo + threadIdx.x; idx < hi; idx += stride) {
        long long local;
        int pitch, rows;
        if (idx < (NSP + 1) * nc) {
            local = idx % nc;
            pitch = nx;
            rows = ny;
        } else if (idx < (NSP + 1) * nc + nxf) {
            local = idx - (NSP + 1) * nc;
            pitch = nx + 1;
            rows = ny;
        } else {
            local = idx - (NSP + 1) * nc - nxf;
            pitch = nx;
            rows = ny + 1;
        }
        const int row = (int)(local / pitch), col = (int)(local - (long long)row * pitch);
        const int pos = dir == 0 ? col : row;
        const int n = dir == 0 ? pitch : rows;
        const long long st = dir == 0 ? 1 : pitch;
        const int m = min(min(pos, n - 1 - pos), 5);
        const double f = in[idx];
        if (m == 0) {
            out[idx] = f;
            continue;
        }
        const double* w = c_filter_w[m - 1];
        const double* p = in + idx - m * st;
        double acc = 0.0;
        for (int k = 0; k <= 2 * m; ++k) acc = fma(w[k], p[k * st], acc);
        out[idx] = fma(-sigma, acc, f);
    }
}

}  // namespace hyp
