/*
 * hyp.h -- C ABI of the GB300 library for the right-hand side and explicit stage update of the
 * compressible multi-species Navier-Stokes equations for air in chemical nonequilibrium
 * (arXiv 2210.05547: Eqs. 1-11 for the equations, Sec. 2.2 for the closure, Sec. 3.1-3.3 for
 * the discretisation, Eq. 26 for the sponge).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Return value: HYP_OK (0) on success, a negative HYP_ERR_* code otherwise; the message of the
 *   last error on the calling thread is available from hyp_last_error().
 * - Device pointers are CUDA global-memory pointers of the current device; host pointers are
 *   ordinary process memory. Each argument says which it is.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Calls that take
 *   a stream are asynchronous with respect to the host: they enqueue kernels and return. Device
 *   status flags (Newton failure, clamped temperature, non-physical state) are read with
 *   hyp_grid_status(), which synchronises the grid's stream.
 * - Ownership: the caller owns every field buffer it passes (state, right-hand side, the
 *   thermo_eval inputs and outputs). The library owns the opaque handles and everything inside
 *   them (gas tables, metrics, sponge, reference state, scratch), and frees them in *_free.
 * - Floating point: FP64 throughout with precision HYP_FP64; HYP_MIXED moves the parts listed at
 *   enum hyp_precision to binary32. No call falls back to the CPU: every arithmetic step of
 *   rhs / rk_stage / thermo_eval runs in CUDA kernels.
 * - A grid handle carries scratch memory: calls that use the same grid (rhs, rk_stage) must not
 *   overlap on the device; serialise them on one stream.
 *
 * State vector layout (2D, ns species, the first species of the table omitted, Sec. 2.1):
 *   centres  (ny rows x nx columns, x fastest): rho, rho_s for s = 1..ns-1, rho*E
 *   x-faces  (ny rows x (nx+1) columns):       rho*u
 *   y-faces  ((ny+1) rows x nx columns):       rho*v
 * concatenated in that order, FP64, nondimensional per Eq. (7). Three-dimensional grids stack nz
 * such planes per field (z slowest) and append rho*w on the z-faces (nz x ny x nx; face k lies
 * between centres k-1 and k of the periodic direction). Total length from hyp_state_size(). The
 * right-hand side has the same layout.
 */
#ifndef HYP_H
#define HYP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Capacity of the species arrays of the ABI structs. The library is built for one species
 * count: libhyp.so for five-species air (N2, O2, NO, N, O; data/air5.dat), libhyp11.so for
 * eleven-species air with ions and electrons (data/air11.dat); a gas table must list exactly the
 * count of the library that loads it. */
#define HYP_MAX_SPECIES 11

enum hyp_gas_kind {
    HYP_GAS_CNEQ = 0,    /* finite-rate chemistry with algebraic diffusion (Sec. 2.2.1) */
    HYP_GAS_FROZEN = 1,  /* frozen composition: no reactions, no diffusion (Sec. 2.2.1) */
    HYP_GAS_CPG = 2,     /* calorically perfect gas, Sutherland viscosity (Eqs. 22, 24) */
    HYP_GAS_TPG = 3,     /* thermally perfect gas: c_p(T) of Eq. 23, Sutherland viscosity,
                            Keyes conductivity (Eqs. 22-25) */
    HYP_GAS_LTE = 4      /* local thermodynamic equilibrium (Sec. 2.2.2, special cases): the
                            composition of minimum Gibbs energy for the element content of the
                            freestream Y_inf, found per point from (rho, e); no species equations
                            (the species fields are carried as passive scalars, unread), heat
                            flux -k_eq grad T with the equilibrium conductivity (see
                            hyp_lte_eval) */
};

/* HYP_FP64: every step in binary64. HYP_MIXED: in binary32 the transport and diffusion
 * coefficients (Blottner, Eucken, Wilke, Chapman-Enskog; Sec. 2.2.1, Eq. 19), the forward-rate
 * exponentials (Eq. 13), the species heat capacities and the weakly populated electronic levels
 * (theta / T >= 9) of the species thermodynamics (Sec. 2.2.1; in the right-hand side, whose
 * neighbouring cells share a choice per level, not in hyp_thermo_eval), the Gaussian filter of
 * the artificial diffusivities (Sec. 3.3), and the interior rows of the compact
 * interpolations and derivatives that feed only the diffusive fluxes (Sec. 3.1); in double-word
 * binary32 (each value a pair of binary32 words) the interior rows of the other compact operators;
 * in binary64 the Newton iteration for the temperature, the vibrational factors and populated
 * electronic levels that set the species energies, equilibrium constants and backward rates,
 * every closure row of the operators, every divergence, the fluxes themselves and the stage
 * update. */
enum hyp_precision { HYP_FP64 = 0, HYP_MIXED = 1 };

enum hyp_error {
    HYP_OK = 0,
    HYP_ERR_ARG = -1,       /* invalid argument (null handle, bad size, unknown kind) */
    HYP_ERR_CUDA = -2,      /* a CUDA runtime call failed (message has the CUDA error) */
    HYP_ERR_IO = -3,        /* gas table could not be read or parsed */
    HYP_ERR_OOM = -4,       /* device allocation failed */
    HYP_ERR_STATUS = -5     /* device status flags set (see hyp_grid_status) */
};

/* Per-point status bits (thermo_eval status mask, hyp_grid_status flags). */
#define HYP_STATUS_NOT_CONVERGED 1u  /* Newton inversion for T did not converge */
#define HYP_STATUS_T_CLAMPED 2u      /* internal energy outside [e(50 K), e(1e5 K)]: T clamped */
#define HYP_STATUS_NONPHYSICAL 4u    /* rho <= 0 */

typedef struct hyp_gas hyp_gas;
typedef struct hyp_grid hyp_grid;
typedef struct hyp_state hyp_state;

/* Freestream that defines the nondimensionalisation of Eq. (7) and the numbers of Eq. (11).
 * reynolds is Re_inf = rho_inf a_inf L_ref / mu_inf (Eq. 11), which fixes L_ref. */
typedef struct {
    double T_inf;                      /* K */
    double p_inf;                      /* Pa */
    double Y_inf[HYP_MAX_SPECIES];     /* mass fractions, table order */
    double mach;                       /* U_inf / a_inf */
    double reynolds;                   /* Re_inf of Eq. (11) */
    double prandtl_cpg;                /* Prandtl number, used by HYP_GAS_CPG only */
} hyp_freestream;

/* Structured grid: nx x ny cells; x uniform on [x0, x1]; y on [y0, y1] with
 * y_stretch 0 = uniform, 1 = tanh wall clustering y = y0 + (y1-y0)(1 - tanh(q(1-s))/tanh q),
 * 2 = the cubic map of Eq. (27) with kappa_y = q; s = j/ny at grid (tau) nodes.
 * nz > 1: a three-dimensional grid with nz uniform, periodic cells on [z0, z1) (nz <= 1: the
 * two-dimensional grid). Three-dimensional grids take the cneq, frozen or cpg gas, the algebraic
 * diffusion and no state filter, and run hyp_rhs / hyp_rk_stage (the two-register RK3) only; the
 * state adds rho w on the z-faces (see the state layout above) and the case may carry a jet. */
typedef struct {
    int32_t nx, ny;
    double x0, x1, y0, y1;
    int32_t y_stretch;
    double y_param;
    int32_t nz;
    double z0, z1;
} hyp_grid_desc;

/* Case: boundary conditions (Sec. 3.2, Fig. 2), sponge (Eq. 26), shock capturing (Sec. 3.3),
 * and the synthetic initial / reference state. */
typedef struct {
    int32_t flow;                  /* 0 flat-plate boundary layer, 1 oblique shock impinging on it */
    int32_t wall;                  /* 1: isothermal no-slip non-catalytic wall at y0; 0: far field */
    double T_wall;                 /* K */
    double delta_coef;             /* boundary-layer thickness delta(x) = delta_coef sqrt(x/(Re Ma)) */
    double minor_species;          /* NO/N/O seeded inside the layer, peak mass fraction scale */
    double shock_deflection_deg;   /* flow deflection of the incident shock (flow = 1) */
    double shock_x;                /* x where the inviscid shock line meets the wall */
    double shock_width;            /* tanh smoothing width of the shock in the initial state */
    double sponge_sigma;           /* sigma_max of the cubic sponge ramps */
    double sponge_in, sponge_out;  /* x-lengths of the inflow / outflow sponges (0 = none) */
    int32_t sponge_top_cells;      /* number of cells in the top sponge */
    int32_t artificial_diffusivity;
    double C_mu, C_beta, C_kappa, C_D;
    double noise_amp;              /* initial state = reference * (1 + noise_amp * noise) */
    const double* noise;           /* HOST, nullable; hyp_state_size() values in [-1, 1] */
    double filter_sigma;           /* > 0: low-pass filter of the state after each RK step, with
                                      this damping of the grid-to-grid mode (see hyp_rk_stage) */
    int32_t diffusion_model;       /* HYP_GAS_CNEQ: 0 the algebraic model of Eq. 18, 1 the
                                      Stefan-Maxwell system of Eq. 17 solved at every face */
    /* Three-dimensional grids: a sonic jet through a circular orifice in the wall (the jet in
     * hypersonic crossflow of Sec. 4). Inside the orifice the wall face holds the Dirichlet mass
     * flux of a sonic jet at T_j = jet_T_ratio T_inf and p_j = jet_J Ma^2 p_inf (so that jet_J is
     * the momentum ratio rho_j v_j^2 / (rho_inf U_inf^2)), blended to the wall by
     * 1/2 (1 - tanh((r - jet_radius) / (jet_edge jet_radius))), r the distance to (jet_x, jet_z)
     * on the periodic domain; the wall temperature of the heat flux blends to T_j the same way. */
    int32_t jet;
    double jet_x, jet_z, jet_radius, jet_edge, jet_J, jet_T_ratio;
} hyp_case;

/* Load a gas table (plain-text SPECIES / LEVEL / REACTION lines, see data/air5.dat) and build
 * the closure of Sec. 2.2 for `kind`, nondimensionalised with `fs` (Eq. 7). The table must list
 * the library's species count (5 or 11, see HYP_MAX_SPECIES); its first species is the omitted
 * one (Sec. 2.1). Charged species (an optional last SPECIES column, the charge) need the
 * eleven-species build: ions diffuse ambipolarly (twice their Eq. 19 coefficient), the electron
 * stays out of the mixing rules and binary pairs and its diffusive flux follows from zero
 * conduction current, J_e = M_e sum_ions J_i / M_i, with the omitted species taking
 * J_0 = -sum_{s>=1} J_s. HYP_GAS_LTE rejects charged species (it conserves N and O only).
 * path: HOST string. fs: HOST. *out: new handle, free with hyp_gas_free. */
int hyp_gas_model_load(const char* path, int kind, const hyp_freestream* fs, hyp_gas** out);

/* Reference scales (HOST array of 13 doubles): rho_inf, a_inf, T_inf, p_inf, mu_inf, k_inf,
 * cp_inf, gamma_inf, R_inf, T_ref, L_ref, Re_inf, Pr_inf (Eqs. 7, 11). n_species may be NULL. */
int hyp_gas_scales(const hyp_gas* gas, int* n_species, double* scales13);

void hyp_gas_free(hyp_gas* gas);

/* Number of doubles in the state vector for this gas and grid. */
int hyp_state_size(const hyp_gas* gas, const hyp_grid_desc* desc, int64_t* n);

/* Build the grid (metrics), sponge strength, reference state Q_ref of Eq. (26) and scratch, and
 * write the initial state into U. U, dQ: DEVICE, caller-owned, hyp_state_size() doubles each;
 * the state handle keeps both pointers as the two Runge-Kutta registers (dQ is zeroed).
 * desc, cas (and cas->noise): HOST. Enqueued on `stream`; the handle's grid uses that stream
 * for its status flag. */
int hyp_state_init(const hyp_gas* gas, const hyp_grid_desc* desc, const hyp_case* cas,
                   double* U, double* dQ, void* stream, hyp_state** out);

/* The grid of a state (valid while the state lives). */
const hyp_grid* hyp_state_grid(const hyp_state* st);

/* Copy grid data to HOST buffers of hyp_state_size() doubles (either may be NULL):
 * U_ref = reference state of Eq. (26); sigma = sponge strength at the node of each entry. */
int hyp_grid_reference(const hyp_grid* grid, double* U_ref_host, double* sigma_host);

/* Read and optionally clear the OR of the per-point status bits raised since the last clear.
 * Synchronises the grid's stream. */
int hyp_grid_status(const hyp_grid* grid, uint32_t* flags, int clear);

/* Temperature (K) at every cell centre from the grid's last hyp_rhs or hyp_rk_stage: the T the
 * closure inverted from the internal energy (Sec. 2.2). hyp_rhs_noalloc keeps its closure in its
 * own scratch and does not change it. T: DEVICE, caller-owned, n_T doubles, n_T = nx*ny
 * (nx*ny*nz for a three-dimensional grid), x fastest. Enqueued on `stream` (order it after the
 * evaluation it reads). HYP_ERR_ARG if n_T is not the cell count or no closure has run on the
 * grid yet. */
int hyp_grid_temperature(const hyp_grid* grid, int64_t n_T, double* T, void* stream);

void hyp_state_free(hyp_state* st);

/* dU/dt = -div F_C + div F_D + S - sigma (U - U_ref)  (Eqs. 5, 6, 26) on the staggered grid,
 * with the closure of Sec. 2.2 at every cell centre, sixth-order compact staggered operators
 * (Sec. 3.1), the boundary conditions of Sec. 3.2 and, if the case enables it, artificial
 * diffusivity (Sec. 3.3). Entries on Dirichlet boundary faces (x-faces at x0 and x1, y-faces at
 * y0 and y1) are set to 0. U, dUdt: DEVICE, caller-owned, hyp_state_size() doubles, must not
 * alias. Uses the grid's scratch. */
int hyp_rhs(const hyp_gas* gas, const hyp_grid* grid, const double* U, double* dUdt,
            int precision, void* stream);

/* One stage (0, 1, 2) of the low-storage two-register third-order Runge-Kutta scheme (Sec. 3.1):
 * dQ <- A_k dQ + dt R(U); U <- U + B_k dQ with A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15),
 * on the registers given to hyp_state_init. dt nondimensional (time unit L_ref / a_inf).
 * If the case sets filter_sigma > 0, stage 2 ends with the low-pass filter of the high-order
 * shock-capturing practice the paper cites (Sec. 3.3): along every grid line of every field,
 * f_i <- f_i - sigma 4^-m sum_{n=-m..m} (-1)^n C(2m, m+n) f_{i+n}, m = 5, or m = d at distance
 * d < 5 from an end of the line (end points unchanged); x lines first, then y lines. */
int hyp_rk_stage(hyp_state* st, int stage, double dt, int precision, void* stream);

/* Time integrators of Sec. 3.1. HYP_RK3_2N: the scheme of hyp_rk_stage. HYP_RK3_TVD: the TVD RK3
 * of Shu and Osher, U1 = U0 + dt R(U0), U2 = 3/4 U0 + 1/4 (U1 + dt R(U1)),
 * U^{n+1} = 1/3 U0 + 2/3 (U2 + dt R(U2)), with the step's start state U0 kept in the second
 * register (dQ). HYP_RK4_2N: the five-stage fourth-order 2N-storage scheme of Carpenter and
 * Kennedy (dQ <- A_k dQ + dt R; U <- U + B_k dQ with their published coefficients). */
enum hyp_rk_scheme { HYP_RK3_2N = 0, HYP_RK3_TVD = 1, HYP_RK4_2N = 2 };

/* One stage (0..2, or 0..4 for HYP_RK4_2N) of `scheme` on the state's two registers; the case's
 * state filter runs after the scheme's last stage. Otherwise as hyp_rk_stage. */
int hyp_rk_stage_scheme(hyp_state* st, int scheme, int stage, double dt, int precision,
                        void* stream);

/* Wall heat flux and wall shear stress of state U (nondimensional, Eq. 7): evaluates the
 * right-hand side on U with the grid's scratch (the result is discarded) and writes
 * q_w[i] = -K dT/dy at the nx wall faces (Eq. 10, K including the artificial conductivity) and
 * tau_w[i] = tau_xy at the nx + 1 wall corners (Eq. 9). U: DEVICE, hyp_state_size() doubles;
 * q_w[nx], tau_w[nx+1]: DEVICE, caller-owned. Skin friction C_f = 2 tau_w / Ma_inf^2.
 * HYP_ERR_ARG if the case has no wall. Uses the grid's scratch like hyp_rhs. */
int hyp_wall_fluxes(const hyp_gas* gas, const hyp_grid* grid, const double* U, double* q_w,
                    double* tau_w, int precision, void* stream);

/* ---- Batched execution (serving many independent solves on one GPU) ----
 * A batch advances several states, each with its own grid size, freestream, case and time step,
 * with every step of the hot path in shared launches: one compact-operator launch per phase over
 * the members' joined line jobs, and one persistent kernel per pointwise step whose blocks walk
 * fixed-size tiles of the members. The kernels run the same arithmetic on each member's own
 * scratch and caches as hyp_rk_stage, so a member's states are bit-identical alone and in any
 * batch. Members must come from gases built from the same table and kind. A batch and its
 * members are used from one host thread; a state may be in one batch at a time and must not be
 * stepped by other calls while it is a member. */
typedef struct hyp_batch hyp_batch;

/* New empty batch computing in `precision` (HYP_FP64 or HYP_MIXED). Free with hyp_batch_free. */
int hyp_batch_create(int precision, hyp_batch** out);

/* Add (remove) a member. dt: the member's nondimensional time step. The state stays owned by the
 * caller; removing it leaves its registers at the last completed step. */
int hyp_batch_add(hyp_batch* b, hyp_state* st, double dt);
int hyp_batch_remove(hyp_batch* b, hyp_state* st);

/* use_graph != 0: capture one step into a CUDA graph and replay it while the membership stays
 * the same. tile: points per persistent-kernel tile, a positive multiple of 128, or 0 (the
 * default) for the autotuner: after a change of membership to a size class (power of two of the
 * total cell count) not seen before, the next steps run one untimed step and then one timed step
 * for each tile size in {256, 512, 1024, 2048}, and the fastest is kept for that class. Those are
 * real steps of every member; the tile size does not change any result. */
int hyp_batch_configure(hyp_batch* b, int use_graph, int tile);

/* Number of members (HOST int). */
int hyp_batch_size(const hyp_batch* b, int* members);

/* Current tile size and whether the autotuner has settled for this membership (HOST ints,
 * each nullable). */
int hyp_batch_tile(const hyp_batch* b, int* tile, int* tuned);

/* nsteps full RK3 steps (three stages and, for members whose case sets it, the state filter)
 * of every member, enqueued on `stream`. */
int hyp_batch_step(hyp_batch* b, int nsteps, void* stream);

void hyp_batch_free(hyp_batch* b);

/* ---- Serving: continuous batching of independent solves ----
 * A server owns one worker thread, one stream and one batch (hyp_batch_*). Requests (a grid, a
 * case, a freestream, a time step and a step count) are submitted from any host thread and queued
 * in arrival order. Between batch steps the worker admits queued requests while the GPU's free
 * memory stays above the reserve after the request's estimated footprint and the member limit
 * is not reached (it builds the gas, the state and the registers on the device), advances the
 * batch by as many steps as the nearest completion allows (at most 8), and retires finished
 * members (status read, registers optionally copied to host memory, device memory freed).
 * Requests that arrive while others run join at the next step boundary. Times are seconds since
 * the server was created, from the host's steady clock. */
typedef struct hyp_server hyp_server;

typedef struct {
    hyp_freestream fs;
    hyp_grid_desc grid;
    hyp_case cas;                  /* cas.noise, if set, is copied at submission */
    double dt;                     /* nondimensional time step */
    int32_t nsteps;                /* RK3 steps to run */
    int32_t keep_result;           /* 1: keep the final state for hyp_server_result */
} hyp_request;

typedef struct {
    double t_submit, t_admit, t_finish;   /* -1 while not reached */
    int32_t done;                         /* 1 when finished */
    uint32_t status;                      /* HYP_STATUS_* bits raised during the solve */
    int32_t error;                        /* HYP_OK, or the error that ended the request */
    int64_t points;                       /* cells of the grid */
    int64_t bytes;                        /* device bytes reserved for it at admission */
} hyp_request_stats;

/* New server. table: gas table path (HOST string) shared by all requests; kind: hyp_gas_kind;
 * precision: HYP_FP64 or HYP_MIXED; reserve_bytes: free device memory kept back at admission;
 * max_members: upper bound on concurrently admitted requests (> 0). */
int hyp_server_create(const char* table, int kind, int precision, int64_t reserve_bytes,
                      int max_members, hyp_server** out);

/* Queue a request (HOST struct, copied). *id: its identifier (0, 1, 2, ... in submission order).
 * Returns immediately. HYP_ERR_ARG for an invalid request (checked here: sizes, dt, nsteps). */
int hyp_server_submit(hyp_server* sv, const hyp_request* req, int64_t* id);

/* Block until request id (or, with id < 0, every request submitted so far) has finished, or
 * timeout_s seconds passed (HYP_ERR_ARG then). */
int hyp_server_wait(hyp_server* sv, int64_t id, double timeout_s);

/* Statistics of one request (HOST struct). */
int hyp_server_stats(hyp_server* sv, int64_t id, hyp_request_stats* out);

/* Final state of a finished request submitted with keep_result (HOST buffer of
 * hyp_state_size() doubles); the server drops its copy afterwards. */
int hyp_server_result(hyp_server* sv, int64_t id, double* U_host);

/* Server-wide counters (HOST, each nullable): steps run by the batch, sum over steps of the
 * member count, device seconds of the steps, largest member count. */
int hyp_server_counters(hyp_server* sv, int64_t* batch_steps, int64_t* member_steps,
                        double* busy_s, int32_t* max_members);

/* Stop the worker after the requests in flight finish and queued ones are dropped, and free. */
void hyp_server_free(hyp_server* sv);

/* The binary64 -> binary32 rounding (nearest, ties to even; magnitudes below 1.18e-38 to signed
 * zero) and the exact widening back that HYP_MIXED uses between its binary64 and binary32
 * parts, done with integer instructions. x[n]: DEVICE input; y[n] (binary32) and back[n]
 * (binary64): DEVICE outputs, each nullable. */
int hyp_round_f32(int64_t n, const double* x, float* y, double* back, void* stream);

/* The binary64 exponential, quotient, reciprocal and logarithm the FP64 closure uses
 * (diagnostics; no counterpart in the paper): exp and log by Tang's table-driven methods, a / b
 * and 1 / b from a binary32 reciprocal refined in binary64, each within 2 ulp; arguments outside
 * their fast ranges (|a| >= 512 for exp, |b| outside [2^-120, 2^120] for the quotients, a outside
 * [2, 2^1000) for log) go through CUDA's exp, division and log. fn 0: out[i] = exp(a[i]); fn 1:
 * out[i] = a[i] / b[i]; fn 2: out[i] = 1 / b[i]; fn 3: out[i] = log(a[i]). a, b (the one a
 * function does not read may be null), out: DEVICE arrays of n doubles. */
int hyp_fp64_fast(int fn, int64_t n, const double* a, const double* b, double* out, void* stream);

/* Pointwise closure of Sec. 2.2 in SI units for n independent states (the work the paper hands
 * to its real-gas library, Sec. 3.4). Inputs (DEVICE): rho[n] kg/m^3, e[n] J/kg internal energy
 * including formation enthalpy (298.15 K reference), Y[ns*n] mass fractions species-major
 * (Y[s*n + i]). Outputs (DEVICE, each nullable): T[n] K, p[n] Pa, wdot[ns*n] kg/(m^3 s) (Eq. 15),
 * mu[n] Pa s, k[n] W/(m K) (frozen), D[ns*n] m^2/s (Eq. 19), status[n] HYP_STATUS_* bits.
 * HYP_ERR_ARG for an HYP_GAS_LTE gas, whose composition is not an input (hyp_lte_eval). */
int hyp_thermo_eval(const hyp_gas* gas, int64_t n, const double* rho, const double* e,
                    const double* Y, double* T, double* p, double* wdot, double* mu, double* k,
                    double* D, uint8_t* status, int precision, void* stream);

/* Mixture internal energy e = sum_s Y_s e_s(T) (Eq. 12), J/kg. T[n], Y[ns*n], e[n]: DEVICE. */
int hyp_thermo_energy(const hyp_gas* gas, int64_t n, const double* T, const double* Y, double* e,
                      void* stream);

/* Closure of a mixture in local thermodynamic equilibrium at n states (HYP_GAS_LTE gas only;
 * Sec. 2.2.2): the temperature from the equilibrium energy at fixed density (safeguarded Newton
 * iteration, relative step 1e-8, from a tabulated start), the composition of minimum Gibbs energy
 * at (T, rho) for the element content of the gas's Y_inf (element potentials by Newton's method),
 * p = rho R_mix T, the Wilke viscosity and frozen conductivity of that composition, and the
 * equilibrium conductivity k_eq = k_frozen + k_reactive, where k_reactive is the heat the
 * algebraic diffusion of Eq. (18) carries when the mole fractions follow the equilibrium at the
 * local pressure: k_reactive = (rho / M_mix) sum_s M_s D_s (dX_s/dT)_p (h_s - h).
 * rho[n] (kg/m^3), e[n] (J/kg): DEVICE inputs. Outputs, DEVICE, each nullable: T[n] (K), p[n]
 * (Pa), Y[ns*n] (mass fractions, species-major), mu[n] (Pa s), k[n] (k_eq, W/(m K)),
 * k_reactive[n], status[n] (HYP_STATUS_* bits). precision: HYP_MIXED takes the transport in
 * binary32 as hyp_thermo_eval does. HYP_ERR_ARG if the gas is not HYP_GAS_LTE. */
int hyp_lte_eval(const hyp_gas* gas, int64_t n, const double* rho, const double* e, double* T,
                 double* p, double* Y, double* mu, double* k, double* k_reactive,
                 uint8_t* status, int precision, void* stream);

/* hyp_rhs without any device allocation of its own scratch (the paper has no counterpart). It is
 * for callers that may not allocate device memory while they run: real-time solver loops that
 * forbid allocation after start-up, and hosts (simulation frameworks, language runtimes, plug-in
 * hosts) that own all device memory through their own allocator and do not let a library call
 * cudaMalloc behind their back. It computes the same right-hand side as hyp_rhs for the same gas,
 * grid and U, within rounding (the Newton inversion starts from 1000 K instead of the grid's
 * previous temperatures). Arguments as for hyp_rhs, always FP64; two-dimensional grids only.
 * - Scratch: every per-call scratch field, the line-sweep storage and the launch plan live in one
 *   file-scope device array of 12 MiB (1,572,864 doubles) that every GPU loading the library holds
 *   until exit. Grids needing more (a few thousand cells, e.g. up to 64 x 64) are rejected with
 *   HYP_ERR_ARG and the required size in hyp_last_error(). The grid's own scratch and predictor
 *   cache are not touched, so hyp_rhs and hyp_rhs_noalloc may be mixed on one grid; its read-only
 *   data (metrics, reference state, sponge, operators) are used. Per-point status bits (Newton,
 *   energy range, rho <= 0) are OR-ed into the grid's status word, read with hyp_grid_status.
 * - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *   that device current.
 * - Each call only enqueues work on `stream` (the launch plan is copied and relocated by a kernel):
 *   no host synchronisation, and no cudaMalloc, cudaFree or other allocating routine.
 * - All calls on a device share the array: it keeps the last call's contents (the parts that must
 *   start at zero are cleared on every call), and calls that overlap on the GPU race. */
int hyp_rhs_noalloc(const hyp_gas* gas, const hyp_grid* grid, const double* U, double* dUdt,
                    void* stream);

/* Event profile of the launches that hyp_rhs / hyp_rk_stage make on a grid (diagnostics; no
 * counterpart in the paper). hyp_grid_profile(grid, 1) clears the totals and starts recording a
 * pair of CUDA events around every launch (on a three-dimensional grid: around the closure's
 * launches only) on the caller's stream; (grid, 0) stops. Reading
 * synchronises on the recorded events and returns, for the first n kernel ids, the summed
 * device time in ms and the launch count (HOST arrays, nullable). Kernel ids run from 0 to
 * hyp_profile_count() - 1; hyp_profile_name(id) is a static string. */
int hyp_grid_profile(const hyp_grid* grid, int enable);
int hyp_grid_profile_read(const hyp_grid* grid, int n, double* ms, int64_t* launches);
int hyp_profile_count(void);
const char* hyp_profile_name(int id);

/* Message of the last failed call on this thread ("" if none). Owned by the library. */
const char* hyp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HYP_H */
