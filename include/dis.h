/*
 * dis.h - C ABI of the GB300 diffuse-interface finite-volume step.
 *
 * One explicit time step of the unified diffuse-interface system for
 * multiphase reactive fluids and elastoplastic solids on regular Cartesian
 * patches (Wallis, Barton & Nikiforakis, arXiv 2009.14555, Section 3):
 * CFL time step, SSP-RK3 (or single-stage MUSCL-Hancock) hyperbolic update
 * with MUSCL(-BVD-THINC) reconstruction of primitives and an HLLD-type
 * elastic Riemann solver (Section 3.1), in planar or cylindrical geometry,
 * then the plastic (Section 3.2) and reactive (Section 3.3) source steps.
 *
 * Conventions shared by every call:
 *   - All functions return an int status (DIS_OK = 0, negative on error).
 *     Nothing aborts or throws across this interface; the text of the last
 *     error of the calling thread is returned by dis_last_error().
 *   - A context is bound to the CUDA device that was current at dis_create
 *     and to one CUDA stream; all device work is ordered on that stream.
 *     Calls on one context are not thread-safe.
 *   - Device pointers must be device memory of that device; host pointers
 *     may be pageable.  The library never keeps a caller pointer after a call
 *     returns, except workspace bound by dis_bind_workspace.
 *   - State arrays ("packed" layout): for each patch in creation order, an
 *     array [nfields][ny][nx] of float64 (x fastest), patches concatenated.
 *     Field order (two materials, material 1 carries the stored volume
 *     fraction; the last field exists only with a reactive material):
 *       conservative 1D: phi1, phi1 rho1, phi2 rho2, rho u, rho E, V11, V22, V33, [phi_y rho_y lam]
 *       conservative 2D: phi1, phi1 rho1, phi2 rho2, rho u, rho v, rho E,
 *                        V11, V12, V21, V22, V33, [phi_y rho_y lam]
 *       primitive    1D: phi1, rho1, rho2, u, p, V11, V22, V33, [lam]
 *       primitive    2D: phi1, rho1, rho2, u, v, p, V11, V12, V21, V22, V33, [lam]
 *     (state vector q of Section 3; V is the elastic stretch tensor in plane
 *     strain; lam is the reaction progress variable, 1 = reactant.)
 */
#ifndef DIS_H
#define DIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DIS_OK = 0,
  DIS_EINVAL = -1,       /* bad argument; nothing was changed */
  DIS_ENOMEM = -2,       /* workspace missing or too small, or allocation failed */
  DIS_ECUDA = -3,        /* a CUDA runtime call failed (text in dis_last_error) */
  DIS_ENONPHYSICAL = -4, /* a step met a state without a real sound speed or positive density, or
                            produced a non-finite value or phi outside [-1e-6, 1+1e-6] */
  DIS_ESTATE = -5        /* call out of order (e.g. step before set_state) */
};

/* DIS_BC_EXTERNAL: the ghost layers of that side are read as stored in the
 * state (filled by the AMR hierarchy's ghost-cell kernel); not accepted by
 * dis_create. */
enum { DIS_BC_TRANSMISSIVE = 0, DIS_BC_PERIODIC = 1, DIS_BC_REFLECTIVE = 2, DIS_BC_EXTERNAL = 3 };
enum { DIS_CONSERVATIVE = 0, DIS_PRIMITIVE = 1 };
enum { DIS_FP64 = 0, DIS_FP32_BULK = 1 };
enum { DIS_PLASTIC_NONE = 0, DIS_PLASTIC_PERFECT = 1, DIS_PLASTIC_RATE = 2, DIS_PLASTIC_JC = 3 };

enum { DIS_RATE_ARRHENIUS = 0, DIS_RATE_SQRT = 1 };

/* Equation-of-state family of a material (Section 2.3), all Mie-Grueneisen
 * with a constant Gruneisen coefficient Gamma = gamma - 1:
 *   DIS_EOS_STIFFENED  reference pressure -gamma p_inf, energy e_inf, shear
 *                      modulus G (the default: zero-filled);
 *   DIS_EOS_ROMENSKII  elastic solid: reference energy
 *                      K0 / (2 rho0 a^2) ((rho/rho0)^a - 1)^2 and its pressure
 *                      rho^2 dE/drho, shear modulus G (rho/rho0)^(b + 1)
 *                      (a, b = alpha, beta; G is G0; p_inf, e_inf unused);
 *   DIS_EOS_JWL        reference pressure A e^(-R1 rho0/rho) + B e^(-R2 rho0/rho),
 *                      energy A / (R1 rho0) e^(-R1 rho0/rho) + B / (R2 rho0)
 *                      e^(-R2 rho0/rho) (a fluid: G must be 0).
 * The shear energy G(rho) J^2 / rho enters the reference curves.  The
 * reactive material must be a stiffened gas without shear modulus (ideal,
 * p_inf = 0, unless it has a product closure of its own). */
enum { DIS_EOS_STIFFENED = 0, DIS_EOS_ROMENSKII = 1, DIS_EOS_JWL = 2 };

/* One material: Mie-Grueneisen closure (Section 2.3; stiffened gas by
 * default, see above) with shear modulus G, plasticity (Section 2.3.2: none, perfect = the
 * chi0 -> infinity limit of ideal plasticity, ideal plasticity with rate
 * chi0, or Johnson-Cook, below), and for a reactive material an ideal-gas reactant/product pair of
 * equal gamma and C_V with heat release Q (Section 2.3.1) and a rate law for
 * the reactant fraction lam (1 = reactant):
 *   DIS_RATE_ARRHENIUS  lam_dot = -A lam exp(-T_act / T)   (zero where T <= 0);
 *   DIS_RATE_SQRT       lam_dot = -A sqrt(lam) where p > p_ign, else 0 (the
 *                       k sqrt(lam) law with a pressure switch of the paper's
 *                       one-dimensional detonation test, Section 4.1; A = k;
 *                       sqrt of max(lam, 0), and the reaction step's result
 *                       is clamped at lam >= 0).
 * rate_law and p_ign are read only for the reactive material; zero-filled
 * (the default of a C initialiser without them) selects Arrhenius. */
typedef struct {
  double gamma, p_inf, e_inf, G;
  int32_t plastic;
  double sigma_y, chi0;
  int32_t reactive;
  double Q, cv, A, T_act;
  int32_t rate_law; /* DIS_RATE_ARRHENIUS or DIS_RATE_SQRT */
  double p_ign;     /* DIS_RATE_SQRT: pressure above which the reaction runs, Pa */
  int32_t eos;      /* DIS_EOS_STIFFENED, DIS_EOS_ROMENSKII or DIS_EOS_JWL */
  double rho0;      /* Romenskii, JWL: reference density */
  double K0, alpha, beta;                 /* Romenskii: bulk modulus, exponents */
  double jwl_A, jwl_B, jwl_R1, jwl_R2;    /* JWL constants */
  /* Reactive material only: a product closure of its own (stiffened gas
   * prod_gamma, prod_p_inf, prod_cv; prod_gamma 0 = the reactant's closure).
   * The reactant is then the material's gamma, p_inf, cv, and the mixture's
   * component densities follow from the temperature equality of Appendix B
   * (a bisection over the reactant's volume share).  Float64 contexts only. */
  double prod_gamma, prod_p_inf, prod_cv;
  /* DIS_PLASTIC_JC (Section 2.3.2), a Romenskii solid with cv > 0: the
   * plastic strain rate chi0 exp((sqrt(3/2) |dev sigma| / sigma_Y - 1) / c3)
   * with sigma_Y = (sigma_y + jc_c2 eps_p^jc_n)(1 - T*^jc_m),
   * T* = (T - jc_T0) / (jc_Tmelt - jc_T0) clamped to [0, 1], and the
   * temperature T = jc_T0 (rho/rho0)^Gamma + (p - p_ref) / (rho Gamma cv) of
   * the Debye form of the thermal energy (Section 2.2), taken at the state
   * entering the plastic step.  The relaxation objective of Section 3.2,
   * J - J* + dt chi(J, eps_p + J* - J), is solved by bisection on [0, J*]
   * (64 halvings) and the material's eps_p grows by J* - J.  The material
   * carries the context's history row (see dis_create).  Float64 contexts,
   * not the adjoint. */
  double jc_c2, jc_c3, jc_n, jc_m, jc_Tmelt, jc_T0;
} dis_material;

/* One Cartesian patch (the single-grid unit of Section 3): nx x ny cells of
 * size dx x dy (ny = 1 and dy ignored in 1D); bc = {x-low, x-high, y-low,
 * y-high} boundary kinds. */
typedef struct {
  int32_t nx, ny;
  double dx, dy;
  int32_t bc[4];
  double x0; /* x of the patch's low face: the radius of its axis-side face in
                cylindrical geometry (0 when the patch touches the axis);
                unused in planar geometry */
} dis_patch;

/* Hyperbolic update of a step: DIS_RK3 is the paper's three-stage
 * Runge-Kutta scheme (Section 3.1, three Riemann solves per face and step);
 * DIS_HANCOCK the single-stage MUSCL-Hancock predictor-corrector (one Riemann
 * solve per face and step, second order; no counterpart in the paper): the
 * per-cell edge states of the same reconstruction move by half a step of the
 * cell's own operator before the face Riemann problems.  Planar geometry.
 * In FP32-bulk contexts one fused kernel per step reads the state and writes
 * a second buffer; the two exchange roles from step to step (the workspace
 * holds two state buffers, the Runge-Kutta form three). */
enum { DIS_RK3 = 0, DIS_HANCOCK = 1 };

/* Geometry: DIS_PLANAR is the Cartesian plane-strain system; DIS_CYLINDRICAL
 * the axisymmetric one of Section 3 (x = r, y = z, theta the third axis): the
 * operator subtracts the geometric source s_g = -(1/r) (0, phi_l rho_l u_r,
 * phi_y rho_y lam u_r, rho u_r^2 - sigma_rr + sigma_thth, rho u_z u_r -
 * sigma_rz, rho E u_r - (u_r sigma_rr + u_z sigma_zr), V_ij u_r / 3 -
 * delta_{i theta} V_ij u_r) at each cell centre r = x0 + (i + 1/2) dx.  A
 * patch on the axis has x0 = 0 and a reflective x-low boundary.
 * Runge-Kutta contexts only (float64 and FP32-bulk). */
enum { DIS_PLANAR = 0, DIS_CYLINDRICAL = 1 };

/* Slope limiter of the MUSCL reconstruction of the primitives (Section 3.1
 * names none): DIS_MINMOD (default), DIS_VANLEER (2 a b / (a + b) of the two
 * one-sided differences a, b when a b > 0, else 0).  The same limiter forms
 * the MUSCL candidate of the MUSCL-BVD-THINC reconstruction of phi1. */
enum { DIS_MINMOD = 0, DIS_VANLEER = 1 };

/* Step options: CFL number (Section 3: fraction of the largest stable step),
 * THINC interface steepening on/off (Appendix A), precision mode, hyperbolic
 * scheme (DIS_RK3 or DIS_HANCOCK; 0 = the paper's), geometry (DIS_PLANAR or
 * DIS_CYLINDRICAL), slope limiter (DIS_MINMOD or DIS_VANLEER; zero-filled =
 * minmod). */
typedef struct {
  double cfl;
  int32_t thinc;
  int32_t precision;
  int32_t scheme;
  int32_t geometry;
  int32_t limiter;
} dis_options;

typedef struct dis_ctx dis_ctx;

/* Create a context for `n_patches` patches of dimension `dim` (1 or 2) with
 * two materials.  Material `reactive_material` (0, 1, or -1 for none)
 * carries the history row phi_y rho_y alpha_y of Section 2.1 (the last
 * conservative field, advected with the material): alpha = lam if it is the
 * reactive material, alpha = eps_p if it is a Johnson-Cook solid
 * (DIS_PLASTIC_JC); one material carries it, so a context holds either a
 * reactive material or a Johnson-Cook one.  `stream` is a cudaStream_t (NULL
 * = legacy default).  Copies `patches` and `opt`.  Returns DIS_EINVAL for
 * bad sizes. */
int dis_create(int dim, int n_patches, const dis_patch* patches, int reactive_material,
               const dis_options* opt, void* stream, dis_ctx** out);

/* Set the two materials (n must be 2).  Copies `m`.  May be called again
 * between steps (new parameters take effect from the next step).  Returns
 * DIS_EINVAL for bad parameters, for a history-row material that is neither
 * reactive nor Johnson-Cook (or a reactive or Johnson-Cook material that is
 * not the history-row material), and for a Johnson-Cook material in an
 * FP32-bulk context. */
int dis_set_materials(dis_ctx* ctx, const dis_material* m, int n);

/* Bytes of device workspace the context needs (state buffers, primitives,
 * face fluxes, staging).  Depends only on the patches, dim and materials. */
size_t dis_workspace_bytes(const dis_ctx* ctx);

/* Lend the context `bytes` of device memory at `dev` (256-byte aligned); the
 * caller keeps it alive until dis_destroy or another bind.  If no workspace
 * is bound when it is first needed, the library allocates its own. */
int dis_bind_workspace(dis_ctx* ctx, void* dev, size_t bytes);

/* Load the state of all patches from `src` (packed layout above).  kind =
 * DIS_PRIMITIVE converts primitives to conservative variables on the device
 * through the closures of Section 2.  src_on_device selects a device or host
 * pointer.  Ordered on the context's stream. */
int dis_set_state(dis_ctx* ctx, int kind, const double* src, int src_on_device);

/* Store the state of all patches into `dst` (packed layout).  kind =
 * DIS_PRIMITIVE returns the recovered primitives (pressure from the mixture
 * pressure function, Appendix B).  A host destination synchronises the
 * stream. */
int dis_get_state(dis_ctx* ctx, int kind, double* dst, int dst_on_device);

/* The state of one patch only, in that patch's packed layout
 * ([nfields][ny][nx], the slice of the whole-state array): the other patches
 * keep theirs.  A context steps once every patch holds a state (set by
 * dis_set_state, dis_set_state_async or per patch).  Host pointers
 * synchronise the stream; device pointers are ordered on it.  Returns
 * DIS_EINVAL (bad patch index, kind or NULL), DIS_ESTATE (materials missing;
 * get: the patch holds no state), DIS_ENOMEM, DIS_ECUDA. */
int dis_set_patch_state(dis_ctx* ctx, int patch, int kind, const double* src, int src_on_device);
int dis_get_patch_state(dis_ctx* ctx, int patch, int kind, double* dst, int dst_on_device);

/* Advance every patch by n_steps time steps, each with its own CFL time step
 * computed on the device from the state at the start of the step (Section
 * 3).  If dt_out is not NULL it receives the last step's dt per patch (host
 * array of n_patches; synchronises).  The step is device-resident: no host
 * synchronisation inside. */
int dis_step(dis_ctx* ctx, int n_steps, double* dt_out);

/* Same with prescribed time steps dt[patch] (host array) for every step. */
int dis_step_fixed_dt(dis_ctx* ctx, int n_steps, const double* dt);

/* Read and clear the device status word: DIS_OK or DIS_ENONPHYSICAL, with the
 * first offending patch and cell (x index + nx * y index) if not NULL.
 * Synchronises the stream. */
int dis_check(dis_ctx* ctx, int* bad_patch, int* bad_cell);

/* Diagnostics of the current state and of the last step call, reduced on the
 * device.  Totals are sums over every interior cell of every patch of the
 * conserved quantities of Section 3 times the cell volume (dx dy; dx in 1D;
 * times 2 pi r in cylindrical geometry): with periodic or reflective
 * boundaries the mass, momentum and energy totals stay constant up to
 * rounding (the source steps conserve them), which is how the step's
 * conservation is checked. */
typedef struct {
  double mass[2];      /* phi_l rho_l, l = 1, 2 */
  double momentum[2];  /* rho u, rho v (0 in 1D) */
  double energy;       /* rho E */
  double reactant;     /* phi_y rho_y lam (0 without a reactive material) */
  double phi_min, phi_max; /* range of the stored volume fraction phi1 */
  double dt_min, dt_max;   /* time step of the last step over the patches (0 before any step) */
  double kernel_ms;        /* device time of the last dis_step / dis_step_fixed_dt call */
  double bytes;            /* algorithmic state traffic of that call: the state read
                              and written once per step (float64: 8 nfields bytes a
                              cell; FP32-bulk: 4 (nfields + 1)) x cells x steps x 2 */
  long long steps;         /* steps since the state was last set */
  long long launches;      /* kernel launches of the last step call */
  int status;              /* DIS_OK or DIS_ENONPHYSICAL (the device status word; not cleared) */
  int bad_patch, bad_cell; /* the first offending patch and cell (x + nx y), or -1 */
} dis_stats;

/* Fill *s (see dis_stats).  Synchronises the stream.  DIS_EINVAL (NULL),
 * DIS_ESTATE (no state), DIS_ECUDA. */
int dis_query(dis_ctx* ctx, dis_stats* s);

/* Total bytes of the packed state for `kind` (nfields x cells x 8). */
size_t dis_state_bytes(const dis_ctx* ctx, int kind);

/* Number of kernel launches made by the last dis_step / dis_step_fixed_dt. */
long long dis_last_launches(const dis_ctx* ctx);

/* FP32-bulk contexts run one kernel per Runge-Kutta stage over tiles of
 * TX x TY cells (primitives of the tile and its halo, faces, update; the last
 * stage also takes the CFL rate of the new state for the next step).  There
 * are DIS_NVARIANTS variants v: tile shape v % 3 (2D 16 x 15, 32 x 15, 32 x 7
 * cells per CTA of 256, 512, 256 threads; 1D 122, 250, 506 cells per CTA of
 * 128, 256, 512 threads) and register budget v / 3 (2D: 768 or 1024 resident
 * threads per SM; 1D: no limit, or at most 64 registers per thread).  The
 * limiter and the closure family are compiled into the kernels: a
 * DIS_VANLEER context of stiffened gases has one variant (5 in 2D, 1 in 1D),
 * a context with a Romenskii or JWL material one (2 in 2D, 1 in 1D; limiter
 * read at run time); changing the materials between the families returns a
 * fixed variant that no longer applies to tuning.  A DIS_HANCOCK context has
 * variants 0 .. 2 (the tile shapes; one kernel per step, about 104 KB of
 * shared memory per 2D CTA), van Leer and general closures the 32 x 7 tile
 * (2) in 2D and the 250-cell tile (1) in 1D.  The first
 * dis_step times one step of every variant (the last stage writing a scratch
 * buffer, so the state is unchanged) and keeps the fastest.  Returns the
 * chosen shape (0 x 0 before tuning or for float64 contexts), precomputed = 0
 * (kept for compatibility), and, if step_ms is not NULL, the tuned time per
 * step of each variant. */
#define DIS_NVARIANTS 6
int dis_tile_choice(const dis_ctx* ctx, int* tx, int* ty, int* precomputed, double* step_ms);

/* Fix the FP32-bulk stage variant (0 .. DIS_NVARIANTS - 1; a context with
 * one variant only that one) or return to tuning on the next step (-1).  For tests and measurements; the
 * result of a step does not depend on the variant beyond float32 rounding
 * order.  DIS_EINVAL for float64 contexts or an out-of-range variant. */
int dis_set_variant(dis_ctx* ctx, int variant);

/* Schedule of a 1D FP32-bulk batch (independent problems, one per patch):
 * 0 = per step one CFL launch and one stage-kernel launch per Runge-Kutta
 * stage over the tiles of all problems (captured as one CUDA graph per
 * step); 1 = one persistent launch per dis_step / dis_step_fixed_dt call
 * that runs all its steps, one CTA per problem (longest problems first),
 * with the problem's CFL rate and stages in turn, so a problem's state stays
 * in L2 between stages and steps; -1 (default) = the autotuner of the first
 * step times both and keeps the faster.  Both run the same tile arithmetic;
 * compiled as separate kernels they may contract multiply-adds differently,
 * so states agree to rounding, not bit for bit.
 * The variant (dis_set_variant) selects the tile length and register budget
 * in either schedule.  DIS_EINVAL for a NULL context, a schedule outside
 * -1..1, or 1 on a float64 or 2D context. */
int dis_set_schedule(dis_ctx* ctx, int schedule);

/* The schedule a step uses (0 or 1; -1 while a tuned context has not stepped)
 * and, if batch_ms is not NULL, the tuned one-step time of the persistent
 * kernel per variant (DIS_NVARIANTS values, 0 where not timed).  DIS_EINVAL
 * for a NULL context. */
int dis_schedule(const dis_ctx* ctx, int* schedule, double* batch_ms);

/* Pipelined host transfers (no counterpart in the paper).  dis_set_state_async
 * copies a host state (the packed layout of dis_set_state; pinned memory for
 * the copies to overlap anything) into one of two library staging buffers on a
 * copy stream and converts it into the context's state on the context's
 * stream, after the copy.  dis_get_state_async converts the state into one of
 * two other staging buffers on the context's stream and copies it to the host
 * buffer on a second copy stream.  Neither waits: a host-to-device copy for
 * the next step, the current step and a device-to-host copy of the previous
 * step can run at the same time.  The caller keeps the host buffers alive and
 * unchanged (resp. unread) until dis_sync, which waits for all three streams.
 * The staging buffers (4 states) are allocated by the first call and released
 * by dis_destroy.  Returns DIS_EINVAL (NULL argument, bad kind), DIS_ESTATE
 * (materials or state missing), DIS_ENOMEM, DIS_ECUDA. */
int dis_set_state_async(dis_ctx* ctx, int kind, const double* host_src);
int dis_get_state_async(dis_ctx* ctx, int kind, double* host_dst);
int dis_sync(dis_ctx* ctx);

/* Diagnostic: advance n_steps CFL steps like dis_step but launch kernel by
 * kernel with CUDA events between launches, and return in kernel_ms[4] the
 * mean device time per launch of the primitive-recovery, x-flux, y-flux (0 in
 * 1D) and update kernels (float64), or, FP32-bulk: slot 0 the CFL pass that
 * only the first step after a new state needs (timed once per step here, on
 * a scratch buffer), slot 1 the stage kernel.  Synchronises after every
 * stage.  DIS_EINVAL for a DIS_HANCOCK context. */
int dis_step_timed(dis_ctx* ctx, int n_steps, double* kernel_ms);

/* ---- Adjoint (reverse mode) of the float64 step -------------------------
 * The paper has no adjoint; these calls differentiate the discrete step of
 * Section 3 (EOS recovery, MUSCL/THINC-BVD reconstruction, elastic HLLD-type
 * fluxes, non-conservative terms, SSP-RK3, plastic radial return of Section
 * 3.2, RK4 reaction of Section 3.3) with every time step frozen at its
 * recorded value.  Branches (limiter, BVD choice, Riemann region, radial
 * return) are differentiated on the side the forward run took. */

/* Parameters with an adjoint: for material l, grad_params[3 l + k] is the
 * derivative with respect to k = 0: shear modulus G, 1: yield stress
 * sigma_y, 2: heat release Q (zero unless l is the reactive material). */
#define DIS_NPARAM 6

/* Forward run recorded for dis_adjoint, from the current state.  Takes
 * n_steps steps of the context's own step (float64 or FP32-bulk), with the
 * CFL time step (dt_in NULL)
 * or with dt_in[n * n_patches + p] (host array), copies the state to a
 * library-owned checkpoint every checkpoint_every steps and records every
 * dt.  If objective_material is 0 or 1 it accumulates the running objective
 *   J = sum_n dt_n sum_cells phi_l (rho u) dx dy     (l = objective_material,
 * states after each step, x momentum of the material's volume fraction) and
 * returns it in J_out (may be NULL).  dt_out (host, n_steps x n_patches, may
 * be NULL) receives the time steps.  Leaves the context at the final state,
 * like dis_step.  Device memory: (ceil(n_steps / checkpoint_every) +
 * 4 checkpoint_every + 8) states and 3 checkpoint_every sets of primitives
 * and face outputs (about 3.5 states each), allocated here, kept for dis_adjoint and
 * released by dis_destroy.  FP32-bulk contexts checkpoint their states in
 * float64 (plus float64 primitive and face buffers for the reverse sweep).
 * In a DIS_CYLINDRICAL context the geometric source of Section 3 is reversed
 * with the rest of the stage, and J is the same plain sum over cells (no
 * factor r).  Both limiters are reversed.  Stiffened-gas contexts reverse
 * every local map by hand; a context with a Romenskii material (Section
 * 2.3) reverses them by dual-number evaluation of the forward closure code
 * (planar geometry only; its G is G_0, and its yield strain follows G(rho)).
 * Returns DIS_EINVAL (bad arguments, a DIS_HANCOCK context: the adjoint
 * covers the Runge-Kutta scheme, a JWL or Johnson-Cook material, a reactive
 * material with a product closure of its own, or a Romenskii material in
 * cylindrical geometry), DIS_ESTATE (no state), DIS_ENOMEM, DIS_ECUDA.
 * Synchronises. */
int dis_adj_forward(dis_ctx* ctx, int n_steps, int checkpoint_every, int objective_material,
                    const double* dt_in, double* dt_out, double* J_out);

/* Reverse sweep of the last dis_adj_forward run: given the adjoint of the
 * final conservative state qbar_final (packed layout of dis_get_state, host
 * or device per qbar_on_device; NULL for zero) and the adjoint jbar of the
 * running objective, writes the gradient with respect to the initial state
 * into grad_init (packed layout, conservative or primitive variables per
 * out_kind; host or device per grad_on_device) and, if grad_params is not
 * NULL, the DIS_NPARAM parameter gradients selected by param_mask (bit k for
 * entry k; the others are set to 0).  Segments of checkpoint_every steps are
 * recomputed from their checkpoints with the float64 step (the state of the
 * context is not touched); for an FP32-bulk run the result is the float64
 * adjoint along a trajectory restarted from the FP32-bulk states at every
 * checkpoint.  Returns DIS_ESTATE without a recorded run, DIS_EINVAL,
 * DIS_ECUDA.  Synchronises. */
int dis_adjoint(dis_ctx* ctx, const double* qbar_final, int qbar_on_device, double jbar, int out_kind,
                double* grad_init, int grad_on_device, double* grad_params, unsigned param_mask);

/* Diagnostic: with on != 0, later dis_adjoint calls reverse every local map
 * (face Riemann problems, face states, THINC-BVD edge values, primitive
 * recovery, source steps) with dual numbers (one forward evaluation per input
 * direction, the reference form) instead of the hand-written reverses; both
 * give the same gradient up to rounding.  Returns DIS_EINVAL for a NULL
 * context. */
int dis_adj_reference(dis_ctx* ctx, int on);

/* Largest patch count accepted by dis_cfl_dt_static. */
#define DIS_STATIC_MAX_PATCHES 16384

/* Per-patch CFL time step of a conservative state, for callers that cannot
 * allocate device memory (code running where an allocation could
 * synchronise the device or be refused, e.g. inside a host callback, under a
 * framework that owns the device allocator, or after all device memory was
 * reserved up front).  The paper has no counterpart: this is the CFL
 * reduction of the step (dt = cfl / max over the patch of
 * sum_d (|u_d| + c_L) / dx_d) without a context.
 *   d_state: device pointer to the packed conservative state of n_patches
 *            patches (layout above) for materials[0..1];
 *   d_dt:    device pointer receiving n_patches float64 time steps; a patch
 *            with a cell that is not hyperbolic (c_L^2 <= 0), has no
 *            positive density, or is not finite gets NaN;
 *   stream:  cudaStream_t the work is ordered on (NULL = legacy default).
 * It allocates nothing: its scratch (per-patch maxima, flags and
 * descriptors) is a fixed area inside the library on each device,
 * DIS_STATIC_MAX_PATCHES entries (about 0.7 MB), held by every GPU that loads
 * the library until the process exits.  The first call on a device looks the
 * area up (with that device current).  Every call copies the patch
 * descriptors from a library host array with an ordinary asynchronous copy,
 * so the call must not be made while its stream is being captured into a
 * CUDA graph.  Each call clears the maxima and flags it uses; calls are
 * serialised on the host, but calls whose device work overlaps (different
 * streams) share the area and race.
 * Returns DIS_EINVAL for n_patches outside 1..DIS_STATIC_MAX_PATCHES, a
 * reactive material with a product closure of its own (not covered), or
 * other bad arguments (nothing is launched), DIS_ECUDA if a CUDA call
 * fails. */
int dis_cfl_dt_static(int dim, int n_patches, const dis_patch* patches,
                      const dis_material* materials, int reactive_material, double cfl,
                      const double* d_state, double* d_dt, void* stream);

/* Diagnostic (no counterpart in the paper): the device's measured
 * fused-multiply-add throughput, float32 and float64, in TFLOP/s (2 FLOP per
 * FMA), from a loop of independent FMA chains on 4 CTAs of 512 threads per
 * SM, best of three timed launches on `stream` (cudaStream_t, NULL = legacy
 * default); ms (may be NULL) receives the two launch times.  The rooflines
 * of the ALU-bound kernels are fractions of these.  Allocates a small output
 * buffer; synchronises.  DIS_EINVAL (NULL output), DIS_ENOMEM, DIS_ECUDA. */
int dis_alu_peaks(void* stream, double* fp32_tflops, double* fp64_tflops, double* ms);

/* ------------------------------------------------------------------------
 * Structured adaptive mesh refinement (Section 3, the AMR platform
 * paragraph: a hierarchy of levels refined recursively by a flagging
 * criterion, ratio 2 in space and time per level, the single-grid update
 * applied to every patch of a level; Section 4.2: difference-based
 * flagging).  The hierarchy covers one rectangular domain.  Level 0 is one
 * patch; level l + 1 refines whole blocks of block x block cells of level l
 * (block cells in 1D) into patches of 2 block x 2 block cells, stepped as
 * one batch.  Per level-0 step (dt_0 = min over levels of 2^l times the CFL
 * step of the cells level l owns), level l takes 2^l steps of dt_0 / 2^l;
 * before each Runge-Kutta stage the ghost cells of level l >= 1 come from
 * level l (copies) or from level l - 1 (conservative linear interpolation in
 * space, minmod slopes, and linear interpolation in time); after the two
 * steps of level l + 1 its mean replaces each covered cell of level l and the
 * conservative rows (phi_l rho_l, rho u, rho E, phi_y rho_y lam) of the level l
 * cells next to it are refluxed with the time- and area-averaged fine fluxes.
 * Every regrid_every level-0 steps the levels are rebuilt from the coarsest:
 * a cell is tagged when the fractional change of phi1, phi_l rho_l, p or a
 * velocity component to a face neighbour exceeds eps (floors: 1 for phi1,
 * u_floor for velocities), tags are dilated by `buffer` cells, and a block is
 * refined when it holds a tag and, on levels >= 1, its neighbouring blocks
 * are refined (proper nesting).  Float64; SSP-RK3 in planar or cylindrical
 * geometry (Section 3, cylindrical symmetry: x = r, y = z), or the
 * single-stage MUSCL-Hancock update (DIS_HANCOCK) in planar geometry, whose
 * one stage takes its ghost cells at the start of each step and registers
 * its fluxes with weight 1.  The cylindrical
 * step is the planar step plus the cell-centre geometric source, so the
 * conservative variables are per unit (r, z) area and the interpolation,
 * average-down and refluxing above act on them as in planar geometry; each
 * level takes the geometric source at its own cell-centre radii.  No
 * counterpart in the paper for the block and nesting rules: the paper's
 * platform leaves them to AMReX. */
typedef struct dis_amr dis_amr;
typedef struct {
  int32_t max_levels;   /* 1 .. 4 */
  int32_t block;        /* block edge in cells of the coarser level, >= 4; divides nx (and ny) */
  double eps;           /* flagging threshold (fractional change) */
  int32_t buffer;       /* tag dilation in cells */
  double u_floor;       /* velocity floor of the fractional change (m/s) */
  int32_t regrid_every; /* level-0 steps between regrids (0 = never after the first) */
} dis_amr_options;

/* domain: the level-0 patch (bc: transmissive, periodic or reflective; in
 * cylindrical geometry x0 >= 0 is the radius of its axis-side face, and a
 * domain on the axis has x0 = 0 and a reflective x-low side); opt: as
 * dis_create (precision DIS_FP64; scheme DIS_RK3 with geometry DIS_PLANAR
 * or DIS_CYLINDRICAL, or DIS_HANCOCK with DIS_PLANAR).  DIS_EINVAL for other
 * options or a block that does not divide the domain; DIS_ECUDA. */
int dis_amr_create(int dim, const dis_patch* domain, int reactive_material, const dis_options* opt,
                   const dis_amr_options* aopt, void* stream, dis_amr** out);
/* Materials of every level (as dis_set_materials). */
int dis_amr_set_materials(dis_amr* h, const dis_material* m, int n);
/* Level-0 state (host or device pointer, kind DIS_CONSERVATIVE or
 * DIS_PRIMITIVE, the layout of dis_set_state for the domain patch); builds
 * the finer levels by flagging and conservative interpolation. */
int dis_amr_set_state(dis_amr* h, const double* src, int kind);
/* n level-0 steps (all levels subcycled, regrids as configured); dt_out
 * (host, may be NULL) receives the n level-0 time steps.  Synchronises.
 * DIS_ENONPHYSICAL if a level lost hyperbolicity (dis_amr_check). */
int dis_amr_step(dis_amr* h, int n_steps, double* dt_out);
/* Number of levels in use and blocks (patches) per level (counts[max_levels],
 * level 0 counts 1). */
int dis_amr_levels(const dis_amr* h, int* n_levels, int* counts);
/* Level `level` as a dense array of the whole domain at that level's
 * resolution (host; the dis_get_state layout of a patch of nx 2^l x ny 2^l
 * cells, kind DIS_CONSERVATIVE or DIS_PRIMITIVE); cells the level does not
 * own hold NaN; active (host, may be NULL) receives 1 for owned cells. */
int dis_amr_get_level(dis_amr* h, int level, int kind, double* dst, unsigned char* active);
/* Sum over the cells no finer level covers of each conservative field times
 * the cell volume (nf values, host). */
int dis_amr_totals(dis_amr* h, double* out);
/* Status of the levels: DIS_OK or DIS_ENONPHYSICAL with the level, block and
 * cell of the first bad cell. */
int dis_amr_check(dis_amr* h, int* level, int* patch, int* cell);
void dis_amr_destroy(dis_amr* h);

/* Thread-local text of the last error (never NULL). */
const char* dis_last_error(void);

void dis_destroy(dis_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DIS_H */
