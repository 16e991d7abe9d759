/*
 * lbm.h - C ABI of the GB300 reactive-mixture lattice Boltzmann library.
 *
 * The library advances the lattice Boltzmann model for reactive mixtures of
 * Sawant, Dorschner & Karlin (arXiv 2108.07605): M species lattices with
 * Stefan-Maxwell diffusion and reaction sources (Sec. 2), a momentum lattice
 * f with the extended equilibrium and an energy lattice g carrying the
 * enthalpy of formation (Sec. 3), the M-th species slaved to f (Sec. 3.7,
 * Eq. strongest), Arrhenius chemistry in l forward-Euler sub-steps at frozen
 * energy (Sec. 2.4, Eq. R3) and the temperature recovered from energy by
 * Newton iteration (Sec. 3.1, Eq. temperature).  Every step runs in CUDA
 * kernels for sm_103a on the caller's stream; there is no CPU fallback.
 *
 * Conventions shared by all entry points
 *  - Units at the boundary are SI: kg/m^3, m/s, K, Pa, J/kg.  Internally the
 *    library uses lattice units dx = dt = 1 with acoustic scaling (Sec. 3.6):
 *    velocities are divided by the reference speed c_ref, dt = dx / c_ref.
 *  - Node index n = x + nx*(y + ny*z), x fastest; N = nx*ny*nz.
 *  - Field arrays: scalar fields [N]; velocity [3][N] (component-major, all
 *    three components even for D2Q9, where u_z is written as 0 and ignored
 *    on input); mass fractions [M][N] (species-major).
 *  - Populations: [lattice][i][N] with lattice 0..M-2 the stored species,
 *    M-1 the momentum lattice f, M the energy lattice g; velocity index
 *    i = (cz+1)*9 + (cy+1)*3 + (cx+1) (D3Q27) or (cy+1)*3 + (cx+1) (D2Q9),
 *    so the opposite of i is Q-1-i.
 *  - "on_device" = 1: pointers are device memory of the handle's GPU and the
 *    call is asynchronous on the handle's stream; 0: host memory, the call
 *    copies and synchronises the stream.
 *  - The caller owns every array it passes.  The library owns its population
 *    buffers, allocated through cfg->dev_alloc (or cudaMalloc when NULL) at
 *    lbm_create and released at lbm_destroy.
 *  - Errors: calls return lbm_status.  Invalid arguments return
 *    LBM_ERR_INVALID without touching state.  Device-side failures (Newton
 *    not converged, non-finite moments) are recorded in a sticky status word
 *    and returned by the next synchronising call (lbm_moments,
 *    lbm_synchronize, lbm_get_populations).  lbm_last_error() gives text.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_MAX_SPECIES 9
#define LBM_MAX_REACTIONS 32
#define LBM_NCP 3

typedef enum {
  LBM_OK = 0,
  LBM_ERR_INVALID = 1,   /* bad argument or configuration                   */
  LBM_ERR_OOM = 2,       /* device allocation failed                        */
  LBM_ERR_CUDA = 3,      /* a CUDA runtime call failed                      */
  LBM_ERR_NEWTON = 4,    /* temperature Newton did not converge (Eq. temperature) */
  LBM_ERR_NONFINITE = 5, /* a non-finite or non-positive density appeared   */
  LBM_ERR_RANGE = 6,     /* size beyond a documented limit                  */
  LBM_ERR_TIMEOUT = 7,   /* a bounded device wait gave up                   */
  LBM_ERR_STATE = 8      /* call out of order (e.g. step before init)       */
} lbm_status;

typedef enum { LBM_D2Q9 = 0, LBM_D3Q27 = 1 } lbm_lattice;

/* Storage precision of the populations.  LBM_FP64: every operation in FP64
 * (the path checked against the oracle to 1e-10).  LBM_FP32_STORE:
 * populations, moments and collision in FP32; the temperature Newton solve
 * and the chemistry in float-float (pairs of FP32, ~48 significant bits);
 * transport in FP32.  LBM_FP16_OFFSET: the FP32 path's arithmetic, with
 * populations stored as FP16 offsets (the storage reading of the paper's
 * lattice weights): h = (f - o) / s, o = the equilibrium population of the
 * mean initial state at rest (per lattice and direction), s = a per-lattice
 * scale; both are fixed by lbm_init_fields from the initial fields (16x
 * headroom over the initial deviations) and kept by checkpoints.  Field
 * tolerances vs FP64 are stated in the tests. */
typedef enum { LBM_FP64 = 0, LBM_FP32_STORE = 1, LBM_FP16_OFFSET = 2 } lbm_precision;

/* Face boundary kinds (Sec. 4): periodic; bounce-back wall (Eq. bb);
 * Tamm-Mott-Smith isothermal wall (Sec. 4.2.2); flux inlet (Sec. 4.3);
 * LODI outlet with convective mass fractions (Sec. 4.4). */
typedef enum {
  LBM_PERIODIC = 0, LBM_BOUNCE_BACK = 1, LBM_TMS_WALL = 2, LBM_INLET = 3,
  LBM_OUTLET = 4
} lbm_bc;

/* Species, thermodynamics, reactions and transport (Sec. 3.6).  Plain data,
 * copied by lbm_create.
 *  Heat capacity  c_p/R_U = cp[a][0] + cp[a][1] T + cp[a][2] T^2.
 *  Enthalpy       h_a = h_formation[a] + int_T0^T c_p dT'  (J/mol, T0 = 298.15 K).
 *  Entropy        s_a = s_standard[a] + int_T0^T c_p/T' dT' (J/(mol K)).
 *  Rate constant  k_f = A T^b exp(-Ea/(R_U T)), SI (m^3/mol)^(order-1)/s.
 *  Reverse rate   k_f / K_c, K_c from the table's Gibbs energies.
 *  Third body     [M] = sum_a efficiency[r][a] C_a multiplies the rate.
 *  Transport      D_ab = D0[a][b] (T/T0)^D_T_exponent (P0/P);
 *                 mu = mu0 (T/T0)^mu_T_exponent; lambda = mu c_p / prandtl. */
typedef struct lbm_mechanism {
  int n_species;                                   /* M, 2..LBM_MAX_SPECIES */
  int n_reactions;                                 /* 0..LBM_MAX_REACTIONS  */
  double molar_mass[LBM_MAX_SPECIES];              /* kg/mol                */
  double cp[LBM_MAX_SPECIES][LBM_NCP];
  double h_formation[LBM_MAX_SPECIES];             /* J/mol at T0           */
  double s_standard[LBM_MAX_SPECIES];              /* J/(mol K) at T0, P0   */
  int nu_f[LBM_MAX_REACTIONS][LBM_MAX_SPECIES];    /* reactant coefficients */
  int nu_r[LBM_MAX_REACTIONS][LBM_MAX_SPECIES];    /* product coefficients  */
  double arrhenius[LBM_MAX_REACTIONS][3];          /* A, b, Ea (J/mol)      */
  int third_body[LBM_MAX_REACTIONS];
  double efficiency[LBM_MAX_REACTIONS][LBM_MAX_SPECIES];
  int reversible[LBM_MAX_REACTIONS];
  double D0[LBM_MAX_SPECIES][LBM_MAX_SPECIES];     /* m^2/s at T0, P0       */
  double D_T_exponent;
  double mu0;                                      /* Pa s at T0            */
  double mu_T_exponent;
  double prandtl;
  /* viscosity_model 0: mu = mu0 (T/T0)^mu_T_exponent; 1: Wilke's mixing rule
   * over the species viscosities mu0_species[a] (T/T0)^mu_T_exponent (Pa s at
   * T0): mu = sum_a X_a mu_a / sum_b X_b Phi_ab, Phi_ab = [1 + (mu_a/mu_b)^1/2
   * (m_b/m_a)^1/4]^2 / [8 (1 + m_a/m_b)]^1/2, X the mole fractions.  In
   * both, lambda = mu C_p / Pr (the paper's transport comes from Cantera,
   * which this library does not carry). */
  int viscosity_model;
  double mu0_species[LBM_MAX_SPECIES];
} lbm_mechanism;

typedef struct lbm_config {
  lbm_lattice lattice;
  int nx, ny, nz;             /* nz = 1 for D2Q9                              */
  lbm_precision precision;
  int substeps;               /* reaction sub-steps l (Eq. R3), >= 1          */
  double dx;                  /* lattice spacing, m                           */
  double c_ref;               /* reference speed, m/s; 0 selects
                                 sqrt(max_a R_a * T_max / 0.9)               */
  double T_max;               /* K, used only by the default c_ref            */
  lbm_mechanism mech;
  lbm_bc face_bc[6];          /* faces -x, +x, -y, +y, -z, +z                  */
  double wall_T[6];           /* TMS wall temperature per face, K             */
  const uint8_t* solid_mask;  /* optional host [N], 1 = solid node (staircase
                                 walls); NULL = no solid nodes                */
  lbm_bc solid_bc;            /* LBM_BOUNCE_BACK or LBM_TMS_WALL              */
  const double* wall_T_nodes; /* optional host [N] TMS target temperature of
                                 each interface node, K; NULL = face values   */
  const double* inlet_u;      /* optional host [3][N] inlet velocity of each
                                 inlet node, m/s; NULL = inlet_u_uniform      */
  double inlet_u_uniform[3];
  double inlet_Y[LBM_MAX_SPECIES];
  double inlet_T, inlet_P;
  double outlet_P;            /* LODI target pressure, Pa                     */
  double outlet_sigma;        /* LODI relaxation factor                       */
  int newton_max_iter;        /* default 50                                   */
  double newton_rtol;         /* default 1e-13                                */
  void* (*dev_alloc)(size_t bytes, void* user);  /* NULL: cudaMalloc          */
  void (*dev_free)(void* ptr, void* user);
  void* alloc_user;
  void* stream;               /* cudaStream_t; NULL = legacy default stream   */
  int device;                 /* CUDA device ordinal                          */
  int inlet_simplified;       /* 1: the simplified flux inlet of Sec. 4.3 -
                                 stop after the local state of step 2 and set
                                 every population of the inlet node to the
                                 local equilibria (u and T take local values,
                                 not the targets); 0 (default): the full
                                 four-step inlet                              */
  const double* wall_dist;    /* optional, host [N]: normal distance from each
                                 node to the wall (lattice units, >= 0 at
                                 fluid nodes), with wall_normal; NULL: the
                                 TMS targets apply at the interface node
                                 itself (walls on the grid or staircase)      */
  const double* wall_normal;  /* optional, host [3][N]: inward unit normal of
                                 the wall at each node.  With both arrays a
                                 TMS interface node takes its targets (Sec.
                                 4.2.2, last paragraph) by linear
                                 interpolation along the normal between the
                                 wall (u = u_a = 0, T = its wall temperature)
                                 and the fluid node x + c_k most aligned with
                                 the normal, from that node's stored
                                 post-collision fields; a node whose x + c_k
                                 is solid or beyond a non-periodic face keeps
                                 the wall values.  Copied at lbm_create.      */
  double outlet_length;       /* LODI length L (lattice units) in the incoming
                                 wave's relaxation K = sigma (1 - Ma^2) c / L;
                                 0 (default): the domain's extent along the
                                 outlet normal.  A slab of a longer domain
                                 gives the whole domain's length.             */
  int chem_fp64;              /* with LBM_FP32_STORE: 1 runs the temperature
                                 Newton solves (Sec. 3.1 Eq. temperature) and
                                 the reaction sub-steps (Sec. 2.4 Eq. R3) in
                                 native FP64 instead of float-float; the
                                 populations, moments, transport and
                                 collision stay FP32.  Ignored for LBM_FP64;
                                 LBM_ERR_INVALID with LBM_FP16_OFFSET.
                                 Default 0.                                   */
} lbm_config;

/* Derived lattice-unit data of a handle. */
typedef struct lbm_info {
  int Q, D, L, M;             /* velocities, dimension, lattices, species     */
  long long n_nodes;
  double c_ref, dt, dx;       /* m/s, s, m                                    */
  size_t bytes_per_population;
  size_t device_bytes;        /* everything the handle allocated              */
  long long steps_done;
} lbm_info;

typedef struct lbm_ctx* lbm_t;

/* Fill *cfg with defaults (D3Q27, FP64, periodic, l = 2, Newton 50 / 1e-13,
 * T_max = 3000 K, outlet_sigma = 0.25).  Mechanism left zeroed. */
void lbm_config_defaults(lbm_config* cfg);

/* Bytes of device memory lbm_create would allocate for cfg, or 0 if cfg is
 * invalid.  Lets a caller admit work against a memory budget. */
size_t lbm_bytes_required(const lbm_config* cfg);

/* Validate cfg, copy it, allocate the handle's device buffers.  Populations
 * are undefined until lbm_init_fields.  On failure *out is NULL. */
lbm_status lbm_create(const lbm_config* cfg, lbm_t* out);

/* Set every population to the equilibria of the given fields (Sec. 4.1,
 * Eqs. faEqGeneral, fEqGeneral, gEqGeneral): species f_a^eq(rho Y_a, u, T)
 * for a < M, the momentum equilibrium f^eq(rho, Y, u, T) (Eq. feq) and the
 * energy equilibrium g^eq(rho, Y, u, T) (Eq. geq_i).  rho [N] kg/m^3,
 * u [3][N] m/s, T [N] K, Y [M][N].  Also sets the temperature guess. */
lbm_status lbm_init_fields(lbm_t h, const double* rho, const double* u,
                           const double* T, const double* Y, int on_device);

/* As lbm_init_fields with the density from the ideal-gas law
 * rho = P / (R T), R = R_U sum_a Y_a/m_a (Sec. 2.1, Eq. eosIdealGas);
 * P [N] in Pa. */
lbm_status lbm_init_fields_pressure(lbm_t h, const double* P, const double* u,
                                    const double* T, const double* Y,
                                    int on_device);

/* Advance nsteps time steps (each: pull streaming, boundary reconstruction,
 * moments, temperature, relaxation, gradients, diffusion velocities,
 * reaction sub-steps, collision of all lattices; Sec. 2.3, Sec. 3, Sec. 4).
 * Asynchronous on the handle's stream. */
lbm_status lbm_step(lbm_t h, int nsteps);

/* Advance several handles by nsteps steps together, in the placement a
 * batch plan of the same handles starts with (see lbm_batch_set_launch):
 * FP64 storage under 311,296 nodes in all, each step is ONE persistent
 * launch over a work-list of the handles' tiles (persistent = 2); else one
 * launch per kernel over the concatenated tiles (128-node tiles, 64
 * interface nodes per boundary block), so many small domains fill the GPU.
 * The handles must share lattice, species count, precision and device; each
 * keeps its own mechanism, units and boundaries.  The work runs on hs[0]'s
 * stream after the earlier work of every handle's stream, and every
 * handle's stream waits for it; with the single launch the call returns
 * after the work (its work-list is freed).  Results equal n separate
 * lbm_step calls to rounding (the same per-node arithmetic, summed in
 * another order where the placements differ). */
lbm_status lbm_batch_step(lbm_t* hs, int n, int nsteps);

/* A batch plan: the batched step of lbm_batch_step for a fixed set of
 * handles, captured once as CUDA graphs (one step and two steps, from either
 * buffer parity) and replayed by lbm_batch_run.  The plan owns a stream; a
 * run waits for every handle's stream and every handle's stream waits for
 * the run.  If a handle is advanced on its own between runs, the next run
 * refreshes the plan's view of it.  Handles must outlive the plan. */
typedef struct lbm_batch_ctx* lbm_batch_t;
lbm_status lbm_batch_create(lbm_t* hs, int n, lbm_batch_t* out);
lbm_status lbm_batch_run(lbm_batch_t b, int nsteps);
lbm_status lbm_batch_destroy(lbm_batch_t b);

/* Kernel placement of a step.  A performance choice only: every placement
 * evaluates the same formulas; they agree to rounding.
 *   chem_lanes     threads per node of the moments and reaction sub-steps
 *                  (Sec. 2.4, Eq. R3): 1 = one thread per node; 4 or 8 = a
 *                  group of that many lanes per node shares the pull, the
 *                  temperature solve and the node's reactions (for grids too
 *                  small to fill the GPU at one thread per node); -1 = by
 *                  grid size.  Interface nodes (boundary reconstruction) take
 *                  their sub-steps, in every placement, with one thread each
 *                  when a grid has at least 19,456 of them and with eight
 *                  lanes each otherwise (the single launch of a plan: one
 *                  thread each).
 *   collide_split  0 = one thread per node does the whole collision; 1 = a
 *                  per-node kernel stores the collision parameters and a
 *                  second kernel updates the directions with nine threads
 *                  per node; -1 = default.
 * Defaults (below 77,824 nodes, four 128-thread blocks per SM of a 152-SM
 * GPU, a grid is small): collide_split 0 for FP64 storage on grids that are
 * not small (except the single launch of a plan, see persistent), else 1;
 * chem_lanes 4 for small FP32-storage grids, else 1.
 * lbm_set_launch rejects other values with LBM_ERR_INVALID. */
typedef struct {
  int chem_lanes;
  int collide_split;
  int persistent;     /* batch plans only: 1 = every batched kernel runs a grid
                         of the blocks the GPU holds at once, each block
                         looping over tiles of the work-list; 2 = the whole
                         step as ONE launch: a grid of the resident blocks
                         claims the items of a work-list in stage order
                         (boundary + sub-steps of 128 interface nodes,
                         moments + sub-steps of a node tile; collision
                         parameters of a node tile once its domain's first
                         stage is done and the collision of 32 nodes once
                         their parameters are, or with collide_split 0 the
                         whole collision of a node tile once its domain's
                         first stage is done), with chem_lanes 1; a
                         dependency wait that outlasts 4 s
                         ends the launch and the handles report
                         LBM_ERR_TIMEOUT; 0 = one block per tile; -1 = the
                         default: 2 for plans of FP64 storage below 311,296
                         nodes in all, else 0 */
  int nodes_per_thread;  /* persistent = 2: nodes per thread of the node
                         tiles, 1, 2 or 4 (tiles of 128, 256, 512 nodes);
                         -1 = 1 */
} lbm_launch;

/* Set / read the handle's placement (lbm_get_launch reports the resolved
 * values). */
lbm_status lbm_set_launch(lbm_t h, const lbm_launch* l);
lbm_status lbm_get_launch(lbm_t h, lbm_launch* l);

/* Autotuner: times trial_steps steps of each placement (chem_lanes 1, 4, 8
 * x collide_split 0, 1) on the handle's own state and keeps the fastest
 * (written to *chosen when not NULL).  The trial steps read the current
 * populations and write the spare buffer without advancing the handle; the
 * temperature guesses they update are restored, so the solve continues
 * exactly as without the call.  Synchronises. */
lbm_status lbm_autotune(lbm_t h, int trial_steps, lbm_launch* chosen);

/* The same for a batch plan: times trial_steps replays of each placement's
 * captured one-step graph over the whole batch (the six placements above,
 * the best of them with persistent grids, and the single launch with split
 * and fused collision, each with 1, 2 and 4 nodes per thread), keeps the
 * fastest and captures the plan's graphs
 * again with it.  A new plan starts with the default placement (see
 * lbm_batch_set_launch). */
lbm_status lbm_batch_autotune(lbm_batch_t b, int trial_steps, lbm_launch* chosen);

/* Set a plan's placement (-1 fields: the default for the batch's precision
 * and total node count) and capture its graphs again; read the placement in
 * use.  A
 * performance choice with no counterpart in the paper: every placement
 * computes the step of Secs. 2-4.  The handles' own lbm_set_launch values do
 * not apply to plans.  l is the caller's; the plan keeps a copy.
 * LBM_ERR_INVALID for a NULL plan or l, or values out of range (the plan is
 * unchanged); LBM_ERR_CUDA if the new graphs cannot be captured (destroy
 * the plan then). */
lbm_status lbm_batch_set_launch(lbm_batch_t b, const lbm_launch* l);

/* The work-list of the single-launch batched step (persistent = 2) for n
 * domains of nodes[k] nodes, n_if[k] of them interface nodes: host only (no
 * device, no handle), the list a plan of such handles uploads.  items
 * receives five values per item, in list order: kind (0 boundary: 128
 * interface nodes from `first`; 1 moments and 2 collision parameters: a
 * tile of 128 x nodes_per_thread nodes; 3 collision: 32 nodes; 4 fused
 * collision: a tile), domain, first (interface index or node), dep (kinds 2
 * and 4: the count of the domain's kind-0 and kind-1 items they wait for;
 * kind 3: the flag it waits for), flag (kind 2: the flag it sets).  Every
 * dependency names items earlier in the list, the property that lets the
 * launch's bounded waits end without a co-residency guarantee.  *nitems and
 * *nsync receive the item and sync-word counts (cap = 0: counts only).
 * LBM_ERR_INVALID for NULL pointers, n < 1, nodes_per_thread not 1, 2 or 4,
 * or a domain with nodes < 1 or n_if outside 0..nodes; LBM_ERR_RANGE if cap
 * (> 0) is below the item count. */
lbm_status lbm_worklist(const long long* nodes, const long long* n_if, int n,
                        int nodes_per_thread, int collide_split, long long* items, int cap,
                        int* nitems, int* nsync);
lbm_status lbm_batch_get_launch(lbm_batch_t b, lbm_launch* l);

/* As lbm_step, and adds each kernel's device time in milliseconds, measured
 * with CUDA events recorded on the handle's stream around every launch:
 * kernel_ms[0] += boundary + moments/temperature (+ chemistry) kernels,
 * kernel_ms[1] += collision
 * kernel (n_kernels >= 2).  Synchronises the stream before returning. */
lbm_status lbm_step_timed(lbm_t h, int nsteps, double* kernel_ms, int n_kernels);

/* Fields of the stored post-collision state in SI units, T from Newton on
 * Eq. temperature.  Any pointer may be NULL to skip that field.
 * rho [N], u [3][N], T [N], Y [M][N], E [N] total specific energy (J/kg).
 * Host pointers (on_device = 0) synchronise and return sticky errors. */
lbm_status lbm_moments(lbm_t h, double* rho, double* u, double* T, double* Y,
                       double* E, int on_device);

/* Flame diagnostics of the stored state, the quantities the paper follows
 * in its microchannel and microtube runs (Sec. 5.3), computed on the device
 * in one pass with FP64 arithmetic whatever the storage: per node the
 * moments, T by Newton on Eq. temperature, the mass production rates of the
 * mechanism and the heat release rate q = -sum_a H_a(T) rho_dot_a (W/m^3,
 * H_a the specific enthalpy with formation, so q < 0 where the reactions are
 * endothermic); then reductions over the fluid nodes in a fixed order (the
 * result does not depend on scheduling).  Synchronises; returns sticky errors. */
typedef struct {
  double hrr_integral;   /* sum of q times the cell volume dx^3 (W); in 2-D the
                            cell area dx^2 (W per metre of depth) */
  double hrr_max;        /* largest q (W/m^3) */
  double flame_x;        /* x coordinate (node index along x times dx, m) of the
                            node with the largest q; among equal maxima the
                            smallest node index (x fastest) */
  double T_max;          /* K */
  double u_max;          /* largest |u| (m/s) */
} lbm_diag;
lbm_status lbm_diagnostics(lbm_t h, lbm_diag* out);
/* The same over the nodes with x in [x0, x0 + nplanes) only (the own planes
 * of a slab, whose partial results combine over the slabs: sums add,
 * maxima take the largest, flame_x that of the largest hrr_max); flame_x is
 * the x coordinate in this handle's grid, NaN (and hrr_max, T_max, u_max
 * -inf) when the planes hold no fluid node.  LBM_ERR_RANGE for planes
 * outside 0..nx-1. */
lbm_status lbm_diagnostics_planes(lbm_t h, int x0, int nplanes, lbm_diag* out);

/* All stored populations converted to FP64, layout [lattice][i][N]
 * (lattice-unit values: species and f in kg/m^3, g in kg/m^3 * J/kg / c_ref^2). */
lbm_status lbm_get_populations(lbm_t h, double* out, int on_device);

/* Wait for the handle's stream; returns and clears nothing else than the
 * sticky device status. */
lbm_status lbm_synchronize(lbm_t h);

/* Checkpoint: raw populations (storage precision), temperature guess and,
 * for FP16 offset storage, the codec (offsets and scales).  lbm_get_state
 * with buf == NULL stores the size. */
lbm_status lbm_get_state(lbm_t h, void* buf, size_t* bytes);
lbm_status lbm_set_state(lbm_t h, const void* buf, size_t bytes);

lbm_status lbm_get_info(lbm_t h, lbm_info* info);

/* Release the handle and its device memory.  Returns the sticky status. */
lbm_status lbm_destroy(lbm_t h);

/* Test hook with no counterpart in the paper: the library's float-float exp
 * and log (the functions of the mixed-precision path's Arrhenius rates and
 * temperature) evaluated on the current device at the host values x[0..n),
 * each first split into float-float (hi = x rounded to FP32, lo = x - hi
 * rounded to FP32).  exp_out and log_out (host, n doubles each) receive
 * hi + lo of the results; log of a value whose hi is not positive is NaN.
 * exp returns +inf above 88.7 and 0 below -103; results below 2^-102 keep
 * only the spacing of FP32's denormals in their low part (float-float has
 * FP32's exponent range).  Allocates and frees its own
 * device scratch; synchronous.  LBM_ERR_INVALID for NULL buffers or n < 0,
 * LBM_ERR_RANGE for n > 2^24, LBM_ERR_CUDA on a device error (message in
 * lbm_last_error(NULL)). */
lbm_status lbm_ff_check(const double* x, long long n, double* exp_out, double* log_out);

/* The FP64 exp of the reaction rates (Sec. 3.6's Arrhenius form and the
 * reverse rates from equilibrium constants: exp of ln k), Tang's
 * table-driven method, at the n points x (host arrays; exp_out receives n
 * values).  A test hook for its accuracy; synchronous.  LBM_ERR_INVALID for
 * NULL buffers or n < 0, LBM_ERR_RANGE for n > 2^24, LBM_ERR_CUDA on a
 * device error. */
lbm_status lbm_exp64_check(const double* x, long long n, double* exp_out);

/* Measured fused-multiply-add throughput of the current device in TFLOP/s
 * (2 FLOP per FMA), FP64 when fp64 != 0, else FP32.  No counterpart in the
 * paper: the ALU roof against which the step's executed operation counts
 * are reported.  Eight independent FMA chains per thread, eight 256-thread
 * blocks per SM, best of three timed launches.  Synchronous; allocates and
 * frees one element of device memory.  LBM_ERR_INVALID for a NULL tflops,
 * LBM_ERR_CUDA on a device error. */
lbm_status lbm_fma_peak(int fp64, double* tflops);

/* Check of the bounded device wait the single-launch batched step uses for
 * its dependencies (no counterpart in the paper): one thread waits for a
 * device word that is already 1 (set_word = 1) or that nothing sets
 * (set_word = 0), giving up after timeout_ns.  result[0] = 1 if the wait saw
 * the word set, result[1] = the abort word afterwards (1 after a timeout),
 * result[2] = the wait's length in microseconds.  Synchronous; on the current
 * device.  LBM_ERR_INVALID for a NULL result or a negative timeout,
 * LBM_ERR_RANGE for timeout_ns > 1e8, LBM_ERR_CUDA on a device error. */
lbm_status lbm_wait_probe(int set_word, long long timeout_ns, long long* result);

/* Allocation-free single step.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory themselves -
 * a solver embedded in an application that owns every device allocation
 * through its own pool, a loop on a latency budget where cudaMalloc/cudaFree
 * would synchronise the device, or a process under a fixed memory budget.
 * It advances caller-owned populations by one step exactly as lbm_step does
 * for a handle created from the same cfg, and calls no allocator.
 *  cfg      the configuration lbm_create takes (periodic faces; cfg->stream,
 *           cfg->device and cfg->precision are honoured, except FP16 offset
 *           storage, whose codec only a handle keeps: LBM_ERR_INVALID; the
 *           allocation hooks are ignored).
 *  pops_in  device, stored populations in cfg->precision, layout
 *           [lattice][i][N] (what lbm_get_populations returns for FP64).
 *  pops_out device, same size, distinct from pops_in; receives the step.
 *  T_guess  device [N] temperature guess in K, read and overwritten with the
 *           step's temperatures (the initial temperatures before the first
 *           step).
 *  error    optional; set to a message on failure (valid until the next
 *           call on the same thread).
 * The per-node scratch lives in a fixed array inside the library sized for
 * LBM_NOALLOC_MAX_NODES nodes: 16 384 x 61 + 32 doubles = 7 995 648 bytes,
 * held by every GPU that loads the library until the process exits, whether
 * or not this function is called; larger grids return LBM_ERR_RANGE.
 * Every call shares that array, so calls that overlap on the GPU race.  The
 * first call on a device looks up the array's device address; make it
 * before any stream capture.  The address is kept for the life of the
 * process: after a cudaDeviceReset of that device do not call this again.
 * The step always runs in the library's fixed placement (one thread per
 * node for the moments with the reaction sub-steps inline, the fused
 * collision kernel), which lbm_step uses after
 * lbm_set_launch({chem_lanes = 1, collide_split = 0}); with that placement
 * the two agree bit for bit, with another to the rounding of the changed
 * summation order.  cfg->device must name a present GPU (LBM_ERR_RANGE).
 * The call waits for its stream and returns the step's device status
 * (LBM_ERR_NEWTON, LBM_ERR_NONFINITE). */
#define LBM_NOALLOC_MAX_NODES 16384
lbm_status lbm_step_noalloc(const lbm_config* cfg, const void* pops_in, void* pops_out,
                            double* T_guess, const char** error);

/* Halo planes for an x-slab domain decomposition (the paper runs on one
 * domain; the slab split keeps every step of Sec. 2-4 local to
 * a node and its neighbours up to two planes away, so a slab that receives
 * its neighbours' two nearest planes before each step advances its own
 * planes exactly as the undivided domain would).
 * lbm_get_planes copies planes x0 .. x0+nplanes-1 of the current state out
 * to buf, lbm_set_planes copies buf into them: the populations
 * [L][Q][nz][ny][nplanes] in the storage precision (8 bytes FP64, 4 bytes
 * FP32), then the temperature guesses [nz][ny][nplanes] as doubles; total
 * nplanes*ny*nz*(L*Q*elem + 8) bytes.  buf is host memory, or device memory
 * on the handle's device when on_device != 0; owned by the caller.
 * Synchronous (the handle's stream is drained).  LBM_ERR_RANGE for planes
 * outside 0..nx-1, LBM_ERR_INVALID for FP16 offset storage (its codec is a
 * property of each handle) or a NULL buffer, LBM_ERR_STATE before
 * lbm_init_fields. */
lbm_status lbm_get_planes(lbm_t h, int x0, int nplanes, void* buf, int on_device);
lbm_status lbm_set_planes(lbm_t h, int x0, int nplanes, const void* buf, int on_device);

/* Text of the last error on h (or of the last lbm_create failure if h is
 * NULL).  Valid until the next call on h. */
const char* lbm_last_error(lbm_t h);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
