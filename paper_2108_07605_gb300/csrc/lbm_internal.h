// Internal declarations shared by the host API (lbm_capi.cu) and the kernels
// (lbm_kernels.cuh and its instantiations).  Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include <cuda_fp16.h>

#include "ff.cuh"

namespace lbm {

constexpr double R_U = 8.314462618;       // J/(mol K)
constexpr double T_REF = 298.15;          // K, T0 of Sec. 3.6
constexpr double P_REF = 101325.0;        // Pa, P0 of Sec. 3.6
constexpr double RHO_TINY = 1e-300;       // u_a := u below this species density

// status bits written by kernels with atomicOr
constexpr int ST_NEWTON = 1;
constexpr int ST_NONFINITE = 2;
constexpr int ST_RANGE = 4;
constexpr int ST_TIMEOUT = 8;   // a bounded device wait gave up

struct DevReaction {
  int nr, np;            // number of reactant / product molecules (<= 3)
  int reac[3], prod[3];  // species index per molecule (repeated for nu = 2)
  int dn;                // sum of product minus reactant coefficients
  int reversible, third_body;
  double lnA, b, EaR;    // ln A, temperature exponent, Ea / R_U
  ff lnA_f, b_f, EaR_f;  // the same as float-float (mixed path)
};

// Mechanism in the forms the kernels evaluate (built on the host).
struct DevMech {
  int M, R;
  double mm[LBM_MAX_SPECIES], inv_mm[LBM_MAX_SPECIES], Ra[LBM_MAX_SPECIES];
  // U_a(T) = u0 + u1 T + u2 T^2 + u3 T^3  (J/kg, incl. formation)
  double u0[LBM_MAX_SPECIES], u1[LBM_MAX_SPECIES], u2[LBM_MAX_SPECIES],
      u3[LBM_MAX_SPECIES];
  // g_a/(R_U T) = g_inv/T + g0 + g1 T + g2 T^2 - a0 ln T
  double g_inv[LBM_MAX_SPECIES], g0[LBM_MAX_SPECIES], g1[LBM_MAX_SPECIES],
      g2[LBM_MAX_SPECIES], a0[LBM_MAX_SPECIES];
  double ln_p0_over_ru;
  DevReaction rx[LBM_MAX_REACTIONS];
  double eff[LBM_MAX_REACTIONS][LBM_MAX_SPECIES];
  // 1/tau_ab = s(node) * K[a][b], K = 1/(m_a m_b D0_ab)
  double K[LBM_MAX_SPECIES][LBM_MAX_SPECIES];
  float Kf[LBM_MAX_SPECIES][LBM_MAX_SPECIES];   // K rounded to FP32 (mixed path)
  double D_T_exp, mu0, mu_T_exp, inv_prandtl;
  // Wilke's mixing rule (wilke = 1): species viscosities at T0 and the
  // T-independent Phi_ab (the species share the T exponent)
  int wilke;
  double mu0_sp[LBM_MAX_SPECIES];
  double wilke_phi[LBM_MAX_SPECIES][LBM_MAX_SPECIES];
  float mu0_sp_s[LBM_MAX_SPECIES];
  float wilke_phi_s[LBM_MAX_SPECIES][LBM_MAX_SPECIES];
  // float-float copies for the mixed path's temperature solve and chemistry
  ff mm_f[LBM_MAX_SPECIES], inv_mm_f[LBM_MAX_SPECIES];
  ff u0_f[LBM_MAX_SPECIES], u1_f[LBM_MAX_SPECIES], u2_f[LBM_MAX_SPECIES], u3_f[LBM_MAX_SPECIES];
  ff g_inv_f[LBM_MAX_SPECIES], g0_f[LBM_MAX_SPECIES], g1_f[LBM_MAX_SPECIES],
      g2_f[LBM_MAX_SPECIES], a0_f[LBM_MAX_SPECIES];
  ff ln_p0_over_ru_f;
  ff eff_f[LBM_MAX_REACTIONS][LBM_MAX_SPECIES];
  // FP32 copies for the mixed path's transport and energy-flux terms
  float inv_mm_s[LBM_MAX_SPECIES], Ra_s[LBM_MAX_SPECIES];
  float D_T_exp_s, mu0_s, mu_T_exp_s, inv_prandtl_s;
};

struct Units {
  double c, inv_c, inv_c2, dx, dt;
  double s_pref;         // R_U^2 dx / (c P0): 1/tau_ab = s_pref rho T^2 (T/T0)^-e K_ab
  double nu_pref;        // 1 / (c dx):  nu_lat = mu / rho * nu_pref
  int substeps;
  int newton_max_iter;
  double newton_rtol;
  // mixed path: float-float and FP32 copies
  ff c2_f, inv_c2_f, dt_sub_f;   // c^2, 1/c^2, dt / substeps
  float newton_rtol_f;           // max(newton_rtol, 4e-13): float-float resolution
  float inv_c2_s, s_pref_s, nu_pref_s;
};

struct Geom {
  int nx, ny, nz;
  long long N;
  // FP16 storage: per population index l*Q + i the codec entry
  // {offset, scale, 1/scale, 0} (nullptr for FP64 / FP32 storage)
  const float4* codec = nullptr;
};

// Kernel launchers (lbm_dispatch.cu).  `S` is the storage type.
// Boundary data of a handle (Sec. 4).  tag == nullptr: periodic box, no
// interface or solid nodes.
constexpr int TAG_BULK = -1;
constexpr int TAG_SOLID = -2;
enum { BK_NONE = 0, BK_BB = 1, BK_TMS = 2, BK_INLET = 3, BK_OUTLET = 4 };

struct BCDev {
  const int* tag = nullptr;        // [N] interface index, TAG_BULK or TAG_SOLID
  const int* if_node = nullptr;    // [n_if] node index of each interface node
  const int* if_info = nullptr;    // kind | outlet axis << 4 | (outlet sign > 0) << 6
  const unsigned* if_inc = nullptr;  // incoming-link mask (bit i = link i)
  const double* if_wallT = nullptr;  // [n_if] TMS target temperature (K)
  const double* if_uin = nullptr;    // [3][n_if] inlet velocity, lattice units
  double* pops = nullptr;            // [L][Q][n_if] reconstructed populations
  // off-grid TMS targets (nullptr: targets at the node): the fluid node x_f
  // of each interface node (-1: none), its normal projection h and the
  // node's normal wall distance delta (lattice units)
  const int* if_nbr = nullptr;
  const double* if_wh = nullptr;
  const double* if_wd = nullptr;
  int n_if = 0;
  int face[6] = {0, 0, 0, 0, 0, 0};
  int has_solid = 0;
  int solid_kind = BK_TMS;
  double rho_in = 0.0, T_in = 0.0, theta_in = 0.0;
  double Y_in[LBM_MAX_SPECIES] = {0};
  double p_out_lat = 0.0, sigma = 0.25;
  double outlet_L = 0.0;          // LODI length (lattice units); 0: the extent
  int inlet_simplified = 0;       // simplified flux inlet (Sec. 4.3)
};

// Kernel placement of a step (lbm_launch, resolved).
struct Launch {
  int chem_lanes = 1;    // 1: chemistry inside the moments kernel; 4 or 8: k_chem lanes per node
  int coll_split = 0;    // 0: fused collision; 1: k_prep + k_coll
  int persistent = 0;    // batched kernels: 1 = grids of the resident blocks, looping over
                         // tiles; 2 = the whole step as one launch over a work-list
  int npt = 1;           // persistent == 2: nodes per thread of the node items (1, 2, 4)
};

struct StepArgs {
  const void* src = nullptr;
  void* dst = nullptr;
  double* rec = nullptr;       // moment records [NF][N]
  double* Tfield = nullptr;    // temperature guess [N]
  int* status = nullptr;
  Geom g;
  Units un;
  BCDev bc;                    // default: periodic box
  Launch lc;                   // default: chemistry and collision one thread per node
  const DevMech* mech_dev = nullptr;   // device copy of the mechanism (k_chem)
  void* cpar = nullptr;        // per-node collision parameters [NF][N] (split collision)
  // optional side stream for the boundary kernel, forked from and joined to
  // the step's stream with these events (all three or none)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// One domain of a batched step (lbm_batch_step): every block of the batched
// grids belongs to exactly one domain (a tile of 128 nodes, or 4 interface
// nodes for the boundary kernel).
struct DomainDev {
  const void* pops[2] = {nullptr, nullptr};   // the handle's two buffers
  int cur0 = 0;                // buffer holding the state at batch parity 0
  void* rec = nullptr;
  double* Tf = nullptr;
  int* status = nullptr;
  Geom g;
  Units un;
  BCDev bc;
  const DevMech* mech = nullptr;   // device copy of the handle's mechanism
  void* cpar = nullptr;        // per-node collision parameters (split collision)
  int block_begin = 0;         // first block of this domain in the node grids
  int bblock_begin = 0;        // first block in the interface-chemistry grid
  int tblock_begin = 0;        // first block in the thread-per-interface-node grid (k_bnode)
  int cblock_begin = 0;        // first block in the chemistry grid (k_chem)
  int kblock_begin = 0;        // first block in the split-collision grid (k_coll)
};

// A side stream with fork / join events (all set, or the step runs on one
// stream).
struct SideStream {
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

// The whole batched step as one launch (Launch::persistent == 2): a
// work-list of items in stage order, claimed by the blocks of a persistent
// grid through an atomic counter.  Stage 1: PI_BND (kPersistBndNodes
// interface nodes: boundary reconstruction, record, reaction sub-steps) and
// PI_MOM (kPersistThreads * npt nodes: moments, sub-steps).  Split
// collision: stage 2, PI_PREP (collision parameters of kPersistThreads * npt
// nodes), after every stage-1 item of its domain; stage 3, PI_COLL
// (kCollNodesPerBlock nodes), after the PI_PREP item holding its nodes.
// Fused collision: stage 2, PI_COLLIDE (the whole collision of
// kPersistThreads * npt nodes, one thread per node), after every stage-1
// item of its domain.  An item waits only on items earlier in the list,
// which blocks already running hold, so every wait ends without any
// assumption on how many blocks are resident.
enum PItemKind : int { PI_BND = 0, PI_MOM = 1, PI_PREP = 2, PI_COLL = 3, PI_COLLIDE = 4 };
struct PItem {
  int kind;     // PItemKind
  int dom;      // domain index
  long long first;   // first interface index (PI_BND) or first node
  int dep;      // PI_PREP, PI_COLLIDE: the domain's stage-1 item count; PI_COLL: the flag
  int flag;     // PI_PREP: the flag it sets
};
constexpr int kPersistThreads = 128;
constexpr int kPersistBndNodes = 128;
// sync words of the work-list: [0] next item, [1] abort, then one stage-1
// completion count per domain, then one flag per PI_PREP item
constexpr int kSyncHead = 2;
// a wait of the persistent step gives up after this long (it sets ST_TIMEOUT)
constexpr long long kPersistTimeoutNs = 4000000000LL;

// Block totals of the batched grids.
struct BatchGrids {
  int nblocks = 0;    // node kernels, 128 nodes per block
  int nbblocks = 0;   // interface-chemistry grid, kIfChemNodesPerBlock nodes per block
  int ntblocks = 0;   // k_bnode, kBndNodesPerBlock interface nodes per block
  int ncblocks = 0;   // k_chem, 128 / chem_lanes nodes per block (0 without it)
  int nkblocks = 0;   // k_coll, 32 nodes per block (0 without it)
  long long n_if_total = 0;   // interface nodes of every domain
  // persistent == 2: the device work-list and its sync words (zeroed before
  // every launch), the domains' interface-node presence
  const PItem* items = nullptr;
  int nitems = 0;
  int* sync = nullptr;
  int nsync = 0;
  int any_if = 0;
  long long timeout_ns = kPersistTimeoutNs;
};

// interface nodes per block of the boundary kernel (one thread each)
constexpr int kBndNodesPerBlock = 64;
// interface nodes per block of the batched interface chemistry (8 lanes each)
constexpr int kIfChemNodesPerBlock = 16;

// Batched step: doms is a device array of ndom domains sharing (D, M, prec)
// and laid out for the placement lc.
cudaError_t launch_batch_step(int D, int M, lbm_precision prec, const DomainDev* doms,
                              int ndom, const BatchGrids& gr, const Launch& lc, int parity,
                              cudaStream_t s, const SideStream& side = SideStream());
// nodes per block of the split-collision kernel k_coll
constexpr int kCollNodesPerBlock = 32;
// fields of the per-node collision parameters (split collision)
int collide_param_fields(int D, int M);
// Set the kernels' attributes (large shared memory) ahead of a stream
// capture, where such calls are not recorded.
cudaError_t prepare_batch_step(int D, int M, lbm_precision prec);

// Per-block partial results of the diagnostics kernel.
struct DiagPart {
  double q_sum;       // sum of q over the block's nodes (W/m^3)
  double q_max;       // largest q
  long long n_max;    // its node (smallest index among equal maxima)
  double T_max, u_max;
};

// Host entry points of one instantiation (lattice, species count, precision)
// of the kernel templates; see lbm_inst.cu.
struct KernelSet {
  cudaError_t (*step)(const DevMech& mech, const StepArgs& a, cudaStream_t s, int which);
  cudaError_t (*batch)(const DomainDev* doms, int ndom, const BatchGrids& gr, const Launch& lc,
                       int parity, cudaStream_t s, const SideStream& side);
  cudaError_t (*prepare)();
  cudaError_t (*init)(const DevMech& mech, const Geom& g, const Units& un,
                      const double* rho_or_P, int is_pressure, const double* u,
                      const double* T, const double* Y, void* pops, double* Tfield,
                      int* status, cudaStream_t s);
  cudaError_t (*out)(const DevMech& mech, const Geom& g, const Units& un, const void* pops,
                     const double* Tfield, double* rho, double* u, double* T, double* Y,
                     double* E, int* status, cudaStream_t s);
  cudaError_t (*diag)(const DevMech& mech, const Geom& g, const Units& un, const void* pops,
                      const double* Tfield, const int* tag, DiagPart* part, int* status,
                      int x0, int x1, cudaStream_t s);
  int record_fields;   // moment-record fields
  int param_fields;    // collision-parameter fields
};
// nullptr for an unsupported combination.  Besides the lbm_precision values,
// prec may be LBM_KPREC_FP32_CHEM64: FP32 storage and lattice arithmetic with
// the temperature solve and the chemistry in native FP64 (cfg->chem_fp64).
constexpr int LBM_KPREC_FP32_CHEM64 = 16;
const KernelSet* kernel_set(int D, int M, lbm_precision prec);
// the kernel-set precision of a configuration
inline lbm_precision kernel_precision(const lbm_config& c) {
  return (c.precision == LBM_FP32_STORE && c.chem_fp64) ? (lbm_precision)LBM_KPREC_FP32_CHEM64
                                                         : c.precision;
}

// which: 0 = moments kernel only, 1 = collision kernel only, -1 = both.
cudaError_t launch_step(int D, int M, lbm_precision prec, const DevMech& mech,
                        const StepArgs& a, cudaStream_t s, int which = -1);
cudaError_t launch_init(int D, int M, lbm_precision prec, const DevMech& mech,
                        const Geom& g, const Units& un, const double* rho_or_P,
                        int is_pressure, const double* u, const double* T,
                        const double* Y, void* pops, double* Tfield, int* status,
                        cudaStream_t s);
cudaError_t launch_moments_out(int D, int M, lbm_precision prec, const DevMech& mech,
                               const Geom& g, const Units& un, const void* pops,
                               const double* Tfield, double* rho, double* u,
                               double* T, double* Y, double* E, int* status,
                               cudaStream_t s);
cudaError_t launch_to_fp64(lbm_precision prec, const void* pops, double* out,
                           long long count, cudaStream_t s, long long N = 1,
                           const float4* codec = nullptr);
// Flame diagnostics over the nodes with x in [x0, x1): per-block partials,
// then their deterministic reduction into out (one DiagPart).
cudaError_t launch_diagnostics(int D, int M, lbm_precision prec, const DevMech& mech,
                               const Geom& g, const Units& un, const void* pops,
                               const double* Tfield, const int* tag, DiagPart* part,
                               DiagPart* out, int* status, int x0, int x1, cudaStream_t s);
// FP16 storage codec (lbm_dispatch.cu)
cudaError_t launch_codec_extent(const float* eq, const float* off, int L, int Q, long long N,
                                unsigned* dev_max, unsigned* abs_max, cudaStream_t s);
cudaError_t launch_codec_encode(const float* eq, void* out, long long count, long long N,
                                const float4* codec, cudaStream_t s);
int record_fields(int D, int M);

// Host helpers defined in lbm_capi.cu.
std::string validate_config(const lbm_config* c);   // "" when valid
void build_device_mechanism(const lbm_mechanism& m, DevMech& d);
void fill_units(const lbm_config& cfg, Units& un);
void fill_mixed_units(Units& un);

}  // namespace lbm
