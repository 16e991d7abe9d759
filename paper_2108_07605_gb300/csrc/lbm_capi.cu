// Host side of the C ABI declared in include/lbm.h: configuration checks,
// mechanism preprocessing, device buffers, launches and error reporting.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "exp64.cuh"
#include "ff.cuh"
#include "lbm_internal.h"

using namespace lbm;

struct lbm_ctx {
  lbm_config cfg;
  int D, Q, M, L, NF;
  Geom g;
  Units un;
  DevMech mech;
  size_t elem;              // bytes per stored population
  void* pops[2] = {nullptr, nullptr};
  int cur = 0;
  double* rec = nullptr;    // moment records (scratch)
  double* Tf = nullptr;     // temperature guess
  int* status = nullptr;    // sticky device status word
  double* io = nullptr;     // staging for host <-> device field copies
  size_t io_bytes = 0;
  BCDev bc;                 // boundary data (device arrays owned by the handle)
  DevMech* mech_dev = nullptr;  // device copy of the mechanism (batched steps)
  void* bc_mem = nullptr;   // one allocation holding every boundary array
  cudaStream_t stream = nullptr;
  size_t bytes = 0;
  long long steps = 0;
  bool initialized = false;
  lbm_launch opt = {-1, -1, -1};  // placement as set (-1: default)
  cudaStream_t side = nullptr;  // boundary kernel, concurrent with the bulk moments
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void* cpar = nullptr;     // per-node collision parameters (split collision)
  float4* codec = nullptr;  // FP16 storage: per-population offset and scale
  std::string err;
};

static thread_local std::string g_create_error;

namespace {

lbm_status fail(lbm_ctx* h, lbm_status st, const std::string& msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return st;
}

lbm_status cuda_fail(lbm_ctx* h, cudaError_t e, const char* where) {
  return fail(h, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Default placement.  The split collision measured faster than the fused
// one on every grid tried (FP32 and FP64, 16k to 524k nodes).  Below
// kSmallGrid nodes a thread-per-node grid holds fewer than four 128-thread
// blocks per SM of a 152-SM GB300, too few warps to hide the latency of the
// float-float chemistry, which then runs with four lanes per node; in FP64
// the extra redundant work of the lanes costs more than it hides.
constexpr long long kSmallGrid = 152LL * 4 * 128;

// Defaults, measured on one GB300.  plan: a batch plan's placement, whose
// default for FP64 storage below kPlanSingleLaunch nodes in total is the
// single launch over the work-list with split collision (14 % faster than
// one launch per kernel on a mix of eight domains of 92k nodes in all; on
// batches of about a million nodes one launch per kernel is 2-6 % faster);
// FP32 and FP16 plans keep one launch per kernel, whose kernels hold fewer
// registers than the single launch.  FP64, a grid that fills the GPU at one
// thread per node: the fused collision (3 % faster on the 600x40x40 tube);
// else the split one.
constexpr long long kPlanSingleLaunch = 4 * kSmallGrid;
Launch resolve_launch(const lbm_launch& opt, long long nodes, lbm_precision prec,
                      bool plan = false) {
  Launch lc;
  const bool small = nodes < kSmallGrid;
  lc.chem_lanes = opt.chem_lanes > 0 ? opt.chem_lanes
                                     : (small && prec == LBM_FP32_STORE ? 4 : 1);
  lc.persistent = opt.persistent >= 0
                      ? opt.persistent
                      : (plan && prec == LBM_FP64 && nodes < kPlanSingleLaunch ? 2 : 0);
  lc.coll_split = opt.collide_split >= 0
                      ? opt.collide_split
                      : (prec == LBM_FP64 && !small && lc.persistent != 2 ? 0 : 1);
  lc.npt = opt.nodes_per_thread > 0 ? opt.nodes_per_thread : 1;
  return lc;
}

// every placement the autotuners try
const Launch kCandidates[] = {{1, 0}, {4, 0}, {8, 0}, {1, 1}, {4, 1}, {8, 1}};

// Domains of a batched step: each handle's tiles follow the previous
// handle's in every grid (128 nodes per node-kernel block, 16 interface nodes
// per interface-chemistry block, 128 / chem_lanes nodes per chemistry block,
// 32 nodes per split-collision block).
void fill_domains(lbm_ctx* const* hs, int n, const Launch& lc, std::vector<DomainDev>& doms,
                  BatchGrids& gr) {
  doms.assign(n, DomainDev());
  gr = BatchGrids();
  for (int k = 0; k < n; ++k) {
    lbm_ctx* h = hs[k];
    DomainDev& d = doms[k];
    d.pops[0] = h->pops[0];
    d.pops[1] = h->pops[1];
    d.cur0 = h->cur;
    d.rec = h->rec;
    d.cpar = h->cpar;
    d.Tf = h->Tf;
    d.status = h->status;
    d.g = h->g;
    d.un = h->un;
    d.bc = h->bc;
    d.mech = h->mech_dev;
    d.block_begin = gr.nblocks;
    d.bblock_begin = gr.nbblocks;
    d.tblock_begin = gr.ntblocks;
    d.cblock_begin = gr.ncblocks;
    d.kblock_begin = gr.nkblocks;
    gr.nblocks += (int)((h->g.N + 127) / 128);
    gr.nbblocks += (h->bc.n_if + kIfChemNodesPerBlock - 1) / kIfChemNodesPerBlock;
    gr.ntblocks += (h->bc.n_if + kBndNodesPerBlock - 1) / kBndNodesPerBlock;
    gr.n_if_total += h->bc.n_if;
    if (lc.chem_lanes > 1) {
      const int per = 128 / lc.chem_lanes;
      gr.ncblocks += (int)((h->g.N + per - 1) / per);
    }
    if (lc.coll_split)
      gr.nkblocks += (int)((h->g.N + kCollNodesPerBlock - 1) / kCollNodesPerBlock);
  }
}

long long total_nodes(lbm_ctx* const* hs, int n) {
  long long t = 0;
  for (int k = 0; k < n; ++k) t += hs[k]->g.N;
  return t;
}

void* dalloc(const lbm_config& c, size_t bytes) {
  if (bytes == 0) return nullptr;
  if (c.dev_alloc) return c.dev_alloc(bytes, c.alloc_user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}

void dfree(const lbm_config& c, void* p) {
  if (!p) return;
  if (c.dev_free) c.dev_free(p, c.alloc_user);
  else cudaFree(p);
}

int lattice_dim(lbm_lattice l) { return l == LBM_D3Q27 ? 3 : 2; }

// component a of velocity i, i = (cz+1)*9 + (cy+1)*3 + (cx+1)
int cvel_host(int i, int a) { return a == 0 ? i % 3 - 1 : (a == 1 ? (i / 3) % 3 - 1 : i / 9 - 1); }

double default_c_ref(const lbm_config& c) {
  double rmax = 0.0;
  for (int a = 0; a < c.mech.n_species; ++a) rmax = std::max(rmax, R_U / c.mech.molar_mass[a]);
  return std::sqrt(rmax * c.T_max / 0.9);
}

// Returns an empty string when cfg is valid.
std::string validate(const lbm_config* c) {
  if (!c) return "config is NULL";
  if (c->lattice != LBM_D3Q27 && c->lattice != LBM_D2Q9) return "unknown lattice";
  if (c->nx < 1 || c->ny < 1 || c->nz < 1) return "grid extents must be >= 1";
  if (c->lattice == LBM_D2Q9 && c->nz != 1) return "D2Q9 needs nz = 1";
  if (c->precision != LBM_FP64 && c->precision != LBM_FP32_STORE &&
      c->precision != LBM_FP16_OFFSET)
    return "precision must be LBM_FP64, LBM_FP32_STORE or LBM_FP16_OFFSET";
  if (c->chem_fp64 != 0 && c->chem_fp64 != 1) return "chem_fp64 must be 0 or 1";
  if (!(c->outlet_length >= 0.0) || !std::isfinite(c->outlet_length))
    return "outlet_length must be >= 0";
  if ((c->wall_dist == nullptr) != (c->wall_normal == nullptr))
    return "wall_dist and wall_normal go together";
  if (c->chem_fp64 && c->precision == LBM_FP16_OFFSET)
    return "chem_fp64 is supported with LBM_FP32_STORE (and implied by LBM_FP64)";
  if (c->substeps < 1 || c->substeps > 64) return "substeps must be in 1..64";
  if (!(c->dx > 0.0) || !std::isfinite(c->dx)) return "dx must be positive";
  if (c->c_ref < 0.0 || !std::isfinite(c->c_ref)) return "c_ref must be >= 0";
  if (c->c_ref == 0.0 && !(c->T_max > 0.0)) return "T_max must be positive when c_ref = 0";
  const lbm_mechanism& m = c->mech;
  if (m.n_species != 2 && m.n_species != 9)
    return "n_species must be 2 or 9 (the species counts the library is compiled for)";
  if (m.n_reactions < 0 || m.n_reactions > LBM_MAX_REACTIONS) return "n_reactions out of range";
  for (int a = 0; a < m.n_species; ++a) {
    if (!(m.molar_mass[a] > 0.0)) return "molar masses must be positive";
    for (int b = 0; b < m.n_species; ++b)
      if (a != b && !(m.D0[a][b] > 0.0)) return "D0 must be positive off the diagonal";
  }
  for (int r = 0; r < m.n_reactions; ++r) {
    int nr = 0, np = 0;
    for (int a = 0; a < m.n_species; ++a) {
      if (m.nu_f[r][a] < 0 || m.nu_r[r][a] < 0) return "stoichiometric coefficients must be >= 0";
      nr += m.nu_f[r][a];
      np += m.nu_r[r][a];
    }
    if (nr < 1 || nr > 3 || np < 1 || np > 3) return "reactions need 1..3 molecules per side";
    if (!(m.arrhenius[r][0] > 0.0)) return "Arrhenius A must be positive";
  }
  if (!(m.mu0 > 0.0) || !(m.prandtl > 0.0)) return "mu0 and prandtl must be positive";
  if (m.viscosity_model != 0 && m.viscosity_model != 1) return "viscosity_model must be 0 or 1";
  if (m.viscosity_model == 1)
    for (int a = 0; a < m.n_species; ++a)
      if (!(m.mu0_species[a] > 0.0)) return "Wilke viscosity needs positive mu0_species";
  bool any_tms = c->solid_mask && c->solid_bc == LBM_TMS_WALL, any_in = false, any_out = false;
  for (int f = 0; f < 6; ++f) {
    const lbm_bc k = c->face_bc[f];
    if (k < LBM_PERIODIC || k > LBM_OUTLET) return "unknown face boundary kind";
    if (c->lattice == LBM_D2Q9 && f >= 4 && k != LBM_PERIODIC)
      return "D2Q9 needs periodic z faces";
    if (k == LBM_TMS_WALL) {
      any_tms = true;
      if (!c->wall_T_nodes && !(c->wall_T[f] > 0.0)) return "TMS face needs wall_T";
    }
    any_in |= k == LBM_INLET;
    any_out |= k == LBM_OUTLET;
  }
  if (c->solid_mask && c->solid_bc != LBM_BOUNCE_BACK && c->solid_bc != LBM_TMS_WALL)
    return "solid_bc must be LBM_BOUNCE_BACK or LBM_TMS_WALL";
  if (c->solid_mask && c->solid_bc == LBM_TMS_WALL && !c->wall_T_nodes)
    return "TMS solid walls need wall_T_nodes";
  if (any_tms && c->wall_T_nodes)
    for (long long n = 0; n < (long long)c->nx * c->ny * c->nz; ++n)
      if (!(c->wall_T_nodes[n] > 0.0)) return "wall_T_nodes must be positive";
  if (any_in) {
    if (!(c->inlet_T > 0.0) || !(c->inlet_P > 0.0)) return "inlet needs inlet_T and inlet_P";
    double ys = 0.0;
    for (int a = 0; a < m.n_species; ++a) {
      if (c->inlet_Y[a] < 0.0) return "inlet_Y must be >= 0";
      ys += c->inlet_Y[a];
    }
    if (std::fabs(ys - 1.0) > 1e-9) return "inlet_Y must sum to 1";
  }
  if (any_out && !(c->outlet_P > 0.0 && c->outlet_sigma >= 0.0))
    return "outlet needs outlet_P > 0 and outlet_sigma >= 0";
  if (c->newton_max_iter < 1 || !(c->newton_rtol >= 0.0)) return "bad Newton parameters";
  if (c->device < 0) return "device must be >= 0";
  return "";
}

void build_mech(const lbm_mechanism& m, DevMech& d) {
  std::memset(&d, 0, sizeof(d));
  d.M = m.n_species;
  d.R = m.n_reactions;
  const double T0 = T_REF;
  for (int a = 0; a < m.n_species; ++a) {
    const double mm = m.molar_mass[a];
    const double a0 = m.cp[a][0], a1 = m.cp[a][1], a2 = m.cp[a][2];
    d.mm[a] = mm;
    d.inv_mm[a] = 1.0 / mm;
    d.Ra[a] = R_U / mm;
    const double poly0 = a0 * T0 + 0.5 * a1 * T0 * T0 + a2 / 3.0 * T0 * T0 * T0;
    d.u0[a] = (m.h_formation[a] - R_U * poly0) / mm;
    d.u1[a] = d.Ra[a] * (a0 - 1.0);
    d.u2[a] = d.Ra[a] * 0.5 * a1;
    d.u3[a] = d.Ra[a] * a2 / 3.0;
    d.g_inv[a] = m.h_formation[a] / R_U - poly0;
    d.g0[a] = a0 - m.s_standard[a] / R_U + a0 * std::log(T0) + a1 * T0 + 0.5 * a2 * T0 * T0;
    d.g1[a] = -0.5 * a1;
    d.g2[a] = -a2 / 6.0;
    d.a0[a] = a0;
    for (int b = 0; b < m.n_species; ++b) {
      d.K[a][b] = a == b ? 0.0 : 1.0 / (mm * m.molar_mass[b] * m.D0[a][b]);
      d.Kf[a][b] = (float)d.K[a][b];
    }
  }
  d.ln_p0_over_ru = std::log(P_REF / R_U);
  for (int r = 0; r < m.n_reactions; ++r) {
    DevReaction& x = d.rx[r];
    x.nr = x.np = 0;
    x.dn = 0;
    for (int a = 0; a < m.n_species; ++a) {
      for (int k = 0; k < m.nu_f[r][a]; ++k) x.reac[x.nr++] = a;
      for (int k = 0; k < m.nu_r[r][a]; ++k) x.prod[x.np++] = a;
      x.dn += m.nu_r[r][a] - m.nu_f[r][a];
      d.eff[r][a] = m.efficiency[r][a];
    }
    x.reversible = m.reversible[r] ? 1 : 0;
    x.third_body = m.third_body[r] ? 1 : 0;
    x.lnA = std::log(m.arrhenius[r][0]);
    x.b = m.arrhenius[r][1];
    x.EaR = m.arrhenius[r][2] / R_U;
    x.lnA_f = ff_host(x.lnA);
    x.b_f = ff_host(x.b);
    x.EaR_f = ff_host(x.EaR);
    for (int a = 0; a < m.n_species; ++a) d.eff_f[r][a] = ff_host(m.efficiency[r][a]);
  }
  d.D_T_exp = m.D_T_exponent;
  d.mu0 = m.mu0;
  d.mu_T_exp = m.mu_T_exponent;
  d.inv_prandtl = 1.0 / m.prandtl;
  for (int a = 0; a < m.n_species; ++a) {
    d.mm_f[a] = ff_host(d.mm[a]);
    d.inv_mm_f[a] = ff_host(d.inv_mm[a]);
    d.u0_f[a] = ff_host(d.u0[a]);
    d.u1_f[a] = ff_host(d.u1[a]);
    d.u2_f[a] = ff_host(d.u2[a]);
    d.u3_f[a] = ff_host(d.u3[a]);
    d.g_inv_f[a] = ff_host(d.g_inv[a]);
    d.g0_f[a] = ff_host(d.g0[a]);
    d.g1_f[a] = ff_host(d.g1[a]);
    d.g2_f[a] = ff_host(d.g2[a]);
    d.a0_f[a] = ff_host(d.a0[a]);
    d.inv_mm_s[a] = (float)d.inv_mm[a];
    d.Ra_s[a] = (float)d.Ra[a];
  }
  d.ln_p0_over_ru_f = ff_host(d.ln_p0_over_ru);
  d.D_T_exp_s = (float)d.D_T_exp;
  d.mu0_s = (float)d.mu0;
  d.mu_T_exp_s = (float)d.mu_T_exp;
  d.inv_prandtl_s = (float)d.inv_prandtl;
  d.wilke = m.viscosity_model == 1 ? 1 : 0;
  for (int a = 0; a < m.n_species; ++a) {
    d.mu0_sp[a] = d.wilke ? m.mu0_species[a] : m.mu0;
    d.mu0_sp_s[a] = (float)d.mu0_sp[a];
  }
  for (int a = 0; a < m.n_species; ++a)
    for (int b = 0; b < m.n_species; ++b) {
      // Wilke's Phi_ab: the species viscosities share the T exponent, so the
      // ratio mu_a/mu_b, and Phi, are the same at every T
      const double ma = m.molar_mass[a], mb = m.molar_mass[b];
      const double r = std::sqrt(d.mu0_sp[a] / d.mu0_sp[b]) * std::pow(mb / ma, 0.25);
      d.wilke_phi[a][b] = (1.0 + r) * (1.0 + r) / std::sqrt(8.0 * (1.0 + ma / mb));
      d.wilke_phi_s[a][b] = (float)d.wilke_phi[a][b];
    }
}

// bytes of a stored population, and of the scratch records' lattice type
size_t elem_size(lbm_precision p) { return p == LBM_FP64 ? 8 : (p == LBM_FP16_OFFSET ? 2 : 4); }
size_t compute_size(lbm_precision p) { return p == LBM_FP64 ? 8 : 4; }

// Interface-node classification (Sec. 4.1): a link i of node x is incoming
// when x - c_i lies beyond a non-periodic face or on a solid node; the node's
// procedure is the one of its incoming links with the highest precedence
// (walls, then inlet, then outlet; the first such link in index order).
struct HostBC {
  bool needed = false, has_solid = false;
  int n_if = 0;
  std::vector<int> tag, if_node, if_info;
  std::vector<unsigned> if_inc;
  std::vector<double> wallT, uin;   // uin [3][n_if], lattice units
  bool offgrid = false;             // off-grid TMS targets (wall_dist, wall_normal)
  std::vector<int> og_nbr;          // [n_if] fluid node x_f, -1: none
  std::vector<double> og_h, og_d;   // [n_if] normal projection of c_k, wall distance
};

int precedence(int k) {
  return (k == BK_BB || k == BK_TMS) ? 3 : (k == BK_INLET ? 2 : (k == BK_OUTLET ? 1 : 0));
}

HostBC classify(const lbm_config& c, double c_ref) {
  HostBC h;
  const int D = lattice_dim(c.lattice);
  const int Q = D == 3 ? 27 : 9;
  const int ext[3] = {c.nx, c.ny, c.nz};
  const long long N = (long long)c.nx * c.ny * c.nz;
  h.has_solid = c.solid_mask != nullptr;
  h.needed = h.has_solid;
  for (int f = 0; f < 6; ++f) h.needed |= c.face_bc[f] != LBM_PERIODIC;
  if (!h.needed) return h;
  h.tag.assign(N, TAG_BULK);
  for (long long n = 0; n < N; ++n) {
    if (h.has_solid && c.solid_mask[n]) { h.tag[n] = TAG_SOLID; continue; }
    const int co[3] = {(int)(n % c.nx), (int)((n / c.nx) % c.ny), (int)(n / ((long long)c.nx * c.ny))};
    int nk = 0, ax = 0, sg = 0, tms_face = -1;
    unsigned inc = 0;
    for (int i = 0; i < Q; ++i) {
      int lk = 0, src[3] = {co[0], co[1], co[2]};
      for (int a = 0; a < D; ++a) {
        int sa = co[a] - cvel_host(i, a);
        int face = -1;
        if (sa < 0) { face = 2 * a; sa += ext[a]; }
        else if (sa >= ext[a]) { face = 2 * a + 1; sa -= ext[a]; }
        src[a] = sa;
        if (face < 0) continue;
        const int fk = c.face_bc[face];
        if (fk == LBM_PERIODIC) continue;
        if (precedence(fk) > precedence(lk)) lk = fk;
        if (fk == LBM_OUTLET) { ax = a; sg = (face & 1) ? 1 : -1; }
        if (fk == LBM_TMS_WALL && tms_face < 0) tms_face = face;
      }
      if (lk == 0 && h.has_solid &&
          c.solid_mask[src[0] + (long long)c.nx * (src[1] + (long long)c.ny * src[2])])
        lk = c.solid_bc;
      if (lk) {
        inc |= 1u << i;
        if (precedence(lk) > precedence(nk)) nk = lk;
      }
    }
    if (!nk) continue;
    h.tag[n] = h.n_if++;
    h.if_node.push_back((int)n);
    h.if_info.push_back(nk | (ax << 4) | ((sg > 0) << 6));
    h.if_inc.push_back(inc);
    h.wallT.push_back(c.wall_T_nodes ? c.wall_T_nodes[n] : (tms_face >= 0 ? c.wall_T[tms_face] : 0.0));
  }
  h.uin.assign(3 * (size_t)h.n_if, 0.0);
  for (int k = 0; k < h.n_if; ++k)
    for (int d = 0; d < 3; ++d)
      h.uin[(size_t)d * h.n_if + k] =
          (c.inlet_u ? c.inlet_u[(long long)d * N + h.if_node[k]] : c.inlet_u_uniform[d]) / c_ref;
  // off-grid TMS targets (Sec. 4.2.2, last paragraph): per TMS node the
  // fluid node x + c_k whose direction is most aligned with the inward
  // normal (first such direction in index order), its projection on the
  // normal and the node's wall distance
  h.offgrid = c.wall_dist && c.wall_normal;
  if (h.offgrid) {
    h.og_nbr.assign(h.n_if, -1);
    h.og_h.assign(h.n_if, 0.0);
    h.og_d.assign(h.n_if, 0.0);
    for (int k = 0; k < h.n_if; ++k) {
      if ((h.if_info[k] & 15) != BK_TMS) continue;
      const long long n = h.if_node[k];
      double nrm[3] = {0.0, 0.0, 0.0};
      for (int d = 0; d < D; ++d) nrm[d] = c.wall_normal[(long long)d * N + n];
      int best = -1;
      double bval = 0.0;
      for (int i = 0; i < Q; ++i) {
        double cc = 0.0, dot = 0.0;
        for (int d = 0; d < D; ++d) cc += cvel_host(i, d) * cvel_host(i, d);
        if (cc == 0.0) continue;
        const double inv = 1.0 / std::sqrt(cc);
        for (int d = 0; d < D; ++d) dot += (cvel_host(i, d) * inv) * nrm[d];
        if (best < 0 || dot > bval) { best = i; bval = dot; }
      }
      const int co[3] = {(int)(n % c.nx), (int)((n / c.nx) % c.ny),
                         (int)(n / ((long long)c.nx * c.ny))};
      int xf[3] = {co[0], co[1], co[2]};
      bool ok = true;
      double hproj = 0.0;
      for (int d = 0; d < D; ++d) {
        int v = co[d] + cvel_host(best, d);
        if (v < 0 || v >= ext[d]) {
          if (c.face_bc[2 * d + (v >= ext[d] ? 1 : 0)] != LBM_PERIODIC) ok = false;
          v = (v + ext[d]) % ext[d];
        }
        xf[d] = v;
        hproj += cvel_host(best, d) * nrm[d];
      }
      const long long nf = xf[0] + (long long)c.nx * (xf[1] + (long long)c.ny * xf[2]);
      if (!ok || (h.has_solid && c.solid_mask[nf])) continue;
      h.og_nbr[k] = (int)nf;
      h.og_h[k] = hproj;
      h.og_d[k] = c.wall_dist[n];
    }
  }
  return h;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

struct Sizes {
  size_t pops, rec, cpar, codec, tf, status, io, bc, total;
};

Sizes sizes_for(const lbm_config& c, const HostBC& hb) {
  const int D = lattice_dim(c.lattice);
  const int Q = D == 3 ? 27 : 9;
  const int M = c.mech.n_species;
  const long long N = (long long)c.nx * c.ny * c.nz;
  Sizes s;
  s.pops = (size_t)(M + 1) * Q * N * elem_size(c.precision);
  s.rec = (size_t)record_fields(D, M) * N * compute_size(c.precision);
  s.cpar = (size_t)collide_param_fields(D, M) * N * compute_size(c.precision);
  s.codec = c.precision == LBM_FP16_OFFSET ? (size_t)(M + 1) * Q * sizeof(float4) : 0;
  s.tf = (size_t)N * sizeof(double);
  s.status = 256;
  s.io = 0;
  s.bc = 0;
  if (hb.needed) {
    const size_t nif = (size_t)hb.n_if;
    s.bc = align256(N * sizeof(int)) + 3 * align256(nif * sizeof(int)) +
           4 * align256(nif * sizeof(double)) + align256((size_t)(M + 1) * Q * nif * sizeof(double));
    if (hb.offgrid) s.bc += align256(nif * sizeof(int)) + 2 * align256(nif * sizeof(double));
  }
  s.total = 2 * s.pops + s.rec + s.cpar + s.codec + s.tf + s.status + s.bc;
  return s;
}

lbm_status check_status(lbm_ctx* h) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "status read");
  if (st & ST_NEWTON) return fail(h, LBM_ERR_NEWTON, "temperature Newton did not converge");
  if (st & ST_NONFINITE) return fail(h, LBM_ERR_NONFINITE, "non-finite or non-positive density or temperature");
  if (st & ST_RANGE) return fail(h, LBM_ERR_RANGE, "value out of range");
  if (st & ST_TIMEOUT) return fail(h, LBM_ERR_TIMEOUT, "a bounded device wait gave up");
  return LBM_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    cudaGetDevice(&now);
    if (prev >= 0 && now != prev) cudaSetDevice(prev);
  }
};

lbm_status ensure_io(lbm_ctx* h, size_t bytes) {
  if (h->io_bytes >= bytes) return LBM_OK;
  if (h->io) {
    cudaStreamSynchronize(h->stream);
    dfree(h->cfg, h->io);
    h->bytes -= h->io_bytes;
    h->io = nullptr;
    h->io_bytes = 0;
  }
  h->io = static_cast<double*>(dalloc(h->cfg, bytes));
  if (!h->io) return fail(h, LBM_ERR_OOM, "staging buffer allocation failed");
  h->io_bytes = bytes;
  h->bytes += bytes;
  return LBM_OK;
}

// FP16 offset storage (reading R19): offsets o_li = the equilibrium
// populations of the mean initial state at rest; per lattice a scale that
// maps 16x the largest initial deviation |f^eq - o| to the FP16 maximum, and
// at least (rho_ref / 27) 2^-12 for species and f, (max |g|) 2^-12 for g, so
// that later growth (trace species forming, the flow speeding up) stays in
// range.  Then the initial equilibria are encoded.
lbm_status init_fp16(lbm_ctx* h, const double* drho, int is_pressure, const double* du,
                     const double* dT, const double* dY) {
  const long long N = h->g.N;
  const int M = h->M, L = h->L, Q = h->Q, LQ = L * Q;
  // mean fields (host)
  std::vector<double> rp(N), T(N), Y((size_t)M * N);
  cudaError_t e = cudaMemcpyAsync(rp.data(), drho, N * sizeof(double), cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(T.data(), dT, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Y.data(), dY, (size_t)M * N * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "FP16 codec: field download");
  std::vector<double> mean(1 + 3 + 1 + M, 0.0);   // rho or P, u (0), T, Y
  for (long long n = 0; n < N; ++n) {
    mean[0] += rp[n];
    mean[4] += T[n];
    for (int a = 0; a < M; ++a) mean[5 + a] += Y[(size_t)a * N + n];
  }
  mean[0] /= N;
  mean[4] /= N;
  for (int a = 0; a < M; ++a) mean[5 + a] /= N;
  // scratch: mean state (1 node), offsets, FP32 equilibria, extents
  const size_t b_mean = mean.size() * sizeof(double), b_off = LQ * sizeof(float),
               b_eq = (size_t)LQ * N * sizeof(float), b_ext = 2 * L * sizeof(unsigned);
  char* tmp = static_cast<char*>(dalloc(h->cfg, b_mean + b_off + b_eq + b_ext + 256 * 4));
  if (!tmp) return fail(h, LBM_ERR_OOM, "FP16 codec: scratch allocation failed");
  double* dmean = reinterpret_cast<double*>(tmp);
  float* off = reinterpret_cast<float*>(tmp + align256(b_mean));
  float* eq = reinterpret_cast<float*>(tmp + align256(b_mean) + align256(b_off));
  unsigned* ext = reinterpret_cast<unsigned*>(tmp + align256(b_mean) + align256(b_off) +
                                              align256(b_eq));
  double* Tdummy = dmean + 4;   // the 1-node init writes its temperature here (unused)
  Geom g1;
  g1.nx = g1.ny = g1.nz = 1;
  g1.N = 1;
  Geom gq = h->g;
  gq.codec = nullptr;
  e = cudaMemcpyAsync(dmean, mean.data(), b_mean, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = launch_init(h->D, M, LBM_FP32_STORE, h->mech, g1, h->un, dmean, is_pressure, dmean + 1,
                    dmean + 4, dmean + 5, off, Tdummy, h->status, h->stream);
  if (e == cudaSuccess)
    e = launch_init(h->D, M, LBM_FP32_STORE, h->mech, gq, h->un, drho, is_pressure, du, dT, dY,
                    eq, h->Tf, h->status, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ext, 0, b_ext, h->stream);
  if (e == cudaSuccess) e = launch_codec_extent(eq, off, L, Q, N, ext, ext + L, h->stream);
  std::vector<float> hoff(LQ);
  std::vector<unsigned> hext(2 * L);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hoff.data(), off, b_off, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hext.data(), ext, b_ext, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    dfree(h->cfg, tmp);
    return cuda_fail(h, e, "FP16 codec");
  }
  double rho_ref = 0.0;
  for (int i = 0; i < Q; ++i) rho_ref += hoff[(M - 1) * Q + i];
  std::vector<float4> table(LQ);
  for (int l = 0; l < L; ++l) {
    float dev, amax;
    std::memcpy(&dev, &hext[l], sizeof(float));
    std::memcpy(&amax, &hext[L + l], sizeof(float));
    const double floor_s = l < M ? rho_ref / 27.0 * 0x1p-12 : amax * 0x1p-12;
    double sc = std::max(16.0 * dev / 65504.0, floor_s);
    if (!(sc > 0.0) || !std::isfinite(sc)) sc = 1.0;
    for (int i = 0; i < Q; ++i)
      table[l * Q + i] = make_float4(hoff[l * Q + i], (float)sc, (float)(1.0 / sc), 0.f);
  }
  e = cudaMemcpyAsync(h->codec, table.data(), LQ * sizeof(float4), cudaMemcpyHostToDevice,
                      h->stream);
  if (e == cudaSuccess)
    e = launch_codec_encode(eq, h->pops[h->cur], (long long)LQ * N, N, h->codec, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // table and scratch in use
  dfree(h->cfg, tmp);
  if (e != cudaSuccess) return cuda_fail(h, e, "FP16 encode");
  return LBM_OK;
}

lbm_status init_common(lbm_ctx* h, const double* rho_or_P, int is_pressure, const double* u,
                       const double* T, const double* Y, int on_device) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID, "handle is NULL");
  if (!rho_or_P || !u || !T || !Y) return fail(h, LBM_ERR_INVALID, "field pointer is NULL");
  DeviceGuard dg(h->cfg.device);
  const long long N = h->g.N;
  const int M = h->M;
  const double *drho = rho_or_P, *du = u, *dT = T, *dY = Y;
  if (!on_device) {
    const size_t need = (size_t)(1 + 3 + 1 + M) * N * sizeof(double);
    lbm_status st = ensure_io(h, need);
    if (st != LBM_OK) return st;
    double* p = h->io;
    const size_t nb = N * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(p, rho_or_P, nb, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + N, u, 3 * nb, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + 4 * N, T, nb, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + 5 * N, Y, M * nb, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "field upload");
    drho = p; du = p + N; dT = p + 4 * N; dY = p + 5 * N;
  }
  cudaError_t e = cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "status reset");
  if (h->cfg.precision == LBM_FP16_OFFSET) {
    const lbm_status st = init_fp16(h, drho, is_pressure, du, dT, dY);
    if (st != LBM_OK) return st;
  } else {
    e = launch_init(h->D, M, kernel_precision(h->cfg), h->mech, h->g, h->un, drho, is_pressure, du, dT,
                    dY, h->pops[h->cur], h->Tf, h->status, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "init kernel");
  }
  // Both buffers start equal: the kernels never write solid nodes, which
  // keep their initial (equilibrium) populations in either buffer.
  e = cudaMemcpyAsync(h->pops[1 - h->cur], h->pops[h->cur],
                      (size_t)h->L * h->Q * N * h->elem, cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "buffer copy");
  h->initialized = true;
  h->steps = 0;
  if (!on_device) return check_status(h);
  return LBM_OK;
}

}  // namespace

namespace lbm {
void fill_mixed_units(Units& un) {
  un.c2_f = ff_host(un.c * un.c);
  un.inv_c2_f = ff_host(un.inv_c2);
  un.dt_sub_f = ff_host(un.dt / un.substeps);
  un.newton_rtol_f = (float)std::max(un.newton_rtol, 4e-13);
  un.inv_c2_s = (float)un.inv_c2;
  un.s_pref_s = (float)un.s_pref;
  un.nu_pref_s = (float)un.nu_pref;
}
// Host helpers shared with the allocation-free entry point (lbm_noalloc.cu).
std::string validate_config(const lbm_config* c) { return validate(c); }
void build_device_mechanism(const lbm_mechanism& m, DevMech& d) { build_mech(m, d); }
void fill_units(const lbm_config& cfg, Units& un) {
  const double c = cfg.c_ref > 0.0 ? cfg.c_ref : default_c_ref(cfg);
  un.c = c;
  un.inv_c = 1.0 / c;
  un.inv_c2 = 1.0 / (c * c);
  un.dx = cfg.dx;
  un.dt = cfg.dx / c;
  un.s_pref = R_U * R_U * cfg.dx / (c * P_REF);
  un.nu_pref = 1.0 / (c * cfg.dx);
  un.substeps = cfg.substeps;
  un.newton_max_iter = cfg.newton_max_iter;
  un.newton_rtol = cfg.newton_rtol;
  fill_mixed_units(un);
}
}  // namespace lbm

namespace {

// The work-list of the single-launch step (PItem): stage 1 (the boundary
// items of every domain, then the moments items), stage 2 (parameter items),
// stage 3 (collision items), each stage domain by domain.  nsync: the sync
// words the launch needs.
void build_worklist(const long long* nodes, const long long* nif, int n, int npt, bool split,
                    std::vector<PItem>& items, int& nsync) {
  items.clear();
  const long long tile = (long long)kPersistThreads * npt;
  std::vector<int> n1(n, 0), pbase(n, 0);
  for (int k = 0; k < n; ++k)
    for (long long f = 0; f < nif[k]; f += kPersistBndNodes, ++n1[k])
      items.push_back(PItem{PI_BND, k, f, 0, 0});
  for (int k = 0; k < n; ++k)
    for (long long f = 0; f < nodes[k]; f += tile, ++n1[k])
      items.push_back(PItem{PI_MOM, k, f, 0, 0});
  int nflag = 0;
  if (!split) {
    for (int k = 0; k < n; ++k)
      for (long long f = 0; f < nodes[k]; f += tile)
        items.push_back(PItem{PI_COLLIDE, k, f, n1[k], 0});
    nsync = kSyncHead + n;
    return;
  }
  for (int k = 0; k < n; ++k) {
    pbase[k] = nflag;
    for (long long f = 0; f < nodes[k]; f += tile)
      items.push_back(PItem{PI_PREP, k, f, n1[k], nflag++});
  }
  for (int k = 0; k < n; ++k)
    for (long long f = 0; f < nodes[k]; f += kCollNodesPerBlock)
      items.push_back(PItem{PI_COLL, k, f, pbase[k] + (int)(f / tile), 0});
  nsync = kSyncHead + n + nflag;
}

void build_worklist(lbm_ctx* const* hs, int n, int npt, bool split, std::vector<PItem>& items,
                    int& nsync) {
  std::vector<long long> nodes(n), nif(n);
  for (int k = 0; k < n; ++k) {
    nodes[k] = hs[k]->g.N;
    nif[k] = hs[k]->bc.n_if;
  }
  build_worklist(nodes.data(), nif.data(), n, npt, split, items, nsync);
}

}  // namespace

extern "C" {

void lbm_config_defaults(lbm_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->lattice = LBM_D3Q27;
  cfg->nx = cfg->ny = cfg->nz = 1;
  cfg->precision = LBM_FP64;
  cfg->substeps = 2;
  cfg->dx = 1e-3;
  cfg->c_ref = 0.0;
  cfg->T_max = 3000.0;
  for (int f = 0; f < 6; ++f) cfg->face_bc[f] = LBM_PERIODIC;
  cfg->outlet_sigma = 0.25;
  cfg->solid_bc = LBM_TMS_WALL;
  cfg->outlet_P = P_REF;
  cfg->inlet_P = P_REF;
  cfg->newton_max_iter = 50;
  cfg->newton_rtol = 1e-13;
}

size_t lbm_bytes_required(const lbm_config* cfg) {
  if (!validate(cfg).empty()) return 0;
  const double c = cfg->c_ref > 0.0 ? cfg->c_ref : default_c_ref(*cfg);
  return sizes_for(*cfg, classify(*cfg, c)).total;
}

lbm_status lbm_create(const lbm_config* cfg, lbm_t* out) {
  if (!out) return fail(nullptr, LBM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  const std::string why = validate(cfg);
  if (!why.empty()) return fail(nullptr, LBM_ERR_INVALID, why);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device >= ndev)
    return fail(nullptr, LBM_ERR_CUDA, "no CUDA device with that ordinal");
  DeviceGuard dg(cfg->device);
  lbm_ctx* h = new lbm_ctx();
  h->cfg = *cfg;
  h->cfg.inlet_u = nullptr;   // not retained
  h->D = lattice_dim(cfg->lattice);
  h->Q = h->D == 3 ? 27 : 9;
  h->M = cfg->mech.n_species;
  h->L = h->M + 1;
  h->NF = record_fields(h->D, h->M);
  h->g.nx = cfg->nx; h->g.ny = cfg->ny; h->g.nz = cfg->nz;
  h->g.N = (long long)cfg->nx * cfg->ny * cfg->nz;
  const double c = cfg->c_ref > 0.0 ? cfg->c_ref : default_c_ref(*cfg);
  h->un.c = c;
  h->un.inv_c = 1.0 / c;
  h->un.inv_c2 = 1.0 / (c * c);
  h->un.dx = cfg->dx;
  h->un.dt = cfg->dx / c;
  h->un.s_pref = R_U * R_U * cfg->dx / (c * P_REF);
  h->un.nu_pref = 1.0 / (c * cfg->dx);
  h->un.substeps = cfg->substeps;
  h->un.newton_max_iter = cfg->newton_max_iter;
  h->un.newton_rtol = cfg->newton_rtol;
  fill_mixed_units(h->un);
  build_mech(cfg->mech, h->mech);
  h->elem = elem_size(cfg->precision);
  h->stream = static_cast<cudaStream_t>(cfg->stream);
  const HostBC hb = classify(*cfg, c);
  const Sizes s = sizes_for(*cfg, hb);
  h->pops[0] = dalloc(h->cfg, s.pops);
  h->pops[1] = dalloc(h->cfg, s.pops);
  h->rec = static_cast<double*>(dalloc(h->cfg, s.rec));
  h->cpar = dalloc(h->cfg, s.cpar);
  if (s.codec) {
    h->codec = static_cast<float4*>(dalloc(h->cfg, s.codec));
    h->g.codec = h->codec;
  }
  h->Tf = static_cast<double*>(dalloc(h->cfg, s.tf));
  h->status = static_cast<int*>(dalloc(h->cfg, s.status));
  h->bytes = s.total;
  h->mech_dev = static_cast<DevMech*>(dalloc(h->cfg, sizeof(DevMech)));
  if (!h->mech_dev) {
    lbm_destroy(h);
    return fail(nullptr, LBM_ERR_OOM, "device allocation failed (mechanism)");
  }
  if (cudaMemcpy(h->mech_dev, &h->mech, sizeof(DevMech), cudaMemcpyHostToDevice) != cudaSuccess) {
    lbm_destroy(h);
    return fail(nullptr, LBM_ERR_CUDA, "mechanism upload failed");
  }
  h->bytes += sizeof(DevMech);
  if (hb.n_if > 0) {
    cudaError_t e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      lbm_destroy(h);
      return fail(nullptr, LBM_ERR_CUDA, std::string("side stream: ") + cudaGetErrorString(e));
    }
  }
  if (hb.needed) {
    h->bc_mem = dalloc(h->cfg, s.bc);
    if (!h->bc_mem) {
      lbm_destroy(h);
      return fail(nullptr, LBM_ERR_OOM, "device allocation failed (boundary data)");
    }
    char* p = static_cast<char*>(h->bc_mem);
    const size_t nif = (size_t)hb.n_if;
    const long long N = h->g.N;
    BCDev& b = h->bc;
    auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
    int* tag = reinterpret_cast<int*>(take(N * sizeof(int)));
    int* if_node = reinterpret_cast<int*>(take(nif * sizeof(int)));
    int* if_info = reinterpret_cast<int*>(take(nif * sizeof(int)));
    unsigned* if_inc = reinterpret_cast<unsigned*>(take(nif * sizeof(unsigned)));
    double* wallT = reinterpret_cast<double*>(take(nif * sizeof(double)));
    double* uin = reinterpret_cast<double*>(take(3 * nif * sizeof(double)));
    b.pops = reinterpret_cast<double*>(take((size_t)h->L * h->Q * nif * sizeof(double)));
    cudaError_t e = cudaMemcpy(tag, hb.tag.data(), N * sizeof(int), cudaMemcpyHostToDevice);
    if (hb.offgrid) {
      int* nbr = reinterpret_cast<int*>(take(nif * sizeof(int)));
      double* wh = reinterpret_cast<double*>(take(nif * sizeof(double)));
      double* wd = reinterpret_cast<double*>(take(nif * sizeof(double)));
      if (nif && e == cudaSuccess)
        e = cudaMemcpy(nbr, hb.og_nbr.data(), nif * sizeof(int), cudaMemcpyHostToDevice);
      if (nif && e == cudaSuccess)
        e = cudaMemcpy(wh, hb.og_h.data(), nif * sizeof(double), cudaMemcpyHostToDevice);
      if (nif && e == cudaSuccess)
        e = cudaMemcpy(wd, hb.og_d.data(), nif * sizeof(double), cudaMemcpyHostToDevice);
      b.if_nbr = nbr;
      b.if_wh = wh;
      b.if_wd = wd;
    }
    if (nif && e == cudaSuccess)
      e = cudaMemcpy(if_node, hb.if_node.data(), nif * sizeof(int), cudaMemcpyHostToDevice);
    if (nif && e == cudaSuccess)
      e = cudaMemcpy(if_info, hb.if_info.data(), nif * sizeof(int), cudaMemcpyHostToDevice);
    if (nif && e == cudaSuccess)
      e = cudaMemcpy(if_inc, hb.if_inc.data(), nif * sizeof(unsigned), cudaMemcpyHostToDevice);
    if (nif && e == cudaSuccess)
      e = cudaMemcpy(wallT, hb.wallT.data(), nif * sizeof(double), cudaMemcpyHostToDevice);
    if (nif && e == cudaSuccess)
      e = cudaMemcpy(uin, hb.uin.data(), 3 * nif * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      lbm_destroy(h);
      return fail(nullptr, LBM_ERR_CUDA, std::string("boundary upload: ") + cudaGetErrorString(e));
    }
    b.tag = tag;
    b.if_node = if_node;
    b.if_info = if_info;
    b.if_inc = if_inc;
    b.if_wallT = wallT;
    b.if_uin = uin;
    b.n_if = hb.n_if;
    for (int f = 0; f < 6; ++f) b.face[f] = cfg->face_bc[f];
    b.has_solid = hb.has_solid ? 1 : 0;
    b.solid_kind = cfg->solid_bc;
    b.sigma = cfg->outlet_sigma;
    b.outlet_L = cfg->outlet_length;
    b.inlet_simplified = cfg->inlet_simplified ? 1 : 0;
    b.p_out_lat = cfg->outlet_P * h->un.inv_c2;
    double Rin = 0.0;
    for (int a = 0; a < h->M; ++a) {
      b.Y_in[a] = cfg->inlet_Y[a];
      Rin += cfg->inlet_Y[a] / cfg->mech.molar_mass[a];
    }
    Rin *= R_U;
    b.T_in = cfg->inlet_T;
    b.rho_in = cfg->inlet_T > 0.0 ? cfg->inlet_P / (Rin * cfg->inlet_T) : 0.0;
    b.theta_in = Rin * cfg->inlet_T * h->un.inv_c2;
  }
  if (!h->pops[0] || !h->pops[1] || !h->rec || !h->cpar || !h->Tf || !h->status ||
      (s.codec && !h->codec)) {
    lbm_destroy(h);
    return fail(nullptr, LBM_ERR_OOM, "device allocation failed");
  }
  cudaError_t e = cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
  if (e != cudaSuccess) {
    lbm_destroy(h);
    return fail(nullptr, LBM_ERR_CUDA, std::string("status reset: ") + cudaGetErrorString(e));
  }
  *out = h;
  return LBM_OK;
}

lbm_status lbm_init_fields(lbm_t h, const double* rho, const double* u, const double* T,
                           const double* Y, int on_device) {
  return init_common(h, rho, 0, u, T, Y, on_device);
}

lbm_status lbm_init_fields_pressure(lbm_t h, const double* P, const double* u,
                                    const double* T, const double* Y, int on_device) {
  return init_common(h, P, 1, u, T, Y, on_device);
}

lbm_status lbm_step(lbm_t h, int nsteps) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID, "handle is NULL");
  if (nsteps < 0) return fail(h, LBM_ERR_INVALID, "nsteps must be >= 0");
  if (!h->initialized) return fail(h, LBM_ERR_STATE, "lbm_step before lbm_init_fields");
  DeviceGuard dg(h->cfg.device);
  StepArgs a;
  a.rec = h->rec;
  a.Tfield = h->Tf;
  a.status = h->status;
  a.g = h->g;
  a.un = h->un;
  a.bc = h->bc;
  a.lc = resolve_launch(h->opt, h->g.N, h->cfg.precision);
  a.mech_dev = h->mech_dev;
  a.cpar = h->cpar;
  a.side = h->side;
  a.ev_fork = h->ev_fork;
  a.ev_join = h->ev_join;
  for (int k = 0; k < nsteps; ++k) {
    a.src = h->pops[h->cur];
    a.dst = h->pops[1 - h->cur];
    cudaError_t e = launch_step(h->D, h->M, kernel_precision(h->cfg), h->mech, a, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
    h->cur = 1 - h->cur;
    ++h->steps;
  }
  return LBM_OK;
}

lbm_status lbm_step_timed(lbm_t h, int nsteps, double* kernel_ms, int n_kernels) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID, "handle is NULL");
  if (nsteps < 0 || !kernel_ms || n_kernels < 2)
    return fail(h, LBM_ERR_INVALID, "need nsteps >= 0 and kernel_ms[2]");
  if (!h->initialized) return fail(h, LBM_ERR_STATE, "lbm_step before lbm_init_fields");
  DeviceGuard dg(h->cfg.device);
  const int nev = 3 * nsteps;
  std::vector<cudaEvent_t> ev(nev, nullptr);
  for (auto& e : ev) cudaEventCreate(&e);
  StepArgs a;
  a.rec = h->rec;
  a.Tfield = h->Tf;
  a.status = h->status;
  a.g = h->g;
  a.un = h->un;
  a.bc = h->bc;
  a.lc = resolve_launch(h->opt, h->g.N, h->cfg.precision);
  a.mech_dev = h->mech_dev;
  a.cpar = h->cpar;
  a.side = h->side;
  a.ev_fork = h->ev_fork;
  a.ev_join = h->ev_join;
  cudaError_t err = cudaSuccess;
  for (int k = 0; k < nsteps && err == cudaSuccess; ++k) {
    a.src = h->pops[h->cur];
    a.dst = h->pops[1 - h->cur];
    cudaEventRecord(ev[3 * k], h->stream);
    err = launch_step(h->D, h->M, kernel_precision(h->cfg), h->mech, a, h->stream, 0);
    cudaEventRecord(ev[3 * k + 1], h->stream);
    if (err == cudaSuccess)
      err = launch_step(h->D, h->M, kernel_precision(h->cfg), h->mech, a, h->stream, 1);
    cudaEventRecord(ev[3 * k + 2], h->stream);
    h->cur = 1 - h->cur;
    ++h->steps;
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
  for (int k = 0; k < nsteps && err == cudaSuccess; ++k) {
    float t0 = 0.f, t1 = 0.f;
    cudaEventElapsedTime(&t0, ev[3 * k], ev[3 * k + 1]);
    cudaEventElapsedTime(&t1, ev[3 * k + 1], ev[3 * k + 2]);
    kernel_ms[0] += t0;
    kernel_ms[1] += t1;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (err != cudaSuccess) return cuda_fail(h, err, "timed step");
  return LBM_OK;
}

lbm_status lbm_set_launch(lbm_t h, const lbm_launch* l) {
  if (!h || !l) return fail(h, LBM_ERR_INVALID, "handle or launch is NULL");
  if (l->chem_lanes != -1 && l->chem_lanes != 1 && l->chem_lanes != 4 && l->chem_lanes != 8)
    return fail(h, LBM_ERR_INVALID, "chem_lanes must be -1, 1, 4 or 8");
  if (l->collide_split < -1 || l->collide_split > 1)
    return fail(h, LBM_ERR_INVALID, "collide_split must be -1, 0 or 1");
  if (l->persistent < -1 || l->persistent > 1)
    return fail(h, LBM_ERR_INVALID, "persistent must be -1, 0 or 1 (2: batch plans only)");
  if (l->nodes_per_thread != -1 && l->nodes_per_thread != 1 && l->nodes_per_thread != 2 &&
      l->nodes_per_thread != 4)
    return fail(h, LBM_ERR_INVALID, "nodes_per_thread must be -1, 1, 2 or 4");
  h->opt = *l;
  return LBM_OK;
}

lbm_status lbm_get_launch(lbm_t h, lbm_launch* l) {
  if (!h || !l) return fail(h, LBM_ERR_INVALID, "handle or launch is NULL");
  const Launch lc = resolve_launch(h->opt, h->g.N, h->cfg.precision);
  l->chem_lanes = lc.chem_lanes;
  l->collide_split = lc.coll_split;
  l->persistent = lc.persistent;
  l->nodes_per_thread = lc.npt;
  return LBM_OK;
}

lbm_status lbm_autotune(lbm_t h, int trial_steps, lbm_launch* chosen) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID, "handle is NULL");
  if (trial_steps < 1) return fail(h, LBM_ERR_INVALID, "trial_steps must be >= 1");
  if (!h->initialized) return fail(h, LBM_ERR_STATE, "lbm_autotune before lbm_init_fields");
  DeviceGuard dg(h->cfg.device);
  const size_t tbytes = (size_t)h->g.N * sizeof(double);
  double* Tsave = static_cast<double*>(dalloc(h->cfg, tbytes));
  if (!Tsave) return fail(h, LBM_ERR_OOM, "autotune scratch allocation failed");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Tsave, h->Tf, tbytes, cudaMemcpyDeviceToDevice, h->stream);
  // trial steps read the current buffer and write the other without
  // advancing the handle; only the temperature guess changes, and it is
  // restored after every candidate
  StepArgs a;
  a.src = h->pops[h->cur];
  a.dst = h->pops[1 - h->cur];
  a.rec = h->rec;
  a.Tfield = h->Tf;
  a.status = h->status;
  a.g = h->g;
  a.un = h->un;
  a.bc = h->bc;
  a.mech_dev = h->mech_dev;
  a.cpar = h->cpar;
  a.side = h->side;
  a.ev_fork = h->ev_fork;
  a.ev_join = h->ev_join;
  float best_ms = 0.f;
  Launch best;
  bool first = true;
  for (const Launch& cand : kCandidates) {
    if (e != cudaSuccess) break;
    a.lc = cand;
    e = launch_step(h->D, h->M, kernel_precision(h->cfg), h->mech, a, h->stream);   // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int t = 0; t < trial_steps && e == cudaSuccess; ++t)
      e = launch_step(h->D, h->M, kernel_precision(h->cfg), h->mech, a, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->Tf, Tsave, tbytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (first || ms < best_ms)) {
      best_ms = ms;
      best = cand;
      first = false;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(h->stream);
  dfree(h->cfg, Tsave);
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
  h->opt.chem_lanes = best.chem_lanes;
  h->opt.collide_split = best.coll_split;
  if (chosen) {
    *chosen = h->opt;
    const Launch r = resolve_launch(h->opt, h->g.N, h->cfg.precision);
    chosen->persistent = r.persistent;
    chosen->nodes_per_thread = r.npt;
  }
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_t* hs, int n, int nsteps) {
  if (!hs || n < 1) return fail(nullptr, LBM_ERR_INVALID, "need at least one handle");
  for (int k = 0; k < n; ++k)
    if (!hs[k]) return fail(nullptr, LBM_ERR_INVALID, "handle is NULL");
  lbm_ctx* h0 = hs[0];
  if (nsteps < 0) return fail(h0, LBM_ERR_INVALID, "nsteps must be >= 0");
  for (int k = 0; k < n; ++k) {
    lbm_ctx* h = hs[k];
    if (!h->initialized) return fail(h0, LBM_ERR_STATE, "lbm_batch_step before lbm_init_fields");
    if (h->D != h0->D || h->M != h0->M || h->cfg.precision != h0->cfg.precision ||
        kernel_precision(h->cfg) != kernel_precision(h0->cfg) ||
        h->cfg.device != h0->cfg.device)
      return fail(h0, LBM_ERR_INVALID,
                  "batched handles must share lattice, species count, precision and device");
    for (int j = 0; j < k; ++j)
      if (hs[j] == h) return fail(h0, LBM_ERR_INVALID, "a handle appears twice in the batch");
  }
  if (nsteps == 0) return LBM_OK;
  DeviceGuard dg(h0->cfg.device);
  std::vector<DomainDev> doms;
  BatchGrids gr;
  // the placement a new plan of these handles starts with (for FP64 under
  // kPlanSingleLaunch nodes: the whole step as one launch over a work-list)
  const Launch lc = resolve_launch(lbm_launch{-1, -1, -1, -1}, total_nodes(hs, n),
                                   hs[0]->cfg.precision, true);
  fill_domains(hs, n, lc, doms, gr);
  // every handle's earlier work precedes the batch; the batch runs on the
  // first handle's stream and each handle's stream waits for it afterwards
  cudaStream_t s0 = h0->stream;
  cudaEvent_t ev = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  for (int k = 1; k < n && e == cudaSuccess; ++k)
    if (hs[k]->stream != s0) {
      e = cudaEventRecord(ev, hs[k]->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s0, ev, 0);
    }
  DomainDev* ddev = static_cast<DomainDev*>(dalloc(h0->cfg, n * sizeof(DomainDev)));
  if (!ddev) e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ddev, doms.data(), n * sizeof(DomainDev), cudaMemcpyHostToDevice, s0);
  std::vector<PItem> items;
  PItem* items_dev = nullptr;
  int* sync_dev = nullptr;
  if (e == cudaSuccess && lc.persistent == 2) {
    int nsync = 0;
    build_worklist(hs, n, lc.npt, lc.coll_split != 0, items, nsync);
    items_dev = static_cast<PItem*>(dalloc(h0->cfg, items.size() * sizeof(PItem)));
    sync_dev = static_cast<int*>(dalloc(h0->cfg, (size_t)nsync * sizeof(int)));
    if (!items_dev || !sync_dev) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(items_dev, items.data(), items.size() * sizeof(PItem),
                          cudaMemcpyHostToDevice, s0);
    gr.items = items_dev;
    gr.nitems = (int)items.size();
    gr.sync = sync_dev;
    gr.nsync = nsync;
  }
  for (int step = 0; step < nsteps && e == cudaSuccess; ++step)
    e = launch_batch_step(h0->D, h0->M, kernel_precision(h0->cfg), ddev, n, gr, lc, step & 1, s0);
  if (e == cudaSuccess) e = cudaEventRecord(ev, s0);
  for (int k = 1; k < n && e == cudaSuccess; ++k)
    if (hs[k]->stream != s0) e = cudaStreamWaitEvent(hs[k]->stream, ev, 0);
  if (ddev || items_dev || sync_dev) {
    // plain cudaFree is not stream-ordered; the host copy of the items must
    // outlive its asynchronous upload
    if (!h0->cfg.dev_free || items_dev) cudaStreamSynchronize(s0);
    dfree(h0->cfg, ddev);
    dfree(h0->cfg, items_dev);
    dfree(h0->cfg, sync_dev);
  }
  if (ev) cudaEventDestroy(ev);
  if (e != cudaSuccess) return cuda_fail(h0, e, "batched step");
  for (int k = 0; k < n; ++k) {
    hs[k]->cur ^= (nsteps & 1);
    hs[k]->steps += nsteps;
  }
  return LBM_OK;
}

}  // extern "C"

struct lbm_batch_ctx {
  std::vector<lbm_ctx*> hs;
  std::vector<int> cur;        // each handle's buffer parity the plan expects
  DomainDev* ddev = nullptr;
  BatchGrids gr;
  Launch lc;                   // placement of the captured step
  SideStream side;             // boundary branch of the captured step
  int parity = 0;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t one[2] = {nullptr, nullptr}, two[2] = {nullptr, nullptr};
  // persistent == 2: the work-list and its sync words on the device
  PItem* items = nullptr;
  int items_cap = 0;
  int* sync = nullptr;
  int sync_cap = 0;
};

namespace {

cudaError_t batch_upload(lbm_batch_ctx* b) {
  std::vector<DomainDev> doms;
  const int n = (int)b->hs.size();
  fill_domains(b->hs.data(), n, b->lc, doms, b->gr);
  for (int k = 0; k < n; ++k) b->cur[k] = b->hs[k]->cur;
  b->parity = 0;
  cudaError_t e = cudaMemcpyAsync(b->ddev, doms.data(), doms.size() * sizeof(DomainDev),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess && b->lc.persistent == 2) {
    std::vector<PItem> items;
    int nsync = 0;
    build_worklist(b->hs.data(), n, b->lc.npt, b->lc.coll_split != 0, items, nsync);
    const lbm_config& cfg = b->hs[0]->cfg;
    if ((int)items.size() > b->items_cap) {
      e = cudaStreamSynchronize(b->stream);
      dfree(cfg, b->items);
      b->items = static_cast<PItem*>(dalloc(cfg, items.size() * sizeof(PItem)));
      b->items_cap = b->items ? (int)items.size() : 0;
      if (!b->items) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess && nsync > b->sync_cap) {
      e = cudaStreamSynchronize(b->stream);
      dfree(cfg, b->sync);
      b->sync = static_cast<int*>(dalloc(cfg, (size_t)nsync * sizeof(int)));
      b->sync_cap = b->sync ? nsync : 0;
      if (!b->sync) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->items, items.data(), items.size() * sizeof(PItem),
                          cudaMemcpyHostToDevice, b->stream);
    b->gr.items = b->items;
    b->gr.nitems = (int)items.size();
    b->gr.sync = b->sync;
    b->gr.nsync = nsync;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e;
}

cudaError_t batch_capture(lbm_batch_ctx* b, int first_parity, int nsteps, cudaGraphExec_t* out) {
  lbm_ctx* h0 = b->hs[0];
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  for (int k = 0; k < nsteps && e == cudaSuccess; ++k)
    e = launch_batch_step(h0->D, h0->M, kernel_precision(h0->cfg), b->ddev, (int)b->hs.size(), b->gr,
                          b->lc, (first_parity + k) & 1, b->stream, b->side);
  const cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  return e;
}

void batch_release_graphs(lbm_batch_ctx* b) {
  for (int p = 0; p < 2; ++p) {
    if (b->one[p]) cudaGraphExecDestroy(b->one[p]);
    if (b->two[p]) cudaGraphExecDestroy(b->two[p]);
    b->one[p] = b->two[p] = nullptr;
  }
}

// graphs of one and of two steps from either buffer parity
cudaError_t batch_capture_all(lbm_batch_ctx* b) {
  batch_release_graphs(b);
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
    e = batch_capture(b, p, 1, &b->one[p]);
    if (e == cudaSuccess) e = batch_capture(b, p, 2, &b->two[p]);
  }
  return e;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_destroy(lbm_batch_t b) {
  if (!b) return LBM_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_release_graphs(b);
  if (b->side.fork) cudaEventDestroy(b->side.fork);
  if (b->side.join) cudaEventDestroy(b->side.join);
  if (b->side.stream) cudaStreamDestroy(b->side.stream);
  if (b->ddev && !b->hs.empty()) dfree(b->hs[0]->cfg, b->ddev);
  if (b->items && !b->hs.empty()) dfree(b->hs[0]->cfg, b->items);
  if (b->sync && !b->hs.empty()) dfree(b->hs[0]->cfg, b->sync);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return LBM_OK;
}

lbm_status lbm_batch_create(lbm_t* hs, int n, lbm_batch_t* out) {
  if (!out) return fail(nullptr, LBM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  lbm_status st = lbm_batch_step(hs, n, 0);          // validation only
  if (st != LBM_OK) return st;
  lbm_ctx* h0 = hs[0];
  DeviceGuard dg(h0->cfg.device);
  lbm_batch_ctx* b = new lbm_batch_ctx();
  b->hs.assign(hs, hs + n);
  b->cur.assign(n, 0);
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side.fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side.join, cudaEventDisableTiming);
  if (e == cudaSuccess) {
    b->ddev = static_cast<DomainDev*>(dalloc(h0->cfg, n * sizeof(DomainDev)));
    if (!b->ddev) e = cudaErrorMemoryAllocation;
  }
  b->lc = resolve_launch(lbm_launch{-1, -1, -1, -1}, total_nodes(hs, n), hs[0]->cfg.precision,
                         true);
  if (e == cudaSuccess) e = batch_upload(b);
  if (e == cudaSuccess) e = prepare_batch_step(h0->D, h0->M, kernel_precision(h0->cfg));
  if (e == cudaSuccess) e = batch_capture_all(b);
  if (e != cudaSuccess) {
    lbm_batch_destroy(b);
    return cuda_fail(h0, e, "batch plan");
  }
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_run(lbm_batch_t b, int nsteps) {
  if (!b) return fail(nullptr, LBM_ERR_INVALID, "plan is NULL");
  lbm_ctx* h0 = b->hs[0];
  if (nsteps < 0) return fail(h0, LBM_ERR_INVALID, "nsteps must be >= 0");
  if (nsteps == 0) return LBM_OK;
  DeviceGuard dg(h0->cfg.device);
  cudaError_t e = cudaSuccess;
  // a handle stepped on its own since the last run: refresh the plan's view
  bool stale = false;
  for (size_t k = 0; k < b->hs.size(); ++k)
    stale |= (b->hs[k]->cur != (b->cur[k] ^ b->parity));
  cudaEvent_t ev = nullptr;
  e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  for (size_t k = 0; k < b->hs.size() && e == cudaSuccess; ++k) {
    e = cudaEventRecord(ev, b->hs[k]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, ev, 0);
  }
  if (e == cudaSuccess && stale) e = batch_upload(b);
  int left = nsteps;
  while (e == cudaSuccess && left >= 2) {
    e = cudaGraphLaunch(b->two[b->parity], b->stream);
    left -= 2;
  }
  if (e == cudaSuccess && left == 1) {
    e = cudaGraphLaunch(b->one[b->parity], b->stream);
    b->parity ^= 1;
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev, b->stream);
  for (size_t k = 0; k < b->hs.size() && e == cudaSuccess; ++k)
    e = cudaStreamWaitEvent(b->hs[k]->stream, ev, 0);
  if (ev) cudaEventDestroy(ev);
  if (e != cudaSuccess) return cuda_fail(h0, e, "batch run");
  for (lbm_ctx* h : b->hs) {
    h->cur ^= (nsteps & 1);
    h->steps += nsteps;
  }
  return LBM_OK;
}

lbm_status lbm_batch_set_launch(lbm_batch_t b, const lbm_launch* l) {
  if (!b || !l) return fail(nullptr, LBM_ERR_INVALID, "plan or launch is NULL");
  lbm_ctx* h0 = b->hs[0];
  if ((l->chem_lanes != -1 && l->chem_lanes != 1 && l->chem_lanes != 4 && l->chem_lanes != 8) ||
      l->collide_split < -1 || l->collide_split > 1 || l->persistent < -1 || l->persistent > 2 ||
      (l->nodes_per_thread != -1 && l->nodes_per_thread != 1 && l->nodes_per_thread != 2 &&
       l->nodes_per_thread != 4))
    return fail(h0, LBM_ERR_INVALID, "placement out of range");
  DeviceGuard dg(h0->cfg.device);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  b->lc = resolve_launch(*l, total_nodes(b->hs.data(), (int)b->hs.size()), h0->cfg.precision,
                         true);
  if (e == cudaSuccess) e = batch_upload(b);
  if (e == cudaSuccess) e = batch_capture_all(b);
  return e == cudaSuccess ? LBM_OK : cuda_fail(h0, e, "batch placement");
}

lbm_status lbm_batch_get_launch(lbm_batch_t b, lbm_launch* l) {
  if (!b || !l) return fail(nullptr, LBM_ERR_INVALID, "plan or launch is NULL");
  l->chem_lanes = b->lc.chem_lanes;
  l->collide_split = b->lc.coll_split;
  l->persistent = b->lc.persistent;
  l->nodes_per_thread = b->lc.npt;
  return LBM_OK;
}

lbm_status lbm_worklist(const long long* nodes, const long long* n_if, int n,
                        int nodes_per_thread, int collide_split, long long* items, int cap,
                        int* nitems, int* nsync) {
  if (!nodes || !n_if || !nitems || !nsync || n < 1 || (cap > 0 && !items))
    return fail(nullptr, LBM_ERR_INVALID, "lbm_worklist: NULL argument or no domain");
  if (nodes_per_thread != 1 && nodes_per_thread != 2 && nodes_per_thread != 4)
    return fail(nullptr, LBM_ERR_INVALID, "lbm_worklist: nodes_per_thread must be 1, 2 or 4");
  for (int k = 0; k < n; ++k)
    if (nodes[k] < 1 || n_if[k] < 0 || n_if[k] > nodes[k])
      return fail(nullptr, LBM_ERR_INVALID, "lbm_worklist: bad domain size");
  std::vector<PItem> list;
  int ns = 0;
  build_worklist(nodes, n_if, n, nodes_per_thread, collide_split != 0, list, ns);
  *nitems = (int)list.size();
  *nsync = ns;
  if ((int)list.size() > cap) return cap > 0 ? fail(nullptr, LBM_ERR_RANGE, "lbm_worklist: cap too small") : LBM_OK;
  for (size_t i = 0; i < list.size(); ++i) {
    long long* o = items + 5 * i;
    o[0] = list[i].kind;
    o[1] = list[i].dom;
    o[2] = list[i].first;
    o[3] = list[i].dep;
    o[4] = list[i].flag;
  }
  return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch_t b, int trial_steps, lbm_launch* chosen) {
  if (!b) return fail(nullptr, LBM_ERR_INVALID, "plan is NULL");
  lbm_ctx* h0 = b->hs[0];
  if (trial_steps < 1) return fail(h0, LBM_ERR_INVALID, "trial_steps must be >= 1");
  DeviceGuard dg(h0->cfg.device);
  const int n = (int)b->hs.size();
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < n && e == cudaSuccess; ++k) e = cudaStreamSynchronize(b->hs[k]->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  // temperature guesses of every handle, restored after each candidate
  std::vector<double*> Tsave(n, nullptr);
  for (int k = 0; k < n && e == cudaSuccess; ++k) {
    const size_t tb = (size_t)b->hs[k]->g.N * sizeof(double);
    Tsave[k] = static_cast<double*>(dalloc(h0->cfg, tb));
    if (!Tsave[k]) e = cudaErrorMemoryAllocation;
    else e = cudaMemcpyAsync(Tsave[k], b->hs[k]->Tf, tb, cudaMemcpyDeviceToDevice, b->stream);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best_ms = 0.f;
  Launch best = b->lc;
  bool first = true;
  // stage 1: the six placements with one block per tile; stage 2: the best
  // of them with persistent grids; stage 3: the whole step as one launch over
  // the work-list, split and fused collision, each with 1, 2 and 4 nodes per
  // thread (tiles of 128, 256, 512 nodes)
  const size_t nc = sizeof(kCandidates) / sizeof(kCandidates[0]);
  const int npts[3] = {1, 2, 4};
  for (size_t ci = 0; ci <= nc + 6; ++ci) {
    if (e != cudaSuccess) break;
    Launch cand;
    if (ci < nc) {
      cand = kCandidates[ci];
    } else if (ci == nc) {
      cand = best;
      cand.persistent = 1;
    } else {
      cand = Launch();
      cand.chem_lanes = 1;
      cand.coll_split = (ci - nc - 1) < 3 ? 1 : 0;
      cand.persistent = 2;
      cand.npt = npts[(ci - nc - 1) % 3];
    }
    b->lc = cand;
    e = batch_upload(b);
    // the candidate as the plan would run it: its captured one-step graph
    // from parity 0, replayed; every trial step recomputes the next state of
    // every handle from its current buffer, advancing none of them
    if (e == cudaSuccess) e = batch_capture_all(b);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->one[0], b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
    for (int t = 0; t < trial_steps && e == cudaSuccess; ++t)
      e = cudaGraphLaunch(b->one[0], b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
    for (int k = 0; k < n && e == cudaSuccess; ++k)
      e = cudaMemcpyAsync(b->hs[k]->Tf, Tsave[k], (size_t)b->hs[k]->g.N * sizeof(double),
                          cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (first || ms < best_ms)) {
      best_ms = ms;
      best = cand;
      first = false;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(b->stream);
  for (int k = 0; k < n; ++k) dfree(h0->cfg, Tsave[k]);
  if (e == cudaSuccess) {
    b->lc = best;
    e = batch_upload(b);
  }
  if (e == cudaSuccess) e = batch_capture_all(b);
  if (e != cudaSuccess) return cuda_fail(h0, e, "batch autotune");
  if (chosen) {
    chosen->chem_lanes = best.chem_lanes;
    chosen->collide_split = best.coll_split;
    chosen->persistent = best.persistent;
    chosen->nodes_per_thread = best.npt;
  }
  return LBM_OK;
}

lbm_status lbm_moments(lbm_t h, double* rho, double* u, double* T, double* Y, double* E,
                       int on_device) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID, "handle is NULL");
  if (!h->initialized) return fail(h, LBM_ERR_STATE, "lbm_moments before lbm_init_fields");
  DeviceGuard dg(h->cfg.device);
  const long long N = h->g.N;
  const int M = h->M;
  if (on_device) {
    cudaError_t e = launch_moments_out(h->D, M, kernel_precision(h->cfg), h->mech, h->g, h->un,
                                       h->pops[h->cur], h->Tf, rho, u, T, Y, E, h->status,
                                       h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
    return LBM_OK;
  }
  const size_t nb = N * sizeof(double);
  lbm_status st = ensure_io(h, (size_t)(1 + 3 + 1 + M + 1) * nb);
  if (st != LBM_OK) return st;
  double* p = h->io;
  double *drho = p, *du = p + N, *dT = p + 4 * N, *dY = p + 5 * N, *dE = p + (5 + M) * N;
  cudaError_t e = launch_moments_out(h->D, M, kernel_precision(h->cfg), h->mech, h->g, h->un,
                                     h->pops[h->cur], h->Tf, rho ? drho : nullptr,
                                     u ? du : nullptr, T ? dT : nullptr, Y ? dY : nullptr,
                                     E ? dE : nullptr, h->status, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
  if (rho && e == cudaSuccess) e = cudaMemcpyAsync(rho, drho, nb, cudaMemcpyDeviceToHost, h->stream);
  if (u && e == cudaSuccess) e = cudaMemcpyAsync(u, du, 3 * nb, cudaMemcpyDeviceToHost, h->stream);
  if (T && e == cudaSuccess) e = cudaMemcpyAsync(T, dT, nb, cudaMemcpyDeviceToHost, h->stream);
  if (Y && e == cudaSuccess) e = cudaMemcpyAsync(Y, dY, M * nb, cudaMemcpyDeviceToHost, h->stream);
  if (E && e == cudaSuccess) e = cudaMemcpyAsync(E, dE, nb, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "moments download");
  return check_status(h);
}

lbm_status lbm_diagnostics_planes(lbm_t h, int x0, int nplanes, lbm_diag* out) {
  if (!h || !out) return fail(h, LBM_ERR_INVALID, "handle or out is NULL");
  if (!h->initialized) return fail(h, LBM_ERR_STATE, "lbm_diagnostics before lbm_init_fields");
  if (x0 < 0 || nplanes < 0 || x0 + (long long)nplanes > h->g.nx)
    return fail(h, LBM_ERR_RANGE, "planes outside 0..nx-1");
  DeviceGuard dg(h->cfg.device);
  const long long nb = (h->g.N + 127) / 128;
  const size_t need = (size_t)(nb + 1) * sizeof(DiagPart);
  lbm_status st = ensure_io(h, need);
  if (st != LBM_OK) return st;
  DiagPart* part = reinterpret_cast<DiagPart*>(h->io);
  DiagPart* dout = part + nb;
  cudaError_t e = launch_diagnostics(h->D, h->M, kernel_precision(h->cfg), h->mech, h->g, h->un,
                                     h->pops[h->cur], h->Tf, h->bc.tag, part, dout, h->status,
                                     x0, x0 + nplanes, h->stream);
  DiagPart r;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&r, dout, sizeof(DiagPart), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics");
  const double cell = h->D == 3 ? h->un.dx * h->un.dx * h->un.dx : h->un.dx * h->un.dx;
  out->hrr_integral = r.q_sum * cell;
  out->hrr_max = r.q_max;
  // no fluid node in the planes: no maximum, no position
  out->flame_x = r.n_max == LLONG_MAX ? NAN : (double)(r.n_max % h->g.nx) * h->un.dx;
  out->T_max = r.T_max;
  out->u_max = r.u_max;
  return check_status(h);
}

lbm_status lbm_diagnostics(lbm_t h, lbm_diag* out) {
  if (!h) return fail(h, LBM_ERR_INVALID, "handle or out is NULL");
  return lbm_diagnostics_planes(h, 0, h->g.nx, out);
}

lbm_status lbm_get_populations(lbm_t h, double* out, int on_device) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID, "handle is NULL");
  if (!out) return fail(h, LBM_ERR_INVALID, "out is NULL");
  if (!h->initialized) return fail(h, LBM_ERR_STATE, "no populations before lbm_init_fields");
  DeviceGuard dg(h->cfg.device);
  const long long count = (long long)h->L * h->Q * h->g.N;
  if (on_device) {
    cudaError_t e = launch_to_fp64(h->cfg.precision, h->pops[h->cur], out, count, h->stream,
                                   h->g.N, h->codec);
    return e == cudaSuccess ? LBM_OK : cuda_fail(h, e, "population conversion");
  }
  lbm_status st = ensure_io(h, (size_t)count * sizeof(double));
  if (st != LBM_OK) return st;
  cudaError_t e = launch_to_fp64(h->cfg.precision, h->pops[h->cur], h->io, count, h->stream,
                                 h->g.N, h->codec);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, h->io, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "population download");
  return check_status(h);
}

// Planes x0 .. x0+nplanes-1 of the stored state: populations [L][Q][nz][ny]
// [nplanes] in the storage precision, then the temperature guesses
// [nz][ny][nplanes] (FP64).  One strided copy each (rows of nplanes values
// at pitch nx), synchronous.
static lbm_status planes_io(lbm_t h, int x0, int nplanes, void* buf, int on_device, bool out) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID, "handle is NULL");
  if (!buf) return fail(h, LBM_ERR_INVALID, "buffer is NULL");
  if (h->cfg.precision == LBM_FP16_OFFSET)
    return fail(h, LBM_ERR_INVALID, "plane copies need FP64 or FP32 storage (FP16 offsets "
                                    "depend on each handle's codec)");
  if (nplanes < 1 || x0 < 0 || x0 + nplanes > h->g.nx)
    return fail(h, LBM_ERR_RANGE, "planes outside 0 .. nx-1");
  if (!h->initialized) return fail(h, LBM_ERR_STATE, "no state before lbm_init_fields");
  DeviceGuard dg(h->cfg.device);
  const size_t rows = (size_t)h->L * h->Q * h->g.nz * h->g.ny;
  const size_t trows = (size_t)h->g.nz * h->g.ny;
  const size_t e1 = h->elem, w = (size_t)nplanes;
  char* pops = static_cast<char*>(h->pops[h->cur]) + (size_t)x0 * e1;
  char* tf = reinterpret_cast<char*>(h->Tf + x0);
  char* b = static_cast<char*>(buf);
  char* bt = b + rows * w * e1;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice
                                     : (out ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
  const size_t pitch = (size_t)h->g.nx * e1, tpitch = (size_t)h->g.nx * sizeof(double);
  cudaError_t e;
  if (out) {
    e = cudaMemcpy2DAsync(b, w * e1, pops, pitch, w * e1, rows, k, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(bt, w * sizeof(double), tf, tpitch, w * sizeof(double), trows, k,
                            h->stream);
  } else {
    e = cudaMemcpy2DAsync(pops, pitch, b, w * e1, w * e1, rows, k, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(tf, tpitch, bt, w * sizeof(double), w * sizeof(double), trows, k,
                            h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "plane copy");
  return LBM_OK;
}

lbm_status lbm_get_planes(lbm_t h, int x0, int nplanes, void* buf, int on_device) {
  return planes_io(h, x0, nplanes, buf, on_device, true);
}

lbm_status lbm_set_planes(lbm_t h, int x0, int nplanes, const void* buf, int on_device) {
  return planes_io(h, x0, nplanes, const_cast<void*>(buf), on_device, false);
}

lbm_status lbm_synchronize(lbm_t h) {
  if (!h) return fail(nullptr, LBM_ERR_INVALID, "handle is NULL");
  DeviceGuard dg(h->cfg.device);
  return check_status(h);
}

static const uint64_t STATE_MAGIC = 0x4c424d5354415445ull;   // "LBMSTATE"

lbm_status lbm_get_state(lbm_t h, void* buf, size_t* bytes) {
  if (!h || !bytes) return fail(h, LBM_ERR_INVALID, "handle or bytes is NULL");
  const size_t pop_bytes = (size_t)h->L * h->Q * h->g.N * h->elem;
  const size_t codec_bytes = h->codec ? (size_t)h->L * h->Q * sizeof(float4) : 0;
  const size_t need = 64 + pop_bytes + h->g.N * sizeof(double) + codec_bytes;
  if (!buf) { *bytes = need; return LBM_OK; }
  if (*bytes < need) return fail(h, LBM_ERR_INVALID, "state buffer too small");
  if (!h->initialized) return fail(h, LBM_ERR_STATE, "no state before lbm_init_fields");
  DeviceGuard dg(h->cfg.device);
  uint64_t hdr[8] = {STATE_MAGIC, (uint64_t)h->D, (uint64_t)h->M, (uint64_t)h->g.nx,
                     (uint64_t)h->g.ny, (uint64_t)h->g.nz, (uint64_t)h->cfg.precision,
                     (uint64_t)h->steps};
  std::memcpy(buf, hdr, 64);
  char* p = static_cast<char*>(buf) + 64;
  cudaError_t e = cudaMemcpyAsync(p, h->pops[h->cur], pop_bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p + pop_bytes, h->Tf, h->g.N * sizeof(double), cudaMemcpyDeviceToHost,
                        h->stream);
  if (e == cudaSuccess && codec_bytes)   // FP16: the codec the populations are encoded with
    e = cudaMemcpyAsync(p + pop_bytes + h->g.N * sizeof(double), h->codec, codec_bytes,
                        cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "state download");
  *bytes = need;
  return check_status(h);
}

lbm_status lbm_set_state(lbm_t h, const void* buf, size_t bytes) {
  if (!h || !buf) return fail(h, LBM_ERR_INVALID, "handle or buffer is NULL");
  const size_t pop_bytes = (size_t)h->L * h->Q * h->g.N * h->elem;
  const size_t codec_bytes = h->codec ? (size_t)h->L * h->Q * sizeof(float4) : 0;
  const size_t need = 64 + pop_bytes + h->g.N * sizeof(double) + codec_bytes;
  if (bytes != need) return fail(h, LBM_ERR_INVALID, "state size does not match this handle");
  uint64_t hdr[8];
  std::memcpy(hdr, buf, 64);
  if (hdr[0] != STATE_MAGIC || hdr[1] != (uint64_t)h->D || hdr[2] != (uint64_t)h->M ||
      hdr[3] != (uint64_t)h->g.nx || hdr[4] != (uint64_t)h->g.ny ||
      hdr[5] != (uint64_t)h->g.nz || hdr[6] != (uint64_t)h->cfg.precision)
    return fail(h, LBM_ERR_INVALID, "state was written by an incompatible handle");
  DeviceGuard dg(h->cfg.device);
  const char* p = static_cast<const char*>(buf) + 64;
  cudaError_t e = cudaMemcpyAsync(h->pops[h->cur], p, pop_bytes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->Tf, p + pop_bytes, h->g.N * sizeof(double), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess && codec_bytes)
    e = cudaMemcpyAsync(h->codec, p + pop_bytes + h->g.N * sizeof(double), codec_bytes,
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->pops[1 - h->cur], h->pops[h->cur], pop_bytes,
                        cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "state upload");
  h->steps = (long long)hdr[7];
  h->initialized = true;
  return LBM_OK;
}

lbm_status lbm_get_info(lbm_t h, lbm_info* info) {
  if (!h || !info) return fail(h, LBM_ERR_INVALID, "handle or info is NULL");
  info->Q = h->Q;
  info->D = h->D;
  info->L = h->L;
  info->M = h->M;
  info->n_nodes = h->g.N;
  info->c_ref = h->un.c;
  info->dt = h->un.dt;
  info->dx = h->un.dx;
  info->bytes_per_population = h->elem;
  info->device_bytes = h->bytes;
  info->steps_done = h->steps;
  return LBM_OK;
}

lbm_status lbm_destroy(lbm_t h) {
  if (!h) return LBM_OK;
  DeviceGuard dg(h->cfg.device);
  lbm_status st = LBM_OK;
  if (h->status) st = check_status(h);
  cudaStreamSynchronize(h->stream);
  dfree(h->cfg, h->pops[0]);
  dfree(h->cfg, h->pops[1]);
  dfree(h->cfg, h->rec);
  dfree(h->cfg, h->cpar);
  dfree(h->cfg, h->codec);
  dfree(h->cfg, h->Tf);
  dfree(h->cfg, h->status);
  dfree(h->cfg, h->io);
  dfree(h->cfg, h->bc_mem);
  dfree(h->cfg, h->mech_dev);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  delete h;
  return st;
}

const char* lbm_last_error(lbm_t h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The FP64 table-driven exp at given points (a test hook for its accuracy).
__global__ void k_exp64_check(const double* __restrict__ x, long long n,
                              double* __restrict__ e) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) e[i] = exp_tang(x[i]);
}

lbm_status lbm_exp64_check(const double* x, long long n, double* exp_out) {
  if (!x || !exp_out || n < 0)
    return fail(nullptr, LBM_ERR_INVALID, "lbm_exp64_check: NULL buffer or negative n");
  if (n > (1LL << 24)) return fail(nullptr, LBM_ERR_RANGE, "lbm_exp64_check: n above 2^24");
  if (n == 0) return LBM_OK;
  double* d = nullptr;
  const size_t b = (size_t)n * sizeof(double);
  cudaError_t e = cudaMalloc(&d, 2 * b);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "lbm_exp64_check allocation");
  e = cudaMemcpy(d, x, b, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_exp64_check<<<(unsigned)((n + 255) / 256), 256>>>(d, n, d + n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(exp_out, d + n, b, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? LBM_OK : cuda_fail(nullptr, e, "lbm_exp64_check");
}

// ---------------------------------------------------------------------------
// Float-float exp and log at given points (a test hook for their accuracy).
__global__ void k_ff_check(const double* __restrict__ x, long long n, double* __restrict__ e,
                           double* __restrict__ l) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ff v = ff_from_double(x[i]);
  e[i] = ff_to_double(ff_exp(v));
  l[i] = v.hi > 0.f ? ff_to_double(ff_log(v)) : __longlong_as_double(0x7ff8000000000000LL);
}

lbm_status lbm_ff_check(const double* x, long long n, double* exp_out, double* log_out) {
  if (!x || !exp_out || !log_out || n < 0)
    return fail(nullptr, LBM_ERR_INVALID, "lbm_ff_check: NULL buffer or negative n");
  if (n > (1LL << 24)) return fail(nullptr, LBM_ERR_RANGE, "lbm_ff_check: n above 2^24");
  if (n == 0) return LBM_OK;
  double* d = nullptr;
  const size_t b = (size_t)n * sizeof(double);
  cudaError_t e = cudaMalloc(&d, 3 * b);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "lbm_ff_check allocation");
  e = cudaMemcpy(d, x, b, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_ff_check<<<(unsigned)((n + 255) / 256), 256>>>(d, n, d + n, d + 2 * n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(exp_out, d + n, b, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(log_out, d + 2 * n, b, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? LBM_OK : cuda_fail(nullptr, e, "lbm_ff_check");
}
