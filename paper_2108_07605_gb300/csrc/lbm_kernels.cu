// Kernels of the reactive-mixture LBM step (thread per node).
//
//   k_moments   pull-stream all lattices, moments, temperature Newton,
//               write the per-node moment record (scratch) and T guess.
//   k_collide   gradients from neighbour records, relaxation parameters,
//               diffusion velocities, reaction sub-steps, collision of all
//               lattices on a second pull gather, store to the other buffer.
//   k_init      populations at the equilibria of given fields.
//   k_out       fields of the stored state (SI units).
//
// Template parameters: D (2 or 3), M (species), S (storage type), RT (type
// of the lattice arithmetic: moments, equilibria, collision).  Temperature,
// transport, diffusion velocities and chemistry always run in FP64.
#include <cmath>

#include "lbm_device.cuh"

namespace lbm {

template <typename S>
__device__ __forceinline__ double ldp(const S* p) { return static_cast<double>(__ldg(p)); }

__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <int D>
__device__ __forceinline__ long long node_shift(int x, int y, int z, int i, int sgn,
                                                const Geom& g) {
  const int sx = wrap1(x + sgn * cvel(i, 0), g.nx);
  const int sy = wrap1(y + sgn * cvel(i, 1), g.ny);
  const int sz = D == 3 ? wrap1(z + sgn * cvel(i, 2), g.nz) : 0;
  return sx + (long long)g.nx * (sy + (long long)g.ny * sz);
}

// Population (lattice l, direction i) entering node n's collision: the
// reconstructed value for interface nodes (tag >= 0), else the streamed one.
template <typename RT, typename S>
__device__ __forceinline__ RT pop_in(const S* __restrict__ src, const BCDev& bc, int tag,
                                     long long N, long long sn, int li) {
  return tag >= 0 ? RT(bc.pops[(long long)li * bc.n_if + tag])
                  : RT(__ldg(src + (long long)li * N + sn));
}

// 1/tau_ab = s * K_ab: the coefficient table in the lattice compute type
template <typename RT> __device__ __forceinline__ RT kcoef(const DevMech& m, int a, int b);
template <> __device__ __forceinline__ double kcoef<double>(const DevMech& m, int a, int b) {
  return m.K[a][b];
}
template <> __device__ __forceinline__ float kcoef<float>(const DevMech& m, int a, int b) {
  return m.Kf[a][b];
}

// threads per block of the node kernels (the shared-memory columns use it)
constexpr int kBS = 128;

// shared memory of the collision kernel per thread: the diffusion-velocity
// matrix, then the axis-factor tables
// (tables only in the FP32 path: in FP64 they would halve the occupancy)
template <int D, int M, typename RT> constexpr int collide_smem_entries() {
  return (sizeof(RT) == 4 && 2 * M * D * 3 > M * M) ? 2 * M * D * 3 : M * M;
}

template <typename R>
__device__ __forceinline__ R pick3(int c, const R (&v)[3]) {
  return c == 0 ? v[1] : (c > 0 ? v[2] : v[0]);
}

template <int D>
__device__ __forceinline__ constexpr int pidx(int a, int b) {
  return a == b ? a : (D == 3 ? (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5)) : 2);
}

// ---------------------------------------------------------------------------
// Moments of the post-stream state + temperature (Sec. 2.1, Sec. 3.1-3.2,
// Sec. 3.7 slaving, Sec. 4.1 pull streaming).
// chem_inline = 0: the reaction sub-steps run in k_chem (one warp per node);
// this kernel then leaves the post-stream species densities rho_a (a < M) in
// the record's increment slots for it.
template <int D, int M, typename S, typename RT>
__device__ __forceinline__ void moments_body(const S* __restrict__ src, RT* __restrict__ rec,
                                             double* __restrict__ Tf, int* __restrict__ status,
                                             const Geom& g, const Units& un, const BCDev& bc,
                                             const DevMech& mech, long long n,
                                             int chem_inline) {
  constexpr int Q = Lat<D>::Q, NP = Lat<D>::NP;
  using RC = Rec<D, M>;
  const long long N = g.N;
  if (n >= N) return;
  const int tag = bc.tag ? bc.tag[n] : TAG_BULK;
  if (tag == TAG_SOLID) return;
  const int x = (int)(n % g.nx);
  const int y = (int)((n / g.nx) % g.ny);
  const int z = (int)(n / ((long long)g.nx * g.ny));

  // sums in the lattice compute type RT
  RT rho = RT(0), rhoE = RT(0), j[D], q[D], P[NP], rs[M], js[M][D];
#pragma unroll
  for (int d = 0; d < D; ++d) { j[d] = RT(0); q[d] = RT(0); }
#pragma unroll
  for (int k = 0; k < NP; ++k) P[k] = RT(0);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    rs[a] = RT(0);
#pragma unroll
    for (int d = 0; d < D; ++d) js[a][d] = RT(0);
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const long long sn = node_shift<D>(x, y, z, i, -1, g);
#pragma unroll
    for (int a = 0; a < M - 1; ++a) {
      const RT v = pop_in<RT>(src, bc, tag, N, sn, a * Q + i);
      rs[a] += v;
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (cvel(i, d) != 0) js[a][d] += cvel(i, d) * v;
    }
    const RT f = pop_in<RT>(src, bc, tag, N, sn, (M - 1) * Q + i);
    rho += f;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (cvel(i, d) != 0) j[d] += cvel(i, d) * f;
#pragma unroll
      for (int e = d; e < D; ++e)
        if (cvel(i, d) * cvel(i, e) != 0) P[pidx<D>(d, e)] += cvel(i, d) * cvel(i, e) * f;
    }
    const RT gv = pop_in<RT>(src, bc, tag, N, sn, M * Q + i);
    rhoE += gv;
#pragma unroll
    for (int d = 0; d < D; ++d)
      if (cvel(i, d) != 0) q[d] += cvel(i, d) * gv;
  }
  // slaved species M (Eq. strongest)
  rs[M - 1] = rho;
#pragma unroll
  for (int d = 0; d < D; ++d) js[M - 1][d] = j[d];
#pragma unroll
  for (int a = 0; a < M - 1; ++a) {
    rs[M - 1] -= rs[a];
#pragma unroll
    for (int d = 0; d < D; ++d) js[M - 1][d] -= js[a][d];
  }
  // node fields in the lattice type; FP64 only for the temperature solve
  const RT inv_rho = RT(1) / rho;
  RT uR[D], YR[M], usqR = RT(0);
#pragma unroll
  for (int d = 0; d < D; ++d) { uR[d] = j[d] * inv_rho; usqR += uR[d] * uR[d]; }
#pragma unroll
  for (int a = 0; a < M; ++a) YR[a] = rs[a] * inv_rho;
  const RT ER = rhoE * inv_rho;
  bool ok;
  double T;
  RT thR;
  if constexpr (sizeof(RT) == 4) {
    // mixed path: the temperature solve in float-float
    ff Yf[M];
    float Rm = 0.f;
#pragma unroll
    for (int a = 0; a < M; ++a) {
      Yf[a] = ff(YR[a]);
      Rm += YR[a] * mech.inv_mm_s[a];
    }
    const ff U = (ff(ER) + ff(-0.5f * usqR)) * un.c2_f;
    const ff Tx = newton_T_ff<M>(mech, Yf, U, ff_from_double(Tf[n]), un.newton_max_iter,
                                 un.newton_rtol_f, ok);
    T = ff_to_double(Tx);
    thR = Rm * float(R_U) * Tx.hi * un.inv_c2_s;
  } else {
    double Y[M];
#pragma unroll
    for (int a = 0; a < M; ++a) Y[a] = double(YR[a]);
    const double U = (double(ER) - 0.5 * double(usqR)) * un.c * un.c;
    T = newton_T<M>(mech, Y, U, Tf[n], un.newton_max_iter, un.newton_rtol, ok);
    double Rmix = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) Rmix += Y[a] * mech.inv_mm[a];
    Rmix *= R_U;
    thR = RT(Rmix * T * un.inv_c2);
  }
  if (!ok) atomicOr(status, ST_NEWTON);
  if (!(rho > RT(0)) || !isfinite(double(rho)) || !isfinite(T)) atomicOr(status, ST_NONFINITE);
  Tf[n] = T;

  // reaction sub-steps at frozen U (Sec. 2.4 Eq. R3): a zero-dimensional
  // reactor per node from its post-stream species densities; T_0 is the T
  // just solved.  The increments drho_a (a < M) go to the record.
  if (!chem_inline) {
#pragma unroll
    for (int a = 0; a < M - 1; ++a) rec[(RC::DRHO + a) * N + n] = rs[a];
  } else if constexpr (sizeof(RT) == 4) {
    const ff Uphys = (ff(ER) + ff(-0.5f * usqR)) * un.c2_f;
    ff r[M], rdot[M];
#pragma unroll
    for (int a = 0; a < M; ++a) r[a] = ff(rs[a]);
    ff Ts = ff_from_double(T);
    const ff rho_f(rho);
    for (int s = 0; s < un.substeps; ++s) {
      if (s > 0) {
        ff Ys[M];
#pragma unroll
        for (int a = 0; a < M; ++a) Ys[a] = r[a] / rho_f;
        bool oks;
        Ts = newton_T_ff<M>(mech, Ys, Uphys, Ts, un.newton_max_iter, un.newton_rtol_f, oks);
        if (!oks) atomicOr(status, ST_NEWTON);
      }
      production_rates_ff<M>(mech, Ts, r, rdot);
#pragma unroll
      for (int a = 0; a < M; ++a) r[a] += un.dt_sub_f * rdot[a];
    }
#pragma unroll
    for (int a = 0; a < M - 1; ++a) rec[(RC::DRHO + a) * N + n] = (r[a] - ff(rs[a])).hi;
  } else {
    const double Uphys = (double(ER) - 0.5 * double(usqR)) * un.c * un.c;
    const double dtr = un.dt / un.substeps;
    const double rho_d = double(rho);
    double r[M], rdot[M];
#pragma unroll
    for (int a = 0; a < M; ++a) r[a] = double(rs[a]);
    double Ts = T;
    for (int s = 0; s < un.substeps; ++s) {
      if (s > 0) {
        double Ys[M];
        const double ir = 1.0 / rho_d;
#pragma unroll
        for (int a = 0; a < M; ++a) Ys[a] = r[a] * ir;
        bool oks;
        Ts = newton_T<M>(mech, Ys, Uphys, Ts, un.newton_max_iter, un.newton_rtol, oks);
        if (!oks) atomicOr(status, ST_NEWTON);
      }
      production_rates<M>(mech, Ts, r, rdot);
#pragma unroll
      for (int a = 0; a < M; ++a) r[a] += dtr * rdot[a];
    }
#pragma unroll
    for (int a = 0; a < M - 1; ++a) rec[(RC::DRHO + a) * N + n] = RT(r[a] - double(rs[a]));
  }

  rec[RC::RHO * N + n] = rho;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    rec[(RC::U + d) * N + n] = uR[d];
    rec[(RC::QF + d) * N + n] = q[d];
    rec[(RC::PHI + d) * N + n] = rho * uR[d] * (RT(1) - RT(3) * thR) - rho * uR[d] * uR[d] * uR[d];
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) rec[(RC::P + k) * N + n] = P[k];
  rec[RC::E * N + n] = ER;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    rec[(RC::Y + a) * N + n] = YR[a];
    // where defined, |j_a| < rho_a, so the quotient lies in (-1, 1) even when
    // rho_a is denormal in FP32 (its reciprocal would overflow)
    const bool tiny = species_velocity_undefined<D, RT>(rs[a], js[a]);
#pragma unroll
    for (int d = 0; d < D; ++d)
      rec[(RC::US + a * D + d) * N + n] = tiny ? uR[d] : js[a][d] / rs[a];
  }
}

// ---------------------------------------------------------------------------
// Reaction sub-steps with one warp per node (Sec. 2.4 Eq. R3), for grids too
// small to fill the GPU at one thread per node: the lanes take the reactions'
// rates of progress, then lanes a < M sum them into the species production
// rates and advance rho_a.  The formulas and their order of evaluation are
// those of production_rates / production_rates_ff, so both placements give
// the same increments.  CT: double (FP64 path) or float-float (mixed path).
template <typename CT> struct Chem;
template <> struct Chem<double> {
  __device__ static double ex(double x) { return exp(x); }
  __device__ static double ln(double x) { return log(x); }
  __device__ static double inv(double x) { return 1.0 / x; }
  __device__ static double inv_mm(const DevMech& m, int a) { return m.inv_mm[a]; }
  __device__ static double mm(const DevMech& m, int a) { return m.mm[a]; }
  __device__ static double gibbs(const DevMech& m, int a, double T, double invT, double lnT) {
    return m.g_inv[a] * invT + m.g0[a] + T * (m.g1[a] + T * m.g2[a]) - m.a0[a] * lnT;
  }
  __device__ static double lnkf(const DevReaction& rx, double lnT, double invT) {
    return rx.lnA + rx.b * lnT - rx.EaR * invT;
  }
  __device__ static double rev_arg(const DevReaction& rx, double lk, double dG, double lp) {
    return lk + dG - rx.dn * lp;
  }
  __device__ static double ln_p0(const DevMech& m) { return m.ln_p0_over_ru; }
  __device__ static double eff(const DevMech& m, int k, int a) { return m.eff[k][a]; }
  __device__ static double dt_sub(const Units& u) { return u.dt / u.substeps; }
  __device__ static double of(double v) { return v; }
  __device__ static double of_T(double T) { return T; }
  template <int M>
  __device__ static double newton(const DevMech& m, const double (&r)[M], double rho, double U,
                                  double T, const Units& un, bool& ok) {
    double Ys[M];
    const double ir = 1.0 / rho;
#pragma unroll
    for (int a = 0; a < M; ++a) Ys[a] = r[a] * ir;
    return newton_T<M>(m, Ys, U, T, un.newton_max_iter, un.newton_rtol, ok);
  }
};
template <> struct Chem<ff> {
  __device__ static ff ex(ff x) { return ff_exp(x); }
  __device__ static ff ln(ff x) { return ff_log(x); }
  __device__ static ff inv(ff x) { return ff(1.f) / x; }
  __device__ static ff inv_mm(const DevMech& m, int a) { return m.inv_mm_f[a]; }
  __device__ static ff mm(const DevMech& m, int a) { return m.mm_f[a]; }
  __device__ static ff gibbs(const DevMech& m, int a, ff T, ff invT, ff lnT) {
    return m.g_inv_f[a] * invT + m.g0_f[a] + T * (m.g1_f[a] + T * m.g2_f[a]) - m.a0_f[a] * lnT;
  }
  __device__ static ff lnkf(const DevReaction& rx, ff lnT, ff invT) {
    return rx.lnA_f + rx.b_f * lnT - rx.EaR_f * invT;
  }
  __device__ static ff rev_arg(const DevReaction& rx, ff lk, ff dG, ff lp) {
    return lk + dG - ff((float)rx.dn) * lp;
  }
  __device__ static ff ln_p0(const DevMech& m) { return m.ln_p0_over_ru_f; }
  __device__ static ff eff(const DevMech& m, int k, int a) { return m.eff_f[k][a]; }
  __device__ static ff dt_sub(const Units& u) { return u.dt_sub_f; }
  __device__ static ff of(float v) { return ff(v); }
  __device__ static ff of_T(double T) { return ff_from_double(T); }
  template <int M>
  __device__ static ff newton(const DevMech& m, const ff (&r)[M], ff rho, ff U, ff T,
                              const Units& un, bool& ok) {
    ff Ys[M];
#pragma unroll
    for (int a = 0; a < M; ++a) Ys[a] = r[a] / rho;
    return newton_T_ff<M>(m, Ys, U, T, un.newton_max_iter, un.newton_rtol_f, ok);
  }
};

template <typename RT> struct ChemType { using type = double; };
template <> struct ChemType<float> { using type = ff; };

// warp scratch entries of k_chem: r, C, G per species and q per reaction
constexpr int kChemScratch = 3 * LBM_MAX_SPECIES + LBM_MAX_REACTIONS;

template <int D, int M, typename RT>
__device__ __forceinline__ void chem_warp_body(RT* __restrict__ rec,
                                               const double* __restrict__ Tf,
                                               int* __restrict__ status, long long N,
                                               const int* __restrict__ tag, const Units& un,
                                               const DevMech& m, long long n, int lane,
                                               typename ChemType<RT>::type* __restrict__ sc) {
  using CT = typename ChemType<RT>::type;
  using X = Chem<CT>;
  using RC = Rec<D, M>;
  if (n >= N) return;
  if (tag && tag[n] == TAG_SOLID) return;
  CT* r = sc;
  CT* C = sc + LBM_MAX_SPECIES;
  CT* G = sc + 2 * LBM_MAX_SPECIES;
  CT* q = sc + 3 * LBM_MAX_SPECIES;
  // the node's post-stream species densities and internal energy, as the
  // moments kernel formed them
  const RT rho = rec[RC::RHO * N + n];
  RT usq = RT(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const RT ud = rec[(RC::U + d) * N + n];
    usq += ud * ud;
  }
  const RT ER = rec[RC::E * N + n];
  CT U;
  if constexpr (sizeof(RT) == 4) U = (ff(ER) + ff(-0.5f * usq)) * un.c2_f;
  else U = (double(ER) - 0.5 * double(usq)) * un.c * un.c;
  CT r0 = CT();
  if (lane < M - 1) {
    const RT v = rec[(RC::DRHO + lane) * N + n];
    r0 = X::of(v);
    r[lane] = r0;
  } else if (lane == M - 1) {
    RT last = rho;
#pragma unroll
    for (int a = 0; a < M - 1; ++a) last -= rec[(RC::DRHO + a) * N + n];
    r[lane] = X::of(last);
  }
  __syncwarp();
  const CT rho_c = X::of(rho);
  CT Ts = X::of_T(Tf[n]);
  for (int s = 0; s < un.substeps; ++s) {
    if (s > 0) {
      CT rl[M];
#pragma unroll
      for (int a = 0; a < M; ++a) rl[a] = r[a];
      bool ok;
      Ts = X::template newton<M>(m, rl, rho_c, U, Ts, un, ok);
      if (!ok && lane == 0) atomicOr(status, ST_NEWTON);
    }
    const CT lnT = X::ln(Ts);
    const CT invT = X::inv(Ts);
    if (lane < M) {
      C[lane] = r[lane] * X::inv_mm(m, lane);
      G[lane] = X::gibbs(m, lane, Ts, invT, lnT);
    }
    __syncwarp();
    const CT lp = X::ln_p0(m) - lnT;   // ln(P0 / (R_U T))
    for (int k = lane; k < m.R; k += 32) {
      const DevReaction& rx = m.rx[k];
      const CT lk = X::lnkf(rx, lnT, invT);
      CT fwd = X::ex(lk);
      for (int j = 0; j < rx.nr; ++j) fwd *= C[rx.reac[j]];
      CT rev = CT();
      if (rx.reversible) {
        CT dG = CT();
        for (int j = 0; j < rx.np; ++j) dG += G[rx.prod[j]];
        for (int j = 0; j < rx.nr; ++j) dG -= G[rx.reac[j]];
        rev = X::ex(X::rev_arg(rx, lk, dG, lp));
        for (int j = 0; j < rx.np; ++j) rev *= C[rx.prod[j]];
      }
      CT qk = fwd - rev;
      if (rx.third_body) {
        CT cm = CT();
#pragma unroll
        for (int a = 0; a < M; ++a) cm += X::eff(m, k, a) * C[a];
        qk *= cm;
      }
      q[k] = qk;
    }
    __syncwarp();
    if (lane < M) {
      CT w = CT();
      for (int k = 0; k < m.R; ++k) {
        const DevReaction& rx = m.rx[k];
        for (int j = 0; j < rx.nr; ++j)
          if (rx.reac[j] == lane) w -= q[k];
        for (int j = 0; j < rx.np; ++j)
          if (rx.prod[j] == lane) w += q[k];
      }
      r[lane] += X::dt_sub(un) * (w * X::mm(m, lane));
    }
    __syncwarp();
  }
  if (lane < M - 1) {
    if constexpr (sizeof(RT) == 4) rec[(RC::DRHO + lane) * N + n] = (r[lane] - r0).hi;
    else rec[(RC::DRHO + lane) * N + n] = RT(r[lane] - r0);
  }
}

// Transport and lattice constants in the parameter type: FP64 for the FP64
// path, FP32 for the mixed path.
template <typename PT> struct MixParams;
template <> struct MixParams<double> {
  __device__ static double inv_mm(const DevMech& m, int a) { return m.inv_mm[a]; }
  __device__ static double Ra(const DevMech& m, int a) { return m.Ra[a]; }
  __device__ static double D_T_exp(const DevMech& m) { return m.D_T_exp; }
  __device__ static double mu0(const DevMech& m) { return m.mu0; }
  __device__ static double mu_T_exp(const DevMech& m) { return m.mu_T_exp; }
  __device__ static double inv_prandtl(const DevMech& m) { return m.inv_prandtl; }
  __device__ static double inv_c2(const Units& u) { return u.inv_c2; }
  __device__ static double s_pref(const Units& u) { return u.s_pref; }
  __device__ static double nu_pref(const Units& u) { return u.nu_pref; }
};
template <> struct MixParams<float> {
  __device__ static float inv_mm(const DevMech& m, int a) { return m.inv_mm_s[a]; }
  __device__ static float Ra(const DevMech& m, int a) { return m.Ra_s[a]; }
  __device__ static float D_T_exp(const DevMech& m) { return m.D_T_exp_s; }
  __device__ static float mu0(const DevMech& m) { return m.mu0_s; }
  __device__ static float mu_T_exp(const DevMech& m) { return m.mu_T_exp_s; }
  __device__ static float inv_prandtl(const DevMech& m) { return m.inv_prandtl_s; }
  __device__ static float inv_c2(const Units& u) { return u.inv_c2_s; }
  __device__ static float s_pref(const Units& u) { return u.s_pref_s; }
  __device__ static float nu_pref(const Units& u) { return u.nu_pref_s; }
};

// ---------------------------------------------------------------------------
// Collision of all lattices (Sec. 2.3 Eq. finalNumericalEquationsReactive;
// Sec. 3.2 Eqs. f, g; Sec. 3.3 Eqs. feqmix, Pex; Sec. 3.4 Eqs. geq_i, gstar,
// gstareq1mom, qdiff, corrFourier, qex; Sec. 2.4 Eq. R3).
template <int D, int M, typename S, typename RT>
__device__ __forceinline__ void collide_body(const S* __restrict__ src, S* __restrict__ dst,
                                             const RT* __restrict__ rec,
                                             const double* __restrict__ Tf,
                                             int* __restrict__ status, const Geom& g,
                                             const Units& un, const BCDev& bc,
                                             const DevMech& mech, long long n) {
  constexpr int Q = Lat<D>::Q, NP = Lat<D>::NP;
  using RC = Rec<D, M>;
  const long long N = g.N;
  if (n >= N) return;
  const int tag = bc.tag ? bc.tag[n] : TAG_BULK;
  if (tag == TAG_SOLID) return;
  const int x = (int)(n % g.nx);
  const int y = (int)((n / g.nx) % g.ny);
  const int z = (int)(n / ((long long)g.nx * g.ny));

  // node scalars in the parameter type PT (FP64 in the FP64 path, FP32 in
  // the mixed path, whose temperature and chemistry run in float-float);
  // lattice-type values (RT) for gradients, the solve and the collision
  using PT = RT;
  using MP = MixParams<PT>;
  const PT rho = PT(rec[RC::RHO * N + n]);
  const double T_d = Tf[n];
  const PT T = PT(T_d);
  const PT E = PT(rec[RC::E * N + n]);
  PT u[D], Y[M];
  RT q[D], P[NP], V[M][D];
  PT usq = PT(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    u[d] = PT(rec[(RC::U + d) * N + n]);
    q[d] = rec[(RC::QF + d) * N + n];
    usq += u[d] * u[d];
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) P[k] = rec[(RC::P + k) * N + n];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    Y[a] = PT(rec[(RC::Y + a) * N + n]);
#pragma unroll
    for (int d = 0; d < D; ++d) V[a][d] = rec[(RC::US + a * D + d) * N + n] - RT(u[d]);
  }

  // isotropic gradients d_a Phi_a and grad Y_a: 3 sum_i w_i c_ia phi(x + c_i)
  RT dPhi[D], gY[M][D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    dPhi[d] = RT(0);
#pragma unroll
    for (int a = 0; a < M; ++a) gY[a][d] = RT(0);
  }
  // ghost values beyond non-periodic faces and on solid nodes: walls Phi = 0,
  // inlet the inlet state's Phi, outlet the node's own Phi; Y the node's own
  RT phi_self[D], phi_in[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    phi_self[d] = RT(0);
    phi_in[d] = RT(0);
  }
  if (bc.tag) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      phi_self[d] = rec[(RC::PHI + d) * N + n];
      const RT ui = tag >= 0 ? RT(bc.if_uin[(long long)d * bc.n_if + tag]) : RT(0);
      const RT rin = RT(bc.rho_in);
      phi_in[d] = rin * ui * (RT(1) - RT(3) * RT(bc.theta_in)) - rin * ui * ui * ui;
    }
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (csq(i, D) == 0) continue;
    long long nb = 0;
    int gk = BK_NONE;
    if (!bc.tag) {
      nb = node_shift<D>(x, y, z, i, +1, g);
    } else {
      int cc[3] = {x + cvel(i, 0), y + cvel(i, 1), D == 3 ? z + cvel(i, 2) : z};
      const int ext[3] = {g.nx, g.ny, g.nz};
#pragma unroll
      for (int a = 0; a < D; ++a) {
        if (cc[a] < 0) {
          if (bc.face[2 * a]) { if (!gk) gk = bc.face[2 * a]; } else cc[a] += ext[a];
        } else if (cc[a] >= ext[a]) {
          if (bc.face[2 * a + 1]) { if (!gk) gk = bc.face[2 * a + 1]; } else cc[a] -= ext[a];
        }
      }
      if (!gk) {
        nb = cc[0] + (long long)g.nx * (cc[1] + (long long)g.ny * cc[2]);
        if (bc.has_solid && bc.tag[nb] == TAG_SOLID) gk = bc.solid_kind;
      }
    }
    const RT w3 = RT(3) * wstd<RT>(i, D);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (cvel(i, d) == 0) continue;
      const RT wc = w3 * RT(cvel(i, d));
      const RT pv = gk == BK_NONE ? __ldg(rec + (RC::PHI + d) * N + nb)
                    : (gk == BK_INLET ? phi_in[d] : (gk == BK_OUTLET ? phi_self[d] : RT(0)));
      dPhi[d] += wc * pv;
#pragma unroll
      for (int a = 0; a < M; ++a)
        gY[a][d] += wc * (gk == BK_NONE ? __ldg(rec + (RC::Y + a) * N + nb) : RT(Y[a]));
    }
  }

  // relaxation parameters (Sec. 2.3 Eqs. betaa, taua; Sec. 3.5 Eqs. mu, lambda)
  PT Rmix = PT(0);
#pragma unroll
  for (int a = 0; a < M; ++a) Rmix += Y[a] * MP::inv_mm(mech, a);
  Rmix *= PT(R_U);
  const PT theta = Rmix * T * MP::inv_c2(un);
  const PT lnTr = log(T * PT(1.0 / T_REF));
  const PT s_tau = MP::s_pref(un) * rho * T * T * exp(-MP::D_T_exp(mech) * lnTr);
  const PT mu = MP::mu0(mech) * exp(MP::mu_T_exp(mech) * lnTr);
  const PT nu = mu / rho * MP::nu_pref(un);
  const PT omega = PT(1) / (nu / theta + PT(0.5));
  const PT omega1 = PT(1) / (nu * MP::inv_prandtl(mech) / theta + PT(0.5));
  PT inv_tau_a[M];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    PT acc = PT(0);
#pragma unroll
    for (int b = 0; b < M; ++b)
      if (b != a) acc += Y[b] * (s_tau * kcoef<PT>(mech, a, b));
    inv_tau_a[a] = acc;
  }

  // diffusion velocities, Eq. transform1: A V = u_a - u  (V holds the rhs).
  // Each thread's matrix lives in shared memory, entry-major with the block's
  // threads contiguous (no bank conflicts): in registers it would not fit
  // beside the node's other state and spills to local memory.
  {
    extern __shared__ unsigned char smem_raw[];
    RT* As = reinterpret_cast<RT*>(smem_raw) + threadIdx.x;
    const int st = kBS;
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
      for (int b = 0; b < M; ++b)
        As[(a * M + b) * st] = RT(a == b ? PT(1) + PT(0.5) * inv_tau_a[a]
                                         : PT(-0.5) * Y[b] * (s_tau * kcoef<PT>(mech, a, b)));
    solve_dd_strided<M, D, RT>(As, st, V);
  }

  // species densities; the reaction increments come from the moments kernel
  PT rs[M];
#pragma unroll
  for (int a = 0; a < M; ++a) rs[a] = rho * Y[a];

  // energy-flux correction W = (omega - omega1)(q* - q^eq), folded form
  const PT U_lat = E - PT(0.5) * usq;
  RT W[D];
  {
    RT diff[D], corr[D];
#pragma unroll
    for (int d = 0; d < D; ++d) { diff[d] = RT(0); corr[d] = RT(0); }
#pragma unroll
    for (int a = 0; a < M; ++a) {
      RT Ha;
      if constexpr (sizeof(RT) == 4) {
        const ff Tf_(T);
        Ha = ((species_U_ff(mech, a, Tf_) + ff(mech.Ra_s[a]) * Tf_) * un.inv_c2_f).hi;
      } else {
        Ha = RT((species_U(mech, a, T_d) + mech.Ra[a] * T_d) * un.inv_c2);
      }
      const RT HY = Ha * RT(Y[a]);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        diff[d] += HY * V[a][d];
        corr[d] += Ha * gY[a][d];
      }
    }
    const RT rhoR = RT(rho), thR = RT(theta), ER = RT(E);
    const RT Pres = rhoR * thR;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const RT ud = RT(u[d]);
      const RT q_eq = rhoR * ud * (ER + thR);
      RT uP = RT(0);
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const RT ub = RT(u[b]);
        const RT Peq = rhoR * ub * ud + (b == d ? Pres : RT(0));
        uP += ub * (P[pidx<D>(b, d)] - Peq);
      }
      const RT q_ex = RT(-0.5) * ud * dPhi[d];
      W[d] = RT(omega - omega1) * (q[d] - q_eq - uP + q_ex) + RT(omega1) * rhoR * diff[d] +
             RT(PT(0.5) * (PT(2) - omega1)) * Pres * corr[d];
    }
  }

  // per-lattice parameters in the collision type
  RT th_a[M], beta[M], Pex[D], uR[D], VR[M][D];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    th_a[a] = RT(MP::Ra(mech, a) * T * MP::inv_c2(un));
    beta[a] = RT(inv_tau_a[a] / (PT(2) + inv_tau_a[a]));
#pragma unroll
    for (int d = 0; d < D; ++d) VR[a][d] = V[a][d];
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    uR[d] = RT(u[d]);
    Pex[d] = RT(theta + u[d] * u[d] + (PT(2) - omega) / (PT(2) * rho * omega) * PT(dPhi[d]));
  }
  // energy equilibrium axis factors: A_c (acting on 1) and B_c (on u^2/2)
  RT Af[D][3], Bf[D][3];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const PT ua = u[d];
    const PT O1 = theta * ua + PT(0.5) * ua * ua * ua;
    const PT O2 = theta * theta + PT(2.5) * theta * ua * ua + PT(0.5) * ua * ua * ua * ua;
    const PT Pd = theta + ua * ua;
    Af[d][0] = RT(PT(0.5) * (Pd - ua));
    Af[d][1] = RT(PT(1) - Pd);
    Af[d][2] = RT(PT(0.5) * (Pd + ua));
    Bf[d][0] = RT(PT(0.5) * (O2 - O1));
    Bf[d][1] = RT(PT(0.5) * ua * ua - O2);
    Bf[d][2] = RT(PT(0.5) * (O2 + O1));
  }
  const RT rhoR = RT(rho), omR = RT(omega), UR = RT(U_lat);
  // species coefficients of the update, hoisted out of the direction loop:
  // f_a += 2 beta_a (rho_a psi_a - f_a) + cF_a sum_b K_ab d_b + drho_a psi_a
  // with cF_a = (beta_a - 1) Y_a s (1/tau_ab = s K_ab)
  RT rsR[M], cF[M - 1], drR[M - 1], two_beta[M - 1];
#pragma unroll
  for (int b = 0; b < M; ++b) rsR[b] = RT(rs[b]);
#pragma unroll
  for (int a = 0; a < M - 1; ++a) {
    cF[a] = RT((inv_tau_a[a] / (PT(2) + inv_tau_a[a]) - PT(1)) * Y[a] * s_tau);
    drR[a] = rec[(RC::DRHO + a) * N + n];
    two_beta[a] = RT(2) * beta[a];
  }

  // Per-species axis factors of psi(u, theta_b) and psi(u + V_b, theta_b)
  // (Eq. prod), tabulated once per node in this thread's shared-memory column
  // (the solve's space, now free): entry ((set*M + b)*D + d)*3 + c + 1.
  extern __shared__ unsigned char smem_raw[];
  RT* tab = reinterpret_cast<RT*>(smem_raw) + threadIdx.x;
  constexpr bool kTab = sizeof(RT) == 4;
  if constexpr (kTab) {
#pragma unroll
    for (int b = 0; b < M; ++b)
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const RT ud = uR[d], Pe = th_a[b] + ud * ud;
        RT* te = tab + ((b * D + d) * 3) * kBS;
        te[0] = RT(0.5) * (Pe - ud);
        te[kBS] = RT(1) - Pe;
        te[2 * kBS] = RT(0.5) * (Pe + ud);
        const RT xs = ud + VR[b][d], Ps = th_a[b] + xs * xs;
        RT* ts = tab + (((M + b) * D + d) * 3) * kBS;
        ts[0] = RT(0.5) * (Ps - xs);
        ts[kBS] = RT(1) - Ps;
        ts[2 * kBS] = RT(0.5) * (Ps + xs);
      }
  }
#pragma unroll 1
  for (int i = 0; i < Q; ++i) {
    const long long sn = node_shift<D>(x, y, z, i, -1, g);
    int c[3];
    c[0] = cvel(i, 0); c[1] = cvel(i, 1); c[2] = D == 3 ? cvel(i, 2) : 0;
    RT pe[M], dd[M];
    if constexpr (kTab) {
      int off[3];
#pragma unroll
      for (int d = 0; d < D; ++d) off[d] = (d * 3 + c[d] + 1) * kBS;
#pragma unroll
      for (int b = 0; b < M; ++b) {
        const RT* te = tab + b * D * 3 * kBS;
        const RT* ts = tab + (M + b) * D * 3 * kBS;
        RT e = te[off[0]], st = ts[off[0]];
#pragma unroll
        for (int d = 1; d < D; ++d) {
          e *= te[off[d]];
          st *= ts[off[d]];
        }
        pe[b] = e;
        dd[b] = rsR[b] * (e - st);
      }
    } else {
#pragma unroll
      for (int b = 0; b < M; ++b) {
        RT e = RT(1), st = RT(1);
#pragma unroll
        for (int d = 0; d < D; ++d) {
          e *= psi1<RT>(c[d], uR[d], th_a[b] + uR[d] * uR[d]);
          const RT xs = uR[d] + VR[b][d];
          st *= psi1<RT>(c[d], xs, th_a[b] + xs * xs);
        }
        pe[b] = e;
        dd[b] = rsR[b] * (e - st);
      }
    }
#pragma unroll
    for (int a = 0; a < M - 1; ++a) {
      RT F = RT(0);
#pragma unroll
      for (int b = 0; b < M; ++b)
        if (b != a) F += kcoef<RT>(mech, a, b) * dd[b];
      const long long off = (long long)(a * Q + i) * N;
      const RT f = pop_in<RT>(src, bc, tag, N, sn, a * Q + i);
      const RT fn = f + two_beta[a] * (rsR[a] * pe[a] - f) + cF[a] * F + drR[a] * pe[a];
      dst[off + n] = S(fn);
    }
    {
      RT fex = rhoR;
#pragma unroll
      for (int d = 0; d < D; ++d) fex *= psi1<RT>(c[d], uR[d], Pex[d]);
      const long long off = (long long)((M - 1) * Q + i) * N;
      const RT f = pop_in<RT>(src, bc, tag, N, sn, (M - 1) * Q + i);
      dst[off + n] = S(f + omR * (fex - f));
    }
    {
      RT prodA = RT(1);
#pragma unroll
      for (int d = 0; d < D; ++d) prodA *= pick3<RT>(c[d], Af[d]);
      RT geq = UR * prodA;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        RT t = pick3<RT>(c[d], Bf[d]);
#pragma unroll
        for (int e = 0; e < D; ++e)
          if (e != d) t *= pick3<RT>(c[e], Af[e]);
        geq += t;
      }
      geq *= rhoR;
      const long long off = (long long)(M * Q + i) * N;
      const RT gv = pop_in<RT>(src, bc, tag, N, sn, M * Q + i);
      RT gn = gv + omR * (geq - gv);
      if (csq(i, D) == 1) {
#pragma unroll
        for (int d = 0; d < D; ++d)
          if (c[d] != 0) gn += (c[d] > 0 ? RT(0.5) : RT(-0.5)) * W[d];
      }
      dst[off + n] = S(gn);
    }
  }
}


// ---------------------------------------------------------------------------
// Boundary reconstruction at interface nodes (Sec. 4).  One warp per
// interface node: lanes stride over the node's L*Q populations, moment sums
// are reduced with warp shuffles, and the per-node scalars (local state,
// Newton temperature, LODI data) are evaluated redundantly by every lane.
// Writes the node's full post-boundary population set to bc.pops, which the
// moments and collision kernels read for that node.
//   bounce-back (Eq. bb): incoming f_i = f_{-i}^post of the node itself;
//   TMS wall (Sec. 4.2.2), flux inlet (Sec. 4.3), outlet (Sec. 4.4): put
//   the first equilibrium A on the incoming links, take the local state
//   `loc` of the result, then every population becomes B + f - f^loc with
//   B = A (wall: target; outlet: outlet data) or, for the inlet, the
//   target equilibrium at (rho^loc, Y^loc, u^in, T^in).

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp-cooperative state_of: every lane returns the same state.
template <int D, int M, typename F>
__device__ void warp_state_of(F fetch, EqSet<D, M>& s, double T_guess, const DevMech& m,
                              const Units& un, int* status, int lane) {
  constexpr int Q = Lat<D>::Q, L = M + 1;
  double rho = 0.0, rhoE = 0.0, j[D], rs[M], js[M][D];
  for (int d = 0; d < D; ++d) j[d] = 0.0;
  for (int a = 0; a < M; ++a) {
    rs[a] = 0.0;
    for (int d = 0; d < D; ++d) js[a][d] = 0.0;
  }
  for (int t = lane; t < L * Q; t += 32) {
    const int l = t / Q, i = t % Q;
    const double v = fetch(l, i);
    if (l < M - 1) {
      rs[l] += v;
      for (int d = 0; d < D; ++d) js[l][d] += cvel(i, d) * v;
    } else if (l == M - 1) {
      rho += v;
      for (int d = 0; d < D; ++d) j[d] += cvel(i, d) * v;
    } else {
      rhoE += v;
    }
  }
  rho = warp_sum(rho);
  rhoE = warp_sum(rhoE);
  for (int d = 0; d < D; ++d) j[d] = warp_sum(j[d]);
  for (int a = 0; a < M - 1; ++a) {
    rs[a] = warp_sum(rs[a]);
    for (int d = 0; d < D; ++d) js[a][d] = warp_sum(js[a][d]);
  }
  rs[M - 1] = rho;
  for (int d = 0; d < D; ++d) js[M - 1][d] = j[d];
  for (int a = 0; a < M - 1; ++a) {
    rs[M - 1] -= rs[a];
    for (int d = 0; d < D; ++d) js[M - 1][d] -= js[a][d];
  }
  s.rho = rho;
  double usq = 0.0;
  for (int d = 0; d < D; ++d) { s.u[d] = j[d] / rho; usq += s.u[d] * s.u[d]; }
  for (int a = 0; a < M; ++a) {
    s.Y[a] = rs[a] / rho;
    const bool tiny = species_velocity_undefined<D, double>(rs[a], js[a]);
    for (int d = 0; d < D; ++d) s.us[a][d] = tiny ? s.u[d] : js[a][d] / rs[a];
  }
  const double U = (rhoE / rho - 0.5 * usq) * un.c * un.c;
  bool ok;
  s.T = newton_T<M>(m, s.Y, U, T_guess, un.newton_max_iter, un.newton_rtol, ok);
  if (!ok && lane == 0) atomicOr(status, ST_NEWTON);
}

template <int D, int M, typename S>
__device__ __forceinline__ void boundary_body(const S* __restrict__ src, const BCDev& bc,
                                              const double* __restrict__ Tf,
                                              int* __restrict__ status, const Geom& g,
                                              const Units& un, const DevMech& mech, int k,
                                              int lane) {
  constexpr int Q = Lat<D>::Q, L = M + 1;
  if (k >= bc.n_if) return;                                         // whole warp leaves
  const long long N = g.N;
  const long long n = bc.if_node[k];
  const int info = bc.if_info[k];
  const int kind = info & 15;
  const unsigned inc = bc.if_inc[k];
  const int x = (int)(n % g.nx);
  const int y = (int)((n / g.nx) % g.ny);
  const int z = (int)(n / ((long long)g.nx * g.ny));
  const long long st = bc.n_if;
  double* P = bc.pops + k;                       // element (l, i) at P[(l Q + i) st]
  for (int t = lane; t < L * Q; t += 32) {       // pull streaming (wrapped address)
    const int l = t / Q, i = t % Q;
    const long long sn = node_shift<D>(x, y, z, i, -1, g);
    P[(long long)t * st] = (inc >> i & 1u) && kind == BK_BB
                               ? ldp(src + (long long)(l * Q + (Q - 1 - i)) * N + n)
                               : ldp(src + (long long)t * N + sn);
  }
  if (kind == BK_BB) return;
  __syncwarp();
  EqSet<D, M> A, B, loc;
  A.own_species_u = B.own_species_u = false;
  if (kind == BK_TMS) {
    // step 1: bounce-back density and mass fractions (Eqs. BBrho, BBY)
    double rho_bb = 0.0, rs[M];
    for (int a = 0; a < M - 1; ++a) rs[a] = 0.0;
    for (int t = lane; t < M * Q; t += 32) {
      const int l = t / Q, i = t % Q;
      const double v = (inc >> i & 1u) ? ldp(src + (long long)(l * Q + (Q - 1 - i)) * N + n)
                                       : P[(long long)t * st];
      if (l < M - 1) rs[l] += v; else rho_bb += v;
    }
    rho_bb = warp_sum(rho_bb);
    for (int a = 0; a < M - 1; ++a) rs[a] = warp_sum(rs[a]);
    A.rho = rho_bb;
    double ysum = 0.0;
    for (int a = 0; a < M - 1; ++a) { A.Y[a] = rs[a] / rho_bb; ysum += A.Y[a]; }
    A.Y[M - 1] = 1.0 - ysum;
    for (int d = 0; d < D; ++d) A.u[d] = 0.0;      // u^tgt = u_a^tgt = 0
    A.T = bc.if_wallT[k];
    eq_prepare(A, mech, un);                         // step 2: target (Eqs. tgtf-tgtfa)
  } else if (kind == BK_INLET) {
    A.rho = bc.rho_in;
    for (int a = 0; a < M; ++a) A.Y[a] = bc.Y_in[a];
    for (int d = 0; d < D; ++d) A.u[d] = bc.if_uin[(long long)d * st + k];
    A.T = bc.T_in;
    eq_prepare(A, mech, un);                         // step 1 (Eqs. in_f-in_fa)
  } else {
    // LODI data from the stored state at x and x - n (Eq. convectiveBC)
    const int ax = (info >> 4) & 3;
    const int sg = (info >> 6) & 1 ? 1 : -1;
    const long long stride = ax == 0 ? 1 : (ax == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
    const long long up = n - sg * stride;
    EqSet<D, M> s0, s1;
    warp_state_of<D, M>([&](int l, int i) { return ldp(src + (long long)(l * Q + i) * N + n); },
                        s0, Tf[n], mech, un, status, lane);
    warp_state_of<D, M>([&](int l, int i) { return ldp(src + (long long)(l * Q + i) * N + up); },
                        s1, Tf[up], mech, un, status, lane);
    double R0 = 0.0, R1 = 0.0, Cv = 0.0;
    for (int a = 0; a < M; ++a) {
      R0 += s0.Y[a] * mech.inv_mm[a];
      R1 += s1.Y[a] * mech.inv_mm[a];
      Cv += s0.Y[a] * (mech.u1[a] + s0.T * (2.0 * mech.u2[a] + 3.0 * s0.T * mech.u3[a]));
    }
    R0 *= R_U;
    R1 *= R_U;
    const double p0 = s0.rho * R0 * s0.T * un.inv_c2;
    const double p1 = s1.rho * R1 * s1.T * un.inv_c2;
    const double un0 = sg * s0.u[ax], un1 = sg * s1.u[ax];
    const double gamma = (Cv + R0) / Cv;
    const double cs = sqrt(gamma * R0 * s0.T * un.inv_c2);
    const double Ma = un0 / cs;
    const double Ln = ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz);
    const double K = bc.sigma * (1.0 - Ma * Ma) * cs / Ln;
    const double L1 = K * (p0 - bc.p_out_lat);
    const double L2 = un0 * (cs * cs * (s0.rho - s1.rho) - (p0 - p1));
    const double L5 = (un0 + cs) * ((p0 - p1) + s0.rho * cs * (un0 - un1));
    A.rho = s0.rho - (L2 + 0.5 * (L5 + L1)) / (cs * cs);
    const double p_o = p0 - 0.5 * (L5 + L1);
    const double un_o = un0 - (L5 - L1) / (2.0 * s0.rho * cs);
    for (int d = 0; d < D; ++d) A.u[d] = s0.u[d] - un0 * (s0.u[d] - s1.u[d]);
    A.u[ax] = sg * un_o;
    double Ro = 0.0;
    for (int a = 0; a < M; ++a) {
      A.Y[a] = s0.Y[a] - un0 * (s0.Y[a] - s1.Y[a]);
      Ro += A.Y[a] * mech.inv_mm[a];
    }
    A.T = p_o * un.c * un.c / (A.rho * R_U * Ro);
    eq_prepare(A, mech, un);                         // step 1 (Eqs. out_f-out_fa)
  }
  // incoming links at A, then the local state (Eqs. locRho-locT and analogues)
  for (int t = lane; t < L * Q; t += 32) {
    const int l = t / Q, i = t % Q;
    if (inc >> i & 1u) P[(long long)t * st] = eq_pop(A, l, i);
  }
  __syncwarp();
  warp_state_of<D, M>([&](int l, int i) { return P[(long long)(l * Q + i) * st]; }, loc,
                      Tf[n], mech, un, status, lane);
  loc.own_species_u = kind == BK_TMS;             // TMS local species use u_a^loc
  eq_prepare(loc, mech, un);
  if (kind == BK_INLET) {                         // target (Eqs. in_tgt_*)
    B.rho = loc.rho;
    for (int a = 0; a < M; ++a) B.Y[a] = loc.Y[a];
    for (int d = 0; d < D; ++d) B.u[d] = A.u[d];
    B.T = bc.T_in;
    eq_prepare(B, mech, un);
  }
  const EqSet<D, M>& Bref = kind == BK_INLET ? B : A;
  __syncwarp();
  for (int t = lane; t < L * Q; t += 32) {
    const int l = t / Q, i = t % Q;
    double& p = P[(long long)t * st];
    p = eq_pop(Bref, l, i) + p - eq_pop(loc, l, i);
  }
}

// ---------------------------------------------------------------------------
// Single-domain kernels: one thread per node (moments, collision), one warp
// per interface node (boundary).
template <int D, int M, typename S, typename RT>
__global__ void __launch_bounds__(128)
k_moments(const S* __restrict__ src, RT* __restrict__ rec, double* __restrict__ Tf,
          int* __restrict__ status, const __grid_constant__ Geom g,
          const __grid_constant__ Units un, const __grid_constant__ BCDev bc,
          const __grid_constant__ DevMech mech, int chem_inline) {
  moments_body<D, M, S, RT>(src, rec, Tf, status, g, un, bc, mech,
                            blockIdx.x * (long long)blockDim.x + threadIdx.x, chem_inline);
}

// one warp per node, kChemWarps nodes per block
constexpr int kChemWarps = kChemNodesPerBlock;

template <int D, int M, typename RT>
__global__ void __launch_bounds__(32 * kChemWarps)
k_chem(RT* __restrict__ rec, const double* __restrict__ Tf, int* __restrict__ status,
       long long N, const int* __restrict__ tag, const __grid_constant__ Units un,
       const DevMech* __restrict__ mech) {
  using CT = typename ChemType<RT>::type;
  __shared__ __align__(16) unsigned char raw[kChemWarps * kChemScratch * sizeof(CT)];
  const int w = threadIdx.x >> 5;
  chem_warp_body<D, M, RT>(rec, Tf, status, N, tag, un, *mech,
                           blockIdx.x * (long long)kChemWarps + w, threadIdx.x & 31,
                           reinterpret_cast<CT*>(raw) + w * kChemScratch);
}

template <int D, int M, typename S, typename RT>
__global__ void __launch_bounds__(128)
k_collide(const S* __restrict__ src, S* __restrict__ dst, const RT* __restrict__ rec,
          const double* __restrict__ Tf, int* __restrict__ status,
          const __grid_constant__ Geom g, const __grid_constant__ Units un,
          const __grid_constant__ BCDev bc, const __grid_constant__ DevMech mech) {
  collide_body<D, M, S, RT>(src, dst, rec, Tf, status, g, un, bc, mech,
                            blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

template <int D, int M, typename S>
__global__ void __launch_bounds__(128)
k_boundary(const S* __restrict__ src, const __grid_constant__ BCDev bc,
           const double* __restrict__ Tf, int* __restrict__ status,
           const __grid_constant__ Geom g, const __grid_constant__ Units un,
           const __grid_constant__ DevMech mech) {
  boundary_body<D, M, S>(src, bc, Tf, status, g, un, mech,
                         blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// Batched kernels: the grid is the concatenation of every domain's tiles; a
// block finds its domain by binary search over the domains' first blocks.
// grid: 0 = node kernels, 1 = boundary kernel, 2 = warp-per-node chemistry
__device__ __forceinline__ int domain_of_block(const DomainDev* __restrict__ d, int ndom,
                                               int b, int grid) {
  int lo = 0, hi = ndom - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int first = grid == 1 ? d[mid].bblock_begin
                                : (grid == 2 ? d[mid].cblock_begin : d[mid].block_begin);
    if (first <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int D, int M, typename S, typename RT>
__global__ void __launch_bounds__(128)
k_moments_batch(const DomainDev* __restrict__ doms, int ndom, int parity, int chem_inline) {
  const DomainDev& d = doms[domain_of_block(doms, ndom, blockIdx.x, 0)];
  const int c = d.cur0 ^ parity;
  moments_body<D, M, S, RT>(static_cast<const S*>(d.pops[c]), static_cast<RT*>(d.rec), d.Tf,
                            d.status, d.g, d.un, d.bc, *d.mech,
                            (blockIdx.x - d.block_begin) * (long long)blockDim.x + threadIdx.x,
                            chem_inline);
}

template <int D, int M, typename RT>
__global__ void __launch_bounds__(32 * kChemWarps)
k_chem_batch(const DomainDev* __restrict__ doms, int ndom) {
  using CT = typename ChemType<RT>::type;
  __shared__ __align__(16) unsigned char raw[kChemWarps * kChemScratch * sizeof(CT)];
  const DomainDev& d = doms[domain_of_block(doms, ndom, blockIdx.x, 2)];
  const int w = threadIdx.x >> 5;
  chem_warp_body<D, M, RT>(static_cast<RT*>(d.rec), d.Tf, d.status, d.g.N, d.bc.tag, d.un,
                           *d.mech,
                           (blockIdx.x - d.cblock_begin) * (long long)kChemWarps + w,
                           threadIdx.x & 31, reinterpret_cast<CT*>(raw) + w * kChemScratch);
}

template <int D, int M, typename S, typename RT>
__global__ void __launch_bounds__(128)
k_collide_batch(const DomainDev* __restrict__ doms, int ndom, int parity) {
  const DomainDev& d = doms[domain_of_block(doms, ndom, blockIdx.x, 0)];
  const int c = d.cur0 ^ parity;
  collide_body<D, M, S, RT>(static_cast<const S*>(d.pops[c]),
                            static_cast<S*>(const_cast<void*>(d.pops[1 - c])),
                            static_cast<const RT*>(d.rec), d.Tf, d.status, d.g, d.un, d.bc,
                            *d.mech,
                            (blockIdx.x - d.block_begin) * (long long)blockDim.x + threadIdx.x);
}

template <int D, int M, typename S>
__global__ void __launch_bounds__(128)
k_boundary_batch(const DomainDev* __restrict__ doms, int ndom, int parity) {
  const DomainDev& d = doms[domain_of_block(doms, ndom, blockIdx.x, 1)];
  const int c = d.cur0 ^ parity;
  boundary_body<D, M, S>(static_cast<const S*>(d.pops[c]), d.bc, d.Tf, d.status, d.g, d.un,
                         *d.mech, (blockIdx.x - d.bblock_begin) * 4 + threadIdx.x / 32,
                         threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// Initial populations at the equilibria of (rho or P, u, T, Y).
template <int D, int M, typename S>
__global__ void k_init(const double* __restrict__ rho_or_P, int is_pressure,
                       const double* __restrict__ uin, const double* __restrict__ Tin,
                       const double* __restrict__ Yin, S* __restrict__ pops,
                       double* __restrict__ Tf, int* __restrict__ status, Geom g, Units un,
                       const __grid_constant__ DevMech mech) {
  constexpr int Q = Lat<D>::Q;
  const long long N = g.N;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double T = Tin[n];
  double Y[M], Rmix = 0.0, U = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    Y[a] = Yin[a * N + n];
    Rmix += Y[a] * mech.inv_mm[a];
    U += Y[a] * species_U(mech, a, T);
  }
  Rmix *= R_U;
  const double rho = is_pressure ? rho_or_P[n] / (Rmix * T) : rho_or_P[n];
  if (!(rho > 0.0) || !isfinite(rho) || !(T > 0.0)) atomicOr(status, ST_NONFINITE);
  double u[D], usq = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) { u[d] = uin[d * N + n] * un.inv_c; usq += u[d] * u[d]; }
  const double theta = Rmix * T * un.inv_c2;
  const double U_lat = U * un.inv_c2;
  for (int i = 0; i < Q; ++i) {
    int c[3] = {cvel(i, 0), cvel(i, 1), D == 3 ? cvel(i, 2) : 0};
    for (int a = 0; a < M - 1; ++a) {
      const double th = mech.Ra[a] * T * un.inv_c2;
      double p = rho * Y[a];
      for (int d = 0; d < D; ++d) p *= psi1<double>(c[d], u[d], th + u[d] * u[d]);
      pops[(long long)(a * Q + i) * N + n] = S(p);
    }
    double f = rho;
    for (int d = 0; d < D; ++d) f *= psi1<double>(c[d], u[d], theta + u[d] * u[d]);
    pops[(long long)((M - 1) * Q + i) * N + n] = S(f);
    double prodA = 1.0, sumB = 0.0;
    double A[3], B[3];
    for (int d = 0; d < D; ++d) {
      const double ua = u[d];
      const double O1 = theta * ua + 0.5 * ua * ua * ua;
      const double O2 = theta * theta + 2.5 * theta * ua * ua + 0.5 * ua * ua * ua * ua;
      A[d] = psi1<double>(c[d], ua, theta + ua * ua);
      B[d] = c[d] == 0 ? 0.5 * ua * ua - O2 : 0.5 * (O2 + c[d] * O1);
      prodA *= A[d];
    }
    for (int d = 0; d < D; ++d) {
      double t = B[d];
      for (int e = 0; e < D; ++e)
        if (e != d) t *= A[e];
      sumB += t;
    }
    pops[(long long)(M * Q + i) * N + n] = S(rho * (U_lat * prodA + sumB));
  }
  (void)usq;
  Tf[n] = T;
}

// ---------------------------------------------------------------------------
// Fields of the stored state: rho, u (m/s), T (Newton, not stored), Y, E (J/kg).
template <int D, int M, typename S>
__global__ void k_out(const S* __restrict__ pops, const double* __restrict__ Tf,
                      double* __restrict__ orho, double* __restrict__ ou,
                      double* __restrict__ oT, double* __restrict__ oY,
                      double* __restrict__ oE, int* __restrict__ status, Geom g, Units un,
                      const __grid_constant__ DevMech mech) {
  constexpr int Q = Lat<D>::Q;
  const long long N = g.N;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= N) return;
  double rho = 0.0, rhoE = 0.0, j[D], rs[M];
  for (int d = 0; d < D; ++d) j[d] = 0.0;
  for (int a = 0; a < M; ++a) rs[a] = 0.0;
  for (int i = 0; i < Q; ++i) {
    for (int a = 0; a < M - 1; ++a) rs[a] += ldp(pops + (long long)(a * Q + i) * N + n);
    const double f = ldp(pops + (long long)((M - 1) * Q + i) * N + n);
    rho += f;
    for (int d = 0; d < D; ++d) j[d] += cvel(i, d) * f;
    rhoE += ldp(pops + (long long)(M * Q + i) * N + n);
  }
  rs[M - 1] = rho;
  for (int a = 0; a < M - 1; ++a) rs[M - 1] -= rs[a];
  double Y[M], u[D], usq = 0.0;
  for (int a = 0; a < M; ++a) Y[a] = rs[a] / rho;
  for (int d = 0; d < D; ++d) { u[d] = j[d] / rho; usq += u[d] * u[d]; }
  const double E = rhoE / rho;
  bool ok;
  const double T = newton_T<M>(mech, Y, (E - 0.5 * usq) * un.c * un.c, Tf[n],
                               un.newton_max_iter, un.newton_rtol, ok);
  if (!ok) atomicOr(status, ST_NEWTON);
  if (orho) orho[n] = rho;
  if (ou) {
    for (int d = 0; d < 3; ++d) ou[d * N + n] = d < D ? u[d] * un.c : 0.0;
  }
  if (oT) oT[n] = T;
  if (oY)
    for (int a = 0; a < M; ++a) oY[a * N + n] = Y[a];
  if (oE) oE[n] = E * un.c * un.c;
}

template <typename S>
__global__ void k_to_fp64(const S* __restrict__ in, double* __restrict__ out, long long count) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x)
    out[k] = static_cast<double>(in[k]);
}

// ---------------------------------------------------------------------------
// dispatch

static inline unsigned blocks_for(long long N, int bs) { return (unsigned)((N + bs - 1) / bs); }

template <int D, int M, typename S, typename RT>
static cudaError_t step_impl(const DevMech& mech, const StepArgs& a, cudaStream_t s,
                             int which) {
  const int bs = 128;
  const unsigned nb = blocks_for(a.g.N, bs);
  if (which != 1) {
    if (a.bc.n_if > 0)
      k_boundary<D, M, S><<<(a.bc.n_if + 3) / 4, 128, 0, s>>>(
          static_cast<const S*>(a.src), a.bc, a.Tfield, a.status, a.g, a.un, mech);
    const int chem_warp = a.chem_warp && a.mech_dev;
    k_moments<D, M, S, RT><<<nb, bs, 0, s>>>(static_cast<const S*>(a.src),
                                             reinterpret_cast<RT*>(a.rec), a.Tfield,
                                             a.status, a.g, a.un, a.bc, mech, !chem_warp);
    if (chem_warp)
      k_chem<D, M, RT><<<blocks_for(a.g.N, kChemWarps), 32 * kChemWarps, 0, s>>>(
          reinterpret_cast<RT*>(a.rec), a.Tfield, a.status, a.g.N, a.bc.tag, a.un, a.mech_dev);
  }
  if (which != 0) {
    const size_t smem = (size_t)collide_smem_entries<D, M, RT>() * bs * sizeof(RT);
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(
          k_collide<D, M, S, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_collide<D, M, S, RT><<<nb, bs, smem, s>>>(
                                             static_cast<const S*>(a.src),
                                             static_cast<S*>(a.dst),
                                             reinterpret_cast<const RT*>(a.rec), a.Tfield,
                                             a.status, a.g, a.un, a.bc, mech);
  }
  return cudaGetLastError();
}

#define LBM_DISPATCH(D_, M_, CALL)                                 \
  if (D == D_ && M == M_) {                                        \
    if (prec == LBM_FP64) return CALL(D_, M_, double, double);     \
    if (prec == LBM_FP32_STORE) return CALL(D_, M_, float, float); \
  }

cudaError_t launch_step(int D, int M, lbm_precision prec, const DevMech& mech,
                        const StepArgs& a, cudaStream_t s, int which) {
#define CALL_STEP(D_, M_, S_, R_) step_impl<D_, M_, S_, R_>(mech, a, s, which)
  LBM_DISPATCH(3, 9, CALL_STEP)
  LBM_DISPATCH(3, 2, CALL_STEP)
  LBM_DISPATCH(2, 9, CALL_STEP)
  LBM_DISPATCH(2, 2, CALL_STEP)
#undef CALL_STEP
  return cudaErrorInvalidValue;
}

cudaError_t launch_init(int D, int M, lbm_precision prec, const DevMech& mech,
                        const Geom& g, const Units& un, const double* rho_or_P,
                        int is_pressure, const double* u, const double* T,
                        const double* Y, void* pops, double* Tfield, int* status,
                        cudaStream_t s) {
  const unsigned nb = blocks_for(g.N, 128);
#define CALL_INIT(D_, M_, S_, R_)                                                       \
  (k_init<D_, M_, S_><<<nb, 128, 0, s>>>(rho_or_P, is_pressure, u, T, Y,               \
                                         static_cast<S_*>(pops), Tfield, status, g, un, \
                                         mech),                                         \
   cudaGetLastError())
  LBM_DISPATCH(3, 9, CALL_INIT)
  LBM_DISPATCH(3, 2, CALL_INIT)
  LBM_DISPATCH(2, 9, CALL_INIT)
  LBM_DISPATCH(2, 2, CALL_INIT)
#undef CALL_INIT
  return cudaErrorInvalidValue;
}

cudaError_t launch_moments_out(int D, int M, lbm_precision prec, const DevMech& mech,
                               const Geom& g, const Units& un, const void* pops,
                               const double* Tfield, double* rho, double* u, double* T,
                               double* Y, double* E, int* status, cudaStream_t s) {
  const unsigned nb = blocks_for(g.N, 128);
#define CALL_OUT(D_, M_, S_, R_)                                                         \
  (k_out<D_, M_, S_><<<nb, 128, 0, s>>>(static_cast<const S_*>(pops), Tfield, rho, u, T, \
                                        Y, E, status, g, un, mech),                      \
   cudaGetLastError())
  LBM_DISPATCH(3, 9, CALL_OUT)
  LBM_DISPATCH(3, 2, CALL_OUT)
  LBM_DISPATCH(2, 9, CALL_OUT)
  LBM_DISPATCH(2, 2, CALL_OUT)
#undef CALL_OUT
  return cudaErrorInvalidValue;
}

cudaError_t launch_to_fp64(lbm_precision prec, const void* pops, double* out,
                           long long count, cudaStream_t s) {
  const unsigned nb = (unsigned)std::min<long long>(blocks_for(count, 256), 152LL * 16);
  if (prec == LBM_FP64)
    k_to_fp64<double><<<nb, 256, 0, s>>>(static_cast<const double*>(pops), out, count);
  else if (prec == LBM_FP32_STORE)
    k_to_fp64<float><<<nb, 256, 0, s>>>(static_cast<const float*>(pops), out, count);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <int D, int M, typename S, typename RT>
static cudaError_t batch_impl(const DomainDev* doms, int ndom, int nblocks, int nbblocks,
                              int ncblocks, int parity, cudaStream_t s) {
  const int bs = 128;
  if (nbblocks > 0)
    k_boundary_batch<D, M, S><<<nbblocks, bs, 0, s>>>(doms, ndom, parity);
  k_moments_batch<D, M, S, RT><<<nblocks, bs, 0, s>>>(doms, ndom, parity, ncblocks == 0);
  if (ncblocks > 0)
    k_chem_batch<D, M, RT><<<ncblocks, 32 * kChemWarps, 0, s>>>(doms, ndom);
  const size_t smem = (size_t)collide_smem_entries<D, M, RT>() * bs * sizeof(RT);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_collide_batch<D, M, S, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_collide_batch<D, M, S, RT><<<nblocks, bs, smem, s>>>(doms, ndom, parity);
  return cudaGetLastError();
}

template <int D, int M, typename S, typename RT>
static cudaError_t batch_prepare_impl() {
  const size_t smem = (size_t)collide_smem_entries<D, M, RT>() * 128 * sizeof(RT);
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k_collide_batch<D, M, S, RT>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t prepare_batch_step(int D, int M, lbm_precision prec) {
#define CALL_PREP(D_, M_, S_, R_) batch_prepare_impl<D_, M_, S_, R_>()
  LBM_DISPATCH(3, 9, CALL_PREP)
  LBM_DISPATCH(3, 2, CALL_PREP)
  LBM_DISPATCH(2, 9, CALL_PREP)
  LBM_DISPATCH(2, 2, CALL_PREP)
#undef CALL_PREP
  return cudaErrorInvalidValue;
}

cudaError_t launch_batch_step(int D, int M, lbm_precision prec, const DomainDev* doms,
                              int ndom, int nblocks, int nbblocks, int ncblocks, int parity,
                              cudaStream_t s) {
#define CALL_BATCH(D_, M_, S_, R_) \
  batch_impl<D_, M_, S_, R_>(doms, ndom, nblocks, nbblocks, ncblocks, parity, s)
  LBM_DISPATCH(3, 9, CALL_BATCH)
  LBM_DISPATCH(3, 2, CALL_BATCH)
  LBM_DISPATCH(2, 9, CALL_BATCH)
  LBM_DISPATCH(2, 2, CALL_BATCH)
#undef CALL_BATCH
  return cudaErrorInvalidValue;
}

int record_fields(int D, int M) {
  if (D == 3) {
    if (M == 9) return Rec<3, 9>::NF;
    if (M == 2) return Rec<3, 2>::NF;
  } else {
    if (M == 9) return Rec<2, 9>::NF;
    if (M == 2) return Rec<2, 2>::NF;
  }
  return -1;
}

}  // namespace lbm
