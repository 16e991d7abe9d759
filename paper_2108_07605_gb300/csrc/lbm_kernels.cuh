// Kernels of the reactive-mixture LBM step (templates; instantiated per
// lattice, species count and precision by lbm_inst.cu).
//
//   k_bnode     one thread per interface node: gather, bounce-back / TMS /
//               inlet / LODI outlet reconstruction, the node's moment record
//               (lbm_bnode.cuh).
//   k_iface_chem, k_chem  the interface nodes' reaction sub-steps (a thread
//               or a lane group per node).
//   k_moments   one thread per bulk node: pull-stream all lattices, moments,
//               temperature Newton, the reaction sub-steps, the moment
//               record (scratch) and the T guess.
//   k_mchem     the same with a group of lanes per node (small grids).
//   k_collide   gradients from neighbour records, relaxation parameters,
//               diffusion velocities, collision of all lattices on a second
//               pull gather, store to the other buffer (fused collision).
//   k_prep, k_coll  the same collision split into a per-node parameter
//               kernel and a nine-threads-per-node direction kernel.
//   k_*_batch   the same bodies over the tiles of several handles.
//   k_step_persist  a whole batched step as one launch over a work-list.
//   k_init      populations at the equilibria of given fields.
//   k_out       fields of the stored state (SI units).
//   k_diag      per-node heat release and flame diagnostics.
//
// Template parameters: D (2 or 3), M (species), S (storage type), RT (type
// of the lattice arithmetic: moments, equilibria, collision).  FP64 storage
// computes everything in FP64.  FP32 and FP16 storage compute the lattice
// arithmetic and transport in FP32 and the temperature Newton solve and the
// chemistry in float-float (ff.cuh) or, with LBM_CHEM64, in FP64.
#include <atomic>
#include <climits>
#include <cmath>
#include <type_traits>

#pragma once

#include "lbm_device.cuh"
#include "lbm_sync.cuh"

// Chemistry mode of the mixed path in this translation unit: with FP32
// lattice arithmetic, the temperature Newton solve and the reaction
// chemistry run in float-float (LBM_CHEM64 = 0) or in native FP64
// (LBM_CHEM64 = 1).  The two modes' templates live in distinct inline
// namespaces, so both can be instantiated in one library.
#ifndef LBM_CHEM64
#define LBM_CHEM64 0
#endif

namespace lbm {
#if LBM_CHEM64
inline namespace chem64 {
#else
inline namespace chemff {
#endif

// float-float Newton and chemistry: FP32 lattice arithmetic, float-float mode
template <typename RT> constexpr bool kFF = sizeof(RT) == 4 && !LBM_CHEM64;
// resident blocks per SM the moments kernels are compiled for (register cap):
// four for the float-float chemistry, two with FP64 chemistry beside FP32
// lattice arithmetic, one in the FP64 path
template <typename RT>
constexpr int kMomentsMinBlocks = kFF<RT> ? 4 : (sizeof(RT) == 4 ? 2 : 1);

// Arithmetic type of a storage type: FP16 storage computes in FP32.
template <typename S> struct ComputeType { using type = S; };
template <> struct ComputeType<__half> { using type = float; };

// Stored-population codec.  FP64 and FP32 storage hold the value itself.
// FP16 storage holds offsets (reading R19): h = (f - o_li) / s_l, o_li the
// equilibrium population at the mean initial state and s_l a per-lattice
// scale, both fixed by lbm_init_fields (codec entry li = {o, s, 1/s, 0}).
template <typename S> struct Codec {
  template <typename R>
  __device__ static R dec(S v, const float4*, int) { return R(v); }
  template <typename R>
  __device__ static S enc(R v, const float4*, int) { return S(v); }
};
template <> struct Codec<__half> {
  template <typename R>
  __device__ static R dec(__half v, const float4* t, int li) {
    const float4 c = __ldg(t + li);
    return R(fmaf(c.y, __half2float(v), c.x));
  }
  template <typename R>
  __device__ static __half enc(R v, const float4* t, int li) {
    const float4 c = __ldg(t + li);
    return __float2half_rn((float(v) - c.x) * c.z);
  }
};

// population li = l*Q + i of node n as FP64 (decoded)
template <typename S>
__device__ __forceinline__ double ldp(const S* pops, long long N, long long n, int li,
                                      const float4* codec) {
  return Codec<S>::template dec<double>(__ldg(pops + (long long)li * N + n), codec, li);
}

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
                                     long long N, long long sn, int li, const float4* codec) {
  return tag >= 0 ? RT(bc.pops[(long long)li * bc.n_if + tag])
                  : Codec<S>::template dec<RT>(__ldg(src + (long long)li * N + sn), codec, li);
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
static_assert(kBS == kChemThreads, "the chemistry's shared-memory slices assume kBS threads");

// shared memory of the collision kernel per thread: the diffusion-velocity
// matrix, then the axis-factor tables (FP32: every axis; FP64 in 3D: the y
// and z axes, the whole table would halve the occupancy)
template <int D, int M, typename RT> constexpr int collide_smem_entries() {
  constexpr int tab = sizeof(RT) == 4 ? 2 * M * D * 3 : (D == 3 ? 2 * M * 2 * 3 : 0);
  return tab > M * M ? tab : M * M;
}

template <int D>
__device__ __forceinline__ constexpr int pidx(int a, int b) {
  return a == b ? a : (D == 3 ? (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5)) : 2);
}

// ---------------------------------------------------------------------------
// Reaction sub-steps of one node by one thread at frozen internal energy
// (Sec. 2.4 Eq. R3): rs the post-stream species densities (the slaved one
// included), rho, ER = E / rho and usqR = |u|^2 of the moments, T_0 = T
// their temperature; dr receives the increments drho_a (a < M - 1).  The
// mixed path runs it in float-float, whose rate arrays live in the thread's
// shared-memory slice (kDynChem: chem_slice, the block's slices of
// chem_slice_bytes in dynamic shared memory; else a static array of the
// calling kernel); FP64 chemistry otherwise.  Blocks of kChemThreads threads.
template <int M>
__device__ __forceinline__ ff* chem_static_slice() {
  __shared__ __align__(8) unsigned char chem_raw[chem_slice_bytes<M, ff>()];
  return reinterpret_cast<ff*>(chem_raw);
}

template <int M, typename RT, bool kDynChem>
__device__ __forceinline__ void node_substeps(const RT (&rs)[M], RT rho, RT ER, RT usqR,
                                              double T, const Units& un, const DevMech& mech,
                                              int* __restrict__ status, void* chem_slice,
                                              RT (&dr)[M - 1]) {
  if constexpr (kFF<RT>) {
    ff* Cs;
    if constexpr (kDynChem) Cs = static_cast<ff*>(chem_slice) + threadIdx.x;
    else Cs = chem_static_slice<M>() + threadIdx.x;
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
      production_rates_ff<M>(mech, Ts, r, rdot, Cs);
#pragma unroll
      for (int a = 0; a < M; ++a) r[a] += un.dt_sub_f * rdot[a];
    }
#pragma unroll
    for (int a = 0; a < M - 1; ++a) dr[a] = (r[a] - ff(rs[a])).hi;
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
    for (int a = 0; a < M - 1; ++a) dr[a] = RT(r[a] - double(rs[a]));
  }
}

// ---------------------------------------------------------------------------
// The node's record from its population sums (Sec. 2.1, Sec. 3.1-3.2, Sec.
// 3.7 slaving): fields, temperature by Newton from the node's previous T,
// and the reaction sub-steps when chem_inline (else the species densities go
// to the increment slots for a separate sub-step kernel).  Used by the
// moments kernels (one thread per node).
template <int D, int M, typename RT, bool kDynChem = false>
__device__ __forceinline__ void moments_finish(RT* __restrict__ rec, double* __restrict__ Tf,
                                               int* __restrict__ status, long long N,
                                               const Units& un, const DevMech& mech,
                                               long long n, int chem_inline, RT rho, RT rhoE,
                                               const RT (&j)[D], const RT (&q)[D],
                                               const RT (&P)[Lat<D>::NP], RT (&rs)[M],
                                               RT (&js)[M][D], void* chem_slice) {
  constexpr int NP = Lat<D>::NP;
  using RC = Rec<D, M>;
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
  if constexpr (kFF<RT>) {
    // mixed path: the temperature solve in float-float
    ff Yf[M];
    float Rm = 0.f;
#pragma unroll
    for (int a = 0; a < M; ++a) {
      Yf[a] = ff(YR[a]);
      Rm += YR[a] * mech.inv_mm_s[a];
    }
    const ff U = (ff(ER) + ff(-0.5f * usqR)) * un.c2_f;
    const ff Tx = newton_T_ff<M>(mech, Yf, U, ff_from_double(__ldcg(Tf + n)), un.newton_max_iter,
                                 un.newton_rtol_f, ok);
    T = ff_to_double(Tx);
    thR = Rm * float(R_U) * Tx.hi * un.inv_c2_s;
  } else {
    double Y[M];
#pragma unroll
    for (int a = 0; a < M; ++a) Y[a] = double(YR[a]);
    const double U = (double(ER) - 0.5 * double(usqR)) * un.c * un.c;
    T = newton_T<M>(mech, Y, U, __ldcg(Tf + n), un.newton_max_iter, un.newton_rtol, ok);
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
  } else {
    RT dr[M - 1];
    node_substeps<M, RT, kDynChem>(rs, rho, ER, usqR, T, un, mech, status, chem_slice, dr);
#pragma unroll
    for (int a = 0; a < M - 1; ++a) rec[(RC::DRHO + a) * N + n] = dr[a];
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
    // rho_a is denormal in FP32 (its reciprocal would overflow: FP32 divides);
    // in FP64 rho_a > 1e-300 where defined, so one reciprocal serves the D
    // components
    const bool tiny = species_velocity_undefined<D, RT>(rs[a], js[a]);
    if constexpr (sizeof(RT) == 8) {
      const RT ira = tiny ? RT(0) : RT(1) / rs[a];
#pragma unroll
      for (int d = 0; d < D; ++d)
        rec[(RC::US + a * D + d) * N + n] = tiny ? uR[d] : js[a][d] * ira;
    } else {
#pragma unroll
      for (int d = 0; d < D; ++d)
        rec[(RC::US + a * D + d) * N + n] = tiny ? uR[d] : js[a][d] / rs[a];
    }
  }
}

// ---------------------------------------------------------------------------
// Moments of the post-stream state + temperature (Sec. 2.1, Sec. 3.1-3.2,
// Sec. 3.7 slaving, Sec. 4.1 pull streaming).
// chem_inline = 0: the reaction sub-steps run in a lane-group kernel
// (k_chem); this kernel then leaves the post-stream species densities rho_a
// (a < M) in the record's increment slots for it.
template <int D, int M, typename S, typename RT, bool kDynChem = false>
__device__ __forceinline__ void moments_body(const S* __restrict__ src, RT* __restrict__ rec,
                                             double* __restrict__ Tf, int* __restrict__ status,
                                             const Geom& g, const Units& un, const BCDev& bc,
                                             const DevMech& mech, long long n,
                                             int chem_inline, void* chem_slice = nullptr) {
  constexpr int Q = Lat<D>::Q, NP = Lat<D>::NP;
  using RC = Rec<D, M>;
  const long long N = g.N;
  if (n >= N) return;
  const int tag = bc.tag ? bc.tag[n] : TAG_BULK;
  if (tag == TAG_SOLID) return;
  const int x = (int)(n % g.nx);
  const int y = (int)((n / g.nx) % g.ny);
  const int z = (int)(n / ((long long)g.nx * g.ny));
  const float4* codec = g.codec;

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
  // rows of three velocities (c_x = -1, 0, 1 at fixed c_y, c_z), rows
  // rolled: the fully unrolled loop is ~27 copies of the body, whose
  // instruction fetch dominates grids too small to keep many warps per SM.
  // A row's populations enter through their sum s and difference d = f_+ -
  // f_- (and f_+ + f_- for P_xx): sum_i c_ix f_i = sum_rows d,
  // sum_i c_iy f_i = sum_rows c_y s, and so on.
#pragma unroll 1
  for (int r = 0; r < Q / 3; ++r) {
    const RT cy = RT(r % 3 - 1), cz = RT(D == 3 ? r / 3 - 1 : 0);
    const long long sn0 = node_shift<D>(x, y, z, 3 * r, -1, g);
    const long long sn1 = node_shift<D>(x, y, z, 3 * r + 1, -1, g);
    const long long sn2 = node_shift<D>(x, y, z, 3 * r + 2, -1, g);
#pragma unroll
    for (int a = 0; a < M - 1; ++a) {
      const RT v0 = pop_in<RT>(src, bc, tag, N, sn0, a * Q + 3 * r, codec);
      const RT v1 = pop_in<RT>(src, bc, tag, N, sn1, a * Q + 3 * r + 1, codec);
      const RT v2 = pop_in<RT>(src, bc, tag, N, sn2, a * Q + 3 * r + 2, codec);
      const RT sr = v0 + v1 + v2;
      rs[a] += sr;
      js[a][0] += v2 - v0;
      js[a][1] += cy * sr;
      if (D == 3) js[a][D - 1] += cz * sr;
    }
    {
      const int l = M - 1;
      const RT f0 = pop_in<RT>(src, bc, tag, N, sn0, l * Q + 3 * r, codec);
      const RT f1 = pop_in<RT>(src, bc, tag, N, sn1, l * Q + 3 * r + 1, codec);
      const RT f2 = pop_in<RT>(src, bc, tag, N, sn2, l * Q + 3 * r + 2, codec);
      const RT sx = f0 + f2, sr = sx + f1, dx = f2 - f0;
      rho += sr;
      j[0] += dx;
      j[1] += cy * sr;
      P[pidx<D>(0, 0)] += sx;
      P[pidx<D>(1, 1)] += (cy * cy) * sr;
      P[pidx<D>(0, 1)] += cy * dx;
      if constexpr (D == 3) {
        j[2] += cz * sr;
        P[pidx<D>(2, 2)] += (cz * cz) * sr;
        P[pidx<D>(0, 2)] += cz * dx;
        P[pidx<D>(1, 2)] += (cy * cz) * sr;
      }
    }
    {
      const int l = M;
      const RT g0 = pop_in<RT>(src, bc, tag, N, sn0, l * Q + 3 * r, codec);
      const RT g1 = pop_in<RT>(src, bc, tag, N, sn1, l * Q + 3 * r + 1, codec);
      const RT g2 = pop_in<RT>(src, bc, tag, N, sn2, l * Q + 3 * r + 2, codec);
      const RT sr = g0 + g1 + g2;
      rhoE += sr;
      q[0] += g2 - g0;
      q[1] += cy * sr;
      if (D == 3) q[D - 1] += cz * sr;
    }
  }
  moments_finish<D, M, RT, kDynChem>(rec, Tf, status, N, un, mech, n, chem_inline, rho, rhoE, j,
                                     q, P, rs, js, chem_slice);
}

// ---------------------------------------------------------------------------
// Reaction sub-steps with several lanes per node (Sec. 2.4 Eq. R3), for
// grids too small to fill the GPU at one thread per node: the node's
// reactions are dealt out over the lanes, which cuts the latency of a node's
// chemistry by about the lane count.  The formulas are those of
// production_rates / production_rates_ff; only the production rates are
// summed in another order (partial sums per lane), so the placements agree
// to rounding.  CT: double (FP64 path) or float-float (mixed path).
__device__ __forceinline__ double shfl_xor_ct(unsigned mask, double v, int o) {
  return __shfl_xor_sync(mask, v, o);
}
__device__ __forceinline__ ff shfl_xor_ct(unsigned mask, ff v, int o) {
  return ff(__shfl_xor_sync(mask, v.hi, o), __shfl_xor_sync(mask, v.lo, o));
}

template <typename CT> struct Chem;
template <> struct Chem<double> {
  __device__ static double ex(double x) { return exp_tang(x); }
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
  __device__ static double ucoef(const DevMech& m, int k, int a) {
    return k == 0 ? m.u0[a] : (k == 1 ? m.u1[a] : (k == 2 ? m.u2[a] : m.u3[a]));
  }
  __device__ static double mag(double x) { return fabs(x); }
  __device__ static double rtol(const Units& u) { return u.newton_rtol; }
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
  __device__ static ff ucoef(const DevMech& m, int k, int a) {
    return k == 0 ? m.u0_f[a] : (k == 1 ? m.u1_f[a] : (k == 2 ? m.u2_f[a] : m.u3_f[a]));
  }
  __device__ static float mag(ff x) { return fabsf(x.hi); }
  __device__ static float rtol(const Units& u) { return u.newton_rtol_f; }
};

template <typename RT> struct ChemType { using type = double; };
template <> struct ChemType<float> { using type = std::conditional_t<LBM_CHEM64 != 0, double, ff>; };

__device__ __forceinline__ double shfl_ct(unsigned mask, double v, int src) {
  return __shfl_sync(mask, v, src);
}
__device__ __forceinline__ ff shfl_ct(unsigned mask, ff v, int src) {
  return ff(__shfl_sync(mask, v.hi, src), __shfl_sync(mask, v.lo, src));
}

// Register r[a] for a lane-dependent species index a (a select per species:
// a runtime index into a register array would put it in local memory).
template <int M, typename CT>
__device__ __forceinline__ CT pick(const CT (&r)[M], int a) {
  CT v = r[0];
#pragma unroll
  for (int b = 1; b < M; ++b)
    if (b == a) v = r[b];
  return v;
}

// Temperature Newton on Eq. temperature for a lane group (the formulas of
// newton_T / newton_T_ff): lane `sub` sums the mixture energy polynomial's
// coefficients over the species a = sub, sub + L, ..., the group adds them
// with a butterfly (every lane ends with the same sums, so every lane takes
// the same iterates), and every lane iterates.
template <int M, int L, typename CT>
__device__ __forceinline__ CT group_newton(const DevMech& m, const CT (&r)[M], CT irho, CT U,
                                           CT T, const Units& un, int sub, unsigned gmask,
                                           bool& ok) {
  using X = Chem<CT>;
  CT c[4] = {CT(), CT(), CT(), CT()};
#pragma unroll
  for (int j = 0; j < (M + L - 1) / L; ++j) {
    const int a = sub + j * L;
    if (a < M) {
      const CT Ya = pick<M, CT>(r, a) * irho;
#pragma unroll
      for (int k = 0; k < 4; ++k) c[k] += Ya * X::ucoef(m, k, a);
    }
  }
#pragma unroll
  for (int o = 1; o < L; o <<= 1)
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] += shfl_xor_ct(gmask, c[k], o);
  const CT two = X::of(2.f), three = X::of(3.f);
  ok = false;
  for (int it = 0; it < un.newton_max_iter; ++it) {
    const CT F = c[0] + T * (c[1] + T * (c[2] + T * c[3])) - U;
    const CT dF = c[1] + T * (two * c[2] + three * T * c[3]);
    const CT dT = -(F / dF);
    T += dT;
    if (X::mag(dT) <= X::rtol(un) * X::mag(T)) { ok = true; break; }
  }
  return T;
}

// The reaction sub-steps of one node by its lane group (Sec. 2.4 Eq. R3),
// from the post-stream species densities r (replaced by the densities after
// the sub-steps), 1/rho, the internal energy U and the temperature T_0 of
// the moments.
template <int M, typename CT, int L>
__device__ __forceinline__ void chem_group_substeps(CT (&r)[M], const CT irho, const CT U,
                                                    CT Ts, const Units& un, const DevMech& m,
                                                    int sub, unsigned gmask,
                                                    int* __restrict__ status) {
  using X = Chem<CT>;
  const int base = (int)(threadIdx.x & 31) - sub;      // the group's first lane
  // the arrays the reaction loop indexes by species: a per-thread slice of
  // shared memory (as in production_rates_ff; 128-thread blocks)
  __shared__ __align__(8) unsigned char chem_raw[3 * M * kChemThreads * sizeof(CT)];
  CT* const Cs = reinterpret_cast<CT*>(chem_raw) + threadIdx.x;
  CT* const Gs = Cs + M * kChemThreads;
  CT* const Ws = Gs + M * kChemThreads;
  for (int s = 0; s < un.substeps; ++s) {
    if (s > 0) {
      bool ok;
      Ts = group_newton<M, L, CT>(m, r, irho, U, Ts, un, sub, gmask, ok);
      if (!ok && sub == 0) atomicOr(status, ST_NEWTON);
    }
    const CT lnT = X::ln(Ts);
    const CT invT = X::inv(Ts);
    // Gibbs functions: lane `sub` evaluates species sub, sub + L, ...; the
    // group exchanges them with shuffles
    CT Gown[(M + L - 1) / L];
#pragma unroll
    for (int j = 0; j < (M + L - 1) / L; ++j) {
      const int a = sub + j * L;
      Gown[j] = a < M ? X::gibbs(m, a, Ts, invT, lnT) : CT();
    }
    // species-indexed arrays in the thread's shared-memory slice (the
    // register copy of C serves the unrolled third-body sums)
    CT C[M];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      C[a] = r[a] * X::inv_mm(m, a);
      Cs[a * kChemThreads] = C[a];
      Gs[a * kChemThreads] = shfl_ct(gmask, Gown[a / L], base + a % L);
      Ws[a * kChemThreads] = CT();
    }
    const CT lp = X::ln_p0(m) - lnT;   // ln(P0 / (R_U T))
    for (int k = sub; k < m.R; k += L) {
      const DevReaction& rx = m.rx[k];
      const CT lk = X::lnkf(rx, lnT, invT);
      CT fwd = X::ex(lk);
      for (int j = 0; j < rx.nr; ++j) fwd *= Cs[rx.reac[j] * kChemThreads];
      CT rev = CT();
      if (rx.reversible) {
        CT dG = CT();
        for (int j = 0; j < rx.np; ++j) dG += Gs[rx.prod[j] * kChemThreads];
        for (int j = 0; j < rx.nr; ++j) dG -= Gs[rx.reac[j] * kChemThreads];
        rev = X::ex(X::rev_arg(rx, lk, dG, lp));
        for (int j = 0; j < rx.np; ++j) rev *= Cs[rx.prod[j] * kChemThreads];
      }
      CT q = fwd - rev;
      if (rx.third_body) {
        CT cm = CT();
#pragma unroll
        for (int a = 0; a < M; ++a) cm += X::eff(m, k, a) * C[a];
        q *= cm;
      }
      for (int j = 0; j < rx.nr; ++j) Ws[rx.reac[j] * kChemThreads] -= q;
      for (int j = 0; j < rx.np; ++j) Ws[rx.prod[j] * kChemThreads] += q;
    }
    CT w[M];
#pragma unroll
    for (int a = 0; a < M; ++a) w[a] = Ws[a * kChemThreads];
    // butterfly sums over the group: every lane ends with the same total
#pragma unroll
    for (int o = 1; o < L; o <<= 1)
#pragma unroll
      for (int a = 0; a < M; ++a) w[a] += shfl_xor_ct(gmask, w[a], o);
#pragma unroll
    for (int a = 0; a < M; ++a) r[a] += X::dt_sub(un) * (w[a] * X::mm(m, a));
  }
}

// Reaction sub-steps of node n by a group of L lanes (L = 4 or 8, aligned
// within the warp): every lane forms the node's state, temperature,
// concentrations and Gibbs functions; lane `sub` takes the reactions
// k = sub, sub + L, ...; the species production rates are summed across the
// group with shuffles, after which every lane holds the same densities.
template <int D, int M, typename RT, int L>
__device__ __forceinline__ void chem_lanes_body(RT* __restrict__ rec,
                                                const double* __restrict__ Tf,
                                                int* __restrict__ status, long long N,
                                                const int* __restrict__ tag, const Units& un,
                                                const DevMech& m, long long n, int sub,
                                                unsigned gmask) {
  using CT = typename ChemType<RT>::type;
  using X = Chem<CT>;
  using RC = Rec<D, M>;
  const RT rho = rec[RC::RHO * N + n];
  RT usq = RT(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const RT ud = rec[(RC::U + d) * N + n];
    usq += ud * ud;
  }
  const RT ER = rec[RC::E * N + n];
  CT U;
  if constexpr (kFF<RT>) U = (ff(ER) + ff(-0.5f * usq)) * un.c2_f;
  else U = (double(ER) - 0.5 * double(usq)) * un.c * un.c;
  // the post-stream species densities the moments kernel left in the
  // increment slots; the slaved species from the mixture density
  CT r[M], r0[M - 1];
  RT last = rho;
#pragma unroll
  for (int a = 0; a < M - 1; ++a) {
    const RT v = rec[(RC::DRHO + a) * N + n];
    last -= v;
    r0[a] = X::of(v);
    r[a] = r0[a];
  }
  r[M - 1] = X::of(last);
  chem_group_substeps<M, CT, L>(r, X::inv(X::of(rho)), U, X::of_T(Tf[n]), un, m, sub, gmask,
                                status);
#pragma unroll
  for (int a = 0; a < M - 1; ++a) {
    if (a % L != sub) continue;
    if constexpr (kFF<RT>) rec[(RC::DRHO + a) * N + n] = (r[a] - r0[a]).hi;
    else rec[(RC::DRHO + a) * N + n] = RT(r[a] - r0[a]);
  }
}

// Moments and reaction sub-steps of node n by a group of L lanes (grids too
// small to fill the GPU at one thread per node; chem_lanes = L).  Lane `sub`
// pulls the directions sub, sub + L, ... of every lattice, the group adds the
// partial sums with a butterfly, every lane forms the node's fields (the
// formulas of moments_finish), the temperature solve is shared as in
// group_newton, the lanes split the record's stores, and the group runs the
// sub-steps from the post-stream densities (chem_group_substeps).  m: the
// mechanism for compile-time indices; mg: its global copy, indexed by lane.
template <int D, int M, typename S, typename RT, int L>
__device__ __forceinline__ void mchem_body(const S* __restrict__ src, RT* __restrict__ rec,
                                           double* __restrict__ Tf, int* __restrict__ status,
                                           const Geom& g, const Units& un, const BCDev& bc,
                                           const DevMech& m, const DevMech& mg, long long n,
                                           int tag, int sub, unsigned gmask) {
  constexpr int Q = Lat<D>::Q, NP = Lat<D>::NP;
  using RC = Rec<D, M>;
  using CT = typename ChemType<RT>::type;
  using X = Chem<CT>;
  const long long N = g.N;
  const int x = (int)(n % g.nx);
  const int y = (int)((n / g.nx) % g.ny);
  const int z = (int)(n / ((long long)g.nx * g.ny));
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
  for (int jd = 0; jd < (Q + L - 1) / L; ++jd) {
    const int i = sub + jd * L;
    if (i < Q) {
      RT c[D];
#pragma unroll
      for (int d = 0; d < D; ++d) c[d] = RT(cvel(i, d));
      const long long sn = node_shift<D>(x, y, z, i, -1, g);
#pragma unroll
      for (int a = 0; a < M - 1; ++a) {
        const RT v = pop_in<RT>(src, bc, tag, N, sn, a * Q + i, g.codec);
        rs[a] += v;
#pragma unroll
        for (int d = 0; d < D; ++d) js[a][d] += c[d] * v;
      }
      const RT f = pop_in<RT>(src, bc, tag, N, sn, (M - 1) * Q + i, g.codec);
      rho += f;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        j[d] += c[d] * f;
#pragma unroll
        for (int e = d; e < D; ++e) P[pidx<D>(d, e)] += c[d] * c[e] * f;
      }
      const RT gv = pop_in<RT>(src, bc, tag, N, sn, M * Q + i, g.codec);
      rhoE += gv;
#pragma unroll
      for (int d = 0; d < D; ++d) q[d] += c[d] * gv;
    }
  }
#pragma unroll
  for (int o = 1; o < L; o <<= 1) {
    rho += __shfl_xor_sync(gmask, rho, o);
    rhoE += __shfl_xor_sync(gmask, rhoE, o);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      j[d] += __shfl_xor_sync(gmask, j[d], o);
      q[d] += __shfl_xor_sync(gmask, q[d], o);
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) P[k] += __shfl_xor_sync(gmask, P[k], o);
#pragma unroll
    for (int a = 0; a < M - 1; ++a) {
      rs[a] += __shfl_xor_sync(gmask, rs[a], o);
#pragma unroll
      for (int d = 0; d < D; ++d) js[a][d] += __shfl_xor_sync(gmask, js[a][d], o);
    }
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
  const RT inv_rho = RT(1) / rho;
  RT uR[D], YR[M], usqR = RT(0);
#pragma unroll
  for (int d = 0; d < D; ++d) { uR[d] = j[d] * inv_rho; usqR += uR[d] * uR[d]; }
#pragma unroll
  for (int a = 0; a < M; ++a) YR[a] = rs[a] * inv_rho;
  const RT ER = rhoE * inv_rho;
  // temperature (Eq. temperature) from the node's previous T, shared solve
  CT U, r[M];
  if constexpr (kFF<RT>) U = (ff(ER) + ff(-0.5f * usqR)) * un.c2_f;
  else U = (double(ER) - 0.5 * double(usqR)) * un.c * un.c;
#pragma unroll
  for (int a = 0; a < M; ++a) r[a] = X::of(rs[a]);
  const CT irho = X::inv(X::of(rho));
  bool ok;
  const CT Tx = group_newton<M, L, CT>(mg, r, irho, U, X::of_T(Tf[n]), un, sub, gmask, ok);
  double T;
  RT thR;
  if constexpr (kFF<RT>) {
    float Rm = 0.f;
#pragma unroll
    for (int a = 0; a < M; ++a) Rm += YR[a] * m.inv_mm_s[a];
    T = ff_to_double(Tx);
    thR = Rm * float(R_U) * Tx.hi * un.inv_c2_s;
  } else {
    double Rmix = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) Rmix += double(YR[a]) * m.inv_mm[a];
    T = Tx;
    thR = RT(Rmix * R_U * T * un.inv_c2);
  }
  if (sub == 0) {
    if (!ok) atomicOr(status, ST_NEWTON);
    if (!(rho > RT(0)) || !isfinite(double(rho)) || !isfinite(T)) atomicOr(status, ST_NONFINITE);
    Tf[n] = T;
  }
  // the record's fields, each stored by one lane of the group
  auto put = [&](int f, RT v) {
    if (f % L == sub) rec[(long long)f * N + n] = v;
  };
  put(RC::RHO, rho);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    put(RC::U + d, uR[d]);
    put(RC::QF + d, q[d]);
    put(RC::PHI + d, rho * uR[d] * (RT(1) - RT(3) * thR) - rho * uR[d] * uR[d] * uR[d]);
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) put(RC::P + k, P[k]);
  put(RC::E, ER);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    put(RC::Y + a, YR[a]);
    const bool tiny = species_velocity_undefined<D, RT>(rs[a], js[a]);
#pragma unroll
    for (int d = 0; d < D; ++d) put(RC::US + a * D + d, tiny ? uR[d] : js[a][d] / rs[a]);
  }
  // reaction sub-steps at frozen U (Sec. 2.4 Eq. R3), T_0 the T just solved
  CT r0[M - 1];
#pragma unroll
  for (int a = 0; a < M - 1; ++a) r0[a] = r[a];
  chem_group_substeps<M, CT, L>(r, irho, U, X::of_T(T), un, mg, sub, gmask, status);
#pragma unroll
  for (int a = 0; a < M - 1; ++a) {
    if constexpr (kFF<RT>) put(RC::DRHO + a, (r[a] - r0[a]).hi);
    else put(RC::DRHO + a, RT(r[a] - r0[a]));
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
  __device__ static double mu0_sp(const DevMech& m, int a) { return m.mu0_sp[a]; }
  __device__ static double wilke_phi(const DevMech& m, int a, int b) {
    return m.wilke_phi[a][b];
  }
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
  __device__ static float mu0_sp(const DevMech& m, int a) { return m.mu0_sp_s[a]; }
  __device__ static float wilke_phi(const DevMech& m, int a, int b) {
    return m.wilke_phi_s[a][b];
  }
};

// ---------------------------------------------------------------------------
// Per-node collision parameters: everything the direction loop needs
// (Sec. 2.3 Eqs. betaa, taua, transform1; Sec. 3.3 Eq. Pex; Sec. 3.4 Eqs.
// gstar, qdiff, corrFourier; Sec. 2.4 Eq. R3).
template <int D, int M, typename RT> struct NodePar {
  RT rho, om, U, theta;          // density, omega, internal energy, R T (lattice)
  RT u[D], Pex[D], W[D];         // velocity, extended diagonal pressure, energy-flux term
  RT th[M], V[M][D], rs[M];      // theta_b, diffusion velocities, rho_b
  RT cF[M - 1], om1[M - 1], hh[M - 1];  // (beta_a - 1) Y_a s, 1 - 2 beta_a, 2 beta_a rho_a + drho_a
};

// Field offsets of NodePar stored field-major [field][N] (split collision).
template <int D, int M> struct CPar {
  static constexpr int TH = 0;
  static constexpr int V = TH + M;
  static constexpr int RS = V + M * D;
  static constexpr int CF = RS + M;
  static constexpr int OM1 = CF + M - 1;
  static constexpr int HH = OM1 + M - 1;
  static constexpr int U = HH + M - 1;
  static constexpr int PEX = U + D;
  static constexpr int W = PEX + D;
  static constexpr int RHO = W + D;
  static constexpr int OM = RHO + 1;
  static constexpr int UL = OM + 1;
  static constexpr int THETA = UL + 1;
  static constexpr int NF = THETA + 1;
};

// The per-node part of the collision of node n (not solid, n < N):
// moments from the record, isotropic gradients, relaxation parameters,
// diffusion velocities, energy-flux correction.  The diffusion-velocity
// solve uses this thread's shared-memory column (M*M entries, stride kBS).
template <int D, int M, typename RT>
__device__ __forceinline__ void node_params(const RT* __restrict__ rec,
                                            const double* __restrict__ Tf, const Geom& g,
                                            const Units& un, const BCDev& bc,
                                            const DevMech& mech, long long n, int tag,
                                            NodePar<D, M, RT>& p) {
  constexpr int Q = Lat<D>::Q, NP = Lat<D>::NP;
  using RC = Rec<D, M>;
  const long long N = g.N;
  const int x = (int)(n % g.nx);
  const int y = (int)((n / g.nx) % g.ny);
  const int z = (int)(n / ((long long)g.nx * g.ny));

  // node scalars in the parameter type PT (FP64 in the FP64 path, FP32 in
  // the mixed path, whose temperature and chemistry run in float-float);
  // lattice-type values (RT) for gradients, the solve and the collision
  using PT = RT;
  using MP = MixParams<PT>;
  const PT rho = PT(rec[RC::RHO * N + n]);
  const double T_d = __ldcg(Tf + n);
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
  // x-rows of neighbours unrolled, rows rolled (instruction footprint, as in
  // the moments kernel)
#pragma unroll 1
  for (int r = 0; r < Q / 3; ++r) {
    const int cyi = r % 3 - 1, czi = D == 3 ? r / 3 - 1 : 0;
#pragma unroll
    for (int ix = 0; ix < 3; ++ix) {
      const int cxi = ix - 1;
      if (ix == 1 && cyi == 0 && czi == 0) continue;          // the rest velocity
      const int cvi[3] = {cxi, cyi, czi};
      long long nb = 0;
      int gk = BK_NONE;
      if (!bc.tag) {
        nb = node_shift<D>(x, y, z, 3 * r + ix, +1, g);
      } else {
        int cc[3] = {x + cxi, y + cyi, D == 3 ? z + czi : z};
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
      // 3 w_i: the product of 2/3 (c = 0) and 1/6 (c = +-1) per axis
      const RT wy = cyi == 0 ? RT(2.0 / 3.0) : RT(1.0 / 6.0);
      const RT wz = D == 3 ? (czi == 0 ? RT(2.0 / 3.0) : RT(1.0 / 6.0)) : RT(1);
      const RT w3 = RT(3) * ((ix == 1 ? RT(2.0 / 3.0) : RT(1.0 / 6.0)) * wy * wz);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (cvi[d] == 0) continue;
        const RT wc = w3 * RT(cvi[d]);
        const RT pv = gk == BK_NONE ? __ldg(rec + (RC::PHI + d) * N + nb)
                      : (gk == BK_INLET ? phi_in[d] : (gk == BK_OUTLET ? phi_self[d] : RT(0)));
        dPhi[d] += wc * pv;
#pragma unroll
        for (int a = 0; a < M; ++a)
          gY[a][d] += wc * (gk == BK_NONE ? __ldg(rec + (RC::Y + a) * N + nb) : RT(Y[a]));
      }
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
  PT mu = MP::mu0(mech);
  if (mech.wilke) {
    // Wilke's mixing rule over the species viscosities (the mole fractions'
    // normalisation cancels between numerator and denominator)
    PT X[M];
#pragma unroll
    for (int a = 0; a < M; ++a) X[a] = Y[a] * MP::inv_mm(mech, a);
    mu = PT(0);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      PT den = PT(0);
#pragma unroll
      for (int b = 0; b < M; ++b) den += X[b] * MP::wilke_phi(mech, a, b);
      mu += X[a] * MP::mu0_sp(mech, a) / den;
    }
  }
  mu *= exp(MP::mu_T_exp(mech) * lnTr);
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
      if constexpr (kFF<RT>) {
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
#pragma unroll
  for (int a = 0; a < M; ++a) {
    p.th[a] = RT(MP::Ra(mech, a) * T * MP::inv_c2(un));
    p.rs[a] = RT(rs[a]);
#pragma unroll
    for (int d = 0; d < D; ++d) p.V[a][d] = V[a][d];
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    p.u[d] = RT(u[d]);
    p.Pex[d] = RT(theta + u[d] * u[d] + (PT(2) - omega) / (PT(2) * rho * omega) * PT(dPhi[d]));
    p.W[d] = W[d];
  }
  p.rho = RT(rho);
  p.om = RT(omega);
  p.U = RT(U_lat);
  p.theta = RT(theta);
  // species coefficients of the update
  //   f_a + 2 beta_a (rho_a psi_a - f_a) + cF_a sum_b K_ab d_b + drho_a psi_a
  //     = f_a om1_a + psi_a hh_a + cF_a sum_b K_ab d_b,
  // cF_a = (beta_a - 1) Y_a s (1/tau_ab = s K_ab), om1_a = 1 - 2 beta_a,
  // hh_a = 2 beta_a rho_a + drho_a
#pragma unroll
  for (int a = 0; a < M - 1; ++a) {
    const PT beta = inv_tau_a[a] / (PT(2) + inv_tau_a[a]);
    p.cF[a] = RT((beta - PT(1)) * Y[a] * s_tau);
    p.om1[a] = RT(PT(1) - PT(2) * beta);
    p.hh[a] = RT(PT(2) * beta * rs[a] + PT(rec[(RC::DRHO + a) * N + n]));
  }
}

// Energy-equilibrium axis factors (the closed form of g^eq, Sec. 3.4 Eq.
// geq_i): A_c acting on 1 and B_c acting on u^2/2, c = -1, 0, 1.
template <int D, typename RT>
__device__ __forceinline__ void energy_factors(const RT (&u)[D], RT theta, RT (&Af)[D][3],
                                               RT (&Bf)[D][3]) {
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const RT ua = u[d];
    const RT O1 = theta * ua + RT(0.5) * ua * ua * ua;
    const RT O2 = theta * theta + RT(2.5) * theta * ua * ua + RT(0.5) * ua * ua * ua * ua;
    const RT Pd = theta + ua * ua;
    Af[d][0] = RT(0.5) * (Pd - ua);
    Af[d][1] = RT(1) - Pd;
    Af[d][2] = RT(0.5) * (Pd + ua);
    Bf[d][0] = RT(0.5) * (O2 - O1);
    Bf[d][1] = RT(0.5) * ua * ua - O2;
    Bf[d][2] = RT(0.5) * (O2 + O1);
  }
}

// Axis factors of psi(u, theta_b) (set 0) and psi(u + V_b, theta_b) (set 1)
// (Eq. prod): entry e = ((set*M + b)*D + d)*3 + c + 1 of a table.
template <int D, int M, typename RT>
__device__ __forceinline__ RT axis_factor(int e, const RT* th, const RT* u, const RT* V) {
  const int c = e % 3 - 1;
  const int d = (e / 3) % D;
  const int b = (e / (3 * D)) % M;
  const int set = e / (3 * D * M);
  const RT xs = set ? u[d] + V[b * D + d] : u[d];
  const RT Ps = th[b] + xs * xs;
  return c == 0 ? RT(1) - Ps : (c > 0 ? RT(0.5) * (Ps + xs) : RT(0.5) * (Ps - xs));
}

// The M + 1 populations of direction i entering node n's collision (pulled
// from node sn, or the boundary-reconstructed ones).
template <int D, int M, typename S, typename RT>
__device__ __forceinline__ void load_direction(const S* __restrict__ src, const BCDev& bc,
                                               int tag, long long N, long long sn, int i,
                                               const float4* codec, RT (&fin)[M + 1]) {
  constexpr int Q = Lat<D>::Q;
#pragma unroll
  for (int l = 0; l <= M; ++l) fin[l] = pop_in<RT>(src, bc, tag, N, sn, l * Q + i, codec);
}

// The part of the equilibria of direction (c_x, c_y, c_z) that depends on
// (c_x, c_y) only, shared by the directions that differ in c_z (the product
// form, Sec. 3.3 Eqs. prod, feqmix; Sec. 3.4 Eq. geq_i):
//   species  e_b = psi_x psi_y of psi(u, theta_b), s_b the same of psi(u + V_b, theta_b);
//   momentum rho psi_x psi_y of the extended equilibrium;
//   energy   g^eq = rho [A_z (U A_x A_y + B_x A_y + A_x B_y) + A_x A_y B_z].
template <int D, int M, typename RT> struct XYPart {
  RT e[M], s[M];
  RT fxy, gP, gQ;
};

template <int D, int M, typename RT, typename PS>
__device__ __forceinline__ void xy_part(const PS& ps, int cx, int cy, XYPart<D, M, RT>& h) {
#pragma unroll
  for (int b = 0; b < M; ++b) {
    h.e[b] = ps.sp(0, b, 0, cx) * ps.sp(0, b, 1, cy);
    h.s[b] = ps.sp(1, b, 0, cx) * ps.sp(1, b, 1, cy);
  }
  h.fxy = ps.rho() * psi1<RT>(cx, ps.u(0), ps.Pex(0)) * psi1<RT>(cy, ps.u(1), ps.Pex(1));
  const RT ax = ps.Af(0, cx), ay = ps.Af(1, cy);
  h.gP = ax * ay;
  h.gQ = ps.U() * h.gP + ps.Bf(0, cx) * ay + ax * ps.Bf(1, cy);
}

// Collision of every lattice in direction i = (c_x, c_y, cz) of node n
// (Sec. 2.3 Eq. finalNumericalEquationsReactive; Sec. 3.2 Eqs. f, g; Sec.
// 3.3 Eq. feqmix), from the shared (c_x, c_y) part h.  PS supplies the
// node's parameters (registers, or the block's shared memory in the split
// placement).  The species update
//   f_a + 2 beta_a (rho_a psi_a - f_a) + cF_a sum_b K_ab d_b + drho_a psi_a
// is evaluated as f_a om1_a + psi_a hh_a + cF_a F_a with the per-node
// om1_a = 1 - 2 beta_a and hh_a = 2 beta_a rho_a + drho_a.
template <int D, int M, typename S, typename RT, typename PS>
__device__ __forceinline__ void collide_direction(const PS& ps, const XYPart<D, M, RT>& h,
                                                  int i, const RT (&fin)[M + 1],
                                                  S* __restrict__ dst, long long N, long long n,
                                                  const DevMech& mech, const float4* codec) {
  constexpr int Q = Lat<D>::Q;
  const int cz = D == 3 ? cvel(i, 2) : 0;
  RT pe[M], dd[M];
#pragma unroll
  for (int b = 0; b < M; ++b) {
    RT e = h.e[b], st = h.s[b];
    if constexpr (D == 3) {
      e *= ps.sp(0, b, 2, cz);
      st *= ps.sp(1, b, 2, cz);
    }
    pe[b] = e;
    dd[b] = ps.rs(b) * (e - st);
  }
#pragma unroll
  for (int a = 0; a < M - 1; ++a) {
    RT F = RT(0);
#pragma unroll
    for (int b = 0; b < M; ++b)
      if (b != a) F += kcoef<RT>(mech, a, b) * dd[b];
    const long long off = (long long)(a * Q + i) * N;
    const RT fn = fin[a] * ps.om1(a) + pe[a] * ps.hh(a) + ps.cF(a) * F;
    dst[off + n] = Codec<S>::enc(fn, codec, a * Q + i);
  }
  {
    RT fex = h.fxy;
    if constexpr (D == 3) fex *= psi1<RT>(cz, ps.u(2), ps.Pex(2));
    const long long off = (long long)((M - 1) * Q + i) * N;
    const RT f = fin[M - 1];
    dst[off + n] = Codec<S>::enc(f + ps.om() * (fex - f), codec, (M - 1) * Q + i);
  }
  {
    RT geq = h.gQ;
    if constexpr (D == 3) geq = ps.Af(2, cz) * h.gQ + h.gP * ps.Bf(2, cz);
    geq *= ps.rho();
    const long long off = (long long)(M * Q + i) * N;
    const RT gv = fin[M];
    RT gn = gv + ps.om() * (geq - gv);
    if (csq(i, D) == 1) {
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (cvel(i, d) != 0) gn += (cvel(i, d) > 0 ? RT(0.5) : RT(-0.5)) * ps.W(d);
    }
    dst[off + n] = Codec<S>::enc(gn, codec, M * Q + i);
  }
}

// Parameters held in registers (fused placement).  The species axis factors
// come from a table in this thread's shared-memory column (FP32, entry stride
// kBS) or are formed directly, except, in FP64 3D, those of the y and z axes,
// tabulated in the column (yztab: entry (((set M + b) 2 + d - 1) 3 + c + 1)
// kBS, d = 1, 2).
template <int D, int M, typename RT> struct RegPar {
  const NodePar<D, M, RT>& p;
  RT Afv[D][3], Bfv[D][3];
  const RT* tab;
  const RT* yztab;
  __device__ RegPar(const NodePar<D, M, RT>& p_, const RT* tab_, const RT* yztab_ = nullptr)
      : p(p_), tab(tab_), yztab(yztab_) {
    energy_factors<D, RT>(p.u, p.theta, Afv, Bfv);
  }
  __device__ RT rho() const { return p.rho; }
  __device__ RT om() const { return p.om; }
  __device__ RT U() const { return p.U; }
  __device__ RT u(int d) const { return p.u[d]; }
  __device__ RT Pex(int d) const { return p.Pex[d]; }
  __device__ RT W(int d) const { return p.W[d]; }
  __device__ RT rs(int a) const { return p.rs[a]; }
  __device__ RT cF(int a) const { return p.cF[a]; }
  __device__ RT om1(int a) const { return p.om1[a]; }
  __device__ RT hh(int a) const { return p.hh[a]; }
  __device__ RT Af(int d, int c) const { return c == 0 ? Afv[d][1] : (c > 0 ? Afv[d][2] : Afv[d][0]); }
  __device__ RT Bf(int d, int c) const { return c == 0 ? Bfv[d][1] : (c > 0 ? Bfv[d][2] : Bfv[d][0]); }
  // species axis factor (set 0: psi(u, theta_b); set 1: psi(u + V_b, theta_b))
  __device__ RT sp(int set, int b, int d, int c) const {
    if (tab) return tab[(((set * M + b) * D + d) * 3 + c + 1) * kBS];
    if (D == 3 && d > 0 && yztab) return yztab[(((set * M + b) * 2 + d - 1) * 3 + c + 1) * kBS];
    const RT xs = set ? p.u[d] + p.V[b][d] : p.u[d];
    return psi1<RT>(c, xs, p.th[b] + xs * xs);
  }
};

// Fused placement: one thread per node does the per-node part and then every
// direction (Sec. 2.3, 3.2-3.4).
template <int D, int M, typename S, typename RT>
__device__ __forceinline__ void collide_body(const S* __restrict__ src, S* __restrict__ dst,
                                             const RT* __restrict__ rec,
                                             const double* __restrict__ Tf,
                                             int* __restrict__ status, const Geom& g,
                                             const Units& un, const BCDev& bc,
                                             const DevMech& mech, long long n) {
  constexpr int Q = Lat<D>::Q;
  const long long N = g.N;
  if (n >= N) return;
  const int tag = bc.tag ? bc.tag[n] : TAG_BULK;
  if (tag == TAG_SOLID) return;
  NodePar<D, M, RT> p;
  node_params<D, M, RT>(rec, Tf, g, un, bc, mech, n, tag, p);
  const int x = (int)(n % g.nx);
  const int y = (int)((n / g.nx) % g.ny);
  const int z = (int)(n / ((long long)g.nx * g.ny));
  // FP32: the species axis factors tabulated once per node in this thread's
  // shared-memory column (the solve's space, now free)
  extern __shared__ unsigned char smem_raw[];
  RT* tab = nullptr;
  RT* yztab = nullptr;
  if constexpr (sizeof(RT) == 4) {
    tab = reinterpret_cast<RT*>(smem_raw) + threadIdx.x;
    constexpr int NT = 2 * M * D * 3;
#pragma unroll
    for (int e = 0; e < NT; ++e)
      tab[e * kBS] = axis_factor<D, M, RT>(e, p.th, p.u, &p.V[0][0]);
  } else if constexpr (D == 3) {
    // FP64: the y- and z-axis factors, psi_c(x_s, theta_b + x_s^2) with
    // x_s = u_d (set 0) or u_d + V_bd (set 1)
    yztab = reinterpret_cast<RT*>(smem_raw) + threadIdx.x;
#pragma unroll
    for (int set = 0; set < 2; ++set)
#pragma unroll
      for (int b = 0; b < M; ++b)
#pragma unroll
        for (int d = 1; d < 3; ++d) {
          const RT xs = set ? p.u[d] + p.V[b][d] : p.u[d];
          const RT Ps = p.th[b] + xs * xs;
#pragma unroll
          for (int c = -1; c <= 1; ++c)
            yztab[(((set * M + b) * 2 + d - 1) * 3 + c + 1) * kBS] = psi1<RT>(c, xs, Ps);
        }
  }
  const RegPar<D, M, RT> ps(p, tab, yztab);
  // directions i = j + 9 k share (c_x, c_y) = direction j's
#pragma unroll 1
  for (int j = 0; j < 9; ++j) {
    XYPart<D, M, RT> h;
    xy_part<D, M, RT>(ps, cvel(j, 0), cvel(j, 1), h);
#pragma unroll 1
    for (int i = j; i < Q; i += 9) {
      RT fin[M + 1];
      load_direction<D, M, S, RT>(src, bc, tag, N, node_shift<D>(x, y, z, i, -1, g), i,
                                  g.codec, fin);
      collide_direction<D, M, S, RT>(ps, h, i, fin, dst, N, n, mech, g.codec);
    }
  }
}

// ---------------------------------------------------------------------------
// Split placement of the collision, for grids too small to fill the GPU at
// one thread per node: k_prep (one thread per node) stores each node's
// parameters field-major; k_coll gives every node kCollTPN threads (one warp
// per direction group, lanes over 32 consecutive nodes), stages the block's
// parameters and axis-factor tables in shared memory, and updates each
// direction as the fused kernel does.
template <int D, int M, typename RT>
__device__ __forceinline__ void prep_body(const RT* __restrict__ rec,
                                          const double* __restrict__ Tf, RT* __restrict__ cp,
                                          const Geom& g, const Units& un, const BCDev& bc,
                                          const DevMech& mech, long long n) {
  using CP = CPar<D, M>;
  const long long N = g.N;
  if (n >= N) return;
  const int tag = bc.tag ? bc.tag[n] : TAG_BULK;
  if (tag == TAG_SOLID) return;
  NodePar<D, M, RT> p;
  node_params<D, M, RT>(rec, Tf, g, un, bc, mech, n, tag, p);
#pragma unroll
  for (int b = 0; b < M; ++b) {
    cp[(CP::TH + b) * N + n] = p.th[b];
    cp[(CP::RS + b) * N + n] = p.rs[b];
#pragma unroll
    for (int d = 0; d < D; ++d) cp[(CP::V + b * D + d) * N + n] = p.V[b][d];
  }
#pragma unroll
  for (int a = 0; a < M - 1; ++a) {
    cp[(CP::CF + a) * N + n] = p.cF[a];
    cp[(CP::OM1 + a) * N + n] = p.om1[a];
    cp[(CP::HH + a) * N + n] = p.hh[a];
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    cp[(CP::U + d) * N + n] = p.u[d];
    cp[(CP::PEX + d) * N + n] = p.Pex[d];
    cp[(CP::W + d) * N + n] = p.W[d];
  }
  cp[CP::RHO * N + n] = p.rho;
  cp[CP::OM * N + n] = p.om;
  cp[CP::UL * N + n] = p.U;
  cp[CP::THETA * N + n] = p.theta;
}

constexpr int kCollNodes = kCollNodesPerBlock;   // nodes per block of k_coll (the lanes)
constexpr int kCollTPN = 9;      // threads per node (warps per block)

// shared-memory entries per node of k_coll: parameters, energy factors,
// species axis-factor tables
template <int D, int M> constexpr int coll_smem_entries() {
  return CPar<D, M>::NF + 6 * D + 2 * M * D * 3;
}

// Parameters of node j of the block, field f at s[f * kCollNodes + j].
template <int D, int M, typename RT> struct SmemPar {
  using CP = CPar<D, M>;
  static constexpr int AF = CP::NF, BF = CP::NF + 3 * D, TAB = CP::NF + 6 * D;
  const RT* s;
  int j;
  __device__ RT get(int f) const { return s[f * kCollNodes + j]; }
  __device__ RT rho() const { return get(CP::RHO); }
  __device__ RT om() const { return get(CP::OM); }
  __device__ RT U() const { return get(CP::UL); }
  __device__ RT u(int d) const { return get(CP::U + d); }
  __device__ RT Pex(int d) const { return get(CP::PEX + d); }
  __device__ RT W(int d) const { return get(CP::W + d); }
  __device__ RT rs(int a) const { return get(CP::RS + a); }
  __device__ RT cF(int a) const { return get(CP::CF + a); }
  __device__ RT om1(int a) const { return get(CP::OM1 + a); }
  __device__ RT hh(int a) const { return get(CP::HH + a); }
  __device__ RT Af(int d, int c) const { return get(AF + d * 3 + c + 1); }
  __device__ RT Bf(int d, int c) const { return get(BF + d * 3 + c + 1); }
  __device__ RT sp(int set, int b, int d, int c) const {
    return get(TAB + ((set * M + b) * D + d) * 3 + c + 1);
  }
};

// One block of TPN warps: nodes n0 .. n0 + 31.  sm holds coll_smem_entries *
// kCollNodes.  The Q directions, taken in the order k = 0 .. Q - 1 with
// direction (k / NZ) + 9 (k % NZ) (NZ = 3 in 3D: the directions of one
// (c_x, c_y) pair in a row), are dealt to the warps in contiguous chunks.
template <int D, int M, typename S, typename RT, int TPN = kCollTPN>
__device__ __forceinline__ void coll_block(const S* __restrict__ src, S* __restrict__ dst,
                                           const RT* __restrict__ cp, const Geom& g,
                                           const BCDev& bc, const DevMech& mech, long long n0,
                                           RT* __restrict__ sm) {
  using CP = CPar<D, M>;
  using SP = SmemPar<D, M, RT>;
  constexpr int Q = Lat<D>::Q;
  constexpr int NT = 2 * M * D * 3;
  const long long N = g.N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long n = n0 + lane;
  const int tag = n < N ? (bc.tag ? bc.tag[n] : TAG_BULK) : TAG_SOLID;
  const bool valid = tag != TAG_SOLID;
  for (int f = w; f < CP::NF; f += TPN)
    sm[f * kCollNodes + lane] = valid ? __ldcg(cp + f * N + n) : RT(0);
  __syncthreads();
  if (valid) {
    if (w == 0) {
      RT u[D], Af[D][3], Bf[D][3];
#pragma unroll
      for (int d = 0; d < D; ++d) u[d] = sm[(CP::U + d) * kCollNodes + lane];
      energy_factors<D, RT>(u, sm[CP::THETA * kCollNodes + lane], Af, Bf);
#pragma unroll
      for (int d = 0; d < D; ++d)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          sm[(SP::AF + d * 3 + k) * kCollNodes + lane] = Af[d][k];
          sm[(SP::BF + d * 3 + k) * kCollNodes + lane] = Bf[d][k];
        }
    }
    for (int e = w; e < NT; e += TPN) {
      const int c = e % 3 - 1;
      const int d = (e / 3) % D;
      const int b = (e / (3 * D)) % M;
      const int set = e / (3 * D * M);
      const RT ud = sm[(CP::U + d) * kCollNodes + lane];
      const RT xs = set ? ud + sm[(CP::V + b * D + d) * kCollNodes + lane] : ud;
      const RT Ps = sm[(CP::TH + b) * kCollNodes + lane] + xs * xs;
      sm[(SP::TAB + e) * kCollNodes + lane] =
          c == 0 ? RT(1) - Ps : (c > 0 ? RT(0.5) * (Ps + xs) : RT(0.5) * (Ps - xs));
    }
  }
  __syncthreads();
  if (!valid) return;
  const SP ps{sm, lane};
  const int x = (int)(n % g.nx);
  const int y = (int)((n / g.nx) % g.ny);
  const int z = (int)(n / ((long long)g.nx * g.ny));
  // software pipeline: the next direction's populations are in flight while
  // this one collides.  FP64 forms the (c_x, c_y) part once per pair and
  // keeps it in registers; FP32 forms it per direction, which keeps k_coll
  // within its 56-register budget.
  constexpr int NZ = D == 3 ? 3 : 1;
  constexpr int CH = (Q + TPN - 1) / TPN;
  const int k0 = w * CH, k1 = min(k0 + CH, Q);
  if (k0 >= k1) return;
  XYPart<D, M, RT> h;
  int jcur = -1;
  RT fa[M + 1], fb[M + 1];
  int i = k0 / NZ + 9 * (k0 % NZ);
  load_direction<D, M, S, RT>(src, bc, tag, N, node_shift<D>(x, y, z, i, -1, g), i, g.codec, fa);
#pragma unroll 1
  for (int k = k0; k < k1; ++k) {
    const int inext = k + 1 < k1 ? (k + 1) / NZ + 9 * ((k + 1) % NZ) : -1;
    if (inext >= 0)
      load_direction<D, M, S, RT>(src, bc, tag, N, node_shift<D>(x, y, z, inext, -1, g), inext,
                                  g.codec, fb);
    const int j = k / NZ;
    if (sizeof(RT) == 4 || j != jcur) {
      xy_part<D, M, RT>(ps, cvel(j, 0), cvel(j, 1), h);
      jcur = j;
    }
    collide_direction<D, M, S, RT>(ps, h, i, fa, dst, N, n, mech, g.codec);
#pragma unroll
    for (int l = 0; l <= M; ++l) fa[l] = fb[l];
    i = inext;
  }
}


#include "lbm_bnode.cuh"

// ---------------------------------------------------------------------------
// Single-domain kernels: one thread per node (moments, collision), one thread
// per interface node (k_bnode: boundary reconstruction and record).
// Node sets: every node, the nodes without boundary reconstruction (the
// bulk), or the interface nodes (whose sub-steps follow k_bnode, on a side
// stream concurrent with the bulk).
enum { NODES_ALL = 0, NODES_BULK = 1, NODES_INTERFACE = 2 };

template <int D, int M, typename S, typename RT>
__global__ void __launch_bounds__(128, kMomentsMinBlocks<RT>)
k_moments(const S* __restrict__ src, RT* __restrict__ rec, double* __restrict__ Tf,
          int* __restrict__ status, const __grid_constant__ Geom g,
          const __grid_constant__ Units un, const __grid_constant__ BCDev bc,
          const __grid_constant__ DevMech mech, int chem_inline, int node_set) {
  // node_set: NODES_ALL or NODES_BULK
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (node_set == NODES_BULK && bc.tag && n < g.N && bc.tag[n] >= 0) return;
  moments_body<D, M, S, RT>(src, rec, Tf, status, g, un, bc, mech, n, chem_inline);
}

// reaction sub-steps, L lanes per node, 128 threads per block.  Node sets:
// every node, the nodes without boundary reconstruction (their chemistry
// runs beside the boundary kernel on the side stream), or the interface
// nodes (entry `first` of the interface list, after the boundary kernel)
template <int D, int M, typename RT, int L>
__device__ __forceinline__ void chem_entry(RT* rec, const double* Tf, int* status, long long N,
                                           const int* tag, const Units& un, const DevMech& m,
                                           long long first, int node_set, const int* if_node,
                                           int n_if) {
  const int lane = threadIdx.x & 31;
  const long long idx = first + threadIdx.x / L;
  long long n = idx;
  if (node_set == NODES_INTERFACE) {                    // the whole group leaves
    if (idx >= n_if) return;
    n = if_node[idx];
  } else {
    if (n >= N) return;
    if (tag && (tag[n] == TAG_SOLID || (node_set == NODES_BULK && tag[n] >= 0))) return;
  }
  const unsigned gmask = (L == 32 ? 0xffffffffu : ((1u << L) - 1u) << (lane & ~(L - 1)));
  chem_lanes_body<D, M, RT, L>(rec, Tf, status, N, tag, un, m, n, lane & (L - 1), gmask);
}

template <int D, int M, typename RT, int L>
__global__ void __launch_bounds__(128)
k_chem(RT* __restrict__ rec, const double* __restrict__ Tf, int* __restrict__ status,
       long long N, const int* __restrict__ tag, const __grid_constant__ Units un,
       const DevMech* __restrict__ mech, int node_set, const int* __restrict__ if_node,
       int n_if) {
  chem_entry<D, M, RT, L>(rec, Tf, status, N, tag, un, *mech, blockIdx.x * (128LL / L), node_set,
                          if_node, n_if);
}

// moments and reaction sub-steps, L lanes per node, 128 threads per block,
// over every node or the nodes without boundary reconstruction
template <int D, int M, typename S, typename RT, int L>
__global__ void __launch_bounds__(128)
k_mchem(const S* __restrict__ src, RT* __restrict__ rec, double* __restrict__ Tf,
        int* __restrict__ status, const __grid_constant__ Geom g,
        const __grid_constant__ Units un, const __grid_constant__ BCDev bc,
        const __grid_constant__ DevMech mech, const DevMech* __restrict__ mech_g,
        int node_set) {
  const int lane = threadIdx.x & 31;
  const long long n = blockIdx.x * (128LL / L) + threadIdx.x / L;
  if (n >= g.N) return;                                  // the whole group leaves
  const int tag = bc.tag ? bc.tag[n] : TAG_BULK;
  if (tag == TAG_SOLID || (node_set == NODES_BULK && tag >= 0)) return;
  const unsigned gmask = ((1u << L) - 1u) << (lane & ~(L - 1));
  mchem_body<D, M, S, RT, L>(src, rec, Tf, status, g, un, bc, mech, *mech_g, n, tag,
                             lane & (L - 1), gmask);
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

template <int D, int M, typename RT>
__global__ void __launch_bounds__(128)
k_prep(const RT* __restrict__ rec, const double* __restrict__ Tf, RT* __restrict__ cp,
       const __grid_constant__ Geom g, const __grid_constant__ Units un,
       const __grid_constant__ BCDev bc, const __grid_constant__ DevMech mech) {
  prep_body<D, M, RT>(rec, Tf, cp, g, un, bc, mech,
                      blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// FP32: four 288-thread blocks per SM (at most 56 registers), so a grid of
// the 16k-node flame fits the GPU in one wave; FP64 would spill
template <int D, int M, typename S, typename RT>
__global__ void __launch_bounds__(32 * kCollTPN, sizeof(RT) == 4 ? 4 : 1)
k_coll(const S* __restrict__ src, S* __restrict__ dst, const RT* __restrict__ cp,
       const __grid_constant__ Geom g, const __grid_constant__ BCDev bc,
       const __grid_constant__ DevMech mech) {
  extern __shared__ __align__(16) unsigned char coll_raw[];
  coll_block<D, M, S, RT>(src, dst, cp, g, bc, mech, blockIdx.x * (long long)kCollNodes,
                          reinterpret_cast<RT*>(coll_raw));
}

// One thread per interface node: reconstruction and record (lbm_bnode.cuh);
// the interface nodes' reaction sub-steps follow in k_chem.
template <int D, int M, typename S>
__global__ void __launch_bounds__(kBnd)
k_bnode(const S* __restrict__ src, const __grid_constant__ BCDev bc, double* __restrict__ Tf,
        int* __restrict__ status, const __grid_constant__ Geom g,
        const __grid_constant__ Units un, const __grid_constant__ DevMech mech,
        typename ComputeType<S>::type* __restrict__ rec) {
  using R = typename ComputeType<S>::type;
  extern __shared__ __align__(16) unsigned char bnd_raw[];
  const int k = blockIdx.x * kBnd + threadIdx.x;
  if (k >= bc.n_if) return;
  bnode_body<D, M, S, R>(src, bc, rec, Tf, status, g, un, mech, k,
                         reinterpret_cast<R*>(bnd_raw) + threadIdx.x,
                         reinterpret_cast<long long*>(
                             bnd_raw + sizeof(R) * bnode_col_entries<D, M>() * kBnd) +
                             threadIdx.x);
}

// ---------------------------------------------------------------------------
// Batched kernels: the grid is the concatenation of every domain's tiles; a
// block finds its domain by binary search over the domains' first blocks.
enum { GRID_NODE = 0, GRID_BOUNDARY = 1, GRID_CHEM = 2, GRID_COLL = 3, GRID_BNODE = 4 };
__device__ __forceinline__ int domain_of_block(const DomainDev* __restrict__ d, int ndom,
                                               int b, int grid) {
  int lo = 0, hi = ndom - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int first = grid == GRID_BOUNDARY ? d[mid].bblock_begin
                      : grid == GRID_CHEM   ? d[mid].cblock_begin
                      : grid == GRID_COLL   ? d[mid].kblock_begin
                      : grid == GRID_BNODE  ? d[mid].tblock_begin
                                            : d[mid].block_begin;
    if (first <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Every batched kernel walks its grid's blocks b = blockIdx.x, + gridDim.x,
// ... below nblk: launched with one block per tile it runs each tile once;
// launched persistent (a grid sized to the blocks resident on the GPU) each
// block processes several tiles in turn.
//
// The block's domain descriptor is copied to shared memory whenever the
// block moves to another domain (k block-uniform, every thread calls it),
// so the bodies read its fields from shared memory rather than reloading
// them from global memory around every store.
struct BlockDomain {
  unsigned char* raw;   // __shared__ storage of sizeof(DomainDev) bytes
  int cur = -1;
  __device__ const DomainDev& get(const DomainDev* __restrict__ doms, int k) {
    if (k != cur) {
      __syncthreads();   // the previous domain's readers are done
      const unsigned* src = reinterpret_cast<const unsigned*>(doms + k);
      unsigned* dst = reinterpret_cast<unsigned*>(raw);
      for (int i = threadIdx.x; i < (int)(sizeof(DomainDev) / 4); i += blockDim.x)
        dst[i] = src[i];
      __syncthreads();
      cur = k;
    }
    return *reinterpret_cast<const DomainDev*>(raw);
  }
};
static_assert(sizeof(DomainDev) % 4 == 0, "domain descriptor copied in 4-byte words");
#define LBM_BLOCK_DOMAIN(name)                                          \
  __shared__ __align__(16) unsigned char name##_raw[sizeof(DomainDev)]; \
  BlockDomain name{name##_raw}
template <int D, int M, typename S, typename RT>
__global__ void __launch_bounds__(128, kMomentsMinBlocks<RT>)
k_moments_batch(const DomainDev* __restrict__ doms, int ndom, int parity, int chem_inline,
                int node_set, int nblk) {
  LBM_BLOCK_DOMAIN(bd);
  // node_set: NODES_ALL or NODES_BULK (the interface nodes' records come from
  // k_bnode_batch)
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const DomainDev& d = bd.get(doms, domain_of_block(doms, ndom, b, GRID_NODE));
    const int c = d.cur0 ^ parity;
    const long long n = (b - d.block_begin) * (long long)blockDim.x + threadIdx.x;
    if (node_set == NODES_BULK && d.bc.tag && n < d.g.N && d.bc.tag[n] >= 0) continue;
    moments_body<D, M, S, RT>(static_cast<const S*>(d.pops[c]), static_cast<RT*>(d.rec), d.Tf,
                              d.status, d.g, d.un, d.bc, *d.mech, n, chem_inline);
  }
}

// NODES_INTERFACE: the interface-chemistry grid (128 / L interface nodes
// per block, L lanes each, as k_chem)
template <int D, int M, typename RT, int L>
__global__ void __launch_bounds__(128)
k_chem_batch(const DomainDev* __restrict__ doms, int ndom, int node_set, int nblk) {
  LBM_BLOCK_DOMAIN(bd);
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    if (node_set == NODES_INTERFACE) {
      const DomainDev& d = bd.get(doms, domain_of_block(doms, ndom, b, GRID_BOUNDARY));
      chem_entry<D, M, RT, L>(static_cast<RT*>(d.rec), d.Tf, d.status, d.g.N, d.bc.tag, d.un,
                              *d.mech, (b - d.bblock_begin) * (128LL / L), NODES_INTERFACE,
                              d.bc.if_node, d.bc.n_if);
    } else {
      const DomainDev& d = bd.get(doms, domain_of_block(doms, ndom, b, GRID_CHEM));
      chem_entry<D, M, RT, L>(static_cast<RT*>(d.rec), d.Tf, d.status, d.g.N, d.bc.tag, d.un,
                              *d.mech, (b - d.cblock_begin) * (128LL / L), node_set, nullptr,
                              0);
    }
  }
}

// the chemistry grid (128 / L nodes per block)
template <int D, int M, typename S, typename RT, int L>
__global__ void __launch_bounds__(128)
k_mchem_batch(const DomainDev* __restrict__ doms, int ndom, int parity, int node_set,
              int nblk) {
  LBM_BLOCK_DOMAIN(bd);
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const DomainDev& d = bd.get(doms, domain_of_block(doms, ndom, b, GRID_CHEM));
    const int c = d.cur0 ^ parity;
    const int lane = threadIdx.x & 31;
    const long long n = (b - d.cblock_begin) * (128LL / L) + threadIdx.x / L;
    if (n >= d.g.N) continue;
    const int tag = d.bc.tag ? d.bc.tag[n] : TAG_BULK;
    if (tag == TAG_SOLID || (node_set == NODES_BULK && tag >= 0)) continue;
    const unsigned gmask = ((1u << L) - 1u) << (lane & ~(L - 1));
    mchem_body<D, M, S, RT, L>(static_cast<const S*>(d.pops[c]), static_cast<RT*>(d.rec), d.Tf,
                               d.status, d.g, d.un, d.bc, *d.mech, *d.mech, n, tag,
                               lane & (L - 1), gmask);
  }
}

template <int D, int M, typename S, typename RT>
__global__ void __launch_bounds__(128)
k_collide_batch(const DomainDev* __restrict__ doms, int ndom, int parity, int nblk) {
  LBM_BLOCK_DOMAIN(bd);
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const DomainDev& d = bd.get(doms, domain_of_block(doms, ndom, b, GRID_NODE));
    const int c = d.cur0 ^ parity;
    collide_body<D, M, S, RT>(static_cast<const S*>(d.pops[c]),
                              static_cast<S*>(const_cast<void*>(d.pops[1 - c])),
                              static_cast<const RT*>(d.rec), d.Tf, d.status, d.g, d.un, d.bc,
                              *d.mech, (b - d.block_begin) * (long long)blockDim.x + threadIdx.x);
  }
}

template <int D, int M, typename RT>
__global__ void __launch_bounds__(128)
k_prep_batch(const DomainDev* __restrict__ doms, int ndom, int nblk) {
  LBM_BLOCK_DOMAIN(bd);
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const DomainDev& d = bd.get(doms, domain_of_block(doms, ndom, b, GRID_NODE));
    prep_body<D, M, RT>(static_cast<const RT*>(d.rec), d.Tf, static_cast<RT*>(d.cpar), d.g,
                        d.un, d.bc, *d.mech,
                        (b - d.block_begin) * (long long)blockDim.x + threadIdx.x);
  }
}

template <int D, int M, typename S, typename RT>
__global__ void __launch_bounds__(32 * kCollTPN, sizeof(RT) == 4 ? 4 : 1)
k_coll_batch(const DomainDev* __restrict__ doms, int ndom, int parity, int nblk) {
  LBM_BLOCK_DOMAIN(bd);
  extern __shared__ __align__(16) unsigned char coll_raw[];
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const DomainDev& d = bd.get(doms, domain_of_block(doms, ndom, b, GRID_COLL));
    const int c = d.cur0 ^ parity;
    // the previous tile's threads are done with the shared memory
    if (b != blockIdx.x) __syncthreads();
    coll_block<D, M, S, RT>(static_cast<const S*>(d.pops[c]),
                            static_cast<S*>(const_cast<void*>(d.pops[1 - c])),
                            static_cast<const RT*>(d.cpar), d.g, d.bc, *d.mech,
                            (b - d.kblock_begin) * (long long)kCollNodes,
                            reinterpret_cast<RT*>(coll_raw));
  }
}

// One thread per interface node over every domain (the batched k_bnode).
template <int D, int M, typename S>
__global__ void __launch_bounds__(kBnd)
k_bnode_batch(const DomainDev* __restrict__ doms, int ndom, int parity, int nblk) {
  LBM_BLOCK_DOMAIN(bd);
  using R = typename ComputeType<S>::type;
  extern __shared__ __align__(16) unsigned char bnd_raw[];
  R* col = reinterpret_cast<R*>(bnd_raw) + threadIdx.x;
  long long* sncol =
      reinterpret_cast<long long*>(bnd_raw + sizeof(R) * bnode_col_entries<D, M>() * kBnd) +
      threadIdx.x;
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const DomainDev& d = bd.get(doms, domain_of_block(doms, ndom, b, GRID_BNODE));
    const int k = (b - d.tblock_begin) * kBnd + threadIdx.x;
    if (k >= d.bc.n_if) continue;
    bnode_body<D, M, S, R>(static_cast<const S*>(d.pops[d.cur0 ^ parity]), d.bc,
                           static_cast<R*>(d.rec), d.Tf, d.status, d.g, d.un, *d.mech, k, col,
                           sncol);
  }
}

// ---------------------------------------------------------------------------
// The whole batched step as one persistent launch over a work-list (PItem,
// lbm_internal.h).  Dependencies go through sync words: a producer block
// fences its stores and then releases a count or a flag; a consumer's first
// thread acquires it (bounded by timeout_ns on the global timer, after which
// it sets the abort word and ST_TIMEOUT in the item's domain) before the
// block reads.  Data written earlier in the same launch is read only after
// such an acquire, and the reads that could meet a line fetched before its
// last write (the temperature guesses and the collision parameters) bypass
// the L1 (ld.global.cg).
// Reaction sub-steps of interface node n (Sec. 2.4 Eq. R3) by one thread,
// from the record the boundary reconstruction left (post-stream species
// densities in the increment slots), as chem_lanes_body does with lanes.
template <int D, int M, typename RT>
__device__ __forceinline__ void iface_substeps(RT* __restrict__ rec, const double* __restrict__ Tf,
                                               int* __restrict__ status, long long N,
                                               const Units& un, const DevMech& mech, long long n,
                                               void* chem_slice) {
  using RC = Rec<D, M>;
  const RT rho = __ldcg(rec + RC::RHO * N + n);
  RT usq = RT(0);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const RT ud = __ldcg(rec + (RC::U + d) * N + n);
    usq += ud * ud;
  }
  const RT ER = __ldcg(rec + RC::E * N + n);
  RT rs[M];
  RT last = rho;
#pragma unroll
  for (int a = 0; a < M - 1; ++a) {
    rs[a] = __ldcg(rec + (RC::DRHO + a) * N + n);
    last -= rs[a];
  }
  rs[M - 1] = last;
  RT dr[M - 1];
  node_substeps<M, RT, true>(rs, rho, ER, usq, __ldcg(Tf + n), un, mech, status, chem_slice, dr);
#pragma unroll
  for (int a = 0; a < M - 1; ++a) rec[(RC::DRHO + a) * N + n] = dr[a];
}

// The interface nodes' sub-steps with one thread per node (grids with at
// least kIfChemThreadNodes interface nodes, which fill the GPU this way):
// the same arithmetic as the lane groups of k_chem without their redundant
// per-lane temperature and Gibbs evaluations.  Float-float rate arrays in
// dynamic shared memory (chem_slice_bytes).
constexpr long long kIfChemThreadNodes = 152LL * 128;

template <int D, int M, typename RT>
__global__ void __launch_bounds__(kChemThreads)
k_iface_chem(RT* __restrict__ rec, const double* __restrict__ Tf, int* __restrict__ status,
             long long N, const int* __restrict__ if_node, int n_if,
             const __grid_constant__ Units un, const DevMech* __restrict__ mech) {
  extern __shared__ __align__(16) unsigned char ic_raw[];
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n_if) return;
  iface_substeps<D, M, RT>(rec, Tf, status, N, un, *mech, if_node[k], ic_raw);
}

// The same over the interface nodes of several handles (batch plans whose
// handles hold at least kIfChemThreadNodes interface nodes in all), on the
// thread-per-interface-node grid of k_bnode_batch.
template <int D, int M, typename RT>
__global__ void __launch_bounds__(kBnd)
k_iface_chem_batch(const DomainDev* __restrict__ doms, int ndom, int nblk) {
  LBM_BLOCK_DOMAIN(bd);
  extern __shared__ __align__(16) unsigned char icb_raw[];
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const DomainDev& d = bd.get(doms, domain_of_block(doms, ndom, b, GRID_BNODE));
    const long long k = (b - d.tblock_begin) * (long long)kBnd + threadIdx.x;
    if (k >= d.bc.n_if) continue;
    iface_substeps<D, M, RT>(static_cast<RT*>(d.rec), d.Tf, d.status, d.g.N, d.un, *d.mech,
                             d.bc.if_node[k], icb_raw);
  }
}

template <typename RT> constexpr int kPersistMinBlocks = sizeof(RT) == 8 ? 2 : 3;
constexpr int kPersistCollWarps = kPersistThreads / 32;

template <int D, int M, typename S, typename RT>
__global__ void __launch_bounds__(kPersistThreads, kPersistMinBlocks<RT>)
k_step_persist(const DomainDev* __restrict__ doms, int ndom, int parity,
               const PItem* __restrict__ items, int nitems, int npt, int* __restrict__ sync,
               long long timeout_ns) {
  LBM_BLOCK_DOMAIN(bd);
  using R = typename ComputeType<S>::type;
  constexpr int Q = Lat<D>::Q;
  extern __shared__ __align__(16) unsigned char ps_raw[];
  __shared__ int s_item, s_go;
  int* const next = sync;
  int* const abort_w = sync + 1;
  int* const done1 = sync + kSyncHead;
  int* const pflag = done1 + ndom;
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = atomicAdd(next, 1);
      int go = it < nitems && !ld_acquire_gpu(abort_w);
      if (go) {
        const PItem w = items[it];
        if (w.kind == PI_PREP || w.kind == PI_COLLIDE)
          go = wait_at_least(done1 + w.dom, w.dep, abort_w, timeout_ns);
        else if (w.kind == PI_COLL) go = wait_at_least(pflag + w.dep, 1, abort_w, timeout_ns);
        if (!go) atomicOr(doms[w.dom].status, ST_TIMEOUT);
      }
      s_item = it;
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const PItem w = items[s_item];
    const DomainDev& d = bd.get(doms, w.dom);
    const int c = d.cur0 ^ parity;
    const S* src = static_cast<const S*>(d.pops[c]);
    RT* rec = static_cast<RT*>(d.rec);
    if (w.kind == PI_BND) {
      // two groups of kBnd threads, each with its boundary columns
      const int grp = threadIdx.x / kBnd, t = threadIdx.x % kBnd;
      constexpr int E = bnode_col_entries<D, M>();
      R* col = reinterpret_cast<R*>(ps_raw) + grp * E * kBnd + t;
      long long* sncol =
          reinterpret_cast<long long*>(ps_raw + sizeof(R) * E * kBnd * (kPersistThreads / kBnd)) +
          grp * Q * kBnd + t;
      const long long k = w.first + threadIdx.x;
      if (k < d.bc.n_if)
        bnode_body<D, M, S, R>(src, d.bc, static_cast<R*>(d.rec), d.Tf, d.status, d.g, d.un,
                               *d.mech, (int)k, col, sncol);
      __syncthreads();   // the columns become the sub-steps' shared-memory slices
      if (k < d.bc.n_if)
        iface_substeps<D, M, RT>(rec, d.Tf, d.status, d.g.N, d.un, *d.mech, d.bc.if_node[k],
                                 ps_raw);
    } else if (w.kind == PI_MOM) {
      for (int j = 0; j < npt; ++j) {
        const long long n = w.first + (long long)j * kPersistThreads + threadIdx.x;
        if (n >= d.g.N) break;
        if (d.bc.tag && d.bc.tag[n] >= 0) continue;   // interface node: PI_BND
        moments_body<D, M, S, RT, true>(src, rec, d.Tf, d.status, d.g, d.un, d.bc, *d.mech, n, 1,
                                        ps_raw);
      }
    } else if (w.kind == PI_PREP) {
      for (int j = 0; j < npt; ++j)
        prep_body<D, M, RT>(rec, d.Tf, static_cast<RT*>(d.cpar), d.g, d.un, d.bc, *d.mech,
                            w.first + (long long)j * kPersistThreads + threadIdx.x);
    } else if (w.kind == PI_COLLIDE) {
      for (int j = 0; j < npt; ++j)
        collide_body<D, M, S, RT>(src, static_cast<S*>(const_cast<void*>(d.pops[1 - c])), rec,
                                  d.Tf, d.status, d.g, d.un, d.bc, *d.mech,
                                  w.first + (long long)j * kPersistThreads + threadIdx.x);
    } else {
      coll_block<D, M, S, RT, kPersistCollWarps>(
          src, static_cast<S*>(const_cast<void*>(d.pops[1 - c])),
          static_cast<const RT*>(d.cpar), d.g, d.bc, *d.mech, w.first,
          reinterpret_cast<RT*>(ps_raw));
    }
    // publish the item: every thread's stores, then the block's release
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      if (w.kind == PI_BND || w.kind == PI_MOM) add_release_gpu(done1 + w.dom, 1);
      else if (w.kind == PI_PREP) st_release_gpu(pflag + w.flag, 1);
    }
  }
}

// dynamic shared memory of k_step_persist: the largest of its items' needs
// (split: parameter and collision items; else fused collision items)
template <int D, int M, typename S, typename RT> constexpr size_t persist_smem(bool split) {
  using R = typename ComputeType<S>::type;
  const size_t bnd = bnode_smem<D, M, R>() * (kPersistThreads / kBnd);
  const size_t prep = (size_t)M * M * kBS * sizeof(RT);
  const size_t coll = (size_t)coll_smem_entries<D, M>() * kCollNodes * sizeof(RT);
  const size_t fused = (size_t)collide_smem_entries<D, M, RT>() * kBS * sizeof(RT);
  const size_t chem = kFF<RT> ? chem_slice_bytes<M, ff>() : 0;
  size_t m = bnd > chem ? bnd : chem;
  if (split) {
    m = m > prep ? m : prep;
    m = m > coll ? m : coll;
  } else {
    m = m > fused ? m : fused;
  }
  return m;
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
      pops[(long long)(a * Q + i) * N + n] = Codec<S>::enc(p, g.codec, a * Q + i);
    }
    double f = rho;
    for (int d = 0; d < D; ++d) f *= psi1<double>(c[d], u[d], theta + u[d] * u[d]);
    pops[(long long)((M - 1) * Q + i) * N + n] = Codec<S>::enc(f, g.codec, (M - 1) * Q + i);
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
    pops[(long long)(M * Q + i) * N + n] =
        Codec<S>::enc(rho * (U_lat * prodA + sumB), g.codec, M * Q + i);
  }
  (void)usq;
  Tf[n] = T;
}

// ---------------------------------------------------------------------------
// Flame diagnostics of the stored state (Sec. 5.3 quantities), one pass:
// per node the moments, T by Newton from the guess, the mass production
// rates and q = -sum_a H_a(T) rho_dot_a (W/m^3, H_a with the enthalpy of
// formation); per block the sum of q, the largest q with its node (the
// smallest index among equal maxima), the largest T and |u| (m/s).  FP64
// whatever the storage.
template <int D, int M, typename S>
__global__ void __launch_bounds__(128)
k_diag(const S* __restrict__ pops, const double* __restrict__ Tf, const int* __restrict__ tag,
       DiagPart* __restrict__ part, int* __restrict__ status, Geom g, Units un,
       const __grid_constant__ DevMech mech, int x0, int x1) {
  constexpr int Q = Lat<D>::Q;
  __shared__ double s_sum[128], s_qmax[128], s_T[128], s_u[128];
  __shared__ long long s_n[128];
  const long long N = g.N;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double q = 0.0, qmax = -INFINITY, Tmax = -INFINITY, umax = -INFINITY;
  long long nmax = LLONG_MAX;
  const int xn = (int)(n % g.nx);   // the nodes with x in [x0, x1) only
  if (n < N && xn >= x0 && xn < x1 && !(tag && tag[n] == TAG_SOLID)) {
    double rho = 0.0, rhoE = 0.0, j[D], rs[M];
    for (int d = 0; d < D; ++d) j[d] = 0.0;
    for (int a = 0; a < M; ++a) rs[a] = 0.0;
    for (int i = 0; i < Q; ++i) {
      for (int a = 0; a < M - 1; ++a) rs[a] += ldp(pops, N, n, a * Q + i, g.codec);
      const double f = ldp(pops, N, n, (M - 1) * Q + i, g.codec);
      rho += f;
      for (int d = 0; d < D; ++d) j[d] += cvel(i, d) * f;
      rhoE += ldp(pops, N, n, M * Q + i, g.codec);
    }
    rs[M - 1] = rho;
    for (int a = 0; a < M - 1; ++a) rs[M - 1] -= rs[a];
    double Y[M], usq = 0.0;
    for (int a = 0; a < M; ++a) Y[a] = rs[a] / rho;
    for (int d = 0; d < D; ++d) usq += (j[d] / rho) * (j[d] / rho);
    bool ok;
    const double T = newton_T<M>(mech, Y, (rhoE / rho - 0.5 * usq) * un.c * un.c, Tf[n],
                                 un.newton_max_iter, un.newton_rtol, ok);
    if (!ok) atomicOr(status, ST_NEWTON);
    double rdot[M];
    production_rates<M>(mech, T, rs, rdot);
    for (int a = 0; a < M; ++a) q -= (species_U(mech, a, T) + mech.Ra[a] * T) * rdot[a];
    qmax = q;
    nmax = n;
    Tmax = T;
    umax = sqrt(usq) * un.c;
  }
  const int t = threadIdx.x;
  s_sum[t] = q;
  s_qmax[t] = qmax;
  s_n[t] = nmax;
  s_T[t] = Tmax;
  s_u[t] = umax;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (t < o) {
      s_sum[t] += s_sum[t + o];
      if (s_qmax[t + o] > s_qmax[t] || (s_qmax[t + o] == s_qmax[t] && s_n[t + o] < s_n[t])) {
        s_qmax[t] = s_qmax[t + o];
        s_n[t] = s_n[t + o];
      }
      s_T[t] = fmax(s_T[t], s_T[t + o]);
      s_u[t] = fmax(s_u[t], s_u[t + o]);
    }
    __syncthreads();
  }
  if (t == 0) part[blockIdx.x] = DiagPart{s_sum[0], s_qmax[0], s_n[0], s_T[0], s_u[0]};
}

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
    for (int a = 0; a < M - 1; ++a) rs[a] += ldp(pops, N, n, a * Q + i, g.codec);
    const double f = ldp(pops, N, n, (M - 1) * Q + i, g.codec);
    rho += f;
    for (int d = 0; d < D; ++d) j[d] += cvel(i, d) * f;
    rhoE += ldp(pops, N, n, M * Q + i, g.codec);
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


// ---------------------------------------------------------------------------
// dispatch

static inline unsigned blocks_for(long long N, int bs) { return (unsigned)((N + bs - 1) / bs); }

// dynamic shared memory of the collision kernels and of k_prep (bytes)
template <int D, int M, typename RT> constexpr size_t fused_smem() {
  return (size_t)collide_smem_entries<D, M, RT>() * kBS * sizeof(RT);
}
template <int D, int M, typename RT> constexpr size_t prep_smem() {
  return (size_t)M * M * kBS * sizeof(RT);
}
template <int D, int M, typename RT> constexpr size_t coll_smem() {
  return (size_t)coll_smem_entries<D, M>() * kCollNodes * sizeof(RT);
}

// Kernel attributes (shared memory above the 48 KB default) of every kernel a
// step may launch; idempotent, and required before a stream capture, where
// attribute calls are not recorded.
template <int D, int M, typename S, typename RT>
static cudaError_t prepare_impl() {
  cudaError_t e = cudaSuccess;
  auto big = [&](const void* f, size_t bytes) {
    if (e == cudaSuccess && bytes > 48 * 1024)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  big((const void*)k_collide<D, M, S, RT>, fused_smem<D, M, RT>());
  big((const void*)k_collide_batch<D, M, S, RT>, fused_smem<D, M, RT>());
  big((const void*)k_prep<D, M, RT>, prep_smem<D, M, RT>());
  big((const void*)k_prep_batch<D, M, RT>, prep_smem<D, M, RT>());
  big((const void*)k_coll<D, M, S, RT>, coll_smem<D, M, RT>());
  big((const void*)k_coll_batch<D, M, S, RT>, coll_smem<D, M, RT>());
  big((const void*)k_bnode<D, M, S>, bnode_smem<D, M, RT>());
  big((const void*)k_bnode_batch<D, M, S>, bnode_smem<D, M, RT>());
  big((const void*)k_step_persist<D, M, S, RT>,
      std::max(persist_smem<D, M, S, RT>(true), persist_smem<D, M, S, RT>(false)));
  return e;
}

template <int D, int M, typename RT>
static void launch_chem(const Launch& lc, cudaStream_t s, RT* rec, const double* Tf,
                        int* status, long long N, const BCDev& bc, const Units& un,
                        const DevMech* mech, int node_set) {
  if (node_set == NODES_INTERFACE && bc.n_if >= kIfChemThreadNodes) {
    const size_t sm = kFF<RT> ? chem_slice_bytes<M, ff>() : 0;
    k_iface_chem<D, M, RT><<<blocks_for(bc.n_if, kChemThreads), kChemThreads, sm, s>>>(
        rec, Tf, status, N, bc.if_node, bc.n_if, un, mech);
    return;
  }
  // fewer interface nodes: on the critical path, 8 lanes each
  const int lanes = node_set == NODES_INTERFACE ? 8 : lc.chem_lanes;
  const long long n = node_set == NODES_INTERFACE ? bc.n_if : N;
  const unsigned nblk = blocks_for(n, 128 / lanes);
  if (nblk == 0) return;
  if (lanes == 4)
    k_chem<D, M, RT, 4><<<nblk, 128, 0, s>>>(rec, Tf, status, N, bc.tag, un, mech, node_set,
                                             bc.if_node, bc.n_if);
  else
    k_chem<D, M, RT, 8><<<nblk, 128, 0, s>>>(rec, Tf, status, N, bc.tag, un, mech, node_set,
                                             bc.if_node, bc.n_if);
}

// prepare_impl once per device and instantiation
template <int D, int M, typename S, typename RT>
static cudaError_t prepare_once() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load() & bit) return cudaSuccess;
  e = prepare_impl<D, M, S, RT>();
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

template <int D, int M, typename S, typename RT>
static cudaError_t step_impl(const DevMech& mech, const StepArgs& a, cudaStream_t s,
                             int which) {
  const int bs = kBS;
  const unsigned nb = blocks_for(a.g.N, bs);
  const cudaError_t pe = prepare_once<D, M, S, RT>();
  if (pe != cudaSuccess) return pe;
  const Launch& lc = a.lc;
  const bool chem_sep = lc.chem_lanes > 1 && a.mech_dev;
  const bool split = lc.coll_split && a.cpar;
  if (which != 1) {
    const S* src = static_cast<const S*>(a.src);
    RT* rec = reinterpret_cast<RT*>(a.rec);
    // chem_lanes > 1: the bulk nodes' moments and reaction sub-steps in one
    // kernel with chem_lanes lanes per node (k_mchem); the boundary warps
    // write their nodes' records and the interface nodes' sub-steps follow
    // in k_chem.  chem_lanes = 1: k_moments with the sub-steps inline, the
    // interface nodes' moments after the boundary kernel.
    auto mchem = [&](cudaStream_t st, int node_set) {
      const unsigned nbm = blocks_for(a.g.N, 128 / lc.chem_lanes);
      if (lc.chem_lanes == 4)
        k_mchem<D, M, S, RT, 4><<<nbm, 128, 0, st>>>(src, rec, a.Tfield, a.status, a.g, a.un,
                                                     a.bc, mech, a.mech_dev, node_set);
      else
        k_mchem<D, M, S, RT, 8><<<nbm, 128, 0, st>>>(src, rec, a.Tfield, a.status, a.g, a.un,
                                                     a.bc, mech, a.mech_dev, node_set);
    };
    // the boundary kernel and the interface nodes' sub-steps run on a side
    // stream beside the bulk moments.  Interface nodes need the handle's
    // device copy of the mechanism (every handle has one; the
    // allocation-free step accepts no interface nodes).
    if (a.bc.n_if > 0 && !a.mech_dev) return cudaErrorInvalidValue;
    const bool fork = a.bc.n_if > 0 && a.side && a.ev_fork && a.ev_join;
    if (fork) {
      cudaError_t e = cudaEventRecord(a.ev_fork, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(a.side, a.ev_fork, 0);
      if (e != cudaSuccess) return e;
      k_bnode<D, M, S><<<blocks_for(a.bc.n_if, kBnd), kBnd, bnode_smem<D, M, RT>(), a.side>>>(
          src, a.bc, a.Tfield, a.status, a.g, a.un, mech, rec);
      launch_chem<D, M, RT>(lc, a.side, rec, a.Tfield, a.status, a.g.N, a.bc, a.un,
                            a.mech_dev, NODES_INTERFACE);
      e = cudaEventRecord(a.ev_join, a.side);
      if (e != cudaSuccess) return e;
      if (chem_sep)
        mchem(s, NODES_BULK);
      else
        k_moments<D, M, S, RT><<<nb, bs, 0, s>>>(src, rec, a.Tfield, a.status, a.g, a.un, a.bc,
                                                 mech, 1, NODES_BULK);
      e = cudaStreamWaitEvent(s, a.ev_join, 0);
      if (e != cudaSuccess) return e;
    } else {
      const bool bnd = a.bc.n_if > 0;
      if (bnd)
        k_bnode<D, M, S><<<blocks_for(a.bc.n_if, kBnd), kBnd, bnode_smem<D, M, RT>(), s>>>(
            src, a.bc, a.Tfield, a.status, a.g, a.un, mech, rec);
      if (chem_sep)
        mchem(s, bnd ? NODES_BULK : NODES_ALL);
      else
        k_moments<D, M, S, RT><<<nb, bs, 0, s>>>(src, rec, a.Tfield, a.status, a.g, a.un, a.bc,
                                                 mech, 1, bnd ? NODES_BULK : NODES_ALL);
      if (bnd)
        launch_chem<D, M, RT>(lc, s, rec, a.Tfield, a.status, a.g.N, a.bc, a.un, a.mech_dev,
                              NODES_INTERFACE);
    }
  }
  if (which != 0) {
    if (split) {
      k_prep<D, M, RT><<<nb, bs, prep_smem<D, M, RT>(), s>>>(
          reinterpret_cast<const RT*>(a.rec), a.Tfield, static_cast<RT*>(a.cpar), a.g, a.un,
          a.bc, mech);
      k_coll<D, M, S, RT><<<blocks_for(a.g.N, kCollNodes), 32 * kCollTPN, coll_smem<D, M, RT>(),
                            s>>>(static_cast<const S*>(a.src), static_cast<S*>(a.dst),
                                 static_cast<const RT*>(a.cpar), a.g, a.bc, mech);
    } else {
      k_collide<D, M, S, RT><<<nb, bs, fused_smem<D, M, RT>(), s>>>(
          static_cast<const S*>(a.src), static_cast<S*>(a.dst),
          reinterpret_cast<const RT*>(a.rec), a.Tfield, a.status, a.g, a.un, a.bc, mech);
    }
  }
  return cudaGetLastError();
}

template <int D, int M, typename S>
static cudaError_t init_impl(const DevMech& mech, const Geom& g, const Units& un,
                             const double* rho_or_P, int is_pressure, const double* u,
                             const double* T, const double* Y, void* pops, double* Tfield,
                             int* status, cudaStream_t s) {
  k_init<D, M, S><<<blocks_for(g.N, 128), 128, 0, s>>>(rho_or_P, is_pressure, u, T, Y,
                                                        static_cast<S*>(pops), Tfield, status,
                                                        g, un, mech);
  return cudaGetLastError();
}

template <int D, int M, typename S>
static cudaError_t diag_impl(const DevMech& mech, const Geom& g, const Units& un,
                             const void* pops, const double* Tfield, const int* tag,
                             DiagPart* part, int* status, int x0, int x1, cudaStream_t s) {
  k_diag<D, M, S><<<blocks_for(g.N, 128), 128, 0, s>>>(static_cast<const S*>(pops), Tfield, tag,
                                                        part, status, g, un, mech, x0, x1);
  return cudaGetLastError();
}

template <int D, int M, typename S>
static cudaError_t out_impl(const DevMech& mech, const Geom& g, const Units& un,
                            const void* pops, const double* Tfield, double* rho, double* u,
                            double* T, double* Y, double* E, int* status, cudaStream_t s) {
  k_out<D, M, S><<<blocks_for(g.N, 128), 128, 0, s>>>(static_cast<const S*>(pops), Tfield,
                                                       rho, u, T, Y, E, status, g, un, mech);
  return cudaGetLastError();
}

// Grid of a batched kernel: one block per tile, or (persistent) at most the
// blocks the GPU holds at once, from the occupancy calculator.
template <typename K>
static int batch_grid(K kernel, int nblk, int threads, size_t smem, bool persistent) {
  if (!persistent || nblk <= 0) return nblk;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
          cudaSuccess ||
      per_sm <= 0)
    return nblk;
  return std::min(nblk, sms * per_sm);
}

template <int D, int M, typename S, typename RT>
static cudaError_t batch_impl(const DomainDev* doms, int ndom, const BatchGrids& gr,
                              const Launch& lc, int parity, cudaStream_t s,
                              const SideStream& side) {
  const int bs = kBS;
  const cudaError_t pe = prepare_once<D, M, S, RT>();
  if (pe != cudaSuccess) return pe;
  if (lc.persistent == 2) {
    // the whole step as one launch over the work-list (sync words zeroed
    // first)
    if (gr.nitems == 0) return cudaSuccess;
    auto kp = k_step_persist<D, M, S, RT>;
    const size_t sm = persist_smem<D, M, S, RT>(lc.coll_split != 0);
    cudaError_t e = cudaMemsetAsync(gr.sync, 0, (size_t)gr.nsync * sizeof(int), s);
    if (e != cudaSuccess) return e;
    kp<<<batch_grid(kp, gr.nitems, kPersistThreads, sm, true), kPersistThreads, sm, s>>>(
        doms, ndom, parity, gr.items, gr.nitems, lc.npt, gr.sync, gr.timeout_ns);
    return cudaGetLastError();
  }
  const int chem_inline = lc.chem_lanes <= 1;
  const bool ps = lc.persistent != 0;
  auto kmom = k_moments_batch<D, M, S, RT>;
  auto kbnd = k_bnode_batch<D, M, S>;
  const size_t sbnd = bnode_smem<D, M, RT>();
  // the reaction sub-steps in k_chem over a node set (the grid of the set)
  static_assert(128 / 8 == kIfChemNodesPerBlock, "interface chemistry: 8 lanes per node");
  auto chem = [&](int node_set, cudaStream_t st) {
    if (node_set == NODES_INTERFACE && gr.n_if_total >= kIfChemThreadNodes) {
      // enough interface nodes to fill the GPU with one thread each
      auto k = k_iface_chem_batch<D, M, RT>;
      const size_t sm = kFF<RT> ? chem_slice_bytes<M, ff>() : 0;
      k<<<batch_grid(k, gr.ntblocks, kBnd, sm, ps), kBnd, sm, st>>>(doms, ndom, gr.ntblocks);
      return;
    }
    const int nb = node_set == NODES_INTERFACE ? gr.nbblocks : gr.ncblocks;
    if (nb == 0) return;
    // the interface nodes are few and on the critical path: 8 lanes each
    if (lc.chem_lanes == 4 && node_set != NODES_INTERFACE) {
      auto k = k_chem_batch<D, M, RT, 4>;
      k<<<batch_grid(k, nb, 128, 0, ps), 128, 0, st>>>(doms, ndom, node_set, nb);
    } else {
      auto k = k_chem_batch<D, M, RT, 8>;
      k<<<batch_grid(k, nb, 128, 0, ps), 128, 0, st>>>(doms, ndom, node_set, nb);
    }
  };
  // chem_lanes > 1: moments and sub-steps of the nodes in one kernel with
  // chem_lanes lanes per node, on the chemistry grid
  auto mchem = [&](int node_set) {
    if (gr.ncblocks == 0) return;
    if (lc.chem_lanes == 4) {
      auto k = k_mchem_batch<D, M, S, RT, 4>;
      k<<<batch_grid(k, gr.ncblocks, 128, 0, ps), 128, 0, s>>>(doms, ndom, parity, node_set,
                                                               gr.ncblocks);
    } else {
      auto k = k_mchem_batch<D, M, S, RT, 8>;
      k<<<batch_grid(k, gr.ncblocks, 128, 0, ps), 128, 0, s>>>(doms, ndom, parity, node_set,
                                                               gr.ncblocks);
    }
  };
  if (gr.nbblocks > 0 && side.stream && side.fork && side.join) {
    // on the side stream, concurrent with the bulk moments: the boundary
    // kernel, then the interface nodes' moments (reaction sub-steps inline)
    // or, with the boundary warps writing the records, their sub-steps
    cudaError_t e = cudaEventRecord(side.fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side.stream, side.fork, 0);
    if (e != cudaSuccess) return e;
    // (the interface nodes: records by the boundary warps, sub-steps with
    // eight lanes per node, whatever the bulk placement)
    kbnd<<<batch_grid(kbnd, gr.ntblocks, kBnd, sbnd, ps), kBnd, sbnd, side.stream>>>(
        doms, ndom, parity, gr.ntblocks);
    chem(NODES_INTERFACE, side.stream);
    e = cudaEventRecord(side.join, side.stream);
    if (e != cudaSuccess) return e;
    if (chem_inline)
      kmom<<<batch_grid(kmom, gr.nblocks, bs, 0, ps), bs, 0, s>>>(doms, ndom, parity, 1,
                                                                  NODES_BULK, gr.nblocks);
    else
      mchem(NODES_BULK);
    e = cudaStreamWaitEvent(s, side.join, 0);
    if (e != cudaSuccess) return e;
  } else {
    const bool bnd_rec = gr.nbblocks > 0;
    if (gr.nbblocks > 0)
      kbnd<<<batch_grid(kbnd, gr.ntblocks, kBnd, sbnd, ps), kBnd, sbnd, s>>>(doms, ndom, parity,
                                                                          gr.ntblocks);
    if (chem_inline)
      kmom<<<batch_grid(kmom, gr.nblocks, bs, 0, ps), bs, 0, s>>>(
          doms, ndom, parity, 1, bnd_rec ? NODES_BULK : NODES_ALL, gr.nblocks);
    else
      mchem(bnd_rec ? NODES_BULK : NODES_ALL);
    if (bnd_rec) chem(NODES_INTERFACE, s);
  }
  if (lc.coll_split) {
    auto kp = k_prep_batch<D, M, RT>;
    auto kc = k_coll_batch<D, M, S, RT>;
    const size_t sp = prep_smem<D, M, RT>(), sc = coll_smem<D, M, RT>();
    kp<<<batch_grid(kp, gr.nblocks, bs, sp, ps), bs, sp, s>>>(doms, ndom, gr.nblocks);
    kc<<<batch_grid(kc, gr.nkblocks, 32 * kCollTPN, sc, ps), 32 * kCollTPN, sc, s>>>(
        doms, ndom, parity, gr.nkblocks);
  } else {
    auto kf = k_collide_batch<D, M, S, RT>;
    const size_t sf = fused_smem<D, M, RT>();
    kf<<<batch_grid(kf, gr.nblocks, bs, sf, ps), bs, sf, s>>>(doms, ndom, parity, gr.nblocks);
  }
  return cudaGetLastError();
}

// The kernel set of one (D, M, precision).
template <int D, int M, typename S, typename RT>
const KernelSet* make_kernel_set() {
  static const KernelSet ks = {&step_impl<D, M, S, RT>, &batch_impl<D, M, S, RT>,
                               &prepare_once<D, M, S, RT>, &init_impl<D, M, S>,
                               &out_impl<D, M, S>, &diag_impl<D, M, S>, Rec<D, M>::NF,
                               CPar<D, M>::NF};
  return &ks;
}

}  // inline namespace
}  // namespace lbm
