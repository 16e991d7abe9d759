// Device-side building blocks of the reactive-mixture LBM step.
//
// Lattice: D3Q27 / D2Q9 product-form velocity sets, index
// i = (cz+1)*9 + (cy+1)*3 + (cx+1) (x fastest), opposite = Q-1-i (Sec. 2.2).
// Thermodynamics, rates and transport are evaluated from the precomputed
// polynomial forms in DevMech (filled on the host from lbm_mechanism).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "exp64.cuh"
#include "lbm_internal.h"

namespace lbm {

template <int D> struct Lat;
template <> struct Lat<3> {
  static constexpr int Q = 27;
  static constexpr int NP = 6;   // xx, yy, zz, xy, xz, yz
};
template <> struct Lat<2> {
  static constexpr int Q = 9;
  static constexpr int NP = 3;   // xx, yy, xy
};

// component a (0 = x, 1 = y, 2 = z) of velocity i
__host__ __device__ constexpr int cvel(int i, int a) {
  return a == 0 ? (i % 3) - 1 : (a == 1 ? ((i / 3) % 3) - 1 : (i / 9) - 1);
}
__host__ __device__ constexpr int csq(int i, int D) {
  return cvel(i, 0) * cvel(i, 0) + cvel(i, 1) * cvel(i, 1) +
         (D == 3 ? cvel(i, 2) * cvel(i, 2) : 0);
}
// Per-axis product-form factor Psi_c(xi, P), Eqs. phi0, phiPlus, phis.
template <typename R>
__device__ __forceinline__ R psi1(int c, R xi, R P) {
  return c == 0 ? (R(1) - P) : (c == 1 ? R(0.5) * (P + xi) : R(0.5) * (P - xi));
}

// Reading R5 of Eq. momentum1: u_a := u when rho_a <= 1e-300 or when some
// |j_a| >= rho_a (impossible for non-negative populations; it arises only
// from cancellation in near-zero densities, where j_a / rho_a is noise).
template <int D, typename R>
__host__ __device__ __forceinline__ bool species_velocity_undefined(R rho_a, const R* j_a) {
  bool bad = sizeof(R) == 4 ? rho_a <= R(0)              // FP32: no value below 1e-300
                            : double(rho_a) <= RHO_TINY;
  for (int d = 0; d < D; ++d) bad |= fabs(j_a[d]) >= rho_a;
  return bad;
}

// Moment-record field offsets ([field][N] scratch in the lattice compute
// type, written by the moments kernel, read by the collision kernel).
template <int D, int M> struct Rec {
  static constexpr int RHO = 0;
  static constexpr int U = 1;
  static constexpr int P = U + D;
  static constexpr int QF = P + Lat<D>::NP;
  static constexpr int E = QF + D;
  static constexpr int Y = E + 1;
  static constexpr int US = Y + M;
  static constexpr int PHI = US + M * D;
  static constexpr int DRHO = PHI + D;          // reaction increments, species a < M
  static constexpr int NF = DRHO + M - 1;
};

// ------------------------------------------------------------------------
// thermodynamics (Sec. 3.1)
// U_a(T) = u0 + u1 T + u2 T^2 + u3 T^3 (J/kg), C_av = dU_a/dT.

template <int M>
__device__ __forceinline__ void mixture_energy_poly(const DevMech& m, const double* Y,
                                                    double c[4]) {
  c[0] = c[1] = c[2] = c[3] = 0.0;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    c[0] += Y[a] * m.u0[a];
    c[1] += Y[a] * m.u1[a];
    c[2] += Y[a] * m.u2[a];
    c[3] += Y[a] * m.u3[a];
  }
}

// Newton on sum_a Y_a U_a(T) = U (Eq. temperature); stops when the update
// satisfies |dT| <= rtol |T| after it is applied; ok = false after max_iter.
template <int M>
__device__ __forceinline__ double newton_T(const DevMech& m, const double* Y, double U,
                                           double T, int max_iter, double rtol, bool& ok) {
  double c[4];
  mixture_energy_poly<M>(m, Y, c);
  ok = false;
  for (int it = 0; it < max_iter; ++it) {
    const double F = c[0] + T * (c[1] + T * (c[2] + T * c[3])) - U;
    const double dF = c[1] + T * (2.0 * c[2] + 3.0 * T * c[3]);
    const double dT = -F / dF;
    T += dT;
    if (fabs(dT) <= rtol * fabs(T)) { ok = true; break; }
  }
  return T;
}

__device__ __forceinline__ double species_U(const DevMech& m, int a, double T) {
  return m.u0[a] + T * (m.u1[a] + T * (m.u2[a] + T * m.u3[a]));
}

// ------------------------------------------------------------------------
// chemistry: mass production rates rho_dot_a (kg/(m^3 s)) at (T, rho_a).
template <int M>
__device__ void production_rates(const DevMech& m, double T, const double* r,
                                 double* rdot) {
  const double lnT = log(T);
  const double invT = 1.0 / T;
  double C[M], G[M], w[M];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    C[a] = r[a] * m.inv_mm[a];
    G[a] = m.g_inv[a] * invT + m.g0[a] + T * (m.g1[a] + T * m.g2[a]) - m.a0[a] * lnT;
    w[a] = 0.0;
  }
  const double ln_p0_rut = m.ln_p0_over_ru - lnT;   // ln(P0 / (R_U T))
  for (int k = 0; k < m.R; ++k) {
    const DevReaction& rx = m.rx[k];
    const double lnkf = rx.lnA + rx.b * lnT - rx.EaR * invT;
    double fwd = exp_tang(lnkf);
    for (int j = 0; j < rx.nr; ++j) fwd *= C[rx.reac[j]];
    double rev = 0.0;
    if (rx.reversible) {
      double dG = 0.0;                               // sum_a nu_a G_a
      for (int j = 0; j < rx.np; ++j) dG += G[rx.prod[j]];
      for (int j = 0; j < rx.nr; ++j) dG -= G[rx.reac[j]];
      // k_r = k_f / K_c, ln K_c = -dG + dn ln(P0/(R_U T))
      rev = exp_tang(lnkf + dG - rx.dn * ln_p0_rut);
      for (int j = 0; j < rx.np; ++j) rev *= C[rx.prod[j]];
    }
    double q = fwd - rev;
    if (rx.third_body) {
      double cm = 0.0;
#pragma unroll
      for (int a = 0; a < M; ++a) cm += m.eff[k][a] * C[a];
      q *= cm;
    }
    for (int j = 0; j < rx.nr; ++j) w[rx.reac[j]] -= q;
    for (int j = 0; j < rx.np; ++j) w[rx.prod[j]] += q;
  }
#pragma unroll
  for (int a = 0; a < M; ++a) rdot[a] = w[a] * m.mm[a];
}

// ------------------------------------------------------------------------
// The same temperature solve and rates in float-float (mixed path).  The
// formulas are those of newton_T and production_rates; the stopping rule
// uses max(rtol, 4e-13), the resolution of float-float sums of the
// formation-energy-sized terms.
__device__ __forceinline__ ff species_U_ff(const DevMech& m, int a, ff T) {
  return m.u0_f[a] + T * (m.u1_f[a] + T * (m.u2_f[a] + T * m.u3_f[a]));
}

template <int M>
__device__ ff newton_T_ff(const DevMech& m, const ff* Y, ff U, ff T, int max_iter,
                          float rtol, bool& ok) {
  ff c0, c1, c2, c3;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    c0 += Y[a] * m.u0_f[a];
    c1 += Y[a] * m.u1_f[a];
    c2 += Y[a] * m.u2_f[a];
    c3 += Y[a] * m.u3_f[a];
  }
  const ff two(2.f), three(3.f);
  ok = false;
  for (int it = 0; it < max_iter; ++it) {
    const ff F = c0 + T * (c1 + T * (c2 + T * c3)) - U;
    const ff dF = c1 + T * (two * c2 + three * T * c3);
    const ff dT = -(F / dF);
    T += dT;
    if (fabsf(dT.hi) <= rtol * fabsf(T.hi)) { ok = true; break; }
  }
  return T;
}

// The arrays the reaction loop indexes by species (concentrations, Gibbs
// functions, rates) live in a per-thread slice of shared memory: a runtime
// index into a register array would put it in local memory.  Every kernel
// that runs the float-float rates has kChemThreads threads per block.
constexpr int kChemThreads = 128;

// bytes of one block's slices (kChemThreads threads, C, G and W per species)
template <int M, typename CT> constexpr size_t chem_slice_bytes() {
  return (size_t)3 * M * kChemThreads * sizeof(CT);
}

// Cs: this thread's slice (entry a of C at Cs[a kChemThreads], then G and W)
template <int M>
__device__ void production_rates_ff(const DevMech& m, ff T, const ff* r, ff* rdot,
                                    ff* const Cs) {
  ff* const Gs = Cs + M * kChemThreads;
  ff* const Ws = Gs + M * kChemThreads;
  const ff lnT = ff_log(T);
  const ff invT = ff(1.f) / T;
  ff C[M];
#pragma unroll
  for (int a = 0; a < M; ++a) {
    C[a] = r[a] * m.inv_mm_f[a];
    Cs[a * kChemThreads] = C[a];
    Gs[a * kChemThreads] =
        m.g_inv_f[a] * invT + m.g0_f[a] + T * (m.g1_f[a] + T * m.g2_f[a]) - m.a0_f[a] * lnT;
    Ws[a * kChemThreads] = ff();
  }
  const ff ln_p0_rut = m.ln_p0_over_ru_f - lnT;
  for (int k = 0; k < m.R; ++k) {
    const DevReaction& rx = m.rx[k];
    const ff lnkf = rx.lnA_f + rx.b_f * lnT - rx.EaR_f * invT;
    ff fwd = ff_exp(lnkf);
    for (int j = 0; j < rx.nr; ++j) fwd *= Cs[rx.reac[j] * kChemThreads];
    ff rev;
    if (rx.reversible) {
      ff dG;
      for (int j = 0; j < rx.np; ++j) dG += Gs[rx.prod[j] * kChemThreads];
      for (int j = 0; j < rx.nr; ++j) dG -= Gs[rx.reac[j] * kChemThreads];
      rev = ff_exp(lnkf + dG - ff((float)rx.dn) * ln_p0_rut);
      for (int j = 0; j < rx.np; ++j) rev *= Cs[rx.prod[j] * kChemThreads];
    }
    ff q = fwd - rev;
    if (rx.third_body) {
      ff cm;
#pragma unroll
      for (int a = 0; a < M; ++a) cm += m.eff_f[k][a] * C[a];
      q *= cm;
    }
    for (int j = 0; j < rx.nr; ++j) Ws[rx.reac[j] * kChemThreads] -= q;
    for (int j = 0; j < rx.np; ++j) Ws[rx.prod[j] * kChemThreads] += q;
  }
#pragma unroll
  for (int a = 0; a < M; ++a) rdot[a] = Ws[a * kChemThreads] * m.mm_f[a];
}

// ------------------------------------------------------------------------
// Gaussian elimination without pivoting for A V = B with 3 right-hand sides,
// the matrix stored with entry (r, c) at A[(r M + c) st].
// A is strictly row diagonally dominant (diagonal 1 + sum of |off-diagonal|),
// so every pivot is at least 1.
template <int M, int D, typename R>
__device__ __forceinline__ void solve_dd_strided(R* A, int st, R (&B)[M][D]) {
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const R inv = R(1) / A[(k * M + k) * st];
#pragma unroll
    for (int r = k + 1; r < M; ++r) {
      const R f = A[(r * M + k) * st] * inv;
#pragma unroll
      for (int c = k + 1; c < M; ++c) A[(r * M + c) * st] -= f * A[(k * M + c) * st];
#pragma unroll
      for (int d = 0; d < D; ++d) B[r][d] -= f * B[k][d];
    }
  }
#pragma unroll
  for (int k = M - 1; k >= 0; --k) {
    const R inv = R(1) / A[(k * M + k) * st];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      R s = B[k][d];
#pragma unroll
      for (int c = k + 1; c < M; ++c) s -= A[(k * M + c) * st] * B[c][d];
      B[k][d] = s * inv;
    }
  }
}

}  // namespace lbm
