// Boundary reconstruction with one thread per interface node (Sec. 4):
// bounce-back (Eq. bb), Tamm-Mott-Smith wall (Sec. 4.2.2, Eqs. BBrho-fatms),
// flux inlet (Sec. 4.3, Eqs. in_f-fa_inlet, and the simplified inlet of the
// same section) and LODI outlet (Sec. 4.4, Eqs. convectiveBC-fa_outlet),
// followed by the node's moment record.  Included by lbm_kernels.cuh inside
// its namespace.
//
// Why a thread per node.  A node's procedure is a chain of scalar steps
// (moment sums over the 270 populations, up to four temperature Newton
// solves, equilibrium parameters) around three passes over its populations.
// Spread over a warp (lane = direction), every scalar step and every
// cross-lane reduction is a full-warp instruction: on GB300, whose FP64
// pipes run two lanes per clock per SM, that made the FP64 boundary kernel
// execute ~63k FP64 FLOP per interface node.  With a thread per node the
// sums are sequential adds and the scalar steps run once per node.  The
// passes run lattice by lattice (compile-time l) and, inside, direction by
// direction: the direction index is the same for every thread of a warp,
// so the branches on c_i are uniform, and each equilibrium population is a
// product of three entries of per-lattice axis-factor tables (Eq. prod)
// built once per lattice and state.  Threads are consecutive interface
// nodes (the list is in node order), so the pull loads of a wall row
// coalesce.
//
// Per-thread arrays (species mass fractions, the TMS local species
// velocities, the pull-source node of every direction) live in this
// thread's shared-memory column, stride kBnd.

constexpr int kBnd = kBndNodesPerBlock;   // threads per block of the boundary kernel

// shared memory per thread: target Y, local Y, a spare Y, the local u_a and
// the target u_a (off-grid TMS targets) (R entries), then the Q pull sources
// (long long)
template <int D, int M> constexpr int bnode_col_entries() { return 3 * M + 2 * M * D; }
template <int D, int M, typename R> constexpr size_t bnode_smem() {
  return (sizeof(R) * bnode_col_entries<D, M>() + sizeof(long long) * Lat<D>::Q) * kBnd;
}

// An equilibrium state of the boundary procedures (Eqs. faEqGeneral,
// fEqGeneral, gEqGeneral): rho, T, theta, U/c^2, u in registers; Y and the
// species velocities in shared memory.
template <int D, int M, typename R> struct BState {
  R rho, T, th, U;
  R u[D];
  R* Y;           // [M], stride kBnd
  R* us;          // [M D] species velocities, stride kBnd (nullptr: u for every species)
  double T_full;  // T to the solve's precision
};

// theta, U/c^2 of a state from its T and Y (the mixture energy as a sum over
// species, float-float in the mixed path)
template <int D, int M, typename R>
__device__ __forceinline__ void bstate_prepare(BState<D, M, R>& s, const DevMech& m,
                                               const Units& un) {
  if constexpr (!kFF<R>) {
    double Rm = 0.0, U = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) {
      const double Ya = double(s.Y[a * kBnd]);
      Rm += Ya * m.inv_mm[a];
      U += Ya * species_U(m, a, double(s.T));
    }
    s.th = R(R_U * Rm * double(s.T) * un.inv_c2);
    s.U = R(U * un.inv_c2);
  } else {
    float Rm = 0.f;
    const ff T(s.T);
    ff U;
#pragma unroll
    for (int a = 0; a < M; ++a) {
      Rm += s.Y[a * kBnd] * m.inv_mm_s[a];
      U += ff(s.Y[a * kBnd]) * species_U_ff(m, a, T);
    }
    s.th = float(R_U) * Rm * s.T * un.inv_c2_s;
    s.U = (U * un.inv_c2_f).hi;
  }
}

// Population sums of a node (every lattice): rho, j, the momentum flux
// tensor P of the f lattice, rho E and q of the g lattice, rho_a and j_a of
// the stored species.
template <int D, int M, typename R> struct BSums {
  R rho, rhoE, j[D], q[D], P[Lat<D>::NP], rs[M], js[M][D];
};

// The macroscopic state of population sums (Eqs. density1, momentum1,
// fdensity, f1momMomentum, g0momTotalEnergy, slaving Eq. strongest): rho,
// u, Y, u_a (reading R5) and T by Newton on Eq. temperature from T_guess,
// then theta and U/c^2 as bstate_prepare.
template <int D, int M, typename R>
__device__ __forceinline__ void bstate_of(BState<D, M, R>& s, const BSums<D, M, R>& z,
                                          double T_guess, const DevMech& m, const Units& un,
                                          int* status) {
  s.rho = z.rho;
  const R irho = R(1) / z.rho;
  R usq = R(0);
#pragma unroll
  for (int d = 0; d < D; ++d) { s.u[d] = z.j[d] * irho; usq += s.u[d] * s.u[d]; }
  R rM = z.rho, jM[D];
#pragma unroll
  for (int d = 0; d < D; ++d) jM[d] = z.j[d];
#pragma unroll
  for (int a = 0; a < M - 1; ++a) {
    rM -= z.rs[a];
#pragma unroll
    for (int d = 0; d < D; ++d) jM[d] -= z.js[a][d];
  }
#pragma unroll
  for (int a = 0; a < M; ++a) {
    const R ra = a < M - 1 ? z.rs[a] : rM;
    s.Y[a * kBnd] = ra * irho;
    if (s.us) {
      R ja[D];
#pragma unroll
      for (int d = 0; d < D; ++d) ja[d] = a < M - 1 ? z.js[a][d] : jM[d];
      const bool tiny = species_velocity_undefined<D, R>(ra, ja);
      if constexpr (sizeof(R) == 8) {
        // rho_a > 1e-300 when not tiny: 1/rho_a is finite
        const R ira = tiny ? R(0) : R(1) / ra;
#pragma unroll
        for (int d = 0; d < D; ++d) s.us[(a * D + d) * kBnd] = tiny ? s.u[d] : ja[d] * ira;
      } else {
        // FP32: a positive rho_a below ~3e-39 has no finite reciprocal
#pragma unroll
        for (int d = 0; d < D; ++d) s.us[(a * D + d) * kBnd] = tiny ? s.u[d] : ja[d] / ra;
      }
    }
  }
  bool ok;
  if constexpr (!kFF<R>) {
    double Y[M];
#pragma unroll
    for (int a = 0; a < M; ++a) Y[a] = double(s.Y[a * kBnd]);
    const double U = (double(z.rhoE * irho) - 0.5 * double(usq)) * un.c * un.c;
    const double T = newton_T<M>(m, Y, U, T_guess, un.newton_max_iter, un.newton_rtol, ok);
    s.T = R(T);
    s.T_full = T;
  } else {
    ff Yf[M];
#pragma unroll
    for (int a = 0; a < M; ++a) Yf[a] = ff(s.Y[a * kBnd]);
    const ff U = (ff(z.rhoE * irho) + ff(-0.5f * usq)) * un.c2_f;
    const ff T = newton_T_ff<M>(m, Yf, U, ff_from_double(T_guess), un.newton_max_iter,
                                un.newton_rtol_f, ok);
    s.T = T.hi;
    s.T_full = ff_to_double(T);
  }
  if (!ok) atomicOr(status, ST_NEWTON);
  bstate_prepare<D, M, R>(s, m, un);
}

// Per-lattice axis-factor tables of a state (Eqs. phi0, phiPlus, phis,
// prod): entry k of an axis is the factor for c = k - 1.  PTab: a species
// or the f lattice, population = pref * prod_d t[d][c_d + 1].  GTab: the g
// lattice by the closed form of Eq. geq_i, A = Psi_c(u_d, theta + u_d^2),
// B = Psi_c applied to u_d^2 / 2.
template <int D, typename R> struct PTab { R pref, t[D][3]; };
template <int D, typename R> struct GTab { R rho, U, A[D][3], B[D][3]; };

template <typename R> __device__ __forceinline__ R sel3(int c, const R (&t)[3]) {
  return c < 0 ? t[0] : (c == 0 ? t[1] : t[2]);
}

template <int D, int M, int l, typename R>
__device__ __forceinline__ void ptab(const BState<D, M, R>& s, PTab<D, R>& e, const DevMech& m,
                                     const Units& un) {
  R th;
  if constexpr (l < M - 1) {
    if constexpr (sizeof(R) == 8) th = R(m.Ra[l] * double(s.T) * un.inv_c2);
    else th = m.Ra_s[l] * s.T * un.inv_c2_s;
    e.pref = s.rho * s.Y[l * kBnd];
  } else {
    th = s.th;
    e.pref = s.rho;
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const R xi = (l < M - 1 && s.us) ? s.us[(l * D + d) * kBnd] : s.u[d];
    const R P = th + xi * xi;
    e.t[d][0] = R(0.5) * (P - xi);
    e.t[d][1] = R(1) - P;
    e.t[d][2] = R(0.5) * (P + xi);
  }
}

template <int D, int M, typename R>
__device__ __forceinline__ void gtab(const BState<D, M, R>& s, GTab<D, R>& g) {
  g.rho = s.rho;
  g.U = s.U;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const R ua = s.u[d];
    const R O1 = s.th * ua + R(0.5) * ua * ua * ua;
    const R O2 = s.th * s.th + R(2.5) * s.th * ua * ua + R(0.5) * ua * ua * ua * ua;
    const R P = s.th + ua * ua;
    g.A[d][0] = R(0.5) * (P - ua);
    g.A[d][1] = R(1) - P;
    g.A[d][2] = R(0.5) * (P + ua);
    g.B[d][0] = R(0.5) * (O2 - O1);
    g.B[d][1] = R(0.5) * ua * ua - O2;
    g.B[d][2] = R(0.5) * (O2 + O1);
  }
}

// Tables of one state for the lattice of the current pass.  row<l>(c_y,
// c_z) forms the part shared by a row of three directions (the population's
// pref t_y t_z; for g, A_y A_z and U A_y A_z + B_y A_z + A_y B_z, since
// g^eq = rho [A_x (U A_y A_z + B_y A_z + A_y B_z) + B_x A_y A_z]); evalx<l>(c_x)
// then finishes a direction of that row.
template <int D, int M, typename R> struct ETab {
  PTab<D, R> p;
  GTab<D, R> g;
  R rp, rP, rQ;
  template <int l>
  __device__ __forceinline__ void build(const BState<D, M, R>& s, const DevMech& m,
                                        const Units& un) {
    if constexpr (l == M) gtab<D, M, R>(s, g);
    else ptab<D, M, l, R>(s, p, m, un);
  }
  template <int l> __device__ __forceinline__ void row(int cy, int cz) {
    if constexpr (l == M) {
      const R ay = sel3(cy, g.A[1]), by = sel3(cy, g.B[1]);
      if constexpr (D == 3) {
        const R az = sel3(cz, g.A[2]), bz = sel3(cz, g.B[2]);
        rP = ay * az;
        rQ = g.U * rP + by * az + ay * bz;
      } else {
        rP = ay;
        rQ = g.U * ay + by;
      }
    } else {
      rp = p.pref * sel3(cy, p.t[1]);
      if constexpr (D == 3) rp *= sel3(cz, p.t[2]);
    }
  }
  template <int l> __device__ __forceinline__ R evalx(int cx) const {
    if constexpr (l == M) return g.rho * (sel3(cx, g.A[0]) * rQ + sel3(cx, g.B[0]) * rP);
    else return rp * sel3(cx, p.t[0]);
  }
};

// Compile-time loop l = B .. E-1: f(std::integral_constant<int, l>{}).
template <int B, int E> struct ForL {
  template <typename Fn> __device__ __forceinline__ static void run(Fn&& f) {
    f(std::integral_constant<int, B>{});
    ForL<B + 1, E>::run(f);
  }
};
template <int E> struct ForL<E, E> {
  template <typename Fn> __device__ __forceinline__ static void run(Fn&&) {}
};

// Population sums of a pass, lattice by lattice: fn.template setup<l>()
// once per lattice, then, row by row, fn.template row<l>(c_y, c_z) and
// fn.template get<l>(i, c) for the row's three directions.
// Directions in rows of three (c_x = -1, 0, 1 at compile time, a row's loads
// in flight together); a row enters through its sum s and difference
// d = f_+ - f_- (and f_+ + f_- for P_xx).  kDensOnly: the densities rho_a,
// rho and rho E only (the bounce-back pass of a wall).
template <int D, int M, typename R, bool kDensOnly = false, typename F>
__device__ __forceinline__ void bsums(F& fn, BSums<D, M, R>& z) {
  constexpr int Q = Lat<D>::Q, NP = Lat<D>::NP;
  ForL<0, M + 1>::run([&](auto lc) {
    constexpr int l = decltype(lc)::value;
    fn.template setup<l>();
    R sum = R(0), sj[D], sP[NP];
#pragma unroll
    for (int d = 0; d < D; ++d) sj[d] = R(0);
#pragma unroll
    for (int p = 0; p < NP; ++p) sP[p] = R(0);
#pragma unroll 1
    for (int yz = 0; yz < Q / 3; ++yz) {
      const int cy = yz % 3 - 1, cz = D == 3 ? yz / 3 - 1 : 0;
      fn.template row<l>(cy, cz);
      R v[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int c[3] = {k - 1, cy, cz};
        v[k] = fn.template get<l>(3 * yz + k, c);
      }
      const R sx = v[0] + v[2], sr = sx + v[1];
      sum += sr;
      if constexpr (!kDensOnly) {
        const R dx = v[2] - v[0];
        sj[0] += dx;
        if (cy != 0) sj[1] += cy > 0 ? sr : -sr;
        if constexpr (D == 3)
          if (cz != 0) sj[2] += cz > 0 ? sr : -sr;
        if constexpr (l == M - 1) {
          sP[pidx<D>(0, 0)] += sx;
          if (cy != 0) {
            sP[pidx<D>(1, 1)] += sr;
            sP[pidx<D>(0, 1)] += cy > 0 ? dx : -dx;
          }
          if constexpr (D == 3) {
            if (cz != 0) {
              sP[pidx<D>(2, 2)] += sr;
              sP[pidx<D>(0, 2)] += cz > 0 ? dx : -dx;
              if (cy != 0) sP[pidx<D>(1, 2)] += cy == cz ? sr : -sr;
            }
          }
        }
      }
    }
    if constexpr (l < M - 1) {
      z.rs[l] = sum;
#pragma unroll
      for (int d = 0; d < D; ++d) z.js[l][d] = sj[d];
    } else if constexpr (l == M - 1) {
      z.rho = sum;
#pragma unroll
      for (int d = 0; d < D; ++d) z.j[d] = sj[d];
#pragma unroll
      for (int p = 0; p < NP; ++p) z.P[p] = sP[p];
    } else {
      z.rhoE = sum;
#pragma unroll
      for (int d = 0; d < D; ++d) z.q[d] = sj[d];
    }
  });
}

// Value functors of bsums.  BPull: the pulled population (source node from
// this thread's column) or, with bbk and an incoming link, the node's own
// opposite post-collision population (Eq. bb).
template <int D, int M, typename S, typename R> struct BPull {
  static constexpr int Q = Lat<D>::Q;
  const S* src;
  const float4* codec;
  long long N, n;
  const long long* sn;      // pull source of direction i at sn[i kBnd]
  unsigned inc;
  bool bbk;
  __device__ __forceinline__ bool incoming(int i) const { return inc >> i & 1u; }
  template <int l> __device__ __forceinline__ void setup() {}
  template <int l> __device__ __forceinline__ void row(int, int) {}
  template <int l> __device__ __forceinline__ R pull(int i) const {
    const bool bb = bbk && incoming(i);
    const long long mm = bb ? n : sn[i * kBnd];
    const int ii = bb ? Q - 1 - i : i;
    return Codec<S>::template dec<R>(__ldg(src + (long long)(l * Q + ii) * N + mm), codec,
                                     l * Q + ii);
  }
  template <int l> __device__ __forceinline__ R get(int i, const int (&)[3]) const {
    return pull<l>(i);
  }
};

// BPull whose values are also stored as the node's reconstructed populations.
template <int D, int M, typename S, typename R> struct BStorePull {
  static constexpr int Q = Lat<D>::Q;
  BPull<D, M, S, R> p;
  double* P;
  long long st;
  template <int l> __device__ __forceinline__ void setup() {}
  template <int l> __device__ __forceinline__ void row(int, int) {}
  template <int l> __device__ __forceinline__ R get(int i, const int (&)[3]) const {
    const R v = p.template pull<l>(i);
    P[(long long)(l * Q + i) * st] = double(v);
    return v;
  }
};

// The stored populations of one node.
template <int D, int M, typename S, typename R> struct BNode {
  static constexpr int Q = Lat<D>::Q;
  const S* src;
  const float4* codec;
  long long N, node;
  template <int l> __device__ __forceinline__ void setup() {}
  template <int l> __device__ __forceinline__ void row(int, int) {}
  template <int l> __device__ __forceinline__ R get(int i, const int (&)[3]) const {
    return Codec<S>::template dec<R>(__ldg(src + (long long)(l * Q + i) * N + node), codec,
                                     l * Q + i);
  }
};

// The local populations: incoming links at the state A, the others pulled.
template <int D, int M, typename S, typename R> struct BLocal {
  BPull<D, M, S, R> p;
  const BState<D, M, R>* A;
  const DevMech* m;
  const Units* un;
  ETab<D, M, R> ta;
  template <int l> __device__ __forceinline__ void setup() {
    ta.template build<l>(*A, *m, *un);
  }
  template <int l> __device__ __forceinline__ void row(int cy, int cz) {
    ta.template row<l>(cy, cz);
  }
  template <int l> __device__ __forceinline__ R get(int i, const int (&c)[3]) const {
    return p.incoming(i) ? ta.template evalx<l>(c[0]) : p.template pull<l>(i);
  }
};

// Step 4: the target Bt + the local populations - the local equilibria L;
// the simplified inlet takes the local equilibria.  Stored as the node's
// reconstructed populations.
template <int D, int M, typename S, typename R> struct BFinal {
  static constexpr int Q = Lat<D>::Q;
  BLocal<D, M, S, R> lo;
  const BState<D, M, R>* Bt;
  const BState<D, M, R>* L;
  bool simple, same;        // same: Bt is the state A of the incoming links
  double* P;
  long long st;
  ETab<D, M, R> tb, tl;
  template <int l> __device__ __forceinline__ void setup() {
    lo.template setup<l>();
    if (!same) tb.template build<l>(*Bt, *lo.m, *lo.un);
    tl.template build<l>(*L, *lo.m, *lo.un);
  }
  template <int l> __device__ __forceinline__ void row(int cy, int cz) {
    lo.template row<l>(cy, cz);
    if (!same) tb.template row<l>(cy, cz);
    tl.template row<l>(cy, cz);
  }
  template <int l> __device__ __forceinline__ R get(int i, const int (&c)[3]) const {
    const R loc = tl.template evalx<l>(c[0]);
    R v;
    if (simple) {
      v = loc;
    } else if (lo.p.incoming(i)) {
      const R a = lo.ta.template evalx<l>(c[0]);
      v = (same ? a : tb.template evalx<l>(c[0])) + a - loc;
    } else {
      v = (same ? lo.ta.template evalx<l>(c[0]) : tb.template evalx<l>(c[0])) +
          lo.p.template pull<l>(i) - loc;
    }
    P[(long long)(l * Q + i) * st] = double(v);
    return v;
  }
};

// The boundary procedure of interface node k and its moment record.
// col: this thread's shared-memory column of R entries, sncol: its column of
// pull sources (both stride kBnd).
template <int D, int M, typename S, typename R>
__device__ __forceinline__ void bnode_body(const S* __restrict__ src, const BCDev& bc,
                                           R* __restrict__ rec, double* __restrict__ Tf,
                                           int* __restrict__ status, const Geom& g,
                                           const Units& un, const DevMech& m, int k,
                                           R* col, long long* sncol) {
  constexpr int Q = Lat<D>::Q, NP = Lat<D>::NP;
  using RC = Rec<D, M>;
  using Pull = BPull<D, M, S, R>;
  const long long N = g.N;
  const long long n = bc.if_node[k];
  const int info = bc.if_info[k];
  const int kind = info & 15;
  const unsigned inc = bc.if_inc[k];
  {
    const int x = (int)(n % g.nx);
    const int y = (int)((n / g.nx) % g.ny);
    const int z = (int)(n / ((long long)g.nx * g.ny));
#pragma unroll 1
    for (int i = 0; i < Q; ++i) sncol[i * kBnd] = node_shift<D>(x, y, z, i, -1, g);
  }
  const long long st = bc.n_if;
  const float4* codec = g.codec;
  BState<D, M, R> A, B, L;
  A.Y = col;
  L.Y = col + M * kBnd;
  B.Y = col + 2 * M * kBnd;                // spare column (outlet upstream state)
  L.us = col + 3 * M * kBnd;
  A.us = B.us = nullptr;
  BSums<D, M, R> z;

  if (kind == BK_BB) {
    // Eq. bb: incoming links take the node's own opposite post-collision
    // populations
    BStorePull<D, M, S, R> out{Pull{src, codec, N, n, sncol, inc, true}, bc.pops + k, st};
    bsums<D, M, R>(out, z);
  } else {
    if (kind == BK_TMS) {
      // step 1, Eqs. BBrho and BBY: bounce-back density and mass fractions
      Pull pull{src, codec, N, n, sncol, inc, true};
      bsums<D, M, R, true>(pull, z);
      A.rho = z.rho;
      const R irho = R(1) / z.rho;
      R ysum = R(0);
#pragma unroll
      for (int a = 0; a < M - 1; ++a) {
        const R Ya = z.rs[a] * irho;
        A.Y[a * kBnd] = Ya;
        ysum += Ya;
      }
      A.Y[(M - 1) * kBnd] = R(1) - ysum;
#pragma unroll
      for (int d = 0; d < D; ++d) A.u[d] = R(0);     // u^tgt = u_a^tgt = 0
      A.T = R(bc.if_wallT[k]);
      if (bc.if_nbr && bc.if_nbr[k] >= 0) {
        // off-grid targets (last paragraph of Sec. 4.2.2; reading R20): the
        // stored state of the fluid node x_f (Newton from this node's own T
        // guess, as for the outlet), interpolated along the wall normal
        // between the wall (at -delta) and x_f (at h)
        BState<D, M, R> sf = B;            // the spare and local-u_a columns, free now
        sf.us = L.us;
        BNode<D, M, S, R> nf{src, codec, N, (long long)bc.if_nbr[k]};
        bsums<D, M, R>(nf, z);
        bstate_of<D, M, R>(sf, z, __ldcg(Tf + n), m, un, status);
        const double h = bc.if_wh[k], dl = bc.if_wd[k];
        const R w = R(dl / (h + dl));
#pragma unroll
        for (int d = 0; d < D; ++d) A.u[d] = w * sf.u[d];
        A.us = col + (3 * M + M * D) * kBnd;
#pragma unroll
        for (int e = 0; e < M * D; ++e) A.us[e * kBnd] = w * sf.us[e * kBnd];
        A.T = R((h * bc.if_wallT[k] + dl * sf.T_full) / (h + dl));
      }
      bstate_prepare<D, M, R>(A, m, un);              // step 2: target (Eqs. tgtf-tgtfa)
    } else if (kind == BK_INLET) {
      A.rho = R(bc.rho_in);
#pragma unroll
      for (int a = 0; a < M; ++a) A.Y[a * kBnd] = R(bc.Y_in[a]);
#pragma unroll
      for (int d = 0; d < D; ++d) A.u[d] = R(bc.if_uin[(long long)d * st + k]);
      A.T = R(bc.T_in);
      bstate_prepare<D, M, R>(A, m, un);              // step 1 (Eqs. in_f-in_fa)
    } else {
      // LODI data from the stored state at x and x - n (Eq. convectiveBC,
      // reading R13); the upstream node's Newton starts from this node's T
      // guess (the bulk moments kernel may be rewriting the upstream one)
      const int ax = (info >> 4) & 3;
      const int sg = (info >> 6) & 1 ? 1 : -1;
      const long long stride =
          ax == 0 ? 1 : (ax == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
      const long long up = n - sg * stride;
      BState<D, M, R> s0 = L, s1 = B;      // the local and spare columns, free until later
      s0.us = s1.us = nullptr;
      BNode<D, M, S, R> n0{src, codec, N, n};
      bsums<D, M, R>(n0, z);
      bstate_of<D, M, R>(s0, z, __ldcg(Tf + n), m, un, status);
      BNode<D, M, S, R> n1{src, codec, N, up};
      bsums<D, M, R>(n1, z);
      bstate_of<D, M, R>(s1, z, __ldcg(Tf + n), m, un, status);
      double R0 = 0.0, R1 = 0.0, Cv = 0.0;
      const double T0 = s0.T, T1 = s1.T;
#pragma unroll
      for (int a = 0; a < M; ++a) {
        const double Y0 = double(s0.Y[a * kBnd]), Y1 = double(s1.Y[a * kBnd]);
        R0 += Y0 * m.inv_mm[a];
        R1 += Y1 * m.inv_mm[a];
        Cv += Y0 * (m.u1[a] + T0 * (2.0 * m.u2[a] + 3.0 * T0 * m.u3[a]));
      }
      R0 *= R_U;
      R1 *= R_U;
      const double r0 = s0.rho, r1 = s1.rho;
      const double p0 = r0 * R0 * T0 * un.inv_c2;
      const double p1 = r1 * R1 * T1 * un.inv_c2;
      const double un0 = sg * double(s0.u[ax]), un1 = sg * double(s1.u[ax]);
      const double gamma = (Cv + R0) / Cv;
      const double cs = sqrt(gamma * R0 * T0 * un.inv_c2);
      const double Ma = un0 / cs;
      const double Ln = bc.outlet_L > 0.0 ? bc.outlet_L : (ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz));
      const double K = bc.sigma * (1.0 - Ma * Ma) * cs / Ln;
      const double L1 = K * (p0 - bc.p_out_lat);
      const double L2 = un0 * (cs * cs * (r0 - r1) - (p0 - p1));
      const double L5 = (un0 + cs) * ((p0 - p1) + r0 * cs * (un0 - un1));
      const double rho_o = r0 - (L2 + 0.5 * (L5 + L1)) / (cs * cs);
      const double p_o = p0 - 0.5 * (L5 + L1);
      const double un_o = un0 - (L5 - L1) / (2.0 * r0 * cs);
      A.rho = R(rho_o);
#pragma unroll
      for (int d = 0; d < D; ++d)
        A.u[d] = R(double(s0.u[d]) - un0 * double(s0.u[d] - s1.u[d]));
      A.u[ax] = R(sg * un_o);
      double Ro = 0.0;
#pragma unroll
      for (int a = 0; a < M; ++a) {
        const double Y0 = double(s0.Y[a * kBnd]);
        const double Ya = Y0 - un0 * (Y0 - double(s1.Y[a * kBnd]));
        A.Y[a * kBnd] = R(Ya);
        Ro += Ya * m.inv_mm[a];
      }
      A.T = R(p_o * un.c * un.c / (rho_o * R_U * Ro));
      bstate_prepare<D, M, R>(A, m, un);              // step 1 (Eqs. out_f-out_fa)
    }
    // the local state: incoming links at A, the others pulled (Eqs.
    // locRho-locT and their inlet / outlet analogues)
    BLocal<D, M, S, R> local{Pull{src, codec, N, n, sncol, inc, false}, &A, &m, &un, {}};
    bsums<D, M, R>(local, z);
    if (kind != BK_TMS) L.us = nullptr;               // TMS local species use u_a^loc
    bstate_of<D, M, R>(L, z, __ldcg(Tf + n), m, un, status);
    if (kind == BK_INLET) {                           // target (Eqs. in_tgt_*)
      B.rho = L.rho;
      B.Y = L.Y;
#pragma unroll
      for (int d = 0; d < D; ++d) B.u[d] = A.u[d];
      B.T = R(bc.T_in);
      bstate_prepare<D, M, R>(B, m, un);
    }
    // step 4 (Eqs. ftms-fatms, f_inlet-fa_inlet, f_outlet-fa_outlet)
    BFinal<D, M, S, R> fin{local, &B, &L, kind == BK_INLET && bc.inlet_simplified != 0,
                           kind != BK_INLET, bc.pops + k, st, {}, {}};
    bsums<D, M, R>(fin, z);
  }

  // the record from the reconstructed populations (the fields the moments
  // kernel records: state with Newton from the node's previous T, energy
  // flux, momentum flux tensor); the reaction sub-steps follow in their own kernel
  BState<D, M, R> s;
  s.Y = A.Y;                                    // the target columns are free now
  s.us = col + 3 * M * kBnd;
  bstate_of<D, M, R>(s, z, __ldcg(Tf + n), m, un, status);
  if (!(s.rho > R(0)) || !isfinite(double(s.rho)) || !isfinite(s.T_full))
    atomicOr(status, ST_NONFINITE);
  Tf[n] = s.T_full;
  R thR;
  if constexpr (sizeof(R) == 4) {
    float Rm = 0.f;
#pragma unroll
    for (int a = 0; a < M; ++a) Rm += s.Y[a * kBnd] * m.inv_mm_s[a];
    thR = Rm * float(R_U) * s.T * un.inv_c2_s;
  } else {
    double Rmix = 0.0;
#pragma unroll
    for (int a = 0; a < M; ++a) Rmix += s.Y[a * kBnd] * m.inv_mm[a];
    thR = R(Rmix * R_U * s.T * un.inv_c2);
  }
  const R rr = s.rho;
#pragma unroll
  for (int a = 0; a < M - 1; ++a) rec[(RC::DRHO + a) * N + n] = s.Y[a * kBnd] * rr;
  rec[RC::RHO * N + n] = rr;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    rec[(RC::U + d) * N + n] = s.u[d];
    rec[(RC::QF + d) * N + n] = z.q[d];
    rec[(RC::PHI + d) * N + n] =
        rr * s.u[d] * (R(1) - R(3) * thR) - rr * s.u[d] * s.u[d] * s.u[d];
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) rec[(RC::P + p) * N + n] = z.P[p];
  rec[RC::E * N + n] = z.rhoE * (R(1) / rr);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    rec[(RC::Y + a) * N + n] = s.Y[a * kBnd];
#pragma unroll
    for (int d = 0; d < D; ++d) rec[(RC::US + a * D + d) * N + n] = s.us[(a * D + d) * kBnd];
  }
}
