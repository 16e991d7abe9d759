// Boundary reconstruction with one thread per interface node (Sec. 4):
// bounce-back (Eq. bb), Tamm-Mott-Smith wall (Sec. 4.2.2, Eqs. BBrho-fatms),
// flux inlet (Sec. 4.3, Eqs. in_f-fa_inlet, and the simplified inlet of the
// same section) and LODI outlet (Sec. 4.4, Eqs. convectiveBC-fa_outlet),
// followed by the node's moment record.  Included by lbm_kernels.cuh inside
// its namespace.
//
// Why a thread per node.  A node's procedure is a chain of scalar steps
// (moment sums over 27 directions x 10 lattices, up to four temperature
// Newton solves, equilibrium parameters) around three passes over its 270
// populations.  Spread over a warp (lane = direction), every scalar step and
// every cross-lane reduction is a full-warp instruction: on GB300, whose
// FP64 pipes run two lanes per clock per SM, that made the FP64 boundary
// kernel execute ~63k FP64 FLOP per interface node.  With a thread per node
// the sums are sequential adds and the scalar steps run once per node; the
// direction loop index is the same for every thread of a warp, so its
// branches on c_i are uniform.  Threads are consecutive interface nodes
// (the list is in node order), so the pull loads of a wall row coalesce.
//
// Per-thread arrays (species mass fractions and the TMS local species
// velocities) live in this thread's shared-memory column, stride kBnd.

constexpr int kBnd = kBndNodesPerBlock;   // threads per block of the boundary kernel

// shared-memory entries per thread: target Y, local Y, local u_a, a spare Y
template <int D, int M> constexpr int bnode_smem_entries() { return 3 * M + M * D; }
template <int D, int M, typename R> constexpr size_t bnode_smem() {
  return sizeof(R) * kBnd * bnode_smem_entries<D, M>();
}

// An equilibrium state of the boundary procedures (Eqs. faEqGeneral,
// fEqGeneral, gEqGeneral): rho, T, theta, U/c^2, u in registers; Y and the
// species velocities in shared memory.
template <int D, int M, typename R> struct BState {
  R rho, T, th, U;
  R u[D];
  R* Y;          // [M], stride kBnd
  R* us;         // [M D] species velocities, stride kBnd (nullptr: u for every species)
  double T_full;  // T to the solve's precision
};

// theta, U/c^2 of a state from its T and Y (the formulas of eq_prepare_warp:
// the mixture energy as a sum over species, float-float in the mixed path)
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

// The macroscopic state of population sums (Eqs. density1, momentum1,
// fdensity, f1momMomentum, g0momTotalEnergy, slaving Eq. strongest): rho,
// u, Y, u_a (reading R5) and T by Newton on Eq. temperature from T_guess
// (the formulas of warp_state_of), then theta and U/c^2 as bstate_prepare.
template <int D, int M, typename R>
__device__ __forceinline__ void bstate_of(BState<D, M, R>& s, R rho, R rhoE, const R (&j)[D],
                                          const R (&rs)[M], const R (&js)[M][D],
                                          double T_guess, const DevMech& m, const Units& un,
                                          int* status) {
  s.rho = rho;
  R usq = R(0);
#pragma unroll
  for (int d = 0; d < D; ++d) { s.u[d] = j[d] / rho; usq += s.u[d] * s.u[d]; }
  R rM = rho, jM[D];
#pragma unroll
  for (int d = 0; d < D; ++d) jM[d] = j[d];
#pragma unroll
  for (int a = 0; a < M - 1; ++a) {
    rM -= rs[a];
#pragma unroll
    for (int d = 0; d < D; ++d) jM[d] -= js[a][d];
  }
#pragma unroll
  for (int a = 0; a < M; ++a) {
    const R ra = a < M - 1 ? rs[a] : rM;
    s.Y[a * kBnd] = ra / rho;
    if (s.us) {
      R ja[D];
#pragma unroll
      for (int d = 0; d < D; ++d) ja[d] = a < M - 1 ? js[a][d] : jM[d];
      const bool tiny = species_velocity_undefined<D, R>(ra, ja);
#pragma unroll
      for (int d = 0; d < D; ++d) s.us[(a * D + d) * kBnd] = tiny ? s.u[d] : ja[d] / ra;
    }
  }
  bool ok;
  if constexpr (!kFF<R>) {
    double Y[M];
#pragma unroll
    for (int a = 0; a < M; ++a) Y[a] = double(s.Y[a * kBnd]);
    const double U = (double(rhoE / rho) - 0.5 * double(usq)) * un.c * un.c;
    const double T = newton_T<M>(m, Y, U, T_guess, un.newton_max_iter, un.newton_rtol, ok);
    s.T = R(T);
    s.T_full = T;
  } else {
    ff Yf[M];
#pragma unroll
    for (int a = 0; a < M; ++a) Yf[a] = ff(s.Y[a * kBnd]);
    const ff U = (ff(rhoE / rho) + ff(-0.5f * usq)) * un.c2_f;
    const ff T = newton_T_ff<M>(m, Yf, U, ff_from_double(T_guess), un.newton_max_iter,
                                un.newton_rtol_f, ok);
    s.T = T.hi;
    s.T_full = ff_to_double(T);
  }
  if (!ok) atomicOr(status, ST_NEWTON);
  bstate_prepare<D, M, R>(s, m, un);
}

// Per-axis factor Psi_c (Eqs. phi0, phiPlus, phis) for a warp-uniform c.
template <typename R> __device__ __forceinline__ R bpsi(int c, R xi, R P) {
  return c == 0 ? R(1) - P : R(0.5) * (c > 0 ? P + xi : P - xi);
}

// Equilibrium population of lattice l (compile-time) in direction with
// velocity c (warp-uniform) of state s (Eqs. faEqGeneral, fEqGeneral,
// gEqGeneral; the energy lattice by the closed form of Eq. geq_i).
template <int D, int M, int l, typename R>
__device__ __forceinline__ R beq(const BState<D, M, R>& s, const int (&c)[3], const DevMech& m,
                                 const Units& un) {
  if constexpr (l < M - 1) {
    R th_l;
    if constexpr (sizeof(R) == 8) th_l = R(m.Ra[l] * double(s.T) * un.inv_c2);
    else th_l = m.Ra_s[l] * s.T * un.inv_c2_s;
    R p = s.rho * s.Y[l * kBnd];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const R xi = s.us ? s.us[(l * D + d) * kBnd] : s.u[d];
      p *= bpsi<R>(c[d], xi, th_l + xi * xi);
    }
    return p;
  } else if constexpr (l == M - 1) {
    R p = s.rho;
#pragma unroll
    for (int d = 0; d < D; ++d) p *= bpsi<R>(c[d], s.u[d], s.th + s.u[d] * s.u[d]);
    return p;
  } else {
    R A[3], B[3], prodA = R(1);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const R ua = s.u[d];
      const R O1 = s.th * ua + R(0.5) * ua * ua * ua;
      const R O2 = s.th * s.th + R(2.5) * s.th * ua * ua + R(0.5) * ua * ua * ua * ua;
      A[d] = bpsi<R>(c[d], ua, s.th + ua * ua);
      B[d] = c[d] == 0 ? R(0.5) * ua * ua - O2 : R(0.5) * (c[d] > 0 ? O2 + O1 : O2 - O1);
      prodA *= A[d];
    }
    R sumB = R(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      R t = B[d];
#pragma unroll
      for (int e = 0; e < D; ++e)
        if (e != d) t *= A[e];
      sumB += t;
    }
    return s.rho * (s.U * prodA + sumB);
  }
}

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

// Population sums sum_i v(l, i) and sum_i c_i v(l, i) of every lattice; the
// functor gives v through fn.begin(i, c) (once per direction) and
// fn.template get<l>(i, c) (compile-time l).
template <int D, int M, typename R, typename F>
__device__ __forceinline__ void bsums(F& fn, R& rho, R& rhoE, R (&j)[D], R (&rs)[M],
                                      R (&js)[M][D]) {
  constexpr int Q = Lat<D>::Q;
  rho = rhoE = R(0);
#pragma unroll
  for (int d = 0; d < D; ++d) j[d] = R(0);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    rs[a] = R(0);
#pragma unroll
    for (int d = 0; d < D; ++d) js[a][d] = R(0);
  }
#pragma unroll 1
  for (int i = 0; i < Q; ++i) {
    const int c[3] = {cvel(i, 0), cvel(i, 1), D == 3 ? cvel(i, 2) : 0};
    fn.begin(i, c);
    auto acc = [&](R v, R& sum, R (&sj)[D]) {
      sum += v;
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (c[d] != 0) sj[d] += c[d] > 0 ? v : -v;
    };
    ForL<0, M - 1>::run([&](auto lc) {
      constexpr int l = decltype(lc)::value;
      acc(fn.template get<l>(i, c), rs[l], js[l]);
    });
    acc(fn.template get<M - 1>(i, c), rho, j);
    rhoE += fn.template get<M>(i, c);
  }
}

// Value functors of bsums.  BPull: the pulled population (wrapped source
// address) or, with bbk and an incoming link, the node's own opposite
// post-collision population (Eq. bb).
template <int D, int M, typename S, typename R> struct BPull {
  static constexpr int Q = Lat<D>::Q;
  const S* src;
  const float4* codec;
  long long N, n, sn;
  int x, y, z;
  const Geom* g;
  unsigned inc;
  bool in_i, bbk;
  __device__ __forceinline__ void begin(int i, const int (&)[3]) {
    in_i = inc >> i & 1u;
    sn = node_shift<D>(x, y, z, i, -1, *g);
  }
  template <int l> __device__ __forceinline__ R get(int i, const int (&)[3]) const {
    const bool bb = bbk && in_i;
    const long long mm = bb ? n : sn;
    const int ii = bb ? Q - 1 - i : i;
    return Codec<S>::template dec<R>(__ldg(src + (long long)(l * Q + ii) * N + mm), codec,
                                     l * Q + ii);
  }
};

// The stored populations of one node.
template <int D, int M, typename S, typename R> struct BNode {
  static constexpr int Q = Lat<D>::Q;
  const S* src;
  const float4* codec;
  long long N, node;
  __device__ __forceinline__ void begin(int, const int (&)[3]) {}
  template <int l> __device__ __forceinline__ R get(int i, const int (&)[3]) const {
    return Codec<S>::template dec<R>(__ldg(src + (long long)(l * Q + i) * N + node), codec,
                                     l * Q + i);
  }
};

// Values written to the node's reconstructed populations as they are summed.
template <int D, int M, typename R, typename F> struct BStore {
  static constexpr int Q = Lat<D>::Q;
  F& f;
  double* P;
  long long st;
  __device__ __forceinline__ void begin(int i, const int (&c)[3]) { f.begin(i, c); }
  template <int l> __device__ __forceinline__ R get(int i, const int (&c)[3]) const {
    const R v = f.template get<l>(i, c);
    P[(long long)(l * Q + i) * st] = double(v);
    return v;
  }
};

// The local populations: incoming links at the state A, the others pulled.
template <int D, int M, typename S, typename R> struct BLocal {
  BPull<D, M, S, R> p;
  const BState<D, M, R>* A;
  const DevMech* m;
  const Units* un;
  __device__ __forceinline__ void begin(int i, const int (&c)[3]) { p.begin(i, c); }
  template <int l> __device__ __forceinline__ R get(int i, const int (&c)[3]) const {
    return p.in_i ? beq<D, M, l, R>(*A, c, *m, *un) : p.template get<l>(i, c);
  }
};

// Step 4: target + local populations - local equilibria; the simplified
// inlet takes the local equilibria.
template <int D, int M, typename S, typename R> struct BFinal {
  BLocal<D, M, S, R>* lo;
  const BState<D, M, R>* Bt;
  const BState<D, M, R>* L;
  bool simple;
  __device__ __forceinline__ void begin(int i, const int (&c)[3]) { lo->begin(i, c); }
  template <int l> __device__ __forceinline__ R get(int i, const int (&c)[3]) const {
    const R loc = beq<D, M, l, R>(*L, c, *lo->m, *lo->un);
    if (simple) return loc;
    return beq<D, M, l, R>(*Bt, c, *lo->m, *lo->un) + lo->template get<l>(i, c) - loc;
  }
};

// The boundary procedure of interface node k and its moment record.
template <int D, int M, typename S, typename R>
__device__ __forceinline__ void bnode_body(const S* __restrict__ src, const BCDev& bc,
                                           R* __restrict__ rec, double* __restrict__ Tf,
                                           int* __restrict__ status, const Geom& g,
                                           const Units& un, const DevMech& m, int k,
                                           R* col) {
  constexpr int Q = Lat<D>::Q, NP = Lat<D>::NP;
  using RC = Rec<D, M>;
  const long long N = g.N;
  const long long n = bc.if_node[k];
  const int info = bc.if_info[k];
  const int kind = info & 15;
  const unsigned inc = bc.if_inc[k];
  const int x = (int)(n % g.nx);
  const int y = (int)((n / g.nx) % g.ny);
  const int z = (int)(n / ((long long)g.nx * g.ny));
  const long long st = bc.n_if;
  const float4* codec = g.codec;
  BState<D, M, R> A, B, L;
  A.Y = col;
  L.Y = col + M * kBnd;
  L.us = col + 2 * M * kBnd;
  B.Y = col + (2 * M + M * D) * kBnd;      // spare column (outlet upstream state)
  A.us = B.us = nullptr;
  R rho, rhoE, j[D], rs[M], js[M][D];

  using Pull = BPull<D, M, S, R>;
  if (kind == BK_BB) {
    // Eq. bb: incoming links take the node's own opposite post-collision
    // populations; the record from the result
    Pull pull{src, codec, N, n, 0, x, y, z, &g, inc, false, true};
    BStore<D, M, R, Pull> out{pull, bc.pops + k, st};
    bsums<D, M, R>(out, rho, rhoE, j, rs, js);
  } else {
    if (kind == BK_TMS) {
      // step 1, Eqs. BBrho and BBY: bounce-back density and mass fractions
      Pull pull{src, codec, N, n, 0, x, y, z, &g, inc, false, true};
      bsums<D, M, R>(pull, rho, rhoE, j, rs, js);
      A.rho = rho;
      R ysum = R(0);
#pragma unroll
      for (int a = 0; a < M - 1; ++a) {
        const R Ya = rs[a] / rho;
        A.Y[a * kBnd] = Ya;
        ysum += Ya;
      }
      A.Y[(M - 1) * kBnd] = R(1) - ysum;
#pragma unroll
      for (int d = 0; d < D; ++d) A.u[d] = R(0);     // u^tgt = u_a^tgt = 0
      A.T = R(bc.if_wallT[k]);
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
      using Node = BNode<D, M, S, R>;
      BState<D, M, R>& s0 = L;           // columns reused before the local state
      BState<D, M, R>& s1 = B;
      L.us = nullptr;
      Node n0{src, codec, N, n};
      bsums<D, M, R>(n0, rho, rhoE, j, rs, js);
      bstate_of<D, M, R>(s0, rho, rhoE, j, rs, js, Tf[n], m, un, status);
      Node n1{src, codec, N, up};
      bsums<D, M, R>(n1, rho, rhoE, j, rs, js);
      bstate_of<D, M, R>(s1, rho, rhoE, j, rs, js, Tf[n], m, un, status);
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
      const double Ln = ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz);
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
      L.us = col + 2 * M * kBnd;
    }
    // the local state: incoming links at A, the others as streamed (Eqs.
    // locRho-locT and their inlet / outlet analogues)
    BLocal<D, M, S, R> local{Pull{src, codec, N, n, 0, x, y, z, &g, inc, false, false}, &A,
                             &m, &un};
    bsums<D, M, R>(local, rho, rhoE, j, rs, js);
    if (kind != BK_TMS) L.us = nullptr;               // TMS local species use u_a^loc
    bstate_of<D, M, R>(L, rho, rhoE, j, rs, js, Tf[n], m, un, status);
    const bool simple = kind == BK_INLET && bc.inlet_simplified;
    if (kind == BK_INLET) {                           // target (Eqs. in_tgt_*)
      B.rho = L.rho;
      B.Y = L.Y;
#pragma unroll
      for (int d = 0; d < D; ++d) B.u[d] = A.u[d];
      B.T = R(bc.T_in);
      bstate_prepare<D, M, R>(B, m, un);
    }
    // step 4 (Eqs. ftms-fatms, f_inlet-fa_inlet, f_outlet-fa_outlet):
    // target + (incoming ? A : streamed) - local; the simplified inlet takes
    // the local equilibria
    BFinal<D, M, S, R> fin{&local, kind == BK_INLET ? &B : &A, &L, simple};
    BStore<D, M, R, BFinal<D, M, S, R>> out{fin, bc.pops + k, st};
    bsums<D, M, R>(out, rho, rhoE, j, rs, js);
  }

  // the record from the reconstructed populations (as boundary_record): the
  // state (Newton from the node's previous T), the energy flux and the
  // momentum flux tensor; the reaction sub-steps are left to k_chem
  R q[D], Pt[NP];
  {
    const double* P = bc.pops + k;
#pragma unroll
    for (int d = 0; d < D; ++d) q[d] = R(0);
#pragma unroll
    for (int p = 0; p < NP; ++p) Pt[p] = R(0);
#pragma unroll 1
    for (int i = 0; i < Q; ++i) {
      const int c[3] = {cvel(i, 0), cvel(i, 1), D == 3 ? cvel(i, 2) : 0};
      const R vf = R(P[(long long)((M - 1) * Q + i) * st]);
      const R vg = R(P[(long long)(M * Q + i) * st]);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (c[d] == 0) continue;
        q[d] += c[d] > 0 ? vg : -vg;
#pragma unroll
        for (int e = d; e < D; ++e)
          if (c[e] != 0) Pt[pidx<D>(d, e)] += (c[d] * c[e] > 0) ? vf : -vf;
      }
    }
  }
  BState<D, M, R> s;
  s.Y = A.Y;                                    // the target columns are free now
  s.us = L.us ? L.us : col + 2 * M * kBnd;
  bstate_of<D, M, R>(s, rho, rhoE, j, rs, js, Tf[n], m, un, status);
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
    rec[(RC::QF + d) * N + n] = q[d];
    rec[(RC::PHI + d) * N + n] =
        rr * s.u[d] * (R(1) - R(3) * thR) - rr * s.u[d] * s.u[d] * s.u[d];
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) rec[(RC::P + p) * N + n] = Pt[p];
  rec[RC::E * N + n] = rhoE * (R(1) / rr);
#pragma unroll
  for (int a = 0; a < M; ++a) {
    rec[(RC::Y + a) * N + n] = s.Y[a * kBnd];
#pragma unroll
    for (int d = 0; d < D; ++d) rec[(RC::US + a * D + d) * N + n] = s.us[(a * D + d) * kBnd];
  }
}
