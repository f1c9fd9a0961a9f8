// Discrete adjoint of one free-surface LBM step (SRT, EQ refilling, no
// surface tension, walls and periodic faces), for gradients of a misfit of
// the surface elevation with respect to the viscosity, the gravity and the
// initial state.
//
// The forward step t -> t+1 (the library's own kernels) is replayed from a
// tape: for every step of a segment the stored PDFs F (post-collision, time
// level t), the cell flags, the interface mass M and the fill level Phi.
// The cell types and every conversion decision are taken from the tape
// (types at t and at t+1 tell which cells filled, emptied, were created or
// turned from liquid into interface), so the step is a smooth function of
// (F, M, Phi) and of the parameters, and its vector-Jacobian product is
// written out here by hand:
//
//   fin_i(x) = F_i(x - c_i)                       fluid source (streaming)
//            = F_i'(x)                            wall (halfway bounce-back)
//            = feq_i(rho_G, u*) + feq_i'(rho_G, u*) - F_i'(x)
//                                                 gas (Eq. nm-fslbm-boundary-condition),
//              u* = sum c F(x) / sum F(x) - g/2
//   m_new(x) = M(x) + sum_i d_i(x)                interface (Eq. nm-fslbm-mass-flux,
//              d_i = F_i'(y) - F_i(x), y = x + c_i liquid;
//              d_i = (Phi_x + Phi_y)/2 * br_i, y interface, br from Thuerey's table
//   rho = sum fin, u = sum c fin / rho + g/2, F = rho g
//   fn_i(x) = fin_i - omega (fin_i - feq_i(rho, u)) + (1 - omega/2) G_i(u, F)
//                                                 (Eqs. nm-lbm-collision, nm-lbm-force-guo)
//   interface at t+1: M1 = base + excess share, Phi1 = M1 / rho;
//     base = m_new (stayed interface), rho (liquid turned interface), 0 (new)
//   filled cell: m_ex = m_new - rho; emptied cell: m_ex = m_new (Eq. nm-fslbm-excess-mass),
//     shared evenly over its interface neighbours at t+1 (counted per direction)
//   new cell: fn(x) = feq(mean rho_y, mean u_y) over its valid neighbours y,
//     rho_y, u_y the moments of F(t+1)(y) (Sec. 3.1, EQ); its rho = sum fn(x)
//
// Every kernel is a gather (one thread per cell, no atomics on the adjoint
// fields); the parameter gradients are accumulated with FP64 atomics.
#pragma once
// Included by fsl_api.cu after fsl_kernels.cuh.

namespace fsl {

// the tape entry of one time level
struct AdjLevel {
  const void* F;          // stored PDFs (storage type of the path), q planes
  const uint8_t* flags;   // cell flags
  const double* M;        // interface mass
  const double* Phi;      // fill level
};

// adjoint fields (arithmetic type R) and accumulators
template <class R>
struct AdjFields {
  R* lF;     // q planes: adjoint of F at the current level (in: t+1, out: t)
  R* lF0;    // q planes: output buffer for the adjoint of F at t
  R* lfin;   // q planes: adjoint of the pulled values fin at t
  R* lM;     // cells: adjoint of M (in: t+1; out: t, in lM0)
  R* lM0;
  R* lP;     // cells: adjoint of Phi (in: t+1; out: t, in lP0)
  R* lP0;
  R* lm1;    // cells: adjoint of the mass at t+1 of interface-at-t+1 cells
  R* lrhoP;  // cells: adjoint of rho through Phi1 = M1 / rho (and the base m = rho)
  R* lmnew;  // cells: adjoint of m_new
  R* lrho;   // cells: adjoint of the collision density rho (all contributions)
  R* lbar;   // 4 per cell: (rho_bar, u_bar) adjoint of a new cell / |V|
  R* lg;     // 3 per cell: adjoint of u* of the gas boundary condition
  double* acc;  // [0] dJ/domega, [1..3] dJ/dg_a
};

template <int Q>
__device__ __forceinline__ int adj_opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

template <int Q, class ST>
__device__ __forceinline__ typename ST::R adj_ld(const void* F, long long plane, int i, int c) {
  using T = typename ST::T;
  return (typename ST::R)ST::ldf(reinterpret_cast<const T*>(F) + i * plane + c, rw<Q>(i));
}

// Thuerey class of an interface cell from the flags of its level: 0 standard,
// 1 no liquid neighbour (NF), 2 no gas neighbour (NE)
template <int Q>
__device__ __forceinline__ int adj_class(const Geom& g, const uint8_t* fl, int x, int y, int z) {
  bool has_liq = false, has_gas = false;
  for (int d = 1; d < Q; ++d) {
    const int t = type_at(fl, nb_at(g, x, y, z, rc(d, 0), rc(d, 1), rc(d, 2)));
    has_liq |= t == T_LIQ;
    has_gas |= t == T_GAS;
  }
  if (!has_liq && has_gas) return 1;
  if (!has_gas && has_liq) return 2;
  return 0;
}

// coefficients of f_in and f_out in the bracket of an interface pair
// (classes of the cell and of its neighbour); simple = plain f_in - f_out
__device__ __forceinline__ void adj_bracket(int cx, int cy, bool simple, int& a_in, int& a_out) {
  a_in = 1;
  a_out = -1;
  if (simple) return;
  if (cx == 0) {
    if (cy == 1) a_out = 0;
    else if (cy == 2) a_in = 0;
  } else if (cx == 1) {
    if (cy != 1) a_in = 0;
  } else {
    if (cy != 2) a_out = 0;
  }
}

template <int Q, class R>
__device__ __forceinline__ R adj_feq(int i, R rho, R ux, R uy, R uz) {
  const R cu = (R)rc(i, 0) * ux + (R)rc(i, 1) * uy + (R)rc(i, 2) * uz;
  const R usq = ux * ux + uy * uy + uz * uz;
  return (R)rw<Q>(i) * rho * ((R)1 + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * usq);
}

// the pulled values at t of a fluid cell, with the kind of each source
// (0 fluid, 1 wall, 2 gas) and the stored moments (rho*, u*) of the cell
template <int Q, class ST>
__device__ __forceinline__ void adj_fin(const Geom& g, const Phys& p, const AdjLevel& L, int c,
                                        int x, int y, int z, typename ST::R* fin, int* kind,
                                        typename ST::R& rs, typename ST::R* us) {
  using R = typename ST::R;
  const long long P = g.plane;
  R r = 0, jx = 0, jy = 0, jz = 0;
  for (int i = 0; i < Q; ++i) {
    const R f = adj_ld<Q, ST>(L.F, P, i, c);
    r += f;
    jx += (R)rc(i, 0) * f;
    jy += (R)rc(i, 1) * f;
    jz += (R)rc(i, 2) * f;
  }
  rs = r;
  us[0] = jx / r - (R)0.5 * (R)p.g[0];
  us[1] = jy / r - (R)0.5 * (R)p.g[1];
  us[2] = jz / r - (R)0.5 * (R)p.g[2];
  const R rhoG = (R)(3.0 * p.p_v);
  for (int i = 0; i < Q; ++i) {
    const int src = nb_at(g, x, y, z, -rc(i, 0), -rc(i, 1), -rc(i, 2));
    const int t = type_at(L.flags, src);
    const int io = adj_opp<Q>(i);
    if (is_fluid(t)) {
      kind[i] = 0;
      fin[i] = adj_ld<Q, ST>(L.F, P, i, src);
    } else if (t == T_OBST) {
      kind[i] = 1;
      fin[i] = adj_ld<Q, ST>(L.F, P, io, c);
    } else {
      kind[i] = 2;
      fin[i] = adj_feq<Q, R>(i, rhoG, us[0], us[1], us[2]) +
               adj_feq<Q, R>(io, rhoG, us[0], us[1], us[2]) - adj_ld<Q, ST>(L.F, P, io, c);
    }
  }
}

// B1: cells that are interface at t+1: adjoint of their mass and of the
// density that divides it
template <int Q, class ST>
__global__ void k_adj_phi(Geom g, Phys p, AdjLevel L0, AdjLevel L1,
                          AdjFields<typename ST::R> A) {
  using R = typename ST::R;
  FSL_GRID_LOOP(k, (unsigned)g.cells) {
    const int c = (int)k;
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    R m1 = 0, rp = 0;
    if (x < g.nx && (L1.flags[c] & F_TYPE) == T_IF) {
      R rho;
      if ((L0.flags[c] & F_TYPE) == T_GAS) {  // new cell: density of its refilled PDFs
        rho = 0;
        for (int i = 0; i < Q; ++i) rho += adj_ld<Q, ST>(L1.F, g.plane, i, c);
      } else {
        R fin[Q], rs, us[3];
        int kind[Q];
        adj_fin<Q, ST>(g, p, L0, c, x, y, z, fin, kind, rs, us);
        rho = 0;
        for (int i = 0; i < Q; ++i) rho += fin[i];
      }
      m1 = A.lM[c] + A.lP[c] / rho;
      rp = -A.lP[c] * (R)L1.Phi[c] / rho;
    }
    A.lm1[c] = m1;
    A.lrhoP[c] = rp;
  }
}

// B2: adjoint of m_new and of the collision density of every fluid cell at t
// (including the excess mass of converted cells, gathered from receivers)
template <int Q, class ST>
__global__ void k_adj_mass(Geom g, Phys p, AdjLevel L0, AdjLevel L1,
                           AdjFields<typename ST::R> A) {
  using R = typename ST::R;
  FSL_GRID_LOOP(k, (unsigned)g.cells) {
    const int c = (int)k;
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    R lmn = 0, lr = 0;
    const int t0 = L0.flags[c] & F_TYPE, t1 = L1.flags[c] & F_TYPE;
    if (x < g.nx && is_fluid(t0)) {
      if (t1 == T_IF) {
        lr = A.lrhoP[c];
        if (t0 == T_IF) lmn = A.lm1[c];  // M1 = m_new + share
        else lr += A.lm1[c];             // liquid turned interface: M1 = rho + share
      } else if (t0 == T_IF && (t1 == T_LIQ || t1 == T_GAS)) {
        // converted: excess mass to the interface neighbours at t+1
        int nr = 0;
        R s = 0;
        for (int d = 1; d < Q; ++d) {
          const int n = nb_at(g, x, y, z, rc(d, 0), rc(d, 1), rc(d, 2));
          if (n >= 0 && (L1.flags[n] & F_TYPE) == T_IF) {
            ++nr;
            s += A.lm1[n];
          }
        }
        const R lex = nr > 0 ? s / (R)nr : (R)0;  // no receiver: lost mass, no later effect
        lmn = lex;                                // m_ex = m_new - rho or m_new
        if (t1 == T_LIQ) lr = -lex;
      }
    }
    A.lmnew[c] = lmn;
    A.lrho[c] = lr;
  }
}

// B3: new cells: adjoint of the means that their equilibrium was built from
template <int Q, class ST>
__global__ void k_adj_refill(Geom g, Phys p, AdjLevel L0, AdjLevel L1,
                             AdjFields<typename ST::R> A) {
  using R = typename ST::R;
  FSL_GRID_LOOP(k, (unsigned)g.cells) {
    const int c = (int)k;
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    R out[4] = {0, 0, 0, 0};
    if (x < g.nx && (L0.flags[c] & F_TYPE) == T_GAS && (L1.flags[c] & F_TYPE) == T_IF) {
      int cnt = 0;
      R rsum = 0, us[3] = {0, 0, 0};
      for (int d = 1; d < Q; ++d) {
        const int n = nb_at(g, x, y, z, rc(d, 0), rc(d, 1), rc(d, 2));
        if (n < 0) continue;
        const int tn0 = L0.flags[n] & F_TYPE, tn1 = L1.flags[n] & F_TYPE;
        if (!is_fluid(tn1) || (tn0 == T_GAS)) continue;  // valid: fluid at t+1, not new
        R r = 0, j[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
          const R f = adj_ld<Q, ST>(L1.F, g.plane, i, n);
          r += f;
          for (int a = 0; a < 3; ++a) j[a] += (R)rc(i, a) * f;
        }
        rsum += r;
        for (int a = 0; a < 3; ++a) us[a] += j[a] / r - (R)0.5 * (R)p.g[a];
        ++cnt;
      }
      if (cnt > 0) {
        const R rb = rsum / (R)cnt;
        const R ub[3] = {us[0] / (R)cnt, us[1] / (R)cnt, us[2] / (R)cnt};
        R lrb = 0, lub[3] = {0, 0, 0};
        for (int i = 0; i < Q; ++i) {
          // fn_i = feq_i(rb, ub); rho of the cell = sum fn
          const R lf = A.lF[i * g.plane + c] + A.lrhoP[c];
          const R cu = (R)rc(i, 0) * ub[0] + (R)rc(i, 1) * ub[1] + (R)rc(i, 2) * ub[2];
          const R usq = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
          const R w = (R)rw<Q>(i);
          lrb += lf * w * ((R)1 + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * usq);
          for (int a = 0; a < 3; ++a)
            lub[a] += lf * w * rb * ((R)3 * (R)rc(i, a) + (R)9 * cu * (R)rc(i, a) - (R)3 * ub[a]);
        }
        // u_y = j_y / rho_y - g/2 for every y: d ub / d g = -1/2
        for (int a = 0; a < 3; ++a) atomicAdd(&A.acc[1 + a], -0.5 * (double)lub[a]);
        out[0] = lrb / (R)cnt;
        for (int a = 0; a < 3; ++a) out[1 + a] = lub[a] / (R)cnt;
      }
    }
    for (int a = 0; a < 4; ++a) A.lbar[4 * (long long)c + a] = out[a];
  }
}

// B4: collision (and gas boundary condition) of every fluid cell at t
template <int Q, class ST>
__global__ void k_adj_collide(Geom g, Phys p, AdjLevel L0, AdjLevel L1,
                              AdjFields<typename ST::R> A) {
  using R = typename ST::R;
  const long long P = g.plane;
  const R om = (R)p.omega, pre = (R)1 - (R)0.5 * om;
  const R gv[3] = {(R)p.g[0], (R)p.g[1], (R)p.g[2]};
  double dom = 0.0, dg[3] = {0.0, 0.0, 0.0};
  FSL_GRID_LOOP(k, (unsigned)g.cells) {
    const int c = (int)k;
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    const int t0 = L0.flags[c] & F_TYPE, t1 = L1.flags[c] & F_TYPE;
    if (x >= g.nx || !is_fluid(t0)) {
      for (int i = 0; i < Q; ++i) A.lfin[i * P + c] = 0;
      for (int a = 0; a < 3; ++a) A.lg[3 * (long long)c + a] = 0;
      continue;
    }
    // adjoint of the post-collision values fn(x) = F(t+1)(x)
    R lfn[Q];
    for (int i = 0; i < Q; ++i) lfn[i] = is_fluid(t1) ? A.lF[i * P + c] : (R)0;
    if (is_fluid(t1)) {
      // this cell's F(t+1) also fed the equilibrium of new neighbours
      R r1 = 0, j1[3] = {0, 0, 0};
      bool any = false;
      for (int d = 1; d < Q; ++d) {
        const int n = nb_at(g, x, y, z, rc(d, 0), rc(d, 1), rc(d, 2));
        if (n >= 0 && (L0.flags[n] & F_TYPE) == T_GAS && (L1.flags[n] & F_TYPE) == T_IF) any = true;
      }
      if (any) {
        for (int i = 0; i < Q; ++i) {
          const R f = adj_ld<Q, ST>(L1.F, P, i, c);
          r1 += f;
          for (int a = 0; a < 3; ++a) j1[a] += (R)rc(i, a) * f;
        }
        for (int d = 1; d < Q; ++d) {
          const int n = nb_at(g, x, y, z, rc(d, 0), rc(d, 1), rc(d, 2));
          if (n < 0 || (L0.flags[n] & F_TYPE) != T_GAS || (L1.flags[n] & F_TYPE) != T_IF) continue;
          const R* lb = A.lbar + 4 * (long long)n;
          for (int i = 0; i < Q; ++i) {
            R v = lb[0];
            for (int a = 0; a < 3; ++a) v += lb[1 + a] * ((R)rc(i, a) - j1[a] / r1) / r1;
            lfn[i] += v;
          }
        }
      }
    }
    R fin[Q], rs, us[3];
    int kind[Q];
    adj_fin<Q, ST>(g, p, L0, c, x, y, z, fin, kind, rs, us);
    R rho = 0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
      rho += fin[i];
      for (int a = 0; a < 3; ++a) j[a] += (R)rc(i, a) * fin[i];
    }
    const R u[3] = {j[0] / rho + (R)0.5 * gv[0], j[1] / rho + (R)0.5 * gv[1], j[2] / rho + (R)0.5 * gv[2]};
    const R F[3] = {rho * gv[0], rho * gv[1], rho * gv[2]};
    R Lr = 0, Lu[3] = {0, 0, 0}, LF[3] = {0, 0, 0};
    double dom_c = 0.0;
    for (int i = 0; i < Q; ++i) {
      const R w = (R)rw<Q>(i);
      const R ci[3] = {(R)rc(i, 0), (R)rc(i, 1), (R)rc(i, 2)};
      const R cu = ci[0] * u[0] + ci[1] * u[1] + ci[2] * u[2];
      const R cF = ci[0] * F[0] + ci[1] * F[1] + ci[2] * F[2];
      const R usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
      const R feq = w * rho * ((R)1 + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * usq);
      const R G = w * ((R)3 * ((ci[0] - u[0]) * F[0] + (ci[1] - u[1]) * F[1] + (ci[2] - u[2]) * F[2]) +
                       (R)9 * cu * cF);
      // fn = fin - om (fin - feq) + pre G
      Lr += lfn[i] * (om * feq / rho);  // d feq / d rho at fixed u
      for (int a = 0; a < 3; ++a) {
        Lu[a] += lfn[i] * (om * w * rho * ((R)3 * ci[a] + (R)9 * cu * ci[a] - (R)3 * u[a]) +
                           pre * w * ((R)-3 * F[a] + (R)9 * ci[a] * cF));
        LF[a] += lfn[i] * pre * w * ((R)3 * (ci[a] - u[a]) + (R)9 * cu * ci[a]);
      }
      dom_c += (double)(lfn[i] * (feq - fin[i] - (R)0.5 * G));
    }
    // F = rho g: through rho and through g
    for (int a = 0; a < 3; ++a) Lr += LF[a] * gv[a];
    dom += dom_c;
    for (int a = 0; a < 3; ++a) dg[a] += (double)((R)0.5 * Lu[a] + LF[a] * rho);
    Lr += A.lrho[c];
    R lfin[Q];
    for (int i = 0; i < Q; ++i) {
      R v = ((R)1 - om) * lfn[i] + Lr;
      for (int a = 0; a < 3; ++a) v += Lu[a] * ((R)rc(i, a) - j[a] / rho) / rho;
      lfin[i] = v;
      A.lfin[i * P + c] = v;
    }
    // gas sources: feq_i + feq_i' at (rho_G, u*)
    R Lg[3] = {0, 0, 0};
    const R rhoG = (R)(3.0 * p.p_v);
    for (int i = 0; i < Q; ++i) {
      if (kind[i] != 2) continue;
      const R w = (R)rw<Q>(i);
      const R cu = (R)rc(i, 0) * us[0] + (R)rc(i, 1) * us[1] + (R)rc(i, 2) * us[2];
      for (int a = 0; a < 3; ++a)
        Lg[a] += lfin[i] * (R)2 * w * rhoG * ((R)9 * cu * (R)rc(i, a) - (R)3 * us[a]);
    }
    for (int a = 0; a < 3; ++a) {
      A.lg[3 * (long long)c + a] = Lg[a];
      dg[a] += -0.5 * (double)Lg[a];  // u* = j*/rho* - g/2
    }
  }
  atomicAdd(&A.acc[0], dom);
  for (int a = 0; a < 3; ++a) atomicAdd(&A.acc[1 + a], dg[a]);
}

// B5: adjoint of the state at t (F, M, Phi) by gathering every use of it
template <int Q, class ST>
__global__ void k_adj_state(Geom g, Phys p, AdjLevel L0, AdjFields<typename ST::R> A) {
  using R = typename ST::R;
  const long long P = g.plane;
  const bool simple = (p.options & 1u) != 0;
  FSL_GRID_LOOP(k, (unsigned)g.cells) {
    const int c = (int)k;
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    const int t0 = L0.flags[c] & F_TYPE;
    if (x >= g.nx || !is_fluid(t0)) {
      for (int i = 0; i < Q; ++i) A.lF0[i * P + c] = 0;
      A.lM0[c] = 0;
      A.lP0[c] = 0;
      continue;
    }
    const bool iface = t0 == T_IF;
    const int cls = iface ? adj_class<Q>(g, L0.flags, x, y, z) : 0;
    const R phx = (R)L0.Phi[c];
    const R lmx = iface ? A.lmnew[c] : (R)0;
    // stored moments of the cell (gas boundary condition)
    R rs = 0, js[3] = {0, 0, 0};
    if (iface) {
      for (int i = 0; i < Q; ++i) {
        const R f = adj_ld<Q, ST>(L0.F, P, i, c);
        rs += f;
        for (int a = 0; a < 3; ++a) js[a] += (R)rc(i, a) * f;
      }
    }
    const R* lg = A.lg + 3 * (long long)c;
    R lphi = 0;
    for (int kd = 0; kd < Q; ++kd) {
      R v = 0;
      const int ko = adj_opp<Q>(kd);
      // the cell in direction c_k: consumer of F_k(x) by streaming, and the
      // partner of the interface pair (x, x + c_k)
      const int n = kd == 0 ? c : nb_at(g, x, y, z, rc(kd, 0), rc(kd, 1), rc(kd, 2));
      const int tn = type_at(L0.flags, n);
      if (kd == 0) {
        v += A.lfin[c];  // rest population streams onto itself
      } else if (is_fluid(tn)) {
        v += A.lfin[kd * P + n];  // streaming
      } else if (tn == T_OBST) {
        v += A.lfin[ko * P + c];  // bounce-back into direction k'
      } else {
        v -= A.lfin[ko * P + c];  // gas: - F_k(x) in fin_k'
      }
      if (iface) {
        for (int a = 0; a < 3; ++a) v += lg[a] * ((R)rc(kd, a) - js[a] / rs) / rs;
      }
      if (kd > 0 && is_fluid(tn)) {
        // pair (x, n): own flux d_k(x) has f_out = F_k(x); n's flux d_k'(n)
        // has f_in = F_k(x)
        const bool n_if = tn == T_IF;
        const R phn = (R)L0.Phi[n];
        const R lmn = n_if ? A.lmnew[n] : (R)0;
        if (iface) {
          if (tn == T_LIQ) {
            v -= lmx;
          } else {
            const int cn = adj_class<Q>(g, L0.flags, n % g.sx, (n / g.sx) % g.ny, n / (g.sx * g.ny));
            int a_in, a_out;
            adj_bracket(cls, cn, simple, a_in, a_out);
            const R half = (R)0.5 * (phx + phn);
            v += half * (R)a_out * lmx;
            // fill-level weights of both fluxes of the pair
            const R fin_x = adj_ld<Q, ST>(L0.F, P, ko, n), fout_x = adj_ld<Q, ST>(L0.F, P, kd, c);
            const R br_x = (R)a_in * fin_x + (R)a_out * fout_x;
            int b_in, b_out;
            adj_bracket(cn, cls, simple, b_in, b_out);
            const R br_n = (R)b_in * fout_x + (R)b_out * fin_x;  // n's f_in = F_k(x), f_out = F_k'(n)
            lphi += (R)0.5 * br_x * lmx + (R)0.5 * br_n * lmn;
            v += half * (R)b_in * lmn;
          }
        } else if (n_if) {
          v += lmn;  // x liquid: d_k'(n) = F_k(x) - F_k'(n)
        }
      }
      A.lF0[kd * P + c] = v;
    }
    A.lM0[c] = lmx;
    A.lP0[c] = lphi;
  }
}

// the observable's adjoint at one time level: d J / d (column height) spread
// over the cells at x = 0 (the column height is their fill levels summed
// over y and averaged over z)
__global__ void k_adj_observe(Geom g, double dj, double* lP_dbl, float* lP_flt) {
  FSL_GRID_LOOP(k, (unsigned)(g.ny * g.nz)) {
    const int c = (int)k * g.sx;  // x = 0 of row k
    const double v = dj / (double)g.nz;
    if (lP_dbl) lP_dbl[c] += v;
    if (lP_flt) lP_flt[c] += (float)v;
  }
}

// the initial state's adjoint: F = feq(rho0, 0), M = phi0 rho0 (interface) or
// rho0 (liquid), Phi = phi0; per cell d J / d rho0 and d J / d phi0 (dense
// x-fastest layout), and the hydrostatic rho0 = 1 + 3 g_a (x_a + 1/2 - h_ref)
// added to d J / d g_a
template <int Q, class ST>
__global__ void k_adj_init(Geom g, Phys p, AdjLevel L0, AdjFields<typename ST::R> A, double h_ref,
                           double* drho0, double* dphi0) {
  using R = typename ST::R;
  double dga = 0.0;
  FSL_GRID_LOOP(k, (unsigned)g.cells) {
    const int c = (int)k;
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    if (x >= g.nx) continue;
    const long long u = x + (long long)g.nx * (y + (long long)g.ny * z);
    const int t0 = L0.flags[c] & F_TYPE;
    double dr = 0.0, dp = 0.0;
    if (is_fluid(t0)) {
      for (int i = 0; i < Q; ++i) dr += (double)A.lF[i * g.plane + c] * rw<Q>(i);
      if (t0 == T_IF) {
        dr += (double)A.lM[c] * L0.Phi[c];
        // rho0 of the cell: M0 / Phi0 when Phi0 > 0, else from the PDFs
        double r0 = 0.0;
        for (int i = 0; i < Q; ++i) r0 += (double)adj_ld<Q, ST>(L0.F, g.plane, i, c);
        dp = (double)A.lM[c] * r0 + (double)A.lP[c];
      } else {
        dr += (double)A.lM[c];
      }
      if (p.gaxis >= 0 && !isnan(h_ref)) {
        const int pa = p.gaxis == 0 ? x : p.gaxis == 1 ? y : z;
        dga += dr * 3.0 * (((double)pa + 0.5) - h_ref);
      }
    }
    drho0[u] = dr;
    dphi0[u] = dp;
  }
  if (p.gaxis >= 0) atomicAdd(&A.acc[1 + p.gaxis], dga);
}

}  // namespace fsl
