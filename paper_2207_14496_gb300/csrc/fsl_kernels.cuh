// FSLBM step kernels, templated on the lattice (Q = 19 | 27) and the PDF
// storage (SF64 | SF32 | SF16 | SBF16).  Each precision family instantiates
// them in its own translation unit (fsl_prec_*.cu); the FP64 unit is compiled
// with -fmad=false so that its arithmetic is bit-reproducible against a plain
// FP64 evaluation in the operation order written here.
//
// One step (Sec. 2 and 3 of the paper), t -> t+1:
//   k_stream_collide  pull streaming (Eq. nm-lbm-streaming), halfway bounce-back,
//                     free-surface anti-bounce-back for PDFs from gas
//                     (Eq. nm-fslbm-boundary-condition), interface mass flux
//                     (Eq. nm-fslbm-mass-flux, Thuerey classes), moments
//                     (Eqs. nm-lbm-density, nm-lbm-velocity), SRT/TRT collision
//                     with Guo forcing (Eqs. nm-lbm-collision, nm-lbm-force-guo),
//                     fill level m/rho (Eq. nm-fslbm-mass), conversion marks
//                     (threshold eps_phi) and warp-ballot compaction of the
//                     interface, to-liquid and to-gas cells;
//   k_fill            commit fill levels; gas neighbours of filled cells become
//                     new interface cells; to-gas neighbours are kept (filling
//                     wins a conflict);
//   k_empty           liquid neighbours of emptied cells become interface;
//   k_finalise        excess mass (Eq. nm-fslbm-excess-mass), type change;
//   k_refill          EQ, EQ+NEQ, GEQ, EXT, AVG refilling (Sec. 3.1);
//   k_excess_share    share per receiver, receiver compaction;
//   k_excess_gather   receivers gather their shares in direction order;
//   k_classify        Thuerey classes and curvature K = -div(n_hat) for the
//                     next step, clean-up of the per-step marks;
//   k_end_step        trace record, counters, step counter.
#pragma once
#include "fsl_lattice.cuh"

namespace fsl {

// ---------------------------------------------------------------- physics
// Equilibrium (Eq. nm-lbm-equilibrium) in working representation.
//   exact:   f_i^eq = w_i rho (1 + 3 cu + 4.5 cu^2 - 1.5 u.u)
//   shifted: f_i^eq - w_i = w_i (drho + rho (3 cu + 4.5 cu^2 - 1.5 u.u)), drho = rho - 1
template <int Q, int I, bool SHIFT, class R>
__device__ __forceinline__ R feq_w(R rho, R drho, R ux, R uy, R uz, R usq) {
  constexpr R w = (R)wgt<Q>(I);
  R cu = dot3<dir_c(I, 0), dir_c(I, 1), dir_c(I, 2)>(ux, uy, uz);
  if (!SHIFT) return w * rho * ((R)1 + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * usq);
  return w * (drho + rho * ((R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * usq));
}

// Guo term without its (1 - lambda/2) prefactor (Eq. nm-lbm-force-guo):
// w_i [3 (c_i - u).F + 9 (c_i.u)(c_i.F)]
template <int Q, int I, class R>
__device__ __forceinline__ R guo_w(R ux, R uy, R uz, R Fx, R Fy, R Fz) {
  constexpr R w = (R)wgt<Q>(I);
  constexpr int cx = dir_c(I, 0), cy = dir_c(I, 1), cz = dir_c(I, 2);
  R cu = dot3<cx, cy, cz>(ux, uy, uz);
  R cF = dot3<cx, cy, cz>(Fx, Fy, Fz);
  R ax = (cx == 0) ? -ux : ((R)cx - ux);
  R ay = (cy == 0) ? -uy : ((R)cy - uy);
  R az = (cz == 0) ? -uz : ((R)cz - uz);
  return w * ((R)3 * (ax * Fx + ay * Fy + az * Fz) + (R)9 * cu * cF);
}

// Zeroth moment (density) of working values, summed i = 0..Q-1.
template <int Q, bool SHIFT, class R>
__device__ __forceinline__ void density(const R* f, R& rho, R& drho) {
  R s = (R)0;
#pragma unroll
  for (int i = 0; i < Q; ++i) s = (i == 0) ? f[0] : s + f[i];
  if (SHIFT) { drho = s; rho = (R)1 + s; }
  else { rho = s; drho = s - (R)1; }
}

// First moment sum_i c_i f_i, summed in direction order with zero terms left out.
template <int Q, class R>
__device__ __forceinline__ void momentum(const R* f, R& jx, R& jy, R& jz) {
  R ax = (R)0, ay = (R)0, az = (R)0;
  bool hx = false, hy = false, hz = false;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int cx = dir_c(i, 0), cy = dir_c(i, 1), cz = dir_c(i, 2);
    if (cx != 0) { R t = cx == 1 ? f[i] : -f[i]; ax = hx ? ax + t : t; hx = true; }
    if (cy != 0) { R t = cy == 1 ? f[i] : -f[i]; ay = hy ? ay + t : t; hy = true; }
    if (cz != 0) { R t = cz == 1 ? f[i] : -f[i]; az = hz ? az + t : t; hz = true; }
  }
  jx = ax; jy = ay; jz = az;
}

template <int Q, bool SHIFT, class R, int I = 0>
__device__ __forceinline__ void feq_all(R* out, R rho, R drho, R ux, R uy, R uz, R usq) {
  if constexpr (I < Q) {
    out[I] = feq_w<Q, I, SHIFT, R>(rho, drho, ux, uy, uz, usq);
    feq_all<Q, SHIFT, R, I + 1>(out, rho, drho, ux, uy, uz, usq);
  }
}
template <int Q, class R, int I = 0>
__device__ __forceinline__ void guo_all(R* out, R ux, R uy, R uz, R Fx, R Fy, R Fz) {
  if constexpr (I < Q) {
    out[I] = guo_w<Q, I, R>(ux, uy, uz, Fx, Fy, Fz);
    guo_all<Q, R, I + 1>(out, ux, uy, uz, Fx, Fy, Fz);
  }
}

// Collision (SRT or TRT) with Guo forcing of the streamed working values fin
// into fout.  Returns u.u for the stability guard.
template <int Q, bool SHIFT, class R>
__device__ __forceinline__ R collide(const R* fin, R* fout, const Phys& p, R& rho_out) {
  R rho, drho, jx, jy, jz;
  density<Q, SHIFT, R>(fin, rho, drho);
  momentum<Q, R>(fin, jx, jy, jz);
  const R gx = (R)p.g[0], gy = (R)p.g[1], gz = (R)p.g[2];
  // Eq. nm-lbm-velocity with F = rho g: u = j / rho + g / 2
  const R ux = jx / rho + (R)0.5 * gx, uy = jy / rho + (R)0.5 * gy, uz = jz / rho + (R)0.5 * gz;
  const R Fx = rho * gx, Fy = rho * gy, Fz = rho * gz;
  const R usq = ux * ux + uy * uy + uz * uz;
  R fe[Q], fg[Q];
  feq_all<Q, SHIFT, R>(fe, rho, drho, ux, uy, uz, usq);
  guo_all<Q, R>(fg, ux, uy, uz, Fx, Fy, Fz);
  if (!p.trt) {
    const R om = (R)p.omega, pre = (R)p.pre_e;
#pragma unroll
    for (int i = 0; i < Q; ++i) fout[i] = fin[i] - om * (fin[i] - fe[i]) + pre * fg[i];
  } else {
    const R le = (R)p.lam_e, lo = (R)p.lam_o, pe = (R)p.pre_e, po = (R)p.pre_o;
    fout[0] = fin[0] - le * (fin[0] - fe[0]) + pe * fg[0];
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const int io = i + 1;
      R fp = (R)0.5 * (fin[i] + fin[io]), fm = (R)0.5 * (fin[i] - fin[io]);
      R ep = (R)0.5 * (fe[i] + fe[io]), em = (R)0.5 * (fe[i] - fe[io]);
      R gp = (R)0.5 * (fg[i] + fg[io]), gm = (R)0.5 * (fg[i] - fg[io]);
      fout[i] = fin[i] - le * (fp - ep) - lo * (fm - em) + pe * gp + po * gm;
      fout[io] = fin[io] - le * (fp - ep) + lo * (fm - em) + pe * gp - po * gm;
    }
  }
  rho_out = rho;
  return usq;
}

// Neighbour coordinates of (x, y, z) along each axis: index 0 -> -1, 1 -> 0,
// 2 -> +1; -1 beyond a wall.
struct Nbr {
  int X[3], Y[3], Z[3];
  int sx, ny;
  __device__ __forceinline__ void setup(const Geom& g, int x, int y, int z) {
    sx = g.sx;
    ny = g.ny;
    X[1] = x; Y[1] = y; Z[1] = z;
    X[0] = x > 0 ? x - 1 : (g.periodic[0] ? g.nx - 1 : -1);
    X[2] = x < g.nx - 1 ? x + 1 : (g.periodic[0] ? 0 : -1);
    Y[0] = y > 0 ? y - 1 : (g.periodic[1] ? g.ny - 1 : -1);
    Y[2] = y < g.ny - 1 ? y + 1 : (g.periodic[1] ? 0 : -1);
    Z[0] = z > 0 ? z - 1 : (g.periodic[2] ? g.nz - 1 : -1);
    Z[2] = z < g.nz - 1 ? z + 1 : (g.periodic[2] ? 0 : -1);
  }
  // cell at offset (dx, dy, dz) in {-1,0,1}^3, -1 beyond a wall
  __device__ __forceinline__ int at(int dx, int dy, int dz) const {
    int a = X[dx + 1], b = Y[dy + 1], c = Z[dz + 1];
    return (a < 0 || b < 0 || c < 0) ? -1 : a + sx * (b + ny * c);
  }
  // same, for a cell known to have no wall in its stencil
  __device__ __forceinline__ int in(int dx, int dy, int dz) const {
    return X[dx + 1] + sx * (Y[dy + 1] + ny * Z[dz + 1]);
  }
};

// Streamed (pre-collision) working values of a LIQUID cell: every stencil
// neighbour is liquid, interface or a wall/obstacle (closed interface layer).
// Shared by the stream-collide pass and the liquid->interface conversion so
// that both obtain bit-identical densities.
template <int Q, class ST>
__device__ __forceinline__ void pull_liquid(const typename ST::T* __restrict__ A, long long plane,
                                            const uint8_t* flags, const Nbr& nb, int c, bool near,
                                            typename ST::R* fin) {
  if (!near) {
#pragma unroll
    for (int i = 0; i < Q; ++i)
      fin[i] = ST::ldw(A + i * plane + nb.in(-dir_c(i, 0), -dir_c(i, 1), -dir_c(i, 2)));
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      int n = nb.at(-dir_c(i, 0), -dir_c(i, 1), -dir_c(i, 2));
      int t = type_at(flags, n);
      if (t == T_OBST) fin[i] = ST::ldw(A + opp(i) * plane + c); /* halfway bounce-back */
      else fin[i] = ST::ldw(A + i * plane + n);
    }
  }
}

// ------------------------------------------------------------ stream-collide
// Pass over all cells: liquid cells stream and collide here; interface cells
// are compacted (warp ballot) into l_if for k_stream_collide_if.
template <int Q, class ST>
__global__ void __launch_bounds__(128) k_stream_collide(Dev d, Geom g, Phys p) {
  using T = typename ST::T;
  using R = typename ST::R;
  constexpr bool SH = ST::kShift;
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int cur = ctrl->step & 1;  // pdf[step & 1] holds f*(t)
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  const T* __restrict__ A = (const T*)d.pdf[cur];
  T* __restrict__ B = (T*)d.pdf[cur ^ 1];
  const long long P = g.plane;
  const int c = x + g.sx * (y + g.ny * z);
  const uint8_t fl = (x < g.nx) ? d.flags[c] : (uint8_t)T_GAS;
  const int type = fl & F_TYPE;
  bool bad = false;
  if (type == T_LIQ) {
    Nbr nb;
    nb.setup(g, x, y, z);
    R fin[Q], fout[Q], rho;
    pull_liquid<Q, ST>(A, P, d.flags, nb, c, (fl & F_NEAR_OBST) != 0, fin);
    const R usq = collide<Q, SH, R>(fin, fout, p, rho);
    if (!(usq < (R)(1.0 / 3.0))) bad = true;
#pragma unroll
    for (int i = 0; i < Q; ++i) ST::stw(B + i * P + c, fout[i]);
  }
  warp_append(type == T_IF, c, &ctrl->n_if, d.l_if);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
    atomicCAS(&ctrl->unstable_step, -1, ctrl->step + 1);
}

// Interface cells (list-driven): free-surface boundary condition for PDFs
// arriving from gas, mass flux, collision, fill level and conversion marks.
template <int Q, class ST>
__global__ void __launch_bounds__(128) k_stream_collide_if(Dev d, Geom g, Phys p) {
  using T = typename ST::T;
  using R = typename ST::R;
  constexpr bool SH = ST::kShift;
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int cur = ctrl->step & 1;
  const T* __restrict__ A = (const T*)d.pdf[cur];
  T* __restrict__ B = (T*)d.pdf[cur ^ 1];
  const long long P = g.plane;
  const unsigned nif = ctrl->n_if;
  bool bad = false;
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < nif; k += gridDim.x * blockDim.x) {
    const int c = d.l_if[k];
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    const uint8_t fl = d.flags[c];
    Nbr nb;
    nb.setup(g, x, y, z);
    R fin[Q], own[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) own[i] = ST::ldw(A + i * P + c);
    // stored post-collision moments at t: u = sum c f* / rho - g / 2
    R rt, drt, jx, jy, jz;
    density<Q, SH, R>(own, rt, drt);
    momentum<Q, R>(own, jx, jy, jz);
    const R utx = jx / rt - (R)0.5 * (R)p.g[0];
    const R uty = jy / rt - (R)0.5 * (R)p.g[1];
    const R utz = jz / rt - (R)0.5 * (R)p.g[2];
    const R utsq = utx * utx + uty * uty + utz * utz;
    const double pg = (p.options & 8u) ? p.p_v - 2.0 * p.sigma * d.kappa[c]
                                       : p.p_v + p.sigma * d.kappa[c];
    const R rg = (R)(3.0 * pg);  // rho_G = p_G / c_s^2
    const R drg = (R)(3.0 * pg - 1.0);
    R feg[Q];
    feq_all<Q, SH, R>(feg, rg, drg, utx, uty, utz, utsq);
    int tn[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int n = nb.at(-dir_c(i, 0), -dir_c(i, 1), -dir_c(i, 2));
      const int t = type_at(d.flags, n);
      tn[i] = t;
      if (is_fluid(t)) fin[i] = ST::ldw(A + i * P + n);
      else if (t == T_OBST) fin[i] = own[opp(i)];             /* halfway bounce-back */
      else fin[i] = feg[i] + feg[opp(i)] - own[opp(i)];       /* anti-bounce-back from gas */
    }
    // Eq. nm-fslbm-mass-flux over i = 1..Q-1 (gas and walls carry none)
    const double phx = d.phi[c];
    const int clsx = fl & (F_NF | F_NE);
    const bool thurey = !(p.options & 1u);
    double dm = 0.0;
    bool dm_has = false;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int io = opp(i);
      const int t = tn[io];  // the neighbour x + c_i sent f_io
      if (t != T_LIQ && t != T_IF) continue;
      // f_in = f*_io(x + c_i) = fin[io], f_out = f*_i(x) = own[i]
      double dd;
      const double both = (double)(fin[io] - own[i]);
      if (t == T_LIQ) {
        dd = both;
      } else {
        const int n = nb.at(dir_c(i, 0), dir_c(i, 1), dir_c(i, 2));
        const int clsn = d.flags[n] & (F_NF | F_NE);
        const double f_in = SH ? (double)fin[io] + wgt<Q>(io) : (double)fin[io];
        const double f_out = SH ? (double)own[i] + wgt<Q>(i) : (double)own[i];
        double br;
        if (!thurey) br = both;
        else if (clsx == 0) br = (clsn == F_NF) ? f_in : (clsn == F_NE) ? -f_out : both;
        else if (clsx == F_NF) br = (clsn == F_NF) ? both : -f_out;
        else br = (clsn == F_NE) ? both : f_in;
        dd = 0.5 * (phx + d.phi[n]) * br;
      }
      dm = dm_has ? dm + dd : dd;
      dm_has = true;
    }
    const double m_new = dm_has ? d.mass[c] + dm : d.mass[c];
    R fout[Q], rho;
    const R usq = collide<Q, SH, R>(fin, fout, p, rho);
    if (!(usq < (R)(1.0 / 3.0))) bad = true;
#pragma unroll
    for (int i = 0; i < Q; ++i) ST::stw(B + i * P + c, fout[i]);
    const double rd = (double)rho;
    const double ph = m_new / rd;  // Eq. nm-fslbm-mass
    d.mass[c] = m_new;
    d.rho[c] = rd;
    d.phinew[c] = ph;
    if (ph > p.thr_hi) {
      d.flags[c] = fl | F_TO_LIQ;
      d.l_fill[atomicAdd(&ctrl->n_fill, 1u)] = c;
    } else if (ph < p.thr_lo) {
      d.flags[c] = fl | F_TO_GAS;
      d.l_empty[atomicAdd(&ctrl->n_empty, 1u)] = c;
    }
  }
  if (bad) atomicCAS(&ctrl->unstable_step, -1, ctrl->step + 1);
}

// ------------------------------------------------------------ conversion
#define FSL_GRID_LOOP(k, n) \
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < (n); k += gridDim.x * blockDim.x)

template <int Q>
__global__ void __launch_bounds__(256) k_fill(Dev d, Geom g) {
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const unsigned nif = ctrl->n_if, nfill = ctrl->n_fill;
  FSL_GRID_LOOP(k, nif + nfill) {
    if (k < nif) {
      const int c = d.l_if[k];
      d.phi[c] = d.phinew[c];
      continue;
    }
    const int c = d.l_fill[k - nif];
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    for (int i = 1; i < Q; ++i) {
      const int n = nb_at(g, x, y, z, rc(i, 0), rc(i, 1), rc(i, 2));
      if (n < 0) continue;
      if ((d.flags[n] & F_TYPE) == T_GAS) {
        uint8_t old = byte_or(d.flags, n, (uint8_t)(F_NEW | T_IF));
        if (!(old & F_NEW)) {
          d.phi[n] = 0.0;
          d.mass[n] = 0.0;
          unsigned slot = atomicAdd(&ctrl->n_new, 1u);
          d.l_new[slot] = n;
        }
      }
      if (d.flags[n] & F_TO_GAS) byte_and(d.flags, n, F_TO_GAS);
    }
  }
}

template <int Q, class ST>
__global__ void __launch_bounds__(256) k_empty(Dev d, Geom g) {
  using R = typename ST::R;
  constexpr bool SH = ST::kShift;
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int cur = ctrl->step & 1;
  const typename ST::T* A = (const typename ST::T*)d.pdf[cur];
  const unsigned ne = ctrl->n_empty;
  FSL_GRID_LOOP(k, ne) {
    const int c = d.l_empty[k];
    if (!(d.flags[c] & F_TO_GAS)) continue;
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    for (int i = 1; i < Q; ++i) {
      const int n = nb_at(g, x, y, z, rc(i, 0), rc(i, 1), rc(i, 2));
      if (n < 0) continue;
      if ((d.flags[n] & F_TYPE) != T_LIQ) continue;
      if (!byte_retype(d.flags, n, T_LIQ, T_IF, &ctrl->timeout)) continue;
      // the liquid cell's density of this step, recomputed exactly as the
      // stream-collide pass obtained it
      int nx_, ny_, nz_;
      cell_xyz(g, n, nx_, ny_, nz_);
      Nbr nb;
      nb.setup(g, nx_, ny_, nz_);
      R fin[Q], rho, drho;
      pull_liquid<Q, ST>(A, g.plane, d.flags, nb, n, (d.flags[n] & F_NEAR_OBST) != 0, fin);
      density<Q, SH, R>(fin, rho, drho);
      d.rho[n] = (double)rho;
      d.mass[n] = (double)rho;
      d.phi[n] = 1.0;
      unsigned slot = atomicAdd(&ctrl->n_l2i, 1u);
      d.l_l2i[slot] = n;
    }
  }
}

static __global__ void __launch_bounds__(256) k_finalise(Dev d) {
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const unsigned nf = ctrl->n_fill, ne = ctrl->n_empty;
  FSL_GRID_LOOP(k, nf + ne) {
    const bool fill = k < nf;
    const int c = fill ? d.l_fill[k] : d.l_empty[k - nf];
    const uint8_t fl = d.flags[c];
    if (fill) {
      d.mex[c] = (d.phi[c] - 1.0) * d.rho[c];
      d.flags[c] = (uint8_t)((fl & ~F_TYPE) | T_LIQ);
      d.phi[c] = 1.0;
      d.mass[c] = d.rho[c];
    } else if (fl & F_TO_GAS) {
      d.mex[c] = d.phi[c] * d.rho[c];
      d.flags[c] = (uint8_t)((fl & ~F_TYPE) | T_GAS);
      d.phi[c] = 0.0;
      d.mass[c] = 0.0;
      atomicAdd(&ctrl->pad[0], 1u);
    }
  }
}

// ------------------------------------------------------------ normals
// Parker-Youngs gradient of phi at cell (x, y, z): per axis a, the centred
// difference across the 3x3 block perpendicular to a with weights 4 (centre),
// 2 (edges), 1 (corners), divided by 32; exact for linear phi.  An axis whose
// block touches a wall or obstacle uses a two-point difference over the
// non-obstacle cells instead (narrowed stencil near obstacles).
__device__ inline void normal_py(const Geom& g, const uint8_t* flags, const double* phi, int x,
                                 int y, int z, double* n) {
  const int p[3] = {x, y, z};
  const int c = x + g.sx * (y + g.ny * z);
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3, cc = (a + 2) % 3;
    if (b > cc) { int t = b; b = cc; cc = t; }
    bool touches = false;
    for (int ob = -1; ob <= 1 && !touches; ++ob)
      for (int oc = -1; oc <= 1 && !touches; ++oc) {
        int dp[3] = {0, 0, 0}, dm[3] = {0, 0, 0};
        dp[a] = 1; dm[a] = -1;
        dp[b] += ob; dm[b] += ob;
        dp[cc] += oc; dm[cc] += oc;
        int yp = nb_at(g, p[0], p[1], p[2], dp[0], dp[1], dp[2]);
        int ym = nb_at(g, p[0], p[1], p[2], dm[0], dm[1], dm[2]);
        if (type_at(flags, yp) == T_OBST || type_at(flags, ym) == T_OBST) touches = true;
      }
    if (!touches) {
      double sum = 0.0;
      for (int ob = -1; ob <= 1; ++ob)
        for (int oc = -1; oc <= 1; ++oc) {
          int dp[3] = {0, 0, 0}, dm[3] = {0, 0, 0};
          dp[a] = 1; dm[a] = -1;
          dp[b] += ob; dm[b] += ob;
          dp[cc] += oc; dm[cc] += oc;
          int yp = nb_at(g, p[0], p[1], p[2], dp[0], dp[1], dp[2]);
          int ym = nb_at(g, p[0], p[1], p[2], dm[0], dm[1], dm[2]);
          double w = (ob == 0 ? 2.0 : 1.0) * (oc == 0 ? 2.0 : 1.0);
          sum += w * (phi[yp] - phi[ym]);
        }
      n[a] = sum / 32.0;
    } else {
      int dp[3] = {0, 0, 0}, dm[3] = {0, 0, 0};
      dp[a] = 1; dm[a] = -1;
      int yp = nb_at(g, p[0], p[1], p[2], dp[0], dp[1], dp[2]);
      int ym = nb_at(g, p[0], p[1], p[2], dm[0], dm[1], dm[2]);
      bool okp = type_at(flags, yp) != T_OBST, okm = type_at(flags, ym) != T_OBST;
      if (okp && okm) n[a] = 0.5 * (phi[yp] - phi[ym]);
      else if (okp) n[a] = phi[yp] - phi[c];
      else if (okm) n[a] = phi[c] - phi[ym];
      else n[a] = 0.0;
    }
  }
}

__device__ inline void unit_normal(const Geom& g, const uint8_t* flags, const double* phi, int x,
                                   int y, int z, double* nh) {
  double n[3];
  normal_py(g, flags, phi, x, y, z, n);
  double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  if (len < 1e-12) {
    nh[0] = nh[1] = nh[2] = 0.0;
  } else {
    nh[0] = n[0] / len;
    nh[1] = n[1] / len;
    nh[2] = n[2] / len;
  }
}

// K = -div(n_hat), central differences over the face neighbours; a wall side
// is replaced by the centre value.
__device__ inline double curvature(const Geom& g, const uint8_t* flags, const double* phi, int x,
                                   int y, int z) {
  double nc[3];
  unit_normal(g, flags, phi, x, y, z, nc);
  double div = 0.0;
  for (int a = 0; a < 3; ++a) {
    int dp[3] = {0, 0, 0}, dm[3] = {0, 0, 0};
    dp[a] = 1; dm[a] = -1;
    int yp = nb_at(g, x, y, z, dp[0], dp[1], dp[2]);
    int ym = nb_at(g, x, y, z, dm[0], dm[1], dm[2]);
    bool okp = type_at(flags, yp) != T_OBST, okm = type_at(flags, ym) != T_OBST;
    double np[3], nm[3], dd;
    if (okp && okm) {
      int px, py, pz, mx, my, mz;
      cell_xyz(g, yp, px, py, pz);
      cell_xyz(g, ym, mx, my, mz);
      unit_normal(g, flags, phi, px, py, pz, np);
      unit_normal(g, flags, phi, mx, my, mz, nm);
      dd = 0.5 * (np[a] - nm[a]);
    } else if (okp) {
      int px, py, pz;
      cell_xyz(g, yp, px, py, pz);
      unit_normal(g, flags, phi, px, py, pz, np);
      dd = np[a] - nc[a];
    } else if (okm) {
      int mx, my, mz;
      cell_xyz(g, ym, mx, my, mz);
      unit_normal(g, flags, phi, mx, my, mz, nm);
      dd = nc[a] - nm[a];
    } else {
      dd = 0.0;
    }
    div += dd;
  }
  return -div;
}

// ------------------------------------------------------------ refilling
// plain FP64 equilibrium for a runtime direction (list kernels, initial state)
template <int Q>
__device__ inline double feq_d(int i, double rho, double ux, double uy, double uz) {
  const double cu = (double)rc(i, 0) * ux + (double)rc(i, 1) * uy + (double)rc(i, 2) * uz;
  const double usq = ux * ux + uy * uy + uz * uz;
  return rw<Q>(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
}

// stored moments of cell n from full PDFs (double): rho = sum f*,
// u = sum c f* / rho - g / 2
template <int Q, class ST>
__device__ inline void stored_moments(const typename ST::T* B, long long plane, int n,
                                      const Phys& p, double& rho, double* u) {
  double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
  double f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = ST::ldf(B + i * plane + n, wgt<Q>(i));
#pragma unroll
  for (int i = 0; i < Q; ++i) r = (i == 0) ? f[0] : r + f[i];
  momentum<Q, double>(f, jx, jy, jz);
  rho = r;
  u[0] = jx / r - 0.5 * p.g[0];
  u[1] = jy / r - 0.5 * p.g[1];
  u[2] = jz / r - 0.5 * p.g[2];
}

__device__ __forceinline__ bool valid_src(const uint8_t* flags, int n) {
  if (n < 0) return false;
  const uint8_t f = flags[n];
  return is_fluid(f & F_TYPE) && !(f & F_NEW);
}

template <int Q, class ST>
__global__ void __launch_bounds__(128) k_refill(Dev d, Geom g, Phys p) {
  using T = typename ST::T;
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int cur = ctrl->step & 1;
  T* B = (T*)d.pdf[cur ^ 1];
  const long long P = g.plane;
  const unsigned nn = ctrl->n_new;
  FSL_GRID_LOOP(k, nn) {
    const int c = d.l_new[k];
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    bool valid[Q];
    int nbr[Q];
    double nrho[Q], nux[Q], nuy[Q], nuz[Q];
    int count = 0;
    double rsum = 0.0, usx = 0.0, usy = 0.0, usz = 0.0;
    valid[0] = false;
    nbr[0] = c;
    for (int i = 1; i < Q; ++i) {
      const int n = nb_at(g, x, y, z, rc(i, 0), rc(i, 1), rc(i, 2));
      nbr[i] = n;
      valid[i] = valid_src(d.flags, n);
      if (valid[i]) {
        double u[3];
        stored_moments<Q, ST>(B, P, n, p, nrho[i], u);
        nux[i] = u[0]; nuy[i] = u[1]; nuz[i] = u[2];
        rsum += nrho[i];
        usx += nux[i]; usy += nuy[i]; usz += nuz[i];
        count += 1;
      }
    }
    double out[Q];
    const double cnt = (double)(count > 0 ? count : 1);
    const double rb = rsum / cnt, ubx = usx / cnt, uby = usy / cnt, ubz = usz / cnt;
    const int scheme = p.refill;
    int dn = -1;
    if (scheme == 1 || scheme == 3) {
      double n3[3];
      normal_py(g, d.flags, d.phi, x, y, z, n3);
      double best = 0.0;
      for (int i = 1; i < Q; ++i) {
        if (!valid[i]) continue;
        const double dot = (double)rc(i, 0) * n3[0] + (double)rc(i, 1) * n3[1] +
                           (double)rc(i, 2) * n3[2];
        if (dn < 0 || dot > best) { dn = i; best = dot; }
      }
    }
    if (count == 0 || ((scheme == 1 || scheme == 3) && dn < 0)) {
      // unreachable for cells created by a filling neighbour; latch the event
      atomicOr(&ctrl->timeout, 2u);
      for (int i = 0; i < Q; ++i) out[i] = rw<Q>(i);
    } else if (scheme == 0) {  // EQ
      for (int i = 0; i < Q; ++i) out[i] = feq_d<Q>(i, rb, ubx, uby, ubz);
    } else if (scheme == 1) {  // EQ+NEQ
      const int yn = nbr[dn];
      for (int i = 0; i < Q; ++i) {
        const double fe = feq_d<Q>(i, rb, ubx, uby, ubz);
        const double fy = ST::ldf(B + i * P + yn, rw<Q>(i));
        double fneq;
        if (p.options & 4u) fneq = fy - fe;
        else fneq = fy - feq_d<Q>(i, nrho[dn], nux[dn], nuy[dn], nuz[dn]);
        out[i] = fe + fneq;
      }
    } else if (scheme == 2) {  // GEQ
      double du[3][3];
      const double ub[3] = {ubx, uby, ubz};
      for (int b = 0; b < 3; ++b) {
        const int dp = 1 + 2 * b, dm = 2 + 2 * b;
        for (int a = 0; a < 3; ++a) {
          const double up = a == 0 ? nux[dp] : a == 1 ? nuy[dp] : nuz[dp];
          const double um = a == 0 ? nux[dm] : a == 1 ? nuy[dm] : nuz[dm];
          if (valid[dp] && valid[dm]) du[a][b] = 0.5 * (up - um);
          else if (valid[dp]) du[a][b] = up - ub[a];
          else if (valid[dm]) du[a][b] = ub[a] - um;
          else du[a][b] = 0.0;
        }
      }
      const double coef = p.geq_coef;
      for (int i = 0; i < Q; ++i) {
        const int cc[3] = {rc(i, 0), rc(i, 1), rc(i, 2)};
        double sum = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            const double S = du[a][b] + du[b][a];
            const double Qab = (a == b ? 1.0 / 3.0 : 0.0) - (double)(cc[a] * cc[b]);
            sum += S * Qab;
          }
        out[i] = feq_d<Q>(i, rb, ubx, uby, ubz) + rw<Q>(i) * rb * coef * sum;
      }
    } else if (scheme == 3) {  // EXT
      const int cx = rc(dn, 0), cy = rc(dn, 1), cz = rc(dn, 2);
      const int y1 = nbr[dn];
      const int y2 = nb_at(g, x, y, z, 2 * cx, 2 * cy, 2 * cz);
      const int y3 = nb_at(g, x, y, z, 3 * cx, 3 * cy, 3 * cz);
      int kk = 1;
      const bool v2 = valid_src(d.flags, y2), v3 = valid_src(d.flags, y3);
      if (v2) kk = v3 ? 3 : 2;
      for (int i = 0; i < Q; ++i) {
        const double w = rw<Q>(i);
        const double f1 = ST::ldf(B + i * P + y1, w);
        if (kk == 3) {
          const double f2 = ST::ldf(B + i * P + y2, w), f3 = ST::ldf(B + i * P + y3, w);
          out[i] = 3.0 * f1 - 3.0 * f2 + f3;
        } else if (kk == 2) {
          const double f2 = ST::ldf(B + i * P + y2, w);
          out[i] = 2.0 * f1 - f2;
        } else {
          out[i] = f1;
        }
      }
    } else {  // AVG
      for (int i = 0; i < Q; ++i) {
        double sum = 0.0;
        for (int j = 1; j < Q; ++j)
          if (valid[j]) sum += ST::ldf(B + i * P + nbr[j], rw<Q>(i));
        out[i] = sum / cnt;
      }
    }
    double r = 0.0;
    for (int i = 0; i < Q; ++i) {
      ST::stf(B + i * P + c, out[i], rw<Q>(i));
      r = (i == 0) ? out[0] : r + out[i];
    }
    d.rho[c] = r;
  }
}

// ------------------------------------------------------------ excess mass
template <int Q>
__global__ void __launch_bounds__(256) k_excess_share(Dev d, Geom g) {
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const unsigned nf = ctrl->n_fill, ne = ctrl->n_empty;
  FSL_GRID_LOOP(k, nf + ne) {
    const bool fill = k < nf;
    const int c = fill ? d.l_fill[k] : d.l_empty[k - nf];
    if (!fill && !(d.flags[c] & F_TO_GAS)) continue;
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    int nr = 0;
    for (int i = 1; i < Q; ++i) {
      const int n = nb_at(g, x, y, z, rc(i, 0), rc(i, 1), rc(i, 2));
      if (type_at(d.flags, n) != T_IF) continue;
      nr++;
      if (byte_or(d.claim, n, 1) == 0) {
        unsigned slot = atomicAdd(&ctrl->n_recv, 1u);
        d.l_recv[slot] = n;
      }
    }
    const double mex = d.mex[c];
    if (nr == 0) {
      d.lost[c] += mex;
      d.mex[c] = 0.0;
    } else {
      d.mex[c] = mex / (double)nr;
    }
  }
}

template <int Q>
__global__ void __launch_bounds__(256) k_excess_gather(Dev d, Geom g) {
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const unsigned nr = ctrl->n_recv;
  FSL_GRID_LOOP(k, nr) {
    const int r = d.l_recv[k];
    int x, y, z;
    cell_xyz(g, r, x, y, z);
    double sum = 0.0;
    for (int i = 1; i < Q; ++i) {
      const int n = nb_at(g, x, y, z, rc(i, 0), rc(i, 1), rc(i, 2));
      if (n >= 0 && (d.flags[n] & (F_TO_LIQ | F_TO_GAS))) sum += d.mex[n];
    }
    d.mass[r] = d.mass[r] + sum;
    d.phi[r] = d.mass[r] / d.rho[r];
  }
}

// ------------------------------------------------------------ classes / curvature
// Thuerey class of an interface cell from its stencil neighbours.
template <int Q>
__device__ inline uint8_t iface_class(const Geom& g, const uint8_t* flags, int x, int y, int z) {
  bool has_liq = false, has_gas = false;
  for (int i = 1; i < Q; ++i) {
    const int t = type_at(flags, nb_at(g, x, y, z, rc(i, 0), rc(i, 1), rc(i, 2)));
    if (t == T_LIQ) has_liq = true;
    if (t == T_GAS) has_gas = true;
  }
  if (!has_liq && has_gas) return F_NF;
  if (!has_gas && has_liq) return F_NE;
  return 0;
}

template <int Q>
__global__ void __launch_bounds__(128) k_classify(Dev d, Geom g, Phys p) {
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const unsigned a = ctrl->n_if, b = ctrl->n_new, e = ctrl->n_l2i;
  FSL_GRID_LOOP(k, a + b + e) {
    const int c = k < a ? d.l_if[k] : (k < a + b ? d.l_new[k - a] : d.l_l2i[k - a - b]);
    const uint8_t fl = d.flags[c];
    uint8_t nf = (uint8_t)(fl & ~(F_TO_LIQ | F_TO_GAS | F_NEW | F_NF | F_NE));
    d.claim[c] = 0;
    if ((fl & F_TYPE) == T_IF) {
      int x, y, z;
      cell_xyz(g, c, x, y, z);
      nf |= iface_class<Q>(g, d.flags, x, y, z);
      d.kappa[c] = (p.sigma != 0.0) ? curvature(g, d.flags, d.phi, x, y, z) : 0.0;
    }
    d.flags[c] = nf;
  }
}

// Deterministic block reduction helpers (fixed tree order).
template <int NT>
__device__ inline double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}
template <int NT>
__device__ inline int block_max(int v, int* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = max(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  int r = sh[0];
  __syncthreads();
  return r;
}

// End of step: optional trace record, counters for the next step, step++.
static __global__ void __launch_bounds__(256) k_end_step(Dev d, Geom g) {
  __shared__ double shd[256];
  __shared__ int shi[256];
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int every = ctrl->trace_every;
  if (every > 0 && ((ctrl->step + 1) % every) == 0) {
    // column height at i = 0: sum_j,k phi / nz
    double s = 0.0;
    const int ncol = g.ny * g.nz;
    for (int k = threadIdx.x; k < ncol; k += 256) s += d.phi[g.sx * k];
    const double col = block_sum<256>(s, shd) / (double)g.nz;
    // front: 1 + max i of an interface cell with j = 0
    int best = -1;
    for (int k = threadIdx.x; k < g.nx * g.nz; k += 256) {
      const int i = k % g.nx, kz = k / g.nx;
      if ((d.flags[i + g.sx * (g.ny * kz)] & F_TYPE) == T_IF) best = max(best, i);
    }
    const int front = block_max<256>(best, shi) + 1;
    best = -1;
    for (int k = threadIdx.x; k < ncol; k += 256) {
      const int j = k % g.ny;
      if ((d.flags[g.sx * k] & F_TYPE) == T_IF) best = max(best, j);
    }
    const int height = block_max<256>(best, shi) + 1;
    if (threadIdx.x == 0) {
      const int slot = ctrl->trace_count % kTraceCapacity;
      d.trace[3 * slot + 0] = col;
      d.trace[3 * slot + 1] = (double)front;
      d.trace[3 * slot + 2] = (double)height;
      ctrl->trace_count += 1;
    }
  }
  if (threadIdx.x == 0) {
    ctrl->last[0] = ctrl->n_fill;
    ctrl->last[1] = ctrl->pad[0];
    ctrl->last[2] = ctrl->n_new;
    ctrl->last[3] = ctrl->n_if;
    ctrl->n_if = ctrl->n_fill = ctrl->n_empty = 0;
    ctrl->n_new = ctrl->n_l2i = ctrl->n_recv = 0;
    ctrl->pad[0] = 0;
    ctrl->step += 1;
  }
}

// ------------------------------------------------------------ initialisation
static __global__ void k_ctrl_reset(Ctrl* ctrl, int trace_every) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    Ctrl z = {};
    z.unstable_step = -1;
    z.trace_every = trace_every;
    *ctrl = z;
  }
}

// types from the staged fill level / obstacle mask (unpadded staging arrays)
static __global__ void k_init_types(Dev d, Geom g, const double* phi0, const uint8_t* obst, int have_obst) {
  const long long total = g.cells;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % g.sx);
    const long long r = c / g.sx;
    uint8_t t = T_GAS;
    double ph = 0.0;
    if (x < g.nx) {
      const long long u = x + (long long)g.nx * r;
      const double v = phi0[u];
      if (have_obst && obst[u]) { t = T_OBST; ph = 0.0; }
      else if (v >= 1.0) { t = T_LIQ; ph = 1.0; }
      else if (v <= 0.0) { t = T_GAS; ph = 0.0; }
      else { t = T_IF; ph = v; }
    }
    d.flags[c] = t;
    d.phi[c] = ph;
  }
}

// closed interface layer: a liquid cell with a gas stencil neighbour becomes interface
template <int Q>
__global__ void k_init_close(Dev d, Geom g) {
  const long long total = g.cells;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(g, (int)c, x, y, z);
    if (x >= g.nx || (d.flags[c] & F_TYPE) != T_LIQ) continue;
    bool gas = false;
    for (int i = 1; i < Q; ++i)
      if (type_at(d.flags, nb_at(g, x, y, z, rc(i, 0), rc(i, 1), rc(i, 2))) == T_GAS)
        gas = true;
    if (gas) d.flags[c] = T_IF;  // fill level stays 1
  }
}

template <int Q, class ST>
__global__ void k_init_state(Dev d, Geom g, Phys p, int cur, const double* u0, double h_ref) {
  using T = typename ST::T;
  T* A = (T*)d.pdf[cur];
  const long long total = g.cells;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(g, (int)c, x, y, z);
    d.claim[c] = 0;
    d.mex[c] = 0.0;
    d.lost[c] = 0.0;
    d.kappa[c] = 0.0;
    d.phinew[c] = 0.0;
    if (x >= g.nx) { d.mass[c] = 0.0; d.rho[c] = 0.0; continue; }
    uint8_t fl = d.flags[c];
    bool near = false;
    for (int i = 1; i < Q; ++i)
      if (type_at(d.flags, nb_at(g, x, y, z, rc(i, 0), rc(i, 1), rc(i, 2))) == T_OBST)
        near = true;
    if (near) d.flags[c] = (uint8_t)(fl | F_NEAR_OBST);
    const int t = fl & F_TYPE;
    double r = 1.0;
    if (p.gaxis >= 0 && !isnan(h_ref)) {
      const int pa = p.gaxis == 0 ? x : p.gaxis == 1 ? y : z;
      r = 1.0 + 3.0 * p.g[p.gaxis] * (((double)pa + 0.5) - h_ref);
    }
    double ux = 0.0, uy = 0.0, uz = 0.0;
    if (u0) {
      const long long u = x + (long long)g.nx * (y + (long long)g.ny * z);
      ux = u0[3 * u]; uy = u0[3 * u + 1]; uz = u0[3 * u + 2];
    }
    if (is_fluid(t)) {
      for (int i = 0; i < Q; ++i) ST::stf(A + i * g.plane + c, feq_d<Q>(i, r, ux, uy, uz), rw<Q>(i));
      d.rho[c] = r;
      d.mass[c] = (t == T_LIQ) ? r : d.phi[c] * r;
    } else {
      d.rho[c] = 0.0;
      d.mass[c] = 0.0;
    }
  }
}

template <int Q>
__global__ void k_init_classes(Dev d, Geom g, Phys p) {
  const long long total = g.cells;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(g, (int)c, x, y, z);
    if (x >= g.nx) continue;
    const uint8_t fl = d.flags[c];
    if ((fl & F_TYPE) != T_IF) continue;
    d.flags[c] = (uint8_t)((fl & ~(F_NF | F_NE)) | iface_class<Q>(g, d.flags, x, y, z));
    d.kappa[c] = (p.sigma != 0.0) ? curvature(g, d.flags, d.phi, x, y, z) : 0.0;
  }
}

// ------------------------------------------------------------ observation
// total mass partial sums: liquid zeroth moment, interface m, lost mass
template <int Q, class ST>
__global__ void __launch_bounds__(256) k_mass_partial(Dev d, Geom g, int cur, double* part) {
  __shared__ double sh[256];
  const typename ST::T* A = (const typename ST::T*)d.pdf[cur];
  double s = 0.0;
  const long long total = g.cells;
  for (long long c = blockIdx.x * 256ll + threadIdx.x; c < total; c += (long long)gridDim.x * 256) {
    const int x = (int)(c % g.sx);
    if (x >= g.nx) continue;
    const int t = d.flags[c] & F_TYPE;
    double v = d.lost[c];
    if (t == T_LIQ) {
      double r = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double f = ST::ldf(A + i * g.plane + c, wgt<Q>(i));
        r = (i == 0) ? f : r + f;
      }
      v += r;
    } else if (t == T_IF) {
      v += d.mass[c];
    }
    s += v;
  }
  const double b = block_sum<256>(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

static __global__ void __launch_bounds__(256) k_sum_partials(const double* part, int n, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) s += part[k];
  const double b = block_sum<256>(s, sh);
  if (threadIdx.x == 0) *out = b;
}

template <int Q, class ST>
__global__ void __launch_bounds__(256) k_umax_partial(Dev d, Geom g, Phys p, int cur, double* part) {
  __shared__ double sh[256];
  const typename ST::T* A = (const typename ST::T*)d.pdf[cur];
  double best = 0.0;
  const long long total = g.cells;
  for (long long c = blockIdx.x * 256ll + threadIdx.x; c < total; c += (long long)gridDim.x * 256) {
    const int x = (int)(c % g.sx);
    if (x >= g.nx || !is_fluid(d.flags[c] & F_TYPE)) continue;
    double r, u[3];
    stored_moments<Q, ST>(A, g.plane, (int)c, p, r, u);
    best = fmax(best, sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  }
  sh[threadIdx.x] = best;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

static __global__ void __launch_bounds__(256) k_max_partials(const double* part, int n, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) s = fmax(s, part[k]);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int t = 128; t > 0; t >>= 1) {
    if ((int)threadIdx.x < t) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + t]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// decode one PDF plane into an unpadded double array
template <int Q, class ST>
__global__ void k_export_plane(Dev d, Geom g, int cur, int i, double* dst) {
  const typename ST::T* A = (const typename ST::T*)d.pdf[cur];
  const long long n = (long long)g.nx * g.ny * g.nz;
  const double w = rw<Q>(i);
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < n;
       u += (long long)gridDim.x * blockDim.x) {
    const long long x = u % g.nx, r = u / g.nx;
    dst[u] = ST::ldf(A + i * g.plane + x + g.sx * r, w);
  }
}

// ------------------------------------------------------------ launch table
template <int Q, class ST>
struct Kernels {
  // the buffer parity is read on the device from the step counter, so the
  // launch sequence is the same for every step (and graph-capturable)
  static cudaError_t step(const Dev& d, const Geom& g, const Phys& p, cudaStream_t s) {
    dim3 b1(128), g1((g.nx + 127) / 128, g.ny, g.nz);
    k_stream_collide<Q, ST><<<g1, b1, 0, s>>>(d, g, p);
    k_stream_collide_if<Q, ST><<<kListBlocks, 128, 0, s>>>(d, g, p);
    k_fill<Q><<<kListBlocks, 256, 0, s>>>(d, g);
    k_empty<Q, ST><<<kListBlocks, 256, 0, s>>>(d, g);
    k_finalise<<<kListBlocks, 256, 0, s>>>(d);
    k_refill<Q, ST><<<kListBlocks, 128, 0, s>>>(d, g, p);
    k_excess_share<Q><<<kListBlocks, 256, 0, s>>>(d, g);
    k_excess_gather<Q><<<kListBlocks, 256, 0, s>>>(d, g);
    k_classify<Q><<<kListBlocks, 128, 0, s>>>(d, g, p);
    k_end_step<<<1, 256, 0, s>>>(d, g);
    return cudaGetLastError();
  }
  static cudaError_t init(const Dev& d, const Geom& g, const Phys& p, int cur, const double* u0,
                          int have_obst, double h_ref, cudaStream_t s) {
    const int blocks = 4 * 152;
    k_ctrl_reset<<<1, 32, 0, s>>>(d.ctrl, 0);
    k_init_types<<<blocks, 256, 0, s>>>(d, g, d.phinew, d.claim, have_obst);
    k_init_close<Q><<<blocks, 256, 0, s>>>(d, g);
    k_init_state<Q, ST><<<blocks, 256, 0, s>>>(d, g, p, cur, u0, h_ref);
    k_init_classes<Q><<<blocks, 128, 0, s>>>(d, g, p);
    return cudaGetLastError();
  }
  static cudaError_t total_mass(const Dev& d, const Geom& g, const Phys&, int cur, double* out,
                                cudaStream_t s) {
    k_mass_partial<Q, ST><<<kReduceBlocks, 256, 0, s>>>(d, g, cur, d.red);
    k_sum_partials<<<1, 256, 0, s>>>(d.red, kReduceBlocks, out);
    return cudaGetLastError();
  }
  static cudaError_t max_velocity(const Dev& d, const Geom& g, const Phys& p, int cur, double* out,
                                  cudaStream_t s) {
    k_umax_partial<Q, ST><<<kReduceBlocks, 256, 0, s>>>(d, g, p, cur, d.red);
    k_max_partials<<<1, 256, 0, s>>>(d.red, kReduceBlocks, out);
    return cudaGetLastError();
  }
  static cudaError_t export_pdf(const Dev& d, const Geom& g, const Phys&, int cur, int i,
                                double* dst, cudaStream_t s) {
    k_export_plane<Q, ST><<<4 * 152, 256, 0, s>>>(d, g, cur, i, dst);
    return cudaGetLastError();
  }
  static const Launch* table() {
    static const Launch L = {&step, &init, &total_mass, &max_velocity, &export_pdf, 11};
    return &L;
  }
};

}  // namespace fsl
