// FSLBM step kernels, templated on the lattice (Q = 19 | 27) and the PDF
// storage (SF64 | SF32 | SF16 | SBF16).  Each precision family instantiates
// them in its own translation unit (k_<storage>_q<Q>.cu).  Every unit is
// compiled with -fmad=false: the FP64 arithmetic is then bit-reproducible
// against a plain FP64 evaluation in the operation order written here, and a
// body inlined into both the single-domain and the batched kernel gives the
// same bits in each.
//
// One step (Sec. 2 and 3 of the paper), t -> t+1:
//   k_stream_collide  (bulk variants) pull streaming (Eq. nm-lbm-streaming),
//                     halfway bounce-back, moments (Eqs. nm-lbm-density,
//                     nm-lbm-velocity), SRT/TRT collision with Guo forcing
//                     (Eqs. nm-lbm-collision, nm-lbm-force-guo) of the liquid
//                     cells; concurrently, on a second stream,
//   k_stream_collide_if  the interface cells of the list built by the previous
//                     step: free-surface anti-bounce-back for PDFs from gas
//                     (Eq. nm-fslbm-boundary-condition), interface mass flux
//                     (Eq. nm-fslbm-mass-flux, Thuerey classes), collision,
//                     fill level m/rho (Eq. nm-fslbm-mass), conversion marks
//                     (threshold eps_phi) and warp-ballot compaction of the
//                     to-liquid and to-gas cells;
//   k_convert         one cooperative launch of five phases separated by
//                     grid-wide barriers (the batched path launches them one
//                     by one):
//     fill            commit fill levels; gas neighbours of filled cells become
//                     new interface cells; to-gas neighbours are kept (filling
//                     wins a conflict);
//     empty           liquid neighbours of emptied cells become interface;
//     finalise/share  type change, excess mass (Eq. nm-fslbm-excess-mass) and
//                     its share per receiver, receiver compaction;
//     refill          EQ, EQ+NEQ, GEQ, EXT, AVG refilling (Sec. 3.1);
//     excess gather   receivers gather their shares in direction order;
//   k_classify        Thuerey classes and curvature K = -div(n_hat) for the
//                     next step, clean-up of the per-step marks, and the next
//                     step's interface list (two lists, by step parity);
//   k_end_step        trace record, counters, step counter.
#pragma once
#include "fsl_lattice.cuh"

namespace fsl {

// A physical parameter in the arithmetic type R: the FP64 value for the FP64
// path, the copy rounded once on the host otherwise.
#define PAR(R, p, name) (sizeof(R) == 8 ? (R)(p).name : (R)(p).f.name)

// Fill level of cell c written together with its FP32 copy (16/32-bit path),
// so that the kernels that read many fill levels per cell in FP32 (interface
// pass, normals, curvature) load 4-byte values and convert none of them.
__device__ __forceinline__ void put_phi(const Dev& d, long long c, double v) {
  d.phi[c] = v;
  if (d.phif) d.phif[c] = (float)v;
}
// the fill levels in the working precision R: the FP32 copy for R = float
template <class R>
__device__ __forceinline__ const R* phi_work(const Dev& d) {
  if constexpr (sizeof(R) == 4) return d.phif;
  else return d.phi;
}

// The member of a batched launch that this block serves (blockIdx.y), copied
// into local values so that the body's stores cannot alias them.
#define FSL_MEMBER(t)                          \
  const Member& mb_ = *(t).m[blockIdx.y];      \
  const Dev d = mb_.d;                         \
  const Geom g = mb_.g;                        \
  const Phys p = mb_.p;                        \
  (void)d;                                     \
  (void)g;                                     \
  (void)p

#define FSL_GRID_LOOP(k, n) \
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < (n); k += gridDim.x * blockDim.x)
// Warp-synchronous grid loop: all lanes of a warp run the same iterations
// (k_ok says whether the lane's index is in range), so warp ballots may be
// used inside to aggregate list appends.
#define FSL_WARP_LOOP(k, k_ok, n)                                                             \
  for (unsigned k##_base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; k##_base < (n);   \
       k##_base += gridDim.x * blockDim.x)                                                    \
    for (unsigned k = k##_base + (threadIdx.x & 31u), k##_once = 1; k##_once; k##_once = 0)  \
      for (bool k_ok = k < (n), k##_o2 = true; k##_o2; k##_o2 = false)

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
//   exact:   rho = f_0 + f_1 + ... + f_{Q-1}, left to right;
//   shifted: drho = d_0 + (d_1 + d_2) + (d_3 + d_4) + ..., opposite pairs first
//            (the order the pairwise collision of the 16/32-bit path uses).
template <int Q, bool SHIFT, class R>
__device__ __forceinline__ void density(const R* f, R& rho, R& drho) {
  R s = f[0];
  if (SHIFT) {
#pragma unroll
    for (int i = 1; i < Q; i += 2) s = s + (f[i] + f[i + 1]);
    drho = s;
    rho = (R)1 + s;
  } else {
#pragma unroll
    for (int i = 1; i < Q; ++i) s = s + f[i];
    rho = s;
    drho = s - (R)1;
  }
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
// The same equilibrium for a direction given as an (unrolled-loop) value:
// identical operations, so identical results.
template <int Q, bool SHIFT, class R>
__device__ __forceinline__ R feq_c(int i, R rho, R drho, R ux, R uy, R uz, R usq) {
  const R w = (R)wgt<Q>(i);
  R cu = dot3r<R>(dir_c(i, 0), dir_c(i, 1), dir_c(i, 2), ux, uy, uz);
  if (!SHIFT) return w * rho * ((R)1 + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * usq);
  return w * (drho + rho * ((R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * usq));
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
  const R gx = PAR(R, p, g[0]), gy = PAR(R, p, g[1]), gz = PAR(R, p, g[2]);
  // Eq. nm-lbm-velocity with F = rho g: u = j / rho + g / 2
  const R ux = jx / rho + (R)0.5 * gx, uy = jy / rho + (R)0.5 * gy, uz = jz / rho + (R)0.5 * gz;
  const R Fx = rho * gx, Fy = rho * gy, Fz = rho * gz;
  const R usq = ux * ux + uy * uy + uz * uz;
  R fe[Q], fg[Q];
  feq_all<Q, SHIFT, R>(fe, rho, drho, ux, uy, uz, usq);
  guo_all<Q, R>(fg, ux, uy, uz, Fx, Fy, Fz);
  R om = PAR(R, p, omega), pre = PAR(R, p, pre_e);
  R le = PAR(R, p, lam_e), lo = PAR(R, p, lam_o), pe = PAR(R, p, pre_e), po = PAR(R, p, pre_o);
  if (p.les_cs > 0.0) {
    // Smagorinsky model (Sec. 2.1): Q_ab = sum_i c_ia c_ib (f_i - f_i^eq),
    // Qbar = sqrt(2 sum_ab Q_ab^2),
    // tau = tau0 + (sqrt(tau0^2 + 2 sqrt(2) C_S^2 Qbar / (rho c_s^4)) - tau0) / 2
    R qq = (R)0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        R qab = (R)0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          const int cc = dir_c(i, a) * dir_c(i, b);
          if (cc != 0) qab = qab + (R)cc * (fin[i] - fe[i]);
        }
        qq = qq + qab * qab;
      }
    const R qbar = sqrt((R)2 * qq);
    const R t0 = PAR(R, p, tau), cs = PAR(R, p, les_cs);
    const R tau = t0 + (R)0.5 * (sqrt(t0 * t0 + (R)2 * sqrt((R)2) * cs * cs * qbar * (R)9 / rho) - t0);
    om = (R)1 / tau;
    pre = (R)1 - (R)0.5 * om;
    le = om;
    lo = (R)1 / ((R)0.5 + PAR(R, p, magic) / ((R)1 / le - (R)0.5));
    pe = (R)1 - (R)0.5 * le;
    po = (R)1 - (R)0.5 * lo;
  }
  if (!p.trt) {
#pragma unroll
    for (int i = 0; i < Q; ++i) fout[i] = fin[i] - om * (fin[i] - fe[i]) + pre * fg[i];
  } else {
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

// direction with the components in mask (bit a = axis a) negated
template <int Q>
__device__ inline int mirror_dir(int i, int mask) {
  const int c0 = (mask & 1) ? -rc(i, 0) : rc(i, 0);
  const int c1 = (mask & 2) ? -rc(i, 1) : rc(i, 1);
  const int c2 = (mask & 4) ? -rc(i, 2) : rc(i, 2);
  for (int j = 0; j < Q; ++j)
    if (rc(j, 0) == c0 && rc(j, 1) == c1 && rc(j, 2) == c2) return j;
  return i;
}

// Neighbour coordinates of (x, y, z) along each axis: index 0 -> -1, 1 -> 0,
// 2 -> +1; -1 beyond a wall.
struct Nbr {
  int X[3], Y[3], Z[3];
  int sx, ny;
  int fs;  // free-slip axes
  __device__ __forceinline__ void setup(const Geom& g, int x, int y, int z) {
    sx = g.sx;
    ny = g.ny;
    fs = g.free_slip;
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
  // Where the PDF f_i arriving at the cell comes from: normally the cell
  // x - c_i, direction i; across free-slip walls (specular reflection) the
  // cell x - c_i with the crossed components removed, in the mirrored
  // direction.  -1 for a no-slip wall or an obstacle (halfway bounce-back).
  // The same source as source() without looking at the cell types: -1 only
  // for a no-slip wall (an obstacle source is recognised by its flag byte).
  template <int Q>
  __device__ __forceinline__ int geo_source(int i, int& dir) const {
    int a = X[1 - dir_c(i, 0)], b = Y[1 - dir_c(i, 1)], c = Z[1 - dir_c(i, 2)];
    const int crossed = (a < 0 ? 1 : 0) | (b < 0 ? 2 : 0) | (c < 0 ? 4 : 0);
    dir = i;
    if (crossed) {
      if ((crossed & fs) != crossed) return -1;
      if (a < 0) a = X[1];
      if (b < 0) b = Y[1];
      if (c < 0) c = Z[1];
      dir = mirror_dir<Q>(i, crossed);
    }
    return a + sx * (b + ny * c);
  }
  template <int Q>
  __device__ __forceinline__ int source(int i, const uint8_t* flags, int& dir) const {
    int a = X[1 - dir_c(i, 0)], b = Y[1 - dir_c(i, 1)], c = Z[1 - dir_c(i, 2)];
    const int crossed = (a < 0 ? 1 : 0) | (b < 0 ? 2 : 0) | (c < 0 ? 4 : 0);
    dir = i;
    if (crossed) {
      if ((crossed & fs) != crossed) return -1;
      if (a < 0) a = X[1];
      if (b < 0) b = Y[1];
      if (c < 0) c = Z[1];
      dir = mirror_dir<Q>(i, crossed);
    }
    const int n = a + sx * (b + ny * c);
    return (flags[n] & F_TYPE) == T_OBST ? -1 : n;
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
      int di;
      const int n = nb.source<Q>(i, flags, di);
      if (n < 0) fin[i] = ST::ldw(A + opp(i) * plane + c); /* halfway bounce-back */
      else fin[i] = ST::ldw(A + di * plane + n);            /* neighbour or mirror image */
    }
  }
}

// ------------------------------------------------------------ 16/32-bit path
// Collision of one cell in the even/odd (opposite-pair) form, FP32, values in
// storage units (offsets f_i - w_i times S).  For a pair (i, i') = (i, opp i):
//   f+ = (f_i + f_i')/2,  f- = (f_i - f_i')/2
//   e+ = w (drho + rho (4.5 cu^2 - 1.5 u.u)),  e- = 3 w rho cu       (Eq. nm-lbm-equilibrium)
//   G+ = w (9 cu cF - 3 u.F),                   G- = 3 w cF           (Eq. nm-lbm-force-guo)
//   f*_i  = f_i  - [lam_e (f+ - e+) - pe G+] - [lam_o (f- - e-) - po G-]
//   f*_i' = f_i' - [lam_e (f+ - e+) - pe G+] + [lam_o (f- - e-) - po G-]
// which is the TRT update with Guo forcing; SRT is lam_o = lam_e = omega.
// Smagorinsky parameters of the 16/32-bit collision (cs = 0: model off)
struct LesLp {
  float cs, tau0, magic, k;  // k = 2 sqrt(2) C_S^2 * 9 (c_s^-4 of the closure)
  int trt;
  __host__ __device__ static LesLp of(const Phys& p) {
    return LesLp{p.f.les_cs, p.f.tau, p.f.magic, p.f.les_k, p.trt};
  }
};

// Arithmetic of the 16/32-bit collision on V = float (one cell) or float2 (two
// cells, the packed FP32 instructions of sm_100+).  Every operation is an
// explicitly rounded add, multiply or fused multiply-add, so the compiler
// contracts nothing and the one-cell and two-cell kernels produce identical
// bits.
__device__ __forceinline__ float vsplat(float s, float) { return s; }
__device__ __forceinline__ float2 vsplat(float s, float2) { return make_float2(s, s); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as fma(b, -1, a): one rounding of the exact difference
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <class V> struct Lanes;
template <> struct Lanes<float> {
  static constexpr int n = 1;
  static __device__ __forceinline__ float& at(float& v, int) { return v; }
};
template <> struct Lanes<float2> {
  static constexpr int n = 2;
  static __device__ __forceinline__ float& at(float2& v, int k) { return k ? v.y : v.x; }
};
// sum_k c_k v_k for constant c in {-1, 0, 1}, starting from the first
// nonzero term (at least one is nonzero for every moving direction)
template <class V>
__device__ __forceinline__ V vdot(int a, int b, int c, V x, V y, V z) {
  V acc = vsplat(0.f, x);
  bool has = false;
  if (a == 1) { acc = x; has = true; }
  if (a == -1) { acc = vsub(vsplat(0.f, x), x); has = true; }
  if (b != 0) acc = has ? (b == 1 ? vadd(acc, y) : vsub(acc, y)) : (b == 1 ? y : vsub(vsplat(0.f, x), y));
  has = has || b != 0;
  if (c != 0) acc = has ? (c == 1 ? vadd(acc, z) : vsub(acc, z)) : (c == 1 ? z : vsub(vsplat(0.f, x), z));
  return acc;
}

template <int Q, class V>
__device__ __forceinline__ V collide_v(const V* f, V* o, float lamE_, float lamO_, float pe_,
                                       float po_, float gx, float gy, float gz, float S,
                                       const LesLp& les) {
  constexpr int NP = (Q - 1) / 2;
  const V z0 = vsplat(0.f, f[0]);
  V sp[NP], dp[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    sp[k] = vadd(f[2 * k + 1], f[2 * k + 2]);
    dp[k] = vsub(f[2 * k + 1], f[2 * k + 2]);
  }
  V acc = f[0];
#pragma unroll
  for (int k = 0; k < NP; ++k) acc = vadd(acc, sp[k]);
  const V drho = vmul(acc, vsplat(1.0f / S, z0));
  const V rho = vadd(vsplat(1.0f, z0), drho);
  // momentum: first contribution assigned, the rest added in direction order
  V jx = z0, jy = z0, jz = z0;
  bool hx = false, hy = false, hz = false;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int i = 2 * k + 1;
    const int c0 = dir_c(i, 0), c1 = dir_c(i, 1), c2 = dir_c(i, 2);
    if (c0 != 0) { jx = hx ? (c0 == 1 ? vadd(jx, dp[k]) : vsub(jx, dp[k])) : (c0 == 1 ? dp[k] : vsub(z0, dp[k])); hx = true; }
    if (c1 != 0) { jy = hy ? (c1 == 1 ? vadd(jy, dp[k]) : vsub(jy, dp[k])) : (c1 == 1 ? dp[k] : vsub(z0, dp[k])); hy = true; }
    if (c2 != 0) { jz = hz ? (c2 == 1 ? vadd(jz, dp[k]) : vsub(jz, dp[k])) : (c2 == 1 ? dp[k] : vsub(z0, dp[k])); hz = true; }
  }
  // 1/(S rho) from the hardware reciprocal (relative error below 2^-22,
  // the same instruction in every variant); S is a power of two
  V kk = rho;
#pragma unroll
  for (int l = 0; l < Lanes<V>::n; ++l) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(Lanes<V>::at(kk, l)));
    Lanes<V>::at(kk, l) = __fmul_rn(r, 1.0f / S);
  }
  const V ux = vfma(jx, kk, vsplat(0.5f * gx, z0));
  const V uy = vfma(jy, kk, vsplat(0.5f * gy, z0));
  const V uz = vfma(jz, kk, vsplat(0.5f * gz, z0));
  const V Fx = vmul(rho, vsplat(gx, z0)), Fy = vmul(rho, vsplat(gy, z0)), Fz = vmul(rho, vsplat(gz, z0));
  const V usq = vfma(uz, uz, vfma(uy, uy, vmul(ux, ux)));
  const V uF = vfma(uz, Fz, vfma(uy, Fy, vmul(ux, Fx)));
  const V cst = vfma(vmul(rho, vsplat(-1.5f, z0)), usq, drho);
  V lamE = vsplat(lamE_, z0), lamO = vsplat(lamO_, z0), pe = vsplat(pe_, z0), po = vsplat(po_, z0);
  if (les.cs > 0.f) {
    // Smagorinsky model (Sec. 2.1) in the pair form: Q_ab = sum_i c_ia c_ib
    // (f_i - f_i^eq) = sum_pairs c_a c_b (f_i + f_i' - 2 e+)
    V qxx = z0, qyy = z0, qzz = z0, qxy = z0, qxz = z0, qyz = z0;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int i = 2 * k + 1;
      const int c = len2(i);
      const float wS = (float)wgt<Q>(i) * S;
      const int c0 = dir_c(i, 0), c1 = dir_c(i, 1), c2 = dir_c(i, 2);
      const V cu = vdot(c0, c1, c2, ux, uy, uz);
      const V Ac = vmul(vsplat(4.5f * wS, z0), rho), Bcc = vmul(vsplat(wS, z0), cst);
      const V dn = vsub(sp[k], vmul(vsplat(2.f, z0), vfma(vmul(Ac, cu), cu, Bcc)));
      (void)c;
      if (c0 != 0) qxx = vadd(qxx, dn);
      if (c1 != 0) qyy = vadd(qyy, dn);
      if (c2 != 0) qzz = vadd(qzz, dn);
      if (c0 * c1 == 1) qxy = vadd(qxy, dn); else if (c0 * c1 == -1) qxy = vsub(qxy, dn);
      if (c0 * c2 == 1) qxz = vadd(qxz, dn); else if (c0 * c2 == -1) qxz = vsub(qxz, dn);
      if (c1 * c2 == 1) qyz = vadd(qyz, dn); else if (c1 * c2 == -1) qyz = vsub(qyz, dn);
    }
    const V dg = vfma(qzz, qzz, vfma(qyy, qyy, vmul(qxx, qxx)));
    const V of = vfma(qyz, qyz, vfma(qxz, qxz, vmul(qxy, qxy)));
    const V qq = vfma(vsplat(2.f, z0), of, dg);
    V rq = qq, rr = rho;
#pragma unroll
    for (int l = 0; l < Lanes<V>::n; ++l) {
      // Q̄ = sqrt(2 Q_ab Q_ab) in lattice units; tau from the quadratic of
      // the Smagorinsky closure
      const float qbar = __fmul_rn(__fsqrt_rn(__fmul_rn(2.f, Lanes<V>::at(rq, l))), 1.0f / S);
      const float t0 = les.tau0;
      const float arg = __fmaf_rn(t0, t0, __fdiv_rn(__fmul_rn(les.k, qbar), Lanes<V>::at(rr, l)));
      const float tau = __fmaf_rn(0.5f, __fsub_rn(__fsqrt_rn(arg), t0), t0);
      const float le = __frcp_rn(tau);
      const float lo = les.trt ? __frcp_rn(__fadd_rn(0.5f, __fdiv_rn(les.magic, __fsub_rn(tau, 0.5f)))) : le;
      Lanes<V>::at(lamE, l) = le;
      Lanes<V>::at(lamO, l) = lo;
      Lanes<V>::at(pe, l) = __fmaf_rn(-0.5f, le, 1.f);
      Lanes<V>::at(po, l) = __fmaf_rn(-0.5f, lo, 1.f);
    }
  }
  // The update of a pair (i, i') regrouped: with f_i = (sp + dp)/2,
  //   f*_i  = a sp + E + (b dp + D),   f*_i' = a sp + E - (b dp + D),
  //   a = (1 - lam_e)/2, b = (1 - lam_o)/2,
  //   E = cu (lam_e A cu + pe 9 wS cF) + wS (lam_e cst - 3 pe u.F)   (even part),
  //   D = lam_o 3 wS rho cu + po 3 wS cF                            (odd part),
  // A = 4.5 wS rho; wS = w_i S.  Per weight class (index |c|^2):
  const V r45 = vmul(vmul(lamE, rho), vsplat(4.5f, z0));
  const V r3 = vmul(vmul(lamO, rho), vsplat(3.0f, z0));
  const V kb = vfma(lamE, cst, vmul(vmul(vsplat(-3.0f, z0), pe), uF));
  V Ap[4], Op[4], K[4], G9[4], G3[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float wS = (float)wgt<Q>(c == 0 ? 0 : c == 1 ? 1 : c == 2 ? 7 : (Q == 27 ? 19 : 7)) * S;
    K[c] = vmul(vsplat(wS, z0), kb);
    if (c == 0) continue;
    Ap[c] = vmul(vsplat(wS, z0), r45);
    Op[c] = vmul(vsplat(wS, z0), r3);
    G9[c] = vmul(vsplat(9.0f * wS, z0), pe);
    G3[c] = vmul(vsplat(3.0f * wS, z0), po);
  }
  const V al = vfma(vsplat(-0.5f, z0), lamE, vsplat(0.5f, z0));
  const V be = vfma(vsplat(-0.5f, z0), lamO, vsplat(0.5f, z0));
  // rest population: (1 - lam_e) f0 + wS0 (lam_e cst - 3 pe u.F)
  o[0] = vfma(vsub(vsplat(1.0f, z0), lamE), f[0], K[0]);
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int i = 2 * k + 1;
    const int c = len2(i);
    const int c0 = dir_c(i, 0), c1 = dir_c(i, 1), c2 = dir_c(i, 2);
    const V cu = vdot(c0, c1, c2, ux, uy, uz);
    const V cF = vdot(c0, c1, c2, Fx, Fy, Fz);
    const V E = vfma(vfma(Ap[c], cu, vmul(G9[c], cF)), cu, K[c]);
    const V D = vfma(Op[c], cu, vmul(G3[c], cF));
    const V Pp = vfma(al, sp[k], E);
    const V Mm = vfma(be, dp[k], D);
    o[i] = vadd(Pp, Mm);
    o[i + 1] = vsub(Pp, Mm);
  }
  return usq;
}

// The same collision of two cells (V = float2) evaluated in sweeps over the
// direction pairs instead of from 2Q values held in registers: fetch(i)
// returns the pulled value pair of direction i (storage units) and is called
// again in each sweep; emit(i, v) receives the post-collision pair.  Sweep 1
// forms the density and momentum sums, an optional middle sweep the
// Smagorinsky momentum flux, and sweep 2 the outputs.  Every accumulator sees
// the same explicitly rounded operations in the same order as in collide_v,
// so the results are bit for bit those of collide_v<Q, float2>; only a few
// moments and per-class constants stay live.  Returns |u|^2 of both cells.
template <int Q, class Fetch, class Emit>
__device__ __forceinline__ float2 collide_2s(Fetch&& fetch, Emit&& emit, float lamE_, float lamO_,
                                             float pe_, float po_, float gx, float gy, float gz,
                                             float S, const LesLp& les) {
  using V = float2;
  constexpr int NP = (Q - 1) / 2;
  const V z0 = make_float2(0.f, 0.f);
  V acc = fetch(0);
  V jx = z0, jy = z0, jz = z0;
  bool hx = false, hy = false, hz = false;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int i = 2 * k + 1;
    const V a = fetch(i), b = fetch(i + 1);
    const V sp = vadd(a, b), dp = vsub(a, b);
    acc = vadd(acc, sp);
    const int c0 = dir_c(i, 0), c1 = dir_c(i, 1), c2 = dir_c(i, 2);
    if (c0 != 0) { jx = hx ? (c0 == 1 ? vadd(jx, dp) : vsub(jx, dp)) : (c0 == 1 ? dp : vsub(z0, dp)); hx = true; }
    if (c1 != 0) { jy = hy ? (c1 == 1 ? vadd(jy, dp) : vsub(jy, dp)) : (c1 == 1 ? dp : vsub(z0, dp)); hy = true; }
    if (c2 != 0) { jz = hz ? (c2 == 1 ? vadd(jz, dp) : vsub(jz, dp)) : (c2 == 1 ? dp : vsub(z0, dp)); hz = true; }
  }
  const V drho = vmul(acc, vsplat(1.0f / S, z0));
  const V rho = vadd(vsplat(1.0f, z0), drho);
  V kk = rho;
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(Lanes<V>::at(kk, l)));
    Lanes<V>::at(kk, l) = __fmul_rn(r, 1.0f / S);
  }
  const V ux = vfma(jx, kk, vsplat(0.5f * gx, z0));
  const V uy = vfma(jy, kk, vsplat(0.5f * gy, z0));
  const V uz = vfma(jz, kk, vsplat(0.5f * gz, z0));
  const V Fx = vmul(rho, vsplat(gx, z0)), Fy = vmul(rho, vsplat(gy, z0)), Fz = vmul(rho, vsplat(gz, z0));
  const V usq = vfma(uz, uz, vfma(uy, uy, vmul(ux, ux)));
  const V uF = vfma(uz, Fz, vfma(uy, Fy, vmul(ux, Fx)));
  const V cst = vfma(vmul(rho, vsplat(-1.5f, z0)), usq, drho);
  V lamE = vsplat(lamE_, z0), lamO = vsplat(lamO_, z0), pe = vsplat(pe_, z0), po = vsplat(po_, z0);
  // the sweeps below read the pulled values again instead of keeping the
  // first sweep's loads alive
  asm volatile("" ::: "memory");
  if (les.cs > 0.f) {
    V qxx = z0, qyy = z0, qzz = z0, qxy = z0, qxz = z0, qyz = z0;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int i = 2 * k + 1;
      const V sp = vadd(fetch(i), fetch(i + 1));
      const float wS = (float)wgt<Q>(i) * S;
      const int c0 = dir_c(i, 0), c1 = dir_c(i, 1), c2 = dir_c(i, 2);
      const V cu = vdot(c0, c1, c2, ux, uy, uz);
      const V Ac = vmul(vsplat(4.5f * wS, z0), rho), Bcc = vmul(vsplat(wS, z0), cst);
      const V dn = vsub(sp, vmul(vsplat(2.f, z0), vfma(vmul(Ac, cu), cu, Bcc)));
      if (c0 != 0) qxx = vadd(qxx, dn);
      if (c1 != 0) qyy = vadd(qyy, dn);
      if (c2 != 0) qzz = vadd(qzz, dn);
      if (c0 * c1 == 1) qxy = vadd(qxy, dn); else if (c0 * c1 == -1) qxy = vsub(qxy, dn);
      if (c0 * c2 == 1) qxz = vadd(qxz, dn); else if (c0 * c2 == -1) qxz = vsub(qxz, dn);
      if (c1 * c2 == 1) qyz = vadd(qyz, dn); else if (c1 * c2 == -1) qyz = vsub(qyz, dn);
    }
    const V dg = vfma(qzz, qzz, vfma(qyy, qyy, vmul(qxx, qxx)));
    const V of = vfma(qyz, qyz, vfma(qxz, qxz, vmul(qxy, qxy)));
    const V qq = vfma(vsplat(2.f, z0), of, dg);
    V rq = qq, rr = rho;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const float qbar = __fmul_rn(__fsqrt_rn(__fmul_rn(2.f, Lanes<V>::at(rq, l))), 1.0f / S);
      const float t0 = les.tau0;
      const float arg = __fmaf_rn(t0, t0, __fdiv_rn(__fmul_rn(les.k, qbar), Lanes<V>::at(rr, l)));
      const float tau = __fmaf_rn(0.5f, __fsub_rn(__fsqrt_rn(arg), t0), t0);
      const float le = __frcp_rn(tau);
      const float lo = les.trt ? __frcp_rn(__fadd_rn(0.5f, __fdiv_rn(les.magic, __fsub_rn(tau, 0.5f)))) : le;
      Lanes<V>::at(lamE, l) = le;
      Lanes<V>::at(lamO, l) = lo;
      Lanes<V>::at(pe, l) = __fmaf_rn(-0.5f, le, 1.f);
      Lanes<V>::at(po, l) = __fmaf_rn(-0.5f, lo, 1.f);
    }
  }
  const V r45 = vmul(vmul(lamE, rho), vsplat(4.5f, z0));
  const V r3 = vmul(vmul(lamO, rho), vsplat(3.0f, z0));
  const V kb = vfma(lamE, cst, vmul(vmul(vsplat(-3.0f, z0), pe), uF));
  V Ap[4], Op[4], K[4], G9[4], G3[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float wS = (float)wgt<Q>(c == 0 ? 0 : c == 1 ? 1 : c == 2 ? 7 : (Q == 27 ? 19 : 7)) * S;
    K[c] = vmul(vsplat(wS, z0), kb);
    if (c == 0) continue;
    Ap[c] = vmul(vsplat(wS, z0), r45);
    Op[c] = vmul(vsplat(wS, z0), r3);
    G9[c] = vmul(vsplat(9.0f * wS, z0), pe);
    G3[c] = vmul(vsplat(3.0f * wS, z0), po);
  }
  const V al = vfma(vsplat(-0.5f, z0), lamE, vsplat(0.5f, z0));
  const V be = vfma(vsplat(-0.5f, z0), lamO, vsplat(0.5f, z0));
  asm volatile("" ::: "memory");
  emit(0, vfma(vsub(vsplat(1.0f, z0), lamE), fetch(0), K[0]));
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int i = 2 * k + 1;
    const int c = len2(i);
    const V a = fetch(i), b = fetch(i + 1);
    const V sp = vadd(a, b), dp = vsub(a, b);
    const int c0 = dir_c(i, 0), c1 = dir_c(i, 1), c2 = dir_c(i, 2);
    const V cu = vdot(c0, c1, c2, ux, uy, uz);
    const V cF = vdot(c0, c1, c2, Fx, Fy, Fz);
    const V E = vfma(vfma(Ap[c], cu, vmul(G9[c], cF)), cu, K[c]);
    const V D = vfma(Op[c], cu, vmul(G3[c], cF));
    const V Pp = vfma(al, sp, E);
    const V Mm = vfma(be, dp, D);
    emit(i, vadd(Pp, Mm));
    emit(i + 1, vsub(Pp, Mm));
  }
  return usq;
}

// pull_liquid's near-obstacle path for the liquid cell (x, y, z), out of line
// so that the rare cells next to a wall cost the fast path no registers.
template <int Q, class ST>
__device__ __noinline__ void pull_near(const typename ST::T* __restrict__ A, long long plane,
                                       const uint8_t* flags, const Geom& g, int x, int y, int z,
                                       typename ST::R* fin) {
  Nbr nb;
  nb.setup(g, x, y, z);
  pull_liquid<Q, ST>(A, plane, flags, nb, x + g.sx * (y + g.ny * z), true, fin);
}

// Pulled value of direction i at a cell next to a wall or obstacle, in
// storage units: f*_i of the source cell x - c_i (or its mirror image across
// free-slip walls, in the mirrored direction), f*_(opp i) of the cell itself
// (halfway bounce-back) where the source is a no-slip wall or an obstacle;
// the same values as pull_liquid's near-obstacle path.  Out of line: used by
// the rare cells with a wall in their stencil.
template <int Q, class ST>
__device__ __noinline__ float pull_one(const typename ST::T* __restrict__ A, long long plane,
                                       const uint8_t* flags, const Geom& g, int x, int y, int z,
                                       int i) {
  const int c = x + g.sx * (y + g.ny * z);
  int a = x - rc(i, 0), b = y - rc(i, 1), e = z - rc(i, 2);
  int crossed = 0;
  if (a < 0 || a >= g.nx) { if (g.periodic[0]) a = a < 0 ? g.nx - 1 : 0; else crossed |= 1; }
  if (b < 0 || b >= g.ny) { if (g.periodic[1]) b = b < 0 ? g.ny - 1 : 0; else crossed |= 2; }
  if (e < 0 || e >= g.nz) { if (g.periodic[2]) e = e < 0 ? g.nz - 1 : 0; else crossed |= 4; }
  int dir = i;
  if (crossed) {
    if ((crossed & g.free_slip) != crossed) return ST::ld1(A + opp(i) * plane + c);
    if (crossed & 1) a = x;
    if (crossed & 2) b = y;
    if (crossed & 4) e = z;
    dir = mirror_dir<Q>(i, crossed);
  }
  const int n = a + g.sx * (b + g.ny * e);
  if ((flags[n] & F_TYPE) == T_OBST) return ST::ld1(A + opp(i) * plane + c);
  return ST::ld1(A + dir * plane + n);
}

template <int Q>
__device__ __forceinline__ float collide_lp(const float* f, float* o, float lamE, float lamO,
                                            float pe, float po, float gx, float gy, float gz,
                                            float S, const LesLp& les, float& rho_out) {
  rho_out = 0.f;
  return collide_v<Q, float>(f, o, lamE, lamO, pe, po, gx, gy, gz, S, les);
}

// Update of two cells (x0, x0 + 1) of row (y, z) by one thread of a warp whose
// 32 threads cover 64 consecutive cells of that row: pairs of PDFs loaded as
// one aligned 4/8-byte word per direction; PDFs pulled from x -/+ 1 come from
// the neighbouring lane by a warp shuffle (one extra scalar load at the
// warp's edge or at a periodic wrap).  Liquid cells next to a wall or
// obstacle take the per-direction bounce-back path.  GATE: the warp reads the
// flag bytes first and leaves without loading PDFs when it holds no liquid
// cell (grids over every cell); without GATE the PDF loads are issued
// together with the flag loads (warps that walk a list of segments with
// liquid).  Warp-uniform call; returns whether a liquid cell reached
// |u|^2 >= 1/3.
template <int Q, class ST, bool PACKED, bool GATE>
__device__ __forceinline__ bool pair_update(const Dev& d, const Geom& g, const Phys& p, int x0,
                                            int y, int z, int lane) {
  using T = typename ST::T;
  constexpr float S = ST::kScaleF;
  const int cur = d.ctrl->step & 1;
  const T* __restrict__ A = (const T*)d.pdf[cur];
  T* __restrict__ B = (T*)d.pdf[cur ^ 1];
  const long long P = g.plane;
  const unsigned FULL = 0xffffffffu;
  const int row = g.sx * (y + g.ny * z);
  const bool in_row = x0 < g.sx;
  const int xc = in_row ? x0 : g.sx - 2;  // clamped pair start for addressing
  uint8_t fl0 = 0, fl1 = 0;
  if (in_row) {
    const uchar2 fl = *reinterpret_cast<const uchar2*>(d.flags + row + x0);
    fl0 = x0 < g.nx ? fl.x : (uint8_t)T_GAS;
    fl1 = x0 + 1 < g.nx ? fl.y : (uint8_t)T_GAS;
  }
  const int t0 = fl0 & F_TYPE, t1 = fl1 & F_TYPE;
  const bool liq0 = t0 == T_LIQ, liq1 = t1 == T_LIQ;
  if (GATE && !__any_sync(FULL, liq0 || liq1)) return false;
  // rows of the y/z neighbours (a wall side maps to the cell's own row: such
  // cells are near-obstacle and never use the fast values); row offsets fit
  // 32 bits (fewer than 2^31 cells), the plane offset i P is uniform
  int Yr[3], Zr[3];
  Yr[1] = y; Zr[1] = z;
  Yr[0] = y > 0 ? y - 1 : (g.periodic[1] ? g.ny - 1 : y);
  Yr[2] = y < g.ny - 1 ? y + 1 : (g.periodic[1] ? 0 : y);
  Zr[0] = z > 0 ? z - 1 : (g.periodic[2] ? g.nz - 1 : z);
  Zr[2] = z < g.nz - 1 ? z + 1 : (g.periodic[2] ? 0 : z);
  const int xm = x0 > 0 ? xc - 1 : (g.periodic[0] ? g.nx - 1 : 0);
  const bool edge_hi = (lane == 31) || (x0 + 2 >= g.nx);
  const int xp = (x0 + 2 < g.nx) ? x0 + 2 : ((g.periodic[0] && x0 + 2 == g.nx) ? 0 : xc);
  const bool wrap0 = g.periodic[0] && x0 + 1 == g.nx;
  // f[i] = (value pulled by cell x0, value pulled by cell x0 + 1)
  float2 f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = dir_c(i, 0), cy = dir_c(i, 1), cz = dir_c(i, 2);
    const T* base = (A + i * P) + g.sx * (Yr[1 - cy] + g.ny * Zr[1 - cz]);
    const float2 v = ST::ld2(base + xc);
    if (cx == 0) {
      f[i] = v;
    } else if (cx == 1) {  // pulled from x - 1
      const float up = __shfl_up_sync(FULL, v.y, 1);
      f[i] = make_float2((lane == 0) ? ST::ld1(base + xm) : up, v.x);
    } else {  // pulled from x + 1
      const float dn = __shfl_down_sync(FULL, v.x, 1);
      f[i] = make_float2(v.y, edge_hi ? ST::ld1(base + xp) : dn);
      // odd periodic width: the pair's first cell ends the row and wraps
      if (wrap0) f[i].x = ST::ld1(base);
    }
  }
  // cells with a wall or obstacle in their stencil.  Domain walls only (no
  // obstacle cell, no free-slip wall): a PDF whose source lies beyond a wall
  // is the cell's own f*_(opp i) (halfway bounce-back), every other pulled
  // value above came from the right row already.  Otherwise the general
  // per-direction path, out of line.
  const bool walls_only = !g.has_obst && !g.free_slip;
  if (walls_only && ((liq0 && (fl0 & F_NEAR_OBST)) || (liq1 && (fl1 & F_NEAR_OBST)))) {
    const bool wl0 = !g.periodic[0] && x0 == 0, wr1 = !g.periodic[0] && x0 + 2 >= g.nx;
    const bool wr0 = !g.periodic[0] && x0 + 1 >= g.nx;
    const bool ylo = !g.periodic[1] && y == 0, yhi = !g.periodic[1] && y == g.ny - 1;
    const bool zlo = !g.periodic[2] && z == 0, zhi = !g.periodic[2] && z == g.nz - 1;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int cx = dir_c(i, 0), cy = dir_c(i, 1), cz = dir_c(i, 2);
      // the source x - c_i crosses a wall in y or z (both cells), or in x
      const bool yz = (cy == 1 && ylo) || (cy == -1 && yhi) || (cz == 1 && zlo) || (cz == -1 && zhi);
      const bool c0 = yz || (cx == 1 && wl0) || (cx == -1 && wr0);
      const bool c1 = yz || (cx == -1 && wr1);
      if (liq0 && (fl0 & F_NEAR_OBST) && c0) f[i].x = ST::ld1(A + opp(i) * P + row + x0);
      if (liq1 && (fl1 & F_NEAR_OBST) && c1) f[i].y = ST::ld1(A + opp(i) * P + row + x0 + 1);
    }
  } else if ((liq0 && (fl0 & F_NEAR_OBST)) || (liq1 && (fl1 & F_NEAR_OBST))) {
    float t[Q];
    if (liq0 && (fl0 & F_NEAR_OBST)) {
      pull_near<Q, ST>(A, P, d.flags, g, x0, y, z, t);
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i].x = t[i] * S;
    }
    if (liq1 && (fl1 & F_NEAR_OBST)) {
      pull_near<Q, ST>(A, P, d.flags, g, x0 + 1, y, z, t);
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i].y = t[i] * S;
    }
  }
  const bool tr = p.trt != 0;
  const float lamE = p.f.lam_e, lamO = tr ? p.f.lam_o : p.f.omega;
  const float pe = p.f.pre_e, po = tr ? p.f.pre_o : p.f.pre_e;
  float2 usq;
  if constexpr (PACKED) {
    // both cells collide together in packed FP32 (a non-liquid partner's
    // result is discarded)
    usq = collide_v<Q, float2>(f, f, lamE, lamO, pe, po, p.f.g[0], p.f.g[1], p.f.g[2], S,
                               LesLp::of(p));
  } else {
    // one cell after the other: fewer values live at once
    usq = make_float2(0.f, 0.f);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!(h ? liq1 : liq0)) continue;
      float c[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) c[i] = Lanes<float2>::at(f[i], h);
      Lanes<float2>::at(usq, h) =
          collide_v<Q, float>(c, c, lamE, lamO, pe, po, p.f.g[0], p.f.g[1], p.f.g[2], S, LesLp::of(p));
#pragma unroll
      for (int i = 0; i < Q; ++i) Lanes<float2>::at(f[i], h) = c[i];
    }
  }
  const bool bad = (liq0 && !(usq.x < (float)(1.0 / 3.0))) || (liq1 && !(usq.y < (float)(1.0 / 3.0)));
  T* out = B + row + x0;
  if (liq0 && liq1) {
#pragma unroll
    for (int i = 0; i < Q; ++i) ST::st2(out + i * P, f[i].x, f[i].y);
  } else if (liq0) {
#pragma unroll
    for (int i = 0; i < Q; ++i) ST::st1(out + i * P, f[i].x);
  } else if (liq1) {
#pragma unroll
    for (int i = 0; i < Q; ++i) ST::st1(out + i * P + 1, f[i].y);
  }
  return bad;
}

// Bulk pass of the 16/32-bit path over every cell: two cells per thread (see
// pair_update), a block of 128 threads covering 256 cells of a row, or
// several rows of a narrower domain (blockDim.x is a multiple of 32, so every
// warp lies in one row); warps without liquid cells leave after their flags.
template <int Q, class ST, int BT, int MINB, bool PACKED>
__global__ void __launch_bounds__(BT, MINB) k_stream_collide_lp(Dev d, Geom g, Phys p) {
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int lane = threadIdx.x & 31;
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
  if (y >= g.ny) return;
  const bool bad = pair_update<Q, ST, PACKED, true>(d, g, p, x0, y, z, lane);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicCAS(&ctrl->unstable_step, -1, ctrl->step + 1);
}

// Bulk pass over the list of 64-cell row segments with liquid (k_tiles<64>):
// persistent warps walk the list with a grid stride, one segment (two cells
// per lane, pair_update without the flag gate) per iteration; the list entry
// of the next iteration is loaded one iteration ahead.  No gas-only warp is
// launched and a warp's flag and PDF loads are in flight together, so every
// segment costs one memory round trip.
template <int Q, class ST>
__device__ __forceinline__ void stream_collide_seg_body(const Dev& d, const Geom& g, const Phys& p, int ntx) {
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int ntl = (int)ctrl->n_tiles;
  const int lane = threadIdx.x & 31;
  const int tw = gridDim.x * (blockDim.x >> 5);
  int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int seg = k < ntl ? d.l_tiles[k] : 0;
  bool bad = false;
  while (k < ntl) {
    const int kn = k + tw;
    const int segn = kn < ntl ? d.l_tiles[kn] : 0;
    const int x0 = (seg % ntx) * 64 + 2 * lane;
    const int row = seg / ntx;
    bad |= pair_update<Q, ST, true, false>(d, g, p, x0, row % g.ny, row / g.ny, lane);
    k = kn;
    seg = segn;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicCAS(&ctrl->unstable_step, -1, ctrl->step + 1);
}
template <int Q, class ST, int MINB>
__global__ void __launch_bounds__(128, MINB) k_stream_collide_seg(Dev d, Geom g, Phys p, int ntx) {
  stream_collide_seg_body<Q, ST>(d, g, p, ntx);
}
template <int Q, class ST>
__global__ void __launch_bounds__(128, 4) kb_stream_collide_seg(MemberTable t) {
  FSL_MEMBER(t);
  stream_collide_seg_body<Q, ST>(d, g, p, (g.nx + 63) / 64);
}


// One liquid cell (x, y, z) per thread, from a warp covering 32 consecutive
// cells of a row: one stored value loaded per direction straight from the
// source cell x - c_i (any alignment; the warp's 32 loads of a direction are
// contiguous), the collision in FP32 on one cell (collide_v<Q, float>, the
// same bits as the two-cell variants), one store per direction.  With a
// single value per direction live, a thread needs about half the registers
// of the two-cell form, so twice the warps fit on an SM.  Returns whether
// the cell is liquid and reached |u|^2 >= 1/3.
template <int Q, class ST>
__device__ __forceinline__ bool cell_update(const Dev& d, const Geom& g, const Phys& p, int x, int y,
                                            int z) {
  using T = typename ST::T;
  constexpr float S = ST::kScaleF;
  const int cur = d.ctrl->step & 1;
  const T* __restrict__ A = (const T*)d.pdf[cur];
  T* __restrict__ B = (T*)d.pdf[cur ^ 1];
  const long long P = g.plane;
  const int row = g.sx * (y + g.ny * z);
  const bool in = x < g.nx;
  const uint8_t fl = in ? d.flags[row + x] : (uint8_t)T_GAS;
  const bool liq = (fl & F_TYPE) == T_LIQ;
  const int xs = in ? x : 0;  // in-row address for the lanes past the row end
  // neighbour rows and columns (a wall side maps to the cell itself: such
  // cells are near-obstacle and take the bounce-back values below)
  const int ym = y > 0 ? y - 1 : (g.periodic[1] ? g.ny - 1 : y);
  const int yp = y < g.ny - 1 ? y + 1 : (g.periodic[1] ? 0 : y);
  const int zm = z > 0 ? z - 1 : (g.periodic[2] ? g.nz - 1 : z);
  const int zp = z < g.nz - 1 ? z + 1 : (g.periodic[2] ? 0 : z);
  const int xm = xs > 0 ? xs - 1 : (g.periodic[0] ? g.nx - 1 : xs);
  const int xq = xs < g.nx - 1 ? xs + 1 : (g.periodic[0] ? 0 : xs);
  float f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = dir_c(i, 0), cy = dir_c(i, 1), cz = dir_c(i, 2);
    const int yy = cy == 0 ? y : (cy == 1 ? ym : yp);
    const int zz = cz == 0 ? z : (cz == 1 ? zm : zp);
    const int xx = cx == 0 ? xs : (cx == 1 ? xm : xq);
    f[i] = ST::ld1((A + i * P) + g.sx * (yy + g.ny * zz) + xx);
  }
  if (liq && (fl & F_NEAR_OBST)) {
    if (!g.has_obst && !g.free_slip) {
      // domain walls only: the directions whose source lies beyond a wall
      // take the cell's own f*_(opp i) (halfway bounce-back)
      const bool xlo = !g.periodic[0] && x == 0, xhi = !g.periodic[0] && x == g.nx - 1;
      const bool ylo = !g.periodic[1] && y == 0, yhi = !g.periodic[1] && y == g.ny - 1;
      const bool zlo = !g.periodic[2] && z == 0, zhi = !g.periodic[2] && z == g.nz - 1;
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int cx = dir_c(i, 0), cy = dir_c(i, 1), cz = dir_c(i, 2);
        const bool cross = (cx == 1 && xlo) || (cx == -1 && xhi) || (cy == 1 && ylo) ||
                           (cy == -1 && yhi) || (cz == 1 && zlo) || (cz == -1 && zhi);
        if (cross) f[i] = ST::ld1(A + opp(i) * P + row + x);
      }
    } else {
      float t[Q];
      pull_near<Q, ST>(A, P, d.flags, g, x, y, z, t);
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i] = t[i] * S;
    }
  }
  const bool tr = p.trt != 0;
  const float lamE = p.f.lam_e, lamO = tr ? p.f.lam_o : p.f.omega;
  const float pe = p.f.pre_e, po = tr ? p.f.pre_o : p.f.pre_e;
  const float usq = collide_v<Q, float>(f, f, lamE, lamO, pe, po, p.f.g[0], p.f.g[1], p.f.g[2], S,
                                        LesLp::of(p));
  if (liq) {
    T* out = B + row + x;
#pragma unroll
    for (int i = 0; i < Q; ++i) ST::st1(out + i * P, f[i]);
  }
  return liq && !(usq < (float)(1.0 / 3.0));
}

// Bulk pass over the list of 64-cell row segments with liquid, one cell per
// thread: persistent warps walk the halves (32 cells) of the listed segments
// with a grid stride, the list entry of the next iteration loaded one
// iteration ahead.
template <int Q, class ST, int MINB>
__global__ void __launch_bounds__(128, MINB) k_stream_collide_c1(Dev d, Geom g, Phys p, int ntx) {
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int nh = 2 * (int)ctrl->n_tiles;
  const int lane = threadIdx.x & 31;
  const int tw = gridDim.x * (blockDim.x >> 5);
  int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int seg = k < nh ? d.l_tiles[k >> 1] : 0;
  bool bad = false;
  while (k < nh) {
    const int kn = k + tw;
    const int segn = kn < nh ? d.l_tiles[kn >> 1] : 0;
    const int x = (seg % ntx) * 64 + 32 * (k & 1) + lane;
    const int row = seg / ntx;
    bad |= cell_update<Q, ST>(d, g, p, x, row % g.ny, row / g.ny);
    k = kn;
    seg = segn;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicCAS(&ctrl->unstable_step, -1, ctrl->step + 1);
}

// Bulk pass of the 16-bit storages with four cells per thread: the four
// stored values of each direction arrive as one aligned 8-byte load and stay
// packed (two 32-bit words) until the collision unpacks them; the values
// pulled from x -/+ 1 are assembled with byte permutes from the neighbouring
// lane's words (warp shuffles), one scalar load at the warp's edges or at a
// periodic wrap.  Same arithmetic as k_stream_collide_lp, twice the bytes in
// flight per thread.
template <int Q, class ST>
__global__ void __launch_bounds__(64) k_stream_collide_lp4(Dev d, Geom g, Phys p) {
  using T = typename ST::T;
  static_assert(sizeof(T) == 2, "16-bit storage only");
  constexpr float S = ST::kScaleF;
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int cur = ctrl->step & 1;
  const T* __restrict__ A = (const T*)d.pdf[cur];
  T* __restrict__ B = (T*)d.pdf[cur ^ 1];
  const long long P = g.plane;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y, z = blockIdx.z;
  const int row = g.sx * (y + g.ny * z);
  const bool in_row = x0 < g.sx;
  const int xc = in_row ? x0 : g.sx - 4;  // clamped group start for addressing
  uint8_t fl[4] = {0, 0, 0, 0};
  if (in_row) {
    const uchar4 f4 = *reinterpret_cast<const uchar4*>(d.flags + row + x0);
    fl[0] = x0 < g.nx ? f4.x : (uint8_t)T_GAS;
    fl[1] = x0 + 1 < g.nx ? f4.y : (uint8_t)T_GAS;
    fl[2] = x0 + 2 < g.nx ? f4.z : (uint8_t)T_GAS;
    fl[3] = x0 + 3 < g.nx ? f4.w : (uint8_t)T_GAS;
  }
  bool anyl = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    anyl |= (fl[k] & F_TYPE) == T_LIQ;
  }
  if (!__any_sync(FULL, anyl)) return;
  int Yr[3], Zr[3];
  Yr[1] = y; Zr[1] = z;
  Yr[0] = y > 0 ? y - 1 : (g.periodic[1] ? g.ny - 1 : y);
  Yr[2] = y < g.ny - 1 ? y + 1 : (g.periodic[1] ? 0 : y);
  Zr[0] = z > 0 ? z - 1 : (g.periodic[2] ? g.nz - 1 : z);
  Zr[2] = z < g.nz - 1 ? z + 1 : (g.periodic[2] ? 0 : z);
  const int xm = x0 > 0 ? xc - 1 : (g.periodic[0] ? g.nx - 1 : 0);
  const bool edge_hi = (lane == 31) || (x0 + 4 >= g.nx);
  const int xp = (x0 + 4 < g.nx) ? x0 + 4 : ((g.periodic[0] && x0 + 4 == g.nx) ? 0 : xc);
  const int kwrap = (g.periodic[0] && x0 < g.nx && x0 + 3 >= g.nx) ? g.nx - 1 - x0 : -1;
  // w[i][0] = (e0, e1), w[i][1] = (e2, e3): the four values pulled by the
  // thread's cells in direction i, low half first
  unsigned w[Q][2];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = dir_c(i, 0), cy = dir_c(i, 1), cz = dir_c(i, 2);
    const T* base = A + i * P + (long long)g.sx * (Yr[1 - cy] + g.ny * Zr[1 - cz]);
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(base + xc));
    if (cx == 0) {
      w[i][0] = v.x;
      w[i][1] = v.y;
    } else if (cx == 1) {  // pulled from x - 1: (left, e0), (e1, e2)
      unsigned left = __shfl_up_sync(FULL, v.y, 1);
      if (lane == 0) left = (unsigned)__ldg(reinterpret_cast<const unsigned short*>(base + xm)) << 16;
      w[i][0] = __byte_perm(left, v.x, 0x5432);
      w[i][1] = __byte_perm(v.x, v.y, 0x5432);
    } else {  // pulled from x + 1: (e1, e2), (e3, right)
      unsigned right = __shfl_down_sync(FULL, v.x, 1);
      if (edge_hi) right = (unsigned)__ldg(reinterpret_cast<const unsigned short*>(base + xp));
      w[i][0] = __byte_perm(v.x, v.y, 0x5432);
      w[i][1] = __byte_perm(v.y, right, 0x5432);
      // periodic row end inside the group (cells 0..2): wraps to x = 0
      if (kwrap >= 0) {
        const unsigned e = (unsigned)__ldg(reinterpret_cast<const unsigned short*>(base));
        if (kwrap == 0) w[i][0] = (w[i][0] & 0xffff0000u) | e;
        else if (kwrap == 1) w[i][0] = (w[i][0] & 0xffffu) | (e << 16);
        else w[i][1] = (w[i][1] & 0xffff0000u) | e;
      }
    }
  }
  const bool tr = p.trt != 0;
  const float lamE = p.f.lam_e, lamO = tr ? p.f.lam_o : p.f.omega;
  const float pe = p.f.pre_e, po = tr ? p.f.pre_o : p.f.pre_e;
  const float gx = p.f.g[0], gy = p.f.g[1], gz = p.f.g[2];
  const LesLp les = LesLp::of(p);
  bool bad = false;
#pragma unroll
  for (int pr = 0; pr < 2; ++pr) {  // cell pairs (0, 1) and (2, 3)
    bool liq[2];
    liq[0] = (fl[2 * pr] & F_TYPE) == T_LIQ;
    liq[1] = (fl[2 * pr + 1] & F_TYPE) == T_LIQ;
    if (!liq[0] && !liq[1]) continue;
    float2 f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = ST::unpack2(w[i][pr]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * pr + h;
      if (liq[h] && (fl[k] & F_NEAR_OBST)) {
        float t[Q];
        Nbr nb;
        nb.setup(g, x0 + k, y, z);
        pull_liquid<Q, ST>(A, P, d.flags, nb, row + x0 + k, true, t);
#pragma unroll
        for (int i = 0; i < Q; ++i) Lanes<float2>::at(f[i], h) = t[i] * S;
      }
    }
    // both cells of the pair collide together in packed FP32
    const float2 usq = collide_v<Q, float2>(f, f, lamE, lamO, pe, po, gx, gy, gz, S, les);
    bad |= (liq[0] && !(usq.x < (float)(1.0 / 3.0))) || (liq[1] && !(usq.y < (float)(1.0 / 3.0)));
#pragma unroll
    for (int i = 0; i < Q; ++i) w[i][pr] = ST::pack2(f[i].x, f[i].y);
    T* out = B + row + x0 + 2 * pr;
    if (liq[0] && liq[1]) {
#pragma unroll
      for (int i = 0; i < Q; ++i) *reinterpret_cast<unsigned*>(out + i * P) = w[i][pr];
    } else if (liq[0]) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        *reinterpret_cast<unsigned short*>(out + i * P) = (unsigned short)(w[i][pr] & 0xffffu);
    } else if (liq[1]) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        *reinterpret_cast<unsigned short*>(out + i * P + 1) = (unsigned short)(w[i][pr] >> 16);
    }
  }
  if (__any_sync(FULL, bad) && lane == 0) atomicCAS(&ctrl->unstable_step, -1, ctrl->step + 1);
}

// Bulk pass of the 16-bit storages, software-pipelined over rows: each block
// covers 256 cells of a row (two per thread) and walks rows r, r + G, r + 2G,
// ... of the domain; while it collides row r, the loads of its next row are
// already in flight (one aligned 4-byte word per direction and thread, plus
// the scalar values the warp's edge lanes need), and the flags are read two
// rows ahead so that the decision to load a row (any liquid cell in the warp)
// never waits.  The loads in flight therefore cover the whole collision
// instead of only the start of a thread's life.
template <int Q, class ST>
__device__ __forceinline__ void pp_fetch(const typename ST::T* __restrict__ A, const Geom& g,
                                         int rr, int xc, int xm, int xp, bool edge_hi, bool wrap0,
                                         int lane, unsigned* w, unsigned* e) {
  const long long P = g.plane;
  const int y = rr % g.ny, z = rr / g.ny;
  int Yr[3], Zr[3];
  Yr[1] = y; Zr[1] = z;
  Yr[0] = y > 0 ? y - 1 : (g.periodic[1] ? g.ny - 1 : y);
  Yr[2] = y < g.ny - 1 ? y + 1 : (g.periodic[1] ? 0 : y);
  Zr[0] = z > 0 ? z - 1 : (g.periodic[2] ? g.nz - 1 : z);
  Zr[2] = z < g.nz - 1 ? z + 1 : (g.periodic[2] ? 0 : z);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = dir_c(i, 0), cy = dir_c(i, 1), cz = dir_c(i, 2);
    const unsigned short* base = reinterpret_cast<const unsigned short*>(A) + i * P +
                                 (long long)g.sx * (Yr[1 - cy] + g.ny * Zr[1 - cz]);
    w[i] = __ldg(reinterpret_cast<const unsigned*>(base + xc));
    e[i] = 0u;
    if (cx == 1 && lane == 0) e[i] = (unsigned)__ldg(base + xm) << 16;
    if (cx == -1 && (wrap0 || edge_hi)) e[i] = (unsigned)__ldg(base + (wrap0 ? 0 : xp));
  }
}

template <int Q, class ST>
__global__ void __launch_bounds__(128, 3) k_stream_collide_pp(Dev d, Geom g, Phys p) {
  using T = typename ST::T;
  static_assert(sizeof(T) == 2, "16-bit storage only");
  constexpr float S = ST::kScaleF;
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int cur = ctrl->step & 1;
  const T* __restrict__ A = (const T*)d.pdf[cur];
  T* __restrict__ B = (T*)d.pdf[cur ^ 1];
  const long long P = g.plane;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int nrows = g.ny * g.nz;
  const int G = gridDim.y;
  int r = blockIdx.y;
  if (r >= nrows) return;
  const bool in_row = x0 < g.sx;
  const int xc = in_row ? x0 : g.sx - 2;
  const int xm = x0 > 0 ? xc - 1 : (g.periodic[0] ? g.nx - 1 : 0);
  const bool edge_hi = (lane == 31) || (x0 + 2 >= g.nx);
  const int xp = (x0 + 2 < g.nx) ? x0 + 2 : ((g.periodic[0] && x0 + 2 == g.nx) ? 0 : xc);
  const bool wrap0 = g.periodic[0] && x0 + 1 == g.nx;
  // the two type bytes of the thread's cells in row rr (gas outside)
  auto flags_of = [&](int rr) -> unsigned {
    if (rr >= nrows || !in_row) return 0u;
    const uchar2 f = *reinterpret_cast<const uchar2*>(d.flags + (long long)rr * g.sx + x0);
    const unsigned a = x0 < g.nx ? f.x : (unsigned)T_GAS;
    const unsigned b = x0 + 1 < g.nx ? f.y : (unsigned)T_GAS;
    return a | (b << 8);
  };
  auto has_liquid = [](unsigned f) {
    return (f & F_TYPE) == T_LIQ || ((f >> 8) & F_TYPE) == T_LIQ;
  };
  const bool tr = p.trt != 0;
  const float lamE = p.f.lam_e, lamO = tr ? p.f.lam_o : p.f.omega;
  const float pe = p.f.pre_e, po = tr ? p.f.pre_o : p.f.pre_e;
  const LesLp les = LesLp::of(p);
  unsigned fc = flags_of(r), fn = flags_of(r + G);
  bool anyc = __any_sync(FULL, has_liquid(fc));
  unsigned w[Q], e[Q];
  if (anyc) pp_fetch<Q, ST>(A, g, r, xc, xm, xp, edge_hi, wrap0, lane, w, e);
  bool bad = false;
  for (;;) {
    const int rn = r + G;
    const unsigned fnn = flags_of(rn + G);
    const bool anyn = __any_sync(FULL, has_liquid(fn));
    unsigned wn[Q], en[Q];
    if (anyn) pp_fetch<Q, ST>(A, g, rn, xc, xm, xp, edge_hi, wrap0, lane, wn, en);
    // row r: interface cells to the list, liquid cells stream and collide
    const long long row = (long long)r * g.sx;
    const uint8_t fl0 = (uint8_t)(fc & 0xffu), fl1 = (uint8_t)(fc >> 8);
    if (anyc) {
      const bool liq0 = (fl0 & F_TYPE) == T_LIQ, liq1 = (fl1 & F_TYPE) == T_LIQ;
      float2 f[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int cx = dir_c(i, 0);
        unsigned word;
        if (cx == 0) {
          word = w[i];
        } else if (cx == 1) {  // (x - 1, x): the left lane's high half, then ours
          unsigned left = __shfl_up_sync(FULL, w[i], 1);
          if (lane == 0) left = e[i];
          word = __byte_perm(left, w[i], 0x5432);
        } else {  // (x + 1, x + 2): our high half, then the right lane's low half
          unsigned right = __shfl_down_sync(FULL, w[i], 1);
          if (edge_hi) right = e[i];
          word = wrap0 ? e[i] : __byte_perm(w[i], right, 0x5432);
        }
        f[i] = ST::unpack2(word);
      }
      const int y = r % g.ny, z = r / g.ny;
      if ((liq0 && (fl0 & F_NEAR_OBST)) || (liq1 && (fl1 & F_NEAR_OBST))) {
        float t[Q];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint8_t fh = h ? fl1 : fl0;
          if ((fh & F_TYPE) == T_LIQ && (fh & F_NEAR_OBST)) {
            Nbr nb;
            nb.setup(g, x0 + h, y, z);
            pull_liquid<Q, ST>(A, P, d.flags, nb, (int)(row + x0 + h), true, t);
#pragma unroll
            for (int i = 0; i < Q; ++i) Lanes<float2>::at(f[i], h) = t[i] * S;
          }
        }
      }
      // both cells of the pair collide together in packed FP32
      const float2 usq =
          collide_v<Q, float2>(f, f, lamE, lamO, pe, po, p.f.g[0], p.f.g[1], p.f.g[2], S, les);
      bad |= (liq0 && !(usq.x < (float)(1.0 / 3.0))) || (liq1 && !(usq.y < (float)(1.0 / 3.0)));
      T* out = B + row + x0;
      if (liq0 && liq1) {
#pragma unroll
        for (int i = 0; i < Q; ++i) *reinterpret_cast<unsigned*>(out + i * P) = ST::pack2(f[i].x, f[i].y);
      } else if (liq0) {
#pragma unroll
        for (int i = 0; i < Q; ++i) ST::st1(out + i * P, f[i].x);
      } else if (liq1) {
#pragma unroll
        for (int i = 0; i < Q; ++i) ST::st1(out + i * P + 1, f[i].y);
      }
    }
    if (rn >= nrows) break;
    r = rn;
    fc = fn;
    fn = fnn;
    anyc = anyn;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      w[i] = wn[i];
      e[i] = en[i];
    }
  }
  if (__any_sync(FULL, bad) && lane == 0) atomicCAS(&ctrl->unstable_step, -1, ctrl->step + 1);
}

}  // namespace fsl
#include "fsl_bulk.cuh"
#include "fsl_bubble.cuh"
namespace fsl {

// ------------------------------------------------------------ stream-collide
// Pass over all cells: liquid cells stream and collide here (interface cells
// are handled by k_stream_collide_if from the step's interface list).
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
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
    atomicCAS(&ctrl->unstable_step, -1, ctrl->step + 1);
}

// Interface cells (list-driven): free-surface boundary condition for PDFs
// arriving from gas, mass flux, collision, fill level and conversion marks.
// (16/32-bit path: five blocks per SM at 96 registers, some spilled; the
// interface list of a 256^3 drop impact then fits in one wave: 90 us at
// three blocks, 70 at four, and the step 2 % faster again at five)
template <int Q, class ST>
__device__ __forceinline__ void stream_collide_if_body(const Dev& d, const Geom& g, const Phys& p) {
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
  const int* lif = list_if(d, ctrl->step);
  bool bad = false;
  FSL_WARP_LOOP(k, ok, nif) {
    bool to_liq = false, to_gas = false;
    const int c = ok ? lif[k] : 0;
    if (ok) {
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
    const R utx = jx / rt - (R)0.5 * PAR(R, p, g[0]);
    const R uty = jy / rt - (R)0.5 * PAR(R, p, g[1]);
    const R utz = jz / rt - (R)0.5 * PAR(R, p, g[2]);
    const R utsq = utx * utx + uty * uty + utz * utz;
    // Eq. nm-fslbm-pressure-gas: volume pressure (per bubble with the bubble
    // model, Eq. nm-fslbm-pressure-volume) and Laplace pressure
    int bub = -1;
    if (g.bubbles) bub = d.blab[c];
    const double pv = bub >= 0 ? d.bp[bub] : p.p_v;
    const double pg = (p.options & 8u) ? pv - 2.0 * p.sigma * d.kappa[c]
                                       : pv + p.sigma * d.kappa[c];
    const R rg = (R)(3.0 * pg);  // rho_G = p_G / c_s^2
    const R drg = (R)(3.0 * pg - 1.0);
    // Eq. nm-fslbm-mass-flux over i = 1..Q-1 (gas and walls carry none), in
    // the working precision (FP64 in the FP64 path)
    const R phx = (R)phi_work<R>(d)[c];
    const int clsx = fl & (F_NF | F_NE);
    const bool thurey = !(p.options & 1u);
    R dm = (R)0;
    bool dm_has = false;
    // Directions in opposite pairs (0 alone, then (1, 2), (3, 4), ...): per
    // direction the source cell of the incoming PDF (-1 beyond a no-slip
    // wall), its flag byte, stored value and fill level (every load with a
    // valid address whatever the type turns out to be, the type only selects
    // among the values), then the pair's two flux terms, which need exactly
    // the pair's values: the sum still runs over i = 1, 2, 3, ... in order,
    // and a pair's loads are dead once its terms are added.
#pragma unroll
    for (int k = 0; k <= (Q - 1) / 2; ++k) {
      const int i0 = k == 0 ? 0 : 2 * k - 1;
      const int np = k == 0 ? 1 : 2;
      // gas equilibria of the pair (Eq. nm-fslbm-boundary-condition)
      const R fe0 = feq_c<Q, SH, R>(i0, rg, drg, utx, uty, utz, utsq);
      const R fe1 = np == 2 ? feq_c<Q, SH, R>(i0 + 1, rg, drg, utx, uty, utz, utsq) : fe0;
      uint8_t fb2[2];
      R ph2[2];
      int tn2[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h >= np) break;
        const int i = i0 + h;
        int di;
        const int n = nb.geo_source<Q>(i, di);
        const int ns = n >= 0 ? n : c;
        fb2[h] = n >= 0 ? d.flags[ns] : (uint8_t)T_OBST;
        const R nv = ST::ldw(A + di * P + ns);
        ph2[h] = (R)phi_work<R>(d)[ns];
        const int t = fb2[h] & F_TYPE;
        tn2[h] = t;
        const R fa = h == 0 ? fe0 : fe1, fo = h == 0 ? fe1 : fe0;
        if (is_fluid(t)) fin[i] = nv;                         /* neighbour or mirror image */
        else if (t == T_OBST) fin[i] = own[opp(i)];          /* halfway bounce-back */
        else fin[i] = fa + fo - own[opp(i)];                 /* anti-bounce-back from gas */
      }
      if (np < 2) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = i0 + h, io = opp(i), ho = 1 - h;  // io = i0 + ho
        // the cell exchanging PDFs with x along c_i (x + c_i, or its mirror
        // image across a free-slip wall) is the source of the incoming f_io
        const int t = tn2[ho];
        if (t != T_LIQ && t != T_IF) continue;
        // f_in = fin[io] (what arrives from it), f_out = f*_i(x) = own[i]
        R dd;
        const R both = fin[io] - own[i];
        if (t == T_LIQ) {
          dd = both;
        } else {
          const int clsn = fb2[ho] & (F_NF | F_NE);
          const R f_in = SH ? fin[io] + (R)wgt<Q>(io) : fin[io];
          const R f_out = SH ? own[i] + (R)wgt<Q>(i) : own[i];
          R br;
          if (!thurey) br = both;
          else if (clsx == 0) br = (clsn == F_NF) ? f_in : (clsn == F_NE) ? -f_out : both;
          else if (clsx == F_NF) br = (clsn == F_NF) ? both : -f_out;
          else br = (clsn == F_NE) ? both : f_in;
          dd = (R)0.5 * (phx + ph2[ho]) * br;
        }
        dm = dm_has ? dm + dd : dd;
        dm_has = true;
      }
    }
    const double m_new = dm_has ? d.mass[c] + (double)dm : d.mass[c];
    R fout[Q], rho;
    R usq;
    if constexpr (SH) {
      // 16/32-bit path: the regrouped pair collision of the bulk kernels, on
      // unscaled offsets (scale 1); rho summed in the same pair order
      R drho;
      density<Q, SH, R>(fin, rho, drho);
      const bool tr = p.trt != 0;
      usq = collide_v<Q, float>(fin, fout, p.f.lam_e, tr ? p.f.lam_o : p.f.omega, p.f.pre_e,
                                tr ? p.f.pre_o : p.f.pre_e, p.f.g[0], p.f.g[1], p.f.g[2], 1.0f,
                                LesLp::of(p));
    } else {
      usq = collide<Q, SH, R>(fin, fout, p, rho);
    }
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
      to_liq = true;
    } else if (ph < p.thr_lo) {
      d.flags[c] = fl | F_TO_GAS;
      to_gas = true;
    }
    }
    warp_append(to_liq, c, &ctrl->n_fill, d.l_fill);
    warp_append(to_gas, c, &ctrl->n_empty, d.l_empty);
  }
  if (bad) atomicCAS(&ctrl->unstable_step, -1, ctrl->step + 1);
}
template <int Q, class ST>
__global__ void __launch_bounds__(128, ST::kShift ? 5 : 1) k_stream_collide_if(Dev d, Geom g, Phys p) {
  stream_collide_if_body<Q, ST>(d, g, p);
}
template <int Q, class ST>
__global__ void __launch_bounds__(128, ST::kShift ? 5 : 1) kb_stream_collide_if(MemberTable t) {
  FSL_MEMBER(t);
  stream_collide_if_body<Q, ST>(d, g, p);
}


// ------------------------------------------------------------ conversion


// lane i of a warp examines direction i of the warp's cell (warp-per-cell
// loops); lanes >= Q stay idle but take part in the ballots.  Consecutive
// items go to consecutive blocks, so that a short list is spread over all SMs
// (its FP64 arithmetic shares each SM's two FP64 lanes with few other items).
#define FSL_WARP_PER_ITEM(k, n)                                                     \
  for (unsigned k = (threadIdx.x >> 5) * gridDim.x + blockIdx.x; k < (n);           \
       k += (gridDim.x * blockDim.x) >> 5)
// one thread per item, spread over the blocks in the same way
#define FSL_SPREAD_LOOP(k, n)                                                       \
  for (unsigned k = threadIdx.x * gridDim.x + blockIdx.x; k < (n);                  \
       k += gridDim.x * blockDim.x)

template <int Q>
__device__ __forceinline__ void fill_body(const Dev& d, const Geom& g) {
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const unsigned nif = ctrl->n_if, nfill = ctrl->n_fill;
  const int* lif = list_if(d, ctrl->step);
  // commit the fill levels computed by the stream-collide pass
  FSL_GRID_LOOP(k, nif) {
    const int c = lif[k];
    put_phi(d, c, d.phinew[c]);
  }
  // gas neighbours of filled cells become new interface cells; a neighbour
  // about to empty is kept (filling wins)
  const int lane = threadIdx.x & 31;
  FSL_WARP_PER_ITEM(k, nfill) {
    int x, y, z;
    cell_xyz(g, d.l_fill[k], x, y, z);
    int n = -1;
    bool created = false;
    if (lane >= 1 && lane < Q) {
      n = nb_at(g, x, y, z, rc(lane, 0), rc(lane, 1), rc(lane, 2));
      if (n >= 0) {
        // one load of the flag byte: marks are only set by the interface
        // pass, and clearing one twice is harmless
        const uint8_t fn = d.flags[n];
        if ((fn & F_TYPE) == T_GAS) {
          const uint8_t old = byte_or(d.flags, n, (uint8_t)(F_NEW | T_IF));
          if (!(old & F_NEW)) {
            put_phi(d, n, 0.0);
            d.mass[n] = 0.0;
            created = true;
          }
        }
        if (fn & F_TO_GAS) byte_and(d.flags, n, F_TO_GAS);
      }
    }
    warp_append(created, n, &ctrl->n_new, d.l_new);
  }
}
template <int Q>
__global__ void __launch_bounds__(256) kb_fill(MemberTable t) {
  FSL_MEMBER(t);
  fill_body<Q>(d, g);
}


template <int Q, class ST>
__device__ __forceinline__ void empty_body(const Dev& d, const Geom& g) {
  using R = typename ST::R;
  constexpr bool SH = ST::kShift;
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int cur = ctrl->step & 1;
  const typename ST::T* A = (const typename ST::T*)d.pdf[cur];
  const unsigned ne = ctrl->n_empty;
  const int lane = threadIdx.x & 31;
  FSL_WARP_PER_ITEM(k, ne) {
    const int c = d.l_empty[k];
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    // the neighbour's flag byte is loaded together with the cell's own
    int n = -1;
    uint8_t fn = 0;
    if (lane >= 1 && lane < Q) {
      n = nb_at(g, x, y, z, rc(lane, 0), rc(lane, 1), rc(lane, 2));
      if (n >= 0) fn = d.flags[n];
    }
    if (!(d.flags[c] & F_TO_GAS)) continue;  // kept by a filling neighbour (warp-uniform)
    bool won = false;
    if (n >= 0 && (fn & F_TYPE) == T_LIQ) {
      // the liquid cell's density of this step, recomputed exactly as the
      // stream-collide pass obtained it (its PDFs are loaded before the type
      // change is claimed, so that the two round trips overlap; a lane whose
      // claim fails drops them)
      int nx_, ny_, nz_;
      cell_xyz(g, n, nx_, ny_, nz_);
      Nbr nb;
      nb.setup(g, nx_, ny_, nz_);
      R fin[Q], rho, drho;
      pull_liquid<Q, ST>(A, g.plane, d.flags, nb, n, (fn & F_NEAR_OBST) != 0, fin);
      density<Q, SH, R>(fin, rho, drho);
      if (byte_retype(d.flags, n, T_LIQ, T_IF, &ctrl->timeout)) {
        d.rho[n] = (double)rho;
        d.mass[n] = (double)rho;
        put_phi(d, n, 1.0);
        won = true;
      }
    }
    warp_append(won, n, &ctrl->n_l2i, d.l_l2i);
  }
}
template <int Q, class ST>
__global__ void __launch_bounds__(256) kb_empty(MemberTable t) {
  FSL_MEMBER(t);
  empty_body<Q, ST>(d, g);
}


// Type of cell c once this step's conversions are applied: a cell marked to
// fill becomes liquid, a cell still marked to empty becomes gas (every marked
// cell is on the fill or the empty list, and the marks of earlier steps were
// cleared by k_classify).  Beyond a wall: T_OBST.
__device__ __forceinline__ int final_type(const uint8_t* flags, int c) {
  if (c < 0) return T_OBST;
  const uint8_t b = flags[c];
  return (b & F_TO_LIQ) ? T_LIQ : (b & F_TO_GAS) ? T_GAS : (b & F_TYPE);
}

// Conversion of the filled and emptied cells with the share of their excess
// mass per receiver (Eq. nm-fslbm-excess-mass), one warp per cell: lane 0
// changes the type and computes the excess mass, lanes 1..Q-1 test the
// neighbour x + c_i, which receives a share when it is an interface cell after
// the conversions (its final type, read from its marks, so that the answer
// does not depend on whether its own conversion was written yet), and claim
// it for the receiver list.  Receivers are counted per direction.
template <int Q>
__device__ __forceinline__ void finalise_share_body(const Dev& d, const Geom& g) {
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const unsigned nf = ctrl->n_fill, ne = ctrl->n_empty;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  FSL_WARP_PER_ITEM(k, nf + ne) {
    const bool fill = k < nf;
    const int c = fill ? d.l_fill[k] : d.l_empty[k - nf];
    const uint8_t fl = d.flags[c];
    if (!fill && !(fl & F_TO_GAS)) continue;  // kept by a filling neighbour (warp-uniform)
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    int n = -1;
    bool recv = false, claimed = false;
    if (lane >= 1 && lane < Q) {
      n = nb_at(g, x, y, z, rc(lane, 0), rc(lane, 1), rc(lane, 2));
      recv = final_type(d.flags, n) == T_IF;
      if (recv) claimed = byte_or(d.claim, n, 1) == 0;
    }
    const int nr = __popc(__ballot_sync(FULL, recv));
    warp_append(claimed, n, &ctrl->n_recv, d.l_recv);
    if (lane == 0) {
      double mex;
      if (fill) {
        mex = (d.phi[c] - 1.0) * d.rho[c];
        d.flags[c] = (uint8_t)((fl & ~F_TYPE) | T_LIQ);
        put_phi(d, c, 1.0);
        d.mass[c] = d.rho[c];
      } else {
        mex = d.phi[c] * d.rho[c];
        d.flags[c] = (uint8_t)((fl & ~F_TYPE) | T_GAS);
        put_phi(d, c, 0.0);
        d.mass[c] = 0.0;
        atomicAdd(&ctrl->n_emptied, 1u);
      }
      if (nr == 0) {
        d.lost[c] += mex;
        d.mex[c] = 0.0;
      } else {
        d.mex[c] = mex / (double)nr;
      }
    }
  }
}
template <int Q>
__global__ void __launch_bounds__(256) kb_finalise_share(MemberTable t) {
  FSL_MEMBER(t);
  finalise_share_body<Q>(d, g);
}


// ------------------------------------------------------------ normals
// Parker-Youngs gradient of phi at cell (x, y, z): per axis a, the centred
// difference across the 3x3 block perpendicular to a with weights 4 (centre),
// 2 (edges), 1 (corners), divided by 32; exact for linear phi.  An axis whose
// block touches a wall or obstacle uses a two-point difference over the
// non-obstacle cells instead (narrowed stencil near obstacles).  RC is the
// compute type: FP64 in the FP64 path, FP32 otherwise.
template <class RC, class PT>
__device__ inline void normal_py(const Geom& g, const uint8_t* flags, const PT* phi, int x,
                                 int y, int z, RC* n) {
  const int p[3] = {x, y, z};
  const int c = x + g.sx * (y + g.ny * z);
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3, cc = (a + 2) % 3;
    if (b > cc) { int t = b; b = cc; cc = t; }
    int yp_[9], ym_[9];
    bool touches = false;
    for (int ob = -1; ob <= 1; ++ob)
      for (int oc = -1; oc <= 1; ++oc) {
        int dp[3] = {0, 0, 0}, dm[3] = {0, 0, 0};
        dp[a] = 1; dm[a] = -1;
        dp[b] += ob; dm[b] += ob;
        dp[cc] += oc; dm[cc] += oc;
        const int k = 3 * (ob + 1) + (oc + 1);
        yp_[k] = nb_at(g, p[0], p[1], p[2], dp[0], dp[1], dp[2]);
        ym_[k] = nb_at(g, p[0], p[1], p[2], dm[0], dm[1], dm[2]);
        if (type_at(flags, yp_[k]) == T_OBST || type_at(flags, ym_[k]) == T_OBST) touches = true;
      }
    if (!touches) {
      RC sum = (RC)0;
      for (int ob = -1; ob <= 1; ++ob)
        for (int oc = -1; oc <= 1; ++oc) {
          const int k = 3 * (ob + 1) + (oc + 1);
          const RC w = (RC)((ob == 0 ? 2.0 : 1.0) * (oc == 0 ? 2.0 : 1.0));
          const RC t = w * ((RC)phi[yp_[k]] - (RC)phi[ym_[k]]);
          sum = (k == 0) ? (RC)0 + t : sum + t;
        }
      n[a] = sum / (RC)32;
    } else {
      const int yp = yp_[4], ym = ym_[4];
      const bool okp = type_at(flags, yp) != T_OBST, okm = type_at(flags, ym) != T_OBST;
      if (okp && okm) n[a] = (RC)0.5 * ((RC)phi[yp] - (RC)phi[ym]);
      else if (okp) n[a] = (RC)phi[yp] - (RC)phi[c];
      else if (okm) n[a] = (RC)phi[c] - (RC)phi[ym];
      else n[a] = (RC)0;
    }
  }
}

template <class RC, class PT>
__device__ inline void unit_normal(const Geom& g, const uint8_t* flags, const PT* phi, int x,
                                   int y, int z, RC* nh) {
  RC n[3];
  normal_py<RC>(g, flags, phi, x, y, z, n);
  const RC len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  if (len < (RC)1e-12) {
    nh[0] = nh[1] = nh[2] = (RC)0;
  } else {
    nh[0] = n[0] / len;
    nh[1] = n[1] / len;
    nh[2] = n[2] / len;
  }
}

// coordinate v wrapped into [0, n) (periodic axes; v within one period)
__device__ __forceinline__ int wrapc(int v, int n) {
  if (v < 0) v += n;
  else if (v >= n) v -= n;
  return (v < 0 || v >= n) ? ((v % n) + n) % n : v;
}

// K = -div(n_hat), central differences over the face neighbours; a wall side
// is replaced by the centre value.
template <class RC, class PT>
__device__ inline RC curvature(const Geom& g, const uint8_t* flags, const PT* phi, int x,
                               int y, int z) {
  RC nc[3];
  unit_normal<RC>(g, flags, phi, x, y, z, nc);
  RC div = (RC)0;
  for (int a = 0; a < 3; ++a) {
    int dp[3] = {0, 0, 0}, dm[3] = {0, 0, 0};
    dp[a] = 1; dm[a] = -1;
    const int yp = nb_at(g, x, y, z, dp[0], dp[1], dp[2]);
    const int ym = nb_at(g, x, y, z, dm[0], dm[1], dm[2]);
    const bool okp = type_at(flags, yp) != T_OBST, okm = type_at(flags, ym) != T_OBST;
    RC np[3], nm[3], dd;
    const int px = wrapc(x + dp[0], g.nx), py = wrapc(y + dp[1], g.ny), pz = wrapc(z + dp[2], g.nz);
    const int mx = wrapc(x + dm[0], g.nx), my = wrapc(y + dm[1], g.ny), mz = wrapc(z + dm[2], g.nz);
    if (okp && okm) {
      unit_normal<RC>(g, flags, phi, px, py, pz, np);
      unit_normal<RC>(g, flags, phi, mx, my, mz, nm);
      dd = (RC)0.5 * (np[a] - nm[a]);
    } else if (okp) {
      unit_normal<RC>(g, flags, phi, px, py, pz, np);
      dd = np[a] - nc[a];
    } else if (okm) {
      unit_normal<RC>(g, flags, phi, mx, my, mz, nm);
      dd = nc[a] - nm[a];
    } else {
      dd = (RC)0;
    }
    div = (a == 0) ? (RC)0 + dd : div + dd;
  }
  return -div;
}

// The same curvature for a cell whose distance-2 neighbourhood holds no wall
// or obstacle: no type checks, wrapped coordinates computed once.  Same
// operation order as curvature(), so the results are identical.
template <class RC, class PT>
__device__ inline RC curvature_open(const Geom& g, const PT* phi, int x, int y, int z) {
  int X[5], Y[5], Z[5];
#pragma unroll
  for (int o = 0; o < 5; ++o) {
    X[o] = wrapc(x + o - 2, g.nx);
    Y[o] = wrapc(y + o - 2, g.ny);
    Z[o] = wrapc(z + o - 2, g.nz);
  }
  RC div = (RC)0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    RC nh[2][3];
#pragma unroll
    for (int sgn = 0; sgn < 2; ++sgn) {
      // point p = centre + (+1 | -1) e_a, in offset coordinates (2 = centre)
      int pc[3] = {2, 2, 2};
      pc[a] += sgn == 0 ? 1 : -1;
      RC v[3][3][3];  // phi around p, v[dz+1][dy+1][dx+1]
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx)
            v[dz + 1][dy + 1][dx + 1] =
                (RC)phi[X[pc[0] + dx] + g.sx * (Y[pc[1] + dy] + g.ny * Z[pc[2] + dz])];
      RC n[3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        int b = (ax + 1) % 3, cc = (ax + 2) % 3;
        if (b > cc) { int t = b; b = cc; cc = t; }
        RC sum = (RC)0;
#pragma unroll
        for (int ob = -1; ob <= 1; ++ob)
#pragma unroll
          for (int oc = -1; oc <= 1; ++oc) {
            int op[3] = {0, 0, 0}, om[3] = {0, 0, 0};
            op[ax] = 1; om[ax] = -1;
            op[b] += ob; om[b] += ob;
            op[cc] += oc; om[cc] += oc;
            const RC w = (RC)((ob == 0 ? 2.0 : 1.0) * (oc == 0 ? 2.0 : 1.0));
            const RC t = w * (v[op[2] + 1][op[1] + 1][op[0] + 1] - v[om[2] + 1][om[1] + 1][om[0] + 1]);
            sum = (ob == -1 && oc == -1) ? (RC)0 + t : sum + t;
          }
        n[ax] = sum / (RC)32;
      }
      // without a branch, so that the loads of all six stencils can be in
      // flight at once
      const RC len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      const bool tiny = len < (RC)1e-12;
      const RC l = tiny ? (RC)1 : len;
      nh[sgn][0] = tiny ? (RC)0 : n[0] / l;
      nh[sgn][1] = tiny ? (RC)0 : n[1] / l;
      nh[sgn][2] = tiny ? (RC)0 : n[2] / l;
    }
    const RC dd = (RC)0.5 * (nh[0][a] - nh[1][a]);
    div = (a == 0) ? (RC)0 + dd : div + dd;
  }
  return -div;
}

// true when no cell within distance 2 of (x, y, z) can be a wall or obstacle
__device__ __forceinline__ bool open_neighbourhood(const Geom& g, int x, int y, int z) {
  if (g.has_obst) return false;
  if (!g.periodic[0] && (x < 2 || x > g.nx - 3)) return false;
  if (!g.periodic[1] && (y < 2 || y > g.ny - 3)) return false;
  if (!g.periodic[2] && (z < 2 || z > g.nz - 3)) return false;
  return true;
}

template <class RC, class PT>
__device__ inline RC curvature_any(const Geom& g, const uint8_t* flags, const PT* phi, int x,
                                   int y, int z) {
  return open_neighbourhood(g, x, y, z) ? curvature_open<RC>(g, phi, x, y, z)
                                        : curvature<RC>(g, flags, phi, x, y, z);
}

// ------------------------------------------------------------ refilling
// plain FP64 equilibrium for a runtime direction (initial state)
template <int Q>
__device__ inline double feq_d(int i, double rho, double ux, double uy, double uz) {
  const double cu = (double)rc(i, 0) * ux + (double)rc(i, 1) * uy + (double)rc(i, 2) * uz;
  const double usq = ux * ux + uy * uy + uz * uz;
  return rw<Q>(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
}

// equilibrium of a runtime direction in working representation (Eq.
// nm-lbm-equilibrium): f_i^eq, or f_i^eq - w_i in the shifted representation
template <int Q, bool SHIFT, class R>
__device__ inline R feq_rt(int i, R rho, R drho, R ux, R uy, R uz) {
  const R cu = (R)rc(i, 0) * ux + (R)rc(i, 1) * uy + (R)rc(i, 2) * uz;
  const R usq = ux * ux + uy * uy + uz * uz;
  const R w = (R)rw<Q>(i);
  if (!SHIFT) return w * rho * ((R)1 + (R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * usq);
  return w * (drho + rho * ((R)3 * cu + (R)4.5 * cu * cu - (R)1.5 * usq));
}

// stored moments of cell n (double, full PDFs): rho = sum f*,
// u = sum c f* / rho - g / 2  (observation kernels)
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

// the same in working representation and precision
template <int Q, class ST>
__device__ inline void stored_moments_w(const typename ST::T* B, long long plane, int n,
                                        const Phys& p, typename ST::R& rho,
                                        typename ST::R& drho, typename ST::R* u) {
  using R = typename ST::R;
  R f[Q], jx, jy, jz;
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = ST::ldw(B + i * plane + n);
  density<Q, ST::kShift, R>(f, rho, drho);
  momentum<Q, R>(f, jx, jy, jz);
  u[0] = jx / rho - (R)0.5 * PAR(R, p, g[0]);
  u[1] = jy / rho - (R)0.5 * PAR(R, p, g[1]);
  u[2] = jz / rho - (R)0.5 * PAR(R, p, g[2]);
}

__device__ __forceinline__ bool valid_src(const uint8_t* flags, int n) {
  if (n < 0) return false;
  const uint8_t f = flags[n];
  return is_fluid(f & F_TYPE) && !(f & F_NEW);
}

// Refilling (Sec. 3.1), one warp per new interface cell: lane i examines the
// neighbour x + c_i and writes the refilled f_i; sums over the valid
// neighbours run in direction order (shuffled to every lane), so the FP64
// result equals a sequential evaluation in that order.
template <int Q, class ST>
__device__ __forceinline__ void refill_body(const Dev& d, const Geom& g, const Phys& p) {
  using T = typename ST::T;
  using R = typename ST::R;
  constexpr bool SH = ST::kShift;
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int cur = ctrl->step & 1;
  T* B = (T*)d.pdf[cur ^ 1];
  const long long P = g.plane;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned nn = ctrl->n_new;
  const int scheme = p.refill;
  FSL_WARP_PER_ITEM(k, nn) {
    const int c = d.l_new[k];
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    int n = -1;
    bool valid = false;
    R nr = (R)0, ndr = (R)0, nu[3] = {(R)0, (R)0, (R)0};
    if (lane >= 1 && lane < Q) {
      n = nb_at(g, x, y, z, rc(lane, 0), rc(lane, 1), rc(lane, 2));
      valid = valid_src(d.flags, n);
      // loaded whatever the flag says (the cell itself beyond a wall), so that
      // the loads need not wait for it; only valid neighbours are used below
      stored_moments_w<Q, ST>(B, P, n >= 0 ? n : c, p, nr, ndr, nu);
    }
    const unsigned vmask = __ballot_sync(FULL, valid);
    const int count = __popc(vmask);
    // rho_bar, u_bar: plain means over the valid neighbours (R7)
    R rsum = (R)0, dsum = (R)0, sx = (R)0, sy = (R)0, sz = (R)0;
    for (int j = 1; j < Q; ++j) {
      const R a = __shfl_sync(FULL, nr, j), b = __shfl_sync(FULL, ndr, j);
      const R vx = __shfl_sync(FULL, nu[0], j), vy = __shfl_sync(FULL, nu[1], j),
              vz = __shfl_sync(FULL, nu[2], j);
      if ((vmask >> j) & 1u) {
        rsum = rsum + a;
        dsum = dsum + b;
        sx = sx + vx;
        sy = sy + vy;
        sz = sz + vz;
      }
    }
    const R cnt = (R)(count > 0 ? count : 1);
    const R rb = rsum / cnt, drb = dsum / cnt;
    const R ubx = sx / cnt, uby = sy / cnt, ubz = sz / cnt;
    // direction best aligned with the interface normal among valid ones
    int dn = -1;
    if (scheme == 1 || scheme == 3) {
      R n3[3];
      normal_py<R>(g, d.flags, phi_work<R>(d), x, y, z, n3);
      R best = (R)0;
      for (int j = 1; j < Q; ++j) {
        if (!((vmask >> j) & 1u)) continue;
        const R dot = (R)rc(j, 0) * n3[0] + (R)rc(j, 1) * n3[1] + (R)rc(j, 2) * n3[2];
        if (dn < 0 || dot > best) { dn = j; best = dot; }
      }
    }
    const int i = lane;
    R out = (R)0;
    const bool bad = count == 0 || ((scheme == 1 || scheme == 3) && dn < 0);
    if (bad) {
      // unreachable for cells created by a filling neighbour; latch the event
      if (lane == 0) atomicOr(&ctrl->timeout, 2u);
      out = SH ? (R)0 : (R)(i < Q ? rw<Q>(i) : 0.0);
    } else if (scheme == 0 || scheme == 1 || scheme == 2) {
      const int li = i < Q ? i : 0;
      const R fe = feq_rt<Q, SH, R>(li, rb, drb, ubx, uby, ubz);
      out = fe;
      if (scheme == 1) {  // EQ+NEQ (R8: the neighbour's own equilibrium)
        const int yn = __shfl_sync(FULL, n, dn);
        const R ry = __shfl_sync(FULL, nr, dn), dry = __shfl_sync(FULL, ndr, dn);
        const R vx = __shfl_sync(FULL, nu[0], dn), vy = __shfl_sync(FULL, nu[1], dn),
                vz = __shfl_sync(FULL, nu[2], dn);
        if (i < Q) {
          const R fy = ST::ldw(B + i * P + yn);
          R fneq;
          if (p.options & 4u) fneq = fy - fe;
          else fneq = fy - feq_rt<Q, SH, R>(i, ry, dry, vx, vy, vz);
          out = fe + fneq;
        }
      } else if (scheme == 2) {  // GEQ (R9: prefactor 1/(2 c_s^2 omega))
        R vel[7][3];
        for (int j = 1; j <= 6; ++j) {
          vel[j][0] = __shfl_sync(FULL, nu[0], j);
          vel[j][1] = __shfl_sync(FULL, nu[1], j);
          vel[j][2] = __shfl_sync(FULL, nu[2], j);
        }
        const R ub[3] = {ubx, uby, ubz};
        R du[3][3];
        for (int b = 0; b < 3; ++b) {
          const int dp = 1 + 2 * b, dm = 2 + 2 * b;
          const bool vp = (vmask >> dp) & 1u, vm = (vmask >> dm) & 1u;
          for (int a = 0; a < 3; ++a) {
            if (vp && vm) du[a][b] = (R)0.5 * (vel[dp][a] - vel[dm][a]);
            else if (vp) du[a][b] = vel[dp][a] - ub[a];
            else if (vm) du[a][b] = ub[a] - vel[dm][a];
            else du[a][b] = (R)0;
          }
        }
        const R coef = PAR(R, p, geq_coef);
        const int cc[3] = {rc(li, 0), rc(li, 1), rc(li, 2)};
        R sum = (R)0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            const R Sab = du[a][b] + du[b][a];
            const R Qab = (a == b ? (R)(1.0 / 3.0) : (R)0) - (R)(cc[a] * cc[b]);
            sum = sum + Sab * Qab;
          }
        out = fe + (R)rw<Q>(li) * rb * coef * sum;
      }
    } else if (scheme == 3) {  // EXT, second order with lower-order fallbacks
      const int cx = rc(dn, 0), cy = rc(dn, 1), cz = rc(dn, 2);
      const int y1 = __shfl_sync(FULL, n, dn);
      const int y2 = nb_at(g, x, y, z, 2 * cx, 2 * cy, 2 * cz);
      const int y3 = nb_at(g, x, y, z, 3 * cx, 3 * cy, 3 * cz);
      int kk = 1;
      const bool v2 = valid_src(d.flags, y2), v3 = valid_src(d.flags, y3);
      if (v2) kk = v3 ? 3 : 2;
      if (i < Q) {
        const R f1 = ST::ldw(B + i * P + y1);
        if (kk == 3) {
          const R f2 = ST::ldw(B + i * P + y2), f3 = ST::ldw(B + i * P + y3);
          out = (R)3 * f1 - (R)3 * f2 + f3;
        } else if (kk == 2) {
          out = (R)2 * f1 - ST::ldw(B + i * P + y2);
        } else {
          out = f1;
        }
      }
    } else {  // AVG
      R sum = (R)0;
      for (int j = 1; j < Q; ++j) {
        const int nj = __shfl_sync(FULL, n, j);
        if (((vmask >> j) & 1u) && i < Q) sum = sum + ST::ldw(B + i * P + nj);
      }
      out = sum / cnt;
    }
    if (i < Q) ST::stw(B + i * P + c, out);
    // density of the refilled cell, summed in direction order
    R r = (R)0;
    for (int j = 0; j < Q; ++j) {
      const R oj = __shfl_sync(FULL, out, j);
      r = (j == 0) ? oj : r + oj;
    }
    if (lane == 0) d.rho[c] = SH ? 1.0 + (double)r : (double)r;
  }
}
template <int Q, class ST>
__global__ void __launch_bounds__(128) kb_refill(MemberTable t) {
  FSL_MEMBER(t);
  refill_body<Q, ST>(d, g, p);
}


// ------------------------------------------------------------ excess mass
// Each receiver gathers the shares of its converted neighbours, summed in
// direction order; one thread per receiver (its flag loads, then its share
// loads, in flight together).
template <int Q>
__device__ __forceinline__ void excess_gather_body(const Dev& d, const Geom& g) {
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const unsigned nr = ctrl->n_recv;
  FSL_SPREAD_LOOP(k, nr) {
    const int r = d.l_recv[k];
    int x, y, z;
    cell_xyz(g, r, x, y, z);
    Nbr nb;
    nb.setup(g, x, y, z);
    const double m0 = d.mass[r], rr = d.rho[r];
    // flag bytes and shares of all neighbours with valid addresses (the cell
    // itself beyond a wall), so that all loads are in flight together and the
    // marks only select which shares are summed
    uint8_t fb[Q];
    double sv[Q];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int n = nb.at(dir_c(i, 0), dir_c(i, 1), dir_c(i, 2));
      const int ns = n >= 0 ? n : r;
      fb[i] = n >= 0 ? d.flags[ns] : (uint8_t)0;
      sv[i] = d.mex[ns];
    }
    double sum = 0.0;
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (fb[i] & (F_TO_LIQ | F_TO_GAS)) sum += sv[i];
    const double m = m0 + sum;
    d.mass[r] = m;
    put_phi(d, r, m / rr);
  }
}
template <int Q>
__global__ void __launch_bounds__(256) kb_excess_gather(MemberTable t) {
  FSL_MEMBER(t);
  excess_gather_body<Q>(d, g);
}


// ------------------------------------------------------------ conversion phase
// Fill, empty, finalise with excess share, refill and excess gather of one
// step in one cooperative launch (all blocks resident).  Each phase reads what the
// previous phases wrote anywhere in the domain, so a grid-wide barrier
// separates them: block arrivals are counted in ctrl->bar (phase k waits for
// k * gridDim.x arrivals), the waits are bounded in time, and a block whose
// wait gives up sets timeout bit 16 and leaves (the blocks still waiting then
// give up in their turn).  The phases run the same bodies as the separate
// kernels of the batched path, in the same order, so the results are the same.
constexpr unsigned long long kBarrierWaitNs = 200000000ull;  // 0.2 s
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool grid_barrier(Ctrl* ctrl, unsigned target) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this block's writes before its arrival
    atomicAdd(&ctrl->bar, 1u);
    int good = 1;
    const unsigned long long t0 = global_ns();
    while (*(volatile unsigned*)&ctrl->bar < target) {
      if (global_ns() - t0 > kBarrierWaitNs) {
        atomicOr(&ctrl->timeout, 16u);
        good = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();  // the other blocks' writes before this block's reads
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}
// Self-check of the bounded wait: one block arrives at a grid barrier whose
// target needs one more arrival than can come, gives up after the time
// bound, latches timeout bit 16, and puts the arrival count back.
static __global__ void k_barrier_selftest(Dev d) {
  Ctrl* ctrl = d.ctrl;
  __shared__ unsigned before;
  if (threadIdx.x == 0) before = *(volatile unsigned*)&ctrl->bar;
  __syncthreads();
  const bool ok = grid_barrier(ctrl, before + 2u);
  if (threadIdx.x == 0) {
    ctrl->bar = before;
    if (ok) atomicOr(&ctrl->timeout, 32u);  // not expected: no second arrival exists
  }
}

template <int Q, class ST>
__global__ void __launch_bounds__(256) k_convert(Dev d, Geom g, Phys p) {
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const unsigned nb = gridDim.x;
  fill_body<Q>(d, g);
  if (!grid_barrier(ctrl, nb)) return;
  empty_body<Q, ST>(d, g);
  if (!grid_barrier(ctrl, 2 * nb)) return;
  finalise_share_body<Q>(d, g);
  if (!grid_barrier(ctrl, 3 * nb)) return;
  refill_body<Q, ST>(d, g, p);
  if (!grid_barrier(ctrl, 4 * nb)) return;
  excess_gather_body<Q>(d, g);
}


// ------------------------------------------------------------ classes / curvature
// Thuerey class of an interface cell from its stencil neighbours.
template <int Q>
__device__ inline uint8_t iface_class(const Geom& g, const uint8_t* flags, int x, int y, int z) {
  Nbr nb;
  nb.setup(g, x, y, z);
  const int c = nb.in(0, 0, 0);
  bool has_liq = false, has_gas = false;
  // every flag load has a valid address (the cell itself beyond a wall), so
  // the q - 1 loads are in flight together
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int n = nb.at(dir_c(i, 0), dir_c(i, 1), dir_c(i, 2));
    const uint8_t b = flags[n >= 0 ? n : c];
    const int t = n >= 0 ? (b & F_TYPE) : T_OBST;
    if (t == T_LIQ) has_liq = true;
    if (t == T_GAS) has_gas = true;
  }
  if (!has_liq && has_gas) return F_NF;
  if (!has_gas && has_liq) return F_NE;
  return 0;
}

template <int Q, class ST>
__device__ __forceinline__ void classify_body(const Dev& d, const Geom& g, const Phys& p) {
  using R = typename ST::R;
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const unsigned a = ctrl->n_if, b = ctrl->n_new, e = ctrl->n_l2i;
  const int* lif = list_if(d, ctrl->step);
  int* lnext = list_if(d, ctrl->step + 1);
  // every interface cell of the next step was interface, new or liquid turned
  // interface in this one: the next step's list is built here
  // block-uniform loop (the append below is block-wide; 128 threads)
  const unsigned n = a + b + e;
  for (unsigned base = blockIdx.x * 128u; base < n; base += gridDim.x * 128u) {
    const unsigned k = base + threadIdx.x;
    const bool ok = k < n;
    const int c = !ok ? 0 : (k < a ? lif[k] : (k < a + b ? d.l_new[k - a] : d.l_l2i[k - a - b]));
    bool is_if = false;
    if (ok) {
      const uint8_t fl = d.flags[c];
      uint8_t nf = (uint8_t)(fl & ~(F_TO_LIQ | F_TO_GAS | F_NEW | F_NF | F_NE));
      d.claim[c] = 0;
      if ((fl & F_TYPE) == T_IF) {
        is_if = true;
        int x, y, z;
        cell_xyz(g, c, x, y, z);
        nf |= iface_class<Q>(g, d.flags, x, y, z);
        d.kappa[c] = (p.sigma != 0.0) ? (double)curvature_any<R>(g, d.flags, phi_work<R>(d), x, y, z) : 0.0;
      }
      d.flags[c] = nf;
    }
    block_append<128>(is_if, c, &ctrl->n_if_next, lnext);
  }
}
template <int Q, class ST>
__global__ void __launch_bounds__(128, 4) k_classify(Dev d, Geom g, Phys p) {
  classify_body<Q, ST>(d, g, p);
}
template <int Q, class ST>
__global__ void __launch_bounds__(128, 4) kb_classify(MemberTable t) {
  FSL_MEMBER(t);
  classify_body<Q, ST>(d, g, p);
}


// The FP32 copy of every fill level (state loaded from a checkpoint).
static __global__ void k_phif_from_phi(Dev d, Geom g) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.cells;
       c += (long long)gridDim.x * blockDim.x)
    d.phif[c] = (float)d.phi[c];
}

// The interface list of the current step from the flags (initial state, state
// loaded from a checkpoint).
static __global__ void k_list_interface(Dev d, Geom g) {
  Ctrl* ctrl = d.ctrl;
  int* lif = list_if(d, ctrl->step);
  FSL_WARP_LOOP(k, ok, (unsigned)g.cells) {
    bool is_if = false;
    if (ok) {
      const int x = (int)(k % (unsigned)g.sx);
      is_if = x < g.nx && (d.flags[k] & F_TYPE) == T_IF;
    }
    warp_append(is_if, (int)k, &ctrl->n_if, lif);
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
// The trace reductions are split over kEndBlocks blocks (fixed partition,
// fixed tree order); the last block to finish combines the partials in block
// order and advances the counters.
constexpr int kEndBlocks = 64;
__device__ __forceinline__ void end_step_body(const Dev& d, const Geom& g) {
  __shared__ double shd[256];
  __shared__ int shi[256];
  __shared__ bool last;
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int every = ctrl->trace_every;
  const bool tracing = every > 0 && ((ctrl->step + 1) % every) == 0;
  double* part = d.red;                         // kEndBlocks column partials
  int* ipart = reinterpret_cast<int*>(d.red + kEndBlocks);  // 2 x kEndBlocks maxima
  if (tracing) {
    const int ncol = g.ny * g.nz;
    const int chunk = (ncol + gridDim.x - 1) / gridDim.x;
    const int k0 = blockIdx.x * chunk, k1 = min(ncol, k0 + chunk);
    double s = 0.0;
    int hbest = -1;
    for (int k = k0 + threadIdx.x; k < k1; k += 256) {
      const long long cidx = (long long)g.sx * k;   // cell (0, j, kz), k = j + ny kz
      s += d.phi[cidx];
      if ((d.flags[cidx] & F_TYPE) == T_IF) hbest = max(hbest, k % g.ny);
    }
    const double bs = block_sum<256>(s, shd);
    const int bh = block_max<256>(hbest, shi);
    // front: cells (i, 0, kz)
    const int nrow = g.nx * g.nz;
    const int rchunk = (nrow + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * rchunk, r1 = min(nrow, r0 + rchunk);
    int fbest = -1;
    for (int k = r0 + threadIdx.x; k < r1; k += 256) {
      const int i = k % g.nx, kz = k / g.nx;
      if ((d.flags[i + (long long)g.sx * g.ny * kz] & F_TYPE) == T_IF) fbest = max(fbest, i);
    }
    const int bf = block_max<256>(fbest, shi);
    if (threadIdx.x == 0) {
      part[blockIdx.x] = bs;
      ipart[blockIdx.x] = bf;
      ipart[kEndBlocks + blockIdx.x] = bh;
    }
  }
  __threadfence();
  if (threadIdx.x == 0) last = atomicAdd(&ctrl->end_blocks, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (tracing) {
    const bool in = (int)threadIdx.x < (int)gridDim.x;
    const double cp = in ? *(volatile double*)&part[threadIdx.x] : 0.0;
    const int fp = in ? *(volatile int*)&ipart[threadIdx.x] : -1;
    const int hp = in ? *(volatile int*)&ipart[kEndBlocks + threadIdx.x] : -1;
    const double col_all = block_sum<256>(cp, shd);
    const int front_all = block_max<256>(fp, shi);
    const int height_all = block_max<256>(hp, shi);
    if (threadIdx.x == 0) {
      shd[0] = col_all;
      shi[0] = front_all;
      shi[1] = height_all;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (tracing) {
      const double col = shd[0];
      const int front = shi[0], height = shi[1];
      const int slot = ctrl->trace_count % kTraceCapacity;
      d.trace[3 * slot + 0] = col / (double)g.nz;
      d.trace[3 * slot + 1] = (double)(front + 1);
      d.trace[3 * slot + 2] = (double)(height + 1);
      ctrl->trace_count += 1;
    }
    ctrl->last[0] = ctrl->n_fill;
    ctrl->last[1] = ctrl->n_emptied;
    ctrl->last[2] = ctrl->n_new;
    ctrl->last[3] = ctrl->n_if;
    ctrl->n_if = ctrl->n_if_next;  // the list k_classify built for the next step
    ctrl->n_if_next = 0;
    ctrl->n_fill = ctrl->n_empty = 0;
    ctrl->n_new = ctrl->n_l2i = ctrl->n_recv = 0;
    ctrl->n_emptied = 0;
    ctrl->end_blocks = 0;
    ctrl->n_tiles = 0;
    ctrl->bar = 0;
    __threadfence();
    ctrl->step += 1;
  }
}
static __global__ void __launch_bounds__(256) k_end_step(Dev d, Geom g) { end_step_body(d, g); }
static __global__ void __launch_bounds__(256) kb_end_step(MemberTable t) {
  FSL_MEMBER(t);
  end_step_body(d, g);
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
    put_phi(d, c, ph);
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

template <int Q, class ST>
__global__ void k_init_classes(Dev d, Geom g, Phys p) {
  using R = typename ST::R;
  const long long total = g.cells;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(g, (int)c, x, y, z);
    if (x >= g.nx) continue;
    const uint8_t fl = d.flags[c];
    if ((fl & F_TYPE) != T_IF) continue;
    d.flags[c] = (uint8_t)((fl & ~(F_NF | F_NE)) | iface_class<Q>(g, d.flags, x, y, z));
    d.kappa[c] = (p.sigma != 0.0) ? (double)curvature_any<R>(g, d.flags, phi_work<R>(d), x, y, z) : 0.0;
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
  static cudaError_t step(const Dev& d, const Geom& g, const Phys& p, cudaStream_t s,
                          const Aux& aux) {
    // the interface pass (its list was built by the previous step) beside the
    // bulk pass: disjoint cells written, same input buffer read
    cudaStream_t si = aux.side ? aux.side : s;
    cudaError_t e = cudaSuccess;
    if (aux.side) {
      e = cudaEventRecord(aux.fork, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(aux.side, aux.fork, 0);
      if (e != cudaSuccess) return e;
    }
    k_stream_collide_if<Q, ST><<<kCellListBlocks, 128, 0, si>>>(d, g, p);
    if (aux.side) {
      e = cudaEventRecord(aux.join, aux.side);
      if (e != cudaSuccess) return e;
    }
    e = pre_bulk(d, g, p, s);
    if (e == cudaSuccess) e = stream_collide(d, g, p, s);
    if (e == cudaSuccess && aux.side) e = cudaStreamWaitEvent(s, aux.join, 0);
    if (e != cudaSuccess) return e;
    e = convert(d, g, p, s);
    if (e != cudaSuccess) return e;
    if (g.bubbles) {
      e = bubble_update<Q>(d, g, p, 0, s);
      if (e != cudaSuccess) return e;
    }
    k_classify<Q, ST><<<kCellListBlocks, 128, 0, s>>>(d, g, p);
    k_end_step<<<kEndBlocks, 256, 0, s>>>(d, g);
    return cudaGetLastError();
  }
  // the conversion phase (k_convert), cooperative: at most four blocks per SM,
  // as many as fit
  static cudaError_t convert(const Dev& d, const Geom& g, const Phys& p, cudaStream_t s) {
    static int grid = 0;
    if (grid == 0) {
      int per_sm = 0, dev = 0, sms = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_convert<Q, ST>, 256, 0);
      if (e != cudaSuccess) return e;
      e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      if (per_sm < 1) return cudaErrorLaunchOutOfResources;
      grid = (per_sm < 4 ? per_sm : 4) * sms;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_convert<Q, ST>, d, g, p);
  }
  static cudaError_t init(const Dev& d, const Geom& g, const Phys& p, int cur, const double* u0,
                          int have_obst, double h_ref, cudaStream_t s) {
    const int blocks = 4 * 152;
    k_ctrl_reset<<<1, 32, 0, s>>>(d.ctrl, 0);
    k_init_types<<<blocks, 256, 0, s>>>(d, g, d.phinew, d.claim, have_obst);
    k_init_close<Q><<<blocks, 256, 0, s>>>(d, g);
    k_init_state<Q, ST><<<blocks, 256, 0, s>>>(d, g, p, cur, u0, h_ref);
    k_init_classes<Q, ST><<<blocks, 128, 0, s>>>(d, g, p);
    k_list_interface<<<blocks, 256, 0, s>>>(d, g);
    if (g.bubbles) return bubble_update<Q>(d, g, p, 1, s);
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
  // resolved bulk-kernel variant of the 16/32-bit path
  static int variant_of(const Geom& g) {
    constexpr bool half = sizeof(typename ST::T) == 2;
    if ((g.variant >= 1 && g.variant <= 4) || g.variant == 6 || g.variant == 8 || g.variant == 9 ||
        g.variant == 10 || g.variant == 12 || g.variant == 13 || g.variant == 14 || g.variant == 15)
      return g.variant;
    if ((g.variant == 5 || g.variant == 7 || g.variant == 11 || g.variant == 16) && half)
      return g.variant;
    return 2;
  }
  // variants that walk the list of liquid tiles of 256 cells
  static bool uses_tiles256(int v) {
    return v == 4 || v == 9 || v == 10 || v == 11 || v == 16;
  }
  // variants that walk the list of liquid segments of 64 cells
  static bool uses_segments64(int v) { return v == 6 || (v >= 12 && v <= 15); }
  // persistent TMA pipeline (one producer warp, four consumer warps) with NS
  // stages and at least MINB blocks per SM
  template <int NS, int MINB>
  static cudaError_t launch_tma(const Dev& d, const Geom& g, const Phys& p, cudaStream_t s) {
    static int grid = 0;
    constexpr size_t smem = BulkRing<Q, ST, NS>::bytes;
    if (grid == 0) {
      cudaError_t e = cudaFuncSetAttribute(k_stream_collide_bulk<Q, ST, NS, MINB>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int per_sm = 0, dev = 0, sms = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_bulk<Q, ST, NS, MINB>,
                                                        kBulkThreads, smem);
      if (e != cudaSuccess) return e;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      grid = (per_sm > 0 ? per_sm : 1) * sms;
    }
    const int ntx = (g.nx + kBulkTX - 1) / kBulkTX;
    k_stream_collide_bulk<Q, ST, NS, MINB><<<grid, kBulkThreads, smem, s>>>(d, g, p, ntx);
    return cudaGetLastError();
  }
  // persistent cp.async pipeline with S stages and at least MINB blocks per SM
  template <int S, int MINB>
  static cudaError_t launch_cpa(const Dev& d, const Geom& g, const Phys& p, cudaStream_t s) {
    static int grid = 0;
    constexpr size_t smem = CpRing<Q, ST, S>::bytes;
    if (grid == 0) {
      cudaError_t e = cudaFuncSetAttribute(k_stream_collide_cpa<Q, ST, S, MINB>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int per_sm = 0, dev = 0, sms = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_cpa<Q, ST, S, MINB>,
                                                        kCpThreads, smem);
      if (e != cudaSuccess) return e;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      grid = (per_sm > 0 ? per_sm : 1) * sms;
    }
    const int ntx = (g.nx + kBulkTX - 1) / kBulkTX;
    k_stream_collide_cpa<Q, ST, S, MINB><<<grid, kCpThreads, smem, s>>>(d, g, p, ntx);
    return cudaGetLastError();
  }
  static cudaError_t pre_bulk(const Dev& d, const Geom& g, const Phys&, cudaStream_t s) {
    if constexpr (ST::kShift) {
      if (uses_tiles256(variant_of(g))) {
        const int ntx = (g.nx + kBulkTX - 1) / kBulkTX;
        const long long ntiles = (long long)ntx * g.ny * g.nz;
        k_tiles<kBulkTX><<<(unsigned)((ntiles + 255) / 256), 256, 0, s>>>(d, g, ntx);
        return cudaGetLastError();
      }
      if (uses_segments64(variant_of(g))) {
        const int ntx = (g.nx + kWarpTX - 1) / kWarpTX;
        const long long ntiles = (long long)ntx * g.ny * g.nz;
        k_tiles<kWarpTX><<<(unsigned)((ntiles + 255) / 256), 256, 0, s>>>(d, g, ntx);
        return cudaGetLastError();
      }
    }
    return cudaSuccess;
  }
  static cudaError_t stream_collide(const Dev& d, const Geom& g, const Phys& p, cudaStream_t s) {
    if constexpr (ST::kShift) {
      const int v = variant_of(g);
      constexpr bool half = sizeof(typename ST::T) == 2;
      if (v == 16) {
        if constexpr (half) return launch_tma<3, 4>(d, g, p, s);
      }
      if (v == 14 || v == 15) {
        static int grid14 = 0, grid15 = 0;
        int& grid = v == 14 ? grid14 : grid15;
        if (grid == 0) {
          int per_sm = 0, dev = 0, sms = 0;
          cudaError_t e = v == 14
              ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_c1<Q, ST, 8>, 128, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_c1<Q, ST, 6>, 128, 0);
          if (e != cudaSuccess) return e;
          cudaGetDevice(&dev);
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
          grid = (per_sm > 0 ? per_sm : 1) * sms;
        }
        const int ntx = (g.nx + kWarpTX - 1) / kWarpTX;
        if (v == 14) k_stream_collide_c1<Q, ST, 8><<<grid, 128, 0, s>>>(d, g, p, ntx);
        else k_stream_collide_c1<Q, ST, 6><<<grid, 128, 0, s>>>(d, g, p, ntx);
        return cudaGetLastError();
      }
      if (v == 12 || v == 13) {
        // persistent warps over the 64-cell segment list: as many blocks as fit
        static int grid12 = 0, grid13 = 0;
        int& grid = v == 12 ? grid12 : grid13;
        if (grid == 0) {
          int per_sm = 0, dev = 0, sms = 0;
          cudaError_t e = v == 12
              ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_seg<Q, ST, 5>, 128, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_seg<Q, ST, 4>, 128, 0);
          if (e != cudaSuccess) return e;
          cudaGetDevice(&dev);
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
          grid = (per_sm > 0 ? per_sm : 1) * sms;
        }
        const int ntx = (g.nx + kWarpTX - 1) / kWarpTX;
        if (v == 12) k_stream_collide_seg<Q, ST, 5><<<grid, 128, 0, s>>>(d, g, p, ntx);
        else k_stream_collide_seg<Q, ST, 4><<<grid, 128, 0, s>>>(d, g, p, ntx);
        return cudaGetLastError();
      }
      if constexpr (half) {
        if (v == 9) return launch_cpa<2, 6>(d, g, p, s);
        if (v == 10) return launch_cpa<3, 4>(d, g, p, s);
        if (v == 11) return launch_cpa<2, 7>(d, g, p, s);
      } else {
        if (v == 9) return launch_cpa<2, 3>(d, g, p, s);
        if (v == 10) return launch_cpa<3, 2>(d, g, p, s);
      }
      if (v == 4) {
        if constexpr (half) return launch_tma<4, 3>(d, g, p, s);
        else return launch_tma<3, 3>(d, g, p, s);
      } else if (v == 6) {
        static int grid = 0;
        constexpr size_t smem = WarpRing<Q, ST>::bytes;
        if (grid == 0) {
          cudaError_t e = cudaFuncSetAttribute(k_stream_collide_wtma<Q, ST>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
          if (e != cudaSuccess) return e;
          int per_sm = 0, dev = 0, sms = 0;
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream_collide_wtma<Q, ST>,
                                                            32 * kWarpsPerBlock, smem);
          if (e != cudaSuccess) return e;
          cudaGetDevice(&dev);
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
          grid = (per_sm > 0 ? per_sm : 1) * sms;
        }
        const int ntx = (g.nx + kWarpTX - 1) / kWarpTX;
        k_stream_collide_wtma<Q, ST><<<grid, 32 * kWarpsPerBlock, smem, s>>>(d, g, p, ntx);
      } else if (v == 7) {
        if constexpr (sizeof(typename ST::T) == 2) {
          // rows split among about 3 blocks per SM x 152 SMs x 2 waves
          const int tx = (g.nx + 255) / 256;
          const int nrows = g.ny * g.nz;
          int G = (152 * 3 * 2 + tx - 1) / tx;
          if (G > nrows) G = nrows;
          dim3 b1(128), g1(tx, G, 1);
          k_stream_collide_pp<Q, ST><<<g1, b1, 0, s>>>(d, g, p);
        }
      } else if (v == 5) {
        if constexpr (sizeof(typename ST::T) == 2) {
          dim3 b1(64), g1((g.nx + 255) / 256, g.ny, g.nz);
          k_stream_collide_lp4<Q, ST><<<g1, b1, 0, s>>>(d, g, p);
        }
      } else {
        // 128 threads, two cells each: rows of up to 256 cells take one warp
        // row per 64 cells, and narrower domains stack rows in the block
        const int half = (g.nx + 1) / 2;
        const int bx = half >= 128 ? 128 : ((half + 31) / 32) * 32;
        const int by = 128 / bx;
        dim3 b1(bx, by), g1((g.nx + 2 * bx - 1) / (2 * bx), (g.ny + by - 1) / by, g.nz);
        if (v == 1)
          k_stream_collide_lp<Q, ST, 128, 4, true><<<g1, b1, 0, s>>>(d, g, p);
        else if (v == 2)
          k_stream_collide_lp<Q, ST, 128, 4, false><<<g1, b1, 0, s>>>(d, g, p);
        else if (v == 3)
          k_stream_collide_lp<Q, ST, 128, 5, true><<<g1, b1, 0, s>>>(d, g, p);
        else
          k_stream_collide_lp<Q, ST, 128, 6, true><<<g1, b1, 0, s>>>(d, g, p);
      }
    } else {
      dim3 b1(128), g1((g.nx + 127) / 128, g.ny, g.nz);
      k_stream_collide<Q, ST><<<g1, b1, 0, s>>>(d, g, p);
    }
    return cudaGetLastError();
  }
  // kernels of one step: interface pass, bulk pass (plus the tile list of
  // the list-driven variants), conversion phase, classify, end of step; six
  // more with the bubble model
  static int launches(const Geom& g) {
    const int bub = g.bubbles ? 6 : 0;
    if constexpr (ST::kShift)
      return ((uses_tiles256(variant_of(g)) || uses_segments64(variant_of(g))) ? 6 : 5) + bub;
    return 5 + bub;
  }
  // One step of n members of this lattice and storage, each kernel launched
  // once for all of them (blockIdx.y = member).  The bulk pass is the
  // segment-list kernel whatever variant a member selected (all variants give
  // the same bits).  16/32-bit storages only; FP64 batches step their members
  // one by one.
  static cudaError_t batch_step(const MemberTable& t, int n, const BatchGrid& bg, cudaStream_t s) {
    if constexpr (ST::kShift) {
      const unsigned m = (unsigned)n;
      kb_stream_collide_if<Q, ST><<<dim3(16, m), 128, 0, s>>>(t);
      kb_tiles<kWarpTX><<<dim3((unsigned)bg.tiles, m), 256, 0, s>>>(t);
      kb_stream_collide_seg<Q, ST><<<dim3(32, m), 128, 0, s>>>(t);
      kb_fill<Q><<<dim3(4, m), 256, 0, s>>>(t);
      kb_empty<Q, ST><<<dim3(4, m), 256, 0, s>>>(t);
      kb_finalise_share<Q><<<dim3(4, m), 256, 0, s>>>(t);
      kb_refill<Q, ST><<<dim3(8, m), 128, 0, s>>>(t);
      kb_excess_gather<Q><<<dim3(4, m), 256, 0, s>>>(t);
      kb_classify<Q, ST><<<dim3(16, m), 128, 0, s>>>(t);
      kb_end_step<<<dim3(kEndBlocks, m), 256, 0, s>>>(t);
      return cudaGetLastError();
    } else {
      (void)t; (void)n; (void)bg; (void)s;
      return cudaErrorNotSupported;
    }
  }
  static const Launch* table() {
    static const Launch L = {&step, &init, &total_mass, &max_velocity, &export_pdf,
                             &pre_bulk, &stream_collide, &launches, &batch_step};
    return &L;
  }
};

}  // namespace fsl
