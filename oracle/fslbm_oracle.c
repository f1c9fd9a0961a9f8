/*
 * Plain FP64 CPU oracle of one free-surface lattice Boltzmann (FSLBM) time step
 * with the five refilling schemes of "Comparison of refilling schemes in the
 * free-surface lattice Boltzmann method" (Schwarzmeier & Ruede, arXiv 2207.14496).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg load it.  It shares no code, header, table or helper with the CUDA
 * library: every lattice table and every formula below is written out here
 * from the paper's equations.
 *
 * Style: slow, sequential loops in the paper's order and notation.  Sums run
 * over lattice directions i = 0..q-1 (or over cells in index order) exactly as
 * written; nothing is fused, blocked or reordered.  Compile with
 * -ffp-contract=off so that a*b+c is never contracted into an FMA.
 *
 * Threads: the per-cell loops whose iteration x writes only cell x's own
 * values and reads nothing that the loop writes (classes, stream/collide,
 * refilling, finalising conversions, the excess-mass gather, curvature, and
 * plain copies) may run on several OpenMP
 * threads (orc_set_threads); every cell's arithmetic is the same in any
 * order, so the results are bit for bit those of one thread.  Loops that
 * write neighbours (conversion), sum across cells (lost mass, bubble sums,
 * observables) or search (bubble labels) always run sequentially.
 *
 * Sections of the paper followed:
 *   Sec. 2.1  collision (Eq. nm-lbm-collision), streaming (Eq. nm-lbm-streaming),
 *             SRT operator (Eq. nm-lbm-collision-operator, read as relaxation
 *             towards f^eq), equilibrium (Eq. nm-lbm-equilibrium), density and
 *             velocity moments (Eqs. nm-lbm-density, nm-lbm-velocity),
 *             viscosity (Eq. nm-lbm-viscosity), Guo forcing (Eq. nm-lbm-force-guo),
 *             bounce-back no-slip walls.
 *   Sec. 2.2  cell types and fill level, cell mass (Eq. nm-fslbm-mass), mass flux
 *             (Eq. nm-fslbm-mass-flux) with the unnecessary-interface treatment of
 *             Thuerey, conversion thresholds, excess mass (Eq. nm-fslbm-excess-mass),
 *             free-surface boundary condition (Eq. nm-fslbm-boundary-condition),
 *             gas and Laplace pressure (Eqs. nm-fslbm-pressure-gas, -laplace),
 *             curvature kappa = -div(n_hat), Parker-Youngs normal.
 *             With the bubble model (option 16): volume pressure per enclosed
 *             gas region (Eq. nm-fslbm-pressure-volume), regions merging and
 *             splitting.
 *   Sec. 3.1  refilling: EQ, EQ+NEQ, GEQ, EXT, AVG.
 *   Sec. 3.2  mass neutrality of refilling (Eq. rs-mass-change).
 *
 * Readings where the paper is silent or garbled (each one is listed with its
 * reason in the design notes of the repository):
 *   R1  step order: classify, stream/collide/flux, convert (fill then empty),
 *       refill, excess mass, normals/curvature.
 *   R2  c_s^2 = 1/3 (the printed sqrt(1/3) is a typo; p0 = c_s^2 rho0 = 1/3).
 *   R3  excess-mass receivers: stencil neighbours that are interface after
 *       refilling (new ones included); no receiver -> lost-mass accumulator.
 *   R4  gas density rho_G = 3 (p_V + sigma K), K = -div(n_hat), n = grad(phi).
 *   R5  Thuerey flux: a cell without liquid neighbours (NF) may only lose mass
 *       to interface neighbours, a cell without gas neighbours (NE) may only
 *       gain; same-class pairs use the plain bracket.
 *   R6  conflicting conversions: filling wins (a to-gas cell next to a
 *       to-liquid cell stays interface).
 *   R7  "surrounding" = stencil neighbours of the velocity set, plain means.
 *   R8  EQ+NEQ non-equilibrium: f_i(y) - f_i^eq(rho_y, u_y) of the neighbour y.
 *   R9  GEQ coefficient w_i rho / (2 c_s^2 omega) (dimensionally consistent
 *       Grad/Chapman-Enskog form; printed nu read as omega).
 *   R10 TRT with lambda_e = omega and magic parameter Lambda; D3Q27 standard
 *       weights.
 *   R11 Parker-Youngs weights 4/2/1 over the 3x3 perpendicular block, /32;
 *       an axis whose block touches an obstacle falls back to a one-sided or
 *       central two-point difference over non-obstacle cells.
 *   R12 hydrostatic initial density, linear: rho = 1 + 3 g_a (x_a - h_ref).
 *   R16 plain IEEE round-to-nearest FP64, no contraction.
 *   R23 bubbles: face-connected regions of gas and interface cells (option
 *       32: gas cells alone, interface cells attached), K = p V carried
 *       through merges (added) and splits (shared by volume); volumes and
 *       shares of K summed in FP64 in cell order.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_GAS 0
#define ORC_IFACE 1
#define ORC_LIQUID 2
#define ORC_OBST 3

#define ORC_REFILL_EQ 0
#define ORC_REFILL_EQ_NEQ 1
#define ORC_REFILL_GEQ 2
#define ORC_REFILL_EXT 3
#define ORC_REFILL_AVG 4

#define ORC_OPT_SIMPLE_FLUX 1u       /* plain Eq. nm-fslbm-mass-flux, no Thuerey */
#define ORC_OPT_GEQ_LITERAL_NU 2u    /* GEQ coefficient 1/(2 c_s^2 nu) as printed */
#define ORC_OPT_NEQ_LITERAL_MEAN 4u  /* f^neq = f(y) - f^eq(rho_bar, u_bar) as printed */
#define ORC_OPT_LAPLACE_LITERAL 8u   /* p_G = p_V - 2 sigma kappa, kappa = -div n_hat */
#define ORC_OPT_BUBBLES 16u          /* volume pressure per enclosed gas region (bubble model) */
#define ORC_OPT_BUBBLE_GAS_ONLY 32u  /* bubbles from gas cells alone (interface cells attached) */

#define CLS_STD 0
#define CLS_NF 1 /* interface cell without liquid neighbour */
#define CLS_NE 2 /* interface cell without gas neighbour */

typedef struct {
  int q;         /* 19 or 27 */
  int trt;       /* 0: SRT, 1: TRT */
  double magic;  /* TRT magic parameter Lambda */
  int refill;    /* ORC_REFILL_* */
  int nx, ny, nz;
  int periodic[3]; /* 1: periodic axis, 0: no-slip walls on both faces */
  double nu;
  double g[3];
  double sigma;
  double p_v;    /* volume (atmospheric) pressure, 1/3 */
  double eps;    /* conversion threshold epsilon_phi */
  unsigned options;
  double les_cs;   /* Smagorinsky constant C_S (Sec. 2.1); 0 = no turbulence model */
  int free_slip[3]; /* non-periodic axis: 1 = free-slip (specular) walls instead of no-slip */
} orc_config;

typedef struct {
  orc_config c;
  int q;
  int cx[27], cy[27], cz[27], opp[27];
  int mirror[27][8]; /* direction with the components in mask (bit a = axis a) negated */
  double w[27];
  long N;
  double tau, omega, lam_e, lam_o;
  unsigned char *type;
  double *f;    /* post-collision PDFs f*(x,t), layout f[i*N + x] */
  double *fn;   /* post-collision PDFs f*(x,t+1) being built */
  double *m, *phi, *rho, *kappa;
  double *phi_t; /* fill levels at time t, read by the mass flux of neighbours */
  double lost;
  long step;
  long unstable_step; /* first step at which |u| >= c_s or a NaN appeared, -1 if none */
  /* per-step scratch */
  unsigned char *cls, *to_liq, *to_gas, *is_new, *conv;
  double *mex, *share;
  int *nr;
  long n_fill, n_empty, n_new;  /* conversion counts of the last step */
  /* bubble model: label (root cell index, -1 none) of every gas and
   * interface cell, the invariant K = p V of every bubble (kept at its root
   * cell), the volume pressure seen by every interface cell; scratch */
  long *blab, *bnew, *bqueue;
  double *bK, *bp;
  double *bKnew, *bV, *bVseen; /* per-bubble sums, kept at the root cell */
  unsigned char *bhas;
} orc_state;

/* ---------------------------------------------------------------- lattice */

/* Direction order: rest, 6 faces, 12 edges, 8 corners; opposite pairs are
 * (1,2), (3,4), ...: opp(i) = i+1 for odd i, i-1 for even i > 0.  D3Q19 is the
 * first 19 directions of D3Q27. */
static const int DIRS[27][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
    {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
    {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};

static void setup_lattice(orc_state *s) {
  int q = s->c.q;
  s->q = q;
  for (int i = 0; i < q; ++i)
    for (int m = 0; m < 8; ++m) {
      int c[3] = {DIRS[i][0], DIRS[i][1], DIRS[i][2]};
      for (int a = 0; a < 3; ++a)
        if (m & (1 << a)) c[a] = -c[a];
      s->mirror[i][m] = -1;
      for (int j = 0; j < q; ++j)
        if (DIRS[j][0] == c[0] && DIRS[j][1] == c[1] && DIRS[j][2] == c[2]) s->mirror[i][m] = j;
    }
  for (int i = 0; i < q; ++i) {
    s->cx[i] = DIRS[i][0];
    s->cy[i] = DIRS[i][1];
    s->cz[i] = DIRS[i][2];
    s->opp[i] = (i == 0) ? 0 : ((i % 2 == 1) ? i + 1 : i - 1);
    int len2 = DIRS[i][0] * DIRS[i][0] + DIRS[i][1] * DIRS[i][1] + DIRS[i][2] * DIRS[i][2];
    if (q == 19) {
      /* Krueger et al., Table 3.3: 1/3, 1/18, 1/36 */
      s->w[i] = (len2 == 0) ? 1.0 / 3.0 : (len2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
    } else {
      /* D3Q27: 8/27, 2/27, 1/54, 1/216 */
      s->w[i] = (len2 == 0) ? 8.0 / 27.0 : (len2 == 1) ? 2.0 / 27.0 : (len2 == 2) ? 1.0 / 54.0 : 1.0 / 216.0;
    }
  }
}

/* ------------------------------------------------------------ geometry */

static long cell_index(const orc_state *s, long i, long j, long k) {
  const orc_config *c = &s->c;
  long n[3] = {c->nx, c->ny, c->nz};
  long p[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    if (p[a] < 0 || p[a] >= n[a]) {
      if (!c->periodic[a]) return -1; /* outside a wall: obstacle */
      p[a] = ((p[a] % n[a]) + n[a]) % n[a];
    }
  }
  return p[0] + n[0] * (p[1] + n[1] * p[2]);
}

static void cell_coords(const orc_state *s, long x, long *i, long *j, long *k) {
  *i = x % s->c.nx;
  *j = (x / s->c.nx) % s->c.ny;
  *k = x / ((long)s->c.nx * s->c.ny);
}

/* neighbour of cell x displaced by mult * c_d; -1 outside a wall */
static long neighbour(const orc_state *s, long x, int d, int mult) {
  long i, j, k;
  cell_coords(s, x, &i, &j, &k);
  return cell_index(s, i + mult * s->cx[d], j + mult * s->cy[d], k + mult * s->cz[d]);
}

static int type_of(const orc_state *s, long x) { return x < 0 ? ORC_OBST : s->type[x]; }

/* Where the PDF f_i arriving at cell x comes from.  Normally the cell x - c_i
 * with direction i.  Across free-slip walls (Sec. 2.1: specular reflection,
 * the wall-normal velocity component reversed) the PDF left the cell x - c_i
 * with the crossed components removed, in the mirrored direction.  Returns
 * -1 for a no-slip wall or an obstacle (halfway bounce-back), else the source
 * cell, with *dir its direction. */
static long pdf_source(const orc_state *s, long x, int i, int *dir) {
  long p0, p1, p2;
  cell_coords(s, x, &p0, &p1, &p2);
  long p[3] = {p0, p1, p2};
  long n[3] = {s->c.nx, s->c.ny, s->c.nz};
  int c[3] = {s->cx[i], s->cy[i], s->cz[i]};
  int crossed = 0;
  long q[3];
  for (int a = 0; a < 3; ++a) {
    q[a] = p[a] - c[a];
    if ((q[a] < 0 || q[a] >= n[a]) && !s->c.periodic[a]) crossed |= 1 << a;
  }
  *dir = i;
  if (crossed) {
    for (int a = 0; a < 3; ++a)
      if ((crossed & (1 << a)) && !s->c.free_slip[a]) return -1;
    for (int a = 0; a < 3; ++a)
      if (crossed & (1 << a)) q[a] = p[a];
    *dir = s->mirror[i][crossed];
  }
  long y = cell_index(s, q[0], q[1], q[2]);
  if (y >= 0 && s->type[y] == ORC_OBST) return -1;
  return y;
}
static int is_fluid_type(int t) { return t == ORC_LIQUID || t == ORC_IFACE; }

/* ------------------------------------------------------------ LBM pieces */

/* Eq. nm-lbm-equilibrium with c_s^2 = 1/3: 1/c_s^2 = 3, 1/(2 c_s^4) = 4.5,
 * 1/(2 c_s^2) = 1.5 */
static double feq(const orc_state *s, int i, double rho, double ux, double uy, double uz) {
  double cu = s->cx[i] * ux + s->cy[i] * uy + s->cz[i] * uz;
  double usq = ux * ux + uy * uy + uz * uz;
  return s->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
}

/* Guo force term of Eq. nm-lbm-force-guo without its (1 - 1/(2 tau)) prefactor:
 * w_i [ (c_i - u)/c_s^2 + (c_i.u) c_i / c_s^4 ] . F */
static double guo(const orc_state *s, int i, double ux, double uy, double uz, double Fx, double Fy,
                  double Fz) {
  double cu = s->cx[i] * ux + s->cy[i] * uy + s->cz[i] * uz;
  double cF = s->cx[i] * Fx + s->cy[i] * Fy + s->cz[i] * Fz;
  return s->w[i] * (3.0 * ((s->cx[i] - ux) * Fx + (s->cy[i] - uy) * Fy + (s->cz[i] - uz) * Fz) +
                    9.0 * cu * cF);
}

/* Moments of stored post-collision PDFs: rho = sum f*, and since sum c f* =
 * rho u + F/2 with F = rho g (both SRT and TRT with Guo forcing),
 * u = sum c f* / rho - g/2. */
static void stored_moments(const orc_state *s, const double *f, long x, double *rho, double *u) {
  const long N = s->N;
  double r = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
  for (int i = 0; i < s->q; ++i) r += f[i * N + x];
  for (int i = 0; i < s->q; ++i) {
    double fi = f[i * N + x];
    jx += s->cx[i] * fi;
    jy += s->cy[i] * fi;
    jz += s->cz[i] * fi;
  }
  *rho = r;
  u[0] = jx / r - 0.5 * s->c.g[0];
  u[1] = jy / r - 0.5 * s->c.g[1];
  u[2] = jz / r - 0.5 * s->c.g[2];
}

/* --------------------------------------------------- normals and curvature */

/* Parker-Youngs normal n = grad(phi) at cell x (reading R11). */
static void normal_py(const orc_state *s, long x, double *n) {
  long i, j, k;
  cell_coords(s, x, &i, &j, &k);
  long p[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    if (b > c) { int t = b; b = c; c = t; }
    int touches_obstacle = 0;
    double sum = 0.0;
    for (int ob = -1; ob <= 1; ++ob) {
      for (int oc = -1; oc <= 1; ++oc) {
        long pp[3] = {p[0], p[1], p[2]}, pm[3] = {p[0], p[1], p[2]};
        pp[a] += 1; pm[a] -= 1;
        pp[b] += ob; pm[b] += ob;
        pp[c] += oc; pm[c] += oc;
        long yp = cell_index(s, pp[0], pp[1], pp[2]);
        long ym = cell_index(s, pm[0], pm[1], pm[2]);
        if (type_of(s, yp) == ORC_OBST || type_of(s, ym) == ORC_OBST) touches_obstacle = 1;
        double wgt = (ob == 0 ? 2.0 : 1.0) * (oc == 0 ? 2.0 : 1.0);
        if (!touches_obstacle) sum += wgt * (s->phi[yp] - s->phi[ym]);
      }
    }
    if (!touches_obstacle) {
      n[a] = sum / 32.0;
    } else {
      /* narrowed stencil: two-point differences along a over non-obstacle cells */
      long pp[3] = {p[0], p[1], p[2]}, pm[3] = {p[0], p[1], p[2]};
      pp[a] += 1; pm[a] -= 1;
      long yp = cell_index(s, pp[0], pp[1], pp[2]);
      long ym = cell_index(s, pm[0], pm[1], pm[2]);
      int okp = type_of(s, yp) != ORC_OBST, okm = type_of(s, ym) != ORC_OBST;
      if (okp && okm) n[a] = 0.5 * (s->phi[yp] - s->phi[ym]);
      else if (okp) n[a] = s->phi[yp] - s->phi[x];
      else if (okm) n[a] = s->phi[x] - s->phi[ym];
      else n[a] = 0.0;
    }
  }
}

static void unit_normal(const orc_state *s, long x, double *nh) {
  double n[3];
  normal_py(s, x, n);
  double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  if (len < 1e-12) {
    nh[0] = nh[1] = nh[2] = 0.0;
  } else {
    nh[0] = n[0] / len;
    nh[1] = n[1] / len;
    nh[2] = n[2] / len;
  }
}

/* K = -div(n_hat) by central differences of n_hat over the face neighbours;
 * a side that is an obstacle is replaced by the centre value (one-sided). */
static double curvature(const orc_state *s, long x) {
  long i, j, k;
  cell_coords(s, x, &i, &j, &k);
  long p[3] = {i, j, k};
  double nc[3];
  unit_normal(s, x, nc);
  double div = 0.0;
  for (int a = 0; a < 3; ++a) {
    long pp[3] = {p[0], p[1], p[2]}, pm[3] = {p[0], p[1], p[2]};
    pp[a] += 1; pm[a] -= 1;
    long yp = cell_index(s, pp[0], pp[1], pp[2]);
    long ym = cell_index(s, pm[0], pm[1], pm[2]);
    int okp = type_of(s, yp) != ORC_OBST, okm = type_of(s, ym) != ORC_OBST;
    double np[3], nm[3], d;
    if (okp && okm) {
      unit_normal(s, yp, np);
      unit_normal(s, ym, nm);
      d = 0.5 * (np[a] - nm[a]);
    } else if (okp) {
      unit_normal(s, yp, np);
      d = np[a] - nc[a];
    } else if (okm) {
      unit_normal(s, ym, nm);
      d = nc[a] - nm[a];
    } else {
      d = 0.0;
    }
    div += d;
  }
  return -div;
}

static void update_curvature(orc_state *s) {
#pragma omp parallel for schedule(static)
  for (long x = 0; x < s->N; ++x) s->kappa[x] = 0.0;
  if (s->c.sigma == 0.0) return;
#pragma omp parallel for schedule(static)
  for (long x = 0; x < s->N; ++x)
    if (s->type[x] == ORC_IFACE) s->kappa[x] = curvature(s, x);
}

/* ------------------------------------------------------------ lifecycle */

/* ------------------------------------------------------------ bubble model */

/* Sec. 2.2, Eq. nm-fslbm-pressure-volume: an enclosed gas volume (a bubble)
 * has the volume pressure p_V(t) = p_V(0) V(0) / V(t).  Bubbles merge and
 * split, so (reading R23) the invariant K = p V is carried per bubble:
 *  - bubbles are the connected components of gas and interface cells,
 *    connected through the 6 face neighbours (with periodic wrap); the
 *    label of a component is its smallest cell index.  Two bubbles merge
 *    when their interface layers touch, and a bubble splits only when a
 *    liquid cell separates its parts;
 *  - with ORC_OPT_BUBBLE_GAS_ONLY the components are those of gas cells
 *    alone, and an interface cell belongs to the bubble with the smallest
 *    label among its gas stencil neighbours (none: no bubble);
 *  - a bubble's volume is sum of w over its cells, w = 1 for gas and
 *    1 - phi for interface cells;
 *  - K of a new component = sum over old bubbles b of K_b times the share
 *    of b's volume (w of the cells labelled b before and now in this
 *    component, over all of b's cells still in a bubble): a bubble that only
 *    changed volume keeps its K, merged bubbles add their K (one common
 *    pressure), a split bubble divides its K in proportion to the volumes
 *    (each part keeps the pressure);
 *  - a component without any old cell starts with K = p_V V (the
 *    configuration's volume pressure), as every bubble does initially;
 *  - the volume pressure of an interface cell is K / V of its bubble.
 * Every sum is a plain FP64 sum over the cells in index order. */
static void bubble_update(orc_state *s, int first) {
  const long N = s->N;
  const int q = s->q;
  long *lab = s->bnew;
  for (long x = 0; x < N; ++x) lab[x] = -1;
  const int gas_only = (s->c.options & ORC_OPT_BUBBLE_GAS_ONLY) != 0;
  /* members: gas cells, and interface cells unless gas_only */
#define BUB_MEMBER(t) ((t) == ORC_GAS || (!gas_only && (t) == ORC_IFACE))
  /* components of members: breadth-first from the smallest unlabelled cell */
  for (long x = 0; x < N; ++x) {
    if (!BUB_MEMBER(s->type[x]) || lab[x] >= 0) continue;
    long head = 0, tail = 0;
    s->bqueue[tail++] = x;
    lab[x] = x;
    while (head < tail) {
      long y = s->bqueue[head++];
      for (int d = 1; d <= 6; ++d) {
        long n = neighbour(s, y, d, 1);
        if (n >= 0 && BUB_MEMBER(s->type[n]) && lab[n] < 0) {
          lab[n] = x;
          s->bqueue[tail++] = n;
        }
      }
    }
  }
#undef BUB_MEMBER
  /* gas_only: interface cells take the smallest label among gas stencil
   * neighbours */
  for (long x = 0; gas_only && x < N; ++x) {
    if (s->type[x] != ORC_IFACE) continue;
    long best = -1;
    for (int d = 1; d < q; ++d) {
      long n = neighbour(s, x, d, 1);
      if (n >= 0 && s->type[n] == ORC_GAS && (best < 0 || lab[n] < best)) best = lab[n];
    }
    lab[x] = best;
  }
  for (long x = 0; x < N; ++x) {
    s->bV[x] = 0.0;
    s->bVseen[x] = 0.0;
    s->bKnew[x] = 0.0;
    s->bhas[x] = 0;
  }
  for (long x = 0; x < N; ++x) {
    if (lab[x] < 0) continue;
    double w = s->type[x] == ORC_GAS ? 1.0 : 1.0 - s->phi[x];
    s->bV[lab[x]] += w;
    if (!first && s->blab[x] >= 0) s->bVseen[s->blab[x]] += w;
  }
  if (!first) {
    for (long x = 0; x < N; ++x) {
      long b = s->blab[x], r = lab[x];
      if (r < 0 || b < 0 || s->bVseen[b] == 0.0) continue;
      double w = s->type[x] == ORC_GAS ? 1.0 : 1.0 - s->phi[x];
      s->bKnew[r] += s->bK[b] * (w / s->bVseen[b]);
      s->bhas[r] = 1;
    }
  }
  for (long x = 0; x < N; ++x) {
    long r = lab[x];
    s->blab[x] = r;
    double V = (r >= 0) ? s->bV[r] : 0.0;
    if (r == x) s->bK[x] = s->bhas[x] ? s->bKnew[x] : s->c.p_v * V;
    else s->bK[x] = 0.0;
  }
  for (long x = 0; x < N; ++x) {
    long r = s->blab[x];
    double V = (r >= 0) ? s->bV[r] : 0.0;
    s->bp[x] = (r >= 0 && V != 0.0) ? s->bK[r] / V : s->c.p_v;
  }
}

void orc_destroy(orc_state *s);

orc_state *orc_create(const orc_config *cfg) {
  if (!cfg || (cfg->q != 19 && cfg->q != 27) || cfg->nx <= 0 || cfg->ny <= 0 || cfg->nz <= 0 ||
      cfg->refill < 0 || cfg->refill > 4 || !(cfg->nu > 0.0))
    return NULL;
  orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
  if (!s) return NULL;
  s->c = *cfg;
  setup_lattice(s);
  s->N = (long)cfg->nx * cfg->ny * cfg->nz;
  /* Eq. nm-lbm-viscosity: nu = c_s^2 (tau - 1/2) */
  s->tau = 3.0 * cfg->nu + 0.5;
  s->omega = 1.0 / s->tau;
  s->lam_e = s->omega;
  /* TRT: Lambda = (1/lam_e - 1/2)(1/lam_o - 1/2) */
  s->lam_o = 1.0 / (0.5 + cfg->magic / (1.0 / s->lam_e - 0.5));
  long N = s->N;
  int q = s->q;
  s->type = (unsigned char *)calloc(N, 1);
  s->f = (double *)calloc((size_t)q * N, sizeof(double));
  s->fn = (double *)calloc((size_t)q * N, sizeof(double));
  s->m = (double *)calloc(N, sizeof(double));
  s->phi = (double *)calloc(N, sizeof(double));
  s->rho = (double *)calloc(N, sizeof(double));
  s->kappa = (double *)calloc(N, sizeof(double));
  s->phi_t = (double *)calloc(N, sizeof(double));
  s->cls = (unsigned char *)calloc(N, 1);
  s->to_liq = (unsigned char *)calloc(N, 1);
  s->to_gas = (unsigned char *)calloc(N, 1);
  s->is_new = (unsigned char *)calloc(N, 1);
  s->conv = (unsigned char *)calloc(N, 1);
  s->mex = (double *)calloc(N, sizeof(double));
  s->share = (double *)calloc(N, sizeof(double));
  s->nr = (int *)calloc(N, sizeof(int));
  s->blab = (long *)calloc(N, sizeof(long));
  s->bnew = (long *)calloc(N, sizeof(long));
  s->bqueue = (long *)calloc(N, sizeof(long));
  s->bK = (double *)calloc(N, sizeof(double));
  s->bKnew = (double *)calloc(N, sizeof(double));
  s->bV = (double *)calloc(N, sizeof(double));
  s->bVseen = (double *)calloc(N, sizeof(double));
  s->bp = (double *)calloc(N, sizeof(double));
  s->bhas = (unsigned char *)calloc(N, 1);
  if (!s->type || !s->f || !s->fn || !s->m || !s->phi || !s->rho || !s->kappa || !s->phi_t || !s->cls ||
      !s->to_liq || !s->to_gas || !s->is_new || !s->conv || !s->mex || !s->share || !s->nr ||
      !s->blab || !s->bnew || !s->bqueue || !s->bK || !s->bKnew || !s->bV || !s->bVseen || !s->bp ||
      !s->bhas) {
    orc_destroy(s);
    return NULL;
  }
  s->unstable_step = -1;
  return s;
}

void orc_destroy(orc_state *s) {
  if (!s) return;
  free(s->type); free(s->f); free(s->fn); free(s->m); free(s->phi); free(s->rho);
  free(s->kappa); free(s->phi_t); free(s->cls); free(s->to_liq); free(s->to_gas); free(s->is_new);
  free(s->conv); free(s->mex); free(s->share); free(s->nr);
  free(s->blab); free(s->bnew); free(s->bqueue); free(s->bK); free(s->bKnew); free(s->bV);
  free(s->bVseen); free(s->bp); free(s->bhas);
  free(s);
}

/* Initial state (readings R12, R13): flags from the fill level, closed
 * interface layer, hydrostatic density, f* = f^eq(rho, u0), m = phi rho. */
int orc_init_fill(orc_state *s, const double *phi0, const double *u0, const unsigned char *obstacle,
                  double h_ref) {
  const long N = s->N;
  const int q = s->q;
  for (long x = 0; x < N; ++x) {
    if (obstacle && obstacle[x]) { s->type[x] = ORC_OBST; s->phi[x] = 0.0; }
    else if (phi0[x] >= 1.0) { s->type[x] = ORC_LIQUID; s->phi[x] = 1.0; }
    else if (phi0[x] <= 0.0) { s->type[x] = ORC_GAS; s->phi[x] = 0.0; }
    else { s->type[x] = ORC_IFACE; s->phi[x] = phi0[x]; }
  }
  /* a liquid cell touching gas becomes interface (closed layer), fill level kept */
  for (long x = 0; x < N; ++x) s->cls[x] = 0;
  for (long x = 0; x < N; ++x) {
    if (s->type[x] != ORC_LIQUID) continue;
    for (int d = 1; d < q; ++d)
      if (type_of(s, neighbour(s, x, d, 1)) == ORC_GAS) s->cls[x] = 1;
  }
  for (long x = 0; x < N; ++x) if (s->cls[x]) { s->type[x] = ORC_IFACE; s->cls[x] = 0; }

  int ga = -1;
  for (int a = 0; a < 3; ++a) if (s->c.g[a] != 0.0) ga = a;
  for (long x = 0; x < N; ++x) {
    long i, j, k;
    cell_coords(s, x, &i, &j, &k);
    double r = 1.0;
    if (ga >= 0 && !isnan(h_ref)) {
      long p[3] = {i, j, k};
      r = 1.0 + 3.0 * s->c.g[ga] * (((double)p[ga] + 0.5) - h_ref);
    }
    double ux = 0.0, uy = 0.0, uz = 0.0;
    if (u0) { ux = u0[3 * x + 0]; uy = u0[3 * x + 1]; uz = u0[3 * x + 2]; }
    if (is_fluid_type(s->type[x])) {
      for (int i2 = 0; i2 < q; ++i2) s->f[i2 * N + x] = feq(s, i2, r, ux, uy, uz);
      s->rho[x] = r;
      s->m[x] = (s->type[x] == ORC_LIQUID) ? r : s->phi[x] * r;
    } else {
      for (int i2 = 0; i2 < q; ++i2) s->f[i2 * N + x] = 0.0;
      s->rho[x] = 0.0;
      s->m[x] = 0.0;
    }
  }
  s->lost = 0.0;
  s->step = 0;
  s->unstable_step = -1;
  update_curvature(s);
  if (s->c.options & ORC_OPT_BUBBLES) bubble_update(s, 1);
  return 0;
}

/* ------------------------------------------------------------ refilling */

/* Sec. 3.1.  Writes the q refilled PDFs of new interface cell x into fn. */
static void refill_cell(orc_state *s, long x) {
  const long N = s->N;
  const int q = s->q;
  const double *fn = s->fn;
  /* valid neighbours: liquid or interface and not newly converted (R7) */
  int valid[27];
  long nbr[27];
  double nrho[27], nu_[27][3];
  int count = 0;
  double rsum = 0.0, usum[3] = {0.0, 0.0, 0.0};
  valid[0] = 0;
  nbr[0] = x;
  for (int d = 1; d < q; ++d) {
    long y = neighbour(s, x, d, 1);
    nbr[d] = y;
    valid[d] = (y >= 0 && is_fluid_type(s->type[y]) && !s->is_new[y]);
    if (valid[d]) {
      stored_moments(s, fn, y, &nrho[d], nu_[d]);
      rsum += nrho[d];
      usum[0] += nu_[d][0];
      usum[1] += nu_[d][1];
      usum[2] += nu_[d][2];
      count += 1;
    }
  }
  double out[27];
  /* count >= 1 always: the cell that filled and created x is a valid neighbour */
  double rb = rsum / (double)count;
  double ub[3] = {usum[0] / (double)count, usum[1] / (double)count, usum[2] / (double)count};
  int scheme = s->c.refill;

  /* direction best aligned with the interface normal, among valid ones */
  int dn = -1;
  if (scheme == ORC_REFILL_EQ_NEQ || scheme == ORC_REFILL_EXT) {
    double n[3];
    normal_py(s, x, n);
    double best = 0.0;
    for (int d = 1; d < q; ++d) {
      if (!valid[d]) continue;
      double dot = s->cx[d] * n[0] + s->cy[d] * n[1] + s->cz[d] * n[2];
      if (dn < 0 || dot > best) { dn = d; best = dot; }
    }
  }

  if (scheme == ORC_REFILL_EQ) {
    for (int i = 0; i < q; ++i) out[i] = feq(s, i, rb, ub[0], ub[1], ub[2]);
  } else if (scheme == ORC_REFILL_EQ_NEQ) {
    long y = nbr[dn];
    for (int i = 0; i < q; ++i) {
      double fe = feq(s, i, rb, ub[0], ub[1], ub[2]);
      double fneq;
      if (s->c.options & ORC_OPT_NEQ_LITERAL_MEAN)
        fneq = fn[i * N + y] - fe;
      else
        fneq = fn[i * N + y] - feq(s, i, nrho[dn], nu_[dn][0], nu_[dn][1], nu_[dn][2]);
      out[i] = fe + fneq;
    }
  } else if (scheme == ORC_REFILL_GEQ) {
    /* velocity derivatives du[a][b] = d u_a / d x_b */
    double du[3][3];
    for (int b = 0; b < 3; ++b) {
      /* face directions +e_b and -e_b are 1+2b and 2+2b */
      int dp = 1 + 2 * b, dm = 2 + 2 * b;
      for (int a = 0; a < 3; ++a) {
        if (valid[dp] && valid[dm]) du[a][b] = 0.5 * (nu_[dp][a] - nu_[dm][a]);
        else if (valid[dp]) du[a][b] = nu_[dp][a] - ub[a];
        else if (valid[dm]) du[a][b] = ub[a] - nu_[dm][a];
        else du[a][b] = 0.0;
      }
    }
    double coef;
    if (s->c.options & ORC_OPT_GEQ_LITERAL_NU) coef = 1.5 / s->c.nu;  /* 1/(2 c_s^2 nu) */
    else coef = 1.5 * s->tau;                                          /* 1/(2 c_s^2 omega) */
    for (int i = 0; i < q; ++i) {
      int c[3] = {s->cx[i], s->cy[i], s->cz[i]};
      double sum = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double S = du[a][b] + du[b][a];
          double Q = (a == b ? 1.0 / 3.0 : 0.0) - (double)(c[a] * c[b]);
          sum += S * Q;
        }
      out[i] = feq(s, i, rb, ub[0], ub[1], ub[2]) + s->w[i] * rb * coef * sum;
    }
  } else if (scheme == ORC_REFILL_EXT) {
    long y1 = neighbour(s, x, dn, 1), y2 = neighbour(s, x, dn, 2), y3 = neighbour(s, x, dn, 3);
    int k = 1; /* y1 is valid by construction of dn */
    int v2 = (y2 >= 0 && is_fluid_type(s->type[y2]) && !s->is_new[y2]);
    int v3 = (y3 >= 0 && is_fluid_type(s->type[y3]) && !s->is_new[y3]);
    if (v2) k = v3 ? 3 : 2;
    for (int i = 0; i < q; ++i) {
      if (k == 3) out[i] = 3.0 * fn[i * N + y1] - 3.0 * fn[i * N + y2] + fn[i * N + y3];
      else if (k == 2) out[i] = 2.0 * fn[i * N + y1] - fn[i * N + y2];
      else out[i] = fn[i * N + y1];
    }
  } else { /* AVG */
    for (int i = 0; i < q; ++i) {
      double sum = 0.0;
      for (int d = 1; d < q; ++d)
        if (valid[d]) sum += fn[i * N + nbr[d]];
      out[i] = sum / (double)count;
    }
  }
  for (int i = 0; i < q; ++i) s->fn[i * N + x] = out[i];
}

/* ------------------------------------------------------------ one step */

static void step_once(orc_state *s) {
  const long N = s->N;
  const int q = s->q;
  const double *g = s->c.g;
  const double eps = s->c.eps;
  const int thurey = !(s->c.options & ORC_OPT_SIMPLE_FLUX);

  /* 1. neighbourhood classes of interface cells from the flags at time t */
#pragma omp parallel for schedule(static)
  for (long x = 0; x < N; ++x) {
    s->cls[x] = CLS_STD;
    if (s->type[x] != ORC_IFACE) continue;
    int has_liq = 0, has_gas = 0;
    for (int d = 1; d < q; ++d) {
      int t = type_of(s, neighbour(s, x, d, 1));
      if (t == ORC_LIQUID) has_liq = 1;
      if (t == ORC_GAS) has_gas = 1;
    }
    if (!has_liq && has_gas) s->cls[x] = CLS_NF;
    else if (!has_gas && has_liq) s->cls[x] = CLS_NE;
  }

#pragma omp parallel for schedule(static)
  for (long x = 0; x < N; ++x) s->phi_t[x] = s->phi[x];

  int unstable = 0;
  /* 2. stream (pull), free-surface and wall boundaries, mass flux, collide */
#pragma omp parallel for schedule(dynamic, 256) reduction(| : unstable)
  for (long x = 0; x < N; ++x) {
    s->to_liq[x] = 0;
    s->to_gas[x] = 0;
    s->is_new[x] = 0;
    s->conv[x] = 0;
    if (!is_fluid_type(s->type[x])) continue;
    const int iface = (s->type[x] == ORC_IFACE);
    double fin[27];
    /* own velocity at time t for the free-surface boundary condition */
    double rho_t = 0.0, ut[3] = {0.0, 0.0, 0.0};
    double rho_g = 0.0;
    if (iface) {
      stored_moments(s, s->f, x, &rho_t, ut);
      double pg;
      /* Eq. nm-fslbm-pressure-volume: the bubble's volume pressure */
      double pv = (s->c.options & ORC_OPT_BUBBLES) ? s->bp[x] : s->c.p_v;
      if (s->c.options & ORC_OPT_LAPLACE_LITERAL) pg = pv - 2.0 * s->c.sigma * s->kappa[x];
      else pg = pv + s->c.sigma * s->kappa[x];
      rho_g = 3.0 * pg; /* rho_G = p_G / c_s^2 */
    }
    for (int i = 0; i < q; ++i) {
      int di;
      long y = pdf_source(s, x, i, &di); /* the PDF f_i arrives from x - c_i */
      int t = type_of(s, y);
      int io = s->opp[i];
      if (is_fluid_type(t)) {
        fin[i] = s->f[di * N + y];
      } else if (t == ORC_OBST) {
        fin[i] = s->f[io * N + x]; /* halfway bounce-back */
      } else {
        /* Eq. nm-fslbm-boundary-condition: anti-bounce-back at the free surface */
        fin[i] = feq(s, i, rho_g, ut[0], ut[1], ut[2]) + feq(s, io, rho_g, ut[0], ut[1], ut[2]) -
                 s->f[io * N + x];
      }
    }
    double m_new = s->m[x];
    if (iface) {
      /* Eq. nm-fslbm-mass-flux, summed as in Eq. rs-mass-change */
      double dm = 0.0;
      for (int i = 1; i < q; ++i) {
        /* the cell exchanging PDFs with x along c_i: x + c_i, or its mirror
         * image across a free-slip wall; f_in is what arrives from it */
        int io = s->opp[i], dj;
        long y = pdf_source(s, x, io, &dj);
        int t = type_of(s, y);
        double d = 0.0;
        if (t == ORC_LIQUID) {
          d = s->f[dj * N + y] - s->f[i * N + x];
        } else if (t == ORC_IFACE) {
          double f_in = s->f[dj * N + y], f_out = s->f[i * N + x];
          double br = f_in - f_out;
          if (thurey) {
            int cx_ = s->cls[x], cy_ = s->cls[y];
            if (cx_ == CLS_STD) br = (cy_ == CLS_NF) ? f_in : (cy_ == CLS_NE) ? -f_out : f_in - f_out;
            else if (cx_ == CLS_NF) br = (cy_ == CLS_NF) ? f_in - f_out : -f_out;
            else br = (cy_ == CLS_NE) ? f_in - f_out : f_in;
          }
          d = 0.5 * (s->phi_t[x] + s->phi_t[y]) * br;
        }
        dm += d;
      }
      m_new = s->m[x] + dm;
    }
    /* Eqs. nm-lbm-density, nm-lbm-velocity with F = rho g */
    double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int i = 0; i < q; ++i) rho += fin[i];
    for (int i = 0; i < q; ++i) {
      jx += s->cx[i] * fin[i];
      jy += s->cy[i] * fin[i];
      jz += s->cz[i] * fin[i];
    }
    double ux = jx / rho + 0.5 * g[0], uy = jy / rho + 0.5 * g[1], uz = jz / rho + 0.5 * g[2];
    double Fx = rho * g[0], Fy = rho * g[1], Fz = rho * g[2];
    double usq = ux * ux + uy * uy + uz * uz;
    if (!(usq < 1.0 / 3.0)) unstable = 1; /* |u| >= c_s, or NaN */
    double fe[27], fg[27];
    for (int i = 0; i < q; ++i) {
      fe[i] = feq(s, i, rho, ux, uy, uz);
      fg[i] = guo(s, i, ux, uy, uz, Fx, Fy, Fz);
    }
    double omega = s->omega, lam_e = s->lam_e, lam_o = s->lam_o;
    if (s->c.les_cs > 0.0) {
      /* Smagorinsky model (Sec. 2.1, Eqs. nm-lbm-turbulence-viscosity to
       * nm-lbm-turublence-relaxation-time): Q_ab = sum_i c_ia c_ib (f_i - f_i^eq),
       * Qbar = sqrt(2 sum_ab Q_ab Q_ab),
       * tau = tau0 + (sqrt(tau0^2 + 2 sqrt(2) C_S^2 Qbar / (rho c_s^4)) - tau0) / 2 */
      int c[27][3];
      for (int i = 0; i < q; ++i) { c[i][0] = s->cx[i]; c[i][1] = s->cy[i]; c[i][2] = s->cz[i]; }
      double qq = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double Qab = 0.0;
          for (int i = 0; i < q; ++i) Qab += (double)(c[i][a] * c[i][b]) * (fin[i] - fe[i]);
          qq += Qab * Qab;
        }
      double qbar = sqrt(2.0 * qq);
      double t0 = s->tau, cs = s->c.les_cs;
      double tau = t0 + 0.5 * (sqrt(t0 * t0 + 2.0 * sqrt(2.0) * cs * cs * qbar * 9.0 / rho) - t0);
      omega = 1.0 / tau;
      lam_e = omega;
      lam_o = 1.0 / (0.5 + s->c.magic / (1.0 / lam_e - 0.5));
    }
    if (!s->c.trt) {
      /* SRT: f* = f - omega (f - f^eq) + (1 - omega/2) F_i */
      double om = omega, pre = 1.0 - 0.5 * omega;
      for (int i = 0; i < q; ++i) s->fn[i * N + x] = fin[i] - om * (fin[i] - fe[i]) + pre * fg[i];
    } else {
      /* TRT: symmetric parts relax with lam_e, antisymmetric with lam_o */
      double le = lam_e, lo = lam_o;
      double pe = 1.0 - 0.5 * le, po = 1.0 - 0.5 * lo;
      s->fn[x] = fin[0] - le * (fin[0] - fe[0]) + pe * fg[0];
      for (int i = 1; i < q; i += 2) {
        int io = i + 1;
        double fp = 0.5 * (fin[i] + fin[io]), fm = 0.5 * (fin[i] - fin[io]);
        double ep = 0.5 * (fe[i] + fe[io]), em = 0.5 * (fe[i] - fe[io]);
        double gp = 0.5 * (fg[i] + fg[io]), gm = 0.5 * (fg[i] - fg[io]);
        s->fn[i * N + x] = fin[i] - le * (fp - ep) - lo * (fm - em) + pe * gp + po * gm;
        s->fn[io * N + x] = fin[io] - le * (fp - ep) + lo * (fm - em) + pe * gp - po * gm;
      }
    }
    s->rho[x] = rho;
    if (iface) {
      s->m[x] = m_new;
      s->phi[x] = m_new / rho; /* Eq. nm-fslbm-mass */
      if (s->phi[x] > 1.0 + eps) s->to_liq[x] = 1;
      else if (s->phi[x] < 0.0 - eps) s->to_gas[x] = 1;
    } else {
      s->m[x] = rho;
      s->phi[x] = 1.0;
    }
  }

  /* 3. conversion, sub-pass 1 (fill): gas neighbours of filled cells become new
   * interface cells; a neighbour about to empty is kept (R6) */
  long n_fill = 0, n_empty = 0, n_new = 0;
  for (long x = 0; x < N; ++x) {
    if (!s->to_liq[x]) continue;
    for (int d = 1; d < q; ++d) {
      long y = neighbour(s, x, d, 1);
      if (y < 0) continue;
      if (s->type[y] == ORC_GAS) {
        s->type[y] = ORC_IFACE;
        s->is_new[y] = 1;
        s->phi[y] = 0.0;
        s->m[y] = 0.0;
      }
      s->to_gas[y] = 0;
    }
  }
  /* sub-pass 2 (empty): liquid neighbours of emptied cells become interface */
  for (long x = 0; x < N; ++x) {
    if (!s->to_gas[x]) continue;
    for (int d = 1; d < q; ++d) {
      long y = neighbour(s, x, d, 1);
      if (y < 0) continue;
      if (s->type[y] == ORC_LIQUID) {
        s->type[y] = ORC_IFACE;
        s->phi[y] = 1.0;
        s->m[y] = s->rho[y];
      }
    }
  }
  /* finalise: Eq. nm-fslbm-excess-mass */
#pragma omp parallel for schedule(static) reduction(+ : n_fill, n_empty)
  for (long x = 0; x < N; ++x) {
    if (s->to_liq[x]) {
      s->mex[x] = (s->phi[x] - 1.0) * s->rho[x];
      s->type[x] = ORC_LIQUID;
      s->phi[x] = 1.0;
      s->m[x] = s->rho[x];
      s->conv[x] = 1;
      n_fill++;
    } else if (s->to_gas[x]) {
      s->mex[x] = s->phi[x] * s->rho[x];
      s->type[x] = ORC_GAS;
      s->phi[x] = 0.0;
      s->m[x] = 0.0;
      s->conv[x] = 1;
      n_empty++;
    }
  }

  /* 4. refill new interface cells from their valid neighbours (Sec. 3.1);
   * a refilled cell reads only valid (not new) neighbours */
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : n_new)
  for (long x = 0; x < N; ++x) {
    if (!s->is_new[x]) continue;
    refill_cell(s, x);
    n_new++;
  }
#pragma omp parallel for schedule(static)
  for (long x = 0; x < N; ++x) {
    if (!s->is_new[x]) continue;
    double r = 0.0;
    for (int i = 0; i < q; ++i) r += s->fn[i * N + x];
    s->rho[x] = r;
  }

  /* 5. excess mass spread evenly over interface neighbours (R3) */
  for (long x = 0; x < N; ++x) {
    if (!s->conv[x]) continue;
    int n_r = 0;
    for (int d = 1; d < q; ++d)
      if (type_of(s, neighbour(s, x, d, 1)) == ORC_IFACE) n_r++;
    s->nr[x] = n_r;
    if (n_r == 0) {
      s->lost += s->mex[x];
      s->share[x] = 0.0;
    } else {
      s->share[x] = s->mex[x] / (double)n_r;
    }
  }
#pragma omp parallel for schedule(static)
  for (long x = 0; x < N; ++x) {
    if (s->type[x] != ORC_IFACE) continue;
    int got = 0;
    double sum = 0.0;
    for (int d = 1; d < q; ++d) {
      long y = neighbour(s, x, d, 1);
      if (y >= 0 && s->conv[y] && s->nr[y] > 0) { sum += s->share[y]; got = 1; }
    }
    if (got) {
      s->m[x] = s->m[x] + sum;
      s->phi[x] = s->m[x] / s->rho[x];
    }
  }

  /* swap PDF buffers: fn now holds f*(t+1) */
  double *tmp = s->f;
  s->f = s->fn;
  s->fn = tmp;

  /* 6. curvature and (bubble model) volume pressure for the next step's gas density */
  update_curvature(s);
  if (s->c.options & ORC_OPT_BUBBLES) bubble_update(s, 0);

  s->step += 1;
  if (unstable && s->unstable_step < 0) s->unstable_step = s->step;
  s->n_fill = n_fill;
  s->n_empty = n_empty;
  s->n_new = n_new;
}

/* Threads for the order-free per-cell loops (1 = sequential); returns the
 * count in effect (1 when built without OpenMP). */
int orc_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
  return n > 0 ? n : 1;
#else
  (void)n;
  return 1;
#endif
}

/* Advance n steps; once an instability has been recorded further steps do
 * nothing (the state stays frozen).  Returns the step counter. */
long orc_step(orc_state *s, long n) {
  for (long k = 0; k < n; ++k) {
    if (s->unstable_step >= 0) break;
    step_once(s);
  }
  return s->step;
}

/* ------------------------------------------------------------ observation */

long orc_num_cells(const orc_state *s) { return s->N; }
long orc_step_count(const orc_state *s) { return s->step; }
long orc_unstable_step(const orc_state *s) { return s->unstable_step; }
double orc_lost_mass(const orc_state *s) { return s->lost; }
void orc_last_counts(const orc_state *s, long *out3) {
  out3[0] = s->n_fill; out3[1] = s->n_empty; out3[2] = s->n_new;
}

void orc_get_types(const orc_state *s, unsigned char *out) { memcpy(out, s->type, s->N); }
void orc_get_pdfs(const orc_state *s, double *out) {
  memcpy(out, s->f, sizeof(double) * s->q * s->N);
}
/* bubble model: label of every cell (-1 none) and the volume pressure seen
 * by every cell (p_V where the model is off or the cell has no bubble) */
void orc_get_bubbles(const orc_state *s, long *lab, double *pressure) {
  for (long x = 0; x < s->N; ++x) {
    if (lab) lab[x] = (s->c.options & ORC_OPT_BUBBLES) ? s->blab[x] : -1;
    if (pressure) pressure[x] = (s->c.options & ORC_OPT_BUBBLES) ? s->bp[x] : s->c.p_v;
  }
}
void orc_get_phi(const orc_state *s, double *out) { memcpy(out, s->phi, sizeof(double) * s->N); }
void orc_get_mass(const orc_state *s, double *out) { memcpy(out, s->m, sizeof(double) * s->N); }
void orc_get_kappa(const orc_state *s, double *out) { memcpy(out, s->kappa, sizeof(double) * s->N); }

/* Total mass: liquid cells count the zeroth moment of their stored PDFs,
 * interface cells their mass m, plus the mass lost for want of receivers. */
double orc_total_mass(const orc_state *s) {
  const long N = s->N;
  double M = 0.0;
  for (long x = 0; x < N; ++x) {
    if (s->type[x] == ORC_LIQUID) {
      double r = 0.0;
      for (int i = 0; i < s->q; ++i) r += s->f[i * N + x];
      M += r;
    } else if (s->type[x] == ORC_IFACE) {
      M += s->m[x];
    }
  }
  return M + s->lost;
}

/* Liquid height in column x = i0: sum over y of phi, averaged over z. */
double orc_column_height(const orc_state *s, int i0) {
  double sum = 0.0;
  for (long k = 0; k < s->c.nz; ++k)
    for (long j = 0; j < s->c.ny; ++j) sum += s->phi[cell_index(s, i0, j, k)];
  return sum / (double)s->c.nz;
}

/* Front position: 1 + largest x of an interface cell in the layer y = 0. */
double orc_front(const orc_state *s) {
  long best = -1;
  for (long k = 0; k < s->c.nz; ++k)
    for (long i = 0; i < s->c.nx; ++i)
      if (s->type[cell_index(s, i, 0, k)] == ORC_IFACE && i > best) best = i;
  return (double)(best + 1);
}

/* Column height: 1 + largest y of an interface cell in the column x = 0. */
double orc_height(const orc_state *s) {
  long best = -1;
  for (long k = 0; k < s->c.nz; ++k)
    for (long j = 0; j < s->c.ny; ++j)
      if (s->type[cell_index(s, 0, j, k)] == ORC_IFACE && j > best) best = j;
  return (double)(best + 1);
}

/* Largest |u| over fluid cells, from the stored PDFs. */
double orc_max_velocity(const orc_state *s) {
  double best = 0.0;
  for (long x = 0; x < s->N; ++x) {
    if (!is_fluid_type(s->type[x])) continue;
    double r, u[3];
    stored_moments(s, s->f, x, &r, u);
    double v = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (v > best) best = v;
  }
  return best;
}

/* ------------------------------------------- single-function test entry points */

/* Parker-Youngs normal and curvature of the current phi field at one cell. */
void orc_normal_at(const orc_state *s, long x, double *n3) { normal_py(s, x, n3); }
double orc_curvature_at(const orc_state *s, long x) { return curvature(s, x); }

/* Overwrite state for hand-built neighbourhood tests: types, phi, stored PDFs. */
void orc_set_state(orc_state *s, const unsigned char *types, const double *phi, const double *pdfs,
                   const double *mass) {
  memcpy(s->type, types, s->N);
  memcpy(s->phi, phi, sizeof(double) * s->N);
  memcpy(s->f, pdfs, sizeof(double) * s->q * s->N);
  if (mass) memcpy(s->m, mass, sizeof(double) * s->N);
  for (long x = 0; x < s->N; ++x) {
    double r = 0.0;
    for (int i = 0; i < s->q; ++i) r += s->f[i * s->N + x];
    s->rho[x] = is_fluid_type(s->type[x]) ? r : 0.0;
  }
  update_curvature(s);
}

/* Refill cell x with the configured scheme from the stored PDFs of its
 * neighbours, treating the cells flagged in new_mask as newly converted.
 * Writes q PDFs to out.  Used to check the schemes on hand-built cells. */
/* Bubble bookkeeping alone, for tests: set cell types and fill levels,
 * then run the bubble update (first = 1: fresh bubbles with K = p_V V). */
void orc_bubble_probe(orc_state *s, const unsigned char *types, const double *phi, int first) {
  for (long x = 0; x < s->N; ++x) {
    s->type[x] = types[x];
    s->phi[x] = phi[x];
  }
  bubble_update(s, first);
}

void orc_refill_probe(orc_state *s, long x, const unsigned char *new_mask, double *out) {
  const long N = s->N;
  memcpy(s->is_new, new_mask, s->N);
  memcpy(s->fn, s->f, sizeof(double) * s->q * N);
  refill_cell(s, x);
  for (int i = 0; i < s->q; ++i) out[i] = s->fn[i * N + x];
  memset(s->is_new, 0, s->N);
}

/* Equilibrium and Guo term as the oracle evaluates them (for moment pins). */
double orc_feq(const orc_state *s, int i, double rho, double ux, double uy, double uz) {
  return feq(s, i, rho, ux, uy, uz);
}
double orc_guo(const orc_state *s, int i, double ux, double uy, double uz, double Fx, double Fy,
               double Fz) {
  return guo(s, i, ux, uy, uz, Fx, Fy, Fz);
}
void orc_lattice(const orc_state *s, int *c3q, double *w, int *opp) {
  for (int i = 0; i < s->q; ++i) {
    c3q[3 * i] = s->cx[i]; c3q[3 * i + 1] = s->cy[i]; c3q[3 * i + 2] = s->cz[i];
    w[i] = s->w[i];
    opp[i] = s->opp[i];
  }
}
void orc_relaxation(const orc_state *s, double *out4) {
  out4[0] = s->tau; out4[1] = s->omega; out4[2] = s->lam_e; out4[3] = s->lam_o;
}
