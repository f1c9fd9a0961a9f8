// Bubble model (Sec. 2.2, Eq. nm-fslbm-pressure-volume): every enclosed gas
// region has the volume pressure p_V(t) = p_V(0) V(0) / V(t), and regions
// merge and split.  The invariant K = p V of every bubble is carried from
// step to step (option FSL_OPT_BUBBLES):
//   - bubbles are the face-connected components of gas and interface cells
//     (periodic wrap included), labelled by their smallest cell index:
//     union-find with atomicMin links (the larger root always points to the
//     smaller one, so the final root is the component's smallest cell), then
//     flattening.  Bubbles merge when their interface layers touch;
//   - with FSL_OPT_BUBBLE_GAS_ONLY the components are those of gas cells
//     alone, and an interface cell belongs to the bubble with the smallest
//     label among its gas stencil neighbours (none: no bubble);
//   - a bubble's volume V is the sum of 1 per gas cell and 1 - phi per
//     interface cell; its new K is the sum, over the cells it holds that
//     were in a bubble b before, of K_b times the cell's share of b's volume
//     still in bubbles; a bubble with no such cell starts at K = p_V V;
//   - interface cells see the volume pressure K / V of their bubble, kept
//     at the bubble's root cell (bp) and read through the cell's label.
// The sums are fixed-point integers, so their value does not depend on the
// order in which the atomics land: with 2^b the smallest power of two not
// below nx*ny*nz, a cell's volume term w counts as round(w 2^vshift) units,
// vshift = 62 - b, and a share of K as round(share 2^kshift) units,
// kshift = vshift - 4 (round to nearest even).  Sums of up to 2^b terms stay
// below 2^63 while |w| < 2 and every share is below 16 (a share is at most
// the bubble's pressure); a term outside that range counts as 0 and marks the
// step unstable.  The union loop is bounded; if it gives up it latches bit 8
// of the control block's error word.
#pragma once
// Included by fsl_kernels.cuh.
#include <cmath>

namespace fsl {

__device__ __forceinline__ int bub_find(const int* L, int x) {
  // labels only ever decrease towards the root, so the walk ends (path
  // halving with atomicMin was measured slower: the hot ancestors contend)
  int r = L[x];
  while (r != x) {
    x = r;
    r = L[x];
  }
  return r;
}

// link the components of cells a and b (roots always point to smaller roots)
__device__ __forceinline__ bool bub_unite(int* L, int a, int b) {
  for (int it = 0; it < (1 << 16); ++it) {
    a = bub_find(L, a);
    b = bub_find(L, b);
    if (a == b) return true;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    // make root b point to the smaller root a, if b is still a root
    const int old = atomicMin(&L[b], a);
    if (old == b) return true;
    b = old;  // b had been linked meanwhile: retry from its new parent
  }
  return false;
}

// sum of v over the lanes of the warp that share key; the lowest such lane
// adds the sum to *dst (integer: exact in any order)
__device__ __forceinline__ void warp_keyed_add(bool on, long long key, long long v,
                                               long long* dst) {
  const unsigned act = __ballot_sync(0xffffffffu, on);
  if (!on) return;
  const unsigned grp = __match_any_sync(act, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(grp) - 1;
  unsigned long long sum = 0;
  unsigned m = grp;
  while (m) {
    const int l = __ffs(m) - 1;
    const long long t = __shfl_sync(grp, v, l);
    if (lane == leader) sum += (unsigned long long)t;
    m &= m - 1;
  }
  if (lane == leader) atomicAdd(reinterpret_cast<unsigned long long*>(dst), sum);
}

// fixed-point scales of the bubble sums
struct BubScale {
  double vs, vinv;  // 2^vshift, 2^-vshift
  double ks, kinv;  // 2^kshift, 2^-kshift
};

inline BubScale bub_scale(const Geom& g) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  int b = 0;
  while ((1LL << b) < n) ++b;
  const int vshift = 62 - b, kshift = vshift - 4;
  return {std::ldexp(1.0, vshift), std::ldexp(1.0, -vshift), std::ldexp(1.0, kshift),
          std::ldexp(1.0, -kshift)};
}

// a cell's volume term in fixed point (0 and *bad when |w| >= 2)
__device__ __forceinline__ long long bub_wq(const Dev& d, int c, double vs, bool& bad) {
  const double w = (d.flags[c] & F_TYPE) == T_GAS ? 1.0 : 1.0 - d.phi[c];
  if (!(fabs(w) < 2.0)) {
    bad = true;
    return 0;
  }
  return __double2ll_rn(w * vs);
}

// cells that make up the components: gas cells, and interface cells unless
// the gas-only reading is selected
__device__ __forceinline__ bool bub_member(const Geom& g, uint8_t fl) {
  const int t = fl & F_TYPE;
  return t == T_GAS || (!g.bub_gas_only && t == T_IF);
}

// every member its own root; clear the sums of the new roots (members) and
// the seen volume of the old roots
static __global__ void k_bub_init(Dev d, Geom g, int first) {
  FSL_GRID_LOOP(k, (unsigned)g.cells) {
    const int c = (int)k;
    const int x = c % g.sx;
    const bool gas = x < g.nx && bub_member(g, d.flags[c]);
    d.bnew[c] = gas ? c : -1;
    if (gas) {
      d.bV[c] = 0;
      d.bKnew[c] = 0;
      d.bhas[c] = 0;
    }
    if (!first && d.blab[c] == c) d.bVseen[c] = 0;
  }
}

static __global__ void k_bub_union(Dev d, Geom g) {
  Ctrl* ctrl = d.ctrl;
  FSL_GRID_LOOP(k, (unsigned)g.cells) {
    const int c = (int)k;
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    if (x >= g.nx || !bub_member(g, d.flags[c])) continue;
    // the three face neighbours below: every face pair (wrap included) once
    const int nbs[3] = {nb_at(g, x, y, z, -1, 0, 0), nb_at(g, x, y, z, 0, -1, 0),
                        nb_at(g, x, y, z, 0, 0, -1)};
    for (int a = 0; a < 3; ++a) {
      const int n = nbs[a];
      if (n >= 0 && n != c && bub_member(g, d.flags[n]))
        if (!bub_unite(d.bnew, c, n)) atomicOr(&ctrl->timeout, 8u);
    }
  }
}

// members point straight at their root; in the gas-only reading an
// interface cell takes the smallest root among its gas stencil neighbours.
// Concurrent finds stay valid: flattening only ever stores a cell's root,
// and (gas-only) interface cells are on no gas cell's path.
template <int Q>
__global__ void k_bub_label(Dev d, Geom g) {
  FSL_GRID_LOOP(k, (unsigned)g.cells) {
    const int c = (int)k;
    int x, y, z;
    cell_xyz(g, c, x, y, z);
    if (x >= g.nx) continue;
    const uint8_t fl = d.flags[c];
    const uint8_t t = fl & F_TYPE;
    if (bub_member(g, fl)) {
      d.bnew[c] = bub_find(d.bnew, c);
    } else if (t == T_IF) {
      int best = -1;
      for (int i = 1; i < Q; ++i) {
        const int n = nb_at(g, x, y, z, rc(i, 0), rc(i, 1), rc(i, 2));
        if (n >= 0 && (d.flags[n] & F_TYPE) == T_GAS) {
          const int l = bub_find(d.bnew, n);
          if (best < 0 || l < best) best = l;
        }
      }
      d.bnew[c] = best;
    }
  }
}

// a step whose bubble sums met an out-of-range term counts as unstable
__device__ __forceinline__ void bub_flag(const Dev& d, bool bad, int first) {
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0 && !first)
    atomicCAS(&d.ctrl->unstable_step, -1, d.ctrl->step + 1);
}

// volume of every new bubble; volume of every old bubble still in bubbles
static __global__ void k_bub_volume(Dev d, Geom g, int first, double vs) {
  FSL_WARP_LOOP(k, ok, (unsigned)g.cells) {
    const int c = ok ? (int)k : 0;
    const int r = ok ? d.bnew[c] : -1;
    const int b = (ok && !first) ? d.blab[c] : -1;
    bool bad = false;
    const long long wq = r >= 0 ? bub_wq(d, c, vs, bad) : 0;
    warp_keyed_add(r >= 0, r, wq, d.bV + (r >= 0 ? r : 0));
    warp_keyed_add(r >= 0 && b >= 0, b, wq, d.bVseen + (b >= 0 ? b : 0));
    bub_flag(d, bad, first);
  }
}

// K of every new bubble from the old bubbles its cells came from
static __global__ void k_bub_kmap(Dev d, Geom g, double vs, double ks) {
  FSL_WARP_LOOP(k, ok, (unsigned)g.cells) {
    const int c = ok ? (int)k : 0;
    const int r = ok ? d.bnew[c] : -1;
    const int b = ok ? d.blab[c] : -1;
    bool on = r >= 0 && b >= 0;
    bool bad = false;
    long long v = 0;
    if (on) {
      const long long vseen = d.bVseen[b];
      on = vseen != 0;
      if (on) {
        const long long wq = bub_wq(d, c, vs, bad);
        const double share = d.bK[b] * ((double)wq / (double)vseen);
        if (fabs(share) < 16.0)
          v = __double2ll_rn(share * ks);
        else
          bad = true;
        d.bhas[r] = 1;
      }
    }
    const long long key = on ? ((long long)r << 32) | (unsigned)b : 0;
    warp_keyed_add(on, key, v, d.bKnew + (on ? r : 0));
    bub_flag(d, bad, 0);
  }
}

// the new labels become the state; K and volume pressure of every bubble at
// its root: the carried sum of K, or p_V V for a bubble without a predecessor
static __global__ void k_bub_commit(Dev d, Geom g, double p_v, double vinv, double kinv) {
  FSL_GRID_LOOP(k, (unsigned)g.cells) {
    const int c = (int)k;
    const int r = d.bnew[c];
    d.blab[c] = r;
    if (r == c) {
      const double V = (double)d.bV[c] * vinv;
      const double K = d.bhas[c] ? (double)d.bKnew[c] * kinv : p_v * V;
      d.bK[c] = K;
      d.bp[c] = V != 0.0 ? K / V : p_v;
    }
  }
}

// volume pressure of every cell (the bubble's, else p_V) into out
static __global__ void k_bub_expand(Dev d, Geom g, double p_v, double* out) {
  FSL_GRID_LOOP(k, (unsigned)g.cells) {
    const int c = (int)k;
    const int r = d.blab[c];
    out[c] = r >= 0 ? d.bp[r] : p_v;
  }
}

// the whole update (first: bubbles of the initial state, K = p_V V)
template <int Q>
cudaError_t bubble_update(const Dev& d, const Geom& g, const Phys& p, int first, cudaStream_t s) {
  // one thread per cell: these passes do one or two dependent memory round
  // trips per cell, so as many cells as possible should be in flight (a
  // grid-stride loop over a small grid would serialise the round trips)
  const unsigned blocks = (unsigned)((g.cells + 255) / 256);
  const BubScale sc = bub_scale(g);
  k_bub_init<<<blocks, 256, 0, s>>>(d, g, first);
  k_bub_union<<<blocks, 256, 0, s>>>(d, g);
  k_bub_label<Q><<<blocks, 256, 0, s>>>(d, g);
  k_bub_volume<<<blocks, 256, 0, s>>>(d, g, first, sc.vs);
  if (!first) k_bub_kmap<<<blocks, 256, 0, s>>>(d, g, sc.vs, sc.ks);
  k_bub_commit<<<blocks, 256, 0, s>>>(d, g, p.p_v, sc.vinv, sc.kinv);
  return cudaGetLastError();
}

}  // namespace fsl
