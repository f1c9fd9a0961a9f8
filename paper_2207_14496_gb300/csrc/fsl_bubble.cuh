// Bubble model (Sec. 2.2, Eq. nm-fslbm-pressure-volume): every enclosed gas
// region has the volume pressure p_V(t) = p_V(0) V(0) / V(t), and regions
// merge and split.  The invariant K = p V of every bubble is carried from
// step to step (option FSL_OPT_BUBBLES):
//   - bubbles are the face-connected components of gas and interface cells
//     (periodic wrap included), labelled by their smallest cell index:
//     union-find with atomicMin links (the larger root always points to the
//     smaller one, so the final root is the component's smallest cell),
//     started from runs of members along x and linked once per overlapping
//     stretch, then flattening.  Bubbles merge when their interface layers
//     touch;
//   - with FSL_OPT_BUBBLE_GAS_ONLY the components are those of gas cells
//     alone, and an interface cell belongs to the bubble with the smallest
//     label among its gas stencil neighbours (none: no bubble);
//   - a bubble's volume V is the sum of 1 per gas cell and 1 - phi per
//     interface cell; its new K is the sum, over the cells it holds that
//     were in a bubble b before, of K_b times the cell's share of b's volume
//     still in bubbles; a bubble with no such cell starts at K = p_V V;
//   - interface cells see the volume pressure K / V of their bubble, kept
//     at the bubble's root cell (bp) and read through the cell's label.
// The sums are fixed-point integers, summed per key in each warp and block
// before one atomic per key and block, so their value does not depend on the
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

// Sum of v over the threads of the block whose keys are equal, added to
// arr[idx] (idx is the same for equal keys) with one atomic per distinct key
// per block: lanes with equal keys are summed in their warp, the warps'
// partial sums are listed in shared memory and summed per key again.  The
// sums are integers, so the result does not depend on the grouping.  If
// flag is non-null, the final adder also sets flag[idx] = 1.  Every thread of
// the block calls it (it synchronises the block); kBubThreads threads.
constexpr int kBubThreads = 256;
struct BubSlots {
  long long key[kBubThreads];
  long long sum[kBubThreads];
  int idx[kBubThreads];
  int n;
};

__device__ __forceinline__ void block_keyed_add(bool on, long long key, long long v, int idx,
                                                long long* arr, uint8_t* flag, BubSlots& sh) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) sh.n = 0;
  __syncthreads();
  const unsigned act = __ballot_sync(FULL, on);
  if (on) {
    const unsigned grp = __match_any_sync(act, key);
    const int leader = __ffs(grp) - 1;
    unsigned long long sum = 0;
    for (unsigned m = grp; m; m &= m - 1) {
      const long long t = __shfl_sync(grp, v, __ffs(m) - 1);
      if (lane == leader) sum += (unsigned long long)t;
    }
    if (lane == leader) {
      const int slot = atomicAdd(&sh.n, 1);
      sh.key[slot] = key;
      sh.sum[slot] = (long long)sum;
      sh.idx[slot] = idx;
    }
  }
  __syncthreads();
  const int j = threadIdx.x;  // warp w sums entries 32 w .. 32 w + 31
  const bool has = j < sh.n;
  const unsigned act2 = __ballot_sync(FULL, has);
  if (has) {
    const long long k2 = sh.key[j];
    const long long v2 = sh.sum[j];
    const unsigned grp = __match_any_sync(act2, k2);
    const int leader = __ffs(grp) - 1;
    unsigned long long sum = 0;
    for (unsigned m = grp; m; m &= m - 1) {
      const long long t = __shfl_sync(grp, v2, __ffs(m) - 1);
      if (lane == leader) sum += (unsigned long long)t;
    }
    if (lane == leader) {
      atomicAdd(reinterpret_cast<unsigned long long*>(arr + sh.idx[j]), sum);
      if (flag) flag[sh.idx[j]] = 1;
    }
  }
  __syncthreads();
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

// Union-find start: every member points at the first cell of its run of
// members within its warp (a warp's 32 cells lie in one row, rows being
// padded to multiples of 32 cells), so a run is one tree before any union; the sums
// of the new roots (members) and the seen volume of the old roots are
// cleared.  One cell per thread, no early exit (warp ballots).
static __global__ void k_bub_init(Dev d, Geom g, int first) {
  const unsigned FULL = 0xffffffffu;
  const unsigned k = blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = k < (unsigned)g.cells;
  const int c = ok ? (int)k : 0;
  const int lane = threadIdx.x & 31;
  const bool mem = ok && c % g.sx < g.nx && bub_member(g, d.flags[c]);
  const unsigned mm = __ballot_sync(FULL, mem);
  const unsigned below = ~mm & ((1u << lane) - 1u);  // non-members left of this lane
  const int start = below ? 32 - __clz(below) : 0;
  if (!ok) return;
  d.bnew[c] = mem ? c - lane + start : -1;
  if (mem) {
    d.bV[c] = 0;
    d.bKnew[c] = 0;
    d.bhas[c] = 0;
  }
  if (!first && d.blab[c] == c) d.bVseen[c] = 0;
}

// Links across runs: the first cell of a run links to its member neighbour
// at x - 1 (the run before it, or the wrap); for the neighbours at y - 1 and
// z - 1, the first cell of every stretch of the run that lies on members
// links (its left neighbour's neighbour is not a member, or it starts the
// run): along a stretch the cells below form one run of the warp below,
// which already shares one root.  Every face-adjacent pair of members ends
// up in one tree.
static __global__ void k_bub_union(Dev d, Geom g) {
  const unsigned FULL = 0xffffffffu;
  Ctrl* ctrl = d.ctrl;
  const unsigned k = blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = k < (unsigned)g.cells;
  const int c = ok ? (int)k : 0;
  const int lane = threadIdx.x & 31;
  const bool mem = ok && c % g.sx < g.nx && bub_member(g, d.flags[c]);
  const unsigned mm = __ballot_sync(FULL, mem);
  if (!mem) return;
  const bool run_start = lane == 0 || !((mm >> (lane - 1)) & 1u);
  int x, y, z;
  cell_xyz(g, c, x, y, z);
  bool fail = false;
  if (run_start) {
    const int n = nb_at(g, x, y, z, -1, 0, 0);
    if (n >= 0 && n != c && bub_member(g, d.flags[n])) fail |= !bub_unite(d.bnew, c, n);
  }
  for (int a = 1; a <= 2; ++a) {
    const int dy = a == 1 ? -1 : 0, dz = a == 2 ? -1 : 0;
    const int n = nb_at(g, x, y, z, 0, dy, dz);
    if (n < 0 || n == c || !bub_member(g, d.flags[n])) continue;
    bool need = run_start;
    if (!need) {
      const int nl = nb_at(g, x - 1, y, z, 0, dy, dz);
      need = !(nl >= 0 && bub_member(g, d.flags[nl]));
    }
    if (need) fail |= !bub_unite(d.bnew, c, n);
  }
  if (fail) atomicOr(&ctrl->timeout, 8u);
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

// Cells per thread of the two summing passes: a warp takes 32 kBubCells
// consecutive cells (lane, lane + 32, ...), and a thread adds the terms of
// its cells that share the first key it meets in registers (inside a bubble
// that is all of them) and adds the others straight to their bubble.
constexpr int kBubCells = 8;

__device__ __forceinline__ long long bub_cell(int j) {
  const long long w = (long long)blockIdx.x * (kBubThreads / 32) + (threadIdx.x >> 5);
  return w * (32 * kBubCells) + 32 * j + (threadIdx.x & 31);
}

// volume of every new bubble; volume of every old bubble still in bubbles
// (no early exit: the sums synchronise the block)
static __global__ void __launch_bounds__(kBubThreads) k_bub_volume(Dev d, Geom g, int first,
                                                                   double vs) {
  __shared__ BubSlots sh;
  int r0 = -1, b0 = -1;
  long long acc_v = 0, acc_s = 0;
  bool bad = false;
  for (int j = 0; j < kBubCells; ++j) {
    const long long c = bub_cell(j);
    if (c >= g.cells) break;
    const int r = d.bnew[c];
    if (r < 0) continue;
    const int b = first ? -1 : d.blab[c];
    const long long wq = bub_wq(d, (int)c, vs, bad);
    if (r0 < 0) r0 = r;
    if (r == r0)
      acc_v += wq;
    else
      atomicAdd(reinterpret_cast<unsigned long long*>(d.bV + r), (unsigned long long)wq);
    if (b < 0) continue;
    if (b0 < 0) b0 = b;
    if (b == b0)
      acc_s += wq;
    else
      atomicAdd(reinterpret_cast<unsigned long long*>(d.bVseen + b), (unsigned long long)wq);
  }
  block_keyed_add(r0 >= 0, r0, acc_v, r0, d.bV, nullptr, sh);
  block_keyed_add(b0 >= 0, b0, acc_s, b0, d.bVseen, nullptr, sh);
  bub_flag(d, bad, first);
}

// K of every new bubble from the old bubbles its cells came from; bubble r
// receives a share (bhas[r] = 1) whenever one of its cells came from an old
// bubble still in bubbles
static __global__ void __launch_bounds__(kBubThreads) k_bub_kmap(Dev d, Geom g, double vs,
                                                                 double ks) {
  __shared__ BubSlots sh;
  long long key0 = -1;
  int r0 = 0;
  long long acc = 0;
  bool bad = false;
  for (int j = 0; j < kBubCells; ++j) {
    const long long c = bub_cell(j);
    if (c >= g.cells) break;
    const int r = d.bnew[c];
    const int b = d.blab[c];
    if (r < 0 || b < 0) continue;
    const long long vseen = d.bVseen[b];
    if (vseen == 0) continue;
    const long long wq = bub_wq(d, (int)c, vs, bad);
    const double share = d.bK[b] * ((double)wq / (double)vseen);
    long long v = 0;
    if (fabs(share) < 16.0)
      v = __double2ll_rn(share * ks);
    else
      bad = true;
    const long long key = ((long long)r << 32) | (unsigned)b;
    if (key0 < 0) {
      key0 = key;
      r0 = r;
    }
    if (key == key0) {
      acc += v;
    } else {
      atomicAdd(reinterpret_cast<unsigned long long*>(d.bKnew + r), (unsigned long long)v);
      d.bhas[r] = 1;
    }
  }
  block_keyed_add(key0 >= 0, key0, acc, r0, d.bKnew, d.bhas, sh);
  bub_flag(d, bad, 0);
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
  const unsigned sum_blocks = (unsigned)((g.cells + kBubThreads * kBubCells - 1) /
                                         (kBubThreads * kBubCells));
  k_bub_volume<<<sum_blocks, kBubThreads, 0, s>>>(d, g, first, sc.vs);
  if (!first) k_bub_kmap<<<sum_blocks, kBubThreads, 0, s>>>(d, g, sc.vs, sc.ks);
  k_bub_commit<<<blocks, 256, 0, s>>>(d, g, p.p_v, sc.vinv, sc.kinv);
  return cudaGetLastError();
}

}  // namespace fsl
