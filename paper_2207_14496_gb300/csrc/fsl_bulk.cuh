// Bulk pass of the 16/32-bit path, staged through shared memory by the TMA.
//
// k_tiles lists, at the start of a step, the tiles (256 cells along x of one
// (y, z) row) that hold liquid cells.
//
// k_stream_collide_bulk is persistent and warp-specialised.  Its producer warp
// walks the CTA's share of the tile list and, for each tile, issues Q + 1
// one-dimensional bulk copies (cp.async.bulk, the untiled TMA form) into a
// ring of shared-memory stages: for each direction i the 256 + 2*8 stored
// values of plane i on the row (y - c_iy, z - c_iz) that the tile pulls
// from (clipped to the row), and the tile's 256 flag bytes.  Each copy group
// completes on the stage's "full" mbarrier.  Four consumer warps, two
// neighbouring cells per thread, wait on "full", pull their 27 (or 19) value
// pairs out of shared memory, collide both cells in packed FP32 (collide_v)
// and store the result to HBM, then release the stage through its "empty"
// mbarrier so that the producer can refill it.  With
// several stages in flight per CTA the HBM traffic does not wait on the
// collision arithmetic.
//
// Alignment: every copy starts at an element index that is a multiple of 8
// (tile starts are multiples of 256, the halo is 8, rows are padded to 32),
// so addresses and byte counts are multiples of 16.  Every mbarrier wait is
// bounded; a wait that gives up latches bit 4 of the control block's error
// word, stops the CTA's loops, and the producer waits (bounded) for the copies
// it issued before the CTA exits.
#pragma once
// Included by fsl_kernels.cuh after collide_lp, pull_liquid and warp_append.

namespace fsl {

constexpr int kBulkTX = 256;    // cells per tile along x
constexpr int kBulkHalo = 8;    // staged halo on each side (keeps copies 16-byte aligned)
constexpr int kBulkSeg = kBulkTX + 2 * kBulkHalo;
constexpr int kBulkConsumers = 4;                      // warps, two cells per thread
constexpr int kBulkThreads = 32 * (kBulkConsumers + 1);  // + one producer warp

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (int it = 0; it < (1 << 20); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ring depth and shared-memory layout per storage type
template <int Q, class ST, int NS = (sizeof(typename ST::T) == 2 ? 4 : 3)>
struct BulkRing {
  static constexpr int stages = NS;
  static constexpr size_t pdf_bytes = (size_t)Q * kBulkSeg * sizeof(typename ST::T);
  static constexpr size_t stage_bytes = pdf_bytes + kBulkTX;  // + flag bytes
  // stages, then full[stages] and empty[stages] barriers, the tile
  // coordinates (x0, row, y, z) of each stage and the abort flag
  static constexpr size_t bytes = stages * stage_bytes + 2 * stages * 8 + 16 * stages + 16;
};

// List the tiles (TX cells along x of one row) with liquid cells.  One thread
// per tile reads the tile's flag bytes in 16-byte words; a block's tiles are
// ranked by warp ballots and appended with one atomic per block (the order of
// the list does not matter to its consumers).  Cells beyond the row's extent
// hold the gas type.
template <int TX>
__device__ __forceinline__ void tiles_body(const Dev& d, const Geom& g, int ntx) {
  static_assert(TX % 32 == 0, "tiles of whole 32-cell row pieces");
  __shared__ int warp_n[8];
  __shared__ unsigned base;
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const long long ntiles = (long long)ntx * g.ny * g.nz;
  const long long k = (long long)blockIdx.x * 256 + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool liq = false;
  if (k < ntiles) {
    const int x0 = (int)(k % ntx) * TX;
    const long long row = k / ntx;
    const int n = (g.sx - x0 < TX ? g.sx - x0 : TX) / 16;  // 16-byte words in the padded row
    const uint4* w = reinterpret_cast<const uint4*>(d.flags + row * g.sx + x0);
    for (int q = 0; q < n && !liq; ++q) {
      const uint4 v = w[q];
      const unsigned u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        // a byte whose type bits are T_LIQ: (b & 3) ^ 2 == 0
        const unsigned t = (u[h] & 0x03030303u) ^ 0x02020202u;
        liq |= ((t - 0x01010101u) & ~t & 0x80808080u) != 0u;
      }
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, liq);
  if (lane == 0) warp_n[warp] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w2 = 0; w2 < 8; ++w2) {
      const int c = warp_n[w2];
      warp_n[w2] = tot;
      tot += c;
    }
    base = tot ? atomicAdd(&ctrl->n_tiles, (unsigned)tot) : 0u;
  }
  __syncthreads();
  if (liq) d.l_tiles[base + warp_n[warp] + __popc(m & ((1u << lane) - 1u))] = (int)k;
}

template <int TX>
__global__ void __launch_bounds__(256) k_tiles(Dev d, Geom g, int ntx) {
  tiles_body<TX>(d, g, ntx);
}
template <int TX>
__global__ void __launch_bounds__(256) kb_tiles(MemberTable t) {
  FSL_MEMBER(t);
  tiles_body<TX>(d, g, (g.nx + TX - 1) / TX);
}


// Update of two neighbouring cells (xa, xa + 1) of row `row` = (y, z), read
// from A and written to B, whose pulled values sit in a staged row segment:
// stage holds, per direction i, the stored values of
// plane i on the source row (y - c_iy, z - c_iz) from x = x0 - halo on, `seg`
// values per direction; li is the staged index of cell xa.  Values are read
// out of shared memory, both cells collide in packed FP32 and the results go
// to HBM.  The periodic wrap along x at the two row ends: wrap = 0, read from
// HBM; 1, the stage holds the wrapped halos; 2, the stage holds the whole row
// (x0 = 0, nx <= the tile width) and the value comes from its other end.
// Liquid cells next to a domain wall (no obstacle cell, no free-slip wall)
// take the halfway bounce-back value for the directions that cross the wall;
// next to an obstacle or a free-slip wall the per-direction path reads HBM.
// Returns whether a liquid cell reached |u|^2 >= 1/3.
template <int Q, class ST>
__device__ __forceinline__ bool bulk_pair(const typename ST::T* __restrict__ A,
                                          typename ST::T* __restrict__ B,
                                          const typename ST::T* stage, int seg, int li, int xa,
                                          int row, int y, int z, uint8_t fl0, uint8_t fl1,
                                          const Dev& d, const Geom& g, const Phys& p,
                                          const LesLp& les, int wrap = 0) {
  using T = typename ST::T;
  constexpr float S = ST::kScaleF;
  const bool liq0 = (fl0 & F_TYPE) == T_LIQ, liq1 = (fl1 & F_TYPE) == T_LIQ;
  if (!liq0 && !liq1) return false;
  const long long P = g.plane;
  float2 f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = dir_c(i, 0);
    if constexpr (sizeof(T) == 2) {
      const unsigned short* sg = reinterpret_cast<const unsigned short*>(stage) + (size_t)i * seg;
      unsigned wv;
      if (cx == 0) {
        wv = *reinterpret_cast<const unsigned*>(sg + li);
      } else {  // (li - cx, li + 1 - cx) straddles a 32-bit word
        wv = (unsigned)sg[li - cx] | ((unsigned)sg[li + 1 - cx] << 16);
      }
      f[i] = ST::unpack2(wv);
    } else {
      const T* sg = stage + (size_t)i * seg;
      f[i] = make_float2(ST::ld1s(sg + li - cx), ST::ld1s(sg + li + 1 - cx));
    }
  }
  if (wrap == 2 && g.periodic[0] && (xa == 0 || xa + 1 >= g.nx - 1)) {
    // the whole row is staged: cell x sits at li - (xa - x)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cx = dir_c(i, 0);
      if (cx == 0) continue;
      const T* sg = stage + (size_t)i * seg;
      if (cx == 1 && xa == 0) f[i].x = ST::ld1s(sg + li + g.nx - 1);
      if (cx == -1 && xa == g.nx - 1) f[i].x = ST::ld1s(sg + li - xa);
      if (cx == -1 && xa + 1 == g.nx - 1) f[i].y = ST::ld1s(sg + li - xa);
    }
  }
  if (wrap == 0 && g.periodic[0] && (xa == 0 || xa + 1 >= g.nx - 1)) {
    // periodic wrap along x: the value comes from the other end of the row
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cx = dir_c(i, 0);
      if (cx == 0) continue;
      const T* src = A + i * P +
                     (long long)g.sx * (((y - dir_c(i, 1) + g.ny) % g.ny) +
                                        g.ny * ((z - dir_c(i, 2) + g.nz) % g.nz));
      if (cx == 1 && xa == 0) f[i].x = ST::ld1(src + g.nx - 1);
      if (cx == -1 && xa == g.nx - 1) f[i].x = ST::ld1(src);
      if (cx == -1 && xa + 1 == g.nx - 1) f[i].y = ST::ld1(src);
    }
  }
  const long long c = (long long)row * g.sx + xa;
  const bool near0 = liq0 && (fl0 & F_NEAR_OBST), near1 = liq1 && (fl1 & F_NEAR_OBST);
  if ((near0 || near1) && !g.has_obst && !g.free_slip) {
    const bool wl0 = !g.periodic[0] && xa == 0, wr0 = !g.periodic[0] && xa + 1 >= g.nx;
    const bool wr1 = !g.periodic[0] && xa + 2 >= g.nx;
    const bool ylo = !g.periodic[1] && y == 0, yhi = !g.periodic[1] && y == g.ny - 1;
    const bool zlo = !g.periodic[2] && z == 0, zhi = !g.periodic[2] && z == g.nz - 1;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int cx = dir_c(i, 0), cy = dir_c(i, 1), cz = dir_c(i, 2);
      const bool yz = (cy == 1 && ylo) || (cy == -1 && yhi) || (cz == 1 && zlo) || (cz == -1 && zhi);
      if (near0 && (yz || (cx == 1 && wl0) || (cx == -1 && wr0))) f[i].x = ST::ld1(A + opp(i) * P + c);
      if (near1 && (yz || (cx == -1 && wr1))) f[i].y = ST::ld1(A + opp(i) * P + c + 1);
    }
  } else if (near0 || near1) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!(h ? near1 : near0)) continue;
      float tv[Q];
      pull_near<Q, ST>(A, P, d.flags, g, xa + h, y, z, tv);
#pragma unroll
      for (int i = 0; i < Q; ++i) Lanes<float2>::at(f[i], h) = tv[i] * S;
    }
  }
  const bool tr = p.trt != 0;
  const float lamE = p.f.lam_e, lamO = tr ? p.f.lam_o : p.f.omega;
  const float pe = p.f.pre_e, po = tr ? p.f.pre_o : p.f.pre_e;
  const float2 usq = collide_v<Q, float2>(f, f, lamE, lamO, pe, po, p.f.g[0], p.f.g[1], p.f.g[2],
                                          S, les);
  T* out = B + c;
  if (liq0 && liq1) {
#pragma unroll
    for (int i = 0; i < Q; ++i) ST::st2(out + i * P, f[i].x, f[i].y);
  } else if (liq0) {
#pragma unroll
    for (int i = 0; i < Q; ++i) ST::st1(out + i * P, f[i].x);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) ST::st1(out + i * P + 1, f[i].y);
  }
  return (liq0 && !(usq.x < (float)(1.0 / 3.0))) || (liq1 && !(usq.y < (float)(1.0 / 3.0)));
}

template <int Q, class ST, int NS, int MINB>
__global__ void __launch_bounds__(kBulkThreads, MINB)
    k_stream_collide_bulk(Dev d, Geom g, Phys p, int ntx) {
  using T = typename ST::T;
  using RING = BulkRing<Q, ST, NS>;
  constexpr int D = RING::stages;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + D * RING::stage_bytes);
  uint64_t* empty = full + D;
  int4* tile_of = reinterpret_cast<int4*>(empty + D);  // (x0, row, y, z) held by each stage
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tile_of + D);
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int cur = ctrl->step & 1;
  const T* __restrict__ A = (const T*)d.pdf[cur];
  T* __restrict__ B = (T*)d.pdf[cur ^ 1];
  const long long P = g.plane;
  const int ntl = (int)ctrl->n_tiles;
  if ((int)blockIdx.x >= ntl) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < D; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kBulkConsumers);
    }
    *abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == kBulkConsumers) {
    // ---------------- producer warp: lane 0 waits for the stage and arms its
    // barrier, lane i < Q copies direction i, lane Q the flags
    int issued = 0;
    bool stop = false;
    for (int j = 0;; ++j) {
      const int ti = blockIdx.x + j * gridDim.x;
      if (ti >= ntl) break;
      const int s = j % D;
      int go = 1;
      if (lane == 0) {
        if (j >= D && !mbar_wait(&empty[s], ((j / D) - 1) & 1)) {
          *abort_flag = 1;
          atomicOr(&ctrl->timeout, 4u);
        }
        go = *abort_flag == 0;
      }
      if (!__shfl_sync(0xffffffffu, go, 0)) {
        stop = true;
        break;
      }
      const int k = d.l_tiles[ti];
      const int x0 = (k % ntx) * kBulkTX;
      const int row = k / ntx;
      const int lo = x0 - kBulkHalo > 0 ? x0 - kBulkHalo : 0;
      const int hi = x0 + kBulkTX + kBulkHalo < g.sx ? x0 + kBulkTX + kBulkHalo : g.sx;
      const unsigned bytes = (unsigned)((hi - lo) * sizeof(T));
      const unsigned fbytes = (unsigned)(g.sx - x0 < kBulkTX ? g.sx - x0 : kBulkTX);
      unsigned char* stage = smem + (size_t)s * RING::stage_bytes;
      if (lane == 0) {
        // published to the consumers by the arrive below
        tile_of[s] = make_int4(x0, row, row % g.ny, row / g.ny);
        mbar_expect_tx(&full[s], bytes * Q + fbytes);
      }
      __syncwarp();
      if (lane < Q) {
        const int i = lane;
        const int y = row % g.ny, z = row / g.ny;
        const int cy = rc(i, 1), cz = rc(i, 2);
        int ys = y - cy, zs = z - cz;
        ys = ys < 0 ? (g.periodic[1] ? g.ny - 1 : y) : (ys >= g.ny ? (g.periodic[1] ? 0 : y) : ys);
        zs = zs < 0 ? (g.periodic[2] ? g.nz - 1 : z) : (zs >= g.nz ? (g.periodic[2] ? 0 : z) : zs);
        const T* src = A + i * P + (long long)g.sx * (ys + g.ny * zs) + lo;
        T* dst = reinterpret_cast<T*>(stage) + (lo - (x0 - kBulkHalo)) + (size_t)i * kBulkSeg;
        bulk_copy_g2s(dst, src, bytes, &full[s]);
      } else if (lane == Q) {
        bulk_copy_g2s(stage + RING::pdf_bytes, d.flags + (long long)row * g.sx + x0, fbytes,
                      &full[s]);
      }
      ++issued;
    }
    if (stop && lane == 0) {
      // let the copies this CTA issued land before its shared memory goes away
      const int first = issued > D ? issued - D : 0;
      for (int j = first; j < issued; ++j) mbar_wait(&full[j % D], (j / D) & 1);
    }
    return;
  }

  // ---------------- consumer warps: two cells (2t, 2t + 1) of the tile per thread
  const LesLp les = LesLp::of(p);
  const int t = threadIdx.x;
  bool bad = false;
  for (int j = 0;; ++j) {
    const int ti = blockIdx.x + j * gridDim.x;
    if (ti >= ntl) break;
    const int s = j % D;
    const bool ok = mbar_wait(&full[s], (j / D) & 1);
    // the decision to stop is taken by the whole warp
    if (__any_sync(0xffffffffu, !ok || *abort_flag != 0)) {
      if (lane == 0) {
        *abort_flag = 1;
        atomicOr(&ctrl->timeout, 4u);
      }
      break;
    }
    const unsigned char* stage = smem + (size_t)s * RING::stage_bytes;
    const int4 tc = tile_of[s];
    const int xa = tc.x + 2 * t;
    const uchar2 f2 = *reinterpret_cast<const uchar2*>(stage + RING::pdf_bytes + 2 * t);
    const uint8_t fl0 = xa < g.nx ? f2.x : (uint8_t)T_GAS;
    const uint8_t fl1 = xa + 1 < g.nx ? f2.y : (uint8_t)T_GAS;
    bad |= bulk_pair<Q, ST>(A, B, reinterpret_cast<const T*>(stage), kBulkSeg, kBulkHalo + 2 * t,
                            xa, tc.y, tc.z, tc.w, fl0, fl1, d, g, p, les,
                            (tc.x == 0 && g.nx <= kBulkTX) ? 2 : 0);
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicCAS(&ctrl->unstable_step, -1, ctrl->step + 1);
}

// ------------------------------------------------------------------------
// Per-warp TMA pipeline.  Every warp owns a ring of shared-memory stages and
// streams its own sequence of 64-cell row segments (listed by k_tiles<64>):
// lane 0 issues the Q + 1 bulk copies of segment j + D - 1 (per direction the
// 64 + 2*8 stored values of the source row, and the 64 flag bytes) while the
// whole warp updates segment j out of its stage, two cells per lane.  No
// barrier spans more than one warp, so a slow warp holds up nobody, and the
// loads in flight occupy shared memory instead of registers.  The stage a
// warp has just read is handed back to the async proxy by a proxy fence
// before lane 0 refills it.  Waits are bounded as in the block-level kernel.
constexpr int kWarpTX = 64;
constexpr int kWarpSeg = kWarpTX + 2 * kBulkHalo;
constexpr int kWarpsPerBlock = 4;

template <int Q, class ST>
struct WarpRing {
  static constexpr bool half = sizeof(typename ST::T) == 2;
  static constexpr int stages = half ? 4 : 3;
  static constexpr int min_blocks = half ? 3 : 2;  // blocks per SM the ring allows
  static constexpr size_t pdf_bytes = (size_t)Q * kWarpSeg * sizeof(typename ST::T);
  static constexpr size_t stage_bytes = (pdf_bytes + kWarpTX + 15) / 16 * 16;
  // per warp: stages, then the full barriers (padded to 16 bytes) and the
  // segment coordinates (x0, row, y, z) of each stage (16-byte aligned)
  static constexpr size_t bar_bytes = (stages * 8 + 15) / 16 * 16;
  static constexpr size_t tail_bytes = bar_bytes + stages * 16;
  static constexpr size_t warp_bytes = stages * stage_bytes + tail_bytes;
  static constexpr size_t bytes = kWarpsPerBlock * warp_bytes;
};

template <int Q, class ST>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, WarpRing<Q, ST>::min_blocks)
    k_stream_collide_wtma(Dev d, Geom g, Phys p, int ntx) {
  using T = typename ST::T;
  using RING = WarpRing<Q, ST>;
  constexpr int D = RING::stages;
  extern __shared__ __align__(128) unsigned char smem[];
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int ntl = (int)ctrl->n_tiles;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kWarpsPerBlock + warp, tw = gridDim.x * kWarpsPerBlock;
  if (gw >= ntl) return;  // whole warp; nothing below synchronises the block
  unsigned char* ring = smem + (size_t)warp * RING::warp_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + D * RING::stage_bytes);
  int4* seg_of = reinterpret_cast<int4*>(ring + D * RING::stage_bytes + RING::bar_bytes);
  if (lane == 0) {
    for (int s = 0; s < D; ++s) mbar_init(&full[s], 1);
    mbar_fence_init();
  }
  __syncwarp();
  const T* __restrict__ A = (const T*)d.pdf[ctrl->step & 1];
  T* __restrict__ B = (T*)d.pdf[(ctrl->step & 1) ^ 1];
  const long long P = g.plane;
  // copies of the warp's jl-th segment into stage jl % D: lane 0 arms the
  // stage's barrier, then lane i < Q issues direction i and lane Q the flags
  // (warp-uniform call)
  auto issue = [&](int jl) {
    const int u = gw + jl * tw;
    if (u >= ntl) return;
    const int s = jl % D;
    const int k = d.l_tiles[u];
    const int x0 = (k % ntx) * kWarpTX;
    const int row = k / ntx;
    const int lo = x0 - kBulkHalo > 0 ? x0 - kBulkHalo : 0;
    const int hi = x0 + kWarpTX + kBulkHalo < g.sx ? x0 + kWarpTX + kBulkHalo : g.sx;
    const unsigned bytes = (unsigned)((hi - lo) * sizeof(T));
    const unsigned fbytes = (unsigned)(g.sx - x0 < kWarpTX ? g.sx - x0 : kWarpTX);
    unsigned char* stage = ring + (size_t)s * RING::stage_bytes;
    if (lane == 0) {
      // published to the warp by the arrive below
      seg_of[s] = make_int4(x0, row, row % g.ny, row / g.ny);
      mbar_expect_tx(&full[s], bytes * Q + fbytes);
    }
    __syncwarp();
    if (lane < Q) {
      const int i = lane;
      const int y = row % g.ny, z = row / g.ny;
      const int cy = rc(i, 1), cz = rc(i, 2);
      int ys = y - cy, zs = z - cz;
      ys = ys < 0 ? (g.periodic[1] ? g.ny - 1 : y) : (ys >= g.ny ? (g.periodic[1] ? 0 : y) : ys);
      zs = zs < 0 ? (g.periodic[2] ? g.nz - 1 : z) : (zs >= g.nz ? (g.periodic[2] ? 0 : z) : zs);
      const T* src = A + i * P + (long long)g.sx * (ys + g.ny * zs) + lo;
      T* dst = reinterpret_cast<T*>(stage) + (lo - (x0 - kBulkHalo)) + (size_t)i * kWarpSeg;
      bulk_copy_g2s(dst, src, bytes, &full[s]);
    } else if (lane == Q) {
      bulk_copy_g2s(stage + RING::pdf_bytes, d.flags + (long long)row * g.sx + x0, fbytes, &full[s]);
    }
  };
  for (int jl = 0; jl < D - 1; ++jl) issue(jl);
  const LesLp les = LesLp::of(p);
  bool bad = false;
  int done = 0;  // segments consumed
  bool abort = false;
  for (int jl = 0;; ++jl) {
    const int u = gw + jl * tw;
    if (u >= ntl) break;
    const int s = jl % D;
    issue(jl + D - 1);  // into the stage released last iteration
    const bool ok = mbar_wait(&full[s], (jl / D) & 1);
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0) atomicOr(&ctrl->timeout, 4u);
      abort = true;
      break;
    }
    const unsigned char* stage = ring + (size_t)s * RING::stage_bytes;
    const int4 tc = seg_of[s];
    const int xa = tc.x + 2 * lane;
    const uchar2 f2 = *reinterpret_cast<const uchar2*>(stage + RING::pdf_bytes + 2 * lane);
    const uint8_t fl0 = xa < g.nx ? f2.x : (uint8_t)T_GAS;
    const uint8_t fl1 = xa + 1 < g.nx ? f2.y : (uint8_t)T_GAS;
    bad |= bulk_pair<Q, ST>(A, B, reinterpret_cast<const T*>(stage), kWarpSeg,
                            kBulkHalo + 2 * lane, xa, tc.y, tc.z, tc.w, fl0, fl1, d, g, p, les);
    // this lane's reads of the stage are complete before the refill
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    done = jl + 1;
  }
  if (abort && lane == 0) {
    // let every copy this warp issued land before its shared memory goes away
    for (int jl = done; jl < done + D; ++jl) {
      if (gw + jl * tw >= ntl) break;
      mbar_wait(&full[jl % D], (jl / D) & 1);
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicCAS(&ctrl->unstable_step, -1, ctrl->step + 1);
}

// ------------------------------------------------------------------------
// Block-wide cp.async pipeline.  Persistent CTAs of 128 threads walk the
// liquid tiles (256 cells of one row, listed by k_tiles<256>) through a ring
// of S shared-memory stages.  Every thread takes part in
// filling a stage: per direction i the stage holds the stored values of
// plane i on the source row (y - c_iy, z - c_iz) for x in [x0 - 8, x0 + 264),
// cut into 34 pieces of 8 values (16 bytes), followed by the tile's 256 flag
// bytes; thread t issues the pieces t, t + 128, ... as asynchronous
// global-to-shared copies (cp.async.cg, one commit group per tile).  Along a
// periodic x axis whose extent is a multiple of 8 the halo pieces beyond the
// row ends are copied from the other end of the row, so no cell reads HBM
// outside the stage (other widths read the wrapped values directly).
// The loads of S - 1 tiles are in flight while the block collides the
// current one, and they occupy shared memory, not registers.  A thread's
// pieces have landed once cp.async.wait_group returns, and the whole stage is
// visible to the block after the barrier that follows; a second barrier keeps
// a stage from being refilled before every thread has read it.  Nothing here
// spins: the waits are the hardware's completion of the copies this thread
// issued.  The collision of a cell pair is pair_2s (same bits as the other
// variants).
//
// Alignment: piece r of a tile starts at x0 - 8 + 8 r (or at that position
// moved by +/- nx across the periodic wrap, with nx a multiple of 8), a
// multiple of 8 elements, and rows are padded to 32 cells, so every piece is
// 16 bytes at 16-byte-aligned addresses.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

constexpr int kCpThreads = 128;  // two cells per thread: one tile of 256 cells

template <int Q, class ST, int S>
struct CpRing {
  static constexpr int stages = S;
  static constexpr int epp = 16 / (int)sizeof(typename ST::T);  // values per piece
  static constexpr int pieces = kBulkSeg / epp;                  // per direction
  static constexpr size_t seg_bytes = (size_t)kBulkSeg * sizeof(typename ST::T);
  static constexpr size_t pdf_bytes = (size_t)Q * seg_bytes;
  static constexpr size_t stage_bytes = pdf_bytes + kBulkTX;  // + flag bytes
  // stages, the tile coordinates (x0, row, y, z) of each stage, then a ring
  // of S + 1 tile ids
  static constexpr size_t bytes = stages * stage_bytes + 16 * stages + 4 * (stages + 1);
  static_assert(seg_bytes % 16 == 0 && stage_bytes % 16 == 0, "16-byte pieces");
  static_assert(kBulkSeg % epp == 0 && kBulkHalo % epp == 0, "whole pieces");
};

// c_iy + 1 and c_iz + 1 of directions 0..26, two bits each (shift 2 i)
__host__ __device__ constexpr unsigned long long pack_cyz(int a) {
  unsigned long long v = 0;
  for (int i = 0; i < 27; ++i) v |= (unsigned long long)(dir_c(i, a) + 1) << (2 * i);
  return v;
}

// Update of two neighbouring cells (xa, xa + 1) from a staged tile in two
// sweeps (collide_2s): the pulled pairs are read out of shared memory once per
// sweep instead of being held in registers.  Cells with a wall or obstacle in
// their stencil, and (edge = true) cells at the two ends of a periodic row
// whose wrapped halo is not staged, take their pulled values from pull_one.
// Same bits as bulk_pair.  Returns whether a liquid cell reached
// |u|^2 >= 1/3.
template <int Q, class ST>
__device__ __forceinline__ bool pair_2s(const typename ST::T* __restrict__ A,
                                        typename ST::T* __restrict__ B,
                                        const typename ST::T* stage, int seg, int li, int xa,
                                        int row, int y, int z, uint8_t fl0, uint8_t fl1,
                                        const uint8_t* flags, const Geom& g, const Phys& p,
                                        const LesLp& les, bool edge) {
  using T = typename ST::T;
  constexpr float S = ST::kScaleF;
  const bool liq0 = (fl0 & F_TYPE) == T_LIQ, liq1 = (fl1 & F_TYPE) == T_LIQ;
  if (!liq0 && !liq1) return false;
  const bool near0 = liq0 && ((fl0 & F_NEAR_OBST) || (edge && (xa == 0 || xa == g.nx - 1)));
  const bool near1 = liq1 && ((fl1 & F_NEAR_OBST) || (edge && xa + 1 == g.nx - 1));
  const long long P = g.plane;
  const long long c = (long long)row * g.sx + xa;
  auto fetch = [&](int i) -> float2 {
    const int cx = dir_c(i, 0);
    float2 v;
    if constexpr (sizeof(T) == 2) {
      const unsigned short* sg = reinterpret_cast<const unsigned short*>(stage) + (size_t)i * seg;
      unsigned wv;
      if (cx == 0) wv = *reinterpret_cast<const unsigned*>(sg + li);
      else wv = (unsigned)sg[li - cx] | ((unsigned)sg[li + 1 - cx] << 16);
      v = ST::unpack2(wv);
    } else {
      const T* sg = stage + (size_t)i * seg;
      if (cx == 0) v = *reinterpret_cast<const float2*>(sg + li);
      else v = make_float2(ST::ld1s(sg + li - cx), ST::ld1s(sg + li + 1 - cx));
    }
    if (near0) v.x = pull_one<Q, ST>(A, P, flags, g, xa, y, z, i);
    if (near1) v.y = pull_one<Q, ST>(A, P, flags, g, xa + 1, y, z, i);
    return v;
  };
  T* out = B + c;
  auto emit = [&](int i, float2 o) {
    if (liq0 && liq1) ST::st2(out + i * P, o.x, o.y);
    else if (liq0) ST::st1(out + i * P, o.x);
    else ST::st1(out + i * P + 1, o.y);
  };
  const bool tr = p.trt != 0;
  const float lamE = p.f.lam_e, lamO = tr ? p.f.lam_o : p.f.omega;
  const float pe = p.f.pre_e, po = tr ? p.f.pre_o : p.f.pre_e;
  const float2 usq = collide_2s<Q>(fetch, emit, lamE, lamO, pe, po, p.f.g[0], p.f.g[1], p.f.g[2],
                                   S, les);
  return (liq0 && !(usq.x < (float)(1.0 / 3.0))) || (liq1 && !(usq.y < (float)(1.0 / 3.0)));
}

// Persistent bulk kernel: tiles handed out dynamically, staged by cp.async,
// collided in two sweeps.  The block takes its next tile from a counter in
// the control block (thread 0, one tile ahead of the copies that need it), so
// that slow tiles (rows along a wall) do not leave other SMs idle; the tile
// ids travel to the other threads through a small ring in shared memory that
// the two barriers of each iteration order.  The last block to finish resets
// the counter for the next launch.  Along a periodic x axis with a width that
// is a multiple of 8 the halos are staged from the other end of the row;
// otherwise the cells at the row ends, like cells next to a wall, read their
// pulled values directly (pull_one).
template <int Q, class ST, int S, int MINB>
__global__ void __launch_bounds__(kCpThreads, MINB)
    k_stream_collide_cpa(Dev d, Geom g, Phys p, int ntx) {
  using T = typename ST::T;
  using RING = CpRing<Q, ST, S>;
  constexpr int EPP = RING::epp, NPC = RING::pieces;
  constexpr int NPIECE = Q * NPC + kBulkTX / 16;  // + flag pieces
  constexpr int PER_T = (NPIECE + kCpThreads - 1) / kCpThreads;
  constexpr unsigned long long CY = pack_cyz(1), CZ = pack_cyz(2);
  extern __shared__ __align__(128) unsigned char smem[];
  int4* tile_of = reinterpret_cast<int4*>(smem + S * RING::stage_bytes);
  int* tid_ring = reinterpret_cast<int*>(tile_of + S);  // S + 1 tile ids
  Ctrl* ctrl = d.ctrl;
  if (frozen(ctrl)) return;
  const int ntl = (int)ctrl->n_tiles;
  const int cur = ctrl->step & 1;
  const T* __restrict__ A = (const T*)d.pdf[cur];
  T* __restrict__ B = (T*)d.pdf[cur ^ 1];
  const long long P = g.plane;
  const int t = threadIdx.x, lane = t & 31;
  const bool wrapx = g.periodic[0] && (g.nx % EPP) == 0 && g.nx >= kBulkHalo;

  // copies of tile list entry u into stage s (block-uniform call; one commit
  // group per call, empty past the end of the list)
  auto issue = [&](int u, int s) {
    if (u < ntl) {
      const int k = d.l_tiles[u];
      const int x0 = (k % ntx) * kBulkTX;
      const int row = k / ntx;
      const int y = row % g.ny, z = row / g.ny;
      unsigned char* stage = smem + (size_t)s * RING::stage_bytes;
      if (t == 0) tile_of[s] = make_int4(x0, row, y, z);
      const int ym = y > 0 ? y - 1 : (g.periodic[1] ? g.ny - 1 : y);
      const int yp = y < g.ny - 1 ? y + 1 : (g.periodic[1] ? 0 : y);
      const int zm = z > 0 ? z - 1 : (g.periodic[2] ? g.nz - 1 : z);
      const int zp = z < g.nz - 1 ? z + 1 : (g.periodic[2] ? 0 : z);
#pragma unroll
      for (int kk = 0; kk < PER_T; ++kk) {
        const int c = t + kk * kCpThreads;
        if (c >= NPIECE) break;
        if (c < Q * NPC) {
          const int i = c / NPC, r = c - i * NPC;
          int xs = x0 - kBulkHalo + EPP * r;
          if (xs < 0) {
            if (!wrapx) continue;
            xs += g.nx;
          } else if (xs >= g.nx) {
            if (!wrapx || xs != g.nx) continue;
            xs = 0;
          }
          const int cy = (int)((CY >> (2 * i)) & 3ull) - 1;
          const int cz = (int)((CZ >> (2 * i)) & 3ull) - 1;
          const int ys = cy == 0 ? y : (cy == 1 ? ym : yp);
          const int zs = cz == 0 ? z : (cz == 1 ? zm : zp);
          const T* src = A + (long long)i * P + (long long)g.sx * (ys + (long long)g.ny * zs) + xs;
          cp_async16(stage + (size_t)i * RING::seg_bytes + 16 * r, src);
        } else {
          const int r = c - Q * NPC;
          if (x0 + 16 * r < g.sx)
            cp_async16(stage + RING::pdf_bytes + 16 * r, d.flags + (long long)row * g.sx + x0 + 16 * r);
        }
      }
    }
    cp_async_commit();
  };

  if (t == 0)
    for (int m = 0; m < S; ++m) tid_ring[m] = (int)atomicAdd(&ctrl->tile_next, 1u);
  __syncthreads();
#pragma unroll
  for (int m = 0; m < S - 1; ++m) issue(tid_ring[m], m);
  const LesLp les = LesLp::of(p);
  bool bad = false;
  for (int j = 0;; ++j) {
    issue(tid_ring[(j + S - 1) % (S + 1)], (j + S - 1) % S);
    cp_async_wait<S - 1>();  // this thread's pieces of tile j have landed
    __syncthreads();         // ... and every other thread's
    const int u = tid_ring[j % (S + 1)];
    if (u >= ntl) break;     // block-uniform; later ids are larger still
    if (t == 0) tid_ring[(j + S) % (S + 1)] = (int)atomicAdd(&ctrl->tile_next, 1u);
    const int s = j % S;
    const unsigned char* stage = smem + (size_t)s * RING::stage_bytes;
    const int4 tc = tile_of[s];
    const int xa = tc.x + 2 * t;
    const uchar2 f2 = *reinterpret_cast<const uchar2*>(stage + RING::pdf_bytes + 2 * t);
    const uint8_t fl0 = xa < g.nx ? f2.x : (uint8_t)T_GAS;
    const uint8_t fl1 = xa + 1 < g.nx ? f2.y : (uint8_t)T_GAS;
    bad |= pair_2s<Q, ST>(A, B, reinterpret_cast<const T*>(stage), kBulkSeg, kBulkHalo + 2 * t,
                          xa, tc.y, tc.z, tc.w, fl0, fl1, d.flags, g, p, les,
                          g.periodic[0] && !wrapx);
    __syncthreads();  // the stage and the ring slot are read before they are refilled
  }
  cp_async_wait<0>();
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicCAS(&ctrl->unstable_step, -1, ctrl->step + 1);
  if (t == 0) {
    __threadfence();
    if (atomicAdd(&ctrl->tile_done, 1u) == gridDim.x - 1) {
      ctrl->tile_next = 0;
      ctrl->tile_done = 0;
    }
  }
}

}  // namespace fsl
