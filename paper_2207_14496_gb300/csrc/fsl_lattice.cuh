// Lattice tables, storage traits and small device helpers of libfsl.
//
// Direction order: rest, 6 faces, 12 edges, 8 corners; opposite pairs are
// (1,2), (3,4), ...; D3Q19 is the first 19 directions of D3Q27.  Weights:
// D3Q19 1/3, 1/18, 1/36 (Krueger et al. 2017, Table 3.3); D3Q27 8/27, 2/27,
// 1/54, 1/216.  c_s^2 = 1/3 (the paper's "sqrt(1/3)" in Sec. 2.1 is a typo:
// p0 = c_s^2 rho0 = 1/3).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "fsl_internal.h"

namespace fsl {

__host__ __device__ constexpr int dir_c(int i, int a) {
  constexpr int D[27][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                            {0, 0, 1},   {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                            {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
                            {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},  {1, 1, 1},
                            {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1},
                            {-1, 1, 1},  {1, -1, -1}};
  return D[i][a];
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr int len2(int i) {
  return dir_c(i, 0) * dir_c(i, 0) + dir_c(i, 1) * dir_c(i, 1) + dir_c(i, 2) * dir_c(i, 2);
}
template <int Q>
__host__ __device__ constexpr double wgt(int i) {
  return Q == 19 ? (len2(i) == 0 ? 1.0 / 3.0 : len2(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0)
                 : (len2(i) == 0 ? 8.0 / 27.0
                                 : len2(i) == 1 ? 2.0 / 27.0 : len2(i) == 2 ? 1.0 / 54.0 : 1.0 / 216.0);
}

// Runtime-indexed copies of the same tables for loops that are not unrolled.
static __constant__ int kDirC[27][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},  {1, 1, 1},   {-1, -1, -1},
    {1, 1, -1},  {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};
static __constant__ double kW19[19] = {
    wgt<19>(0),  wgt<19>(1),  wgt<19>(2),  wgt<19>(3),  wgt<19>(4),  wgt<19>(5),  wgt<19>(6),
    wgt<19>(7),  wgt<19>(8),  wgt<19>(9),  wgt<19>(10), wgt<19>(11), wgt<19>(12), wgt<19>(13),
    wgt<19>(14), wgt<19>(15), wgt<19>(16), wgt<19>(17), wgt<19>(18)};
static __constant__ double kW27[27] = {
    wgt<27>(0),  wgt<27>(1),  wgt<27>(2),  wgt<27>(3),  wgt<27>(4),  wgt<27>(5),  wgt<27>(6),
    wgt<27>(7),  wgt<27>(8),  wgt<27>(9),  wgt<27>(10), wgt<27>(11), wgt<27>(12), wgt<27>(13),
    wgt<27>(14), wgt<27>(15), wgt<27>(16), wgt<27>(17), wgt<27>(18), wgt<27>(19), wgt<27>(20),
    wgt<27>(21), wgt<27>(22), wgt<27>(23), wgt<27>(24), wgt<27>(25), wgt<27>(26)};
__device__ __forceinline__ int rc(int i, int a) { return kDirC[i][a]; }
template <int Q>
__device__ __forceinline__ double rw(int i) {
  return Q == 19 ? kW19[i] : kW27[i];
}

// (a x + b y) + c z for integer a, b, c in {-1, 0, 1}, summed left to right
// with the zero terms left out.  Equal to the full expression up to the sign
// of an exact zero, which no later operation observes.
template <int A, int B, int C, class R>
__device__ __forceinline__ R dot3(R x, R y, R z) {
  R acc = R(0);
  bool has = false;
  if (A != 0) { acc = (A == 1) ? x : -x; has = true; }
  if (B != 0) { R t = (B == 1) ? y : -y; acc = has ? acc + t : t; has = true; }
  if (C != 0) { R t = (C == 1) ? z : -z; acc = has ? acc + t : t; has = true; }
  return acc;
}

// Same with the coefficients as (unrolled-loop) values instead of template
// arguments.
template <class R>
__device__ __forceinline__ R dot3r(int a, int b, int c, R x, R y, R z) {
  R acc = R(0);
  bool has = false;
  if (a != 0) { acc = (a == 1) ? x : -x; has = true; }
  if (b != 0) { R t = (b == 1) ? y : -y; acc = has ? acc + t : t; has = true; }
  if (c != 0) { R t = (c == 1) ? z : -z; acc = has ? acc + t : t; has = true; }
  return acc;
}

// ----------------------------------------------------------------- storage
// Working representation inside the stream-collide kernel:
//   FP64: f itself (operation order identical to a plain FP64 evaluation);
//   FP32 / FP16 / BF16: the offset d = f - w_i (computed in FP32), which keeps
//   the small deviations from the lattice weights representable.
struct SF64 {
  using T = double;
  using R = double;
  static constexpr bool kShift = false;
  static __device__ __forceinline__ R ldw(const T* p) { return __ldg(p); }
  static __device__ __forceinline__ void stw(T* p, R v) { *p = v; }
  static __device__ __forceinline__ double ldf(const T* p, double) { return __ldg(p); }
  static __device__ __forceinline__ void stf(T* p, double f, double) { *p = f; }
};
struct SF32 {
  using T = float;
  using T2 = float2;
  using R = float;
  static constexpr bool kShift = true;
  static constexpr float kScaleF = 1.0f;
  // raw stored value(s) as float, in storage units (offset x kScaleF)
  static __device__ __forceinline__ float ld1(const T* p) { return __ldg(p); }
  static __device__ __forceinline__ float ld1s(const T* p) { return *p; }
  static __device__ __forceinline__ float2 ld2(const T* p) {
    return __ldg(reinterpret_cast<const float2*>(p));
  }
  static __device__ __forceinline__ void st1(T* p, float a) { *p = a; }
  static __device__ __forceinline__ void st2(T* p, float a, float b) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
  }
  static __device__ __forceinline__ R ldw(const T* p) { return __ldg(p); }
  static __device__ __forceinline__ void stw(T* p, R v) { *p = v; }
  static __device__ __forceinline__ double ldf(const T* p, double w) { return w + (double)__ldg(p); }
  static __device__ __forceinline__ void stf(T* p, double f, double w) { *p = (float)(f - w); }
};
// FP16 offsets scaled by 2^15 so that offsets down to ~1e-9 stay normal and
// offsets up to 2 fit the format's range.
struct SF16 {
  using T = __half;
  using T2 = __half2;
  using R = float;
  static constexpr bool kShift = true;
  static constexpr float kScale = 32768.0f, kInv = 1.0f / 32768.0f;
  static constexpr float kScaleF = 32768.0f;
  static __device__ __forceinline__ float ld1(const T* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ float ld1s(const T* p) { return __half2float(*p); }
  static __device__ __forceinline__ float2 ld2(const T* p) {
    return __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
  }
  static __device__ __forceinline__ void st1(T* p, float a) { *p = __float2half_rn(a); }
  static __device__ __forceinline__ void st2(T* p, float a, float b) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
  }
  // the 16 bits that st1 would store
  static __device__ __forceinline__ unsigned bits(float a) {
    return (unsigned)__half_as_ushort(__float2half_rn(a));
  }
  // two stored values packed in a 32-bit word (low half first) and back
  static __device__ __forceinline__ float2 unpack2(unsigned w) {
    __half2 h;
    memcpy(&h, &w, 4);
    return __half22float2(h);
  }
  static __device__ __forceinline__ unsigned pack2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    unsigned w;
    memcpy(&w, &h, 4);
    return w;
  }
  static __device__ __forceinline__ R ldw(const T* p) { return __half2float(__ldg(p)) * kInv; }
  static __device__ __forceinline__ void stw(T* p, R v) { *p = __float2half_rn(v * kScale); }
  static __device__ __forceinline__ double ldf(const T* p, double w) {
    return w + (double)(__half2float(__ldg(p)) * kInv);
  }
  static __device__ __forceinline__ void stf(T* p, double f, double w) {
    *p = __float2half_rn((float)(f - w) * kScale);
  }
};
struct SBF16 {
  using T = __nv_bfloat16;
  using T2 = __nv_bfloat162;
  using R = float;
  static constexpr bool kShift = true;
  static constexpr float kScaleF = 1.0f;
  static __device__ __forceinline__ float ld1(const T* p) { return __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ float ld1s(const T* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ float2 ld2(const T* p) {
    return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
  }
  static __device__ __forceinline__ void st1(T* p, float a) { *p = __float2bfloat16_rn(a); }
  static __device__ __forceinline__ void st2(T* p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
  }
  static __device__ __forceinline__ unsigned bits(float a) {
    return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(a));
  }
  static __device__ __forceinline__ float2 unpack2(unsigned w) {
    __nv_bfloat162 h;
    memcpy(&h, &w, 4);
    return __bfloat1622float2(h);
  }
  static __device__ __forceinline__ unsigned pack2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    unsigned w;
    memcpy(&w, &h, 4);
    return w;
  }
  static __device__ __forceinline__ R ldw(const T* p) { return __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ void stw(T* p, R v) { *p = __float2bfloat16_rn(v); }
  static __device__ __forceinline__ double ldf(const T* p, double w) {
    return w + (double)__bfloat162float(__ldg(p));
  }
  static __device__ __forceinline__ void stf(T* p, double f, double w) {
    *p = __float2bfloat16_rn((float)(f - w));
  }
};

// ----------------------------------------------------------------- geometry
__device__ __forceinline__ void cell_xyz(const Geom& g, int c, int& x, int& y, int& z) {
  x = c % g.sx;
  int r = c / g.sx;
  y = r % g.ny;
  z = r / g.ny;
}

// Cell at (x + dx, y + dy, z + dz) with periodic wrap; -1 beyond a wall.
__device__ __forceinline__ int nb_at(const Geom& g, int x, int y, int z, int dx, int dy, int dz) {
  x += dx;
  y += dy;
  z += dz;
  if (x < 0 || x >= g.nx) {
    if (!g.periodic[0]) return -1;
    x = ((x % g.nx) + g.nx) % g.nx;
  }
  if (y < 0 || y >= g.ny) {
    if (!g.periodic[1]) return -1;
    y = ((y % g.ny) + g.ny) % g.ny;
  }
  if (z < 0 || z >= g.nz) {
    if (!g.periodic[2]) return -1;
    z = ((z % g.nz) + g.nz) % g.nz;
  }
  return x + g.sx * (y + g.ny * z);
}

__device__ __forceinline__ int type_at(const uint8_t* flags, int c) {
  return c < 0 ? T_OBST : (flags[c] & F_TYPE);
}
__device__ __forceinline__ bool is_fluid(int t) { return t == T_LIQ || t == T_IF; }

// the interface list consumed in step `step` (built by step - 1)
__device__ __forceinline__ int* list_if(const Dev& d, int step) { return (step & 1) ? d.l_if2 : d.l_if; }

// frozen: an instability was latched in an earlier step
__device__ __forceinline__ bool frozen(const Ctrl* ctrl) {
  int u = *(volatile const int*)&ctrl->unstable_step;
  int s = *(volatile const int*)&ctrl->step;
  return u >= 0 && u <= s;
}

// Warp-aggregated append of the lanes whose pred is set to list[*count++].
__device__ __forceinline__ void warp_append(bool pred, int value, unsigned* count, int* list) {
  unsigned mask = __ballot_sync(0xffffffffu, pred);
  if (mask == 0) return;
  int lane = threadIdx.x & 31;
  int leader = __ffs(mask) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(count, (unsigned)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) list[base + __popc(mask & ((1u << lane) - 1u))] = value;
}

// The same for a whole block of NT threads (all of them call it): one atomic
// per block instead of one per warp.  Lists with one entry for most threads
// (the next step's interface list) otherwise queue thousands of same-address
// atomics per step.
template <int NT>
__device__ __forceinline__ void block_append(bool pred, int value, unsigned* count, int* list) {
  constexpr int NW = NT / 32;
  __shared__ unsigned wbase[NW];
  __shared__ unsigned bbase;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  if (lane == 0) wbase[warp] = (unsigned)__popc(mask);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < NW; ++w) {
      const unsigned c = wbase[w];
      wbase[w] = t;
      t += c;
    }
    bbase = t ? atomicAdd(count, t) : 0u;
  }
  __syncthreads();
  if (pred) list[bbase + wbase[warp] + (unsigned)__popc(mask & ((1u << lane) - 1u))] = value;
  __syncthreads();  // wbase and bbase are reused by the block's next call
}

// Atomic OR / AND on the byte of a flag array through its aligned 32-bit word.
__device__ __forceinline__ uint8_t byte_or(uint8_t* a, int c, uint8_t bits) {
  unsigned* word = reinterpret_cast<unsigned*>(reinterpret_cast<uintptr_t>(a + c) & ~uintptr_t(3));
  unsigned sh = 8u * (unsigned)(reinterpret_cast<uintptr_t>(a + c) & 3u);
  unsigned old = atomicOr(word, (unsigned)bits << sh);
  return (uint8_t)(old >> sh);
}
__device__ __forceinline__ void byte_and(uint8_t* a, int c, uint8_t bits) {
  unsigned* word = reinterpret_cast<unsigned*>(reinterpret_cast<uintptr_t>(a + c) & ~uintptr_t(3));
  unsigned sh = 8u * (unsigned)(reinterpret_cast<uintptr_t>(a + c) & 3u);
  atomicAnd(word, ~((unsigned)bits << sh));
}
// Change the type of a cell from `from` to `to` if it still is `from`;
// returns true for the one caller that made the change.  The compare-and-swap
// retries only while other bytes of the same word change; the retry count is
// capped and a cap hit is latched in *err.
__device__ __forceinline__ bool byte_retype(uint8_t* a, int c, int from, int to, unsigned* err) {
  unsigned* word = reinterpret_cast<unsigned*>(reinterpret_cast<uintptr_t>(a + c) & ~uintptr_t(3));
  unsigned sh = 8u * (unsigned)(reinterpret_cast<uintptr_t>(a + c) & 3u);
  unsigned old = *(volatile unsigned*)word;
  for (int tries = 0;; ++tries) {
    if (tries >= (1 << 16)) {
      atomicOr(err, 1u);
      return false;
    }
    unsigned b = (old >> sh) & 0xffu;
    if ((int)(b & F_TYPE) != from) return false;
    unsigned nb = (b & ~(unsigned)F_TYPE) | (unsigned)to;
    unsigned repl = (old & ~(0xffu << sh)) | (nb << sh);
    unsigned prev = atomicCAS(word, old, repl);
    if (prev == old) return true;
    old = prev;
  }
}

}  // namespace fsl
