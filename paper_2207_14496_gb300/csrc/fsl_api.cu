// Host side of the C ABI declared in include/fsl.h: configuration checks,
// workspace carving, initial state, step launches (captured into CUDA graphs),
// observation, checkpointing.  No device memory is allocated here; every
// device buffer is carved out of the caller's workspace.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "fsl.h"
#include "fsl_kernels.cuh"
#include "fsl_adjoint.cuh"

using namespace fsl;

namespace {

thread_local std::string g_err;

fsl_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return FSL_ERR_CUDA;
}
#define FSL_CK(call)                                   \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr long long kPlaneSkew = 512;  // elements added to every PDF plane

enum Region {
  R_PDF0, R_PDF1, R_FLAGS, R_CLAIM, R_PHI, R_PHINEW, R_MASS, R_RHO, R_KAPPA, R_MEX, R_LOST, R_PHIF,
  R_LIF, R_LIF2, R_LFILL, R_LEMPTY, R_LNEW, R_LL2I, R_LRECV, R_LTILES, R_CTRL, R_TRACE, R_RED,
  R_BLAB, R_BNEW, R_BK, R_BKNEW, R_BV, R_BVSEEN, R_BP, R_BHAS, R_SELF, R_COUNT
};

bool valid_config(const fsl_config* c) {
  if (!c) return false;
  if (c->lattice != FSL_D3Q19 && c->lattice != FSL_D3Q27) return false;
  if (c->collision != FSL_SRT && c->collision != FSL_TRT) return false;
  if (c->precision < FSL_FP64 || c->precision > FSL_MIXED_BF16) return false;
  if (c->refill < FSL_REFILL_EQ || c->refill > FSL_REFILL_AVG) return false;
  if (c->nx < 1 || c->ny < 1 || c->nz < 1) return false;
  if (!(c->nu > 0.0) || !std::isfinite(c->nu)) return false;
  if (c->collision == FSL_TRT && !(c->trt_magic > 0.0)) return false;
  if (!(c->eps_phi >= 0.0)) return false;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(c->gravity[a])) return false;
  if (!std::isfinite(c->sigma) || !std::isfinite(c->p_volume)) return false;
  if (!(c->les_cs >= 0.0) || !std::isfinite(c->les_cs)) return false;
  const long long sx = ((long long)c->nx + 31) / 32 * 32;
  const long long cells = sx * c->ny * (long long)c->nz;
  const long long plane = (cells + 127) / 128 * 128 + kPlaneSkew;
  if (plane * (long long)c->lattice >= (1ll << 31) * 8ll) return false;
  if (cells >= (1ll << 31) - 1) return false;
  return true;
}

void make_geom(const fsl_config* c, Geom* g) {
  g->nx = c->nx;
  g->ny = c->ny;
  g->nz = c->nz;
  g->sx = (c->nx + 31) / 32 * 32;
  g->cells = (long long)g->sx * c->ny * c->nz;
  // planes padded to 128 elements plus a skew, so that the q planes (which a
  // warp streams from at once) do not start at multiples of a large power of
  // two from each other and spread over the HBM channels
  g->plane = (g->cells + 127) / 128 * 128 + kPlaneSkew;
  for (int a = 0; a < 3; ++a) g->periodic[a] = c->periodic[a] ? 1 : 0;
  g->has_obst = 0;
  g->variant = FSL_VARIANT_DEFAULT;
  g->free_slip = 0;
  g->bubbles = (c->options & FSL_OPT_BUBBLES) ? 1 : 0;
  g->bub_gas_only = (c->options & FSL_OPT_BUBBLE_GAS_ONLY) ? 1 : 0;
  for (int a = 0; a < 3; ++a)
    if (c->free_slip[a] && !c->periodic[a]) g->free_slip |= 1 << a;
}

void make_phys(const fsl_config* c, Phys* p) {
  std::memset(p, 0, sizeof(*p));
  p->q = c->lattice;
  p->trt = c->collision == FSL_TRT;
  p->refill = c->refill;
  p->options = c->options;
  // Eq. nm-lbm-viscosity: nu = c_s^2 (tau - 1/2)
  p->tau = 3.0 * c->nu + 0.5;
  p->omega = 1.0 / p->tau;
  p->lam_e = p->omega;
  // TRT magic parameter Lambda = (1/lam_e - 1/2)(1/lam_o - 1/2)
  p->lam_o = 1.0 / (0.5 + c->trt_magic / (1.0 / p->lam_e - 0.5));
  p->pre_e = 1.0 - 0.5 * p->lam_e;
  p->pre_o = 1.0 - 0.5 * p->lam_o;
  p->gaxis = -1;
  for (int a = 0; a < 3; ++a) {
    p->g[a] = c->gravity[a];
    if (c->gravity[a] != 0.0) p->gaxis = a;
  }
  p->sigma = c->sigma;
  p->p_v = c->p_volume;
  p->eps = c->eps_phi;
  // GEQ prefactor: 1/(2 c_s^2 omega) = 1.5 tau, or the printed 1/(2 c_s^2 nu)
  p->geq_coef = (c->options & FSL_OPT_GEQ_LITERAL_NU) ? 1.5 / c->nu : 1.5 * p->tau;
  p->thr_hi = 1.0 + c->eps_phi;
  p->thr_lo = 0.0 - c->eps_phi;
  p->magic = c->trt_magic;
  p->les_cs = c->les_cs;
  p->f.tau = (float)p->tau;
  p->f.omega = (float)p->omega;
  p->f.lam_e = (float)p->lam_e;
  p->f.lam_o = (float)p->lam_o;
  p->f.pre_e = (float)p->pre_e;
  p->f.pre_o = (float)p->pre_o;
  for (int a = 0; a < 3; ++a) p->f.g[a] = (float)p->g[a];
  p->f.sigma = (float)p->sigma;
  p->f.p_v = (float)p->p_v;
  p->f.eps = (float)p->eps;
  p->f.geq_coef = (float)p->geq_coef;
  p->f.thr_hi = (float)p->thr_hi;
  p->f.thr_lo = (float)p->thr_lo;
  p->f.magic = (float)p->magic;
  p->f.les_cs = (float)p->les_cs;
  p->f.les_k = (float)(2.0 * std::sqrt(2.0) * p->les_cs * p->les_cs * 9.0);
}

void region_sizes(const fsl_config* c, const Geom& g, size_t* sz) {
  const size_t sb = storage_bytes(c->precision);
  const size_t cells = (size_t)g.cells;
  sz[R_PDF0] = sz[R_PDF1] = (size_t)g.plane * c->lattice * sb;
  sz[R_FLAGS] = sz[R_CLAIM] = cells;
  sz[R_PHI] = sz[R_PHINEW] = sz[R_MASS] = sz[R_RHO] = sz[R_KAPPA] = sz[R_MEX] = sz[R_LOST] =
      cells * sizeof(double);
  // the FP32 copy of the fill level that the 16/32-bit kernels read
  sz[R_PHIF] = c->precision == FSL_FP64 ? 0 : cells * sizeof(float);
  for (int r = R_LIF; r <= R_LRECV; ++r) sz[r] = cells * sizeof(int);
  // tile lists of the shared-memory variants: up to one entry per 64 cells of a row
  sz[R_LTILES] = (size_t)((g.nx + 63) / 64) * g.ny * g.nz * sizeof(int);
  sz[R_CTRL] = sizeof(Ctrl);
  {
    const size_t bc = (c->options & FSL_OPT_BUBBLES) ? cells : 0;
    sz[R_BLAB] = sz[R_BNEW] = bc * sizeof(int);
    sz[R_BK] = sz[R_BKNEW] = sz[R_BV] = sz[R_BVSEEN] = sz[R_BP] = bc * 8;
    sz[R_BHAS] = bc;
  }
  sz[R_TRACE] = (size_t)kTraceCapacity * 3 * sizeof(double);
  sz[R_RED] = (size_t)(2 * kReduceBlocks + 16) * sizeof(double);
  // the handle's own member record for batched launches
  sz[R_SELF] = sizeof(Member);
}

size_t layout(const fsl_config* c, const Geom& g, size_t* off) {
  size_t sz[R_COUNT];
  region_sizes(c, g, sz);
  size_t at = 0;
  for (int r = 0; r < R_COUNT; ++r) {
    off[r] = at;
    at = align256(at + sz[r]);
  }
  return at;
}

const Launch* pick(int precision, int q) {
  const bool q19 = q == 19;
  switch (precision) {
    case FSL_FP64: return q19 ? launch_fp64_q19() : launch_fp64_q27();
    case FSL_FP32: return q19 ? launch_fp32_q19() : launch_fp32_q27();
    case FSL_MIXED_FP16: return q19 ? launch_fp16_q19() : launch_fp16_q27();
    case FSL_MIXED_BF16: return q19 ? launch_bf16_q19() : launch_bf16_q27();
  }
  return nullptr;
}

}  // namespace

void fsl::set_error_text(const char* msg) { g_err = msg ? msg : ""; }

size_t fsl::storage_bytes(int precision) {
  return precision == FSL_FP64 ? 8 : precision == FSL_FP32 ? 4 : 2;
}

// ------------------------------------------------------------ observation kernels
namespace {

// column height at i = 0, front (j = 0 layer) and height (i = 0 column)
__global__ void k_small_obs(Dev d, Geom g, double* out) {
  __shared__ double shd[256];
  __shared__ int shi[256];
  double s = 0.0;
  const int ncol = g.ny * g.nz;
  for (int k = threadIdx.x; k < ncol; k += 256) s += d.phi[(long long)g.sx * k];
  const double col = block_sum<256>(s, shd) / (double)g.nz;
  int best = -1;
  for (int k = threadIdx.x; k < g.nx * g.nz; k += 256) {
    const int i = k % g.nx, kz = k / g.nx;
    if ((d.flags[i + (long long)g.sx * g.ny * kz] & F_TYPE) == T_IF) best = max(best, i);
  }
  const int front = block_max<256>(best, shi) + 1;
  best = -1;
  for (int k = threadIdx.x; k < ncol; k += 256)
    if ((d.flags[(long long)g.sx * k] & F_TYPE) == T_IF) best = max(best, k % g.ny);
  const int height = block_max<256>(best, shi) + 1;
  if (threadIdx.x == 0) {
    out[0] = col;
    out[1] = (double)front;
    out[2] = (double)height;
  }
}

__global__ void __launch_bounds__(256) k_lost_partial(Dev d, Geom g, double* part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (long long c = blockIdx.x * 256ll + threadIdx.x; c < g.cells; c += (long long)gridDim.x * 256)
    if ((int)(c % g.sx) < g.nx) s += d.lost[c];
  const double b = block_sum<256>(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

__global__ void k_count_types(Dev d, Geom g, unsigned long long* out) {
  unsigned long long liq = 0, itf = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.cells;
       c += (long long)gridDim.x * blockDim.x) {
    if ((int)(c % g.sx) >= g.nx) continue;
    const int t = d.flags[c] & F_TYPE;
    liq += (t == T_LIQ);
    itf += (t == T_IF);
  }
  atomicAdd(&out[0], liq);
  atomicAdd(&out[1], itf);
}

__global__ void k_set_trace(Ctrl* ctrl, int every) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctrl->trace_every = every;
    ctrl->trace_count = 0;
  }
}

}  // namespace

// ------------------------------------------------------------ handle
struct fsl_handle {
  fsl_config cfg;
  Geom g;
  Phys p;
  Dev d;
  const Launch* L;
  cudaStream_t stream;
  size_t bytes;
  size_t off[R_COUNT];
  bool ready;
  int trace_every;
  std::map<int, cudaGraphExec_t> graphs;
  unsigned gen = 0;  // bumped whenever captured launch parameters may change
  char* base = nullptr;         // start of the workspace
  Aux aux = {nullptr, nullptr, nullptr};  // side stream of the interface pass
  double h_ref = 0.0;           // hydrostatic reference height of the last fsl_init_fill
};

namespace {

fsl_status read_ctrl(fsl_handle* h, Ctrl* c) {
  FSL_CK(cudaMemcpyAsync(c, h->d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  FSL_CK(cudaStreamSynchronize(h->stream));
  return FSL_OK;
}

fsl_status copy_field(fsl_handle* h, const void* dev, size_t elem, void* host) {
  // padded rows (pitch sx) -> dense host rows (nx)
  FSL_CK(cudaMemcpy2DAsync(host, (size_t)h->g.nx * elem, dev, (size_t)h->g.sx * elem,
                           (size_t)h->g.nx * elem, (size_t)h->g.ny * h->g.nz,
                           cudaMemcpyDeviceToHost, h->stream));
  FSL_CK(cudaStreamSynchronize(h->stream));
  return FSL_OK;
}

const size_t kGraphChunk = 64;

}  // namespace

extern "C" {

fsl_status fsl_workspace_bytes(const fsl_config* cfg, size_t* bytes) {
  if (!valid_config(cfg) || !bytes) return FSL_ERR_ARG;
  Geom g;
  make_geom(cfg, &g);
  size_t off[R_COUNT];
  *bytes = layout(cfg, g, off);
  return FSL_OK;
}

fsl_status fsl_create(const fsl_config* cfg, void* d_workspace, size_t bytes, void* cuda_stream,
                      fsl_handle** out) {
  if (!out) return FSL_ERR_ARG;
  *out = nullptr;
  if (!valid_config(cfg)) return FSL_ERR_ARG;
  if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u)) return FSL_ERR_WORKSPACE;
  const Launch* L = pick(cfg->precision, cfg->lattice);
  if (!L) return FSL_ERR_ARG;
  fsl_handle* h = new (std::nothrow) fsl_handle();
  if (!h) return FSL_ERR_ARG;
  h->cfg = *cfg;
  make_geom(cfg, &h->g);
  make_phys(cfg, &h->p);
  h->bytes = layout(cfg, h->g, h->off);
  if (bytes < h->bytes) {
    delete h;
    return FSL_ERR_WORKSPACE;
  }
  char* base = static_cast<char*>(d_workspace);
  h->base = base;
  Dev& d = h->d;
  d.pdf[0] = base + h->off[R_PDF0];
  d.pdf[1] = base + h->off[R_PDF1];
  d.flags = reinterpret_cast<uint8_t*>(base + h->off[R_FLAGS]);
  d.claim = reinterpret_cast<uint8_t*>(base + h->off[R_CLAIM]);
  d.phi = reinterpret_cast<double*>(base + h->off[R_PHI]);
  d.phinew = reinterpret_cast<double*>(base + h->off[R_PHINEW]);
  d.phif = cfg->precision == FSL_FP64 ? nullptr : reinterpret_cast<float*>(base + h->off[R_PHIF]);
  d.mass = reinterpret_cast<double*>(base + h->off[R_MASS]);
  d.rho = reinterpret_cast<double*>(base + h->off[R_RHO]);
  d.kappa = reinterpret_cast<double*>(base + h->off[R_KAPPA]);
  d.mex = reinterpret_cast<double*>(base + h->off[R_MEX]);
  d.lost = reinterpret_cast<double*>(base + h->off[R_LOST]);
  d.l_if = reinterpret_cast<int*>(base + h->off[R_LIF]);
  d.l_if2 = reinterpret_cast<int*>(base + h->off[R_LIF2]);
  d.l_fill = reinterpret_cast<int*>(base + h->off[R_LFILL]);
  d.l_empty = reinterpret_cast<int*>(base + h->off[R_LEMPTY]);
  d.l_new = reinterpret_cast<int*>(base + h->off[R_LNEW]);
  d.l_l2i = reinterpret_cast<int*>(base + h->off[R_LL2I]);
  d.l_recv = reinterpret_cast<int*>(base + h->off[R_LRECV]);
  d.l_tiles = reinterpret_cast<int*>(base + h->off[R_LTILES]);
  d.ctrl = reinterpret_cast<Ctrl*>(base + h->off[R_CTRL]);
  d.blab = reinterpret_cast<int*>(base + h->off[R_BLAB]);
  d.bnew = reinterpret_cast<int*>(base + h->off[R_BNEW]);
  d.bK = reinterpret_cast<double*>(base + h->off[R_BK]);
  d.bKnew = reinterpret_cast<long long*>(base + h->off[R_BKNEW]);
  d.bV = reinterpret_cast<long long*>(base + h->off[R_BV]);
  d.bVseen = reinterpret_cast<long long*>(base + h->off[R_BVSEEN]);
  d.bp = reinterpret_cast<double*>(base + h->off[R_BP]);
  d.bhas = reinterpret_cast<uint8_t*>(base + h->off[R_BHAS]);
  d.trace = reinterpret_cast<double*>(base + h->off[R_TRACE]);
  d.red = reinterpret_cast<double*>(base + h->off[R_RED]);
  d.redi = nullptr;
  h->L = L;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  {
    // the interface pass runs on a high-priority side stream beside the bulk
    // pass; if it cannot be created the step uses one stream
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    Aux a = {nullptr, nullptr, nullptr};
    if (cudaStreamCreateWithPriority(&a.side, cudaStreamNonBlocking, hi) == cudaSuccess &&
        cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming) == cudaSuccess) {
      h->aux = a;
    } else {
      if (a.join) cudaEventDestroy(a.join);
      if (a.fork) cudaEventDestroy(a.fork);
      if (a.side) cudaStreamDestroy(a.side);
      cudaGetLastError();
    }
  }
  h->ready = false;
  h->trace_every = 0;
  *out = h;
  return FSL_OK;
}

fsl_status fsl_init_fill(fsl_handle* h, const double* phi, const double* u0,
                         const unsigned char* obstacle, double h_ref) {
  if (!h || !phi) return FSL_ERR_ARG;
  const size_t n = (size_t)h->g.nx * h->g.ny * h->g.nz;
  // staging: fill level in phinew, obstacle bytes in claim, u0 in the second
  // PDF buffer (all unpadded); the init kernels move them into place
  FSL_CK(cudaMemcpyAsync(h->d.phinew, phi, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  if (obstacle)
    FSL_CK(cudaMemcpyAsync(h->d.claim, obstacle, n, cudaMemcpyHostToDevice, h->stream));
  double* su = nullptr;
  if (u0) {
    su = static_cast<double*>(h->d.pdf[1]);
    FSL_CK(cudaMemcpyAsync(su, u0, 3 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  }
  // interior obstacles disable the obstacle-free fast paths; captured step
  // graphs hold the geometry by value and are rebuilt
  h->g.has_obst = 0;
  if (obstacle)
    for (size_t k = 0; k < n; ++k)
      if (obstacle[k]) { h->g.has_obst = 1; break; }
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  ++h->gen;
  h->h_ref = h_ref;
  FSL_CK(h->L->init(h->d, h->g, h->p, 0, su, obstacle ? 1 : 0, h_ref, h->stream));
  k_set_trace<<<1, 32, 0, h->stream>>>(h->d.ctrl, h->trace_every);
  FSL_CK(cudaGetLastError());
  FSL_CK(cudaStreamSynchronize(h->stream));
  h->ready = true;
  return FSL_OK;
}

fsl_status fsl_step(fsl_handle* h, int nsteps) {
  if (!h || nsteps < 0) return FSL_ERR_ARG;
  if (!h->ready) return FSL_ERR_STATE;
  if (nsteps == 0) return FSL_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (h->stream) FSL_CK(cudaStreamIsCapturing(h->stream, &cs));
  if (!h->stream || cs != cudaStreamCaptureStatusNone) {
    // legacy default stream (not capturable) or a capture owned by the caller
    for (int k = 0; k < nsteps; ++k) FSL_CK(h->L->step(h->d, h->g, h->p, h->stream, h->aux));
    return FSL_OK;
  }
  int left = nsteps;
  while (left > 0) {
    const int chunk = left >= (int)kGraphChunk ? (int)kGraphChunk : left;
    auto it = h->graphs.find(chunk);
    if (it == h->graphs.end()) {
      cudaGraph_t graph;
      FSL_CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t le = cudaSuccess;
      for (int k = 0; k < chunk && le == cudaSuccess; ++k) le = h->L->step(h->d, h->g, h->p, h->stream, h->aux);
      cudaError_t ee = cudaStreamEndCapture(h->stream, &graph);
      if (le != cudaSuccess) return cuda_fail(le, "step launch during capture");
      if (ee != cudaSuccess) return cuda_fail(ee, "cudaStreamEndCapture");
      cudaGraphExec_t exec;
      cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
      it = h->graphs.emplace(chunk, exec).first;
    }
    FSL_CK(cudaGraphLaunch(it->second, h->stream));
    left -= chunk;
  }
  return FSL_OK;
}

fsl_status fsl_observe(fsl_handle* h, int what, void* host_out, size_t bytes) {
  if (!h || !host_out) return FSL_ERR_ARG;
  if (!h->ready) return FSL_ERR_STATE;
  const size_t n = (size_t)h->g.nx * h->g.ny * h->g.nz;
  const int q = h->cfg.lattice;
  Ctrl c;
  fsl_status st = read_ctrl(h, &c);
  if (st != FSL_OK) return st;
  const int cur = c.step & 1;
  double* dout = h->d.red + 2 * kReduceBlocks;  // device result slots
  switch (what) {
    case FSL_OBS_TOTAL_MASS:
    case FSL_OBS_MAX_VELOCITY:
    case FSL_OBS_LOST_MASS: {
      if (bytes < sizeof(double)) return FSL_ERR_ARG;
      if (what == FSL_OBS_TOTAL_MASS) FSL_CK(h->L->total_mass(h->d, h->g, h->p, cur, dout, h->stream));
      else if (what == FSL_OBS_MAX_VELOCITY)
        FSL_CK(h->L->max_velocity(h->d, h->g, h->p, cur, dout, h->stream));
      else {
        k_lost_partial<<<kReduceBlocks, 256, 0, h->stream>>>(h->d, h->g, h->d.red);
        k_sum_partials<<<1, 256, 0, h->stream>>>(h->d.red, kReduceBlocks, dout);
        FSL_CK(cudaGetLastError());
      }
      FSL_CK(cudaMemcpyAsync(host_out, dout, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      FSL_CK(cudaStreamSynchronize(h->stream));
      return FSL_OK;
    }
    case FSL_OBS_COLUMN_HEIGHT:
    case FSL_OBS_FRONT:
    case FSL_OBS_HEIGHT: {
      if (bytes < sizeof(double)) return FSL_ERR_ARG;
      k_small_obs<<<1, 256, 0, h->stream>>>(h->d, h->g, dout);
      FSL_CK(cudaGetLastError());
      double v[3];
      FSL_CK(cudaMemcpyAsync(v, dout, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
      FSL_CK(cudaStreamSynchronize(h->stream));
      const double r = what == FSL_OBS_COLUMN_HEIGHT ? v[0] : what == FSL_OBS_FRONT ? v[1] : v[2];
      std::memcpy(host_out, &r, sizeof(double));
      return FSL_OK;
    }
    case FSL_OBS_STATUS: {
      if (bytes < 2 * sizeof(int64_t)) return FSL_ERR_ARG;
      int64_t v[2] = {c.unstable_step >= 0 ? (int64_t)FSL_ERR_UNSTABLE
                                           : (c.timeout ? (int64_t)FSL_ERR_TIMEOUT : 0),
                      (int64_t)c.unstable_step};
      std::memcpy(host_out, v, sizeof(v));
      return FSL_OK;
    }
    case FSL_OBS_STEP: {
      if (bytes < sizeof(int64_t)) return FSL_ERR_ARG;
      int64_t v = c.step;
      std::memcpy(host_out, &v, sizeof(v));
      return FSL_OK;
    }
    case FSL_OBS_COUNTS: {
      if (bytes < 4 * sizeof(int64_t)) return FSL_ERR_ARG;
      int64_t v[4] = {c.last[0], c.last[1], c.last[2], c.last[3]};
      std::memcpy(host_out, v, sizeof(v));
      return FSL_OK;
    }
    case FSL_OBS_TRACE: {
      const int cnt = c.trace_count < kTraceCapacity ? c.trace_count : kTraceCapacity;
      if (bytes < (size_t)cnt * 3 * sizeof(double)) return FSL_ERR_ARG;
      std::vector<double> ring((size_t)kTraceCapacity * 3);
      FSL_CK(cudaMemcpyAsync(ring.data(), h->d.trace, ring.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
      FSL_CK(cudaStreamSynchronize(h->stream));
      const int first = c.trace_count - cnt;
      double* o = static_cast<double*>(host_out);
      for (int k = 0; k < cnt; ++k) {
        const int slot = (first + k) % kTraceCapacity;
        for (int j = 0; j < 3; ++j) o[3 * k + j] = ring[3 * slot + j];
      }
      return FSL_OK;
    }
    case FSL_OBS_FIELD_PDF: {
      if (bytes < (size_t)q * n * sizeof(double)) return FSL_ERR_ARG;
      double* o = static_cast<double*>(host_out);
      for (int i = 0; i < q; ++i) {
        FSL_CK(h->L->export_pdf(h->d, h->g, h->p, cur, i, h->d.phinew, h->stream));
        FSL_CK(cudaMemcpyAsync(o + (size_t)i * n, h->d.phinew, n * sizeof(double),
                               cudaMemcpyDeviceToHost, h->stream));
      }
      FSL_CK(cudaStreamSynchronize(h->stream));
      return FSL_OK;
    }
    case FSL_OBS_FIELD_TYPES: {
      if (bytes < n) return FSL_ERR_ARG;
      st = copy_field(h, h->d.flags, 1, host_out);
      if (st != FSL_OK) return st;
      unsigned char* o = static_cast<unsigned char*>(host_out);
      for (size_t k = 0; k < n; ++k) o[k] &= F_TYPE;
      return FSL_OK;
    }
    case FSL_OBS_FIELD_PHI:
      if (bytes < n * sizeof(double)) return FSL_ERR_ARG;
      return copy_field(h, h->d.phi, sizeof(double), host_out);
    case FSL_OBS_FIELD_MASS:
      if (bytes < n * sizeof(double)) return FSL_ERR_ARG;
      return copy_field(h, h->d.mass, sizeof(double), host_out);
    case FSL_OBS_FIELD_KAPPA:
      if (bytes < n * sizeof(double)) return FSL_ERR_ARG;
      return copy_field(h, h->d.kappa, sizeof(double), host_out);
    case FSL_OBS_FIELD_BUBBLE: {
      if (bytes < n * sizeof(int)) return FSL_ERR_ARG;
      int* o = static_cast<int*>(host_out);
      if (!h->g.bubbles) {
        for (size_t k = 0; k < n; ++k) o[k] = -1;
        return FSL_OK;
      }
      fsl_status st2 = copy_field(h, h->d.blab, sizeof(int), host_out);
      if (st2 != FSL_OK) return st2;
      // padded cell index -> dense index x + nx (y + ny z)
      for (size_t k = 0; k < n; ++k)
        if (o[k] >= 0) o[k] = (o[k] % h->g.sx) + h->g.nx * (o[k] / h->g.sx);
      return FSL_OK;
    }
    case FSL_OBS_FIELD_PRESSURE: {
      if (bytes < n * sizeof(double)) return FSL_ERR_ARG;
      if (!h->g.bubbles) {
        double* o = static_cast<double*>(host_out);
        for (size_t k = 0; k < n; ++k) o[k] = h->p.p_v;
        return FSL_OK;
      }
      // the pressure lives at each bubble's root: expand it per cell into the
      // next-K scratch, which the next step re-initialises anyway
      double* tmp = reinterpret_cast<double*>(h->d.bKnew);
      k_bub_expand<<<(unsigned)((h->g.cells + 255) / 256), 256, 0, h->stream>>>(h->d, h->g,
                                                                              h->p.p_v, tmp);
      FSL_CK(cudaGetLastError());
      return copy_field(h, tmp, sizeof(double), host_out);
    }
  }
  return FSL_ERR_ARG;
}

fsl_status fsl_set_trace(fsl_handle* h, int every) {
  if (!h || every < 0) return FSL_ERR_ARG;
  h->trace_every = every;
  if (h->ready) {
    k_set_trace<<<1, 32, 0, h->stream>>>(h->d.ctrl, every);
    FSL_CK(cudaGetLastError());
  }
  return FSL_OK;
}

int fsl_trace_capacity(void) { return kTraceCapacity; }

// checkpoint: current PDF buffer, flags, phi, mass, kappa, lost, control block
fsl_status fsl_state_bytes(const fsl_handle* h, size_t* bytes) {
  if (!h || !bytes) return FSL_ERR_ARG;
  size_t sz[R_COUNT];
  region_sizes(&h->cfg, h->g, sz);
  *bytes = sz[R_PDF0] + sz[R_FLAGS] + sz[R_PHI] + sz[R_MASS] + sz[R_KAPPA] + sz[R_LOST] +
           sz[R_BLAB] + sz[R_BK] + sz[R_BP] + sizeof(Ctrl);
  return FSL_OK;
}

static fsl_status state_parts(fsl_handle* h, int cur, std::vector<std::pair<char*, size_t>>& parts) {
  size_t sz[R_COUNT];
  region_sizes(&h->cfg, h->g, sz);
  parts.clear();
  parts.push_back({static_cast<char*>(h->d.pdf[cur]), sz[R_PDF0]});
  parts.push_back({reinterpret_cast<char*>(h->d.flags), sz[R_FLAGS]});
  parts.push_back({reinterpret_cast<char*>(h->d.phi), sz[R_PHI]});
  parts.push_back({reinterpret_cast<char*>(h->d.mass), sz[R_MASS]});
  parts.push_back({reinterpret_cast<char*>(h->d.kappa), sz[R_KAPPA]});
  parts.push_back({reinterpret_cast<char*>(h->d.lost), sz[R_LOST]});
  if (h->g.bubbles) {
    parts.push_back({reinterpret_cast<char*>(h->d.blab), sz[R_BLAB]});
    parts.push_back({reinterpret_cast<char*>(h->d.bK), sz[R_BK]});
    parts.push_back({reinterpret_cast<char*>(h->d.bp), sz[R_BP]});
  }
  return FSL_OK;
}

fsl_status fsl_save(fsl_handle* h, void* host_dst, size_t bytes) {
  if (!h || !host_dst) return FSL_ERR_ARG;
  if (!h->ready) return FSL_ERR_STATE;
  size_t need;
  fsl_state_bytes(h, &need);
  if (bytes < need) return FSL_ERR_ARG;
  Ctrl c;
  fsl_status st = read_ctrl(h, &c);
  if (st != FSL_OK) return st;
  std::vector<std::pair<char*, size_t>> parts;
  state_parts(h, c.step & 1, parts);
  char* o = static_cast<char*>(host_dst);
  for (auto& pr : parts) {
    FSL_CK(cudaMemcpyAsync(o, pr.first, pr.second, cudaMemcpyDeviceToHost, h->stream));
    o += pr.second;
  }
  FSL_CK(cudaStreamSynchronize(h->stream));
  std::memcpy(o, &c, sizeof(Ctrl));
  return FSL_OK;
}

fsl_status fsl_load(fsl_handle* h, const void* host_src, size_t bytes) {
  if (!h || !host_src) return FSL_ERR_ARG;
  size_t need;
  fsl_state_bytes(h, &need);
  if (bytes < need) return FSL_ERR_ARG;
  Ctrl c;
  std::memcpy(&c, static_cast<const char*>(host_src) + need - sizeof(Ctrl), sizeof(Ctrl));
  if (c.step < 0) return FSL_ERR_ARG;
  std::vector<std::pair<char*, size_t>> parts;
  state_parts(h, c.step & 1, parts);
  const char* s = static_cast<const char*>(host_src);
  // the flag bytes follow the PDF buffer: interior obstacles switch the
  // obstacle-free fast paths off, and captured graphs hold the geometry
  const unsigned char* fl = reinterpret_cast<const unsigned char*>(s + parts[0].second);
  h->g.has_obst = 0;
  for (int z = 0; z < h->g.nz && !h->g.has_obst; ++z)
    for (int y = 0; y < h->g.ny && !h->g.has_obst; ++y)
      for (int x = 0; x < h->g.nx; ++x)
        if ((fl[x + (size_t)h->g.sx * (y + (size_t)h->g.ny * z)] & F_TYPE) == T_OBST) {
          h->g.has_obst = 1;
          break;
        }
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  ++h->gen;
  for (auto& pr : parts) {
    FSL_CK(cudaMemcpyAsync(pr.first, s, pr.second, cudaMemcpyHostToDevice, h->stream));
    s += pr.second;
  }
  // per-step scratch restarts empty: counters zero, claim bytes zero
  c.n_if = c.n_fill = c.n_empty = c.n_new = c.n_l2i = c.n_recv = 0;
  c.n_emptied = c.end_blocks = c.n_tiles = 0;
  c.tile_next = c.tile_done = 0;
  c.bar = 0;
  c.trace_every = h->trace_every;
  c.trace_count = 0;
  c.n_if_next = 0;
  FSL_CK(cudaMemcpyAsync(h->d.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
  FSL_CK(cudaMemsetAsync(h->d.claim, 0, (size_t)h->g.cells, h->stream));
  // the interface list of the loaded step, from the loaded flags
  k_list_interface<<<4 * 152, 256, 0, h->stream>>>(h->d, h->g);
  FSL_CK(cudaGetLastError());
  // the FP32 copy of the loaded fill levels
  if (h->d.phif) {
    k_phif_from_phi<<<4 * 152, 256, 0, h->stream>>>(h->d, h->g);
    FSL_CK(cudaGetLastError());
  }
  FSL_CK(cudaStreamSynchronize(h->stream));
  h->ready = true;
  return FSL_OK;
}

fsl_status fsl_destroy(fsl_handle* h) {
  if (!h) return FSL_ERR_ARG;
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  if (h->aux.side) {
    cudaStreamSynchronize(h->aux.side);
    cudaEventDestroy(h->aux.fork);
    cudaEventDestroy(h->aux.join);
    cudaStreamDestroy(h->aux.side);
  }
  delete h;
  return FSL_OK;
}

// ---------------------------------------------------------------- adjoint
struct fsl_adjoint {
  fsl_handle* h = nullptr;
  int nsteps = 0, every = 0, nseg = 0;
  long long step0 = 0;  // step counter of the handle when the forward pass started
  size_t fbytes = 0, cells = 0;
  char* ckpt = nullptr;    // nseg + 1 workspace copies
  char* tF = nullptr;      // every + 1 levels of stored PDFs
  uint8_t* tFl = nullptr;  // every + 1 levels of flags
  double* tM = nullptr;    // every + 1 levels of mass
  double* tP = nullptr;    // every + 1 levels of fill level
  char* fld = nullptr;     // adjoint fields
  double* acc = nullptr;   // 8 accumulators
  double* dinit = nullptr; // 2 x dense cells: d J / d rho0, d J / d phi0
  std::vector<double> column;
  bool forward_done = false;
};

extern "C++" {
namespace {

bool adjoint_supported(const fsl_handle* h) {
  const fsl_config& c = h->cfg;
  return (c.precision == FSL_FP64 || c.precision == FSL_FP32) && c.collision == FSL_SRT &&
         c.refill == FSL_REFILL_EQ && c.sigma == 0.0 && c.les_cs == 0.0 && h->g.free_slip == 0 &&
         h->g.has_obst == 0 && h->g.bubbles == 0;
}

size_t adjoint_layout(const fsl_handle* h, int nsteps, int every, size_t* off) {
  const int nseg = (nsteps + every - 1) / every;
  const size_t sb = storage_bytes(h->cfg.precision);
  const size_t rb = h->cfg.precision == FSL_FP64 ? 8 : 4;
  const size_t cells = (size_t)h->g.cells;
  const size_t fbytes = (size_t)h->cfg.lattice * (size_t)h->g.plane * sb;
  const size_t dense = (size_t)h->g.nx * h->g.ny * h->g.nz;
  size_t sz[8];
  sz[0] = (size_t)(nseg + 1) * align256(h->bytes);
  sz[1] = (size_t)(every + 1) * align256(fbytes);
  sz[2] = (size_t)(every + 1) * align256(cells);
  sz[3] = (size_t)(every + 1) * align256(cells * 8);
  sz[4] = (size_t)(every + 1) * align256(cells * 8);
  // fields: 4 q-plane arrays (lF, lF0, lfin, spare) + 10 cell arrays + 4 + 3 per cell
  sz[5] = align256(rb * (4 * (size_t)h->cfg.lattice * h->g.plane + 17 * cells));
  sz[6] = 256;
  sz[7] = align256(2 * dense * 8);
  size_t total = 0;
  for (int k = 0; k < 8; ++k) {
    if (off) off[k] = total;
    total += align256(sz[k]);
  }
  return total;
}

template <class R>
AdjFields<R> adjoint_fields(fsl_adjoint* a) {
  const fsl_handle* h = a->h;
  const size_t qp = (size_t)h->cfg.lattice * h->g.plane, n = (size_t)h->g.cells;
  R* b = reinterpret_cast<R*>(a->fld);
  AdjFields<R> f;
  f.lF = b;
  f.lF0 = b + qp;
  f.lfin = b + 2 * qp;
  R* cb = b + 4 * qp;
  f.lM = cb;
  f.lM0 = cb + n;
  f.lP = cb + 2 * n;
  f.lP0 = cb + 3 * n;
  f.lm1 = cb + 4 * n;
  f.lrhoP = cb + 5 * n;
  f.lmnew = cb + 6 * n;
  f.lrho = cb + 7 * n;
  f.lbar = cb + 10 * n;  // 4 per cell
  f.lg = cb + 14 * n;    // 3 per cell
  f.acc = a->acc;
  return f;
}

// copy the handle's current state into tape level j
fsl_status adjoint_record(fsl_adjoint* a, int j, long long step) {
  fsl_handle* h = a->h;
  const int cur = (int)(step & 1);
  FSL_CK(cudaMemcpyAsync(a->tF + (size_t)j * align256(a->fbytes), h->d.pdf[cur], a->fbytes,
                         cudaMemcpyDeviceToDevice, h->stream));
  FSL_CK(cudaMemcpyAsync(a->tFl + (size_t)j * align256(a->cells), h->d.flags, a->cells,
                         cudaMemcpyDeviceToDevice, h->stream));
  FSL_CK(cudaMemcpyAsync(a->tM + (size_t)j * align256(a->cells * 8) / 8, h->d.mass, a->cells * 8,
                         cudaMemcpyDeviceToDevice, h->stream));
  FSL_CK(cudaMemcpyAsync(a->tP + (size_t)j * align256(a->cells * 8) / 8, h->d.phi, a->cells * 8,
                         cudaMemcpyDeviceToDevice, h->stream));
  return FSL_OK;
}

AdjLevel adjoint_level(const fsl_adjoint* a, int j) {
  AdjLevel L;
  L.F = a->tF + (size_t)j * align256(a->fbytes);
  L.flags = a->tFl + (size_t)j * align256(a->cells);
  L.M = a->tM + (size_t)j * align256(a->cells * 8) / 8;
  L.Phi = a->tP + (size_t)j * align256(a->cells * 8) / 8;
  return L;
}

template <int Q, class ST>
fsl_status adjoint_step(fsl_adjoint* a, const AdjLevel& L0, const AdjLevel& L1) {
  using R = typename ST::R;
  fsl_handle* h = a->h;
  AdjFields<R> f = adjoint_fields<R>(a);
  const int blocks = (int)((a->cells + 255) / 256);
  k_adj_phi<Q, ST><<<blocks, 256, 0, h->stream>>>(h->g, h->p, L0, L1, f);
  k_adj_mass<Q, ST><<<blocks, 256, 0, h->stream>>>(h->g, h->p, L0, L1, f);
  k_adj_refill<Q, ST><<<blocks, 256, 0, h->stream>>>(h->g, h->p, L0, L1, f);
  k_adj_collide<Q, ST><<<blocks, 256, 0, h->stream>>>(h->g, h->p, L0, L1, f);
  k_adj_state<Q, ST><<<blocks, 256, 0, h->stream>>>(h->g, h->p, L0, f);
  FSL_CK(cudaGetLastError());
  // the level-t adjoint becomes the input of the next (earlier) step
  const size_t rb = sizeof(R);
  const size_t qp = (size_t)h->cfg.lattice * h->g.plane;
  FSL_CK(cudaMemcpyAsync(f.lF, f.lF0, qp * rb, cudaMemcpyDeviceToDevice, h->stream));
  FSL_CK(cudaMemcpyAsync(f.lM, f.lM0, a->cells * rb, cudaMemcpyDeviceToDevice, h->stream));
  FSL_CK(cudaMemcpyAsync(f.lP, f.lP0, a->cells * rb, cudaMemcpyDeviceToDevice, h->stream));
  return FSL_OK;
}

template <int Q, class ST>
fsl_status adjoint_init(fsl_adjoint* a, const AdjLevel& L0) {
  using R = typename ST::R;
  fsl_handle* h = a->h;
  AdjFields<R> f = adjoint_fields<R>(a);
  const size_t dense = (size_t)h->g.nx * h->g.ny * h->g.nz;
  k_adj_init<Q, ST><<<(unsigned)((a->cells + 255) / 256), 256, 0, h->stream>>>(
      h->g, h->p, L0, f, h->h_ref, a->dinit, a->dinit + dense);
  FSL_CK(cudaGetLastError());
  return FSL_OK;
}

fsl_status adjoint_dispatch_step(fsl_adjoint* a, const AdjLevel& L0, const AdjLevel& L1) {
  const int q = a->h->cfg.lattice;
  if (a->h->cfg.precision == FSL_FP64)
    return q == 19 ? adjoint_step<19, SF64>(a, L0, L1) : adjoint_step<27, SF64>(a, L0, L1);
  return q == 19 ? adjoint_step<19, SF32>(a, L0, L1) : adjoint_step<27, SF32>(a, L0, L1);
}

fsl_status adjoint_dispatch_init(fsl_adjoint* a, const AdjLevel& L0) {
  const int q = a->h->cfg.lattice;
  if (a->h->cfg.precision == FSL_FP64)
    return q == 19 ? adjoint_init<19, SF64>(a, L0) : adjoint_init<27, SF64>(a, L0);
  return q == 19 ? adjoint_init<19, SF32>(a, L0) : adjoint_init<27, SF32>(a, L0);
}

}  // namespace
}  // extern "C++"

fsl_status fsl_adjoint_workspace_bytes(const fsl_handle* h, int nsteps, int every, size_t* bytes) {
  if (!h || !bytes || nsteps < 1 || every < 1 || nsteps > kTraceCapacity) return FSL_ERR_ARG;
  if (!adjoint_supported(h)) return FSL_ERR_ARG;
  *bytes = adjoint_layout(h, nsteps, every, nullptr);
  return FSL_OK;
}

fsl_status fsl_adjoint_create(fsl_handle* h, int nsteps, int every, void* d_workspace,
                              size_t bytes, fsl_adjoint** out) {
  if (!h || !out || nsteps < 1 || every < 1 || nsteps > kTraceCapacity) return FSL_ERR_ARG;
  if (!adjoint_supported(h) || !h->ready) return FSL_ERR_ARG;
  if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u)) return FSL_ERR_WORKSPACE;
  size_t off[8];
  if (bytes < adjoint_layout(h, nsteps, every, off)) return FSL_ERR_WORKSPACE;
  fsl_adjoint* a = new fsl_adjoint;
  a->h = h;
  a->nsteps = nsteps;
  a->every = every;
  a->nseg = (nsteps + every - 1) / every;
  a->cells = (size_t)h->g.cells;
  a->fbytes = (size_t)h->cfg.lattice * (size_t)h->g.plane * storage_bytes(h->cfg.precision);
  char* b = static_cast<char*>(d_workspace);
  a->ckpt = b + off[0];
  a->tF = b + off[1];
  a->tFl = reinterpret_cast<uint8_t*>(b + off[2]);
  a->tM = reinterpret_cast<double*>(b + off[3]);
  a->tP = reinterpret_cast<double*>(b + off[4]);
  a->fld = b + off[5];
  a->acc = reinterpret_cast<double*>(b + off[6]);
  a->dinit = reinterpret_cast<double*>(b + off[7]);
  *out = a;
  return FSL_OK;
}

fsl_status fsl_adjoint_forward(fsl_adjoint* a, double* column) {
  if (!a || !column) return FSL_ERR_ARG;
  fsl_handle* h = a->h;
  Ctrl c;
  fsl_status st = read_ctrl(h, &c);
  if (st != FSL_OK) return st;
  a->step0 = c.step;
  const int saved_every = h->trace_every;
  st = fsl_set_trace(h, 1);
  if (st != FSL_OK) return st;
  const size_t wb = align256(h->bytes);
  for (int k = 0; k < a->nseg; ++k) {
    FSL_CK(cudaMemcpyAsync(a->ckpt + (size_t)k * wb, h->base, h->bytes, cudaMemcpyDeviceToDevice,
                           h->stream));
    const int len = std::min(a->every, a->nsteps - k * a->every);
    st = fsl_step(h, len);
    if (st != FSL_OK) return st;
  }
  FSL_CK(cudaMemcpyAsync(a->ckpt + (size_t)a->nseg * wb, h->base, h->bytes,
                         cudaMemcpyDeviceToDevice, h->stream));
  std::vector<double> tr((size_t)a->nsteps * 3);
  st = fsl_observe(h, FSL_OBS_TRACE, tr.data(), tr.size() * sizeof(double));
  if (st != FSL_OK) return st;
  a->column.resize(a->nsteps);
  for (int t = 0; t < a->nsteps; ++t) a->column[t] = column[t] = tr[3 * (size_t)t];
  // the final state keeps the trace setting the caller had
  h->trace_every = saved_every;
  k_set_trace<<<1, 32, 0, h->stream>>>(h->d.ctrl, saved_every);
  FSL_CK(cudaGetLastError());
  FSL_CK(cudaMemcpyAsync(a->ckpt + (size_t)a->nseg * wb, h->base, h->bytes,
                         cudaMemcpyDeviceToDevice, h->stream));
  FSL_CK(cudaStreamSynchronize(h->stream));
  a->forward_done = true;
  return FSL_OK;
}

fsl_status fsl_adjoint_backward(fsl_adjoint* a, const double* dj_dcolumn, double* out) {
  if (!a || !dj_dcolumn || !out) return FSL_ERR_ARG;
  if (!a->forward_done) return FSL_ERR_STATE;
  fsl_handle* h = a->h;
  const size_t wb = align256(h->bytes);
  const size_t rb = h->cfg.precision == FSL_FP64 ? 8 : 4;
  const size_t qp = (size_t)h->cfg.lattice * h->g.plane;
  const size_t dense = (size_t)h->g.nx * h->g.ny * h->g.nz;
  FSL_CK(cudaMemsetAsync(a->fld, 0, rb * (4 * qp + 17 * a->cells), h->stream));
  FSL_CK(cudaMemsetAsync(a->acc, 0, 8 * sizeof(double), h->stream));
  double* lP_dbl = rb == 8 ? reinterpret_cast<double*>(a->fld) + 4 * qp + 2 * a->cells : nullptr;
  float* lP_flt = rb == 4 ? reinterpret_cast<float*>(a->fld) + 4 * qp + 2 * a->cells : nullptr;
  for (int k = a->nseg - 1; k >= 0; --k) {
    const int t0 = k * a->every;
    const int len = std::min(a->every, a->nsteps - t0);
    // replay the segment from its checkpoint, recording every level
    FSL_CK(cudaMemcpyAsync(h->base, a->ckpt + (size_t)k * wb, h->bytes, cudaMemcpyDeviceToDevice,
                           h->stream));
    fsl_status st = adjoint_record(a, 0, a->step0 + t0);
    if (st != FSL_OK) return st;
    for (int j = 1; j <= len; ++j) {
      st = fsl_step(h, 1);
      if (st != FSL_OK) return st;
      st = adjoint_record(a, j, a->step0 + t0 + j);
      if (st != FSL_OK) return st;
    }
    for (int j = len; j >= 1; --j) {
      k_adj_observe<<<(h->g.ny * h->g.nz + 255) / 256, 256, 0, h->stream>>>(
          h->g, dj_dcolumn[t0 + j - 1], lP_dbl, lP_flt);
      FSL_CK(cudaGetLastError());
      st = adjoint_dispatch_step(a, adjoint_level(a, j - 1), adjoint_level(a, j));
      if (st != FSL_OK) return st;
    }
  }
  // level 0 of the first segment is the initial state
  fsl_status st = adjoint_dispatch_init(a, adjoint_level(a, 0));
  if (st != FSL_OK) return st;
  double acc[4];
  FSL_CK(cudaMemcpyAsync(acc, a->acc, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
  FSL_CK(cudaMemcpyAsync(out + 4, a->dinit, 2 * dense * sizeof(double), cudaMemcpyDeviceToHost,
                         h->stream));
  // leave the handle at the end of the forward pass
  FSL_CK(cudaMemcpyAsync(h->base, a->ckpt + (size_t)a->nseg * wb, h->bytes,
                         cudaMemcpyDeviceToDevice, h->stream));
  FSL_CK(cudaStreamSynchronize(h->stream));
  // omega = 1 / (3 nu + 1/2): d omega / d nu = -3 omega^2
  out[0] = acc[0] * (-3.0 * h->p.omega * h->p.omega);
  out[1] = acc[1];
  out[2] = acc[2];
  out[3] = acc[3];
  return FSL_OK;
}

fsl_status fsl_adjoint_destroy(fsl_adjoint* a) {
  if (!a) return FSL_ERR_ARG;
  delete a;
  return FSL_OK;
}

// ------------------------------------------------------------------ batch
struct fsl_batch {
  std::vector<fsl_handle*> hs;
  bool batched = false;           // one launch per kernel for all members
  cudaStream_t stream = nullptr;  // graph launches
  cudaStream_t cap = nullptr;     // private stream, used only for captures
  std::vector<cudaEvent_t> ev;    // per member: its stream's queued work
  cudaEvent_t done = nullptr;
  int chunk = 8;
  std::vector<unsigned> gens;     // member generations the graphs were captured at
  std::map<int, cudaGraphExec_t> graphs;
};

namespace {

void batch_drop_graphs(fsl_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

// Whether the batch can run as one launch per kernel and step for all its
// members: 16/32-bit storages and no bubble model.
bool batchable(const fsl_batch* b) {
  for (const fsl_handle* h : b->hs)
    if (storage_bytes(h->cfg.precision) == 8 || h->g.bubbles) return false;
  return true;
}

// Each member's record (device pointers, geometry, parameters) into its own
// workspace, where the batched kernels read it.
fsl_status write_member_records(fsl_batch* b) {
  for (fsl_handle* h : b->hs) {
    const Member m = {h->d, h->g, h->p};
    FSL_CK(cudaMemcpyAsync(h->base + h->off[R_SELF], &m, sizeof(Member), cudaMemcpyHostToDevice,
                           b->stream));
  }
  FSL_CK(cudaStreamSynchronize(b->stream));
  return FSL_OK;
}

// One graph of `steps` steps of the batch, one launch per kernel for the
// members of each launch table (lattice and storage), at most kBatchMax
// members per launch.
fsl_status batch_capture_joint(fsl_batch* b, int steps, cudaGraphExec_t* out) {
  fsl_status st = write_member_records(b);
  if (st != FSL_OK) return st;
  struct Group {
    const Launch* L;
    MemberTable t;
    int n;
    BatchGrid bg;
  };
  std::vector<Group> groups;
  for (fsl_handle* h : b->hs) {
    Group* gp = nullptr;
    for (Group& q : groups)
      if (q.L == h->L && q.n < kBatchMax) gp = &q;
    if (!gp) {
      groups.push_back(Group{h->L, {}, 0, {1}});
      gp = &groups.back();
    }
    gp->t.m[gp->n++] = reinterpret_cast<const Member*>(h->base + h->off[R_SELF]);
    const long long ntiles = (long long)((h->g.nx + 63) / 64) * h->g.ny * h->g.nz;
    const int tb = (int)((ntiles + 255) / 256);
    if (tb > gp->bg.tiles) gp->bg.tiles = tb;
  }
  cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture (batch)");
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < steps && le == cudaSuccess; ++k)
    for (const Group& q : groups)
      if (le == cudaSuccess) le = q.L->batch_step(q.t, q.n, q.bg, b->cap);
  cudaGraph_t g;
  e = cudaStreamEndCapture(b->cap, &g);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (e == cudaSuccess) cudaGraphDestroy(g);
    return cuda_fail(le != cudaSuccess ? le : e, "batch capture");
  }
  cudaError_t ie = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate (batch)");
  return FSL_OK;
}

// one graph of `steps` steps of every member: a child graph per member, no
// edges between them
fsl_status batch_capture(fsl_batch* b, int steps, cudaGraphExec_t* out) {
  if (b->batched) return batch_capture_joint(b, steps, out);
  cudaGraph_t parent;
  FSL_CK(cudaGraphCreate(&parent, 0));
  for (fsl_handle* h : b->hs) {
    cudaGraph_t g;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaGraphDestroy(parent);
      return cuda_fail(e, "cudaStreamBeginCapture (batch)");
    }
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < steps && le == cudaSuccess; ++k) le = h->L->step(h->d, h->g, h->p, b->cap, h->aux);
    e = cudaStreamEndCapture(b->cap, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (e == cudaSuccess) cudaGraphDestroy(g);
      cudaGraphDestroy(parent);
      return cuda_fail(le != cudaSuccess ? le : e, "batch member capture");
    }
    cudaGraphNode_t node;
    e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, g);
    cudaGraphDestroy(g);  // the child node holds its own copy
    if (e != cudaSuccess) {
      cudaGraphDestroy(parent);
      return cuda_fail(e, "cudaGraphAddChildGraphNode");
    }
  }
  cudaError_t ie = cudaGraphInstantiate(out, parent, 0);
  cudaGraphDestroy(parent);
  if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate (batch)");
  return FSL_OK;
}

}  // namespace

fsl_status fsl_batch_create(fsl_handle* const* handles, int n, void* cuda_stream, int chunk,
                            fsl_batch** out) {
  if (!handles || n < 1 || !out || !cuda_stream || chunk < 1 || chunk > (int)kGraphChunk)
    return FSL_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!handles[i] || !handles[i]->ready) return FSL_ERR_ARG;
  fsl_batch* b = new fsl_batch;
  b->hs.assign(handles, handles + n);
  b->stream = (cudaStream_t)cuda_stream;
  b->chunk = chunk;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  b->ev.assign(n, nullptr);
  for (int i = 0; i < n && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    fsl_batch_destroy(b);
    return cuda_fail(e, "batch streams/events");
  }
  *out = b;
  return FSL_OK;
}

fsl_status fsl_batch_step(fsl_batch* b, int nsteps) {
  if (!b || nsteps < 0) return FSL_ERR_ARG;
  if (nsteps == 0) return FSL_OK;
  const size_t n = b->hs.size();
  bool stale = b->gens.size() != n;
  for (size_t i = 0; i < n && !stale; ++i) stale = b->gens[i] != b->hs[i]->gen;
  if (stale) {
    for (fsl_handle* h : b->hs)
      if (!h->ready) return FSL_ERR_STATE;
    b->batched = batchable(b);
    batch_drop_graphs(b);
    b->gens.resize(n);
    for (size_t i = 0; i < n; ++i) b->gens[i] = b->hs[i]->gen;
  }
  // after everything already queued on the members' streams
  for (size_t i = 0; i < n; ++i) {
    FSL_CK(cudaEventRecord(b->ev[i], b->hs[i]->stream));
    FSL_CK(cudaStreamWaitEvent(b->stream, b->ev[i], 0));
  }
  int left = nsteps;
  while (left > 0) {
    const int c = left >= b->chunk ? b->chunk : left;
    auto it = b->graphs.find(c);
    if (it == b->graphs.end()) {
      cudaGraphExec_t exec;
      fsl_status st = batch_capture(b, c, &exec);
      if (st != FSL_OK) return st;
      it = b->graphs.emplace(c, exec).first;
    }
    FSL_CK(cudaGraphLaunch(it->second, b->stream));
    left -= c;
  }
  // members' later work after the batched steps
  FSL_CK(cudaEventRecord(b->done, b->stream));
  for (fsl_handle* h : b->hs) FSL_CK(cudaStreamWaitEvent(h->stream, b->done, 0));
  return FSL_OK;
}

fsl_status fsl_batch_destroy(fsl_batch* b) {
  if (!b) return FSL_ERR_ARG;
  batch_drop_graphs(b);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->done) cudaEventDestroy(b->done);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return FSL_OK;
}

fsl_status fsl_lattice_table(int lattice, int* c3q, double* w) {
  if (lattice != FSL_D3Q19 && lattice != FSL_D3Q27) return FSL_ERR_ARG;
  for (int i = 0; i < lattice; ++i) {
    for (int a = 0; a < 3; ++a)
      if (c3q) c3q[3 * i + a] = dir_c(i, a);
    if (w) w[i] = lattice == 19 ? wgt<19>(i) : wgt<27>(i);
  }
  return FSL_OK;
}

int fsl_launches_per_step(const fsl_handle* h) { return h ? h->L->launches_per_step(h->g) : 0; }

fsl_status fsl_set_variant(fsl_handle* h, int variant) {
  if (!h || variant < FSL_VARIANT_DEFAULT || variant > FSL_VARIANT_TMA_R96) return FSL_ERR_ARG;
  if ((variant == FSL_VARIANT_QUAD_64 || variant == FSL_VARIANT_PAIR_PIPE ||
       variant == FSL_VARIANT_CPA_R96 || variant == FSL_VARIANT_TMA_R96) &&
      storage_bytes(h->cfg.precision) != 2)
    return FSL_ERR_ARG;
  h->g.variant = variant;
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  ++h->gen;
  return FSL_OK;
}

int fsl_get_variant(const fsl_handle* h) { return h ? h->g.variant : -1; }

fsl_status fsl_kernel_stats(fsl_handle* h, int kernel, int reps, double* out4) {
  if (!h || !out4 || reps < 1 ||
      (kernel != FSL_KERNEL_STREAM_COLLIDE && kernel != FSL_KERNEL_BULK_PASS))
    return FSL_ERR_ARG;
  if (!h->ready) return FSL_ERR_STATE;
  const bool with_pre = kernel == FSL_KERNEL_BULK_PASS;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(h->d.red + 2 * kReduceBlocks + 8);
  FSL_CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), h->stream));
  k_count_types<<<kReduceBlocks, 256, 0, h->stream>>>(h->d, h->g, cnt);
  FSL_CK(cudaGetLastError());
  unsigned long long nc[2];
  FSL_CK(cudaMemcpyAsync(nc, cnt, sizeof(nc), cudaMemcpyDeviceToHost, h->stream));
  cudaEvent_t e0, e1;
  FSL_CK(cudaEventCreate(&e0));
  FSL_CK(cudaEventCreate(&e1));
  double total_ms = 0.0;
  cudaError_t err = cudaSuccess;
  // work lists of the current state (interface cells, liquid tiles), untimed
  // unless the pre-pass is part of what is measured
  if (!with_pre) {
    err = cudaMemsetAsync(&h->d.ctrl->n_tiles, 0, sizeof(unsigned), h->stream);
    if (err == cudaSuccess) err = h->L->pre_bulk(h->d, h->g, h->p, h->stream);
  }
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    // the tile list is rebuilt by the pre-pass
    if (with_pre)
      err = cudaMemsetAsync(&h->d.ctrl->n_tiles, 0, sizeof(unsigned), h->stream);
    if (err == cudaSuccess) err = cudaEventRecord(e0, h->stream);
    if (err == cudaSuccess && with_pre) err = h->L->pre_bulk(h->d, h->g, h->p, h->stream);
    if (err == cudaSuccess) err = h->L->stream_collide(h->d, h->g, h->p, h->stream);
    if (err == cudaSuccess) err = cudaEventRecord(e1, h->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    total_ms += ms;
  }
  if (err == cudaSuccess) err = cudaMemsetAsync(&h->d.ctrl->n_tiles, 0, sizeof(unsigned), h->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_fail(err, "fsl_kernel_stats");
  const double sb = (double)storage_bytes(h->cfg.precision);
  const double cells = (double)h->g.nx * h->g.ny * h->g.nz;
  out4[0] = total_ms / reps;
  // liquid cells read and write q PDFs; every cell's flag byte is read
  out4[1] = (double)nc[0] * 2.0 * h->cfg.lattice * sb + cells * 1.0;
  out4[2] = (double)nc[0];
  out4[3] = (double)nc[1];
  return FSL_OK;
}

fsl_status fsl_selftest_wait(fsl_handle* h) {
  if (!h) return FSL_ERR_ARG;
  if (!h->ready) return FSL_ERR_STATE;
  k_barrier_selftest<<<1, 256, 0, h->stream>>>(h->d);
  FSL_CK(cudaGetLastError());
  FSL_CK(cudaStreamSynchronize(h->stream));
  return FSL_OK;
}

const char* fsl_status_string(fsl_status s) {
  switch (s) {
    case FSL_OK: return "ok";
    case FSL_ERR_ARG: return "invalid argument";
    case FSL_ERR_CUDA: return "CUDA runtime error";
    case FSL_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case FSL_ERR_UNSTABLE: return "unstable: |u| >= c_s or NaN";
    case FSL_ERR_TIMEOUT: return "bounded device wait gave up";
    case FSL_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* fsl_last_error(void) { return g_err.c_str(); }

}  // extern "C"
