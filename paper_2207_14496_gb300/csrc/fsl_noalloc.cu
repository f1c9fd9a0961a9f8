// Allocation-free total mass of a state held in caller-owned device arrays.
//
// Some callers cannot allocate device memory at the point where they need this
// observable: code inside a host callback or inside another allocator's
// bookkeeping, a process whose device-memory budget is fixed up front, or a
// loop that must not let a cudaMalloc synchronise the device.  This entry
// point therefore takes its reduction scratch (one partial sum per block)
// from a file-scope static device array instead of a workspace.  The array is
// modest (kMaxBlocks doubles, 16 KiB) and every GPU that loads the library
// keeps it until the process exits.
//
// The first call on each device looks up the array's device address (with
// that device current), caches it, and loads every kernel this entry point
// can launch, so that later calls load nothing; make that first call before
// any stream capture.  All calls share the array: each call overwrites the
// partials it uses (nothing has to start at zero), and calls whose kernels
// overlap on the GPU (different streams without ordering) race on it.
#include <cstdint>
#include <mutex>

#include "fsl.h"
#include "fsl_lattice.cuh"

namespace {

using namespace fsl;

constexpr int kThreads = 256;
constexpr long long kCellsPerBlock = 16384;  // fixed partition -> deterministic sum
constexpr int kMaxBlocks = 2048;             // scratch capacity
constexpr long long kMaxCells = kCellsPerBlock * kMaxBlocks;
constexpr int kMaxDevices = 64;

// Reduction scratch shared by every call on a device.  In host code this name
// is only a stand-in for the device symbol: its device address comes from
// cudaGetSymbolAddress (scratch_on_current_device) and is passed to the kernels.
static __device__ __align__(256) double g_mass_partials[kMaxBlocks];

std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};

cudaError_t load_kernels();

// Device address of the scratch on the current device, looked up once per
// device (with that device current), together with loading the kernels.
cudaError_t scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mass_partials);
    if (e != cudaSuccess) return e;
    e = load_kernels();
    if (e != cudaSuccess) return e;
    g_scratch[dev] = p;
  }
  *out = static_cast<double*>(g_scratch[dev]);
  return cudaSuccess;
}

// Per block: the cells [b * kCellsPerBlock, (b + 1) * kCellsPerBlock); liquid
// cells count the zeroth moment of their stored PDFs (direction order),
// interface cells their mass, plus the per-cell lost mass when given.
template <int Q, class ST>
__global__ void __launch_bounds__(kThreads)
    k_mass_dense_partial(const typename ST::T* pdf, const uint8_t* types, const double* mass,
                         const double* lost, long long n, double* part) {
  __shared__ double sh[kThreads];
  const long long c0 = blockIdx.x * kCellsPerBlock;
  const long long c1 = c0 + kCellsPerBlock < n ? c0 + kCellsPerBlock : n;
  double s = 0.0;
  for (long long c = c0 + threadIdx.x; c < c1; c += kThreads) {
    const int t = types[c] & F_TYPE;
    double v = lost ? lost[c] : 0.0;
    if (t == T_LIQ) {
      double r = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double f = ST::ldf(pdf + i * n + c, wgt<Q>(i));
        r = (i == 0) ? f : r + f;
      }
      v += r;
    } else if (t == T_IF) {
      v += mass[c];
    }
    s += v;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kThreads) k_mass_dense_final(const double* part, int nb,
                                                                double* out) {
  __shared__ double sh[kThreads];
  double s = 0.0;
  for (int k = threadIdx.x; k < nb; k += kThreads) s += part[k];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// Launch errors are read with cudaPeekAtLastError, which leaves an error of
// unrelated earlier work in place for its owner (it is reported here too).
template <int Q, class ST>
cudaError_t launch(const void* pdf, const uint8_t* types, const double* mass, const double* lost,
                   long long n, double* scratch, double* out, cudaStream_t s) {
  const int nb = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
  k_mass_dense_partial<Q, ST><<<nb, kThreads, 0, s>>>(
      static_cast<const typename ST::T*>(pdf), types, mass, lost, n, scratch);
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) return e;
  k_mass_dense_final<<<1, kThreads, 0, s>>>(scratch, nb, out);
  return cudaPeekAtLastError();
}

// Loads the module code of every kernel above on the current device (with
// lazy module loading a kernel is otherwise loaded at its first launch).
cudaError_t load_kernels() {
  const void* fns[] = {
      (const void*)k_mass_dense_partial<19, SF64>,  (const void*)k_mass_dense_partial<27, SF64>,
      (const void*)k_mass_dense_partial<19, SF32>,  (const void*)k_mass_dense_partial<27, SF32>,
      (const void*)k_mass_dense_partial<19, SF16>,  (const void*)k_mass_dense_partial<27, SF16>,
      (const void*)k_mass_dense_partial<19, SBF16>, (const void*)k_mass_dense_partial<27, SBF16>,
      (const void*)k_mass_dense_final};
  for (const void* f : fns) {
    cudaFuncAttributes a;
    const cudaError_t e = cudaFuncGetAttributes(&a, f);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" fsl_status fsl_total_mass_noalloc(const fsl_config* cfg, const void* d_pdf,
                                             const unsigned char* d_types, const double* d_mass,
                                             const double* d_lost, double* d_out,
                                             void* cuda_stream) {
  if (!cfg || !d_pdf || !d_types || !d_mass || !d_out) return FSL_ERR_ARG;
  if (cfg->lattice != FSL_D3Q19 && cfg->lattice != FSL_D3Q27) return FSL_ERR_ARG;
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return FSL_ERR_ARG;
  const long long n = (long long)cfg->nx * cfg->ny * cfg->nz;
  if (n > kMaxCells) {
    set_error_text("fsl_total_mass_noalloc: more cells than the static scratch holds "
                   "(limit 33554432 cells)");
    return FSL_ERR_ARG;
  }
  double* scratch = nullptr;
  const cudaError_t se = scratch_on_current_device(&scratch);
  if (se != cudaSuccess) {
    set_error_text(cudaGetErrorString(se));
    return FSL_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const bool q19 = cfg->lattice == FSL_D3Q19;
  cudaError_t e;
  switch (cfg->precision) {
    case FSL_FP64:
      e = q19 ? launch<19, SF64>(d_pdf, d_types, d_mass, d_lost, n, scratch, d_out, s)
              : launch<27, SF64>(d_pdf, d_types, d_mass, d_lost, n, scratch, d_out, s);
      break;
    case FSL_FP32:
      e = q19 ? launch<19, SF32>(d_pdf, d_types, d_mass, d_lost, n, scratch, d_out, s)
              : launch<27, SF32>(d_pdf, d_types, d_mass, d_lost, n, scratch, d_out, s);
      break;
    case FSL_MIXED_FP16:
      e = q19 ? launch<19, SF16>(d_pdf, d_types, d_mass, d_lost, n, scratch, d_out, s)
              : launch<27, SF16>(d_pdf, d_types, d_mass, d_lost, n, scratch, d_out, s);
      break;
    case FSL_MIXED_BF16:
      e = q19 ? launch<19, SBF16>(d_pdf, d_types, d_mass, d_lost, n, scratch, d_out, s)
              : launch<27, SBF16>(d_pdf, d_types, d_mass, d_lost, n, scratch, d_out, s);
      break;
    default:
      return FSL_ERR_ARG;
  }
  if (e != cudaSuccess) {
    set_error_text(cudaGetErrorString(e));
    return FSL_ERR_CUDA;
  }
  return FSL_OK;
}
