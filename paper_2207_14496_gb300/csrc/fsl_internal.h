// Internal declarations shared by the host ABI (fsl_api.cu) and the kernel
// translation units (one per precision family).  Not installed; the public
// interface is include/fsl.h.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace fsl {

// Cell-type codes (low two bits of the flag byte).
enum : uint8_t { T_GAS = 0, T_IF = 1, T_LIQ = 2, T_OBST = 3 };
// Flag bits above the type.
enum : uint8_t {
  F_TYPE = 3,
  F_NF = 4,        // interface cell without liquid neighbour (Thuerey class)
  F_NE = 8,        // interface cell without gas neighbour
  F_TO_LIQ = 16,   // fill level above 1 + eps this step (converts to liquid)
  F_TO_GAS = 32,   // fill level below -eps this step (converts to gas)
  F_NEW = 64,      // gas cell that became interface this step (to be refilled)
  F_NEAR_OBST = 128  // some stencil neighbour is a wall or obstacle (static)
};

// Device control block (one per handle, in the workspace).
struct Ctrl {
  int step;            // steps completed
  int unstable_step;   // first step with |u| >= c_s or NaN, -1 if none
  unsigned n_if;       // interface cells of this step (list built by the previous step)
  unsigned n_fill;     // cells marked to fill
  unsigned n_empty;    // cells marked to empty
  unsigned n_new;      // gas -> interface cells
  unsigned n_l2i;      // liquid -> interface cells
  unsigned n_recv;     // excess-mass receivers
  unsigned last[4];    // previous step: filled, emptied (after conflicts), new, interface
  int trace_every;     // 0: no trace
  int trace_count;     // records written (ring index = count % capacity)
  unsigned timeout;    // error bits: 1 CAS retry cap, 2 refill without source, 4 copy wait gave up,
                       // 8 bubble union retry cap, 16 grid barrier wait gave up,
                       // 32 a self-checked barrier passed that could not
  unsigned n_emptied;  // to-gas cells actually converted this step
  unsigned end_blocks; // end-of-step blocks finished
  unsigned n_tiles;    // tiles holding liquid cells, listed this step (16/32-bit path)
  unsigned n_if_next;  // interface cells of the next step (appended by k_classify)
  unsigned tile_next;  // next tile handed out by the dynamically scheduled bulk kernel
  unsigned tile_done;  // blocks of that kernel finished (the last one resets both)
  unsigned bar;        // block arrivals at the grid barriers of the conversion kernel
                       // (reset by the end-of-step kernel)
};

constexpr int kTraceCapacity = 1 << 16;
constexpr int kListBlocks = 2 * 152;  // grid of the list-driven kernels
// grid of the two kernels that run one thread per interface cell (tens of
// thousands per step): enough threads for one cell each, so that their
// latency-bound neighbourhood reads overlap across many warps
constexpr int kCellListBlocks = 8 * 152;
constexpr int kReduceBlocks = 4 * 152;

struct Geom {
  int nx, ny, nz;
  int sx;              // padded row stride (elements/cells)
  long long cells;     // padded cell count nz*ny*sx
  long long plane;     // PDF plane stride in elements (>= cells, 128-element multiple)
  int periodic[3];
  int has_obst;        // the initial state had interior obstacle cells
  int free_slip;       // bit a: the walls of non-periodic axis a are free-slip (specular)
  int variant;         // bulk kernel of the 16/32-bit path (FSL_VARIANT_*; 0 = default)
  int bubbles;         // bubble model on (FSL_OPT_BUBBLES)
  int bub_gas_only;    // bubbles from gas cells alone (FSL_OPT_BUBBLE_GAS_ONLY)
};

struct Phys {
  int q;
  int trt;
  int refill;
  unsigned options;
  double tau, omega, lam_e, lam_o;  // SRT omega; TRT even/odd rates
  double pre_e, pre_o;              // 1 - lam/2 Guo prefactors (pre_e also SRT)
  double g[3];
  int gaxis;                        // last axis with nonzero g, -1 if none
  double sigma, p_v, eps;
  double geq_coef;                  // 1/(2 c_s^2 omega) = 1.5 tau, or 1.5/nu
  double thr_hi, thr_lo;            // 1 + eps, 0 - eps
  double magic;                     // TRT magic parameter
  double les_cs;                    // Smagorinsky constant, 0 = no turbulence model
  // the same parameters rounded once to FP32 on the host, so that the 16/32-bit
  // kernels execute no FP64 conversion (GB300 has two FP64 lanes per SM)
  struct {
    float tau, omega, lam_e, lam_o, pre_e, pre_o, g[3], sigma, p_v, eps, geq_coef, thr_hi,
        thr_lo, magic, les_cs;
    float les_k;  // 2 sqrt(2) C_S^2 * 9, the Smagorinsky closure's constant
  } f;
};

struct Dev {
  void* pdf[2];       // ping-pong PDF buffers (storage type of the precision)
  uint8_t* flags;
  uint8_t* claim;     // receiver claim bytes (zero between steps)
  double* phi;        // fill level
  float* phif;        // FP32 copy of phi, written with it (16/32-bit path; null in FP64)
  double* phinew;     // fill level computed by stream-collide (interface cells)
  double* mass;       // cell mass (interface cells)
  double* rho;        // density recorded this step (interface cells)
  double* kappa;      // curvature K (interface cells)
  double* mex;        // excess mass of converted cells / share per receiver
  double* lost;       // per-cell lost excess mass (no receiver)
  int* l_if;   // interface list of even steps
  int* l_if2;  // interface list of odd steps
  int* l_fill;
  int* l_empty;
  int* l_new;
  int* l_l2i;
  int* l_recv;
  int* l_tiles;       // tiles (256 cells along x of one row) holding liquid cells
  Ctrl* ctrl;
  double* trace;      // kTraceCapacity * 3 doubles
  double* red;        // reduction scratch, kReduceBlocks * 2 doubles
  int* redi;          // integer reduction scratch
  // bubble model (empty when off): label per cell and its next value, K = p V
  // and volume pressure per bubble (at its root cell), the next K and the
  // volumes as fixed-point sums
  int* blab;
  int* bnew;
  double* bK;
  long long* bKnew;
  long long* bV;
  long long* bVseen;
  double* bp;
  uint8_t* bhas;
};

// One member of a batch of independent domains, as the batched kernels read
// it: a copy of the handle's device pointers, geometry and parameters kept in
// the handle's own workspace (region written by the host before a capture).
struct Member {
  Dev d;
  Geom g;
  Phys p;
};
// Members of one batched launch, one per blockIdx.y (a kernel parameter).
constexpr int kBatchMax = 256;
struct MemberTable {
  const Member* m[kBatchMax];
};
// Grid extent along x of each batched kernel, per member (the kernels' own
// loops cover whatever cells, list entries or segments the member holds).
struct BatchGrid {
  int tiles;  // blocks of the segment-list pre-pass (largest member)
};

// Per-precision-family launch table, implemented in fsl_prec_*.cu.
// Side stream and events of a handle: the interface pass of a step runs on
// `side`, forked from and joined back to the step's stream, concurrently with
// the bulk pass (the two write disjoint cells).  side == nullptr: one stream.
struct Aux {
  cudaStream_t side;
  cudaEvent_t fork, join;
};

struct Launch {
  // one full time step from pdf[step & 1] to pdf[(step + 1) & 1]
  cudaError_t (*step)(const Dev&, const Geom&, const Phys&, cudaStream_t, const Aux&);
  // initial state into pdf[cur] (cur = 0); staged: fill level in d.phinew and
  // obstacle bytes in d.claim (both unpadded), u0 (3N doubles, unpadded) in
  // stage_u or null
  cudaError_t (*init)(const Dev&, const Geom&, const Phys&, int cur, const double* stage_u,
                      int have_obstacle, double h_ref, cudaStream_t);
  // total mass (fluid zeroth moments + interface m + lost) into out (device double)
  cudaError_t (*total_mass)(const Dev&, const Geom&, const Phys&, int cur, double* out,
                            cudaStream_t);
  // max |u| over fluid cells into out (device double)
  cudaError_t (*max_velocity)(const Dev&, const Geom&, const Phys&, int cur, double* out,
                              cudaStream_t);
  // decode plane i of pdf[cur] into dst (device, nx*ny*nz doubles, unpadded)
  cudaError_t (*export_pdf)(const Dev&, const Geom&, const Phys&, int cur, int i, double* dst,
                            cudaStream_t);
  // work lists the bulk kernel needs (interface cells, liquid tiles), or null
  cudaError_t (*pre_bulk)(const Dev&, const Geom&, const Phys&, cudaStream_t);
  // the bulk stream-collide kernel alone (timing)
  cudaError_t (*stream_collide)(const Dev&, const Geom&, const Phys&, cudaStream_t);
  // kernel launches of one step
  int (*launches_per_step)(const Geom&);
  // one time step of n members (one launch per kernel for all of them)
  cudaError_t (*batch_step)(const MemberTable& t, int n, const BatchGrid& bg, cudaStream_t);
};

// Launch tables, one translation unit per (storage, lattice).
const Launch* launch_fp64_q19();
const Launch* launch_fp64_q27();
const Launch* launch_fp32_q19();
const Launch* launch_fp32_q27();
const Launch* launch_fp16_q19();
const Launch* launch_fp16_q27();
const Launch* launch_bf16_q19();
const Launch* launch_bf16_q27();

size_t storage_bytes(int precision);

// text returned by fsl_last_error() on this thread
void set_error_text(const char* msg);

}  // namespace fsl
