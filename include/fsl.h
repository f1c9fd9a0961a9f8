/*
 * fsl.h -- C ABI of libfsl, a GB300 (sm_103a) free-surface lattice Boltzmann
 * (FSLBM) time step with the five refilling schemes compared in Schwarzmeier &
 * Ruede, "Comparison of refilling schemes in the free-surface lattice
 * Boltzmann method" (arXiv 2207.14496).
 *
 * One handle advances one domain.  Every step runs entirely in the library's
 * CUDA kernels on the stream bound at creation:
 *   1. pull stream + collide (SRT Eq. nm-lbm-collision-operator, or TRT) with
 *      Guo forcing (Eq. nm-lbm-force-guo), halfway bounce-back at walls, the
 *      free-surface anti-bounce-back condition (Eq. nm-fslbm-boundary-condition)
 *      for PDFs arriving from gas, and the interface mass flux
 *      (Eq. nm-fslbm-mass-flux, Sec. 2.2, with Thuerey's treatment of
 *      unnecessary interface cells);
 *   2. cell conversion with the threshold epsilon_phi (Sec. 2.2) over
 *      warp-ballot-compacted candidate lists;
 *   3. refilling of gas->interface cells (Sec. 3.1: EQ, EQ+NEQ, GEQ, EXT, AVG);
 *   4. excess-mass redistribution (Eq. nm-fslbm-excess-mass);
 *   5. Parker-Youngs normals and curvature kappa = -div(n_hat) (Sec. 2.2) for
 *      the Laplace pressure (Eqs. nm-fslbm-pressure-gas, nm-fslbm-pressure-laplace);
 *   6. with FSL_OPT_BUBBLES, the volume pressure of every enclosed gas region
 *      (Eq. nm-fslbm-pressure-volume), carried through merges and splits.
 *
 * Conventions for every entry point
 *   - Status: 0 on success, a negative fsl_status on failure.  No entry point
 *     aborts or traps; device-side conditions (instability, a bubble sum
 *     term out of range, a bounded device loop that gave up) are latched in a
 *     device status word and reported by fsl_observe(FSL_OBS_STATUS).
 *   - Memory: the caller owns the device workspace (one allocation of
 *     fsl_workspace_bytes bytes, 256-byte aligned) and the CUDA stream.  The
 *     library never calls cudaMalloc/cudaFree; it mallocs only the small host
 *     handle and temporary host buffers inside fsl_observe.
 *   - Synchronisation: fsl_step is asynchronous on the bound stream.
 *     fsl_init_fill, fsl_observe, fsl_save and fsl_load synchronise the stream
 *     before returning, so host buffers may be reused immediately.
 *   - Threading: a handle is bound to one stream and is not thread-safe.
 *   - Layout of host arrays: cell (i, j, k) at index i + nx (j + ny k), x
 *     fastest; PDF arrays are q planes of nx*ny*nz values, direction order
 *     rest, 6 faces, 12 edges (, 8 corners) as listed in fsl_lattice_table.
 */
#ifndef FSL_H
#define FSL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fsl_handle fsl_handle;

typedef enum {
  FSL_OK = 0,
  FSL_ERR_ARG = -1,       /* invalid argument or configuration */
  FSL_ERR_CUDA = -2,      /* a CUDA runtime call failed (message: fsl_last_error) */
  FSL_ERR_WORKSPACE = -3, /* workspace missing, misaligned or too small */
  FSL_ERR_UNSTABLE = -4,  /* |u| >= c_s or a NaN appeared; steps are frozen */
  FSL_ERR_TIMEOUT = -5,   /* a bounded device wait gave up */
  FSL_ERR_STATE = -6      /* call out of order (e.g. step before init_fill) */
} fsl_status;

enum { FSL_D3Q19 = 19, FSL_D3Q27 = 27 };
enum { FSL_SRT = 0, FSL_TRT = 1 };
/* PDF storage / collision precision.  FP64: FP64 storage and arithmetic,
 * bit-reproducible against a plain FP64 evaluation in the documented
 * operation order.  FP32: FP32 storage and arithmetic.  MIXED_FP16 /
 * MIXED_BF16: PDFs stored as 16-bit offsets f_i - w_i (FP16 scaled by 2^15),
 * collision and mass flux in FP32; cell mass, excess mass and reductions stay
 * FP64 in every mode. */
enum { FSL_FP64 = 0, FSL_FP32 = 1, FSL_MIXED_FP16 = 2, FSL_MIXED_BF16 = 3 };
/* Refilling schemes of Sec. 3.1. */
enum { FSL_REFILL_EQ = 0, FSL_REFILL_EQ_NEQ = 1, FSL_REFILL_GEQ = 2, FSL_REFILL_EXT = 3,
       FSL_REFILL_AVG = 4 };
/* Reading switches (fsl_config.options). */
enum {
  FSL_OPT_SIMPLE_FLUX = 1u,      /* plain Eq. nm-fslbm-mass-flux, no Thuerey table */
  FSL_OPT_GEQ_LITERAL_NU = 2u,   /* GEQ prefactor 1/(2 c_s^2 nu) as printed (default 1/(2 c_s^2 omega)) */
  FSL_OPT_NEQ_LITERAL_MEAN = 4u, /* EQ+NEQ: f_i(y) - f_i^eq(rho_bar, u_bar) as printed */
  FSL_OPT_LAPLACE_LITERAL = 8u,  /* p_G = p_V - 2 sigma kappa (default p_G = p_V + sigma K) */
  FSL_OPT_BUBBLES = 16u,         /* bubble model (Sec. 2.2, Eq. nm-fslbm-pressure-volume):
                                    every face-connected region of gas and interface cells
                                    has its own volume pressure p_V(0) V(0)/V(t), p V
                                    carried through merges and splits; p_volume is the
                                    initial pressure */
  FSL_OPT_BUBBLE_GAS_ONLY = 32u  /* with FSL_OPT_BUBBLES: regions of gas cells alone, each
                                    interface cell attached to the smallest-labelled
                                    region among its gas stencil neighbours */
};

typedef struct {
  int lattice;      /* FSL_D3Q19 | FSL_D3Q27 */
  int collision;    /* FSL_SRT | FSL_TRT */
  double trt_magic; /* TRT magic parameter Lambda (3/16 typical) */
  int precision;    /* FSL_FP64 | FSL_FP32 | FSL_MIXED_FP16 | FSL_MIXED_BF16 */
  int refill;       /* FSL_REFILL_* */
  int nx, ny, nz;   /* cells; each >= 1 */
  int periodic[3];  /* per axis: 1 periodic, 0 no-slip (bounce-back) walls on both faces */
  double nu;        /* kinematic viscosity, lattice units; tau = 3 nu + 1/2 */
  double gravity[3];/* body acceleration g; force F = rho g (Guo) */
  double sigma;     /* surface tension (0: no Laplace pressure) */
  double p_volume;  /* volume (atmospheric) gas pressure, 1/3 for rho = 1 */
  double eps_phi;   /* conversion threshold epsilon_phi (1e-2 in the paper) */
  unsigned options; /* FSL_OPT_* */
  double les_cs;    /* Smagorinsky constant C_S (Sec. 2.1, 0.1 in the paper's dam breaks);
                       0 disables the turbulence model */
  int free_slip[3]; /* per non-periodic axis: 1 = free-slip (specular) walls, 0 = no-slip */
} fsl_config;

/* Workspace size for a configuration.  bytes: out.  FSL_ERR_ARG for an
 * invalid configuration. */
fsl_status fsl_workspace_bytes(const fsl_config* cfg, size_t* bytes);

/* Bind a configuration to a caller-owned device workspace and CUDA stream
 * (cudaStream_t passed as void*; NULL = legacy default stream).
 * d_workspace: device pointer, 256-byte aligned, >= fsl_workspace_bytes.
 * out: receives the host handle (release with fsl_destroy).  The handle
 * creates one high-priority side stream and two events of its own (no device
 * memory): each step runs its interface-cell pass there, forked from and
 * joined back to the bound stream, beside the bulk pass; fsl_destroy
 * releases them. */
fsl_status fsl_create(const fsl_config* cfg, void* d_workspace, size_t bytes, void* cuda_stream,
                      fsl_handle** out);

/* Initial state (Sec. 2.2 cell types): phi (host, N doubles) gives the fill
 * level; phi >= 1 liquid, phi <= 0 gas, else interface; a liquid cell touching
 * gas becomes interface (closed layer).  u0 (host, 3N doubles, xyz per cell)
 * or NULL for rest.  obstacle (host, N bytes, nonzero = solid) or NULL.
 * h_ref: height along the gravity axis where rho = 1; the initial density is
 * rho = 1 + 3 g_a (x_a + 1/2 - h_ref) (hydrostatic); NaN disables it.
 * PDFs start at f^eq(rho, u0), m = phi rho.  Synchronises the stream. */
fsl_status fsl_init_fill(fsl_handle* h, const double* phi, const double* u0,
                         const unsigned char* obstacle, double h_ref);

/* Advance nsteps time steps (asynchronous).  After an instability has been
 * latched, further steps do nothing.  Launch sequence is captured once into a
 * CUDA graph per distinct nsteps and replayed. */
fsl_status fsl_step(fsl_handle* h, int nsteps);

/* Observables (fsl_observe `what`).  host_out must hold `bytes` bytes. */
enum {
  FSL_OBS_TOTAL_MASS = 1,    /* double: sum of liquid zeroth moments + interface m + lost mass */
  FSL_OBS_COLUMN_HEIGHT = 2, /* double: sum_j phi(0, j, k), averaged over k (surface elevation + depth) */
  FSL_OBS_FRONT = 3,         /* double: 1 + largest i of an interface cell with j = 0 */
  FSL_OBS_HEIGHT = 4,        /* double: 1 + largest j of an interface cell with i = 0 */
  FSL_OBS_MAX_VELOCITY = 5,  /* double: max |u| over fluid cells */
  FSL_OBS_STATUS = 6,        /* int64[2]: {FSL_OK or FSL_ERR_UNSTABLE, first unstable step or -1} */
  FSL_OBS_STEP = 7,          /* int64: steps taken */
  FSL_OBS_COUNTS = 8,        /* int64[4]: last step's {filled, emptied, new interface, interface} */
  FSL_OBS_LOST_MASS = 9,     /* double: mass of converted cells that had no interface neighbour */
  FSL_OBS_TRACE = 10,        /* double[3 * steps]: per step {column height at i=0, front, height} */
  FSL_OBS_FIELD_PDF = 16,    /* double[q N]: stored post-collision PDFs (valid in fluid cells) */
  FSL_OBS_FIELD_TYPES = 17,  /* uint8[N]: 0 gas, 1 interface, 2 liquid, 3 obstacle */
  FSL_OBS_FIELD_PHI = 18,    /* double[N]: fill level */
  FSL_OBS_FIELD_MASS = 19,   /* double[N]: cell mass m (meaningful in interface cells) */
  FSL_OBS_FIELD_KAPPA = 20,  /* double[N]: curvature K = -div(n_hat) (interface cells, sigma != 0) */
  FSL_OBS_FIELD_BUBBLE = 21, /* int32[N]: bubble of each gas or interface cell (dense index of
                                the bubble's smallest cell), -1 none or model off */
  FSL_OBS_FIELD_PRESSURE = 22 /* double[N]: volume pressure seen by each cell (p_volume where
                                the model is off or the cell has no bubble) */
};
/* Reads an observable into host memory; synchronises the stream.
 * FSL_ERR_ARG if `bytes` is smaller than the observable. FSL_OBS_TRACE holds
 * at most fsl_trace_capacity steps (oldest first; extra steps overwrite the
 * ring) and writes min(steps, capacity) records. */
fsl_status fsl_observe(fsl_handle* h, int what, void* host_out, size_t bytes);

/* Enable (every >= 1) or disable (0) the per-step trace of
 * FSL_OBS_TRACE; clears the ring.  Capacity in steps: fsl_trace_capacity. */
fsl_status fsl_set_trace(fsl_handle* h, int every);
int fsl_trace_capacity(void);

/* Checkpoint: fsl_state_bytes gives the size; fsl_save copies the full
 * simulation state to host memory, fsl_load restores it (same config).
 * Resuming from a checkpoint is bit-identical to an uninterrupted run. */
fsl_status fsl_state_bytes(const fsl_handle* h, size_t* bytes);
fsl_status fsl_save(fsl_handle* h, void* host_dst, size_t bytes);
fsl_status fsl_load(fsl_handle* h, const void* host_src, size_t bytes);

/* Release the handle (the workspace and stream stay with the caller). */
fsl_status fsl_destroy(fsl_handle* h);

/* Lattice table used by the library: c (3q ints) and w (q doubles).
 * FSL_ERR_ARG for an unknown lattice. */
fsl_status fsl_lattice_table(int lattice, int* c3q, double* w);

/* Number of kernel launches one fsl_step(1) issues. */
int fsl_launches_per_step(const fsl_handle* h);

/* Bulk stream-collide kernel of the FP32 / FP16 / BF16 storages (the FP64
 * path has one kernel).  All variants collide two neighbouring cells at once
 * in packed FP32 and give identical results (same explicitly rounded
 * arithmetic on the same inputs); they differ in how the stored values reach
 * the registers:
 *   PAIR, PAIR_R96, PAIR_R80, PAIR_R128: two cells per thread, 128 threads
 *     per block (tiles of 256 cells along x), one aligned 2-value load per
 *     direction, values pulled from x -/+ 1 exchanged between lanes by warp
 *     shuffles.  PAIR, PAIR_R96 and PAIR_R80 collide both cells together in
 *     packed FP32 with at most 128, 96 and 80 registers per thread (four,
 *     five and six blocks per SM); PAIR_R128 collides them one after the
 *     other (128 registers);
 *   TMA: persistent, tiles of 256 cells with liquid (listed by a pre-pass)
 *     staged in shared memory by bulk copies through a ring of
 *     mbarrier-guarded stages, one producer warp and four consumer warps;
 *   QUAD_64 (16-bit storages only): four cells per thread, 64 threads per
 *     block, one 8-byte load per direction kept packed until the collision;
 *   WARP_TMA: persistent, every warp streams its own 64-cell row segments
 *     with liquid (listed by a pre-pass) through a private ring of
 *     shared-memory stages filled by bulk copies, two cells per lane;
 *   PAIR_PIPE (16-bit storages only): as PAIR_R128, but each block walks a
 *     strided sequence of rows and issues the loads of its next row before
 *     colliding the current one (software pipelining over rows);
 *   CPA, CPA_DEEP, CPA_R96: persistent, tiles of 256 cells with liquid
 *     (listed by a pre-pass) staged in a ring of shared-memory stages by
 *     16-byte asynchronous copies (cp.async) that all 128 threads of a block
 *     issue; the copies of the next tiles are in flight while the block
 *     collides the current one.  16-bit storages: CPA 3 stages and 4 blocks
 *     per SM, CPA_DEEP 4 stages and 3 blocks, CPA_R96 (16-bit only) 2 stages
 *     and 5 blocks (at most 102 registers); FP32: CPA 2 stages and 3 blocks,
 *     CPA_DEEP 3 stages and 2 blocks;
 *   SEG, SEG_R128: persistent warps walk the list of 64-cell row segments
 *     with liquid (listed by a pre-pass), two cells per lane as in PAIR, with
 *     the flag and PDF loads of a segment in flight together (no warp is
 *     spent on gas-only rows); at most 96 (SEG) or 128 (SEG_R128) registers;
 *   CELL, CELL_R80: as SEG, but one cell per thread: one value loaded per
 *     direction straight from the source cell (no shuffles), the collision
 *     on one cell in FP32, at most 64 (CELL) or 80 (CELL_R80) registers;
 *   TMA_R96 (16-bit storages only): as TMA with three stages and four blocks
 *     per SM (at most 102 registers), sixteen consumer warps per SM.
 * DEFAULT is PAIR_R128; the Python autotuner
 * (paper_2207_14496_gb300.autotune) measures the variants instead.
 * fsl_set_variant drops captured step graphs; FSL_ERR_ARG for an unknown
 * variant and for QUAD_64, PAIR_PIPE, CPA_R96 or TMA_R96 with FP32 storage. */
enum { FSL_VARIANT_DEFAULT = 0, FSL_VARIANT_PAIR = 1, FSL_VARIANT_PAIR_R128 = 2,
       FSL_VARIANT_PAIR_R96 = 3, FSL_VARIANT_TMA = 4, FSL_VARIANT_QUAD_64 = 5,
       FSL_VARIANT_WARP_TMA = 6, FSL_VARIANT_PAIR_PIPE = 7, FSL_VARIANT_PAIR_R80 = 8,
       FSL_VARIANT_CPA = 9, FSL_VARIANT_CPA_DEEP = 10, FSL_VARIANT_CPA_R96 = 11,
       FSL_VARIANT_SEG = 12, FSL_VARIANT_SEG_R128 = 13, FSL_VARIANT_CELL = 14,
       FSL_VARIANT_CELL_R80 = 15, FSL_VARIANT_TMA_R96 = 16 };
fsl_status fsl_set_variant(fsl_handle* h, int variant);
int fsl_get_variant(const fsl_handle* h);

/* Measurement of one kernel on the current state, for roofline reports.
 * kernel: FSL_KERNEL_STREAM_COLLIDE, the bulk pull stream-collide pass over
 * all cells (Eqs. nm-lbm-collision, nm-lbm-streaming; liquid cells), timed
 * alone; FSL_KERNEL_BULK_PASS, the same pass together with the list pre-pass
 * that some variants launch before it (what one step spends on the bulk).
 * Launches it `reps` times on the bound stream, each bracketed by CUDA
 * events, and leaves the simulation state unchanged (the pass only reads the
 * current PDF buffer and writes the other one).  out4 (host, 4 doubles):
 * average launch time in ms, algorithmic bytes per launch (liquid cells x
 * 2 q x storage bytes + one flag byte per cell), number of liquid cells,
 * number of interface cells.  Synchronises
 * the stream.  FSL_ERR_ARG for another kernel code or reps < 1. */
enum { FSL_KERNEL_STREAM_COLLIDE = 1, FSL_KERNEL_BULK_PASS = 2 };
fsl_status fsl_kernel_stats(fsl_handle* h, int kernel, int reps, double* out4);

/* Self-check of the library's bounded device waits (failure path).  Launches
 * one block on the bound stream that waits at the conversion phase's grid
 * barrier for an arrival that never comes; the wait gives up after its time
 * bound (0.2 s), the handle's timeout bit is latched, and from then on
 * fsl_observe(FSL_OBS_STATUS) reports FSL_ERR_TIMEOUT, as after any device
 * wait that gave up.  Nothing else of the state changes; the CUDA context
 * stays usable.  Synchronises the stream.  FSL_ERR_STATE before
 * fsl_init_fill. */
fsl_status fsl_selftest_wait(fsl_handle* h);

/* Total mass of a state held in caller-owned device arrays, for callers that
 * cannot allocate device memory when they need it (inside a host callback or
 * another allocator, under a fixed device-memory budget, or in a loop that
 * must not let an allocation synchronise the device).  The paper has no
 * counterpart: this is a library convenience.  It allocates nothing: its
 * reduction scratch is a static 16 KiB device array inside the library,
 * shared by all calls; calls whose kernels overlap on the GPU race on it.
 * The first call on each device looks up that array and loads the entry
 * point's kernels (make it before any stream capture).
 *   cfg: lattice, precision, nx/ny/nz (other fields ignored);
 *   d_pdf: device, q planes of nx*ny*nz stored values in the dense layout
 *     (x fastest, no row padding) and the storage of cfg->precision (FP64:
 *     f_i; FP32: f_i - w_i; FP16: (f_i - w_i) * 2^15; BF16: f_i - w_i);
 *   d_types: device, nx*ny*nz type codes (0 gas, 1 interface, 2 liquid, 3 obstacle);
 *   d_mass: device, nx*ny*nz doubles (read in interface cells);
 *   d_lost: device, nx*ny*nz doubles of lost mass per cell, or NULL;
 *   d_out: device, one double: sum of liquid zeroth moments + interface mass + lost mass;
 *   cuda_stream: the stream to run on (cudaStream_t as void*).
 * Asynchronous.  FSL_ERR_ARG for a null pointer, a bad lattice or size, or
 * more than 33554432 cells (the scratch limit; message in fsl_last_error). */
fsl_status fsl_total_mass_noalloc(const fsl_config* cfg, const void* d_pdf,
                                  const unsigned char* d_types, const double* d_mass,
                                  const double* d_lost, double* d_out, void* cuda_stream);

/* Batched stepping of many independent domains (the paper runs one domain at
 * a time; this is the throughput form for sets of small problems of uneven
 * sizes and refilling schemes).  A batch groups existing handles, each with
 * its own configuration, workspace and state; fsl_batch_step advances every
 * member by nsteps with one CUDA-graph launch per chunk of steps on the
 * batch's stream.  When every member stores 16- or 32-bit PDFs and none runs
 * the bubble model, each kernel of a step is launched once for all members
 * of a lattice and storage (up to 256 members per launch, one member per
 * blockIdx.y; the member reads its pointers, geometry and parameters from a
 * record in its own workspace), so a step of the whole batch costs ten
 * launches; otherwise each member's kernels form an independent branch
 * (a child graph per member, no edges between members).  Either way the GPU
 * runs the domains side by side instead of one after another.
 *   handles: host array of n >= 1 handles, all initialised (fsl_init_fill or
 *     fsl_load done) and bound to streams of one device; the batch keeps the
 *     pointers, not the array; the handles must outlive the batch;
 *   cuda_stream: the stream the graphs launch on (cudaStream_t as void*, not
 *     the legacy default stream);
 *   chunk: steps per captured graph, 1..64 (each member contributes
 *     chunk x fsl_launches_per_step kernel nodes to a graph);
 *   out: receives the batch (release with fsl_batch_destroy, which leaves the
 *     handles alone).
 * fsl_batch_step orders itself after the work already queued on every
 * member's stream and queues the members' later work after it, so
 * fsl_observe on a member sees the batched steps.  A member that was
 * re-initialised, loaded or given another variant since the last capture is
 * recaptured.  Each member's results are bit-identical to fsl_step on it
 * alone.  Errors: FSL_ERR_ARG (null, n < 1, chunk out of range, a null or
 * uninitialised member), FSL_ERR_CUDA (capture, instantiation or launch). */
typedef struct fsl_batch fsl_batch;
fsl_status fsl_batch_create(fsl_handle* const* handles, int n, void* cuda_stream, int chunk,
                            fsl_batch** out);
fsl_status fsl_batch_step(fsl_batch* b, int nsteps);
fsl_status fsl_batch_destroy(fsl_batch* b);

/* Discrete adjoint of the step, for gradients of a misfit of the surface
 * elevation (Sec. 4.1's observable: the column height sum_y phi(0, y, z),
 * averaged over z) with respect to the viscosity, the gravity and the
 * initial state.  The paper has no adjoint; this is the differentiation
 * pattern built around its method.  Scope: FP64 or FP32 storage, SRT, EQ
 * refilling, no surface tension, no turbulence model, no-slip walls or
 * periodic faces, no interior obstacles, no bubble model (FSL_ERR_ARG
 * otherwise).  Cell types
 * and every conversion decision of the forward run are replayed, so the
 * gradient is that of the step map with those decisions fixed (the usual
 * discrete adjoint of a free-surface scheme); the stream-collide, the
 * free-surface boundary condition, the interface mass flux, the fill-level
 * update, the excess-mass redistribution and the EQ refilling are
 * differentiated by hand-written kernels.
 *   fsl_adjoint_workspace_bytes: device bytes for `nsteps` steps with a
 *     checkpoint every `every` steps (1 <= nsteps <= fsl_trace_capacity());
 *     memory grows with nsteps / every whole-state copies plus every + 1
 *     recorded levels;
 *   fsl_adjoint_create: binds the adjoint to an initialised handle; the
 *     caller owns the 256-byte-aligned device workspace (released after
 *     fsl_adjoint_destroy); the adjoint runs on the handle's stream;
 *   fsl_adjoint_forward: advances the handle by nsteps from its current
 *     state (time level 0) and writes the column height after each step to
 *     column (host, nsteps doubles); checkpoints whole states on the device;
 *   fsl_adjoint_backward: given dJ/dcolumn(t) for t = 1..nsteps (host,
 *     nsteps doubles) writes out (host, 4 + 2 nx ny nz doubles): dJ/dnu,
 *     dJ/dg_x, dJ/dg_y, dJ/dg_z (the gravity's direct effect and its effect
 *     through the hydrostatic initial density of fsl_init_fill), then
 *     dJ/drho0 and dJ/dphi0 per cell of the level-0 state (dense, x fastest;
 *     rho0 the initial density, phi0 the initial fill level of interface
 *     cells).  Replays each segment from its checkpoint; leaves the handle at
 *     the end of the forward pass.  FSL_ERR_STATE before a forward pass.
 * Synchronous (they synchronise the handle's stream). */
typedef struct fsl_adjoint fsl_adjoint;
fsl_status fsl_adjoint_workspace_bytes(const fsl_handle* h, int nsteps, int every, size_t* bytes);
fsl_status fsl_adjoint_create(fsl_handle* h, int nsteps, int every, void* d_workspace,
                              size_t bytes, fsl_adjoint** out);
fsl_status fsl_adjoint_forward(fsl_adjoint* a, double* column);
fsl_status fsl_adjoint_backward(fsl_adjoint* a, const double* dj_dcolumn, double* out);
fsl_status fsl_adjoint_destroy(fsl_adjoint* a);

/* Static description of a status code; last CUDA error text of this thread. */
const char* fsl_status_string(fsl_status s);
const char* fsl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FSL_H */
