/*
 * ns.h - C ABI of the GB300 (sm_103a) fractional-step Navier-Stokes hot path.
 *
 * The method (Ha, Park & You, arXiv:1812.01178):
 *   Sec. 2.1  incompressible NS, Eq. (NScontinuity) and Eq. (NSmomentum), on a staggered grid:
 *             u on x-faces, v on y-faces, w on z-faces, p at cell centres; uniform x and z,
 *             wall-clustered y; no-slip wall at the bottom, no-slip or stress-free top;
 *             periodic z; x periodic (channel) or inflow / convective outflow (flat plate).
 *   Sec. 2.2  semi-implicit fractional step: low-storage RK3 (convection) + Crank-Nicolson
 *             (viscous), ADI factorisation into tridiagonal solves along x, y and z, Poisson
 *             equation by Fourier transforms in x and z plus tridiagonal solves in y, projection
 *             with the pseudo-pressure phi.
 *   Sec. 3.2  PDD / PPT divide-and-conquer solution of tridiagonal systems, Eqs. (smidentity)
 *             to (xppt): used here for the contiguous x-lines, split across the lanes of a warp.
 *
 * Units and layout.  Every field is a dense array of double with x fastest, then y, then z:
 *   u : nz * ny     * nx   (x-face i, y-centre j, z-centre k)
 *   v : nz * (ny+1) * nx   (x-centre i, y-face j, z-centre k); rows j = 0 and j = ny are the
 *                          walls and hold 0
 *   w : nz * ny     * nx   (x-centre i, y-centre j, z-face k)
 *   p : nz * ny     * nx   (cell centres)
 * Element (i, j, k) of u is u[(k * ny + j) * nx + i].  With inflow / outflow in x (bc_x = 1)
 * u holds faces i = 0..nx-1, face 0 being the inflow (fixed in time), and five boundary planes
 * complete the state (x fastest within a plane is not used: index k * rows + j):
 *   u_out : nz * ny      u on the outflow face x = Lx (advanced by the convective condition
 *                        dU/dt + U_c dU/dx = 0 and shifted so the outflow flux equals the inflow
 *                        flux before every Poisson solve)
 *   v_in, v_out : nz * (ny+1)   v on the inflow / outflow face (inflow fixed, outflow convected)
 *   w_in, w_out : nz * ny       w on the inflow / outflow face (same)
 * v and w see these faces through linear ghost cells (ghost = 2 f_face - f_adjacent).  All device pointers must be 256-byte
 * aligned (cudaMalloc / torch allocations are).  nx and nz are 2^a 3^b with a >= 3 (the
 * mixed radix-2/4/3 FFT of Sec. 2.2; multiples of 8) in [8, 4096], and nx must admit a partition
 * shape of the x solver (ns_set_partition).  ny is in [4, 1024].  Other sizes give NS_ERR_SIZE
 * (ns_workspace_bytes returns 0 for them).
 *
 * Ownership.  Fields and the workspace are allocated by the caller (device memory) and are
 * never freed by the library.  The library owns only the opaque context (host memory) and the
 * CUDA graph it captures.  If ns_init gets workspace == NULL, the library allocates the
 * workspace itself with cudaMalloc and frees it in ns_destroy.
 *
 * Streams.  All work is enqueued on the stream passed to ns_init (a cudaStream_t cast to
 * void*; NULL means the legacy default stream).  No call synchronises the host except
 * ns_sync and the *_host entry points.
 *
 * Errors.  Every call returns an ns_status.  Argument errors are detected before any work is
 * enqueued.  Asynchronous CUDA failures surface as NS_ERR_CUDA at the next call that checks
 * the stream (ns_sync, ns_step_host).  ns_last_error(ctx) gives a one-line message.  No call
 * aborts the process or throws.
 */
#ifndef NS_GB300_H
#define NS_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ns_ctx ns_ctx;

typedef enum {
  NS_OK = 0,
  NS_ERR_ARG = 1,        /* NULL pointer, bad enum value, misaligned pointer */
  NS_ERR_SIZE = 2,       /* grid size outside the supported range */
  NS_ERR_CUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  NS_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up (status word set) */
  NS_ERR_STATE = 5,      /* call made in the wrong state (e.g. during graph capture) */
  NS_ERR_UNSUPPORTED = 6 /* option not built */
} ns_status;

/* Precision of the increment path (Sec. 2.2 solves everything in one precision; the mixed
 * form is this library's addition):
 *   NS_FP64  : every stage in FP64.
 *   NS_MIXED : RHS stencils and the ADI increment solves in FP32 (r, delta and N_prev stored
 *              as float); state accumulation u* = u + delta, divergence, the Poisson solve
 *              (all modes) and the projection stay FP64. */
enum { NS_FP64 = 0, NS_MIXED = 1 };

typedef struct {
  int nx, ny, nz;        /* cells in x, y, z */
  double lx, lz;         /* domain lengths in the periodic directions */
  const double* yf;      /* ny+1 strictly increasing y-face coordinates, HOST memory, read
                            only during ns_init (Sec. 2.1: wall-clustered y grid) */
  int bc_x;              /* 0: periodic x; 1: inflow at x = 0, convective outflow at x = Lx */
  int bc_ytop;           /* 0: no-slip top wall, 1: stress-free top (v = 0, du/dy = dw/dy = 0) */
  double re;             /* Reynolds number of Eq. (NSmomentum); re <= 0 means inviscid */
  double fx;             /* constant body force along x (drives channel flow) */
  double dt;             /* time step, fixed for the lifetime of the context */
  int precision;         /* NS_FP64 or NS_MIXED */
  double u_conv;         /* convection speed U_c of the outflow condition (bc_x = 1 only) */
  int pressure_update;   /* NS_PRESSURE_DELTA or NS_PRESSURE_KIM_MOIN */
  int recycle_i;         /* 0: fixed inflow planes; else the u face 1..nx-1 recycled to the inflow */
  double delta_in;       /* inlet boundary-layer thickness of the recycling (recycle_i != 0) */
} ns_config;

/* Recycling inflow (Sec. 2.1 names the method of Lund, Wu & Squires, J. Comput. Phys. 140,
 * 1998).  With bc_x = 1 and recycle_i != 0, every time step first rewrites the inflow planes
 * (u on face 0, v_in, w_in) from the u face recycle_i, with v and w there averaged from the
 * centres recycle_i - 1 and recycle_i:
 *   means U, V, W are spanwise averages of that plane, fluctuations the plane minus them;
 *   delta_rec is the first height where U reaches 0.99 u_conv (linear between centres);
 *   gamma = (delta_rec / delta_in)^(1/8) is the inlet-to-recycle friction-velocity ratio;
 *   the row at height y takes mean and fluctuation at y gamma (inner) and y delta_rec / delta_in
 *   (outer) by linear interpolation (0 at the wall for u, w), inner mean gamma U, outer
 *   gamma U + (1 - gamma) u_conv, mean V unscaled, mean W zero, fluctuations times gamma, blended
 *   by W(y / delta_in) = (1 + tanh(4 (eta - 0.2) / (0.6 eta + 0.2)) / tanh 4) / 2 (1 above 1).
 * recycle_i outside [1, nx-1], delta_in <= 0, or recycle_i != 0 with bc_x = 0 give NS_ERR_ARG. */

/* Pressure update of each sub-step after the projection (the paper names only the
 * pseudo-pressure phi, Sec. 2.2):
 *   NS_PRESSURE_DELTA    : p = p + phi.
 *   NS_PRESSURE_KIM_MOIN : p = p + phi - beta_k L phi, beta_k = alpha_k dt / (2 Re), L = D G the
 *                          operator of the Poisson solve (Kim & Moin, J. Comput. Phys. 59, 1985),
 *                          which makes the pressure consistent to second order in time.
 * The velocities are the same under both. */
enum { NS_PRESSURE_DELTA = 0, NS_PRESSURE_KIM_MOIN = 1 };

typedef struct {
  double* u;             /* device pointers, layouts above; updated in place */
  double* v;
  double* w;
  double* p;
  double* u_out;         /* boundary planes (bc_x = 1 only, else ignored and may be NULL) */
  double* v_in;
  double* v_out;
  double* w_in;
  double* w_out;
} ns_fields;

/* Workspace bytes needed by ns_init for this configuration (0 if cfg is invalid). */
size_t ns_workspace_bytes(const ns_config* cfg);

/* Create a context: validates cfg, computes the line-independent coefficient tables of every
 * ADI factor (Sec. 2.2) and of the partitioned x solver (Sec. 3.2: spikes v, w of Eq. (blockAY)
 * and the reduced-system eliminators), the Poisson y factors per (kx, kz) and the FFT twiddles,
 * and stores them in the workspace.  `fields` are the caller's state arrays (N_prev is kept in
 * the workspace).  Returns NS_ERR_SIZE / NS_ERR_ARG / NS_ERR_UNSUPPORTED / NS_ERR_CUDA. */
ns_status ns_init(ns_ctx** out, const ns_config* cfg, const ns_fields* fields,
                  void* workspace, size_t ws_bytes, void* cuda_stream);

/* Explicit right-hand side of RK3 sub-step `substep` (0, 1, 2), Sec. 2.2 in delta form:
 *   r_i = dt [ -gamma_k N_i(u) - zeta_k N_prev_i - alpha_k G_i p + (alpha_k/Re) L u_i + alpha_k f_i ]
 * with N = divergence-form convection (Eq. NSmomentum, 2nd-order central), L the viscous
 * operator and G the pressure gradient.  Writes r into the workspace buffers NS_BUF_RU/RV/RW
 * and -dt gamma_k N(u) into NS_BUF_NU/NV/NW: N is formed and kept already multiplied by its weight
 * in r, and read back by the next sub-step as N_prev with weight zeta_(k+1) / gamma_k (substep 0
 * ignores it). */
ns_status ns_rhs(ns_ctx* ctx, int substep);

/* One ADI factor (Sec. 2.2): solves (I - beta_k delta_dd) x = r in place on the r buffers for
 * all three components, beta_k = alpha_k dt / (2 Re).
 *   dir 0: x-lines (contiguous, periodic): each line split into P partitions across the lanes
 *          of a warp and solved with PDD or PPT (Sec. 3.2, Eqs. blockAx - xppt).
 *   dir 1: y-lines (stride nx), one thread per line, precomputed Thomas factors.
 *   dir 2: z-lines (stride nx*ny, periodic), one thread per line; then forms the intermediate
 *          velocity u* = u + delta in the caller's u, v, w (FP64 accumulation). */
ns_status ns_adi_sweep(ns_ctx* ctx, int dir, int substep);

/* Pressure Poisson solve of sub-step `substep` (Sec. 2.2): b = D u* / (alpha_k dt); forward
 * real FFT along z and complex FFT along x; one complex tridiagonal solve along y per (kx, kz)
 * with zero normal gradient at both y boundaries (the singular (0,0) mode is gauged by
 * phi_hat(j=0) = 0); inverse FFTs.  Writes phi into NS_BUF_PHI.  substep = -1 uses scale 1
 * (b = D u), for making an initial field divergence-free.
 * NS_MIXED: b is formed in FP64 and kept (in NS_BUF_SPEC), the transforms run in FP32 on a
 * complex64 spectrum held over NS_BUF_RU/RV (phi1 in NS_BUF_RW: the three r buffers are scratch of
 * the solve), the y solves keep FP64 arithmetic, and one refinement on the FP64 residual
 * b - D G phi1 gives phi = phi1 + phi2 (FP64) at the accuracy of the FP64 solve. */
ns_status ns_poisson_solve(ns_ctx* ctx, int substep);

/* Projection of sub-step `substep` (Sec. 2.2): u = u* - alpha_k dt G phi, p = p + phi.
 * substep = -1 projects with scale 1 and leaves p unchanged. */
ns_status ns_project(ns_ctx* ctx, int substep);

/* One full RK3 sub-step: ns_rhs, (outflow update), ns_adi_sweep x/y/z, (outflow mass-flux
 * correction), ns_poisson_solve, ns_project; the bracketed stages run only with bc_x = 1. */
ns_status ns_substep(ns_ctx* ctx, int substep);

/* nsteps time steps of three sub-steps each (Table 1 counts one step = three sub-steps).
 * The three sub-steps are captured once as a CUDA graph and replayed. */
ns_status ns_step(ns_ctx* ctx, int nsteps);

/* Time step at a fixed CFL number (the paper's runs hold CFL = 1.0, Sec. 4).
 *
 * ns_convective_rate: *rate = max over cells of |u| (1/dx) + |v_c| (1/dy_j) + |w| (1/dz) of the current
 * fields, with u and w the values on the cell's lower x and z faces and v_c the average of its two
 * y faces, so that the convective CFL number is dt * rate.  One device max-reduction on the
 * context's stream, then a synchronising 8-byte read.  NS_ERR_STATE if the fields hold a
 * non-finite value.
 *
 * ns_set_dt: make dt the time step of the following sub-steps.  Rebuilds every table that
 * depends on dt (RHS rows, ADI factors and PDD/PPT tables, with the PDD admissibility test of the
 * automatic mode redone, and the sub-step constants) on the host and copies them to the workspace
 * asynchronously.  The first call switches the kernels to reading the sub-step constants from the
 * workspace and drops the captured graphs once (the next ns_step captures again); later calls
 * keep them.  dt must be positive and finite (NS_ERR_ARG).  Synchronises the stream on entry.
 *
 * ns_step_cfl: nsteps steps, each preceded by dt = cfl / rate of the velocity at its start.  The
 * rate, dt and every dt-dependent table are computed on the device inside the captured step graph
 * (rate reduction, then two kernels that build the same tables as ns_set_dt, with the same
 * operations and roundings, so the steps are bitwise those of ns_convective_rate + ns_set_dt +
 * ns_step); the host reads the dt log back once per 1024 steps.  dts, if not NULL, receives the
 * nsteps values of dt (host array).  cfl must be positive and finite (NS_ERR_ARG).  A rate that is
 * not positive and finite (a non-finite field, or fluid at rest) keeps the previous dt for that
 * step and makes the call return NS_ERR_STATE after the run of steps it fell in (the message names
 * the step); the fields are then not a solution.  Synchronises the stream. */
ns_status ns_convective_rate(ns_ctx* ctx, double* rate);
ns_status ns_set_dt(ns_ctx* ctx, double dt);
ns_status ns_step_cfl(ns_ctx* ctx, int nsteps, double cfl, double* dts);

/* Number of kernel launches in one ns_step time step: the kernel nodes of the step's graph (it is
 * captured here if ns_step has not run yet).  -1 on error (ns_last_error). */
int ns_launches_per_step(ns_ctx* ctx);

/* ns_step with per-kernel timing: replays a captured step that also records a CUDA event before
 * every kernel (and after the last) on the context's stream, waits for each step, and adds each
 * kernel's event-to-event time (ms) into kernel_ms[ns_kernel_name index], summed over the three
 * sub-steps and nsteps steps.  kernel_ms: host array of at least ns_kernel_count() floats (zeroed
 * first).  The state advances exactly as with ns_step. */
ns_status ns_step_profiled(ns_ctx* ctx, int nsteps, float* kernel_ms, int nk);

/* Number of kernel slots in one sub-step, and the name of slot idx, in launch order: recycle,
 * rhs, outflow, adi_x, adi_y, adi_z, flux_correct, poisson_div_fftz, poisson_x_fwd,
 * poisson_tdma_y, poisson_x_inv, poisson_ifftz, poisson_refine, project ("" if idx is out of
 * range).  recycle launches only in sub-step 0 with recycle_i != 0; outflow and flux_correct only
 * with bc_x = 1; poisson_refine (the FP64 residual and the second FP32 Poisson pass, five kernels)
 * only with NS_MIXED (an idle slot's time is 0); poisson_x_* are FFTs for periodic x and cosine
 * transforms (DCT-II / its inverse) for inflow / outflow. */
int ns_kernel_count(void);
const char* ns_kernel_name(int idx);

/* End-to-end variant of ns_step for callers whose state lives in HOST memory: copies u, v, w,
 * p from the host arrays (pinned memory recommended) to the context's device fields, runs
 * nsteps steps, copies them back and synchronises.  Host arrays use the device layout. */
ns_status ns_step_host(ns_ctx* ctx, double* u, double* v, double* w, double* p, int nsteps);

/* Make the current velocity discretely divergence-free (with bc_x = 1: outflow mass-flux
 * correction first; then ns_poisson_solve(-1) + ns_project(-1)). */
ns_status ns_make_divergence_free(ns_ctx* ctx);

/* Partitioning of the x-line solver (Sec. 3.2): P partitions of M = nx/P rows per line, P a
 * power of two from 1 to 32, M in {1, 2, 3, 4, 6, 8, 9, 12, 16} (rows held in registers) or, at
 * P = 32, M in {24, 32, 48, 64, 96, 128} (long lines staged in shared memory); other P give NS_ERR_ARG.
 * mode 0 = automatic (PDD when the coupling PDD drops is below its tolerance for every sub-step,
 * else PPT), 1 = PPT, 2 = PDD.  Rebuilds the tables and drops the captured graph.  The default P
 * is the largest admissible one with at least 8 rows per partition.
 *
 * dir 1 / 2: the y / z lines of the mixed form (NS_MIXED with nx a multiple of 32; otherwise
 * NS_ERR_UNSUPPORTED).  P = 0 solves every line whole, one thread per line; a nonzero P must be
 * the one partition shape the line kernels are built for (8 x {4, 6, 8, 12, 16, 24, 32},
 * 16 x {18, 32}, 32 x 32 rows; it is the default when the line length has one), else NS_ERR_ARG.
 * mode must be NS_PART_AUTO: PDD when the coupling it drops is below the FP32 tolerance for every
 * sub-step, else PPT.  Other dir: NS_ERR_ARG. */
enum { NS_PART_AUTO = 0, NS_PART_PPT = 1, NS_PART_PDD = 2 };
ns_status ns_set_partition(ns_ctx* ctx, int dir, int P, int mode);

/* Query the partitioning in use: *P, *mode (NS_PART_PPT or NS_PART_PDD) and the largest
 * coupling PDD drops over the three sub-steps (the admissibility measure).  dir 1 / 2 (y / z
 * lines): *P = 0 for lines solved whole (reported as NS_PART_PPT, dropped 0). */
ns_status ns_get_partition(ns_ctx* ctx, int dir, int* P, int* mode, double* pdd_dropped);

/* Pick P and the PDD/PPT mode for the x solver by timing every admissible P on the context's
 * stream (CUDA events), and, in the mixed form with nx a multiple of 32, the y and z line shapes
 * (partitioned or whole), each by timing its sweep.  Leaves the fastest installed.  The timed
 * sweeps run on the current r buffers and velocity; both are saved to temporary device memory
 * (cudaMalloc, freed before return) and restored.  Synchronises the stream. */
ns_status ns_autotune(ns_ctx* ctx);

/* Workspace buffers, for inspection and for stage-by-stage testing. */
enum {
  NS_BUF_RU = 0, NS_BUF_RV = 1, NS_BUF_RW = 2,   /* r / delta (double, or float if NS_MIXED) */
  NS_BUF_NU = 3, NS_BUF_NV = 4, NS_BUF_NW = 5,   /* -dt gamma_k N of the last ns_rhs (double, or
                                                   float if NS_MIXED) */
  NS_BUF_PHI = 6,                               /* phi, double, nz*ny*nx */
  NS_BUF_SPEC = 7,                              /* spectral buffer, complex double,
                                                   (nz/2+1)*ny*nx, layout [kz][j][kx]; NS_MIXED:
                                                   the FP64 right-hand side of the Poisson solve */
  NS_BUF_POIS_MODE = 8                          /* NS_MIXED only: one byte per Poisson mode,
                                                   layout [kz][kx], (nz/2+1)*nx; 1 where its y
                                                   solve may run in FP32 arithmetic (kz > 0 and
                                                   the Skeel condition number of its y matrix
                                                   <= 4096), 0 where it runs in FP64.  With nx
                                                   a multiple of 16 the solve goes by tiles of 16
                                                   kx, in FP32 only where all 16 flags are 1, the
                                                   other tiles in float-float arithmetic (about
                                                   48 bits) from the FP64 factors.
                                                   NS_ERR_UNSUPPORTED for an FP64 context */
};
ns_status ns_get_buffer(ns_ctx* ctx, int which, void** ptr, size_t* bytes);

/* Context-free Poisson solve that allocates nothing (this entry point has no counterpart in the
 * paper).  It serves callers that may not call cudaMalloc: plugins inside a host framework that
 * owns all device memory through its own pool allocator, and fixed-latency loops that must not
 * allocate after start-up (an allocation can synchronise the device and take unbounded time).
 *
 * Computes the same phi as ns_poisson_solve(ctx, substep) for an NS_FP64 context made from cfg
 * (nx, ny, nz, lx, lz, yf and, for substep >= 0, dt are used; bc_x must be 0): D G phi = D u / s
 * with s = alpha_k dt (substep k = 0, 1, 2) or s = 1 (substep = -1).  The solve runs in FP64
 * only: cfg->precision must be NS_FP64 (NS_MIXED gives NS_ERR_UNSUPPORTED, other values
 * NS_ERR_ARG).  u, v, w: caller's device arrays in the field layouts above (read); phi: caller's
 * device array nz*ny*nx (written); all four 256-byte aligned (else NS_ERR_ARG).
 * Work goes on cuda_stream: the call queues the upload of small coefficient tables from static
 * host buffers, then synchronises cuda_stream (so earlier work on that stream completes first and
 * the host buffers may be reused), then queues the kernels and returns without waiting for them.
 *
 * Scratch: one file-scope device array of NS_STATIC_SCRATCH_BYTES, held by every GPU that loads
 * the library until the process exits.  A grid needing more (about 2 * 16 * (nz/2+1) * ny * nx
 * bytes) is rejected with NS_ERR_SIZE and a message; no cudaMalloc, cudaFree or other
 * allocating routine is called.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and sets kernel attributes; make that first call before any
 * stream capture.  Every call shares the array and rewrites what it reads, so results do not
 * depend on earlier calls, but calls that overlap on the GPU (e.g. on two streams) race.
 * Errors: NS_ERR_ARG / NS_ERR_SIZE / NS_ERR_UNSUPPORTED / NS_ERR_CUDA, message in
 * ns_last_error(NULL) on the calling thread. */
#define NS_STATIC_SCRATCH_BYTES (48u * 1024u * 1024u)
ns_status ns_poisson_solve_static(const ns_config* cfg, const double* u, const double* v, const double* w,
                                  double* phi, int substep, void* cuda_stream);

/* ---------------------------------------------------------------------------------------------
 * Batched ensembles: n independent instances (periodic x, one precision, any sizes) advanced
 * together.  Each stage of a sub-step is one persistent launch for the whole ensemble (per kernel
 * variant): its blocks walk the blocks of every instance, reading each instance's arguments from a
 * device table; one time step is one captured CUDA graph.  cfgs[i] / fields[i] describe instance
 * i exactly as for ns_init.  The workspace (caller-owned, or library-owned if NULL) holds every
 * instance's workspace plus the launch tables.
 * ------------------------------------------------------------------------------------------- */
typedef struct ns_batch ns_batch;

/* Workspace bytes for the ensemble (0 if any cfg is invalid, not periodic in x, or the
 * precisions differ). */
size_t ns_batch_workspace_bytes(const ns_config* cfgs, int n);

ns_status ns_batch_init(ns_batch** out, const ns_config* cfgs, const ns_fields* fields, int n,
                        void* workspace, size_t ws_bytes, void* cuda_stream);

/* nsteps time steps of every instance (graph captured on first use and replayed). */
ns_status ns_batch_step(ns_batch* b, int nsteps);

/* Number of kernel launches in one batched time step (3 sub-steps x stages x kernel variants). */
int ns_batch_launches_per_step(ns_batch* b);

/* Pick each instance's x partitioning by timing (as ns_autotune, x solver only: instances keep
 * their default y and z line shapes, so that instances of one size share launches), then
 * re-plan. */
ns_status ns_batch_autotune(ns_batch* b);

/* Set instance i's x partitioning (as ns_set_partition) and re-plan. */
ns_status ns_batch_set_partition(ns_batch* b, int i, int P, int mode);

/* The context of instance i (for its buffers, partition query or single-instance calls on the
 * batch's stream), NULL if out of range.  Owned by the batch. */
ns_ctx* ns_batch_instance(ns_batch* b, int i);

ns_status ns_batch_sync(ns_batch* b);
const char* ns_batch_last_error(ns_batch* b);
void ns_batch_destroy(ns_batch* b);

/* ---------------------------------------------------------------------------------------------
 * y-slab decomposition (Sec. 3.2, "Domain decomposition using parallel algorithms"; Algorithm 1):
 * the domain is cut into p slabs of whole x-z planes, slab r owning the cell rows [j0, j1) of y
 * (ns_slab_rows) and, of v, the faces j0 .. j1-1 (the last slab also the top face ny).  One slab
 * is one GPU's share in the paper's multi-GPU method.  Everything along x and z is local to a slab;
 * the y sweep of the ADI factorisation is split across slabs by PDD (Sec. 3.2, Eq. (Zpdd): one
 * exchange of end values with the two neighbours, Algorithm 1) or PPT (Eq. (Zppt): all-gather of
 * the end values), and the Poisson y solve of every (kx, kz) line by PPT.  With inflow /
 * convective outflow in x, the outflow mass-flux correction sums every slab's share (FLUX
 * exchange, an all-gather of one double); with the recycling inflow (recycle_i != 0) every slab
 * packs the recycle-plane samples of its rows (RCY exchange, an all-gather) and, in sub-step 0,
 * writes the inflow rows it holds from the whole plane (Sec. 2.1; the recycling of one context).
 * Built for NS_FP64 (with either pressure update; the PHI exchange carries phi of each slab's end
 * rows both ways, for the gradient and for the Kim-Moin Laplacian); other precisions give
 * NS_ERR_ARG; every slab needs at least 3 rows (ny >= 3 p).
 *
 * Local fields.  A slab's u, w, p hold rows j0-hb .. j1+ha-1 and its v the faces j0-hb .. j1+ha,
 * where hb = (r > 0) and ha = (r < p-1) are the halo rows below and above (layouts as above with
 * ny replaced by the local row count nyl + hb + ha); so do the five boundary planes of inflow /
 * outflow x.  The caller fills the owned rows (and, for the boundary planes, the halo rows too);
 * the halo rows of u, v, w, p are filled by the exchanges.
 *
 * Exchanges.  A sub-step is six phases (NS_SLAB_*) with an exchange after each:
 *   PACK (before the first sub-step only) -> HALO, RCY -> RHS -> ADIY -> ADIZ -> VSTAR, FLUX -> POIS
 *   -> POIS -> PHI -> PHI -> PROJECT -> HALO (ready for the next sub-step's RHS), and RCY after
 *   the PROJECT of sub-step 2
 * where the exchange named after a phase is NS_XCH_<name> (FLUX only matters with inflow /
 * outflow x; with periodic x it carries nothing the slabs read; RCY has slots of 0 bytes, and
 * nothing to move, without recycling).  For exchange x every slab has a send
 * buffer of ns_slab_slot_bytes bytes and a receive buffer of p such slots; after the phase that
 * writes its send buffer, the caller copies slab s's send buffer into slot s of every slab r that
 * reads it (ns_slab_slots: slots lo .. hi of slab r; the slab's own slot, where read, it writes
 * itself).  Between GPUs that is NCCL send / receive between neighbours or an all-gather; on one
 * GPU, device copies.  Buffers come from ns_slab_buffers.
 * ------------------------------------------------------------------------------------------- */
typedef struct ns_slab ns_slab;
enum { NS_XCH_HALO = 0, NS_XCH_ADIY = 1, NS_XCH_VSTAR = 2, NS_XCH_POIS = 3, NS_XCH_PHI = 4, NS_XCH_FLUX = 5,
       NS_XCH_RCY = 6, NS_XCH_COUNT = 7 };
enum { NS_SLAB_PACK = 0, NS_SLAB_RHS = 1, NS_SLAB_ADIZ = 2, NS_SLAB_POIS = 3, NS_SLAB_PHI = 4,
       NS_SLAB_PROJECT = 5 };

/* Rows [*j0, *j1) of slab r of p on ny rows (as even as possible).  Host only. */
ns_status ns_slab_rows(int ny, int p, int r, int* j0, int* j1);

/* Bytes of one exchange slot of kind xch for the whole-domain cfg (0 if invalid).  Host only. */
size_t ns_slab_slot_bytes(const ns_config* cfg, int p, int xch);

/* The slots lo .. hi (inclusive) of its receive buffer that slab r reads in exchange xch; ymode is
 * the slab's y-sweep mode (NS_PART_PDD: neighbours only; NS_PART_PPT: every slab).  Host only. */
ns_status ns_slab_slots(int p, int r, int xch, int ymode, int* lo, int* hi);

/* Host-only reference of the slab algebra (no device work): solves the tridiagonal line
 * a_j x_{j-1} + b_j x_j + c_j x_{j+1} = d_j of n unknowns (a_0, c_{n-1} ignored) cut into p blocks
 * as ns_slab_rows cuts ny rows, with the tables the slabs use (the same builder): every block of
 * A~ solved alone, the end values gathered, and the reduced system of Sec. 3.2 solved by PPT
 * (Eq. (Zppt), exact) or PDD (Eq. (Zpdd), the couplings between interfaces dropped), then each
 * block corrected.  mode is NS_PART_PPT or NS_PART_PDD; x (n doubles, host) receives the solution;
 * *dropped (if not NULL) the largest coupling PDD drops.  NS_ERR_ARG for NULL arrays, p < 1 or
 * n < 2p; NS_ERR_STATE for a singular reduced system. */
ns_status ns_slab_solve_line_host(int n, const double* a, const double* b, const double* c, const double* d, int p,
                                  int mode, double* x, double* dropped);

/* Workspace bytes of slab r (its sub-grid context, the slab tables and the exchange buffers); 0 if
 * the configuration is not supported. */
size_t ns_slab_workspace_bytes(const ns_config* cfg, int p, int r);

/* Create slab r of p of the whole-domain configuration cfg on `local` fields (device pointers,
 * 256-byte aligned, layouts above).  ymode: NS_PART_AUTO (PDD when the coupling it drops is at most
 * 1e-15 in every sub-step, else PPT), NS_PART_PPT or NS_PART_PDD for the y sweep.  The tables of
 * the y sweep and of the Poisson y solve (block factors, spikes, reduced-system rows) are built on
 * the host once.  workspace: caller's device memory of ns_slab_workspace_bytes, or NULL (the
 * library allocates it and frees it in ns_slab_destroy).  Errors: NS_ERR_ARG / NS_ERR_SIZE /
 * NS_ERR_CUDA / NS_ERR_STATE (a singular reduced system), message in ns_last_error(NULL). */
ns_status ns_slab_init(ns_slab** out, const ns_config* cfg, int p, int r, int ymode, const ns_fields* local,
                       void* workspace, size_t ws_bytes, void* cuda_stream);

/* Enqueue phase `phase` of RK3 sub-step `substep` on the slab's stream: it first reads the
 * receive buffer of the exchange before it, then runs its kernels and writes the send buffer of
 * the exchange after it. */
ns_status ns_slab_phase(ns_slab* s, int phase, int substep);

/* Send buffer, receive buffer and slot bytes of exchange xch (device pointers, slab-owned). */
ns_status ns_slab_buffers(ns_slab* s, int xch, void** send, void** recv, size_t* slot_bytes);

/* The y-sweep mode in use (NS_PART_PDD or NS_PART_PPT) and the largest coupling PDD drops. */
ns_status ns_slab_mode(ns_slab* s, int* ymode, double* ydrop);

/* The sub-grid context (for ns_get_buffer and the like); owned by the slab. */
ns_ctx* ns_slab_context(ns_slab* s);

ns_status ns_slab_sync(ns_slab* s);
const char* ns_slab_last_error(ns_slab* s);
void ns_slab_destroy(ns_slab* s);

/* Measurement aid (no counterpart in the paper): the FP64 FMA throughput of this GPU, the
 * denominator of the FP64-ALU roofline the solver's FP64 kernels are measured against.  Enqueues
 * one kernel of n_blocks blocks of 256 threads on cuda_stream; every thread runs 8 independent
 * chains of n_iter dependent FMAs (x = x * b + c), i.e. 16 * n_iter flops per thread, and writes
 * the sum of its chains to out[block * 256 + thread] (caller's device array of n_blocks * 256
 * doubles, written only).  Time it with CUDA events recorded on cuda_stream.  NS_ERR_ARG for a
 * NULL out or n_blocks, n_iter < 1; NS_ERR_CUDA if the launch fails (message in
 * ns_last_error(NULL) on the calling thread). */
ns_status ns_fp64_fma_probe(double* out, int n_blocks, int n_iter, void* cuda_stream);

/* Wait for all work on the context's stream; reports asynchronous CUDA errors. */
ns_status ns_sync(ns_ctx* ctx);

/* Last error message of the context (never NULL; "" when none).  ctx may be NULL, giving the
 * message of the last failed ns_init or ns_poisson_solve_static on this thread. */
const char* ns_last_error(ns_ctx* ctx);

/* Destroy the context (frees the graph and a library-allocated workspace, not the fields). */
void ns_destroy(ns_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* NS_GB300_H */
