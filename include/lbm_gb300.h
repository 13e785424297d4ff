/*
 * lbm_gb300.h -- C ABI of the GB300 (sm_103a) two-phase lattice Boltzmann library.
 *
 * The library advances the D2Q9 pseudopotential lattice Boltzmann method with curved solid walls
 * of Yu, Li & Wen, "Modified curved boundary scheme for two-phase lattice Boltzmann simulations"
 * (arXiv:1908.09235).  One time step is
 *   (i)  a fused pass over every fluid node: density and velocity (Eq. 5), the pseudopotential
 *        interaction force of Eq. (16) from psi(rho) of the eight neighbours, BGK collision with
 *        Guo forcing (Eqs. 1, 2, 4) and streaming (Eq. 3);
 *  (ii)  a pass over the boundary nodes that sets the populations entering the fluid across the
 *        curved wall, with the scheme chosen at creation: halfway bounce-back, Filippova-Haenel
 *        (Eqs. 7-10), Mei-Luo-Shyy (Eqs. 7, 8, 10, 11), linear / quadratic Bouzidi (Eqs. 12, 13),
 *        Zhao-Yong (Eq. 14), modified scheme A (Eqs. 15, 17, 18), modified scheme B
 *        (Eqs. 19-22) or the fictitious density of Bao et al. (Eq. 23).
 * Everything in (i) and (ii) runs in CUDA kernels on one GPU; the host only validates arguments,
 * builds the Carnahan-Starling constants and copies fields in and out.
 *
 * Conventions.  Node (i, j) sits at position (i, j) in lattice units, i in [0, nx), j in [0, ny);
 * its linear index is j*nx + i (row-major, y outer).  The outer box is periodic in x and y (x
 * becomes a channel with a velocity inlet and an outlet after lbm_set_inflow, Sec. 4.2).
 * D2Q9 directions: 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 * All host arrays are caller-owned and are read or written only during the call.  Device state is
 * owned by the context and released by lbm_destroy.  Functions return an lbm_status; a non-zero
 * status is also recorded as the context's sticky error (lbm_last_error) and makes every later
 * call on that context return the same status, except lbm_destroy and lbm_last_error.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, library-owned */

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,    /* invalid argument; nothing was changed                              */
  LBM_ENOMEM = 2,    /* device allocation failed                                           */
  LBM_ECUDA = 3,     /* a CUDA call failed (message in lbm_last_error)                     */
  LBM_EUNSTABLE = 4, /* a density became non-positive or not finite (detected by lbm_mass) */
  LBM_ETIMEOUT = 5,  /* a bounded device wait gave up                                      */
  LBM_ESTATE = 6     /* call out of order (e.g. lbm_step before any initialisation)       */
} lbm_status;

/* Curved-wall scheme applied at every boundary link (Sec. 2.2 and Sec. 4.1). */
typedef enum {
  LBM_HBB = 0,        /* halfway bounce-back: f_abar(x_b, t+1) = f*_a(x_b, t)              */
  LBM_FH = 1,         /* Filippova-Haenel, Eqs. (7)-(10); rejected when |tau - 1| < 1e-3   */
  LBM_MLS = 2,        /* Mei-Luo-Shyy, Eqs. (7), (8), (10), (11)                          */
  LBM_BOUZIDI_L = 3,  /* linear interpolated bounce-back, Eq. (12)                        */
  LBM_BOUZIDI_Q = 4,  /* quadratic interpolated bounce-back, Eq. (13)                     */
  LBM_ZHAO_YONG = 5,  /* single-node scheme, Eq. (14)                                     */
  LBM_MOD_A = 6,      /* modified scheme A: MLS, then f_0(x_b) += leakage, Eqs. (15)-(18) */
  LBM_MOD_B = 7,      /* modified scheme B: MLS with the fictitious density of Eq. (22)   */
  LBM_BAO = 8,        /* MLS with the fictitious density of Eq. (23) (Bao et al.)         */
  LBM_BOUZIDI_L_A = 9 /* linear Bouzidi, then the rest-population correction of Eq. (18)  */
} lbm_scheme;

/* How populations are stored in device memory.  Arithmetic is FP64 for LBM_FP64 and FP32 for
 * the deviation formats, which store f_a - w_a rho_ref: LBM_FP32_DEV all nine as FP32;
 * LBM_FP16_DEV the rest population f_0 (which does not stream) as FP32 and the eight moving ones
 * as FP16 (20 bytes per node and lattice).  In both the rest population takes the node's stored
 * mass minus the rounded moving populations, so the bulk step keeps mass to FP32 accuracy.  The
 * boundary pass computes the incoming link values in the same arithmetic (FP32 for the deviation
 * formats) and keeps each boundary node's mass balance in FP64: the imbalance between its stored
 * outgoing and incoming values, and the rounding residue of its rest population, carried from
 * step to step, so the mass-conserving schemes stay conserving. */
typedef enum { LBM_FP64 = 0, LBM_FP32_DEV = 1, LBM_FP16_DEV = 2 } lbm_precision;

typedef enum { LBM_EOS_NONE = 0, LBM_EOS_EXP = 1, LBM_EOS_CS = 2 } lbm_eos_kind;

typedef struct {
  double cx, cy, r;      /* centre and radius in lattice units                                  */
  int32_t solid_outside; /* 0: nodes with |x - c| <= r are solid; 1: nodes with |x - c| >= r are  */
  int32_t pad;
} lbm_circle;

/* Solid geometry.  A node is solid if any circle or wall makes it solid.  The wall fraction q of a
 * link (Eq. 6) is the smallest t in (0, 1] at which x_b + t e_a meets a circle whose solid region
 * holds x_s = x_b + e_a, or the wall's q when x_s is a wall row.  Every circle, widened by two
 * nodes, must lie inside the box: links never cross the periodic seam into a circle. */
typedef struct {
  int32_t nx, ny;       /* lattice size, each in [4, 65536], 9*nx*ny < 2^31            */
  int32_t n_circles;    /* number of entries in circles (may be 0)                        */
  int32_t pad;
  const lbm_circle* circles;
  double wall_q_lo;     /* > 0: row 0 is a flat solid wall and its links have this q      */
  double wall_q_hi;     /* > 0: row ny-1 is a flat solid wall and its links have this q   */
} lbm_geometry;

/* Fluid model.  psi(rho) of Eq. (16): LBM_EOS_EXP psi0*exp(-rho0/rho) (Sec. 3.2); LBM_EOS_CS
 * psi = sqrt(2 (p(rho) - rho/3) / G) with the Carnahan-Starling pressure
 * p = rho R T (1 + eta + eta^2 - eta^3)/(1 - eta)^3 - a rho^2, eta = b rho / 4, T = T_over_Tc*T_c;
 * LBM_EOS_NONE: single phase (no interaction force).  Solid nodes take psi(rho_wall), the
 * virtual wall density that sets the contact angle (Sec. 3.2).  Body force density:
 * rho*(gx, gy) plus azim_C / r along e_theta about (azim_cx, azim_cy) when azim_C != 0. */
typedef struct {
  int32_t kind; /* lbm_eos_kind */
  int32_t pad;
  double G;     /* interaction strength; attractive (phase separating) when negative        */
  double psi0, rho0;
  double a, b, R, T_over_Tc;
  double rho_wall;
  double gx, gy;
  double azim_C, azim_cx, azim_cy;
} lbm_eos;

/* Device allocation hook: return device memory of at least `bytes` bytes (256-byte aligned) or
 * NULL.  When no hook is given the library uses cudaMallocAsync/cudaFreeAsync on its stream. */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* user);
typedef void (*lbm_free_fn)(void* ptr, void* user);

typedef struct {
  int32_t precision;   /* lbm_precision, default LBM_FP64                                     */
  int32_t graph_steps; /* time steps per captured CUDA graph in lbm_step; 0 = default (32)    */
  void* stream;        /* cudaStream_t for all work of the context; NULL = legacy default     */
  lbm_alloc_fn alloc;  /* optional device allocation hook (both or neither)                   */
  lbm_free_fn free;
  void* alloc_user;
  double rho_ref;      /* reference density of the deviation formats; <= 0: the smallest       *
                        * initial fluid density, set by lbm_init_fields / lbm_init_droplet.     *
                        * Used rounded to the nearest FP32 value                                */
  int32_t kernel_path; /* step kernel, all with the same results bit for bit:                  *
                        * 0: the fastest measured: for FP32/FP16 deviations with nx % 4 == 0    *
                        *    and ny >= 8 (FP16: 12) the vectorised kernel (population vectors   *
                        *    of 16 B; the two psi-ring rows of tiles away from the x seam staged *
                        *    by tensor copies (TMA), the rest of the halo by cp.async), otherwise *
                        *    the scalar tiles; a copy wait that expires is reported as           *
                        *    LBM_ETIMEOUT by lbm_mass;                                           *
                        * 1: the scalar tile kernel (one node per thread and row);              *
                        * 2: FP32 deviations on lattices with nx % 16 == 0, nx, ny >= 64: a     *
                        *    persistent kernel that stages tiles by TMA; otherwise as 0;         *
                        * 3: the vectorised kernel wherever nx % 4 == 0 (FP64: nx % 2 == 0) and *
                        *    ny >= 8 (FP16: 12), FP64 included, its halo staged by cp.async     *
                        *    only; otherwise the scalar tiles;                                   *
                        * 4: the same as 0                                                       */
  int32_t track_force; /* nonzero: the wall pass records the momentum exchange for lbm_force   *
                        * (also switched on by lbm_set_inflow); off by default, it costs the   *
                        * wall pass a few microseconds per step; ignored by batches            */
} lbm_options;

typedef struct {
  int32_t nx, ny;
  int64_t n_fluid;          /* fluid nodes                                                   */
  int64_t n_boundary_nodes; /* fluid nodes with at least one cut link                        */
  int64_t n_links;          /* cut links                                                     */
  int64_t steps;            /* time steps taken since the last initialisation                */
  int64_t device_bytes;     /* device memory held by the context                             */
  int64_t fallbacks;        /* reserved (always 0)                                           */
  double T;                 /* absolute temperature of the Carnahan-Starling EOS (0 otherwise) */
  double psi_wall;          /* psi(rho_wall)                                                 */
} lbm_info_t;

/* Create a context: validates the arguments, builds on the GPU the solid flags and the list of
 * boundary links with q (Eq. 6) in canonical order (node index, then direction), and allocates
 * two population lattices.  tau > 0.5 is the relaxation time (nu = (tau - 1/2)/3).  `opt` may be
 * NULL.  On success *out receives the context; on failure *out is NULL. */
lbm_status lbm_create(const lbm_geometry* geometry, const lbm_eos* eos, double tau, int32_t scheme,
                      const lbm_options* opt, lbm_ctx** out);

/* Maxwell equal-area coexistence densities of the Carnahan-Starling EOS at eos->T_over_Tc
 * (host computation, no context needed).  LBM_EINVAL unless kind == LBM_EOS_CS and T < T_c. */
lbm_status lbm_coexistence(const lbm_eos* eos, double* rho_l, double* rho_v);

/* Initialise f = f_eq(rho, u) (Eq. 4) at every fluid node from caller-owned host arrays of nx*ny
 * doubles (ux, uy may be NULL for zero).  Blocks until the upload is done. */
lbm_status lbm_init_fields(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy);

/* Initialise a droplet: rho = (rho_in + rho_out)/2 - (rho_in - rho_out)/2 tanh(2 (r - R)/W),
 * r the distance to (cx, cy), u = 0, f = f_eq (computed on the GPU). */
lbm_status lbm_init_droplet(lbm_ctx* ctx, double cx, double cy, double R, double W, double rho_in,
                            double rho_out);

/* Advance n >= 0 time steps, asynchronously on the context's stream (whole graphs of
 * graph_steps steps, the remainder launched one by one). */
lbm_status lbm_step(lbm_ctx* ctx, int32_t n);

/* Advance n >= 1 steps without graphs, recording CUDA events around every kernel on the
 * context's stream; blocks until done and returns the summed milliseconds of the fused step
 * kernel, of the boundary kernel, and from the first event to the last.  Any pointer may be NULL. */
lbm_status lbm_step_timed(lbm_ctx* ctx, int32_t n, double* ms_step_kernel, double* ms_boundary,
                          double* ms_total);

/* Total mass sum over fluid nodes and directions of f (FP64, fixed summation order, so repeated
 * calls on the same state agree bit for bit).  Blocks.  Returns LBM_EUNSTABLE (sticky) when a
 * fluid density is not finite or not positive. */
lbm_status lbm_mass(lbm_ctx* ctx, double* out);

/* Density and velocity (Eq. 5, with the half-force term) of every node into caller-owned host
 * arrays of nx*ny doubles; solid nodes get NaN.  Blocks. */
lbm_status lbm_fields(lbm_ctx* ctx, double* rho, double* ux, double* uy);

/* The same into device arrays of nx*ny doubles, asynchronously on the context's stream. */
lbm_status lbm_fields_device(lbm_ctx* ctx, double* rho, double* ux, double* uy);

/* Node flags into a caller-owned host array of nx*ny bytes: bit 0 solid, bit 1 boundary node
 * (fluid with at least one cut link).  Blocks. */
lbm_status lbm_flags(lbm_ctx* ctx, uint8_t* flags);

/* Boundary links in canonical order.  *n_inout holds the capacity of the three arrays on entry
 * and the number of links on return; arrays may be NULL to query the count only.  LBM_EINVAL if
 * the capacity is too small (the count is still returned).  Blocks. */
lbm_status lbm_links(lbm_ctx* ctx, int32_t* node, uint8_t* dir, double* q, int64_t* n_inout);

/* Sizes and counters of the context (nodes, fluid nodes, boundary nodes, cut links, steps since
 * the last initialisation, device bytes held, the absolute temperature of a Carnahan-Starling
 * fluid, psi of the virtual wall density).  Host-only; never blocks and works on a context in
 * error. */
lbm_status lbm_info(lbm_ctx* ctx, lbm_info_t* out);

/* Channel flow past solid bodies (Sec. 4.2, steady flow past a circular cylinder): from the next
 * step on (and with the force recorded for lbm_force), column i = 0 is a velocity inlet with
 * the uniform profile (u_in, 0) imposed by Zou and
 * He's rule for the three populations entering from the left, and column i = nx - 1 is a
 * fully developed outlet (the three populations entering from the right are those of column
 * nx - 2).  y stays periodic.  Single-phase flows only (eos kind LBM_EOS_NONE: the psi stencil is
 * not defined at an open end); |u_in| < 0.5; nx >= 3.  Takes effect for lbm_step, lbm_step_timed
 * and later graphs; there is no call to return to a periodic x. */
lbm_status lbm_set_inflow(lbm_ctx* ctx, double u_in);

/* Force on all solid nodes during the last time step by momentum exchange (Sec. 4.2, after Mei
 * et al. 2002): the sum over cut links of e_a (f*_a(x_b, t) + f_abar(x_b, t+1)), the incoming
 * value being the one the curved-wall scheme wrote, in lattice units (momentum per step).
 * FP64, per boundary node in a fixed lane order, then over boundary nodes in ascending order on
 * the host.  Blocks.  0 before the first recorded step and when there are no cut links.
 * LBM_ESTATE unless the context records the force (lbm_options.track_force or
 * lbm_set_inflow).  The drag coefficient of Sec. 4.2 is fx / (0.5 rho U0^2 D). */
lbm_status lbm_force(lbm_ctx* ctx, double* fx, double* fy);

/* ---- Checkpoint and resume ------------------------------------------------------------------
 * (No counterpart in the paper: a server preempts lattices and resumes them later.)  A state
 * blob holds everything the later steps of a lattice depend on: a header naming the lattice
 * (nx, ny, precision, scheme, EOS kind, tau), the step count, rho_ref, the channel settings of
 * lbm_set_inflow, then the current populations in the storage format (lattice layout, one
 * lattice) and the FP64 rounding carry of each boundary node (zeros for FP64 storage).
 * Restored into a context created with the same arguments, the run continues bit for bit. */
/* Size in bytes of the state blob of this context. */
lbm_status lbm_state_bytes(const lbm_ctx* ctx, int64_t* bytes);
/* Write the state into the caller-owned host buffer of `bytes` bytes (at least
 * lbm_state_bytes).  Blocks.  LBM_ESTATE before the first initialisation, LBM_EINVAL for a short
 * buffer. */
lbm_status lbm_save_state(lbm_ctx* ctx, void* buf, int64_t bytes);
/* Replace the context's state (populations, carry, step count, rho_ref, channel settings) by a
 * blob from lbm_save_state.  Blocks.  LBM_EINVAL when the blob is short, not a state blob, or
 * names another lattice (size, precision, scheme, EOS kind, tau); LBM_ESTATE for a lattice that
 * belongs to a batch (its state lives in the batch's tables). */
lbm_status lbm_load_state(lbm_ctx* ctx, const void* buf, int64_t bytes);

/* Self-test of the bounded device waits (those of the TMA-staged step kernel, which give up
 * after a time limit and report LBM_ETIMEOUT instead of hanging): one CTA waits on an mbarrier
 * phase for at most limit_ns nanoseconds (1 .. 1e10).  complete != 0: an arrival completes the
 * phase first; the call returns LBM_OK with *completed = 1.  complete = 0: nothing completes
 * it, the wait gives up after limit_ns; the call returns LBM_ETIMEOUT with *completed = 0.  The
 * device stays usable either way.  stream: a cudaStream_t or NULL.  Blocks.  Needs no context;
 * LBM_EINVAL for a limit out of range. */
lbm_status lbm_selftest_bounded_wait(int64_t limit_ns, int32_t complete, void* stream,
                                     int32_t* completed);

/* Throughput of the GPU's FP64 fused multiply-add pipe, measured (measurement support; the
 * paper has no counterpart: the FP64 step of the method is bound by this pipe on GB300, and its
 * roofline needs the pipe's rate).  One untimed and one timed launch of a kernel that fills the
 * GPU with one wave of resident blocks, each thread running 8 independent chains of iters
 * dependent FP64 FMAs; CUDA events on `stream` (cudaStream_t or NULL) around the timed launch.
 *   iters    FMAs per chain, 1 .. 2^24 (about 1e5 gives a launch of tens of milliseconds)
 *   gflops   receives 2 x FMAs / time in GFLOP/s      ms  receives the timed launch in ms
 * Blocks until done.  LBM_EINVAL for bad arguments, LBM_ECUDA if a CUDA call fails. */
lbm_status lbm_probe_fp64_fma(int32_t iters, void* stream, double* gflops, double* ms);

/* Total mass of caller-owned device arrays without allocating any memory.  (This entry point
 * has no counterpart in the paper; it serves callers that cannot allocate device memory: a host
 * framework that already holds the device memory in its own pool, or a latency-critical loop
 * that must not call cudaMalloc, which may synchronise the whole device.)
 *   f           device array of 9*nx*ny populations [a][j][i]: FP64 values for LBM_FP64, FP32
 *               values f_a - w_a rho_ref for LBM_FP32_DEV (the layout of this library);
 *               LBM_FP16_DEV is not accepted
 *   flags       device array of nx*ny bytes, bit 0 = solid (skipped); NULL: every node is fluid
 *   mass_out    device pointer: receives sum over fluid nodes of sum_a f_a (FP64, fixed order)
 *   status_out  device pointer: receives LBM_OK, or LBM_EUNSTABLE if a fluid density is not
 *               finite or not positive
 *   stream      cudaStream_t the two kernels run on (asynchronously); NULL = legacy stream
 * The reduction's scratch is a fixed device array of 2 x 8192 doubles (128 KiB) inside the
 * library, held by every GPU that loads the library until the process exits; hence at most
 * 8192 x 8192 = 67,108,864 nodes (larger lattices return LBM_EINVAL).  All calls on a device share
 * that array: calls whose kernels overlap on the GPU race and give wrong results, so serialise
 * them (e.g. one stream).  The first call on a device looks up the array's device address (no
 * allocation) and should come before any stream capture; the address is kept for the life of
 * the process, so resetting the device (cudaDeviceReset) after that first call is not supported:
 * the next call would launch with the old address.  Returns LBM_EINVAL for bad arguments,
 * LBM_ECUDA if a launch fails; the mass and status arrive on the stream. */
lbm_status lbm_mass_noalloc(const void* f, const uint8_t* flags, int32_t nx, int32_t ny,
                            int32_t precision, double rho_ref, double* mass_out,
                            int32_t* status_out, void* stream);

/* ---- Batches: many lattices advanced together -------------------------------------------------
 * (No counterpart in the paper, which advances one lattice at a time: batches serve many
 * independent lattices of different sizes, step budgets and parameters at once, for throughput
 * and for the serving loop of paper_1908_09235_gb300/serve.py.)
 * A batch holds up to max_domains lattices of one precision and one EOS kind.  One batch step is
 * three kernel launches for all of them (a persistent step kernel over a queue of tiles, a
 * persistent boundary kernel over all boundary nodes, and a kernel that advances each lattice's
 * state), replayed from a CUDA graph; lattices join and leave between steps and each stops at its
 * own step budget.  A lattice gives the same bits alone (lbm_step) and inside any batch. */
typedef struct lbm_batch lbm_batch;

typedef struct {
  lbm_geometry geometry;
  lbm_eos eos;
  double tau;
  int32_t scheme;   /* lbm_scheme */
  int32_t init;     /* 1: droplet (cx, cy, R, W, rho_in, rho_out); 0: rho = rho_in, u = 0 */
  double cx, cy, R, W, rho_in, rho_out;
} lbm_domain;

/* How the CTAs of a batch's persistent step kernel work through its queue of tiles.  The
 * tiles of one lattice stand together, row by row; results are the same bits under every
 * schedule and tile height (only the order of independent tiles changes). */
typedef enum {
  LBM_SCHED_STRIDED = 0,              /* CTA k takes tiles k, k + G, k + 2G, ... (G CTAs);
                                         lattices in slot order                            */
  LBM_SCHED_CLAIM = 1,                /* CTAs claim the next tile from a device counter;
                                         lattices in slot order                            */
  LBM_SCHED_CLAIM_LARGEST_FIRST = 2   /* CTAs claim tiles; lattices by tile count, largest
                                         first (ties in slot order)                        */
} lbm_schedule;

typedef struct {
  int32_t active;          /* lattices in the batch                                         */
  int32_t tiles;           /* tiles in the current table (-1 before the first step)         */
  int32_t tile_rows, tile_cols;
  int64_t nodes, fluid_nodes, boundary_links;
  int64_t device_bytes;    /* device memory of the batch and its lattices                   */
  int32_t schedule;        /* lbm_schedule of the tile queue                                */
  int32_t pad;
} lbm_batch_info_t;

/* One candidate timed by lbm_batch_tune: tile height, schedule, mean step-kernel time. */
typedef struct {
  int32_t tile_rows;
  int32_t schedule;
  double ms;
} lbm_tune_trial;

/* opt: stream and allocation hook for the batch and every lattice in it (precision is taken
 * from the argument).  Starts with 32-row tiles (FP64: 16) and LBM_SCHED_CLAIM
 * (lbm_batch_tune, lbm_batch_set_schedule change them).  LBM_EINVAL for bad arguments. */
lbm_status lbm_batch_create(int32_t precision, int32_t eos_kind, int32_t max_domains,
                            const lbm_options* opt, lbm_batch** out);
/* Create, initialise and add a lattice with a budget of `steps` time steps; *slot receives its
 * index.  LBM_ENOMEM when no slot or no device memory is free (nothing is added), LBM_EINVAL
 * when d->eos.kind differs from the batch's. */
lbm_status lbm_batch_add(lbm_batch* b, const lbm_domain* d, int64_t steps, int32_t* slot);
lbm_status lbm_batch_remove(lbm_batch* b, int32_t slot);          /* frees its memory */
lbm_status lbm_batch_set_steps(lbm_batch* b, int32_t slot, int64_t steps); /* new budget */
/* Advance every lattice by n steps or until its budget is spent (asynchronous). */
lbm_status lbm_batch_step(lbm_batch* b, int32_t n);
/* As lbm_batch_step without graphs, with CUDA events around each kernel; blocks and returns
 * the total time and the summed times of the step kernel and of boundary + advance kernels. */
lbm_status lbm_batch_step_timed(lbm_batch* b, int32_t n, double* ms_total, double* ms_step_kernel,
                                double* ms_boundary);
/* Steps done and left of a lattice (blocks). */
lbm_status lbm_batch_progress(lbm_batch* b, int32_t slot, int64_t* steps_done,
                              int64_t* steps_left);
/* Steps left of slots 0..n-1 in one call (-1 for an empty slot); blocks. */
lbm_status lbm_batch_poll(lbm_batch* b, int32_t n, int64_t* steps_left);
/* The lattice's context, current as of this call, for lbm_mass, lbm_fields, lbm_info (blocks).
 * It stays owned by the batch; do not step or destroy it directly. */
lbm_status lbm_batch_domain(lbm_batch* b, int32_t slot, lbm_ctx** ctx);
/* Time the step kernel (mean of trial_steps launches after two warm-up launches) for each tile
 * height (8, 16, 32 rows; FP64: 8, 16) under each lbm_schedule on the current batch, without
 * changing any lattice's state, and keep the fastest pair; *tile_rows receives its height and
 * lbm_batch_info its schedule.  LBM_EINVAL for trial_steps < 1. */
lbm_status lbm_batch_tune(lbm_batch* b, int32_t trial_steps, int32_t* tile_rows);
/* The candidates of the last lbm_batch_tune in the order timed: up to max into out, their
 * number into *n (0 before any tuning). */
lbm_status lbm_batch_tune_trials(const lbm_batch* b, int32_t max, lbm_tune_trial* out,
                                 int32_t* n);
/* Set the tile height (8, 16, 32; FP64: 8, 16) and schedule by hand (takes effect at the next
 * step; a captured graph is dropped).  LBM_EINVAL for other values. */
lbm_status lbm_batch_set_schedule(lbm_batch* b, int32_t tile_rows, int32_t schedule);
lbm_status lbm_batch_info(lbm_batch* b, lbm_batch_info_t* out);
/* Device bytes a lattice would need in a batch of the given precision (upper estimate). */
lbm_status lbm_domain_bytes(const lbm_domain* d, int32_t precision, int64_t* bytes);
const char* lbm_batch_last_error(const lbm_batch* b);
void lbm_batch_destroy(lbm_batch* b);

/* Message of the sticky error, or "" when there is none.  Valid until the next call. */
const char* lbm_last_error(const lbm_ctx* ctx);
const char* lbm_status_string(lbm_status s);

/* Release device memory and the context (NULL is ignored).  Synchronises the stream. */
void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
