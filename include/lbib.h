/*
 * lbib — C ABI of the coupled lattice-Boltzmann / immersed-boundary time step
 * for three-bead microswimmers (Geyer et al., "Lattice Boltzmann Simulations
 * of Two Linear Microswimmers Using the Immersed Boundary Method",
 * arXiv 2202.12147), implemented as CUDA kernels for sm_103a.
 *
 * One coupled step (Sec. 2, in this order):
 *   1. bead centres R_b = mean of the bead's mesh nodes        (Fig. 1 caption)
 *   2. drive f^d(t) and spring forces f^s(R) per swimmer       (Sec. 2.2)
 *   3. membrane forces f^part = -dW/dr on each node (linear FEM) (Sec. 2.2)
 *      and f^tot = f^part + (f^d + f^s)/N_v                    (Sec. 2.2)
 *   4. force spreading F(x) = sum_j f^tot_j Delta(x - r_j)     (Sec. 2.3, Eq. spreading)
 *   5. D3Q19 BGK collide with body force, then stream           (Sec. 2.1, Eqs. lbe, lbm:equilibrium)
 *   6. velocity interpolation rdot_j = sum_x u(x) Delta(x-r_j) (Sec. 2.3, Eq. interpolation)
 *   7. front tracking r_j += rdot_j (dt = 1)                   (Sec. 2.3)
 *
 * Conventions shared by every call:
 *   - Every function returns an int status: LBIB_OK (0) or a negative code.
 *     Nothing aborts or throws across this boundary.  lbib_last_error() gives
 *     a message for the most recent failure on the calling thread.
 *   - Lattice nodes sit at integer coordinates 0..n-1 of a periodic box,
 *     cell index = x + nx*(y + ny*z).  Lagrangian node coordinates are
 *     unwrapped doubles (they may leave [0, n)).
 *   - Large device buffers are owned by the caller (allocate them with the
 *     sizes from lbib_required_sizes), borrowed by the context and must
 *     outlive it.  The context owns only host metadata, a private capture
 *     stream, CUDA graphs and a small pinned host block.
 *   - Work is queued on the stream given to lb_init.  Calls are asynchronous
 *     unless stated otherwise; device-side errors (non-finite values, unstable
 *     node speeds) are latched in device memory and reported by the next
 *     synchronising call (swimmer_state, lb_sync, the lb_get_* calls).
 */
#ifndef LBIB_H
#define LBIB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LBIB_OK 0
#define LBIB_EINVAL -1     /* invalid argument, detected before any launch */
#define LBIB_ECUDA -2      /* a CUDA runtime call failed */
#define LBIB_ENONFINITE -3 /* a density, velocity or node position became NaN/Inf */
#define LBIB_EUNSTABLE -4  /* a node moved faster than 0.1 lattice units per step */
#define LBIB_ETIMEOUT -5   /* a bounded device-side wait gave up */
#define LBIB_ESIZE -6      /* a buffer is too small or a size exceeds a limit */

/* ---- options ----------------------------------------------------------- */
/* Population storage.  Every format stores the shifted deviation
 * d_i = f_i - w_i rho0 (F32 as is; F16/BF16 as d_i / w_i * store_scale);
 * collisions always run in FP32. */
#define LBIB_F32 0
#define LBIB_F16 1
#define LBIB_BF16 2
/* Body-force inclusion: Guo's source term, or the paper's Shan-Chen velocity
 * shift rho u^eq = sum f c + tau F (Sec. 2.1, Eq. sc). */
#define LBIB_GUO 0
#define LBIB_SHAN_CHEN 1
/* Discrete delta kernel (Sec. 2.3): Peskin's 4-point kernel (4^3 stencil) or
 * the paper's 2-point linear kernel (2^3 stencil). */
#define LBIB_PESKIN4 0
#define LBIB_LINEAR2 1

/* Fluid box.  tau > 1/2 is the BGK relaxation time (viscosity
 * nu = (tau - 1/2)/3, Sec. 2.1); rho0 the rest density; g a uniform
 * force density added in every cell (zero for swimmer runs).
 * deterministic = 1 makes spreading bitwise reproducible run to run
 * (fixed-point integer accumulation instead of float atomics).
 * store_scale: scale S of the F16/BF16 formats, 0 selects 4096. */
typedef struct {
    int nx, ny, nz;
    double tau;
    double rho0;
    int storage;
    int forcing;
    int kernel;
    int deterministic;
    double g[3];
    double store_scale;
} lb_params;

/* One bead: its mesh nodes [node_start, node_start + node_count) and
 * triangles [tri_start, tri_start + tri_count) of the structure arrays, and
 * its membrane (Sec. 2.2):
 *   law = LBIB_NEOHOOKE: strain energy Gs/2 (I1 - 1 + 1/(I2 + 1)) per
 *         reference area (Gs the small-strain shear modulus);
 *   law = LBIB_SKALAK:   Gs/4 (I1^2 + 2 I1 - 2 I2 + C I2^2) (Gs = kappa_s,
 *         kappa_a / kappa_s = 1 + 2 C);
 *   kb >= 0: bending modulus of the Helfrich energy, discretised per edge
 *         after Kantor and Nelson as 2 sqrt(3) kb (1 - cos(theta - theta0)),
 *         theta the angle between the normals of the edge's two triangles
 *         and theta0 its value in the rest shape (needs a closed surface:
 *         every edge on exactly two triangles of the bead);
 *   kv >= 0: volume penalty kv/2 (V - V0)^2 / V0 (Eq. vol_cons), V0 the
 *         enclosed volume of the rest shape (closed, outward surface).
 * Zero kb or kv switches the term off. */
#define LBIB_NEOHOOKE 0
#define LBIB_SKALAK 1
typedef struct {
    int node_start, node_count;
    int tri_start, tri_count;
    double Gs;
    int law;
    double C;
    double kb;
    double kv;
} lbib_bead;

/* One three-bead swimmer (Sec. 2.2).  bead[0..2] index the bead table in
 * swimming-axis order.  Springs: stiffness k_spring, rest length L_spring.
 * Drive along x on bead b: amp[b] sin(2 pi t / period + phase[b]); with
 * balance = 1 the middle bead instead carries -(f_0 + f_2), the paper's
 * protocol (f1 = A sin(wt), f3 = B sin(wt + alpha), f2 = -f1 - f3). */
typedef struct {
    int bead[3];
    double k_spring, L_spring;
    double amp[3], phase[3];
    int balance;
    double period;
} lbib_swimmer;

/* The Lagrangian structure.  All pointers are HOST memory, read during
 * lb_init only.  rest_nodes (n_nodes x 3, row-major) is both the
 * stress-free membrane shape and the initial node positions; tris
 * (n_tris x 3) are global node ids, counter-clockwise seen from outside. */
typedef struct {
    int n_beads, n_swimmers, n_nodes, n_tris;
    const lbib_bead *beads;
    const lbib_swimmer *swimmers;
    const double *rest_nodes;
    const int *tris;
} lbib_structure;

/* Caller-owned device buffers (each 256-byte aligned) of at least the sizes
 * lbib_required_sizes returns, in this order. */
#define LBIB_NBUF 3
typedef struct {
    void *pops;   /* populations: 19 planes of the padded cell count */
    void *fields; /* force density F and velocity u per cell, tile flags */
    void *aux;    /* node positions, node forces/velocities, mesh tables, control block */
} lbib_buffers;

/* Observables of one swimmer (Sec. 3, Eq. vel_swim; the Reynolds numbers of
 * Sec. 3 with nu = (tau - 1/2)/3 and a the bead's rest radius).  All FP64.
 * Period boundaries are the steps where floor(t / period) increases; x_cm is
 * recorded there on the device. */
typedef struct {
    long long step;        /* time steps taken since lb_init */
    double R[3][3];        /* bead centres, unwrapped */
    double V[3][3];        /* bead velocities: mean interpolated node velocity of the last step */
    double F[3][3];        /* sum of the total nodal forces of each bead at the last force evaluation */
    double T[3][3];        /* torque of those forces about each bead centre */
    double x_cm[3];        /* mean of the three bead centres */
    double disp[3];        /* x_cm minus x_cm at lb_init */
    long long periods;     /* drive periods completed since lb_init */
    double v_period[3];    /* mean swimming velocity over the last completed period,
                              (x_cm(kT) - x_cm((k-1)T)) / T (Sec. 3, Eq. vel_swim);
                              zero before the first period ends */
    double re_swim;        /* |v_period| L_swim / nu, L_swim = outer bead distance + 2a */
    double re_bead;        /* max_b |V_b| a / nu (bead velocities of the last step) */
} lbib_swimmer_state;

typedef struct lbib_ctx lbib_ctx;

/* Version string of the library. */
const char *lbib_version(void);
/* Message for a status code. */
const char *lbib_strerror(int status);
/* Message of the most recent failure on the calling thread. */
const char *lbib_last_error(void);

/* The library's D3Q19 velocity set (Sec. 2.1): c[19][3] and w[19], in the
 * order the population planes are stored.  Opposite directions are adjacent
 * (i, i+1 for odd i). */
int lbib_lattice(int *c, double *w);

/* Byte sizes of the three caller buffers for this box and structure.
 * out_bytes[LBIB_NBUF].  structure may be NULL (no swimmers). */
int lbib_required_sizes(const lb_params *p, const lbib_structure *s, size_t *out_bytes);

/* Create a context over caller buffers.  Uploads the mesh tables (reference
 * metrics per triangle, node-to-triangle lists), sets every population to
 * rest (f_i = w_i rho0, Sec. 2.1 with u = 0), places the nodes at rest_nodes
 * and captures the CUDA graphs of the step.  stream: a cudaStream_t (NULL =
 * legacy default stream).  Synchronous.  *out receives the context. */
int lb_init(const lb_params *p, const lbib_structure *s, const lbib_buffers *b, void *stream, lbib_ctx **out);

/* Advance n_steps full coupled steps (1-7 above) asynchronously on the
 * context stream, replaying the captured 16-step CUDA graph from even steps
 * and launching the kernels of the remaining single steps directly (faster
 * than a one-step graph replay).  The environment variable LBIB_GRAPHS=0
 * launches every step's kernels directly; the results are the same either
 * way. */
int lb_step(lbib_ctx *ctx, long long n_steps);

/* Steps 1-4 alone at the current positions and time: evaluate f^tot on every
 * node and add its spread into the force field F; the next lb_step applies
 * and clears F.  For tests and custom coupling. */
int ib_spread(lbib_ctx *ctx);

/* Step 6 alone: interpolate the velocity field u held in the fields buffer
 * at the current node positions, without moving the nodes.  node_vel_out is
 * a DEVICE pointer to n_nodes x 3 floats.  (lb_step writes u only in the
 * tiles around the nodes; lb_set_velocity fills it everywhere.) */
int ib_interpolate(lbib_ctx *ctx, float *node_vel_out);

/* Copy one swimmer's observables to host memory.  Synchronises the context
 * stream and reports latched device errors. */
int swimmer_state(lbib_ctx *ctx, int swimmer, lbib_swimmer_state *out);
/* Asynchronous form: queues the evaluation of every swimmer's observables and
 * a copy of the n_swimmers records into HOST memory `out` on the context
 * stream, and returns.  The records are valid after the next synchronising
 * call (lb_sync); `out` should be page-locked for the copy to overlap the
 * following steps, and must not be reused before then.  Device errors
 * surface at that synchronising call. */
int swimmer_state_async(lbib_ctx *ctx, lbib_swimmer_state *out);

/* Trajectory of one swimmer at one step, written on the device by every
 * coupled step (the last block of step 7, after the bead centres have moved
 * with the mean velocity of their nodes, Fig. 1 caption).  FP64. */
typedef struct {
    long long step;     /* steps taken since lb_init once this step completed */
    double x_cm[3];     /* mean of the three bead centres */
    double R[3][3];     /* bead centres, unwrapped */
    double V[3][3];     /* mean interpolated node velocity of each bead in this step */
} lbib_track_point;

/* Steps of trajectory points a context keeps on the device (a ring). */
#define LBIB_TRACK_STEPS 256

/* Queue a copy of the trajectory points of the last n_steps completed steps
 * into HOST memory out[n_steps][n_swimmers] (oldest step first) on the stream
 * that advances the context (its own, or its batch's), and return.
 * 1 <= n_steps <= LBIB_TRACK_STEPS and n_steps <= the steps taken since
 * lb_init (else LBIB_EINVAL, nothing queued).  Like swimmer_state_async, the
 * points are valid after the next synchronising call; `out` should be
 * page-locked.  The ring is part of the checkpoint, so points written before
 * lb_checkpoint survive lb_restore. */
int lb_track(lbib_ctx *ctx, long long n_steps, lbib_track_point *out);

/* Wait for queued work and report latched device errors. */
int lb_sync(lbib_ctx *ctx);

/* Density and momentum velocity u = sum f c / rho (no force term) of the
 * current populations into DEVICE arrays rho[n_cells], u[n_cells x 3]. */
int lb_get_macros(lbib_ctx *ctx, float *rho, float *u);

/* Current populations as raw f_i (not deviations), HOST array [19][n_cells]
 * in lbib_lattice order, FP64.  Synchronous. */
int lb_get_populations(lbib_ctx *ctx, double *host_f);
/* Replace the populations with raw f_i from HOST [19][n_cells] FP64. */
int lb_set_populations(lbib_ctx *ctx, const double *host_f);

/* Node positions as HOST n_nodes x 3 FP64 (get is synchronous). */
int lb_get_nodes(lbib_ctx *ctx, double *host_xyz);
int lb_set_nodes(lbib_ctx *ctx, const double *host_xyz);

/* Total nodal forces f^tot of the last force evaluation, HOST n_nodes x 3. */
int ib_get_node_forces(lbib_ctx *ctx, float *host_f);
/* The force field F currently accumulated, HOST n_cells x 3. */
int lb_get_force_field(lbib_ctx *ctx, float *host_F);
/* Overwrite the velocity field u with HOST n_cells x 3 values. */
int lb_set_velocity(lbib_ctx *ctx, const float *host_u);

/* Timing hook.  With on = 1, every launch of the main fluid kernel (the
 * update of every tile no node stencil touches) is bracketed by a pair of
 * CUDA events on the context stream: lb_step replays a 16-step graph captured
 * with an event-record node before and after each main-kernel launch (fresh
 * events for every replay), and launches single steps one by one; with on =
 * 0 (the default) it replays the plain graphs.  Switching on captures that
 * graph the first time (LBIB_GRAPHS=0: launches one by one throughout) and
 * discards earlier measurements. */
int lb_profile(lbib_ctx *ctx, int on);
/* Sum of the bracketed fluid-kernel durations in milliseconds and the
 * number of launches measured since profiling was switched on.
 * Synchronises the context stream. */
int lb_profile_read(lbib_ctx *ctx, double *total_ms, long long *launches);

/* Deterministic force spreading that allocates nothing.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory themselves -- code inside a framework whose caching
 * allocator owns all device memory (a cudaMalloc there competes with it and
 * can fail), or a loop that must keep its memory footprint fixed after
 * start-up.  It needs no context and no caller scratch.
 *
 * Computes F(x) = sum_j f_j Delta(x - r_j) on a periodic nx x ny x nz box
 * with the same fixed-point accumulation as a
 * deterministic context, so the result is bitwise reproducible and equals
 * the force field ib_spread produces for the same positions and forces.
 *   nodes        DEVICE, n_nodes x 3 FP64 unwrapped positions (row-major)
 *   node_forces  DEVICE, n_nodes x 3 FP32 nodal forces
 *   kernel       LBIB_PESKIN4 or LBIB_LINEAR2
 *   F_out        DEVICE, n_cells x 3 FP32, cell = x + nx*(y + ny*z); every
 *                entry is written
 *   stream       cudaStream_t the work is queued on (asynchronous)
 * The accumulation grid is a static device array inside this library holding
 * at most 262144 cells (64^3; 6 MiB, kept by every GPU that loads the library
 * until the process exits); larger boxes are rejected with LBIB_ESIZE before
 * anything is launched.  The first call on each device looks up the array's
 * device address (with that device current) and caches it: make that first
 * call before any stream capture.  Every call clears the part of the array it
 * uses, then accumulates into it, so calls whose work overlaps on the GPU (on
 * different streams, or on two host threads) race and corrupt each other's
 * results; serialise them.  No cudaMalloc, cudaFree or allocating library
 * routine is called. */
int ib_spread_fixed_noalloc(const double *nodes, const float *node_forces, int n_nodes, int nx, int ny, int nz,
                            int kernel, float *F_out, void *stream);

/* Number of cells in the fluid tiles marked for the next step (the tiles the
 * delta-kernel stencils of the current node positions touch; they are updated
 * with the force field by the immersed-boundary stream, every other cell by
 * the main fluid kernel).  Synchronous. */
int lb_marked_cells(lbib_ctx *ctx, long long *cells);

/* ---- batches of independent boxes -------------------------------------
 * A batch advances many contexts (each its own periodic box with its own
 * swimmers, as in the single-box problem of Sec. 2) with one set of kernel
 * launches per step for all of them: every launch covers the tiles, nodes or
 * triangles of every box, on the same two-stream schedule as lb_step, and
 * the step sequence is captured in CUDA graphs.  The contexts keep their own
 * buffers and accessors (swimmer_state, lb_get_*). */
typedef struct lbib_batch lbib_batch;

/* Group n contexts.  They must share storage, forcing, delta kernel and the
 * deterministic flag, have taken the same number of steps, and use the same
 * stream (the batch works on the stream of ctxs[0]); n <= 1024.  The contexts
 * must outlive the batch, and lb_step on a batched context fails with
 * LBIB_EINVAL until the batch is destroyed.  Synchronous. */
int lb_batch_create(lbib_ctx *const *ctxs, int n, lbib_batch **out);
/* Advance every box of the batch by n_steps coupled steps (asynchronous). */
int lb_batch_step(lbib_batch *b, long long n_steps);
/* Timing hook of the batch, as lb_profile / lb_profile_read: brackets every
 * batched main fluid launch with CUDA events. */
int lb_batch_profile(lbib_batch *b, int on);
int lb_batch_profile_read(lbib_batch *b, double *total_ms, long long *launches);
/* Launch-shape autotuner of a batch.  The main fluid update of every box-size
 * class can run one, two or four adjacent cells per thread (four for 16-bit
 * storage only; the count must divide the row length), which sets its block
 * shape; the marked-tile launch walks its flat work list with a grid of
 * blocks whose size trades load balance for launch width.  lb_batch_autotune
 * times real steps of the batch with CUDA events: first `steps_per_trial`
 * steps (rounded up to an even number, >= 2) per cells-per-thread candidate,
 * timing each class's launches, then as many per marked-grid candidate,
 * timing whole steps; it keeps the fastest choice of each, re-captures the
 * batch's CUDA graph and fills `report` (may be NULL).  The tuning steps are
 * ordinary steps of every box (the candidates differ in launch shape only),
 * so the batch advances by report->steps_taken steps.  Synchronous. */
#define LBIB_TUNE_MAX_CLASSES 32
typedef struct {
    int n_classes;                                /* box-size classes (first 32 reported) */
    int class_dims[LBIB_TUNE_MAX_CLASSES][3];     /* nx, ny, nz of the class */
    int class_boxes[LBIB_TUNE_MAX_CLASSES];       /* boxes in the class */
    int class_cells_per_thread[LBIB_TUNE_MAX_CLASSES]; /* chosen */
    double class_us[LBIB_TUNE_MAX_CLASSES][3];    /* mean main-fluid launch time for 1, 2, 4 cells per
                                                     thread, microseconds (0: not a candidate) */
    int marked_candidates[4];                     /* marked-tile grid sizes tried */
    double marked_step_us[4];                     /* mean step time for each, microseconds */
    int marked_blocks;                            /* chosen */
    long long steps_taken;                        /* steps the tuning advanced the batch by */
} lbib_batch_tuning;
int lb_batch_autotune(lbib_batch *b, int steps_per_trial, lbib_batch_tuning *report);
/* Release the batch (not the contexts).  Synchronises. */
int lb_batch_destroy(lbib_batch *b);

/* ---- checkpoint / resume ----------------------------------------------
 * A checkpoint is a versioned binary blob: a header (format version, box,
 * storage, forcing and kernel, determinism flag, structure counts, buffer
 * sizes, step, a 64-bit checksum of the payload) followed by the context's
 * three device buffers as they are (populations in their stored format and
 * AA parity, force/velocity fields and tile stamps, node positions, bead
 * centres, mesh tables, control block, swimmer accumulators).  Restoring it
 * into a context over the same box and structure continues the run exactly:
 * with deterministic spreading, bitwise as if it had never stopped. */
/* Bytes of a checkpoint blob of this context. */
int lb_checkpoint_size(lbib_ctx *ctx, size_t *bytes);
/* Write the blob into HOST memory of at least lb_checkpoint_size bytes.
 * Synchronous; reports a latched device error instead of saving. */
int lb_checkpoint(lbib_ctx *ctx, void *host_buf, size_t bytes);
/* Load a blob written by lb_checkpoint (HOST memory).  LBIB_EINVAL for a
 * blob of another format, box, scheme or structure, or with a checksum
 * mismatch; LBIB_ESIZE if truncated; LBIB_EINVAL while batched.
 * Synchronous. */
int lb_restore(lbib_ctx *ctx, const void *host_buf, size_t bytes);

/* Release the context (not the caller's buffers).  Synchronises.  Fails with
 * LBIB_EINVAL while the context belongs to a batch. */
int lb_destroy(lbib_ctx *ctx);

/* ---- adjoint: gradients with respect to the drive --------------------
 * Reverse-mode derivative of the coupled step (the one of the header comment,
 * Sec. 2.1-2.3) over n_steps steps, for gradients of swimmer displacements
 * x_cm(T) - x_cm(0) (Sec. 3, Eq. vel_swim) with respect to every bead's drive
 * amplitude and phase (Sec. 2.2, driving-force equation, generalised to
 * f_b = A_b sin(2 pi t / period + phi_b) on each bead b).
 *
 * The engine runs its own forward step on a plain layout (two population
 * arrays, push streaming, full per-step records) in FP32 or FP64 fluid
 * precision; node positions, forces and every node-level derivative are
 * FP64.  It keeps a checkpoint (populations + node positions) every K steps
 * and, sweeping backward, recomputes each K-step segment from its checkpoint
 * before reversing it, so memory grows with n_steps / K + K states rather
 * than n_steps.  Full K-step segments replay captured CUDA graphs in both
 * sweeps (LBIB_GRAPHS=0 launches them step by step).  Only Guo forcing and the 4-point kernel (differentiable; the
 * 2-point kernel is not) are supported.  The drive parameter vector of
 * swimmer s is theta[6 s .. 6 s + 5] = (A_1, A_2, A_3, phi_1, phi_2, phi_3)
 * in the order of lbib_swimmer.bead; for a swimmer with balance = 1 the
 * middle bead carries -(f_1 + f_3) and its entries A_2, phi_2 are unused
 * (their gradient is 0). */
#define LBIB_F64 3 /* adjoint engine only: FP64 fluid state */

typedef struct lbib_adjoint lbib_adjoint;

/* Bytes of device workspace an engine needs: params as for lb_init with
 * storage LBIB_F32 or LBIB_F64, forcing LBIB_GUO, kernel LBIB_PESKIN4;
 * n_steps >= 1 steps per sweep; a checkpoint every K >= 1 steps. */
int lb_adjoint_required_bytes(const lb_params *params, const lbib_structure *structure, long long n_steps, int K,
                              size_t *bytes);
/* Create an engine on a caller-owned DEVICE workspace of at least
 * lb_adjoint_required_bytes (256-byte aligned; borrowed, must outlive the
 * engine).  The initial state is the rest state (f_i = w_i rho0, nodes at the
 * rest shape) and theta is taken from the structure's swimmers.  Work is
 * queued on `stream`.  Synchronous. */
int lb_adjoint_create(const lb_params *params, const lbib_structure *structure, long long n_steps, int K,
                      void *workspace, size_t workspace_bytes, void *stream, lbib_adjoint **out);
/* Replace the drive parameters: HOST theta, n_swimmers x 6.  Invalidates the
 * last forward sweep. */
int lb_adjoint_set_drive(lbib_adjoint *a, const double *theta);
/* Replace the initial state: HOST populations f (19 x n_cells, raw f_i in the
 * order of lbib_lattice, cell = x + nx*(y + ny*z)) and/or node positions r
 * (n_nodes x 3); NULL keeps that part.  Invalidates the last forward sweep. */
int lb_adjoint_set_initial(lbib_adjoint *a, const double *f, const double *r);
/* Forward sweep: n_steps coupled steps from the initial state, storing the
 * checkpoints.  disp (HOST, n_swimmers x 3, may be NULL) receives every
 * swimmer's x_cm(T) - x_cm(0).  Synchronous; LBIB_ENONFINITE or
 * LBIB_EUNSTABLE if the run blew up. */
int lb_adjoint_forward(lbib_adjoint *a, double *disp);
/* Reverse sweep of the last forward sweep for the objective
 *   L = sum_s seed_disp[s] . disp_s + <seed_f, f(T)> + <seed_r, r(T)>
 * (HOST seeds: seed_disp n_swimmers x 3, required; seed_f 19 x n_cells and
 * seed_r n_nodes x 3 optional, NULL = 0).  Writes HOST outputs
 * grad_theta (n_swimmers x 6, required) = dL/dtheta and, if not NULL,
 * grad_f0 (19 x n_cells) = dL/df(0) and grad_r0 (n_nodes x 3) = dL/dr(0).
 * Synchronous.  LBIB_EINVAL without a valid forward sweep. */
int lb_adjoint_backward(lbib_adjoint *a, const double *seed_disp, const double *seed_f, const double *seed_r,
                        double *grad_theta, double *grad_f0, double *grad_r0);
/* State after the last forward sweep (HOST, layouts as lb_adjoint_set_initial;
 * either pointer may be NULL).  Synchronous. */
int lb_adjoint_get_final(lbib_adjoint *a, double *f, double *r);
/* Device time of the last forward and backward sweeps, milliseconds (CUDA
 * events on the engine's stream), and the number of kernel launches each
 * made. */
int lb_adjoint_timing(lbib_adjoint *a, double *forward_ms, double *backward_ms, long long *forward_launches,
                      long long *backward_launches);
/* Release the engine (not the workspace).  Synchronises. */
int lb_adjoint_destroy(lbib_adjoint *a);

#ifdef __cplusplus
}
#endif
#endif /* LBIB_H */
