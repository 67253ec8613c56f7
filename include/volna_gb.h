/*
 * volna_gb.h -- C ABI of the GB300 (sm_103a) finite-volume shallow-water step.
 *
 * The library advances the 2D nonlinear shallow water equations
 *     dH/dt + div(H u) = 0,
 *     d(H u)/dt + div(H u (x) u + g H^2 / 2 I) = -g H grad(h)
 * (Giles et al., "Performance analysis of Volna-OP2", Sec. 2.1) on an
 * unstructured triangular mesh with the cell-centred finite-volume scheme of
 * Sec. 2: MUSCL reconstruction with least-squares gradients and the
 * Barth-Jespersen limiter (Sec. 2.4, Eq. recon), skipped below the dry
 * threshold; the HLL flux with the wave speeds of Sec. 2.2 and a hydrostatic
 * wet/dry interface; the wall ghost cell of Sec. 2.5; SSP-RK(2,2) in time
 * with a CFL time step (Sec. 2.3).
 *
 * Conventions
 *  - Every call returns an int status: VG_OK (0) or a negative VG_E* code.
 *    vg_last_error() gives a message for the last failing call on a context.
 *  - Host buffers belong to the caller; the library copies them in or out
 *    before returning.  Device buffers made by the library belong to the
 *    context and are freed by vg_destroy().  *_dev calls take caller-owned
 *    device memory and never free it.
 *  - Cell arrays passed in or out are in the caller's ORIGINAL cell order;
 *    the library renumbers cells internally for locality.
 *  - A context is used by one host thread at a time; contexts are independent
 *    (no global state).
 *  - Work is queued on the context's CUDA stream.  vg_step() and the get
 *    calls synchronise that stream before returning.
 */
#ifndef VOLNA_GB_H
#define VOLNA_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VG_OK 0
#define VG_EINVAL (-1)      /* bad argument, bad mesh, gauge outside the mesh   */
#define VG_ENOMEM (-2)      /* host or device allocation failed                 */
#define VG_ECUDA (-3)       /* a CUDA runtime call failed (message has details) */
#define VG_ENONFINITE (-4)  /* a NaN/Inf appeared in the state or the time step */
#define VG_ENEGDEPTH (-5)   /* negative depth met with params.strict_positivity */
#define VG_ETIMEOUT (-6)    /* a bounded device-side wait gave up                */
#define VG_ESTATE (-7)      /* call out of order (no mesh, no state, ...)        */

#define VG_RENUMBER_NONE 0
#define VG_RENUMBER_MORTON 1
#define VG_RENUMBER_RCM 2
#define VG_RENUMBER_HILBERT 3

/* Boundary kinds (vg_set_boundary). */
#define VG_BOUNDARY_WALL 1
#define VG_BOUNDARY_OPEN 2
#define VG_BOUNDARY_ABSORBING 3

typedef struct vg_ctx vg_ctx;

/* Scheme and run parameters.  Defaults from vg_default_params(). */
typedef struct vg_params {
    double g;              /* gravity (the paper does not state it): 9.81          */
    double cfl;            /* Courant number of the time-step rule: 0.9            */
    double h_threshold;    /* dry threshold H_threshold of Sec. 2.4 (m): 1e-5      */
    double dt_fixed;       /* > 0: fixed time step instead of the CFL rule: 0      */
    double dt_max;         /* > 0: upper clamp of the time step: 0 (none)          */
    double t_end;          /* > 0: the step reaching t_end is shortened to end on
                              it and later steps do not move: 0 (none)             */
    int32_t order;         /* 1 first order, 2 MUSCL (Sec. 2.4): 2                 */
    int32_t gauge_every;   /* record gauges every this many steps: 1               */
    int32_t strict_positivity; /* 1: vg_step fails with VG_ENEGDEPTH when a stage
                              produced a negative depth (otherwise it is emptied
                              and counted): 0                                      */
    int32_t block_cells;   /* cells per thread block of the step kernels
                              (32..512, multiple of 32, at most 256 in a batch;
                              0 = library default 256;
                              halved automatically while the block and its
                              two-ring halo exceed shared memory)                 */
    int32_t block_threads; /* threads per thread block of the step kernels: a
                              multiple of 32 from block_cells to 2 x block_cells
                              and at most 512 (the extra threads share the halo
                              and face work); 0 = block_cells                  */
    int32_t fp64_literal;  /* FP64 contexts and batches: 1 evaluates every formula
                              as written, without multiply-add contraction, so
                              the result equals a plain FP64 implementation of
                              the scheme (the oracle's order) bit for bit; 0 lets
                              the compiler contract multiply-adds and divides
                              once where the literal form divides several times
                              by the same value: about 1.8x faster, rounding
                              differences only, but over long runs with moving
                              shorelines those decide discontinuous switches
                              (a thin film's velocity, hence the CFL step)
                              differently, so trajectories drift apart.  The
                              adjoint always runs the literal form: 1           */
    int32_t rk_unfused;    /* 1: vg_step and vg_advance_to run the SSP-RK(2,2)
                              stage updates (Sec. 2.3) as kernels of their own,
                              with w1 and R(w1) in device memory (two more
                              [3][N] arrays, allocated by vg_set_params or
                              vg_mesh_upload), instead of forming w1 inside the
                              second residual kernel and ending it with the
                              update: the same arithmetic cell by cell, kept
                              to measure what the fusion saves.  Batches, the
                              adjoint and vg_step_noalloc always run fused: 0 */
} vg_params;

/* Run diagnostics (vg_get_diagnostics). */
typedef struct vg_diag {
    double t;              /* simulated time                                      */
    double last_dt;        /* time step of the last step                          */
    double mass;           /* sum_K |K| H_K                                       */
    double min_H;          /* smallest depth                                      */
    int64_t steps;         /* steps taken with dt > 0                              */
    int64_t neg_count;     /* negative depths met (and emptied) so far             */
    int64_t dry_count;     /* cells with H <= H_threshold                          */
    int64_t launches;      /* kernels launched by the library so far               */
    int64_t n_records;     /* gauge records available to vg_get_gauges             */
} vg_diag;

/* Library version (major * 10000 + minor * 100 + patch). */
int vg_version(void);

/* Human-readable name of a status code; static storage. */
const char *vg_strerror(int code);

/* Fill *p with the defaults listed in vg_params. */
int vg_default_params(vg_params *p);

/*
 * Create a context on CUDA device `device` computing in FP32 (precision 32) or
 * FP64 (precision 64).  cuda_stream is a cudaStream_t to queue work on (for
 * example a torch stream), or NULL for a stream owned by the context.
 */
int vg_create(vg_ctx **out, int precision, int device, void *cuda_stream);

/* Free the context and all device memory it owns.  NULL is allowed. */
void vg_destroy(vg_ctx *ctx);

/* Message for the last failing call on ctx; valid until the next call on ctx. */
const char *vg_last_error(vg_ctx *ctx);

/*
 * Upload an unstructured triangular mesh (Sec. 2.2: cell-centred finite volumes
 * on triangles) with per-vertex bathymetry depth h (positive down, z = -h,
 * Sec. 2.1).
 *   xy[nv][2]   vertex coordinates (m), row major
 *   tri[nc][3]  vertex ids per triangle; clockwise triangles are reoriented
 *   depth_v[nv] depth at each vertex; the bed is the piecewise linear bed of
 *               the vertex depths: each cell's bed is the mean of its three,
 *               and each face's bed (under the face values of a cell that
 *               reconstructs, Sec. 2.4) the mean of its two
 *   renumber    VG_RENUMBER_NONE / _MORTON (Z-order of centroids) / _RCM
 *               (reverse Cuthill-McKee on the face graph) / _HILBERT
 *               (Hilbert-curve order of centroids: compact blocks, the
 *               smallest halos of the four)
 * Every edge must belong to one or two triangles; one-triangle edges are walls
 * (Sec. 2.5).  Returns VG_EINVAL for an out-of-range or repeated vertex id, a
 * zero-area triangle or a non-manifold edge.  Replaces any previous mesh and
 * clears the state and gauges.
 */
int vg_mesh_upload(vg_ctx *ctx, int64_t nv, const double *xy, int64_t nc, const int32_t *tri,
                   const double *depth_v, int renumber);

/* new_of_old[nc]: the internal index of each original cell. */
int vg_get_permutation(vg_ctx *ctx, int32_t *new_of_old);

/* Number of clockwise triangles that vg_mesh_upload reoriented. */
int vg_get_flipped(vg_ctx *ctx, int64_t *n_flipped);

int vg_set_params(vg_ctx *ctx, const vg_params *p);
int vg_get_params(vg_ctx *ctx, vg_params *p);

/*
 * Set the conserved state w = (H, Hu, Hv) (Sec. 2.2) at time t from host FP64
 * arrays of nc values in the original cell order (converted to the context's
 * precision).  Depths must be finite and >= 0 (VG_EINVAL otherwise).  Clears
 * the gauge record and, if gauges are set, records eta = H + z at t.
 * Page-locked (pinned) buffers are read in place by the import kernel.
 */
int vg_set_state(vg_ctx *ctx, const double *H, const double *Hu, const double *Hv, double t);

/* Same from device arrays of the context's precision (float or double), in the
   original cell order, read on the context stream. */
int vg_set_state_dev(vg_ctx *ctx, const void *H, const void *Hu, const void *Hv, double t);

/* Copy the state out to host FP64 arrays in the original order; *t may be NULL. */
int vg_get_state(vg_ctx *ctx, double *H, double *Hu, double *Hv, double *t);

/*
 * vg_set_state / vg_get_state with host FP32 arrays (nc values each, original
 * cell order), half the bytes over the CPU-GPU link.  An FP32 context loses
 * nothing by it: vg_get_state_f32 returns exactly the FP32 rounding of what
 * vg_get_state returns (H is formed in FP64 from the stored eta and bed, then
 * rounded once).  An FP64 context widens the inputs and rounds the outputs.
 * Page-locked (pinned) buffers are read or written in place by the import /
 * export kernels; pageable ones go through a device staging copy.  Errors as
 * vg_set_state / vg_get_state.
 */
int vg_set_state_f32(vg_ctx *ctx, const float *H, const float *Hu, const float *Hv, double t);
int vg_get_state_f32(vg_ctx *ctx, float *H, float *Hu, float *Hv, double *t);

/* Copy the state out to device arrays of the context's precision. */
int vg_get_state_dev(vg_ctx *ctx, void *H, void *Hu, void *Hv);

/*
 * Virtual gauges (Sec. 3: free-surface elevation recorded at fixed points):
 * xy[n][2] points, each resolved to the cell containing it (on an edge or a
 * vertex: the lowest original cell id).  A point outside the mesh returns
 * VG_EINVAL.  The gauge value is eta = H + z of that cell.  Clears the record
 * and records the current state if one is set.  n = 0 removes the gauges.
 */
int vg_set_gauges(vg_ctx *ctx, int32_t n, const double *xy);

/* Cells (original ids) that vg_set_gauges resolved, cells[n]. */
int vg_get_gauge_cells(vg_ctx *ctx, int32_t *cells);

/*
 * Advance n_steps SSP-RK(2,2) steps (Sec. 2.3) on the device; the time step of
 * each comes from the CFL rule on the stage-1 wave speeds,
 *   dt = cfl * min_K |K| / (3 max_f l_f a_f),
 * unless params.dt_fixed > 0, clamped by dt_max and t_end.  The whole loop
 * stays on the device (CUDA-graph replays); the call synchronises once at the
 * end and returns VG_ENONFINITE / VG_ENEGDEPTH if a step went wrong.
 */
int vg_step(vg_ctx *ctx, int64_t n_steps);

/* Step until the simulated time reaches t (the last step is shortened). */
int vg_advance_to(vg_ctx *ctx, double t);

/*
 * Gauge records so far: t[k] and eta[k][n_gauges] for k < min(*n_rec, cap).
 * *n_rec receives the number of records held.  Either array may be NULL.
 */
int vg_get_gauges(vg_ctx *ctx, double *t, double *eta, int64_t cap, int64_t *n_rec);

/* Diagnostics of the current state; synchronises the context stream. */
int vg_get_diagnostics(vg_ctx *ctx, vg_diag *d);

/*
 * Per-kernel timing.  With enable != 0, later vg_step calls launch kernel by
 * kernel (no graph) with CUDA events around each launch on the context
 * stream, and accumulate device time per kernel.  vg_get_profile returns, for
 * up to n kernels, their names (static strings), launch counts and total
 * milliseconds; *n_out receives the number of kernels timed: "stage1",
 * "stage2", "post_step", "bed_update", and with rk_unfused "rk_update1",
 * "residual_w1", "rk_update2" (in that order; a kernel never launched has 0).
 */
int vg_profile(vg_ctx *ctx, int enable);
int vg_get_profile(vg_ctx *ctx, int32_t n, const char **names, int64_t *launches, double *ms,
                   int32_t *n_out);

/* Bytes of device memory the context holds. */
int vg_device_bytes(vg_ctx *ctx, int64_t *bytes);

/*
 * One time step that allocates no device memory.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc when they step
 * -- a caller whose memory pool is fully reserved, a real-time loop that must
 * not touch the allocator, or a framework that forbids device allocations
 * after its set-up phase.
 *
 * The step's scratch (the stage-1 residual and the step scalars) lives in one
 * file-scope device array of fixed size inside the library, so a mesh may have
 * at most VG_NOALLOC_MAX_CELLS cells (VG_EINVAL otherwise).  The array (about
 * 6 MiB) is committed on a device at set-up, when a context first uploads a
 * mesh there: vg_mesh_upload looks up its address (with that device current)
 * and loads the kernels this call uses, so the call itself loads and allocates
 * nothing; the array is held until the process exits.
 *
 *   ctx     a context with a mesh (vg_mesh_upload, vg_set_params) and no moving
 *           bed (vg_set_bed_motion set: VG_ESTATE, since this call steps the
 *           static bed); its state, time, gauges and diagnostics are neither
 *           read nor changed
 *   w_in    device array [3][nc] of the context's precision: the state at time t
 *           in the library's internal cell order (vg_get_permutation gives
 *           new_of_old) -- rows H, Hu, Hv for FP64 contexts; for FP32 contexts
 *           the first row holds eta = H + z instead of H
 *   w_out   device array of the same shape receiving the state after one step;
 *           must not alias w_in
 *   t       time of w_in (for the t_end clamp)
 *   dt_out  host pointer receiving the step's dt (may be NULL)
 *
 * Work runs on the context's stream; the call waits for it.  All calls share
 * the scratch array and leave the last call's contents in it; each call clears
 * the scalars it needs before its kernels run, but calls that overlap on the
 * GPU (other streams or host threads) race on the array.  Returns
 * VG_ENONFINITE or VG_ENEGDEPTH (with params.strict_positivity) like vg_step.
 */
#define VG_NOALLOC_MAX_CELLS 262144
int vg_step_noalloc(vg_ctx *ctx, const void *w_in, void *w_out, double t, double *dt_out);


/* ------------------------------------------------------------------------
 * Discrete adjoint (FP64 contexts).  The run of n_steps SSP-RK(2,2) steps
 * (Sec. 2.3) from the current state, with a fixed or the CFL time step, is a
 * smooth map almost everywhere (branches -- wet/dry switches, limiter and wave-speed
 * choices, HLL regions -- frozen where the run takes them), and the gauge
 * records eta_g(t_n) = H + z of the gauge cells (Sec. 3 gauges) are outputs of
 * it.  vg_adj_backward returns the gradient of any scalar J(eta) given
 * dJ/deta, with respect to the initial state and the bathymetry.  Every
 * boundary kind of vg_set_boundary (wall, open, absorbing) and a moving bed
 * (vg_set_bed_motion) are differentiated.
 * ------------------------------------------------------------------------ */

/* Replace the per-vertex bathymetry depth (as in vg_mesh_upload) of the
   uploaded mesh; the cell beds and the face beds are recomputed.  The state is
   unchanged. */
int vg_set_depth(vg_ctx *ctx, const double *depth_v);

/*
 * Forward run for the adjoint: n_steps steps from the current state with the
 * fixed time step dt > 0, or, for dt = 0, the CFL time step of every step (the
 * rule of Sec. 2.3 with the context's cfl and dt_max; t_end is ignored),
 * recording the gauges at the start and after every step (vg_get_gauges then
 * returns n_steps + 1 records).  With dt = 0 the backward pass differentiates
 * through each step's time step as well: dt depends on the state through the
 * cell of smallest bound |K| / (3 max_f l_f a_f) (a tie goes to the lowest
 * original cell id) and its face of largest l_f a_f (a tie to the first local
 * face); a step clamped by dt_max does not depend on the state.  The state at
 * every checkpoint_every-th step is kept on the device, and vg_adj_backward
 * recomputes each segment of checkpoint_every steps once, recording it (about
 * r = 192 bytes per cell and step with a fixed dt, 216 with CFL steps, against
 * 24 per checkpoint).  0 picks the segment length that minimises device memory,
 * round(sqrt(24 n_steps / r)): recordings and checkpoints then take about equal
 * shares, 2 sqrt(24 r n_steps) bytes per cell in all (about 6.1 KB per cell for
 * 2000 steps).  The context's state advances to step n_steps.  dt < 0 or
 * non-finite: VG_EINVAL.
 */
int vg_adj_forward(vg_ctx *ctx, int64_t n_steps, double dt, int64_t checkpoint_every);

/* The same forward run for binomial checkpointing: only the first state is
 * kept, and vg_adj_backward reverses the steps with `slots` (1..4096) state
 * buffers on the device, recomputing forward steps along Griewank's binomial
 * schedule (the split of each range minimises the recomputed steps: found by
 * dynamic programming for up to 2048 steps, by halving beyond).  Device memory
 * is slots + 3 states plus one step's recordings, instead of the sqrt(N)
 * segment of recordings -- for meshes whose sqrt(N) segment does not fit --
 * at the price of recomputation (for N steps and s slots about N log N / log s
 * forward steps).  The gradients equal those of vg_adj_forward bit for bit. */
int vg_adj_forward_binomial(vg_ctx *ctx, int64_t n_steps, double dt, int32_t slots);

/*
 * Reverse sweep of the last vg_adj_forward run.  dJ_deta[n_steps + 1][G] is the
 * derivative of J with respect to each gauge record.  Outputs (host FP64,
 * original cell / vertex order; any may be NULL): dJ/dH0, dJ/dHu0, dJ/dHv0 [nc]
 * for the initial state, dJ/dz [nc] for the cell beds z_K alone (the face beds
 * held fixed), dJ/ddepth [nv] for the vertex depths, through both the cell beds
 * (z_K = -mean of its three vertex depths) and the face beds under the face
 * values of reconstructing cells (z_f = -mean of the face's two vertex
 * depths).  Scratch device memory
 * is allocated for the sweep and freed at its end; the first sweep on a mesh
 * also builds a list of its faces (4 bytes per face) that the context keeps
 * until the mesh is replaced.  No forward run: VG_ESTATE; allocation failure:
 * VG_ENOMEM.
 */
int vg_adj_backward(vg_ctx *ctx, const double *dJ_deta, double *dJ_dH0, double *dJ_dHu0, double *dJ_dHv0,
                    double *dJ_dz, double *dJ_ddepth);

/* After vg_adj_backward of a run with a moving bed (vg_set_bed_motion set
   during vg_adj_forward): dJ/duplift_v and dJ/donset_v [nv] (host, either may
   be NULL) -- the gradient with respect to the rupture history.  The bed of
   step n is the vertex-mean bed at its start time t_n; onset times act where a
   vertex is inside its rise (0 < (t_n - onset_v) / rise < 1), and with the CFL
   time step the dependence of every later t_n on each step's dt is included.
   No such run: VG_ESTATE.  The paper has no counterpart (its source model is
   not given). */
int vg_adj_bed_gradient(vg_ctx *ctx, double *dJ_duplift, double *dJ_donset);

/* Open (transmissive) boundary.  The paper's solver has walls (Sec. 2.5: a
 * ghost with mirrored normal velocity) and leaves other boundary conditions to
 * Dutykh et al. 2011.  Marks the n boundary edges edges[k] = (a, b) (original
 * vertex ids, either order; [n][2] int32, host, copied) open and every other
 * boundary face a wall: an open face takes as ghost the cell's own state, so
 * the reconstruction sees no jump across it and its flux is the physical flux
 * of the face state (zero-gradient outflow; waves leave with little
 * reflection).  n = 0 makes every boundary face a wall again.  An edge that is
 * not a boundary edge: VG_EINVAL, nothing changed.  The adjoint
 * differentiates through open faces as well. */
int vg_set_open_boundary(vg_ctx *ctx, int64_t n, const int32_t *edges);

/* Boundary kinds per edge: edges as for vg_set_open_boundary, kinds[k]
 * (int32, host, copied; NULL: all open) VG_BOUNDARY_WALL, VG_BOUNDARY_OPEN or
 * VG_BOUNDARY_ABSORBING; every other boundary face a wall.  An absorbing face
 * (a reading: the paper defers such conditions to Dutykh et al. 2011) takes the
 * characteristic ghost of a sea at rest at eta = 0 beyond the boundary: the
 * outgoing Riemann invariant u_n + 2c comes from the face state, the incoming
 * u_n - 2c = -2 c_0 from the rest state (c_0 = sqrt(g max(0, -z)) on the face's
 * bed), giving u_n,g = (R+ + R-)/2, c_g = max(0, (R+ - R-)/4), depth c_g^2 / g,
 * tangential velocity kept; the reconstruction sees it as the open ghost.
 * Waves leave with far less reflection than through open faces, and water
 * above or below the outer level flows out or in.  An edge that is not a
 * boundary edge or an unknown kind: VG_EINVAL, nothing changed.  The adjoint
 * differentiates all three kinds, the absorbing ghost's dependence on the bed
 * (through c_0) included. */
int vg_set_boundary(vg_ctx *ctx, int64_t n, const int32_t *edges, const int32_t *kinds);

/* Moving bed: the time-dependent depth h(x, y, t) of Sec. 2.1 (the governing
 * equations conserve the total depth H = h + eta while the bed moves), read as
 * a kinematic rupture: vertex v rises by uplift_v [nv] (metres, positive up),
 * linearly over `rise` seconds from its onset time onset_v [nv]:
 *     depth_v(t) = depth0_v - uplift_v * min(1, max(0, (t - onset_v) / rise))
 * (rise = 0: a step at onset), with depth0 the depths of vg_mesh_upload /
 * vg_set_depth.  The cell beds z_K = -(mean of their vertices' depths) and face
 * beds z_f = -(mean of the face's two vertex depths) are set at the end of
 * every step to the bed of the step's end time, keeping H (the
 * free surface follows the bed; no mass is created), before the gauges record;
 * vg_set_state (and this call, for the current state) sets the bed of the
 * state's time.  uplift_v = NULL removes the motion and restores the static
 * bed (keeping H).  Host arrays, caller-owned, copied; non-finite values or a
 * negative rise: VG_EINVAL.  One extra launch per step while set.  While it
 * is set, vg_step_noalloc and vg_set_depth fail with VG_ESTATE.  The
 * adjoint (vg_adj_forward / vg_adj_backward) differentiates through it, and
 * vg_adj_bed_gradient returns the gradients with respect to uplift_v and
 * onset_v. */
int vg_set_bed_motion(vg_ctx *ctx, const double *uplift_v, const double *onset_v, double rise);

/* ------------------------------------------------------------------------
 * Batched ensembles (uncertainty quantification): many scenarios -- initial
 * states of the same scheme -- on several meshes of uneven size, advanced
 * together.  Each scenario has its own time and its own CFL time step; one
 * batched step is one persistent launch per stage over every (mesh, block)
 * work item for all scenarios, replayed from a CUDA graph.  Results equal
 * those of one context per scenario bit for bit (same kernels, same order).
 * ------------------------------------------------------------------------ */
typedef struct vg_batch vg_batch;

/* precision 32 or 64, CUDA device, cudaStream_t or NULL (as vg_create). */
int vg_batch_create(vg_batch **out, int precision, int device, void *cuda_stream);
void vg_batch_destroy(vg_batch *b);
const char *vg_batch_last_error(vg_batch *b);

/* Parameters shared by all scenarios (vg_params, gauge_every included). */
int vg_batch_set_params(vg_batch *b, const vg_params *p);

/* Add a mesh (arguments as vg_mesh_upload) carrying n_scenarios scenarios;
   *mesh_id receives its index.  At most 512 scenarios per batch.  All meshes
   must end up with the same block size. */
int vg_batch_add_mesh(vg_batch *b, int64_t nv, const double *xy, int64_t nc, const int32_t *tri,
                      const double *depth_v, int renumber, int32_t n_scenarios, int32_t *mesh_id);

/* State of one scenario from host FP64 arrays in the mesh's original cell order
   (as vg_set_state), at time t. */
int vg_batch_set_state(vg_batch *b, int32_t mesh_id, int32_t scenario, const double *H, const double *Hu,
                       const double *Hv, double t);

/* State, time and step count of one scenario (t, steps may be NULL). */
int vg_batch_get_state(vg_batch *b, int32_t mesh_id, int32_t scenario, double *H, double *Hu, double *Hv,
                       double *t, int64_t *steps);

/* n_steps batched steps of every scenario (each with its own dt). */
int vg_batch_step(vg_batch *b, int64_t n_steps);

/* Step until every scenario reaches t_end (each stops exactly there), or
   max_steps; *steps_taken receives the batched steps run. */
int vg_batch_run(vg_batch *b, double t_end, int64_t max_steps, int64_t *steps_taken);

/* Autotuner: times n_steps batched steps from the current state for each
   candidate launch shape -- block size (64, 128, 256 cells per thread block)
   times resident CTAs per SM (as many as fit, and one and two fewer: fewer CTAs
   leave each more L1 for the mesh data its scenarios share) -- restores the
   state after each, and keeps the fastest; *best_block, *best_ctas_per_sm (0:
   as many as fit) and *best_ms_per_step report it (any may be NULL). */
int vg_batch_autotune(vg_batch *b, int32_t n_steps, int32_t *best_block, int32_t *best_ctas_per_sm,
                      double *best_ms_per_step);

/* Virtual gauges of one mesh, shared by all its scenarios (as vg_set_gauges:
   xy [n][2] in the mesh's coordinates, each located in its containing cell,
   ties to the lowest original cell id; a point outside the mesh: VG_EINVAL;
   n = 0 removes them).  Every scenario of the mesh then records eta = H + z of
   the gauge cells at its current time now, at vg_batch_set_state, and after
   every gauge_every of its own steps (a scenario that has reached t_end no
   longer records), the same records as a context of its own.  Records are
   kept in device rings and moved to host memory by the library whenever it
   reads the scenarios' scalars (every vg_batch_step and vg_batch_run call
   does, often enough that no record is lost). */
int vg_batch_set_gauges(vg_batch *b, int32_t mesh_id, int32_t n, const double *xy);

/* Open boundary edges of one mesh, shared by all its scenarios (as
   vg_set_open_boundary). */
int vg_batch_set_open_boundary(vg_batch *b, int32_t mesh_id, int64_t n, const int32_t *edges);

/* Boundary kinds per edge of one mesh, shared by all its scenarios (as
   vg_set_boundary). */
int vg_batch_set_boundary(vg_batch *b, int32_t mesh_id, int64_t n, const int32_t *edges, const int32_t *kinds);

/* Records of one scenario: t [cap] and eta [cap][G] (G = the mesh's gauge
   count), copied up to cap records; *n_rec receives the number held (may
   exceed cap).  Any of t, eta, n_rec may be NULL. */
int vg_batch_get_gauges(vg_batch *b, int32_t mesh_id, int32_t scenario, double *t, double *eta, int64_t cap,
                        int64_t *n_rec);

/* Meshes, scenarios, total cells over all scenarios, kernels launched. */
int vg_batch_info(vg_batch *b, int32_t *n_meshes, int32_t *n_scenarios, int64_t *cells, int64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* VOLNA_GB_H */
