/*
 * dsea.h -- C ABI of the GB300 slice-streamed Lennard-Jones NVE library.
 *
 * The library advances a periodic box of Lennard-Jones molecules with the
 * velocity-Verlet scheme of Algorithm 1 (Sec. 4), the box cut into slices
 * perpendicular to x, each slice at least one cutoff wide (Sec. 3, Sec. 4),
 * every slice updated from itself and its left and right neighbours
 * (O_in = O_out = 1, Sec. 4) and the (slice, step) updates streamed in a
 * time-skewed cyclic order through a ring of persistent on-chip stages
 * (Sec. 3.1 data flow, Sec. 3.3 worker firing rule).
 *
 * Conventions for every call:
 *  - returns DSEA_OK (0) or a negative DSEA_ERR_* code; dsea_status_string()
 *    names it;
 *  - host arrays passed in are read during the call and stay owned by the
 *    caller; outputs go to caller-allocated host arrays;
 *  - positions, velocities and forces are AoS (x, y, z) per atom, FP64, in
 *    the original atom-ID order (atom i at [3i, 3i+2]);
 *  - reduced LJ units: sigma = epsilon = m = 1;
 *  - calls on one box are not thread-safe; different boxes may be driven from
 *    different host threads;
 *  - work is enqueued on the CUDA stream given at creation; errors raised on
 *    the device (capacity, migration, timeout) are reported by the next call
 *    that synchronises with the box (dsea_sync or any dsea_read_*).
 */
#ifndef DSEA_H
#define DSEA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define DSEA_OK 0
#define DSEA_ERR_INVALID_ARG -1 /* bad pointer, size or geometry */
#define DSEA_ERR_OOM -2         /* device or host allocation failed */
#define DSEA_ERR_CUDA -3        /* a CUDA runtime call failed */
#define DSEA_ERR_TIMEOUT -4     /* a bounded device-side wait expired */
#define DSEA_ERR_CAPACITY -5    /* a cell received more atoms than its slots */
#define DSEA_ERR_MIGRATION -6   /* an atom moved farther than one slice in one step */
#define DSEA_ERR_BUDGET -7      /* a served job cannot fit the memory budget */
#define DSEA_ERR_STATE -8       /* call out of order (e.g. no kernel registered) */
#define DSEA_ERR_NOT_FOUND -9   /* unknown job id */
#define DSEA_ERR_NO_DEVICE -10  /* no CUDA device available */
#define DSEA_ERR_BOUNDS -12     /* checked build only: a kernel met an index out of range
                                   (it skipped the access; the box's state is not valid) */
#define DSEA_ERR_RANGE -13      /* the slice thermostat met 32 atoms with a kinetic energy of
                                   1024 epsilon or more (a temperature near 21): beyond the
                                   range of its exact fixed-point sums */

/* ---- enums ------------------------------------------------------------- */
#define DSEA_FP64 0  /* all pair arithmetic in FP64 */
#define DSEA_MIXED 1 /* FP32 pair arithmetic on cell-centred coordinates;
                        FP64 absolute positions, position update, reductions */

#define DSEA_KERNEL_LJ_TS 1 /* truncated-shifted LJ 12-6 (Sec. 4, Algorithm 1) */

#define DSEA_SCHED_RING 0     /* one persistent launch per advance: stages pull
                                 (slice, step) units in time-skewed cyclic order
                                 and wait on their neighbours' completion */
#define DSEA_SCHED_STEPWISE 1 /* one launch per step over all units (same
                                 per-unit arithmetic, bitwise equal results) */

typedef struct dsea_box dsea_box;
typedef struct dsea_batch dsea_batch;
typedef struct dsea_server dsea_server;

/* Optional device allocator (e.g. PyTorch's caching allocator).  alloc
 * returns a device pointer of at least `bytes` bytes, aligned to 256 bytes,
 * or NULL; free releases it.  NULL allocator = cudaMalloc / cudaFree. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} dsea_allocator;

/* Per-box kernel parameters (the "registered kernel", Sec. 3.3). */
typedef struct {
    double rc;         /* cutoff radius, sigma; 2.5 in every workload (Sec. 4) */
    double dt;         /* timestep, tau */
    int precision;     /* DSEA_FP64 or DSEA_MIXED */
    int schedule;      /* DSEA_SCHED_RING or DSEA_SCHED_STEPWISE */
    int tile_y;        /* home cells per work unit along y; tile_y = tile_z = 0:
                          automatic (see below) */
    int tile_z;        /* home cells per work unit along z */
    int cell_capacity; /* atom slots per cell; 0 = from the density */
    int ctas;          /* CTAs of a ring launch (one stage each in the FP64 form, one per
                          warp in the mixed form); 0 = automatic: the autotuner's choice
                          for the size class when it has one, else in the mixed form
                          n_slices x min(units per slice, 160) warps (all resident CTAs
                          when that is at least 90 % of them), in the FP64 form all
                          resident CTAs.  Launches of several boxes (batches, the
                          server) use the mixed rule summed over their boxes. */
    double temperature; /* NVT: target kT/epsilon of the slice thermostat (Sec. 4.1,
                           md_thermo_a/b and md_v3b); 0 = NVE.  Each step scales the
                           synchronised velocities of slice j by sqrt(T0 / T'_j), T'_j
                           the slice's temperature after the previous step's scaling
                           (factor 1 at the first step) */
} dsea_params;

/* Automatic work-unit shape (tile_y = tile_z = 0).  A box takes, in order:
 * the dsea_autotune choice cached for its size class; in the mixed form,
 * where a unit is one warp's, the launch-filling shape of the box alone (the
 * largest of 4x4, 3x3, 2x4, 2x2, 1x4, 1x2 home cells whose units per step
 * reach twice the warp stages one launch keeps resident, 32 per SM; else
 * 1x2); in the FP64 form 2 x 4.  Boxes on the automatic shape are re-shaped
 * together when they share a launch: dsea_batch_create and each server
 * launch apply the launch-filling rule to the units of all of them.  Only one
 * of the two set: that side as given, the other 2 (y) or 4 (z).  A shape
 * larger than the box, or whose stage does not fit a unit's shared memory,
 * is shrunk (longer side first).  The shape never changes a result. */

/* Boundary along x (the slicing axis).  y and z are always periodic. */
#define DSEA_BOUNDARY_PERIODIC 0 /* minimum image along x as well */
#define DSEA_BOUNDARY_MIRROR 1   /* specular mirror walls at x = 0 and x = Lx (Sec. 3
                                    requirement (3); the mirror of Sec. 4.2): no pair
                                    across them; an atom carried past a wall is
                                    reflected and its x velocity reversed */

/* A box as the caller describes it (Sec. 4: cubic volume of edge b, but any
 * orthorhombic box works).  n_slices = 0 means one slice per cell layer
 * along x (the paper's choice N_S = N_xyz, Sec. 4). */
typedef struct {
    int n_slices;
    double box[3];     /* edge lengths Lx, Ly, Lz */
    int64_t n_atoms;
    const double *pos; /* host, 3 n_atoms, any values (wrapped into the box); with mirror
                          walls every x must lie in [0, Lx) */
    const double *vel; /* host, 3 n_atoms, or NULL for zero velocities */
    int boundary_x;    /* DSEA_BOUNDARY_PERIODIC or DSEA_BOUNDARY_MIRROR */
} dsea_box_desc;

/* Observables at the box's current step, all FP64:
 *   U  = sum over pairs i<j of the shifted pair energy (Algorithm 1's U),
 *   W  = sum over pairs i<j of r_ij . F_ij (24 times Algorithm 1's V),
 *   KE = 1/2 sum_i v_i^2 at the synchronised velocity v(t_step). */
typedef struct {
    int64_t step;
    double U, W, KE;
} dsea_observables;

/* Geometry and memory of a box, for inspection. */
typedef struct {
    int n_slices, cells_per_slice_x;
    int cells[3];
    int tile_y, tile_z, units_per_step;
    int cell_capacity;
    int precision, schedule;
    int64_t n_atoms, step;
    size_t device_bytes; /* device memory the box holds now (also before registration:
                            its copy of the initial state) */
    double cell_edge[3];
    int boundary_x;
} dsea_box_info;

/* ---- box lifecycle ----------------------------------------------------- */

/* Create a box from host positions and velocities (Sec. 3, "the user
 * provides slices of the dataset"; Sec. 4 geometry).  The box is cut into
 * n_slices slices along x of width Lx / n_slices >= rc and into cells of edge
 * >= rc; needs >= 3 slices and >= 3 cells per axis (checked by
 * dsea_register_kernel, which knows rc).  The cell count per axis is the
 * paper's floor(L / rc) at liquid density; below rho = 8 / rc^3 the cells
 * grow (edge (8 / rho)^(1/3), at most 1.5 rc, still at least 3 per axis) so
 * that each holds about eight atoms.  The positions and velocities are
 * copied to device buffers owned by the box (through `allocator`) and the
 * positions checked there; the call returns once the copies are complete, so
 * the caller may reuse its arrays at once (pinned host memory makes the
 * copies faster).  Errors: DSEA_ERR_INVALID_ARG for a bad box, boundary code,
 * an x outside [0, Lx) with mirror walls (all checked before any device
 * call) or a non-finite position; DSEA_ERR_NO_DEVICE, DSEA_ERR_OOM,
 * DSEA_ERR_CUDA.  The cell state itself is allocated by
 * dsea_register_kernel.  `cuda_stream` is a cudaStream_t (NULL = the legacy
 * default stream).  *out receives the handle. */
int dsea_box_create(const dsea_box_desc *desc, const dsea_allocator *allocator,
                    void *cuda_stream, dsea_box **out);

/* Register the per-slice kernel (Sec. 3.3: the user kernel with input and
 * output order).  kind must be DSEA_KERNEL_LJ_TS and o_in = o_out = 1
 * (Sec. 4); params may be NULL for rc 2.5, dt 0.005, FP64, ring schedule.
 * Allocates the slice/cell state on the device, bins the atoms, releases
 * the box's copy of the initial state and makes the box ready to advance. */
int dsea_register_kernel(dsea_box *box, int kind, int o_in, int o_out, const dsea_params *params);

/* Advance n_steps >= 0 velocity-Verlet steps (Algorithm 1), asynchronously
 * on the box's stream. */
int dsea_advance(dsea_box *box, int64_t n_steps);

/* Wait for the box's queued work; returns the first device-side error. */
int dsea_sync(dsea_box *box);

/* Read the current state in atom-ID order into host arrays of 3 n doubles
 * (n must equal the box's atom count).  Positions are wrapped into the box.
 * Velocities and forces are synchronised with the positions (a force pass
 * at the current positions runs on first read after an advance). */
int dsea_read_positions(dsea_box *box, double *out_xyz, int64_t n);
int dsea_read_velocities(dsea_box *box, double *out_xyz, int64_t n);
int dsea_read_forces(dsea_box *box, double *out_xyz, int64_t n);

/* Observables at the current step (Algorithm 1's U and V, and KE): FP64
 * sums of per-cell partials (each cell's atoms in canonical order) over the
 * cells in a fixed order, so the same bits whatever the unit shape, stage
 * count, batch or server launch the box ran in. */
int dsea_read_observables(dsea_box *box, dsea_observables *out);

/* Spatially resolved observables at the current step (Sec. 4.2: per-slice
 * results): for each slice j (n must equal the slice count) the sums over the
 * atoms of slice j of half their pair energies (U[j]), half their pair
 * virials (W[j]) and their kinetic energies (KE[j]), and the atom count
 * (N[j]); host arrays of n entries; any pointer may be NULL.  Slice j holds
 * the atoms of cell layers [j cps, (j+1) cps) along x.  Synchronising. */
int dsea_read_profiles(dsea_box *box, double *U, double *W, double *KE, int64_t *N, int n);

int dsea_box_get_info(const dsea_box *box, dsea_box_info *out);

int dsea_box_destroy(dsea_box *box);

/* ---- many boxes in one persistent launch -------------------------------- */

/* Group n boxes (same device, same stream, same precision, all registered)
 * so that one persistent launch advances all of them; the launch is captured
 * once in a CUDA graph per distinct step vector and replayed.  Mixed-precision
 * boxes on the automatic unit shape take the launch-filling shape of the
 * whole batch (see dsea_params).  The boxes stay owned by the caller and must
 * outlive the batch. */
int dsea_batch_create(dsea_box *const *boxes, int n, dsea_batch **out);

/* Advance box k by steps[k] >= 0 steps, all in one launch. */
int dsea_batch_advance(dsea_batch *batch, const int64_t *steps);

int dsea_batch_destroy(dsea_batch *batch);

/* ---- autotuning -------------------------------------------------------- */

/* Time each candidate work-unit shape (tile_y x tile_z home cells), then at
 * the fastest shape each ring stage count (all resident CTAs, 3/4, 1/2 and
 * 1/4 of them, against the default rule), for trial_steps steps each from a
 * snapshot of the box's state (taken through the box's allocator, restored
 * after each trial), and keep the fastest; a fixed stage count is kept only
 * when it is at least 3 % faster than the default.  The choice is cached per
 * size class (total cells and mean atoms per cell in octaves, cells along y
 * and z up to 16, cell layers per slice, cell capacity, precision), applied
 * to the box and used as the default shape and stage count of later boxes of
 * the same class.  The tile shape never
 * changes a result: each atom's force is summed in the same order whatever
 * the shape.  *chosen (may be NULL) receives the parameters in effect. */
int dsea_autotune(dsea_box *box, int trial_steps, dsea_params *chosen);

/* Choose one unit shape for every box of a batch: each candidate (the same
 * list as dsea_autotune's) is applied to all boxes, shrunk per box where its
 * cells or its shared-memory stage do not allow it, and the batch is timed
 * over trial_steps steps in one dsea_batch_advance from snapshots of every
 * box's state, which are restored after each trial.  The boxes keep the
 * fastest shape; *tile_y, *tile_z (may be NULL) receive it.  Many boxes in
 * one launch fill the GPU by themselves, so the batch's best shape is
 * usually larger than what dsea_autotune picks for a small box alone.  The
 * boxes leave the automatic shape; the lone-box cache is not changed.  The
 * snapshots, as large as every box's state, come from each box's allocator
 * and are released before the call returns; DSEA_ERR_OOM if they do not fit
 * (the boxes are unchanged).  The shape never changes a result.  Results:
 * DSEA_OK, DSEA_ERR_INVALID_ARG (NULL batch, trial_steps <= 0), or a latched
 * device error of a box. */
int dsea_batch_autotune(dsea_batch *batch, int trial_steps, int *tile_y, int *tile_z);

/* ---- serving ----------------------------------------------------------- */

/* A continuous-batching server: jobs (boxes with a step count) are admitted
 * while their device state fits mem_budget_bytes, kept resident, and
 * advanced together in persistent launches of at most segment_steps steps;
 * jobs join and leave between launches.  A host thread drives the device.
 * With tile_y = tile_z = 0 in params, each launch re-shapes the jobs present
 * by the launch-filling rule (see dsea_params): small units while few jobs
 * run, larger ones once they fill the GPU together. */
int dsea_server_create(size_t mem_budget_bytes, const dsea_params *params, int segment_steps,
                       void *cuda_stream, dsea_server **out);

/* Which resident jobs each launch advances (set at any time; the next launch
 * uses it).  DSEA_SERVE_SHORTEST, the default: the jobs with the least
 * remaining work first (remaining atom-steps at the server's measured rate,
 * minus 0.1 x the seconds since the job arrived, so that a waiting job's
 * turn always comes), taken in that order until they hold 2^21 atoms (a
 * launch that size still fills the GPU).  DSEA_SERVE_ALL: every resident job
 * in every launch.  A job's results do not depend on the policy, only when
 * it finishes.  DSEA_ERR_INVALID_ARG for another value. */
#define DSEA_SERVE_ALL 0
#define DSEA_SERVE_SHORTEST 1
int dsea_server_set_policy(dsea_server *srv, int policy);

/* Queue a job; the box description is copied.  *job_id receives its id. */
int dsea_server_submit(dsea_server *srv, const dsea_box_desc *desc, int64_t steps,
                       uint64_t *job_id);

/* *state: 0 queued, 1 running, 2 done, or a negative error code. */
int dsea_server_poll(dsea_server *srv, uint64_t job_id, int *state);

/* Copy a finished job's final positions and velocities (3 n doubles each,
 * atom-ID order, may be NULL) and observables, then release it.  *t_arrive,
 * *t_done (seconds on the server clock, may be NULL) give its latency. */
int dsea_server_result(dsea_server *srv, uint64_t job_id, double *pos, double *vel,
                       dsea_observables *obs, double *t_arrive, double *t_done);

/* Block until every submitted job is done or failed. */
int dsea_server_drain(dsea_server *srv);

/* Server clock (seconds since creation), for stamping arrivals. */
double dsea_server_clock(const dsea_server *srv);

/* Cumulative atom-steps advanced and busy device seconds. */
int dsea_server_stats(const dsea_server *srv, double *atom_steps, double *busy_seconds,
                      int *launches);

int dsea_server_destroy(dsea_server *srv);

/* ---- forces without device allocation ------------------------------------ */

/* The paper has no counterpart to this call.  It is for callers that cannot
 * let a library allocate device memory: hosts that reserve all GPU memory in
 * their own pool up front and refuse outside cudaMalloc calls, and
 * latency-bound loops where cudaMalloc / cudaFree would synchronise the device.
 * It computes, for one configuration, the forces and (U, W, KE) that a box
 * registered with DSEA_KERNEL_LJ_TS would report at its current step, using
 * the same kernels, but it allocates nothing: its scratch is one fixed 64 MiB
 * device array that the library holds on every GPU that loads it until the
 * process exits.
 *   pos_dev   device, 3 n_atoms FP64 positions (AoS, atom-ID order), read only;
 *   vel_dev   device, 3 n_atoms FP64 velocities, or NULL (then KE = 0);
 *   box       host, 3 edge lengths; one slice per cell layer, cells >= rc;
 *   precision DSEA_FP64 or DSEA_MIXED;
 *   forces_dev device, 3 n_atoms FP64 output (atom-ID order);
 *   obs3_dev  device, 3 FP64 outputs (U, W, KE), or NULL;
 *   cuda_stream work is queued there; before returning, the call waits for
 *             that stream (and only that stream) to finish, because it reads
 *             a status word back to the host.
 * Returns DSEA_ERR_SCRATCH_LIMIT, before touching the GPU, when the box needs
 * more than the 64 MiB (at density 0.8: about 290,000 atoms in FP64, 240,000
 * in the mixed form).  Because every call waits for its stream and reads the
 * status word back, no call may be made while a stream is being captured
 * into a CUDA graph (the first call on a device also looks up the array's
 * device address, which capture does not allow either).  Every call shares
 * the array: calls that overlap on the GPU, from other streams or host
 * threads, race and must be serialised by the caller. */
#define DSEA_ERR_SCRATCH_LIMIT -11 /* problem larger than the fixed scratch */
int dsea_forces_noalloc(const double *pos_dev, const double *vel_dev, int64_t n_atoms,
                        const double *box, double rc, int precision, double *forces_dev,
                        double *obs3_dev, void *cuda_stream);

/* ---- arithmetic peak probes ---------------------------------------------- */

/* The paper has no counterpart to this call: it measures the denominators of
 * the roofline the benchmark reports.  kind DSEA_PROBE_FP32: scalar FP32
 * fused multiply-adds (2 flops each); DSEA_PROBE_FP32X2: packed two-lane FP32
 * FMAs (fma.rn.f32x2, 4 flops each); DSEA_PROBE_FP64: FP64 FMAs.  8 CTAs of
 * 256 threads per SM, 8 independent chains per thread; *tflops receives the
 * counted flops over the CUDA-event time of the fastest of three launches
 * on `cuda_stream` (after an untimed warm-up launch).  The call allocates a small device
 * buffer, waits for the stream and returns DSEA_OK, DSEA_ERR_INVALID_ARG,
 * DSEA_ERR_NO_DEVICE or DSEA_ERR_CUDA. */
#define DSEA_PROBE_FP32 0
#define DSEA_PROBE_FP32X2 1
#define DSEA_PROBE_FP64 2
int dsea_probe_peak(int kind, void *cuda_stream, double *tflops);

/* ---- failure-detection testing hooks -------------------------------------- */

/* No GPU fault is involved.  DSEA_DEBUG_WITHHOLD_SLICE: during the next ring
 * advances, slice `value` never reports its first level complete, so every
 * unit that depends on it waits until the bounded wait expires, the launch
 * stops and the next synchronising call returns DSEA_ERR_TIMEOUT (the box is
 * then unusable); -1 turns the hook off.  DSEA_DEBUG_WAIT_LIMIT_NS: the
 * bounded-wait limit in nanoseconds (default 5 s). */
#define DSEA_DEBUG_WITHHOLD_SLICE 1
#define DSEA_DEBUG_WAIT_LIMIT_NS 2
int dsea_debug_set(dsea_box *box, int key, int64_t value);

/* ---- the generic slice ring (Sec. 3.1, 3.3) ------------------------------ */

/* A sliced dataset streamed through a registered slice kernel: the paper's
 * model of "the user provides slices of the dataset" and a kernel with O_in
 * input and O_out output neighbours (Sec. 3.3, caller_worker), for explicit
 * algorithms other than the built-in Lennard-Jones step.  Each slice has two
 * device buffers of slice_bytes (step parity: a step never overwrites its own
 * inputs, Sec. 3.1).  n_workers CUDA streams are the workers: worker k runs
 * the steps s = k mod n_workers, each step sweeping every slice once in a
 * cyclic order that starts (O_in + O_out) s slices further than at step 0;
 * unit (j, s) starts after units (j - R .. j + R, s - 1), R = O_in + O_out,
 * which finalise its inputs and are the last readers of the buffers it
 * overwrites.  Units of one step run one after another, so outputs shared
 * with neighbouring units (O_out > 0) are never written concurrently. */
typedef struct dsea_dataset dsea_dataset;

/* A slice kernel ("caller_worker" launcher).  Computes step + 1 from step for
 * slice `slice` by enqueueing device work on `stream` (a cudaStream_t):
 *   in[k],  k = 0 .. 2 O_in:  device view of slice (slice - O_in + k) mod n at `step` (read only);
 *   out[k], k = 0 .. 2 O_out: device view of slice (slice - O_out + k) mod n at step + 1.
 * out[O_out] is the slice's own output; views of other slices are shared with
 * their units.  Returns 0, or a negative DSEA_ERR_* that stops the run. */
typedef int (*dsea_slice_fn)(void *user, int slice, int64_t step, const void *const *in, void *const *out,
                             size_t slice_bytes, void *stream);

/* Create a dataset of n_slices zero-filled slices (2 (O_in + O_out) + 1 <=
 * n_slices, 1 <= n_workers <= 64).  allocator: as for boxes (NULL =
 * cudaMalloc).  cuda_stream: the caller's stream, which runs ordered with
 * every dsea_dataset_run.  INVALID_ARG, NO_DEVICE, OOM. */
int dsea_dataset_create(int n_slices, size_t slice_bytes, int o_in, int o_out, int n_workers,
                        const dsea_allocator *allocator, void *cuda_stream, dsea_dataset **out);

/* Copy host bytes into (out of) slice `slice` at the current step; bytes must
 * equal slice_bytes.  Synchronising. */
int dsea_dataset_write_slice(dsea_dataset *ds, int slice, const void *host, size_t bytes);
int dsea_dataset_read_slice(dsea_dataset *ds, int slice, void *host, size_t bytes);

/* Register the slice kernel (replaces any previous one). */
int dsea_dataset_register(dsea_dataset *ds, dsea_slice_fn fn, void *user);

/* Enqueue n_steps steps of every slice in the ring order; asynchronous with
 * respect to the host (the caller's stream waits for them).  STATE without a
 * registered kernel; a kernel's negative status is returned. */
int dsea_dataset_run(dsea_dataset *ds, int64_t n_steps);

/* Steps completed (queued) so far; -1 for NULL. */
int64_t dsea_dataset_step(const dsea_dataset *ds);

int dsea_dataset_destroy(dsea_dataset *ds);

/* The dataset's dispatch order without a GPU: for k = 0 .. n_slices n_steps - 1
 * the slice, absolute step and worker of the k-th unit, steps start_step .. */
int dsea_dataset_plan(int n_slices, int o_in, int o_out, int n_workers, int64_t n_steps, int64_t start_step,
                      int32_t *out_slice, int64_t *out_step, int32_t *out_worker);

/* A slice kernel shipped with the library, for tests and examples: one
 * explicit FP32 step of the heat equation u_t = u_xx on a periodic rod whose
 * slices hold slice_bytes / 4 grid values each (O_in = 1, O_out = 0):
 * u'[i] = u[i] + a (u[i-1] - 2 u[i] + u[i+1]), a = *(const float *)user,
 * evaluated in that order with every operation rounded (no contraction). */
int dsea_example_heat1d(void *user, int slice, int64_t step, const void *const *in, void *const *out,
                        size_t slice_bytes, void *stream);

/* ---- host-side schedule introspection (no GPU needed) ------------------- */

/* The order in which the ring dispatches the units of one box: for
 * k = 0 .. n_slices * units_per_slice * n_steps - 1, out_slice[k] and
 * out_step[k] name the slice and relative step of the k-th unit.  Every
 * unit's dependencies (slices j-2 .. j+2 at the previous step, periodic)
 * come earlier in this order. */
int dsea_ring_order(int n_slices, int units_per_slice, int64_t n_steps, int64_t start_step,
                    int32_t *out_slice, int32_t *out_step);

/* Human-readable name of a status code. */
const char *dsea_status_string(int status);

/* Library version, e.g. "0.1.0". */
const char *dsea_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DSEA_H */
