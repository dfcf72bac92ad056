// dsea_internal.h -- device-side box descriptor and the launch entry points
// shared by the CUDA translation units of the library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

// DSEA_CHECKED=1 builds the checked variant of the library: every computed
// global index (slots, cells, atom ids, units, slices) and shared-memory list
// position is tested before it is used; an index out of range sets
// kErrBounds and the access is skipped.  The release build defines it 0, and
// the checks compile to nothing.
#ifndef DSEA_CHECKED
#define DSEA_CHECKED 0
#endif

namespace dsea {

constexpr int kThreads = 256;            // threads per work-unit CTA
constexpr int kWarps = kThreads / 32;
constexpr int kMaxStagedCells = 2048;    // staged neighbourhood cells per unit (upper bound)
constexpr int kObsStride = 4;            // per-cell partials of a force pass: U, W, KE, atom count

// Device error word values (first error wins).
enum : int {
    kErrNone = 0,
    kErrCapacity = 1,   // a cell or the shared-memory stage overflowed
    kErrMigration = 2,  // an atom left slices j-1..j+1 in one step
    kErrTimeout = 3,    // a bounded dependency wait expired
    kErrBounds = 4,     // checked build: an index out of range (the access was skipped)
    kErrRange = 5,      // a thermostat kinetic energy beyond its fixed-point range
};

// One box as the kernels see it.  Slot layout: the state of a step lives in
// one of two buffers (step parity).  Cell c owns slots [c*cap, c*cap + cap);
// per-slot arrays are SoA (component k of slot t at k*n_slots + t).  Within
// a cell, the atoms that stayed in it during the last step fill the front
// slots in the cell's canonical order and the atoms that arrived fill the
// back slots (the last one first); readers order the arrivals by atom id.
struct BoxDev {
    // geometry (Sec. 4: cells of edge >= rc, slices of cps cell layers in x)
    double L[3];
    double lc[3];
    double inv_lc[3];
    float lcf[3];
    float inv_lcf[3];   // 1 / lcf, rounded
    int nc[3];
    int n_slices;
    int cps;
    // work units: tile_y x tile_z home cells (all cps layers of one slice)
    int tile_y, tile_z, tiles_y, tiles_z, units_per_slice;
    int cap;
    int precision;
    int walls_x;       // 1: mirror walls at x = 0 and x = Lx (no wrap along x)
    int staged_cells;  // max staged cells of a unit
    int smem_atoms;    // staged atoms the unit's shared memory holds
    int64_t n_cells;
    int64_t n_slots;   // n_cells * cap
    int64_t n_atoms;
    // pair law (Algorithm 1)
    double rc2, ushift, dt;
    float rc2f, ushiftf;
    // state, two step-parity buffers
    unsigned long long *cnt[2];  // per cell: (tag << 32) | stayers, tag = step + 1
    unsigned long long *arr[2];  // per cell: (tag << 32) | arrivals
    int *id[2];     // FP64 form: atom ids (the mixed form keeps them in q.w)
    double *r[2];   // FP64 form: absolute positions; mixed: relative to the atom's cell centre
    double *v[2];   // FP64 form: velocities (half-step after the first step), 3 * n_slots
    float *vf[2];   // mixed form: the same velocities in FP32, 3 * n_slots
    float4 *q[2];   // mixed: cell-centred FP32 coordinates, atom id bits in .w
    // per advance
    int64_t step;   // absolute step of the current state
    int w_is_sync;  // 1 until the first step: v holds v(t0), not v(t-dt/2)
    int withhold_slice;   // testing hook: this slice never reports completion (-1 = off)
    unsigned *done;       // [n_slices] completed units of the running launch, then
                          // [n_slices] units whose thermostat partial is written
    int *err;             // device error word
    double *unit_obs;     // [n_cells * kObsStride] (U, W, KE, N) of each home cell, from a force pass
    // slice thermostat (T0 > 0): per unit (KE, N) of the synchronised velocities before
    // scaling (KE as an int64 fixed-point word), and per slice the factor of the step,
    // both by step parity
    double T0;
    double *th_part[2];   // [units_per_step * 2]
    double *th_lam[2];    // [n_slices]
    double *out_r, *out_v, *out_f;  // readback by atom id, 3 * n_atoms each
    long long wait_limit_ns;        // bounded-wait limit of the ring
};

// Slice processed by the jj-th slice group of level s_abs in the ring's
// dispatch order: each level starts two slices after the previous one.
__host__ __device__ inline int ring_slice(int jj, long long s_abs, int n_slices)
{
    return (int)((jj + 2 * (s_abs % n_slices)) % n_slices);
}

// Dynamic shared memory bytes a unit of this box needs.
size_t unit_smem_bytes(int precision, int staged_cells, int smem_atoms);

// Largest dynamic shared memory a unit may use on this device.
size_t max_unit_smem_bytes();

// Bin atoms (device AoS pos/vel, atom-ID order) into the buffer of `box.step`.
// flag = 1 if any of a[0..n) is not finite (flag is left alone otherwise).
cudaError_t launch_check_finite(const double *a, long long n, int *flag, cudaStream_t stream);
cudaError_t launch_bin(const BoxDev &host_box, const BoxDev *dev_box, const double *pos,
                       const double *vel, cudaStream_t stream);

// One step of all units of one box, one launch (no device waits).
cudaError_t launch_step(const BoxDev &host_box, const BoxDev *dev_box, int64_t s_abs,
                        int first_step, cudaStream_t stream);

// Force pass at the current state: forces, synchronised velocities and
// positions scattered by atom id, plus (U, W, KE, N) partials per home cell.
cudaError_t launch_force_pass(const BoxDev &host_box, const BoxDev *dev_box, cudaStream_t stream);

// Deterministic fixed-order sum of the per-cell partials into out3 (device).
cudaError_t launch_obs_reduce(const double *cell_obs, long long n_cells, double *out3,
                              cudaStream_t stream);

// The persistent ring over one or more boxes (same precision).
struct RingPlan {
    const BoxDev *boxes;        // device array [n_boxes]
    const int64_t *step_base;   // [n_steps + 1] first ticket of each relative step
    const int64_t *cum_units;   // [n_boxes + 1] prefix sums of units per step
    const int *active;          // [n_steps] boxes active at each relative step
    int n_boxes;
    int n_steps;                // relative steps in this launch (max over boxes)
    int64_t total;              // tickets
    unsigned long long *ticket; // dispenser
    int *err;                   // launch-wide error word
};
cudaError_t launch_ring(const RingPlan &plan, int precision, size_t smem_bytes, int ctas,
                        cudaStream_t stream);

// Occupancy of the ring kernel (CTAs per SM) for a shared-memory size.
int ring_ctas_per_sm(int precision, size_t smem_bytes);

}  // namespace dsea
