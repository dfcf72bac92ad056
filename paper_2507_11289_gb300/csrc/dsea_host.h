// dsea_host.h -- host-side objects shared by the C-ABI translation units
// (dsea_api.cu, dsea_server.cu); not part of the ABI.
#pragma once

#include "dsea.h"
#include "dsea_internal.h"

#include <nvtx3/nvToolsExt.h>

#include <map>
#include <utility>
#include <vector>

// A named NVTX range over a scope of host code (the library's calls and the
// server's phases show up by name on a profiler's timeline; without a tool
// attached a range costs a call through a null hook).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct dsea_box {
    int device = 0;
    cudaStream_t stream = nullptr;
    dsea_allocator alloc{};
    bool has_alloc = false;
    int n_slices_req = 0;
    double L[3] = {0, 0, 0};
    int walls_x = 0;                  // DSEA_BOUNDARY_MIRROR along x
    double *d_pos0 = nullptr;         // device copies of the caller's positions and
    double *d_vel0 = nullptr;         // velocities until the kernel is registered
    bool has_vel = false;
    bool registered = false;
    dsea_params params{};
    double mean_cap = 0;              // expected atoms per cell used for stage sizing
    bool tile_auto = false;           // unit shape not requested: launches may re-choose it
    dsea::BoxDev hb{};
    dsea::BoxDev *db = nullptr;
    std::vector<std::pair<void *, size_t>> allocs;   // live device allocations and their sizes
    size_t device_bytes = 0;
    // ring plan buffers of single-box launches
    int64_t *d_step_base = nullptr;
    int64_t step_base_cap = 0;
    int64_t *d_cum = nullptr;
    int *d_active = nullptr;
    unsigned long long *d_ticket = nullptr;
    int *d_launch_err = nullptr;
    double *d_obs3 = nullptr;
    double obs3[3] = {0, 0, 0};
    bool outputs_valid = false;
    int latched = DSEA_OK;            // first device error seen
};

namespace dsea {

// Reusable buffers of a persistent launch over several boxes.  The host half
// is pinned so that a captured graph can re-read it on every replay.
struct MultiPlan {
    int cap_boxes = 0;
    int64_t cap_steps = 0;
    BoxDev *d_boxes = nullptr, *h_boxes = nullptr;
    int64_t *d_cum = nullptr, *h_cum = nullptr;
    int64_t *d_step_base = nullptr, *h_step_base = nullptr;
    int *d_active = nullptr, *h_active = nullptr;
    unsigned long long *d_ticket = nullptr;
    int *d_err = nullptr;
    // filled by multi_prepare
    int n = 0;
    int64_t smax = 0, total = 0;
    size_t smem = 0;
    int precision = 0;
    int64_t want_warps = 0;   // mixed form: the stage-count rule summed over the boxes
    std::vector<int> order;
};

// Make room for n boxes and smax steps (frees and reallocates as needed).
int multi_reserve(MultiPlan &mp, int n, int64_t smax);
// Host half of a launch advancing boxes[k] by steps[k]; the pinned buffers
// must not be in use by an earlier launch.
int multi_prepare(MultiPlan &mp, dsea_box *const *boxes, const int64_t *steps, int n);
// Enqueue the plan upload, the counter resets and the ring launch.
int multi_enqueue(MultiPlan &mp, dsea_box *const *boxes, cudaStream_t stream);
// After the launch has been enqueued: advance the host step counters.
void multi_commit(dsea_box *const *boxes, const int64_t *steps, int n);
void multi_free(MultiPlan &mp);

// Give every mixed-precision box of a launch whose unit shape is automatic
// (tile_auto) the launch-filling shape of the whole set: the largest candidate
// whose units per step, over all boxes, reach twice the resident warp stages.
// Host arithmetic only; a shape never changes a result.
void retile_for_launch(dsea_box *const *boxes, int n);

// Geometry, cell capacity and work-unit shape of a box (no allocation).
int box_geometry(int n_slices, const double *L, int64_t n_atoms, dsea_params &p, BoxDev &hb);

// Device bytes a box of this description would hold once registered.
int estimate_box_bytes(const dsea_box_desc *desc, const dsea_params *params, size_t *bytes);

// Force pass + read-back of positions, velocities (and observables) into host
// arrays (any may be NULL); synchronises the box.
int read_state(dsea_box *b, double *pos, double *vel, dsea_observables *obs);

}  // namespace dsea
