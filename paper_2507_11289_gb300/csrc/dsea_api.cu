// dsea_api.cu -- host side of the C ABI declared in include/dsea.h: box
// lifecycle, the two launch forms of an advance, read-back, many-box batches
// replayed from CUDA graphs, the work-unit autotuner and schedule
// introspection.
#include "dsea_host.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

using dsea::BoxDev;

struct dsea_batch {
    std::vector<dsea_box *> boxes;
    cudaStream_t stream = nullptr;
    int precision = 0;
    dsea::MultiPlan mp;
    cudaEvent_t done_ev = nullptr;
    std::map<std::vector<int64_t>, cudaGraphExec_t> graphs;
};

namespace {

int map_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return DSEA_OK;
    if (e == cudaErrorMemoryAllocation) return DSEA_ERR_OOM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return DSEA_ERR_NO_DEVICE;
    return DSEA_ERR_CUDA;
}

int map_device_error(int code)
{
    switch (code) {
    case dsea::kErrNone: return DSEA_OK;
    case dsea::kErrCapacity: return DSEA_ERR_CAPACITY;
    case dsea::kErrMigration: return DSEA_ERR_MIGRATION;
    case dsea::kErrTimeout: return DSEA_ERR_TIMEOUT;
    case dsea::kErrBounds: return DSEA_ERR_BOUNDS;
    case dsea::kErrRange: return DSEA_ERR_RANGE;
    default: return DSEA_ERR_CUDA;
    }
}

#define CU(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return map_cuda(e_); \
    } while (0)

void *dev_alloc(dsea_box *b, size_t bytes)
{
    void *p = nullptr;
    bytes = std::max<size_t>(bytes, 256);
    if (b->has_alloc) {
        p = b->alloc.alloc(bytes, b->alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        b->allocs.emplace_back(p, bytes);
        b->device_bytes += bytes;
    }
    return p;
}

void dev_release(dsea_box *b, void *p)
{
    if (b->has_alloc) b->alloc.free(p, b->alloc.ctx);
    else cudaFree(p);
}

// Free one allocation of the box before the box itself goes.
void dev_free(dsea_box *b, void *p)
{
    for (size_t k = 0; k < b->allocs.size(); ++k) {
        if (b->allocs[k].first != p) continue;
        dev_release(b, p);
        b->device_bytes -= b->allocs[k].second;
        b->allocs.erase(b->allocs.begin() + (long)k);
        return;
    }
}

void dev_free_all(dsea_box *b)
{
    for (auto &a : b->allocs) dev_release(b, a.first);
    b->allocs.clear();
    b->device_bytes = 0;
}

// Copy the caller's positions (and velocities) into device buffers of the
// box and check that they are finite; waits for the copies, so the caller may
// reuse its arrays as soon as dsea_box_create returns.
int upload_initial_state(dsea_box *b, const dsea_box_desc *desc)
{
    const long long n3 = 3LL * desc->n_atoms;
    if (n3 == 0) return DSEA_OK;
    const size_t nb = sizeof(double) * (size_t)n3;
    b->d_pos0 = (double *)dev_alloc(b, nb);
    if (b->has_vel) b->d_vel0 = (double *)dev_alloc(b, nb);
    int *d_flag = (int *)dev_alloc(b, sizeof(int));
    if (!b->d_pos0 || (b->has_vel && !b->d_vel0) || !d_flag) return DSEA_ERR_OOM;
    CU(cudaMemsetAsync(d_flag, 0, sizeof(int), b->stream));
    CU(cudaMemcpyAsync(b->d_pos0, desc->pos, nb, cudaMemcpyHostToDevice, b->stream));
    if (b->has_vel) CU(cudaMemcpyAsync(b->d_vel0, desc->vel, nb, cudaMemcpyHostToDevice, b->stream));
    CU(dsea::launch_check_finite(b->d_pos0, n3, d_flag, b->stream));
    int flag = 0;
    CU(cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    dev_free(b, d_flag);
    return flag ? DSEA_ERR_INVALID_ARG : DSEA_OK;
}

int num_sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// Stages (CTAs) of a mixed-form ring launch when the caller leaves the count
// to the library.  A slice's units at one level can only run while its
// neighbours' previous level completes, so only about kSliceWarps units of a
// slice run at once usefully.  More warps mostly wait: measured on lone
// boxes of 32k-187k atoms, all 608 resident CTAs ran 20-38 % slower than
// n_slices x min(units per slice, 160) warps, while from 296k atoms on, all
// stages were as fast or faster.  The launch uses all resident stages unless
// the rule asks for at most 90 % of them.  `want_warps` is the rule summed
// over the launch's boxes; `full` the resident count.
constexpr int kSliceWarps = 160;

int64_t slice_rule_warps(const BoxDev &hb)
{
    return (int64_t)hb.n_slices * std::min<int64_t>(hb.units_per_slice, kSliceWarps);
}

int mixed_ring_ctas(int64_t want_warps, int full)
{
    const int64_t want = (want_warps + dsea::kWarps - 1) / dsea::kWarps;
    return want < (int64_t)(0.9 * full) ? (int)std::max<int64_t>(want, 1) : full;
}

// Fill the work-unit shape fields of hb for a (ty, tz) tile.
bool apply_tile(BoxDev &hb, double mean_cap, int ty, int tz)
{
    ty = std::max(1, std::min(ty, hb.nc[1]));
    tz = std::max(1, std::min(tz, hb.nc[2]));
    hb.tile_y = ty;
    hb.tile_z = tz;
    hb.tiles_y = (hb.nc[1] + ty - 1) / ty;
    hb.tiles_z = (hb.nc[2] + tz - 1) / tz;
    hb.units_per_slice = hb.tiles_y * hb.tiles_z;
    hb.staged_cells = (hb.cps + 2) * (ty + 2) * (tz + 2);
    if (hb.staged_cells > dsea::kMaxStagedCells) return false;
    // room for the expected stage plus a quarter, never more than every slot;
    // a multiple of 4
    const double expect = hb.staged_cells * mean_cap * 1.25 + 64.0;
    const double worst = (double)hb.staged_cells * hb.cap;
    hb.smem_atoms = ((int)std::ceil(std::min(expect, worst)) + 3) & ~3;
    return dsea::unit_smem_bytes(hb.precision, hb.staged_cells, hb.smem_atoms) <=
           dsea::max_unit_smem_bytes();
}

// The requested unit shape, or the largest one below it (shrinking the longer
// side first) whose stage fits one unit's shared memory; false if not even one
// cell's does.
bool fit_tile(BoxDev &hb, double mean_cap, int ty, int tz)
{
    while (!apply_tile(hb, mean_cap, ty, tz)) {
        if (ty == 1 && tz == 1) return false;
        if (tz >= ty && tz > 1) --tz;
        else --ty;
    }
    return true;
}

// Launch-filling unit shape of the mixed form, where a unit is one warp's: the
// largest of these shapes whose units per step (summed over every box of the
// launch) reach twice the warp stages the launch keeps resident (32 per SM:
// 4 CTAs of 8 warps), else the smallest.  Below about two units per stage the
// slice dependencies of the ring leave warps idle; above it a larger unit
// gathers each neighbour cell for more home cells.  On batches of 1 to 512
// boxes (3k to 11M atoms) the rule picks the fastest of the six shapes or
// one within 1.5 % of it.
constexpr int kFillShapes[][2] = {{4, 4}, {3, 3}, {2, 4}, {2, 2}, {1, 4}, {1, 2}};
constexpr int kNumFillShapes = 6;

int64_t units_with_tile(BoxDev hb, double mean_cap, int ty, int tz)
{
    if (!fit_tile(hb, mean_cap, ty, tz)) return 0;
    return (int64_t)hb.n_slices * hb.units_per_slice;
}

template <class UnitsOf>
int pick_filling_shape(UnitsOf units_of)
{
    const int64_t want = 2LL * num_sms() * 32;
    for (int ci = 0; ci < kNumFillShapes; ++ci)
        if (units_of(ci) >= want) return ci;
    return kNumFillShapes - 1;
}

int upload_desc(dsea_box *b)
{
    CU(cudaMemcpyAsync(b->db, &b->hb, sizeof(BoxDev), cudaMemcpyHostToDevice, b->stream));
    return DSEA_OK;
}

int check_device_error(dsea_box *b)
{
    if (b->latched != DSEA_OK) return b->latched;
    CU(cudaStreamSynchronize(b->stream));
    int code = 0;
    CU(cudaMemcpy(&code, b->hb.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (code != 0) b->latched = map_device_error(code);
    return b->latched;
}

int ring_launch_single(dsea_box *b, int64_t n)
{
    BoxDev &hb = b->hb;
    const int64_t U = (int64_t)hb.n_slices * hb.units_per_slice;
    if (n + 1 > b->step_base_cap) {
        // grow the plan arrays; the box keeps its old ones if an allocation fails
        const int64_t cap = std::max<int64_t>(n + 1, 1024);
        int64_t *sb = (int64_t *)dev_alloc(b, sizeof(int64_t) * cap);
        int *act = (int *)dev_alloc(b, sizeof(int) * cap);
        if (!sb || !act) {
            if (sb) dev_free(b, sb);
            if (act) dev_free(b, act);
            return DSEA_ERR_OOM;
        }
        std::vector<int> ones(cap, 1);
        const cudaError_t e = cudaMemcpyAsync(act, ones.data(), sizeof(int) * ones.size(), cudaMemcpyHostToDevice,
                                              b->stream);
        if (e == cudaSuccess) cudaStreamSynchronize(b->stream);   // `ones` is pageable and local
        if (e != cudaSuccess) {
            dev_free(b, sb);
            dev_free(b, act);
            return map_cuda(e);
        }
        if (b->d_step_base) dev_free(b, b->d_step_base);
        if (b->d_active) dev_free(b, b->d_active);
        b->d_step_base = sb;
        b->d_active = act;
        b->step_base_cap = cap;
    }
    std::vector<int64_t> sb(n + 1);
    for (int64_t s = 0; s <= n; ++s) sb[s] = s * U;
    CU(cudaMemcpyAsync(b->d_step_base, sb.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice,
                       b->stream));
    const int64_t cum[2] = {0, U};
    CU(cudaMemcpyAsync(b->d_cum, cum, sizeof(cum), cudaMemcpyHostToDevice, b->stream));
    int rc = upload_desc(b);
    if (rc) return rc;
    CU(cudaMemsetAsync(hb.done, 0, sizeof(unsigned) * 2 * hb.n_slices, b->stream));
    CU(cudaMemsetAsync(b->d_ticket, 0, sizeof(unsigned long long), b->stream));
    CU(cudaMemsetAsync(b->d_launch_err, 0, sizeof(int), b->stream));
    dsea::RingPlan plan{};
    plan.boxes = b->db;
    plan.step_base = b->d_step_base;
    plan.cum_units = b->d_cum;
    plan.active = b->d_active;
    plan.n_boxes = 1;
    plan.n_steps = (int)n;
    plan.total = n * U;
    plan.ticket = b->d_ticket;
    plan.err = b->d_launch_err;
    const size_t smem = dsea::unit_smem_bytes(hb.precision, hb.staged_cells, hb.smem_atoms);
    int ctas = b->params.ctas;
    if (ctas <= 0) {
        ctas = num_sms() * std::max(1, dsea::ring_ctas_per_sm(hb.precision, smem));
        if (hb.precision == DSEA_MIXED) ctas = mixed_ring_ctas(slice_rule_warps(hb), ctas);
    }
    if ((int64_t)ctas > plan.total) ctas = (int)plan.total;
    CU(dsea::launch_ring(plan, hb.precision, smem, ctas, b->stream));
    return DSEA_OK;
}

int advance_impl(dsea_box *b, int64_t n)
{
    BoxDev &hb = b->hb;
    if (n == 0) return DSEA_OK;
    int rc = upload_desc(b);
    if (rc) return rc;
    if (b->params.schedule == DSEA_SCHED_STEPWISE) {
        for (int64_t s = 0; s < n; ++s) {
            if (hb.T0 > 0.0)   // the thermostat's per-slice unit counts restart every step
                CU(cudaMemsetAsync(hb.done + hb.n_slices, 0, sizeof(unsigned) * hb.n_slices, b->stream));
            CU(dsea::launch_step(hb, b->db, hb.step + s, (hb.w_is_sync && s == 0) ? 1 : 0, b->stream));
        }
        hb.step += n;
        hb.w_is_sync = 0;
    } else {
        const int64_t chunk = 4096;   // bounded plan arrays per launch
        for (int64_t done = 0; done < n; done += chunk) {
            const int64_t m = std::min(chunk, n - done);
            rc = ring_launch_single(b, m);
            if (rc) return rc;
            hb.step += m;
            hb.w_is_sync = 0;
        }
    }
    b->outputs_valid = false;
    return DSEA_OK;
}

int ensure_outputs(dsea_box *b)
{
    if (b->outputs_valid) return check_device_error(b);
    BoxDev &hb = b->hb;
    if (!hb.out_r) {   // all three or none
        const size_t bytes = sizeof(double) * 3 * (size_t)std::max<int64_t>(hb.n_atoms, 1);
        double *o[3];
        for (auto &q : o) q = (double *)dev_alloc(b, bytes);
        if (!o[0] || !o[1] || !o[2]) {
            for (double *q : o)
                if (q) dev_free(b, q);
            return DSEA_ERR_OOM;
        }
        hb.out_r = o[0];
        hb.out_v = o[1];
        hb.out_f = o[2];
    }
    int rc = upload_desc(b);
    if (rc) return rc;
    CU(dsea::launch_force_pass(hb, b->db, b->stream));
    CU(dsea::launch_obs_reduce(hb.unit_obs, hb.n_cells, b->d_obs3, b->stream));
    CU(cudaMemcpyAsync(b->obs3, b->d_obs3, sizeof(b->obs3), cudaMemcpyDeviceToHost, b->stream));
    rc = check_device_error(b);
    if (rc) return rc;
    b->outputs_valid = true;
    return DSEA_OK;
}

int read_array(dsea_box *b, double *out, int64_t n)
{
    if (!b || !out || n != b->hb.n_atoms) return DSEA_ERR_INVALID_ARG;
    if (!b->registered) return DSEA_ERR_STATE;
    return ensure_outputs(b);
}

struct TuneKey {
    int occ, size, nc1, nc2, cps, cap, precision;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(occ, size, nc1, nc2, cps, cap, precision) <
               std::tie(o.occ, o.size, o.nc1, o.nc2, o.cps, o.cap, o.precision);
    }
};
// Size class of the autotuner cache.  The best unit shape depends on
// - the total number of cells (in octaves): smaller units give a small box
//   enough units to fill the GPU, larger ones save per-unit work in a big box;
// - the mean atoms per cell (in half-octaves): per-cell costs dominate dilute
//   boxes, pair work dense ones;
// - the cells per axis in the unit plane (up to 16: the edge units' share);
// - the cell layers per slice, the cell capacity and the precision.
TuneKey size_class(const int *nc, int cps, int cap, int precision, int64_t n_atoms)
{
    const double cells = (double)nc[0] * nc[1] * nc[2];
    const double mean = cells > 0 ? (double)n_atoms / cells : 0.0;
    const int occ = (int)std::floor(2.0 * std::log2(mean + 1.0));
    const int size = (int)std::floor(std::log2(std::max(cells, 1.0)));
    return TuneKey{occ, size, std::min(nc[1], 16), std::min(nc[2], 16), cps, cap, precision};
}
// A copy of the state buffers an advance reads (cell counts, IDs, positions,
// velocities, pair records of the current parity) and the step counters, so
// that timing trials leave a box as they found it.
struct BoxSnapshot {
    dsea_box *b = nullptr;
    int parity = 0;
    int64_t step0 = 0;
    int sync0 = 0;
    bool mixed = false;
    size_t b_cnt = 0, b_id = 0, b_r = 0, b_v = 0, b_q = 0;
    void *s_cnt = nullptr, *s_id = nullptr, *s_r = nullptr, *s_v = nullptr, *s_q = nullptr;

    int save(dsea_box *box)
    {
        b = box;
        const BoxDev &hb = b->hb;
        parity = (int)(hb.step & 1);
        step0 = hb.step;
        sync0 = hb.w_is_sync;
        mixed = hb.precision == DSEA_MIXED;
        b_cnt = sizeof(unsigned long long) * 2 * hb.n_cells;
        b_id = sizeof(int) * hb.n_slots;
        b_r = sizeof(double) * 3 * hb.n_slots;
        b_q = sizeof(float4) * hb.n_slots;
        b_v = (mixed ? sizeof(float) : sizeof(double)) * 3 * hb.n_slots;
        // through the box's own allocator (the caller's pool, when it gave one)
        s_cnt = dev_alloc(b, b_cnt);
        if (!mixed) s_id = dev_alloc(b, b_id);
        s_r = dev_alloc(b, b_r);
        s_v = dev_alloc(b, b_v);
        if (mixed) s_q = dev_alloc(b, b_q);
        if (!s_cnt || (!mixed && !s_id) || !s_r || !s_v || (mixed && !s_q)) {
            release();
            return DSEA_ERR_OOM;
        }
        return copy(true);
    }
    // copies back and resets the step counters; the other parity's stale
    // counts are zeroed so that they cannot match
    int restore()
    {
        b->hb.step = step0;
        b->hb.w_is_sync = sync0;
        return copy(false);
    }
    void release()
    {
        for (void *q : {s_cnt, s_id, s_r, s_v, s_q})
            if (q) dev_free(b, q);
        s_cnt = s_id = s_r = s_v = s_q = nullptr;
    }
    ~BoxSnapshot() { release(); }

  private:
    int copy(bool save)
    {
        BoxDev &hb = b->hb;
        const int p = parity;
        auto c = [&](void *snap, void *live, size_t bytes) {
            return save ? cudaMemcpyAsync(snap, live, bytes, cudaMemcpyDeviceToDevice, b->stream)
                        : cudaMemcpyAsync(live, snap, bytes, cudaMemcpyDeviceToDevice, b->stream);
        };
        cudaError_t e = c(s_cnt, hb.cnt[p], b_cnt);
        if (e == cudaSuccess && s_id) e = c(s_id, hb.id[p], b_id);
        if (e == cudaSuccess) e = c(s_r, hb.r[p], b_r);
        if (e == cudaSuccess) e = c(s_v, mixed ? (void *)hb.vf[p] : (void *)hb.v[p], b_v);
        if (e == cudaSuccess && s_q) e = c(s_q, hb.q[p], b_q);
        if (e == cudaSuccess && !save) e = cudaMemsetAsync(hb.cnt[p ^ 1], 0, b_cnt, b->stream);
        return map_cuda(e);
    }
};

std::mutex g_tune_mu;
// What the autotuner chose for a size class: the unit shape and the ring's
// stage count (0: the default rule).
struct TuneChoice {
    int ty, tz, ctas;
};
std::map<TuneKey, TuneChoice> g_tune_cache;

// Geometry, cell capacity, pair constants and work-unit shape of a box
// (Sec. 4: slices along x of width >= rc, cells of edge >= rc); validates p
// and fills in its automatic fields.
int setup_geometry(int n_slices_req, const double *L, int64_t n_atoms, dsea_params &p, BoxDev &hb,
                   double &mean_cap)
{
    if (!(p.rc > 0.0) || !(p.dt > 0.0) || !std::isfinite(p.rc) || !std::isfinite(p.dt))
        return DSEA_ERR_INVALID_ARG;
    if (p.precision != DSEA_FP64 && p.precision != DSEA_MIXED) return DSEA_ERR_INVALID_ARG;
    if (p.schedule != DSEA_SCHED_RING && p.schedule != DSEA_SCHED_STEPWISE) return DSEA_ERR_INVALID_ARG;
    if (p.tile_y < 0 || p.tile_z < 0 || p.cell_capacity < 0 || p.ctas < 0) return DSEA_ERR_INVALID_ARG;
    // geometry (Sec. 4): slices along x of width >= rc, cubic-ish cells >= rc.
    // The paper's count floor(b / rc) per axis holds at liquid density; in a
    // dilute box (below rho = 8 / rc^3, 0.51 at rc = 2.5) a cell of edge rc
    // holds one or two atoms, and every home cell pays for gathering its
    // 27-cell neighbourhood for them.  There the target edge grows to
    // (8 / rho)^(1/3), at most 1.5 rc, so that a cell holds about eight atoms
    // (more at the 1.5 rc limit's densities); the stencil stays 27 cells of
    // edge >= rc, so every pair within rc is still met exactly once per atom.
    const double vol_box = L[0] * L[1] * L[2];
    const double rho = vol_box > 0.0 ? (double)n_atoms / vol_box : 0.0;
    const double edge = rho > 0.0 ? std::min(1.5 * p.rc, std::max(p.rc, std::cbrt(12.0 / rho))) : 1.5 * p.rc;
    auto cells_along = [&](double len) {   // edge near `edge`, within [rc, 1.5 rc]; at least 3 cells
        const int n_max = (int)std::floor(len / p.rc);
        int n = std::max((int)std::floor(len / edge), (int)std::ceil(len / (1.5 * p.rc)));
        n = std::min(n, n_max);
        return std::max(n, std::min(3, n_max));
    };
    int n_s = n_slices_req, cps = 1;
    if (n_s == 0) {
        n_s = cells_along(L[0]);
    } else {
        const double w = L[0] / n_s;
        if (w < p.rc) return DSEA_ERR_INVALID_ARG;
        cps = (int)std::floor(w / edge);
        if (cps < 1 || w / cps > 1.5 * p.rc) cps = (int)std::floor(w / p.rc);   // layers no wider than 1.5 rc
    }
    const int ncy = cells_along(L[1]), ncz = cells_along(L[2]);
    if (n_s < 3 || cps < 1 || (int64_t)n_s * cps < 3 || ncy < 3 || ncz < 3) return DSEA_ERR_INVALID_ARG;
    hb.n_slices = n_s;
    hb.cps = cps;
    hb.nc[0] = n_s * cps;
    hb.nc[1] = ncy;
    hb.nc[2] = ncz;
    for (int d = 0; d < 3; ++d) {
        hb.L[d] = L[d];
        hb.lc[d] = L[d] / hb.nc[d];
        hb.inv_lc[d] = 1.0 / hb.lc[d];
        hb.lcf[d] = (float)hb.lc[d];
        hb.inv_lcf[d] = 1.0f / hb.lcf[d];
    }
    hb.n_cells = (int64_t)hb.nc[0] * hb.nc[1] * hb.nc[2];
    if (hb.n_cells >= ((int64_t)1 << 31)) return DSEA_ERR_INVALID_ARG;
    const double vol = hb.lc[0] * hb.lc[1] * hb.lc[2];
    const double mean = hb.n_cells > 0 ? (double)n_atoms / (double)hb.n_cells : 0.0;
    // a cell may hold liquid at rho ~ 0.9 even in a dilute box (phase separation)
    mean_cap = std::max(mean, 0.9 * vol);
    int cap = p.cell_capacity;
    if (cap <= 0) {
        cap = (int)std::ceil(mean_cap + 6.0 * std::sqrt(mean_cap) + 6.0);
        cap = std::max(8, cap);
    }
    cap = (cap + 3) / 4 * 4;   // slot ranges start 16-byte aligned in every per-slot array
    if (cap > 128) return DSEA_ERR_INVALID_ARG;   // a staging warp orders up to 128 arrivals
    hb.cap = cap;
    hb.n_slots = hb.n_cells * cap;
    if (hb.n_slots >= ((int64_t)1 << 31)) return DSEA_ERR_INVALID_ARG;
    hb.precision = p.precision;
    hb.rc2 = p.rc * p.rc;
    hb.rc2f = (float)hb.rc2;
    const double rc6i = 1.0 / (hb.rc2 * hb.rc2 * hb.rc2);
    hb.ushift = -4.0 * (rc6i * rc6i - rc6i);
    hb.ushiftf = (float)hb.ushift;
    hb.dt = p.dt;
    hb.step = 0;
    hb.w_is_sync = 1;
    hb.withhold_slice = -1;
    hb.wait_limit_ns = 5000000000LL;   // 5 s
    // work-unit shape: requested, cached by the autotuner, or by default the
    // launch-filling shape of the box alone (mixed form, a warp's unit) or
    // 2 x 4 home cells (FP64 form, a CTA's unit: two CTAs' staging fit one
    // SM's shared memory)
    int ty = p.tile_y, tz = p.tile_z;
    if (ty == 0 && tz == 0) {
        std::unique_lock<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(size_class(hb.nc, cps, cap, p.precision, n_atoms));
        if (it != g_tune_cache.end()) {
            ty = it->second.ty;
            tz = it->second.tz;
            if (p.ctas == 0) p.ctas = it->second.ctas;
        } else if (p.precision == DSEA_MIXED) {
            lk.unlock();
            const int ci = pick_filling_shape(
                [&](int c) { return units_with_tile(hb, mean_cap, kFillShapes[c][0], kFillShapes[c][1]); });
            ty = kFillShapes[ci][0];
            tz = kFillShapes[ci][1];
        }
    }
    ty = ty ? ty : 2;
    tz = tz ? tz : 4;
    if (!fit_tile(hb, mean_cap, ty, tz)) return DSEA_ERR_INVALID_ARG;   // one cell's stage does not fit
    p.tile_y = hb.tile_y;
    p.tile_z = hb.tile_z;
    p.cell_capacity = cap;
    hb.n_atoms = n_atoms;
    return DSEA_OK;

}


}  // namespace

namespace {

// Registration proper; dsea_register_kernel undoes it when it fails.
int register_impl(dsea_box *b, const dsea_params *params)
{
    dsea_params p{2.5, 0.005, DSEA_FP64, DSEA_SCHED_RING, 0, 0, 0, 0, 0.0};
    if (params) p = *params;
    if (!(p.temperature >= 0.0) || !std::isfinite(p.temperature)) return DSEA_ERR_INVALID_ARG;
    CU(cudaSetDevice(b->device));
    BoxDev &hb = b->hb;
    const bool tile_auto = p.tile_y == 0 && p.tile_z == 0;
    int rc0 = setup_geometry(b->n_slices_req, b->L, hb.n_atoms, p, hb, b->mean_cap);
    if (rc0) return rc0;
    b->tile_auto = tile_auto;
    hb.walls_x = b->walls_x;
    const int n_s = hb.n_slices;
    b->params = p;

    // device state
    b->db = (BoxDev *)dev_alloc(b, sizeof(BoxDev));
    hb.err = (int *)dev_alloc(b, sizeof(int));
    hb.done = (unsigned *)dev_alloc(b, sizeof(unsigned) * 2 * n_s);   // completion, thermostat counts
    const int64_t max_units = hb.n_cells;   // any tile shape has at most one unit per cell
    hb.unit_obs = (double *)dev_alloc(b, sizeof(double) * dsea::kObsStride * (size_t)max_units);
    hb.T0 = p.temperature;
    for (int q = 0; q < 2; ++q) {
        hb.th_part[q] = nullptr;
        hb.th_lam[q] = nullptr;
        if (hb.T0 > 0.0) {
            hb.th_part[q] = (double *)dev_alloc(b, sizeof(double) * 2 * (size_t)max_units);
            hb.th_lam[q] = (double *)dev_alloc(b, sizeof(double) * n_s);
            if (!hb.th_part[q] || !hb.th_lam[q]) return DSEA_ERR_OOM;
        }
    }
    b->d_obs3 = (double *)dev_alloc(b, sizeof(double) * 3);
    b->d_cum = (int64_t *)dev_alloc(b, sizeof(int64_t) * 2);
    b->d_ticket = (unsigned long long *)dev_alloc(b, sizeof(unsigned long long));
    b->d_launch_err = (int *)dev_alloc(b, sizeof(int));
    if (!b->db || !hb.err || !hb.done || !hb.unit_obs || !b->d_obs3 || !b->d_cum || !b->d_ticket ||
        !b->d_launch_err)
        return DSEA_ERR_OOM;
    for (int q = 0; q < 2; ++q) {
        // stayer and arrival counts of every cell, one allocation
        hb.cnt[q] = (unsigned long long *)dev_alloc(b, sizeof(unsigned long long) * 2 * hb.n_cells);
        hb.arr[q] = hb.cnt[q] ? hb.cnt[q] + hb.n_cells : nullptr;
        hb.r[q] = (double *)dev_alloc(b, sizeof(double) * 3 * hb.n_slots);
        hb.id[q] = nullptr;
        hb.v[q] = nullptr;
        hb.vf[q] = nullptr;
        hb.q[q] = nullptr;
        if (p.precision == DSEA_MIXED) {   // the atom id travels in q.w
            hb.vf[q] = (float *)dev_alloc(b, sizeof(float) * 3 * hb.n_slots);
            hb.q[q] = (float4 *)dev_alloc(b, sizeof(float4) * hb.n_slots);
        } else {
            hb.id[q] = (int *)dev_alloc(b, sizeof(int) * hb.n_slots);
            hb.v[q] = (double *)dev_alloc(b, sizeof(double) * 3 * hb.n_slots);
        }
        if (!hb.cnt[q] || !hb.r[q] ||
            (p.precision == DSEA_MIXED ? (!hb.vf[q] || !hb.q[q]) : (!hb.v[q] || !hb.id[q])))
            return DSEA_ERR_OOM;
        CU(cudaMemsetAsync(hb.cnt[q], 0, sizeof(unsigned long long) * 2 * hb.n_cells, b->stream));
    }
    CU(cudaMemsetAsync(hb.err, 0, sizeof(int), b->stream));
    // bin the initial atoms (copied to the device by dsea_box_create) into the
    // buffer of step 0, then release those copies
    int rc = upload_desc(b);
    if (!rc) rc = map_cuda(dsea::launch_bin(hb, b->db, b->d_pos0, b->d_vel0, b->stream));
    if (!rc) rc = check_device_error(b);
    if (rc) return rc;
    if (b->d_pos0) dev_free(b, b->d_pos0);
    if (b->d_vel0) dev_free(b, b->d_vel0);
    b->d_pos0 = b->d_vel0 = nullptr;
    b->registered = true;
    return DSEA_OK;
}

}  // namespace

extern "C" {

const char *dsea_version(void) { return "0.1.0"; }

const char *dsea_status_string(int s)
{
    switch (s) {
    case DSEA_OK: return "ok";
    case DSEA_ERR_INVALID_ARG: return "invalid argument";
    case DSEA_ERR_OOM: return "out of memory";
    case DSEA_ERR_CUDA: return "CUDA runtime error";
    case DSEA_ERR_TIMEOUT: return "bounded device wait expired";
    case DSEA_ERR_CAPACITY: return "cell capacity exceeded";
    case DSEA_ERR_MIGRATION: return "atom moved farther than one slice in a step";
    case DSEA_ERR_BUDGET: return "job exceeds the memory budget";
    case DSEA_ERR_STATE: return "call out of order";
    case DSEA_ERR_NOT_FOUND: return "unknown job";
    case DSEA_ERR_NO_DEVICE: return "no CUDA device";
    case DSEA_ERR_SCRATCH_LIMIT: return "problem exceeds the fixed no-allocation scratch";
    case DSEA_ERR_BOUNDS: return "index out of range (checked build)";
    case DSEA_ERR_RANGE: return "thermostat kinetic energy beyond its fixed-point range";
    default: return "unknown status";
    }
}

int dsea_box_create(const dsea_box_desc *desc, const dsea_allocator *allocator, void *cuda_stream,
                    dsea_box **out)
{
    NvtxRange nvtx_range("dsea_box_create");
    if (!desc || !out || desc->n_atoms < 0 || desc->n_slices < 0) return DSEA_ERR_INVALID_ARG;
    if (desc->n_atoms > 0 && !desc->pos) return DSEA_ERR_INVALID_ARG;
    if (desc->n_atoms >= (int64_t)1 << 31) return DSEA_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(desc->box[d] > 0.0) || !std::isfinite(desc->box[d])) return DSEA_ERR_INVALID_ARG;
    if (desc->boundary_x != DSEA_BOUNDARY_PERIODIC && desc->boundary_x != DSEA_BOUNDARY_MIRROR)
        return DSEA_ERR_INVALID_ARG;
    if (desc->boundary_x == DSEA_BOUNDARY_MIRROR)
        for (int64_t i = 0; i < desc->n_atoms; ++i)
            if (!(desc->pos[3 * i] >= 0.0 && desc->pos[3 * i] < desc->box[0])) return DSEA_ERR_INVALID_ARG;
    if (allocator && (!allocator->alloc || !allocator->free)) return DSEA_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return DSEA_ERR_NO_DEVICE;
    }
    dsea_box *b = new (std::nothrow) dsea_box();
    if (!b) return DSEA_ERR_OOM;
    cudaGetDevice(&b->device);
    b->stream = (cudaStream_t)cuda_stream;
    if (allocator) {
        b->alloc = *allocator;
        b->has_alloc = true;
    }
    b->n_slices_req = desc->n_slices;
    b->walls_x = desc->boundary_x == DSEA_BOUNDARY_MIRROR ? 1 : 0;
    for (int d = 0; d < 3; ++d) b->L[d] = desc->box[d];
    b->hb.n_atoms = desc->n_atoms;
    b->has_vel = desc->vel != nullptr;
    const int rc = upload_initial_state(b, desc);
    if (rc) {
        cudaStreamSynchronize(b->stream);
        dev_free_all(b);
        delete b;
        return rc;
    }
    *out = b;
    return DSEA_OK;
}

int dsea_register_kernel(dsea_box *b, int kind, int o_in, int o_out, const dsea_params *params)
{
    NvtxRange nvtx_range("dsea_register_kernel");
    if (!b) return DSEA_ERR_INVALID_ARG;
    if (b->registered) return DSEA_ERR_STATE;
    if (kind != DSEA_KERNEL_LJ_TS || o_in != 1 || o_out != 1) return DSEA_ERR_INVALID_ARG;
    // a failed registration leaves the box as dsea_box_create made it: what it
    // allocated is released and the descriptor restored, so it may be retried
    const size_t n_allocs0 = b->allocs.size();
    const BoxDev hb0 = b->hb;
    const dsea_params p0 = b->params;
    const double mean_cap0 = b->mean_cap;
    const int rc = register_impl(b, params);
    if (rc) {
        cudaStreamSynchronize(b->stream);
        cudaGetLastError();
        while (b->allocs.size() > n_allocs0) {
            const auto a = b->allocs.back();
            b->allocs.pop_back();
            dev_release(b, a.first);
            b->device_bytes -= a.second;
        }
        b->hb = hb0;
        b->params = p0;
        b->mean_cap = mean_cap0;
        b->tile_auto = false;
        b->latched = DSEA_OK;
    }
    return rc;
}


int dsea_advance(dsea_box *b, int64_t n_steps)
{
    NvtxRange nvtx_range("dsea_advance");
    if (!b || n_steps < 0) return DSEA_ERR_INVALID_ARG;
    if (!b->registered) return DSEA_ERR_STATE;
    if (b->latched) return b->latched;
    return advance_impl(b, n_steps);
}

int dsea_sync(dsea_box *b)
{
    if (!b) return DSEA_ERR_INVALID_ARG;
    if (!b->registered) return DSEA_ERR_STATE;
    return check_device_error(b);
}

int dsea_read_positions(dsea_box *b, double *out, int64_t n)
{
    NvtxRange nvtx_range("dsea_read_positions");
    int rc = read_array(b, out, n);
    if (rc) return rc;
    CU(cudaMemcpyAsync(out, b->hb.out_r, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    return DSEA_OK;
}

int dsea_read_velocities(dsea_box *b, double *out, int64_t n)
{
    NvtxRange nvtx_range("dsea_read_velocities");
    int rc = read_array(b, out, n);
    if (rc) return rc;
    CU(cudaMemcpyAsync(out, b->hb.out_v, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    return DSEA_OK;
}

int dsea_read_forces(dsea_box *b, double *out, int64_t n)
{
    NvtxRange nvtx_range("dsea_read_forces");
    int rc = read_array(b, out, n);
    if (rc) return rc;
    CU(cudaMemcpyAsync(out, b->hb.out_f, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    return DSEA_OK;
}

int dsea_read_observables(dsea_box *b, dsea_observables *out)
{
    NvtxRange nvtx_range("dsea_read_observables");
    if (!b || !out) return DSEA_ERR_INVALID_ARG;
    if (!b->registered) return DSEA_ERR_STATE;
    int rc = ensure_outputs(b);
    if (rc) return rc;
    out->step = b->hb.step;
    out->U = b->obs3[0];
    out->W = b->obs3[1];
    out->KE = b->obs3[2];
    return DSEA_OK;
}

int dsea_read_profiles(dsea_box *b, double *U, double *W, double *KE, int64_t *N, int n)
{
    NvtxRange nvtx_range("dsea_read_profiles");
    if (!b) return DSEA_ERR_INVALID_ARG;
    if (!b->registered) return DSEA_ERR_STATE;
    const BoxDev &hb = b->hb;
    if (n != hb.n_slices) return DSEA_ERR_INVALID_ARG;
    int rc = ensure_outputs(b);
    if (rc) return rc;
    // per-cell partials; slice j owns the contiguous cells of its cps x-layers
    const int64_t per_slice = (int64_t)hb.cps * hb.nc[1] * hb.nc[2];
    std::vector<double> part((size_t)dsea::kObsStride * hb.n_cells);
    CU(cudaMemcpy(part.data(), hb.unit_obs, sizeof(double) * part.size(), cudaMemcpyDeviceToHost));
    for (int j = 0; j < n; ++j) {   // the slice's cells in order
        double u = 0.0, w = 0.0, k = 0.0, c = 0.0;
        for (int64_t t = 0; t < per_slice; ++t) {
            const double *q = &part[(size_t)dsea::kObsStride * ((size_t)j * per_slice + t)];
            u += q[0];
            w += q[1];
            k += q[2];
            c += q[3];
        }
        if (U) U[j] = u;
        if (W) W[j] = w;
        if (KE) KE[j] = k;
        if (N) N[j] = (int64_t)c;
    }
    return DSEA_OK;
}

int dsea_box_get_info(const dsea_box *b, dsea_box_info *o)
{
    if (!b || !o) return DSEA_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    const BoxDev &hb = b->hb;
    o->n_atoms = hb.n_atoms;
    o->step = hb.step;
    o->boundary_x = b->walls_x ? DSEA_BOUNDARY_MIRROR : DSEA_BOUNDARY_PERIODIC;
    o->device_bytes = b->device_bytes;
    if (!b->registered) return DSEA_OK;
    o->n_slices = hb.n_slices;
    o->cells_per_slice_x = hb.cps;
    for (int d = 0; d < 3; ++d) {
        o->cells[d] = hb.nc[d];
        o->cell_edge[d] = hb.lc[d];
    }
    o->tile_y = hb.tile_y;
    o->tile_z = hb.tile_z;
    o->units_per_step = hb.n_slices * hb.units_per_slice;
    o->cell_capacity = hb.cap;
    o->precision = hb.precision;
    o->schedule = b->params.schedule;
    return DSEA_OK;
}

int dsea_box_destroy(dsea_box *b)
{
    NvtxRange nvtx_range("dsea_box_destroy");
    if (!b) return DSEA_ERR_INVALID_ARG;
    cudaStreamSynchronize(b->stream);   // nothing of the box's may still run
    dev_free_all(b);
    delete b;
    return DSEA_OK;
}

int dsea_debug_set(dsea_box *b, int key, int64_t value)
{
    if (!b || !b->registered) return DSEA_ERR_INVALID_ARG;
    switch (key) {
    case DSEA_DEBUG_WITHHOLD_SLICE: b->hb.withhold_slice = (int)value; return DSEA_OK;
    case DSEA_DEBUG_WAIT_LIMIT_NS:
        if (value <= 0) return DSEA_ERR_INVALID_ARG;
        b->hb.wait_limit_ns = value;
        return DSEA_OK;
    default: return DSEA_ERR_INVALID_ARG;
    }
}

// ---- batches ----------------------------------------------------------------

int dsea_batch_create(dsea_box *const *boxes, int n, dsea_batch **out)
{
    if (!boxes || n <= 0 || !out) return DSEA_ERR_INVALID_ARG;
    for (int k = 0; k < n; ++k) {
        if (!boxes[k] || !boxes[k]->registered) return DSEA_ERR_STATE;
        if (boxes[k]->stream != boxes[0]->stream || boxes[k]->device != boxes[0]->device ||
            boxes[k]->hb.precision != boxes[0]->hb.precision)
            return DSEA_ERR_INVALID_ARG;
        for (int q = 0; q < k; ++q)
            if (boxes[q] == boxes[k]) return DSEA_ERR_INVALID_ARG;
    }
    dsea_batch *bt = new (std::nothrow) dsea_batch();
    if (!bt) return DSEA_ERR_OOM;
    bt->boxes.assign(boxes, boxes + n);
    dsea::retile_for_launch(bt->boxes.data(), n);   // boxes on the automatic shape fill the launch together
    bt->stream = boxes[0]->stream;
    bt->precision = boxes[0]->hb.precision;
    if (cudaEventCreateWithFlags(&bt->done_ev, cudaEventDisableTiming) != cudaSuccess ||
        dsea::multi_reserve(bt->mp, n, 1024) != DSEA_OK) {
        cudaGetLastError();
        dsea_batch_destroy(bt);
        return DSEA_ERR_OOM;
    }
    *out = bt;
    return DSEA_OK;
}

int dsea_batch_advance(dsea_batch *bt, const int64_t *steps)
{
    NvtxRange nvtx_range("dsea_batch_advance");
    if (!bt || !steps) return DSEA_ERR_INVALID_ARG;
    const int n = (int)bt->boxes.size();
    int64_t smax = 0;
    for (int k = 0; k < n; ++k) {
        if (steps[k] < 0) return DSEA_ERR_INVALID_ARG;
        if (bt->boxes[k]->latched) return bt->boxes[k]->latched;
        smax = std::max(smax, steps[k]);
    }
    if (smax == 0) return DSEA_OK;
    if (smax > ((int64_t)1 << 30)) return DSEA_ERR_INVALID_ARG;
    CU(cudaEventSynchronize(bt->done_ev));   // the previous replay has read the pinned plan
    if (smax + 1 > bt->mp.cap_steps) {
        for (auto &kv : bt->graphs) cudaGraphExecDestroy(kv.second);   // they hold old buffers
        bt->graphs.clear();
        int rc = dsea::multi_reserve(bt->mp, n, smax);
        if (rc) return rc;
    }
    int rc = dsea::multi_prepare(bt->mp, bt->boxes.data(), steps, n);
    if (rc) return rc;
    std::vector<int64_t> key(2 * n + 3);
    for (int k = 0; k < n; ++k) {
        key[k] = bt->mp.order[k];
        key[n + k] = steps[bt->mp.order[k]];
    }
    key[2 * n] = (int64_t)bt->mp.smem;
    key[2 * n + 1] = bt->mp.total;   // the grid is sized by the units of the whole run
    key[2 * n + 2] = bt->mp.want_warps;   // and by the stage-count rule
    auto it = bt->graphs.find(key);
    if (it == bt->graphs.end()) {
        cudaStream_t st = bt->stream;
        bool own = false;
        if (st == nullptr) {   // the legacy stream cannot be captured: capture on a side stream
            CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            own = true;
        }
        // occupancy queries set kernel attributes: do them before capturing
        dsea::ring_ctas_per_sm(bt->precision, bt->mp.smem);
        CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int erc = dsea::multi_enqueue(bt->mp, bt->boxes.data(), st);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (own) cudaStreamDestroy(st);
        if (erc) {
            if (g) cudaGraphDestroy(g);
            return erc;
        }
        if (e != cudaSuccess) return map_cuda(e);
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return map_cuda(e);
        it = bt->graphs.emplace(key, ex).first;
    }
    CU(cudaGraphLaunch(it->second, bt->stream));
    CU(cudaEventRecord(bt->done_ev, bt->stream));
    dsea::multi_commit(bt->boxes.data(), steps, n);
    return DSEA_OK;
}

int dsea_batch_destroy(dsea_batch *bt)
{
    if (!bt) return DSEA_ERR_INVALID_ARG;
    if (bt->done_ev) {
        cudaEventSynchronize(bt->done_ev);
        cudaEventDestroy(bt->done_ev);
    }
    for (auto &kv : bt->graphs) cudaGraphExecDestroy(kv.second);
    dsea::multi_free(bt->mp);
    delete bt;
    return DSEA_OK;
}

// ---- autotuner ----------------------------------------------------------------

int dsea_autotune(dsea_box *b, int trial_steps, dsea_params *chosen)
{
    NvtxRange nvtx_range("dsea_autotune");
    if (!b || trial_steps <= 0) return DSEA_ERR_INVALID_ARG;
    if (!b->registered) return DSEA_ERR_STATE;
    int rc = check_device_error(b);
    if (rc) return rc;
    BoxDev &hb = b->hb;
    const TuneKey key = size_class(hb.nc, hb.cps, hb.cap, hb.precision, hb.n_atoms);
    TuneChoice best{hb.tile_y, hb.tile_z, b->params.ctas};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        BoxSnapshot snap;
        rc = snap.save(b);
        if (rc) return rc;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const int sched = b->params.schedule;
        const int ctas0 = b->params.ctas;
        const BoxDev saved = hb;
        b->params.schedule = DSEA_SCHED_RING;
        // one trial: a warm-up step, then trial_steps timed, then the state restored
        auto trial = [&](const BoxDev &shape, int ctas, float &ms) -> int {
            hb = shape;
            b->params.ctas = ctas;
            int r = advance_impl(b, 1);
            if (!r) {
                cudaEventRecord(e0, b->stream);
                r = advance_impl(b, trial_steps);
                cudaEventRecord(e1, b->stream);
            }
            if (!r) r = check_device_error(b);
            ms = 0;
            if (!r) cudaEventElapsedTime(&ms, e0, e1);
            const int rr = snap.restore();
            return r ? r : rr;
        };
        // 1. the unit shape (mixed units are one warp's, FP64 units one CTA's),
        //    at the default stage count
        static const int cand_mixed[][2] = {{1, 2}, {2, 2}, {1, 4}, {2, 4}, {3, 3}, {4, 4}};
        static const int cand_f64[][2] = {{2, 2}, {2, 4}, {3, 3}, {4, 4}, {4, 8}, {8, 4}, {6, 6}, {8, 8}};
        const bool tune_mixed = hb.precision == DSEA_MIXED;
        const int n_cand = tune_mixed ? 6 : 8;
        float best_ms = 1e30f;
        BoxDev best_shape = saved;
        for (int ci = 0; ci < n_cand && !rc; ++ci) {
            const int *c = tune_mixed ? cand_mixed[ci] : cand_f64[ci];
            BoxDev t = saved;
            if (!apply_tile(t, b->mean_cap, c[0], c[1])) continue;
            if (t.tile_y != c[0] || t.tile_z != c[1]) continue;   // clipped duplicate
            float ms = 0;
            rc = trial(t, 0, ms);
            if (!rc && ms < best_ms) {
                best_ms = ms;
                best_shape = t;
                best = {t.tile_y, t.tile_z, 0};
            }
        }
        // 2. the stage count at that shape: all resident stages and fractions
        //    of them against the default rule (0)
        if (!rc) {
            const size_t smem = dsea::unit_smem_bytes(best_shape.precision, best_shape.staged_cells,
                                                      best_shape.smem_atoms);
            const int full = num_sms() * std::max(1, dsea::ring_ctas_per_sm(best_shape.precision, smem));
            int tried[5] = {0, 0, 0, 0, 0};
            int n_tried = 0;
            for (int q : {4, 3, 2, 1}) {
                const int c = std::max(1, full * q / 4);
                bool dup = false;
                for (int k = 0; k < n_tried; ++k) dup = dup || tried[k] == c;
                if (dup) continue;
                tried[n_tried++] = c;
                float ms = 0;
                rc = trial(best_shape, c, ms);
                if (rc) break;
                if (ms < 0.97f * best_ms) {   // a fixed count must beat the default clearly
                    best_ms = ms;
                    best.ctas = c;
                }
            }
        }
        b->params.schedule = sched;
        b->params.ctas = ctas0;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamSynchronize(b->stream);
        snap.release();
        hb = saved;
        if (rc) return rc;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    apply_tile(hb, b->mean_cap, best.ty, best.tz);
    b->params.tile_y = hb.tile_y;
    b->params.tile_z = hb.tile_z;
    b->params.ctas = best.ctas;
    b->tile_auto = false;
    b->outputs_valid = false;
    if (chosen) *chosen = b->params;
    return DSEA_OK;
}

int dsea_batch_autotune(dsea_batch *bt, int trial_steps, int *tile_y, int *tile_z)
{
    NvtxRange nvtx_range("dsea_batch_autotune");
    if (!bt || trial_steps <= 0) return DSEA_ERR_INVALID_ARG;
    const int n = (int)bt->boxes.size();
    for (dsea_box *b : bt->boxes) {
        const int rc = check_device_error(b);
        if (rc) return rc;
    }
    std::vector<BoxSnapshot> snaps(n);
    std::vector<BoxDev> saved(n);
    for (int k = 0; k < n; ++k) {
        const int rc = snaps[k].save(bt->boxes[k]);
        if (rc) return rc;
        saved[k] = bt->boxes[k]->hb;
    }
    // the same candidates as a lone box's; every box takes the candidate,
    // shrunk where its cells or its stage do not allow it
    static const int cand_mixed[][2] = {{1, 2}, {2, 2}, {1, 4}, {2, 4}, {3, 3}, {4, 4}};
    static const int cand_f64[][2] = {{2, 2}, {2, 4}, {3, 3}, {4, 4}, {4, 8}, {8, 4}, {6, 6}, {8, 8}};
    const bool mixed = bt->precision == DSEA_MIXED;
    const int n_cand = mixed ? 6 : 8;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return DSEA_ERR_CUDA;
    }
    std::vector<int64_t> warm(n, 1), trial(n, trial_steps);
    std::pair<int, int> best{0, 0};
    float best_ms = 1e30f;
    int rc = DSEA_OK;
    for (int ci = 0; ci < n_cand && !rc; ++ci) {
        const int *c = mixed ? cand_mixed[ci] : cand_f64[ci];
        for (int k = 0; k < n && !rc; ++k) {
            dsea_box *b = bt->boxes[k];
            b->hb = saved[k];
            if (!fit_tile(b->hb, b->mean_cap, c[0], c[1])) rc = DSEA_ERR_INVALID_ARG;
        }
        if (rc) break;
        rc = dsea_batch_advance(bt, warm.data());
        if (!rc) rc = map_cuda(cudaEventRecord(e0, bt->stream));
        if (!rc) rc = dsea_batch_advance(bt, trial.data());
        if (!rc) rc = map_cuda(cudaEventRecord(e1, bt->stream));
        for (int k = 0; k < n && !rc; ++k) rc = check_device_error(bt->boxes[k]);
        float ms = 0;
        if (!rc) rc = map_cuda(cudaEventElapsedTime(&ms, e0, e1));
        for (int k = 0; k < n; ++k) {
            const int rrc = snaps[k].restore();
            if (!rc) rc = rrc;
        }
        if (!rc && ms < best_ms) {
            best_ms = ms;
            best = {c[0], c[1]};
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(bt->stream);
    for (int k = 0; k < n; ++k) {
        dsea_box *b = bt->boxes[k];
        b->hb = saved[k];
        if (!rc) {
            fit_tile(b->hb, b->mean_cap, best.first, best.second);
            b->tile_auto = false;
        }
        b->params.tile_y = b->hb.tile_y;
        b->params.tile_z = b->hb.tile_z;
        b->outputs_valid = false;
        snaps[k].release();
    }
    if (rc) return rc;
    if (tile_y) *tile_y = best.first;
    if (tile_z) *tile_z = best.second;
    return DSEA_OK;
}

// ---- schedule introspection ---------------------------------------------------

int dsea_ring_order(int n_slices, int units_per_slice, int64_t n_steps, int64_t start_step,
                    int32_t *out_slice, int32_t *out_step)
{
    if (n_slices < 3 || units_per_slice < 1 || n_steps < 0 || start_step < 0 || !out_slice || !out_step)
        return DSEA_ERR_INVALID_ARG;
    const int64_t U = (int64_t)n_slices * units_per_slice;
    for (int64_t t = 0; t < n_steps * U; ++t) {
        const int64_t s = t / U, m = t - s * U;
        const int jj = (int)(m / units_per_slice);
        out_slice[t] = dsea::ring_slice(jj, start_step + s, n_slices);
        out_step[t] = (int32_t)s;
    }
    return DSEA_OK;
}

}  // extern "C"

// ---- shared host machinery (used by batches and the server) -------------------

namespace dsea {

void retile_for_launch(dsea_box *const *boxes, int n)
{
    int64_t fixed = 0;
    bool any = false;
    for (int k = 0; k < n; ++k) {
        const dsea_box *b = boxes[k];
        if (b->tile_auto && b->hb.precision == DSEA_MIXED) any = true;
        else fixed += (int64_t)b->hb.n_slices * b->hb.units_per_slice;
    }
    if (!any) return;
    const int ci = pick_filling_shape([&](int c) {
        int64_t u = fixed;
        for (int k = 0; k < n; ++k) {
            const dsea_box *b = boxes[k];
            if (b->tile_auto && b->hb.precision == DSEA_MIXED)
                u += units_with_tile(b->hb, b->mean_cap, kFillShapes[c][0], kFillShapes[c][1]);
        }
        return u;
    });
    for (int k = 0; k < n; ++k) {
        dsea_box *b = boxes[k];
        if (!(b->tile_auto && b->hb.precision == DSEA_MIXED)) continue;
        if (fit_tile(b->hb, b->mean_cap, kFillShapes[ci][0], kFillShapes[ci][1])) {
            b->params.tile_y = b->hb.tile_y;
            b->params.tile_z = b->hb.tile_z;
        }
    }
}

void multi_free(MultiPlan &mp)
{
    if (mp.d_boxes) cudaFree(mp.d_boxes);
    if (mp.h_boxes) cudaFreeHost(mp.h_boxes);
    if (mp.d_cum) cudaFree(mp.d_cum);
    if (mp.h_cum) cudaFreeHost(mp.h_cum);
    if (mp.d_step_base) cudaFree(mp.d_step_base);
    if (mp.h_step_base) cudaFreeHost(mp.h_step_base);
    if (mp.d_active) cudaFree(mp.d_active);
    if (mp.h_active) cudaFreeHost(mp.h_active);
    if (mp.d_ticket) cudaFree(mp.d_ticket);
    if (mp.d_err) cudaFree(mp.d_err);
    mp = MultiPlan();
}

int multi_reserve(MultiPlan &mp, int n, int64_t smax)
{
    if (n <= mp.cap_boxes && smax + 1 <= mp.cap_steps) return DSEA_OK;
    const int nb = std::max(n, mp.cap_boxes);
    const int64_t ns = std::max<int64_t>(smax + 1, mp.cap_steps);
    multi_free(mp);
    bool ok = cudaMalloc(&mp.d_boxes, sizeof(BoxDev) * nb) == cudaSuccess &&
              cudaMallocHost(&mp.h_boxes, sizeof(BoxDev) * nb) == cudaSuccess &&
              cudaMalloc(&mp.d_cum, sizeof(int64_t) * (nb + 1)) == cudaSuccess &&
              cudaMallocHost(&mp.h_cum, sizeof(int64_t) * (nb + 1)) == cudaSuccess &&
              cudaMalloc(&mp.d_step_base, sizeof(int64_t) * ns) == cudaSuccess &&
              cudaMallocHost(&mp.h_step_base, sizeof(int64_t) * ns) == cudaSuccess &&
              cudaMalloc(&mp.d_active, sizeof(int) * ns) == cudaSuccess &&
              cudaMallocHost(&mp.h_active, sizeof(int) * ns) == cudaSuccess &&
              cudaMalloc(&mp.d_ticket, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&mp.d_err, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        multi_free(mp);
        return DSEA_ERR_OOM;
    }
    mp.cap_boxes = nb;
    mp.cap_steps = ns;
    return DSEA_OK;
}

int multi_prepare(MultiPlan &mp, dsea_box *const *boxes, const int64_t *steps, int n)
{
    int64_t smax = 0;
    for (int k = 0; k < n; ++k) smax = std::max(smax, steps[k]);
    int rc = multi_reserve(mp, n, smax);
    if (rc) return rc;
    // boxes with more steps first: the active boxes of each level are a prefix
    mp.order.resize(n);
    for (int k = 0; k < n; ++k) mp.order[k] = k;
    std::stable_sort(mp.order.begin(), mp.order.end(),
                     [&](int a, int c) { return steps[a] > steps[c]; });
    mp.smem = 0;
    mp.want_warps = 0;
    mp.precision = n > 0 ? boxes[0]->hb.precision : 0;
    mp.h_cum[0] = 0;
    for (int k = 0; k < n; ++k) {
        dsea_box *b = boxes[mp.order[k]];
        if (b->hb.precision != mp.precision) return DSEA_ERR_INVALID_ARG;
        mp.h_boxes[k] = b->hb;
        mp.want_warps += slice_rule_warps(b->hb);
        mp.h_cum[k + 1] = mp.h_cum[k] + (int64_t)b->hb.n_slices * b->hb.units_per_slice;
        mp.smem = std::max(mp.smem, unit_smem_bytes(b->hb.precision, b->hb.staged_cells, b->hb.smem_atoms));
    }
    int64_t total = 0;
    int act = n;
    for (int64_t s = 0; s < smax; ++s) {
        while (act > 0 && steps[mp.order[act - 1]] <= s) --act;
        mp.h_active[s] = act;
        mp.h_step_base[s] = total;
        total += mp.h_cum[act];
    }
    mp.h_step_base[smax] = total;
    mp.n = n;
    mp.smax = smax;
    mp.total = total;
    return DSEA_OK;
}

int multi_enqueue(MultiPlan &mp, dsea_box *const *boxes, cudaStream_t st)
{
    if (mp.total == 0) return DSEA_OK;
    const int n = mp.n;
    CU(cudaMemcpyAsync(mp.d_boxes, mp.h_boxes, sizeof(BoxDev) * n, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(mp.d_cum, mp.h_cum, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(mp.d_step_base, mp.h_step_base, sizeof(int64_t) * (mp.smax + 1),
                       cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(mp.d_active, mp.h_active, sizeof(int) * mp.smax, cudaMemcpyHostToDevice, st));
    for (int k = 0; k < n; ++k)
        CU(cudaMemsetAsync(boxes[k]->hb.done, 0, sizeof(unsigned) * 2 * boxes[k]->hb.n_slices, st));
    CU(cudaMemsetAsync(mp.d_ticket, 0, sizeof(unsigned long long), st));
    CU(cudaMemsetAsync(mp.d_err, 0, sizeof(int), st));
    RingPlan plan{};
    plan.boxes = mp.d_boxes;
    plan.step_base = mp.d_step_base;
    plan.cum_units = mp.d_cum;
    plan.active = mp.d_active;
    plan.n_boxes = n;
    plan.n_steps = (int)mp.smax;
    plan.total = mp.total;
    plan.ticket = mp.d_ticket;
    plan.err = mp.d_err;
    int ctas = num_sms() * std::max(1, ring_ctas_per_sm(mp.precision, mp.smem));
    if (mp.precision == DSEA_MIXED) ctas = mixed_ring_ctas(mp.want_warps, ctas);
    if ((int64_t)ctas > mp.total) ctas = (int)mp.total;
    CU(launch_ring(plan, mp.precision, mp.smem, ctas, st));
    return DSEA_OK;
}

void multi_commit(dsea_box *const *boxes, const int64_t *steps, int n)
{
    for (int k = 0; k < n; ++k) {
        if (steps[k] <= 0) continue;
        boxes[k]->hb.step += steps[k];
        boxes[k]->hb.w_is_sync = 0;
        boxes[k]->outputs_valid = false;
    }
}

int estimate_box_bytes(const dsea_box_desc *desc, const dsea_params *params, size_t *bytes)
{
    if (!desc || !bytes) return DSEA_ERR_INVALID_ARG;
    dsea_params p{2.5, 0.005, DSEA_FP64, DSEA_SCHED_RING, 0, 0, 0, 0, 0.0};
    if (params) p = *params;
    BoxDev hb{};
    double mean_cap = 0;
    int rc = setup_geometry(desc->n_slices, desc->box, desc->n_atoms, p, hb, mean_cap);
    if (rc) return rc;
    const size_t per_slot = 3 * sizeof(double) + (p.precision == DSEA_MIXED ? 3 * sizeof(float) + sizeof(float4)
                                                                            : sizeof(int) + 3 * sizeof(double));
    size_t b = 2 * ((size_t)hb.n_cells * 2 * sizeof(unsigned long long) + (size_t)hb.n_slots * per_slot);
    b += (size_t)hb.n_cells * dsea::kObsStride * sizeof(double);   // per-cell observable partials
    if (p.temperature > 0.0) b += (size_t)hb.n_cells * 4 * sizeof(double);   // thermostat partials
    b += (size_t)desc->n_atoms * 9 * sizeof(double);           // read-back arrays
    b += 64 * 1024;                                            // descriptors, counters, plans
    *bytes = b;
    return DSEA_OK;
}

int read_state(dsea_box *b, double *pos, double *vel, dsea_observables *obs)
{
    if (!b || !b->registered) return DSEA_ERR_STATE;
    int rc = ensure_outputs(b);
    if (rc) return rc;
    const size_t nb = sizeof(double) * 3 * (size_t)b->hb.n_atoms;
    if (pos) CU(cudaMemcpyAsync(pos, b->hb.out_r, nb, cudaMemcpyDeviceToHost, b->stream));
    if (vel) CU(cudaMemcpyAsync(vel, b->hb.out_v, nb, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    if (obs) {
        obs->step = b->hb.step;
        obs->U = b->obs3[0];
        obs->W = b->obs3[1];
        obs->KE = b->obs3[2];
    }
    return DSEA_OK;
}

}  // namespace dsea

namespace dsea {

int box_geometry(int n_slices, const double *L, int64_t n_atoms, dsea_params &p, BoxDev &hb)
{
    double mean_cap = 0;
    return setup_geometry(n_slices, L, n_atoms, p, hb, mean_cap);
}

}  // namespace dsea
