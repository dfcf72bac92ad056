// dsea_noalloc.cu -- forces and observables of one configuration without any
// device allocation.
//
// Some callers cannot let a library call cudaMalloc: a host that hands all
// device memory to one arena up front (a framework's pool or a scheduler's
// fixed reservation) and rejects allocations it did not make, or a
// latency-bound loop where cudaMalloc / cudaFree would synchronise the device
// and stall every other stream.  For them, dsea_forces_noalloc runs the same
// binning and force-pass kernels as a box does, but takes all of its scratch
// (cell slots, counts, per-cell partials, the box descriptor) from one fixed,
// file-scope device array instead of allocating it.  The caller passes the
// inputs and outputs.
//
// The array is kScratchBytes (64 MiB) on every GPU that loads the library,
// held until the process exits.  Every call shares it, and it keeps the last
// call's contents: the counts that must start at zero are cleared on every
// call, and calls that overlap on the GPU (other streams, other host threads)
// race on it.
#include "dsea_host.h"

#include <mutex>

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of this GPU's copy of the scratch array.  On the first call
// on a device (that device current) this asks the runtime for the symbol's
// address; later calls reuse it.
int scratch_base(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return DSEA_ERR_NO_DEVICE;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return DSEA_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DSEA_OK;
}

}  // namespace

extern "C" int dsea_forces_noalloc(const double *pos_dev, const double *vel_dev, int64_t n_atoms,
                                   const double *box, double rc, int precision, double *forces_dev,
                                   double *obs3_dev, void *cuda_stream)
{
    NvtxRange nvtx_range("dsea_forces_noalloc");
    if (n_atoms < 0 || !box || (n_atoms > 0 && (!pos_dev || !forces_dev))) return DSEA_ERR_INVALID_ARG;
    if (n_atoms >= ((int64_t)1 << 31)) return DSEA_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    dsea_params p{rc, 0.005, precision, DSEA_SCHED_STEPWISE, 0, 0, 0, 0, 0.0};
    dsea::BoxDev hb{};
    int rc0 = dsea::box_geometry(0, box, n_atoms, p, hb);
    if (rc0) return rc0;
    // carve the scratch: descriptor, error word, counts, slots, partials, read-back
    const size_t n3 = 3 * (size_t)(n_atoms > 0 ? n_atoms : 1);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += up256(bytes);
        return at;
    };
    const size_t o_desc = take(sizeof(dsea::BoxDev));
    const size_t o_err = take(sizeof(int));
    const size_t o_cnt = take(sizeof(unsigned long long) * 2 * hb.n_cells);   // stayers, arrivals
    const size_t o_id = precision == DSEA_MIXED ? 0 : take(sizeof(int) * hb.n_slots);
    const size_t o_r = take(sizeof(double) * 3 * hb.n_slots);
    const size_t o_v = take((precision == DSEA_MIXED ? sizeof(float) : sizeof(double)) * 3 * hb.n_slots);
    const size_t o_q = precision == DSEA_MIXED ? take(sizeof(float4) * hb.n_slots) : 0;
    const size_t o_obs = take(sizeof(double) * dsea::kObsStride * (size_t)hb.n_cells);   // per-cell partials
    const size_t o_outr = take(sizeof(double) * n3);
    const size_t o_outv = take(sizeof(double) * n3);
    if (off > kScratchBytes) return DSEA_ERR_SCRATCH_LIMIT;
    void *base_v = nullptr;
    rc0 = scratch_base(&base_v);
    if (rc0) return rc0;
    unsigned char *base = static_cast<unsigned char *>(base_v);
    dsea::BoxDev *db = reinterpret_cast<dsea::BoxDev *>(base + o_desc);
    hb.err = reinterpret_cast<int *>(base + o_err);
    for (int q = 0; q < 2; ++q) {   // one configuration: step 0 uses buffer 0 only
        hb.cnt[q] = reinterpret_cast<unsigned long long *>(base + o_cnt);
        hb.arr[q] = hb.cnt[q] + hb.n_cells;
        hb.id[q] = precision == DSEA_MIXED ? nullptr : reinterpret_cast<int *>(base + o_id);
        hb.r[q] = reinterpret_cast<double *>(base + o_r);
        hb.v[q] = precision == DSEA_MIXED ? nullptr : reinterpret_cast<double *>(base + o_v);
        hb.vf[q] = precision == DSEA_MIXED ? reinterpret_cast<float *>(base + o_v) : nullptr;
        hb.q[q] = precision == DSEA_MIXED ? reinterpret_cast<float4 *>(base + o_q) : nullptr;
    }
    hb.unit_obs = reinterpret_cast<double *>(base + o_obs);
    hb.out_r = reinterpret_cast<double *>(base + o_outr);
    hb.out_v = reinterpret_cast<double *>(base + o_outv);
    hb.out_f = forces_dev;
    hb.done = nullptr;
    hb.step = 0;
    hb.w_is_sync = 1;
    hb.withhold_slice = -1;
    hb.wait_limit_ns = 5000000000LL;
    // the scratch keeps the previous call's contents: clear what must start at zero
    cudaError_t e = cudaMemsetAsync(hb.cnt[0], 0, sizeof(unsigned long long) * 2 * hb.n_cells, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(hb.err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(db, &hb, sizeof(hb), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = dsea::launch_bin(hb, db, pos_dev, vel_dev, st);
    if (e == cudaSuccess) e = dsea::launch_force_pass(hb, db, st);
    if (e == cudaSuccess && obs3_dev) e = dsea::launch_obs_reduce(hb.unit_obs, hb.n_cells, obs3_dev, st);
    // the status word comes back on the caller's stream, and only that stream
    // is waited for (a plain cudaMemcpy would also wait for every blocking
    // stream of the device)
    int code = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&code, hb.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DSEA_ERR_CUDA;
    }
    switch (code) {
    case 0: return DSEA_OK;
    case dsea::kErrCapacity: return DSEA_ERR_CAPACITY;
    case dsea::kErrMigration: return DSEA_ERR_MIGRATION;
    case dsea::kErrTimeout: return DSEA_ERR_TIMEOUT;
    default: return DSEA_ERR_CUDA;
    }
}
