// dsea_dataset.cu -- the generic slice ring: any explicit per-slice kernel
// streamed over a sliced dataset in the time-skewed cyclic order (Sec. 3.1),
// with the kernel registered as in Sec. 3.3 ("caller_worker": a host launcher
// that receives 2 O_in + 1 input and 2 O_out + 1 output slice views).
//
// Every slice keeps two device buffers (step parity), so a step never
// overwrites its own inputs.  K workers are K CUDA streams; worker k runs the
// steps s = k mod K, each step sweeping all slices once in a cyclic order that
// starts (O_in + O_out) s slices further than the previous one.  Unit (j, s)
// waits, by events, for the units (j - R .. j + R, s - 1), R = O_in + O_out:
// they finalise its inputs (slices j - O_in .. j + O_in at step s) and they
// are the last readers of the buffers its outputs overwrite.  Units of one
// step run one after another on their worker's stream, so outputs shared
// between neighbouring units (O_out > 0) are never written concurrently.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "dsea_host.h"

struct dsea_dataset {
    int n_slices = 0;
    size_t slice_bytes = 0;
    int o_in = 0, o_out = 0, n_workers = 1;
    int device = 0;
    cudaStream_t user_stream = nullptr;
    dsea_allocator alloc{};
    bool has_alloc = false;
    std::vector<void *> buf[2];          // [parity][slice]
    std::vector<cudaStream_t> workers;
    std::vector<cudaEvent_t> ev[2];      // [parity of the step][slice]: unit done
    cudaEvent_t start_ev = nullptr;
    dsea_slice_fn fn = nullptr;
    void *user = nullptr;
    int64_t step = 0;                    // steps completed
    bool have_prev = false;              // events of step - 1 were recorded by a run
};

namespace {

int wrapi(int64_t i, int n)
{
    int64_t r = i % n;
    return (int)(r < 0 ? r + n : r);
}

void *ds_alloc(dsea_dataset *d, size_t bytes)
{
    void *p = nullptr;
    if (d->has_alloc) {
        p = d->alloc.alloc(bytes, d->alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void ds_free(dsea_dataset *d, void *p)
{
    if (!p) return;
    if (d->has_alloc) d->alloc.free(p, d->alloc.ctx);
    else cudaFree(p);
}

// Slice swept at position i of step s (relative to the dataset's first step).
int sweep_slice(int i, int64_t s, int n, int R)
{
    return wrapi((int64_t)i + (int64_t)R * s, n);
}

}  // namespace

extern "C" {

int dsea_dataset_plan(int n_slices, int o_in, int o_out, int n_workers, int64_t n_steps, int64_t start_step,
                      int32_t *out_slice, int64_t *out_step, int32_t *out_worker)
{
    if (n_slices < 1 || o_in < 0 || o_out < 0 || n_workers < 1 || n_steps < 0 || start_step < 0)
        return DSEA_ERR_INVALID_ARG;
    if (2 * (o_in + o_out) + 1 > n_slices) return DSEA_ERR_INVALID_ARG;
    if (n_steps > 0 && (!out_slice || !out_step || !out_worker)) return DSEA_ERR_INVALID_ARG;
    const int R = o_in + o_out;
    int64_t k = 0;
    for (int64_t s = start_step; s < start_step + n_steps; ++s)
        for (int i = 0; i < n_slices; ++i, ++k) {
            out_slice[k] = sweep_slice(i, s, n_slices, R);
            out_step[k] = s;
            out_worker[k] = (int32_t)(s % n_workers);
        }
    return DSEA_OK;
}

int dsea_dataset_create(int n_slices, size_t slice_bytes, int o_in, int o_out, int n_workers,
                        const dsea_allocator *allocator, void *cuda_stream, dsea_dataset **out)
{
    if (!out || n_slices < 1 || slice_bytes == 0 || o_in < 0 || o_out < 0 || n_workers < 1 || n_workers > 64)
        return DSEA_ERR_INVALID_ARG;
    if (2 * (o_in + o_out) + 1 > n_slices) return DSEA_ERR_INVALID_ARG;   // distinct views
    if (allocator && (!allocator->alloc || !allocator->free)) return DSEA_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return DSEA_ERR_NO_DEVICE;
    }
    dsea_dataset *d = new (std::nothrow) dsea_dataset();
    if (!d) return DSEA_ERR_OOM;
    cudaGetDevice(&d->device);
    d->n_slices = n_slices;
    d->slice_bytes = slice_bytes;
    d->o_in = o_in;
    d->o_out = o_out;
    d->n_workers = n_workers;
    d->user_stream = (cudaStream_t)cuda_stream;
    if (allocator) {
        d->alloc = *allocator;
        d->has_alloc = true;
    }
    bool ok = true;
    for (int q = 0; q < 2 && ok; ++q) {
        d->buf[q].assign(n_slices, nullptr);
        d->ev[q].assign(n_slices, nullptr);
        for (int j = 0; j < n_slices && ok; ++j) {
            d->buf[q][j] = ds_alloc(d, slice_bytes);
            ok = d->buf[q][j] && cudaMemsetAsync(d->buf[q][j], 0, slice_bytes, d->user_stream) == cudaSuccess &&
                 cudaEventCreateWithFlags(&d->ev[q][j], cudaEventDisableTiming) == cudaSuccess;
        }
    }
    d->workers.assign(n_workers, nullptr);
    for (int k = 0; k < n_workers && ok; ++k)
        ok = cudaStreamCreateWithFlags(&d->workers[k], cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&d->start_ev, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        dsea_dataset_destroy(d);
        return DSEA_ERR_OOM;
    }
    *out = d;
    return DSEA_OK;
}

int dsea_dataset_write_slice(dsea_dataset *d, int slice, const void *host, size_t bytes)
{
    if (!d || !host || slice < 0 || slice >= d->n_slices || bytes != d->slice_bytes) return DSEA_ERR_INVALID_ARG;
    if (cudaSetDevice(d->device) != cudaSuccess) return DSEA_ERR_CUDA;
    for (auto s : d->workers)
        if (cudaStreamSynchronize(s) != cudaSuccess) return DSEA_ERR_CUDA;
    if (cudaMemcpyAsync(d->buf[d->step & 1][slice], host, bytes, cudaMemcpyHostToDevice, d->user_stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(d->user_stream) != cudaSuccess)
        return DSEA_ERR_CUDA;
    return DSEA_OK;
}

int dsea_dataset_read_slice(dsea_dataset *d, int slice, void *host, size_t bytes)
{
    if (!d || !host || slice < 0 || slice >= d->n_slices || bytes != d->slice_bytes) return DSEA_ERR_INVALID_ARG;
    if (cudaSetDevice(d->device) != cudaSuccess) return DSEA_ERR_CUDA;
    for (auto s : d->workers)
        if (cudaStreamSynchronize(s) != cudaSuccess) return DSEA_ERR_CUDA;
    if (cudaMemcpy(host, d->buf[d->step & 1][slice], bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return DSEA_ERR_CUDA;
    return DSEA_OK;
}

int dsea_dataset_register(dsea_dataset *d, dsea_slice_fn fn, void *user)
{
    if (!d || !fn) return DSEA_ERR_INVALID_ARG;
    d->fn = fn;
    d->user = user;
    return DSEA_OK;
}

int dsea_dataset_run(dsea_dataset *d, int64_t n_steps)
{
    NvtxRange nvtx_range("dsea_dataset_run");
    if (!d || n_steps < 0) return DSEA_ERR_INVALID_ARG;
    if (!d->fn) return DSEA_ERR_STATE;
    if (n_steps == 0) return DSEA_OK;
    if (cudaSetDevice(d->device) != cudaSuccess) return DSEA_ERR_CUDA;
    const int n = d->n_slices, R = d->o_in + d->o_out;
    const int nin = 2 * d->o_in + 1, nout = 2 * d->o_out + 1;
    std::vector<const void *> in(nin);
    std::vector<void *> out(nout);
    // every worker starts after the work already queued on the caller's stream
    if (cudaEventRecord(d->start_ev, d->user_stream) != cudaSuccess) return DSEA_ERR_CUDA;
    for (auto s : d->workers)
        if (cudaStreamWaitEvent(s, d->start_ev, 0) != cudaSuccess) return DSEA_ERR_CUDA;
    int rc = DSEA_OK;
    for (int64_t s = d->step; s < d->step + n_steps && rc == DSEA_OK; ++s) {
        cudaStream_t st = d->workers[s % d->n_workers];
        const int pin = (int)(s & 1), pout = pin ^ 1;
        for (int i = 0; i < n && rc == DSEA_OK; ++i) {
            const int j = sweep_slice(i, s, n, R);
            if (s > d->step || d->have_prev) {
                // the units j - R .. j + R of step s - 1 ran one after another on one
                // stream: waiting for the one swept last covers all of them
                int last = wrapi(j - R, n), last_i = -1;
                for (int dlt = -R; dlt <= R; ++dlt) {
                    const int jj = wrapi(j + dlt, n);
                    const int ii = wrapi((int64_t)jj - (int64_t)R * (s - 1), n);   // its sweep position
                    if (ii > last_i) {
                        last_i = ii;
                        last = jj;
                    }
                }
                if (cudaStreamWaitEvent(st, d->ev[pout][last], 0) != cudaSuccess) rc = DSEA_ERR_CUDA;
            }
            for (int k = 0; k < nin; ++k) in[k] = d->buf[pin][wrapi(j - d->o_in + k, n)];
            for (int k = 0; k < nout; ++k) out[k] = d->buf[pout][wrapi(j - d->o_out + k, n)];
            if (rc == DSEA_OK) {
                const int urc = d->fn(d->user, j, s, in.data(), out.data(), d->slice_bytes, (void *)st);
                if (urc != 0) rc = urc < 0 ? urc : DSEA_ERR_CUDA;
            }
            if (rc == DSEA_OK && cudaEventRecord(d->ev[pin][j], st) != cudaSuccess) rc = DSEA_ERR_CUDA;
        }
    }
    // the caller's stream waits for every worker
    for (auto s : d->workers) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return DSEA_ERR_CUDA;
        cudaEventRecord(e, s);
        cudaStreamWaitEvent(d->user_stream, e, 0);
        cudaEventDestroy(e);
    }
    if (rc != DSEA_OK) return rc;
    d->step += n_steps;
    d->have_prev = true;
    return cudaGetLastError() == cudaSuccess ? DSEA_OK : DSEA_ERR_CUDA;
}

int64_t dsea_dataset_step(const dsea_dataset *d)
{
    return d ? d->step : -1;
}

int dsea_dataset_destroy(dsea_dataset *d)
{
    if (!d) return DSEA_ERR_INVALID_ARG;
    cudaSetDevice(d->device);
    for (auto s : d->workers)
        if (s) cudaStreamSynchronize(s);
    for (int q = 0; q < 2; ++q) {
        for (void *p : d->buf[q]) ds_free(d, p);
        for (cudaEvent_t e : d->ev[q])
            if (e) cudaEventDestroy(e);
    }
    for (auto s : d->workers)
        if (s) cudaStreamDestroy(s);
    if (d->start_ev) cudaEventDestroy(d->start_ev);
    cudaGetLastError();
    delete d;
    return DSEA_OK;
}

}  // extern "C"

// ---- a slice kernel shipped with the library: explicit 1D heat equation -----

namespace {

// One explicit step of u_t = u_xx on a periodic rod cut into equal slices:
// u'[i] = u[i] + a (u[i-1] - 2 u[i] + u[i+1]), a = dt / dx^2, the end values
// coming from the neighbouring slices (O_in = 1).  FP32 with explicit
// roundings (no contraction), so the result matches a plain CPU evaluation
// bit for bit; 8 bytes of memory traffic per point and step.
__global__ void k_heat1d(const float *left, const float *mid, const float *right, float *out, long long m, float a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const float ul = i > 0 ? mid[i - 1] : left[m - 1];
        const float ur = i + 1 < m ? mid[i + 1] : right[0];
        const float u = mid[i];
        const float lap = __fadd_rn(__fsub_rn(ul, __fmul_rn(2.0f, u)), ur);
        out[i] = __fadd_rn(u, __fmul_rn(a, lap));
    }
}

// The same step, four points per float4 (m a multiple of 4, 16-byte aligned
// views): the values left and right of a quad are single loads that mostly
// hit L1, and each thread keeps two quads in flight.
__device__ __forceinline__ float heat_point(float ul, float u, float ur, float a)
{
    return __fadd_rn(u, __fmul_rn(a, __fadd_rn(__fsub_rn(ul, __fmul_rn(2.0f, u)), ur)));
}

__device__ __forceinline__ void heat_quad(const float *left, const float *mid, const float *right, float *out,
                                          long long m, long long q, float a)
{
    const float4 u = reinterpret_cast<const float4 *>(mid)[q];
    const long long i = 4 * q;
    const float ul = i > 0 ? mid[i - 1] : left[m - 1];
    const float ur = i + 4 < m ? mid[i + 4] : right[0];
    reinterpret_cast<float4 *>(out)[q] = make_float4(heat_point(ul, u.x, u.y, a), heat_point(u.x, u.y, u.z, a),
                                                     heat_point(u.y, u.z, u.w, a), heat_point(u.z, u.w, ur, a));
}

__global__ void k_heat1d_v4(const float *left, const float *mid, const float *right, float *out, long long m,
                            float a)
{
    const long long n4 = m >> 2, stride = (long long)gridDim.x * blockDim.x;
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; q + stride < n4; q += 2 * stride) {
        heat_quad(left, mid, right, out, m, q, a);
        heat_quad(left, mid, right, out, m, q + stride, a);
    }
    if (q < n4) heat_quad(left, mid, right, out, m, q, a);
}

}  // namespace

extern "C" int dsea_example_heat1d(void *user, int slice, int64_t step, const void *const *in, void *const *out,
                                   size_t slice_bytes, void *stream)
{
    (void)slice;
    (void)step;
    if (!user || !in || !out || slice_bytes % sizeof(float) != 0) return DSEA_ERR_INVALID_ARG;
    const float a = *static_cast<const float *>(user);
    const long long m = (long long)(slice_bytes / sizeof(float));
    const float *l = static_cast<const float *>(in[0]), *c = static_cast<const float *>(in[1]),
                *r = static_cast<const float *>(in[2]);
    float *o = static_cast<float *>(out[0]);
    const int threads = 256;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long full = (long long)std::max(sms, 1) * 8;   // 8 CTAs of 256 fill an SM
    const bool quads = m % 4 == 0 && (reinterpret_cast<uintptr_t>(c) & 15) == 0 &&
                       (reinterpret_cast<uintptr_t>(o) & 15) == 0;
    if (quads) {
        const long long blocks = std::min<long long>((m / 4 + threads - 1) / threads, full);
        k_heat1d_v4<<<(int)std::max<long long>(blocks, 1), threads, 0, (cudaStream_t)stream>>>(l, c, r, o, m, a);
    } else {
        const long long blocks = std::min<long long>((m + threads - 1) / threads, full);
        k_heat1d<<<(int)std::max<long long>(blocks, 1), threads, 0, (cudaStream_t)stream>>>(l, c, r, o, m, a);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : DSEA_ERR_CUDA;
}
