// dsea_kernels.cu -- sm_103a kernels of the slice-streamed LJ NVE step.
//
// A work unit is the home cells of one slice (its cps cell layers along x)
// within a tile_y x tile_z block of cells in (y, z).  For every home cell the
// step computes the force on each home atom from the 27 neighbour cells
// (Algorithm 1's first loop, Sec. 4.1 "md_v3a"), then kicks and drifts the
// atom (Algorithm 1's second and third loops, "md_v3aa" / "md_v3b") and
// writes it to the cell it moved to in the next-step buffer, which may belong
// to slice j-1, j or j+1 (O_out = 1, Sec. 4).  Every per-atom sum runs in an
// order fixed by the box state alone (neighbour cells in a fixed order, each
// cell's atoms in its canonical order), so results do not depend on the unit
// shape, the launch form or the batch.
//
// The FP64 form runs a unit per CTA: it stages the unit's neighbourhood into
// shared memory as absolute positions and evaluates pairs in FP64.
//
// The mixed form runs a unit per warp: for each home cell the warp gathers
// the 27-cell neighbourhood into a flat list of FP32 coordinates in the home
// cell's centred frame and evaluates pairs in packed FP32x2 arithmetic;
// velocities are FP32; the absolute positions, their update and every
// reduction stay FP64 (FP64 issues at a small fraction of the FP32 rate on
// this GPU, so the mixed form spends about a dozen FP64 operations per
// atom-step).
#include "dsea_internal.h"

namespace dsea {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void set_error(int *err, int code)
{
    atomicCAS(err, 0, code);
}

// Checked build (DSEA_CHECKED): whether 0 <= i < n, recording kErrBounds when
// not, so that the caller skips the access.  Always true in the release build.
__device__ __forceinline__ bool idx_ok(int *err, long long i, long long n)
{
#if DSEA_CHECKED
    if (i < 0 || i >= n) {
        set_error(err, kErrBounds);
        return false;
    }
#else
    (void)err; (void)i; (void)n;
#endif
    return true;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_int(const int *p)
{
    return *reinterpret_cast<const volatile int *>(p);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Asynchronous 16-byte global -> shared copy that bypasses L1 (.cg), so data
// other SMs wrote earlier in the same persistent launch is always seen (L1 is
// not kept coherent with other SMs' writes).  Both addresses 16-B aligned.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// floor(a / d) for 0 <= a < 2^22 through the FP32 reciprocal inv_d = 1/d
// (a few instructions instead of an integer division).  Exact: (a + 1/2)/d
// lies at least 1/(2d) away from an integer, far above the rounding error.
__device__ __forceinline__ int qdiv(int a, float inv_d)
{
    return (int)(((float)a + 0.5f) * inv_d);
}

__device__ __forceinline__ float inv_of(int d)
{
    return __frcp_rn((float)d);
}

// Shared-memory carve-up of one FP64 unit.
struct Layout {
    size_t cnt, nst, start, gcell, atoms, atomsf, id, slot, scr, queue, red, cellke, lam, band, ctr, total;
};

// Depth of the per-lane queue of in-range candidates in the FP64 pair loop.
constexpr int kQueueDepth = 32;

__host__ __device__ inline Layout make_layout(int staged_cells, int smem_atoms)
{
    Layout L;
    size_t o = 0;
    L.cnt = o;   o += sizeof(int) * staged_cells;
    L.nst = o;   o += sizeof(int) * staged_cells;   // stayers of each staged cell
    L.start = o; o += sizeof(int) * (staged_cells + 1);
    L.gcell = o; o += sizeof(int) * staged_cells;
    o = align16(o);
    L.atoms = o; o += 3 * sizeof(double) * smem_atoms;   // x[], y[], z[]
    L.atomsf = o; o += 3 * sizeof(float) * smem_atoms;   // FP32 copies relative to the unit's corner
    L.id = o;    o += sizeof(int) * smem_atoms;
    L.slot = o;  o += sizeof(int) * smem_atoms;
    o = align16(o);
    L.scr = o;   o += sizeof(double) * kThreads * 5;     // partial sums of split home atoms
    L.queue = o; o += sizeof(int) * kThreads * kQueueDepth;   // queued in-range candidates
    L.red = o;   o += sizeof(double) * kWarps * 4;
    L.cellke = o; o += sizeof(double) * 2 * staged_cells;   // thermostat: (KE, N) per home cell
    L.lam = o;   o += 16;
    L.band = o;  o += 16;                               // FP32 pre-test thresholds
    L.ctr = o;   o += 16;
    L.total = align16(o);
    return L;
}

__device__ __forceinline__ int wrap_index(int i, int n)
{
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

// The slice thermostat sums kinetic energies in fixed point, so that a
// slice's total is the same however its cells are grouped into units (unit
// shape, stage count, batch, server launch): each chunk of at most 32 home
// atoms sums its atoms' FP64 energies in canonical order, rounds the sum to
// a multiple of 2^-40 epsilon (4.5e-13 at most per chunk), and the
// multiples add as integers, exactly.  A chunk of 1024 epsilon or more (32
// epsilon per atom, a temperature near 21) is out of range, and so is a
// unit whose int64 sum would overflow: kErrRange.  Slice totals are summed
// in 128 bits.
constexpr double kKeScale = 1099511627776.0;   // 2^40 per epsilon
constexpr double kKeChunkMax = 1024.0;          // 2^10 epsilon

__device__ __forceinline__ long long ke_fixed(double ke, int *err)
{
    if (!(ke >= 0.0 && ke < kKeChunkMax)) {
        set_error(err, kErrRange);
        return 0;
    }
    return __double2ll_rn(ke * kKeScale);
}

// acc += v for non-negative fixed-point energies, or kErrRange on overflow.
__device__ __forceinline__ void ke_add(long long &acc, long long v, int *err)
{
    if (acc > 0x7fffffffffffffffLL - v) set_error(err, kErrRange);
    else acc += v;
}

// Butterfly sum of a 128-bit integer over the warp: the same total in every lane.
__device__ __forceinline__ __int128 warp_sum_i128(__int128 v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((unsigned __int128)v >> 64);
        const unsigned long long lo2 = __shfl_xor_sync(kFull, lo, o), hi2 = __shfl_xor_sync(kFull, hi, o);
        v += (__int128)(((unsigned __int128)hi2 << 64) | lo2);
    }
    return v;
}

// The slice thermostat's factor for slice j at step s_abs + 1 (Sec. 4.1,
// md_thermo_a/b): sqrt(T0 / T'), with T' = 2 lp^2 KE / (3 N) the slice's
// temperature after step s_abs's scaling by lp, KE and N summed exactly over
// the fixed-point partials the slice's units wrote at step s_abs (the KE
// word holds an int64).  Warp-wide; every lane returns the factor.
__device__ __forceinline__ double slice_lambda_next(const BoxDev &B, int j, long long s_abs, double lp, int lane)
{
    const int q = (int)(s_abs & 1);
    const int ups = B.units_per_slice;
    const double *part = B.th_part[q] + 2LL * j * ups;
    __int128 kef = 0;
    long long n = 0;
    // eight partials per lane in flight at once: one L2 round trip, not eight
    for (int t0 = lane; t0 < ups; t0 += 32 * 8) {
        double kv[8], nv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int t = t0 + 32 * k;
            kv[k] = t < ups ? __ldcg(part + 2 * t) : 0.0;
            nv[k] = t < ups ? __ldcg(part + 2 * t + 1) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            kef += (__int128)__double_as_longlong(kv[k]);
            n += (long long)nv[k];
        }
    }
    kef = warp_sum_i128(kef);
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(kFull, n, o);
    const double ke = (double)kef / kKeScale;
    const double ke_after = lp * lp * ke;
    return (n > 0 && ke_after > 0.0) ? sqrt(B.T0 * 3.0 * (double)n / (2.0 * ke_after)) : 1.0;
}

// The factor of slice j at step s_abs: 1 at the first step, else the value
// the slice's last unit of the previous step published (slice_publish).
__device__ __forceinline__ double slice_factor(const BoxDev &B, int j, long long s_abs, bool first_step)
{
    return first_step ? 1.0 : __ldcg(B.th_lam[(int)(s_abs & 1)] + j);
}

// After a unit of slice j at relative level s_rel of this launch (step
// s_abs, factor lam) wrote its partial: count it on the slice's counter
// (after the per-slice completion counters in `done`); the level's last unit
// computes the factor of step s_abs + 1 from all the partials and publishes
// it before its own completion is counted, so the next level's units, which
// wait for that completion, find it.  One computation per slice and step
// instead of one per unit.  Warp-wide.
__device__ __forceinline__ void slice_publish(const BoxDev &B, int j, long long s_abs, int s_rel, double lam,
                                              int lane)
{
    unsigned last = 0;
    if (lane == 0 && idx_ok(B.err, j, B.n_slices)) {
        __threadfence();   // this unit's partial before the count
        const unsigned want = (unsigned)B.units_per_slice * (unsigned)(s_rel + 1);
        last = atomicAdd(B.done + B.n_slices + j, 1u) + 1u == want ? 1u : 0u;
    }
    last = __shfl_sync(kFull, last, 0);
    if (!last) return;
    __threadfence();   // the other units' partials, counted before this one
    const double l = slice_lambda_next(B, j, s_abs, lam, lane);
    if (lane == 0) {
        B.th_lam[(int)((s_abs + 1) & 1)][j] = l;
        __threadfence();
    }
    __syncwarp();
}

// Force accumulators of one lane (FP64 form).
struct Acc64 {
    double fx, fy, fz, u, w;
};

// Packed FP32x2 arithmetic (sm_100+): two pairs' worth of FP32 work per
// issued instruction, each half rounded exactly as its scalar counterpart.
#define DSEA_F2_OP(NAME, OP)                                                                \
    __device__ __forceinline__ float2 NAME(float2 a, float2 b)                              \
    {                                                                                       \
        float2 d;                                                                           \
        asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2,%3};\n\tmov.b64 rb, {%4,%5};\n\t" OP \
            " rd, ra, rb;\n\tmov.b64 {%0,%1}, rd;}"                                         \
            : "=f"(d.x), "=f"(d.y)                                                          \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                      \
        return d;                                                                           \
    }
DSEA_F2_OP(f2add, "add.rn.f32x2")
DSEA_F2_OP(f2sub, "sub.rn.f32x2")
DSEA_F2_OP(f2mul, "mul.rn.f32x2")
#undef DSEA_F2_OP

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2,%3};\n\tmov.b64 rb, {%4,%5};\n\t"
        "mov.b64 rc, {%6,%7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0,%1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ float2 f2splat(float x) { return make_float2(x, x); }

// Unrolling of the mixed form's pair loop over the neighbour list.
#ifndef DSEA_PAIR_UNROLL_N
#define DSEA_PAIR_UNROLL_N 2
#endif
#define DSEA_PRAGMA(x) _Pragma(#x)
#define DSEA_UNROLL(n) DSEA_PRAGMA(unroll n)

// 0 < r2 <= rc2 on the bit patterns of non-negative floats (excludes the atom
// itself, at r2 == 0, in the same test as the cutoff).
__device__ __forceinline__ bool in_cutoff(float r2, unsigned rc2_bits)
{
    return (__float_as_uint(r2) - 1u) < rc2_bits;
}

// 1.0f if a <= b, else 0.0f (one instruction; multiplies a force to zero
// beyond the cutoff).
__device__ __forceinline__ float le_mask(float a, float b)
{
    float d;
    asm("set.le.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// Neighbour pruning (both forms): a candidate farther than the cutoff from
// the bounding box of the home atoms a warp evaluates is out of range of all
// of them.  The test runs in FP32 with these margins, far above its rounding.
constexpr float kFarAway = 1.0e4f;            // coordinate of a padding entry (never within the cutoff)
constexpr float kBoxMargin = 1.0e-4f;         // widening of the home atoms' bounding box
constexpr float kReachMargin = 1.0e-3f;       // widening of rc^2

// A signed integer that orders as the float f does (finite f; -0 just
// below +0), and back: positive floats order as their bit patterns, negative
// ones in reverse, so the magnitude bits of negatives are flipped.
__device__ __forceinline__ int ordered_int(float f)
{
    const int i = __float_as_int(f);
    return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float ordered_float(int i)
{
    return __int_as_float(i ^ ((i >> 31) & 0x7fffffff));
}

// Squared distance from (x, y, z) to the box [lo, hi] (0 inside).
__device__ __forceinline__ float box_dist2(float x, float y, float z, const float lo[3], const float hi[3])
{
    const float dx = fmaxf(fmaxf(lo[0] - x, x - hi[0]), 0.f);
    const float dy = fmaxf(fmaxf(lo[1] - y, y - hi[1]), 0.f);
    const float dz = fmaxf(fmaxf(lo[2] - z, z - hi[2]), 0.f);
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Warp-wide bounding box of the points held by lanes with `own` set (empty:
// lo > hi), widened by kBoxMargin.
__device__ __forceinline__ void warp_box(bool own, float x, float y, float z, float lo[3], float hi[3])
{
    const float c[3] = {x, y, z};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lo[d] = ordered_float(__reduce_min_sync(kFull, ordered_int(own ? c[d] : kFarAway))) - kBoxMargin;
        hi[d] = ordered_float(__reduce_max_sync(kFull, ordered_int(own ? c[d] : -kFarAway))) + kBoxMargin;
    }
}

// Accumulators of the two home atoms a lane carries (packed halves).
struct Acc2 {
    float2 fx, fy, fz, u, w;
};

// Two candidate pairs at once in packed FP32x2: half 0 of (XS, YS, ZS) against
// half 0 of (XJ, YJ, ZJ), half 1 against half 1.  EXACT: the cutoff test
// also excludes r2 == 0 (an atom against itself; needed in the home cell)
// and masks the energy terms; otherwise the force is masked by multiplying
// with the 0/1 cutoff mask, which gives the same bits for every pair of
// distinct atoms.
template <bool EXACT, bool OBS>
__device__ __forceinline__ void pair2(const float2 XS, const float2 YS, const float2 ZS, const float2 XJ,
                                      const float2 YJ, const float2 ZJ, float rc2f, unsigned rcb, float ushiftf,
                                      Acc2 &a)
{
    const float2 DX = f2sub(XS, XJ);
    const float2 DY = f2sub(YS, YJ);
    const float2 DZ = f2sub(ZS, ZJ);
    const float2 R2 = f2fma(DZ, DZ, f2fma(DY, DY, f2mul(DX, DX)));
    const float2 R2I = make_float2(rcp_approx(R2.x), rcp_approx(R2.y));
    const float2 A = f2mul(R2I, R2I);
    const float2 R6 = f2mul(A, R2I);
    // F_abs = 24 (2 r^-12 - r^-6) / r^2 = r^-8 (48 r^-6 - 24)
    float2 FS = f2mul(f2mul(A, A), f2fma(R6, f2splat(48.f), f2splat(-24.f)));
    bool in0 = true, in1 = true;
    if (EXACT) {
        in0 = in_cutoff(R2.x, rcb);
        in1 = in_cutoff(R2.y, rcb);
        FS.x = in0 ? FS.x : 0.f;
        FS.y = in1 ? FS.y : 0.f;
    } else {
        FS = f2mul(FS, make_float2(le_mask(R2.x, rc2f), le_mask(R2.y, rc2f)));
    }
    a.fx = f2fma(DX, FS, a.fx);
    a.fy = f2fma(DY, FS, a.fy);
    a.fz = f2fma(DZ, FS, a.fz);
    if (OBS) {
        // 4 (r^-12 - r^-6) + U_shift, and r_ij . F_ij
        float2 u = f2fma(f2mul(f2splat(4.f), R6), f2add(R6, f2splat(-1.f)), f2splat(ushiftf));
        u.x = in0 ? u.x : 0.f;
        u.y = in1 ? u.y : 0.f;
        a.u = f2add(a.u, u);
        a.w = f2fma(R2, FS, a.w);
    }
}

// The force terms of one pair in range, in FP64 on absolute (periodically
// shifted) positions.
template <bool OBS>
__device__ __forceinline__ void pair_f64(double xi, double yi, double zi, double xj, double yj,
                                         double zj, double ushift, Acc64 &a)
{
    const double dx = xi - xj, dy = yi - yj, dz = zi - zj;
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double r2i = 1.0 / r2;
    const double r6i = r2i * r2i * r2i;
    const double fs = 24.0 * (2.0 * r6i * r6i - r6i) * r2i;
    a.fx += dx * fs;
    a.fy += dy * fs;
    a.fz += dz * fs;
    if (OBS) {
        a.u += 4.0 * (r6i * r6i - r6i) + ushift;
        a.w += r2 * fs;
    }
}

// Whether a candidate pair counts: within the (inclusive) cutoff and not the
// atom itself; the same r2 as pair_f64 computes.
__device__ __forceinline__ bool in_range_f64(double xi, double yi, double zi, double xj, double yj, double zj,
                                             double rc2)
{
    const double dx = xi - xj, dy = yi - yj, dz = zi - zj;
    const double r2 = dx * dx + dy * dy + dz * dz;
    return r2 <= rc2 && r2 > 0.0;
}

// Reserve one slot per active lane in cell `dest` of the next-step buffer;
// lanes with the same destination share one compare-and-swap (warp
// aggregation).  Returns the slot index within the cell, or -1 for inactive
// lanes.
__device__ __forceinline__ int reserve_slot(unsigned long long *cnt, long long dest, bool active,
                                            unsigned tag, int lane, int *err)
{
    const long long key = active ? dest : -1 - (long long)lane;
    const unsigned grp = __match_any_sync(kFull, key);
    const int leader = __ffs(grp) - 1;
    const int rank = __popc(grp & ((1u << lane) - 1u));
    int base = 0;
    if (active && lane == leader) {
        const unsigned gsize = __popc(grp);
        unsigned long long *p = cnt + dest;
        unsigned long long old = *reinterpret_cast<volatile unsigned long long *>(p);
        int tries = 0;
        while (true) {
            const unsigned c = ((unsigned)(old >> 32) == tag) ? (unsigned)old : 0u;
            const unsigned long long nv = ((unsigned long long)tag << 32) | (unsigned long long)(c + gsize);
            const unsigned long long prev = atomicCAS(p, old, nv);
            if (prev == old) {
                base = (int)c;
                break;
            }
            old = prev;
            if (++tries > (1 << 20)) {   // lock-free, so this never triggers in practice
                set_error(err, kErrTimeout);
                base = 1 << 29;
                break;
            }
        }
    }
    base = __shfl_sync(kFull, base, leader);
    return active ? base + rank : -1;
}

// Slot in the next-step buffer for each active lane's atom, whose new cell is
// `dest`; `hcell` is the home cell the warp processes.  Atoms that stay take
// the next front slots of their cell in the order the warp processes them
// (the cell's canonical order), counted in n_stay (warp-uniform); atoms that
// move reserve the next back slot of their new cell through its arrival
// counter.  Returns -1 for inactive lanes and on overflow (error set).
__device__ __forceinline__ long long place_slot(const BoxDev &B, int pn, long long hcell, long long dest,
                                                bool own, unsigned tag, int lane, int &n_stay)
{
    const bool stay = own && dest == hcell;
    const unsigned bs = __ballot_sync(kFull, stay);
    const int k_stay = n_stay + __popc(bs & ((1u << lane) - 1u));
    n_stay += __popc(bs);
    // most chunks have no atom that changes cell: skip the reservation then
    const int k = __any_sync(kFull, own && !stay) ? reserve_slot(B.arr[pn], dest, own && !stay, tag, lane, B.err)
                                                  : -1;
    if (!own) return -1;
    if (stay) return hcell * B.cap + k_stay;   // stayers never outnumber the cell's atoms
    if (k >= B.cap) {
        set_error(B.err, kErrCapacity);
        return -1;
    }
    return dest * B.cap + (B.cap - 1 - k);
}

// Write one atom into slot `slot` of buffer `pn` (FP64 form).
__device__ __forceinline__ void store_f64(const BoxDev &B, int pn, long long slot, int aid, double x,
                                          double y, double z, double vx, double vy, double vz)
{
    const long long S = B.n_slots;
    if (!idx_ok(B.err, slot, S)) return;
    B.id[pn][slot] = aid;
    B.r[pn][slot] = x;
    B.r[pn][S + slot] = y;
    B.r[pn][2 * S + slot] = z;
    B.v[pn][slot] = vx;
    B.v[pn][S + slot] = vy;
    B.v[pn][2 * S + slot] = vz;
}

// Write one atom into slot `slot` of buffer `pn` (mixed form): FP64 position
// relative to its cell centre, FP32 velocity, FP32 copy of the position with
// the atom id in .w.
__device__ __forceinline__ void store_mixed(const BoxDev &B, int pn, long long slot, int aid, double x,
                                            double y, double z, float vx, float vy, float vz, float qx,
                                            float qy, float qz)
{
    const long long S = B.n_slots;
    if (!idx_ok(B.err, slot, S)) return;
    B.r[pn][slot] = x;
    B.r[pn][S + slot] = y;
    B.r[pn][2 * S + slot] = z;
    B.vf[pn][slot] = vx;
    B.vf[pn][S + slot] = vy;
    B.vf[pn][2 * S + slot] = vz;
    B.q[pn][slot] = make_float4(qx, qy, qz, __int_as_float(aid));
}

__device__ __forceinline__ double wrap_coord(double x, double L)
{
    if (x >= L) x -= L;
    else if (x < 0.0) x += L;
    if (x >= L) x -= L;        // x = -tiny rounds to L: fold back to 0
    if (x < 0.0) x = 0.0;
    return x;
}

__device__ __forceinline__ int cell_of(double x, double inv_lc, int n)
{
    int c = (int)(x * inv_lc);
    return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

// Destination of a mixed-form atom along one axis.  The atom sat in cell cg
// at FP64 position r relative to that cell's centre (FP32 copy q) and moves
// by d (FP32).  The cell offset is decided in FP32; r becomes the FP64
// position relative to the destination cell's centre and qn its FP32 copy.
// Returns the destination cell, wrapped periodically (a relative position
// needs no wrap), or, with `mirror`, reflected at the walls of the axis:
// unwrapped cell u < 0 becomes -1 - u, u >= nc becomes 2 nc - 1 - u, and
// the relative position changes sign (the caller reverses the velocity).
// Three FP64 operations in the common case.
__device__ __forceinline__ int move_axis(double &r, float q, float d, int cg, double lc, float inv_lcf, int nc,
                                         bool mirror, float &qn, bool &reflected)
{
    const int o = (int)floorf(fmaf(q + d, inv_lcf, 0.5f));   // cell offset, usually -1, 0 or 1
    double rn = r + (double)d;                               // FP64 position update
    if (o != 0) rn -= (double)o * lc;                        // rebase on the new cell's centre
    int c = cg + o;
    reflected = mirror && (c < 0 || c >= nc);
    if (reflected) {
        c = c < 0 ? -1 - c : 2 * nc - 1 - c;
        rn = -rn;
    }
    r = rn;
    qn = (float)rn;
    c = c < 0 ? c + nc : (c >= nc ? c - nc : c);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// The FP64 work unit.  One CTA = all home cells of one slice (its cps cell
// layers along x) within a tile_y x tile_z block of cells in (y, z).  It
//   1. stages the counts of its neighbourhood cells (home cells plus one cell
//      layer around them, periodic) and an exclusive scan of them,
//   2. stages the atoms of those cells into shared memory in each cell's
//      canonical order (stayers in slot order, then arrivals by atom id), as
//      absolute positions shifted to the periodic image next to the unit,
//      with FP32 copies relative to the unit's corner,
//   3. computes, warp per home cell, the force on each home atom from the 27
//      neighbour cells (Algorithm 1's first loop, Sec. 4.1 "md_v3a"): per
//      neighbour cell the candidates near the home atoms' bounding box, their
//      cutoff tests settled in FP32 where provably exact, the force terms of
//      the pairs in range queued per lane and evaluated on full warps,
//   4. (INTEGRATE) kicks and drifts each home atom (Algorithm 1's second and
//      third loops) and writes it to the cell it moved to in the next-step
//      buffer, which may belong to slice j-1, j or j+1 (O_out = 1, Sec. 4),
//   5. (OBS) reduces U, W and KE of its home atoms in FP64 ("stat_collect").
// s_abs: absolute step of the input state.
template <bool INTEGRATE, bool OBS>
__device__ void run_unit_f64(const BoxDev &B, int j, int tile, long long s_abs, bool first_step,
                             int s_rel, char *smem)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int p = (int)(s_abs & 1);
    const unsigned tag = (unsigned)(s_abs + 1);
    const Layout Ly = make_layout(B.staged_cells, B.smem_atoms);
    int *s_cnt = reinterpret_cast<int *>(smem + Ly.cnt);
    int *s_nst = reinterpret_cast<int *>(smem + Ly.nst);
    int *s_start = reinterpret_cast<int *>(smem + Ly.start);
    int *s_gcell = reinterpret_cast<int *>(smem + Ly.gcell);
    int *s_slot = reinterpret_cast<int *>(smem + Ly.slot);
    double *s_cellke = reinterpret_cast<double *>(smem + Ly.cellke);
    double *s_lam = reinterpret_cast<double *>(smem + Ly.lam);
    float *s_band = reinterpret_cast<float *>(smem + Ly.band);
    int *s_ctr = reinterpret_cast<int *>(smem + Ly.ctr);
    const bool thermo = INTEGRATE && B.T0 > 0.0;   // uniform across the CTA
    double *s_x = reinterpret_cast<double *>(smem + Ly.atoms);
    double *s_y = s_x + B.smem_atoms;
    double *s_z = s_y + B.smem_atoms;
    float *s_xf = reinterpret_cast<float *>(smem + Ly.atomsf);
    float *s_yf = s_xf + B.smem_atoms;
    float *s_zf = s_yf + B.smem_atoms;
    int *s_id = reinterpret_cast<int *>(smem + Ly.id);

    // unit geometry
    const int tyi = qdiv(tile, inv_of(B.tiles_z)), tzi = tile - tyi * B.tiles_z;
    const int y0 = tyi * B.tile_y, z0 = tzi * B.tile_z;
    const int ny = min(B.tile_y, B.nc[1] - y0), nz = min(B.tile_z, B.nc[2] - z0);
    const int x0 = j * B.cps, nx = B.cps;
    const int EY = ny + 2, EZ = nz + 2;
    const int n_staged = (nx + 2) * EY * EZ;
    const float inv_eyez = inv_of(EY * EZ), inv_ez = inv_of(EZ), inv_nynz = inv_of(ny * nz),
                inv_nz = inv_of(nz), inv_cps = inv_of(B.cps);

    // 1. counts of the staged cells
    if (tid == 0) {
        *s_ctr = 0;
        // the pair loop's FP32 pre-test: band, rc2 + band, rc2 - band (see there)
        const double E = fmax((nx + 2) * B.lc[0], fmax((ny + 2) * B.lc[1], (nz + 2) * B.lc[2]));
        const double band = 4.0 * (6.0 * sqrt(B.rc2) * E + 3.0 * B.rc2) * 0x1p-24;
        s_band[0] = (float)band;
        s_band[1] = (float)(B.rc2 + band);
        s_band[2] = (float)(B.rc2 - band);
    }
    for (int k = tid; k < n_staged; k += kThreads) {
        const int lx = qdiv(k, inv_eyez), rem = k - lx * EY * EZ, ly = qdiv(rem, inv_ez), lz = rem - ly * EZ;
        const int gx = wrap_index(x0 - 1 + lx, B.nc[0]);
        const int gy = wrap_index(y0 - 1 + ly, B.nc[1]);
        const int gz = wrap_index(z0 - 1 + lz, B.nc[2]);
        const int gc = (gx * B.nc[1] + gy) * B.nc[2] + gz;
        const bool beyond = (B.walls_x && (x0 - 1 + lx < 0 || x0 - 1 + lx >= B.nc[0])) ||   // past a wall
                            !idx_ok(B.err, gc, B.n_cells);
        const unsigned long long ws = beyond ? 0ull : __ldcg(B.cnt[p] + gc);
        const unsigned long long wa = beyond ? 0ull : __ldcg(B.arr[p] + gc);
        int n_s = ((unsigned)(ws >> 32) == tag) ? (int)(unsigned)ws : 0;   // stayers (front)
        int n_a = ((unsigned)(wa >> 32) == tag) ? (int)(unsigned)wa : 0;   // arrivals (back)
        if (n_s + n_a > B.cap) {   // the two ends met: the cell overflowed
            set_error(B.err, kErrCapacity);
            n_s = min(n_s, B.cap);
            n_a = B.cap - n_s;
        }
        s_cnt[k] = n_s + n_a;
        s_nst[k] = n_s;
        s_gcell[k] = gc;
    }
    __syncthreads();
    // 2. exclusive scan (warp 0, contiguous chunks per lane)
    if (warp == 0) {
        const int per = (n_staged + 31) / 32;
        const int b = lane * per, e = min(b + per, n_staged);
        int sum = 0;
        for (int k = b; k < e; ++k) sum += s_cnt[k];
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        int run = incl - sum;
        for (int k = b; k < e; ++k) {
            s_start[k] = run;
            run += s_cnt[k];
        }
        if (lane == 31) s_start[n_staged] = incl;
    }
    __syncthreads();
    if (s_start[n_staged] > B.smem_atoms) {   // uniform across the CTA
        if (tid == 0) set_error(B.err, kErrCapacity);
        return;
    }
    // 3. stage atoms in each cell's canonical order: the stayers (front
    // slots) as they are, then the arrivals (back slots) ordered by atom id
    const long long S = B.n_slots;
    // the unit's lower corner in the staged frame: FP32 copies relative to it
    // serve the exact-by-construction cutoff pre-test of the pair loop
    const double ref_x = (x0 - 1) * B.lc[0], ref_y = (y0 - 1) * B.lc[1], ref_z = (z0 - 1) * B.lc[2];
    for (int k = warp; k < n_staged; k += kWarps) {
        const int c = s_cnt[k];
        if (c == 0) continue;
        const int n_s = s_nst[k], n_a = c - n_s;
        const long long base = (long long)s_gcell[k] * B.cap;
        const int st = s_start[k];
        // periodic image shift of this staged cell
        const int lx = qdiv(k, inv_eyez), rem = k - lx * EY * EZ, ly = qdiv(rem, inv_ez), lz = rem - ly * EZ;
        const int ux = x0 - 1 + lx, uy = y0 - 1 + ly, uz = z0 - 1 + lz;
        const double shx = ux < 0 ? -B.L[0] : (ux >= B.nc[0] ? B.L[0] : 0.0);
        const double shy = uy < 0 ? -B.L[1] : (uy >= B.nc[1] ? B.L[1] : 0.0);
        const double shz = uz < 0 ? -B.L[2] : (uz >= B.nc[2] ? B.L[2] : 0.0);
        for (int a = lane; a < n_s; a += 32) {
            const long long slot = base + a;
            s_slot[st + a] = (int)slot;
            const double x = __ldcg(B.r[p] + slot) + shx, y = __ldcg(B.r[p] + S + slot) + shy,
                         z = __ldcg(B.r[p] + 2 * S + slot) + shz;
            s_x[st + a] = x;
            s_y[st + a] = y;
            s_z[st + a] = z;
            s_xf[st + a] = (float)(x - ref_x);
            s_yf[st + a] = (float)(y - ref_y);
            s_zf[st + a] = (float)(z - ref_z);
            s_id[st + a] = __ldcg(B.id[p] + slot);
        }
        if (n_a == 0) continue;
        // arrivals: rank by atom id among themselves (up to 4 per lane)
        const int fa = st + n_s;                      // staged position of the first arrival
        const long long abase = base + B.cap - n_a;   // slot of the first arrival
        if (n_a > 128) {
            if (lane == 0) set_error(B.err, kErrCapacity);
            continue;
        }
        const int nm = (n_a + 31) >> 5;
        int idm[4];
        double xm[4], ym[4], zm[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int a = lane + 32 * m;
            idm[m] = 0x7fffffff;
            if (m < nm && a < n_a) {
                const long long slot = abase + a;
                xm[m] = __ldcg(B.r[p] + slot) + shx;
                ym[m] = __ldcg(B.r[p] + S + slot) + shy;
                zm[m] = __ldcg(B.r[p] + 2 * S + slot) + shz;
                idm[m] = __ldcg(B.id[p] + slot);
            }
        }
        int rk[4] = {0, 0, 0, 0};
#pragma unroll
        for (int mb = 0; mb < 4; ++mb) {
            if (mb < nm) {
                const int lim = min(32, n_a - 32 * mb);
                for (int t = 0; t < lim; ++t) {
                    const int o = __shfl_sync(kFull, idm[mb], t);
#pragma unroll
                    for (int m = 0; m < 4; ++m)
                        if (m < nm) rk[m] += (o < idm[m]) ? 1 : 0;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int a = lane + 32 * m;
            if (m < nm && a < n_a) {
                const int dst = fa + rk[m];
                s_slot[dst] = (int)(abase + a);
                s_x[dst] = xm[m];
                s_y[dst] = ym[m];
                s_z[dst] = zm[m];
                s_xf[dst] = (float)(xm[m] - ref_x);
                s_yf[dst] = (float)(ym[m] - ref_y);
                s_zf[dst] = (float)(zm[m] - ref_z);
                s_id[dst] = idm[m];
            }
        }
    }
    if (thermo && tid == 0) *s_lam = slice_factor(B, j, s_abs, first_step);   // this step's factor
    __syncthreads();

    // 4./5. forces, then kick, drift and rebin, warp per home cell.  Without
    // a reduction the home cells are handed out dynamically; with one, in a
    // fixed order so that the unit's partial sums are reproducible.
    double red_u = 0.0, red_w = 0.0, red_k = 0.0, red_n = 0.0;
    const int n_home = nx * ny * nz;
    const int pn = p ^ 1;
    const double lam = thermo ? *s_lam : 1.0;
    const unsigned tag_next = tag + 1u;
    const double dt = B.dt;
    const double kick = first_step ? 0.5 * dt : dt;
    int h = OBS ? warp : 0;
    if (!OBS) {
        if (lane == 0) h = atomicAdd(s_ctr, 1);
        h = __shfl_sync(kFull, h, 0);
    }
    while (h < n_home) {
        const int hx = qdiv(h, inv_nynz), hr = h - hx * ny * nz, hy = qdiv(hr, inv_nz), hz = hr - hy * nz;
        const int kh = ((hx + 1) * EY + (hy + 1)) * EZ + (hz + 1);
        const int n_i = s_cnt[kh];
        const int hs = s_start[kh];
        const long long hcell = s_gcell[kh];
        int n_stay = 0;   // atoms of this cell that stay in it, written to its front slots in order
        long long cell_ke = 0;   // thermostat: the cell's KE before scaling, fixed point
        for (int ib = 0; ib < n_i; ib += 32) {
            const int nin = min(32, n_i - ib);
            const float inv_nin = inv_of(nin);
            const int ns = qdiv(32, inv_nin);
            const int g = qdiv(lane, inv_nin), li = lane - g * nin;
            const bool act = g < ns;
            const int is = hs + ib + li;
            const bool own = lane < nin;
            long long slot = 0;
            if (own) slot = s_slot[is];
            if (own && !idx_ok(B.err, slot, B.n_slots)) slot = 0;   // checked build: read a valid slot
            Acc64 a64 = {0.0, 0.0, 0.0, 0.0, 0.0};
            // The warp's scratch (32 x 5 doubles) holds, during the pair loop, the
            // pruned list of one neighbour cell (ints 0..127) and the chunk's
            // bounding box in FP32 relative to its first atom (box at float 192,
            // reference atom at double 104), re-read per cell to spare registers.
            int *plist = reinterpret_cast<int *>(smem + Ly.scr) + warp * 32 * 10;
            float *s_box = reinterpret_cast<float *>(plist) + 192;
            double *s_ref = reinterpret_cast<double *>(plist) + 104;
            {
                const double xr = s_x[hs + ib], yr = s_y[hs + ib], zr = s_z[hs + ib];
                const int ih = hs + ib + (own ? lane : 0);
                float lo[3], hi[3];
                warp_box(own, (float)(s_x[ih] - xr), (float)(s_y[ih] - yr), (float)(s_z[ih] - zr), lo, hi);
                if (lane == 0) {
                    for (int d = 0; d < 3; ++d) {
                        s_box[d] = lo[d];
                        s_box[3 + d] = hi[d];
                    }
                    s_ref[0] = xr;
                    s_ref[1] = yr;
                    s_ref[2] = zr;
                }
                __syncwarp();
            }
            const double xi = act ? s_x[is] : 0.0, yi = act ? s_y[is] : 0.0, zi = act ? s_z[is] : 0.0;
            // Candidates are tested first; a lane queues the staged index of each
            // one in range and, once some lane's queue is full, the warp evaluates
            // the queued force terms, each lane in its own candidate order.  So
            // the FP64 force arithmetic runs on (nearly) full warps, not once per
            // candidate trip in which any lane has a pair in range.
            int *myq = reinterpret_cast<int *>(smem + Ly.queue) + warp * 32 * kQueueDepth + lane;
            int nq = 0;
            // FP32 pre-test.  The FP32 coordinates (|x| <= E, the unit's extent)
            // carry an error of at most E 2^-24 each and the FP32 subtraction
            // adds at most |d| 2^-24, so near the cutoff (|d_k| <= r <= rc) each
            // component is off by at most (2E + rc) 2^-24; squaring and summing
            // (sum |d_k| <= sqrt(3) r) gives 2 sqrt(3) rc (2E + rc) 2^-24, and the
            // three roundings of r2 add 3 rc^2 2^-24: to first order the FP32 r2
            // is within (6.93 rc E + 6.47 rc^2) 2^-24 of the FP64 one.  The band
            // is 4 (6 rc E + 3 rc^2) 2^-24 = (24 rc E + 12 rc^2) 2^-24: more than
            // 1.8 times that at any E, three times at the extents of a unit (E
            // of three cells or more).  Outside (band, rc2 - band) and above rc2 + band
            // the FP64 test would decide the same way; in between it decides.
            const float xif = act ? s_xf[is] : 0.f, yif = act ? s_yf[is] : 0.f, zif = act ? s_zf[is] : 0.f;
            auto drain = [&]() {
                const int nmax = __reduce_max_sync(kFull, nq);
                for (int i = 0; i < nmax; ++i)
                    if (i < nq) {
                        const int q = myq[32 * i];
                        pair_f64<OBS>(xi, yi, zi, s_x[q], s_y[q], s_z[q], B.ushift, a64);
                    }
                nq = 0;
            };
            auto offer = [&](bool valid, int q) {   // warp-wide: every lane calls it
                if (valid) {
                    const float dx = xif - s_xf[q], dy = yif - s_yf[q], dz = zif - s_zf[q];
                    const float r2f = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    bool in;
                    if (r2f > s_band[1]) in = false;
                    else if (r2f < s_band[2] && r2f > s_band[0]) in = true;
                    else in = in_range_f64(xi, yi, zi, s_x[q], s_y[q], s_z[q], B.rc2);
                    if (in) myq[32 * nq++] = q;
                }
                if (__any_sync(kFull, nq == kQueueDepth)) drain();
            };
            for (int ox = -1; ox <= 1; ++ox)
                for (int oy = -1; oy <= 1; ++oy)
                    for (int oz = -1; oz <= 1; ++oz) {
                        const int kn = ((hx + 1 + ox) * EY + (hy + 1 + oy)) * EZ + (hz + 1 + oz);
                        const int cs = s_start[kn], cn = s_cnt[kn];
                        if (kn == kh) {   // the home cell: every atom
                            for (int b = 0; b < cn; b += ns) offer(act && b + g < cn, cs + b + g);
                            continue;
                        }
                        // the cell's atoms within the cutoff of the box, in order (at most
                        // cap <= 128 of them); the others would all fail the cutoff test
                        int m = 0;
                        for (int t0 = 0; t0 < cn; t0 += 32) {
                            const int t = t0 + lane;
                            bool keep = false;
                            if (t < cn) {
                                const volatile float *vb = s_box;
                                const volatile double *vr = s_ref;
                                const float lo[3] = {vb[0], vb[1], vb[2]}, hi[3] = {vb[3], vb[4], vb[5]};
                                keep = box_dist2((float)(s_x[cs + t] - vr[0]), (float)(s_y[cs + t] - vr[1]),
                                                 (float)(s_z[cs + t] - vr[2]), lo, hi) <=
                                       B.rc2f + kReachMargin;
                            }
                            const unsigned kept = __ballot_sync(kFull, keep);
                            if (keep) plist[m + __popc(kept & ((1u << lane) - 1u))] = cs + t;
                            m += __popc(kept);
                        }
                        __syncwarp();
                        for (int b = 0; b < m; b += ns) {
                            const bool v = act && b + g < m;
                            offer(v, v ? plist[b + g] : 0);
                        }
                        __syncwarp();   // the queue holds staged indices: plist may be rewritten
                    }
            drain();
            // combine the ns partial sums of each home atom in split order
            double fx = a64.fx, fy = a64.fy, fz = a64.fz, uu = a64.u, ww = a64.w;
            if (ns > 1) {
                double *scr = reinterpret_cast<double *>(smem + Ly.scr) + warp * 32 * 5;
                scr[lane * 5 + 0] = a64.fx; scr[lane * 5 + 1] = a64.fy; scr[lane * 5 + 2] = a64.fz;
                scr[lane * 5 + 3] = a64.u;  scr[lane * 5 + 4] = a64.w;
                __syncwarp();
                if (g == 0) {
                    for (int gg = 1; gg < ns; ++gg) {
                        const int o = (li + gg * nin) * 5;
                        fx += scr[o]; fy += scr[o + 1]; fz += scr[o + 2]; uu += scr[o + 3]; ww += scr[o + 4];
                    }
                }
                __syncwarp();
            }
            int aid = 0;
            double rx = 0, ry = 0, rz = 0, vx = 0, vy = 0, vz = 0;
            if (own) {
                aid = s_id[is];
                rx = __ldcg(B.r[p] + slot);
                ry = __ldcg(B.r[p] + S + slot);
                rz = __ldcg(B.r[p] + 2 * S + slot);
                vx = __ldcg(B.v[p] + slot);
                vy = __ldcg(B.v[p] + S + slot);
                vz = __ldcg(B.v[p] + 2 * S + slot);
                if (OBS) {
                    const double hk = first_step ? 0.0 : 0.5 * dt;
                    const double sx = vx + hk * fx, sy = vy + hk * fy, sz = vz + hk * fz;
                    red_u += 0.5 * uu;
                    red_w += 0.5 * ww;
                    red_k += 0.5 * (sx * sx + sy * sy + sz * sz);
                    red_n += 1.0;
                    if (!INTEGRATE && idx_ok(B.err, aid, B.n_atoms)) {
                        const long long o = 3LL * aid;
                        B.out_f[o] = fx; B.out_f[o + 1] = fy; B.out_f[o + 2] = fz;
                        B.out_v[o] = sx; B.out_v[o + 1] = sy; B.out_v[o + 2] = sz;
                        B.out_r[o] = rx; B.out_r[o + 1] = ry; B.out_r[o + 2] = rz;
                    }
                }
            }
            if (thermo) {
                // synchronised v(t) = v(t - dt/2) + F dt/2 (v(t0) itself at the start), its KE,
                // then v(t + dt/2) = lam v(t) + F dt/2 (md_v3b)
                double ke = 0.0;
                if (own) {
                    const double hk = first_step ? 0.0 : 0.5 * dt;
                    const double sx = vx + hk * fx, sy = vy + hk * fy, sz = vz + hk * fz;
                    ke = 0.5 * (sx * sx + sy * sy + sz * sz);
                    vx = lam * sx + 0.5 * dt * fx;
                    vy = lam * sy + 0.5 * dt * fy;
                    vz = lam * sz + 0.5 * dt * fz;
                }
                for (int o = 16; o > 0; o >>= 1) ke += __shfl_xor_sync(kFull, ke, o);
                ke_add(cell_ke, ke_fixed(ke, B.err), B.err);
            }
            if (INTEGRATE) {
                long long dest = 0;
                if (own) {
                    if (!thermo) {
                        vx += kick * fx;   // v(t + dt/2) = v(t - dt/2) + F dt
                        vy += kick * fy;
                        vz += kick * fz;
                    }
                    rx += vx * dt;   // r(t + dt) = r(t) + v(t + dt/2) dt
                    if (B.walls_x && (rx < 0.0 || rx >= B.L[0])) {   // mirror at the wall
                        rx = rx < 0.0 ? -rx : 2.0 * B.L[0] - rx;
                        vx = -vx;
                    }
                    rx = wrap_coord(rx, B.L[0]);
                    ry = wrap_coord(ry + vy * dt, B.L[1]);
                    rz = wrap_coord(rz + vz * dt, B.L[2]);
                    const int cx = cell_of(rx, B.inv_lc[0], B.nc[0]);
                    const int cy = cell_of(ry, B.inv_lc[1], B.nc[1]);
                    const int cz = cell_of(rz, B.inv_lc[2], B.nc[2]);
                    const int dj = qdiv(cx, inv_cps) - j;
                    const int djm = dj < -1 ? dj + B.n_slices : (dj > 1 ? dj - B.n_slices : dj);
                    if (djm < -1 || djm > 1) set_error(B.err, kErrMigration);
                    dest = ((long long)cx * B.nc[1] + cy) * B.nc[2] + cz;
                }
                const long long slot_n = place_slot(B, pn, hcell, dest, own, tag_next, lane, n_stay);
                if (slot_n >= 0) store_f64(B, pn, slot_n, aid, rx, ry, rz, vx, vy, vz);
            }
            __syncwarp();
        }
        // every home cell publishes how many atoms stayed in it, empty or not
        if (INTEGRATE && lane == 0 && idx_ok(B.err, hcell, B.n_cells))
            B.cnt[pn][hcell] = ((unsigned long long)tag_next << 32) | (unsigned long long)n_stay;
        if (thermo && lane == 0) {
            s_cellke[2 * h] = __longlong_as_double(cell_ke);
            s_cellke[2 * h + 1] = (double)n_i;
        }
        if (OBS) {   // the cell's (U, W, KE, N): its lanes' sums by a fixed xor tree
            for (int o = 16; o > 0; o >>= 1) {
                red_u += __shfl_xor_sync(kFull, red_u, o);
                red_w += __shfl_xor_sync(kFull, red_w, o);
                red_k += __shfl_xor_sync(kFull, red_k, o);
                red_n += __shfl_xor_sync(kFull, red_n, o);
            }
            if (lane == 0 && idx_ok(B.err, hcell, B.n_cells)) {
                double *o = B.unit_obs + (long long)kObsStride * hcell;
                o[0] = red_u;
                o[1] = red_w;
                o[2] = red_k;
                o[3] = red_n;
            }
            red_u = red_w = red_k = red_n = 0.0;
        }
        if (OBS) {
            h += kWarps;
        } else {
            if (lane == 0) h = atomicAdd(s_ctr, 1);
            h = __shfl_sync(kFull, h, 0);
        }
    }
    if (thermo) {   // the unit's (KE, N) before scaling, home cells in order; the next factor
        __syncthreads();
        if (warp == 0) {
            if (lane == 0) {
                long long ke = 0;   // fixed point: exact in any order
                double n = 0.0;
                for (int q = 0; q < n_home; ++q) {
                    ke_add(ke, __double_as_longlong(s_cellke[2 * q]), B.err);
                    n += s_cellke[2 * q + 1];
                }
                const long long u = (long long)j * B.units_per_slice + tile;
                if (idx_ok(B.err, u, B.n_cells)) {   // n_cells: units allocated
                    B.th_part[p][2 * u] = __longlong_as_double(ke);
                    B.th_part[p][2 * u + 1] = n;
                }
            }
            __syncwarp();
            slice_publish(B, j, s_abs, s_rel, lam, lane);
        }
    }
}

// ---- mixed form: one warp per home cell ----------------------------------------
//
// A warp gathers the 27-cell neighbourhood of its home cell straight from the
// state in L2 into a flat list in its own shared memory, every neighbour's
// FP32 coordinates shifted into the home cell's centred frame (home cell
// first, then the 26 others in (ox, oy, oz) order), and evaluates its home
// atoms against that list with packed FP32x2 arithmetic, then kicks, drifts
// and rebins them.  The list stores entries in pairs, [x0 x1 y0 y1 | z0 z1 -
// -], so that one pair of neighbours loads straight into the halves of packed
// operands; each lane holds two home atoms as splatted operands and meets two
// neighbours per loop trip (four candidate pairs).  While the list is built,
// every neighbour farther than the cutoff from the home atoms' bounding box is
// dropped (about 40 % of the candidate pairs of a uniform fluid at rho = 0.8,
// 356 -> 223 per atom): it is out of range of every home atom, so only
// masked zeros are lost.  The home cell's
// segment and the whole list are padded to an even length with a far-away
// dummy.  A neighbourhood longer than the list is gathered in windows of
// kListAtoms entries.
// There is no unit-wide staging, so warps never wait for each other.

#ifndef DSEA_LIST_ATOMS
#define DSEA_LIST_ATOMS 400
#endif
constexpr int kListAtoms = DSEA_LIST_ATOMS;   // list window (entries, even) of one warp
constexpr int kHomeMax = 128;                 // largest cell capacity (slots of one home cell)

// Per-warp shared memory of the mixed form.  The context fields are written
// once per home cell and read back through volatile loads where they are
// needed, so that no register holds them across the pair loop.
struct WarpArea {
    float4 list[kListAtoms];   // kListAtoms / 2 entry pairs: [x0 x1 y0 y1], [z0 z1 w0 w1] (w: home atoms' ids)
    unsigned char hslot[kHomeMax];   // slot of each home atom within its cell, canonical order
    long long s_abs;           // step of the input state
    long long hcell;           // home cell
    int j, tile, first;        // unit and first-step flag
    int rel, box;              // ring: relative step and box of the unit
    int hx, hy, hz;            // home cell coordinates
    int n_home, total, built;  // home atoms, list length (padded), window held by the list
    int wlen;                  // entries of the held window after pruning (even)
    float bb[6];               // pruning box: low corner, high corner (home frame)
    int n_stay;                // atoms that stayed in the home cell so far
    double lam;                // slice thermostat: the factor of this step (1 without)
    long long ke_fix;          // slice thermostat: the unit's KE before scaling (fixed point)
    double n_acc;              // and its atoms
};

// Per-lane FP64 accumulators of a force pass: U, W and KE halves, atoms.
struct ObsAcc {
    double u, w, k, n;
};

// Entry e of the list window: its x (y, z and the id bits follow at +2,
// +4 and +6 floats).
__device__ __forceinline__ float *list_entry(WarpArea &wa, int e)
{
    return reinterpret_cast<float *>(&wa.list[2 * (e >> 1)]) + (e & 1);
}

// Unit offsets (ox, oy, oz) of the 27 neighbourhood cells in (ox, oy, oz)
// order, padded with zeros to 32 rows so that any 5-bit index stays inside;
// one table per CTA, filled (fill_offsets) by every kernel that builds
// mixed-form lists before its first list.
__shared__ float4 g_offsets[32];

__device__ __forceinline__ void fill_offsets()
{
    const int k = threadIdx.x;
    if (k < 32)
        g_offsets[k] = k < 27 ? make_float4((float)(k / 9 - 1), (float)((k / 3) % 3 - 1), (float)(k % 3 - 1), 0.f)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
}

// Lane c (< 27) of a warp describes one cell of the neighbourhood of home
// cell (hx, hy, hz): lane 0 the home cell, lanes 1..26 the others.
struct NbrCell {
    int gc;           // global cell index
    int n_s, n_a;     // stayers (front slots) and arrivals (back slots)
    int pre;          // first list entry of the cell
    int kk;           // index of the cell's offset in g_offsets (13: the home cell)
};

// The neighbourhood of a home cell; `total` receives the list length, padded
// to even (the home segment is padded to even as well).
__device__ __forceinline__ NbrCell nbr_cell(const BoxDev &B, int p, unsigned tag, int hx, int hy, int hz,
                                            int lane, int &total)
{
    NbrCell c = {0, 0, 0, 0, 13};
    const int kk = lane == 0 ? 13 : (lane <= 13 ? lane - 1 : lane);
    const int ox = kk / 9 - 1;
    if (lane < 27 && !(B.walls_x && (hx + ox < 0 || hx + ox >= B.nc[0]))) {   // nothing beyond a wall
        const int oy = (kk / 3) % 3 - 1, oz = kk % 3 - 1;
        const int gx = wrap_index(hx + ox, B.nc[0]), gy = wrap_index(hy + oy, B.nc[1]),
                  gz = wrap_index(hz + oz, B.nc[2]);
        const int gc = (gx * B.nc[1] + gy) * B.nc[2] + gz;
        const bool ok = idx_ok(B.err, gc, B.n_cells);
        const unsigned long long ws = ok ? __ldcg(B.cnt[p] + gc) : 0ull, wa = ok ? __ldcg(B.arr[p] + gc) : 0ull;
        int n_s = ((unsigned)(ws >> 32) == tag) ? (int)(unsigned)ws : 0;
        int n_a = ((unsigned)(wa >> 32) == tag) ? (int)(unsigned)wa : 0;
        if (n_s + n_a > B.cap) {   // the two ends met: the cell overflowed
            set_error(B.err, kErrCapacity);
            n_s = min(n_s, B.cap);
            n_a = B.cap - n_s;
        }
        c.gc = gc;
        c.n_s = n_s;
        c.n_a = n_a;
        c.kk = kk;
    }
    const int n = c.n_s + c.n_a;
    const int nl = lane == 0 ? (n + 1) & ~1 : n;   // the home segment ends on a pair boundary
    int incl = nl;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    c.pre = incl - nl;
    const int t = __shfl_sync(kFull, incl, 31);
    total = (t + 1) & ~1;
    return c;
}

// Copy list entries [w0, w0 + kListAtoms) of the neighbourhood into the
// warp's list (lane c copies its cell's share).  A cell's canonical order is
// its stayers in slot order, then its arrivals ordered by atom id.  Home
// cell entries also record their slot.  Padding entries sit far away.  The
// stayers arrive by asynchronous 16-byte copies (all of a cell's in flight at
// once) as whole entries; each lane then tags its cell's entries with the
// cell's offset index (in w, whose atom id is not needed for a neighbour),
// and one warp-wide pass shifts every entry into the home frame by its
// tag's offset, drops the entries beyond the cutoff of the home atoms'
// bounding box and writes the rest, in order, into the
// [x0 x1 y0 y1 | z0 z1 w0 w1] pair layout in place.  wa.wlen receives the
// window's entry count after that pass.  (A per-lane shift pass over each
// cell's entries cost more shared-memory wavefronts: its lanes touch
// scattered 16-byte entries.)
__device__ __forceinline__ void build_window(const BoxDev &B, int p, const NbrCell &c, int total, int w0,
                                             int lane, WarpArea &wa)
{
    const int w1 = w0 + kListAtoms;
    float4 *raw = wa.list;   // entry e of the window at raw[e] until the pair pass
    if (lane < 27) {
        const float4 *q = B.q[p];
        const long long base = (long long)c.gc * B.cap;
        // stayers: canonical position i = slot offset i
        const int lo = max(0, w0 - c.pre), hi = min(c.n_s, w1 - c.pre);
        for (int i = lo; i < hi; ++i) {
            if (!idx_ok(B.err, c.pre + i - w0, kListAtoms) || !idx_ok(B.err, i, B.cap)) continue;
            cp_async16(&raw[c.pre + i - w0], q + base + i);
            if (lane == 0 && idx_ok(B.err, i, kHomeMax)) wa.hslot[i] = (unsigned char)i;
        }
        // arrivals: slot cap-1-k holds the k-th arrival; order them by id
        const long long abase = base + B.cap - c.n_a;
        const int a0 = c.pre + c.n_s;
        const int n_arr = (a0 < w1 && a0 + c.n_a > w0) ? c.n_a : 0;
        for (int t = 0; t < n_arr; ++t) {
            int r = 0;
            const long long slot = abase + t;
            const float4 a = __ldcg(q + slot);
            if (c.n_a > 1) {
                const int id = __float_as_int(a.w);
                for (int u = 0; u < c.n_a; ++u)
                    r += (__float_as_int(__ldcg(q + abase + u).w) < id) ? 1 : 0;
            }
            const int cp = a0 + r;   // canonical list position
            if (cp >= w0 && cp < w1) {
                raw[cp - w0] = a;
                if (lane == 0 && idx_ok(B.err, c.n_s + r, kHomeMax))
                    wa.hslot[c.n_s + r] = (unsigned char)(B.cap - c.n_a + t);
            }
        }
        // padding: after an odd home cell, and after an odd list
        const int pad0 = c.n_s + c.n_a;   // lane 0: the home cell's count
        if (lane == 0 && (pad0 & 1) && pad0 >= w0 && pad0 < w1)
            raw[pad0 - w0] = make_float4(kFarAway, kFarAway, kFarAway, 0.f);
        if (lane == 26 && c.pre + c.n_s + c.n_a < total && total - 1 >= w0 && total - 1 < w1)
            raw[total - 1 - w0] = make_float4(kFarAway, kFarAway, kFarAway, 0.f);
        cp_async_wait_all();
        if (lane > 0) {   // tag each entry with its cell's offset (the id is not needed any more)
            const int e0 = max(c.pre, w0), e1 = min(c.pre + c.n_s + c.n_a, w1);
            for (int e = e0; e < e1; ++e) reinterpret_cast<int *>(&raw[e - w0])[3] = c.kk;
        }
    }
    __syncwarp();
    const int n_raw = min(kListAtoms, total - w0);
    const int nh = __shfl_sync(kFull, c.n_s + c.n_a, 0);
    const int k0 = w0 == 0 ? (nh + 1) & ~1 : 0;
    // the home atoms' bounding box (window 0 holds them at its front)
    float lo[3] = {kFarAway, kFarAway, kFarAway}, hi[3] = {-kFarAway, -kFarAway, -kFarAway};
    if (w0 == 0) {
        for (int e = lane; e < nh; e += 32) {
            const float4 a = raw[e];
            lo[0] = fminf(lo[0], a.x); lo[1] = fminf(lo[1], a.y); lo[2] = fminf(lo[2], a.z);
            hi[0] = fmaxf(hi[0], a.x); hi[1] = fmaxf(hi[1], a.y); hi[2] = fmaxf(hi[2], a.z);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {   // warp min / max on order-preserving integer images
            lo[d] = ordered_float(__reduce_min_sync(kFull, ordered_int(lo[d]))) - kBoxMargin;
            hi[d] = ordered_float(__reduce_max_sync(kFull, ordered_int(hi[d]))) + kBoxMargin;
        }
        if (lane == 0) {
            for (int d = 0; d < 3; ++d) {
                wa.bb[d] = lo[d];
                wa.bb[3 + d] = hi[d];
            }
        }
        __syncwarp();
    } else {
        const volatile WarpArea &v = wa;
        for (int d = 0; d < 3; ++d) {
            lo[d] = v.bb[d];
            hi[d] = v.bb[3 + d];
        }
    }
    // The home segment (window 0 only) goes into the pair layout whole.
    for (int b = lane; b < (k0 >> 1); b += 32) {
        const float4 e0 = raw[2 * b], e1 = raw[2 * b + 1];
        raw[2 * b] = make_float4(e0.x, e1.x, e0.y, e1.y);
        raw[2 * b + 1] = make_float4(e0.z, e1.z, e0.w, e1.w);
    }
    // Every other entry is kept only if it lies within the cutoff (plus a
    // rounding margin) of the box, which holds every home atom; a dropped
    // entry is out of range of all of them, so its pair terms would all have
    // been masked to zero.  Kept entries are compacted in order into the
    // pair layout, in place: an entry never moves up, and each 64-entry
    // sweep (two entries per lane, which overlaps their loads and tests) writes
    // below the entries the next sweep reads.  Only x, y and z are stored: a
    // neighbour's w (its tag) is not read again; the home atoms' ids come
    // from the home segment.
    const float reach2 = B.rc2f + kReachMargin;
    const unsigned below = (1u << lane) - 1u;
    int m = k0;
    auto load_test = [&](int e, float4 &a) -> bool {
        if (e >= n_raw) return false;
        a = raw[e];
        // into the home cell's frame: the same FP32 sum as shifting by ox lc
        // (ox lc is exact); a padding entry (tag 0) stays far away
        const float4 o = g_offsets[__float_as_int(a.w) & 31];
        const volatile float *lc = B.lcf;
        a.x = fmaf(o.x, lc[0], a.x);
        a.y = fmaf(o.y, lc[1], a.y);
        a.z = fmaf(o.z, lc[2], a.z);
        return box_dist2(a.x, a.y, a.z, lo, hi) <= reach2;
    };
    for (int e0 = k0; e0 < n_raw; e0 += 64) {   // two entries per lane per sweep
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        const bool ka = load_test(e0 + lane, a), kb = load_test(e0 + 32 + lane, b);
        const unsigned kA = __ballot_sync(kFull, ka), kB = __ballot_sync(kFull, kb);
        __syncwarp();
        if (ka && idx_ok(B.err, m + __popc(kA & below), kListAtoms)) {
            float *d = list_entry(wa, m + __popc(kA & below));
            d[0] = a.x; d[2] = a.y; d[4] = a.z;
        }
        m += __popc(kA);
        if (kb && idx_ok(B.err, m + __popc(kB & below), kListAtoms)) {
            float *d = list_entry(wa, m + __popc(kB & below));
            d[0] = b.x; d[2] = b.y; d[4] = b.z;
        }
        m += __popc(kB);
    }
    if (m & 1) {   // pad the window to whole pairs
        if (lane == 0) {
            float *d = list_entry(wa, m);
            d[0] = kFarAway; d[2] = kFarAway; d[4] = kFarAway;
        }
        ++m;
    }
    if (lane == 0) wa.wlen = m;
    __syncwarp();
}

// Forces on home atoms [ib, ib + nin) of the warp's home cell from the whole
// neighbourhood (all windows), packed FP32x2: each lane carries two home
// atoms (splatted) and meets one entry pair of the list per trip; the ns lane
// groups take each window's pairs by stride (group g every ns-th pair from
// g; the home segment, which holds the atoms themselves, with the exact
// cutoff test).  The partial sums are combined in a fixed order (halves, then
// groups), so each atom's force is summed in an order fixed by the box
// state.  Lane l < nin returns the totals of home atom ib + l.
template <bool OBS>
__device__ __forceinline__ void home_forces(const BoxDev &B, WarpArea &wa, int ib, int lane, float &fx,
                                            float &fy, float &fz, float &uu, float &ww)
{
    const volatile WarpArea &v = wa;
    const int total = v.total, n_home = v.n_home;
    const int nin = min(32, n_home - ib);
    const int np = (nin + 1) >> 1;
    const float inv_np = inv_of(np);
    const int ns = qdiv(32, inv_np);
    const int g = qdiv(lane, inv_np), pi = lane - g * np;
    const bool act = g < ns;
    Acc2 a0 = {f2splat(0.f), f2splat(0.f), f2splat(0.f), f2splat(0.f), f2splat(0.f)}, a1 = a0;
    float2 X0 = f2splat(0.f), Y0 = X0, Z0 = X0, X1 = X0, Y1 = X0, Z1 = X0;
    const int n_win = (total + kListAtoms - 1) / kListAtoms;
    for (int w = 0; w < n_win; ++w) {
        if (v.built != w) {   // only when the neighbourhood exceeds one window
            const long long s_abs = v.s_abs;
            int tt = 0;
            const NbrCell c = nbr_cell(B, (int)(s_abs & 1), (unsigned)(s_abs + 1), v.hx, v.hy, v.hz, lane, tt);
            build_window(B, (int)(s_abs & 1), c, tt, w * kListAtoms, lane, wa);
            if (lane == 0) wa.built = w;
            __syncwarp();
        }
        if (act) {
            if (w == 0) {   // the home atoms sit at the front of window 0
                const float *h0 = list_entry(wa, ib + 2 * pi);
                const float *h1 = list_entry(wa, ib + min(2 * pi + 1, nin - 1));   // odd nin: repeat
                X0 = f2splat(h0[0]); Y0 = f2splat(h0[2]); Z0 = f2splat(h0[4]);
                X1 = f2splat(h1[0]); Y1 = f2splat(h1[2]); Z1 = f2splat(h1[4]);
            }
            const unsigned rcb = __float_as_uint(B.rc2f);
            const float rc2f = B.rc2f, ush = B.ushiftf;
            const int wp = v.wlen >> 1;                                      // entry pairs in the window
            const int hp = w == 0 ? (n_home + 1) >> 1 : 0;                  // home segment pairs
            const float4 *L = wa.list;
            for (int t = g; t < hp; t += ns) {
                const float4 xy = L[2 * t], zw = L[2 * t + 1];
                const float2 XJ = make_float2(xy.x, xy.y), YJ = make_float2(xy.z, xy.w), ZJ = make_float2(zw.x, zw.y);
                pair2<true, OBS>(X0, Y0, Z0, XJ, YJ, ZJ, rc2f, rcb, ush, a0);
                pair2<true, OBS>(X1, Y1, Z1, XJ, YJ, ZJ, rc2f, rcb, ush, a1);
            }
            // group g takes pairs hp + g, hp + g + ns, ...: at most four groups read
            // distinct bank quarters in every trip
            const float4 *lp = L + 2 * (hp + g);
            const float4 *le = L + 2 * wp;
            const int stride = 2 * ns;
            DSEA_UNROLL(DSEA_PAIR_UNROLL_N)
            for (; lp < le; lp += stride) {
                const float4 xy = lp[0];
                const float2 ZJ = *reinterpret_cast<const float2 *>(lp + 1);
                const float2 XJ = make_float2(xy.x, xy.y), YJ = make_float2(xy.z, xy.w);
                pair2<OBS, OBS>(X0, Y0, Z0, XJ, YJ, ZJ, rc2f, rcb, ush, a0);
                pair2<OBS, OBS>(X1, Y1, Z1, XJ, YJ, ZJ, rc2f, rcb, ush, a1);
            }
        }
    }
    // per lane: home atom 0 of the pair in .x, atom 1 in .y (halves summed)
    const float2 FX = make_float2(a0.fx.x + a0.fx.y, a1.fx.x + a1.fx.y);
    const float2 FY = make_float2(a0.fy.x + a0.fy.y, a1.fy.x + a1.fy.y);
    const float2 FZ = make_float2(a0.fz.x + a0.fz.y, a1.fz.x + a1.fz.y);
    const float2 UU = make_float2(a0.u.x + a0.u.y, a1.u.x + a1.u.y);
    const float2 WW = make_float2(a0.w.x + a0.w.y, a1.w.x + a1.w.y);
    // combine the ns partials of each atom pair into lane pi (group 0) by a
    // fixed tree over the groups: at distance d, group g (a multiple of 2d)
    // adds group g + d when it exists; at most five levels
    float2 SX = FX, SY = FY, SZ = FZ, SU = UU, SW = WW;
#pragma unroll 1
    for (int d = 1; d < ns; d <<= 1) {
        const int off = d * np;   // lane + off < ns * np <= 32 whenever it is added
        const bool add = (g & (2 * d - 1)) == 0 && g + d < ns;
        float t;
        t = __shfl_down_sync(kFull, SX.x, off); if (add) SX.x += t;
        t = __shfl_down_sync(kFull, SX.y, off); if (add) SX.y += t;
        t = __shfl_down_sync(kFull, SY.x, off); if (add) SY.x += t;
        t = __shfl_down_sync(kFull, SY.y, off); if (add) SY.y += t;
        t = __shfl_down_sync(kFull, SZ.x, off); if (add) SZ.x += t;
        t = __shfl_down_sync(kFull, SZ.y, off); if (add) SZ.y += t;
        if (OBS) {
            t = __shfl_down_sync(kFull, SU.x, off); if (add) SU.x += t;
            t = __shfl_down_sync(kFull, SU.y, off); if (add) SU.y += t;
            t = __shfl_down_sync(kFull, SW.x, off); if (add) SW.x += t;
            t = __shfl_down_sync(kFull, SW.y, off); if (add) SW.y += t;
        }
    }
    // atom l (l < nin) is half l & 1 of the pair held by lane l >> 1
    const int from = (lane >> 1) < np ? (lane >> 1) : 0;
    const bool hi = lane & 1;
    float t0, t1;
    t0 = __shfl_sync(kFull, SX.x, from); t1 = __shfl_sync(kFull, SX.y, from); fx = hi ? t1 : t0;
    t0 = __shfl_sync(kFull, SY.x, from); t1 = __shfl_sync(kFull, SY.y, from); fy = hi ? t1 : t0;
    t0 = __shfl_sync(kFull, SZ.x, from); t1 = __shfl_sync(kFull, SZ.y, from); fz = hi ? t1 : t0;
    if (OBS) {
        t0 = __shfl_sync(kFull, SU.x, from); t1 = __shfl_sync(kFull, SU.y, from); uu = hi ? t1 : t0;
        t0 = __shfl_sync(kFull, SW.x, from); t1 = __shfl_sync(kFull, SW.y, from); ww = hi ? t1 : t0;
    }
}

// Kick, drift and rebin (INTEGRATE) or read back (OBS without INTEGRATE) the
// home atoms [ib, ib + 32) of the warp's home cell, given their forces;
// OBS adds their U, W and KE halves and their count to red.  With the slice
// thermostat, the synchronised velocity is scaled by wa.lam before the drift
// (md_v3b) and its KE before scaling is added to the unit's total.
template <bool INTEGRATE, bool OBS>
__device__ __forceinline__ void home_update(const BoxDev &B, WarpArea &wa, int ib, int lane, float fx, float fy,
                                            float fz, float uu, float ww, ObsAcc &red)
{
    const volatile WarpArea &v = wa;
    const long long s_abs = v.s_abs;
    const int p = (int)(s_abs & 1), pn = p ^ 1;
    const unsigned tag_next = (unsigned)(s_abs + 2);
    const bool first_step = v.first != 0;
    const long long S = B.n_slots;
    const float dtf = (float)B.dt;
    const int n_home = v.n_home;
    const bool own = lane < n_home - ib;
    long long slot = 0;
    int aid = 0;
    float4 qo = make_float4(0.f, 0.f, 0.f, 0.f);
    double rr[3] = {0.0, 0.0, 0.0};
    float vv[3] = {0.f, 0.f, 0.f};
    if (own) {
        slot = v.hcell * B.cap + (idx_ok(B.err, ib + lane, kHomeMax) ? wa.hslot[ib + lane] : 0);
        if (!idx_ok(B.err, slot, B.n_slots)) slot = 0;   // checked build: read a valid slot
        if (v.total <= kListAtoms) {
            const float *f = list_entry(wa, ib + lane);
            qo = make_float4(f[0], f[2], f[4], f[6]);
        } else {
            qo = __ldcg(B.q[p] + slot);
        }
        aid = __float_as_int(qo.w);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            rr[d] = __ldcg(B.r[p] + d * S + slot);
            vv[d] = __ldcg(B.vf[p] + d * S + slot);
        }
        if (OBS) {
            // synchronised velocity v(t) = v(t - dt/2) + F dt/2 (v(t0) itself at the start)
            const float hk = first_step ? 0.f : 0.5f * dtf;
            const float sx = fmaf(hk, fx, vv[0]), sy = fmaf(hk, fy, vv[1]), sz = fmaf(hk, fz, vv[2]);
            red.u += 0.5 * (double)uu;
            red.w += 0.5 * (double)ww;
            red.k += 0.5 * (double)fmaf(sx, sx, fmaf(sy, sy, sz * sz));
            red.n += 1.0;
            if (!INTEGRATE && idx_ok(B.err, aid, B.n_atoms)) {   // absolute: cell centre plus relative
                const long long o = 3LL * aid;
                B.out_f[o] = fx; B.out_f[o + 1] = fy; B.out_f[o + 2] = fz;
                B.out_v[o] = sx; B.out_v[o + 1] = sy; B.out_v[o + 2] = sz;
                B.out_r[o] = ((double)v.hx + 0.5) * B.lc[0] + rr[0];
                B.out_r[o + 1] = ((double)v.hy + 0.5) * B.lc[1] + rr[1];
                B.out_r[o + 2] = ((double)v.hz + 0.5) * B.lc[2] + rr[2];
            }
        }
    }
    if (INTEGRATE && B.T0 > 0.0) {
        // synchronised v(t) = v(t - dt/2) + F dt/2 (v(t0) itself at the start), its KE,
        // then v(t + dt/2) = lam v(t) + F dt/2 (md_v3b)
        double ke = 0.0;
        if (own) {
            const float hk = first_step ? 0.f : 0.5f * dtf, lamf = (float)v.lam;
            const float sx = fmaf(hk, fx, vv[0]), sy = fmaf(hk, fy, vv[1]), sz = fmaf(hk, fz, vv[2]);
            ke = 0.5 * (double)fmaf(sx, sx, fmaf(sy, sy, sz * sz));
            vv[0] = fmaf(0.5f * dtf, fx, lamf * sx);
            vv[1] = fmaf(0.5f * dtf, fy, lamf * sy);
            vv[2] = fmaf(0.5f * dtf, fz, lamf * sz);
        }
        for (int o = 16; o > 0; o >>= 1) ke += __shfl_xor_sync(kFull, ke, o);
        if (lane == 0) {
            long long acc = wa.ke_fix;
            ke_add(acc, ke_fixed(ke, B.err), B.err);
            wa.ke_fix = acc;
            wa.n_acc += (double)min(32, n_home - ib);
        }
    }
    if (INTEGRATE) {
        long long dest = 0;
        float qn[3] = {0.f, 0.f, 0.f};
        if (own) {
            if (!(B.T0 > 0.0)) {
                const float kf = first_step ? 0.5f * dtf : dtf;
                vv[0] = fmaf(kf, fx, vv[0]);   // v(t + dt/2) = v(t - dt/2) + F dt
                vv[1] = fmaf(kf, fy, vv[1]);
                vv[2] = fmaf(kf, fz, vv[2]);
            }
            const float q3[3] = {qo.x, qo.y, qo.z};
            const int cg[3] = {v.hx, v.hy, v.hz};
            int c3[3];
            bool refl[3];
#pragma unroll
            for (int d = 0; d < 3; ++d)   // r(t + dt) = r(t) + v(t + dt/2) dt, in FP64
                c3[d] = move_axis(rr[d], q3[d], vv[d] * dtf, cg[d], B.lc[d], B.inv_lcf[d], B.nc[d],
                                  d == 0 && B.walls_x, qn[d], refl[d]);
            if (refl[0]) vv[0] = -vv[0];   // reflected at a mirror wall
            const int dj = qdiv(c3[0], inv_of(B.cps)) - v.j;
            const int djm = dj < -1 ? dj + B.n_slices : (dj > 1 ? dj - B.n_slices : dj);
            if (djm < -1 || djm > 1) set_error(B.err, kErrMigration);
            dest = ((long long)c3[0] * B.nc[1] + c3[1]) * B.nc[2] + c3[2];
        }
        int n_stay = v.n_stay;
        const long long slot_n = place_slot(B, pn, v.hcell, dest, own, tag_next, lane, n_stay);
        if (slot_n >= 0)
            store_mixed(B, pn, slot_n, aid, rr[0], rr[1], rr[2], vv[0], vv[1], vv[2], qn[0], qn[1], qn[2]);
        __syncwarp();
        if (lane == 0) wa.n_stay = n_stay;
    }
}

// One home cell (wa.hx, wa.hy, wa.hz) of the mixed form, warp-wide: its
// neighbourhood into the list, forces, then home_update per 32 home atoms;
// INTEGRATE publishes how many atoms stayed in the cell.
template <bool INTEGRATE, bool OBS>
__device__ __forceinline__ void mixed_home_cell(const BoxDev &B, WarpArea &wa, ObsAcc &red)
{
    const int lane = threadIdx.x & 31;
    const volatile WarpArea &v = wa;
    {
        const long long s_abs = v.s_abs;
        const int hx = v.hx, hy = v.hy, hz = v.hz;
        int total = 0;
        const NbrCell c = nbr_cell(B, (int)(s_abs & 1), (unsigned)(s_abs + 1), hx, hy, hz, lane, total);
        build_window(B, (int)(s_abs & 1), c, total, 0, lane, wa);
        if (lane == 0) {
            wa.n_home = c.n_s + c.n_a;
            wa.hcell = c.gc;
            wa.total = total;
            wa.built = 0;
            wa.n_stay = 0;
        }
        __syncwarp();
    }
    for (int ib = 0; ib < v.n_home; ib += 32) {
        float fx = 0.f, fy = 0.f, fz = 0.f, uu = 0.f, ww = 0.f;
        home_forces<OBS>(B, wa, ib, lane, fx, fy, fz, uu, ww);
        home_update<INTEGRATE, OBS>(B, wa, ib, lane, fx, fy, fz, uu, ww, red);
    }
    if (OBS) {   // the cell's (U, W, KE, N): its lanes' sums by a fixed xor tree
        for (int o = 16; o > 0; o >>= 1) {
            red.u += __shfl_xor_sync(kFull, red.u, o);
            red.w += __shfl_xor_sync(kFull, red.w, o);
            red.k += __shfl_xor_sync(kFull, red.k, o);
            red.n += __shfl_xor_sync(kFull, red.n, o);
        }
        if (lane == 0 && idx_ok(B.err, v.hcell, B.n_cells)) {
            double *o = B.unit_obs + (long long)kObsStride * v.hcell;
            o[0] = red.u;
            o[1] = red.w;
            o[2] = red.k;
            o[3] = red.n;
        }
        red = ObsAcc{0.0, 0.0, 0.0, 0.0};
    }
    // the home cell publishes how many atoms stayed in it, empty or not
    if (INTEGRATE && lane == 0 && idx_ok(B.err, v.hcell, B.n_cells))
        B.cnt[(int)(v.s_abs & 1) ^ 1][v.hcell] = ((unsigned long long)(unsigned)(v.s_abs + 2) << 32) |
                                                  (unsigned long long)(unsigned)v.n_stay;
    __syncwarp();   // the list and slot table are reused by the next home cell
}

// Before a unit's home cells: the slice thermostat's factor and the unit's
// accumulators (INTEGRATE with T0 > 0 only).
template <bool INTEGRATE>
__device__ __forceinline__ void mixed_unit_begin(const BoxDev &B, WarpArea &wa, int j, long long s_abs,
                                                 bool first_step, int lane)
{
    if (!INTEGRATE || !(B.T0 > 0.0)) return;
    if (lane == 0) {
        wa.lam = slice_factor(B, j, s_abs, first_step);
        wa.ke_fix = 0;
        wa.n_acc = 0.0;
    }
    __syncwarp();
}

// After a unit's home cells: its (KE, N) before scaling and the factor, for
// the slice's units of the next step.
template <bool INTEGRATE>
__device__ __forceinline__ void mixed_unit_end(const BoxDev &B, WarpArea &wa, int j, int tile, long long s_abs,
                                               int s_rel, int lane)
{
    if (!INTEGRATE || !(B.T0 > 0.0)) return;
    __syncwarp();
    if (lane == 0) {
        const int p = (int)(s_abs & 1);
        const long long u = (long long)j * B.units_per_slice + tile;
        if (idx_ok(B.err, u, B.n_cells)) {   // n_cells: units allocated
            B.th_part[p][2 * u] = __longlong_as_double(wa.ke_fix);
            B.th_part[p][2 * u + 1] = wa.n_acc;
        }
    }
    __syncwarp();
    const volatile WarpArea &v = wa;
    slice_publish(B, j, s_abs, s_rel, v.lam, lane);
}

// Home cell h of unit (j, tile) (z fastest, then y, then x) into wa.hx/hy/hz.
__device__ __forceinline__ int unit_cell_count(const BoxDev &B, int tile)
{
    const int tyi = qdiv(tile, inv_of(B.tiles_z)), tzi = tile - tyi * B.tiles_z;
    return B.cps * min(B.tile_y, B.nc[1] - tyi * B.tile_y) * min(B.tile_z, B.nc[2] - tzi * B.tile_z);
}
__device__ __forceinline__ void set_unit_cell(const BoxDev &B, WarpArea &wa, int j, int tile, int h)
{
    const int tyi = qdiv(tile, inv_of(B.tiles_z)), tzi = tile - tyi * B.tiles_z;
    const int y0 = tyi * B.tile_y, z0 = tzi * B.tile_z;
    const int ny = min(B.tile_y, B.nc[1] - y0), nz = min(B.tile_z, B.nc[2] - z0);
    const int nyz = ny * nz;
    const int lx = qdiv(h, inv_of(nyz)), r = h - lx * nyz, ly = qdiv(r, inv_of(nz));
    if ((threadIdx.x & 31) == 0) {
        wa.hx = j * B.cps + lx;
        wa.hy = y0 + ly;
        wa.hz = z0 + (r - ly * nz);
    }
    __syncwarp();
}

// ---- kernels ---------------------------------------------------------------

template <int PREC>
__global__ void __launch_bounds__(kThreads) k_bin(const BoxDev *bp, const double *pos,
                                                  const double *vel)
{
    const BoxDev &B = *bp;
    const int lane = threadIdx.x & 31;
    const int p = (int)(B.step & 1);
    const unsigned tag = (unsigned)(B.step + 1);
    const long long n = B.n_atoms;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const long long i = i0 + threadIdx.x;
        const bool own = i < n;
        double x = 0, y = 0, z = 0, vx = 0, vy = 0, vz = 0;
        int cx = 0, cy = 0, cz = 0;
        long long dest = 0;
        if (own) {
            x = pos[3 * i]; y = pos[3 * i + 1]; z = pos[3 * i + 2];
            x -= B.L[0] * floor(x / B.L[0]);
            y -= B.L[1] * floor(y / B.L[1]);
            z -= B.L[2] * floor(z / B.L[2]);
            x = wrap_coord(x, B.L[0]);
            y = wrap_coord(y, B.L[1]);
            z = wrap_coord(z, B.L[2]);
            if (vel) {
                vx = vel[3 * i]; vy = vel[3 * i + 1]; vz = vel[3 * i + 2];
            }
            cx = cell_of(x, B.inv_lc[0], B.nc[0]);
            cy = cell_of(y, B.inv_lc[1], B.nc[1]);
            cz = cell_of(z, B.inv_lc[2], B.nc[2]);
            dest = ((long long)cx * B.nc[1] + cy) * B.nc[2] + cz;
        }
        // every initial atom is an arrival (back slots); readers order them by id
        const int k = reserve_slot(B.arr[p], dest, own, tag, lane, B.err);
        if (own) {
            const long long slot = dest * B.cap + (B.cap - 1 - k);
            if (k >= B.cap) {
                set_error(B.err, kErrCapacity);
            } else if (PREC == 1) {
                // FP64 positions relative to the centre of the atom's cell, and their FP32 copies
                const double rx = x - ((double)cx + 0.5) * B.lc[0];
                const double ry = y - ((double)cy + 0.5) * B.lc[1];
                const double rz = z - ((double)cz + 0.5) * B.lc[2];
                store_mixed(B, p, slot, (int)i, rx, ry, rz, (float)vx, (float)vy, (float)vz, (float)rx, (float)ry,
                            (float)rz);
            } else {
                store_f64(B, p, slot, (int)i, x, y, z, vx, vy, vz);
            }
        }
    }
}

// After binning: one warp per cell moves the cell's arrivals (every atom
// k_bin placed, in the order its atomics gave) to the front slots in atom-id
// order, after any stayers, and makes them stayers.  That is the cell's
// canonical order already (stayers in slot order, then arrivals by id), so
// no result changes; but the first step's readers then find stayers and
// skip ranking a whole cell of arrivals, a quadratic loop of dependent loads
// that made the first step ten times slower than the rest.  All of a cell's
// records are read into registers before any is written: the two slot ranges
// may overlap.
template <int PREC>
__global__ void __launch_bounds__(kThreads) k_settle(const BoxDev *bp)
{
    const BoxDev &B = *bp;
    const int lane = threadIdx.x & 31;
    const int p = (int)(B.step & 1);
    const unsigned tag = (unsigned)(B.step + 1);
    const long long S = B.n_slots;
    const long long warps = (long long)gridDim.x * (kThreads / 32);
    for (long long gc = (long long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5); gc < B.n_cells;
         gc += warps) {
        const unsigned long long ws = B.cnt[p][gc], wa = B.arr[p][gc];
        const int n_s = ((unsigned)(ws >> 32) == tag) ? (int)(unsigned)ws : 0;
        const int n_a = ((unsigned)(wa >> 32) == tag) ? (int)(unsigned)wa : 0;
        if (n_a == 0 || n_s + n_a > B.cap || n_a > 128) continue;   // nothing to do, or overflowed
        const long long abase = gc * B.cap + B.cap - n_a;            // the first arrival's slot
        int idm[4];
        double rx[4], ry[4], rz[4], vx[4], vy[4], vz[4];
        float4 qm[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int a = lane + 32 * m;
            idm[m] = 0x7fffffff;
            if (a < n_a) {
                const long long slot = abase + a;
                rx[m] = B.r[p][slot];
                ry[m] = B.r[p][S + slot];
                rz[m] = B.r[p][2 * S + slot];
                if (PREC == 1) {
                    vx[m] = B.vf[p][slot];
                    vy[m] = B.vf[p][S + slot];
                    vz[m] = B.vf[p][2 * S + slot];
                    qm[m] = B.q[p][slot];
                    idm[m] = __float_as_int(qm[m].w);
                } else {
                    vx[m] = B.v[p][slot];
                    vy[m] = B.v[p][S + slot];
                    vz[m] = B.v[p][2 * S + slot];
                    idm[m] = B.id[p][slot];
                }
            }
        }
        // rank by id among the cell's arrivals (ids are distinct)
        int rk[4] = {0, 0, 0, 0};
#pragma unroll
        for (int mb = 0; mb < 4; ++mb) {   // n_a is the same on every lane
            const int lim = min(32, n_a - 32 * mb);
            for (int t = 0; t < lim; ++t) {
                const int o = __shfl_sync(kFull, idm[mb], t);
#pragma unroll
                for (int m = 0; m < 4; ++m) rk[m] += (o < idm[m]) ? 1 : 0;
            }
        }
        __syncwarp();
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int a = lane + 32 * m;
            if (a < n_a) {
                const long long slot = gc * B.cap + n_s + rk[m];
                B.r[p][slot] = rx[m];
                B.r[p][S + slot] = ry[m];
                B.r[p][2 * S + slot] = rz[m];
                if (PREC == 1) {
                    B.vf[p][slot] = (float)vx[m];
                    B.vf[p][S + slot] = (float)vy[m];
                    B.vf[p][2 * S + slot] = (float)vz[m];
                    B.q[p][slot] = qm[m];
                } else {
                    B.v[p][slot] = vx[m];
                    B.v[p][S + slot] = vy[m];
                    B.v[p][2 * S + slot] = vz[m];
                    B.id[p][slot] = idm[m];
                }
            }
        }
        if (lane == 0) {
            B.cnt[p][gc] = ((unsigned long long)tag << 32) | (unsigned long long)(n_s + n_a);
            B.arr[p][gc] = (unsigned long long)tag << 32;
        }
    }
}

// FP64 form, one step or force pass: one CTA per unit.
template <bool INTEGRATE, bool OBS>
__global__ void __launch_bounds__(kThreads) k_units_f64(const BoxDev *bp, long long s_abs, int first)
{
    extern __shared__ __align__(16) char smem[];
    __shared__ BoxDev sB;
    if (threadIdx.x == 0) sB = *bp;
    __syncthreads();
    const int u = blockIdx.x;
    const int j = u / sB.units_per_slice, tile = u - j * sB.units_per_slice;
    run_unit_f64<INTEGRATE, OBS>(sB, j, tile, s_abs, first != 0, 0, smem);   // one step per launch
}

// Mixed form, one step or force pass: one warp per unit (warp w of block b
// takes unit b * kWarps + w); the unit's home cells in order.
template <bool INTEGRATE, bool OBS>
__global__ void __launch_bounds__(kThreads) k_units_mixed(const BoxDev *bp, long long s_abs, int first)
{
    extern __shared__ __align__(16) char smem[];
    __shared__ BoxDev sB;
    if (threadIdx.x == 0) sB = *bp;
    fill_offsets();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int u = blockIdx.x * kWarps + warp;
    if (u >= sB.n_slices * sB.units_per_slice) return;
    WarpArea &wa = reinterpret_cast<WarpArea *>(smem)[warp];
    const int j = u / sB.units_per_slice, tile = u - j * sB.units_per_slice;
    if (lane == 0) {
        wa.s_abs = s_abs;
        wa.j = j;
        wa.first = first;
    }
    ObsAcc red = {0.0, 0.0, 0.0, 0.0};
    mixed_unit_begin<INTEGRATE>(sB, wa, j, s_abs, first != 0, lane);
    const int n = unit_cell_count(sB, tile);
    for (int h = 0; h < n; ++h) {
        set_unit_cell(sB, wa, j, tile, h);
        mixed_home_cell<INTEGRATE, OBS>(sB, wa, red);
    }
    mixed_unit_end<INTEGRATE>(sB, wa, j, tile, s_abs, 0, lane);   // one step per launch
}

// Global (U, W, KE) from the per-cell partials of a force pass, in a fixed
// order that depends only on the cell count: thread t sums cells t, t + 1024,
// ..., then a fixed tree over the threads.
__global__ void __launch_bounds__(1024) k_obs_reduce(const double *cell_obs, long long n, double *out3)
{
    __shared__ double s[3][1024];
    double a = 0, b = 0, c = 0;
    for (long long i = threadIdx.x; i < n; i += 1024) {
        a += cell_obs[kObsStride * i];
        b += cell_obs[kObsStride * i + 1];
        c += cell_obs[kObsStride * i + 2];
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    s[2][threadIdx.x] = c;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s[0][threadIdx.x] += s[0][threadIdx.x + o];
            s[1][threadIdx.x] += s[1][threadIdx.x + o];
            s[2][threadIdx.x] += s[2][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out3[0] = s[0][0];
        out3[1] = s[1][0];
        out3[2] = s[2][0];
    }
}

// The persistent ring of the FP64 form: every CTA is one on-chip stage that
// repeatedly takes the next ticket, waits (bounded) until the five slices
// its unit reads at the previous level are complete, runs the unit and
// reports completion.  Tickets are dispensed step-major and, within a step,
// slice by slice from an offset that advances two slices per step, so level
// s trails level s-1 by about five slices (the time-skewed cyclic order of
// Sec. 3.1 / Table 1).  A CTA only waits on tickets smaller than its own, all
// of which were taken by running CTAs, so the ring always progresses.
#ifndef DSEA_RING_MIN_BLOCKS
#define DSEA_RING_MIN_BLOCKS 4   // CTAs per SM the register allocation must allow (mixed form)
#endif
// The FP64 unit's staging and force queues fill enough shared memory that an SM
// holds two of its CTAs, so its registers are budgeted for two (128 per thread)
// rather than spilled to fit four.
#ifndef DSEA_RING_F64_MIN_BLOCKS
#define DSEA_RING_F64_MIN_BLOCKS 2
#endif
__global__ void __launch_bounds__(kThreads, DSEA_RING_F64_MIN_BLOCKS) k_ring_f64(RingPlan plan)
{
    extern __shared__ __align__(16) char smem[];
    __shared__ BoxDev sB;
    __shared__ int s_dec[3];
    __shared__ int s_box;
    __shared__ int s_go;
    const int tid = threadIdx.x;
    if (tid == 0) s_box = -1;
    __syncthreads();
    while (true) {
        // thread 0 takes the next ticket, decodes it into (relative step, box,
        // slice, tile), loads the box's descriptor if it changed, and waits
        // (bounded) until slices j-2..j+2 of the previous level are complete.
        // A box that has already failed (capacity, migration) drains its
        // remaining units without work so that nothing waits on it; a wait that
        // expires stops the whole launch and marks every box of it.
        if (tid == 0) {
            int go = 1;   // 0: stop the CTA, 1: run the unit, 2: skip it
            const long long t = (long long)atomicAdd(plan.ticket, 1ULL);
            if (t >= plan.total) {
                go = 0;
            } else {
                int lo = 0, hi = plan.n_steps - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (plan.step_base[mid] <= t) lo = mid; else hi = mid - 1;
                }
                const int s_rel = lo;
                const long long r = t - plan.step_base[s_rel];
                int bl = 0, bh = plan.active[s_rel] - 1;
                while (bl < bh) {
                    const int mid = (bl + bh + 1) >> 1;
                    if (plan.cum_units[mid] <= r) bl = mid; else bh = mid - 1;
                }
                if (bl != s_box) {   // no other thread reads sB between the unit barriers
                    sB = plan.boxes[bl];
                    s_box = bl;
                }
                const int m = (int)(r - plan.cum_units[bl]);
                const int ups = sB.units_per_slice;
                idx_ok(sB.err, m, (long long)sB.n_slices * ups);   // checked build: a bad unit fails the box
                const int jj = m / ups;
                const int j = ring_slice(jj, sB.step + s_rel, sB.n_slices);
                s_dec[0] = s_rel;
                s_dec[1] = j;
                s_dec[2] = m - jj * ups;
                if (ld_volatile_int(plan.err) != 0) go = 0;
                else if (ld_volatile_int(sB.err) != 0) go = 2;
                if (go == 1 && s_rel > 0) {
                    const unsigned need = (unsigned)ups * (unsigned)s_rel;
                    const unsigned long long t0 = global_ns();
                    for (int d = -2; d <= 2 && go == 1; ++d) {
                        if (sB.walls_x && (j + d < 0 || j + d >= sB.n_slices)) continue;   // no slice past a wall
                        const int k = wrap_index(j + d, sB.n_slices);
                        if (!idx_ok(sB.err, k, sB.n_slices)) continue;
                        unsigned sleep = 32;
                        while (ld_acquire(sB.done + k) < need) {
                            if (ld_volatile_int(plan.err) != 0) { go = 0; break; }
                            if ((long long)(global_ns() - t0) > sB.wait_limit_ns) {
                                atomicCAS(plan.err, 0, kErrTimeout);
                                for (int q = 0; q < plan.n_boxes; ++q) set_error(plan.boxes[q].err, kErrTimeout);
                                go = 0;
                                break;
                            }
                            __nanosleep(sleep);
                            if (sleep < 1024) sleep <<= 1;
                        }
                    }
                }
            }
            s_go = go;
        }
        __syncthreads();
        if (s_go == 0) break;
        const int s_rel = s_dec[0], j = s_dec[1], tile = s_dec[2];
        const long long s_abs = sB.step + s_rel;
        if (s_go == 1)
            run_unit_f64<true, false>(sB, j, tile, s_abs, s_rel == 0 && sB.w_is_sync, s_rel, smem);
        __threadfence();
        __syncthreads();
        if (tid == 0 && !(j == sB.withhold_slice && s_rel == 0) && idx_ok(sB.err, j, sB.n_slices))
            atomicAdd(sB.done + j, 1u);
    }
}

// The persistent ring of the mixed form: every warp is one stage.  Lane 0
// takes the next ticket, the warp loads the ticket's box descriptor into its
// own shared memory if it changed, lane 0 waits (bounded) until slices
// j-2..j+2 of the previous level are complete, the warp runs the unit's home
// cells and reports completion.  Same dispatch order, dependency rule and
// failure handling as the CTA-level ring; a warp only waits on tickets
// smaller than its own, all taken by running warps.
__global__ void __launch_bounds__(kThreads, DSEA_RING_MIN_BLOCKS) k_ring_mixed(RingPlan plan)
{
    extern __shared__ __align__(16) char smem[];
    __shared__ BoxDev s_box[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpArea &wa = reinterpret_cast<WarpArea *>(smem)[warp];
    const volatile WarpArea &v = wa;
    BoxDev &B = s_box[warp];
    ObsAcc red = {0.0, 0.0, 0.0, 0.0};   // unused (no reduction in the ring)
    if (lane == 0) wa.box = -1;
    fill_offsets();
    while (true) {
        int go = 1;   // 0: stop the warp, 1: run the unit, 2: skip it
        int bl = 0;
        long long r = 0;
        if (lane == 0) {
            const long long t = (long long)atomicAdd(plan.ticket, 1ULL);
            if (t >= plan.total) {
                go = 0;
            } else {
                int lo = 0, hi = plan.n_steps - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (plan.step_base[mid] <= t) lo = mid; else hi = mid - 1;
                }
                wa.rel = lo;
                r = t - plan.step_base[lo];
                int bh = plan.active[lo] - 1;
                while (bl < bh) {
                    const int mid = (bl + bh + 1) >> 1;
                    if (plan.cum_units[mid] <= r) bl = mid; else bh = mid - 1;
                }
            }
        }
        go = __shfl_sync(kFull, go, 0);
        if (go == 0) break;
        bl = __shfl_sync(kFull, bl, 0);
        if (bl != v.box) {   // the warp's copy of the box descriptor
            const int *src = reinterpret_cast<const int *>(plan.boxes + bl);
            int *dst = reinterpret_cast<int *>(&B);
            for (int i = lane; i < (int)(sizeof(BoxDev) / sizeof(int)); i += 32) dst[i] = src[i];
            __syncwarp();
            if (lane == 0) wa.box = bl;
        }
        __syncwarp();
        if (lane == 0) {
            const int s_rel = wa.rel;
            const int m = (int)(r - plan.cum_units[bl]);
            const int ups = B.units_per_slice;
            idx_ok(B.err, m, (long long)B.n_slices * ups);   // checked build: a bad unit fails the box
            const int jj = m / ups;
            const int j = ring_slice(jj, B.step + s_rel, B.n_slices);
            wa.j = j;
            wa.tile = m - jj * ups;
            wa.s_abs = B.step + s_rel;
            wa.first = (s_rel == 0 && B.w_is_sync) ? 1 : 0;
            if (ld_volatile_int(plan.err) != 0) go = 0;
            else if (ld_volatile_int(B.err) != 0) go = 2;
            if (go == 1 && s_rel > 0) {
                const unsigned need = (unsigned)ups * (unsigned)s_rel;
                const unsigned long long t0 = global_ns();
                for (int d = -2; d <= 2 && go == 1; ++d) {
                    if (B.walls_x && (j + d < 0 || j + d >= B.n_slices)) continue;   // no slice past a wall
                    const int k = wrap_index(j + d, B.n_slices);
                    if (!idx_ok(B.err, k, B.n_slices)) continue;
                    unsigned sleep = 32;
                    while (ld_acquire(B.done + k) < need) {
                        if (ld_volatile_int(plan.err) != 0) { go = 0; break; }
                        if ((long long)(global_ns() - t0) > B.wait_limit_ns) {
                            atomicCAS(plan.err, 0, kErrTimeout);
                            for (int q = 0; q < plan.n_boxes; ++q) set_error(plan.boxes[q].err, kErrTimeout);
                            go = 0;
                            break;
                        }
                        __nanosleep(sleep);
                        if (sleep < 1024) sleep <<= 1;
                    }
                }
            }
        }
        go = __shfl_sync(kFull, go, 0);
        if (go == 0) break;
        if (go == 1) {
            mixed_unit_begin<true>(B, wa, v.j, v.s_abs, v.first != 0, lane);
            const int n = unit_cell_count(B, v.tile);
            for (int h = 0; h < n; ++h) {
                set_unit_cell(B, wa, v.j, v.tile, h);
                mixed_home_cell<true, false>(B, wa, red);
            }
            mixed_unit_end<true>(B, wa, v.j, v.tile, v.s_abs, v.rel, lane);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            const int j = v.j;
            if (!(j == B.withhold_slice && v.rel == 0) && idx_ok(B.err, j, B.n_slices)) atomicAdd(B.done + j, 1u);
        }
    }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t unit_smem_bytes(int precision, int staged_cells, int smem_atoms)
{
    if (precision == 1) return sizeof(WarpArea) * kWarps;   // per-warp lists, whatever the unit
    return make_layout(staged_cells, smem_atoms).total;
}

size_t max_unit_smem_bytes()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // the kernels also hold a static copy of the box descriptor and a few words
    return (size_t)v > 4096 ? (size_t)v - 4096 : 0;
}

__global__ void __launch_bounds__(256) k_check_finite(const double *a, long long n, int *flag)
{
    bool bad = false;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
        bad |= !isfinite(a[i]);
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) *flag = 1;
}

cudaError_t launch_check_finite(const double *a, long long n, int *flag, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    k_check_finite<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(a, n, flag);
    return cudaGetLastError();
}

cudaError_t launch_bin(const BoxDev &hb, const BoxDev *db, const double *pos, const double *vel,
                       cudaStream_t stream)
{
    if (hb.n_atoms == 0) return cudaSuccess;
    const long long blocks = (hb.n_atoms + kThreads - 1) / kThreads;
    const int grid = (int)(blocks < 65535 ? blocks : 65535);
    if (hb.precision == 1) k_bin<1><<<grid, kThreads, 0, stream>>>(db, pos, vel);
    else k_bin<0><<<grid, kThreads, 0, stream>>>(db, pos, vel);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long sblocks = (hb.n_cells + kThreads / 32 - 1) / (kThreads / 32);
    const int sgrid = (int)(sblocks < 65535 ? sblocks : 65535);
    if (hb.precision == 1) k_settle<1><<<sgrid, kThreads, 0, stream>>>(db);
    else k_settle<0><<<sgrid, kThreads, 0, stream>>>(db);
    return cudaGetLastError();
}

template <int PREC, bool INTEGRATE, bool OBS>
static cudaError_t launch_units(const BoxDev &hb, const BoxDev *db, long long s_abs, int first,
                                cudaStream_t stream)
{
    const size_t smem = unit_smem_bytes(PREC, hb.staged_cells, hb.smem_atoms);
    const int units = hb.n_slices * hb.units_per_slice;
    if (PREC == 1) {
        cudaError_t e = set_smem(k_units_mixed<INTEGRATE, OBS>, smem);
        if (e != cudaSuccess) return e;
        const int grid = (units + kWarps - 1) / kWarps;
        k_units_mixed<INTEGRATE, OBS><<<grid, kThreads, smem, stream>>>(db, s_abs, first);
        return cudaGetLastError();
    }
    cudaError_t e = set_smem(k_units_f64<INTEGRATE, OBS>, smem);
    if (e != cudaSuccess) return e;
    k_units_f64<INTEGRATE, OBS><<<units, kThreads, smem, stream>>>(db, s_abs, first);
    return cudaGetLastError();
}

cudaError_t launch_step(const BoxDev &hb, const BoxDev *db, int64_t s_abs, int first_step,
                        cudaStream_t stream)
{
    return hb.precision == 1 ? launch_units<1, true, false>(hb, db, s_abs, first_step, stream)
                             : launch_units<0, true, false>(hb, db, s_abs, first_step, stream);
}

cudaError_t launch_force_pass(const BoxDev &hb, const BoxDev *db, cudaStream_t stream)
{
    return hb.precision == 1 ? launch_units<1, false, true>(hb, db, hb.step, hb.w_is_sync, stream)
                             : launch_units<0, false, true>(hb, db, hb.step, hb.w_is_sync, stream);
}

cudaError_t launch_obs_reduce(const double *cell_obs, long long n_cells, double *out3, cudaStream_t stream)
{
    k_obs_reduce<<<1, 1024, 0, stream>>>(cell_obs, n_cells, out3);
    return cudaGetLastError();
}

cudaError_t launch_ring(const RingPlan &plan, int precision, size_t smem_bytes, int ctas,
                        cudaStream_t stream)
{
    if (plan.total == 0) return cudaSuccess;
    cudaError_t e;
    if (precision == 1) {
        e = set_smem(k_ring_mixed, smem_bytes);
        if (e != cudaSuccess) return e;
        k_ring_mixed<<<ctas, kThreads, smem_bytes, stream>>>(plan);
    } else {
        e = set_smem(k_ring_f64, smem_bytes);
        if (e != cudaSuccess) return e;
        k_ring_f64<<<ctas, kThreads, smem_bytes, stream>>>(plan);
    }
    return cudaGetLastError();
}

int ring_ctas_per_sm(int precision, size_t smem_bytes)
{
    int n = 0;
    if (precision == 1) {
        set_smem(k_ring_mixed, smem_bytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ring_mixed, kThreads, smem_bytes);
    } else {
        set_smem(k_ring_f64, smem_bytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ring_f64, kThreads, smem_bytes);
    }
    return n;
}

}  // namespace dsea
