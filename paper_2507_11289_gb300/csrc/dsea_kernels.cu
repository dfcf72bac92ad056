// dsea_kernels.cu -- sm_103a kernels of the slice-streamed LJ NVE step.
//
// One work unit = all home cells of one slice (its cps cell layers along x)
// within a tile_y x tile_z block of cells in (y, z).  A unit
//   1. stages the counts of its neighbourhood cells (home cells plus one cell
//      layer around them, periodic) and an exclusive scan of them,
//   2. stages the atoms of those cells into shared memory, each cell sorted
//      by atom id (so every sum below runs in an order fixed by the state
//      alone: the same whatever the unit shape, launch form or batch),
//   3. computes, warp per home cell, the force on each home atom from the 27
//      neighbour cells (Algorithm 1's first loop, Sec. 4.1 "md_v3a"),
//   4. (INTEGRATE) kicks and drifts each home atom (Algorithm 1's second and
//      third loops, "md_v3aa" / "md_v3b") and appends it to the cell it
//      moved to in the next-step buffer, which may belong to slice j-1, j or
//      j+1 (O_out = 1, Sec. 4); warp-aggregated atomics reserve the slots,
//   5. (OBS) reduces U, W and KE of its home atoms in FP64 ("stat_collect").
//
// The FP64 form evaluates pairs on absolute positions and keeps velocities in
// FP64.  The mixed form evaluates pairs in packed FP32x2 arithmetic on FP32
// coordinates relative to each atom's cell centre and keeps velocities in
// FP32; FP64 is kept for the absolute positions, the position update and
// every reduction (FP64 issues at a small fraction of the FP32 rate on this
// GPU, so the mixed form spends about a dozen FP64 operations per atom-step).
#include "dsea_internal.h"

namespace dsea {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPrefBytes = 32 * (3 * 8 + 3 * 4);   // per warp: own atoms' r (FP64) and v (FP32)

__device__ __forceinline__ void set_error(int *err, int code)
{
    atomicCAS(err, 0, code);
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
// other CTAs wrote earlier in the same persistent launch is always seen (L1
// is not kept coherent with other SMs' writes).  Both addresses 16-B aligned.
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

// Shared-memory carve-up of one unit.
struct Layout {
    size_t cnt, nst, start, gcell, atoms, id, slot, scr, ctab, tab, red, ctr, total;
};

__host__ __device__ inline Layout make_layout(int precision, int staged_cells, int smem_atoms)
{
    Layout L;
    size_t o = 0;
    L.cnt = o;   o += sizeof(int) * staged_cells;
    L.nst = o;   o += sizeof(int) * staged_cells;   // stayers of each staged cell
    L.start = o; o += sizeof(int) * (staged_cells + 1);
    L.gcell = o; o += sizeof(int) * staged_cells;
    o = align16(o);
    L.atoms = o;
    if (precision == 1) {
        o += sizeof(float4) * smem_atoms;       // x, y, z, id bits
        L.id = 0;
    } else {
        o += 3 * sizeof(double) * smem_atoms;   // x[], y[], z[]
        L.id = o;
        o += sizeof(int) * smem_atoms;
    }
    L.slot = o; o += sizeof(int) * smem_atoms;
    o = align16(o);
    L.scr = o;                                  // FP64: partial sums; mixed: r/v prefetch
    o += precision == 1 ? (size_t)kWarps * kPrefBytes : sizeof(double) * kThreads * 5;
    L.ctab = o; o += sizeof(double) * kWarps * 9;   // mixed: neighbour cell centres
    L.tab = o;  o += sizeof(int2) * kWarps * 32;     // mixed: neighbour cell table per warp
    L.red = o;  o += sizeof(double) * kWarps * 3;
    L.ctr = o;  o += 16;
    L.total = align16(o);
    return L;
}

__device__ __forceinline__ int wrap_index(int i, int n)
{
    return i < 0 ? i + n : (i >= n ? i - n : i);
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

// Unrolling of the 27-cell stencil loops of the mixed force routine.
#ifndef DSEA_CELL_UNROLL
#define DSEA_CELL_UNROLL _Pragma("unroll 1")
#endif

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

// Accumulators of the two home atoms a lane carries (packed halves).
struct Acc2 {
    float2 fx, fy, fz, u, w;
};

// Two home atoms (XS, YS, ZS: already in the neighbour cell's frame) against
// one staged neighbour.  EXACT: the cutoff test also excludes r2 == 0 (the
// atom itself; needed in the home cell) and masks the energy terms; otherwise
// the force is masked by multiplying with the 0/1 cutoff mask, which gives
// the same bits for every pair of distinct atoms.
template <bool EXACT, bool OBS>
__device__ __forceinline__ void pair2(const float2 XS, const float2 YS, const float2 ZS, const float4 pj,
                                      float rc2f, unsigned rcb, float ushiftf, Acc2 &a)
{
    const float2 DX = f2sub(XS, f2splat(pj.x));
    const float2 DY = f2sub(YS, f2splat(pj.y));
    const float2 DZ = f2sub(ZS, f2splat(pj.z));
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

// Mixed-form forces on the atoms of one home cell chunk (nin <= 32 atoms
// starting at staged index `base`), warp-wide.  Each lane carries two home
// atoms and evaluates both against the same staged neighbour with packed
// FP32x2 arithmetic; lanes split each neighbour cell's atoms by stride ns.
// The ns partial sums of an atom are then combined in split order, so each
// atom's force is summed in an order fixed by the box state.  Lane l < nin
// returns the totals of atom base + l.
template <bool OBS>
__device__ __forceinline__ void packed_forces(const BoxDev &B, const float4 *s_q, const int *s_start,
                                              const int *s_cnt, int2 *tab, int hx, int hy, int hz, int EY,
                                              int EZ, int base, int nin, int lane, float &fx, float &fy,
                                              float &fz, float &uu, float &ww)
{
    const int np = (nin + 1) >> 1;
    const float inv_np = inv_of(np);
    const int ns = qdiv(32, inv_np);
    const int g = qdiv(lane, inv_np), pi = lane - g * np;
    const bool act = g < ns;
    const int a0 = 2 * pi, a1 = min(2 * pi + 1, nin - 1);   // odd nin: the last pair repeats an atom
    Acc2 acc = {f2splat(0.f), f2splat(0.f), f2splat(0.f), f2splat(0.f), f2splat(0.f)};
    // table of the 26 neighbour cells: staged start and prefix of the counts
    // (lane 26 holds the total), so the cells read as one list
    {
        int cs = 0, cn = 0;
        if (lane < 26) {
            const int kk = lane + (lane >= 13 ? 1 : 0);
            const int ox = kk / 9 - 1, oy = (kk / 3) % 3 - 1, oz = kk % 3 - 1;
            const int kn = ((hx + 1 + ox) * EY + (hy + 1 + oy)) * EZ + (hz + 1 + oz);
            cs = s_start[kn];
            cn = s_cnt[kn];
        }
        int incl = cn;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane <= 26) tab[lane] = make_int2(cs, incl - cn);
        __syncwarp();
    }
    if (act) {
        const float4 q0 = s_q[base + a0], q1 = s_q[base + a1];
        const float2 X = make_float2(q0.x, q1.x), Y = make_float2(q0.y, q1.y), Z = make_float2(q0.z, q1.z);
        const unsigned rcb = __float_as_uint(B.rc2f);
        const float rc2f = B.rc2f, ush = B.ushiftf;
        // the home cell (it holds the atoms themselves: exact test), split by stride
        {
            const int kh = ((hx + 1) * EY + (hy + 1)) * EZ + (hz + 1);
            const float4 *qc = s_q + s_start[kh];
            const int cn = s_cnt[kh];
            for (int t = g; t < cn; t += ns) pair2<true, OBS>(X, Y, Z, qc[t], rc2f, rcb, ush, acc);
        }
        // the 26 neighbour cells as one list, an equal contiguous share per split
        const int M = tab[26].y;
        const int chunk = qdiv(M + ns - 1, inv_of(ns));
        int t = g * chunk;
        const int e = min(M, t + chunk);
        if (t < e) {
            int lo = 0, hi = 25;   // the cell holding list position t
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (tab[mid].y <= t) lo = mid; else hi = mid - 1;
            }
            int k = lo;
            int end = tab[k + 1].y, off = tab[k].x - tab[k].y;
            float2 XS, YS, ZS;
            auto frame = [&](int kc) {   // home atoms in neighbour cell kc's centred frame
                const int kk = kc + (kc >= 13 ? 1 : 0);
                XS = f2sub(X, f2splat((float)(kk / 9 - 1) * B.lcf[0]));
                YS = f2sub(Y, f2splat((float)((kk / 3) % 3 - 1) * B.lcf[1]));
                ZS = f2sub(Z, f2splat((float)(kk % 3 - 1) * B.lcf[2]));
            };
            frame(k);
            for (; t < e; ++t) {
                while (t == end) {   // next non-empty cell
                    ++k;
                    end = tab[k + 1].y;
                    off = tab[k].x - tab[k].y;
                    frame(k);
                }
                if (OBS) pair2<true, true>(XS, YS, ZS, s_q[off + t], rc2f, rcb, ush, acc);
                else pair2<false, false>(XS, YS, ZS, s_q[off + t], rc2f, rcb, ush, acc);
            }
        }
    }
    const float2 FX = acc.fx, FY = acc.fy, FZ = acc.fz, UU = acc.u, WW = acc.w;
    // combine the ns partials of each atom pair into lane pi, in split order
    float2 SX = FX, SY = FY, SZ = FZ, SU = UU, SW = WW;
    for (int gg = 1; gg < ns; ++gg) {
        const int src = pi + gg * np;   // < ns * np <= 32
        SX.x += __shfl_sync(kFull, FX.x, src); SX.y += __shfl_sync(kFull, FX.y, src);
        SY.x += __shfl_sync(kFull, FY.x, src); SY.y += __shfl_sync(kFull, FY.y, src);
        SZ.x += __shfl_sync(kFull, FZ.x, src); SZ.y += __shfl_sync(kFull, FZ.y, src);
        if (OBS) {
            SU.x += __shfl_sync(kFull, UU.x, src); SU.y += __shfl_sync(kFull, UU.y, src);
            SW.x += __shfl_sync(kFull, WW.x, src); SW.y += __shfl_sync(kFull, WW.y, src);
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

// One candidate pair in FP64 on absolute (periodically shifted) positions.
template <bool OBS>
__device__ __forceinline__ void pair_f64(double xi, double yi, double zi, double xj, double yj,
                                         double zj, double rc2, double ushift, Acc64 &a)
{
    const double dx = xi - xj, dy = yi - yj, dz = zi - zj;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 <= rc2 && r2 > 0.0) {
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
    const int k = reserve_slot(B.arr[pn], dest, own && !stay, tag, lane, B.err);
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
    B.id[pn][slot] = aid;
    B.r[pn][slot] = x;
    B.r[pn][S + slot] = y;
    B.r[pn][2 * S + slot] = z;
    B.v[pn][slot] = vx;
    B.v[pn][S + slot] = vy;
    B.v[pn][2 * S + slot] = vz;
}

// Write one atom into slot `slot` of buffer `pn` (mixed form): FP64 absolute
// position, FP32 velocity, FP32 coordinates relative to its cell centre.
__device__ __forceinline__ void store_mixed(const BoxDev &B, int pn, long long slot, int aid, double x,
                                            double y, double z, float vx, float vy, float vz, float qx,
                                            float qy, float qz)
{
    const long long S = B.n_slots;
    B.id[pn][slot] = aid;
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

// Destination of a mixed-form atom along one axis.  The atom sat in home cell
// `cg` with FP32 coordinate q relative to its centre and moved by d (FP32).
// Returns the unwrapped destination cell and sets the new FP32 coordinate
// relative to that cell's centre (from the FP64 position) and the wrapped
// FP64 position.  ctab3 holds the FP64 centres of cells cg-1, cg, cg+1.
__device__ __forceinline__ int move_axis(double &r, float q, float d, int cg, const double *ctab3,
                                         double lc, float inv_lcf, double L, int nc, float &qn)
{
    const int o = (int)floorf(fmaf(q + d, inv_lcf, 0.5f));   // cell offset, usually -1, 0 or 1
    const int cu = cg + o;
    const double ru = r + (double)d;                         // FP64 position update (unwrapped)
    const double cen = (o >= -1 && o <= 1) ? ctab3[o + 1] : ((double)cu + 0.5) * lc;
    qn = (float)(ru - cen);
    int c = cu;
    double rw = ru;
    if (c < 0) {
        c += nc;
        rw += L;
    } else if (c >= nc) {
        c -= nc;
        rw -= L;
    }
    r = rw;
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// The work unit (see file header).  s_abs: absolute step of the input state.
template <int PREC, bool INTEGRATE, bool OBS>
__device__ void run_unit(const BoxDev &B, int j, int tile, long long s_abs, bool first_step,
                         int unit_id, char *smem)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int p = (int)(s_abs & 1);
    const unsigned tag = (unsigned)(s_abs + 1);
    const Layout Ly = make_layout(PREC, B.staged_cells, B.smem_atoms);
    int *s_cnt = reinterpret_cast<int *>(smem + Ly.cnt);
    int *s_nst = reinterpret_cast<int *>(smem + Ly.nst);
    int *s_start = reinterpret_cast<int *>(smem + Ly.start);
    int *s_gcell = reinterpret_cast<int *>(smem + Ly.gcell);
    int *s_slot = reinterpret_cast<int *>(smem + Ly.slot);
    double *s_red = reinterpret_cast<double *>(smem + Ly.red);
    int *s_ctr = reinterpret_cast<int *>(smem + Ly.ctr);
    float4 *s_q = reinterpret_cast<float4 *>(smem + Ly.atoms);
    double *s_x = reinterpret_cast<double *>(smem + Ly.atoms);
    double *s_y = s_x + B.smem_atoms;
    double *s_z = s_y + B.smem_atoms;
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
    if (tid == 0) *s_ctr = 0;
    for (int k = tid; k < n_staged; k += kThreads) {
        const int lx = qdiv(k, inv_eyez), rem = k - lx * EY * EZ, ly = qdiv(rem, inv_ez), lz = rem - ly * EZ;
        const int gx = wrap_index(x0 - 1 + lx, B.nc[0]);
        const int gy = wrap_index(y0 - 1 + ly, B.nc[1]);
        const int gz = wrap_index(z0 - 1 + lz, B.nc[2]);
        const int gc = (gx * B.nc[1] + gy) * B.nc[2] + gz;
        const unsigned long long ws = __ldcg(B.cnt[p] + gc), wa = __ldcg(B.arr[p] + gc);
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
    // slots) as they are, then the arrivals (back slots) ordered by atom id.
    // Mixed form: every warp issues asynchronous 16-byte copies of its cells'
    // two slot ranges and moves on; after one wait and barrier, each cell's
    // arrivals are ordered in place.  FP64 form: lanes load their atoms (L2)
    // and write them to their place.
    const long long S = B.n_slots;
    if (PREC == 1) {
        for (int k = warp; k < n_staged; k += kWarps) {
            const int c = s_cnt[k];
            if (c == 0) continue;
            const int n_s = s_nst[k], n_a = c - n_s;
            const long long base = (long long)s_gcell[k] * B.cap;
            const int st = s_start[k];
            for (int a = lane; a < c; a += 32) {
                const long long src = a < n_s ? base + a : base + B.cap - n_a + (a - n_s);
                cp_async16(s_q + st + a, B.q[p] + src);
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }
    for (int k = warp; k < n_staged; k += kWarps) {
        const int c = s_cnt[k];
        if (c == 0) continue;
        const int n_s = s_nst[k], n_a = c - n_s;
        const long long base = (long long)s_gcell[k] * B.cap;
        const int st = s_start[k];
        double shx = 0.0, shy = 0.0, shz = 0.0;
        if (PREC == 0) {   // periodic image shift of this staged cell
            const int lx = qdiv(k, inv_eyez), rem = k - lx * EY * EZ, ly = qdiv(rem, inv_ez), lz = rem - ly * EZ;
            const int ux = x0 - 1 + lx, uy = y0 - 1 + ly, uz = z0 - 1 + lz;
            shx = ux < 0 ? -B.L[0] : (ux >= B.nc[0] ? B.L[0] : 0.0);
            shy = uy < 0 ? -B.L[1] : (uy >= B.nc[1] ? B.L[1] : 0.0);
            shz = uz < 0 ? -B.L[2] : (uz >= B.nc[2] ? B.L[2] : 0.0);
        }
        for (int a = lane; a < n_s; a += 32) {
            const long long slot = base + a;
            s_slot[st + a] = (int)slot;
            if (PREC == 0) {
                s_x[st + a] = __ldcg(B.r[p] + slot) + shx;
                s_y[st + a] = __ldcg(B.r[p] + S + slot) + shy;
                s_z[st + a] = __ldcg(B.r[p] + 2 * S + slot) + shz;
                s_id[st + a] = __ldcg(B.id[p] + slot);
            }
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
        float4 qm[4];
        double xm[4], ym[4], zm[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int a = lane + 32 * m;
            idm[m] = 0x7fffffff;
            if (m < nm && a < n_a) {
                if (PREC == 1) {
                    qm[m] = s_q[fa + a];
                    idm[m] = __float_as_int(qm[m].w);
                } else {
                    const long long slot = abase + a;
                    xm[m] = __ldcg(B.r[p] + slot) + shx;
                    ym[m] = __ldcg(B.r[p] + S + slot) + shy;
                    zm[m] = __ldcg(B.r[p] + 2 * S + slot) + shz;
                    idm[m] = __ldcg(B.id[p] + slot);
                }
            }
        }
        int rk[4] = {0, 0, 0, 0};
        if (nm == 1) {
            for (int t = 0; t < n_a; ++t) rk[0] += (__shfl_sync(kFull, idm[0], t) < idm[0]) ? 1 : 0;
        } else {
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
        }
        __syncwarp();   // every lane has read the arrivals before any writes
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int a = lane + 32 * m;
            if (m < nm && a < n_a) {
                const int dst = fa + rk[m];
                s_slot[dst] = (int)(abase + a);
                if (PREC == 1) {
                    s_q[dst] = qm[m];
                } else {
                    s_x[dst] = xm[m];
                    s_y[dst] = ym[m];
                    s_z[dst] = zm[m];
                    s_id[dst] = idm[m];
                }
            }
        }
    }
    __syncthreads();

    // 4./5. forces, then kick, drift and rebin, warp per home cell.  Without
    // a reduction the home cells are handed out dynamically; with one, in a
    // fixed order so that the unit's partial sums are reproducible.
    double red_u = 0.0, red_w = 0.0, red_k = 0.0;
    const int n_home = nx * ny * nz;
    const int pn = p ^ 1;
    const unsigned tag_next = tag + 1u;
    const double dt = B.dt;
    const double kick = first_step ? 0.5 * dt : dt;
    const float dtf = (float)dt;
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
        const int cg[3] = {x0 + hx, y0 + hy, z0 + hz};   // home cell (within the box)
        const long long hcell = s_gcell[kh];
        int n_stay = 0;   // atoms of this cell that stay in it, written to its front slots in order
        double *ctab = reinterpret_cast<double *>(smem + Ly.ctab) + warp * 9;
        if (PREC == 1) {
            if (lane < 9) {
                const int ax = lane / 3, o = lane - 3 * (lane / 3) - 1;
                ctab[lane] = ((double)(cg[ax] + o) + 0.5) * B.lc[ax];
            }
            __syncwarp();
        }
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
            if (PREC == 1) {
                // prefetch the home cell's positions (FP64) and velocities (FP32)
                // in slot order, 16-byte copies, while the forces are computed
                // (cells of up to 32 atoms; larger ones are read after)
                char *pref = smem + Ly.scr + (size_t)warp * kPrefBytes;
                double *pr = reinterpret_cast<double *>(pref);          // [3][32]
                float *pv = reinterpret_cast<float *>(pref + 32 * 3 * 8);  // [3][32]
                const long long hbase = (long long)s_gcell[kh] * B.cap;
                const int n_front = s_nst[kh];   // stayers: slots [0, n_front); arrivals at the back
                const bool pf = n_front <= 32;
                if (pf) {
                    const int n2 = (n_front + 1) >> 1, n4 = (n_front + 3) >> 2;
                    for (int d = 0; d < 3; ++d) {
                        if (lane < n2) cp_async16(pr + 32 * d + 2 * lane, B.r[p] + d * S + hbase + 2 * lane);
                        if (lane < n4) cp_async16(pv + 32 * d + 4 * lane, B.vf[p] + d * S + hbase + 4 * lane);
                    }
                }
                float fx = 0.f, fy = 0.f, fz = 0.f, uu = 0.f, ww = 0.f;
                packed_forces<OBS>(B, s_q, s_start, s_cnt, reinterpret_cast<int2 *>(smem + Ly.tab) + warp * 32,
                                   hx, hy, hz, EY, EZ, hs + ib, nin, lane, fx,
                                   fy, fz, uu, ww);
                cp_async_wait_all();
                __syncwarp();
                int aid = 0;
                double rr[3] = {0.0, 0.0, 0.0};
                float vv[3] = {0.f, 0.f, 0.f};
                float4 qo = make_float4(0.f, 0.f, 0.f, 0.f);
                if (own) {
                    qo = s_q[is];
                    aid = __float_as_int(qo.w);
                    for (int d = 0; d < 3; ++d) {
                        const int a = (int)(slot - hbase);
                        const bool hit = pf && a < n_front;
                        rr[d] = hit ? pr[32 * d + a] : __ldcg(B.r[p] + d * S + slot);
                        vv[d] = hit ? pv[32 * d + a] : __ldcg(B.vf[p] + d * S + slot);
                    }
                    if (OBS) {
                        // synchronised velocity v(t) = v(t - dt/2) + F dt/2 (v(t0) itself at the start)
                        const float hk = first_step ? 0.f : 0.5f * dtf;
                        const float sx = fmaf(hk, fx, vv[0]), sy = fmaf(hk, fy, vv[1]), sz = fmaf(hk, fz, vv[2]);
                        red_u += 0.5 * (double)uu;
                        red_w += 0.5 * (double)ww;
                        red_k += 0.5 * (double)fmaf(sx, sx, fmaf(sy, sy, sz * sz));
                        if (!INTEGRATE) {
                            const long long o = 3LL * aid;
                            B.out_f[o] = fx; B.out_f[o + 1] = fy; B.out_f[o + 2] = fz;
                            B.out_v[o] = sx; B.out_v[o + 1] = sy; B.out_v[o + 2] = sz;
                            B.out_r[o] = rr[0]; B.out_r[o + 1] = rr[1]; B.out_r[o + 2] = rr[2];
                        }
                    }
                }
                __syncwarp();   // the prefetch area is reused by the next chunk
                if (INTEGRATE) {
                    long long dest = 0;
                    float qn[3] = {0.f, 0.f, 0.f};
                    if (own) {
                        const float kf = first_step ? 0.5f * dtf : dtf;
                        vv[0] = fmaf(kf, fx, vv[0]);   // v(t + dt/2) = v(t - dt/2) + F dt
                        vv[1] = fmaf(kf, fy, vv[1]);
                        vv[2] = fmaf(kf, fz, vv[2]);
                        const float q3[3] = {qo.x, qo.y, qo.z};
                        int c3[3];
                        for (int d = 0; d < 3; ++d)   // r(t + dt) = r(t) + v(t + dt/2) dt, in FP64
                            c3[d] = move_axis(rr[d], q3[d], vv[d] * dtf, cg[d], ctab + 3 * d, B.lc[d],
                                              1.0f / B.lcf[d], B.L[d], B.nc[d], qn[d]);
                        const int dj = qdiv(c3[0], inv_cps) - j;
                        const int djm = dj < -1 ? dj + B.n_slices : (dj > 1 ? dj - B.n_slices : dj);
                        if (djm < -1 || djm > 1) set_error(B.err, kErrMigration);
                        dest = ((long long)c3[0] * B.nc[1] + c3[1]) * B.nc[2] + c3[2];
                    }
                    const long long slot_n = place_slot(B, pn, hcell, dest, own, tag_next, lane, n_stay);
                    if (slot_n >= 0)
                        store_mixed(B, pn, slot_n, aid, rr[0], rr[1], rr[2], vv[0], vv[1], vv[2], qn[0], qn[1],
                                    qn[2]);
                }
            } else {
                Acc64 a64 = {0.0, 0.0, 0.0, 0.0, 0.0};
                if (act) {
                    const double xi = s_x[is], yi = s_y[is], zi = s_z[is];
                    for (int ox = -1; ox <= 1; ++ox)
                        for (int oy = -1; oy <= 1; ++oy)
                            for (int oz = -1; oz <= 1; ++oz) {
                                const int kn = ((hx + 1 + ox) * EY + (hy + 1 + oy)) * EZ + (hz + 1 + oz);
                                const int cs = s_start[kn], cn = s_cnt[kn];
                                for (int t = g; t < cn; t += ns)
                                    pair_f64<OBS>(xi, yi, zi, s_x[cs + t], s_y[cs + t], s_z[cs + t],
                                                  B.rc2, B.ushift, a64);
                            }
                }
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
                        if (!INTEGRATE) {
                            const long long o = 3LL * aid;
                            B.out_f[o] = fx; B.out_f[o + 1] = fy; B.out_f[o + 2] = fz;
                            B.out_v[o] = sx; B.out_v[o + 1] = sy; B.out_v[o + 2] = sz;
                            B.out_r[o] = rx; B.out_r[o + 1] = ry; B.out_r[o + 2] = rz;
                        }
                    }
                }
                if (INTEGRATE) {
                    long long dest = 0;
                    if (own) {
                        vx += kick * fx;   // v(t + dt/2) = v(t - dt/2) + F dt
                        vy += kick * fy;
                        vz += kick * fz;
                        rx = wrap_coord(rx + vx * dt, B.L[0]);   // r(t + dt) = r(t) + v(t + dt/2) dt
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
            }
            __syncwarp();
        }
        // every home cell publishes how many atoms stayed in it, empty or not
        if (INTEGRATE && lane == 0)
            B.cnt[pn][hcell] = ((unsigned long long)tag_next << 32) | (unsigned long long)n_stay;
        if (OBS) {
            h += kWarps;
        } else {
            if (lane == 0) h = atomicAdd(s_ctr, 1);
            h = __shfl_sync(kFull, h, 0);
        }
    }
    if (OBS) {
        // fixed-order FP64 reduction: xor tree in the warp, then warps in order
        for (int o = 16; o > 0; o >>= 1) {
            red_u += __shfl_xor_sync(kFull, red_u, o);
            red_w += __shfl_xor_sync(kFull, red_w, o);
            red_k += __shfl_xor_sync(kFull, red_k, o);
        }
        if (lane == 0) {
            s_red[warp * 3 + 0] = red_u;
            s_red[warp * 3 + 1] = red_w;
            s_red[warp * 3 + 2] = red_k;
        }
        __syncthreads();
        if (tid == 0) {
            double u = 0, w = 0, k = 0;
            for (int q = 0; q < kWarps; ++q) {
                u += s_red[q * 3];
                w += s_red[q * 3 + 1];
                k += s_red[q * 3 + 2];
            }
            B.unit_obs[3LL * unit_id] = u;
            B.unit_obs[3LL * unit_id + 1] = w;
            B.unit_obs[3LL * unit_id + 2] = k;
        }
    }
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
                // FP32 coordinates relative to the centre of the atom's cell
                const float qx = (float)(x - ((double)cx + 0.5) * B.lc[0]);
                const float qy = (float)(y - ((double)cy + 0.5) * B.lc[1]);
                const float qz = (float)(z - ((double)cz + 0.5) * B.lc[2]);
                store_mixed(B, p, slot, (int)i, x, y, z, (float)vx, (float)vy, (float)vz, qx, qy, qz);
            } else {
                store_f64(B, p, slot, (int)i, x, y, z, vx, vy, vz);
            }
        }
    }
}

template <int PREC, bool INTEGRATE, bool OBS>
__global__ void __launch_bounds__(kThreads) k_units(const BoxDev *bp, long long s_abs, int first)
{
    extern __shared__ __align__(16) char smem[];
    __shared__ BoxDev sB;
    if (threadIdx.x == 0) sB = *bp;
    __syncthreads();
    const int u = blockIdx.x;
    const int j = u / sB.units_per_slice, tile = u - j * sB.units_per_slice;
    run_unit<PREC, INTEGRATE, OBS>(sB, j, tile, s_abs, first != 0, u, smem);
}

__global__ void __launch_bounds__(256) k_obs_reduce(const double *unit_obs, int n, double *out3)
{
    __shared__ double s[3][256];
    double a = 0, b = 0, c = 0;
    for (int i = threadIdx.x; i < n; i += 256) {
        a += unit_obs[3LL * i];
        b += unit_obs[3LL * i + 1];
        c += unit_obs[3LL * i + 2];
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    s[2][threadIdx.x] = c;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
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

// The persistent ring: every CTA is one on-chip stage that repeatedly takes
// the next ticket, waits (bounded) until the five slices its unit reads at
// the previous level are complete, runs the unit and reports completion.
// Tickets are dispensed step-major and, within a step, slice by slice from
// an offset that advances two slices per step, so level s trails level s-1
// by about five slices (the time-skewed cyclic order of Sec. 3.1 / Table 1).
// A CTA only waits on tickets smaller than its own, all of which were taken
// by running CTAs, so the ring always progresses.
#ifndef DSEA_RING_MIN_BLOCKS
#define DSEA_RING_MIN_BLOCKS 4   // CTAs per SM the register allocation must allow
#endif
template <int PREC>
__global__ void __launch_bounds__(kThreads, DSEA_RING_MIN_BLOCKS) k_ring(RingPlan plan)
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
                        const int k = wrap_index(j + d, sB.n_slices);
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
            run_unit<PREC, true, false>(sB, j, tile, s_abs, s_rel == 0 && sB.w_is_sync, 0, smem);
        __threadfence();
        __syncthreads();
        if (tid == 0 && !(j == sB.withhold_slice && s_rel == 0)) atomicAdd(sB.done + j, 1u);
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
    return make_layout(precision, staged_cells, smem_atoms).total;
}

size_t max_unit_smem_bytes()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // the kernels also hold a static copy of the box descriptor and a few words
    return (size_t)v > 4096 ? (size_t)v - 4096 : 0;
}

cudaError_t launch_bin(const BoxDev &hb, const BoxDev *db, const double *pos, const double *vel,
                       cudaStream_t stream)
{
    if (hb.n_atoms == 0) return cudaSuccess;
    const long long blocks = (hb.n_atoms + kThreads - 1) / kThreads;
    const int grid = (int)(blocks < 65535 ? blocks : 65535);
    if (hb.precision == 1) k_bin<1><<<grid, kThreads, 0, stream>>>(db, pos, vel);
    else k_bin<0><<<grid, kThreads, 0, stream>>>(db, pos, vel);
    return cudaGetLastError();
}

template <int PREC, bool INTEGRATE, bool OBS>
static cudaError_t launch_units(const BoxDev &hb, const BoxDev *db, long long s_abs, int first,
                                cudaStream_t stream)
{
    const size_t smem = unit_smem_bytes(PREC, hb.staged_cells, hb.smem_atoms);
    cudaError_t e = set_smem(k_units<PREC, INTEGRATE, OBS>, smem);
    if (e != cudaSuccess) return e;
    const int grid = hb.n_slices * hb.units_per_slice;
    k_units<PREC, INTEGRATE, OBS><<<grid, kThreads, smem, stream>>>(db, s_abs, first);
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

cudaError_t launch_obs_reduce(const double *unit_obs, int n_units, double *out3, cudaStream_t stream)
{
    k_obs_reduce<<<1, 256, 0, stream>>>(unit_obs, n_units, out3);
    return cudaGetLastError();
}

cudaError_t launch_ring(const RingPlan &plan, int precision, size_t smem_bytes, int ctas,
                        cudaStream_t stream)
{
    if (plan.total == 0) return cudaSuccess;
    cudaError_t e;
    if (precision == 1) {
        e = set_smem(k_ring<1>, smem_bytes);
        if (e != cudaSuccess) return e;
        k_ring<1><<<ctas, kThreads, smem_bytes, stream>>>(plan);
    } else {
        e = set_smem(k_ring<0>, smem_bytes);
        if (e != cudaSuccess) return e;
        k_ring<0><<<ctas, kThreads, smem_bytes, stream>>>(plan);
    }
    return cudaGetLastError();
}

int ring_ctas_per_sm(int precision, size_t smem_bytes)
{
    int n = 0;
    if (precision == 1) {
        set_smem(k_ring<1>, smem_bytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ring<1>, kThreads, smem_bytes);
    } else {
        set_smem(k_ring<0>, smem_bytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ring<0>, kThreads, smem_bytes);
    }
    return n;
}

}  // namespace dsea
