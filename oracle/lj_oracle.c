/*
 * lj_oracle.c -- plain, slow, FP64 CPU reference for the truncated-shifted
 * Lennard-Jones NVE velocity-Verlet step of the paper's molecular-dynamics
 * case study (Sec. 4, Algorithm 1).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or constant with the CUDA path of this repository.
 *
 * Units are reduced Lennard-Jones units: sigma = epsilon = m = 1 (Sec. 4).
 * Positions are absolute Cartesian coordinates in a periodic orthorhombic
 * box [0,Lx) x [0,Ly) x [0,Lz); all arrays are AoS xyz, atom i at [3i..3i+2].
 *
 * Readings of the paper used here (each is listed with its reason in the
 * project's design notes):
 *   - pair force: F_abs = 24 (2 r^-12 - r^-6) / r^2, F_i += r_ij F_abs with
 *     r_ij = r_i - r_j (Algorithm 1);
 *   - cutoff test is inclusive, r^2 <= rc^2 (Algorithm 1);
 *   - "truncated and shifted" (Sec. 4) means u(rc) = 0, so the energy of a
 *     pair is u = 4 (r^-12 - r^-6) - 4 (rc^-12 - rc^-6); the force is not
 *     shifted;
 *   - the virial reported is the physical W = sum_{i<j} r_ij . F_ij, which is
 *     24 times the quantity Algorithm 1 accumulates as V;
 *   - by default all three axes are periodic with the minimum-image
 *     convention (the workloads ask for a periodic box); with walls_x set,
 *     the x axis instead ends in mirror walls at x = 0 and x = Lx (Sec. 3
 *     requirement (3) keeps x non-periodic; Sec. 4.2 places a mirror at the
 *     domain boundaries): no pair interacts across them, and an atom whose
 *     update takes it past a wall is mirrored back -- its x coordinate is
 *     reflected in the wall and the x components of its velocity and of the
 *     force it carries into the next velocity update change sign (a
 *     specular wall; the paper does not describe the mirror further);
 *   - step 1 of Algorithm 1 starts with F_old := -F(r_0), so the first
 *     velocity update leaves v_0 unchanged and the loop is standard velocity
 *     Verlet; a run of n steps ends with one more force evaluation at r_n and
 *     the closing half kick, so the returned state is synchronised
 *     (r_n, v_n, F_n).
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Planted-mistake builds for the mutation tests (tests/test_oracle_mutants.py):
 * 0 = the oracle as written; any other value compiles one deliberate error so the
 * tests can show that the pins detect it.  Never set outside those tests. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG -1
#define ORACLE_ERR_CELLS -2
#define ORACLE_ERR_OOM -3

/* Energy shift so that the pair energy vanishes at rc (Sec. 4: truncated and
 * shifted LJ 12-6). */
static double lj_shift(double rc)
{
    double rc2i = 1.0 / (rc * rc);
    double rc6i = rc2i * rc2i * rc2i;
    return -4.0 * (rc6i * rc6i - rc6i);
}

/* One pair at squared distance r2 <= rc^2, Algorithm 1: returns F_abs (the
 * factor that multiplies the separation vector r_ij) and the shifted energy
 * of the pair. */
static void lj_pair_terms(double r2, double ushift, double *fabs_out, double *u_out)
{
    double r2i = 1.0 / r2;
    double r6i = r2i * r2i * r2i;    /* sigma^6 / r^6  */
    double r12i = r6i * r6i;         /* sigma^12 / r^12 */
    *fabs_out = 24.0 * ((ORACLE_MUTANT == 1 ? 1.0 : 2.0) * r12i - r6i) * r2i;
    *u_out = 4.0 * (r12i - r6i) + (ORACLE_MUTANT == 2 ? -ushift : ushift);
}

/* Minimum-image component of a separation along a periodic axis of length L. */
static double min_image(double d, double L)
{
    return ORACLE_MUTANT == 3 ? d : d - L * nearbyint(d / L);
}

/* Separation along axis `axis`: minimum image, except along x between mirror
 * walls, where there is no periodic image. */
static double sep(double d, const double *box, int axis, int walls_x)
{
    if (axis == 0 && walls_x && ORACLE_MUTANT != 10) return d;
    return min_image(d, box[axis]);
}

/* Pair energy and radial force (positive = repulsive) of one pair at distance
 * r; zero beyond rc.  A closed-form probe of the pair law. */
int oracle_pair(double r, double rc, double *force_radial, double *energy)
{
    if (!(r > 0.0) || !(rc > 0.0) || !force_radial || !energy) return ORACLE_ERR_ARG;
    double r2 = r * r;
    if (ORACLE_MUTANT == 8 ? r2 < rc * rc : r2 <= rc * rc) {
        double fa, u;
        lj_pair_terms(r2, lj_shift(rc), &fa, &u);
        *force_radial = fa * r;
        *energy = u;
    } else {
        *force_radial = 0.0;
        *energy = 0.0;
    }
    return ORACLE_OK;
}

/* O(N^2) minimum-image sum over unordered pairs i<j, each pair applied to
 * both atoms (Newton's third law).  F: out, 3n.  U, W: out, totals.
 * walls_x: mirror walls along x (no periodic image along x). */
int oracle_forces_brute_w(int64_t n, const double *pos, const double *box, double rc, int walls_x,
                          double *F, double *U, double *W)
{
    if (n < 0 || !pos || !box || !F || !U || !W || !(rc > 0.0)) return ORACLE_ERR_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(box[d] >= 2.0 * rc)) return ORACLE_ERR_ARG; /* minimum image needs L >= 2 rc */
    double rc2 = rc * rc, ushift = lj_shift(rc);
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    double u_sum = 0.0, w_sum = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = sep(pos[3 * i + 0] - pos[3 * j + 0], box, 0, walls_x);
            double dy = sep(pos[3 * i + 1] - pos[3 * j + 1], box, 1, walls_x);
            double dz = sep(pos[3 * i + 2] - pos[3 * j + 2], box, 2, walls_x);
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 <= rc2) {
                double fa, u;
                lj_pair_terms(r2, ushift, &fa, &u);
                F[3 * i + 0] += dx * fa; F[3 * j + 0] -= dx * fa;
                F[3 * i + 1] += dy * fa; F[3 * j + 1] -= dy * fa;
                F[3 * i + 2] += dz * fa; F[3 * j + 2] -= dz * fa;
                u_sum += u;
                w_sum += r2 * fa; /* r_ij . F_ij = r^2 F_abs */
            }
        }
    }
    *U = u_sum;
    *W = w_sum;
    return ORACLE_OK;
}

int oracle_forces_brute(int64_t n, const double *pos, const double *box, double rc, double *F, double *U,
                        double *W)
{
    return oracle_forces_brute_w(n, pos, box, rc, 0, F, U, W);
}

/* Linked-cell list (a textbook cell list, Sec. 4): cells of edge
 * l_d = L_d / floor(L_d / rc) >= rc along each axis. */
typedef struct {
    int nc[3];
    double cl[3];
    int64_t *head; /* first atom of each cell, -1 if empty */
    int64_t *next; /* next atom in the same cell, -1 at the end */
} cell_list;

static int cell_coord(double x, double L, double cl, int nc)
{
    double w = x - L * floor(x / L); /* wrap into [0, L) */
    int c = (int)floor(w / cl);
    if (c < 0) c = 0;
    if (c >= nc) c = nc - 1;
    return c;
}

static int build_cells(int64_t n, const double *pos, const double *box, double rc, cell_list *cl)
{
    for (int d = 0; d < 3; ++d) {
        cl->nc[d] = (int)floor(box[d] / rc);
        if (cl->nc[d] < 3) return ORACLE_ERR_CELLS; /* 27 distinct neighbour cells need >= 3 */
        cl->cl[d] = box[d] / cl->nc[d];
    }
    int64_t ncell = (int64_t)cl->nc[0] * cl->nc[1] * cl->nc[2];
    cl->head = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    cl->next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!cl->head || !cl->next) {
        free(cl->head);
        free(cl->next);
        return ORACLE_ERR_OOM;
    }
    for (int64_t c = 0; c < ncell; ++c) cl->head[c] = -1;
    /* insert in reverse so each cell lists its atoms in increasing index order */
    for (int64_t i = n - 1; i >= 0; --i) {
        int cx = cell_coord(pos[3 * i + 0], box[0], cl->cl[0], cl->nc[0]);
        int cy = cell_coord(pos[3 * i + 1], box[1], cl->cl[1], cl->nc[1]);
        int cz = cell_coord(pos[3 * i + 2], box[2], cl->cl[2], cl->nc[2]);
        int64_t c = ((int64_t)cx * cl->nc[1] + cy) * cl->nc[2] + cz;
        cl->next[i] = cl->head[c];
        cl->head[c] = i;
    }
    return ORACLE_OK;
}

static void free_cells(cell_list *cl)
{
    free(cl->head);
    free(cl->next);
}

/* Force, half pair energy and half pair virial on atom i from the atoms of its
 * 27 neighbour cells, as the first loop of Algorithm 1 does per molecule:
 * every neighbour j within rc adds r_ij F_abs to F_i, half of the pair energy
 * to U and half of the pair virial to W. */
static void atom_from_cells(int64_t i, const double *pos, const double *box, double rc2,
                            double ushift, int walls_x, const cell_list *cl, double *f3,
                            double *u_half, double *w_half)
{
    int c0[3];
    for (int d = 0; d < 3; ++d) c0[d] = cell_coord(pos[3 * i + d], box[d], cl->cl[d], cl->nc[d]);
    double fx = 0.0, fy = 0.0, fz = 0.0, uu = 0.0, ww = 0.0;
    for (int ox = -1; ox <= 1; ++ox)
        for (int oy = -1; oy <= 1; ++oy)
            for (int oz = -1; oz <= (ORACLE_MUTANT == 4 ? 0 : 1); ++oz) {
                if (walls_x && (c0[0] + ox < 0 || c0[0] + ox >= cl->nc[0])) continue; /* beyond a wall */
                int cx = (c0[0] + ox + cl->nc[0]) % cl->nc[0];
                int cy = (c0[1] + oy + cl->nc[1]) % cl->nc[1];
                int cz = (c0[2] + oz + cl->nc[2]) % cl->nc[2];
                int64_t c = ((int64_t)cx * cl->nc[1] + cy) * cl->nc[2] + cz;
                for (int64_t j = cl->head[c]; j >= 0; j = cl->next[j]) {
                    if (j == i) continue;
                    double dx = sep(pos[3 * i + 0] - pos[3 * j + 0], box, 0, walls_x);
                    double dy = sep(pos[3 * i + 1] - pos[3 * j + 1], box, 1, walls_x);
                    double dz = sep(pos[3 * i + 2] - pos[3 * j + 2], box, 2, walls_x);
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 <= rc2) {
                        double fa, u;
                        lj_pair_terms(r2, ushift, &fa, &u);
                        fx += dx * fa;
                        fy += dy * fa;
                        fz += dz * fa;
                        uu += 0.5 * u;
                        ww += 0.5 * (ORACLE_MUTANT == 7 ? 1.0 : r2) * fa;
                    }
                }
            }
    f3[0] = fx;
    f3[1] = fy;
    f3[2] = fz;
    *u_half = uu;
    *w_half = ww;
}

/* Cell-list force on every atom (27-cell stencil, directed pairs).  The atoms
 * are independent, so with OpenMP they are shared among threads; each atom's
 * sum, and the U and W sums over atoms (taken afterwards in atom order), are
 * the same with any thread count. */
int oracle_forces_cells_w(int64_t n, const double *pos, const double *box, double rc, int walls_x,
                          double *F, double *U, double *W)
{
    if (n < 0 || !pos || !box || !F || !U || !W || !(rc > 0.0)) return ORACLE_ERR_ARG;
    cell_list cl;
    int rcode = build_cells(n, pos, box, rc, &cl);
    if (rcode) return rcode;
    double *half = (double *)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    if (!half) {
        free_cells(&cl);
        return ORACLE_ERR_OOM;
    }
    double rc2 = rc * rc, ushift = lj_shift(rc), u_sum = 0.0, w_sum = 0.0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        atom_from_cells(i, pos, box, rc2, ushift, walls_x, &cl, &F[3 * i], &half[2 * i], &half[2 * i + 1]);
    for (int64_t i = 0; i < n; ++i) {
        u_sum += half[2 * i];
        w_sum += half[2 * i + 1];
    }
    free(half);
    free_cells(&cl);
    *U = u_sum;
    *W = w_sum;
    return ORACLE_OK;
}

/* Threads of the OpenMP force loop (n <= 0: the runtime's default, all
 * cores); returns the count now in effect (1 without OpenMP). */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int oracle_forces_cells(int64_t n, const double *pos, const double *box, double rc, double *F, double *U,
                        double *W)
{
    return oracle_forces_cells_w(n, pos, box, rc, 0, F, U, W);
}

/* Force and per-atom half energy / half virial for a subset of atoms only
 * (idx[0..m-1]); used to check sampled atoms of boxes too large for a full
 * oracle pass.  F: out, 3m; u_atom, w_atom: out, m (may be NULL). */
int oracle_forces_subset_w(int64_t n, const double *pos, const double *box, double rc, int walls_x,
                           int64_t m, const int64_t *idx, double *F, double *u_atom, double *w_atom)
{
    if (n < 0 || m < 0 || !pos || !box || !idx || !F || !(rc > 0.0)) return ORACLE_ERR_ARG;
    for (int64_t k = 0; k < m; ++k)
        if (idx[k] < 0 || idx[k] >= n) return ORACLE_ERR_ARG;
    cell_list cl;
    int rcode = build_cells(n, pos, box, rc, &cl);
    if (rcode) return rcode;
    double rc2 = rc * rc, ushift = lj_shift(rc);
    for (int64_t k = 0; k < m; ++k) {
        double uh, wh;
        const int64_t i = ORACLE_MUTANT == 14 ? (idx[k] + 1) % n : idx[k];
        atom_from_cells(i, pos, box, rc2, ushift, walls_x, &cl, &F[3 * k], &uh, &wh);
        if (u_atom) u_atom[k] = uh;
        if (w_atom) w_atom[k] = wh;
    }
    free_cells(&cl);
    return ORACLE_OK;
}

int oracle_forces_subset(int64_t n, const double *pos, const double *box, double rc, int64_t m,
                         const int64_t *idx, double *F, double *u_atom, double *w_atom)
{
    return oracle_forces_subset_w(n, pos, box, rc, 0, m, idx, F, u_atom, w_atom);
}

static int forces_any(int use_cells, int64_t n, const double *pos, const double *box, double rc, int walls_x,
                      double *F, double *U, double *W)
{
    return use_cells ? oracle_forces_cells_w(n, pos, box, rc, walls_x, F, U, W)
                     : oracle_forces_brute_w(n, pos, box, rc, walls_x, F, U, W);
}

static double kinetic(int64_t n, const double *vel)
{
    double s = 0.0;
    for (int64_t k = 0; k < 3 * n; ++k) s += vel[k] * vel[k];
    return 0.5 * s;
}

/* Mirror walls at x = 0 and x = Lx: an atom past a wall is reflected back,
 * and the x components of its velocity and of the force it carries into the
 * next velocity update (F_old) change sign. */
static void mirror_walls(int64_t n, double *pos, double *vel, double *f_old, const double *box)
{
    for (int64_t i = 0; i < n; ++i) {
        double x = pos[3 * i];
        if (x < 0.0 || x >= box[0]) {
            pos[3 * i] = x < 0.0 ? -x : 2.0 * box[0] - x;
            if (ORACLE_MUTANT != 9) {
                vel[3 * i] = -vel[3 * i];
                f_old[3 * i] = -f_old[3 * i];
            }
        }
    }
}

static void wrap_positions(int64_t n, double *pos, const double *box, int walls_x)
{
    for (int64_t i = 0; i < n; ++i)
        for (int d = walls_x ? 1 : 0; d < 3; ++d) {
            double x = pos[3 * i + d];
            if (x >= box[d] || x < 0.0) x -= box[d] * floor(x / box[d]);
            if (x >= box[d]) x -= box[d]; /* rounding guard: keep x in [0, L) */
            pos[3 * i + d] = x;
        }
}

/* Velocity-Verlet NVE run (Algorithm 1) of `steps` iterations.
 *   pos, vel: in/out, 3n; on return the synchronised state (r_n, v_n).
 *   F:        out, 3n, the force at r_n.
 *   obs:      out, 3 * (steps + 1) doubles (may be NULL): (U, W, KE) at
 *             steps 0..n, each taken where r, v and F are synchronised.
 * Positions are wrapped into the box after every update, the periodic
 * counterpart of storing each molecule in the slice it moved to (Sec. 4.1);
 * with walls_x the x coordinate is mirrored at the walls instead.  The
 * initial positions must then lie in [0, Lx).
 */
/* Slice of an atom at x: the cell layer floor(x / l) of nc_x layers of
 * width l = Lx / nc_x (computed as x * (1 / l)), clamped into the box, and the
 * slice holding that layer among slices of cps layers each. */
static int slice_of(double x, double Lx, int nc_x, int cps)
{
    double inv = 1.0 / (Lx / nc_x);
    int c = (int)(x * inv);
    if (c < 0) c = 0;
    if (c >= nc_x) c = nc_x - 1;
    return c / cps;
}

/* The slice thermostat (md_thermo_a/b, md_v3b, Sec. 4.1), read as velocity
 * scaling per slice with the factor taken from the previous step: the
 * synchronised velocities of the atoms of slice j at step s are multiplied by
 * lambda_j(s) = sqrt(T0 / T'_j(s-1)), where T'_j(s-1) = 2 lambda_j(s-1)^2
 * KE_j(s-1) / (3 N_j(s-1)) is the temperature slice j reached after the
 * previous step's scaling (KE_j, N_j measured before it).  lambda = 1 at the
 * first step and after an empty slice.  lam: in, lambda_j(s-1); out,
 * lambda_j(s). */
static void slice_thermostat(int64_t n, const double *pos, double *vel, const double *box, int nc_x, int cps,
                             double T0, const double *prev /* [n_slices][2]: KE, N */, double *lam)
{
    int ns = nc_x / cps;
    for (int j = 0; j < ns; ++j) {
        double ke = prev[2 * j], cnt = prev[2 * j + 1];
        double ke_after = (ORACLE_MUTANT == 11 ? 1.0 : lam[j] * lam[j]) * ke;
        const double ratio = T0 * 3.0 * cnt / (2.0 * ke_after);
        lam[j] = (cnt > 0.0 && ke_after > 0.0) ? (ORACLE_MUTANT == 13 ? ratio : sqrt(ratio)) : 1.0;
    }
    for (int64_t i = 0; i < n; ++i) {
        int j = slice_of(pos[3 * i], box[0], nc_x, cps);
        for (int d = 0; d < 3; ++d) vel[3 * i + d] *= lam[j];
    }
}

/* Kinetic energy and atom count of every slice (out: [n_slices][2]). */
static void slice_stats(int64_t n, const double *pos, const double *vel, const double *box, int nc_x, int cps,
                        double *out)
{
    int ns = nc_x / cps;
    for (int j = 0; j < 2 * ns; ++j) out[j] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        int j = slice_of(pos[3 * i], box[0], nc_x, cps);
        double v2 = 0.0;
        for (int d = 0; d < 3; ++d) v2 += vel[3 * i + d] * vel[3 * i + d];
        out[2 * j] += 0.5 * v2;
        out[2 * j + 1] += 1.0;
    }
}

/* Spatially resolved statistics (Sec. 4.2): per slice j, the sum over its
 * atoms of half their pair energies (U_j), of half their pair virials (W_j),
 * of their kinetic energies (KE_j), and the atom count N_j; slices as in
 * slice_of().  out: [n_slices][4] = (U_j, W_j, KE_j, N_j). */
int oracle_profiles(int64_t n, const double *pos, const double *vel, const double *box, double rc, int walls_x,
                    int nc_x, int cps, double *out)
{
    if (n < 0 || !pos || !box || !out || !(rc > 0.0) || nc_x < 1 || cps < 1 || nc_x % cps != 0)
        return ORACLE_ERR_ARG;
    int ns = nc_x / cps;
    for (int j = 0; j < 4 * ns; ++j) out[j] = 0.0;
    cell_list cl;
    int rcode = build_cells(n, pos, box, rc, &cl);
    if (rcode) return rcode;
    double rc2 = rc * rc, ushift = lj_shift(rc);
    for (int64_t i = 0; i < n; ++i) {
        double f3[3], uh, wh;
        atom_from_cells(i, pos, box, rc2, ushift, walls_x, &cl, f3, &uh, &wh);
        int j = slice_of(pos[3 * i], box[0], nc_x, cps);
        double v2 = 0.0;
        if (vel)
            for (int d = 0; d < 3; ++d) v2 += vel[3 * i + d] * vel[3 * i + d];
        out[4 * j + 0] += (ORACLE_MUTANT == 12 ? 2.0 : 1.0) * uh;
        out[4 * j + 1] += wh;
        out[4 * j + 2] += 0.5 * v2;
        out[4 * j + 3] += 1.0;
    }
    free_cells(&cl);
    return ORACLE_OK;
}

/* Velocity-Verlet run with the optional slice thermostat (NVT when T0 > 0)
 * and mirror walls.  nc_x / cps define the slices (nc_x cell layers along x,
 * cps layers per slice); stats (may be NULL) receives, for steps 0..n,
 * [s][j][2] = (KE_j, N_j) of every slice before that step's scaling. */
int oracle_run_ex(int64_t n, double *pos, double *vel, const double *box, double rc, double dt,
                  int64_t steps, int use_cells, int walls_x, int nc_x, int cps, double T0, double *F,
                  double *obs, double *stats)
{
    if (n < 0 || steps < 0 || !pos || !vel || !box || !F || !(rc > 0.0)) return ORACLE_ERR_ARG;
    if (T0 < 0.0 || ((T0 > 0.0 || stats) && (nc_x < 1 || cps < 1 || nc_x % cps != 0))) return ORACLE_ERR_ARG;
    const int ns = (T0 > 0.0 || stats) ? nc_x / cps : 0;
    double *f_old = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *st = (double *)calloc((size_t)(2 * ns + 2) * 2 + (size_t)ns + 1, sizeof(double)); /* this and the previous step, lambda */
    if (!f_old || !st) {
        free(f_old);
        free(st);
        return ORACLE_ERR_OOM;
    }
    if (walls_x)
        for (int64_t i = 0; i < n; ++i)
            if (!(pos[3 * i] >= 0.0 && pos[3 * i] < box[0])) {
                free(f_old);
                free(st);
                return ORACLE_ERR_ARG;
            }
    wrap_positions(n, pos, box, walls_x);
    double U, W;
    int rcode = forces_any(use_cells, n, pos, box, rc, walls_x, F, &U, &W); /* F(r_0) */
    if (rcode) {
        free(f_old);
        free(st);
        return rcode;
    }
    double *cur = st, *prev = st + (2 * ns + 2), *lam = st + 2 * (2 * ns + 2);
    for (int j = 0; j < ns; ++j) lam[j] = 1.0;
    /* F_old := -F(r_0): the first velocity update leaves v_0 unchanged. */
    for (int64_t k = 0; k < 3 * n; ++k) f_old[k] = -F[k];
    for (int64_t s = 0; s <= steps; ++s) {
        if (s > 0) {
            for (int64_t k = 0; k < 3 * n; ++k) f_old[k] = F[k]; /* F_old = F_new */
            rcode = forces_any(use_cells, n, pos, box, rc, walls_x, F, &U, &W); /* F_new = F(r_s) */
            if (rcode) break;
        }
        /* second loop of Algorithm 1: v += (F_new + F_old) dt / 2 -> v_s */
        for (int64_t k = 0; k < 3 * n; ++k)
            vel[k] = vel[k] + (F[k] + (ORACLE_MUTANT == 5 ? 0.0 : f_old[k])) * 0.5 * dt;
        if (obs) {
            obs[3 * s + 0] = U;
            obs[3 * s + 1] = W;
            obs[3 * s + 2] = kinetic(n, vel);
        }
        if (ns > 0) {
            slice_stats(n, pos, vel, box, nc_x, cps, cur);
            if (stats)
                for (int j = 0; j < 2 * ns; ++j) stats[(size_t)s * 2 * ns + j] = cur[j];
        }
        if (s == steps) break; /* closing half kick done: state is (r_n, v_n, F_n) */
        /* md_v3b: the thermostat scales the synchronised velocities, with the
         * factors measured at the previous step (none at the first) */
        if (T0 > 0.0 && s > 0) slice_thermostat(n, pos, vel, box, nc_x, cps, T0, prev, lam);
        double *t = prev;
        prev = cur;
        cur = t;
        /* third loop of Algorithm 1: r += v dt + F_new dt^2 / 2 */
        for (int64_t k = 0; k < 3 * n; ++k)
            pos[k] = pos[k] + vel[k] * dt + (ORACLE_MUTANT == 6 ? 0.0 : F[k] * 0.5 * dt * dt);
        if (walls_x) {
            /* the force of this step becomes F_old of the next one: carry it
             * (F_new) through the mirror together with the velocity */
            mirror_walls(n, pos, vel, F, box);
        }
        wrap_positions(n, pos, box, walls_x);
    }
    free(f_old);
    free(st);
    return rcode;
}

int oracle_run_w(int64_t n, double *pos, double *vel, const double *box, double rc, double dt, int64_t steps,
                 int use_cells, int walls_x, double *F, double *obs)
{
    return oracle_run_ex(n, pos, vel, box, rc, dt, steps, use_cells, walls_x, 0, 0, 0.0, F, obs, NULL);
}

int oracle_run(int64_t n, double *pos, double *vel, const double *box, double rc, double dt, int64_t steps,
               int use_cells, double *F, double *obs)
{
    return oracle_run_w(n, pos, vel, box, rc, dt, steps, use_cells, 0, F, obs);
}
