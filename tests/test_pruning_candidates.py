"""Candidates per atom of the neighbour-pruning schemes at rho = 0.8, counted
on a disordered fcc-derived configuration with the mixed form's cell geometry
(cells of edge 2.57, 13.5 atoms each; the 1M box has 2.55 and 13.2).

The mixed form prunes each home cell's 27-cell neighbourhood to the entries
within rc of the bounding box of the home cell's atoms.  Cluster pairs (the
home cell's atoms split into spatial clusters of k, each pruned against the
neighbour clusters' bounding boxes) keep more candidates than that for
k = 4 and 8: at this density a cluster of 4 atoms is about 1.7 sigma wide,
so the box-to-box test reaches far past the home atoms.  Only k = 2 keeps
fewer, at the price of a pruned list per pair of home atoms.  These counts
are the design's reason for pruning per home cell."""
import numpy as np
import pytest

from paper_2507_11289_gb300 import inputs

RC = 2.5


def _setup():
    pos, box = inputs.fcc_lattice(15, 0.8)
    pos = inputs.jitter(pos, box, 0.35, 3)
    L = box[0]
    nc = int(L // RC)
    lc = L / nc
    cell = np.floor(pos / lc).astype(int) % nc
    cid = (cell[:, 0] * nc + cell[:, 1]) * nc + cell[:, 2]
    cells = {}
    for i in np.argsort(cid, kind="stable"):
        cells.setdefault(int(cid[i]), []).append(int(i))
    return pos, L, nc, lc, cells


def _neighbours(c, nc):
    x, y, z = c // (nc * nc), (c // nc) % nc, c % nc
    return [(((x + a) % nc) * nc + (y + b) % nc) * nc + (z + d) % nc
            for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1)]


def _clusters(p, k, lc):
    """Chunks of k atoms after sorting by half-cell octant, then x, y, z."""
    oc = np.floor((p - p.min(0)) / (lc / 2 + 1e-9)).clip(0, 1).astype(int)
    code = oc[:, 0] * 4 + oc[:, 1] * 2 + oc[:, 2]
    p = p[np.lexsort((p[:, 2], p[:, 1], p[:, 0], code))]
    return [(p[i:i + k].min(0), p[i:i + k].max(0), len(p[i:i + k])) for i in range(0, len(p), k)]


def test_cell_box_pruning_beats_cluster_pairs_of_four_and_eight():
    pos, L, nc, lc, cells = _setup()
    rng = np.random.default_rng(0)
    sample = rng.choice(sorted(cells), 150, replace=False)

    def rel(ids, ref):
        d = pos[ids] - ref
        return d - L * np.round(d / L)

    exact, cellbox, clus = [], [], {2: [], 4: [], 8: []}
    for c in sample:
        home = np.array(cells[c])
        ref = pos[home[0]]
        nb = np.concatenate([np.array(cells[k]) for k in _neighbours(c, nc)])
        h, n = rel(home, ref), rel(nb, ref)
        d2 = ((h[:, None, :] - n[None, :, :]) ** 2).sum(-1)
        exact.append(((d2 <= RC * RC) & (d2 > 0)).sum(1).mean())
        lo, hi = h.min(0), h.max(0)
        dd = np.maximum(np.maximum(lo - n, n - hi), 0.0)
        cellbox.append(((dd * dd).sum(1) <= RC * RC).sum())
        for k in clus:
            hcl = _clusters(h, k, lc)
            ncl = [cl for kk in _neighbours(c, nc) for cl in _clusters(rel(np.array(cells[kk]), ref), k, lc)]
            nlo = np.array([a for a, _, _ in ncl])
            nhi = np.array([b for _, b, _ in ncl])
            nn = np.array([m for _, _, m in ncl])
            tot = 0
            for lo1, hi1, m1 in hcl:
                g = np.maximum(np.maximum(lo1 - nhi, nlo - hi1), 0.0)
                tot += m1 * nn[(g * g).sum(1) <= RC * RC].sum()
            clus[k].append(tot / len(home))
    e, cb = np.mean(exact), np.mean(cellbox)
    c2, c4, c8 = (np.mean(clus[k]) for k in (2, 4, 8))
    print(f"candidates per atom: in range {e:.1f}; home-cell box {cb:.0f}; "
          f"cluster pairs of 2 / 4 / 8: {c2:.0f} / {c4:.0f} / {c8:.0f}")
    assert e == pytest.approx(4 * np.pi / 3 * RC ** 3 * 0.8, rel=0.05)
    assert c4 > cb and c8 > c4
    assert c2 < cb


def test_home_clusters_against_neighbour_atoms_cost_list_room():
    """The finer scheme, each cluster of k home atoms pruning the neighbour
    atoms against its own box, does cut the candidates below the cell box
    (about 133 per atom for k = 4, 177 for k = 8, against 228), but each home
    cell then keeps one list per cluster: about 480 entries for k = 4, more
    than the 400-entry list window of a warp, and every raw neighbour entry is
    tested against each of the cell's clusters instead of once."""
    pos, L, nc, lc, cells = _setup()
    rng = np.random.default_rng(0)
    sample = rng.choice(sorted(cells), 150, replace=False)

    def rel(ids, ref):
        d = pos[ids] - ref
        return d - L * np.round(d / L)

    cand = {16: [], 8: [], 4: []}
    kept = {16: [], 8: [], 4: []}
    n_clusters = {16: [], 8: [], 4: []}
    for c in sample:
        home = np.array(cells[c])
        ref = pos[home[0]]
        n = rel(np.concatenate([np.array(cells[k]) for k in _neighbours(c, nc)]), ref)
        h = rel(home, ref)
        for k in cand:
            tot = st = 0
            hcl = _clusters(h, k, lc)
            for lo, hi, m in hcl:
                dd = np.maximum(np.maximum(lo - n, n - hi), 0.0)
                keep = int(((dd * dd).sum(1) <= RC * RC).sum())
                tot += m * keep
                st += keep
            cand[k].append(tot / len(home))
            kept[k].append(st)
            n_clusters[k].append(len(hcl))
    c16, c8, c4 = (np.mean(cand[k]) for k in (16, 8, 4))
    s16, s8, s4 = (np.mean(kept[k]) for k in (16, 8, 4))
    print(f"home clusters x neighbour atoms, candidates per atom k=16/8/4: {c16:.0f} / {c8:.0f} / {c4:.0f}; "
          f"list entries per home cell {s16:.0f} / {s8:.0f} / {s4:.0f}; "
          f"box tests per raw entry {np.mean(n_clusters[16]):.1f} / {np.mean(n_clusters[8]):.1f} / "
          f"{np.mean(n_clusters[4]):.1f}")
    assert c4 < c8 < c16 and c4 < 0.65 * c16          # fewer candidates...
    assert s4 > 400 and s4 > 1.8 * s16                 # ...for lists beyond a warp's window
    assert np.mean(n_clusters[4]) > 3                  # and a box test per cluster per entry
