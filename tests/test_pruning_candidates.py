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
