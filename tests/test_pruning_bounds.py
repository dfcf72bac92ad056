"""The rounding arguments behind the two neighbour-pruning shortcuts, checked
on random configurations in NumPy float32 (no GPU).  Unfused float32
operations round more often than the kernels' fused ones, so passing here is
the stricter case.

1. Mixed form: an entry is dropped when its squared distance to the home
   atoms' bounding box, widened by 1e-4 per side, exceeds rc^2 + 1e-3.  Such
   an entry must fail the FP32 pair cutoff test against every home atom.
2. FP64 form: a candidate is settled in FP32 (coordinates relative to the
   unit's corner, extent E) unless its FP32 r^2 lies in the band
   [rc^2 - b, rc^2 + b] or at or below b, with b = 4 (6 rc E + 3 rc^2) 2^-24.
   Every such decision must agree with the FP64 test 0 < r^2 <= rc^2.
"""
import numpy as np
import pytest

RC = 2.5
RC2 = RC * RC
F32 = np.float32


def f32_r2(d):
    d = d.astype(F32)
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


@pytest.mark.parametrize("n_home,seed", [(1, 1), (2, 2), (13, 3), (40, 4)])
def test_mixed_form_dropped_entries_are_out_of_range(n_home, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    lc = 2.545
    for _ in range(40):
        home = rng.uniform(-lc / 2, lc / 2, (n_home, 3)).astype(F32)
        # candidates concentrated near the edge of the box's rc-neighbourhood
        cand = rng.uniform(-1.5 * lc, 1.5 * lc, (4000, 3)).astype(F32)
        lo = home.min(0) - F32(1e-4)
        hi = home.max(0) + F32(1e-4)
        d = np.maximum(np.maximum(lo - cand, cand - hi), F32(0))
        dist2 = f32_r2(d)
        dropped = dist2 > F32(RC2) + F32(1e-3)
        assert dropped.any() and (~dropped).any()
        r2 = f32_r2(home[None, :, :] - cand[dropped][:, None, :])
        assert np.all(r2 > F32(RC2)), "a dropped entry is within the cutoff of a home atom"


def band(E):
    return 4.0 * (6.0 * np.sqrt(RC2) * E + 3.0 * RC2) * 2.0 ** -24


def fp32_r2_error_bound(E):
    """First-order bound on |FP32 r^2 - FP64 r^2| near the cutoff: coordinate
    roundings (E 2^-24 each) and the subtraction's (rc 2^-24) per component,
    squared and summed (sum |d_k| <= sqrt(3) rc), plus three roundings of
    r^2 (3 rc^2 2^-24)."""
    rc = np.sqrt(RC2)
    return (2.0 * np.sqrt(3.0) * rc * (2.0 * E + rc) + 3.0 * RC2) * 2.0 ** -24


@pytest.mark.parametrize("E", [0.0, 1.0, 7.5, 15.0, 40.0, 1000.0])
def test_fp64_form_band_covers_the_error_bound(E):
    assert band(E) >= 1.8 * fp32_r2_error_bound(E)
    if E >= 7.5:                        # a unit spans three cells of edge >= rc
        assert band(E) >= 3.0 * fp32_r2_error_bound(E)


@pytest.mark.parametrize("E,seed", [(15.0, 5), (40.0, 6), (1000.0, 7)])
def test_fp64_form_fp32_decisions_agree_with_fp64(E, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    b = band(E)
    lo_in, hi_out, tiny = F32(RC2 - b), F32(RC2 + b), F32(b)
    n = 400_000
    corner = rng.uniform(-2000.0, 2000.0, 3)                    # the unit's corner, FP64
    xi = corner + rng.uniform(0.0, E, (n, 3))
    # partners at distances spread tightly around the cutoff, some exactly on it
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    r = RC * (1.0 + rng.normal(0.0, 2e-5, n))
    r[::97] = RC
    xj = xi + u * r[:, None]
    r2 = ((xi - xj) ** 2).sum(1)                                # the FP64 decision
    in64 = (r2 <= RC2) & (r2 > 0.0)
    r2f = f32_r2((xi - corner).astype(F32) - (xj - corner).astype(F32))
    # the stated bound holds on every sample (and the band is wider still)
    assert np.abs(r2f.astype(np.float64) - r2).max() <= fp32_r2_error_bound(E)
    sure_out = r2f > hi_out
    sure_in = (r2f < lo_in) & (r2f > tiny)
    assert not np.any(sure_out & in64)
    assert not np.any(sure_in & ~in64)
    # the band is narrow: almost every candidate is settled in FP32 at the
    # extents units have (E of a few cells)
    settled = (sure_out | sure_in).mean()
    if E <= 40.0:
        assert settled > 0.5
    # and the same point is never settled "in" against itself
    same = f32_r2(((xi - corner).astype(F32) - (xi - corner).astype(F32))[:10])
    assert np.all(same <= tiny)
