"""Parity of the CUDA light curves (rs_light_curves) with the FP64 oracle (oracle.light_curve).

Both sides read the same float32 map (the oracle promotes it to float64).  The pixel set a sample
covers must be that of the float64 definition, so disc-profile curves agree to rounding of the
sums; Gaussian weights are float32 on the device.  The tolerance is derived per sample: a relative
weight error delta_p changes the weighted mean by at most sum_p w_p delta_p |mu_p - mu| / sum_p w_p
(first order).  The device's exponent E_p carries at most u (5 E + 4 sqrt(a E)) (offsets in pixel
units known to u (1 + |offset|), a = pix^2 / (2 s^2); the float64 sample position adds ~2^-53 of
its pixel index, negligible for these maps), the scaling by log2(e) one more rounding of E, the
hardware base-2 exponential at most 2^-21 relative: delta_p = u (8 E + 8 sqrt(a E) + 16) covers
these with room.  Where the device takes the weight as the product of the column and row factors
2^-ex 2^-ey (separable Gaussian, chord interiors), each factor's exponent carries the same kinds of
rounding over a smaller magnitude and the two exponentials stay within 2^-20 = 16 u together; the
product's own rounding enters the row sum (one more term in its budget).  Both sums are positive; each row of the support (at most n_r = 2 R / pix + 3
pixels) is summed in float32 with fused multiply-adds, relative error <= (n_r + 1) u, and the rows
are folded into compensated pairs whose float-float quotient adds ~2u: (2 n_r + 10) u |mu| covers
the sums.  The tests allow twice the resulting first-order bound.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import rs_inputs as ri
from gpu_helpers import dev, rs

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
G, D = oracle.PROFILE_GAUSSIAN, oracle.PROFILE_DISC


def _gpu(maps, windows, tracks, profile, s):
    m = rs()
    tmaps = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev()) for a in maps]
    mtr = [m.Track(t.map, t.y0, t.step, t.n) for t in tracks]
    mu, dm = m.light_curves(tmaps, windows, mtr, profile, s)
    torch.cuda.synchronize()
    return mu.cpu().numpy(), dm.cpu().numpy()


def _oracle(maps, windows, tracks, profile, s):
    mus, dms = [], []
    for t in tracks:
        w = windows[t.map]
        a, b = oracle.light_curve(maps[t.map].astype(np.float64), w.lo, w.hi, profile, s, t.y0, t.step, t.n)
        mus.append(a)
        dms.append(b)
    return (np.concatenate(mus), np.concatenate(dms)) if mus else (np.zeros(0), np.zeros(0))


def _bound(mu_map, w, profile, s, y, ref):
    """Twice the first-order error bound of the device result at sample y (see module docstring)."""
    mu_map = mu_map.astype(np.float64)
    n1, n0 = mu_map.shape
    pix0 = (w.hi[0] - w.lo[0]) / n0
    pix1 = (w.hi[1] - w.lo[1]) / n1
    cx = w.lo[0] + (np.arange(n0) + 0.5) * pix0
    cy = w.lo[1] + (np.arange(n1) + 0.5) * pix1
    dx = cx[None, :] - y[0]
    dy = cy[:, None] - y[1]
    d2 = dx * dx + dy * dy
    if profile == G:
        inside = d2 <= (6.0 * s) * (6.0 * s)
        E = d2 / (2.0 * s * s)
        a = max(pix0, pix1) ** 2 / (2.0 * s * s)
        wgt = np.where(inside, np.exp(-E), 0.0)
        delta = U * (8.0 * E + 8.0 * np.sqrt(a * E) + 16.0)
    else:
        inside = d2 <= s * s
        wgt = inside.astype(np.float64)
        delta = np.zeros_like(d2)
    sw = wgt.sum()
    if sw == 0:
        return 0.0
    first = (wgt * delta * np.abs(mu_map - ref)).sum() / sw
    n_r = min(2.0 * (6.0 * s if profile == G else s) / pix0 + 3.0, n0)   # longest row of the support
    return 2.0 * (first + (2.0 * n_r + 10.0) * U * abs(ref))


def _compare(maps, windows, tracks, profile, s, label):
    got, got_dm = _gpu(maps, windows, tracks, profile, s)
    want, want_dm = _oracle(maps, windows, tracks, profile, s)
    assert got.shape == want.shape
    nan_g, nan_w = np.isnan(got), np.isnan(want)
    assert np.array_equal(nan_g, nan_w), f"{label}: NaN pattern differs"
    k = 0
    worst = 0.0
    for t in tracks:
        for j in range(t.n):
            if not nan_w[k]:
                y = (t.y0[0] + j * t.step[0], t.y0[1] + j * t.step[1])
                b = _bound(maps[t.map], windows[t.map], profile, s, y, want[k])
                err = abs(got[k] - want[k])
                assert err <= b, f"{label}: sample {k}: |{got[k]} - {want[k]}| = {err:.3e} > bound {b:.3e}"
                worst = max(worst, err / b if b > 0 else 0.0)
            k += 1
    ok = ~nan_w & np.isfinite(want_dm)
    assert np.all(np.abs(got_dm[ok] - want_dm[ok]) <= 1e-5), label
    return worst


def _window(npix, lo=(-2.0, -1.0), hi=(2.0, 1.8)):
    return ri.Window(lo=lo, hi=hi, npix=npix)


@pytest.mark.parametrize("profile,s_pix", [(G, 0.3), (G, 2.0), (G, 9.0), (D, 0.4), (D, 3.0), (D, 12.5)])
def test_caustic_map_parity(profile, s_pix):
    """Random tracks (some starting outside the map) over a non-square-pixel caustic map."""
    w = _window((200, 150))                          # pixels 0.02 x 0.018667
    mu = ri.caustic_map(w.npix, seed=11)
    tracks = ri.random_tracks([w], n_per_map=10, n_samples=40, step_pix=0.7, seed=5, margin_pix=-12.0)
    s = s_pix * (w.hi[0] - w.lo[0]) / w.npix[0]
    _compare([mu], [w], tracks, profile, s, f"profile {profile} s {s_pix} px")


def test_far_samples_are_nan_and_edges():
    """Samples whose profile misses the map give NaN on both sides; tracks along and across the edges."""
    w = _window((64, 48))
    mu = ri.caustic_map(w.npix, seed=3)
    pix = (w.hi[0] - w.lo[0]) / 64
    s = 1.5 * pix
    tracks = [
        ri.Track(0, (w.lo[0] - 40 * pix, 0.1), (2 * pix, 0.0), 60),           # enters from the left
        ri.Track(0, (w.hi[0] + 100 * pix, 0.3), (0.0, 0.0), 3),              # far outside: NaN
        ri.Track(0, (w.lo[0], w.lo[1]), (0.5 * pix, 0.5 * pix), 50),        # from the corner
        ri.Track(0, (0.0, w.hi[1] + 8 * pix), (pix, -0.1 * pix), 40),        # just above the top edge
    ]
    for profile in (G, D):
        _compare([mu], [w], tracks, profile, s if profile == G else 4 * s, f"edges {profile}")
    got, _ = _gpu([mu], [w], tracks[1:2], G, s)
    assert np.all(np.isnan(got))


def test_batched_maps_and_output_order():
    """Several maps of different sizes and windows in one call, tracks interleaved, empty tracks between."""
    wins = [_window((96, 80)), ri.Window(lo=(10.0, -3.0), hi=(11.5, -1.0), npix=(128, 160)),
            ri.Window(lo=(-0.5, -0.5), hi=(0.5, 0.5), npix=(33, 47))]
    maps = [ri.caustic_map(w.npix, seed=20 + k) for k, w in enumerate(wins)]
    tr = ri.random_tracks(wins, n_per_map=4, n_samples=25, step_pix=1.3, seed=9, margin_pix=2.0)
    order = [tr[0], ri.Track(1, (10.5, -2.0), (0.0, 0.0), 0), tr[5], tr[9], tr[1],
             ri.Track(2, (0.0, 0.0), (0.01, 0.0), 0), tr[11], tr[6], tr[2], tr[10], tr[3], tr[4], tr[7], tr[8]]
    s = 0.03
    _compare(maps, wins, order, G, s, "batched gaussian")
    _compare(maps, wins, order, D, s, "batched disc")


@pytest.mark.parametrize("r,count", [(1, 5), (2, 13), (5, 81)])
def test_disc_exact_on_lattice_ties(r, count):
    """Disc radius equal to lattice distances (d^2 == s^2 exactly for the rim pixels): the device must
    take the float64 decision, giving exactly the Gauss-circle count N(r) (mean exactly 2)."""
    w = ri.Window(lo=(0.0, 0.0), hi=(8.0, 8.0), npix=(32, 32))              # dyadic pixel 0.25
    mu = np.ones((32, 32), np.float32)
    mu[16, 16] = 1.0 + count
    y = 16.5 * 0.25
    got, _ = _gpu([mu], [w], [ri.Track(0, (y, y), (0.0, 0.0), 1)], D, r * 0.25)
    assert got[0] == 2.0


def test_gaussian_cut_on_lattice_ties():
    """Gaussian cut 6 s exactly on lattice distances (3 pixels): membership at the rim as in float64."""
    w = ri.Window(lo=(0.0, 0.0), hi=(8.0, 8.0), npix=(32, 32))
    mu = ri.caustic_map((32, 32), seed=4)
    y = 16.5 * 0.25
    tracks = [ri.Track(0, (y, y), (0.25, 0.0), 4), ri.Track(0, (y, y), (0.25, 0.25), 4)]
    _compare([mu], [w], tracks, G, 0.125, "gaussian lattice ties")


def test_oracle_shot_map():
    """Light curves of a magnification map that the oracle itself shot (tiny field, Eq. 4)."""
    spec = ri.tiny_field()
    counts, _ = oracle.shoot_field(spec)
    mu = oracle.magnification(counts, spec.grid.spacing, spec.window.lo, spec.window.hi,
                              spec.window.npix).astype(np.float32)
    w = spec.window
    tracks = ri.random_tracks([w], n_per_map=6, n_samples=50, step_pix=0.9, seed=2, margin_pix=4.0)
    pix = (w.hi[0] - w.lo[0]) / w.npix[0]
    _compare([mu], [w], tracks, G, 1.7 * pix, "oracle map gaussian")
    _compare([mu], [w], tracks, D, 2.2 * pix, "oracle map disc")


def test_bench_scale_sampled():
    """The light-curve bench workload (64 maps of 512^2..1024^2 pixels, 16 tracks of 2048 samples per
    map, Gaussian source of 2 pixels), in the bench's single launch; 48 sampled outputs are checked
    one by one against the oracle."""
    maps, wins, tracks, s = ri.light_curve_workload()
    got, _ = _gpu(maps, wins, tracks, G, s)
    assert got.shape[0] == sum(t.n for t in tracks)
    rng = np.random.default_rng(77)
    offs = np.cumsum([0] + [t.n for t in tracks])
    for g in rng.integers(0, got.shape[0], size=48):
        ti = int(np.searchsorted(offs, g, side="right") - 1)
        t = tracks[ti]
        k = int(g - offs[ti])
        y = (t.y0[0] + k * t.step[0], t.y0[1] + k * t.step[1])
        w = wins[t.map]
        want, _ = oracle.light_curve(maps[t.map].astype(np.float64), w.lo, w.hi, G, s, y, (0.0, 0.0), 1)
        if np.isnan(want[0]):
            assert np.isnan(got[g])
            continue
        b = _bound(maps[t.map], w, G, s, y, want[0])
        assert abs(got[g] - want[0]) <= b, (g, got[g], want[0], b)


def _bits_equal(a, b):
    """Bitwise equality of float64 tensors (NaN samples included)."""
    return torch.equal(a.contiguous().view(torch.int64), b.contiguous().view(torch.int64))


def test_plan_matches_one_shot_and_replays_in_a_graph():
    """A plan launched directly, replayed from a captured CUDA graph, and after its map was rewritten in
    place gives bitwise the one-shot results for the current map contents."""
    m = rs()
    wins = [_window((96, 80)), _window((64, 64))]
    maps = [torch.from_numpy(ri.caustic_map(w.npix, seed=40 + k)).to(dev()) for k, w in enumerate(wins)]
    tr = ri.random_tracks(wins, n_per_map=3, n_samples=30, step_pix=0.8, seed=3, margin_pix=1.0)
    mtr = [m.Track(t.map, t.y0, t.step, t.n) for t in tr]
    s = 0.05
    plan = m.LightCurvePlan(maps, wins, mtr, m.RS_PROFILE_GAUSSIAN, s)
    try:
        ref_mu, ref_dm = m.light_curves(maps, wins, mtr, m.RS_PROFILE_GAUSSIAN, s)
        plan.launch()
        torch.cuda.synchronize()
        assert _bits_equal(plan.mu, ref_mu) and _bits_equal(plan.dm, ref_dm)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            plan.launch(side)                       # warm-up on the capture stream
            side.synchronize()
            with torch.cuda.graph(g, stream=side):
                plan.launch(side)
        plan.mu.zero_()
        maps[1].mul_(2.0)                           # the plan reads the buffers at every launch
        g.replay()
        torch.cuda.synchronize()
        ref2, _ = m.light_curves(maps, wins, mtr, m.RS_PROFILE_GAUSSIAN, s)
        assert _bits_equal(plan.mu, ref2)
        n0 = 3 * 30
        assert _bits_equal(plan.mu[:n0], ref_mu[:n0]) and _bits_equal(plan.mu[n0:], 2 * ref_mu[n0:])
    finally:
        plan.close()


@pytest.mark.parametrize("profile,radius", [(D, 100.0), (G, 100.0 / 6.0)])
def test_large_support_rim_crosses_map(profile, radius):
    """A support of ~5000 pixels radius whose rim crosses the map: hundreds of rim pixels fall inside
    the guard band and take the float64 decision; the interior of each chord is summed untested."""
    w = _window((200, 150))
    mu = ri.caustic_map(w.npix, seed=11)
    tracks = [ri.Track(0, (-100.0 + 0.3, 0.2), (0.0123, 0.0071), 6),
              ri.Track(0, (0.1, 1.0 + 100.0 - 0.4), (0.0031, -0.009), 6)]
    _compare([mu], [w], tracks, profile, radius, f"large support {profile}")
