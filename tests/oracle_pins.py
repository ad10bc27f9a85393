"""Checks that pin the CPU oracle to facts fixed outside of it.

None of these retypes the oracle's formulas.  Each check compares the
oracle with something independent:

* a hand-worked frame (``tests/golden/hand_frame_40x36.json``);
* a brute-force tile-overlap test written as exact comparisons of the
  rounded box edges against every tile's pixel boundary (no floor, no
  clamp, no division);
* Python's arbitrary-precision running sum for the scan;
* Python's ``sorted`` (documented stable) for the sort, plus an O(m^2)
  insertion sort on tiny inputs;
* invariants (permutation, order, stability, partition of the ranges).

The checks take an ``Oracle`` object so the same checks can also be run
against deliberately broken builds of the oracle (see
``test_oracle_mutants.py``) to show that each plausible mistake fails at
least one of them.
"""
from __future__ import annotations

import json
import math
import os
import struct

import numpy as np

from paper_2511_16298_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_frame_40x36.json")


def f32_bits(v: float) -> int:
    return struct.unpack("<I", struct.pack("<f", v))[0]


# ------------------------------------------------------------ brute force
def brute_cover(x, y, r, width, height):
    """Tiles (ty, tx) whose 16x16 pixel square meets the Gaussian's box.

    The box edges are the float32-rounded values s1 = x - r and
    s2 = (x + r) + 15 (same for y).  Column tx is covered iff its right
    pixel boundary 16*tx + 16 lies in (s1, s2].  Every comparison is exact
    (float32 values against small integers)."""
    gx, gy = -(-width // 16), -(-height // 16)
    if r <= 0:
        return []
    rf = np.float32(r)
    xf, yf = np.float32(x), np.float32(y)
    sx1 = float(np.float32(xf - rf))
    sx2 = float(np.float32(np.float32(xf + rf) + np.float32(15.0)))
    sy1 = float(np.float32(yf - rf))
    sy2 = float(np.float32(np.float32(yf + rf) + np.float32(15.0)))
    cols = [tx for tx in range(gx) if 16 * tx + 16 > sx1 and 16 * tx + 16 <= sx2]
    rows = [ty for ty in range(gy) if 16 * ty + 16 > sy1 and 16 * ty + 16 <= sy2]
    return [(ty, tx) for ty in rows for tx in cols]


def brute_frame(g, width, height):
    """Brute-force pairs in emission order: Gaussian, then row, then column."""
    gx = -(-width // 16)
    pairs = []
    counts = []
    for i, rec in enumerate(g):
        cov = brute_cover(float(rec["x"]), float(rec["y"]), int(rec["radius"]), width, height)
        counts.append(len(cov))
        for ty, tx in cov:
            pairs.append(((ty * gx + tx) << 32 | f32_bits(float(rec["depth"])), i))
    return counts, pairs


def tiny_frame(seed: int):
    """Tiny frame with many edge positions: means on and next to tile
    boundaries (+-1 ulp), off-screen means, culled and large radii."""
    rng = np.random.default_rng(seed)
    width = int(rng.integers(1, 65))
    height = int(rng.integers(1, 65))
    n = int(rng.integers(1, 51))
    kind = rng.integers(0, 3, size=(n, 2))
    base = rng.integers(-3, 6, size=(n, 2)) * 16.0 + rng.choice([0.0, 0.5, 15.0, 15.5], size=(n, 2))
    xy = np.where(kind == 0, rng.uniform(-40, 100, size=(n, 2)), base)
    xy = xy.astype(np.float32)
    bump = rng.choice([-1, 0, 1], size=(n, 2))
    xy = np.where(kind == 2, np.nextafter(xy, np.where(bump > 0, np.inf, -np.inf)).astype(np.float32), xy)
    r = rng.choice([0, 1, 2, 3, 7, 8, 9, 15, 16, 17, 31, 40, 100], size=n)
    depth = rng.uniform(0.1, 20.0, size=n)
    g = synth.records(xy[:, 0], xy[:, 1], depth, r)
    return g, width, height


# ----------------------------------------------------------------- checks
def check_golden(O):
    d = json.load(open(GOLDEN))
    gs = d["gaussians"]
    g = synth.records([q["x"] for q in gs], [q["y"] for q in gs], [q["depth"] for q in gs],
                      [q["radius"] for q in gs])
    W, H = d["width"], d["height"]
    st, counts = O.count_tiles(g, W, H)
    assert st == 0 and counts.tolist() == d["counts"], counts
    st, offsets, m = O.scan(counts)
    assert st == 0 and offsets.tolist() == d["offsets"] and m == d["m"]
    st, keys, values = O.duplicate(g, offsets, m, W, H)
    assert st == 0
    exp_keys = [t << 32 | f32_bits(z) for t, z in zip(d["unsorted_tiles"], d["unsorted_depths"])]
    assert keys.tolist() == exp_keys and values.tolist() == d["unsorted_values"]
    st, sk, sv = O.sort_pairs(keys, values)
    exp_sorted = [t << 32 | f32_bits(z) for t, z in zip(d["sorted_tiles"], d["sorted_depths"])]
    assert st == 0 and sk.tolist() == exp_sorted and sv.tolist() == d["sorted_values"]
    st, ranges = O.tile_ranges(sk, len(d["ranges"]))
    assert st == 0 and ranges.tolist() == d["ranges"]
    for k, v in d["float32_bits"].items():
        assert f32_bits(float(k)) == int(v, 16)


def check_count_and_duplicate_bruteforce(O, seeds=range(40)):
    for seed in seeds:
        g, W, H = tiny_frame(seed)
        counts_bf, pairs_bf = brute_frame(g, W, H)
        st, counts = O.count_tiles(g, W, H)
        assert st == 0, (seed, st)
        assert counts.tolist() == counts_bf, (seed, W, H)
        st, offsets, m = O.scan(counts)
        assert st == 0 and m == len(pairs_bf)
        st, keys, values = O.duplicate(g, offsets, m, W, H)
        assert st == 0
        assert list(zip(keys.tolist(), values.tolist())) == pairs_bf, (seed, W, H)


def check_special_cases(O):
    W, H = 256, 128  # 16 x 8 tiles
    T = 128
    cases = [
        # (x, y, r, expected count)
        (8.5, 8.5, 1, 1),          # stays inside one tile
        (-100.0, 50.0, 5, 0),      # fully left of the screen
        (50.0, 500.0, 5, 0),       # fully below the screen
        (128.0, 64.0, 1000, T),    # radius covering the screen
        (0.0, 0.0, 1, 1),          # corner: box [-1,1] -> tile 0 only
        (16.0, 16.0, 1, 4),        # box [15,17] straddles 2x2 tiles
        (255.9, 127.9, 1, 1),      # last tile
        (10.0, 10.0, 0, 0),        # culled
        (10.0, 10.0, -3, 0),       # negative radius: culled
    ]
    g = synth.records([c[0] for c in cases], [c[1] for c in cases], [1.0] * len(cases),
                      [c[2] for c in cases])
    st, counts = O.count_tiles(g, W, H)
    assert st == 0 and counts.tolist() == [c[3] for c in cases], counts
    # one tile image: every visible Gaussian hits tile 0
    g1 = synth.records([3.0, 20.0], [3.0, 3.0], [1.0, 2.0], [2, 1])
    st, c1 = O.count_tiles(g1, 16, 16)
    assert st == 0 and c1.tolist() == [1, 0]
    # n = 0
    st, c0 = O.count_tiles(g[:0], W, H)
    assert st == 0 and len(c0) == 0
    st, r0 = O.tile_ranges(np.zeros(0, np.uint64), 5)
    assert st == 0 and (r0 == 0).all()


def check_validity(O):
    W, H = 64, 64
    bad = [
        (10.0, 10.0, float("nan"), 3),
        (10.0, 10.0, float("inf"), 3),
        (10.0, 10.0, -1.0, 3),
        (10.0, 10.0, 0.0, 3),
        (10.0, 10.0, -0.0, 3),
        (float("nan"), 10.0, 1.0, 3),
        (10.0, float("inf"), 1.0, 3),
    ]
    for x, y, z, r in bad:
        g = synth.records([5.0, x], [5.0, y], [1.0, z], [2, r])
        st, _ = O.count_tiles(g, W, H)
        assert st == 1, (x, y, z)
    ok = [
        (10.0, 10.0, float("nan"), 0),      # culled: not checked
        (-500.0, 10.0, -1.0, 3),             # off-screen: depth not checked
        (10.0, 10.0, 1e-45, 3),              # smallest subnormal is > 0
        (float("nan"), 10.0, 1.0, 0),        # culled NaN mean
    ]
    for x, y, z, r in ok:
        g = synth.records([x], [y], [z], [r])
        st, _ = O.count_tiles(g, W, H)
        assert st == 0, (x, y, z, r)
    st, _ = O.count_tiles(synth.records([1.0], [1.0], [1.0], [1]), 0, 16)
    assert st == 1


def check_scan(O):
    rng = np.random.default_rng(7)
    for n in (0, 1, 2, 31, 1000, 4097):
        c = rng.integers(0, 3000, size=n).astype(np.uint32)
        st, off, total = O.scan(c)
        run = 0
        exp = []
        for v in c.tolist():
            exp.append(run)
            run += v
        assert st == 0 and off.tolist() == exp and total == run
    st, _, total = O.scan(np.array([2**31, 2**31 - 1], dtype=np.uint32))
    assert st == 0 and total == 2**32 - 1
    st, _, total = O.scan(np.array([2**31, 2**31], dtype=np.uint32))
    assert st == 3 and total == 2**32


def check_sort(O):
    rng = np.random.default_rng(11)
    for m, nkeys, wide in ((0, 1, False), (1, 1, False), (2, 1, False), (17, 3, False),
                           (300, 20, False), (5000, 50, True), (20000, 2000, True)):
        if wide:
            pool = rng.integers(0, 2**63, size=nkeys, dtype=np.uint64) * np.uint64(2) \
                + rng.integers(0, 2, size=nkeys, dtype=np.uint64)
        else:
            pool = rng.integers(0, 1 << 40, size=nkeys, dtype=np.uint64)
        keys = pool[rng.integers(0, nkeys, size=m)] if m else np.zeros(0, np.uint64)
        values = rng.permutation(m).astype(np.uint32)
        st, sk, sv = O.sort_pairs(keys, values)
        assert st == 0
        kl, vl = keys.tolist(), values.tolist()
        order = sorted(range(m), key=lambda k: kl[k])  # Python's sort is stable
        assert sk.tolist() == [kl[k] for k in order]
        assert sv.tolist() == [vl[k] for k in order]
        # invariants
        assert sorted(zip(sk.tolist(), sv.tolist())) == sorted(zip(kl, vl))
        assert all(a <= b for a, b in zip(sk.tolist(), sk.tolist()[1:]))
    # O(m^2) insertion sort on a tiny case with ties
    keys = np.array([5, 3, 5, 1, 3, 3, 9, 0, 5], dtype=np.uint64)
    values = np.arange(9, dtype=np.uint32)[::-1].copy()
    pairs = list(zip(keys.tolist(), values.tolist()))
    out = []
    for p in pairs:
        j = len(out)
        while j > 0 and out[j - 1][0] > p[0]:
            j -= 1
        out.insert(j, p)
    st, sk, sv = O.sort_pairs(keys, values)
    assert list(zip(sk.tolist(), sv.tolist())) == out


def check_frame_invariants(O, frames):
    """Full pipeline on frames: permutation of the duplicated pairs, keys
    non-decreasing, equal keys with increasing values (the lemma: equal
    keys come from distinct Gaussians emitted in index order), ranges
    partition [0, m) in tile order and match per-tile brute-force counts."""
    for fr in frames:
        d = O.sort_frame(fr.gaussians, fr.width, fr.height)
        assert d["status"] == 0
        k, v = d["keys"].astype(np.uint64), d["values"].astype(np.int64)
        m = d["m"]
        assert len(k) == m
        assert np.all(k[1:] >= k[:-1])
        tie = k[1:] == k[:-1]
        assert np.all(v[1:][tie] > v[:-1][tie])
        uk, uv = d["unsorted_keys"], d["unsorted_values"]
        a = np.lexsort((uv, uk))
        assert np.array_equal(uk[a], k) and np.array_equal(uv[a].astype(np.int64), v)
        T = fr.num_tiles
        r = d["ranges"].astype(np.int64)
        tiles = (k >> np.uint64(32)).astype(np.int64)
        per_tile = np.bincount(tiles, minlength=T) if m else np.zeros(T, np.int64)
        assert (r[:, 1] - r[:, 0] == per_tile).all()
        assert (r[per_tile == 0] == 0).all()
        nz = np.nonzero(per_tile)[0]
        if len(nz):
            assert r[nz[0], 0] == 0 and r[nz[-1], 1] == m
            assert (r[nz[1:], 0] == r[nz[:-1], 1]).all()
            for t in nz[:: max(1, len(nz) // 50)]:
                assert (tiles[r[t, 0]:r[t, 1]] == t).all()


def check_float_order(samples: int = 10_000_000):
    """For positive finite float32 a, b: a < b iff bits(a) < bits(b).  This
    is the premise that lets the key carry raw depth bits."""
    rng = np.random.default_rng(3)
    u = rng.integers(1, 0x7F800000, size=(samples, 2), dtype=np.uint32)
    f = u.view(np.float32)
    assert np.all(np.isfinite(f)) and np.all(f > 0)
    assert np.array_equal(f[:, 0] < f[:, 1], u[:, 0] < u[:, 1])
    edge = np.array([1e-45, 1.17549435e-38, 1.1754942e-38, 1.0, np.nextafter(np.float32(1), 2),
                     3.4028235e38, np.nextafter(np.float32(3.4028235e38), 0)], dtype=np.float32)
    eb = edge.view(np.uint32)
    for i in range(len(edge)):
        for j in range(len(edge)):
            assert (edge[i] < edge[j]) == (eb[i] < eb[j])


# ------------------------------------------------------------ preprocessing
def _cam(rot=None, trans=(0.0, 0.0, 0.0), fx=1000.0, fy=1000.0, cx=640.0, cy=360.0,
         near=0.2, width=1280, height=720):
    c = np.zeros((), dtype=synth.CAMERA)
    c["rot"] = np.eye(3).reshape(9) if rot is None else np.asarray(rot, dtype=np.float64).reshape(9)
    c["trans"] = trans
    c["fx"], c["fy"], c["cx"], c["cy"], c["near_z"] = fx, fy, cx, cy, near
    c["width"], c["height"] = width, height
    return c


def _g3(points, covs, opacity=0.5):
    """points: (n, 3); covs: (n, 3, 3) symmetric."""
    points = np.asarray(points, dtype=np.float64)
    covs = np.asarray(covs, dtype=np.float64)
    g = np.zeros(len(points), dtype=synth.GAUSSIAN3D)
    g["x"], g["y"], g["z"] = points[:, 0], points[:, 1], points[:, 2]
    g["opacity"] = opacity
    c = np.zeros(len(points), dtype=synth.COV3D)
    for name, (i, j) in (("xx", (0, 0)), ("xy", (0, 1)), ("xz", (0, 2)), ("yy", (1, 1)),
                         ("yz", (1, 2)), ("zz", (2, 2))):
        c[name] = covs[:, i, j]
    return g, c


def _footprint(a, b, c):
    """Closed forms of a symmetric 2x2 [[a, b], [b, c]] in float64: the
    larger eigenvalue with the 0.1 floor on the discriminant, the 3-sigma
    radius (before ceil) and the inverse as (c, -b, a) / det."""
    mid = 0.5 * (a + c)
    det = a * c - b * b
    lam = mid + math.sqrt(max(0.1, mid * mid - det))
    return 3.0 * math.sqrt(lam), np.array([c / det, -b / det, a / det])


def _check_case(O, pt, cov, cam, expect_xy, s2, tag):
    """One Gaussian against closed forms: projected mean, depth, conic
    (relative 2e-6 plus 1e-6 times the determinant's cancellation factor)
    and the radius (exact, cases whose 3-sigma value lies
    within 1e-3 of an integer are not used)."""
    g, c = _g3([pt], [cov])
    st, rec, con = O.preprocess(g, c, cam)
    assert st == 0, tag
    r3, conic = _footprint(*s2)
    assert abs(r3 - round(r3)) > 1e-3, f"{tag}: pick a case away from an integer radius"
    assert rec["radius"][0] == math.ceil(r3), (tag, rec["radius"][0], r3)
    assert np.allclose([rec["x"][0], rec["y"][0]], expect_xy, rtol=1e-6, atol=1e-4), tag
    assert rec["depth"][0] == np.float32(pt[2]), tag
    a, b, c = s2
    kappa = (abs(a * c) + b * b) / (a * c - b * b)  # cancellation in the determinant
    assert np.allclose(con[0, :3], conic, rtol=2e-6 + kappa * 1e-6, atol=1e-9), (tag, con[0], conic)
    assert con[0, 3] == np.float32(0.5), tag


def check_preprocess(O):
    """Projection of single Gaussians whose 2D footprint has a closed form
    (identity camera unless stated; fx = fy = 1000, 1280x720, centre
    (640, 360), near plane 0.2):
    * on the optical axis, isotropic sigma s at depth z: footprint
      (fx s / z)^2 + 0.3 on both axes, no cross term; equal axes put the
      0.1 floor on the discriminant;
    * off axis (X, Y, Z), diagonal covariance: with u = X/Z, v = Y/Z,
      a = fx^2 (sx^2 + u^2 sz^2) / Z^2 + 0.3, b = fx fy u v sz^2 / Z^2,
      c = fy^2 (sy^2 + v^2 sz^2) / Z^2 + 0.3;
    * a slope beyond 1.3 x the half field of view: u is clamped to
      0.65 W / fx in the footprint but not in the projected mean;
    * on the axis with a full covariance: a = (fx/Z)^2 Sxx + 0.3,
      b = fx fy / Z^2 Sxy, c = (fy/Z)^2 Syy + 0.3;
    * invariance: rotating the scene and the camera together changes
      nothing; culling at the near plane, behind the camera, for
      non-finite means and for a negative covariance."""
    fx = fy = 1000.0
    cam = _cam()
    # on axis, isotropic
    for z, s in ((5.0, 0.0075), (2.0, 0.011), (10.0, 0.3), (40.0, 0.21)):
        k = (fx * s / z) ** 2 + 0.3
        _check_case(O, (0.0, 0.0, z), np.eye(3) * s * s, cam, (640.0, 360.0), (k, 0.0, k), f"axis z={z}")
    # off axis, diagonal covariance
    for (X, Y, Z), (sx, sy, sz) in (((0.7, -0.4, 6.0), (0.02, 0.05, 0.09)),
                                     ((-1.1, 0.9, 3.5), (0.004, 0.003, 0.2)),
                                     ((2.0, 1.0, 9.0), (0.1, 0.02, 0.03))):
        u, v = X / Z, Y / Z
        a = fx * fx * (sx * sx + u * u * sz * sz) / (Z * Z) + 0.3
        b = fx * fy * u * v * sz * sz / (Z * Z)
        c = fy * fy * (sy * sy + v * v * sz * sz) / (Z * Z) + 0.3
        _check_case(O, (X, Y, Z), np.diag([sx * sx, sy * sy, sz * sz]), cam,
                    (fx * u + 640.0, fy * v + 360.0), (a, b, c), f"off axis {X},{Y},{Z}")
    # slope clamped (u = 1.4 > 0.65 * 1280 / 1000 = 0.832)
    X, Z, sx, sy, sz = 7.0, 5.0, 0.01, 0.02, 0.05
    lim = 0.65 * 1280 / fx
    a = fx * fx * (sx * sx + lim * lim * sz * sz) / (Z * Z) + 0.3
    c = fy * fy * (sy * sy) / (Z * Z) + 0.3
    _check_case(O, (X, 0.0, Z), np.diag([sx * sx, sy * sy, sz * sz]), cam,
                (fx * X / Z + 640.0, 360.0), (a, 0.0, c), "clamped slope")
    # on axis, full covariance
    S = np.array([[0.0009, 0.0004, -0.0002], [0.0004, 0.0016, 0.0003], [-0.0002, 0.0003, 0.0025]])
    Z = 4.0
    a = (fx / Z) ** 2 * S[0, 0] + 0.3
    b = fx * fy / Z ** 2 * S[0, 1]
    c = (fy / Z) ** 2 * S[1, 1] + 0.3
    _check_case(O, (0.0, 0.0, Z), S, cam, (640.0, 360.0), (a, b, c), "full covariance")

    # invariance under a common rotation of scene and camera
    rng = np.random.default_rng(11)
    pts = np.stack([rng.uniform(-2, 2, 64), rng.uniform(-1, 1, 64), rng.uniform(3, 12, 64)], 1)
    A = rng.normal(size=(64, 3, 3)) * 0.03
    covs = A @ A.transpose(0, 2, 1) + np.eye(3) * 1e-4
    g, cv = _g3(pts, covs)
    st0, rec0, con0 = O.preprocess(g, cv, cam)
    th = 0.7
    Q = np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])
    g2, cv2 = _g3(pts @ Q.T, Q @ covs @ Q.T)
    st1, rec1, con1 = O.preprocess(g2, cv2, _cam(rot=Q.T))
    assert st0 == st1 == 0
    assert np.allclose(rec0["x"], rec1["x"], rtol=1e-5, atol=2e-3)
    assert np.allclose(rec0["y"], rec1["y"], rtol=1e-5, atol=2e-3)
    assert np.allclose(rec0["depth"], rec1["depth"], rtol=1e-5)
    assert np.allclose(con0, con1, rtol=2e-3, atol=1e-6)
    assert np.all(np.abs(rec0["radius"] - rec1["radius"]) <= 1)
    assert np.mean(rec0["radius"] == rec1["radius"]) > 0.9

    # culling: at the near plane, just beyond it, behind, non-finite, negative covariance
    near = np.float32(0.2)
    beyond = float(np.nextafter(near, np.float32(1)))
    pts = [(0, 0, float(near)), (0, 0, beyond), (0, 0, -3.0), (float("nan"), 0, 5.0),
           (0, 0, float("inf")), (0, 0, 5.0)]  # the point at infinite depth: depth not finite
    covs = [np.eye(3) * 1e-4] * 5 + [-np.eye(3)]
    g, cv = _g3(pts, covs)
    st, rec, con = O.preprocess(g, cv, cam)
    assert st == 0
    assert list(rec["radius"]) == [0, rec["radius"][1], 0, 0, 0, 0]
    assert rec["radius"][1] > 0 and rec["depth"][1] == np.float32(beyond)
    for i in (0, 2, 3, 4, 5):
        assert tuple(rec[i]) == (0.0, 0.0, 0.0, 0) and not np.any(con[i])
    # invalid camera
    bad = _cam(fx=0.0)
    assert O.preprocess(g, cv, bad)[0] == 1


# ------------------------------------------------------------ rendering
def _render_case(O, gs, order_by_tile, width, height, bg=(0.1, 0.2, 0.3)):
    """gs: list of (x, y, a, b, c, opacity, (r, g, bl)); order_by_tile: per
    tile the list of Gaussian indices front to back."""
    n = len(gs)
    rec = np.zeros(n, dtype=synth.GAUSSIAN2D)
    conic = np.zeros((n, 4), dtype=np.float32)
    rgb = np.zeros((n, 3), dtype=np.float32)
    for i, (x, y, a, b, c, o, col) in enumerate(gs):
        rec[i] = (x, y, 1.0 + i, 5)
        conic[i] = (a, b, c, o)
        rgb[i] = col
    values, ranges = [], np.zeros((len(order_by_tile), 2), dtype=np.uint32)
    for t, lst in enumerate(order_by_tile):
        ranges[t] = (len(values), len(values) + len(lst))
        values += lst
    st, img = O.render(rec, conic, rgb, np.array(values, dtype=np.uint32), ranges, width, height, bg)
    assert st == 0
    return img.astype(np.float64)


def _alpha(o, a, b, c, dx, dy):
    p = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy
    if p > 0:
        return 0.0
    al = min(0.99, o * math.exp(p))
    return 0.0 if al < 1.0 / 255.0 else al


def check_render(O):
    """Front-to-back blending against closed forms in float64 (tolerance
    1e-5; pixels whose alpha lies within 1e-4 of the 1/255 cut are not
    used): one Gaussian over a 16x16 tile (colour alpha + (1 - alpha)
    background, Gaussian falloff through the conic, cut below 1/255); two
    Gaussians in both orders (order matters); opaque layers stopping when
    the transmittance would drop below 1e-4 (three of five contribute at
    alpha 0.95); an indefinite conic (pixels with positive exponent are
    skipped); tiles of a 64x20 image (row-major tile ids, each pixel sees
    only its own tile's list); an opaque Gaussian (alpha capped at 0.99); an
    empty list (background)."""
    bg = np.array([0.1, 0.2, 0.3])
    col = np.array([1.0, 0.5, 0.25])
    g0 = (5.0, 7.0, 0.5, 0.0, 0.5, 0.6, tuple(col))
    img = _render_case(O, [g0], [[0]], 16, 16)
    for py in range(16):
        for px in range(16):
            dx, dy = 5.0 - px, 7.0 - py
            p = -0.25 * (dx * dx + dy * dy)
            raw = 0.6 * math.exp(p)
            if abs(raw - 1 / 255) < 1e-4:
                continue
            al = _alpha(0.6, 0.5, 0.0, 0.5, dx, dy)
            assert np.allclose(img[py, px], col * al + (1 - al) * bg, atol=1e-5), (px, py)
    # two Gaussians at one point, both orders
    c2 = np.array([0.0, 0.0, 1.0])
    g1 = (5.0, 7.0, 0.5, 0.0, 0.5, 0.5, tuple(c2))
    a0, a1 = 0.6, 0.5
    front = _render_case(O, [g0, g1], [[0, 1]], 16, 16)[7, 5]
    back = _render_case(O, [g0, g1], [[1, 0]], 16, 16)[7, 5]
    assert np.allclose(front, col * a0 + c2 * a1 * (1 - a0) + (1 - a0) * (1 - a1) * bg, atol=1e-6)
    assert np.allclose(back, c2 * a1 + col * a0 * (1 - a1) + (1 - a0) * (1 - a1) * bg, atol=1e-6)
    # opaque layers: alpha = 0.95 each; T = 0.05, 0.0025, 1.25e-4, then 6.25e-6 < 1e-4 stops
    cols = [np.array(v) for v in ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1))]
    layers = [(3.0, 3.0, 0.5, 0.0, 0.5, 0.95, tuple(cc)) for cc in cols]
    px = _render_case(O, layers, [[0, 1, 2, 3, 4]], 16, 16)[3, 3]
    want = sum(cols[k] * 0.95 * 0.05 ** k for k in range(3)) + 0.05 ** 3 * bg
    assert np.allclose(px, want, atol=1e-6), (px, want)
    # indefinite conic: power = -dx dy > 0 where dx dy < 0
    gi = (8.0, 8.0, 0.0, 1.0, 0.0, 0.5, tuple(col))
    img = _render_case(O, [gi], [[0]], 16, 16)
    for (qx, qy) in ((9, 7), (7, 9), (12, 3)):
        assert np.allclose(img[qy, qx], bg, atol=1e-7)
    al = _alpha(0.5, 0.0, 1.0, 0.0, 8.0 - 9, 8.0 - 9)
    assert al > 0 and np.allclose(img[9, 9], col * al + (1 - al) * bg, atol=1e-5)
    # tiles of a 64x20 image: 4 x 2 tiles, the Gaussian listed in tile 1 only (row 0, column 1)
    gt = (20.0, 5.0, 0.02, 0.0, 0.02, 0.8, tuple(col))
    img = _render_case(O, [gt], [[], [0], [], [], [], [], [], []], 64, 20)
    assert np.allclose(img[5, 20], col * 0.8 + 0.2 * bg, atol=1e-6)
    assert np.allclose(img[5, 15], bg, atol=1e-7) and np.allclose(img[16, 20], bg, atol=1e-7)
    assert np.allclose(img[5, 32], bg, atol=1e-7)
    inside = _alpha(0.8, 0.02, 0.0, 0.02, 20.0 - 31, 5.0 - 15)
    assert np.allclose(img[15, 31], col * inside + (1 - inside) * bg, atol=1e-5)
    # an opaque Gaussian: alpha capped at 0.99
    go = (4.0, 4.0, 0.5, 0.0, 0.5, 1.0, tuple(col))
    assert np.allclose(_render_case(O, [go], [[0]], 16, 16)[4, 4], col * 0.99 + 0.01 * bg, atol=1e-6)
    # empty list: background everywhere
    img = _render_case(O, [g0], [[]], 16, 16)
    assert np.allclose(img, np.broadcast_to(bg, img.shape), atol=1e-7)


# ------------------------------------------------------------ 32-bit normalised key
def check_normalized(O):
    """The 32-bit key (tile << 10 | normalised depth) against hand-computed
    cases: three visible depths 1, 2, 3 in one tile map to 0, 512, 1023
    (range 2, scale 512, the top clamped to 1023) while a culled Gaussian
    with a smaller depth does not move the range; depths closer than
    range/1024 collapse and keep index order (where the exact sort reverses
    them); tiles come first; well-separated depths reproduce the exact
    sort's values; more than 2^20 tiles are rejected; ranges partition the
    list."""
    g = synth.records([4.0, 8.0, 12.0, 5.0], [4.0, 8.0, 12.0, 5.0], [3.0, 1.0, 2.0, 0.5], [2, 2, 2, 0])
    st, k, v, r = O.sort_frame_normalized(g, 16, 16)
    assert st == 0
    assert list(k) == [0, 512, 1023] and list(v) == [1, 2, 0]
    assert list(r[0]) == [0, 3]
    # collapse: depth 1.0005 (index 0) and 1.0 (index 1) share q = 0 (range 2)
    g = synth.records([4.0, 6.0, 8.0], [4.0, 6.0, 8.0], [1.0005, 1.0, 3.0], [2, 2, 2])
    st, k, v, r = O.sort_frame_normalized(g, 16, 16)
    assert list(k) == [0, 0, 1023] and list(v) == [0, 1, 2]
    exact = O.sort_frame(g, 16, 16)
    assert list(exact["values"]) == [1, 0, 2]
    # tile first: a far Gaussian in tile 0 before a near one in tile 1 (32x16 image)
    g = synth.records([4.0, 20.0], [4.0, 4.0], [9.0, 1.0], [2, 2])
    st, k, v, r = O.sort_frame_normalized(g, 32, 16)
    assert list(k) == [1023, (1 << 10) | 0] and list(v) == [0, 1]
    assert [list(x) for x in r] == [[0, 1], [1, 2]]
    # well-separated depths (step 4 over a range of 1996: every q distinct)
    rng = np.random.default_rng(5)
    n = 500
    x = rng.uniform(0, 200, n)
    y = rng.uniform(0, 120, n)
    d = 1.0 + 4.0 * rng.permutation(n)
    g = synth.records(x, y, d, rng.integers(1, 30, n))
    st, k, v, r = O.sort_frame_normalized(g, 200, 120)
    exact = O.sort_frame(g, 200, 120)
    assert st == 0 and np.array_equal(v, exact["values"])
    assert np.array_equal(k >> 10, (exact["keys"] >> np.uint64(32)).astype(np.uint32))
    assert np.array_equal(r, exact["ranges"])
    # more than 2^20 tiles
    g1 = synth.records([4.0], [4.0], [1.0], [2])
    assert O.sort_frame_normalized(g1, 16400, 16400)[0] == 1
    # ranges partition the list in tile order
    fr = synth.frame_small(1, n=3000, width=200, height=150)
    st, k, v, r = O.sort_frame_normalized(fr.gaussians, fr.width, fr.height)
    assert np.all(np.diff(k.astype(np.int64)) >= 0)
    nz = r[r[:, 1] > r[:, 0]]
    assert nz[0, 0] == 0 and nz[-1, 1] == len(k) and np.all(nz[1:, 0] == nz[:-1, 1])


ALL_CHECKS = (check_golden, check_count_and_duplicate_bruteforce, check_special_cases,
              check_validity, check_scan, check_sort, check_preprocess, check_render, check_normalized)


def run_all(O) -> list[str]:
    """Names of the checks that fail for oracle ``O``."""
    failed = []
    for check in ALL_CHECKS:
        try:
            if check is check_count_and_duplicate_bruteforce:
                check(O, seeds=range(60))
            else:
                check(O)
        except AssertionError:
            failed.append(check.__name__)
    return failed


if __name__ == "__main__":  # run every check against the library named on the command line
    import sys
    from oracle import oracle as _O
    print(json.dumps(run_all(_O.Oracle(_O.load(sys.argv[1])))))
