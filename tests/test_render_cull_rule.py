"""The render kernel's per-warp culling rule, restated in float32 numpy and
checked against the kernel's own per-pixel cut test on a scene of extreme
conics (CPU; no GPU).

The rule (render kernel, staging step): with K = -2 cut, Q = [[a, b],
[b, c]] the conic and det = ac - b^2 by one fused multiply-add, a warp
(rows 2w, 2w+1 of a 16x16 tile) is left out when every row lies farther
from the mean than sqrt(1.0201 K a / det) + 0.25 (tested on squares), and
every warp when the tile's columns lie farther than sqrt(1.0201 K c / det)
+ 0.25; flat (det <= 1e-3 ac), indefinite or non-finite conics reach every
warp, and K < 0 reaches none.  The cut test a pixel applies: power =
dx (A dx + B dy) + C dy^2 with A = -a/2, B = -b, C = -c/2 as two fused
multiply-adds; the step passes when cut <= power <= 0.  A culled step
that would pass is a violation: the culling must only drop steps the cut
test drops.  This checks the rule's mathematics (the ellipse's extents and
the margins); the GPU tests check the kernel's images against the oracle.
"""
import numpy as np


f32 = np.float32


def fma32(x, y, z):
    """x * y + z rounded once to float32 (the float64 product of two
    float32 values is exact)."""
    return (np.asarray(x, np.float64) * np.asarray(y, np.float64) + np.asarray(z, np.float64)).astype(f32)


def scene(seed, n, W, H):
    """Conics with axis ratios up to 3000 at random angles, 3 % indefinite,
    one in twenty opacities below 1/255."""
    rng = np.random.default_rng(seed)
    s1 = np.exp(rng.uniform(np.log(0.3), np.log(12.0), n))
    s2 = np.minimum(s1 * np.exp(rng.uniform(0.0, np.log(3000.0), n)), 120.0)
    th = rng.uniform(0.0, np.pi, n)
    cs, sn = np.cos(th), np.sin(th)
    i1, i2 = 1.0 / s1 ** 2, 1.0 / s2 ** 2
    a = cs * cs * i1 + sn * sn * i2
    b = cs * sn * (i1 - i2)
    c = sn * sn * i1 + cs * cs * i2
    bad = rng.random(n) < 0.03
    b = np.where(bad, np.sqrt(a * c) * rng.uniform(1.01, 3.0, n), b)
    op = np.where(rng.random(n) < 0.05, rng.uniform(0.002, 0.0039, n), rng.uniform(0.02, 0.6, n))
    con = np.stack([a, b, c, op], 1).astype(f32)
    x = rng.uniform(-20.0, W + 20.0, n).astype(f32)
    y = rng.uniform(-20.0, H + 20.0, n).astype(f32)
    rad = np.where(bad, np.minimum(np.ceil(3 * np.maximum(s1, s2)), 12), np.minimum(np.ceil(3 * np.maximum(s1, s2)), 360))
    return x, y, rad.astype(np.int64), con


def warp_masks(x, y, con, tx0, ty0):
    a, b, c, op = (con[:, k] for k in range(4))
    with np.errstate(all="ignore"):
        cut = np.where(op > 0, -np.log(f32(255.0) * op).astype(f32), f32(np.inf)).astype(f32)
        K = (f32(-2.0) * cut).astype(f32)
        ac = (a * c).astype(f32)
        det = fma32(-b, b, ac)
        ok = (a > 0) & (c > 0) & (det > f32(1e-3) * ac) & (K < f32(1e30))
        hy2 = ((K * a).astype(f32) / det).astype(f32) * f32(1.0201)
        hx2 = ((K * c).astype(f32) / det).astype(f32) * f32(1.0201)
        ok &= (hy2 < f32(1e30)) & (hx2 < f32(1e30))
        ex = np.maximum(np.maximum(tx0 - x, x - (tx0 + f32(15))) - f32(0.25), f32(0)).astype(f32)
        xmiss = (ex * ex).astype(f32) > hx2
        yr = (y - ty0).astype(f32)
        m = np.zeros(len(x), np.uint32)
        for w in range(8):
            r0 = f32(2 * w)
            ey = np.maximum(np.maximum(r0 - yr, yr - (r0 + f32(1))) - f32(0.25), f32(0)).astype(f32)
            m |= ((ey * ey).astype(f32) <= hy2).astype(np.uint32) << w
    m = np.where(ok, np.where(xmiss, 0, m), 0xFF).astype(np.uint32)
    return np.where(K < 0, 0, m).astype(np.uint32), cut


def test_cull_rule_drops_only_steps_the_cut_test_drops():
    W, H = 640, 368
    x, y, rad, con = scene(11, 1500, W, H)
    px = np.arange(256) & 15
    py = np.arange(256) >> 4
    warp = np.arange(256) >> 5
    culled = total = violations = 0
    for ty in range(H // 16):
        for tx in range(W // 16):
            tx0, ty0 = f32(tx * 16), f32(ty * 16)
            # Gaussians whose rectangle touches the tile (the sort's rule, loosely)
            sel = ((x + rad >= tx0) & (x - rad <= tx0 + 16) & (y + rad >= ty0) & (y - rad <= ty0 + 16))
            if not sel.any():
                continue
            gx, gy, gc = x[sel], y[sel], con[sel]
            mask, cut = warp_masks(gx, gy, gc, tx0, ty0)
            A = (f32(-0.5) * gc[:, 0]).astype(f32)
            B = (-gc[:, 1]).astype(f32)
            C = (f32(-0.5) * gc[:, 2]).astype(f32)
            dx = (gx[:, None] - (tx0 + px).astype(f32)[None, :]).astype(f32)
            dy = (gy[:, None] - (ty0 + py).astype(f32)[None, :]).astype(f32)
            with np.errstate(all="ignore"):
                power = fma32(dx, fma32(A[:, None], dx, (B[:, None] * dy).astype(f32)),
                              ((C[:, None] * dy).astype(f32) * dy).astype(f32))
                passes = (power <= 0) & (power >= cut[:, None])
            kept = ((mask[:, None] >> warp[None, :]) & 1).astype(bool)
            violations += int((passes & ~kept).sum())
            culled += int((~kept).sum())
            total += kept.size
    assert total > 1_000_000
    assert culled > 0.3 * total  # the rule does cull
    assert violations == 0
