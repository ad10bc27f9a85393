"""Rendering (tdgs_render) against the CPU oracle's blend.

Both sides blend in float32 in the same order; they differ only through
exp (the GPU's expf against the C library's), whose last-bit differences
can flip a threshold decision (the 1/255 cut or the 1e-4 stop) now and
then.  The bar: no pixel channel off by more than 0.02 (a few flipped
contributions of at most 1/255 each), at most 0.1 % of pixels off by more
than 1e-4, and a mean absolute difference below 1e-6."""
import numpy as np
import pytest
import torch

from paper_2511_16298_gb300 import synth
from paper_2511_16298_gb300 import tdgs as T

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
BG = (0.2, 0.3, 0.4)


@pytest.fixture(scope="module")
def ctx():
    from paper_2511_16298_gb300 import build
    build.build()
    c = T.Context(0)
    yield c
    c.close()


def dev_scene(sc):
    g = torch.from_numpy(sc.gaussians.view(np.float32).reshape(-1, 4).copy()).to(DEV)
    c = torch.from_numpy(sc.cov.view(np.float32).reshape(-1, 8).copy()).to(DEV)
    rgb = torch.from_numpy(sc.rgb.copy()).to(DEV)
    return g, c, rgb


def oracle_image(oracle, sc, cam):
    st, rec, con = oracle.preprocess(sc.gaussians, sc.cov, cam)
    W, H = int(cam["width"]), int(cam["height"])
    ref = oracle.sort_frame(rec, W, H)
    assert ref["status"] == 0
    st, img = oracle.render(rec, con, sc.rgb, ref["values"], ref["ranges"], W, H, BG)
    assert st == 0
    return img, ref["m"]


def compare(got, want, frac=1e-3, mean=1e-6):
    d = np.abs(got.astype(np.float64) - want.astype(np.float64))
    assert d.max() <= 0.02, d.max()
    per_px = d.max(axis=2)
    assert np.mean(per_px > 1e-4) <= frac, np.mean(per_px > 1e-4)
    assert d.mean() < mean, d.mean()


@pytest.mark.parametrize("view", [0, 1, 2, 5])
def test_render_matches_oracle(ctx, oracle, view):
    sc = synth.scene3d(seed=2, n=30_000, views=6, width=640, height=360, scale0=0.05)
    g, c, rgb = dev_scene(sc)
    img, m = ctx.render_frame_3d(g, c, rgb, sc.cameras[view], BG)
    want, m_ref = oracle_image(oracle, sc, sc.cameras[view])
    assert m == m_ref and m > 0
    compare(img.cpu().numpy(), want)


def test_render_odd_image_size(ctx, oracle):
    """Partial edge tiles: 200 x 75 pixels."""
    sc = synth.scene3d(seed=4, n=5_000, views=2, width=200, height=75, scale0=0.08)
    g, c, rgb = dev_scene(sc)
    img, m = ctx.render_frame_3d(g, c, rgb, sc.cameras[1], BG)
    want, _ = oracle_image(oracle, sc, sc.cameras[1])
    compare(img.cpu().numpy(), want)


def test_render_empty_frame_is_background(ctx):
    sc = synth.scene3d(seed=5, n=1000, views=1, width=64, height=48)
    cam = sc.cameras[0].copy()
    cam["trans"] = (0.0, 0.0, -1000.0)  # everything behind the camera
    g, c, rgb = dev_scene(sc)
    img, m = ctx.render_frame_3d(g, c, rgb, cam, BG)
    assert m == 0
    assert torch.allclose(img, torch.tensor(BG, device=DEV).expand_as(img))


def test_render_scene_full_size(ctx, oracle):
    """The 500,000-Gaussian scene seen by one 1280x720 camera."""
    sc = synth.scene3d(seed=0, n=500_000, views=1)
    g, c, rgb = dev_scene(sc)
    img, m = ctx.render_frame_3d(g, c, rgb, sc.cameras[0], BG)
    want, m_ref = oracle_image(oracle, sc, sc.cameras[0])
    assert m == m_ref
    compare(img.cpu().numpy(), want)


def test_render_heaviest_first_path(ctx, oracle):
    """An image with more tiles than one wave of resident blocks (3600 at
    1280x720) takes the ordered path: a tile-order launch, then the blend;
    a 320x180 image (240 tiles, fewer than two blocks per SM) renders in
    raster order without it.  Both images match the oracle."""
    sc = synth.scene3d(seed=6, n=40_000, views=2, scale0=0.05)
    g, c, rgb = dev_scene(sc)
    small = sc.cameras[1].copy()
    small["width"], small["height"], small["cx"], small["cy"] = 320, 180, 160.0, 90.0
    for cam, ordered in ((sc.cameras[0], True), (small, False)):
        ctx.enable_timing(True)
        img, m = ctx.render_frame_3d(g, c, rgb, cam, BG)
        kt = ctx.kernel_times()
        ctx.enable_timing(False)
        assert kt["render"]["launches"] == 1
        assert ("render_order" in kt) == ordered, kt.keys()
        want, m_ref = oracle_image(oracle, sc, cam)
        assert m == m_ref and m > 0
        compare(img.cpu().numpy(), want)


def test_render_ordered_empty_frame_is_background(ctx):
    """Ordered path with every tile empty (the order kernel's all-zero
    maximum): the image is the background."""
    sc = synth.scene3d(seed=7, n=2000, views=1)
    cam = sc.cameras[0].copy()
    cam["trans"] = (0.0, 0.0, -1000.0)
    g, c, rgb = dev_scene(sc)
    img, m = ctx.render_frame_3d(g, c, rgb, cam, BG)
    assert m == 0
    assert torch.allclose(img, torch.tensor(BG, device=DEV).expand_as(img))


def test_render_ordered_skewed_tiles(ctx, oracle):
    """The scene pushed into the bottom-right corner of a 1280x720 image
    (principal point there): a few heavy tiles, thousands of empty ones,
    on the ordered path."""
    sc = synth.scene3d(seed=8, n=20_000, views=1, scale0=0.05)
    cam = sc.cameras[0].copy()
    cam["cx"], cam["cy"] = 1200.0, 680.0  # principal point near the far corner
    g, c, rgb = dev_scene(sc)
    img, m = ctx.render_frame_3d(g, c, rgb, cam, BG)
    want, m_ref = oracle_image(oracle, sc, cam)
    assert m == m_ref and m > 0
    compare(img.cpu().numpy(), want)


def test_render_4k_image(ctx, oracle):
    """3840x2160 (32,400 tiles): the tile-order kernel's block loops over
    many tiles per thread."""
    sc = synth.scene3d(seed=9, n=20_000, views=1, width=3840, height=2160, scale0=0.05)
    cam = sc.cameras[0].copy()
    cam["fx"], cam["fy"] = 3325.5, 3325.5
    g, c, rgb = dev_scene(sc)
    img, m = ctx.render_frame_3d(g, c, rgb, cam, BG)
    want, m_ref = oracle_image(oracle, sc, cam)
    assert m == m_ref and m > 0
    compare(img.cpu().numpy(), want)


def test_render_inverted_ranges_are_empty(ctx, oracle):
    """A range whose start is past its end holds no Gaussians, on the GPU
    as in the oracle's loop; inverted here: every seventh tile and the
    heaviest one (the first in heaviest-first order)."""
    sc = synth.scene3d(seed=10, n=30_000, views=1, scale0=0.05)
    cam = sc.cameras[0]
    g, c, rgb = dev_scene(sc)
    k, v, r, m, rec, con = ctx.sort_frame_3d(g, c, cam, copy=True)
    rr = r.cpu().numpy().view(np.uint32).copy()
    lens = rr[:, 1].astype(np.int64) - rr[:, 0]
    flip = np.zeros(len(rr), dtype=bool)
    flip[::7] = True
    flip[int(np.argmax(lens))] = True
    flip &= lens > 0
    assert flip.sum() > 10
    rr[flip] = rr[flip][:, ::-1]
    W, H = int(cam["width"]), int(cam["height"])
    r2 = torch.from_numpy(rr.view(np.int32)).to(DEV)
    img = ctx.render(rec, con, rgb, v, r2, W, H, BG)
    rec_h = rec.cpu().numpy().view(synth.GAUSSIAN2D).reshape(-1)
    st, want = oracle.render(rec_h, con.cpu().numpy(), sc.rgb, v.cpu().numpy().view(np.uint32), rr, W, H, BG)
    assert st == 0
    compare(img.cpu().numpy(), want)
    gx = (W + 15) // 16
    t = int(np.argmax(lens))
    tile = img[(t // gx) * 16:(t // gx) * 16 + 16, (t % gx) * 16:(t % gx) * 16 + 16].cpu()
    assert torch.allclose(tile, torch.tensor(BG).expand_as(tile))


def extreme_conics(seed, n, W, H):
    """Records and conics built directly (no projection): 2D covariances
    with axis ratios from 1 to 3000 at random angles (so det / ac runs
    from 1 down to about 1e-6, on both sides of the culling's 1e-3
    threshold), scales from 0.3 to 12 pixels, opacities from 0.02 to 0.6
    with one in twenty below 1/255 (no pixel passes) and 3 % of the conics
    indefinite (b^2 > ac, which reach every warp; their rectangles capped
    at 12 pixels).  Sparse enough that most pixels do not saturate."""
    rng = np.random.default_rng(seed)
    s1 = np.exp(rng.uniform(np.log(0.3), np.log(12.0), n))
    ratio = np.exp(rng.uniform(0.0, np.log(3000.0), n))
    s2 = np.minimum(s1 * ratio, 120.0)
    th = rng.uniform(0.0, np.pi, n)
    cs, sn = np.cos(th), np.sin(th)
    # Q = R diag(1/s1^2, 1/s2^2) R^T in float64, rounded to float32
    i1, i2 = 1.0 / s1 ** 2, 1.0 / s2 ** 2
    a = cs * cs * i1 + sn * sn * i2
    b = cs * sn * (i1 - i2)
    c = sn * sn * i1 + cs * cs * i2
    bad = rng.random(n) < 0.03
    b = np.where(bad, np.sqrt(a * c) * rng.uniform(1.01, 3.0, n), b)
    op = np.where(rng.random(n) < 0.05, rng.uniform(0.002, 0.0039, n), rng.uniform(0.02, 0.6, n))
    con = np.stack([a, b, c, op], 1).astype(np.float32)
    rec = np.zeros(n, dtype=synth.GAUSSIAN2D)
    rec["x"] = rng.uniform(-20.0, W + 20.0, n).astype(np.float32)
    rec["y"] = rng.uniform(-20.0, H + 20.0, n).astype(np.float32)
    rec["depth"] = rng.uniform(0.5, 50.0, n).astype(np.float32)
    rad = np.ceil(3.0 * np.maximum(s1, s2))
    rec["radius"] = np.where(bad, np.minimum(rad, 12), np.minimum(rad, 360)).astype(np.int32)
    rgb = rng.random((n, 3)).astype(np.float32)
    return rec, con, rgb


@pytest.mark.parametrize("W,H", [(1280, 720), (320, 180)])
def test_render_extreme_conics(ctx, oracle, W, H):
    """Elongated, near-singular and indefinite conics and tiny opacities,
    on the ordered (1280x720) and raster-order (320x180) paths: the
    per-warp culling must leave every pixel as the oracle's blend has it.
    Each side sorts the records itself (compared first) and renders with
    its own lists.

    Bar: max |d| <= 0.02 as everywhere (a Gaussian culled wrongly would
    move a pixel by up to alpha * colour), but up to 1 % of pixels above
    1e-4 and a mean below 1e-5: with axis ratios up to 3000 the exponent's
    terms nearly cancel, and the kernel's fused form dx (A dx + B dy) +
    C dy^2 rounds differently from the oracle's written order.  A CPU
    blend with the kernel's form, float32 exp and no culling differs from
    the oracle on 0.16 % (1280x720) and 0.12 % (320x180) of pixels, mean
    1.8e-6 and 1.2e-6."""
    rec, con, rgb = extreme_conics(11, 3000 if W > 640 else 800, W, H)
    g = tdgs_records(rec)
    k, v, r, m = ctx.sort_frame(g, W, H, copy=True)
    ref = oracle.sort_frame(rec, W, H)
    assert ref["status"] == 0 and m == ref["m"] > 0
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ref["values"])
    assert np.array_equal(r.cpu().numpy().view(np.uint32).reshape(-1), ref["ranges"].reshape(-1))
    img = ctx.render(g, torch.from_numpy(con).to(DEV), torch.from_numpy(rgb).to(DEV), v, r, W, H, BG)
    st, want = oracle.render(rec, con, rgb, ref["values"], ref["ranges"], W, H, BG)
    assert st == 0
    compare(img.cpu().numpy(), want, frac=1e-2, mean=1e-5)


def tdgs_records(rec):
    return torch.from_numpy(np.ascontiguousarray(rec).view(np.int32).reshape(-1, 4).copy()).to(DEV)
