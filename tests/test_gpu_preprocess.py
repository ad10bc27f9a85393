"""Parity of the preprocessing stage (tdgs_preprocess, tdgs_sort_frame_3d)
with the CPU oracle.

Both sides compute in float32 with the same pinned operation order and no
fused multiply-adds, so records (mean, depth, radius) and conics must be
bit-identical; the sorted output of the 3D frame must equal the oracle's
five steps on the oracle's own records."""
import functools
import math

import numpy as np
import pytest
import torch

from paper_2511_16298_gb300 import synth
from paper_2511_16298_gb300 import tdgs as T
from tests import oracle_pins as P

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    from paper_2511_16298_gb300 import build
    build.build()
    c = T.Context(0)
    yield c
    c.close()


def dev3(scene_g, scene_cov):
    g = torch.from_numpy(np.ascontiguousarray(scene_g).view(np.float32).reshape(-1, 4).copy()).to(DEV)
    c = torch.from_numpy(np.ascontiguousarray(scene_cov).view(np.float32).reshape(-1, 8).copy()).to(DEV)
    return g, c


def rec_bits(rec: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(rec).view(np.uint32).reshape(-1, 4)


@functools.lru_cache(maxsize=1)
def small_scene():
    return synth.scene3d(seed=1, n=20_000, views=6, width=640, height=360)


def edge_gaussians():
    """Near plane, behind the camera, non-finite, degenerate and huge
    covariances, slopes beyond the clamp, points off screen."""
    near = float(np.float32(0.2))
    beyond = float(np.nextafter(np.float32(0.2), np.float32(1)))
    pts = [(0, 0, near), (0, 0, beyond), (0, 0, -4.0), (math.nan, 0, 3.0), (0, math.inf, 3.0),
           (0, 0, math.inf), (0.1, 0.2, 3.0), (0.1, 0.2, 3.0), (0.1, 0.2, 3.0), (9.0, 0.1, 2.0),
           (-9.0, 5.0, 2.0), (40.0, 40.0, 1.0), (0, 0, 1e-3 + 0.2), (0, 0, 5.0), (0.1, 0.2, 3.0)]
    eye = np.eye(3)
    covs = [eye * 1e-4, eye * 1e-4, eye * 1e-4, eye * 1e-4, eye * 1e-4, eye * 1e-4,
            np.zeros((3, 3)), -eye, eye * 1e13, np.diag([1e-4, 4e-4, 9e-2]),
            np.array([[0.01, 0.004, 0.0], [0.004, 0.02, 0.001], [0.0, 0.001, 0.03]]),
            eye * 1e-2, eye * 50.0, np.full((3, 3), math.nan), eye * 1e30]
    return P._g3(pts, covs)


@pytest.mark.parametrize("view", range(6))
def test_preprocess_bit_exact(ctx, oracle, view):
    sc = small_scene()
    g, c = dev3(sc.gaussians, sc.cov)
    rec, con = ctx.preprocess(g, c, sc.cameras[view])
    st, orec, ocon = oracle.preprocess(sc.gaussians, sc.cov, sc.cameras[view])
    assert st == 0
    got = rec.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, rec_bits(orec))
    assert np.array_equal(con.cpu().numpy().view(np.uint32), ocon.view(np.uint32))
    assert (orec["radius"] > 0).sum() > 1000  # the case exercises visible Gaussians


def test_preprocess_edge_cases(ctx, oracle):
    g3, cov = edge_gaussians()
    cam = P._cam()
    g, c = dev3(g3, cov)
    rec, con = ctx.preprocess(g, c, cam)
    st, orec, ocon = oracle.preprocess(g3, cov, cam)
    assert st == 0
    assert np.array_equal(rec.cpu().numpy().view(np.uint32), rec_bits(orec))
    assert np.array_equal(con.cpu().numpy().view(np.uint32), ocon.view(np.uint32))
    assert orec["radius"][8] == 1 << 30  # huge covariance: radius capped
    assert orec["radius"][14] == 0       # the determinant overflows: culled


def test_preprocess_without_conic_and_empty(ctx, oracle):
    sc = small_scene()
    g, c = dev3(sc.gaussians, sc.cov)
    rec, con = ctx.preprocess(g, c, sc.cameras[0], with_conic=False)
    assert con is None
    st, orec, _ = oracle.preprocess(sc.gaussians, sc.cov, sc.cameras[0])
    assert np.array_equal(rec.cpu().numpy().view(np.uint32), rec_bits(orec))
    e = torch.empty((0, 4), dtype=torch.float32, device=DEV)
    r0, c0 = ctx.preprocess(e, torch.empty((0, 8), dtype=torch.float32, device=DEV), sc.cameras[0])
    assert r0.shape == (0, 4) and c0.shape == (0, 4)


def test_preprocess_rejects_bad_camera(ctx):
    sc = small_scene()
    g, c = dev3(sc.gaussians[:10], sc.cov[:10])
    for field, val in (("fx", 0.0), ("fy", -1.0), ("fx", math.inf), ("width", 0), ("height", 0)):
        cam = sc.cameras[0].copy()
        cam[field] = val
        with pytest.raises(T.TdgsError) as e:
            ctx.preprocess(g, c, cam)
        assert e.value.status == T.INVALID_ARGUMENT
    with pytest.raises(T.TdgsError):  # misaligned records
        ctx.preprocess(g, c, sc.cameras[0], records=torch.empty(41 * 4, dtype=torch.int32, device=DEV)[1:41].view(10, 4))


@pytest.mark.parametrize("view", [0, 3])
def test_sort_frame_3d_matches_oracle(ctx, oracle, view):
    sc = small_scene()
    cam = sc.cameras[view]
    g, c = dev3(sc.gaussians, sc.cov)
    k, v, r, m, rec, con = ctx.sort_frame_3d(g, c, cam, copy=True)
    st, orec, ocon = oracle.preprocess(sc.gaussians, sc.cov, cam)
    assert np.array_equal(rec.cpu().numpy().view(np.uint32), rec_bits(orec))
    assert np.array_equal(con.cpu().numpy().view(np.uint32), ocon.view(np.uint32))
    ref = oracle.sort_frame(orec, int(cam["width"]), int(cam["height"]))
    assert ref["status"] == 0 and m == ref["m"] and m > 0
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ref["keys"])
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ref["values"])
    assert np.array_equal(r.cpu().numpy().view(np.uint32), ref["ranges"])


def test_scene_full_size_bit_exact(ctx, oracle):
    """The 500,000-Gaussian scene (the benchmark's 3D workload), camera 0:
    every record and conic."""
    sc = synth.scene3d(seed=0, n=500_000, views=2)
    g, c = dev3(sc.gaussians, sc.cov)
    k, v, r, m, rec, con = ctx.sort_frame_3d(g, c, sc.cameras[0], copy=True)
    st, orec, ocon = oracle.preprocess(sc.gaussians, sc.cov, sc.cameras[0])
    assert np.array_equal(rec.cpu().numpy().view(np.uint32), rec_bits(orec))
    assert np.array_equal(con.cpu().numpy().view(np.uint32), ocon.view(np.uint32))
    ref = oracle.sort_frame(orec, 1280, 720)
    assert m == ref["m"]
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ref["keys"])
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ref["values"])
    assert np.array_equal(r.cpu().numpy().view(np.uint32), ref["ranges"])


@pytest.mark.parametrize("nv", [1, 5])
def test_sort_views_3d_matches_per_camera_oracle(ctx, oracle, nv):
    """A batch of cameras over one 3D scene: every view equals the oracle's
    preprocessing and sort for that camera alone (local tile ids and
    indices), and the projected records are the oracle's."""
    sc = small_scene()
    g, c = dev3(sc.gaussians, sc.cov)
    cams = sc.cameras[:nv]
    res = ctx.sort_views_3d(g, c, cams, copy=True)
    rec_all, con_all = ctx.projected(sc.n * nv)
    rec_all = rec_all.cpu().numpy().view(np.uint32)
    con_all = con_all.cpu().numpy().view(np.uint32)
    for v in range(nv):
        st, orec, ocon = oracle.preprocess(sc.gaussians, sc.cov, cams[v])
        assert np.array_equal(rec_all[v * sc.n:(v + 1) * sc.n], rec_bits(orec))
        assert np.array_equal(con_all[v * sc.n:(v + 1) * sc.n], ocon.view(np.uint32))
        ref = oracle.sort_frame(orec, int(cams[v]["width"]), int(cams[v]["height"]))
        k, vv, r, m = res[v]
        assert m == ref["m"]
        assert np.array_equal(k.cpu().numpy().view(np.uint64), ref["keys"])
        assert np.array_equal(vv.cpu().numpy().view(np.uint32), ref["values"])
        assert np.array_equal(r.cpu().numpy().view(np.uint32), ref["ranges"])


def test_sort_views_3d_full_scene_sampled(ctx, oracle):
    """The 64-camera 3D batch (500,000 Gaussians, the benchmark's workload):
    total pairs equal the per-camera frames and three views are checked
    against the oracle."""
    sc = synth.scene3d(seed=0)
    g, c = dev3(sc.gaussians, sc.cov)
    res = ctx.sort_views_3d(g, c, sc.cameras, copy=True)
    assert len(res) == 64
    for v in (0, 31, 63):
        st, orec, _ = oracle.preprocess(sc.gaussians, sc.cov, sc.cameras[v])
        ref = oracle.sort_frame(orec, 1280, 720)
        k, vv, r, m = res[v]
        assert m == ref["m"]
        assert np.array_equal(k.cpu().numpy().view(np.uint64), ref["keys"])
        assert np.array_equal(vv.cpu().numpy().view(np.uint32), ref["values"])
        assert np.array_equal(r.cpu().numpy().view(np.uint32), ref["ranges"])


def test_sort_views_3d_mixed_resolutions(ctx, oracle):
    """Cameras of different image sizes in one 3D batch."""
    sc = small_scene()
    cams = sc.cameras[:3].copy()
    cams[1]["width"], cams[1]["height"], cams[1]["cx"], cams[1]["cy"] = 200, 90, 100.0, 45.0
    cams[2]["width"], cams[2]["height"], cams[2]["cx"], cams[2]["cy"] = 1000, 700, 500.0, 350.0
    g, c = dev3(sc.gaussians, sc.cov)
    res = ctx.sort_views_3d(g, c, cams, copy=True)
    for v in range(3):
        st, orec, _ = oracle.preprocess(sc.gaussians, sc.cov, cams[v])
        ref = oracle.sort_frame(orec, int(cams[v]["width"]), int(cams[v]["height"]))
        k, vv, r, m = res[v]
        assert m == ref["m"]
        assert np.array_equal(k.cpu().numpy().view(np.uint64), ref["keys"])
        assert np.array_equal(vv.cpu().numpy().view(np.uint32), ref["values"])
        assert np.array_equal(r.cpu().numpy().view(np.uint32), ref["ranges"])
