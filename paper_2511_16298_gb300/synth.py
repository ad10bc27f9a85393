"""Seeded synthetic inputs for the 3DGS tile depth sort.

This module only draws random numbers and arranges them into the projected
Gaussian records that the sort step consumes (Sec. II-A, "Duplication with
Tiles": a 2D mean, a view depth and a pixel radius per Gaussian; Table IV
packs exactly these four values into one record).  It holds none of the
sorting method's arithmetic: no tile rectangles, no keys, no scans.  Both
the CUDA path and the CPU oracle are fed from here, so neither depends on
the other for its inputs.

The paper evaluates on trained scenes (Tanks and Temples, DeepBlending,
Synthetic-NeRF) that are not available; the workloads below are seeded
stand-ins with the sizes and value distributions of those frames:

* ``frame_small``  - 10,000 Gaussians, 256x256, uniform means.
* ``frame_scene``  - 1,000,000 Gaussians, 1280x720, 70 % clustered means.
* ``frame_large``  - 3,000,000 Gaussians, 1920x1080, 85 % clustered means,
  5 % of depths quantised to a 1/8 grid (many exact key ties).
* ``multiview``    - one 500,000-Gaussian 3D scene seen by 64 pinhole
  cameras (the projection happens here, as part of input generation).
* ``request_trace``- a Poisson stream of frames of mixed size/resolution.
* ``scene3d``      - the unprojected input of the preprocessing step: the
  multiview scene's means with opacities and anisotropic 3D covariances
  (Table I packing), and the same camera lattice as world-to-camera blocks.
  Building each covariance from its scales and rotation is input generation;
  projecting it is the method's and is not done here.

All draws use ``numpy.random.default_rng(seed)`` in float64 and are rounded
to float32 at the end; radius = ceil(3 * sigma) computed in float64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# One projected Gaussian: 2D mean (px), view depth, integer pixel radius.
GAUSSIAN2D = np.dtype(
    [("x", "<f4"), ("y", "<f4"), ("depth", "<f4"), ("radius", "<i4")], align=True
)
assert GAUSSIAN2D.itemsize == 16

TILE = 16  # screen tiles are 16x16 pixels (Sec. II-A)


@dataclasses.dataclass
class Frame:
    """One view to sort: image size and its projected Gaussians."""

    width: int
    height: int
    gaussians: np.ndarray  # GAUSSIAN2D records
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.gaussians.shape[0])

    @property
    def grid(self) -> tuple[int, int]:
        return (self.width + TILE - 1) // TILE, (self.height + TILE - 1) // TILE

    @property
    def num_tiles(self) -> int:
        gx, gy = self.grid
        return gx * gy

    @property
    def tile_bits(self) -> int:
        t = self.num_tiles
        return 0 if t <= 1 else int(t - 1).bit_length()


def records(x, y, depth, radius) -> np.ndarray:
    """Pack four equal-length arrays into GAUSSIAN2D records."""
    n = len(x)
    g = np.empty(n, dtype=GAUSSIAN2D)
    g["x"] = np.asarray(x, dtype=np.float64).astype(np.float32)
    g["y"] = np.asarray(y, dtype=np.float64).astype(np.float32)
    g["depth"] = np.asarray(depth, dtype=np.float64).astype(np.float32)
    g["radius"] = np.asarray(radius, dtype=np.int64).astype(np.int32)
    return g


def _radius(sigma: np.ndarray) -> np.ndarray:
    return np.ceil(3.0 * sigma).astype(np.int64)


def _means(rng, n, width, height, cluster_frac, n_centres, centre_sd):
    n_cl = int(round(cluster_frac * n))
    centres = rng.uniform((0.0, 0.0), (width, height), size=(n_centres, 2))
    which = rng.integers(0, n_centres, size=n_cl)
    clustered = centres[which] + rng.normal(0.0, centre_sd, size=(n_cl, 2))
    uniform = rng.uniform((0.0, 0.0), (width, height), size=(n - n_cl, 2))
    pts = np.concatenate([clustered, uniform], axis=0)
    return pts[rng.permutation(n)]


def frame_small(seed: int = 0, n: int = 10_000, width: int = 256, height: int = 256) -> Frame:
    """10k Gaussians on 256x256: uniform means, sigma ~ lognormal(ln 3, 0.6)
    clipped to [1, 64], depth ~ U[0.2, 50]."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform((0.0, 0.0), (width, height), size=(n, 2))
    sigma = np.clip(rng.lognormal(math.log(3.0), 0.6, size=n), 1.0, 64.0)
    depth = rng.uniform(0.2, 50.0, size=n)
    return Frame(width, height, records(xy[:, 0], xy[:, 1], depth, _radius(sigma)),
                 f"small-{n}-{width}x{height}-s{seed}")


def frame_scene(seed: int = 0, n: int = 1_000_000, width: int = 1280, height: int = 720) -> Frame:
    """Scene-scale frame: 70 % of means around 32 centres (sd 60 px), 30 %
    uniform; sigma ~ lognormal(ln 4, 0.8) clipped to [1, 256];
    depth ~ lognormal(ln 5, 0.7).  Means are not clipped to the image."""
    rng = np.random.default_rng(seed)
    xy = _means(rng, n, width, height, 0.70, 32, 60.0)
    sigma = np.clip(rng.lognormal(math.log(4.0), 0.8, size=n), 1.0, 256.0)
    depth = rng.lognormal(math.log(5.0), 0.7, size=n)
    return Frame(width, height, records(xy[:, 0], xy[:, 1], depth, _radius(sigma)),
                 f"scene-{n}-{width}x{height}-s{seed}")


def frame_large(seed: int = 0, n: int = 3_000_000, width: int = 1920, height: int = 1080) -> Frame:
    """Large frame: 85 % of means around 128 centres (sd 40 px);
    sigma ~ lognormal(ln 3, 1.0) clipped to [1, 512];
    depth ~ lognormal(ln 8, 0.9), then 5 % of the Gaussians (chosen by the
    RNG) get depth round(d*8)/8, which is exact in binary and creates many
    equal keys, so stability is exercised."""
    rng = np.random.default_rng(seed)
    xy = _means(rng, n, width, height, 0.85, 128, 40.0)
    sigma = np.clip(rng.lognormal(math.log(3.0), 1.0, size=n), 1.0, 512.0)
    depth = rng.lognormal(math.log(8.0), 0.9, size=n)
    q = rng.random(n) < 0.05
    depth[q] = np.maximum(np.round(depth[q] * 8.0) / 8.0, 0.125)
    return Frame(width, height, records(xy[:, 0], xy[:, 1], depth, _radius(sigma)),
                 f"large-{n}-{width}x{height}-s{seed}")


def frame_random(seed: int, n: int, width: int, height: int, *, max_sigma: float = 64.0,
                 offscreen: float = 0.1, culled: float = 0.05, depth_ties: float = 0.0) -> Frame:
    """Small mixed frames for parity sweeps: some means off-screen, some
    Gaussians culled (radius 0), optional depth ties."""
    rng = np.random.default_rng(seed)
    margin = 2.0 * max_sigma
    x = rng.uniform(-margin * offscreen * 4, width + margin * offscreen * 4, size=n)
    y = rng.uniform(-margin * offscreen * 4, height + margin * offscreen * 4, size=n)
    sigma = np.clip(rng.lognormal(math.log(3.0), 0.9, size=n), 1.0, max_sigma)
    r = _radius(sigma)
    r[rng.random(n) < culled] = 0
    depth = rng.lognormal(math.log(6.0), 0.8, size=n)
    if depth_ties > 0:
        t = rng.random(n) < depth_ties
        depth[t] = np.maximum(np.round(depth[t] * 2.0) / 2.0, 0.5)
    return Frame(width, height, records(x, y, depth, r), f"random-{n}-{width}x{height}-s{seed}")


# ---------------------------------------------------------------- multi-view
@dataclasses.dataclass
class MultiView:
    """A 3D scene seen by several cameras; each view is a Frame whose
    records index the scene's Gaussian array."""

    views: list[Frame]
    scale0: float
    seed: int


def _fibonacci_sphere(k: int) -> np.ndarray:
    i = np.arange(k, dtype=np.float64) + 0.5
    phi = np.arccos(1.0 - 2.0 * i / k)
    theta = math.pi * (1.0 + 5.0 ** 0.5) * i
    return np.stack([np.cos(theta) * np.sin(phi), np.cos(phi), np.sin(theta) * np.sin(phi)], 1)


def multiview(seed: int = 0, n: int = 500_000, views: int = 64, width: int = 1280,
              height: int = 720, scale0: float = 0.05, cam_radius: float = 15.0,
              dist_range: tuple[float, float] = (0.25, 1.0), jitter_radius: float = 8.0) -> MultiView:
    """One scene, many cameras.  Means ~ U[0,1)^3 * 10 - 5; isotropic scale
    s ~ lognormal(ln scale0, 0.5); camera v sits on a Fibonacci lattice of
    directions at distance cam_radius * f_v, f_v log-uniform in
    ``dist_range`` (some cameras inside the cube), looking at the origin
    plus a jitter drawn uniformly from a ball of radius ``jitter_radius``
    (some look partly away), up = +y.  Pinhole with fx = fy = 1108.5,
    principal point at the image centre.  Per view: depth = view-space z,
    radius 0 (culled) where z <= 0.2, otherwise r = ceil(3 * fx * s / z)
    and the mean is projected.  The defaults spread the views' pair counts
    over about 0.4M-4.2M (seed 0: 151M pairs in all), the uneven per-view
    load a batched multi-view sort is for."""
    rng = np.random.default_rng(seed)
    mean3 = rng.random((n, 3)) * 10.0 - 5.0
    scale = rng.lognormal(math.log(scale0), 0.5, size=n)
    u = rng.normal(size=(views, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    jitter = u * (jitter_radius * rng.random(views) ** (1.0 / 3.0))[:, None]
    lo, hi = dist_range
    eye = _fibonacci_sphere(views) * (cam_radius * lo * (hi / lo) ** rng.random(views))[:, None]
    fx = fy = 1108.5
    cx, cy = width / 2.0, height / 2.0
    out = []
    for v in range(views):
        fwd = jitter[v] - eye[v]
        fwd /= np.linalg.norm(fwd)
        up = np.array([0.0, 1.0, 0.0])
        right = np.cross(fwd, up)
        if np.linalg.norm(right) < 1e-6:
            right = np.array([1.0, 0.0, 0.0])
        right /= np.linalg.norm(right)
        down = np.cross(fwd, right)
        rel = mean3 - eye[v]
        xc = rel @ right
        yc = rel @ down
        zc = rel @ fwd
        ok = zc > 0.2
        zs = np.where(ok, zc, 1.0)
        px = fx * xc / zs + cx
        py = fy * yc / zs + cy
        r = np.where(ok, np.ceil(3.0 * fx * scale / zs), 0).astype(np.int64)
        depth = np.where(ok, zc, 1.0)
        out.append(Frame(width, height, records(px, py, depth, r), f"view{v}"))
    return MultiView(out, scale0, seed)


# ------------------------------------------------------------ 3D scene input
# Table I packing: Group 1 = mean and opacity (one 16-byte texel), Group 2 =
# the six entries of the symmetric 3D covariance (two texels).
GAUSSIAN3D = np.dtype([("x", "<f4"), ("y", "<f4"), ("z", "<f4"), ("opacity", "<f4")])
COV3D = np.dtype([("xx", "<f4"), ("xy", "<f4"), ("xz", "<f4"), ("yy", "<f4"), ("yz", "<f4"),
                  ("zz", "<f4"), ("pad0", "<f4"), ("pad1", "<f4")])
# World-to-camera block of a pinhole camera: p_cam = rot @ p + trans.
CAMERA = np.dtype([("rot", "<f4", (9,)), ("trans", "<f4", (3,)), ("fx", "<f4"), ("fy", "<f4"),
                   ("cx", "<f4"), ("cy", "<f4"), ("near_z", "<f4"), ("width", "<u4"),
                   ("height", "<u4")])
assert GAUSSIAN3D.itemsize == 16 and COV3D.itemsize == 32 and CAMERA.itemsize == 76


@dataclasses.dataclass
class Scene3D:
    """Unprojected Gaussians and the cameras that see them."""

    gaussians: np.ndarray  # GAUSSIAN3D
    cov: np.ndarray        # COV3D
    cameras: np.ndarray    # CAMERA, one per view
    seed: int
    rgb: np.ndarray = None  # (n, 3) float32 colours in [0, 1) (Table IV, Group 3)

    @property
    def n(self) -> int:
        return int(self.gaussians.shape[0])


def camera(eye, target, width: int, height: int, fx: float = 1108.5, fy: float = 1108.5,
           near_z: float = 0.2) -> np.ndarray:
    """One CAMERA block looking from ``eye`` at ``target`` with up = +y:
    camera axes right, down, forward (rows of rot), principal point at the
    image centre."""
    eye = np.asarray(eye, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    if np.linalg.norm(right) < 1e-6:
        right = np.array([1.0, 0.0, 0.0])
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    rot = np.stack([right, down, fwd])
    c = np.zeros((), dtype=CAMERA)
    c["rot"] = rot.reshape(9).astype(np.float32)
    c["trans"] = (-(rot @ eye)).astype(np.float32)
    c["fx"], c["fy"] = fx, fy
    c["cx"], c["cy"] = width / 2.0, height / 2.0
    c["near_z"] = near_z
    c["width"], c["height"] = width, height
    return c


def scene3d(seed: int = 0, n: int = 500_000, views: int = 64, width: int = 1280, height: int = 720,
            scale0: float = 0.03, cam_radius: float = 15.0) -> Scene3D:
    """Means ~ U[0,1)^3 * 10 - 5 (the multiview scene's distribution);
    per-axis scales s0 * lognormal(0, 0.5); rotations uniform (normalised
    Gaussian quaternions); cov = Rq diag(s^2) Rq^T in float64, rounded to
    float32; opacity ~ U[0.05, 1); colours ~ U[0, 1)^3 (drawn last).
    Cameras: Fibonacci lattice of a sphere
    of radius ``cam_radius`` looking at the origin plus a jitter uniform in
    a ball of radius 4, fx = fy = 1108.5, near plane 0.2."""
    rng = np.random.default_rng(seed)
    mean3 = rng.random((n, 3)) * 10.0 - 5.0
    scales = scale0 * np.exp(rng.normal(0.0, 0.5, size=(n, 3)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    rq = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1),
    ], 1)  # (n, 3, 3)
    s3 = np.einsum("nij,nj,nkj->nik", rq, scales * scales, rq)
    g = np.empty(n, dtype=GAUSSIAN3D)
    g["x"], g["y"], g["z"] = (mean3[:, k].astype(np.float32) for k in range(3))
    g["opacity"] = rng.uniform(0.05, 1.0, size=n).astype(np.float32)
    cov = np.zeros(n, dtype=COV3D)
    for name, (i, j) in (("xx", (0, 0)), ("xy", (0, 1)), ("xz", (0, 2)), ("yy", (1, 1)),
                         ("yz", (1, 2)), ("zz", (2, 2))):
        cov[name] = s3[:, i, j].astype(np.float32)
    eye = _fibonacci_sphere(views) * cam_radius
    u = rng.normal(size=(views, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    jitter = u * (4.0 * rng.random(views) ** (1.0 / 3.0))[:, None]
    cams = np.stack([camera(eye[v], jitter[v], width, height) for v in range(views)])
    rgb = rng.random((n, 3)).astype(np.float32)
    return Scene3D(g, cov, cams, seed, rgb)


# ------------------------------------------------------------ request trace
RESOLUTIONS = ((640, 360), (1280, 720), (1920, 1080))


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    n: int
    width: int
    height: int
    seed: int

    def frame(self) -> Frame:
        """Frame of this request, drawn like the scene-scale frame."""
        return frame_scene(self.seed, self.n, self.width, self.height)

    def window(self, base_n: int) -> int:
        """First Gaussian of this request's window in a request pool base
        frame of base_n Gaussians (drawn from the request's seed)."""
        return int(np.random.default_rng(self.seed).integers(0, base_n))


def request_pool(base_n: int = 3_000_000, base_seed: int = 500) -> dict:
    """Gaussians for a long request stream without generating every frame:
    per resolution, a base frame drawn like the scene-scale frame
    (base_seed + resolution index), shuffled, and stored twice in a row, so
    that a request of n <= base_n Gaussians is the contiguous slice
    [w, w + n) at its window offset w -- a random subset with the scene
    frame's distribution.  Returns {(width, height): records (2 * base_n)}."""
    out = {}
    for k, (w, h) in enumerate(RESOLUTIONS):
        fr = frame_scene(base_seed + k, base_n, w, h)
        g = fr.gaussians[np.random.default_rng(base_seed + 10 + k).permutation(base_n)]
        out[(w, h)] = np.concatenate([g, g])
    return out


def request_trace(seed: int = 0, count: int = 2000, rate_hz: float = 200.0,
                  n_lo: int = 100_000, n_hi: int = 3_000_000) -> list[Request]:
    """Poisson arrivals at ``rate_hz``; N log-uniform in [n_lo, n_hi];
    resolution uniform over 640x360, 1280x720, 1920x1080; per-request
    seed 1000 + id."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps) - gaps[0]
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count)).astype(np.int64)
    res = rng.integers(0, len(RESOLUTIONS), size=count)
    return [Request(i, float(t[i]), int(ns[i]), *RESOLUTIONS[int(res[i])], 1000 + i)
            for i in range(count)]


CONFIGS = {
    "small": frame_small,
    "scene": frame_scene,
    "large": frame_large,
}
