"""Seeded scene, camera and flag generators (input synthesis only).

Every array is produced by ``numpy.random.default_rng(seed)``; the same seed always
gives the same bytes.  The scenes stand in for the indoor RGBD workloads of the
paper's evaluation (rooms of tens of square metres scanned at 640x480 to
1200x680, Section 4 and the supplementary dataset details): flattened Gaussians
lying on walls, floors, ceilings and boxes, 85-90% opaque (alpha 0.99) and the
rest nearly transparent (Section 3.1 fixes the opaque/transparent split).

Conventions shared with the rasterizer (Section 3.1, the ray definition):
  * quaternions are (w, x, y, z);
  * a camera pose is camera-to-world: ``p_world = R @ p_cam + t``; camera axes are
    x right, y down, z forward; pixel (x, y) has its centre at integer coordinates.
"""

from __future__ import annotations

import dataclasses
import math
from typing import Iterator, List, Optional, Sequence, Tuple

import numpy as np

F32 = np.float32


@dataclasses.dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    R: np.ndarray  # [3,3] float32, camera-to-world rotation (columns: right, down, forward)
    t: np.ndarray  # [3] float32, camera centre in world coordinates

    def copy(self) -> "Camera":
        return dataclasses.replace(self, R=self.R.copy(), t=self.t.copy())


@dataclasses.dataclass
class Scene:
    means: np.ndarray  # [N,3] float32
    scales: np.ndarray  # [N,3] float32, linear metres
    quats: np.ndarray  # [N,4] float32, (w,x,y,z), not necessarily unit
    opacity: np.ndarray  # [N] float32
    colors: np.ndarray  # [N,C] float32
    unstable: np.ndarray  # [N] uint8 (1 = unstable)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def channels(self) -> int:
        return int(self.colors.shape[1])

    def subset(self, idx: np.ndarray) -> "Scene":
        return Scene(*(np.ascontiguousarray(a[idx]) for a in
                       (self.means, self.scales, self.quats, self.opacity, self.colors, self.unstable)))

    def copy(self) -> "Scene":
        return self.subset(np.arange(self.n))


# ----------------------------------------------------------------------------- helpers

def _shoemake_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed unit quaternions (Shoemake, Graphics Gems III)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([b * np.cos(2 * np.pi * u3),           # w
                  a * np.sin(2 * np.pi * u2),           # x
                  a * np.cos(2 * np.pi * u2),           # y
                  b * np.sin(2 * np.pi * u3)], axis=1)  # z
    return q


def _matrix_to_quat(M: np.ndarray) -> np.ndarray:
    """Rotation matrices [...,3,3] -> unit quaternions [...,4] (w,x,y,z), Shepperd's method."""
    M = np.asarray(M, dtype=np.float64)
    m00, m11, m22 = M[..., 0, 0], M[..., 1, 1], M[..., 2, 2]
    tr = m00 + m11 + m22
    cand = np.stack([tr, m00, m11, m22], axis=-1)
    k = np.argmax(cand, axis=-1)
    q = np.zeros(M.shape[:-2] + (4,))
    # case w largest
    s = np.sqrt(np.maximum(1.0 + tr, 1e-300)) * 2
    qw = np.stack([0.25 * s, (M[..., 2, 1] - M[..., 1, 2]) / s,
                   (M[..., 0, 2] - M[..., 2, 0]) / s, (M[..., 1, 0] - M[..., 0, 1]) / s], -1)
    s = np.sqrt(np.maximum(1.0 + m00 - m11 - m22, 1e-300)) * 2
    qx = np.stack([(M[..., 2, 1] - M[..., 1, 2]) / s, 0.25 * s,
                   (M[..., 0, 1] + M[..., 1, 0]) / s, (M[..., 0, 2] + M[..., 2, 0]) / s], -1)
    s = np.sqrt(np.maximum(1.0 - m00 + m11 - m22, 1e-300)) * 2
    qy = np.stack([(M[..., 0, 2] - M[..., 2, 0]) / s, (M[..., 0, 1] + M[..., 1, 0]) / s,
                   0.25 * s, (M[..., 1, 2] + M[..., 2, 1]) / s], -1)
    s = np.sqrt(np.maximum(1.0 - m00 - m11 + m22, 1e-300)) * 2
    qz = np.stack([(M[..., 1, 0] - M[..., 0, 1]) / s, (M[..., 0, 2] + M[..., 2, 0]) / s,
                   (M[..., 1, 2] + M[..., 2, 1]) / s, 0.25 * s], -1)
    for case, val in enumerate((qw, qx, qy, qz)):
        sel = k == case
        q[sel] = val[sel]
    q /= np.linalg.norm(q, axis=-1, keepdims=True)
    return q


def _quat_mul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    aw, ax, ay, az = np.moveaxis(a, -1, 0)
    bw, bx, by, bz = np.moveaxis(b, -1, 0)
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], -1)


def _tangent_basis(n: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Two unit vectors spanning the plane orthogonal to unit vector ``n`` [3]."""
    helper = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u = np.cross(n, helper)
    u /= np.linalg.norm(u)
    v = np.cross(n, u)
    return u, v


def look_at_camera(position: Sequence[float], yaw: float, pitch: float, width: int, height: int,
                   f: float, cx: Optional[float] = None, cy: Optional[float] = None) -> Camera:
    """Pinhole camera at ``position`` (world z up) looking along (yaw, pitch), roll 0."""
    fwd = np.array([math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), math.sin(pitch)])
    right = np.array([math.sin(yaw), -math.cos(yaw), 0.0])
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=1)
    return Camera(fx=float(f), fy=float(f),
                  cx=float((width - 1) / 2 if cx is None else cx),
                  cy=float((height - 1) / 2 if cy is None else cy),
                  width=int(width), height=int(height),
                  R=R.astype(F32), t=np.asarray(position, dtype=F32))


def identity_camera(width: int, height: int, f: float, cx: float, cy: float) -> Camera:
    return Camera(fx=float(f), fy=float(f), cx=float(cx), cy=float(cy), width=int(width),
                  height=int(height), R=np.eye(3, dtype=F32), t=np.zeros(3, dtype=F32))


def disc_gaussian(center: Sequence[float], normal: Sequence[float], radius: float, thickness: float,
                  opacity: float, color: Sequence[float], twist: float = 0.0,
                  radius2: Optional[float] = None) -> Scene:
    """One flattened Gaussian ("surfel disc") whose smallest axis is along ``normal``."""
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    u, v = _tangent_basis(n)
    t1 = math.cos(twist) * u + math.sin(twist) * v
    t2 = np.cross(n, t1)
    R = np.stack([t1, t2, n], axis=1)
    q = _matrix_to_quat(R)
    r2 = radius if radius2 is None else radius2
    col = np.asarray(color, dtype=F32).reshape(1, -1)
    return Scene(means=np.asarray(center, dtype=F32).reshape(1, 3),
                 scales=np.array([[radius, r2, thickness]], dtype=F32),
                 quats=q.reshape(1, 4).astype(F32),
                 opacity=np.array([opacity], dtype=F32),
                 colors=col,
                 unstable=np.ones(1, dtype=np.uint8))


def concat_scenes(scenes: Sequence[Scene]) -> Scene:
    return Scene(*(np.ascontiguousarray(np.concatenate([getattr(s, k) for s in scenes], axis=0))
                   for k in ("means", "scales", "quats", "opacity", "colors", "unstable")))


# ----------------------------------------------------------------------------- configuration 1

def scatter_scene(seed: int, n: int = 2000) -> Tuple[Scene, Camera]:
    """Free-floating random ellipsoids in front of an identity camera.

    Means: x,y ~ U[-1,1] m, z ~ U[1.5,4] m; scales log-uniform in [0.01,0.1] m per
    axis; uniform random rotations; RGB ~ U[0,1]; the first half opaque (0.99) and
    the second half transparent (0.05), then shuffled.  Camera 160x120, f = 150,
    principal point (79.5, 59.5), identity pose.
    """
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(1.5, 4.0, n)], 1)
    scales = np.exp(rng.uniform(math.log(0.01), math.log(0.1), (n, 3)))
    quats = _shoemake_quats(rng, n)
    colors = rng.uniform(0, 1, (n, 3))
    opacity = np.where(np.arange(n) < n // 2, 0.99, 0.05)
    perm = rng.permutation(n)
    scene = Scene(means=means[perm].astype(F32), scales=scales[perm].astype(F32),
                  quats=quats[perm].astype(F32), opacity=opacity[perm].astype(F32),
                  colors=colors[perm].astype(F32), unstable=np.ones(n, dtype=np.uint8))
    cam = identity_camera(160, 120, 150.0, 79.5, 59.5)
    return scene, cam


def stack_scene(seed: int, n: int = 1600, size: int = 32, f: float = 60.0) -> Tuple[Scene, Camera]:
    """A deep stack of faint, wide ellipsoids on the optical axis of a small identity camera:
    the pixels near the centre composite hundreds of fragments before their transmission
    runs out, so the render tiles there hold lists of several hundred entries.

    Means: x, y ~ N(0, 0.04) m, z ~ U[1.5, 3] m; scales log-uniform in [0.08, 0.2] m per
    axis; uniform random rotations; opacity ~ U[0.015, 0.04]; RGB ~ U[0, 1]; every other
    Gaussian unstable.  Camera size x size, focal length f, centred principal point.
    """
    rng = np.random.default_rng(seed)
    means = np.stack([rng.normal(0, 0.04, n), rng.normal(0, 0.04, n), rng.uniform(1.5, 3.0, n)], 1)
    scales = np.exp(rng.uniform(math.log(0.08), math.log(0.2), (n, 3)))
    quats = _shoemake_quats(rng, n)
    scene = Scene(means=means.astype(F32), scales=scales.astype(F32), quats=quats.astype(F32),
                  opacity=rng.uniform(0.015, 0.04, n).astype(F32), colors=rng.uniform(0, 1, (n, 3)).astype(F32),
                  unstable=(np.arange(n) % 2 == 0).astype(np.uint8))
    c = 0.5 * (size - 1)
    return scene, identity_camera(size, size, f, c, c)


# ----------------------------------------------------------------------------- rooms

@dataclasses.dataclass
class Layout:
    size: Tuple[float, float, float]
    faces: List[Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]]  # (origin, edge a, edge b, normal)
    boxes: List[Tuple[np.ndarray, np.ndarray]]  # (min corner, max corner)


def _rect(o, a, b, n):
    return (np.asarray(o, float), np.asarray(a, float), np.asarray(b, float), np.asarray(n, float))


def _room_layout(rng: np.random.Generator, size=(6.0, 5.0, 3.0), grid=(1, 1), door=1.0,
                 n_boxes: int = 20) -> Layout:
    Lx, Ly, Lz = size
    faces = [
        _rect((0, 0, 0), (Lx, 0, 0), (0, Ly, 0), (0, 0, 1)),    # floor
        _rect((0, 0, Lz), (Lx, 0, 0), (0, Ly, 0), (0, 0, -1)),  # ceiling
        _rect((0, 0, 0), (Lx, 0, 0), (0, 0, Lz), (0, 1, 0)),
        _rect((0, Ly, 0), (Lx, 0, 0), (0, 0, Lz), (0, -1, 0)),
        _rect((0, 0, 0), (0, Ly, 0), (0, 0, Lz), (1, 0, 0)),
        _rect((Lx, 0, 0), (0, Ly, 0), (0, 0, Lz), (-1, 0, 0)),
    ]
    gx, gy = grid
    # interior walls (two-sided) with one door gap per room-to-room segment
    for k in range(1, gx):
        x = Lx * k / gx
        for j in range(gy):
            y0, y1 = Ly * j / gy, Ly * (j + 1) / gy
            mid = 0.5 * (y0 + y1)
            for (s0, s1) in ((y0, mid - door / 2), (mid + door / 2, y1)):
                for sgn in (1, -1):
                    faces.append(_rect((x, s0, 0), (0, s1 - s0, 0), (0, 0, Lz), (sgn, 0, 0)))
    for k in range(1, gy):
        y = Ly * k / gy
        for i in range(gx):
            x0, x1 = Lx * i / gx, Lx * (i + 1) / gx
            mid = 0.5 * (x0 + x1)
            for (s0, s1) in ((x0, mid - door / 2), (mid + door / 2, x1)):
                for sgn in (1, -1):
                    faces.append(_rect((s0, y, 0), (s1 - s0, 0, 0), (0, 0, Lz), (0, sgn, 0)))
    boxes = []
    for _ in range(n_boxes):
        e = rng.uniform(0.2, 1.2, 3)
        lo = np.array([rng.uniform(0, Lx - e[0]), rng.uniform(0, Ly - e[1]), 0.0])
        hi = lo + e
        boxes.append((lo, hi))
        ex, ey, ez = e
        faces += [
            _rect((lo[0], lo[1], hi[2]), (ex, 0, 0), (0, ey, 0), (0, 0, 1)),   # top
            _rect((lo[0], lo[1], 0), (0, ey, 0), (0, 0, ez), (-1, 0, 0)),
            _rect((hi[0], lo[1], 0), (0, ey, 0), (0, 0, ez), (1, 0, 0)),
            _rect((lo[0], lo[1], 0), (ex, 0, 0), (0, 0, ez), (0, -1, 0)),
            _rect((lo[0], hi[1], 0), (ex, 0, 0), (0, 0, ez), (0, 1, 0)),
        ]
    return Layout(size=(Lx, Ly, Lz), faces=faces, boxes=boxes)


def _gaussians_on_faces(rng: np.random.Generator, layout: Layout, n: int, opaque_frac: float,
                        channels: int) -> Scene:
    faces = layout.faces
    areas = np.array([np.linalg.norm(a) * np.linalg.norm(b) for (_, a, b, _) in faces])
    face_id = rng.choice(len(faces), size=n, p=areas / areas.sum())
    uv = rng.random((n, 2))
    O = np.stack([f[0] for f in faces])[face_id]
    A = np.stack([f[1] for f in faces])[face_id]
    B = np.stack([f[2] for f in faces])[face_id]
    Nrm = np.stack([f[3] for f in faces])[face_id]
    pos = O + uv[:, :1] * A + uv[:, 1:] * B
    # rotation: third axis along the face normal, random twist in the plane
    tb = [_tangent_basis(f[3]) for f in faces]
    U = np.stack([t[0] for t in tb])[face_id]
    V = np.stack([t[1] for t in tb])[face_id]
    tw = rng.uniform(0, 2 * np.pi, n)[:, None]
    T1 = np.cos(tw) * U + np.sin(tw) * V
    T2 = np.cross(Nrm, T1)
    Rm = np.stack([T1, T2, Nrm], axis=2)
    quats = _matrix_to_quat(Rm)
    s_in = np.exp(rng.uniform(math.log(0.005), math.log(0.030), (n, 2)))
    scales = np.concatenate([s_in, np.full((n, 1), 0.001)], axis=1)
    opaque = rng.random(n) < opaque_frac
    opacity = np.where(opaque, 0.99, 0.05)
    base = rng.uniform(0.2, 0.8, (len(faces), channels))
    omega = rng.normal(0, 2 * np.pi, (len(faces), channels, 3))
    phase = rng.uniform(0, 2 * np.pi, (len(faces), channels))
    smooth = base[face_id] + 0.1 * np.sin(np.einsum("nck,nk->nc", omega[face_id], pos) + phase[face_id])
    residual = rng.normal(0, 0.1, (n, channels))
    colors = np.where(opaque[:, None], smooth, residual)
    # transparent Gaussians float 2 mm off the surface, on the room side
    pos = np.where(opaque[:, None], pos, pos + 0.002 * Nrm)
    return Scene(means=pos.astype(F32), scales=scales.astype(F32), quats=quats.astype(F32),
                 opacity=opacity.astype(F32), colors=colors.astype(F32),
                 unstable=np.ones(n, dtype=np.uint8))


def room_scene(seed: int, n: int, channels: int = 3, opaque_frac: float = 0.85,
               size=(6.0, 5.0, 3.0), grid=(1, 1), n_boxes: int = 20) -> Tuple[Scene, Layout]:
    """Box room (floor, ceiling, inward walls) plus random axis-aligned boxes on the floor.

    ``n`` flattened Gaussians are placed area-uniformly on the visible faces:
    in-plane scales log-uniform in [5,30] mm, normal scale 1 mm, third axis along the
    face normal with a random in-plane twist.  ``opaque_frac`` of them are opaque
    (0.99) with a smooth per-face colour, the rest transparent (0.05) with residual
    colours ~ N(0, 0.1), offset 2 mm off the surface.
    """
    rng = np.random.default_rng(seed)
    layout = _room_layout(rng, size=size, grid=grid, n_boxes=n_boxes)
    return _gaussians_on_faces(rng, layout, n, opaque_frac, channels), layout


def multiroom_scene(seed: int, n: int, channels: int = 3, opaque_frac: float = 0.85,
                    size=(12.0, 10.0, 3.0), grid=(2, 2), n_boxes: int = 40) -> Tuple[Scene, Layout]:
    """A grid of rooms with two-sided interior walls and 1 m door gaps."""
    return room_scene(seed, n, channels=channels, opaque_frac=opaque_frac, size=size, grid=grid,
                      n_boxes=n_boxes)


def room_camera_candidates(seed: int, layout: Layout, width: int = 640, height: int = 480,
                           f: float = 600.0) -> Iterator[Camera]:
    """Endless seeded stream of poses inside the layout (shrunk by 0.5 m), outside boxes.

    yaw ~ U[0, 2pi), pitch ~ U[-20, 20] degrees, roll 0.
    """
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz = layout.size
    while True:
        pos = np.array([rng.uniform(0.5, Lx - 0.5), rng.uniform(0.5, Ly - 0.5), rng.uniform(0.5, Lz - 0.5)])
        yaw = rng.uniform(0, 2 * np.pi)
        pitch = math.radians(rng.uniform(-20, 20))
        inside = any(np.all(pos > lo - 0.2) and np.all(pos < hi + 0.2) for lo, hi in layout.boxes)
        if inside:
            continue
        yield look_at_camera(pos, yaw, pitch, width, height, f)


def flag_blobs(scene: Scene, cameras: Sequence[Camera], n_unstable: int, n_blobs: int,
               seed: int, n_in_view: Optional[int] = None) -> np.ndarray:
    """Flag the ``n_unstable`` Gaussians nearest to ``n_blobs`` centres.

    The first ``n_in_view`` centres (default: all) are the positions of random Gaussians
    that lie in front of one of the cameras inside its field of view (a plain pinhole
    containment test used only to choose inputs); the others are random Gaussians
    anywhere in the scene.
    """
    rng = np.random.default_rng(seed)
    p = scene.means.astype(np.float64)
    cand = np.zeros(scene.n, dtype=bool)
    for cam in cameras:
        pc = (p - cam.t.astype(np.float64)) @ cam.R.astype(np.float64)
        z = pc[:, 2]
        ok = z > 0.5
        with np.errstate(divide="ignore", invalid="ignore"):
            ok &= np.abs(pc[:, 0] / z) < 0.45 * cam.width / cam.fx
            ok &= np.abs(pc[:, 1] / z) < 0.45 * cam.height / cam.fy
        cand |= ok
    pool = np.flatnonzero(cand)
    if pool.size == 0:
        pool = np.arange(scene.n)
    k_view = n_blobs if n_in_view is None else min(n_in_view, n_blobs)
    picks = list(rng.choice(pool, size=k_view, replace=False))
    if n_blobs > k_view:
        picks += list(rng.choice(scene.n, size=n_blobs - k_view, replace=False))
    centers = p[np.array(picks)].astype(np.float32)
    p32 = scene.means.astype(np.float32)
    dist = np.min(np.stack([np.linalg.norm(p32 - c, axis=1) for c in centers], 1), axis=1)
    flags = np.zeros(scene.n, dtype=np.uint8)
    flags[np.argpartition(dist, n_unstable - 1)[:n_unstable]] = 1
    return flags


def sh_coefficients(seed: int, n: int, degree: int, dc_range=(1.0, 3.5), rest_sigma: float = 0.15) -> np.ndarray:
    """Random SH colour coefficients [n, (degree+1)^2, 3] float32: the degree-0 term uniform in
    dc_range (a colour of about 0.28 to 1 after the basis constant), the others N(0, rest_sigma)."""
    rng = np.random.default_rng(seed)
    K = (degree + 1) ** 2
    c = rng.normal(0.0, rest_sigma, (n, K, 3))
    c[:, 0, :] = rng.uniform(dc_range[0], dc_range[1], (n, 3))
    return c.astype(F32)


def jitter_scene(scene: Scene, seed: int, pos_sigma: float = 0.003, log_scale_sigma: float = 0.05,
                 rot_deg: float = 2.0, color_sigma: float = 0.03) -> Scene:
    """Perturbed copy used to render a fixed target image for the L1 losses."""
    rng = np.random.default_rng(seed)
    n = scene.n
    means = scene.means + rng.normal(0, pos_sigma, (n, 3))
    scales = scene.scales * np.exp(rng.normal(0, log_scale_sigma, (n, 3)))
    axis = rng.normal(0, 1, (n, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    half = math.radians(rot_deg) / 2
    dq = np.concatenate([np.full((n, 1), math.cos(half)), math.sin(half) * axis], axis=1)
    quats = _quat_mul(dq, scene.quats.astype(np.float64))
    colors = scene.colors + rng.normal(0, color_sigma, scene.colors.shape)
    return Scene(means=means.astype(F32), scales=scales.astype(F32), quats=quats.astype(F32),
                 opacity=scene.opacity.copy(), colors=colors.astype(F32), unstable=scene.unstable.copy())


def random_masks(seed: int, frames: int, height: int, width: int, lo: float, hi: float) -> np.ndarray:
    """Blob-shaped pixel masks with per-frame coverage drawn in [lo, hi] (for ABI tests)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:height, 0:width]
    out = np.zeros((frames, height, width), dtype=np.uint8)
    for f in range(frames):
        target = rng.uniform(lo, hi)
        m = np.zeros((height, width), dtype=bool)
        while m.mean() < target:
            cx, cy = rng.uniform(0, width), rng.uniform(0, height)
            r = rng.uniform(0.05, 0.2) * min(width, height)
            m |= (xx - cx) ** 2 + (yy - cy) ** 2 < r * r
        out[f] = m
    return out
