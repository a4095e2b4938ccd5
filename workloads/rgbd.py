"""Synthetic RGB-D reconstruction stream of voxel-block keys.

A camera moves along +y through a corridor: a ground plane (z = 0), two walls
(x = +-width/2) and spheres standing on the ground every few metres.  Each
frame samples `per_frame` surface points in the band the camera sees
(y in [cam_y + near, cam_y + near + depth]), area-weighted across the visible
surfaces.  It perturbs each point along its viewing ray with depth-dependent
Gaussian noise (sigma = sigma0 + sigma1 * d^2, the usual shape of
structured-light depth noise), converts it to an 8 mm voxel and then to the
8^3-voxel block holding it, and packs the block coordinates as three signed
21-bit fields: key = (x & M) | (y & M) << 21 | (z & M) << 42, M = 2^21 - 1.

Every random number comes from the counter-based splitmix64 streams, so a
frame's candidates are a pure function of (params, frame).  Nothing here
implements hash-container behaviour.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import splitmix as sm

M21 = (1 << 21) - 1


@dataclass(frozen=True)
class RGBDParams:
    frames: int = 300
    per_frame: int = 400_000
    voxel: float = 0.008          # m
    block_voxels: int = 8         # block edge in voxels (64 mm)
    width: float = 34.0           # corridor width (m): ~9.96M blocks, ~88 % present over 300 frames
    wall_height: float = 5.0      # m
    speed: float = 0.8            # camera advance per frame (m)
    near: float = 0.5             # m
    depth: float = 12.0           # visible band along y (m)
    cam_height: float = 1.6       # m
    sway: float = 3.0             # lateral camera sway amplitude (m)
    sigma0: float = 0.01          # depth noise at zero range (m)
    sigma1: float = 0.0003        # depth noise growth (1/m)
    sphere_every: float = 5.0     # one sphere per this many metres of corridor
    seed: int = 0

    @property
    def block(self) -> float:
        return self.voxel * self.block_voxels


def pack(bx: np.ndarray, by: np.ndarray, bz: np.ndarray) -> np.ndarray:
    """Three signed 21-bit block coordinates -> int64 key (bit 63 is 0)."""
    m = np.int64(M21)
    return ((bx.astype(np.int64) & m) | ((by.astype(np.int64) & m) << 21) | ((bz.astype(np.int64) & m) << 42))


def unpack(keys: np.ndarray):
    k = np.asarray(keys, dtype=np.int64)
    out = []
    for sh in (0, 21, 42):
        c = (k >> sh) & M21
        out.append(np.where(c >= 1 << 20, c - (1 << 21), c))
    return out


def _spheres(p: RGBDParams):
    """Sphere centres and radii along the corridor (deterministic)."""
    n = int((p.frames * p.speed + p.near + p.depth) / p.sphere_every) + 2
    u = sm.uniform01(2500, p.seed, 0, 3 * n).reshape(3, n)
    r = 0.6 + 1.6 * u[0]
    cx = (u[1] - 0.5) * (p.width - 2 * r - 1.0)
    cy = (np.arange(n) + 0.5) * p.sphere_every + (u[2] - 0.5) * p.sphere_every * 0.5
    return np.stack([cx, cy, r], axis=1)


def camera(p: RGBDParams, f: int) -> np.ndarray:
    y = f * p.speed
    x = p.sway * np.sin(2 * np.pi * f / 60.0)
    return np.array([x, y, p.cam_height])


def frame_points(p: RGBDParams, f: int) -> np.ndarray:
    """Noisy surface points seen in frame f, shape (per_frame, 3)."""
    n = p.per_frame
    cam = camera(p, f)
    y0 = cam[1] + p.near
    y1 = y0 + p.depth
    sph = _spheres(p)
    vis = sph[(sph[:, 1] > y0 - sph[:, 2]) & (sph[:, 1] < y1 + sph[:, 2])]
    areas = np.concatenate([[p.width * p.depth, p.wall_height * p.depth, p.wall_height * p.depth],
                            4 * np.pi * vis[:, 2] ** 2])
    cum = np.cumsum(areas) / areas.sum()
    u = sm.uniform01(2000 + f, p.seed, 0, 6 * n).reshape(6, n)
    surf = np.searchsorted(cum, u[0], side="right")
    pts = np.empty((n, 3))
    # ground
    g = surf == 0
    pts[g, 0] = (u[1, g] - 0.5) * p.width
    pts[g, 1] = y0 + u[2, g] * p.depth
    pts[g, 2] = 0.0
    # walls
    for s, x in ((1, -p.width / 2), (2, p.width / 2)):
        w = surf == s
        pts[w, 0] = x
        pts[w, 1] = y0 + u[1, w] * p.depth
        pts[w, 2] = u[2, w] * p.wall_height
    # spheres: uniform on the sphere (z = cos theta uniform)
    sp = surf >= 3
    idx = surf[sp] - 3
    c = vis[idx]
    cz = 2 * u[1, sp] - 1
    phi = 2 * np.pi * u[2, sp]
    rxy = np.sqrt(np.maximum(0.0, 1 - cz * cz))
    pts[sp, 0] = c[:, 0] + c[:, 2] * rxy * np.cos(phi)
    pts[sp, 1] = c[:, 1] + c[:, 2] * rxy * np.sin(phi)
    pts[sp, 2] = c[:, 2] + c[:, 2] * cz          # resting on the ground
    # noise along the viewing ray (Box-Muller from two uniforms)
    d = pts - cam
    dist = np.linalg.norm(d, axis=1)
    gauss = np.sqrt(-2 * np.log(np.maximum(u[3], 1e-300))) * np.cos(2 * np.pi * u[4])
    sigma = p.sigma0 + p.sigma1 * dist * dist
    pts += d / dist[:, None] * (gauss * sigma)[:, None]
    return pts


def frame_keys(p: RGBDParams, f: int) -> np.ndarray:
    """Packed int64 block keys of the frame's candidates (with duplicates)."""
    b = np.floor(frame_points(p, f) / p.block).astype(np.int64)
    return pack(b[:, 0], b[:, 1], b[:, 2])


def all_frame_keys(p: RGBDParams, workers: int = 8) -> list[np.ndarray]:
    """frame_keys for every frame, computed by a process pool started with
    spawn (safe in a process that already holds a CUDA context)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(frame_keys, [p] * p.frames, range(p.frames), chunksize=4))


def values_of(keys: np.ndarray) -> np.ndarray:
    """Mapped value: hash(key) mod 2^31 as int32 (splitmix64 of the key)."""
    return (sm.value_of(np.asarray(keys, dtype=np.int64).view(np.uint64)) % np.uint64(1 << 31)).astype(np.int32)


def calibrate(p: RGBDParams, frames: int | None = None) -> dict:
    """Present fraction of the candidates and the final distinct block count,
    from a dense occupancy grid over the corridor's block range."""
    frames = p.frames if frames is None else frames
    b = p.block
    xlo = int(np.floor(-p.width / 2 / b)) - 8
    ylo = -8
    zlo = -8
    nx = int(np.ceil(p.width / b)) + 16
    ny = int(np.ceil((frames * p.speed + p.near + p.depth + 3) / b)) + 16
    nz = int(np.ceil((p.wall_height + 4.5) / b)) + 16
    seen = np.zeros((nx, ny, nz), dtype=bool)
    present = []
    for f in range(frames):
        bb = np.floor(frame_points(p, f) / b).astype(np.int64)
        ix, iy, iz = bb[:, 0] - xlo, bb[:, 1] - ylo, bb[:, 2] - zlo
        ok = (ix >= 0) & (ix < nx) & (iy >= 0) & (iy < ny) & (iz >= 0) & (iz < nz)
        ix, iy, iz = ix[ok], iy[ok], iz[ok]
        present.append(seen[ix, iy, iz].mean())
        seen[ix, iy, iz] = True
    return {"present_mean": float(np.mean(present[1:])) if frames > 1 else 0.0,
            "present_last": float(present[-1]), "blocks": int(seen.sum())}
