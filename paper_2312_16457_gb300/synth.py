"""Seeded synthetic inputs for the block renderer: baked blocks, cameras, rays
and deferred-MLP weights.

This module holds no step of the rendering method.  It only produces the
arrays that the renderer and its FP64 oracle both consume, so the two sides
always read identical inputs:

* a world density field made of Gaussian blobs plus a dense ground slab,
  stored per block as pre-activation log-density (channel 0);
* smooth diffuse / specular pre-activation fields with per-vertex noise
  (channels 1-7) in the 3D grid, and uniform noise of amplitude 0.1 in the
  three planes (the "features summed" layout of a MERF-style block);
* ground-plane block partitions with 2x2-merged coarser LOD levels, every
  level sampling the same world field at its own vertices;
* pinhole cameras (aerial, oblique) and random ray batches;
* deferred-MLP weights drawn from N(0, 0.3^2), globally or per block.

Scalar parameters come from numpy's PCG64 generator; per-element noise comes
from a counter-based integer hash evaluated with int64 tensor arithmetic that
never overflows, so CPU and GPU produce the same noise.  The arrays are
float32 ("FP32 master"), in the layouts the C ABI documents: grid
[z][y][x][8], planes [v][u][8] for the xy, xz and yz planes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

NCH = 8
MLP_NPARAM = 499
# unbounded boundary blocks: the xy sides that extend to infinity, and the flag
EXT_XLO, EXT_XHI, EXT_YLO, EXT_YHI, CONTRACTED = 1, 2, 4, 8, 16
_MASK32 = 0xFFFFFFFF


# --------------------------------------------------------------------------
# data containers


@dataclass
class Block:
    """One baked block: world AABB, resolutions, LOD links and FP32 arrays."""

    lo: tuple
    hi: tuple
    R: int
    P: int
    level: int = 1
    parent: int = -1
    grid: Optional[torch.Tensor] = None  # [R, R, R, 8] float32, [z][y][x][c]
    planes: List[torch.Tensor] = field(default_factory=list)  # 3 x [P, P, 8]
    unbounded: int = 0  # 0, or CONTRACTED | the xy sides (EXT_*) that extend to infinity

    def to(self, device) -> "Block":
        return Block(self.lo, self.hi, self.R, self.P, self.level, self.parent,
                     self.grid.to(device), [p.to(device) for p in self.planes], self.unbounded)


@dataclass
class Camera:
    c2w: np.ndarray  # (3, 4) float64, OpenGL axes (camera looks along -z)
    width: int
    height: int
    fov_y_deg: float

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


@dataclass
class Scene:
    blocks: List[Block]
    box_lo: tuple
    box_hi: tuple
    lod_thresh: List[float] = field(default_factory=list)  # per level, 1 = finest
    occ_cell: int = 4
    occ_thresh: float = 0.01

    @property
    def n_levels(self) -> int:
        return max(b.level for b in self.blocks)

    def ids_at_level(self, level: int) -> List[int]:
        return [i for i, b in enumerate(self.blocks) if b.level == level]

    def nbytes_master(self) -> int:
        return sum(b.grid.numel() * 4 + sum(p.numel() * 4 for p in b.planes) for b in self.blocks)


# --------------------------------------------------------------------------
# counter-based noise


def _hash32(x: torch.Tensor) -> torch.Tensor:
    """Integer avalanche hash on values in [0, 2^32); int64 arithmetic whose
    products stay below 2^63."""
    x = x ^ (x >> 16)
    x = (x * 0x45D9F3B) & _MASK32
    x = x ^ (x >> 16)
    x = (x * 0x45D9F3B) & _MASK32
    x = x ^ (x >> 16)
    return x


def _salt(*keys: int) -> int:
    h = 0x9E3779B9
    for k in keys:
        v = torch.tensor([(h ^ (k & _MASK32)) & _MASK32], dtype=torch.int64)
        h = int(_hash32(v)[0])
    return h


def uniform_noise(n: int, lo: float, hi: float, *keys: int, device="cpu") -> torch.Tensor:
    """n float32 values uniform on [lo, hi), a pure function of (keys, index)."""
    s = _salt(*keys)
    idx = torch.arange(n, dtype=torch.int64, device=device)
    h = _hash32((idx ^ s) & _MASK32)
    h = _hash32((h + (s >> 7)) & _MASK32)
    u = h.to(torch.float64) * (1.0 / 4294967296.0)
    return (lo + (hi - lo) * u).to(torch.float32)


# --------------------------------------------------------------------------
# world field


@dataclass
class WorldField:
    centers: np.ndarray  # (n, 3)
    radii: np.ndarray  # (n,)
    peak: float
    slab_top: float
    slab_sigma: float
    omega: np.ndarray  # (7, 3) spatial frequencies of channels 1-7
    phase: np.ndarray  # (7,)
    amp: float
    grid_noise: float
    plane_noise: float
    seed: int

    def log_density(self, x, y, z):
        """ln(max(sigma, 1e-4)) at world points (float64 tensors, same shape)."""
        sig = torch.zeros_like(x)
        # blobs within 5 radii of the sampled region
        lo = np.array([float(x.min()), float(y.min()), float(z.min())])
        hi = np.array([float(x.max()), float(y.max()), float(z.max())])
        for c, r in zip(self.centers, self.radii):
            if np.any(c < lo - 5 * r) or np.any(c > hi + 5 * r):
                continue
            d2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
            sig = sig + self.peak * torch.exp(-d2 / (2.0 * r * r))
        sig = torch.where(z < self.slab_top, sig + self.slab_sigma, sig)
        return torch.log(torch.clamp(sig, min=1e-4))

    def smooth(self, ch: int, x, y, z):
        w = self.omega[ch - 1]
        return self.amp * torch.sin(w[0] * x + w[1] * y + w[2] * z + self.phase[ch - 1])


def make_field(seed: int, box_lo, box_hi, n_blobs: int, r_range, blob_lo=None, blob_hi=None,
               slab_frac=0.1, peak=20.0, slab_sigma=20.0) -> WorldField:
    rng = np.random.default_rng(seed)
    blo = np.asarray(blob_lo if blob_lo is not None else box_lo, dtype=np.float64)
    bhi = np.asarray(blob_hi if blob_hi is not None else box_hi, dtype=np.float64)
    centers = rng.uniform(blo, bhi, size=(n_blobs, 3))
    radii = rng.uniform(r_range[0], r_range[1], size=n_blobs)
    dirs = rng.normal(size=(7, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    omega = dirs * rng.uniform(2.0, 6.0, size=(7, 1))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=7)
    slab_top = box_lo[2] + slab_frac * (box_hi[2] - box_lo[2])
    return WorldField(centers, radii, peak, slab_top, slab_sigma, omega, phase, 1.5, 0.5, 0.1, seed)


def _axis(lo: float, hi: float, n: int, device) -> torch.Tensor:
    i = torch.arange(n, dtype=torch.float64, device=device)
    return lo + i * ((hi - lo) / (n - 1))


def _vertex_world(us, lo, hi):
    """World positions of the vertices of an unbounded block, whose grid spans
    contracted coordinates u in [-2, 2]^3: the point whose contraction is u
    (for u in the shell, |x| = 1 / (2 - ||u||_inf) on the coordinates that
    reach the norm and u_i times that on the others; ||u|| is capped at
    2 - 1e-3, i.e. 1000 half extents from the centre)."""
    uu = torch.stack(us, 0)
    m = uu.abs().amax(0).clamp(max=2.0 - 1e-3)
    big = 1.0 / (2.0 - m)
    x = torch.where(m <= 1.0, uu, torch.where(uu.abs() >= m, torch.sign(uu) * big, uu * big))
    return [0.5 * (lo[a] + hi[a]) + 0.5 * (hi[a] - lo[a]) * x[a] for a in range(3)]


def bake_block(fld: WorldField, lo, hi, R: int, P: int, key: int, level=1, parent=-1,
               device="cpu", unbounded=0) -> Block:
    """Sample the world field at the block's vertices (vertex 0 at lo, R-1 at
    hi; for an unbounded block vertex 0 at u = -2, R-1 at u = 2)."""
    lo = tuple(float(np.float32(v)) for v in lo)
    hi = tuple(float(np.float32(v)) for v in hi)
    if unbounded & CONTRACTED:
        us = torch.meshgrid(*(_axis(-2.0, 2.0, R, device),) * 3, indexing="ij")  # (z, y, x)
        xx, yy, zz = _vertex_world([us[2], us[1], us[0]], lo, hi)
    else:
        xs, ys, zs = (_axis(lo[a], hi[a], R, device) for a in range(3))
        zz, yy, xx = torch.meshgrid(zs, ys, xs, indexing="ij")
    grid = torch.empty((R, R, R, NCH), dtype=torch.float32, device=device)
    grid[..., 0] = fld.log_density(xx, yy, zz).to(torch.float32)
    n = R * R * R
    for ch in range(1, NCH):
        sm = fld.smooth(ch, xx, yy, zz).to(torch.float32)
        nz = uniform_noise(n, -fld.grid_noise, fld.grid_noise, fld.seed, key, 0, ch, device=device)
        grid[..., ch] = sm + nz.view(R, R, R)
    del zz, yy, xx
    planes = []
    for pl in range(3):
        nz = uniform_noise(P * P * NCH, -fld.plane_noise, fld.plane_noise, fld.seed, key, 1 + pl,
                           device=device)
        planes.append(nz.view(P, P, NCH).contiguous())
    return Block(lo, hi, R, P, level, parent, grid.contiguous(), planes, unbounded)


# --------------------------------------------------------------------------
# scenes


def single_block_scene(seed=1, R=64, P=256, device="cpu") -> Scene:
    """One block on [-1, 1]^3: 8 blobs (peak sigma 20, radius 0.1-0.3) with
    centres in [-0.7, 0.7]^3 and a ground slab z < -0.8."""
    fld = make_field(seed, (-1, -1, -1), (1, 1, 1), 8, (0.1, 0.3), (-0.7,) * 3, (0.7,) * 3)
    b = bake_block(fld, (-1, -1, -1), (1, 1, 1), R, P, key=0, device=device)
    return Scene([b], (-1, -1, -1), (1, 1, 1))


def city_scene(seed: int, M: int, side: float, res: Sequence[tuple], height=2.0,
               blobs_per_area=2.0, lod_thresh=None, device="cpu", levels=None, unbounded=False,
               blob_top=0.5, blob_r=(0.1, 0.3)) -> Scene:
    """M x M ground blocks of the given side at LOD 1, merged 2x2 per level.

    res[l] = (R, P) of level l+1.  Blob centres are uniform over the ground
    and the lowest blob_top of the height (half by default) so that they
    cross block borders; blob radii are blob_r times half a block side.
    unbounded=True (one level only) makes the blocks on the scene's boundary
    unbounded: contracted, extending to infinity across their boundary sides
    (the ground slab then continues to the horizon)."""
    L = len(res) if levels is None else levels
    assert not unbounded or L == 1
    half = 0.5 * M * side
    box_lo = (-half, -half, -0.5 * height)
    box_hi = (half, half, 0.5 * height)
    area = (2 * half) ** 2
    fld = make_field(seed, box_lo, box_hi, int(round(blobs_per_area * area)),
                     (blob_r[0] * side / 2, blob_r[1] * side / 2), (-half, -half, box_lo[2]),
                     (half, half, box_lo[2] + blob_top * height))
    blocks: List[Block] = []
    level_index = {}
    for lev in range(L, 0, -1):  # coarse first so parents have indices
        m = M // (2 ** (lev - 1))
        s = side * 2 ** (lev - 1)
        R, P = res[lev - 1]
        for j in range(m):
            for i in range(m):
                lo = (-half + i * s, -half + j * s, box_lo[2])
                hi = (-half + (i + 1) * s, -half + (j + 1) * s, box_hi[2])
                parent = level_index.get((lev + 1, i // 2, j // 2), -1)
                key = lev * 100000 + j * 1000 + i
                ext = 0
                if unbounded:
                    ext = (EXT_XLO if i == 0 else 0) | (EXT_XHI if i == m - 1 else 0) | \
                          (EXT_YLO if j == 0 else 0) | (EXT_YHI if j == m - 1 else 0)
                    ext = ext | CONTRACTED if ext else 0
                blocks.append(bake_block(fld, lo, hi, R, P, key, lev, parent, device, ext))
                level_index[(lev, i, j)] = len(blocks) - 1
    thr = list(lod_thresh) if lod_thresh is not None else [2.0 * side * 2 ** l for l in range(L)]
    return Scene(blocks, box_lo, box_hi, thr)


# --------------------------------------------------------------------------
# cameras, rays, MLP


def look_at(pos, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    pos = np.asarray(pos, np.float64)
    fwd = np.asarray(target, np.float64) - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    cup = np.cross(right, fwd)
    c2w = np.zeros((3, 4))
    c2w[:, 0] = right
    c2w[:, 1] = cup
    c2w[:, 2] = -fwd
    c2w[:, 3] = pos
    return c2w


def camera(pos, target, width, height, fov_y_deg=60.0) -> Camera:
    return Camera(look_at(pos, target), int(width), int(height), float(fov_y_deg))


def random_aerial_cameras(n: int, seed: int, half: float, altitude, sizes, fov=60.0) -> List[Camera]:
    """n aerial poses above a [-half, half]^2 ground looking down at 30-60 deg."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(n):
        w, h = sizes[int(rng.integers(len(sizes)))]
        alt = rng.uniform(*altitude)
        pitch = math.radians(rng.uniform(30.0, 60.0))
        yaw = rng.uniform(0.0, 2.0 * math.pi)
        tgt = np.array([rng.uniform(-0.6 * half, 0.6 * half), rng.uniform(-0.6 * half, 0.6 * half), -1.0])
        dist = (alt - tgt[2]) / math.tan(pitch)
        pos = tgt + np.array([-dist * math.cos(yaw), -dist * math.sin(yaw), alt - tgt[2]])
        cams.append(camera(pos, tgt, w, h, fov))
    return cams


def random_rays(n: int, seed: int, box_lo, box_hi, device="cpu"):
    """Origins on a sphere of radius 1.5 x the box diagonal around the box
    centre, aimed at uniform points inside the box; float32 (n, 3) each."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(box_lo, np.float64)
    hi = np.asarray(box_hi, np.float64)
    ctr = 0.5 * (lo + hi)
    rad = 1.5 * np.linalg.norm(hi - lo)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    o = ctr + rad * v
    tgt = rng.uniform(lo, hi, size=(n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return (torch.from_numpy(o.astype(np.float32)).to(device),
            torch.from_numpy(d.astype(np.float32)).to(device))


def mlp_weights(seed: int, std=0.3) -> np.ndarray:
    """499 deferred-MLP parameters ~ N(0, std^2): W1[10][16], b1[16], W2[16][16],
    b2[16], W3[16][3], b3[3], weights stored input-major."""
    return np.random.default_rng(seed).normal(0.0, std, size=MLP_NPARAM).astype(np.float32)


def block_mlp_nparam(n_freq: int) -> int:
    """Parameters of one per-block deferred MLP whose input is [C_d (3), F (4),
    d (3), sin / cos of d at n_freq octaves (6 n_freq)]: 16 n_in + 339."""
    return 16 * (10 + 6 * n_freq) + 16 + 256 + 16 + 48 + 3


def block_mlp_weights(seed: int, n_blocks: int, n_freq: int, std=0.3, spread=0.1) -> np.ndarray:
    """Per-block deferred-MLP parameters, [n_blocks, block_mlp_nparam(n_freq)]
    float32: one shared draw ~ N(0, std^2) plus an independent N(0, spread^2)
    perturbation per block, so neighbouring blocks' MLPs differ a little (the
    per-block models of the paper are trained separately on the same scene)."""
    rng = np.random.default_rng(seed)
    n = block_mlp_nparam(n_freq)
    base = rng.normal(0.0, std, size=n)
    return (base[None, :] + rng.normal(0.0, spread, size=(n_blocks, n))).astype(np.float32)


# --------------------------------------------------------------------------
# the five workloads (full sizes; tests pass smaller resolutions)


def workload_unbounded(R=64, P=256, device="cpu", width=160, height=90):
    """2x2 blocks of side 2, all on the scene's boundary and unbounded
    (contracted), one camera low inside the scene looking out at the horizon;
    scene seed 6, per-block MLP seed 106."""
    sc = city_scene(6, 2, 2.0, [(R, P)], device=device, unbounded=True)
    cam = camera((-0.3, -0.2, 0.4), (6.0, 3.5, -0.6), width, height, 70.0)
    return sc, [cam], mlp_weights(106)


def workload_single_block(R=64, P=256, device="cpu", width=128, height=128):
    """Single block [-1,1]^3, 64^3 grid + 256^2 planes, one 128x128 camera at
    (0, -2.5, 0.8) looking at the origin, fov 60 deg; scene seed 1, MLP seed 101."""
    sc = single_block_scene(1, R, P, device)
    cam = camera((0.0, -2.5, 0.8), (0.0, 0.0, 0.0), width, height, 60.0)
    return sc, [cam], mlp_weights(101)


def workload_city_4x4(R=256, P=1024, device="cpu", width=1280, height=720):
    """4x4 ground blocks of side 2 (scene 8 x 8 x 2), 256^3 grids + 1024^2
    planes; one oblique camera at altitude 6 (3x the scene height), 45 deg
    pitch, 40 deg vertical field of view framing the scene; scene seed 2,
    MLP seed 102."""
    sc = city_scene(2, 4, 2.0, [(R, P)], device=device)
    cam = camera((0.0, -6.5, 6.0), (0.0, 0.5, -1.0), width, height, 40.0)
    return sc, [cam], mlp_weights(102)


# A sparser city: blob centres in the lowest fifth of the height and radii of
# 0.05-0.15 half block sides (the dense default: lower half, 0.1-0.3), so the
# upper part of every block is empty air, as above a real city's ground.
SPARSE_CITY = dict(blob_top=0.2, blob_r=(0.05, 0.15))


def workload_city_lod(res=((256, 1024), (128, 512), (64, 256)), device="cpu", width=1920, height=1080,
                      lod_thresh=(12.5, 16.5, 0.0), sparse=False):
    """8x8 LOD-1 blocks of side 2 with 3 LOD levels (64 + 16 + 4 blocks),
    one 1920x1080 aerial camera (altitude 9, oblique) that sees every block;
    the thresholds keep the near blocks at level 1 and the far ones coarser.
    Scene seed 3, MLP seed 103; sparse=True: the SPARSE_CITY generator setting."""
    sc = city_scene(3, 8, 2.0, list(res), lod_thresh=list(lod_thresh), device=device,
                    **(SPARSE_CITY if sparse else {}))
    cam = camera((0.0, -13.0, 9.0), (0.0, -0.5, -1.0), width, height, 60.0)
    return sc, [cam], mlp_weights(103)


def workload_grad(R=128, P=512, n_rays=1 << 20, device="cpu"):
    """2x2 blocks of side 2 (FP32 parameters), 2^20 random rays; the fit
    target is the render of the same layout baked from seed 40."""
    sc = city_scene(4, 2, 2.0, [(R, P)], device=device)
    tgt = city_scene(40, 2, 2.0, [(R, P)], device=device)
    o, d = random_rays(n_rays, 4, sc.box_lo, sc.box_hi, device)
    return sc, tgt, o, d, mlp_weights(104), mlp_weights(140)


def workload_batch(res=((128, 512), (64, 256), (32, 128)), n_views=64, device="cpu",
                   sizes=((640, 360), (1280, 720), (1920, 1080))):
    """16x16-block city (side 2, 3 LOD levels), 64 aerial views with sizes
    drawn from 360p / 720p / 1080p; scene seed 5, MLP seed 105."""
    sc = city_scene(5, 16, 2.0, list(res), lod_thresh=[10.0, 20.0, 0.0], device=device)
    cams = random_aerial_cameras(n_views, 5, 16.0, (6.0, 14.0), list(sizes))
    return sc, cams, mlp_weights(105)
