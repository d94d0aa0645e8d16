"""FP64 CPU oracle for block-based volume rendering (City-on-Web, arXiv 2312.16457).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's timed CPU baseline may import this package.  The product path
(``paper_2312_16457_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``cow_oracle.c`` (plain C, FP64, OpenMP over rays);
this module compiles it with gcc (``build()``), loads it with ctypes and wraps
it for numpy / torch-CPU inputs produced by the shared seeded generator.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cow_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

MODE_BLOCKWISE, MODE_SINGLE_PASS, MODE_ALPHA_NORM = 0, 1, 2
DTYPES = {"fp32": 0, "fp16": 1, "bf16": 2, "fp8": 3}


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, -O2, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OrcBlock(C.Structure):
    _fields_ = [("lo", C.c_float * 3), ("hi", C.c_float * 3), ("R", C.c_int32), ("P", C.c_int32),
                ("occ_cell", C.c_int32), ("level", C.c_int32), ("parent", C.c_int32),
                ("is_f64", C.c_int32), ("grid", C.c_void_p), ("planes", C.c_void_p * 3),
                ("occ", C.c_void_p), ("unbounded", C.c_int32)]


class OrcCamera(C.Structure):
    _fields_ = [("c2w", C.c_double * 12), ("width", C.c_int32), ("height", C.c_int32),
                ("fov_y_deg", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        i32, i64, dbl, flt = C.c_int32, C.c_int64, C.c_double, C.c_float
        sig = {
            "orc_f32_to_f16": (C.c_uint16, [flt]), "orc_f16_to_f64": (dbl, [C.c_uint16]),
            "orc_f32_to_bf16": (C.c_uint16, [flt]), "orc_bf16_to_f64": (dbl, [C.c_uint16]),
            "orc_f32_to_e4m3": (C.c_uint8, [flt]), "orc_e4m3_to_f64": (dbl, [C.c_uint8]),
            "orc_e4m3_scale_exp": (i32, [flt]),
            "orc_quantize": (None, [P, i64, i32, P, P, P]),
            "orc_pixel_ray": (None, [P, i32, i32, P, P]),
            "orc_occ_cells": (i32, [i32, i32]),
            "orc_set_threads": (i32, [i32]),
            "orc_occupancy": (None, [P, i32, i32, flt, P]),
            "orc_feature_at": (dbl, [P, P, P]),
            "orc_mlp": (None, [P, P, i64, P]),
            "orc_render_view": (None, [P, i32, P, i32, P, P, i32, P, i64, P, P, P]),
            "orc_render_rays": (None, [P, i32, P, i32, P, P, i64, P, i32, P, P, P]),
            "orc_sort_ids_for_ray": (None, [P, P, i32, P, P]),
            "orc_ray_samples": (i64, [P, P, i32, P, P, P, P, P, i64]),
            "orc_ray_sample_steps": (i64, [P, P, i32, P, P, P, i64]),
            "orc_contract": (None, [P, P]),
            "orc_render_rays_grad": (None, [P, i32, P, i32, P, P, i64, P, P, P, P, P]),
            "orc_block_ztop": (dbl, [P]),
            "orc_select_lod": (i32, [P, i32, P, P, i32, P, i32]),
            "orc_sort_view": (None, [P, P, i32, P, P]),
            "orc_sparsity_loss_grad": (dbl, [P, i32, P, i32, P, i64, dbl, P, P]),
            "orc_opacity_loss_grad": (dbl, [P, i32, P, i32, P, P, i64, dbl, P, P]),
            "orc_pe_dim": (i32, [i32]),
            "orc_block_mlp_nparam": (i32, [i32]),
            "orc_pe": (None, [P, i32, P]),
            "orc_render_view_block_mlp": (None, [P, i32, P, i32, P, P, i32, P, i64, P, P, P]),
            "orc_render_rays_block_mlp": (None, [P, i32, P, i32, P, P, i64, P, i32, P, P, P]),
            "orc_render_rays_block_mlp_grad": (None, [P, i32, P, i32, P, P, i64, P, i32, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _np(x, dtype=np.float32) -> np.ndarray:
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(x, dtype=dtype)


def set_threads(n: int) -> int:
    """Threads of the oracle's parallel loops; returns the new maximum."""
    return int(lib().orc_set_threads(int(n)))


def make_camera(cam) -> OrcCamera:
    c = OrcCamera()
    c.c2w[:] = [float(v) for v in np.asarray(cam.c2w, np.float64).reshape(12)]
    c.width, c.height, c.fov_y_deg = int(cam.width), int(cam.height), float(cam.fov_y_deg)
    return c


# ---------------------------------------------------------------------------
# storage formats


def f32_to_f16_bits(x: float) -> int:
    return int(lib().orc_f32_to_f16(float(x)))


def f32_to_bf16_bits(x: float) -> int:
    return int(lib().orc_f32_to_bf16(float(x)))


def f32_to_e4m3_bits(x: float) -> int:
    return int(lib().orc_f32_to_e4m3(float(x)))


def f16_value(b: int) -> float:
    return float(lib().orc_f16_to_f64(int(b)))


def bf16_value(b: int) -> float:
    return float(lib().orc_bf16_to_f64(int(b)))


def e4m3_value(b: int) -> float:
    return float(lib().orc_e4m3_to_f64(int(b)))


def e4m3_scale_exp(amax: float) -> int:
    return int(lib().orc_e4m3_scale_exp(float(amax)))


def channel_scale_exps(x, dtype: str) -> np.ndarray:
    """Per-channel power-of-two scale exponents: FP8 maps each channel's
    max |x| to at most 448; the other formats use scale 1."""
    if dtype != "fp8":
        return np.zeros(8, np.int32)
    a = np.abs(_np(x)).reshape(-1, 8).max(axis=0)
    return np.array([e4m3_scale_exp(float(v)) for v in a], np.int32)


def quantize(x, dtype: str, scale_exp: Optional[np.ndarray] = None):
    """Encode float32 values (channel-interleaved, 8 channels) into the storage
    format; returns (bits, dequantized float32)."""
    xf = _np(x).reshape(-1)
    dt = DTYPES[dtype]
    bits = np.empty(xf.shape, {0: np.float32, 1: np.uint16, 2: np.uint16, 3: np.uint8}[dt])
    deq = np.empty(xf.shape, np.float32)
    se = None if scale_exp is None else np.ascontiguousarray(scale_exp, np.int32)
    lib().orc_quantize(_ptr(xf), xf.size, dt, _ptr(se), _ptr(bits), _ptr(deq))
    return bits, deq


# ---------------------------------------------------------------------------
# geometry


def occ_cells(R: int, C_: int) -> int:
    return int(lib().orc_occ_cells(R, C_))


def occupancy(grid, R: int, C_: int = 4, thresh: float = 0.01) -> np.ndarray:
    g = _np(grid).reshape(-1)
    nc = occ_cells(R, C_)
    bits = np.zeros(((nc ** 3 + 31) // 32,), np.uint32)
    lib().orc_occupancy(_ptr(g), R, C_, float(thresh), _ptr(bits))
    return bits


def pixel_rays(cam, pixels: Optional[Sequence[int]] = None):
    """FP32 origins / directions of pixel-centre rays (row-major linear index)."""
    oc = make_camera(cam)
    pix = np.arange(cam.width * cam.height) if pixels is None else np.asarray(pixels)
    o = np.empty((len(pix), 3), np.float32)
    d = np.empty((len(pix), 3), np.float32)
    ob = (C.c_float * 3)()
    db = (C.c_float * 3)()
    for k, lin in enumerate(pix):
        lib().orc_pixel_ray(C.byref(oc), int(lin % cam.width), int(lin // cam.width), ob, db)
        o[k] = list(ob)
        d[k] = list(db)
    return o, d


class OracleScene:
    """The oracle's view of a synthetic scene: host arrays plus occupancy bits
    computed by the oracle itself.

    values: "master" (FP32 arrays as given), or a storage format name
    ("fp16", "bf16", "fp8", "bf16_fp8" for a BF16 grid with FP8 planes, or
    "fp8_bf16d" for FP8 everywhere but the grid's log-density channel, which
    is BF16) to run on the oracle's own dequantisation of the master, or "f64"
    to hold float64 copies (finite differences)."""

    def __init__(self, scene, values: str = "master"):
        self.scene = scene
        self.values = values
        self._keep = []
        nb = len(scene.blocks)
        self.blocks = (OrcBlock * nb)()
        self.grids: List[np.ndarray] = []
        self.planes: List[List[np.ndarray]] = []
        self.occ: List[np.ndarray] = []
        for i, b in enumerate(scene.blocks):
            f64 = values == "f64"
            g = _np(b.grid, np.float64 if f64 else np.float32)
            pls = [_np(p, np.float64 if f64 else np.float32) for p in b.planes]
            bits = occupancy(_np(b.grid), b.R, scene.occ_cell, scene.occ_thresh)
            if values in ("fp16", "bf16", "fp8", "bf16_fp8", "fp8_bf16d"):
                gv, pv = {"bf16_fp8": ("bf16", "fp8"), "fp8_bf16d": ("fp8", "fp8")}.get(values, (values, values))
                gq = quantize(g, gv, channel_scale_exps(g, gv))[1].reshape(g.shape)
                if values == "fp8_bf16d":  # the log-density channel of the grid in BF16, unscaled
                    gq[..., 0] = quantize(g[..., 0], "bf16")[1].reshape(g.shape[:-1])
                g = gq
                pls = [quantize(p, pv, channel_scale_exps(p, pv))[1].reshape(p.shape) for p in pls]
            ob = self.blocks[i]
            ob.lo[:] = [float(v) for v in b.lo]
            ob.hi[:] = [float(v) for v in b.hi]
            ob.R, ob.P, ob.occ_cell, ob.level, ob.parent = b.R, b.P, scene.occ_cell, b.level, b.parent
            ob.is_f64 = 1 if f64 else 0
            ob.grid = g.ctypes.data
            for k in range(3):
                ob.planes[k] = pls[k].ctypes.data
            ob.occ = bits.ctypes.data
            ob.unbounded = int(getattr(b, "unbounded", 0))
            self.grids.append(g)
            self.planes.append(pls)
            self.occ.append(bits)

    def ptr(self):
        return C.cast(self.blocks, C.c_void_p)

    def __len__(self):
        return len(self.scene.blocks)

    def ztop(self, i: int) -> float:
        return float(lib().orc_block_ztop(C.byref(self.blocks[i])))


def select_lod(osc: OracleScene, cam, lod_thresh: Sequence[float]) -> np.ndarray:
    oc = make_camera(cam)
    th = np.ascontiguousarray(lod_thresh, np.float64)
    cap = len(osc)
    out = np.zeros(max(cap, 1), np.int32)
    n = lib().orc_select_lod(osc.ptr(), len(osc), C.byref(oc), _ptr(th), len(th), _ptr(out), cap)
    assert n <= cap
    return out[:n].copy()


def sort_view(osc: OracleScene, ids: Sequence[int], cam) -> np.ndarray:
    oc = make_camera(cam)
    a = np.ascontiguousarray(ids, np.int32)
    out = np.empty_like(a)
    lib().orc_sort_view(osc.ptr(), _ptr(a), len(a), C.byref(oc), _ptr(out))
    return out


def sort_ids_for_ray(osc: OracleScene, ids: Sequence[int], o) -> np.ndarray:
    a = np.ascontiguousarray(ids, np.int32)
    out = np.empty_like(a)
    of = np.ascontiguousarray(o, np.float32)
    lib().orc_sort_ids_for_ray(osc.ptr(), _ptr(a), len(a), _ptr(of), _ptr(out))
    return out


def _mlp64(mlp):
    return None if mlp is None else np.ascontiguousarray(_np(mlp, np.float64))


def render_view(osc: OracleScene, cam, order: Sequence[int], mlp=None, mode: int = MODE_BLOCKWISE,
                pixels: Optional[Sequence[int]] = None):
    """Returns (rgb [n,3], aux [n,8], nsamp [n]) in float64 / int32 for the
    given pixels (linear indices) or the whole image."""
    oc = make_camera(cam)
    ordr = np.ascontiguousarray(order, np.int32)
    pix = None if pixels is None else np.ascontiguousarray(pixels, np.int64)
    n = cam.width * cam.height if pix is None else len(pix)
    rgb = np.zeros((n, 3))
    aux = np.zeros((n, 8))
    ns = np.zeros(n, np.int32)
    w = _mlp64(mlp)
    lib().orc_render_view(osc.ptr(), len(osc), _ptr(ordr), len(ordr), C.byref(oc), _ptr(w), mode,
                          _ptr(pix), 0 if pix is None else len(pix), _ptr(rgb), _ptr(aux), _ptr(ns))
    return rgb, aux, ns


def pe_dim(n_freq: int) -> int:
    return int(lib().orc_pe_dim(n_freq))


def block_mlp_nparam(n_freq: int) -> int:
    """Parameters of one per-block deferred MLP with n_freq PE frequencies."""
    return int(lib().orc_block_mlp_nparam(n_freq))


def pe(d, n_freq: int) -> np.ndarray:
    """PE(d) of one direction: d, then sin(2^l d), cos(2^l d) for l < n_freq."""
    dd = np.ascontiguousarray(d, np.float64).reshape(3)
    out = np.zeros(pe_dim(n_freq))
    lib().orc_pe(_ptr(dd), n_freq, _ptr(out))
    return out


def render_view_block_mlp(osc: OracleScene, cam, order: Sequence[int], mlps, n_freq: int,
                          pixels: Optional[Sequence[int]] = None):
    """Per-block deferred MLPs blended by Eq. 5.  mlps: [n_blocks, nparam]
    (row i = block i of the scene).  Returns (rgb, aux, nsamp) like render_view."""
    oc = make_camera(cam)
    ordr = np.ascontiguousarray(order, np.int32)
    pix = None if pixels is None else np.ascontiguousarray(pixels, np.int64)
    n = cam.width * cam.height if pix is None else len(pix)
    w = np.ascontiguousarray(_np(mlps, np.float64))
    assert w.shape == (len(osc), block_mlp_nparam(n_freq)), w.shape
    rgb = np.zeros((n, 3))
    aux = np.zeros((n, 8))
    ns = np.zeros(n, np.int32)
    lib().orc_render_view_block_mlp(osc.ptr(), len(osc), _ptr(ordr), len(ordr), C.byref(oc), _ptr(w), n_freq,
                                    _ptr(pix), 0 if pix is None else len(pix), _ptr(rgb), _ptr(aux), _ptr(ns))
    return rgb, aux, ns


def render_rays_block_mlp(osc: OracleScene, ids: Sequence[int], o, d, mlps, n_freq: int):
    """Independent rays with per-block MLPs (Eq. 5); each ray sorts ids from
    its own origin.  mlps: [n_blocks, nparam].  Returns (rgb, aux, nsamp)."""
    of, df = _np(o).reshape(-1, 3), _np(d).reshape(-1, 3)
    n = of.shape[0]
    a = np.ascontiguousarray(ids, np.int32)
    w = np.ascontiguousarray(_np(mlps, np.float64))
    assert w.shape == (len(osc), block_mlp_nparam(n_freq)), w.shape
    rgb = np.zeros((n, 3))
    aux = np.zeros((n, 8))
    ns = np.zeros(n, np.int32)
    lib().orc_render_rays_block_mlp(osc.ptr(), len(osc), _ptr(a), len(a), _ptr(of), _ptr(df), n, _ptr(w), n_freq,
                                    _ptr(rgb), _ptr(aux), _ptr(ns))
    return rgb, aux, ns


def render_rays_block_mlp_grad(osc: OracleScene, ids: Sequence[int], o, d, mlps, n_freq: int, dL_drgb):
    """Analytic FP64 gradient of sum(dL_drgb * rgb) of render_rays_block_mlp
    w.r.t. every grid, plane and per-block MLP parameter; returns (grids,
    planes, mlps) as float64 arrays shaped like the parameters."""
    of, df = _np(o).reshape(-1, 3), _np(d).reshape(-1, 3)
    n = of.shape[0]
    a = np.ascontiguousarray(ids, np.int32)
    w = np.ascontiguousarray(_np(mlps, np.float64))
    assert w.shape == (len(osc), block_mlp_nparam(n_freq)), w.shape
    g = np.ascontiguousarray(_np(dL_drgb, np.float64).reshape(n, 3))
    gg, gp, gptr, pptr = _grad_arrays(osc)
    gm = np.zeros(w.shape, np.float64)
    lib().orc_render_rays_block_mlp_grad(osc.ptr(), len(osc), _ptr(a), len(a), _ptr(of), _ptr(df), n, _ptr(w),
                                         n_freq, _ptr(g), C.cast(gptr, C.c_void_p), C.cast(pptr, C.c_void_p),
                                         _ptr(gm))
    planes = [gp[3 * i:3 * i + 3] for i in range(len(gg))]
    return gg, planes, gm


def render_rays(osc: OracleScene, ids: Sequence[int], o, d, mlp=None, mode: int = MODE_BLOCKWISE):
    of, df = _np(o).reshape(-1, 3), _np(d).reshape(-1, 3)
    n = of.shape[0]
    a = np.ascontiguousarray(ids, np.int32)
    rgb = np.zeros((n, 3))
    aux = np.zeros((n, 8))
    ns = np.zeros(n, np.int32)
    w = _mlp64(mlp)
    lib().orc_render_rays(osc.ptr(), len(osc), _ptr(a), len(a), _ptr(of), _ptr(df), n, _ptr(w), mode,
                          _ptr(rgb), _ptr(aux), _ptr(ns))
    return rgb, aux, ns


def ray_samples(osc: OracleScene, order: Sequence[int], o, d, cap: int = 1 << 16):
    a = np.ascontiguousarray(order, np.int32)
    of, df = _np(o).reshape(3), _np(d).reshape(3)
    t = np.zeros(cap)
    blk = np.zeros(cap, np.int32)
    al = np.zeros(cap)
    n = lib().orc_ray_samples(osc.ptr(), _ptr(a), len(a), _ptr(of), _ptr(df), _ptr(t), _ptr(blk), _ptr(al), cap)
    n = min(n, cap)
    return t[:n], blk[:n], al[:n]


def ray_sample_steps(osc: OracleScene, order: Sequence[int], o, d, cap: int = 1 << 16) -> np.ndarray:
    """The step (delta) of each occupied sample of one ray, in ray_samples order."""
    a = np.ascontiguousarray(order, np.int32)
    of, df = _np(o).reshape(3), _np(d).reshape(3)
    out = np.zeros(cap)
    n = min(lib().orc_ray_sample_steps(osc.ptr(), _ptr(a), len(a), _ptr(of), _ptr(df), _ptr(out), cap), cap)
    return out[:n]


def contract(x) -> np.ndarray:
    """Eq. 16 (FP64) of one normalised point."""
    xx = np.ascontiguousarray(x, np.float64).reshape(3)
    u = np.zeros(3)
    lib().orc_contract(_ptr(xx), _ptr(u))
    return u


def render_rays_grad(osc: OracleScene, ids: Sequence[int], o, d, mlp, dL_drgb):
    """Analytic FP64 gradient of sum(dL_drgb * rgb) w.r.t. every grid, plane
    and MLP parameter; returns (grids, planes, mlp) as float64 arrays shaped
    like the parameters."""
    of, df = _np(o).reshape(-1, 3), _np(d).reshape(-1, 3)
    n = of.shape[0]
    a = np.ascontiguousarray(ids, np.int32)
    g = np.ascontiguousarray(_np(dL_drgb, np.float64).reshape(n, 3))
    gg = [np.zeros(x.shape, np.float64) for x in osc.grids]
    gp = [np.zeros(x.shape, np.float64) for pl in osc.planes for x in pl]
    gm = np.zeros(499, np.float64)
    gptr = (C.c_void_p * len(gg))(*[x.ctypes.data for x in gg])
    pptr = (C.c_void_p * len(gp))(*[x.ctypes.data for x in gp])
    lib().orc_render_rays_grad(osc.ptr(), len(osc), _ptr(a), len(a), _ptr(of), _ptr(df), n, _ptr(_mlp64(mlp)),
                               _ptr(g), C.cast(gptr, C.c_void_p), C.cast(pptr, C.c_void_p), _ptr(gm))
    planes = [gp[3 * i:3 * i + 3] for i in range(len(gg))]
    return gg, planes, gm


def _grad_arrays(osc):
    gg = [np.zeros(x.shape, np.float64) for x in osc.grids]
    gp = [np.zeros(x.shape, np.float64) for pl in osc.planes for x in pl]
    gptr = (C.c_void_p * len(gg))(*[x.ctypes.data for x in gg])
    pptr = (C.c_void_p * len(gp))(*[x.ctypes.data for x in gp])
    return gg, gp, gptr, pptr


def sparsity_loss_grad(osc: OracleScene, ids: Sequence[int], points, weight: float = 1.0, grad: bool = True):
    """Eq. 7 at the given FP32 points: returns (weight * loss, grid grads,
    plane grads) (gradients None when grad is False)."""
    pf = _np(points).reshape(-1, 3)
    a = np.ascontiguousarray(ids, np.int32)
    gg, gp, gptr, pptr = _grad_arrays(osc)
    loss = lib().orc_sparsity_loss_grad(osc.ptr(), len(osc), _ptr(a), len(a), _ptr(pf), pf.shape[0], float(weight),
                                        C.cast(gptr, C.c_void_p) if grad else None,
                                        C.cast(pptr, C.c_void_p) if grad else None)
    if not grad:
        return loss, None, None
    return loss, gg, [gp[3 * i:3 * i + 3] for i in range(len(gg))]


def opacity_loss_grad(osc: OracleScene, ids: Sequence[int], o, d, weight: float = 1.0, grad: bool = True):
    """Eq. 8 over ray batches (mean over rays of the sum over blocks)."""
    of, df = _np(o).reshape(-1, 3), _np(d).reshape(-1, 3)
    a = np.ascontiguousarray(ids, np.int32)
    gg, gp, gptr, pptr = _grad_arrays(osc)
    loss = lib().orc_opacity_loss_grad(osc.ptr(), len(osc), _ptr(a), len(a), _ptr(of), _ptr(df), of.shape[0],
                                       float(weight), C.cast(gptr, C.c_void_p) if grad else None,
                                       C.cast(pptr, C.c_void_p) if grad else None)
    if not grad:
        return loss, None, None
    return loss, gg, [gp[3 * i:3 * i + 3] for i in range(len(gg))]


def mlp(w, x) -> np.ndarray:
    xf = np.ascontiguousarray(_np(x, np.float64).reshape(-1, 10))
    out = np.zeros((xf.shape[0], 3))
    lib().orc_mlp(_ptr(_mlp64(w)), _ptr(xf), xf.shape[0], _ptr(out))
    return out


def feature_at(osc: OracleScene, i: int, p) -> np.ndarray:
    f = np.zeros(8)
    pp = np.ascontiguousarray(p, np.float64)
    lib().orc_feature_at(C.byref(osc.blocks[i]), _ptr(pp), _ptr(f))
    return f
