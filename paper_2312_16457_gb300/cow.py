"""ctypes binding of libcow's C ABI (include/cow.h): argument marshalling only.

Every step of rendering runs in libcow's CUDA kernels; this module converts
torch tensors / numpy arrays to pointers and back.  There is no CPU fallback:
if ``libcow.so`` has not been built, the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np
import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcow.so")
_lib = None

# "bf16_fp8": BF16 grid, FP8-E4M3 planes (quad layout); "fp8_bf16d": FP8-E4M3
# features with the grid's log-density channel in BF16
DTYPES = {"fp32": 0, "fp16": 1, "bf16": 2, "fp8": 3, "bf16_fp8": 4, "fp8_bf16d": 5}
LOAD_BRICKS = 1
ELEM_BYTES = {"fp32": 4, "fp16": 2, "bf16": 2, "fp8": 1}


def tensor_storage(storage: str, tensor: int) -> str:
    """Storage of tensor 0 (grid) or 1-3 (planes) of a context."""
    if storage == "bf16_fp8":
        return "bf16" if tensor == 0 else "fp8"
    if storage == "fp8_bf16d":
        return "bf16" if tensor == 4 else "fp8"
    return storage
FLAG_MLP_BF16 = 1
FLAG_BLOCK_MLPS = 2
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "UNSUPPORTED", 5: "TIMEOUT", 6: "DEVICE_ASSERT"}

# every symbol include/cow.h declares
EXPORTS = ["cow_load_blocks", "cow_load_blocks_ex", "cow_save_scene", "cow_load_scene", "cow_free", "cow_num_blocks", "cow_block_ztop", "cow_select_lod", "cow_sort_blocks",
           "cow_render", "cow_render_rays", "cow_render_partials", "cow_composite_over", "cow_render_rays_f64", "cow_render_rays_block_t", "cow_set_schedule", "cow_set_tile_order", "cow_set_block_mlps",
           "cow_sync_check", "cow_set_test_hooks", "cow_export_occupancy", "cow_export_occupancy_coarse", "cow_set_residency",
           "cow_set_block_unbounded",
           "cow_get_residency", "cow_block_bytes", "cow_plan_view_order", "cow_refine_view_order", "cow_sparsity_loss", "cow_opacity_loss",
           "cow_export_packed", "cow_gather_peak", "cow_reduce_peak", "cow_render_backward", "cow_render_backward_noalloc",
           "cow_render_backward_block_mlps",
           "cow_update_features", "cow_adam_step", "cow_mse_grad", "cow_batch_create", "cow_batch_free",
           "cow_batch_set_views", "cow_batch_render", "cow_batch_set_config", "cow_batch_tune",
           "cow_batch_last_groups", "cow_batch_set_run_fraction", "cow_batch_set_records", "cow_batch_get_config",
           "cow_batch_set_schedule", "cow_batch_get_schedule", "cow_set_ray_order", "cow_render_rays_block_state",
           "cow_render_backward_block_mlps_state", "cow_tune_schedule", "cow_last_error",
           "cow_version"]
SCHEDULES = {"warp": 0, "thread": 1, "thread_const": 2}


class Residency(C.Structure):
    _fields_ = [("budget_bytes", C.c_int64), ("resident_bytes", C.c_int64), ("resident_blocks", C.c_int32),
                ("uploads", C.c_int64), ("upload_bytes", C.c_int64), ("evictions", C.c_int64),
                ("evictions_waiting_last_call", C.c_int64)]


class CowError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libcow {STATUS.get(status, status)}: {msg}")
        self.status = status


class BlockDesc(C.Structure):
    _fields_ = [("lo", C.c_float * 3), ("hi", C.c_float * 3), ("lod", C.c_int32), ("parent", C.c_int32),
                ("grid_res", C.c_int32), ("plane_res", C.c_int32), ("grid", C.c_void_p),
                ("planes", C.c_void_p * 3)]


class Camera(C.Structure):
    _fields_ = [("c2w", C.c_double * 12), ("width", C.c_int32), ("height", C.c_int32), ("fov_y_deg", C.c_double)]


def lib_path() -> str:
    return _LIB_PATH


def lib():
    """Load libcow.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libcow.so is not built ({_LIB_PATH}); run __graft_entry__.build() first")
        L = C.CDLL(_LIB_PATH)
        P, i32, i64, dbl, flt, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_float, C.c_uint32
        sig = {
            "cow_load_blocks": [P, P, i32, i32, flt, i32, P],
            "cow_load_blocks_ex": [P, P, i32, i32, flt, i32, u32, P],
            "cow_save_scene": [P, C.c_char_p],
            "cow_load_scene": [P, C.c_char_p, P],
            "cow_free": [P],
            "cow_num_blocks": [P, P],
            "cow_block_ztop": [P, i32, P],
            "cow_select_lod": [P, P, P, i32, P, i32, P],
            "cow_sort_blocks": [P, P, P, i32, P],
            "cow_render": [P, P, i32, P, P, P, flt, u32, P, P, P, P],
            "cow_render_rays": [P, P, P, i64, P, i32, P, flt, u32, P, P, P, P],
            "cow_render_partials": [P, P, P, i64, P, i32, P, P],
            "cow_render_rays_f64": [P, P, P, i64, P, i32, P, P, P, P, P, P],
            "cow_composite_over": [P, P, P, i64, P, i32, P, P, u32, P, P, P],
            "cow_sync_check": [P, P],
            "cow_set_test_hooks": [P, u32, u32],
            "cow_set_schedule": [P, i32],
            "cow_set_tile_order": [P, i32],
            "cow_set_block_mlps": [P, P, i32, i32, P],
            "cow_export_occupancy": [P, i32, P, i64],
            "cow_export_occupancy_coarse": [P, i32, P, i64],
            "cow_set_residency": [P, i64, P],
            "cow_set_block_unbounded": [P, i32, i32, P],
            "cow_sparsity_loss": [P, P, i64, P, i32, flt, P, P, P, P],
            "cow_opacity_loss": [P, P, P, i64, P, i32, P, flt, P, P, P, P],
            "cow_render_rays_block_t": [P, P, P, i64, P, i32, P, u32, P, P, P, P, P],
            "cow_get_residency": [P, P],
            "cow_block_bytes": [P, i32, P],
            "cow_plan_view_order": [P, i32, P, P, i32, i64, P, P, P],
            "cow_refine_view_order": [P, i32, P, P, i32, i64, P, i32, P],
            "cow_export_packed": [P, i32, i32, P, i64, P],
            "cow_gather_peak": [i32, i64, i32, P, P],
            "cow_reduce_peak": [i64, i32, P, P],
            "cow_render_backward": [P, P, P, i64, P, i32, P, flt, P, P, P, P, P, P],
            "cow_render_backward_noalloc": [P, P, P, i64, P, i32, P, flt, P, P, P, P, P, P],
            "cow_render_backward_block_mlps": [P, P, P, i64, P, i32, P, P, P, P, P],
            "cow_update_features": [P, i32, P, P, P, P, P],
            "cow_adam_step": [P, P, P, P, i64, flt, flt, flt, flt, i32, P],
            "cow_mse_grad": [P, P, i64, P, P, P],
            "cow_batch_create": [P, i32, i32, P],
            "cow_batch_free": [P],
            "cow_batch_set_views": [P, P, i32, P, P, P],
            "cow_batch_render": [P, P, flt, u32, P, P, P, i32, P],
            "cow_batch_set_config": [P, i32, i32],
            "cow_batch_last_groups": [P, P],
            "cow_batch_set_run_fraction": [P, flt],
            "cow_batch_set_records": [P, i32],
            "cow_batch_get_config": [P, P, P, P],
            "cow_batch_set_schedule": [P, i32],
            "cow_set_ray_order": [P, i32],
            "cow_render_rays_block_state": [P, P, P, i64, P, i32, P, P, P],
            "cow_render_backward_block_mlps_state": [P, P, P, i64, P, i32, P, P, P, P, P, P],
            "cow_batch_get_schedule": [P, P],
            "cow_tune_schedule": [P, P, i32, P, P, P, flt, u32, P, i32, P, P, P, P],
            "cow_batch_tune": [P, P, flt, u32, P, i32, P, P, P, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.cow_last_error.restype = C.c_char_p
        L.cow_last_error.argtypes = []
        L.cow_version.restype = C.c_int32
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise CowError(rc, lib().cow_last_error().decode(errors="replace"))


def _camera(cam) -> Camera:
    c = Camera()
    c.c2w[:] = [float(v) for v in np.asarray(cam.c2w, np.float64).reshape(12)]
    c.width, c.height, c.fov_y_deg = int(cam.width), int(cam.height), float(cam.fov_y_deg)
    return c


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        assert t.is_contiguous()
        return t.data_ptr()
    return t.ctypes.data


def _as_f32(t):
    if isinstance(t, torch.Tensor):
        return t.detach().to(torch.float32).contiguous()
    return np.ascontiguousarray(t, np.float32)


class Context:
    """A packed scene on one GPU (wraps cow_ctx)."""

    def __init__(self, scene, storage: str = "fp32", occ_thresh: Optional[float] = None,
                 occ_cell: Optional[int] = None, stream=None, bricks: bool = False):
        """bricks=True stores the grids brick-sparse (cow_load_blocks_ex with
        COW_LOAD_BRICKS): only the 16^3-voxel bricks with occupied cells."""
        self.storage = storage
        self.bricks = bricks
        self.scene = scene
        n = len(scene.blocks)
        descs = (BlockDesc * n)()
        keep = []
        for i, b in enumerate(scene.blocks):
            d = descs[i]
            d.lo[:] = [float(v) for v in b.lo]
            d.hi[:] = [float(v) for v in b.hi]
            d.lod, d.parent, d.grid_res, d.plane_res = int(b.level), int(b.parent), int(b.R), int(b.P)
            g = _as_f32(b.grid)
            pls = [_as_f32(p) for p in b.planes]
            keep += [g, *pls]
            d.grid = _ptr(g)
            for k in range(3):
                d.planes[k] = _ptr(pls[k])
        self._ctx = C.c_void_p()
        th = scene.occ_thresh if occ_thresh is None else occ_thresh
        cc = scene.occ_cell if occ_cell is None else occ_cell
        _check(lib().cow_load_blocks_ex(C.byref(self._ctx), descs, n, DTYPES[storage], float(th), int(cc),
                                        LOAD_BRICKS if bricks else 0, _stream_ptr(stream)))
        self.n_blocks = n
        self.schedule = "thread_const"  # the library default
        for i, b in enumerate(scene.blocks):
            if getattr(b, "unbounded", 0):
                self.set_unbounded(i, b.unbounded, stream)
        del keep

    def close(self):
        if self._ctx:
            lib().cow_free(self._ctx)
            self._ctx = C.c_void_p()

    def save(self, path: str):
        """Write the packed scene to a file (cow_save_scene)."""
        _check(lib().cow_save_scene(self._ctx, os.fsencode(path)))

    @classmethod
    def load(cls, path: str, scene=None, stream=None) -> "Context":
        """A context from a packed scene file (cow_load_scene); `scene` (the
        synthetic description, optional) is kept for inspection helpers."""
        self = cls.__new__(cls)
        self._ctx = C.c_void_p()
        _check(lib().cow_load_scene(C.byref(self._ctx), os.fsencode(path), _stream_ptr(stream)))
        n = C.c_int32()
        _check(lib().cow_num_blocks(self._ctx, C.byref(n)))
        self.n_blocks = n.value
        self.scene = scene
        self.storage = None
        self.bricks = None
        self.schedule = "thread_const"
        return self

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- App. D ------------------------------------------------------------
    def select_lod(self, cam, lod_thresh: Sequence[float]) -> np.ndarray:
        th = np.ascontiguousarray(lod_thresh, np.float64)
        out = np.zeros(max(self.n_blocks, 1), np.int32)
        n = C.c_int32()
        c = _camera(cam)
        _check(lib().cow_select_lod(self._ctx, C.byref(c), _ptr(th), len(th), _ptr(out), self.n_blocks, C.byref(n)))
        return out[:n.value].copy()

    def sort_blocks(self, cam, ids: Sequence[int]) -> np.ndarray:
        a = np.ascontiguousarray(ids, np.int32)
        out = np.empty_like(a)
        c = _camera(cam)
        _check(lib().cow_sort_blocks(self._ctx, C.byref(c), _ptr(a), len(a), _ptr(out)))
        return out

    def ztop(self, i: int) -> float:
        v = C.c_double()
        _check(lib().cow_block_ztop(self._ctx, int(i), C.byref(v)))
        return v.value

    # --- rendering ---------------------------------------------------------
    def render(self, cams, ids_per_view, mlp, ert_eps: float = 0.0, mlp_bf16: bool = False, aux: bool = True,
               nsamp: bool = False, out=None, stream=None, device="cuda", block_mlps: bool = False):
        """Render views; returns (rgb, aux, nsamp) tensors with one row per
        pixel (views concatenated).  `out` may pass preallocated tensors
        (device or pinned host).  block_mlps=True renders with the per-block
        MLPs of set_block_mlps blended by Eq. 5 (`mlp` is then unused)."""
        cams = list(cams)
        cc = (Camera * len(cams))(*[_camera(c) for c in cams])
        offs = np.zeros(len(cams) + 1, np.int32)
        for v, ids in enumerate(ids_per_view):
            offs[v + 1] = offs[v] + len(ids)
        flat = np.ascontiguousarray(np.concatenate([np.asarray(i, np.int32) for i in ids_per_view])
                                    if offs[-1] > 0 else np.zeros(1, np.int32), np.int32)
        npix = sum(int(c.width) * int(c.height) for c in cams)
        if out is None:
            rgb = torch.empty((npix, 3), dtype=torch.float32, device=device)
            ax = torch.empty((npix, 8), dtype=torch.float32, device=device) if aux else None
            ns = torch.empty((npix,), dtype=torch.int32, device=device) if nsamp else None
        else:
            rgb, ax, ns = out
        m = None if mlp is None else (mlp if isinstance(mlp, torch.Tensor) else _as_f32(mlp))
        flags = (FLAG_MLP_BF16 if mlp_bf16 else 0) | (FLAG_BLOCK_MLPS if block_mlps else 0)
        _check(lib().cow_render(self._ctx, cc, len(cams), _ptr(flat), _ptr(offs), _ptr(m), float(ert_eps),
                                flags, _ptr(rgb), _ptr(ax), _ptr(ns), _stream_ptr(stream)))
        return rgb, ax, ns

    def set_block_mlps(self, mlps, n_freq: int, stream=None):
        """Per-block deferred MLPs: [n_blocks, 16 (10 + 6 n_freq) + 339] FP32
        (row i for block i), host or device; None removes them."""
        if mlps is None:
            _check(lib().cow_set_block_mlps(self._ctx, None, 0, 0, _stream_ptr(stream)))
            return
        m = _as_f32(mlps)
        _check(lib().cow_set_block_mlps(self._ctx, _ptr(m), int(m.shape[0]), int(n_freq), _stream_ptr(stream)))
        self._block_mlp_src = m  # a device source stays alive until the stream has copied it

    def render_rays(self, o: torch.Tensor, d: torch.Tensor, ids: Sequence[int], mlp, ert_eps: float = 0.0,
                    mlp_bf16: bool = False, aux: bool = True, nsamp: bool = False, stream=None,
                    block_mlps: bool = False):
        """Independent rays; block_mlps=True blends each ray's blocks by Eq. 5
        with the per-block MLPs of set_block_mlps (`mlp` is then unused)."""
        n = o.shape[0]
        o = o.contiguous()
        d = d.contiguous()
        a = np.ascontiguousarray(ids, np.int32)
        rgb = torch.empty((n, 3), dtype=torch.float32, device=o.device)
        ax = torch.empty((n, 8), dtype=torch.float32, device=o.device) if aux else None
        ns = torch.empty((n,), dtype=torch.int32, device=o.device) if nsamp else None
        m = None if mlp is None else (mlp if isinstance(mlp, torch.Tensor) else _as_f32(mlp))
        flags = (FLAG_MLP_BF16 if mlp_bf16 else 0) | (FLAG_BLOCK_MLPS if block_mlps else 0)
        _check(lib().cow_render_rays(self._ctx, _ptr(o), _ptr(d), n, _ptr(a), len(a), _ptr(m), float(ert_eps),
                                     flags, _ptr(rgb), _ptr(ax), _ptr(ns), _stream_ptr(stream)))
        return rgb, ax, ns

    def render_rays_f64(self, o: torch.Tensor, d: torch.Tensor, ids: Sequence[int], mlp64: torch.Tensor, grids64,
                        planes64, stream=None):
        """FP64 render for finite-difference checks (cow_render_rays_f64):
        grids64[i] / planes64[i][k] FP64 device tensors of every block (None
        for blocks outside ids); returns (rgb, aux) FP64."""
        a = np.ascontiguousarray(ids, np.int32)
        nb = self.n_blocks
        gg = (C.c_void_p * nb)(*[_ptr(g) if g is not None else None for g in grids64])
        flat = []
        for i in range(nb):
            pl = planes64[i] if planes64[i] is not None else [None, None, None]
            flat += [_ptr(t) if t is not None else None for t in pl]
        gp = (C.c_void_p * (3 * nb))(*flat)
        n = o.shape[0]
        rgb = torch.empty((n, 3), dtype=torch.float64, device=o.device)
        ax = torch.empty((n, 8), dtype=torch.float64, device=o.device)
        _check(lib().cow_render_rays_f64(self._ctx, _ptr(o.contiguous()), _ptr(d.contiguous()), n, _ptr(a), len(a),
                                         _ptr(mlp64.contiguous()), gg, gp, _ptr(rgb), _ptr(ax), _stream_ptr(stream)))
        return rgb, ax

    def render_partials(self, o: torch.Tensor, d: torch.Tensor, ids: Sequence[int], stream=None) -> torch.Tensor:
        """Per-block partials (C_d^k, F^k, T^k) of a ray batch: [n, len(ids), 8]."""
        a = np.ascontiguousarray(ids, np.int32)
        out = torch.empty((o.shape[0], len(a), 8), dtype=torch.float32, device=o.device)
        _check(lib().cow_render_partials(self._ctx, _ptr(o.contiguous()), _ptr(d.contiguous()), o.shape[0], _ptr(a),
                                         len(a), _ptr(out), _stream_ptr(stream)))
        return out

    def composite_over(self, o: torch.Tensor, d: torch.Tensor, ids: Sequence[int], partials: torch.Tensor, mlp,
                       mlp_bf16: bool = False, aux: bool = True, stream=None):
        """K2: the partials folded near to far (Eq. 12-13) and shaded (Eq. 3)."""
        a = np.ascontiguousarray(ids, np.int32)
        n = o.shape[0]
        rgb = torch.empty((n, 3), dtype=torch.float32, device=o.device)
        ax = torch.empty((n, 8), dtype=torch.float32, device=o.device) if aux else None
        m = mlp if isinstance(mlp, torch.Tensor) else torch.from_numpy(_as_f32(mlp)).to(o.device)
        _check(lib().cow_composite_over(self._ctx, _ptr(o.contiguous()), _ptr(d.contiguous()), n, _ptr(a), len(a),
                                        _ptr(partials.contiguous()), _ptr(m), FLAG_MLP_BF16 if mlp_bf16 else 0,
                                        _ptr(rgb), _ptr(ax), _stream_ptr(stream)))
        return rgb, ax

    def render_backward(self, o, d, ids, mlp, aux, dL_drgb, grad_grids, grad_planes, grad_mlp,
                        ert_eps: float = 0.0, stream=None, noalloc: bool = False):
        """Accumulate dL/d(features, MLP) of a ray batch into the given FP32
        device tensors (grad_grids[i]: R^3 x 8, grad_planes[i][k]: P^2 x 8,
        grad_mlp: 499; None skips a block).  noalloc=True calls the variant
        that allocates nothing (at most 65536 rays per call)."""
        a = np.ascontiguousarray(ids, np.int32)
        nb = self.n_blocks
        gg = (C.c_void_p * nb)(*[_ptr(g) if g is not None else None for g in grad_grids])
        flat = []
        for i in range(nb):
            pl = grad_planes[i] if grad_planes[i] is not None else [None, None, None]
            flat += [_ptr(t) if t is not None else None for t in pl]
        gp = (C.c_void_p * (3 * nb))(*flat)
        fn = lib().cow_render_backward_noalloc if noalloc else lib().cow_render_backward
        _check(fn(self._ctx, _ptr(o.contiguous()), _ptr(d.contiguous()), o.shape[0], _ptr(a), len(a), _ptr(mlp),
                  float(ert_eps), _ptr(aux), _ptr(dL_drgb.contiguous()), gg, gp, _ptr(grad_mlp), _stream_ptr(stream)))

    def render_backward_block_mlps(self, o, d, ids, dL_drgb, grad_grids, grad_planes, grad_block_mlps,
                                   stream=None):
        """Accumulate dL/d(features, per-block MLPs) of a ray batch rendered
        with block_mlps=True (no early termination) into FP32 device tensors;
        grad_block_mlps: [n_blocks, block_mlp_nparam(n_freq)]."""
        a = np.ascontiguousarray(ids, np.int32)
        gg, gp = self._grad_tables((grad_grids, grad_planes))
        _check(lib().cow_render_backward_block_mlps(self._ctx, _ptr(o.contiguous()), _ptr(d.contiguous()), o.shape[0],
                                                    _ptr(a), len(a), _ptr(dL_drgb.contiguous()), gg, gp,
                                                    _ptr(grad_block_mlps), _stream_ptr(stream)))

    def render_rays_block_state(self, o, d, ids, stream=None):
        """Per-block MLP forward without early termination that also returns
        the per-(ray, block) state the backward's first march would compute:
        (rgb [n, 3], state [n, len(ids), 8])."""
        a = np.ascontiguousarray(ids, np.int32)
        n = o.shape[0]
        rgb = torch.empty((n, 3), dtype=torch.float32, device=o.device)
        state = torch.empty((n, len(a), 8), dtype=torch.float32, device=o.device)
        _check(lib().cow_render_rays_block_state(self._ctx, _ptr(o.contiguous()), _ptr(d.contiguous()), n, _ptr(a),
                                                 len(a), _ptr(rgb), _ptr(state), _stream_ptr(stream)))
        return rgb, state

    def render_backward_block_mlps_state(self, o, d, ids, state, dL_drgb, grad_grids, grad_planes, grad_block_mlps,
                                         stream=None):
        """cow_render_backward_block_mlps from the forward's state (one march)."""
        a = np.ascontiguousarray(ids, np.int32)
        gg, gp = self._grad_tables((grad_grids, grad_planes))
        _check(lib().cow_render_backward_block_mlps_state(
            self._ctx, _ptr(o.contiguous()), _ptr(d.contiguous()), o.shape[0], _ptr(a), len(a), _ptr(state),
            _ptr(dL_drgb.contiguous()), gg, gp, _ptr(grad_block_mlps), _stream_ptr(stream)))

    def _grad_tables(self, grads):
        if grads is None:
            return None, None
        grad_grids, grad_planes = grads
        nb = self.n_blocks
        gg = (C.c_void_p * nb)(*[_ptr(g) if g is not None else None for g in grad_grids])
        flat = []
        for i in range(nb):
            pl = grad_planes[i] if grad_planes[i] is not None else [None, None, None]
            flat += [_ptr(t) if t is not None else None for t in pl]
        return gg, (C.c_void_p * (3 * nb))(*flat)

    def sparsity_loss(self, points, ids, weight: float = 1.0, loss=None, grads=None, stream=None):
        """Eq. 7 at device points (n x 3): adds weight * loss to `loss` (a
        1-element device tensor, created when None, returned) and, when
        grads = (grad_grids, grad_planes) is given, the density gradient."""
        a = np.ascontiguousarray(ids, np.int32)
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float32, device=points.device)
        gg, gp = self._grad_tables(grads)
        p = points.contiguous()
        _check(lib().cow_sparsity_loss(self._ctx, _ptr(p), p.shape[0], _ptr(a), len(a), float(weight), _ptr(loss),
                                       gg, gp, _stream_ptr(stream)))
        return loss

    def opacity_loss(self, o, d, ids, weight: float = 1.0, loss=None, grads=None, block_T=None, stream=None):
        """Eq. 8 over a ray batch (device o, d): as sparsity_loss.  block_T:
        the in-block transmittances of render_rays_block_t on the same rays
        and ids (each block is then marched once instead of twice)."""
        a = np.ascontiguousarray(ids, np.int32)
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float32, device=o.device)
        gg, gp = self._grad_tables(grads)
        oc, dc = o.contiguous(), d.contiguous()
        _check(lib().cow_opacity_loss(self._ctx, _ptr(oc), _ptr(dc), oc.shape[0], _ptr(a), len(a), _ptr(block_T),
                                      float(weight), _ptr(loss), gg, gp, _stream_ptr(stream)))
        return loss

    def render_rays_block_t(self, o, d, ids, mlp, mlp_bf16: bool = False, stream=None):
        """render_rays without early termination; returns (rgb, aux, block_T)
        with block_T[r, k] the transmittance of block ids[k] alone (-1: no
        occupied sample)."""
        n = o.shape[0]
        a = np.ascontiguousarray(ids, np.int32)
        rgb = torch.empty((n, 3), dtype=torch.float32, device=o.device)
        ax = torch.empty((n, 8), dtype=torch.float32, device=o.device)
        bt = torch.empty((n, len(a)), dtype=torch.float32, device=o.device)
        m = mlp if isinstance(mlp, torch.Tensor) else _as_f32(mlp)
        oc, dc = o.contiguous(), d.contiguous()
        _check(lib().cow_render_rays_block_t(self._ctx, _ptr(oc), _ptr(dc), n, _ptr(a), len(a), _ptr(m),
                                             FLAG_MLP_BF16 if mlp_bf16 else 0, _ptr(rgb), _ptr(ax), None, _ptr(bt),
                                             _stream_ptr(stream)))
        return rgb, ax, bt

    def update_features(self, i: int, grid, planes, stream=None):
        """Re-pack block i's features from new FP32 arrays (occupancy kept)."""
        g = _as_f32(grid)
        pls = [_as_f32(p) for p in planes]
        _check(lib().cow_update_features(self._ctx, int(i), _ptr(g), _ptr(pls[0]), _ptr(pls[1]), _ptr(pls[2]),
                                         _stream_ptr(stream)))

    def tune_schedule(self, cams, ids_per_view, mlp, out_rgb, ert_eps: float = 0.0, reps: int = 2, stream=None):
        """Times every marching schedule and tile order on these views and
        keeps the fastest (cow_tune_schedule); returns (schedule, strip, ms)."""
        cams = list(cams)
        cc = (Camera * len(cams))(*[_camera(c) for c in cams])
        flat, offs = _views_csr(ids_per_view)
        m = mlp if isinstance(mlp, torch.Tensor) else _as_f32(mlp)
        s, t, ms = C.c_int32(), C.c_int32(), C.c_float()
        _check(lib().cow_tune_schedule(self._ctx, cc, len(cams), _ptr(flat), _ptr(offs), _ptr(m), float(ert_eps), 0,
                                       _ptr(out_rgb), int(reps), _stream_ptr(stream), C.byref(s), C.byref(t),
                                       C.byref(ms)))
        self.schedule = {v: k for k, v in SCHEDULES.items()}[s.value]
        return self.schedule, t.value, ms.value

    RAY_ORDERS = {"given": 0, "coherent": 1}

    def set_ray_order(self, mode: str):
        """Processing order of ray batches: "coherent" (default; rays grouped by
        entry cell and direction) or "given"."""
        _check(lib().cow_set_ray_order(self._ctx, self.RAY_ORDERS[mode]))

    def set_schedule(self, name: str):
        """"thread_const" (default: one ray per thread, block records in the
        kernel parameter buffer), "thread" (records in shared memory) or
        "warp" (one ray per warp)."""
        _check(lib().cow_set_schedule(self._ctx, SCHEDULES[name]))
        self.schedule = name

    def set_tile_order(self, strip_tiles: int):
        """0: raster tile order; k > 0: vertical strips of k tile columns."""
        _check(lib().cow_set_tile_order(self._ctx, int(strip_tiles)))

    def set_test_hooks(self, skip_record_copy: bool = False, wait_polls: int = 0):
        """Tests of the bounded device waits (cow_set_test_hooks)."""
        _check(lib().cow_set_test_hooks(self._ctx, 1 if skip_record_copy else 0, int(wait_polls)))

    def sync_check(self, stream=None):
        _check(lib().cow_sync_check(self._ctx, _stream_ptr(stream)))

    # --- inspection --------------------------------------------------------
    def occupancy(self, i: int) -> np.ndarray:
        b = self.scene.blocks[i]
        nc = -(-(b.R - 1) // self.scene.occ_cell)
        words = (nc ** 3 + 31) // 32
        out = np.zeros(words, np.uint32)
        _check(lib().cow_export_occupancy(self._ctx, int(i), _ptr(out), words))
        return out

    def set_unbounded(self, i: int, flags: int, stream=None):
        """Block i becomes an unbounded (contracted) boundary block: flags =
        16 | the xy sides extended to infinity (1 -x, 2 +x, 4 -y, 8 +y); 0
        makes it bounded again."""
        _check(lib().cow_set_block_unbounded(self._ctx, int(i), int(flags), _stream_ptr(stream)))

    # --- dynamic loading ---------------------------------------------------
    def set_residency(self, budget_bytes: int, stream=None):
        """Keep at most budget_bytes of packed features on the device (0 = all)."""
        _check(lib().cow_set_residency(self._ctx, int(budget_bytes), _stream_ptr(stream)))

    def residency(self) -> dict:
        r = Residency()
        _check(lib().cow_get_residency(self._ctx, C.byref(r)))
        return {k: getattr(r, k) for k, _ in Residency._fields_}

    def block_bytes(self, i: int) -> int:
        out = C.c_int64()
        _check(lib().cow_block_bytes(self._ctx, int(i), C.byref(out)))
        return out.value

    def occupancy_coarse(self, i: int) -> np.ndarray:
        """Coarse level of block i's occupancy grid: one bit per 4^3 cells."""
        b = self.scene.blocks[i]
        nc = -(-(b.R - 1) // self.scene.occ_cell)
        nc2 = -(-nc // 4)
        words = (nc2 ** 3 + 31) // 32
        out = np.zeros(words, np.uint32)
        _check(lib().cow_export_occupancy_coarse(self._ctx, int(i), _ptr(out), words))
        return out

    def packed(self, i: int, tensor: int):
        b = self.scene.blocks[i]
        n = b.R ** 3 if tensor == 4 else (b.R ** 3 if tensor == 0 else b.P ** 2) * 8
        dt = {"fp32": np.float32, "fp16": np.uint16, "bf16": np.uint16,
              "fp8": np.uint8}[tensor_storage(self.storage, tensor)]
        out = np.zeros(n, dt)
        se = np.zeros(8, np.int32)
        _check(lib().cow_export_packed(self._ctx, int(i), int(tensor), _ptr(out), out.nbytes, _ptr(se)))
        return out, se


def _views_csr(ids_per_view):
    offs = np.zeros(len(ids_per_view) + 1, np.int32)
    for v, ids in enumerate(ids_per_view):
        offs[v + 1] = offs[v] + len(ids)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(i, np.int32) for i in ids_per_view])
                                if offs[-1] > 0 else np.zeros(1, np.int32), np.int32)
    return flat, offs


def refine_view_order(block_bytes: Sequence[int], ids_per_view, budget_bytes: int, order, max_evals: int = 2000):
    """Improve a view order by single-view moves under the same loading rule
    (cow_refine_view_order); returns (order, bytes loaded in it)."""
    bb = np.ascontiguousarray(block_bytes, np.int64)
    flat, offs = _views_csr(ids_per_view)
    out = np.ascontiguousarray(order, np.int32).copy()
    n = C.c_int64()
    _check(lib().cow_refine_view_order(_ptr(bb), len(bb), _ptr(flat), _ptr(offs), len(ids_per_view),
                                       int(budget_bytes), _ptr(out), int(max_evals), C.byref(n)))
    return out, n.value


def plan_view_order(block_bytes: Sequence[int], ids_per_view, budget_bytes: int):
    """Residency-aware view order (host only): returns (order, bytes loaded in
    that order, bytes loaded in the given order) under the LRU rule of
    Context.set_residency, from a cold start, one view per render call."""
    bb = np.ascontiguousarray(block_bytes, np.int64)
    flat, offs = _views_csr(ids_per_view)
    order = np.zeros(len(ids_per_view), np.int32)
    planned, given = C.c_int64(), C.c_int64()
    _check(lib().cow_plan_view_order(_ptr(bb), len(bb), _ptr(flat), _ptr(offs), len(ids_per_view), int(budget_bytes),
                                     _ptr(order), C.byref(planned), C.byref(given)))
    return order, planned.value, given.value


def gather_peak(bytes_per_load: int, buffer_bytes: int, iters: int = 256, stream=None) -> float:
    """Random-gather throughput (useful GB/s) of bytes_per_load-byte loads from
    a buffer of buffer_bytes (see cow_gather_peak)."""
    v = C.c_double()
    _check(lib().cow_gather_peak(int(bytes_per_load), int(buffer_bytes), int(iters), C.byref(v), _stream_ptr(stream)))
    return v.value


def reduce_peak(buffer_bytes: int, iters: int = 256, stream=None) -> float:
    """Random non-returning float4 reductions per second (10^9) into a
    device buffer (cow_reduce_peak)."""
    out = C.c_double()
    _check(lib().cow_reduce_peak(int(buffer_bytes), int(iters), C.byref(out), _stream_ptr(stream)))
    return out.value


def adam_step(param: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, lr: float, step: int,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None):
    """In-place Adam update of an FP32 device tensor (cow_adam_step)."""
    _check(lib().cow_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), float(lr), float(beta1),
                               float(beta2), float(eps), int(step), _stream_ptr(stream)))


def mse_grad(rgb: torch.Tensor, target: torch.Tensor, stream=None):
    """(dL/drgb, loss) of the mean squared error (cow_mse_grad); loss is a
    1-element device tensor."""
    g = torch.empty_like(rgb)
    loss = torch.empty(1, dtype=torch.float32, device=rgb.device)
    _check(lib().cow_mse_grad(_ptr(rgb.contiguous()), _ptr(target.contiguous()), rgb.numel(), _ptr(g), _ptr(loss),
                              _stream_ptr(stream)))
    return g, loss


class Batch:
    """Many cameras rendered by one persistent launch (cow_batch_*)."""

    TILE_SHAPES = {0: (16, 8), 1: (8, 8), 2: (16, 16), 3: (32, 8), 4: (8, 4)}  # 4: warp items

    def __init__(self, ctx: Context, max_views: int, max_ids: int):
        self.ctx = ctx
        self._b = C.c_void_p()
        _check(lib().cow_batch_create(ctx._ctx, int(max_views), int(max_ids), C.byref(self._b)))
        self.n_pixels = 0

    def close(self):
        if self._b:
            lib().cow_batch_free(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_views(self, cams, ids_per_view) -> int:
        cams = list(cams)
        cc = (Camera * len(cams))(*[_camera(c) for c in cams])
        offs = np.zeros(len(cams) + 1, np.int32)
        for v, ids in enumerate(ids_per_view):
            offs[v + 1] = offs[v] + len(ids)
        flat = np.ascontiguousarray(np.concatenate([np.asarray(i, np.int32) for i in ids_per_view])
                                    if offs[-1] > 0 else np.zeros(1, np.int32), np.int32)
        n = C.c_int64()
        _check(lib().cow_batch_set_views(self._b, cc, len(cams), _ptr(flat), _ptr(offs), C.byref(n)))
        self.n_pixels = n.value
        return n.value

    def render(self, mlp, out_rgb, out_aux=None, out_nsamp=None, ert_eps: float = 0.0, mlp_bf16: bool = False,
               graph: bool = False, stream=None):
        _check(lib().cow_batch_render(self._b, _ptr(mlp), float(ert_eps), FLAG_MLP_BF16 if mlp_bf16 else 0,
                                      _ptr(out_rgb), _ptr(out_aux), _ptr(out_nsamp), 1 if graph else 0,
                                      _stream_ptr(stream)))

    def last_groups(self) -> int:
        """Launches of the last render: 1, or the runs of views served one
        after another under a residency budget."""
        n = C.c_int32()
        _check(lib().cow_batch_last_groups(self._b, C.byref(n)))
        return n.value

    RECORDS = {"param": 0, "shared": 1}

    def set_records(self, mode: str):
        """Record placement of the batched kernels: "param" (runs, records in
        the parameter buffer) or "shared" (staged in shared memory)."""
        _check(lib().cow_batch_set_records(self._b, self.RECORDS[mode]))

    def config(self):
        """(tile shape, CTAs per SM, record placement) in use."""
        t, c, r = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().cow_batch_get_config(self._b, C.byref(t), C.byref(c), C.byref(r)))
        return self.TILE_SHAPES[t.value], c.value, {v: k for k, v in self.RECORDS.items()}[r.value]

    SCHEDULES = {"queue": 0, "grid": 1}

    def set_schedule(self, sched: str):
        """"queue" (persistent launches over the (view, tile) work queue) or
        "grid" (the view marcher, one launch per group of views)."""
        _check(lib().cow_batch_set_schedule(self._b, self.SCHEDULES[sched]))

    def schedule(self) -> str:
        k = C.c_int32()
        _check(lib().cow_batch_get_schedule(self._b, C.byref(k)))
        return {v: n for n, v in self.SCHEDULES.items()}[k.value]

    def set_run_fraction(self, frac: float):
        """Under a residency budget: the fraction of it one run may fill."""
        _check(lib().cow_batch_set_run_fraction(self._b, float(frac)))

    def set_config(self, tile_cfg: int, ctas_per_sm: int):
        _check(lib().cow_batch_set_config(self._b, int(tile_cfg), int(ctas_per_sm)))

    def tune(self, mlp, out_rgb, ert_eps: float = 0.0, mlp_bf16: bool = False, reps: int = 2, stream=None):
        t, c, ms = C.c_int32(), C.c_int32(), C.c_float()
        _check(lib().cow_batch_tune(self._b, _ptr(mlp), float(ert_eps), FLAG_MLP_BF16 if mlp_bf16 else 0,
                                    _ptr(out_rgb), int(reps), _stream_ptr(stream), C.byref(t), C.byref(c), C.byref(ms)))
        return t.value, c.value, ms.value
