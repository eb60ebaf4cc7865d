"""ctypes binding of librg.so (include/rg.h): argument marshalling only.

Every step of the render runs in the library's CUDA kernels. PyTorch provides
device memory for outputs and the current CUDA stream. There is no CPU
fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librg.so")

RG_OK = 0
STATUS = {0: "RG_OK", 1: "RG_ERR_INVALID_ARG", 2: "RG_ERR_OOM", 3: "RG_ERR_CUDA", 4: "RG_ERR_CAPACITY",
          5: "RG_ERR_TIMEOUT", 6: "RG_ERR_BUSY", 7: "RG_ERR_NOT_READY", 8: "RG_ERR_UNSUPPORTED"}
RG_STORE_FP32 = 1
RG_STORE_COMPACT = 2
RG_SH_SCALE_BAND = 0
RG_SH_SCALE_BAND_GAUSS = 1
RG_MODE_EXACT = 0
RG_MODE_ROOFGS = 1
RG_FLAG_EXACT_EXP = 1 << 0
RG_FLAG_SINGLE_PIXEL = 1 << 1
RG_FLAG_SORT_FULL_KEY = 1 << 2
RG_FLAG_QUAD_PIXEL = 1 << 3
RG_FLAG_STAGE_EVENTS = 1 << 8
RG_FLAG_BATCH_CHECKED = 1 << 9
RG_FLAG_TEST_STALL_SORT = 1 << 10
RG_FLAG_BATCH_FUSED = 1 << 11
RG_FLAG_BATCH_LANES = 1 << 12
RG_FLAG_TILE_COUNTING_SORT = 1 << 13
RG_FLAG_ORDERED_FRONT_END = 1 << 14
RG_INSPECT_KEYS = 1
RG_INSPECT_VALUES = 2
RG_INSPECT_RANGES = 3
RG_INSPECT_SH_CODES = 4
RG_INSPECT_SH_SCALES = 5
RG_INSPECT_GAUSS_SCALE = 6
RG_INSPECT_GEOM16 = 7
RG_INSPECT_LOG_OPACITY = 8

# every entry point include/rg.h declares
EXPORTS = ["rg_scene_create", "rg_scene_destroy", "rg_scene_reserve", "rg_render", "rg_scene_check",
           "rg_stage_times", "rg_inspect", "rg_eval_fast_exp", "rg_render_batch", "rg_backward", "rg_submit",
           "rg_poll", "rg_last_error", "rg_version", "rg_sort_pairs_noalloc", "rg_batch_plan_info",
           "rg_server_create", "rg_server_destroy", "rg_server_stats", "rg_server_reset_stats", "rg_scene_save",
           "rg_scene_load"]


class RgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, str(status)), msg))
        self.status = status


class RgCamera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("znear", C.c_float), ("zfar", C.c_float), ("bg", C.c_float * 3)]


class RgSceneDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("on_device", C.c_int32), ("means", C.c_void_p),
                ("scales", C.c_void_p), ("quats", C.c_void_p), ("opacities", C.c_void_p), ("sh", C.c_void_p),
                ("storage", C.c_uint32), ("sh_scale_mode", C.c_int32)]


class RgOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("flags", C.c_uint32), ("tile_w", C.c_int32), ("tile_h", C.c_int32)]


class RgGrads(C.Structure):
    _fields_ = [("means", C.c_void_p), ("scales", C.c_void_p), ("quats", C.c_void_p), ("opacities", C.c_void_p),
                ("sh", C.c_void_p)]


class RgServerConfig(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("memory_budget", C.c_int64), ("max_width", C.c_int32),
                ("max_height", C.c_int32), ("mode", C.c_int32), ("flags", C.c_uint32), ("calibration", C.c_void_p)]


class RgServerStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("pending", C.c_int64), ("slots", C.c_int32), ("max_in_flight", C.c_int32),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("slot_bytes", C.c_int64),
                ("p50_delivered_ms", C.c_double), ("p99_delivered_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class RgStats(C.Structure):
    _fields_ = [("n_gaussians", C.c_int64), ("n_front", C.c_int64), ("n_visible", C.c_int64),
                ("n_entries", C.c_int64), ("capacity", C.c_int64), ("n_pairs", C.c_int64), ("n_blends", C.c_int64),
                ("regrown", C.c_int32), ("sort_passes", C.c_int32), ("b_t", C.c_int32),
                ("b_d", C.c_int32), ("tiles_x", C.c_int32), ("tiles_y", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load librg.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("librg.so is not built (run __graft_entry__.build() or "
                               "python paper_2608_15785_gb300/build.py); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.rg_scene_create.argtypes = [C.POINTER(RgSceneDesc), P, C.POINTER(P)]
        L.rg_scene_destroy.argtypes = [P]
        L.rg_scene_reserve.argtypes = [P, C.c_int64]
        L.rg_render.argtypes = [P, C.POINTER(RgCamera), C.POINTER(RgOpts), P, C.POINTER(RgStats), P]
        L.rg_scene_check.argtypes = [P, P]
        L.rg_stage_times.argtypes = [P, C.POINTER(C.c_float), C.POINTER(C.c_int32)]
        L.rg_inspect.argtypes = [P, C.c_int32, P, C.c_int64, C.POINTER(C.c_int64)]
        L.rg_eval_fast_exp.argtypes = [P, P, C.c_int64, P]
        L.rg_render_batch.argtypes = [P, P, P, C.c_int32, C.POINTER(RgOpts), P, P]
        L.rg_batch_plan_info.argtypes = [P, P, P, C.c_int32, C.POINTER(RgOpts), P, P, P, P, P]
        L.rg_backward.argtypes = [P, C.POINTER(RgCamera), C.POINTER(RgOpts), P, C.POINTER(RgGrads), P]
        L.rg_submit.argtypes = [P, C.POINTER(RgCamera), C.c_int32, C.POINTER(C.c_uint64)]
        L.rg_poll.argtypes = [P, C.c_uint64, P]
        L.rg_server_create.argtypes = [P, C.c_int32, C.POINTER(RgServerConfig), C.POINTER(P)]
        L.rg_server_destroy.argtypes = [P]
        L.rg_server_stats.argtypes = [P, C.POINTER(RgServerStats)]
        L.rg_server_reset_stats.argtypes = [P]
        L.rg_sort_pairs_noalloc.argtypes = [P, P, C.c_int64, C.c_int32, P, P]
        L.rg_last_error.restype = C.c_char_p
        L.rg_last_error.argtypes = []
        L.rg_version.restype = C.c_int32
        for name in EXPORTS:
            if name not in ("rg_last_error", "rg_version"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def check(status: int):
    if status != RG_OK:
        raise RgError(status, lib().rg_last_error().decode())


def camera_struct(cam) -> RgCamera:
    c = RgCamera()
    for i, x in enumerate(np.asarray(cam.R, dtype=np.float32).reshape(9)):
        c.R[i] = float(x)
    for i, x in enumerate(np.asarray(cam.t, dtype=np.float32).reshape(3)):
        c.t[i] = float(x)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.znear, c.zfar = float(cam.znear), float(cam.zfar)
    for i, x in enumerate(np.asarray(cam.bg, dtype=np.float32).reshape(3)):
        c.bg[i] = float(x)
    return c


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _mode(mode) -> int:
    if isinstance(mode, str):
        return {"exact": RG_MODE_EXACT, "roofgs": RG_MODE_ROOFGS}[mode]
    return int(mode)


class Scene:
    """A resident scene on the current CUDA device (rg_scene_create)."""

    def __init__(self, scene, storage: int = RG_STORE_FP32 | RG_STORE_COMPACT,
                 sh_scale_mode: int = RG_SH_SCALE_BAND, stream=None):
        import torch
        L = lib()
        arrs = [scene.means, scene.scales, scene.quats, scene.opacities, scene.sh]
        on_dev = all(isinstance(a, torch.Tensor) and a.is_cuda for a in arrs)
        if on_dev:
            keep = [a.contiguous().float() for a in arrs]
            ptrs = [a.data_ptr() for a in keep]
        else:
            keep = [np.ascontiguousarray(a if not isinstance(a, torch.Tensor) else a.cpu().numpy(), dtype=np.float32)
                    for a in arrs]
            ptrs = [a.ctypes.data for a in keep]
        d = RgSceneDesc()
        d.n = int(keep[0].shape[0])
        d.sh_degree = int(getattr(scene, "sh_degree", 3))
        d.on_device = 1 if on_dev else 0
        d.means, d.scales, d.quats, d.opacities, d.sh = ptrs
        d.storage = int(storage)
        d.sh_scale_mode = int(sh_scale_mode)
        h = C.c_void_p()
        check(L.rg_scene_create(C.byref(d), _stream_ptr(stream), C.byref(h)))
        self._h = h
        self.n = d.n

    @property
    def handle(self):
        return self._h

    def save(self, path: str):
        """Write the scene's stored buffers to a file (rg_scene_save)."""
        check(lib().rg_scene_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str, stream=None) -> "Scene":
        """A resident scene from a file written by save() (rg_scene_load), no re-encoding."""
        h = C.c_void_p()
        check(lib().rg_scene_load(os.fsencode(path), _stream_ptr(stream), C.byref(h)))
        obj = cls.__new__(cls)
        obj._h = h
        with open(path, "rb") as f:  # header: magic[8], version u32, storage u32, n i64, ...
            obj.n = int(np.frombuffer(f.read(24)[16:24], dtype="<i8")[0])
        return obj

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rg_scene_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, cam, mode="roofgs", flags: int = 0, out=None, stats: bool = False, stream=None, tile=(16, 16)):
        """Render one view; returns a [3, H, W] float32 CUDA tensor (and stats if asked).
        tile: (16, 16), (32, 8) or (8, 32) pixels."""
        import torch
        c = camera_struct(cam)
        if out is None:
            out = torch.empty((3, c.height, c.width), dtype=torch.float32, device="cuda")
        o = RgOpts(_mode(mode), int(flags), int(tile[0]), int(tile[1]))
        st = RgStats() if stats else None
        check(lib().rg_render(self._h, C.byref(c), C.byref(o), C.c_void_p(out.data_ptr()),
                              C.byref(st) if st is not None else None, _stream_ptr(stream)))
        return (out, st.as_dict()) if stats else out

    def backward(self, cam, dL_dimg, stream=None, tile=(16, 16)) -> dict:
        """Gradients of L w.r.t. the FP32 attributes, given dL/dimage of the exact-mode render."""
        import torch
        g = {"means": torch.empty((self.n, 3), device="cuda"), "scales": torch.empty((self.n, 3), device="cuda"),
             "quats": torch.empty((self.n, 4), device="cuda"), "opacities": torch.empty((self.n,), device="cuda"),
             "sh": torch.empty((self.n, 16, 3), device="cuda")}
        gg = RgGrads(*(g[k].data_ptr() for k in ("means", "scales", "quats", "opacities", "sh")))
        c = camera_struct(cam)
        o = RgOpts(RG_MODE_EXACT, 0, int(tile[0]), int(tile[1]))
        d = dL_dimg.contiguous().float()
        check(lib().rg_backward(self._h, C.byref(c), C.byref(o), C.c_void_p(d.data_ptr()), C.byref(gg),
                                _stream_ptr(stream)))
        return g

    def reserve(self, n_entries: int):
        check(lib().rg_scene_reserve(self._h, int(n_entries)))

    def check(self, stream=None):
        check(lib().rg_scene_check(self._h, _stream_ptr(stream)))

    def stage_times(self):
        ms = (C.c_float * 7)()
        fr = C.c_int32()
        check(lib().rg_stage_times(self._h, ms, C.byref(fr)))
        return list(ms), fr.value

    def inspect(self, what: int) -> np.ndarray:
        nb = C.c_int64()
        check(lib().rg_inspect(self._h, int(what), None, 0, C.byref(nb)))
        dtype = {RG_INSPECT_KEYS: np.uint8, RG_INSPECT_VALUES: np.uint32, RG_INSPECT_RANGES: np.uint32,
                 RG_INSPECT_SH_CODES: np.int8, RG_INSPECT_SH_SCALES: np.float32, RG_INSPECT_GAUSS_SCALE: np.uint16,
                 RG_INSPECT_GEOM16: np.uint16, RG_INSPECT_LOG_OPACITY: np.float32}[what]
        buf = np.zeros(nb.value, dtype=np.uint8)
        check(lib().rg_inspect(self._h, int(what), buf.ctypes.data_as(C.c_void_p), nb.value, C.byref(nb)))
        return buf.view(dtype)


def render_batch(scenes, scene_idx, cams, mode="roofgs", flags: int = 0, outs=None, stream=None, tile=(0, 0)):
    """Render many views in one captured graph (rg_render_batch); returns the list of [3, H, W] tensors.
    tile (0, 0): the plan's autotuner picks the tile shape."""
    import torch
    n = len(cams)
    if outs is None:
        outs = [torch.empty((3, int(c.height), int(c.width)), dtype=torch.float32, device="cuda") for c in cams]
    hs = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    idx = (C.c_int32 * n)(*[int(i) for i in scene_idx])
    cs = (RgCamera * n)(*[camera_struct(c) for c in cams])
    ptrs = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    o = RgOpts(_mode(mode), int(flags), int(tile[0]), int(tile[1]))
    check(lib().rg_render_batch(hs, idx, cs, n, C.byref(o), ptrs, _stream_ptr(stream)))
    return outs


def batch_plan_info(scenes, scene_idx, cams, mode="roofgs", flags: int = 0, tile=(0, 0), with_path=False):
    """(lanes, pixels per thread, tile width, tile height[, fused]) the plan of these views uses."""
    n = len(cams)
    hs = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
    idx = (C.c_int32 * n)(*[int(i) for i in scene_idx])
    cs = (RgCamera * n)(*[camera_struct(c) for c in cams])
    o = RgOpts(_mode(mode), int(flags), int(tile[0]), int(tile[1]))
    lanes, ppt, tw, th, fused = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    check(lib().rg_batch_plan_info(hs, idx, cs, n, C.byref(o), C.byref(lanes), C.byref(ppt), C.byref(tw),
                                   C.byref(th), C.byref(fused)))
    if with_path:
        return lanes.value, ppt.value, tw.value, th.value, bool(fused.value)
    return lanes.value, ppt.value, tw.value, th.value


class Server:
    """Request loop over resident scenes (rg_server_create / rg_submit / rg_poll)."""

    def __init__(self, scenes, max_width, max_height, mode="roofgs", flags=0, max_slots=0, memory_budget=0,
                 calibration=None):
        self._scenes = list(scenes)
        hs = (C.c_void_p * len(scenes))(*[s.handle.value for s in scenes])
        self._cal = camera_struct(calibration) if calibration is not None else None
        cfg = RgServerConfig(int(max_slots), int(memory_budget), int(max_width), int(max_height), _mode(mode),
                             int(flags), C.cast(C.pointer(self._cal), C.c_void_p) if self._cal is not None else None)
        h = C.c_void_p()
        check(lib().rg_server_create(hs, len(scenes), C.byref(cfg), C.byref(h)))
        self._h = h

    def submit(self, cam, scene: int) -> int:
        t = C.c_uint64()
        check(lib().rg_submit(self._h, C.byref(camera_struct(cam)), int(scene), C.byref(t)))
        return t.value

    def poll(self, ticket: int, out) -> bool:
        """True once the image has been copied into `out` ([3, H, W] CUDA or pinned host tensor); False while not ready."""
        st = lib().rg_poll(self._h, C.c_uint64(ticket), C.c_void_p(out.data_ptr()))
        if st == 7:  # RG_ERR_NOT_READY
            return False
        check(st)
        return True

    def stats(self) -> dict:
        s = RgServerStats()
        check(lib().rg_server_stats(self._h, C.byref(s)))
        return s.as_dict()

    def reset_stats(self):
        check(lib().rg_server_reset_stats(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eval_fast_exp(P, stream=None):
    """Device evaluation of the rasterizer's bit-level exponential (Eq. (24))."""
    import torch
    P = P.contiguous().float()
    out = torch.empty_like(P)
    check(lib().rg_eval_fast_exp(C.c_void_p(P.data_ptr()), C.c_void_p(out.data_ptr()), P.numel(), _stream_ptr(stream)))
    return out


def version() -> int:
    return lib().rg_version()
