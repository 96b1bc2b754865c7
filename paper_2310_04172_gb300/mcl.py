"""Thin Python binding of the C ABI in include/mcl.h (ctypes).

Functions carry the C names and only marshal arguments: torch tensors (CUDA,
contiguous, the dtype the C call expects) become device pointers, the current
torch stream becomes the cudaStream_t. Every step of the computation runs in
the CUDA kernels of libmcl.so; there is no CPU fallback. If the library is
missing, loading raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmcl.so")

MCL_OK, MCL_EINVAL, MCL_ENOMEM, MCL_EBUSY, MCL_ETIMEDOUT, MCL_ECUDA, MCL_EINTERNAL = range(7)
MCL_MAP_DENSE, MCL_MAP_BRICK = 0, 1
MCL_F32, MCL_F16, MCL_I16 = 0, 1, 2
MCL_LAYOUT_LINEAR, MCL_LAYOUT_BLOCK4 = 0, 1
MCL_INDEX_AUTO, MCL_INDEX_HASH, MCL_INDEX_GRID = 0, 1, 2
MCL_LOGPROD, MCL_SUM = 0, 1
MCL_NEGLECT_OUTSIDE = 1
MCL_TRILINEAR = 2
PHASES = ("pose", "pack", "sensor", "reduce", "normalise", "resample", "motion", "other")

_c_void_p, _i64, _i32, _u32, _u64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                     ctypes.c_uint32, ctypes.c_uint64)


class mcl_map_desc(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("kind", _i32), ("dtype", _i32),
                ("origin", ctypes.c_float * 3), ("voxel", ctypes.c_float),
                ("inv_voxel", ctypes.c_float), ("truncation", ctypes.c_float),
                ("dims", _i64 * 3), ("n_bricks", _i64), ("brick_coords", _c_void_p),
                ("device_layout", _i32), ("index", _i32)]


class mcl_map_info(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("device_bytes", _i64), ("n_bricks", _i64),
                ("hash_capacity", _i64), ("hash_max_probe", _i32), ("device", _i32),
                ("score_sigma", ctypes.c_float), ("score_outside", ctypes.c_float),
                ("index", _i32), ("reserved", _i32), ("index_bytes", _i64)]


class mcl_sensor_params(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("sigma_hit", ctypes.c_float), ("mode", _i32),
                ("flags", _u32), ("points_per_chunk", _i32), ("lanes_per_particle", _i32),
                ("particles_per_item", _i32), ("unroll", _i32), ("pipeline", _i32),
                ("particle_order", _i32), ("item_order", _i32), ("scan_rings", _i32)]


class mcl_sensor_plan(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("points_per_chunk", _i32), ("lanes_per_particle", _i32),
                ("particles_per_item", _i32), ("unroll", _i32), ("pipeline", _i32),
                ("particle_order", _i32), ("threads", _i32), ("grid", _i32),
                ("blocks_per_sm", _i32), ("num_sms", _i32), ("n_items", _i64),
                ("workspace_bytes", _i64), ("item_order", _i32), ("blocks_per_sweep", _i32)]


class mcl_profile(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("launches", _i64 * 8), ("ms", ctypes.c_double * 8)]


class mcl_tune_params(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("max_particles", _i32), ("repeats", _i32),
                ("use_cache", _i32), ("tune_summation", _i32), ("cache_path", ctypes.c_char_p)]


class mcl_tune_result(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("best", mcl_sensor_params), ("best_ms", ctypes.c_double),
                ("default_ms", ctypes.c_double), ("candidates", _i32), ("from_cache", _i32)]


class mcl_session_update(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("map", _c_void_p), ("particles", _c_void_p), ("P", _i64),
                ("scan", _c_void_p), ("N", _i64), ("sigma_hit", ctypes.c_float), ("mode", _i32),
                ("flags", _u32), ("logw", _c_void_p), ("w", _c_void_p), ("resample_idx", _c_void_p),
                ("particles_out", _c_void_p), ("estimate", _c_void_p), ("scan_rings", _i32)]


class mcl_batch_params(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("points_per_chunk", _i32), ("lanes_per_particle", _i32),
                ("particles_per_item", _i32), ("unroll", _i32), ("pipeline", _i32),
                ("particle_order", _i32), ("use_graph", _i32), ("item_order", _i32)]


class mcl_batch_info(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("n_sessions", _i32), ("n_groups", _i32), ("n_items", _i64),
                ("total_evals", _i64), ("workspace_bytes", _i64), ("kernels_per_run", _i32),
                ("graph_captured", _i32)]


class mcl_server_desc(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("hbm_budget_bytes", _i64), ("max_sessions", _i32),
                ("max_in_flight", _i32), ("max_batch", _i32), ("shape", mcl_batch_params)]


class mcl_session_desc(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("map", _c_void_p), ("P", _i64), ("max_N", _i64),
                ("particles", _c_void_p), ("sigma_hit", ctypes.c_float), ("mode", _i32),
                ("flags", _u32), ("motion_sigma", ctypes.c_float * 6), ("seed", _u64),
                ("first_step", _i64), ("scan_rings", _i32)]


class mcl_session_info(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("P", _i64), ("max_N", _i64), ("step", _i64), ("seed", _u64),
                ("device_bytes", _i64)]





class mcl_server_stats(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("completed", _i64), ("superseded", _i64), ("batches", _i64),
                ("evals", _i64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_batch_sessions", ctypes.c_double),
                ("wall_s", ctypes.c_double), ("evals_per_s", ctypes.c_double),
                ("bytes_in_use", _i64), ("sessions", _i32), ("in_flight", _i32)]


class mcl_estimate(ctypes.Structure):
    _fields_ = [("weight_sum", ctypes.c_double), ("n_eff", ctypes.c_double),
                ("mean_pose", ctypes.c_double * 6), ("quat", ctypes.c_double * 4),
                ("rpy", ctypes.c_double * 3), ("concentration", ctypes.c_double),
                ("argmax", _i64), ("best_pose", ctypes.c_float * 6), ("best_w", ctypes.c_float),
                ("reserved", _i32)]


ESTIMATE_BYTES = ctypes.sizeof(mcl_estimate)


class mcl_result(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("status", _i32), ("latency_ms", ctypes.c_double),
                ("evals", _i64), ("step", _i64), ("estimate", mcl_estimate)]


class mcl_filter_desc(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("map", _c_void_p), ("P", _i64), ("max_points", _i64),
                ("sensor", mcl_sensor_params), ("motion_sigma", ctypes.c_float * 6), ("seed", _u64),
                ("use_graph", _i32), ("max_graphs", _i32), ("first_step", _i64)]


class mcl_filter_state(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("particles", _c_void_p), ("logw", _c_void_p),
                ("w", _c_void_p), ("idx", _c_void_p), ("estimate", _c_void_p), ("P", _i64),
                ("steps", _i64), ("graph_launches", _i64), ("last_r", ctypes.c_double),
                ("device_bytes", _i64), ("graphs", _i32), ("reserved", _i32)]


class MclError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"mcl status {status}: {message}")
        self.status = status


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes) of every exported entry point
SIGNATURES = {
    "mcl_last_error": (ctypes.c_char_p, []),
    "mcl_version": (_i32, []),
    "mcl_sync": (_i32, [_c_void_p]),
    "mcl_map_create": (_i32, [ctypes.POINTER(mcl_map_desc), _c_void_p, ctypes.POINTER(_c_void_p)]),
    "mcl_map_destroy": (_i32, [_c_void_p]),
    "mcl_map_create_score": (_i32, [_c_void_p, ctypes.c_float, _i32, ctypes.POINTER(_c_void_p)]),
    "mcl_map_get_info": (_i32, [_c_void_p, ctypes.POINTER(mcl_map_info)]),
    "mcl_map_lookup": (_i32, [_c_void_p, _c_void_p, _i64, _c_void_p, _c_void_p, _c_void_p]),
    "mcl_sensor_update": (_i32, [_c_void_p, _c_void_p, _i64, _c_void_p, _i64,
                                 ctypes.POINTER(mcl_sensor_params), _c_void_p, _c_void_p, _c_void_p]),
    "mcl_normalise": (_i32, [_c_void_p, _i64, _c_void_p, _c_void_p, _c_void_p]),
    "mcl_pose_estimate": (_i32, [_c_void_p, _c_void_p, _i64, _c_void_p, _c_void_p]),
    "mcl_sensor_update_estimate": (_i32, [_c_void_p, _c_void_p, _i64, _c_void_p, _i64,
                                          ctypes.POINTER(mcl_sensor_params), _c_void_p, _c_void_p,
                                          _c_void_p, _c_void_p]),
    "mcl_pose_to_matrix": (_i32, [_c_void_p, _i64, _c_void_p, _c_void_p]),
    "mcl_sensor_plan_get": (_i32, [_c_void_p, _i64, _i64, ctypes.POINTER(mcl_sensor_params),
                                   ctypes.POINTER(mcl_sensor_plan)]),
    "mcl_resample": (_i32, [_c_void_p, _i64, ctypes.c_double, _c_void_p, _c_void_p, _c_void_p,
                            _c_void_p]),
    "mcl_resample_noalloc": (_i32, [_c_void_p, _i64, ctypes.c_double, _c_void_p, _c_void_p,
                                    _c_void_p, _c_void_p]),
    "mcl_motion_update": (_i32, [_c_void_p, _i64, _c_void_p, _c_void_p, _u64, _u64, _c_void_p]),
    "mcl_autotune": (_i32, [_c_void_p, _c_void_p, _i64, _c_void_p, _i64,
                            ctypes.POINTER(mcl_sensor_params), ctypes.POINTER(mcl_tune_params),
                            ctypes.POINTER(mcl_tune_result), _c_void_p]),
    "mcl_batch_create": (_i32, [ctypes.POINTER(mcl_session_update), _i32,
                                ctypes.POINTER(mcl_batch_params), ctypes.POINTER(_c_void_p)]),
    "mcl_batch_set_offsets": (_i32, [_c_void_p, _c_void_p, _c_void_p]),
    "mcl_batch_run": (_i32, [_c_void_p, _c_void_p]),
    "mcl_batch_get_info": (_i32, [_c_void_p, ctypes.POINTER(mcl_batch_info)]),
    "mcl_batch_destroy": (_i32, [_c_void_p]),
    "mcl_filter_create": (_i32, [ctypes.POINTER(mcl_filter_desc), _c_void_p, ctypes.POINTER(_c_void_p)]),
    "mcl_filter_step": (_i32, [_c_void_p, _c_void_p, _c_void_p, _i64, _c_void_p, _c_void_p]),
    "mcl_filter_reset": (_i32, [_c_void_p, _c_void_p, _c_void_p]),
    "mcl_filter_get_state": (_i32, [_c_void_p, ctypes.POINTER(mcl_filter_state)]),
    "mcl_filter_destroy": (_i32, [_c_void_p]),
    "mcl_server_create": (_i32, [ctypes.POINTER(mcl_server_desc), ctypes.POINTER(_c_void_p)]),
    "mcl_session_open": (_i32, [_c_void_p, ctypes.POINTER(mcl_session_desc), ctypes.POINTER(_c_void_p)]),
    "mcl_submit_scan": (_i32, [_c_void_p, _c_void_p, _i64, _c_void_p, ctypes.POINTER(_u64)]),
    "mcl_wait": (_i32, [_c_void_p, _u64, _i32, ctypes.POINTER(mcl_result)]),
    "mcl_session_read": (_i32, [_c_void_p, _c_void_p, _c_void_p, _i32]),
    "mcl_session_get_info": (_i32, [_c_void_p, ctypes.POINTER(mcl_session_info), _i32]),
    "mcl_session_close": (_i32, [_c_void_p]),
    "mcl_server_get_stats": (_i32, [_c_void_p, _i32, ctypes.POINTER(mcl_server_stats)]),
    "mcl_server_pause": (_i32, [_c_void_p, _i32]),
    "mcl_server_destroy": (_i32, [_c_void_p]),
    "mcl_selftest_wait": (_i32, [ctypes.POINTER(ctypes.c_double), _c_void_p]),
    "mcl_gather_bench": (_i32, [_c_void_p, _i64, _i32, _i32, _i32, _u64, _c_void_p]),
    "mcl_workspace_release": (_i32, [_c_void_p]),
    "mcl_profile_begin": (_i32, []),
    "mcl_profile_end": (_i32, [ctypes.POINTER(mcl_profile)]),
}


def lib():
    """The loaded libmcl.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                                   "(or python -m paper_2310_04172_gb300._build); there is no fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(status: int):
    if status != MCL_OK:
        raise MclError(status, lib().mcl_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype=None, shape_last=None, name="tensor"):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape_last is not None and (t.dim() != 2 or t.shape[1] != shape_last):
        raise ValueError(f"{name} must have shape (n, {shape_last})")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ API (C names)
def mcl_version() -> int:
    return int(lib().mcl_version())


def mcl_sync(stream=None):
    _check(lib().mcl_sync(_stream(stream)))


def mcl_selftest_wait(stream=None) -> float:
    """Runs the bounded-wait failure path on the device; returns the seconds waited."""
    t = ctypes.c_double()
    _check(lib().mcl_selftest_wait(ctypes.byref(t), _stream(stream)))
    return t.value


class Map:
    """Owning handle of a device-resident TSDF map (mcl_map_t)."""

    def __init__(self, handle, desc):
        self.handle = handle
        self.desc = desc

    def info(self) -> dict:
        inf = mcl_map_info(struct_size=ctypes.sizeof(mcl_map_info))
        _check(lib().mcl_map_get_info(self.handle, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in mcl_map_info._fields_ if k != "struct_size"}

    def close(self):
        if self.handle:
            _check(lib().mcl_map_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mcl_map_create(kind: int, dtype: int, origin, voxel: float, truncation: float, dims,
                   values: np.ndarray, brick_coords: np.ndarray | None = None,
                   inv_voxel: float = 0.0, device_layout: int = MCL_LAYOUT_LINEAR,
                   index: int = MCL_INDEX_AUTO) -> Map:
    """Upload a dense or brick TSDF (host arrays) to the current device."""
    values = np.ascontiguousarray(values)
    d = mcl_map_desc(struct_size=ctypes.sizeof(mcl_map_desc), kind=kind, dtype=dtype)
    d.origin[:] = [float(x) for x in origin]
    d.voxel, d.inv_voxel, d.truncation = float(voxel), float(inv_voxel), float(truncation)
    d.dims[:] = [int(x) for x in dims]
    keep = [values]
    if kind == MCL_MAP_BRICK:
        bc = np.ascontiguousarray(brick_coords, np.int32).reshape(-1, 3)
        keep.append(bc)
        d.n_bricks = len(bc)
        d.brick_coords = bc.ctypes.data_as(ctypes.c_void_p)
        d.device_layout = device_layout
        d.index = index
    h = ctypes.c_void_p()
    _check(lib().mcl_map_create(ctypes.byref(d), values.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
    return Map(h, d)


def map_from_scene(m, device_layout: int = MCL_LAYOUT_LINEAR, index: int = MCL_INDEX_AUTO) -> Map:
    """Upload a ``scenes.DenseMap`` / ``scenes.BrickMap`` (input generator objects)."""
    if m.kind == "dense":
        return mcl_map_create(MCL_MAP_DENSE, m.dtype, m.origin, np.float32(m.voxel), np.float32(m.tau),
                              m.dims, m.values, inv_voxel=m.inv_voxel)
    return mcl_map_create(MCL_MAP_BRICK, m.dtype, m.origin, np.float32(m.voxel), np.float32(m.tau),
                          m.dims, m.values, m.coords, inv_voxel=m.inv_voxel,
                          device_layout=device_layout, index=index)


def mcl_map_create_score(m: Map, sigma_hit: float, dtype: int = MCL_F16) -> Map:
    """Score map of `m` for sigma_hit (values exp(-d^2 / (2 sigma^2)), FP16 or FP32)."""
    h = ctypes.c_void_p()
    _check(lib().mcl_map_create_score(m.handle, float(sigma_hit), int(dtype), ctypes.byref(h)))
    return Map(h, ("score", m.desc, float(sigma_hit), int(dtype)))


def mcl_map_destroy(m: Map):
    m.close()


def mcl_map_lookup(m: Map, points, out_index=None, out_value=None, stream=None):
    import torch
    n = points.shape[0]
    if out_index is None:
        out_index = torch.empty(n, dtype=torch.int64, device=points.device)
    if out_value is None:
        out_value = torch.empty(n, dtype=torch.float32, device=points.device)
    _check(lib().mcl_map_lookup(m.handle, _dev_ptr(points, torch.float32, 3, "points"), n,
                                _dev_ptr(out_index, torch.int64, None, "out_index"),
                                _dev_ptr(out_value, torch.float32, None, "out_value"), _stream(stream)))
    return out_index, out_value


def sensor_params(sigma_hit: float = 0.1, mode: int = MCL_LOGPROD, flags: int = 0,
                  points_per_chunk: int = 0, lanes_per_particle: int = 0,
                  particles_per_item: int = 0, unroll: int = 0,
                  pipeline: int = 0, particle_order: int = 0,
                  item_order: int = 0, scan_rings: int = 0) -> mcl_sensor_params:
    return mcl_sensor_params(struct_size=ctypes.sizeof(mcl_sensor_params), sigma_hit=sigma_hit,
                             mode=mode, flags=flags, points_per_chunk=points_per_chunk,
                             lanes_per_particle=lanes_per_particle,
                             particles_per_item=particles_per_item, unroll=unroll,
                             pipeline=pipeline, particle_order=particle_order,
                             item_order=item_order, scan_rings=scan_rings)


def mcl_sensor_update(m: Map, particles, scan, params: mcl_sensor_params, logw=None, w=None,
                      stream=None):
    import torch
    P, N = particles.shape[0], scan.shape[0]
    _check(lib().mcl_sensor_update(m.handle, _dev_ptr(particles, torch.float32, 6, "particles"), P,
                                   _dev_ptr(scan, torch.float32, 3, "scan"), N, ctypes.byref(params),
                                   _dev_ptr(logw, torch.float32, None, "logw"),
                                   _dev_ptr(w, torch.float32, None, "w"), _stream(stream)))
    return logw, w


def estimate_buffer(device=None):
    """Device buffer for one mcl_estimate (uint8 tensor of ESTIMATE_BYTES)."""
    import torch
    return torch.zeros(ESTIMATE_BYTES, dtype=torch.uint8, device=device or "cuda")


def estimate_to_dict(buf) -> dict:
    """Reads an mcl_estimate from a device (or host) buffer into a dict of
    numpy values (synchronises with the buffer's producer through .cpu())."""
    if isinstance(buf, (bytes, bytearray, memoryview)):
        raw = bytes(buf)
    elif hasattr(buf, "cpu"):
        raw = bytes(buf.cpu().numpy().tobytes())
    else:
        raw = bytes(np.asarray(buf).tobytes())
    e = mcl_estimate.from_buffer_copy(raw[:ESTIMATE_BYTES])
    return {
        "weight_sum": e.weight_sum, "n_eff": e.n_eff,
        "mean_pose": np.array(e.mean_pose[:], np.float64), "quat": np.array(e.quat[:], np.float64),
        "rpy": np.array(e.rpy[:], np.float64), "concentration": e.concentration,
        "argmax": int(e.argmax), "best_pose": np.array(e.best_pose[:], np.float32),
        "best_w": float(np.float32(e.best_w)),
    }


def _est_ptr(out):
    import torch
    if out is None:
        return None
    p = _dev_ptr(out, torch.uint8, None, "out")
    if out.numel() < ESTIMATE_BYTES:
        raise ValueError(f"out must hold {ESTIMATE_BYTES} bytes")
    return p


def mcl_pose_estimate(particles, w, out, stream=None):
    import torch
    _check(lib().mcl_pose_estimate(_dev_ptr(particles, torch.float32, 6, "particles"),
                                   _dev_ptr(w, torch.float32, None, "w"), particles.shape[0],
                                   _est_ptr(out), _stream(stream)))
    return out


def mcl_sensor_update_estimate(m: Map, particles, scan, params: mcl_sensor_params, logw, w, out,
                               stream=None):
    import torch
    P, N = particles.shape[0], scan.shape[0]
    _check(lib().mcl_sensor_update_estimate(
        m.handle, _dev_ptr(particles, torch.float32, 6, "particles"), P,
        _dev_ptr(scan, torch.float32, 3, "scan"), N, ctypes.byref(params),
        _dev_ptr(logw, torch.float32, None, "logw"), _dev_ptr(w, torch.float32, None, "w"),
        _est_ptr(out), _stream(stream)))
    return logw, w, out


def mcl_sensor_plan_get(m: Map, P: int, N: int, params: mcl_sensor_params) -> dict:
    pl = mcl_sensor_plan(struct_size=ctypes.sizeof(mcl_sensor_plan))
    _check(lib().mcl_sensor_plan_get(m.handle, P, N, ctypes.byref(params), ctypes.byref(pl)))
    return {k: getattr(pl, k) for k, _ in mcl_sensor_plan._fields_ if k != "struct_size"}


def mcl_normalise(logw, w, out_stats=None, stream=None):
    import torch
    _check(lib().mcl_normalise(_dev_ptr(logw, torch.float32, None, "logw"), logw.shape[0],
                               _dev_ptr(w, torch.float32, None, "w"),
                               _dev_ptr(out_stats, torch.float32, None, "out_stats"), _stream(stream)))
    return w


def mcl_pose_to_matrix(particles, out_mat, stream=None):
    import torch
    _check(lib().mcl_pose_to_matrix(_dev_ptr(particles, torch.float32, 6, "particles"),
                                    particles.shape[0], _dev_ptr(out_mat, torch.float32, 12, "out_mat"),
                                    _stream(stream)))
    return out_mat


def mcl_resample(w, r: float, idx, particles_in=None, particles_out=None, stream=None):
    import torch
    _check(lib().mcl_resample(_dev_ptr(w, torch.float32, None, "w"), w.shape[0], float(r),
                              _dev_ptr(idx, torch.int32, None, "idx"),
                              _dev_ptr(particles_in, torch.float32, 6, "particles_in"),
                              _dev_ptr(particles_out, torch.float32, 6, "particles_out"),
                              _stream(stream)))
    return idx


def mcl_resample_noalloc(w, r: float, idx, particles_in=None, particles_out=None, stream=None):
    """mcl_resample without any device allocation (static scratch, P <= 2^20)."""
    import torch
    _check(lib().mcl_resample_noalloc(_dev_ptr(w, torch.float32, None, "w"), w.shape[0], float(r),
                                      _dev_ptr(idx, torch.int32, None, "idx"),
                                      _dev_ptr(particles_in, torch.float32, 6, "particles_in"),
                                      _dev_ptr(particles_out, torch.float32, 6, "particles_out"),
                                      _stream(stream)))
    return idx


def mcl_motion_update(particles, delta, sigma, seed: int, step: int, stream=None):
    import torch
    d = (ctypes.c_float * 6)(*[float(x) for x in delta])
    s = (ctypes.c_float * 6)(*[float(x) for x in sigma])
    _check(lib().mcl_motion_update(_dev_ptr(particles, torch.float32, 6, "particles"),
                                   particles.shape[0], d, s, int(seed) & (2**64 - 1),
                                   int(step) & (2**64 - 1), _stream(stream)))
    return particles


def mcl_autotune(m: Map, particles, scan, base: mcl_sensor_params, max_particles: int = 0,
                 repeats: int = 0, cache_path: str | None = None, tune_summation: bool = False,
                 stream=None):
    """Tuned launch shape (mcl_sensor_params) and the timing record as a dict."""
    import torch
    tp = mcl_tune_params(struct_size=ctypes.sizeof(mcl_tune_params), max_particles=max_particles,
                         repeats=repeats, use_cache=int(cache_path is not None),
                         tune_summation=int(bool(tune_summation)),
                         cache_path=cache_path.encode() if cache_path else None)
    res = mcl_tune_result(struct_size=ctypes.sizeof(mcl_tune_result))
    _check(lib().mcl_autotune(m.handle, _dev_ptr(particles, torch.float32, 6, "particles"),
                              particles.shape[0], _dev_ptr(scan, torch.float32, 3, "scan"),
                              scan.shape[0], ctypes.byref(base), ctypes.byref(tp), ctypes.byref(res),
                              _stream(stream)))
    best = mcl_sensor_params()
    ctypes.pointer(best)[0] = res.best
    info = {"best_ms": res.best_ms, "default_ms": res.default_ms, "candidates": res.candidates,
            "from_cache": bool(res.from_cache),
            "shape": {k: getattr(res.best, k) for k in ("points_per_chunk", "lanes_per_particle",
                                                         "particles_per_item", "unroll", "pipeline",
                                                         "particle_order", "item_order")}}
    return best, info


class Batch:
    """Owning handle of a batched step plan (mcl_batch_t). `sessions` is a list of
    dicts with keys map, particles, scan, logw, w, and optionally sigma_hit,
    mode, flags, resample_idx, particles_out, estimate (a buffer from
    estimate_buffer()), scan_rings; the CUDA tensors stay referenced."""

    def __init__(self, sessions, points_per_chunk=0, lanes_per_particle=0, particles_per_item=0,
                 unroll=0, pipeline=0, particle_order=0, use_graph=False, item_order=0):
        import torch
        arr = (mcl_session_update * len(sessions))()
        self._keep = []
        for i, s in enumerate(sessions):
            u = arr[i]
            u.struct_size = ctypes.sizeof(mcl_session_update)
            u.map = s["map"].handle
            u.particles = _dev_ptr(s["particles"], torch.float32, 6, "particles")
            u.P = s["particles"].shape[0]
            u.scan = _dev_ptr(s["scan"], torch.float32, 3, "scan")
            u.N = s["scan"].shape[0]
            u.sigma_hit = float(s.get("sigma_hit", 0.1))
            u.mode = int(s.get("mode", MCL_LOGPROD))
            u.flags = int(s.get("flags", 0))
            u.logw = _dev_ptr(s.get("logw"), torch.float32, None, "logw")
            u.w = _dev_ptr(s.get("w"), torch.float32, None, "w")
            u.resample_idx = _dev_ptr(s.get("resample_idx"), torch.int32, None, "resample_idx")
            u.particles_out = _dev_ptr(s.get("particles_out"), torch.float32, 6, "particles_out")
            u.estimate = _est_ptr(s.get("estimate"))
            u.scan_rings = int(s.get("scan_rings", 0))
            self._keep.append(s)
        bp = mcl_batch_params(struct_size=ctypes.sizeof(mcl_batch_params),
                              points_per_chunk=points_per_chunk, lanes_per_particle=lanes_per_particle,
                              particles_per_item=particles_per_item, unroll=unroll, pipeline=pipeline,
                              particle_order=particle_order, use_graph=int(bool(use_graph)),
                              item_order=item_order)
        h = ctypes.c_void_p()
        _check(lib().mcl_batch_create(arr, len(sessions), ctypes.byref(bp), ctypes.byref(h)))
        self.handle = h
        self.n = len(sessions)

    def set_offsets(self, r, stream=None):
        buf = np.ascontiguousarray(r, np.float64)
        if buf.shape != (self.n,):
            raise ValueError(f"need {self.n} offsets")
        _check(lib().mcl_batch_set_offsets(self.handle, buf.ctypes.data_as(ctypes.c_void_p),
                                           _stream(stream)))
        self._r = buf  # the copy may still read the host buffer

    def run(self, stream=None):
        _check(lib().mcl_batch_run(self.handle, _stream(stream)))

    def info(self) -> dict:
        inf = mcl_batch_info(struct_size=ctypes.sizeof(mcl_batch_info))
        _check(lib().mcl_batch_get_info(self.handle, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in mcl_batch_info._fields_ if k != "struct_size"}

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().mcl_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mcl_batch_create(sessions, **kw) -> Batch:
    return Batch(sessions, **kw)


def mcl_batch_run(batch: Batch, stream=None):
    batch.run(stream)


def mcl_batch_set_offsets(batch: Batch, r, stream=None):
    batch.set_offsets(r, stream)


def mcl_batch_get_info(batch: Batch) -> dict:
    return batch.info()


def mcl_batch_destroy(batch: Batch):
    batch.close()


MCL_RESULT_DONE, MCL_RESULT_SUPERSEDED, MCL_RESULT_CLOSED = 0, 1, 2


class Filter:
    """Owning handle of a device-resident particle filter (mcl_filter_t): one
    call runs motion update, sensor update with pose estimate and resampling.
    `particles` is a CUDA float32 (P, 6) tensor (copied)."""

    def __init__(self, m: Map, particles, max_points: int, params: mcl_sensor_params = None,
                 motion_sigma=(0.0,) * 6, seed: int = 0, use_graph: bool = True,
                 max_graphs: int = 0, first_step: int = 0):
        import torch
        d = mcl_filter_desc(struct_size=ctypes.sizeof(mcl_filter_desc), map=m.handle,
                            P=particles.shape[0], max_points=int(max_points),
                            sensor=params if params is not None else sensor_params(),
                            seed=int(seed), use_graph=int(bool(use_graph)), max_graphs=max_graphs,
                            first_step=int(first_step))
        for k in range(6):
            d.motion_sigma[k] = float(motion_sigma[k])
        h = ctypes.c_void_p()
        _check(lib().mcl_filter_create(ctypes.byref(d), _dev_ptr(particles, torch.float32, 6, "particles"),
                                       ctypes.byref(h)))
        self.handle = h
        self.map = m
        self.P = particles.shape[0]

    def step(self, scan, delta=None, out=None, stream=None):
        import torch
        dv = None
        if delta is not None:
            dv = (ctypes.c_float * 6)(*[float(x) for x in np.asarray(delta, np.float32).reshape(6)])
        _check(lib().mcl_filter_step(self.handle, dv, _dev_ptr(scan, torch.float32, 3, "scan"),
                                     scan.shape[0], _est_ptr(out), _stream(stream)))
        return out

    def reset(self, particles, stream=None):
        import torch
        _check(lib().mcl_filter_reset(self.handle, _dev_ptr(particles, torch.float32, 6, "particles"),
                                      _stream(stream)))

    def state(self) -> dict:
        st = mcl_filter_state(struct_size=ctypes.sizeof(mcl_filter_state))
        _check(lib().mcl_filter_get_state(self.handle, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in mcl_filter_state._fields_ if k != "struct_size"}

    def tensors(self) -> dict:
        """Torch views of the filter's device arrays (no copy; valid while the
        filter lives; read them after the stream's work finished)."""
        import torch
        st = self.state()
        P = self.P
        out = {name: _device_view(st[name], shape, dt)
               for name, shape, dt in (("particles", (P, 6), torch.float32), ("logw", (P,), torch.float32),
                                       ("w", (P,), torch.float32), ("idx", (P,), torch.int32))}
        out["estimate"] = _device_view(st["estimate"], (ESTIMATE_BYTES,), torch.uint8)
        return out

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().mcl_filter_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _device_view(ptr: int, shape, dtype):
    """A torch tensor viewing device memory owned by the library (no copy),
    through the CUDA array interface."""
    import torch
    typestr = {torch.float32: "<f4", torch.int32: "<i4", torch.uint8: "|u1"}[dtype]

    class _Iface:
        __cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                    "data": (int(ptr), False), "version": 3, "strides": None}
    return torch.as_tensor(_Iface(), device="cuda")


def mcl_filter_create(m: Map, particles, max_points: int, **kw) -> Filter:
    return Filter(m, particles, max_points, **kw)


def mcl_filter_step(f: Filter, scan, delta=None, out=None, stream=None):
    return f.step(scan, delta, out, stream)


def mcl_filter_reset(f: Filter, particles, stream=None):
    f.reset(particles, stream)


def mcl_filter_get_state(f: Filter) -> dict:
    return f.state()


def mcl_filter_destroy(f: Filter):
    f.close()


class Server:
    """Serving loop handle (mcl_server_t): device-resident sessions, continuous batching."""

    def __init__(self, hbm_budget_bytes: int, max_sessions: int, max_in_flight: int = 2,
                 max_batch: int = 0, **shape):
        d = mcl_server_desc(struct_size=ctypes.sizeof(mcl_server_desc),
                            hbm_budget_bytes=int(hbm_budget_bytes), max_sessions=max_sessions,
                            max_in_flight=max_in_flight, max_batch=max_batch)
        d.shape = mcl_batch_params(struct_size=ctypes.sizeof(mcl_batch_params), **shape)
        h = ctypes.c_void_p()
        _check(lib().mcl_server_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h

    def open(self, m: Map, particles: np.ndarray, max_N: int, sigma_hit: float = 0.1,
             mode: int = MCL_LOGPROD, flags: int = 0, motion_sigma=(0,) * 6, seed: int = 0,
             first_step: int = 0, scan_rings: int = 0):
        parts = np.ascontiguousarray(particles, np.float32).reshape(-1, 6)
        d = mcl_session_desc(struct_size=ctypes.sizeof(mcl_session_desc), map=m.handle, P=len(parts),
                             max_N=int(max_N), particles=parts.ctypes.data_as(ctypes.c_void_p),
                             sigma_hit=sigma_hit, mode=mode, flags=flags, seed=int(seed),
                             first_step=int(first_step), scan_rings=int(scan_rings))
        d.motion_sigma[:] = [float(x) for x in motion_sigma]
        h = ctypes.c_void_p()
        _check(lib().mcl_session_open(self.handle, ctypes.byref(d), ctypes.byref(h)))
        return Session(self, h, len(parts))

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        r = mcl_result(struct_size=ctypes.sizeof(mcl_result))
        _check(lib().mcl_wait(self.handle, int(ticket), int(timeout_ms), ctypes.byref(r)))
        out = {"status": r.status, "latency_ms": r.latency_ms, "evals": r.evals, "step": r.step}
        if r.status == MCL_RESULT_DONE:
            out["estimate"] = estimate_to_dict(bytes(r.estimate))
        return out

    def stats(self, reset: bool = False) -> dict:
        st = mcl_server_stats(struct_size=ctypes.sizeof(mcl_server_stats))
        _check(lib().mcl_server_get_stats(self.handle, int(bool(reset)), ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in mcl_server_stats._fields_ if k != "struct_size"}

    def pause(self, on: bool = True):
        _check(lib().mcl_server_pause(self.handle, int(bool(on))))

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().mcl_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Session:
    def __init__(self, server: Server, handle, P: int):
        self.server, self.handle, self.P = server, handle, P

    def submit(self, scan: np.ndarray, delta=None) -> int:
        sc = np.ascontiguousarray(scan, np.float32).reshape(-1, 3)
        dl = None if delta is None else np.ascontiguousarray(delta, np.float32).reshape(6)
        t = ctypes.c_uint64()
        _check(lib().mcl_submit_scan(self.handle, sc.ctypes.data_as(ctypes.c_void_p), len(sc),
                                     None if dl is None else dl.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(t)))
        return t.value

    def info(self, timeout_ms: int = -1) -> dict:
        st = mcl_session_info(struct_size=ctypes.sizeof(mcl_session_info))
        _check(lib().mcl_session_get_info(self.handle, ctypes.byref(st), int(timeout_ms)))
        return {k: getattr(st, k) for k, _ in mcl_session_info._fields_ if k != "struct_size"}

    def read(self, timeout_ms: int = -1):
        parts = np.empty((self.P, 6), np.float32)
        w = np.empty(self.P, np.float32)
        _check(lib().mcl_session_read(self.handle, parts.ctypes.data_as(ctypes.c_void_p),
                                      w.ctypes.data_as(ctypes.c_void_p), int(timeout_ms)))
        return parts, w

    def close(self):
        if self.handle:
            _check(lib().mcl_session_close(self.handle))
            self.handle = None


def mcl_server_create(hbm_budget_bytes, max_sessions, **kw) -> Server:
    return Server(hbm_budget_bytes, max_sessions, **kw)


def mcl_session_open(server: Server, m: Map, particles, max_N, **kw) -> Session:
    return server.open(m, particles, max_N, **kw)


def mcl_submit_scan(session: Session, scan, delta=None) -> int:
    return session.submit(scan, delta)


def mcl_wait(server: Server, ticket: int, timeout_ms: int = -1) -> dict:
    return server.wait(ticket, timeout_ms)


def mcl_session_read(session: Session, timeout_ms: int = -1):
    return session.read(timeout_ms)


def mcl_session_get_info(session: Session, timeout_ms: int = -1) -> dict:
    return session.info(timeout_ms)


def mcl_session_close(session: Session):
    session.close()


def mcl_server_get_stats(server: Server, reset: bool = False) -> dict:
    return server.stats(reset)


def mcl_server_pause(server: Server, on: bool = True):
    server.pause(on)


def mcl_server_destroy(server: Server):
    server.close()


def mcl_gather_bench(buf, blocks: int, iters: int, seed: int = 1, stream=None) -> int:
    """Launch the gather microbenchmark over a CUDA tensor (int16/float16 or float32
    elements); returns the number of gathers issued."""
    es = buf.element_size()
    _check(lib().mcl_gather_bench(_dev_ptr(buf, None, None, "buf"), buf.numel(), es, int(blocks),
                                  int(iters), int(seed), _stream(stream)))
    return int(blocks) * 256 * int(iters) * 8


def mcl_workspace_release(stream=None):
    _check(lib().mcl_workspace_release(_stream(stream)))


def mcl_profile_begin():
    _check(lib().mcl_profile_begin())


def mcl_profile_end() -> dict:
    p = mcl_profile(struct_size=ctypes.sizeof(mcl_profile))
    _check(lib().mcl_profile_end(ctypes.byref(p)))
    return {name: {"launches": int(p.launches[i]), "ms": float(p.ms[i])}
            for i, name in enumerate(PHASES)}
