"""Thin ctypes binding of the C ABI in ``include/contact_manifold.h``.

Functions keep the C names and only marshal arguments: torch tensors are
passed as raw device pointers, the stream as the torch stream's handle.  Every
step of the manifold runs in the CUDA library; there is no Python or CPU
compute path, and importing this module fails if the library is not built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libcontact_manifold.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(
        f"{_LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")

_lib = ctypes.CDLL(_LIB_PATH)

CM_OK, CM_ERR_INVALID_ARG, CM_ERR_OOM, CM_ERR_CUDA = 0, 1, 2, 3
CM_ERR_ADMISSION, CM_ERR_TIMEOUT, CM_ERR_NOT_FOUND, CM_ERR_DEVICE = 4, 5, 6, 7
CM_BOX, CM_CAPSULE, CM_CYLINDER, CM_ELLIPSOID, CM_HULL, CM_SQ_UNION = 0, 1, 2, 3, 4, 5
CM_FLAG_NO_EE, CM_FLAG_ONE_SIDED, CM_FLAG_HARD = 1, 2, 4
CM_MAX_K = 16


class cm_geometry_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dims", ctypes.c_float * 3),
                ("n_verts", ctypes.c_int32), ("verts", ctypes.POINTER(ctypes.c_float)),
                ("n_edges", ctypes.c_int32), ("edges", ctypes.POINTER(ctypes.c_int32)),
                ("n_planes", ctypes.c_int32), ("planes", ctypes.POINTER(ctypes.c_float))]


class cm_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("w_reg", ctypes.c_float), ("eps_clip", ctypes.c_float),
                ("eps_min", ctypes.c_float), ("eps_comp", ctypes.c_float), ("K", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("top_verts", ctypes.c_int32), ("top_edges", ctypes.c_int32),
                ("trace_iters", ctypes.c_int32)]


class cm_geometry_info(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dims", ctypes.c_float * 3), ("n_verts", ctypes.c_int32),
                ("n_edges", ctypes.c_int32), ("n_planes", ctypes.c_int32)]


class cm_request_desc(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int32), ("with_backward", ctypes.c_int32),
                ("pair_geoms", ctypes.c_void_p), ("poses", ctypes.c_void_p), ("dims", ctypes.c_void_p),
                ("tau", ctypes.c_void_p), ("grad_out", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("grad_poses", ctypes.c_void_p), ("grad_dims", ctypes.c_void_p)]


_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_SIGS = {
    "cm_default_params": (None, [ctypes.POINTER(cm_params)]),
    "cm_last_error": (ctypes.c_char_p, []),
    "cm_create_context": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "cm_destroy_context": (None, [_vp]),
    "cm_create_geometry": (ctypes.c_int, [_vp, ctypes.POINTER(cm_geometry_desc),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "cm_sync_geometry": (ctypes.c_int, [_vp]),
    "cm_destroy_geometry": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "cm_num_geometries": (ctypes.c_int32, [_vp]),
    "cm_create_hull_geometry": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "cm_get_geometry": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(cm_geometry_info), _vp, _vp, _vp]),
    "cm_create_primitive_geometry": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_float),
                                                    ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "cm_check_device_error": (ctypes.c_int, [_vp]),
    "cm_contact_manifold_fwd": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp,
                                               ctypes.POINTER(cm_params), _vp, _vp]),
    "cm_contact_manifold_bwd": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp,
                                               ctypes.POINTER(cm_params), _vp, _vp, _vp, _vp]),
    "cm_contact_manifold_fwd_noalloc": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp,
                                                       ctypes.POINTER(cm_params), _vp, _vp]),
    "cm_saved_stride": (ctypes.c_int, [_vp, ctypes.POINTER(cm_params), ctypes.POINTER(ctypes.c_int64)]),
    "cm_candidate_offsets": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.POINTER(cm_params), _vp]),
    "cm_contact_manifold_fwd_dump": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp,
                                                    ctypes.POINTER(cm_params), _vp, _vp, ctypes.c_int64, _vp, _vp]),
    "cm_contact_manifold_fwd_save": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp,
                                                    ctypes.POINTER(cm_params), _vp, _vp, ctypes.c_int64, _vp]),
    "cm_contact_manifold_bwd_saved": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp,
                                                     ctypes.POINTER(cm_params), _vp, ctypes.c_int64, _vp, _vp,
                                                     _vp, _vp]),
    "cm_autotune": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.POINTER(cm_params),
                                   _vp, _vp, _vp, _vp, _vp]),
    "cm_get_launch_shape": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32)]),
    "cm_plan_create": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.POINTER(cm_params),
                                      _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "cm_plan_launch": (ctypes.c_int, [_vp, _vp]),
    "cm_plan_destroy": (None, [_vp]),
    "cm_server_start": (ctypes.c_int, [_vp, ctypes.POINTER(cm_params), ctypes.c_int32, ctypes.c_int32]),
    "cm_submit": (ctypes.c_int, [_vp, ctypes.POINTER(cm_request_desc), ctypes.POINTER(_u64)]),
    "cm_poll": (ctypes.c_int, [_vp, _u64, ctypes.POINTER(ctypes.c_int32)]),
    "cm_wait": (ctypes.c_int, [_vp, _u64, ctypes.c_int32]),
    "cm_request_latency": (ctypes.c_int, [_vp, _u64, ctypes.POINTER(ctypes.c_double)]),
    "cm_release": (ctypes.c_int, [_vp, _u64]),
    "cm_server_stats": (ctypes.c_int, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "cm_server_stop": (ctypes.c_int, [_vp]),
    "cm_ee_witness_batch": (ctypes.c_int, [ctypes.c_int32, _vp, ctypes.POINTER(cm_params), _vp, _vp]),
    "cm_vf_witness_batch": (ctypes.c_int, [ctypes.c_int32, _vp, ctypes.POINTER(cm_params), _vp, _vp]),
    "cm_measure_pipe_peaks": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_double)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class CMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def _check(status):
    if status != CM_OK:
        raise CMError(status, cm_last_error())


def cm_last_error() -> str:
    return _lib.cm_last_error().decode()


def cm_default_params(**overrides) -> cm_params:
    p = cm_params()
    _lib.cm_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def cm_create_context(device: int = 0, hbm_budget_bytes: int = 0):
    h = _vp()
    _check(_lib.cm_create_context(device, hbm_budget_bytes, ctypes.byref(h)))
    return h


def cm_destroy_context(ctx) -> None:
    _lib.cm_destroy_context(ctx)


def cm_create_geometry(ctx, kind, dims, verts, edges, planes=None) -> int:
    v = np.ascontiguousarray(verts, dtype=np.float32)
    e = np.ascontiguousarray(edges, dtype=np.int32)
    p = None if planes is None or len(planes) == 0 else np.ascontiguousarray(planes, dtype=np.float32)
    d = cm_geometry_desc()
    d.kind = int(kind)
    for i in range(3):
        d.dims[i] = float(dims[i])
    d.n_verts = int(v.shape[0])
    d.verts = v.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    d.n_edges = int(e.shape[0])
    d.edges = e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    d.n_planes = 0 if p is None else int(p.shape[0])
    d.planes = None if p is None else p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    gid = ctypes.c_int32()
    _check(_lib.cm_create_geometry(ctx, ctypes.byref(d), ctypes.byref(gid)))
    return gid.value


def cm_sync_geometry(ctx) -> None:
    _check(_lib.cm_sync_geometry(ctx))


def cm_destroy_geometry(ctx, geom_id) -> None:
    _check(_lib.cm_destroy_geometry(ctx, int(geom_id)))


def cm_num_geometries(ctx) -> int:
    return int(_lib.cm_num_geometries(ctx))


def cm_create_hull_geometry(ctx, points) -> int:
    """Registers the convex hull of ``points`` ((n, 3), converted to float64) and returns its id."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    if pts.ndim != 2 or pts.shape[1] != 3:
        raise ValueError("points must have shape (n, 3)")
    gid = ctypes.c_int32()
    _check(_lib.cm_create_hull_geometry(ctx, pts.ctypes.data, int(pts.shape[0]), ctypes.byref(gid)))
    return gid.value


def cm_create_primitive_geometry(ctx, kind, dims, tess=0) -> int:
    """Registers a primitive whose mesh the library generates at resolution ``tess``."""
    d = (ctypes.c_float * 3)(*[float(x) for x in dims])
    gid = ctypes.c_int32()
    _check(_lib.cm_create_primitive_geometry(ctx, int(kind), d, int(tess), ctypes.byref(gid)))
    return gid.value


def cm_get_geometry(ctx, geom_id) -> dict:
    """A registered geometry as the library holds it: kind, dims, verts (V, 4), edges (E, 2),
    planes (F, 4; hulls only)."""
    info = cm_geometry_info()
    _check(_lib.cm_get_geometry(ctx, int(geom_id), ctypes.byref(info), None, None, None))
    v = np.zeros((info.n_verts, 4), dtype=np.float32)
    e = np.zeros((info.n_edges, 2), dtype=np.int32)
    p = np.zeros((info.n_planes, 4), dtype=np.float32)
    _check(_lib.cm_get_geometry(ctx, int(geom_id), ctypes.byref(info), v.ctypes.data, e.ctypes.data,
                                p.ctypes.data if info.n_planes else None))
    return {"kind": int(info.kind), "dims": np.array(list(info.dims), dtype=np.float32),
            "verts": v, "edges": e, "planes": p}


def cm_check_device_error(ctx) -> None:
    _check(_lib.cm_check_device_error(ctx))


def _ptr(t):
    return None if t is None else _vp(t.data_ptr())


def _stream_handle(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return _vp(s.cuda_stream)


def _check_tensor(t, name, dtype, shape0):
    import torch
    if t is None:
        return
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if t.shape[0] != shape0:
        raise ValueError(f"{name} has {t.shape[0]} rows, expected {shape0}")
    del torch


def cm_contact_manifold_fwd(ctx, pair_geoms, poses, dims, tau, params, out, stream=None) -> None:
    """Launch the forward manifold on torch CUDA tensors (see the C header for layouts)."""
    import torch
    n = int(pair_geoms.shape[0])
    _check_tensor(pair_geoms, "pair_geoms", torch.int32, n)
    _check_tensor(poses, "poses", torch.float32, n)
    _check_tensor(dims, "dims", torch.float32, n)
    _check_tensor(tau, "tau", torch.float32, n)
    _check_tensor(out, "out", torch.float32, n)
    _check(_lib.cm_contact_manifold_fwd(ctx, n, _ptr(pair_geoms), _ptr(poses), _ptr(dims), _ptr(tau),
                                        ctypes.byref(params), _ptr(out), _stream_handle(stream)))


def cm_contact_manifold_bwd(ctx, pair_geoms, poses, dims, tau, params, grad_out, grad_poses, grad_dims,
                            stream=None) -> None:
    """Launch the adjoint on torch CUDA tensors (see the C header for layouts)."""
    import torch
    n = int(pair_geoms.shape[0])
    _check_tensor(pair_geoms, "pair_geoms", torch.int32, n)
    _check_tensor(poses, "poses", torch.float32, n)
    _check_tensor(dims, "dims", torch.float32, n)
    _check_tensor(tau, "tau", torch.float32, n)
    _check_tensor(grad_out, "grad_out", torch.float32, n)
    _check_tensor(grad_poses, "grad_poses", torch.float32, n)
    _check_tensor(grad_dims, "grad_dims", torch.float32, n)
    _check(_lib.cm_contact_manifold_bwd(ctx, n, _ptr(pair_geoms), _ptr(poses), _ptr(dims), _ptr(tau),
                                        ctypes.byref(params), _ptr(grad_out), _ptr(grad_poses),
                                        _ptr(grad_dims), _stream_handle(stream)))


def cm_candidate_offsets(ctx, pair_geoms, params):
    """(n + 1,) int64 first candidate row of each pair (host numpy ids (n, 2) in)."""
    import numpy as np
    pg = np.ascontiguousarray(pair_geoms, dtype=np.int32)
    off = np.zeros(pg.shape[0] + 1, dtype=np.int64)
    _check(_lib.cm_candidate_offsets(ctx, int(pg.shape[0]), pg.ctypes.data, ctypes.byref(params), off.ctypes.data))
    return off


def cm_contact_manifold_fwd_dump(ctx, pair_geoms, poses, dims, tau, params, out, candidates, offsets,
                                 stream=None) -> None:
    """Forward manifold that also writes every candidate row (rows, 8) at ``offsets`` (device int64)."""
    import torch
    n = int(pair_geoms.shape[0])
    _check_tensor(pair_geoms, "pair_geoms", torch.int32, n)
    _check_tensor(poses, "poses", torch.float32, n)
    _check_tensor(dims, "dims", torch.float32, n)
    _check_tensor(tau, "tau", torch.float32, n)
    _check_tensor(out, "out", torch.float32, n)
    _check_tensor(offsets, "candidate_offsets", torch.int64, n + 1)
    if not candidates.is_cuda or candidates.dtype != torch.float32 or not candidates.is_contiguous():
        raise ValueError("candidates must be a contiguous CUDA float32 tensor")
    _check(_lib.cm_contact_manifold_fwd_dump(ctx, n, _ptr(pair_geoms), _ptr(poses), _ptr(dims), _ptr(tau),
                                             ctypes.byref(params), _ptr(out), _ptr(candidates),
                                             int(candidates.numel() // 8), _ptr(offsets), _stream_handle(stream)))


def cm_saved_stride(ctx, params) -> int:
    """Floats per pair of the forward's record for the adjoint (cm_contact_manifold_fwd_save)."""
    v = ctypes.c_int64()
    _check(_lib.cm_saved_stride(ctx, ctypes.byref(params), ctypes.byref(v)))
    return int(v.value)


def cm_contact_manifold_fwd_save(ctx, pair_geoms, poses, dims, tau, params, out, saved, stream=None) -> None:
    """Forward manifold that also writes each pair's record for the adjoint into ``saved``
    ((n, stride) float32, stride >= cm_saved_stride)."""
    import torch
    n = int(pair_geoms.shape[0])
    _check_tensor(pair_geoms, "pair_geoms", torch.int32, n)
    _check_tensor(poses, "poses", torch.float32, n)
    _check_tensor(dims, "dims", torch.float32, n)
    _check_tensor(tau, "tau", torch.float32, n)
    _check_tensor(out, "out", torch.float32, n)
    _check_tensor(saved, "saved", torch.float32, n)
    _check(_lib.cm_contact_manifold_fwd_save(ctx, n, _ptr(pair_geoms), _ptr(poses), _ptr(dims), _ptr(tau),
                                             ctypes.byref(params), _ptr(out), _ptr(saved),
                                             int(saved.shape[1]) if saved.dim() == 2 else 0,
                                             _stream_handle(stream)))


def cm_contact_manifold_bwd_saved(ctx, pair_geoms, poses, dims, tau, params, saved, grad_out, grad_poses,
                                  grad_dims, stream=None) -> None:
    """Adjoint from the records a cm_contact_manifold_fwd_save call wrote for the same inputs."""
    import torch
    n = int(pair_geoms.shape[0])
    _check_tensor(pair_geoms, "pair_geoms", torch.int32, n)
    _check_tensor(poses, "poses", torch.float32, n)
    _check_tensor(dims, "dims", torch.float32, n)
    _check_tensor(tau, "tau", torch.float32, n)
    _check_tensor(saved, "saved", torch.float32, n)
    _check_tensor(grad_out, "grad_out", torch.float32, n)
    _check_tensor(grad_poses, "grad_poses", torch.float32, n)
    _check_tensor(grad_dims, "grad_dims", torch.float32, n)
    _check(_lib.cm_contact_manifold_bwd_saved(ctx, n, _ptr(pair_geoms), _ptr(poses), _ptr(dims), _ptr(tau),
                                              ctypes.byref(params), _ptr(saved),
                                              int(saved.shape[1]) if saved.dim() == 2 else 0, _ptr(grad_out),
                                              _ptr(grad_poses), _ptr(grad_dims), _stream_handle(stream)))


def cm_contact_manifold_fwd_noalloc(ctx, pair_geoms, poses, dims, tau, params, out, stream=None) -> None:
    """Allocation-free variant of cm_contact_manifold_fwd (fixed in-library scratch)."""
    import torch
    n = int(pair_geoms.shape[0])
    _check_tensor(pair_geoms, "pair_geoms", torch.int32, n)
    _check_tensor(poses, "poses", torch.float32, n)
    _check_tensor(dims, "dims", torch.float32, n)
    _check_tensor(tau, "tau", torch.float32, n)
    _check_tensor(out, "out", torch.float32, n)
    _check(_lib.cm_contact_manifold_fwd_noalloc(ctx, n, _ptr(pair_geoms), _ptr(poses), _ptr(dims), _ptr(tau),
                                                ctypes.byref(params), _ptr(out), _stream_handle(stream)))


def cm_autotune(ctx, pair_geoms, poses, dims, tau, params, out, grad_out=None, grad_poses=None,
                grad_dims=None, stream=None) -> None:
    """Pick and remember the fastest launch shape for this batch (see the C header)."""
    n = int(pair_geoms.shape[0])
    _check(_lib.cm_autotune(ctx, n, _ptr(pair_geoms), _ptr(poses), _ptr(dims), _ptr(tau), ctypes.byref(params),
                            _ptr(out), _ptr(grad_out), _ptr(grad_poses), _ptr(grad_dims), _stream_handle(stream)))


def cm_get_launch_shape(ctx, n_pairs, backward=False, flags=0):
    b, p, o = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.cm_get_launch_shape(ctx, n_pairs, int(backward), flags, ctypes.byref(b), ctypes.byref(p),
                                    ctypes.byref(o)))
    return b.value, p.value, o.value


def cm_plan_create(ctx, pair_geoms, poses, dims, tau, params, out, grad_out=None, grad_poses=None,
                   grad_dims=None):
    """Capture the step of this batch in a CUDA graph; returns the plan handle."""
    h = _vp()
    n = int(pair_geoms.shape[0])
    _check(_lib.cm_plan_create(ctx, n, _ptr(pair_geoms), _ptr(poses), _ptr(dims), _ptr(tau), ctypes.byref(params),
                               _ptr(out), _ptr(grad_out), _ptr(grad_poses), _ptr(grad_dims), ctypes.byref(h)))
    return h


def cm_plan_launch(plan, stream=None) -> None:
    _check(_lib.cm_plan_launch(plan, _stream_handle(stream)))


def cm_plan_destroy(plan) -> None:
    _lib.cm_plan_destroy(plan)


_KEEPALIVE = {}


def _host_ptr(a):
    """Address of a host buffer: a CPU torch tensor or a numpy array (kept alive by the caller)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("request buffers must be contiguous host tensors")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("request buffers must be C-contiguous")
    return a.ctypes.data


def cm_server_start(ctx, params, max_batch_pairs=65536, n_streams=4) -> None:
    _check(_lib.cm_server_start(ctx, ctypes.byref(params), max_batch_pairs, n_streams))


def cm_submit(ctx, pair_geoms, poses, out, dims=None, tau=None, grad_out=None, grad_poses=None,
              grad_dims=None) -> int:
    """Queue a request on host buffers; returns its ticket.  The buffers are kept alive
    by this module until cm_release."""
    d = cm_request_desc()
    d.n_pairs = int(pair_geoms.shape[0])
    d.with_backward = 1 if grad_out is not None else 0
    d.pair_geoms, d.poses, d.dims, d.tau = (_host_ptr(pair_geoms), _host_ptr(poses), _host_ptr(dims),
                                            _host_ptr(tau))
    d.grad_out, d.out, d.grad_poses, d.grad_dims = (_host_ptr(grad_out), _host_ptr(out), _host_ptr(grad_poses),
                                                    _host_ptr(grad_dims))
    t = _u64()
    _check(_lib.cm_submit(ctx, ctypes.byref(d), ctypes.byref(t)))
    _KEEPALIVE[(ctx.value, t.value)] = (pair_geoms, poses, out, dims, tau, grad_out, grad_poses, grad_dims)
    return t.value


def cm_poll(ctx, ticket) -> bool:
    done = ctypes.c_int32()
    _check(_lib.cm_poll(ctx, ticket, ctypes.byref(done)))
    return bool(done.value)


def cm_wait(ctx, ticket, timeout_ms=-1) -> None:
    """Block until the request is done; timeout_ms < 0 waits for ever."""
    while True:
        st = _lib.cm_wait(ctx, ticket, 1000 if timeout_ms < 0 else timeout_ms)
        if st == CM_ERR_TIMEOUT and timeout_ms < 0:
            continue
        _check(st)
        return


def cm_request_latency(ctx, ticket) -> float:
    v = ctypes.c_double()
    _check(_lib.cm_request_latency(ctx, ticket, ctypes.byref(v)))
    return v.value


def cm_release(ctx, ticket) -> None:
    _check(_lib.cm_release(ctx, ticket))
    _KEEPALIVE.pop((ctx.value, ticket), None)


def cm_server_stats(ctx):
    a, b, c = _u64(), _u64(), _u64()
    _check(_lib.cm_server_stats(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def cm_server_stop(ctx) -> None:
    _check(_lib.cm_server_stop(ctx))
    for k in [k for k in _KEEPALIVE if k[0] == ctx.value]:
        _KEEPALIVE.pop(k)


def cm_ee_witness_batch(queries, params, out, stream=None) -> None:
    """Edge-edge witness points of n queries (n, 12) -> out (n, 8) on the current device."""
    _check(_lib.cm_ee_witness_batch(int(queries.shape[0]), _ptr(queries), ctypes.byref(params), _ptr(out),
                                    _stream_handle(stream)))


def cm_vf_witness_batch(queries, params, out, stream=None) -> None:
    """Vertex-triangle witness points of n queries (n, 12) -> out (n, 4) on the current device."""
    _check(_lib.cm_vf_witness_batch(int(queries.shape[0]), _ptr(queries), ctypes.byref(params), _ptr(out),
                                    _stream_handle(stream)))


def cm_measure_pipe_peaks(device: int = 0):
    """(FP32 FMA flop/s, MUFU ex2 op/s) measured on ``device``."""
    f, m = ctypes.c_double(), ctypes.c_double()
    _check(_lib.cm_measure_pipe_peaks(device, ctypes.byref(f), ctypes.byref(m)))
    return f.value, m.value


def exported_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return sorted(_SIGS)
