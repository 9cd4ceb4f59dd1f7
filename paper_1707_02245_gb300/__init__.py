"""Python binding of the GB300 PDHG photoacoustic reconstruction library (C ABI: include/pat.h).

Argument marshalling only: every step of the reconstruction runs in the CUDA library
``_lib/libpat_pdhg.so`` (build it with ``paper_1707_02245_gb300.build.build()``).  The
functions below carry the C names and take device pointers as integers or as objects
with a ``data_ptr()`` method (e.g. torch CUDA tensors); streams are ``cudaStream_t``
handles as integers (0 = default stream) or objects with a ``cuda_stream`` attribute.

There is no CPU fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

PAT_OK = 0
PAT_ERR_INVALID_ARG = -1
PAT_ERR_CUDA = -2
PAT_ERR_OOM = -3
PAT_ERR_NONFINITE = -4
PAT_ERR_TIMEOUT = -5

PAT_TV, PAT_TGV, PAT_DTV, PAT_WAV = 0, 1, 2, 3
PAT_PRECOND_DIAG, PAT_PRECOND_SCALAR2 = 0, 1
PAT_STATUS_CONVERGED, PAT_STATUS_MAXITER, PAT_STATUS_DIVERGED = 0, 1, 2
PAT_ADAPT_NONE, PAT_ADAPT_BALANCE = 0, 1

EXPORTED = [
    "pat_create_geometry", "pat_destroy_geometry", "pat_forward", "pat_adjoint",
    "pat_direction_field", "pat_params_default", "pat_reconstruct", "pat_reconstruct_batched",
    "pat_steps", "pat_duality_gap", "pat_error_string", "pat_last_error", "pat_geometry_info",
    "pat_adjoint_worklist",
    "pat_profile_enable", "pat_profile_read", "pat_kernel_launches", "pat_adjoint_noalloc",
    "pat_tune_step_ratio", "pat_tune_step_ratio_batched", "pat_preprocess", "pat_wavelet_transform",
    "pat_dtcwt_transform",
    "pat_time_phases", "pat_forward_plan", "pat_geometry_set_shapes", "pat_geometry_get_shapes", "pat_tune_shapes",
    # learned warm start (include/pat_unet.h)
    "pat_conv3x3_forward", "pat_conv3x3_backward_data", "pat_conv3x3_backward_weight", "pat_nn_wait_timeouts",
    "pat_unet_create", "pat_unet_destroy", "pat_unet_num_params", "pat_unet_get_params",
    "pat_unet_set_params", "pat_unet_forward", "pat_unet_backward", "pat_unet_train_step",
    "pat_warm_start_features", "pat_warm_start_state", "pat_warm_start_target", "pat_warm_start",
]
PAT_WARM_CHANNELS = 8
PAT_WARM_V_SCALE = 10.0
PHASES = ["forward_prox", "adj_clear", "adjoint", "update", "gap"]


class PatError(RuntimeError):
    def __init__(self, code: int, where: str, message: str):
        super().__init__(f"{where}: {message} (code {code})")
        self.code = code


class pat_geometry_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("ymin", ctypes.c_double), ("ymax", ctypes.c_double), ("n_det", ctypes.c_int),
                ("det_xy_host", ctypes.POINTER(ctypes.c_double)), ("n_t", ctypes.c_int),
                ("r0", ctypes.c_double), ("dr", ctypes.c_double), ("quad_m", ctypes.c_int)]


class pat_params(ctypes.Structure):
    _fields_ = [("reg", ctypes.c_int), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("gamma", ctypes.c_double), ("xi_dev", ctypes.c_void_p), ("iters", ctypes.c_int),
                ("tol", ctypes.c_double), ("gap_every", ctypes.c_int), ("precond", ctypes.c_int),
                ("theta", ctypes.c_double), ("box_u", ctypes.c_double), ("box_v", ctypes.c_double),
                ("x0_dev", ctypes.c_void_p), ("xbar0_dev", ctypes.c_void_p), ("y0_dev", ctypes.c_void_p),
                ("x_out_dev", ctypes.c_void_p), ("xbar_out_dev", ctypes.c_void_p),
                ("y_out_dev", ctypes.c_void_p), ("step_ratio", ctypes.c_double), ("adapt", ctypes.c_int),
                ("wavelet_levels", ctypes.c_int), ("x_lo0_dev", ctypes.c_void_p),
                ("x_lo_out_dev", ctypes.c_void_p), ("wavelet_kind", ctypes.c_int),
                ("dtcwt_h1_host", ctypes.c_void_p), ("dtcwt_l1", ctypes.c_int),
                ("dtcwt_hq_host", ctypes.c_void_p), ("dtcwt_lq", ctypes.c_int)]


class pat_shapes(ctypes.Structure):
    _fields_ = [("forward", ctypes.c_int), ("adjoint_waves", ctypes.c_int), ("update_tile", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PAT_FWD_AUTO, PAT_FWD_SLAB_TWO, PAT_FWD_SLAB_ONE, PAT_FWD_GLOBAL = -1, 0, 1, 2
PAT_UPD_32X4, PAT_UPD_32X8, PAT_UPD_64X4 = 0, 1, 2
PAT_WAVELET_DWT, PAT_WAVELET_DTCWT = 0, 1


class pat_unet_desc(ctypes.Structure):
    _fields_ = [("in_ch", ctypes.c_int), ("out_ch", ctypes.c_int), ("base_ch", ctypes.c_int),
                ("levels", ctypes.c_int), ("seed", ctypes.c_ulonglong)]


class pat_info(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int), ("status", ctypes.c_int), ("primal", ctypes.c_double),
                ("dual", ctypes.c_double), ("gap", ctypes.c_double), ("rel_gap", ctypes.c_double),
                ("residual", ctypes.c_double), ("ms", ctypes.c_double), ("step_ratio", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.lib_path()


def load(path: str | None = None) -> ctypes.CDLL:
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or library_path()
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library not built: {p} is missing; run paper_1707_02245_gb300.build.build()")
    lib = ctypes.CDLL(p)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "pat_create_geometry": (i, [ctypes.POINTER(pat_geometry_desc), ctypes.POINTER(vp)]),
        "pat_destroy_geometry": (None, [vp]),
        "pat_forward": (i, [vp, vp, vp, vp]),
        "pat_adjoint": (i, [vp, vp, vp, vp]),
        "pat_adjoint_noalloc": (i, [vp, vp, vp, vp]),
        "pat_direction_field": (i, [i, vp, d, vp, vp]),
        "pat_params_default": (None, [ctypes.POINTER(pat_params)]),
        "pat_reconstruct": (i, [vp, vp, ctypes.POINTER(pat_params), vp, ctypes.POINTER(pat_info), vp]),
        "pat_reconstruct_batched": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(pat_params),
                                        ctypes.POINTER(vp), ctypes.POINTER(pat_info), vp]),
        "pat_steps": (i, [vp, ctypes.POINTER(pat_params), vp, vp, vp, vp, vp, vp]),
        "pat_duality_gap": (i, [vp, vp, ctypes.POINTER(pat_params), vp, vp, ctypes.POINTER(d), vp]),
        "pat_preprocess": (i, [vp, vp, vp, ctypes.POINTER(d), d, vp, vp]),
        "pat_wavelet_transform": (i, [i, i, vp, vp, i, vp]),
        "pat_dtcwt_transform": (i, [i, i, vp, i, vp, i, vp, vp, i, vp]),
        "pat_tune_step_ratio_batched": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(pat_params),
                                            ctypes.POINTER(d), i, i, ctypes.POINTER(d), ctypes.POINTER(d), vp]),
        "pat_tune_step_ratio": (i, [vp, vp, ctypes.POINTER(pat_params), ctypes.POINTER(d), i, i, ctypes.POINTER(d),
                                    ctypes.POINTER(d), vp]),
        "pat_time_phases": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(pat_params), i,
                                ctypes.POINTER(d), vp]),
        "pat_geometry_set_shapes": (i, [vp, ctypes.POINTER(pat_shapes)]),
        "pat_geometry_get_shapes": (i, [vp, ctypes.POINTER(pat_shapes)]),
        "pat_tune_shapes": (i, [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(pat_params), i,
                                ctypes.c_char_p, ctypes.POINTER(pat_shapes), vp]),
        "pat_error_string": (ctypes.c_char_p, [i]),
        "pat_last_error": (ctypes.c_char_p, []),
        "pat_geometry_info": (i, [vp, ctypes.POINTER(ctypes.c_longlong)]),
        "pat_adjoint_worklist": (i, [ctypes.POINTER(pat_geometry_desc), i, vp, ctypes.c_longlong, vp,
                                     ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
        "pat_forward_plan": (i, [ctypes.POINTER(pat_geometry_desc), i, i, vp, ctypes.c_longlong, vp,
                                 ctypes.c_longlong, vp, ctypes.c_longlong, vp, ctypes.c_longlong,
                                 ctypes.POINTER(ctypes.c_longlong)]),
        "pat_profile_enable": (i, [i]),
        "pat_profile_read": (i, [ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong), i]),
        "pat_kernel_launches": (ctypes.c_longlong, []),
        "pat_conv3x3_forward": (i, [vp, i, i, i, i, vp, vp, i, i, vp, vp]),
        "pat_conv3x3_backward_data": (i, [vp, i, i, i, i, vp, i, vp, vp]),
        "pat_conv3x3_backward_weight": (i, [vp, vp, i, i, i, i, i, vp, vp, vp]),
        "pat_nn_wait_timeouts": (i, [ctypes.POINTER(ctypes.c_uint)]),
        "pat_unet_create": (i, [ctypes.POINTER(pat_unet_desc), ctypes.POINTER(vp)]),
        "pat_unet_destroy": (None, [vp]),
        "pat_unet_num_params": (ctypes.c_longlong, [vp]),
        "pat_unet_get_params": (i, [vp, vp]),
        "pat_unet_set_params": (i, [vp, vp]),
        "pat_unet_forward": (i, [vp, vp, i, i, i, vp, vp]),
        "pat_unet_backward": (i, [vp, vp, vp, vp]),
        "pat_unet_train_step": (i, [vp, vp, vp, ctypes.POINTER(ctypes.c_float), i, i, i, ctypes.c_float, vp, vp]),
        "pat_warm_start_features": (i, [vp, vp, vp, i, vp]),
        "pat_warm_start_state": (i, [vp, vp, i, ctypes.POINTER(pat_params), vp, vp, vp, vp]),
        "pat_warm_start_target": (i, [vp, vp, vp, ctypes.POINTER(pat_params), vp, i, vp]),
        "pat_warm_start": (i, [vp, vp, vp, ctypes.POINTER(pat_params), vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s or None
    return int(getattr(s, "cuda_stream"))


def _check(code: int, where: str):
    if code != PAT_OK:
        lib = load()
        raise PatError(code, where, lib.pat_last_error().decode(errors="replace"))


# ---- C-named entry points --------------------------------------------------------

def _geometry_desc(n, det_xy, n_t, r0, dr, quad_m, extent):
    """(desc, detector array); the array must outlive every use of desc."""
    det = np.ascontiguousarray(np.asarray(det_xy, dtype=np.float64).reshape(-1))
    desc = pat_geometry_desc(n=n, xmin=extent[0], xmax=extent[1], ymin=extent[2], ymax=extent[3],
                             n_det=det.size // 2,
                             det_xy_host=det.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             n_t=n_t, r0=r0, dr=dr, quad_m=quad_m)
    return desc, det


def pat_create_geometry(n: int, det_xy, n_t: int, r0: float, dr: float, quad_m: int,
                        extent=(-1.0, 1.0, -1.0, 1.0)) -> int:
    lib = load()
    desc, _det = _geometry_desc(n, det_xy, n_t, r0, dr, quad_m, extent)
    out = ctypes.c_void_p()
    _check(lib.pat_create_geometry(ctypes.byref(desc), ctypes.byref(out)), "pat_create_geometry")
    return out.value


def pat_adjoint_worklist(n: int, det_xy, n_t: int, r0: float, dr: float, quad_m: int, slots: int,
                         extent=(-1.0, 1.0, -1.0, 1.0)) -> dict:
    """The K^T work list (host only when slots > 0): rays (S x 4: detector, angle, first
    radius index, prefix in the tile; sentinels {-1, 0, 0, tile total}), items (I x 5:
    tile, first segment, segments, first and end candidate) and the candidate count."""
    lib = load()
    desc, _det = _geometry_desc(n, det_xy, n_t, r0, dr, quad_m, extent)
    cnt = (ctypes.c_longlong * 3)()
    _check(lib.pat_adjoint_worklist(ctypes.byref(desc), slots, None, 0, None, 0, cnt), "pat_adjoint_worklist")
    rays = np.zeros((cnt[0], 4), dtype=np.int32)
    items = np.zeros((cnt[1], 5), dtype=np.int32)
    _check(lib.pat_adjoint_worklist(ctypes.byref(desc), slots, rays.ctypes.data, cnt[0], items.ctypes.data, cnt[1],
                                    cnt), "pat_adjoint_worklist")
    return {"rays": rays, "items": items, "candidates": int(cnt[2])}


def pat_forward_plan(n: int, det_xy, n_t: int, r0: float, dr: float, quad_m: int, sms: int,
                     budget_bytes: int = 0, extent=(-1.0, 1.0, -1.0, 1.0)) -> dict:
    """The K work plan (host only when sms > 0; see include/pat.h): slabs (= CTAs per
    cluster), rows per slab, shared-memory row stride, units (U x 4), CTAs (C x 4), round
    offsets, the clusters' row groups, the points inside the windows and the CTA's shared
    memory."""
    lib = load()
    desc, _det = _geometry_desc(n, det_xy, n_t, r0, dr, quad_m, extent)
    info = (ctypes.c_longlong * 8)()
    _check(lib.pat_forward_plan(ctypes.byref(desc), budget_bytes, sms, None, 0, None, 0, None, 0, None, 0, info),
           "pat_forward_plan")
    U, C, O = int(info[3]), int(info[4]), int(info[7])
    G = det_xy.shape[0] * ((n_t + 7) // 8)
    units = np.zeros((U, 4), dtype=np.int32)
    ctas = np.zeros((C, 4), dtype=np.int32)
    roff = np.zeros(O, dtype=np.int32)
    rgs = np.zeros(G, dtype=np.int32)
    _check(lib.pat_forward_plan(ctypes.byref(desc), budget_bytes, sms, units.ctypes.data, U, ctas.ctypes.data, C,
                                roff.ctypes.data, O, rgs.ctypes.data, G, info), "pat_forward_plan")
    return {"slabs": int(info[0]), "rows": int(info[1]), "stride": int(info[2]), "units": units, "ctas": ctas,
            "roff": roff, "rgs": rgs, "evaluated": int(info[5]), "smem": int(info[6])}


def pat_destroy_geometry(g: int) -> None:
    load().pat_destroy_geometry(g)


def pat_forward(g: int, u_dev, y_dev, stream=None) -> None:
    _check(load().pat_forward(g, _ptr(u_dev), _ptr(y_dev), _stream(stream)), "pat_forward")


def pat_adjoint(g: int, y_dev, u_dev, stream=None) -> None:
    _check(load().pat_adjoint(g, _ptr(y_dev), _ptr(u_dev), _stream(stream)), "pat_adjoint")


def pat_adjoint_noalloc(g: int, y_dev, u_dev, stream=None) -> None:
    """K^T y without any device allocation during the call (see include/pat.h)."""
    _check(load().pat_adjoint_noalloc(g, _ptr(y_dev), _ptr(u_dev), _stream(stream)), "pat_adjoint_noalloc")


def pat_direction_field(n: int, w_dev, eta: float, xi_dev, stream=None) -> None:
    _check(load().pat_direction_field(n, _ptr(w_dev), eta, _ptr(xi_dev), _stream(stream)), "pat_direction_field")


def pat_params_default() -> pat_params:
    p = pat_params()
    load().pat_params_default(ctypes.byref(p))
    return p


def make_params(reg=PAT_TV, alpha=0.05, beta=1.0, gamma=0.95, xi=None, iters=100, tol=0.0, gap_every=10,
                precond=PAT_PRECOND_DIAG, theta=1.0, box_u=2.0, box_v=4.0, x0=None, xbar0=None, y0=None,
                x_out=None, xbar_out=None, y_out=None, step_ratio=1.0, adapt=PAT_ADAPT_NONE,
                wavelet_levels=4, x_lo0=None, x_lo_out=None, wavelet_kind=0, dtcwt_filters=None) -> pat_params:
    """dtcwt_filters: None (the closed-form defaults) or (level-1 low-pass, Q-shift low-pass of
    tree a) as float64 sequences."""
    p = pat_params_default()
    p.reg, p.alpha, p.beta, p.gamma = reg, alpha, beta, gamma
    p.xi_dev = _ptr(xi)
    p.iters, p.tol, p.gap_every, p.precond = iters, tol, gap_every, precond
    p.theta, p.box_u, p.box_v = theta, box_u, box_v
    p.x0_dev, p.xbar0_dev, p.y0_dev = _ptr(x0), _ptr(xbar0), _ptr(y0)
    p.x_out_dev, p.xbar_out_dev, p.y_out_dev = _ptr(x_out), _ptr(xbar_out), _ptr(y_out)
    p.step_ratio, p.adapt, p.wavelet_levels = step_ratio, adapt, wavelet_levels
    p.x_lo0_dev, p.x_lo_out_dev = _ptr(x_lo0), _ptr(x_lo_out)
    p.wavelet_kind = wavelet_kind
    fl = None
    if dtcwt_filters is not None:
        fl = [(ctypes.c_double * len(h))(*[float(v) for v in h]) for h in dtcwt_filters]
        p.dtcwt_h1_host, p.dtcwt_l1 = ctypes.cast(fl[0], ctypes.c_void_p).value, len(fl[0])
        p.dtcwt_hq_host, p.dtcwt_lq = ctypes.cast(fl[1], ctypes.c_void_p).value, len(fl[1])
    # keep the buffers alive as long as the parameter block that points at them
    p._keep = [xi, x0, xbar0, y0, x_out, xbar_out, y_out, x_lo0, x_lo_out, fl]
    return p


def pat_reconstruct(g: int, f_dev, params: pat_params, u_dev, stream=None) -> dict:
    info = pat_info()
    _check(load().pat_reconstruct(g, _ptr(f_dev), ctypes.byref(params), _ptr(u_dev), ctypes.byref(info),
                                  _stream(stream)), "pat_reconstruct")
    return info.as_dict()


def pat_reconstruct_batched(geoms, fs, params, us, stream=None) -> list[dict]:
    n = len(geoms)
    G = (ctypes.c_void_p * n)(*geoms)
    F = (ctypes.c_void_p * n)(*[_ptr(f) for f in fs])
    U = (ctypes.c_void_p * n)(*[_ptr(u) for u in us])
    P = (pat_params * n)(*params)
    infos = (pat_info * n)()
    _check(load().pat_reconstruct_batched(n, G, F, P, U, infos, _stream(stream)), "pat_reconstruct_batched")
    return [infos[i].as_dict() for i in range(n)]


def pat_steps(g: int, params: pat_params, sig_q=None, tau_u=None, sig_r=None, sig_s=None, tau_v=None,
              stream=None) -> None:
    _check(load().pat_steps(g, ctypes.byref(params), _ptr(sig_q), _ptr(tau_u), _ptr(sig_r), _ptr(sig_s),
                            _ptr(tau_v), _stream(stream)), "pat_steps")


def pat_duality_gap(g: int, f_dev, params: pat_params, x_dev, y_dev, stream=None) -> dict:
    out = (ctypes.c_double * 4)()
    _check(load().pat_duality_gap(g, _ptr(f_dev), ctypes.byref(params), _ptr(x_dev), _ptr(y_dev), out,
                                  _stream(stream)), "pat_duality_gap")
    return {"primal": out[0], "dual": out[1], "gap": out[2], "rel_gap": out[3]}


def pat_tune_step_ratio(g: int, f_dev, params: pat_params, candidates, probe_iters: int, stream=None):
    """Returns (best s, [relative gap of each probe])."""
    c = (ctypes.c_double * len(candidates))(*[float(v) for v in candidates])
    best = ctypes.c_double()
    gaps = (ctypes.c_double * len(candidates))()
    _check(load().pat_tune_step_ratio(g, _ptr(f_dev), ctypes.byref(params), c, len(candidates), probe_iters,
                                      ctypes.byref(best), gaps, _stream(stream)), "pat_tune_step_ratio")
    return best.value, list(gaps)


def pat_tune_step_ratio_batched(geoms, fs, params, candidates, probe_iters: int, stream=None):
    """Returns ([best s per problem], [[relative gap of each probe] per problem])."""
    n, c = len(geoms), len(candidates)
    G = (ctypes.c_void_p * n)(*geoms)
    F = (ctypes.c_void_p * n)(*[_ptr(f) for f in fs])
    Pp = (pat_params * n)(*params)
    C = (ctypes.c_double * c)(*[float(v) for v in candidates])
    best = (ctypes.c_double * n)()
    gaps = (ctypes.c_double * (n * c))()
    _check(load().pat_tune_step_ratio_batched(n, G, F, Pp, C, c, probe_iters, best, gaps, _stream(stream)),
           "pat_tune_step_ratio_batched")
    return list(best), [list(gaps[i * c:(i + 1) * c]) for i in range(n)]


def pat_geometry_set_shapes(g: int, forward: int = PAT_FWD_AUTO, adjoint_waves: int = 1,
                            update_tile: int = PAT_UPD_32X4) -> None:
    s = pat_shapes(forward, adjoint_waves, update_tile)
    _check(load().pat_geometry_set_shapes(g, ctypes.byref(s)), "pat_geometry_set_shapes")


def pat_geometry_get_shapes(g: int) -> dict:
    s = pat_shapes()
    _check(load().pat_geometry_get_shapes(g, ctypes.byref(s)), "pat_geometry_get_shapes")
    return s.as_dict()


def pat_tune_shapes(geoms, fs, params, reps: int = 50, cache_path=None, stream=None) -> list:
    """Times the launch-shape candidates of every geometry on its problem (see
    include/pat.h), keeps the fastest, caches them in the JSON file cache_path and returns
    the chosen shapes per problem."""
    n = len(geoms)
    G = (ctypes.c_void_p * n)(*geoms)
    F = (ctypes.c_void_p * n)(*[_ptr(f) for f in fs])
    Pp = (pat_params * n)(*params)
    out = (pat_shapes * n)()
    path = cache_path.encode() if cache_path else None
    _check(load().pat_tune_shapes(n, G, F, Pp, int(reps), path, out, _stream(stream)), "pat_tune_shapes")
    return [out[i].as_dict() for i in range(n)]


def pat_time_phases(geoms, fs, params, reps: int, stream=None) -> dict:
    """Microseconds per launch of each phase of the batched iteration, each phase timed
    alone in a CUDA graph of ``reps`` launches after ``params[0].iters`` iterations
    (see include/pat.h).  Returns {phase name: us}."""
    n = len(geoms)
    G = (ctypes.c_void_p * n)(*geoms)
    F = (ctypes.c_void_p * n)(*[_ptr(f) for f in fs])
    Pp = (pat_params * n)(*params)
    us = (ctypes.c_double * len(PHASES))()
    _check(load().pat_time_phases(n, G, F, Pp, int(reps), us, _stream(stream)), "pat_time_phases")
    return {name: us[k] for k, name in enumerate(PHASES)}


def pat_dtcwt_transform(n: int, levels: int, in_dev, out_dev, inverse: bool = False, filters=None,
                        stream=None) -> None:
    """W in (out: 4 n^2 floats) or W^T in (in: 4 n^2 floats, out: n^2) of the dual-tree
    complex wavelet transform (see include/pat.h); filters: None or (h1, hq)."""
    h1 = hq = None
    l1 = lq = 0
    if filters is not None:
        h1 = (ctypes.c_double * len(filters[0]))(*[float(v) for v in filters[0]])
        hq = (ctypes.c_double * len(filters[1]))(*[float(v) for v in filters[1]])
        l1, lq = len(h1), len(hq)
    _check(load().pat_dtcwt_transform(n, levels, h1, l1, hq, lq, _ptr(in_dev), _ptr(out_dev), 1 if inverse else 0,
                                      _stream(stream)), "pat_dtcwt_transform")


def pat_wavelet_transform(n: int, levels: int, in_dev, out_dev, inverse: bool = False, stream=None) -> None:
    _check(load().pat_wavelet_transform(n, levels, _ptr(in_dev), _ptr(out_dev), 1 if inverse else 0, _stream(stream)),
           "pat_wavelet_transform")


def pat_preprocess(g: int, p_dev, pcal_dev, xp, eps_rel: float, f_dev, stream=None) -> None:
    """Pre-processed data f from pressures p and calibrations p_cal (see include/pat.h)."""
    x = (ctypes.c_double * 2)(float(xp[0]), float(xp[1]))
    _check(load().pat_preprocess(g, _ptr(p_dev), _ptr(pcal_dev), x, float(eps_rel), _ptr(f_dev), _stream(stream)),
           "pat_preprocess")


def pat_geometry_info(g: int) -> dict:
    out = (ctypes.c_longlong * 6)()
    _check(load().pat_geometry_info(g, out), "pat_geometry_info")
    return {"n": out[0], "n_det": out[1], "n_t": out[2], "quad_m": out[3], "points_per_apply": out[4],
            "points_on_grid": out[5]}


def pat_error_string(code: int) -> str:
    return load().pat_error_string(code).decode()


def pat_last_error() -> str:
    return load().pat_last_error().decode(errors="replace")


def pat_profile_enable(on: bool) -> None:
    _check(load().pat_profile_enable(1 if on else 0), "pat_profile_enable")


def pat_profile_read(reset: bool = False) -> dict:
    ms = (ctypes.c_double * len(PHASES))()
    cnt = (ctypes.c_longlong * len(PHASES))()
    _check(load().pat_profile_read(ms, cnt, 1 if reset else 0), "pat_profile_read")
    return {ph: (ms[i], cnt[i]) for i, ph in enumerate(PHASES)}


def pat_kernel_launches() -> int:
    return int(load().pat_kernel_launches())


# ---- learned warm start (include/pat_unet.h) -------------------------------------
# bfloat16 tensors are passed by pointer (their 16-bit patterns); torch.bfloat16 CUDA
# tensors work as they are.

def pat_conv3x3_forward(x_dev, batch, h, w, cin, w_dev, bias_dev, cout, relu, y_dev, stream=None) -> None:
    _check(load().pat_conv3x3_forward(_ptr(x_dev), batch, h, w, cin, _ptr(w_dev), _ptr(bias_dev), cout,
                                      1 if relu else 0, _ptr(y_dev), _stream(stream)), "pat_conv3x3_forward")


def pat_conv3x3_backward_data(dy_dev, batch, h, w, cout, w_dev, cin, dx_dev, stream=None) -> None:
    _check(load().pat_conv3x3_backward_data(_ptr(dy_dev), batch, h, w, cout, _ptr(w_dev), cin, _ptr(dx_dev),
                                            _stream(stream)), "pat_conv3x3_backward_data")


def pat_conv3x3_backward_weight(x_dev, dy_dev, batch, h, w, cin, cout, dw_dev, db_dev=None, stream=None) -> None:
    _check(load().pat_conv3x3_backward_weight(_ptr(x_dev), _ptr(dy_dev), batch, h, w, cin, cout, _ptr(dw_dev),
                                              _ptr(db_dev), _stream(stream)), "pat_conv3x3_backward_weight")


def pat_nn_wait_timeouts() -> int:
    """Bounded waits of the tensor-memory convolutions that ran out since the library loaded."""
    v = ctypes.c_uint()
    _check(load().pat_nn_wait_timeouts(ctypes.byref(v)), "pat_nn_wait_timeouts")
    return int(v.value)


def pat_unet_create(in_ch=8, out_ch=8, base_ch=32, levels=4, seed=0) -> int:
    desc = pat_unet_desc(in_ch=in_ch, out_ch=out_ch, base_ch=base_ch, levels=levels, seed=seed)
    out = ctypes.c_void_p()
    _check(load().pat_unet_create(ctypes.byref(desc), ctypes.byref(out)), "pat_unet_create")
    return out.value


def pat_unet_destroy(net: int) -> None:
    load().pat_unet_destroy(net)


def pat_unet_num_params(net: int) -> int:
    return int(load().pat_unet_num_params(net))


def pat_unet_get_params(net: int) -> np.ndarray:
    out = np.empty(pat_unet_num_params(net), dtype=np.float32)
    _check(load().pat_unet_get_params(net, out.ctypes.data), "pat_unet_get_params")
    return out


def pat_unet_set_params(net: int, params) -> None:
    a = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    if a.size != pat_unet_num_params(net):
        raise ValueError("pat_unet_set_params: wrong number of parameters")
    _check(load().pat_unet_set_params(net, a.ctypes.data), "pat_unet_set_params")


def pat_unet_forward(net: int, x_dev, batch, h, w, y_dev, stream=None) -> None:
    _check(load().pat_unet_forward(net, _ptr(x_dev), batch, h, w, _ptr(y_dev), _stream(stream)), "pat_unet_forward")


def pat_unet_backward(net: int, dy_dev, grad_dev, stream=None) -> None:
    _check(load().pat_unet_backward(net, _ptr(dy_dev), _ptr(grad_dev), _stream(stream)), "pat_unet_backward")


def pat_unet_train_step(net: int, x_dev, target_dev, ch_weight, batch, h, w, lr, loss_dev=None, stream=None) -> None:
    cw = (ctypes.c_float * len(ch_weight))(*[float(v) for v in ch_weight])
    _check(load().pat_unet_train_step(net, _ptr(x_dev), _ptr(target_dev), cw, batch, h, w, float(lr), _ptr(loss_dev),
                                      _stream(stream)), "pat_unet_train_step")


def pat_warm_start_features(g: int, f_dev, x_dev, in_ch=8, stream=None) -> None:
    _check(load().pat_warm_start_features(g, _ptr(f_dev), _ptr(x_dev), in_ch, _stream(stream)),
           "pat_warm_start_features")


def pat_warm_start_state(g: int, pred_dev, out_ch, params: pat_params, f_dev, x0_dev, y0_dev, stream=None) -> None:
    _check(load().pat_warm_start_state(g, _ptr(pred_dev), out_ch, ctypes.byref(params), _ptr(f_dev), _ptr(x0_dev),
                                       _ptr(y0_dev), _stream(stream)), "pat_warm_start_state")


def pat_warm_start_target(g: int, x_dev, y_dev, params: pat_params, target_dev, out_ch=8, stream=None) -> None:
    _check(load().pat_warm_start_target(g, _ptr(x_dev), _ptr(y_dev), ctypes.byref(params), _ptr(target_dev), out_ch,
                                        _stream(stream)), "pat_warm_start_target")


def pat_warm_start(g: int, net: int, f_dev, params: pat_params, x0_dev, y0_dev, stream=None) -> None:
    _check(load().pat_warm_start(g, net, _ptr(f_dev), ctypes.byref(params), _ptr(x0_dev), _ptr(y0_dev),
                                 _stream(stream)), "pat_warm_start")


# ---- a small owner of a geometry handle -----------------------------------------

@dataclass
class Geometry:
    """Owns a pat_geometry handle; sizes mirror pat_geometry_desc."""
    n: int
    det_xy: np.ndarray
    n_t: int
    r0: float
    dr: float
    quad_m: int
    extent: tuple = (-1.0, 1.0, -1.0, 1.0)

    def __post_init__(self):
        self.det_xy = np.asarray(self.det_xy, dtype=np.float64).reshape(-1, 2)
        self.handle = pat_create_geometry(self.n, self.det_xy, self.n_t, self.r0, self.dr, self.quad_m,
                                          self.extent)

    @property
    def n_det(self) -> int:
        return self.det_xy.shape[0]

    def close(self):
        if getattr(self, "handle", None):
            pat_destroy_geometry(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return pat_geometry_info(self.handle)
