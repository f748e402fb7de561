"""ctypes binding of the ABD-IPC C-ABI (``include/ipc_b300.h``).

Argument marshalling only: every step of the method runs in the CUDA library.
The function and method names follow the C entry points.  PyTorch provides the
device workspace (one uint8 tensor) and the CUDA stream.  There is no CPU
fallback: a missing library raises at import of this module's loader.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# IPC_B300_CHECKS=1 loads the bounds-checked build (see ipc_check_report)
LIB_PATH = os.path.join(_HERE, "libipc_b300_checks.so" if os.environ.get("IPC_B300_CHECKS") == "1"
                        else "libipc_b300.so")

IPC_OK, IPC_EINVAL, IPC_ENOMEM, IPC_ENOTCONV, IPC_EINTERSECT, IPC_EINVERTED, IPC_EOVERFLOW, IPC_ECUDA = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ENOTCONV", "EINTERSECT", "EINVERTED", "EOVERFLOW", "ECUDA"]

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint8)


class ipc_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double * 3), ("dhat", C.c_double), ("kappa", C.c_double),
                ("newton_tol", C.c_double), ("pcg_rel_tol", C.c_double), ("newton_max", C.c_int),
                ("pcg_max", C.c_int), ("ls_max", C.c_int), ("accd_max", C.c_int), ("accd_s", C.c_double),
                ("al_kappa", C.c_double), ("al_max", C.c_int), ("ee_mollifier", C.c_double),
                ("precision", C.c_int), ("max_pairs_per_env", C.c_int), ("friction_mu", C.c_double),
                ("friction_eps_v", C.c_double), ("newton_abs_after", C.c_int),
                ("rollout_pcg_window", C.c_int), ("pcg_fused", C.c_int), ("pcg_iters_per_launch", C.c_int)]


class ipc_scene_desc(C.Structure):
    _fields_ = [("n_verts", C.c_int), ("n_tets", C.c_int), ("rest_x", _dp), ("tets", _ip), ("pad_id", _ip),
                ("pinned", _up), ("attach_body", _ip), ("E", C.c_double), ("nu", C.c_double), ("rho", C.c_double),
                ("n_bodies", C.c_int), ("body_nv", _ip), ("body_rest_x", _dp), ("body_nt", _ip),
                ("body_tris", _ip), ("body_rho", _dp), ("body_kappa_s", _dp), ("body_driven", _up),
                ("pad_self_contact", _up)]


class ipc_sensor(C.Structure):
    _fields_ = [("env", C.c_int), ("pad", C.c_int), ("origin", C.c_double * 3), ("axis_u", C.c_double * 3),
                ("axis_v", C.c_double * 3), ("normal", C.c_double * 3), ("pitch", C.c_double)]


class ipc_tuning(C.Structure):
    _fields_ = [("spmv_unroll", C.c_int), ("pcg_ctas_per_sm", C.c_int), ("spmv_us", C.c_float * 3),
                ("grid_ctas_per_sm", C.c_int * 3), ("grid_us", C.c_float * 3),
                ("assemble_block", C.c_int), ("assemble_us", C.c_float * 3),
                ("pairs_ctas_per_sm", C.c_int), ("pairs_us", C.c_float * 3),
                ("pcg_iter_bound", C.c_int), ("pcg_iter_us", C.c_float * 2)]


class ipc_step_stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("pcg_iters", C.c_int), ("ls_trials", C.c_int),
                ("al_updates", C.c_int), ("max_pairs", C.c_int), ("newton_env_iters", C.c_longlong),
                ("al_env_updates", C.c_longlong), ("ccd_limited", C.c_longlong), ("alpha_sum", C.c_double),
                ("accd_iters", C.c_longlong), ("accd_iters_max", C.c_int),
                ("ms_total", C.c_double), ("pair_evals", C.c_longlong), ("swept_pairs", C.c_longlong),
                ("loop_iters", C.c_longlong), ("pcg_launches", C.c_longlong),
                ("act_pair_iters", C.c_longlong)]


_lib = None


def lib():
    """Load libipc_b300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library missing: {LIB_PATH} (run python -m paper_2504_12908_b300.build)")
        L = C.CDLL(LIB_PATH)
        vp, i32, dbl = C.c_void_p, C.c_int, C.c_double
        sig = {
            "ipc_default_params": (None, [C.POINTER(ipc_params)]),
            "ipc_workspace_bytes": (i32, [C.POINTER(ipc_scene_desc), i32, C.POINTER(ipc_params), C.POINTER(C.c_size_t)]),
            "ipc_create_envs": (i32, [C.POINTER(ipc_scene_desc), i32, C.POINTER(ipc_params), vp, C.c_size_t, vp,
                                      C.POINTER(vp)]),
            "ipc_destroy": (i32, [vp]),
            "ipc_last_error": (C.c_char_p, [vp]),
            "ipc_num_envs": (i32, [vp]),
            "ipc_check_report": (i32, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_longlong)]),
            "ipc_env_sizes": (i32, [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
            "ipc_body_com": (i32, [vp, i32, i32, _dp]),
            "ipc_set_state": (i32, [vp, i32, _dp, _dp, _dp, _dp]),
            "ipc_get_state": (i32, [vp, i32, _dp, _dp, _dp, _dp]),
            "ipc_set_targets": (i32, [vp, i32, _dp]),
            "ipc_reset_env": (i32, [vp, i32, C.POINTER(ipc_scene_desc)]),
            "ipc_set_targets_all": (i32, [vp, _dp]),
            "ipc_set_targets_all_device": (i32, [vp, vp]),
            "ipc_step": (i32, [vp, _ip, i32, _ip, C.POINTER(ipc_step_stats)]),
            "ipc_step_results": (i32, [vp, _ip, C.POINTER(ipc_step_stats)]),
            "ipc_rollout": (i32, [vp, _ip, i32, i32, _ip, vp, _ip, _ip, C.POINTER(ipc_step_stats)]),
            "ipc_rollout_results": (i32, [vp, _ip, _ip, C.POINTER(ipc_step_stats)]),
            "ipc_read_gel_surface": (i32, [vp, i32, _dp, i32, C.POINTER(i32)]),
            "ipc_read_gel_surface_all": (i32, [vp, _dp, C.c_size_t, C.POINTER(C.c_size_t)]),
            "ipc_read_gel_surface_all_noalloc": (i32, [vp, _dp, C.c_size_t, C.POINTER(C.c_size_t)]),
            "ipc_env_stats": (i32, [vp, i32, _ip]),
            "ipc_set_graph_mode": (i32, [vp, i32]),
            "ipc_autotune": (i32, [vp, i32, C.POINTER(ipc_tuning)]),
            "ipc_gel_vertex_rows": (i32, [vp, i32, i32, _ip, _ip]),
            "ipc_sensor_triangles": (i32, [vp, C.POINTER(ipc_sensor), _ip, i32, C.POINTER(i32)]),
            "ipc_tactile_maps_device": (i32, [vp, i32, i32, i32, vp, vp, vp, i32, vp, vp, vp, vp]),
            "ipc_markers_device": (i32, [vp, i32, vp, vp, vp, vp, vp]),
            "ipc_debug_eval": (i32, [vp, i32, _dp, _dp, _dp, _dp]),
            "ipc_debug_pairs": (i32, [vp, i32, _dp, _dp, _ip, i32, C.POINTER(i32)]),
            "ipc_debug_newton_dir": (i32, [vp, i32, _dp, C.POINTER(i32)]),
            "ipc_debug_pcg_wait_out": (i32, [vp, i32, C.POINTER(i32), C.POINTER(C.c_float)]),
            "ipc_debug_accd": (i32, [vp, i32, _dp, _dp]),
            "ipc_profile_enable": (i32, [vp, i32]),
            "ipc_profile_reset": (i32, [vp]),
            "ipc_profile_count": (i32, [vp]),
            "ipc_profile_get": (i32, [vp, i32, C.POINTER(C.c_char_p), C.POINTER(C.c_longlong),
                                      C.POINTER(C.c_double)]),
            "ipc_launch_count": (C.c_longlong, [vp]),
            "ipc_system_sizes": (i32, [vp, i32, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                       C.POINTER(i32), C.POINTER(i32)]),
            "ipc_k_tet": (i32, [i32, vp, vp, vp, dbl, dbl, vp, vp, vp, i32, vp]),
            "ipc_k_barrier": (i32, [i32, vp, vp, vp, vp, dbl, vp, vp, vp, i32, vp]),
            "ipc_k_accd": (i32, [i32, vp, vp, vp, dbl, i32, vp, vp, vp]),
            "ipc_fma_peaks": (i32, [vp, C.c_size_t, _dp, _dp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


EXPORTED = ["ipc_default_params", "ipc_workspace_bytes", "ipc_create_envs", "ipc_destroy", "ipc_last_error",
            "ipc_num_envs", "ipc_check_report", "ipc_env_sizes", "ipc_body_com", "ipc_set_state", "ipc_get_state", "ipc_set_targets", "ipc_reset_env",
            "ipc_set_targets_all", "ipc_set_targets_all_device", "ipc_step", "ipc_step_results", "ipc_rollout", "ipc_rollout_results", "ipc_read_gel_surface", "ipc_read_gel_surface_all",
            "ipc_read_gel_surface_all_noalloc", "ipc_env_stats", "ipc_set_graph_mode", "ipc_gel_vertex_rows", "ipc_sensor_triangles",
            "ipc_tactile_maps_device", "ipc_markers_device", "ipc_autotune",
            "ipc_debug_eval", "ipc_debug_pairs", "ipc_debug_newton_dir", "ipc_debug_pcg_wait_out", "ipc_debug_accd",
            "ipc_profile_enable", "ipc_profile_reset", "ipc_profile_count", "ipc_profile_get", "ipc_launch_count",
            "ipc_system_sizes", "ipc_k_tet", "ipc_k_barrier", "ipc_k_accd", "ipc_fma_peaks"]


class IpcError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


def _ptr(a: Optional[np.ndarray], ct):
    if a is None:
        return None
    return a.ctypes.data_as(ct)


def params_from(p) -> ipc_params:
    """ipc_params from any object with the SolverParams attribute names."""
    out = ipc_params()
    lib().ipc_default_params(C.byref(out))
    out.dt = p.dt
    for k in range(3):
        out.gravity[k] = p.gravity[k]
    for name in ("dhat", "kappa", "newton_tol", "pcg_rel_tol", "accd_s", "al_kappa", "ee_mollifier"):
        setattr(out, name, float(getattr(p, name)))
    for name in ("newton_max", "pcg_max", "ls_max", "accd_max", "al_max"):
        setattr(out, name, int(getattr(p, name)))
    out.precision = int(getattr(p, "precision", 0))
    out.max_pairs_per_env = int(getattr(p, "max_pairs_per_env", 0))
    out.friction_mu = float(getattr(p, "friction_mu", 0.0))
    out.friction_eps_v = float(getattr(p, "friction_eps_v", 1e-3))
    out.newton_abs_after = int(getattr(p, "newton_abs_after", 1000000))
    out.rollout_pcg_window = int(getattr(p, "rollout_pcg_window", 0))
    out.pcg_fused = int(getattr(p, "pcg_fused", 1))
    out.pcg_iters_per_launch = int(getattr(p, "pcg_iters_per_launch", 8))
    return out


class _SceneArrays:
    """Keeps the numpy buffers of one scene descriptor alive."""

    def __init__(self, sc):
        self.x = np.ascontiguousarray(sc.gel_x, dtype=np.float64)
        self.t = np.ascontiguousarray(sc.gel_tets, dtype=np.int32)
        self.pad = np.ascontiguousarray(sc.gel_obj, dtype=np.int32)
        self.pin = np.ascontiguousarray(sc.pinned, dtype=np.uint8)
        self.att = np.ascontiguousarray(sc.attach, dtype=np.int32)
        bs = sc.bodies
        self.bnv = np.array([b.rest_x.shape[0] for b in bs], dtype=np.int32)
        self.bx = np.ascontiguousarray(np.concatenate([b.rest_x for b in bs]) if bs else np.zeros((0, 3)),
                                       dtype=np.float64)
        self.bnt = np.array([b.tris.shape[0] for b in bs], dtype=np.int32)
        self.bt = np.ascontiguousarray(np.concatenate([b.tris for b in bs]) if bs else np.zeros((0, 3)),
                                       dtype=np.int32)
        self.brho = np.array([b.rho for b in bs], dtype=np.float64)
        self.bk = np.array([b.kappa_s for b in bs], dtype=np.float64)
        self.bd = np.array([1 if b.driven else 0 for b in bs], dtype=np.uint8)
        selfc = getattr(sc, "self_contact", None)
        self.selfc = None if selfc is None else np.ascontiguousarray(np.asarray(selfc, dtype=bool), dtype=np.uint8)
        d = ipc_scene_desc()
        d.n_verts, d.n_tets = self.x.shape[0], self.t.shape[0]
        d.rest_x, d.tets, d.pad_id = _ptr(self.x, _dp), _ptr(self.t, _ip), _ptr(self.pad, _ip)
        d.pinned, d.attach_body = _ptr(self.pin, _up), _ptr(self.att, _ip)
        d.E, d.nu, d.rho = float(sc.E), float(sc.nu), float(sc.rho)
        d.n_bodies = len(bs)
        d.body_nv, d.body_rest_x, d.body_nt = _ptr(self.bnv, _ip), _ptr(self.bx, _dp), _ptr(self.bnt, _ip)
        d.body_tris, d.body_rho, d.body_kappa_s = _ptr(self.bt, _ip), _ptr(self.brho, _dp), _ptr(self.bk, _dp)
        d.body_driven = _ptr(self.bd, _up)
        if self.selfc is not None:
            n_pads = int(self.pad.max()) + 1 if self.pad.size else 1
            if self.selfc.shape != (n_pads,):
                raise ValueError(f"self_contact needs one flag per pad ({n_pads})")
            d.pad_self_contact = _ptr(self.selfc, _up)
        self.desc = d


def _descs(scenes: Sequence) -> tuple:
    """Descriptor array; identical scene objects share one descriptor (the
    library then preprocesses them once)."""
    cache = {}
    keep = []
    arr = (ipc_scene_desc * len(scenes))()
    for i, sc in enumerate(scenes):
        k = id(sc)
        if k not in cache:
            cache[k] = _SceneArrays(sc)
            keep.append(cache[k])
        arr[i] = cache[k].desc
    return arr, keep


def workspace_bytes(scenes: Sequence, params) -> int:
    arr, keep = _descs(scenes)
    prm = params_from(params)
    n = C.c_size_t(0)
    st = lib().ipc_workspace_bytes(arr, len(scenes), C.byref(prm), C.byref(n))
    if st != IPC_OK:
        raise IpcError(st, "ipc_workspace_bytes")
    return int(n.value)


class Envs:
    """A batch of environments on one GPU (one ipc_ctx)."""

    def __init__(self, scenes: Sequence, params, device: str = "cuda:0", stream=None):
        import torch
        self._torch = torch
        self.scenes = list(scenes)
        self.params = params
        arr, self._keep = _descs(self.scenes)
        self._prm = params_from(params)
        n = C.c_size_t(0)
        L = lib()
        st = L.ipc_workspace_bytes(arr, len(self.scenes), C.byref(self._prm), C.byref(n))
        if st != IPC_OK:
            raise IpcError(st, "ipc_workspace_bytes")
        self.ws_bytes = int(n.value)
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        ctx = C.c_void_p()
        st = L.ipc_create_envs(arr, len(self.scenes), C.byref(self._prm), C.c_void_p(self.workspace.data_ptr()),
                               self.ws_bytes, C.c_void_p(self.stream.cuda_stream), C.byref(ctx))
        self._ctx = ctx
        if st != IPC_OK:
            msg = L.ipc_last_error(ctx).decode() if ctx.value else ""
            if ctx.value:
                L.ipc_destroy(ctx)
            self._ctx = None
            raise IpcError(st, msg)
        self.n_envs = len(self.scenes)
        self.sizes = []
        for e in range(self.n_envs):
            nv, nb, ns = C.c_int(), C.c_int(), C.c_int()
            L.ipc_env_sizes(ctx, e, C.byref(nv), C.byref(nb), C.byref(ns))
            self.sizes.append((nv.value, nb.value, ns.value))
        self.max_bodies = max([s[1] for s in self.sizes] + [0])

    # ------------------------------------------------------------------
    def _check(self, st: int, what: str):
        if st != IPC_OK:
            raise IpcError(st, f"{what}: {lib().ipc_last_error(self._ctx).decode()}")

    def close(self):
        if self._ctx is not None:
            lib().ipc_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ API
    def body_com(self, env: int, body: int) -> np.ndarray:
        out = np.zeros(3)
        self._check(lib().ipc_body_com(self._ctx, env, body, _ptr(out, _dp)), "ipc_body_com")
        return out

    def rest_y(self, env: int) -> np.ndarray:
        nb = self.sizes[env][1]
        y = np.zeros((nb, 12))
        for b in range(nb):
            y[b, :3] = self.body_com(env, b)
            y[b, 3:] = np.eye(3).T.ravel()
        return y

    def set_state(self, env: int, x=None, v=None, y=None, ydot=None) -> int:
        a = [None if t is None else np.ascontiguousarray(t, dtype=np.float64) for t in (x, v, y, ydot)]
        return lib().ipc_set_state(self._ctx, env, *[_ptr(t, _dp) for t in a])

    def get_state(self, env: int):
        nv, nb, _ = self.sizes[env]
        x, v = np.zeros((nv, 3)), np.zeros((nv, 3))
        y, yd = np.zeros((nb, 12)), np.zeros((nb, 12))
        self._check(lib().ipc_get_state(self._ctx, env, _ptr(x, _dp), _ptr(v, _dp), _ptr(y, _dp), _ptr(yd, _dp)),
                    "ipc_get_state")
        return x, v, y, yd

    def reset_env(self, env: int, scene):
        """Put a new scene of the same topology into env slot `env`, at its
        rest state (ipc_reset_env)."""
        arr, keep = _descs([scene])
        self._check(lib().ipc_reset_env(self._ctx, env, arr), "ipc_reset_env")
        self.scenes[env] = scene
        del keep

    def set_targets(self, env: int, y_target: np.ndarray):
        t = np.ascontiguousarray(y_target, dtype=np.float64)
        self._check(lib().ipc_set_targets(self._ctx, env, _ptr(t, _dp)), "ipc_set_targets")

    def set_targets_all(self, y_targets: np.ndarray):
        t = np.ascontiguousarray(y_targets, dtype=np.float64)
        self._check(lib().ipc_set_targets_all(self._ctx, _ptr(t, _dp)), "ipc_set_targets_all")

    def set_targets_all_device(self, dev_targets):
        """dev_targets: CUDA float64 tensor [n_envs][max_bodies][12]."""
        self._check(lib().ipc_set_targets_all_device(self._ctx, C.c_void_p(dev_targets.data_ptr())),
                    "ipc_set_targets_all_device")

    def step(self, env_ids: Optional[Sequence[int]] = None, wait: bool = True):
        """Returns (per-env status array, stats dict).  wait=False only
        enqueues the step (no host round trip in graph mode 2) and returns
        None; step_results() reads the results later."""
        ids = None if env_ids is None else np.ascontiguousarray(env_ids, dtype=np.int32)
        n = self.n_envs if ids is None else len(ids)
        self._last_n = n
        if not wait:
            self._check(lib().ipc_step(self._ctx, _ptr(ids, _ip), n, None, None), "ipc_step")
            return None
        status = np.zeros(n, dtype=np.int32)
        stats = ipc_step_stats()
        self._check(lib().ipc_step(self._ctx, _ptr(ids, _ip), n, _ptr(status, _ip), C.byref(stats)), "ipc_step")
        return status, {k: getattr(stats, k) for k, _ in ipc_step_stats._fields_}

    def step_results(self):
        """(per-env status array, stats dict) of the last step (synchronises)."""
        status = np.zeros(getattr(self, "_last_n", self.n_envs), dtype=np.int32)
        stats = ipc_step_stats()
        self._check(lib().ipc_step_results(self._ctx, _ptr(status, _ip), C.byref(stats)), "ipc_step_results")
        return status, {k: getattr(stats, k) for k, _ in ipc_step_stats._fields_}

    def rollout(self, n_steps: int, dev_targets, env_ids: Optional[Sequence[int]] = None, wait: bool = True,
                steps_per_env: Optional[Sequence[int]] = None):
        """n_steps steps of each env, every env on its own schedule
        (ipc_rollout).  dev_targets: CUDA float64 tensor
        [n_steps][n_envs][max_bodies][12] (kept alive by this object until
        the results are read), or None without bodies.  steps_per_env
        (aligned with env_ids) caps each env's steps.  Returns (status,
        steps taken, stats dict), or None with wait=False (rollout_results()
        reads them)."""
        ids = None if env_ids is None else np.ascontiguousarray(env_ids, dtype=np.int32)
        n = self.n_envs if ids is None else len(ids)
        lim = None if steps_per_env is None else np.ascontiguousarray(steps_per_env, dtype=np.int32)
        if lim is not None and len(lim) != n:
            raise ValueError("steps_per_env must have one entry per listed env")
        if dev_targets is not None:
            mb = max(self.max_bodies, 1)
            if (not dev_targets.is_cuda or dev_targets.dtype != self._torch_float64()
                    or tuple(dev_targets.shape) != (n_steps, self.n_envs, mb, 12) or not dev_targets.is_contiguous()):
                raise ValueError(f"dev_targets must be a contiguous CUDA float64 tensor of shape "
                                 f"{(n_steps, self.n_envs, mb, 12)}")
        self._roll_n = n
        self._roll_targets = dev_targets
        ptr = None if dev_targets is None else C.c_void_p(dev_targets.data_ptr())
        if not wait:
            self._check(lib().ipc_rollout(self._ctx, _ptr(ids, _ip), n, int(n_steps), _ptr(lim, _ip), ptr, None, None,
                                          None), "ipc_rollout")
            return None
        status = np.zeros(n, dtype=np.int32)
        steps = np.zeros(n, dtype=np.int32)
        stats = ipc_step_stats()
        self._check(lib().ipc_rollout(self._ctx, _ptr(ids, _ip), n, int(n_steps), _ptr(lim, _ip), ptr,
                                      _ptr(status, _ip), _ptr(steps, _ip), C.byref(stats)), "ipc_rollout")
        self._roll_targets = None
        return status, steps, {k: getattr(stats, k) for k, _ in ipc_step_stats._fields_}

    def rollout_results(self):
        """(status, steps taken, stats dict) of the last rollout (synchronises)."""
        n = getattr(self, "_roll_n", self.n_envs)
        status = np.zeros(n, dtype=np.int32)
        steps = np.zeros(n, dtype=np.int32)
        stats = ipc_step_stats()
        self._check(lib().ipc_rollout_results(self._ctx, _ptr(status, _ip), _ptr(steps, _ip), C.byref(stats)),
                    "ipc_rollout_results")
        self._roll_targets = None
        return status, steps, {k: getattr(stats, k) for k, _ in ipc_step_stats._fields_}

    @staticmethod
    def _torch_float64():
        import torch
        return torch.float64

    ENV_STATS = ("status", "newton", "al", "pcg", "ls_trials", "ccd_limited", "accd_max", "pairs", "accd_iters",
                 "pair_evals", "swept_pairs")

    def env_stats(self, env: int) -> dict:
        """Counters of the last step that included `env` (ipc_env_stats)."""
        out = np.zeros(len(self.ENV_STATS), dtype=np.int32)
        self._check(lib().ipc_env_stats(self._ctx, env, _ptr(out, _ip)), "ipc_env_stats")
        return dict(zip(self.ENV_STATS, (int(v) for v in out)))

    def read_gel_surface(self, env: int) -> np.ndarray:
        n = self.sizes[env][2]
        out = np.zeros((n, 3))
        w = C.c_int()
        self._check(lib().ipc_read_gel_surface(self._ctx, env, _ptr(out, _dp), n, C.byref(w)), "ipc_read_gel_surface")
        return out

    @staticmethod
    def _check_out_rows(out: np.ndarray, what: str):
        """A caller's output array must be C-contiguous float64 [rows][3]: the
        library writes 3 doubles per row up to out.shape[0] rows."""
        if not isinstance(out, np.ndarray) or out.dtype != np.float64 or out.ndim != 2 or out.shape[1] != 3 \
                or not out.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{what}: out must be a C-contiguous float64 array of shape (rows, 3), got "
                             f"{getattr(out, 'dtype', type(out))} {getattr(out, 'shape', '')}")

    def read_gel_surface_all(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        tot = sum(s[2] for s in self.sizes)
        if out is None:
            out = np.zeros((tot, 3))
        self._check_out_rows(out, "read_gel_surface_all")
        w = C.c_size_t()
        self._check(lib().ipc_read_gel_surface_all(self._ctx, _ptr(out, _dp), out.shape[0], C.byref(w)),
                    "ipc_read_gel_surface_all")
        return out

    def read_gel_surface_all_noalloc(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        """Same as read_gel_surface_all through the entry point that stages in
        a fixed device array compiled into the library (no device allocation,
        no workspace scratch; at most 262144 rows in total)."""
        tot = sum(s[2] for s in self.sizes)
        if out is None:
            out = np.zeros((tot, 3))
        self._check_out_rows(out, "read_gel_surface_all_noalloc")
        w = C.c_size_t()
        self._check(lib().ipc_read_gel_surface_all_noalloc(self._ctx, _ptr(out, _dp), out.shape[0], C.byref(w)),
                    "ipc_read_gel_surface_all_noalloc")
        return out

    # ------------------------------------------------------------ tactile outputs
    def gel_vertex_rows(self, env: int, verts) -> np.ndarray:
        v = np.ascontiguousarray(verts, dtype=np.int32).ravel()
        out = np.zeros_like(v)
        self._check(lib().ipc_gel_vertex_rows(self._ctx, env, len(v), _ptr(v, _ip), _ptr(out, _ip)),
                    "ipc_gel_vertex_rows")
        return out.reshape(np.shape(verts))

    @staticmethod
    def _sensor(sd) -> "ipc_sensor":
        s = ipc_sensor()
        s.env, s.pad, s.pitch = int(sd["env"]), int(sd.get("pad", 0)), float(sd["pitch"])
        for name in ("origin", "axis_u", "axis_v", "normal"):
            arr = getattr(s, name)
            for k in range(3):
                arr[k] = float(sd[name][k])
        return s

    def sensor_triangles(self, sd) -> np.ndarray:
        """Global row triples of a sensor's front-face triangles."""
        s = self._sensor(sd)
        n = C.c_int(0)
        self._check(lib().ipc_sensor_triangles(self._ctx, C.byref(s), None, 0, C.byref(n)), "ipc_sensor_triangles")
        out = np.zeros((n.value, 3), np.int32)
        self._check(lib().ipc_sensor_triangles(self._ctx, C.byref(s), _ptr(out, _ip), n.value, C.byref(n)),
                    "ipc_sensor_triangles")
        return out

    def prepare_sensors(self, sensors, height: int, width: int) -> dict:
        """Device tables of a set of sensors (dicts with env, pad, origin,
        axis_u, axis_v, normal, pitch), reused by tactile_maps."""
        torch = self._torch
        tris = [self.sensor_triangles(sd) for sd in sensors]
        off = np.concatenate([[0], np.cumsum([len(t) for t in tris])]).astype(np.int32)
        rows = np.concatenate(tris).astype(np.int32) if len(tris) else np.zeros((0, 3), np.int32)
        frames = np.array([list(sd["origin"]) + list(sd["axis_u"]) + list(sd["axis_v"]) + list(sd["normal"])
                           + [sd["pitch"]] for sd in sensors], dtype=np.float64)
        n = len(sensors)
        with torch.cuda.device(self.device):
            return {"n": n, "H": int(height), "W": int(width), "n_tri": int(off[-1]),
                    "frames": torch.as_tensor(frames, device=self.device),
                    "off": torch.as_tensor(off, device=self.device),
                    "rows": torch.as_tensor(rows.reshape(-1, 3), device=self.device),
                    "keys": torch.empty((n, height, width), dtype=torch.int64, device=self.device)}

    def tactile_maps(self, prep: dict, normals: bool = True):
        """(depth [n, H, W], normal [n, H, W, 3] or None, hit [n, H, W] uint8),
        CUDA tensors written on the ctx stream."""
        torch = self._torch
        n, H, W = prep["n"], prep["H"], prep["W"]
        depth = torch.empty((n, H, W), dtype=torch.float64, device=self.device)
        normal = torch.empty((n, H, W, 3), dtype=torch.float64, device=self.device) if normals else None
        hit = torch.empty((n, H, W), dtype=torch.uint8, device=self.device)
        self._check(lib().ipc_tactile_maps_device(self._ctx, n, H, W, _vp(prep["frames"]), _vp(prep["off"]),
                                                  _vp(prep["rows"]), prep["n_tri"], _vp(prep["keys"]), _vp(depth),
                                                  _vp(normal), _vp(hit)), "ipc_tactile_maps_device")
        return depth, normal, hit

    def prepare_markers(self, env: int, tri_verts, bary) -> dict:
        """Device tables of markers on coated triangles of one env: tri_verts
        [m, 3] user vertex ids, bary [m, 3]; the rest positions are taken
        from the env's current state (call before stepping for flows)."""
        torch = self._torch
        rows = self.gel_vertex_rows(env, tri_verts).astype(np.int32)
        with torch.cuda.device(self.device):
            prep = {"m": rows.shape[0], "rows": torch.as_tensor(rows, device=self.device),
                    "bary": torch.as_tensor(np.asarray(bary, dtype=np.float64), device=self.device)}
        prep["rest"], _ = self.markers(prep)
        return prep

    def markers(self, prep: dict):
        """(positions [m, 3], flows [m, 3] or None) as CUDA tensors."""
        torch = self._torch
        m = prep["m"]
        pos = torch.empty((m, 3), dtype=torch.float64, device=self.device)
        rest = prep.get("rest")
        flow = torch.empty((m, 3), dtype=torch.float64, device=self.device) if rest is not None else None
        self._check(lib().ipc_markers_device(self._ctx, m, _vp(prep["rows"]), _vp(prep["bary"]), _vp(rest),
                                             _vp(pos), _vp(flow)), "ipc_markers_device")
        return pos, flow

    def autotune(self, reps: int = 10) -> dict:
        """Pick the PCG mat-vec's slots in flight per lane and the persistent
        PCG grid by timing them on this batch's current system (call between
        steps)."""
        t = ipc_tuning()
        self._check(lib().ipc_autotune(self._ctx, int(reps), C.byref(t)), "ipc_autotune")
        return {"spmv_unroll": t.spmv_unroll, "pcg_ctas_per_sm": t.pcg_ctas_per_sm,
                "spmv_us": {u: round(float(t.spmv_us[k]), 2) for k, u in enumerate((2, 4, 8))},
                "grid_us": {int(t.grid_ctas_per_sm[k]): round(float(t.grid_us[k]), 2) for k in range(3)},
                "assemble_block": t.assemble_block,
                "assemble_us": {b: round(float(t.assemble_us[k]), 2) for k, b in enumerate((64, 128, 256))},
                "pairs_ctas_per_sm": t.pairs_ctas_per_sm,
                "pairs_us": {c: round(float(t.pairs_us[k]), 2) for k, c in enumerate((4, 8, 16))},
                "pcg_iter_bound": t.pcg_iter_bound,
                "pcg_iter_us": {b: round(float(t.pcg_iter_us[k]), 2) for k, b in enumerate((1, 0))}}

    def set_graph_mode(self, mode=1):
        """CUDA-graph execution: 0 plain launches, 1 (or True) each PCG solve
        as one graph, 2 the whole step as one graph.  Needs a capturable
        stream: pass stream= a torch.cuda.Stream at creation."""
        mode = int(mode) if not isinstance(mode, bool) else (1 if mode else 0)
        self._check(lib().ipc_set_graph_mode(self._ctx, mode), "ipc_set_graph_mode")

    # ------------------------------------------------------------ profiling
    def profile_enable(self, on: bool = True):
        self._check(lib().ipc_profile_enable(self._ctx, 1 if on else 0), "ipc_profile_enable")

    def profile_reset(self):
        self._check(lib().ipc_profile_reset(self._ctx), "ipc_profile_reset")

    def profile(self) -> dict:
        """{kernel class: (launches, device ms)} since the last reset."""
        out = {}
        for i in range(lib().ipc_profile_count(self._ctx)):
            name, n, ms = C.c_char_p(), C.c_longlong(), C.c_double()
            self._check(lib().ipc_profile_get(self._ctx, i, C.byref(name), C.byref(n), C.byref(ms)),
                        "ipc_profile_get")
            out[name.value.decode()] = (int(n.value), float(ms.value))
        return out

    def check_report(self) -> dict:
        """First bounds violation recorded by a checked build (ipc_check_report)."""
        built, code, idx = C.c_int(), C.c_int(), C.c_longlong()
        self._check(lib().ipc_check_report(self._ctx, C.byref(built), C.byref(code), C.byref(idx)),
                    "ipc_check_report")
        return {"checks_built": bool(built.value), "code": int(code.value), "index": int(idx.value)}

    def launch_count(self) -> int:
        return int(lib().ipc_launch_count(self._ctx))

    def system_sizes(self, env: int) -> dict:
        rb, sb, r, t = C.c_longlong(), C.c_longlong(), C.c_int(), C.c_int()
        self._check(lib().ipc_system_sizes(self._ctx, env, C.byref(rb), C.byref(sb), C.byref(r), C.byref(t)),
                    "ipc_system_sizes")
        return {"real_blocks": rb.value, "stored_blocks": sb.value, "rows": r.value, "tets": t.value}

    # ------------------------------------------------------------ diagnostics
    def ndof(self, env: int) -> int:
        nv, nb, _ = self.sizes[env]
        return 3 * nv + 12 * nb

    def debug_eval(self, env: int, vec: Optional[np.ndarray] = None):
        n = self.ndof(env)
        E = np.zeros(1)
        g = np.zeros(n)
        hv = np.zeros(n) if vec is not None else None
        v = None if vec is None else np.ascontiguousarray(vec, dtype=np.float64)
        self._check(lib().ipc_debug_eval(self._ctx, env, _ptr(E, _dp), _ptr(g, _dp), _ptr(v, _dp), _ptr(hv, _dp)),
                    "ipc_debug_eval")
        return float(E[0]), g, hv

    def debug_pairs(self, env: int, cv_x: np.ndarray, cv_x_end: Optional[np.ndarray] = None, capacity=None):
        cap = capacity or 200000
        out = np.zeros((cap, 5), dtype=np.int32)
        n = C.c_int()
        a = np.ascontiguousarray(cv_x, dtype=np.float64)
        b = None if cv_x_end is None else np.ascontiguousarray(cv_x_end, dtype=np.float64)
        st = lib().ipc_debug_pairs(self._ctx, env, _ptr(a, _dp), _ptr(b, _dp), _ptr(out, _ip), cap, C.byref(n))
        self._check(st, "ipc_debug_pairs")
        return out[:min(n.value, cap)]

    def debug_newton_dir(self, env: int):
        p = np.zeros(self.ndof(env))
        it = C.c_int()
        self._check(lib().ipc_debug_newton_dir(self._ctx, env, _ptr(p, _dp), C.byref(it)), "ipc_debug_newton_dir")
        return p, it.value

    def debug_pcg_wait_out(self, env: int):
        """Make the multi-iteration PCG kernel's bounded waits run out for
        env (ipc_debug_pcg_wait_out): (the env's status, the launch's ms)."""
        st, ms = C.c_int(), C.c_float()
        self._check(lib().ipc_debug_pcg_wait_out(self._ctx, env, C.byref(st), C.byref(ms)), "ipc_debug_pcg_wait_out")
        return st.value, float(ms.value)

    def debug_accd(self, env: int, direction: np.ndarray) -> float:
        a = np.zeros(1)
        d = np.ascontiguousarray(direction, dtype=np.float64)
        self._check(lib().ipc_debug_accd(self._ctx, env, _ptr(d, _dp), _ptr(a, _dp)), "ipc_debug_accd")
        return float(a[0])


# ---------------------------------------------------------------- element kernels
def _stream_ptr(t):
    import torch
    return C.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _vp(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _filter_code(project) -> int:
    """Eigenvalue filter code of the element kernels: False -> 0 (raw),
    True / "clamp" -> 1, "abs" -> 2."""
    if not project:
        return 0
    return 2 if project == "abs" else 1


def k_tet(x, Dm_inv, vol, mu: float, lam: float, energy=None, grad=None, hess=None, project=True):
    """Neo-Hookean element kernel on torch float64 CUDA tensors."""
    n = int(x.shape[0])
    st = lib().ipc_k_tet(n, _vp(x), _vp(Dm_inv), _vp(vol), float(mu), float(lam), _vp(energy), _vp(grad),
                         _vp(hess), _filter_code(project), _stream_ptr(x))
    if st != IPC_OK:
        raise IpcError(st, "ipc_k_tet")


def k_barrier(X, is_ee, weight, eps_x, dhat: float, energy=None, grad=None, hess=None, project=True,
              hess_fp32=False):
    """Pair barrier element kernel on torch CUDA tensors; hess_fp32 forms and
    projects the Hessian in FP32 (the mixed-precision step's arithmetic)."""
    n = int(X.shape[0])
    st = lib().ipc_k_barrier(n, _vp(X), _vp(is_ee), _vp(weight), _vp(eps_x), float(dhat), _vp(energy), _vp(grad),
                             _vp(hess), _filter_code(project) | (8 if hess_fp32 else 0), _stream_ptr(X))
    if st != IPC_OK:
        raise IpcError(st, "ipc_k_barrier")


def k_accd(X0, P, is_ee, s: float, max_iter: int, toi, iters=None):
    n = int(X0.shape[0])
    st = lib().ipc_k_accd(n, _vp(X0), _vp(P), _vp(is_ee), float(s), int(max_iter), _vp(toi), _vp(iters),
                          _stream_ptr(X0))
    if st != IPC_OK:
        raise IpcError(st, "ipc_k_accd")


def fma_peaks(device="cuda:0") -> dict:
    """Measured FP64 / FP32 FMA throughput of the device, TFLOP/s."""
    import torch
    dev = torch.device(device)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    buf = torch.empty(n_sm * 8 * 256, dtype=torch.float64, device=dev)
    f64, f32 = C.c_double(), C.c_double()
    st = lib().ipc_fma_peaks(_vp(buf), buf.numel() * 8, C.byref(f64), C.byref(f32), _stream_ptr(buf))
    if st != IPC_OK:
        raise IpcError(st, "ipc_fma_peaks")
    return {"fp64_tflops": f64.value, "fp32_tflops": f32.value}
