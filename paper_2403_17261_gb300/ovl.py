"""Thin ctypes binding of libovl (the C ABI declared in ``include/ovl.h``).

Functions keep the C names (``ovl_create``, ``ovl_step``, ...) and only
marshal arguments; every step of the method runs in the library's CUDA
kernels (and its host-side membership code).  ``Simulation`` bundles a
context with numpy/torch conveniences.

There is no fallback: if the library is missing or cannot be loaded,
``load_library`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

# The library launches a step's per-class kernels on up to seven streams; with
# CUDA's default of 8 hardware queues some of them would share one and run in
# turn.  The setting counts only if it is in place before the process first
# uses CUDA (importing this module before torch initialises CUDA is enough).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libovl.so")

OVL_OK = 0
OVL_ERR_ARG = -1
OVL_ERR_CUDA = -2
OVL_ERR_CAPACITY = -3
OVL_ERR_TIMEOUT = -4
OVL_ERR_NONFINITE = -5
OVL_ERR_MEMBERSHIP = -6
OVL_FLAG_RESIDUAL = 1
OVL_FLAG_TIMING = 2
OVL_FLAG_AUTOTUNE = 4
OVL_FLAG_FEATURES = 8
OVL_WS_PREVIOUS, OVL_WS_MLP, OVL_WS_MLP_NEW = 0, 1, 2
OVL_LB_BODIES, OVL_LB_CONTACTS = 0, 1
OVL_WEIGHTS_GEODESIC, OVL_WEIGHTS_UNIFORM = 0, 1
OVL_MLP_N_PARAMS = 5187
OVL_N_FEATURES = 12

EXPORTED = [
    "ovl_default_params", "ovl_create", "ovl_destroy", "ovl_last_error", "ovl_phase_name",
    "ovl_scene_upload", "ovl_set_partition", "ovl_set_membership", "ovl_read_membership",
    "ovl_assign_overlap", "ovl_set_state", "ovl_read_state", "ovl_set_step_index",
    "ovl_set_warmstart", "ovl_read_warmstart", "ovl_step", "ovl_load_balance", "ovl_sync", "ovl_joint_error",
    "ovl_read_stats", "ovl_read_contacts", "ovl_read_graph", "ovl_read_entries", "ovl_read_pairs",
    "ovl_read_worker_stats", "ovl_read_solve_plan", "ovl_read_contact_points", "ovl_step_n", "ovl_save", "ovl_load", "ovl_autotune_export", "ovl_autotune_import",
    "ovl_geodesics_static", "ovl_set_warmstart_mode", "ovl_read_features", "ovl_mlp_set_params",
    "ovl_mlp_get_params", "ovl_mlp_forward", "ovl_log_reserve", "ovl_log_enable", "ovl_log_size",
    "ovl_log_append", "ovl_log_read", "ovl_mlp_train", "ovl_mlp_grad", "ovl_mlp_loss",
    "ovl_host_load_balance", "ovl_host_assign_overlap",
    "ovl_box_plane_contacts", "ovl_sphere_box_contacts", "ovl_box_box_contacts", "ovl_box_plane_step",
    "ovl_box_scene_contacts",
]


class OvlError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libovl error {code}: {msg}")
        self.code = code


class ovl_params(C.Structure):
    _fields_ = [("gravity", C.c_float * 3), ("margin", C.c_float), ("erp", C.c_float),
                ("slop", C.c_float), ("warmstart", C.c_float), ("lb_activate", C.c_int32),
                ("lb_deact_every", C.c_int32), ("res_tol", C.c_float),
                ("res_check_every", C.c_int32), ("pgs_threads", C.c_int32), ("flags", C.c_int32),
                ("pgs_cluster", C.c_int32), ("smem_slot_limit", C.c_int32),
                ("lb_load", C.c_int32), ("weights", C.c_int32)]


_fp, _ip, _u64p, _u8p = C.POINTER(C.c_float), C.POINTER(C.c_int32), C.POINTER(C.c_uint64), C.POINTER(C.c_uint8)


class ovl_train_desc(C.Structure):
    _fields_ = [("first", C.c_int64), ("count", C.c_int64), ("batch", C.c_int32),
                ("steps", C.c_int32), ("sampling", C.c_int32), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("seed", C.c_uint64)]


class ovl_scene_desc(C.Structure):
    _fields_ = [("n_bodies", C.c_int32), ("state", _fp), ("radius", _fp), ("inv_mass", _fp),
                ("n_planes", C.c_int32), ("planes", _fp), ("plane_scene", _ip),
                ("n_joints", C.c_int32), ("joint_bodies", _ip), ("joint_anchors", _fp),
                ("n_scenes", C.c_int32), ("scene_of_body", _ip), ("scene_mu", _fp),
                ("scene_dt", _fp), ("scene_flags", _ip), ("scene_gamma", _ip), ("scene_beta", _ip),
                ("n_sets", _ip), ("half_extents", _fp)]


class ovl_stats(C.Structure):
    _fields_ = [("n_contacts", C.c_int64), ("n_adjacency", C.c_int64), ("n_entries", C.c_int64),
                ("n_pairs", C.c_int64), ("n_rows", C.c_int64), ("n_overlap", C.c_int64),
                ("n_workers", C.c_int32), ("max_colours", C.c_int32), ("max_iters", C.c_int32),
                ("device_status", C.c_int32), ("residual_rms", C.c_double),
                ("residual_max", C.c_double), ("phase_ms", C.c_float * 12),
                ("n_launches", C.c_int64), ("solve_cluster", C.c_int32), ("solve_threads", C.c_int32),
                ("solve_rows_per_thread", C.c_int32), ("colour_rounds_max", C.c_int32),
                ("lb_candidates", C.c_int64), ("lb_host_ms", C.c_double),
                ("solve_ctas", C.c_int64), ("solve_ctas_masses", C.c_int64)]


_lib = None


def load_library(path: str | None = None):
    """Loads libovl.so (built by ``build.py``); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OvlError(OVL_ERR_CUDA, f"{p} is missing: build it with paper_2403_17261_gb300.build.build()")
    L = C.CDLL(p)
    vp = C.c_void_p
    sig = {
        "ovl_default_params": [C.POINTER(ovl_params)],
        "ovl_create": [C.POINTER(vp), C.POINTER(ovl_params), vp],
        "ovl_destroy": [vp],
        "ovl_scene_upload": [vp, C.POINTER(ovl_scene_desc)],
        "ovl_set_partition": [vp, _ip],
        "ovl_set_membership": [vp, _u64p],
        "ovl_read_membership": [vp, _u64p],
        "ovl_assign_overlap": [vp],
        "ovl_set_state": [vp, vp, C.c_int32],
        "ovl_read_state": [vp, vp, C.c_int32],
        "ovl_set_step_index": [vp, C.c_int64],
        "ovl_set_warmstart": [vp, C.c_int64, _ip, _u64p, _fp],
        "ovl_read_warmstart": [vp, C.c_int64, C.POINTER(C.c_int64), _ip, _u64p, _fp],
        "ovl_step": [vp, C.c_float, C.c_int32],
        "ovl_load_balance": [vp, C.c_int32],
        "ovl_joint_error": [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "ovl_sync": [vp],
        "ovl_read_stats": [vp, C.POINTER(ovl_stats)],
        "ovl_read_contacts": [vp, _ip, _fp, _fp, _fp],
        "ovl_read_graph": [vp, _ip, _ip],
        "ovl_read_entries": [vp, _ip, _ip, _u8p, _fp, _fp],
        "ovl_read_pairs": [vp, _ip, _u64p, _ip, _fp],
        "ovl_read_worker_stats": [vp, _ip, C.POINTER(C.c_double), C.POINTER(C.c_int64), _ip],
        "ovl_read_solve_plan": [vp, _ip],
        "ovl_read_contact_points": [vp, _ip, _fp],
        "ovl_step_n": [vp, C.c_float, C.c_int32, C.c_int32, _ip],
        "ovl_save": [vp, vp, C.c_size_t, C.POINTER(C.c_size_t)],
        "ovl_load": [vp, vp, C.c_size_t],
        "ovl_autotune_export": [vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)],
        "ovl_autotune_import": [vp, C.c_char_p],
        "ovl_set_warmstart_mode": [vp, C.c_int32],
        "ovl_read_features": [vp, _fp, _fp, _ip, _fp],
        "ovl_mlp_set_params": [vp, _fp, C.c_int32],
        "ovl_mlp_get_params": [vp, _fp, C.c_int32],
        "ovl_mlp_forward": [vp, C.c_int64, _fp, _fp],
        "ovl_log_reserve": [vp, C.c_int64],
        "ovl_log_enable": [vp, C.c_int32],
        "ovl_log_size": [vp, C.POINTER(C.c_int64)],
        "ovl_log_append": [vp, C.c_int64, _fp, _fp],
        "ovl_log_read": [vp, C.c_int64, C.c_int64, _fp, _fp],
        "ovl_mlp_train": [vp, C.POINTER(ovl_train_desc), _fp],
        "ovl_mlp_grad": [vp, C.c_int64, C.c_int64, _fp, C.POINTER(C.c_double)],
        "ovl_mlp_loss": [vp, C.c_int64, C.c_int64, C.POINTER(C.c_double)],
        "ovl_geodesics_static": [C.c_int32, C.c_int32, C.c_int32, vp, vp, C.c_int32, vp, vp,
                                 C.c_int32, vp, vp, C.c_char_p, C.c_int32],
        "ovl_host_load_balance": [C.c_int32, _ip, C.c_int32, _ip, _ip, _u64p, _ip, _ip, C.c_int64, _ip, _ip,
                                  C.c_int32, C.c_int32, C.c_int32],
        "ovl_host_assign_overlap": [C.c_int32, _ip, C.c_int32, _ip, _ip, _fp, C.c_int32, _ip, _u64p],
        "ovl_box_plane_contacts": [C.c_int32, _fp, _fp, _fp, C.c_float, C.c_int32, _ip, _fp, _fp, _fp],
        "ovl_sphere_box_contacts": [C.c_int32, _fp, _fp, _fp, C.c_float, C.c_int32, _ip, _fp, _fp, _fp],
        "ovl_box_box_contacts": [C.c_int32, _fp, _fp, _fp, _fp, C.c_float, C.c_int32, _ip, _fp, _fp, _fp, _ip],
        "ovl_box_plane_step": [C.c_int32, _fp, _fp, _fp, _fp, C.c_float, C.c_float, _fp, C.c_float, C.c_float,
                               C.c_float, C.c_int32, C.c_int32, _fp, _ip, _fp],
        "ovl_box_scene_contacts": [C.c_int32, _fp, _fp, _fp, _fp, _ip, C.c_int32, _ip, C.c_int32, _fp, _ip,
                                   C.c_float, C.c_int32, C.c_int64, C.POINTER(C.c_int64), _ip, _ip, _fp, _fp, _fp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int32
    L.ovl_last_error.argtypes = [vp]
    L.ovl_last_error.restype = C.c_char_p
    L.ovl_phase_name.argtypes = [C.c_int32]
    L.ovl_phase_name.restype = C.c_char_p
    if path is None:
        _lib = L
    return L


def _check(ctx, rc: int):
    if rc != OVL_OK:
        msg = load_library().ovl_last_error(ctx).decode() if ctx else "no context"
        raise OvlError(rc, msg)


def _ptr(a, t):
    return a.ctypes.data_as(t)


# ---------------------------------------------------------------------------
# functions with the C names
# ---------------------------------------------------------------------------

def ovl_default_params(**overrides) -> ovl_params:
    p = ovl_params()
    load_library().ovl_default_params(C.byref(p))
    for k, v in overrides.items():
        if k == "gravity":
            for i in range(3):
                p.gravity[i] = v[i]
        else:
            setattr(p, k, v)
    return p


def ovl_create(params: ovl_params | None = None, stream: int | None = None):
    h = C.c_void_p()
    rc = load_library().ovl_create(C.byref(h), C.byref(params) if params is not None else None,
                                   C.c_void_p(stream) if stream else None)
    if rc != OVL_OK:
        raise OvlError(rc, "ovl_create failed (is a CUDA device available?)")
    return h


def ovl_destroy(ctx):
    load_library().ovl_destroy(ctx)


class _SceneArrays:
    """Keeps the contiguous host arrays alive for the duration of the upload."""

    def __init__(self, scene):
        he = getattr(scene, "half_extents", None)
        f32 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.float32))
        self.half = None if he is None else f32(he).reshape(-1, 3)
        i32 = lambda a: np.ascontiguousarray(np.asarray(a, dtype=np.int32))
        self.state = f32(scene.state).reshape(-1, 13)
        self.radius, self.inv_mass = f32(scene.radius), f32(scene.inv_mass)
        self.planes = f32(scene.planes).reshape(-1, 4)
        self.plane_scene = i32(scene.plane_scene)
        self.joints = i32(scene.joints).reshape(-1, 2)
        self.anchors = f32(scene.anchors).reshape(-1, 6)
        self.sob = i32(scene.scene_of_body)
        self.mu, self.dt = f32(scene.scene_mu), f32(scene.scene_dt)
        self.flags, self.gamma = i32(scene.scene_flags), i32(scene.scene_gamma)
        self.beta, self.n_sets = i32(scene.scene_beta), i32(scene.n_sets)
        d = ovl_scene_desc()
        d.n_bodies = self.state.shape[0]
        d.state, d.radius, d.inv_mass = _ptr(self.state, _fp), _ptr(self.radius, _fp), _ptr(self.inv_mass, _fp)
        d.n_planes = self.planes.shape[0]
        d.planes, d.plane_scene = _ptr(self.planes, _fp), _ptr(self.plane_scene, _ip)
        d.n_joints = self.joints.shape[0]
        d.joint_bodies, d.joint_anchors = _ptr(self.joints, _ip), _ptr(self.anchors, _fp)
        d.n_scenes = self.mu.shape[0]
        d.scene_of_body = _ptr(self.sob, _ip)
        d.scene_mu, d.scene_dt = _ptr(self.mu, _fp), _ptr(self.dt, _fp)
        d.scene_flags, d.scene_gamma = _ptr(self.flags, _ip), _ptr(self.gamma, _ip)
        d.scene_beta, d.n_sets = _ptr(self.beta, _ip), _ptr(self.n_sets, _ip)
        d.half_extents = _ptr(self.half, _fp) if self.half is not None else None
        self.desc = d


def ovl_scene_upload(ctx, scene):
    arr = _SceneArrays(scene)
    _check(ctx, load_library().ovl_scene_upload(ctx, C.byref(arr.desc)))


def ovl_set_partition(ctx, set_of_body):
    s = np.ascontiguousarray(np.asarray(set_of_body, dtype=np.int32))
    _check(ctx, load_library().ovl_set_partition(ctx, _ptr(s, _ip)))


def ovl_set_membership(ctx, masks):
    m = np.ascontiguousarray(np.asarray(masks, dtype=np.uint64))
    _check(ctx, load_library().ovl_set_membership(ctx, _ptr(m, _u64p)))


def ovl_read_membership(ctx, n):
    m = np.zeros(n, np.uint64)
    _check(ctx, load_library().ovl_read_membership(ctx, _ptr(m, _u64p)))
    return m


def ovl_assign_overlap(ctx):
    _check(ctx, load_library().ovl_assign_overlap(ctx))


def ovl_set_state(ctx, state, on_device: bool = False):
    if on_device:
        _check(ctx, load_library().ovl_set_state(ctx, C.c_void_p(int(state)), 1))
    else:
        s = np.ascontiguousarray(np.asarray(state, dtype=np.float32))
        _check(ctx, load_library().ovl_set_state(ctx, s.ctypes.data_as(C.c_void_p), 0))


def ovl_read_state(ctx, out, on_device: bool = False):
    if on_device:
        _check(ctx, load_library().ovl_read_state(ctx, C.c_void_p(int(out)), 1))
    else:
        assert out.dtype == np.float32 and out.flags["C_CONTIGUOUS"]
        _check(ctx, load_library().ovl_read_state(ctx, out.ctypes.data_as(C.c_void_p), 0))
    return out


def ovl_set_step_index(ctx, k: int):
    _check(ctx, load_library().ovl_set_step_index(ctx, int(k)))


def ovl_set_warmstart(ctx, part, key, lam):
    part = np.ascontiguousarray(np.asarray(part, dtype=np.int32))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float32)).reshape(-1, 3)
    _check(ctx, load_library().ovl_set_warmstart(ctx, part.shape[0], _ptr(part, _ip), _ptr(key, _u64p),
                                                 _ptr(lam, _fp)))


def ovl_read_warmstart(ctx):
    n = C.c_int64()
    L = load_library()
    _check(ctx, L.ovl_read_warmstart(ctx, 0, C.byref(n), None, None, None))
    m = n.value
    part, key, lam = np.zeros(max(m, 1), np.int32), np.zeros(max(m, 1), np.uint64), np.zeros((max(m, 1), 3), np.float32)
    _check(ctx, L.ovl_read_warmstart(ctx, m, C.byref(n), _ptr(part, _ip), _ptr(key, _u64p), _ptr(lam, _fp)))
    return part[:m], key[:m], lam[:m]


def ovl_step(ctx, dt: float, iters: int):
    _check(ctx, load_library().ovl_step(ctx, float(dt), int(iters)))


def ovl_load_balance(ctx, flags: int = 3):
    _check(ctx, load_library().ovl_load_balance(ctx, int(flags)))


def ovl_sync(ctx):
    _check(ctx, load_library().ovl_sync(ctx))


def ovl_autotune_export(ctx) -> str:
    n = C.c_size_t()
    L = load_library()
    _check(ctx, L.ovl_autotune_export(ctx, None, 0, C.byref(n)))
    buf = C.create_string_buffer(n.value + 1)
    _check(ctx, L.ovl_autotune_export(ctx, buf, n.value + 1, C.byref(n)))
    return buf.value.decode()


def ovl_autotune_import(ctx, text: str):
    _check(ctx, load_library().ovl_autotune_import(ctx, text.encode()))


def _dev_ptr(a):
    """Device address of a CUDA tensor (anything with data_ptr()) or an int."""
    return C.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else int(a))


def ovl_geodesics_static(n_bodies: int, n_workers: int, beta: int, row_ptr, col, n_adj: int,
                         mask, entry_ptr, n_entries: int, D, stream: int | None = None):
    """D(o,i) of one scene into the device array D, allocating no device memory.

    Arrays are device arrays (CUDA tensors or raw addresses): row_ptr int32
    [n+1], col int32 [n_adj], mask uint64/int64 [n], entry_ptr int32 [n+1],
    D uint8 [n_entries].  Overlapping calls on one device race; see ovl.h."""
    buf = C.create_string_buffer(256)
    rc = load_library().ovl_geodesics_static(
        n_bodies, n_workers, beta, _dev_ptr(row_ptr), _dev_ptr(col), n_adj, _dev_ptr(mask),
        _dev_ptr(entry_ptr), n_entries, _dev_ptr(D), C.c_void_p(stream) if stream else None,
        buf, len(buf))
    if rc != OVL_OK:
        raise OvlError(rc, buf.value.decode())


def _i32c(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def ovl_host_load_balance(masks, scene_of_body, n_sets, scene_gamma, row_ptr, col, contact_pairs,
                          contact_count=None, do_activate: bool = True, do_deactivate: bool = True,
                          threads: int = 1):
    """Algorithm 6 (with Algorithm 7) by the library's host code, no GPU
    needed; returns the new masks (the input is not modified)."""
    m = np.array(masks, dtype=np.uint64, copy=True)
    sob, ns, sg = _i32c(scene_of_body), _i32c(n_sets), _i32c(scene_gamma)
    rp, cl = _i32c(row_ptr), _i32c(col)
    cp = _i32c(contact_pairs).reshape(-1, 2)
    cc = None if contact_count is None else _i32c(contact_count)
    rc = load_library().ovl_host_load_balance(
        m.shape[0], _ptr(sob, _ip), ns.shape[0], _ptr(ns, _ip), _ptr(sg, _ip), _ptr(m, _u64p),
        _ptr(rp, _ip), _ptr(cl, _ip), cp.shape[0], _ptr(cp, _ip), None if cc is None else _ptr(cc, _ip),
        int(do_activate), int(do_deactivate), int(threads))
    _check(None, rc)
    return m


def ovl_host_assign_overlap(masks, scene_of_body, n_sets, scene_gamma, inv_mass, joints):
    """Algorithms 2-3 by the library's host code, no GPU needed; returns the
    new masks (the input is not modified)."""
    m = np.array(masks, dtype=np.uint64, copy=True)
    sob, ns, sg = _i32c(scene_of_body), _i32c(n_sets), _i32c(scene_gamma)
    im = np.ascontiguousarray(inv_mass, dtype=np.float32)
    j = _i32c(joints).reshape(-1, 2)
    rc = load_library().ovl_host_assign_overlap(
        m.shape[0], _ptr(sob, _ip), ns.shape[0], _ptr(ns, _ip), _ptr(sg, _ip),
        _ptr(im, _fp), j.shape[0], _ptr(j, _ip), _ptr(m, _u64p))
    _check(None, rc)
    return m


def _f32c(a, cols):
    return np.ascontiguousarray(a, dtype=np.float32).reshape(-1, cols)


def _box_out(n):
    return (np.zeros(n, np.int32), np.zeros((n, 4, 3), np.float32), np.zeros((n, 4), np.float32),
            np.zeros((n, 3), np.float32))


def ovl_box_plane_contacts(pose, half, plane, margin: float, on_gpu: bool = True):
    """Box-plane contacts per pair (pose [n,7], half [n,3], plane [n,4]).
    Returns (count, points [n,4,3], gaps [n,4], normal [n,3])."""
    pose, half, plane = _f32c(pose, 7), _f32c(half, 3), _f32c(plane, 4)
    n = pose.shape[0]
    cnt, pts, gaps, nrm = _box_out(n)
    _check(None, load_library().ovl_box_plane_contacts(
        n, _ptr(pose, _fp), _ptr(half, _fp), _ptr(plane, _fp), float(margin), int(on_gpu), _ptr(cnt, _ip),
        _ptr(pts, _fp), _ptr(gaps, _fp), _ptr(nrm, _fp)))
    return cnt, pts, gaps, nrm


def ovl_sphere_box_contacts(sphere, pose, half, margin: float, on_gpu: bool = True):
    """Sphere-box contacts per pair (sphere [n,4] = centre, radius).  Returns
    (count, points [n,4,3], gaps [n,4], normal [n,3]); gaps[:, 0] always
    holds the gap."""
    sphere, pose, half = _f32c(sphere, 4), _f32c(pose, 7), _f32c(half, 3)
    n = pose.shape[0]
    cnt, pts, gaps, nrm = _box_out(n)
    _check(None, load_library().ovl_sphere_box_contacts(
        n, _ptr(sphere, _fp), _ptr(pose, _fp), _ptr(half, _fp), float(margin), int(on_gpu), _ptr(cnt, _ip),
        _ptr(pts, _fp), _ptr(gaps, _fp), _ptr(nrm, _fp)))
    return cnt, pts, gaps, nrm


def ovl_box_box_contacts(pose_a, half_a, pose_b, half_b, margin: float, on_gpu: bool = True):
    """Box-box contacts per pair.  Returns (count, points [n,4,3], gaps [n,4],
    normal [n,3], axis [n])."""
    pa, ha, pb, hb = _f32c(pose_a, 7), _f32c(half_a, 3), _f32c(pose_b, 7), _f32c(half_b, 3)
    n = pa.shape[0]
    cnt, pts, gaps, nrm = _box_out(n)
    axis = np.zeros(n, np.int32)
    _check(None, load_library().ovl_box_box_contacts(
        n, _ptr(pa, _fp), _ptr(ha, _fp), _ptr(pb, _fp), _ptr(hb, _fp), float(margin), int(on_gpu),
        _ptr(cnt, _ip), _ptr(pts, _fp), _ptr(gaps, _fp), _ptr(nrm, _fp), _ptr(axis, _ip)))
    return cnt, pts, gaps, nrm, axis


def ovl_box_plane_step(pose, half, inv_mass, plane, vel, mu=0.5, dt=1 / 60, gravity=(0.0, 0.0, -9.81), erp=0.2,
                       slop=0.0, margin=0.02, iters=200, on_gpu: bool = True):
    """One velocity step of independent boxes on their static planes (box
    rows).  vel [n,6] = (v, omega).  Returns (vel' [n,6], count [n],
    impulses [n,4,3] as (n, t1, t2) per contact)."""
    pose, half, plane = _f32c(pose, 7), _f32c(half, 3), _f32c(plane, 4)
    im = np.ascontiguousarray(inv_mass, dtype=np.float32).reshape(-1)
    v = np.array(vel, dtype=np.float32, copy=True).reshape(-1, 6)
    g = np.ascontiguousarray(gravity, dtype=np.float32).reshape(3)
    n = pose.shape[0]
    cnt, lam = np.zeros(n, np.int32), np.zeros((n, 4, 3), np.float32)
    _check(None, load_library().ovl_box_plane_step(
        n, _ptr(pose, _fp), _ptr(half, _fp), _ptr(im, _fp), _ptr(plane, _fp), float(mu), float(dt), _ptr(g, _fp),
        float(erp), float(slop), float(margin), int(iters), int(on_gpu), _ptr(v, _fp), _ptr(cnt, _ip),
        _ptr(lam, _fp)))
    return v, cnt, lam


def ovl_box_scene_contacts(scene, margin: float = 0.05, on_gpu: bool = True, cap: int | None = None):
    """All contacts of a scene with boxes (Scene with half_extents), in
    canonical order.  Returns dict(ab [m,2], k [m], phi [m], normal [m,3],
    point [m,3])."""
    st = np.ascontiguousarray(scene.state, dtype=np.float32).reshape(-1, 13)
    n = st.shape[0]
    rad = np.ascontiguousarray(scene.radius, dtype=np.float32)
    im = np.ascontiguousarray(scene.inv_mass, dtype=np.float32)
    he = np.zeros((n, 3), np.float32) if scene.half_extents is None else _f32c(scene.half_extents, 3)
    sob = np.ascontiguousarray(scene.scene_of_body, dtype=np.int32)
    sf = np.ascontiguousarray(scene.scene_flags, dtype=np.int32)
    pl = _f32c(scene.planes, 4)
    ps = np.ascontiguousarray(scene.plane_scene, dtype=np.int32)
    L = load_library()
    total = C.c_int64(0)
    cap = 16 * n + 64 if cap is None else cap
    while True:
        ab, k = np.zeros((cap, 2), np.int32), np.zeros(cap, np.int32)
        phi, nrm, pt = np.zeros(cap, np.float32), np.zeros((cap, 3), np.float32), np.zeros((cap, 3), np.float32)
        rc = L.ovl_box_scene_contacts(n, _ptr(st, _fp), _ptr(rad, _fp), _ptr(im, _fp), _ptr(he, _fp), _ptr(sob, _ip),
                                      sf.shape[0], _ptr(sf, _ip), pl.shape[0], _ptr(pl, _fp), _ptr(ps, _ip),
                                      float(margin), int(on_gpu), cap, C.byref(total), _ptr(ab, _ip), _ptr(k, _ip),
                                      _ptr(phi, _fp), _ptr(nrm, _fp), _ptr(pt, _fp))
        if rc == OVL_ERR_CAPACITY:
            cap = int(total.value)
            continue
        _check(None, rc)
        m = int(total.value)
        return dict(ab=ab[:m], k=k[:m], phi=phi[:m], normal=nrm[:m], point=pt[:m])


def ovl_step_n(ctx, dt: float, iters: int, nsteps: int) -> int:
    """nsteps timesteps; returns the number completed (raises on an error)."""
    done = C.c_int32(0)
    rc = load_library().ovl_step_n(ctx, float(dt), int(iters), int(nsteps), C.byref(done))
    _check(ctx, rc)
    return int(done.value)


def ovl_save(ctx) -> bytes:
    """Checkpoint of the simulation state (host bytes)."""
    L = load_library()
    n = C.c_size_t(0)
    _check(ctx, L.ovl_save(ctx, None, 0, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(ctx, L.ovl_save(ctx, buf, n.value, C.byref(n)))
    return buf.raw[:n.value]


def ovl_load(ctx, blob: bytes) -> None:
    buf = C.create_string_buffer(bytes(blob), len(blob))
    _check(ctx, load_library().ovl_load(ctx, buf, len(blob)))


def checkpoint_step_index(blob: bytes) -> int:
    """The step index stored in a checkpoint's header."""
    return int(np.frombuffer(bytes(blob[32:40]), dtype=np.int64)[0])


def ovl_read_stats(ctx) -> dict:
    s = ovl_stats()
    _check(ctx, load_library().ovl_read_stats(ctx, C.byref(s)))
    out = {k: getattr(s, k) for k, _ in ovl_stats._fields_ if k != "phase_ms"}
    L = load_library()
    out["phase_ms"] = {L.ovl_phase_name(i).decode(): s.phase_ms[i] for i in range(11)}
    return out


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class Simulation:
    """One libovl context holding one (possibly batched) scene."""

    def __init__(self, scene, params: ovl_params | dict | None = None, stream: int | None = None,
                 partition: bool = True):
        if isinstance(params, dict) or params is None:
            kw = dict(lb_activate=scene.lb_activate, lb_deact_every=scene.lb_deact_every)
            kw.update(params or {})
            params = ovl_default_params(**kw)
        self.params = params
        self.scene = scene
        self._step_index = 0      # mirrors the context's step counter
        self.n = scene.n_bodies
        self.n_parts = int(np.sum(scene.n_sets))
        self.ctx = ovl_create(params, stream)
        ovl_scene_upload(self.ctx, scene)
        if partition:
            ovl_set_partition(self.ctx, scene.set_of_body)
            if scene.assign_overlap:
                ovl_assign_overlap(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            ovl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # membership / state -------------------------------------------------------
    def set_partition(self, sets):
        ovl_set_partition(self.ctx, sets)

    def set_membership(self, masks):
        ovl_set_membership(self.ctx, masks)

    def membership(self):
        return ovl_read_membership(self.ctx, self.n)

    def assign_overlap(self):
        ovl_assign_overlap(self.ctx)

    def set_state(self, state):
        if hasattr(state, "data_ptr"):
            ovl_set_state(self.ctx, state.data_ptr(), on_device=True)
        else:
            ovl_set_state(self.ctx, state)

    def state(self, out=None):
        if out is not None and hasattr(out, "data_ptr"):
            ovl_read_state(self.ctx, out.data_ptr(), on_device=True)
            return out
        o = np.zeros((self.n, 13), np.float32) if out is None else out
        return ovl_read_state(self.ctx, o)

    def set_step_index(self, k):
        ovl_set_step_index(self.ctx, k)
        self._step_index = int(k)

    def step_index_value(self) -> int:
        """Index of the next step (load-balance cadence)."""
        return self._step_index

    def set_warmstart(self, part, key, lam):
        ovl_set_warmstart(self.ctx, part, key, lam)

    def warmstart(self):
        return ovl_read_warmstart(self.ctx)

    # stepping -----------------------------------------------------------------
    def step(self, dt: float = 0.0, iters: int | None = None):
        ovl_step(self.ctx, dt, self.scene.iters if iters is None else iters)
        self._step_index += 1

    def step_n(self, nsteps: int, dt: float = 0.0, iters: int | None = None) -> int:
        done = C.c_int32(0)
        rc = load_library().ovl_step_n(self.ctx, float(dt), int(self.scene.iters if iters is None else iters),
                                       int(nsteps), C.byref(done))
        self._step_index += int(done.value)   # steps completed before any error
        _check(self.ctx, rc)
        return int(done.value)

    def save(self) -> bytes:
        return ovl_save(self.ctx)

    def load(self, blob: bytes):
        ovl_load(self.ctx, blob)
        self._step_index = checkpoint_step_index(blob)

    def autotune_export(self) -> str:
        return ovl_autotune_export(self.ctx)

    def autotune_import(self, text: str):
        ovl_autotune_import(self.ctx, text)

    def load_balance(self, flags: int = 3):
        ovl_load_balance(self.ctx, flags)

    def joint_error(self) -> dict:
        """Sum and largest pivot gap over the joints of the current state (m)."""
        s, m = C.c_double(), C.c_double()
        _check(self.ctx, load_library().ovl_joint_error(self.ctx, C.byref(s), C.byref(m)))
        return dict(sum=s.value, max=m.value)

    def sync(self):
        ovl_sync(self.ctx)

    # records of the last step -------------------------------------------------
    def stats(self) -> dict:
        return ovl_read_stats(self.ctx)

    def contacts(self):
        m = self.stats()["n_contacts"]
        mm = max(m, 1)
        ab, phi = np.zeros((mm, 2), np.int32), np.zeros(mm, np.float32)
        nn, t1 = np.zeros((mm, 3), np.float32), np.zeros((mm, 3), np.float32)
        _check(self.ctx, load_library().ovl_read_contacts(self.ctx, _ptr(ab, _ip), _ptr(phi, _fp),
                                                          _ptr(nn, _fp), _ptr(t1, _fp)))
        return ab[:m], phi[:m], nn[:m], t1[:m]

    def contact_points(self):
        """(manifold index [m], point [m,3]) of the last step's contacts;
        zeros for sphere contacts."""
        m = self.stats()["n_contacts"]
        mm = max(m, 1)
        k, p = np.zeros(mm, np.int32), np.zeros((mm, 3), np.float32)
        _check(self.ctx, load_library().ovl_read_contact_points(self.ctx, _ptr(k, _ip), _ptr(p, _fp)))
        return k[:m], p[:m]

    def graph(self):
        m = self.stats()["n_adjacency"]
        rp, col = np.zeros(self.n + 1, np.int32), np.zeros(max(m, 1), np.int32)
        _check(self.ctx, load_library().ovl_read_graph(self.ctx, _ptr(rp, _ip), _ptr(col, _ip)))
        return rp, col[:m]

    def entries(self):
        ne = self.stats()["n_entries"]
        m = max(ne, 1)
        ep, part = np.zeros(self.n + 1, np.int32), np.zeros(m, np.int32)
        D, w, cp = np.zeros(m, np.uint8), np.zeros(m, np.float32), np.zeros((m, 13), np.float32)
        _check(self.ctx, load_library().ovl_read_entries(self.ctx, _ptr(ep, _ip), _ptr(part, _ip),
                                                         _ptr(D, _u8p), _ptr(w, _fp), _ptr(cp, _fp)))
        return dict(entry_ptr=ep, part=part[:ne], D=D[:ne], weight=w[:ne], copies=cp[:ne])

    def pairs(self):
        npr = self.stats()["n_pairs"]
        m = max(npr, 1)
        part, key = np.zeros(m, np.int32), np.zeros(m, np.uint64)
        colour, lam = np.zeros(m, np.int32), np.zeros((m, 3), np.float32)
        _check(self.ctx, load_library().ovl_read_pairs(self.ctx, _ptr(part, _ip), _ptr(key, _u64p),
                                                       _ptr(colour, _ip), _ptr(lam, _fp)))
        return dict(part=part[:npr], key=key[:npr], colour=colour[:npr], lam=lam[:npr])

    def worker_stats(self):
        P = self.n_parts
        it, rs = np.zeros(P, np.int32), np.zeros(P, np.float64)
        rows, cols = np.zeros(P, np.int64), np.zeros(P, np.int32)
        _check(self.ctx, load_library().ovl_read_worker_stats(
            self.ctx, _ptr(it, _ip), rs.ctypes.data_as(C.POINTER(C.c_double)),
            rows.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(cols, _ip)))
        return dict(iters=it, res_sq=rs, rows=rows, colours=cols)

    def solve_plan(self):
        """CTAs (one cluster) that solved each worker in the last step."""
        ctas = np.zeros(max(self.n_parts, 1), np.int32)
        _check(self.ctx, load_library().ovl_read_solve_plan(self.ctx, _ptr(ctas, _ip)))
        return ctas[:self.n_parts]

    # learned warm start ----------------------------------------------------------

    def set_warmstart_mode(self, mode: int):
        _check(self.ctx, load_library().ovl_set_warmstart_mode(self.ctx, int(mode)))

    def features(self):
        """Per pair of the last step: features [12], scale, previous-impulse
        flag and the warm-start impulses the solve started from."""
        npr = self.stats()["n_pairs"]
        m = max(npr, 1)
        f, sc = np.zeros((m, 12), np.float32), np.zeros(m, np.float32)
        found, lam0 = np.zeros(m, np.int32), np.zeros((m, 3), np.float32)
        _check(self.ctx, load_library().ovl_read_features(self.ctx, _ptr(f, _fp), _ptr(sc, _fp),
                                                          _ptr(found, _ip), _ptr(lam0, _fp)))
        return dict(feat=f[:npr], scale=sc[:npr], found=found[:npr].astype(bool), lam0=lam0[:npr])

    def mlp_set_params(self, theta):
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
        _check(self.ctx, load_library().ovl_mlp_set_params(self.ctx, _ptr(th, _fp), th.size))

    def mlp_params(self):
        th = np.zeros(OVL_MLP_N_PARAMS, np.float32)
        _check(self.ctx, load_library().ovl_mlp_get_params(self.ctx, _ptr(th, _fp), th.size))
        return th

    def mlp_forward(self, feat):
        f = np.ascontiguousarray(np.asarray(feat, dtype=np.float32)).reshape(-1, 12)
        y = np.zeros((max(len(f), 1), 3), np.float32)
        _check(self.ctx, load_library().ovl_mlp_forward(self.ctx, len(f), _ptr(f, _fp), _ptr(y, _fp)))
        return y[:len(f)]

    def log_reserve(self, capacity: int):
        _check(self.ctx, load_library().ovl_log_reserve(self.ctx, int(capacity)))

    def log_enable(self, on: bool = True):
        _check(self.ctx, load_library().ovl_log_enable(self.ctx, int(bool(on))))

    def log_size(self) -> int:
        n = C.c_int64()
        _check(self.ctx, load_library().ovl_log_size(self.ctx, C.byref(n)))
        return n.value

    def log_append(self, feat, target):
        f = np.ascontiguousarray(np.asarray(feat, dtype=np.float32)).reshape(-1, 12)
        t = np.ascontiguousarray(np.asarray(target, dtype=np.float32)).reshape(-1, 3)
        assert len(f) == len(t)
        _check(self.ctx, load_library().ovl_log_append(self.ctx, len(f), _ptr(f, _fp), _ptr(t, _fp)))

    def log_read(self, first: int = 0, n: int | None = None):
        n = self.log_size() - first if n is None else n
        f, t = np.zeros((max(n, 1), 12), np.float32), np.zeros((max(n, 1), 3), np.float32)
        _check(self.ctx, load_library().ovl_log_read(self.ctx, first, n, _ptr(f, _fp), _ptr(t, _fp)))
        return f[:n], t[:n]

    def mlp_train(self, first: int, count: int, batch: int, steps: int, sampling: int = 1,
                  lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
                  seed: int = 0):
        d = ovl_train_desc(first=first, count=count, batch=batch, steps=steps, sampling=sampling,
                           lr=lr, beta1=beta1, beta2=beta2, eps=eps, seed=seed)
        loss = np.zeros(max(steps, 1), np.float32)
        _check(self.ctx, load_library().ovl_mlp_train(self.ctx, C.byref(d), _ptr(loss, _fp)))
        return loss[:steps]

    def mlp_grad(self, first: int, count: int):
        g = np.zeros(OVL_MLP_N_PARAMS, np.float32)
        loss = C.c_double()
        _check(self.ctx, load_library().ovl_mlp_grad(self.ctx, first, count, _ptr(g, _fp), C.byref(loss)))
        return loss.value, g

    def mlp_loss(self, first: int, count: int) -> float:
        loss = C.c_double()
        _check(self.ctx, load_library().ovl_mlp_loss(self.ctx, first, count, C.byref(loss)))
        return loss.value
