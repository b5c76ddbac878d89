"""ctypes wrapper around the FP64 C oracle (``ovl_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``; never by the library.

``build()`` compiles the oracle with gcc (``-O2 -ffp-contract=off``, no
fused multiply-add) into ``oracle/_build/``.  ``OracleSim`` mirrors one
simulation: scene arrays are widened exactly from FP32 to FP64, and every
record of the last step (contacts, graph, membership, geodesics, weights,
copies, constraint colours and impulses) can be read back for comparison.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ovl_oracle.c")
BOX_SRC = os.path.join(HERE, "box_oracle.c")   # box contact decisions the step takes in FP32
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libovl_oracle.so")
# the same source with FP32 sweeps (-DORC_REAL=float): the precision floor of
# the algorithm itself, for comparisons only
LIB_PATH_F32 = os.path.join(BUILD_DIR, "libovl_oracle_f32sweeps.so")

DEFAULT_PARAMS = dict(gravity=(0.0, 0.0, -9.81), margin=0.05, erp=0.2, slop=0.001, warmstart=1.0,
                      lb_activate=1, lb_deact_every=1, res_tol=0.0, res_check_every=0, lb_load=0,
                      weights=0)


class OrcParams(C.Structure):
    _fields_ = [("gravity", C.c_double * 3), ("margin", C.c_double), ("erp", C.c_double),
                ("slop", C.c_double), ("warmstart", C.c_double), ("lb_activate", C.c_int),
                ("lb_deact_every", C.c_int), ("res_tol", C.c_double),
                ("res_check_every", C.c_int), ("lb_load", C.c_int),
                ("weights", C.c_int)]


def _build_one(path: str, defines: list[str], force: bool) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(SRC)
            or os.path.getmtime(path) < os.path.getmtime(BOX_SRC)):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-std=c11", "-shared", "-fPIC"]
                              + defines + ["-o", tmp, SRC, BOX_SRC, "-lm"])
        os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    _build_one(LIB_PATH_F32, ["-DORC_REAL=float"], force)
    return _build_one(LIB_PATH, [], force)


_lib = None
_lib_f32 = None

P = C.POINTER
dp, ip, i64p, u64p, u8p = P(C.c_double), P(C.c_int), P(C.c_int64), P(C.c_uint64), P(C.c_uint8)


def lib(sweeps: str = "f64"):
    """The oracle library; sweeps="f32" gives the FP32-sweep build."""
    global _lib, _lib_f32
    if sweeps == "f32":
        if _lib_f32 is None:
            build()
            _lib_f32 = _declare(C.CDLL(LIB_PATH_F32))
        return _lib_f32
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def _declare(L):
    if True:
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [P(OrcParams), C.c_int, dp, dp, dp, C.c_int, dp, ip, C.c_int, ip, dp,
                                 C.c_int, ip, dp, dp, ip, ip, ip, ip]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_partition.argtypes = [C.c_void_p, ip]
        L.orc_set_partition.restype = C.c_int
        L.orc_set_masks.argtypes = [C.c_void_p, u64p]
        L.orc_set_shapes.argtypes = [C.c_void_p, dp]
        L.orc_set_shapes.restype = C.c_int
        L.orc_set_masks.restype = C.c_int
        L.orc_get_masks.argtypes = [C.c_void_p, u64p]
        L.orc_set_state.argtypes = [C.c_void_p, dp]
        L.orc_get_state.argtypes = [C.c_void_p, dp]
        L.orc_set_step_index.argtypes = [C.c_void_p, C.c_int64]
        L.orc_get_step_index.argtypes = [C.c_void_p]
        L.orc_get_step_index.restype = C.c_int64
        L.orc_assign.argtypes = [C.c_void_p]
        L.orc_assign.restype = C.c_int
        L.orc_set_warmstart.argtypes = [C.c_void_p, C.c_int64, ip, u64p, dp]
        L.orc_warmstart_size.argtypes = [C.c_void_p]
        L.orc_warmstart_size.restype = C.c_int64
        L.orc_get_warmstart.argtypes = [C.c_void_p, ip, u64p, dp]
        L.orc_step.argtypes = [C.c_void_p, C.c_double, C.c_int]
        L.orc_step.restype = C.c_int
        L.orc_get_counts.argtypes = [C.c_void_p, i64p]
        L.orc_get_contacts.argtypes = [C.c_void_p, ip, dp, dp, dp]
        L.orc_get_contact_points.argtypes = [C.c_void_p, ip, dp]
        L.orc_get_contact_amb.argtypes = [C.c_void_p, dp]
        L.orc_get_graph.argtypes = [C.c_void_p, ip, ip]
        L.orc_get_entries.argtypes = [C.c_void_p, i64p, ip, u8p, dp, dp]
        L.orc_get_pairs.argtypes = [C.c_void_p, ip, ip, i64p, u64p, ip, dp]
        L.orc_get_part_stats.argtypes = [C.c_void_p, ip, dp, i64p, ip]
        L.orc_get_features.argtypes = [C.c_void_p, dp, dp, ip, u8p]
        L.orc_get_metrics.argtypes = [C.c_void_p, dp]
        L.orc_joint_error.argtypes = [C.c_void_p, dp]
        L.orc_contacts.restype = C.c_int64
        L.orc_contacts.argtypes = [C.c_int, dp, dp, dp, C.c_int, dp, ip, ip, ip, C.c_double, C.c_int,
                                   C.c_int64, ip, dp, dp, dp]
        L.orc_graph.restype = C.c_int64
        L.orc_graph.argtypes = [C.c_int, dp, C.c_int64, ip, ip, C.c_int64, ip, ip]
        L.orc_load_balance.argtypes = [C.c_int, u64p, ip, ip, C.c_int, ip, ip, C.c_int64, ip, ip, ip,
                                       C.c_int, C.c_int, i64p]
        L.orc_is_bridge.restype = C.c_int
        L.orc_is_bridge.argtypes = [C.c_int, u64p, ip, ip, C.c_int]
        L.orc_assign_overlap.argtypes = [C.c_int, u64p, ip, ip, C.c_int, dp, C.c_int, ip, ip]
        L.orc_geodesics.argtypes = [C.c_int, u64p, ip, ip, ip, ip, u8p]
        L.orc_weights.argtypes = [C.c_int, u8p, dp]
        L.orc_blend.argtypes = [C.c_int, dp, dp, dp]
        L.orc_colour.restype = C.c_int
        L.orc_colour.argtypes = [C.c_int, ip, u64p, C.c_int, ip]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        L.orc_mix64.restype = C.c_uint64
        L.orc_mix64.argtypes = [C.c_uint64]
    return L


def _ptr(a, t):
    return a.ctypes.data_as(t)


def set_threads(n: int) -> None:
    """Threads for the per-body contact search and the per-worker solve
    (1 = the caller's thread only).  Results do not depend on it."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _u64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


# ---------------------------------------------------------------------------
# standalone stage functions
# ---------------------------------------------------------------------------

def contacts(state, radius, inv_mass, planes, plane_scene=None, scene_of_body=None,
             scene_flags=None, margin=0.05, use_grid=True):
    """Contacts of a state in canonical order: (ab [m,2], phi, n [m,3], t1 [m,3])."""
    st = _f64(state).reshape(-1, 13)
    n = st.shape[0]
    pl = _f64(planes).reshape(-1, 4)
    ps = _i32(np.zeros(pl.shape[0]) if plane_scene is None else plane_scene)
    sob = _i32(np.zeros(n) if scene_of_body is None else scene_of_body)
    sf = _i32([1] if scene_flags is None else scene_flags)
    r, im = _f64(radius), _f64(inv_mass)
    L = lib()
    cap = 0
    dummy_i = np.zeros(2, np.int32)
    dummy_d = np.zeros(3, np.float64)
    m = L.orc_contacts(n, _ptr(st, dp), _ptr(r, dp), _ptr(im, dp), pl.shape[0], _ptr(pl, dp),
                       _ptr(ps, ip), _ptr(sob, ip), _ptr(sf, ip), margin, int(use_grid), cap,
                       _ptr(dummy_i, ip), _ptr(dummy_d, dp), _ptr(dummy_d, dp), _ptr(dummy_d, dp))
    ab = np.zeros((max(m, 1), 2), np.int32)
    phi = np.zeros(max(m, 1), np.float64)
    nn = np.zeros((max(m, 1), 3), np.float64)
    t1 = np.zeros((max(m, 1), 3), np.float64)
    L.orc_contacts(n, _ptr(st, dp), _ptr(r, dp), _ptr(im, dp), pl.shape[0], _ptr(pl, dp),
                   _ptr(ps, ip), _ptr(sob, ip), _ptr(sf, ip), margin, int(use_grid), m,
                   _ptr(ab, ip), _ptr(phi, dp), _ptr(nn, dp), _ptr(t1, dp))
    return ab[:m], phi[:m], nn[:m], t1[:m]


def graph(n, inv_mass, edges):
    """Sorted, deduplicated adjacency (row_ptr [n+1], col) of the given edges."""
    e = _i32(edges).reshape(-1, 2)
    eu, ev = _i32(e[:, 0]), _i32(e[:, 1])
    im = _f64(inv_mass)
    rp = np.zeros(n + 1, np.int32)
    cap = 2 * e.shape[0] + 1
    col = np.zeros(cap, np.int32)
    m = lib().orc_graph(n, _ptr(im, dp), e.shape[0], _ptr(eu, ip), _ptr(ev, ip), cap,
                        _ptr(rp, ip), _ptr(col, ip))
    return rp, col[:m]


def load_balance(masks, scene_of_body, n_sets, row_ptr, col, contact_pairs, scene_gamma,
                 do_activate=True, do_deactivate=True, weights=None):
    """Algorithm 6 on a copy of the masks; returns the new masks.  ``weights``
    (int64 per body) replaces the body count in the loads <W>; None counts
    every active body once (Table 1)."""
    m = _u64(masks).copy()
    n = m.shape[0]
    sob = _i32(scene_of_body)
    ns = _i32(n_sets)
    base = _i32(np.concatenate([[0], np.cumsum(ns)]))
    cp = _i32(contact_pairs).reshape(-1, 2)
    ca, cb = _i32(cp[:, 0]), _i32(cp[:, 1])
    rp, cl, sg = _i32(row_ptr), _i32(col), _i32(scene_gamma)
    wt = None if weights is None else np.ascontiguousarray(weights, dtype=np.int64)
    assert wt is None or wt.shape == (n,)
    lib().orc_load_balance(n, _ptr(m, u64p), _ptr(sob, ip), _ptr(base, ip), int(base[-1]),
                           _ptr(rp, ip), _ptr(cl, ip), cp.shape[0], _ptr(ca, ip), _ptr(cb, ip),
                           _ptr(sg, ip), int(do_activate), int(do_deactivate),
                           None if weights is None else _ptr(wt, i64p))
    return m


def is_bridge(masks, row_ptr, col, b):
    m = _u64(masks)
    return bool(lib().orc_is_bridge(m.shape[0], _ptr(m, u64p), _ptr(_i32(row_ptr), ip),
                                    _ptr(_i32(col), ip), int(b)))


def assign_overlap(masks, scene_of_body, n_sets, inv_mass, joints, scene_gamma):
    """Algorithms 2-3 on a copy of the masks; returns the new masks."""
    m = _u64(masks).copy()
    n = m.shape[0]
    sob = _i32(scene_of_body)
    ns = _i32(n_sets)
    base = _i32(np.concatenate([[0], np.cumsum(ns)]))
    j = _i32(joints).reshape(-1, 2)
    lib().orc_assign_overlap(n, _ptr(m, u64p), _ptr(sob, ip), _ptr(base, ip), int(base[-1]),
                             _ptr(_f64(inv_mass), dp), j.shape[0], _ptr(j, ip),
                             _ptr(_i32(scene_gamma), ip))
    return m


def geodesics(masks, scene_of_body, scene_beta, row_ptr, col):
    """D per entry (bodies in order, their workers ascending); 255 = not met."""
    m = _u64(masks)
    ne = int(sum(bin(int(x)).count("1") for x in m))
    D = np.zeros(max(ne, 1), np.uint8)
    lib().orc_geodesics(m.shape[0], _ptr(m, u64p), _ptr(_i32(scene_of_body), ip),
                        _ptr(_i32(scene_beta), ip), _ptr(_i32(row_ptr), ip), _ptr(_i32(col), ip),
                        _ptr(D, u8p))
    return D[:ne]


def weights(D):
    d = np.ascontiguousarray(np.asarray(D, dtype=np.uint8))
    w = np.zeros(d.shape[0], np.float64)
    lib().orc_weights(d.shape[0], _ptr(d, u8p), _ptr(w, dp))
    return w


def blend(copies, w):
    c = _f64(copies).reshape(-1, 13)
    ww = _f64(w)
    out = np.zeros(13, np.float64)
    lib().orc_blend(c.shape[0], _ptr(c, dp), _ptr(ww, dp), _ptr(out, dp))
    return out


def colour(body_slots, prio, n_local):
    bs = _i32(body_slots).reshape(-1, 2)
    pr = _u64(prio)
    out = np.zeros(max(bs.shape[0], 1), np.int32)
    nc = lib().orc_colour(bs.shape[0], _ptr(bs, ip), _ptr(pr, u64p), int(n_local), _ptr(out, ip))
    return nc, out[:bs.shape[0]]


def mix64(x: int) -> int:
    return int(lib().orc_mix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


# ---------------------------------------------------------------------------
# the whole simulation
# ---------------------------------------------------------------------------

class OracleSim:
    """FP64 simulation of a scene; ``step`` runs one timestep of Algorithm 1.
    sweeps="f32": the same algorithm with its PGS sweeps in FP32 (the
    precision floor of the method's own arithmetic, for comparisons)."""

    def __init__(self, scene, params: dict | None = None, sweeps: str = "f64"):
        p = dict(DEFAULT_PARAMS)
        p["lb_activate"] = scene.lb_activate
        p["lb_deact_every"] = scene.lb_deact_every
        if params:
            p.update(params)
        self.params = p
        cp = OrcParams()
        for k in range(3):
            cp.gravity[k] = p["gravity"][k]
        cp.margin, cp.erp, cp.slop, cp.warmstart = p["margin"], p["erp"], p["slop"], p["warmstart"]
        cp.lb_activate, cp.lb_deact_every = int(p["lb_activate"]), int(p["lb_deact_every"])
        cp.res_tol, cp.res_check_every = float(p["res_tol"]), int(p["res_check_every"])
        cp.lb_load = int(p["lb_load"])
        cp.weights = int(p["weights"])
        self._params = cp
        self.scene = scene
        self.n = scene.n_bodies
        self.n_parts = int(np.sum(scene.n_sets))
        self._keep = [_f64(scene.state), _f64(scene.radius), _f64(scene.inv_mass),
                      _f64(scene.planes), _i32(scene.plane_scene), _i32(scene.joints),
                      _f64(scene.anchors), _i32(scene.scene_of_body), _f64(scene.scene_mu),
                      _f64(scene.scene_dt), _i32(scene.scene_flags), _i32(scene.scene_gamma),
                      _i32(scene.scene_beta), _i32(scene.n_sets)]
        k = self._keep
        self._L = L = lib(sweeps)
        self._h = L.orc_create(C.byref(cp), self.n, _ptr(k[0], dp), _ptr(k[1], dp), _ptr(k[2], dp),
                               scene.planes.shape[0], _ptr(k[3], dp), _ptr(k[4], ip),
                               scene.joints.shape[0], _ptr(k[5], ip), _ptr(k[6], dp),
                               scene.n_scenes, _ptr(k[7], ip), _ptr(k[8], dp), _ptr(k[9], dp),
                               _ptr(k[10], ip), _ptr(k[11], ip), _ptr(k[12], ip), _ptr(k[13], ip))
        he = getattr(scene, "half_extents", None)
        if he is not None and np.any(np.asarray(he) > 0):
            self._half = _f64(np.asarray(he).reshape(self.n, 3))
            if L.orc_set_shapes(self._h, _ptr(self._half, dp)) != 0:
                raise ValueError("negative half extent")
        rc = L.orc_set_partition(self._h, _ptr(_i32(scene.set_of_body), ip))
        if rc != 0:
            raise ValueError(f"invalid partition ({rc})")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and getattr(self, "_L", None) is not None:
            self._L.orc_destroy(h)
            self._h = None

    # setup / state -----------------------------------------------------------
    def assign_overlap(self):
        self._L.orc_assign(self._h)

    def set_masks(self, masks):
        rc = self._L.orc_set_masks(self._h, _ptr(_u64(masks), u64p))
        if rc != 0:
            raise ValueError(f"invalid membership ({rc})")

    def masks(self):
        out = np.zeros(self.n, np.uint64)
        self._L.orc_get_masks(self._h, _ptr(out, u64p))
        return out

    def set_state(self, st):
        self._L.orc_set_state(self._h, _ptr(_f64(st).reshape(-1, 13), dp))

    def state(self):
        out = np.zeros((self.n, 13), np.float64)
        self._L.orc_get_state(self._h, _ptr(out, dp))
        return out

    def set_step_index(self, k):
        self._L.orc_set_step_index(self._h, int(k))

    def step_index(self):
        return int(self._L.orc_get_step_index(self._h))

    def set_warmstart(self, part, key, lam):
        part, key, lam = _i32(part), _u64(key), _f64(lam).reshape(-1, 3)
        self._L.orc_set_warmstart(self._h, part.shape[0], _ptr(part, ip), _ptr(key, u64p), _ptr(lam, dp))

    def warmstart(self):
        n = self._L.orc_warmstart_size(self._h)
        part = np.zeros(max(n, 1), np.int32)
        key = np.zeros(max(n, 1), np.uint64)
        lam = np.zeros((max(n, 1), 3), np.float64)
        self._L.orc_get_warmstart(self._h, _ptr(part, ip), _ptr(key, u64p), _ptr(lam, dp))
        return part[:n], key[:n], lam[:n]

    # stepping ----------------------------------------------------------------
    def step(self, dt: float = 0.0, iters: int | None = None):
        it = self.scene.iters if iters is None else iters
        rc = self._L.orc_step(self._h, float(dt), int(it))
        if rc != 0:
            raise RuntimeError(f"oracle step failed ({rc})")

    # last-step records -------------------------------------------------------
    def counts(self):
        c = np.zeros(5, np.int64)
        self._L.orc_get_counts(self._h, _ptr(c, i64p))
        return dict(contacts=int(c[0]), adjacency=int(c[1]), entries=int(c[2]), pairs=int(c[3]),
                    parts=int(c[4]))

    def contacts(self):
        m = self.counts()["contacts"]
        ab = np.zeros((max(m, 1), 2), np.int32)
        phi = np.zeros(max(m, 1))
        nn = np.zeros((max(m, 1), 3))
        t1 = np.zeros((max(m, 1), 3))
        self._L.orc_get_contacts(self._h, _ptr(ab, ip), _ptr(phi, dp), _ptr(nn, dp), _ptr(t1, dp))
        return ab[:m], phi[:m], nn[:m], t1[:m]


    def contact_points(self):
        """(manifold index [m], contact point [m,3]) of the last step's
        contacts; points are zero for sphere contacts."""
        m = self.counts()["contacts"]
        k, p = np.zeros(m, np.int32), np.zeros((m, 3))
        self._L.orc_get_contact_points(self._h, _ptr(k, ip), _ptr(p, dp))
        return k, p

    def contact_ambiguity(self):
        """Per contact of the last step: how close its box decisions came to
        their thresholds, in bands (< 1: an FP32 computation may decide the
        pair otherwise); inf for sphere contacts."""
        m = self.counts()["contacts"]
        a = np.zeros(max(m, 1))
        self._L.orc_get_contact_amb(self._h, _ptr(a, dp))
        return a[:m]

    def graph(self):
        m = self.counts()["adjacency"]
        rp = np.zeros(self.n + 1, np.int32)
        col = np.zeros(max(m, 1), np.int32)
        self._L.orc_get_graph(self._h, _ptr(rp, ip), _ptr(col, ip))
        return rp, col[:m]

    def entries(self):
        ne = self.counts()["entries"]
        ep = np.zeros(self.n + 1, np.int64)
        part = np.zeros(max(ne, 1), np.int32)
        D = np.zeros(max(ne, 1), np.uint8)
        w = np.zeros(max(ne, 1))
        cp = np.zeros((max(ne, 1), 13))
        self._L.orc_get_entries(self._h, _ptr(ep, i64p), _ptr(part, ip), _ptr(D, u8p), _ptr(w, dp),
                              _ptr(cp, dp))
        return dict(entry_ptr=ep, part=part[:ne], D=D[:ne], weight=w[:ne], copies=cp[:ne])

    def pairs(self):
        m = self.counts()["pairs"]
        mm = max(m, 1)
        part, kind = np.zeros(mm, np.int32), np.zeros(mm, np.int32)
        cidx, key = np.zeros(mm, np.int64), np.zeros(mm, np.uint64)
        colour_, lam = np.zeros(mm, np.int32), np.zeros((mm, 3))
        self._L.orc_get_pairs(self._h, _ptr(part, ip), _ptr(kind, ip), _ptr(cidx, i64p),
                            _ptr(key, u64p), _ptr(colour_, ip), _ptr(lam, dp))
        return dict(part=part[:m], kind=kind[:m], cidx=cidx[:m], key=key[:m], colour=colour_[:m],
                    lam=lam[:m])

    N_FEATURES = 12
    DEPTH_CAP = 8

    def features(self):
        """Learned-warm-start features of the last step: per pair [12], the
        scale s, whether previous impulses existed; per body the depth to O."""
        m = self.counts()["pairs"]
        mm = max(m, 1)
        f, sc, found = np.zeros((mm, 12)), np.zeros(mm), np.zeros(mm, np.int32)
        depth = np.zeros(max(self.n, 1), np.uint8)
        self._L.orc_get_features(self._h, _ptr(f, dp), _ptr(sc, dp), _ptr(found, ip), _ptr(depth, u8p))
        return dict(feat=f[:m], scale=sc[:m], found=found[:m].astype(bool), depth=depth[:self.n])

    def part_stats(self):
        n = self.n_parts
        it, rs = np.zeros(n, np.int32), np.zeros(n)
        rows, cols = np.zeros(n, np.int64), np.zeros(n, np.int32)
        self._L.orc_get_part_stats(self._h, _ptr(it, ip), _ptr(rs, dp), _ptr(rows, i64p), _ptr(cols, ip))
        return dict(iters=it, res_sq=rs, rows=rows, colours=cols)

    def metrics(self):
        out = np.zeros(4)
        self._L.orc_get_metrics(self._h, _ptr(out, dp))
        return dict(residual_rms=out[0], residual_max=out[1], joint_gap_max=out[2], joint_gap_sum=out[3])

    def joint_error(self):
        """Sum and largest pivot gap over the joints of the current state (m)."""
        out = np.zeros(2)
        self._L.orc_joint_error(self._h, _ptr(out, dp))
        return dict(sum=float(out[0]), max=float(out[1]))
