"""ctypes wrapper of box_oracle.c -- TEST INFRASTRUCTURE ONLY: the FP64
reference geometry of box contacts (sphere-box, box-plane, box-box), the
shapes of the paper's Building and Bridge scenes (Section 6).  Only tests and
the build step use it; the CUDA library never does.

Conventions: the normal points from the first shape towards the second; a
gap is positive when apart; a contact exists when gap <= margin;
quaternions are (w, x, y, z)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "box_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libbox_oracle.so")

_lib = None
_dp = C.POINTER(C.c_double)


def build(force: bool = False) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.box_plane.argtypes = [_dp, _dp, _dp, _dp, C.c_double, _dp, _dp, _dp, _dp]
        L.box_plane.restype = C.c_int
        L.sphere_box.argtypes = [_dp, C.c_double, _dp, _dp, _dp, C.c_double, _dp, _dp, _dp, _dp]
        L.sphere_box.restype = C.c_int
        L.box_box.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, C.c_double, _dp, _dp, _dp,
                              C.POINTER(C.c_int), _dp, _dp]
        L.box_box.restype = C.c_int
        L.box_box_axes.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.box_box_axes.restype = None
        L.box_inv_inertia_world.argtypes = [_dp, _dp, C.c_double, _dp]
        L.box_inv_inertia_world.restype = None
        L.box_plane_step.argtypes = [_dp, _dp, _dp, C.c_double, _dp, C.c_double, C.c_double, _dp, C.c_double,
                                     C.c_double, C.c_double, C.c_int, _dp, _dp, _dp]
        L.box_plane_step.restype = C.c_int
        _lib = L
    return _lib


def _v(x, n):
    a = np.ascontiguousarray(x, dtype=np.float64).reshape(n)
    return a, a.ctypes.data_as(_dp)


def box_plane(c, q, h, plane, margin=0.0, with_amb=False):
    """Vertices of the box within the margin of the plane n.x = d (plane =
    (n, d), n unit out of the solid), the 4 deepest at most.  Returns
    (points [k,3], gaps [k], normal [3] = -n), and with with_amb the
    closeness of its decisions to their thresholds in bands (< 1: an FP32
    computation may decide otherwise)."""
    (c, pc), (q, pq), (h, ph), (pl, pp) = _v(c, 3), _v(q, 4), _v(h, 3), _v(plane, 4)
    pts, gaps, nrm, amb = np.zeros(12), np.zeros(4), np.zeros(3), C.c_double(np.inf)
    k = lib().box_plane(pc, pq, ph, pp, float(margin), pts.ctypes.data_as(_dp), gaps.ctypes.data_as(_dp),
                        nrm.ctypes.data_as(_dp), C.byref(amb))
    out = (pts[: 3 * k].reshape(k, 3), gaps[:k], nrm)
    return out + (amb.value,) if with_amb else out


def sphere_box(s, r, c, q, h, margin=0.0, with_amb=False):
    """Returns (hit, point on the box [3], normal sphere->box [3], gap)
    (+ amb with with_amb, as box_plane)."""
    (s, ps), (c, pc), (q, pq), (h, ph) = _v(s, 3), _v(c, 3), _v(q, 4), _v(h, 3)
    pt, nrm, gap, amb = np.zeros(3), np.zeros(3), C.c_double(), C.c_double(np.inf)
    hit = lib().sphere_box(ps, float(r), pc, pq, ph, float(margin), pt.ctypes.data_as(_dp),
                           nrm.ctypes.data_as(_dp), C.byref(gap), C.byref(amb))
    out = (bool(hit), pt, nrm, gap.value)
    return out + (amb.value,) if with_amb else out


def box_box(cA, qA, hA, cB, qB, hB, margin=0.0, with_amb=False):
    """Returns (points [k,3], gaps [k], normal A->B [3], axis, separation)
    (+ amb with with_amb, as box_plane); k = 0 when some axis separates the
    boxes by more than the margin (axis and separation are then undefined)."""
    args = [_v(cA, 3), _v(qA, 4), _v(hA, 3), _v(cB, 3), _v(qB, 4), _v(hB, 3)]
    pts, gaps, nrm = np.zeros(12), np.zeros(4), np.zeros(3)
    axis, sep, amb = C.c_int(-1), C.c_double(np.nan), C.c_double(np.inf)
    k = lib().box_box(*[p for _, p in args], float(margin), pts.ctypes.data_as(_dp), gaps.ctypes.data_as(_dp),
                      nrm.ctypes.data_as(_dp), C.byref(axis), C.byref(sep), C.byref(amb))
    out = (pts[: 3 * k].reshape(k, 3), gaps[:k], nrm, axis.value, sep.value)
    return out + (amb.value,) if with_amb else out


def box_box_axes(cA, qA, hA, cB, qB, hB):
    """Separations along the 15 candidate axes (-inf where parallel edges
    give no axis)."""
    args = [_v(cA, 3), _v(qA, 4), _v(hA, 3), _v(cB, 3), _v(qB, 4), _v(hB, 3)]
    out = np.zeros(15)
    lib().box_box_axes(*[p for _, p in args], out.ctypes.data_as(_dp))
    return out


def box_inv_inertia_world(q, h, inv_mass):
    """World inverse inertia (3x3) of a solid box."""
    (q, pq), (h, ph) = _v(q, 4), _v(h, 3)
    out = np.zeros(9)
    lib().box_inv_inertia_world(pq, ph, float(inv_mass), out.ctypes.data_as(_dp))
    return out.reshape(3, 3)


def box_plane_step(x, q, h, inv_mass, plane, v, w, mu=0.5, dt=1 / 60, g=(0.0, 0.0, -9.81), erp=0.2, slop=0.0,
                   margin=0.02, iters=200):
    """One PGS velocity step of a box on a static plane.  Returns
    (v', w', impulses [k,3] as (n, t1, t2) per contact, contact points,
    gaps)."""
    (x, px), (q, pq), (h, ph), (pl, pp), (gg, pg) = _v(x, 3), _v(q, 4), _v(h, 3), _v(plane, 4), _v(g, 3)
    v2, w2 = np.array(v, dtype=np.float64).copy(), np.array(w, dtype=np.float64).copy()
    lam = np.zeros(12)
    k = lib().box_plane_step(px, pq, ph, float(inv_mass), pp, float(mu), float(dt), pg, float(erp), float(slop),
                             float(margin), int(iters), v2.ctypes.data_as(_dp), w2.ctypes.data_as(_dp),
                             lam.ctypes.data_as(_dp))
    pts, gaps, _ = box_plane(x, q, h, plane, margin)
    return v2, w2, lam[: 3 * k].reshape(k, 3), pts, gaps
