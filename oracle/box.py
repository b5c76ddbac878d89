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
        L.box_plane.argtypes = [_dp, _dp, _dp, _dp, C.c_double, _dp, _dp, _dp]
        L.box_plane.restype = C.c_int
        L.sphere_box.argtypes = [_dp, C.c_double, _dp, _dp, _dp, C.c_double, _dp, _dp, _dp]
        L.sphere_box.restype = C.c_int
        L.box_box.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, C.c_double, _dp, _dp, _dp,
                              C.POINTER(C.c_int), _dp]
        L.box_box.restype = C.c_int
        L.box_box_axes.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.box_box_axes.restype = None
        _lib = L
    return _lib


def _v(x, n):
    a = np.ascontiguousarray(x, dtype=np.float64).reshape(n)
    return a, a.ctypes.data_as(_dp)


def box_plane(c, q, h, plane, margin=0.0):
    """Vertices of the box within the margin of the plane n.x = d (plane =
    (n, d), n unit out of the solid), the 4 deepest at most.  Returns
    (points [k,3], gaps [k], normal [3] = -n)."""
    (c, pc), (q, pq), (h, ph), (pl, pp) = _v(c, 3), _v(q, 4), _v(h, 3), _v(plane, 4)
    pts, gaps, nrm = np.zeros(12), np.zeros(4), np.zeros(3)
    k = lib().box_plane(pc, pq, ph, pp, float(margin), pts.ctypes.data_as(_dp), gaps.ctypes.data_as(_dp),
                        nrm.ctypes.data_as(_dp))
    return pts[: 3 * k].reshape(k, 3), gaps[:k], nrm


def sphere_box(s, r, c, q, h, margin=0.0):
    """Returns (hit, point on the box [3], normal sphere->box [3], gap)."""
    (s, ps), (c, pc), (q, pq), (h, ph) = _v(s, 3), _v(c, 3), _v(q, 4), _v(h, 3)
    pt, nrm, gap = np.zeros(3), np.zeros(3), C.c_double()
    hit = lib().sphere_box(ps, float(r), pc, pq, ph, float(margin), pt.ctypes.data_as(_dp),
                           nrm.ctypes.data_as(_dp), C.byref(gap))
    return bool(hit), pt, nrm, gap.value


def box_box(cA, qA, hA, cB, qB, hB, margin=0.0):
    """Returns (points [k,3], gaps [k], normal A->B [3], axis, separation);
    k = 0 when some axis separates the boxes by more than the margin (axis
    and separation are then undefined)."""
    args = [_v(cA, 3), _v(qA, 4), _v(hA, 3), _v(cB, 3), _v(qB, 4), _v(hB, 3)]
    pts, gaps, nrm = np.zeros(12), np.zeros(4), np.zeros(3)
    axis, sep = C.c_int(-1), C.c_double(np.nan)
    k = lib().box_box(*[p for _, p in args], float(margin), pts.ctypes.data_as(_dp), gaps.ctypes.data_as(_dp),
                      nrm.ctypes.data_as(_dp), C.byref(axis), C.byref(sep))
    return pts[: 3 * k].reshape(k, 3), gaps[:k], nrm, axis.value, sep.value


def box_box_axes(cA, qA, hA, cB, qB, hB):
    """Separations along the 15 candidate axes (-inf where parallel edges
    give no axis)."""
    args = [_v(cA, 3), _v(qA, 4), _v(hA, 3), _v(cB, 3), _v(qB, 4), _v(hB, 3)]
    out = np.zeros(15)
    lib().box_box_axes(*[p for _, p in args], out.ctypes.data_as(_dp))
    return out
