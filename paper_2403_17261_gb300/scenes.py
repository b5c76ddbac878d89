"""Seeded synthetic scenes for the overlapping-partition rigid-body step.

This module only *generates inputs*: sphere lattices, hanging chains, bowls,
initial partitions and their parameters.  It contains none of the method's
arithmetic (no contacts, no solve, no weights, no blending), so both the CUDA
library and the FP64 oracle can be fed from it without sharing any code.

The paper's scenes (Bowl, Building, Chain Net, bridges; Table 2 of Section 6)
are not available, so the workloads below stand in for them:

* ``pile_small``   -- 256 spheres, 8x8x4 lattice on a ground plane, 2 sets split
                      at x = 0 (the Bowl scene's shape, scaled down).
* ``chain``        -- 4096-sphere hanging chain with ball joints, 8 contiguous
                      sets (the Two-way Bridge / Figure 3 chain).
* ``pile_large``   -- 262,144 spheres in a 64^3 lattice falling into a bowl of
                      four inclined planes, 64 sets from k-means (the Bowl scene).
* ``batched``      -- 512 independent scenes (half piles, half chains), 1-16
                      uneven sets each.
* small closed-form scenes used by the oracle's own pins (resting sphere,
  sphere column, incline, pendulum, free flight).

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) turned
into U[0,1) doubles with 53 bits; every float input is generated in FP64 and
rounded to FP32 once, so both sides consume identical values.

State layout (13 floats per body, the paper's Eq. 8): position x (3),
quaternion q = (w, x, y, z) (4), linear velocity (3), angular velocity (3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """SplitMix64 stream: state += golden gamma, output = finaliser(state)."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            idx = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + idx * _GOLDEN
            self.state = self.state + np.uint64(n) * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u


@dataclass
class Scene:
    """Arrays describing one (possibly batched) simulation, ready for upload.

    Bodies of one scene are contiguous and ``scene_of_body`` is non-decreasing.
    Plane rows are (nx, ny, nz, d): the plane is n.p = d and n.p >= d is free space.
    Joint rows are body indices (a, b) with -1 meaning the world; anchors are
    (anchor_a, anchor_b), each in its body's frame, or in world coordinates for
    a world end.
    """

    name: str
    state: np.ndarray            # float32 [n,13]
    radius: np.ndarray           # float32 [n]
    inv_mass: np.ndarray         # float32 [n] (0 = static)
    planes: np.ndarray           # float32 [np,4]
    plane_scene: np.ndarray      # int32 [np]
    joints: np.ndarray           # int32 [nj,2]
    anchors: np.ndarray          # float32 [nj,6]
    scene_of_body: np.ndarray    # int32 [n]
    scene_mu: np.ndarray         # float32 [ns]
    scene_dt: np.ndarray         # float32 [ns]
    scene_flags: np.ndarray      # int32 [ns]; bit 0 = sphere-sphere contacts on
    scene_gamma: np.ndarray      # int32 [ns]  overlap growth depth
    scene_beta: np.ndarray       # int32 [ns]  weight search depth
    n_sets: np.ndarray           # int32 [ns]  workers per scene
    set_of_body: np.ndarray      # int32 [n]   initial worker (scene-local index)
    iters: int = 20
    steps: int = 60
    lb_activate: int = 1
    lb_deact_every: int = 1
    assign_overlap: bool = False  # run the articulated assignment at setup
    meta: dict = field(default_factory=dict)
    # float32 [n,3] half extents, or None: every body a sphere.  A row of
    # zeros is a sphere; a positive row is a box (radius = its bounding
    # radius).  The step does not simulate boxes yet.
    half_extents: np.ndarray | None = None

    @property
    def n_bodies(self) -> int:
        return int(self.state.shape[0])

    @property
    def n_scenes(self) -> int:
        return int(self.scene_mu.shape[0])


def _identity_state(pos: np.ndarray) -> np.ndarray:
    n = pos.shape[0]
    st = np.zeros((n, 13), dtype=np.float64)
    st[:, 0:3] = pos
    st[:, 3] = 1.0
    return st.astype(np.float32)


def _single(name, pos, radius, inv_mass, planes, mu, dt, flags, gamma, beta, n_sets, set_of_body,
            joints=None, anchors=None, **kw) -> Scene:
    n = pos.shape[0]
    if joints is None:
        joints = np.zeros((0, 2), dtype=np.int32)
        anchors = np.zeros((0, 6), dtype=np.float32)
    planes = np.asarray(planes, dtype=np.float64).reshape(-1, 4).astype(np.float32)
    return Scene(
        name=name,
        state=_identity_state(pos),
        radius=np.asarray(radius, dtype=np.float64).astype(np.float32).reshape(n),
        inv_mass=np.asarray(inv_mass, dtype=np.float64).astype(np.float32).reshape(n),
        planes=planes,
        plane_scene=np.zeros(planes.shape[0], dtype=np.int32),
        joints=np.asarray(joints, dtype=np.int32).reshape(-1, 2),
        anchors=np.asarray(anchors, dtype=np.float64).astype(np.float32).reshape(-1, 6),
        scene_of_body=np.zeros(n, dtype=np.int32),
        scene_mu=np.array([mu], dtype=np.float32),
        scene_dt=np.array([dt], dtype=np.float32),
        scene_flags=np.array([flags], dtype=np.int32),
        scene_gamma=np.array([gamma], dtype=np.int32),
        scene_beta=np.array([beta], dtype=np.int32),
        n_sets=np.array([n_sets], dtype=np.int32),
        set_of_body=np.asarray(set_of_body, dtype=np.int32).reshape(n),
        **kw,
    )


# ----------------------------------------------------------------------------
# Workload scenes
# ----------------------------------------------------------------------------

def _lattice_pile(nx, ny, nz, spacing, z0, jitter, rng, count=None):
    """Lattice centres, x fastest: id = i + nx*(j + ny*k); centred in x and y."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pos = np.stack([(i - (nx - 1) / 2.0) * spacing,
                    (j - (ny - 1) / 2.0) * spacing,
                    z0 + k * spacing], axis=-1).reshape(-1, 3).astype(np.float64)
    if count is not None:
        pos = pos[:count]
    if jitter > 0:
        pos = pos + rng.uniform(pos.size, -jitter, jitter).reshape(pos.shape)
    return pos


def pile_small(seed: int = 0) -> Scene:
    """256 spheres r=0.5, m=1 in an 8x8x4 lattice (spacing 1) + U(-0.01,0.01)
    jitter on a ground plane z=0; mu=0.5, dt=1/60, 20 iterations, 60 steps;
    two sets split at x = 0; overlap growth depth 1, weight search depth 4."""
    rng = SplitMix64(seed)
    pos = _lattice_pile(8, 8, 4, 1.0, 0.5, 0.01, rng)
    n = pos.shape[0]
    sets = (pos[:, 0].astype(np.float32) >= 0).astype(np.int32)
    return _single("pile_small", pos, np.full(n, 0.5), np.ones(n), [[0, 0, 1, 0]],
                   mu=0.5, dt=1.0 / 60.0, flags=1, gamma=1, beta=4, n_sets=2,
                   set_of_body=sets, iters=20, steps=60, lb_deact_every=1)


def _chain_geometry(n, span, drop, ground_z, radius):
    """U-shaped polyline from (-span/2,0,0) down to the ground, along x, and up
    to (+span/2,0,0); n sphere centres at arc lengths (i+1)*l, l = path/(n+1).
    Joint pivots sit halfway between consecutive centres (and between each end
    sphere and its world anchor)."""
    bottom = ground_z + radius
    p0 = np.array([-span / 2, 0.0, 0.0])
    p1 = np.array([-span / 2, 0.0, bottom])
    p2 = np.array([span / 2, 0.0, bottom])
    p3 = np.array([span / 2, 0.0, 0.0])
    seg = [p0, p1, p2, p3]
    lens = [np.linalg.norm(seg[k + 1] - seg[k]) for k in range(3)]
    total = sum(lens)
    ell = total / (n + 1)

    def at(s):
        for k in range(3):
            if s <= lens[k] or k == 2:
                t = min(max(s / lens[k], 0.0), 1.0)
                return seg[k] + t * (seg[k + 1] - seg[k])
            s -= lens[k]

    centres = np.array([at((i + 1) * ell) for i in range(n)])
    joints = []
    anchors = []
    # world -> sphere 0
    piv = 0.5 * (p0 + centres[0])
    joints.append((-1, 0))
    anchors.append(np.concatenate([piv, piv - centres[0]]))
    for i in range(1, n):
        piv = 0.5 * (centres[i - 1] + centres[i])
        joints.append((i - 1, i))
        anchors.append(np.concatenate([piv - centres[i - 1], piv - centres[i]]))
    piv = 0.5 * (centres[n - 1] + p3)
    joints.append((n - 1, -1))
    anchors.append(np.concatenate([piv - centres[n - 1], piv]))
    return centres, np.array(joints, dtype=np.int32), np.array(anchors), ell


def chain(seed: int = 1, n: int = 4096, n_sets: int = 8, gamma: int = 2, beta: int | None = None,
          iters: int = 50) -> Scene:
    """Hanging chain: n spheres r=0.1, m~U(0.5,2), ball joints, ends fixed to
    world anchors 300 m apart, ground plane at z=-50 (the lower run rests on it).
    8 contiguous sets; articulated overlap assignment with growth depth gamma
    (2), weight search depth beta (2 gamma + 2); dt=1/120, 50 iterations, 120
    steps."""
    rng = SplitMix64(seed)
    centres, joints, anchors, ell = _chain_geometry(n, 300.0, 50.0, -50.0, 0.1)
    mass = rng.uniform(n, 0.5, 2.0)
    sets = (np.arange(n) * n_sets) // n
    sc = _single("chain", centres, np.full(n, 0.1), 1.0 / mass, [[0, 0, 1, -50.0]],
                 mu=0.5, dt=1.0 / 120.0, flags=0, gamma=gamma,
                 beta=2 * gamma + 2 if beta is None else beta, n_sets=n_sets,
                 set_of_body=sets, joints=joints, anchors=anchors, iters=iters, steps=120,
                 lb_deact_every=1, assign_overlap=True)
    sc.meta["link_length"] = ell
    return sc


def kmeans_sets(pos: np.ndarray, k: int, seed: int, iters: int = 50) -> np.ndarray:
    """FP64 Lloyd k-means with k-means++ seeding (Arthur & Vassilvitskii 2007);
    ties go to the lower centroid index.  Returns the cluster of every point."""
    rng = SplitMix64(seed)
    x = pos.astype(np.float64)
    n = x.shape[0]
    first = min(int(rng.uniform(1)[0] * n), n - 1)
    cent = [x[first]]
    d2 = np.sum((x - cent[0]) ** 2, axis=1)
    for _ in range(1, k):
        c = np.cumsum(d2)
        r = rng.uniform(1)[0] * c[-1]
        idx = min(int(np.searchsorted(c, r, side="right")), n - 1)
        cent.append(x[idx])
        d2 = np.minimum(d2, np.sum((x - x[idx]) ** 2, axis=1))
    cent = np.array(cent)
    xx = np.sum(x * x, axis=1)[:, None]
    for _ in range(iters):
        dist = xx - 2.0 * x @ cent.T + np.sum(cent * cent, axis=1)[None, :]
        lab = np.argmin(dist, axis=1)
        cnt = np.bincount(lab, minlength=k).astype(np.float64)
        new = np.stack([np.bincount(lab, weights=x[:, a], minlength=k) for a in range(3)], axis=1)
        keep = cnt > 0
        cent[keep] = new[keep] / cnt[keep, None]
    dist = xx - 2.0 * x @ cent.T + np.sum(cent * cent, axis=1)[None, :]
    return np.argmin(dist, axis=1).astype(np.int32)


def bowl_planes(angle_deg: float = 30.0) -> np.ndarray:
    """Four planes through the origin forming an inverted square pyramid."""
    s, c = math.sin(math.radians(angle_deg)), math.cos(math.radians(angle_deg))
    return np.array([[s, 0, c, 0], [-s, 0, c, 0], [0, s, c, 0], [0, -s, c, 0]], dtype=np.float64)


def pile_large(seed: int = 2, side: int = 64, n_sets: int = 64, z0: float = 24.0) -> Scene:
    """side^3 spheres (default 262,144), spacing 1.25, x/y centred, bottom layer
    at z=z0 (24), r~U(0.4,0.6), density 1; bowl of 4 planes at 30 degrees; mu=0.6,
    dt=1/60, 30 iterations, 300 steps; sets from k-means on the initial
    positions; growth depth 2, weight search depth 6; load-balance removals
    every 10 steps."""
    rng = SplitMix64(seed)
    pos = _lattice_pile(side, side, side, 1.25, z0, 0.0, rng)
    n = pos.shape[0]
    r = rng.uniform(n, 0.4, 0.6).astype(np.float32).astype(np.float64)
    mass = (4.0 / 3.0) * math.pi * r ** 3
    sets = kmeans_sets(pos.astype(np.float32), n_sets, seed)
    return _single("pile_large", pos, r, 1.0 / mass, bowl_planes(), mu=0.6, dt=1.0 / 60.0,
                   flags=1, gamma=2, beta=6, n_sets=n_sets, set_of_body=sets, iters=30,
                   steps=300, lb_deact_every=10)


def box_planes(half: float) -> np.ndarray:
    """Floor z = 0 and four walls at x, y = +-half, facing inwards."""
    return np.array([[0, 0, 1, 0], [1, 0, 0, -half], [-1, 0, 0, -half],
                     [0, 1, 0, -half], [0, -1, 0, -half]], dtype=np.float64)


def pile_mixed(seed: int = 5, side: int = 128, layers: int = 16, n_sets: int = 64,
               big_radius: float = 1.25, big_layers: int = 2) -> Scene:
    """Bodies with very unequal contact counts, standing in for the floor
    pieces of the paper's Building scene (Section 6): big_layers layers of big
    spheres (radius big_radius, square lattice of spacing 2 big_radius + 0.25)
    resting on the floor of a box, under a side x side x layers lattice of
    small spheres (spacing 1.25, r~U(0.4,0.6)); density 1.  The default has
    262,144 small and 6728 big spheres; a settled big sphere touches tens of
    small ones, a small one about six.  mu=0.6, dt=1/60, 30 iterations; sets
    from k-means on the initial positions; growth depth 2, weight search
    depth 6; load-balance removals every 10 steps."""
    rng = SplitMix64(seed)
    width = side * 1.25
    sp_big = 2.0 * big_radius + 0.25
    nbig = max(1, int(round(width / sp_big)))
    half = max(width, nbig * sp_big) / 2.0 + 0.25
    big = _lattice_pile(nbig, nbig, big_layers, sp_big, big_radius + 0.01, 0.0, rng)
    small = _lattice_pile(side, side, layers, 1.25, big_layers * sp_big + 0.5, 0.0, rng)
    pos = np.concatenate([big, small])
    r = np.concatenate([np.full(big.shape[0], big_radius),
                        rng.uniform(small.shape[0], 0.4, 0.6).astype(np.float32).astype(np.float64)])
    mass = (4.0 / 3.0) * math.pi * r ** 3
    sets = kmeans_sets(pos.astype(np.float32), n_sets, seed)
    return _single("pile_mixed", pos, r, 1.0 / mass, box_planes(half), mu=0.6, dt=1.0 / 60.0,
                   flags=1, gamma=2, beta=6, n_sets=n_sets, set_of_body=sets, iters=30,
                   steps=300, lb_deact_every=10)


def _uneven_sets(rng: SplitMix64, order: np.ndarray, n_sets: int) -> np.ndarray:
    """Cut the given body order at sorted U(0,1) fractions into n_sets pieces."""
    n = order.shape[0]
    cuts = np.sort(rng.uniform(n_sets - 1)) if n_sets > 1 else np.zeros(0)
    bounds = np.concatenate([[0], np.floor(cuts * n).astype(np.int64), [n]])
    bounds = np.maximum.accumulate(bounds)
    sets = np.zeros(n, dtype=np.int32)
    for s in range(n_sets):
        sets[order[bounds[s]:bounds[s + 1]]] = s
    # every set keeps at least one body when possible
    return sets


def concat_scenes(name: str, parts: list[Scene], **kw) -> Scene:
    """Stack independent scenes into one batch (bodies, planes, joints offset)."""
    off = 0
    st, rad, im, pl, ps, jo, an, sob = [], [], [], [], [], [], [], []
    for s_idx, sc in enumerate(parts):
        st.append(sc.state); rad.append(sc.radius); im.append(sc.inv_mass)
        pl.append(sc.planes); ps.append(np.full(sc.planes.shape[0], s_idx, dtype=np.int32))
        j = sc.joints.copy()
        j[j >= 0] += off
        jo.append(j); an.append(sc.anchors)
        sob.append(np.full(sc.n_bodies, s_idx, dtype=np.int32))
        off += sc.n_bodies
    cat = lambda xs, dt: np.concatenate(xs).astype(dt)
    return Scene(
        name=name,
        state=cat(st, np.float32), radius=cat(rad, np.float32), inv_mass=cat(im, np.float32),
        planes=np.concatenate(pl).astype(np.float32).reshape(-1, 4), plane_scene=cat(ps, np.int32),
        joints=np.concatenate(jo).astype(np.int32).reshape(-1, 2),
        anchors=np.concatenate(an).astype(np.float32).reshape(-1, 6),
        scene_of_body=cat(sob, np.int32),
        scene_mu=cat([p.scene_mu for p in parts], np.float32),
        scene_dt=cat([p.scene_dt for p in parts], np.float32),
        scene_flags=cat([p.scene_flags for p in parts], np.int32),
        scene_gamma=cat([p.scene_gamma for p in parts], np.int32),
        scene_beta=cat([p.scene_beta for p in parts], np.int32),
        n_sets=cat([p.n_sets for p in parts], np.int32),
        set_of_body=cat([p.set_of_body for p in parts], np.int32),
        **kw,
    )


def batched(seed: int = 3, n_scenes: int = 512, lo: int = 64, hi: int = 16384) -> Scene:
    """n_scenes independent scenes with log-uniform sizes in [lo, hi]: even
    scenes are piles like ``pile_small`` (ceil(sqrt(B/4)) square layers, 4 high,
    truncated to B), odd scenes are chains like ``chain`` with every length
    scaled by B/4096.  Each scene has U{1..16} sets cut at sorted uniform
    fractions of the body order; dt 1/60 (piles) and 1/120 (chains); 30
    iterations, 100 steps."""
    rng = SplitMix64(seed)
    sizes = np.rint(np.exp(rng.uniform(n_scenes, math.log(lo), math.log(hi)))).astype(np.int64)
    nsets = np.minimum(1 + np.floor(rng.uniform(n_scenes) * 16).astype(np.int64), 16)
    parts = []
    for s in range(n_scenes):
        b = int(sizes[s])
        ns = int(min(nsets[s], b))
        if s % 2 == 0:
            side = int(math.ceil(math.sqrt(b / 4.0)))
            # the first b lattice sites (lowest layers first), then jitter
            pos = _lattice_pile(side, side, 4, 1.0, 0.5, 0.01, rng, count=b)
            n = pos.shape[0]
            order = np.argsort(pos[:, 0], kind="stable")
            sets = _uneven_sets(rng, order, ns)
            parts.append(_single(f"pile{s}", pos, np.full(n, 0.5), np.ones(n), [[0, 0, 1, 0]],
                                 mu=0.5, dt=1.0 / 60.0, flags=1, gamma=1, beta=4, n_sets=ns,
                                 set_of_body=sets))
        else:
            sc = b / 4096.0
            centres, joints, anchors, _ = _chain_geometry(b, 300.0 * sc, 50.0 * sc, -50.0 * sc, 0.1)
            mass = rng.uniform(b, 0.5, 2.0)
            sets = _uneven_sets(rng, np.arange(b), ns)
            parts.append(_single(f"chain{s}", centres, np.full(b, 0.1), 1.0 / mass,
                                 [[0, 0, 1, -50.0 * sc]], mu=0.5, dt=1.0 / 120.0, flags=0,
                                 gamma=2, beta=6, n_sets=ns, set_of_body=sets, joints=joints,
                                 anchors=anchors))
    out = concat_scenes("batched", parts, iters=30, steps=100, lb_deact_every=1,
                        assign_overlap=True)
    out.meta["sizes"] = sizes
    return out


# ----------------------------------------------------------------------------
# Small scenes with closed-form answers (used by the oracle's pins)
# ----------------------------------------------------------------------------

def resting_sphere(mass: float = 2.0, radius: float = 0.5, dt: float = 1.0 / 60.0) -> Scene:
    """One sphere touching the ground plane z=0 exactly (gap 0), at rest."""
    pos = np.array([[0.25, -0.5, radius]])
    return _single("resting_sphere", pos, [radius], [1.0 / mass], [[0, 0, 1, 0]], mu=0.5,
                   dt=dt, flags=1, gamma=0, beta=2, n_sets=1, set_of_body=[0], iters=20, steps=1)


def sphere_column(k: int = 4, mass: float = 1.0, radius: float = 0.5, mu: float = 0.0,
                  dt: float = 1.0 / 60.0, iters: int = 400) -> Scene:
    """k equal spheres stacked exactly (gaps 0) on the ground plane z=0."""
    pos = np.array([[0.0, 0.0, radius * (2 * i + 1)] for i in range(k)])
    return _single("sphere_column", pos, np.full(k, radius), np.full(k, 1.0 / mass),
                   [[0, 0, 1, 0]], mu=mu, dt=dt, flags=1, gamma=0, beta=2, n_sets=1,
                   set_of_body=np.zeros(k), iters=iters, steps=1)


def incline_sphere(theta_deg: float = 20.0, mass: float = 1.5, radius: float = 0.3,
                   mu: float = 0.5, dt: float = 1.0 / 60.0) -> Scene:
    """One sphere touching a plane through the origin tilted by theta about y
    (normal (-sin, 0, cos)), at rest; the slope runs along the contact's second
    tangent direction."""
    th = math.radians(theta_deg)
    nrm = np.array([-math.sin(th), 0.0, math.cos(th)])
    pos = (radius * nrm)[None, :]
    return _single("incline_sphere", pos, [radius], [1.0 / mass], [[nrm[0], nrm[1], nrm[2], 0.0]],
                   mu=mu, dt=dt, flags=1, gamma=0, beta=2, n_sets=1, set_of_body=[0],
                   iters=20, steps=1)


def pendulum(length: float = 1.0, mass: float = 1.3, radius: float = 0.1, angle_deg: float = 0.0,
             dt: float = 1.0 / 120.0) -> Scene:
    """A sphere hanging from a world pivot at the origin by a ball joint whose
    pivot is at distance ``length`` from the centre; ``angle_deg`` tilts the
    initial rod in the x-z plane (0 = hanging straight down, at rest)."""
    a = math.radians(angle_deg)
    c = np.array([length * math.sin(a), 0.0, -length * math.cos(a)])
    joints = np.array([[-1, 0]])
    anchors = np.array([[0.0, 0.0, 0.0, -c[0], -c[1], -c[2]]])
    return _single("pendulum", c[None, :], [radius], [1.0 / mass], np.zeros((0, 4)), mu=0.5,
                   dt=dt, flags=1, gamma=0, beta=2, n_sets=1, set_of_body=[0], joints=joints,
                   anchors=anchors, iters=50, steps=600)


def free_flight(n: int = 3, seed: int = 9, dt: float = 1.0 / 60.0) -> Scene:
    """n spheres far apart with random linear and angular velocities, no planes."""
    rng = SplitMix64(seed)
    pos = np.stack([np.arange(n) * 10.0, np.zeros(n), np.full(n, 5.0)], axis=1)
    sc = _single("free_flight", pos, np.full(n, 0.5), np.full(n, 0.7), np.zeros((0, 4)), mu=0.5,
                 dt=dt, flags=1, gamma=0, beta=2, n_sets=1, set_of_body=np.zeros(n), iters=10,
                 steps=1)
    st = sc.state.astype(np.float64)
    st[:, 7:13] = rng.uniform(n * 6, -2.0, 2.0).reshape(n, 6)
    sc.state = st.astype(np.float32)
    return sc


def random_pile(n: int, seed: int, n_sets: int = 3, box: float = 3.0, radius_lo: float = 0.3,
                radius_hi: float = 0.5, planes=None, mu: float = 0.5, gamma: int = 1,
                beta: int = 4) -> Scene:
    """n spheres at random positions in a box (overlaps allowed), random radii
    and masses, random velocities; sets by x-slabs.  Used for brute-force and
    parity cases at small sizes."""
    rng = SplitMix64(seed)
    pos = np.stack([rng.uniform(n, -box, box), rng.uniform(n, -box, box),
                    rng.uniform(n, 0.3, 2 * box)], axis=1)
    r = rng.uniform(n, radius_lo, radius_hi)
    m = rng.uniform(n, 0.5, 2.0)
    if planes is None:
        planes = [[0, 0, 1, 0]]
    order = np.argsort(pos[:, 0].astype(np.float32), kind="stable")
    sets = np.zeros(n, dtype=np.int32)
    sets[order] = (np.arange(n) * n_sets) // n
    sc = _single(f"random_pile{n}", pos, r, 1.0 / m, planes, mu=mu, dt=1.0 / 60.0, flags=1,
                 gamma=gamma, beta=beta, n_sets=n_sets, set_of_body=sets, iters=20, steps=1)
    st = sc.state.astype(np.float64)
    st[:, 7:10] = rng.uniform(n * 3, -1.0, 1.0).reshape(n, 3)
    st[:, 10:13] = rng.uniform(n * 3, -2.0, 2.0).reshape(n, 3)
    sc.state = st.astype(np.float32)
    return sc


def spinning_sphere(omega_y: float = 3.0, height: float = 0.5, radius: float = 0.5,
                    mass: float = 1.0, dt: float = 1.0 / 60.0) -> Scene:
    """One sphere above the ground plane z=0 with its centre at ``height``
    (height < radius: penetrating), spinning about y, no linear velocity."""
    pos = np.array([[0.0, 0.0, height]])
    sc = _single("spinning_sphere", pos, [radius], [1.0 / mass], [[0, 0, 1, 0]], mu=0.5, dt=dt,
                 flags=1, gamma=0, beta=2, n_sets=1, set_of_body=[0], iters=20, steps=1)
    st = sc.state.astype(np.float64)
    st[0, 11] = omega_y
    sc.state = st.astype(np.float32)
    return sc


def head_on(speed: float = 1.0, gap: float = 0.0, radius: float = 0.5, mass: float = 1.0,
            dt: float = 1.0 / 60.0) -> Scene:
    """Two free spheres on the x axis, ``gap`` apart, moving towards each other
    at ``speed`` each; no planes."""
    pos = np.array([[0.0, 0.0, 5.0], [2 * radius + gap, 0.0, 5.0]])
    sc = _single("head_on", pos, [radius, radius], [1.0 / mass, 1.0 / mass], np.zeros((0, 4)),
                 mu=0.5, dt=dt, flags=1, gamma=0, beta=2, n_sets=1, set_of_body=[0, 0], iters=20,
                 steps=1)
    st = sc.state.astype(np.float64)
    st[0, 7], st[1, 7] = speed, -speed
    sc.state = st.astype(np.float32)
    return sc


# ----------------------------------------------------------------------------
# Learned warm start: seeded parameters and synthetic training rows
# ----------------------------------------------------------------------------

MLP_LAYERS = (12, 64, 64, 3)
MLP_N_PARAMS = 12 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3


def _box_body(c, h, density=1.0):
    """state row, bounding radius and inverse mass of a resting solid box"""
    h = np.asarray(h, np.float64)
    return c, float(np.linalg.norm(h)), 1.0 / (8.0 * h[0] * h[1] * h[2] * density)


def _box_scene(name, bodies, joints, anchors, planes, mu, dt, n_sets, gamma, beta, seed, iters, **kw):
    """bodies: (centre, half extents (zeros = sphere of radius r), radius,
    inverse mass, velocity)"""
    pos = np.array([b[0] for b in bodies], np.float64)
    st = _identity_state(pos)
    st[:, 7:10] = np.array([b[4] for b in bodies], np.float32)
    he = np.array([b[1] for b in bodies], np.float32)
    sc = _single(name, pos, np.array([b[2] for b in bodies]), np.array([b[3] for b in bodies]), planes, mu=mu,
                 dt=dt, flags=1, gamma=gamma, beta=beta, n_sets=n_sets,
                 set_of_body=kmeans_sets(pos, n_sets, seed), joints=joints, anchors=anchors, iters=iters, **kw)
    sc.state = st
    sc.half_extents = he
    return sc


def box_building(seed: int = 7, storeys: int = 12, cells: int = 10, cell: float = 2.0, col_half: float = 0.15,
                 storey_h: float = 1.6, slab_half: float = 0.1, balls: int = 2, n_sets: int = 16,
                 mu: float = 0.6, dt: float = 1.0 / 60.0, iters: int = 30) -> Scene:
    """Stand-in for the Building scene (Section 6: floors, walls and columns
    brought down by two cannon balls, gamma = 0).  Storey s has a column at
    every vertex of a cells x cells grid (pitch `cell`) and a slab over every
    cell, resting on the column tops; the next storey's columns stand on
    the slabs.  Everything touches (gap 0) on a ground plane z = 0.  Then
    `balls` spheres of radius 0.8 fly at the building's side at 15 m/s.
    Defaults: 12 storeys, 2652 boxes and 2 balls (the paper's scene has
    2408 bodies)."""
    hcol = storey_h - 2.0 * slab_half
    bodies = []
    for s in range(storeys):
        base = s * storey_h
        for i in range(cells + 1):
            for j in range(cells + 1):
                c, r, im = _box_body([i * cell, j * cell, base + hcol / 2], [col_half, col_half, hcol / 2])
                bodies.append((c, [col_half, col_half, hcol / 2], r, im, [0, 0, 0]))
        for i in range(cells):
            for j in range(cells):
                h = [cell / 2, cell / 2, slab_half]
                c, r, im = _box_body([(i + 0.5) * cell, (j + 0.5) * cell, base + hcol + slab_half], h)
                bodies.append((c, h, r, im, [0, 0, 0]))
    rb = 0.8
    for k in range(balls):
        y = cells * cell * (k + 1) / (balls + 1)
        bodies.append(([-6.0, y, 3.0 + 2.0 * k], [0, 0, 0], rb, 1.0 / (4.0 / 3.0 * np.pi * rb ** 3 * 8.0),
                       [15.0, 0, 0]))
    planes = np.array([[0.0, 0.0, 1.0, 0.0]])
    return _box_scene("box_building", bodies, np.zeros((0, 2), np.int32), np.zeros((0, 6), np.float32), planes,
                      mu, dt, n_sets, 0, 6, seed, iters)


def plank_bridge(seed: int = 8, planks: int = 1589, half=(0.5, 1.0, 0.05), gap: float = 0.02, height: float = 4.0,
                 balls: int = 2, n_sets: int = 8, gamma: int = 6, beta: int = 14, mu: float = 0.5,
                 dt: float = 1.0 / 60.0, iters: int = 50) -> Scene:
    """Stand-in for the Two-way bridge (Section 6: a long bridge of 3180
    joint constraints, gamma = 6).  Planks of half extents `half` lie in a
    row along x, `gap` apart; ball joints join neighbours at both y edges,
    and the two end planks are jointed to the world the same way: 2 planks
    + 2 joints (3180 at the default 1589 planks).  `balls` spheres of radius
    0.6 fall onto the deck from 2 m above it.  The setup runs the articulated
    assignment (Algorithms 2-3), so that joints across workers start in the
    overlap.  The deck starts straight and taut; it settles by stretching its
    joints a few millimetres."""
    hx, hy, hz = half
    pitch = 2 * hx + gap
    bodies = []
    for i in range(planks):
        c, r, im = _box_body([i * pitch, 0.0, height], half)
        bodies.append((c, list(half), r, im, [0, 0, 0]))
    joints, anchors = [], []
    e = hx + gap / 2
    for sy in (-hy, hy):
        joints.append((-1, 0))
        anchors.append([-e, sy, height, -e, sy, 0.0])          # world pivot, plank 0's own
        for i in range(planks - 1):
            joints.append((i, i + 1))
            anchors.append([e, sy, 0.0, -e, sy, 0.0])
        joints.append((planks - 1, -1))
        anchors.append([e, sy, 0.0, (planks - 1) * pitch + e, sy, height])
    rb = 0.6
    for k in range(balls):
        x = (planks - 1) * pitch * (k + 1) / (balls + 1)
        bodies.append(([x, 0.0, height + hz + 2.0], [0, 0, 0], rb, 1.0 / (4.0 / 3.0 * np.pi * rb ** 3 * 4.0),
                       [0, 0, 0]))
    planes = np.zeros((0, 4))
    return _box_scene("plank_bridge", bodies, np.array(joints, np.int32), np.array(anchors, np.float32), planes,
                      mu, dt, n_sets, gamma, beta, seed, iters, assign_overlap=True)


def bf16_grid(x) -> np.ndarray:
    """FP32 values rounded to the nearest BF16 value (ties to even), still
    stored as FP32: inputs that BF16 arithmetic represents exactly."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def mlp_init_params(seed: int = 5, bias_scale: float = 0.0, bf16_exact: bool = False,
                    zero_output: bool = False) -> np.ndarray:
    """Initial parameters of the 12-64-64-3 network in the C ABI's layout
    (W1 [12][64], b1, W2 [64][64], b2, W3 [64][3], b3): weights uniform in
    +-sqrt(6 / fan_in) (He et al. 2015, uniform form), biases uniform in
    +-bias_scale (zero by default); FP32, optionally on the BF16 grid.
    zero_output: W3 = 0 (the network then starts as the plain warm start)."""
    rng = SplitMix64(seed)
    parts = []
    for fan_in, fan_out in zip(MLP_LAYERS[:-1], MLP_LAYERS[1:]):
        lim = math.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(fan_in * fan_out, -lim, lim))
        parts.append(rng.uniform(fan_out, -bias_scale, bias_scale) if bias_scale > 0 else np.zeros(fan_out))
    if zero_output:
        parts[-2] = np.zeros_like(parts[-2])
    th = np.concatenate(parts).astype(np.float32)
    return bf16_grid(th) if bf16_exact else th


def synthetic_rows(n: int, seed: int = 6) -> tuple[np.ndarray, np.ndarray]:
    """n rows of (12 features, 3 targets) in the ranges the step produces
    (FP32): scaled velocities in +-3, penetration in [0, 2], previous impulses
    around 1, inverse masses in [0, 4], degrees in [0, 1.5], depth in [0, 1];
    targets near the previous impulses.  For gradient and training checks."""
    rng = SplitMix64(seed)
    f = np.zeros((n, 12))
    f[:, 0:3] = rng.uniform(3 * n, -3.0, 3.0).reshape(n, 3)
    f[:, 3] = rng.uniform(n, 0.0, 2.0)
    f[:, 4] = rng.uniform(n, 0.0, 2.0)
    f[:, 5:7] = rng.uniform(2 * n, -0.5, 0.5).reshape(n, 2)
    f[:, 7:9] = rng.uniform(2 * n, 0.0, 4.0).reshape(n, 2)
    f[:, 9:11] = rng.uniform(2 * n, 0.0, 1.5).reshape(n, 2)
    f[:, 11] = rng.uniform(n, 0.0, 1.0)
    t = f[:, 4:7] + rng.uniform(3 * n, -0.3, 0.3).reshape(n, 3)
    return f.astype(np.float32), t.astype(np.float32)


WORKLOADS = {
    "pile_small": pile_small,
    "chain": chain,
    "pile_large": pile_large,
    "pile_mixed": pile_mixed,
    "batched": batched,
    "building": box_building,
    "bridge": plank_bridge,
}
