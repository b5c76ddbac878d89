"""Parity at full size, in the launch configuration the bench times, on
sampled outputs the oracle's definitions fix one by one:

- contacts of sampled bodies: brute force with the FP32 contact test the
  method decides with (same rounding order), against the step's contact list;
- the constraint graph rows of those bodies: their dynamic partners;
- colours of sampled workers: the oracle's greedy colouring of the worker's
  own constraints (priorities mix64(key), canonical order) equals the GPU's;
- geodesic distances of sampled overlap bodies: breadth-first search on the
  step's graph and masks (Eq 16), exactly; their weights (Eq 15);
- the blend of sampled bodies (Algorithm 4, Eq 11-14) from the step's copies
  and weights; positions of the copies: x + h v;
- every impulse within its bounds: lambda_n >= 0, |lambda_t| <= mu lambda_n;
  every dynamic body in at least one worker.

Large pile: 262,144 spheres, 64 workers, after the 150-step settle the bench
uses; batch: 512 scenes, 1.5 M bodies, 4389 workers."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_17261_gb300 import scenes as S

pytestmark = pytest.mark.gpu

MARGIN = np.float32(0.05)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _f32(x):
    return np.asarray(x, dtype=np.float32)


def _contact_partners(a, st0, sc, cand):
    """Sphere partners b > a of body a (FP32 test, the kernels' rounding order)
    and the planes it touches, as the contact list's second entries."""
    n = sc.n_bodies
    pa = st0[a, 0:3]
    ra = sc.radius[a]
    dyn_a = sc.inv_mass[a] > 0
    s = sc.scene_of_body[a]
    out = []
    if sc.scene_flags[s] & 1:
        for b in cand:
            if b <= a or sc.scene_of_body[b] != s:
                continue
            if not dyn_a and not sc.inv_mass[b] > 0:
                continue
            d = _f32(st0[b, 0:3]) - _f32(pa)
            d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
            rs = (np.float32(ra) + np.float32(sc.radius[b])) + MARGIN
            if d2 <= rs * rs:
                out.append(int(b))
    if dyn_a:
        for k in np.nonzero(sc.plane_scene == s)[0]:
            pl = _f32(sc.planes[k])
            dotp = (pl[0] * pa[0] + pl[1] * pa[1]) + pl[2] * pa[2]
            gap = (dotp - pl[3]) - np.float32(ra)
            if gap <= MARGIN:
                out.append(n + int(k))
    return sorted(out)


def _bfs_depths(o, rp, col, beta):
    depth = {o: 0}
    frontier = [o]
    for d in range(1, beta + 1):
        nxt = []
        for u in frontier:
            for v in col[rp[u]:rp[u + 1]]:
                v = int(v)
                if v not in depth:
                    depth[v] = d
                    nxt.append(v)
        frontier = nxt
    return depth


def _check_step(sim, sc, st0, rng, n_bodies=2000, n_workers=8, n_overlap=400):
    n = sc.n_bodies
    ab, phi, nn, t1 = sim.contacts()
    rp, col = sim.graph()
    masks = sim.membership()
    ent = sim.entries()
    pr = sim.pairs()
    st1 = sim.state()
    dyn = sc.inv_mass > 0
    # every dynamic body is in some worker
    assert np.all(masks[dyn] != 0) and np.all(masks[~dyn] == 0)

    # contacts and graph rows of sampled bodies
    from scipy.spatial import cKDTree
    tree = cKDTree(st0[:, 0:3].astype(np.float64))
    reach = 2.0 * float(sc.radius.max()) + float(MARGIN) + 1e-3
    first = np.searchsorted(ab[:, 0], np.arange(n + 1))
    sample = rng.choice(n, size=min(n_bodies, n), replace=False)
    for a in sample:
        cand = tree.query_ball_point(st0[a, 0:3].astype(np.float64), reach)
        want = _contact_partners(int(a), st0, sc, cand)
        got = sorted(int(x) for x in ab[first[a]:first[a + 1], 1])
        assert got == want, (int(a), got, want)
    # graph row of a dynamic body: its dynamic contact and joint partners
    partners = {}
    for a_, b_ in ab:
        if b_ < n and dyn[a_] and dyn[b_]:
            partners.setdefault(int(a_), set()).add(int(b_))
            partners.setdefault(int(b_), set()).add(int(a_))
    for a_, b_ in sc.joints:
        if a_ >= 0 and b_ >= 0 and dyn[a_] and dyn[b_]:
            partners.setdefault(int(a_), set()).add(int(b_))
            partners.setdefault(int(b_), set()).add(int(a_))
    for a in sample:
        row = [int(x) for x in col[rp[a]:rp[a + 1]]]
        assert row == sorted(partners.get(int(a), set())), int(a)

    # colours of sampled workers against the oracle's greedy colouring
    P = int(np.sum(sc.n_sets))
    part_base = np.concatenate([[0], np.cumsum(sc.n_sets)])
    wstart = np.searchsorted(pr["part"], np.arange(P + 1))
    sizes = np.diff(wstart)
    chosen = rng.choice(np.nonzero(sizes > 0)[0], size=min(n_workers, int(np.sum(sizes > 0))), replace=False)
    joint_bit = np.uint64(1) << np.uint64(62)
    for p in chosen:
        s = int(np.searchsorted(part_base, p, side="right") - 1)
        w = p - part_base[s]
        active = np.nonzero((masks >> np.uint64(w)) & np.uint64(1))[0]
        active = active[sc.scene_of_body[active] == s]
        slot = {int(b): i for i, b in enumerate(active)}
        keys = pr["key"][wstart[p]:wstart[p + 1]]
        bs = np.full((keys.shape[0], 2), -1, np.int32)
        for q, key in enumerate(keys):
            if key & joint_bit:
                a_, b_ = sc.joints[int(key & ~joint_bit)]
            else:
                a_, b_ = int(key >> np.uint64(32)), int((key & np.uint64(0xFFFFFFFF)) >> np.uint64(2))
            for e, x in enumerate((a_, b_)):
                if 0 <= x < n and dyn[x]:
                    bs[q, e] = slot[int(x)]
        prio = np.array([O.mix64(int(k)) for k in keys], dtype=np.uint64)
        _, colours = O.colour(bs, prio, len(active))
        assert np.array_equal(colours, pr["colour"][wstart[p]:wstart[p + 1]]), int(p)

    # geodesic distances and weights of sampled overlap bodies
    ep = ent["entry_ptr"]
    k_of = np.diff(ep)
    over = np.nonzero(k_of >= 2)[0]
    if over.size:
        for o in rng.choice(over, size=min(n_overlap, over.size), replace=False):
            s = int(sc.scene_of_body[o])
            beta = int(sc.scene_beta[s])
            depth = _bfs_depths(int(o), rp, col, beta)
            workers = [w for w in range(64) if (int(masks[o]) >> w) & 1]
            want = []
            for wk in workers:
                ds = [d for v, d in depth.items() if d >= 1 and int(masks[v]) == (1 << wk)]
                want.append(min(ds) if ds else 255)
            got = [int(x) for x in ent["D"][ep[o]:ep[o + 1]]]
            assert got == want, (int(o), got, want)
            inv = np.array([1.0 / d if d != 255 else 0.0 for d in want])
            wref = inv / inv.sum() if inv.sum() > 0 else np.full(len(want), 1.0 / len(want))
            np.testing.assert_allclose(ent["weight"][ep[o]:ep[o + 1]], wref, rtol=0, atol=1e-6)

    # blend and copies of sampled bodies
    h = np.float32(sc.scene_dt[0])
    cp = ent["copies"]
    for b in rng.choice(np.nonzero(dyn)[0], size=min(n_bodies, int(dyn.sum())), replace=False):
        e0, e1 = ep[b], ep[b + 1]
        c = cp[e0:e1]
        hb = np.float32(sc.scene_dt[sc.scene_of_body[b]])
        # each copy integrated x + h v from the blended state, in FP32
        assert np.array_equal(c[:, 0:3], (st0[b, 0:3] + hb * c[:, 7:10]).astype(np.float32)), int(b)
        wgt = ent["weight"][e0:e1].astype(np.float64)
        if e1 - e0 == 1:
            assert np.array_equal(st1[b], c[0]), int(b)
            continue
        v = (wgt[:, None] * c[:, 7:13].astype(np.float64)).sum(axis=0)
        np.testing.assert_allclose(st1[b, 7:13], v, rtol=0, atol=1e-5 * max(1.0, np.abs(v).max()))
        xref = st0[b, 0:3].astype(np.float64) + float(hb) * v[0:3]
        np.testing.assert_allclose(st1[b, 0:3], xref, rtol=0, atol=2e-5 + 3e-7 * np.abs(xref).max())
        q = c[:, 3:7].astype(np.float64)
        sign = np.where((q * q[0]).sum(axis=1) < 0, -1.0, 1.0)
        sign[0] = 1.0
        qb = (wgt[:, None] * sign[:, None] * q).sum(axis=0)
        qb /= np.linalg.norm(qb)
        np.testing.assert_allclose(st1[b, 3:7], qb, rtol=0, atol=1e-6)

    # impulse bounds (box friction on the current normal impulse)
    contact = (pr["key"] & joint_bit) == 0
    lam = pr["lam"][contact]
    mu = sc.scene_mu[sc.scene_of_body[(pr["key"][contact] >> np.uint64(32)).astype(np.int64)]]
    assert np.all(lam[:, 0] >= 0)
    assert np.all(np.abs(lam[:, 1]) <= mu * lam[:, 0]) and np.all(np.abs(lam[:, 2]) <= mu * lam[:, 0])
    return dict(contacts=int(ab.shape[0]), pairs=int(pr["key"].shape[0]), overlap=int(over.size))


def test_pile_large_sampled():
    from paper_2403_17261_gb300 import ovl
    sc = S.pile_large()
    sim = ovl.Simulation(sc)
    try:
        for _ in range(152):
            sim.step()
        rng = np.random.default_rng(7)
        for _ in range(2):
            st0 = sim.state()
            sim.step()
            rep = _check_step(sim, sc, st0, rng)
        assert rep["contacts"] > 300_000 and rep["overlap"] > 10_000
    finally:
        sim.close()


def test_batched_sampled():
    from paper_2403_17261_gb300 import ovl
    sc = S.batched()
    sim = ovl.Simulation(sc)
    try:
        sim.step()
        rng = np.random.default_rng(8)
        st0 = sim.state()
        sim.step()
        rep = _check_step(sim, sc, st0, rng, n_workers=12, n_overlap=300)
        assert rep["contacts"] > 1_000_000
    finally:
        sim.close()
