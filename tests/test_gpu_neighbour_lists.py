"""Neighbour-list reuse: the cell list and the per-sphere candidate lists are
rebuilt only when some aggregate may have moved more than half the skin.

Each sphere sums its contacts in the order of its partners' indices, so the
trajectory must be bitwise the same whatever the skin, the cell size and the
steps at which the lists were rebuilt; the tests below check exactly that, and
that rebuilds happen when (and only when) the motion or a state write needs
them.
"""
import numpy as np
import pytest

from paper_2311_11322_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("COM", "VEL", "QUAT", "OMEGA", "FORCE", "TORQUE", "SPHERE_FC", "SPHERE_TC", "CONTACTS")


@pytest.fixture(scope="module")
def dem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2311_11322_gb300 import dem as D
    return D


def _run(dem, ic, p, steps, skin, cell_factor=1.0):
    with dem.World() as w:
        w.set_tuning("skin", skin)
        w.set_tuning("cell_factor", cell_factor)
        pid = w.add_pile(ic, p)
        w.step(steps)
        w.sync()
        out = {f: w.read(pid, f) for f in FIELDS}
        return out, w.info(pid)


@pytest.mark.parametrize("prec", [W.PRECISION_FP64, W.PRECISION_MIXED])
def test_skin_and_cell_size_do_not_change_results(dem, prec):
    """Dense lattice set moving (about 1e-4 R per step): searching afresh every
    step, reusing lists with a small skin (rebuilds every few dozen steps) and
    with a large skin on larger cells give bit-identical states, forces and
    contact histories."""
    ic, p = W.dense_lattice(n_spheres=4000, seed=1, precision=prec, speed=0.01)
    steps = 50
    ref, info0 = _run(dem, ic, p, steps, skin=0.0)
    assert info0["rebuilds"] == steps
    assert ref["CONTACTS"][:, 0].sum() > 10_000
    reb = {}
    for skin, cf in ((0.01, 1.0), (0.3, 1.5)):
        got, info = _run(dem, ic, p, steps, skin=skin, cell_factor=cf)
        assert info["skin"] > 0
        reb[skin] = info["rebuilds"]
        for f in FIELDS:
            assert np.array_equal(got[f], ref[f]), (skin, cf, f)
    assert 1 < reb[0.01] < steps           # the motion forced rebuilds mid-run
    assert 1 <= reb[0.3] < reb[0.01]


def test_long_candidate_lists_do_not_change_results(dem):
    """A violently overlapping cluster with more than 24 candidates for some
    spheres (long lists, many pairs per tile): results still do not depend on
    the skin."""
    ic, p = W.random_cluster(5, n_agg=120, box=5.0, precision=W.PRECISION_MIXED)
    agg = np.repeat(np.arange(len(ic.counts)), ic.counts)
    d = np.linalg.norm(ic.pos[:, None] - ic.pos[None], axis=2)
    near = (d < ic.radius[:, None] + ic.radius[None]) & (agg[:, None] != agg[None])
    assert near.sum(1).max() > 24         # long lists at the first step
    ref, info0 = _run(dem, ic, p, 40, skin=0.0)
    got, info = _run(dem, ic, p, 40, skin=0.5)
    assert info0["rebuilds"] == 40
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), f


def test_lists_kept_while_at_rest_and_rebuilt_after_writes(dem):
    """Dense lattice with slow motion: one rebuild at the first step only; a
    state write forces a rebuild at the next step."""
    ic, p = W.dense_lattice(n_spheres=4000, seed=2, precision=W.PRECISION_MIXED)
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        w.step(30)
        w.sync()
        assert w.info(pid)["rebuilds"] == 1
        w.write(pid, "VEL", w.read(pid, "VEL"))
        assert w.info(pid)["rebuild_next"] == 1
        w.step(5)
        w.sync()
        assert w.info(pid)["rebuilds"] == 2


def test_batched_piles_rebuild_independently(dem):
    """Piles in one batch rebuild independently: a fast pile rebuilds often,
    a pile at rest keeps its lists, and each matches its solo run bitwise."""
    fast = W.random_cluster(8, n_agg=60, box=5.0, precision=W.PRECISION_MIXED)
    ic_s, p_s = W.dense_lattice(n_spheres=2000, seed=9, precision=W.PRECISION_MIXED)
    slow = (ic_s, p_s.replace(max_contacts=fast[1].max_contacts))
    solo = []
    for ic, p in (fast, slow):
        with dem.World() as w:
            w.set_tuning("skin", 0.02)
            pid = w.add_pile(ic, p)
            w.step(60)
            solo.append((w.read(pid, "COM"), w.read(pid, "TORQUE"), w.info(pid)["rebuilds"]))
    with dem.World() as w:
        w.set_tuning("skin", 0.02)
        ids = [w.add_pile(*fast), w.add_pile(*slow)]
        w.step(60)
        for pid, (com, tq, nreb) in zip(ids, solo):
            assert np.array_equal(w.read(pid, "COM"), com)
            assert np.array_equal(w.read(pid, "TORQUE"), tq)
            assert w.info(pid)["rebuilds"] == nreb
        assert w.info(ids[0])["rebuilds"] > w.info(ids[1])["rebuilds"]


@pytest.mark.parametrize("prec", [W.PRECISION_FP64, W.PRECISION_MIXED])
def test_inbox_ranges_do_not_change_results(dem, prec):
    """Each contact tile evaluates the pairs inside it once and shares both
    halves through its inbox; tiles whose lists do not fit are split into
    sphere ranges, and pairs between ranges are evaluated by both.  Forcing
    small ranges (most pairs then cross) must give bit-identical states,
    forces and histories: every pair's shares come from the same canonical
    evaluation and every sphere sums them in partner order.  The one-thread-
    per-sphere form (each pair evaluated by both spheres) must agree too."""
    ic, p = W.dense_lattice(n_spheres=4000, seed=3, precision=prec, speed=0.01)
    res = []
    for mode, cap in ((1, 1280), (1, 96), (1, 40), (0, 1280)):
        with dem.World() as w:
            w.set_tuning("contact_mode", mode)
            w.set_tuning("contact_inbox", cap)
            assert w.get_tuning("contact_inbox") == cap and w.get_tuning("contact_mode") == mode
            pid = w.add_pile(ic, p)
            w.step(30)
            w.sync()
            res.append({f: w.read(pid, f) for f in FIELDS})
    assert res[0]["CONTACTS"][:, 0].sum() > 10_000
    for got in res[1:]:
        for f in FIELDS:
            assert np.array_equal(got[f], res[0][f]), f


def test_lists_longer_than_the_inbox(dem):
    """FP64 tiles hold 640 list entries in their inbox, so a 32-sphere slice of
    a list longer than 20 entries does not fit; the tile form then evaluates
    that slice sphere by sphere and must still agree bitwise with the
    one-thread-per-sphere form, without flagging the pile.  (The mixed path's
    inbox holds 1,280 entries: lists of more than 40.)"""
    from scipy.spatial import cKDTree
    ic, p = W.random_cluster(5, n_agg=40, box=4.0, precision=W.PRECISION_FP64)
    p = p.replace(G=W.G_SI * 1e4, max_contacts=32)
    res, skin = [], None
    for mode in (0, 1):
        with dem.World() as w:
            w.set_tuning("contact_mode", mode)
            w.set_tuning("skin", 0.3)
            pid = w.add_pile(ic, p)
            skin = w.info(pid)["skin"]
            w.step(3)
            w.sync()
            assert w.flags(pid) & dem.DEM_FLAG_SLOTS == 0
            res.append({f: w.read(pid, f) for f in FIELDS})
    # candidate lists at the first step: spheres of other aggregates within the
    # radii sum plus the skin (the positions have barely moved by then)
    agg = np.repeat(np.arange(len(ic.counts)), ic.counts)
    n = np.zeros(len(ic.pos), int)
    for i, j in cKDTree(ic.pos).query_pairs(2.0 * ic.radius.max() + skin):
        if agg[i] != agg[j] and np.linalg.norm(ic.pos[i] - ic.pos[j]) < ic.radius[i] + ic.radius[j] + skin:
            n[i] += 1
            n[j] += 1
    assert n.max() >= 22, n.max()
    for f in FIELDS:
        assert np.array_equal(res[1][f], res[0][f]), f
