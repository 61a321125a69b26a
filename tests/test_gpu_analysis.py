"""Bulk shape and spin of a pile and the radius-growth watch (Sec. 4.1, 4.2).

The device's bulk record is compared with the oracle's on states the oracle
produced (written into the library with dem_write_state); the watch latched
inside the step graph is compared with a host scan over dem_pile_bulk at the
same step cadence, which must find the same step and the same record bit for
bit (the graph evaluates the same kernels on the same state).
"""
import math

import numpy as np
import pytest

from paper_2311_11322_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SCALAR = ("mass", "radius", "density", "period", "p_crit", "planet_dist")
VECTOR = ("com", "vcom", "axes", "spin", "L", "moments")


@pytest.fixture(scope="module")
def dem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2311_11322_gb300 import dem as D
    return D


def _load_oracle_state(w, pid, pile):
    w.write(pid, "COM", pile.r)
    w.write(pid, "VEL", pile.v)
    w.write(pid, "QUAT", pile.q)
    w.write(pid, "OMEGA_BODY", pile.wb)
    w.write(pid, "PLANET", pile.planet)


def _cases():
    ic1, p1 = W.config1(0, precision=W.PRECISION_FP64)
    ic2, p2 = W.random_cluster(3, n_agg=80, box=6.0, precision=W.PRECISION_MIXED)
    rng = np.random.default_rng(5)
    ic3 = W.lattice_pile(rng, 300, shapes=("tetra", "rod4", "cube8"))
    p3 = W.settled_params(ic3, 1.0, precision=W.PRECISION_MIXED)
    from paper_2311_11322_gb300 import analysis
    p3, _ = analysis.encounter_params(p3, ic3, start_roche=1.5)
    return [("config1 fp64", ic1, p1, 30), ("random cluster mixed", ic2, p2, 20),
            ("lattice pile + planet", ic3, p3, 5)]


@pytest.mark.parametrize("case", range(3))
def test_bulk_matches_oracle(dem, case):
    import oracle
    oracle.build()
    name, ic, p, steps = _cases()[case]
    pile = oracle.Pile(ic, p)
    pile.step(steps)
    rng = np.random.default_rng(case)
    pile.v = pile.v + rng.standard_normal(pile.v.shape) * 1e-3      # some net spin
    ref = pile.bulk()
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        _load_oracle_state(w, pid, pile)
        got = w.bulk(pid)
    scale = {"com": 1.0 + np.abs(ref["com"]).max(), "vcom": np.abs(pile.v).max(),
             "L": np.abs(ref["L"]).max(), "spin": np.abs(ref["spin"]).max(),
             "moments": ref["moments"].max(), "axes": ref["axes"].max()}
    for k in VECTOR:
        err = np.abs(got[k] - ref[k]).max() / scale[k]
        assert err < 1e-11, (name, k, got[k], ref[k])
    for k in SCALAR:
        if math.isinf(ref[k]):
            assert math.isinf(got[k]), (name, k)
        else:
            assert got[k] == pytest.approx(ref[k], rel=1e-11, abs=1e-300), (name, k)
    assert (got["planet_dist"] > 0) == (p.ext_mass > 0)


def test_watch_latches_where_a_host_scan_finds_the_growth(dem):
    """A cluster expanding in a uniform radial flow: the watch, evaluated
    every 3 steps in the graph, latches at the first multiple of 3 whose bulk
    radius reaches 1.02 R_b0; a second world stepping 3 at a time and reading
    dem_pile_bulk finds the same step and the same record."""
    ic, p = W.random_cluster(9, n_agg=60, box=8.0, speed=0.05, precision=W.PRECISION_MIXED)
    m = W.sphere_mass(ic.radius, ic.density)
    first = np.concatenate([[0], np.cumsum(ic.counts)[:-1]])
    M = np.add.reduceat(m, first)
    com = np.add.reduceat(m[:, None] * ic.pos, first) / M[:, None]
    c = (M[:, None] * com).sum(0) / M.sum()
    ic.vel = ic.vel + 0.02 * (com - c)          # R_b grows ~2% per second
    growth, every = 0.02, 3
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        before = w.bulk(pid)
        k0 = w.graph_kernel_count()
        w.watch(pid, growth, every)
        assert w.graph_kernel_count() == k0 + 1
        res = w.watch_result(pid)
        assert res["armed"] and res["fired_step"] is None
        for k in before:
            assert np.array_equal(res["at_arm"][k], before[k]), k
        steps = 0
        while res["fired_step"] is None and steps < 6000:
            w.step(7)
            steps += 7
            res = w.watch_result(pid)
        assert res["fired_step"] is not None
        fired = res["fired_step"]
        assert fired % every == 0
        w.step(50)                       # latched: later steps change nothing
        again = w.watch_result(pid)
        assert again["fired_step"] == fired
        for k in again["at_fire"]:
            assert np.array_equal(again["at_fire"][k], res["at_fire"][k]), k
        w.watch(pid, 0.0)
        assert not w.watch_result(pid)["armed"]
        assert w.graph_kernel_count() == k0
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        R0 = w.bulk(pid)["radius"]
        n = 0
        while True:
            w.step(every)
            n += every
            b = w.bulk(pid)
            if b["radius"] >= (1.0 + growth) * R0:
                break
        assert n == fired
        for k in b:
            assert np.array_equal(b[k], res["at_fire"][k]), k


def test_watch_survives_relayout_and_batching(dem):
    """A watch armed on the second pile of a world keeps its reference record
    when the first pile is removed (the layout is compacted), and a pile
    without a watch is never evaluated."""
    a = W.random_cluster(1, n_agg=40, box=6.0, precision=W.PRECISION_MIXED)
    b = W.random_cluster(2, n_agg=50, box=6.0, precision=W.PRECISION_MIXED)
    b = (b[0], b[1].replace(max_contacts=a[1].max_contacts))
    with dem.World() as w:
        ia, ib = w.add_pile(*a), w.add_pile(*b)
        w.watch(ib, 0.5, 4)
        w.step(8)
        armed = w.watch_result(ib)
        assert w.watch_result(ia)["armed"] is False
        w.remove(ia)
        after = w.watch_result(ib)
        assert after["armed"] and after["every"] == 4
        for k in armed["at_arm"]:
            assert np.array_equal(after["at_arm"][k], armed["at_arm"][k]), k
        w.step(4)
        assert w.watch_result(ib)["armed"]


def test_bulk_of_a_single_sphere(dem):
    """Degenerate pile, one free sphere: its own equal-moment ellipsoid (axes =
    radius, bulk density = its density, P_crit = sqrt(3 pi / (G rho))), at rest
    (infinite period), no planet."""
    ic = W.PileIC(counts=np.array([1], np.int32), pos=np.array([[3.0, -1.0, 2.0]]),
                  radius=np.array([2.5]), density=np.array([1800.0]))
    p = W.Params(dt=0.01, kn=1e3, kt=2e3 / 7, eps=0.1, precision=W.PRECISION_MIXED)
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        b = w.bulk(pid)
    assert np.allclose(b["axes"], 2.5, rtol=1e-12)
    assert b["radius"] == pytest.approx(2.5, rel=1e-12)
    assert b["density"] == pytest.approx(1800.0, rel=1e-12)
    assert b["p_crit"] == pytest.approx(math.sqrt(3 * math.pi / (p.G * 1800.0)), rel=1e-12)
    assert math.isinf(b["period"]) and b["planet_dist"] == 0.0
    assert np.allclose(b["com"], [3.0, -1.0, 2.0], atol=1e-12)


def test_watch_rejects_bad_arguments(dem):
    ic, p = W.random_cluster(4, n_agg=10, box=4.0, precision=W.PRECISION_MIXED)
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        for g, e in ((-0.1, 1), (float("nan"), 1), (0.1, 0)):
            with pytest.raises(dem.DemError):
                w.watch(pid, g, e)
        with pytest.raises(dem.DemError):
            w.watch(pid + 7, 0.1, 1)
        with pytest.raises(dem.DemError):
            w.bulk(pid + 7)


def test_spinup_run_reports_a_critical_spin_ratio(dem):
    """A small progenitor settles, is re-added with a spin ramp (Sec. 4.1)
    and spun until its bulk radius has grown 5%: the latch comes with a
    finite spin period and a positive critical spin ratio."""
    from paper_2311_11322_gb300 import analysis
    rng = np.random.default_rng(3)
    ic = W.lattice_pile(rng, 250, shapes=("tetra",))
    p = W.settled_params(ic, 1.0, precision=W.PRECISION_MIXED)
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        ic_s = analysis.settled(w, pid, 3000)
    with dem.World() as w:
        probe = w.add_pile(ic_s, p)
        b0 = w.bulk(probe)
    omega_c = 2 * math.pi / b0["p_crit"]
    ps = analysis.spinup_params(p, ic_s, 3.0 * omega_c, 20_000)
    with dem.World() as w:
        pid = w.add_pile(ic_s, ps)
        res = analysis.run_until_growth(w, pid, 0.05, every=10, max_steps=40_000, chunk=2_000)
    assert res["fired_step"] is not None
    ratio = analysis.critical_spin_ratio(res)
    assert math.isfinite(ratio) and ratio > 0
    assert res["at_fire"]["radius"] >= 1.05 * res["at_arm"]["radius"]
