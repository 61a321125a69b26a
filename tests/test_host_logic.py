"""Host-side logic on CPU: the serving loop against a fake engine, pile
sharding across ranks (also under a 2-rank gloo group), workload generators."""
import os

import numpy as np
import pytest

from paper_2311_11322_gb300 import serve, shard
from paper_2311_11322_gb300 import workloads as W


class FakeWorld:
    """Stand-in engine with the World interface: piles advance a counter."""

    def __init__(self, fail_pile_after=None):
        self.piles = {}
        self.next = 0
        self.log = []
        self.fail_after = fail_pile_after or {}

    def add_pile(self, ic, p):
        pid = self.next
        self.next += 1
        self.piles[pid] = {"n": len(ic.radius), "steps": 0}
        self.log.append(("add", pid))
        return pid

    def step(self, n, piles=None, check=True):
        for pid, st in self.piles.items():
            st["steps"] += n
        self.log.append(("step", n, tuple(sorted(self.piles))))
        return 0

    def sync(self, check=True):
        return 0

    def flags(self, pid):
        lim = self.fail_after.get(pid)
        return 2 if lim is not None and self.piles[pid]["steps"] >= lim else 0

    def read(self, pid, field):
        return np.full(3, float(self.piles[pid]["steps"]))

    def remove(self, pid):
        del self.piles[pid]
        self.log.append(("remove", pid))


class VirtualClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


def fake_footprint(n, a, k, prec):
    return 1000 * n


def req(rid, n, steps, t):
    ic = W.PileIC(counts=np.ones(n, np.int32), pos=np.zeros((n, 3)), radius=np.ones(n),
                  density=np.ones(n))
    return serve.Request(rid=rid, ic=ic, params=W.Params(), steps=steps, t_arrival=t)


def test_server_admits_by_budget_and_slots_and_finishes_all():
    clk = VirtualClock()
    w = FakeWorld()
    srv = serve.Server(w, fake_footprint, budget_bytes=1000 * 250, max_piles=2, chunk=50,
                       clock=clk, sleep=clk.sleep)
    reqs = [req(0, 100, 120, 0.0), req(1, 100, 60, 0.0), req(2, 100, 30, 0.0), req(3, 200, 10, 5.0)]
    st = srv.run(reqs)
    assert st["completed"] == 4 and st["failed"] == 0
    # never more than 2 piles, never more than the budget
    live = set()
    for e in w.log:
        if e[0] == "add":
            live.add(e[1])
            assert len(live) <= 2
        elif e[0] == "remove":
            live.discard(e[1])
    # each request ran exactly its number of steps
    for r in srv.done:
        assert r.result["COM"][0] == r.steps
    # the third request waited for a slot; the 200-sphere one waited for memory
    r2 = [r for r in srv.done if r.rid == 2][0]
    assert r2.t_admit is not None
    steps_taken = [e for e in w.log if e[0] == "step"]
    assert steps_taken[0][1] == 50          # chunk-limited
    assert st["p50_time_to_finish_s"] is not None


def test_server_rejects_oversize_and_retires_failed_piles():
    clk = VirtualClock()
    w = FakeWorld(fail_pile_after={0: 20})
    srv = serve.Server(w, fake_footprint, budget_bytes=1000 * 150, max_piles=4, chunk=10,
                       clock=clk, sleep=clk.sleep)
    reqs = [req(0, 100, 100, 0.0), req(1, 500, 10, 0.0), req(2, 40, 30, 0.0)]
    st = srv.run(reqs)
    status = {r.rid: r.status for r in srv.done}
    assert status == {0: "failed", 1: "failed", 2: "done"}
    assert "budget" in [r for r in srv.done if r.rid == 1][0].result["error"]
    assert st["completed"] == 1


def test_server_overlaps_late_arrivals():
    """A request arriving while another runs is admitted at the next round
    boundary and runs alongside it."""
    clk = VirtualClock()

    class TimedWorld(FakeWorld):
        def step(self, n, piles=None, check=True):
            clk.t += 0.01 * n
            return super().step(n, piles, check)

    w = TimedWorld()
    srv = serve.Server(w, fake_footprint, budget_bytes=10 ** 9, max_piles=8, chunk=10,
                       clock=clk, sleep=clk.sleep)
    srv.run([req(0, 10, 200, 0.0), req(1, 10, 50, 0.35)])
    overlap = [e for e in w.log if e[0] == "step" and len(e[2]) == 2]
    assert overlap, "the late request never ran together with the first"


def test_shard_is_complete_disjoint_and_balanced():
    rng = np.random.default_rng(0)
    sizes = W.pile_sizes_config4(rng, 256)
    for ws in (1, 2, 4, 8):
        sh = shard.shard_piles(sizes, ws)
        flat = sorted(k for s in sh for k in s)
        assert flat == list(range(len(sizes)))
        assert shard.imbalance(sizes, sh) < 1.1
    assert shard.shard_piles(sizes, 4) == shard.shard_piles(sizes, 4)


def _gloo_worker(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    rng = np.random.default_rng(1)
    sizes = W.pile_sizes_config4(rng, 64)
    mine = shard.shard_piles(sizes, ws)[rank]
    # every rank derives the same placement: gather and compare
    objs = [None] * ws
    dist.all_gather_object(objs, mine)
    # max over ranks of a per-rank time, as bench.py reduces it
    t = torch.tensor([float(sum(sizes[k] ** 2 for k in mine))], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, objs, float(t.item())))
    dist.destroy_process_group()


def test_shard_under_two_rank_gloo_group():
    import multiprocessing as mp
    torch = pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    ps = [ctx.Process(target=_gloo_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, objs0, t0), (r1, objs1, t1) = sorted(out)
    assert objs0 == objs1
    assert sorted(objs0[0] + objs0[1]) == list(range(64))
    assert t0 == t1 and t0 > 0


def test_workloads_are_seeded_and_consistent():
    a, pa = W.config1(3)
    b, pb = W.config1(3)
    assert np.array_equal(a.pos, b.pos) and pa == pb
    assert a.n_sph == 1000 and a.n_agg == 250
    ic, p = W.config2(0, n_spheres=3001, ball=300.0)
    assert ic.n_sph == 3001
    # touching spheres inside each aggregate
    first = np.concatenate([[0], np.cumsum(ic.counts)[:-1]])
    for a_, c in zip(first[:50], ic.counts[:50]):
        if c >= 2:
            d = np.linalg.norm(ic.pos[a_] - ic.pos[a_ + 1])
            assert d == pytest.approx(2 * ic.radius[a_], rel=1e-12) or c == 4
    dl, _ = W.dense_lattice(n_spheres=4000, seed=1)
    assert dl.n_sph == 4000
    tr = W.config5_trace(0, n_arrivals=10)
    assert all(1000 <= t["n_spheres"] <= 100000 for t in tr)
    assert all(tr[k]["t_arrival"] < tr[k + 1]["t_arrival"] for k in range(9))


def test_e2_collapse_populations():
    """The profiling collapse of Sec. 3: 2e4 spheres of 50 m, as free spheres, as
    one grain shape (2,500 cubes ... 10,000 dumbbells) or as a mix; members of
    every shape touch, bounding spheres do not overlap."""
    for kind, n_agg in (("spheres", 20_000), ("dumbbell", 10_000), ("cube8", 2_500),
                        ("diamond", 5_000), ("rod4", 5_000), ("tetra", 5_000)):
        ic, p = W.e2_collapse(kind, seed=1)
        assert ic.n_sph == 20_000 and ic.n_agg == n_agg
        assert np.all(ic.radius == 50.0)
        assert p.eps == 5.0 and p.dt > 0
    ic, _ = W.e2_collapse("mixed", seed=1)
    assert ic.n_sph == 20_000 and 2_500 < ic.n_agg < 20_000
    sizes = set(ic.counts.tolist())
    assert {2, 4, 8} <= sizes
    for sh in W.E_SHAPES:
        o = W.shape_offsets(sh, 1.0)
        d = np.linalg.norm(o[:, None] - o[None], axis=2)
        np.fill_diagonal(d, np.inf)
        assert abs(d.min() - 2.0) < 1e-12          # touching, never overlapping
        assert abs(o.mean(axis=0)).max() < 1e-12   # offsets about the centre
        assert len(o) == W.SHAPE_SIZE[sh]


# ---------------------------------------------------------------- analysis runs (host side)
class _FakeWatchWorld:
    """Stands in for a World: the watch latches after a set number of steps."""

    def __init__(self, latch_after, at_arm, at_fire):
        self.latch_after, self.at_arm, self.at_fire = latch_after, at_arm, at_fire
        self.steps, self.armed, self.stepped = 0, None, []

    def watch(self, pile, growth, every):
        self.armed = (pile, growth, every)

    def step(self, n, piles=None):
        self.steps += n
        self.stepped.append((n, tuple(piles)))

    def watch_result(self, pile):
        fired = self.latch_after if self.steps >= self.latch_after else None
        return {"fired_step": fired, "growth": self.armed[1], "every": self.armed[2], "armed": True,
                "at_arm": self.at_arm, "at_fire": self.at_fire if fired is not None else None}


def test_run_until_growth_polls_the_watch_and_stops():
    from paper_2311_11322_gb300 import analysis
    w = _FakeWatchWorld(12_500, {"p_crit": 100.0, "density": 1000.0}, {"period": 123.0, "planet_dist": 5e6})
    res = analysis.run_until_growth(w, 7, 0.05, every=10, max_steps=100_000, chunk=5_000)
    assert w.armed == (7, 0.05, 10)
    assert res["fired_step"] == 12_500 and res["steps_run"] == 15_000
    assert all(p == (7,) for _, p in w.stepped)
    assert analysis.critical_spin_ratio(res) == pytest.approx(1.23)
    # Roche normalisation: d / (1.26 R (rho_M / rho_m)^(1/3))
    d_roche = 1.26 * W.EARTH_RADIUS * (5514.0 / 1000.0) ** (1 / 3)
    assert analysis.disruption_ratio(res) == pytest.approx(5e6 / d_roche)
    never = _FakeWatchWorld(10 ** 9, {"p_crit": 1.0, "density": 1.0}, {})
    res = analysis.run_until_growth(never, 0, 0.005, max_steps=20_000, chunk=3_000)
    assert res["fired_step"] is None and res["steps_run"] == 20_000
    assert analysis.critical_spin_ratio(res) is None and analysis.disruption_ratio(res) is None


def test_spinup_and_encounter_parameters():
    """The spin ramp reaches the target over the stated steps about the axis;
    the encounter starts the planet on the incoming branch at the requested
    multiple of the Roche distance with the requested periapsis."""
    import math
    from paper_2311_11322_gb300 import analysis
    rng = np.random.default_rng(2)
    ic = W.lattice_pile(rng, 60, shapes=("tetra",))
    p = W.settled_params(ic, 1.0)
    ps = analysis.spinup_params(p, ic, 2e-3, 4000, axis=(0.0, 3.0, 4.0))
    assert np.allclose(np.array(ps.spin_inc) * 4000, [0.0, 1.2e-3, 1.6e-3])
    pe, orb = analysis.encounter_params(p, ic, periapsis_rp=1.2, v_inf_kms=3.0, start_roche=3.0)
    assert pe.ext_mass == W.EARTH_MASS
    assert orb["q"] == pytest.approx(1.2 * W.EARTH_RADIUS) and orb["vinf"] == pytest.approx(3e3)
    m = W.sphere_mass(ic.radius, ic.density)
    com = (m[:, None] * ic.pos).sum(0) / m.sum()
    rel = np.array(pe.ext_pos) - com
    d_roche = 1.26 * W.EARTH_RADIUS * (5514.0 / (2500.0 * 0.6)) ** (1 / 3)
    assert np.linalg.norm(rel) == pytest.approx(3.0 * d_roche, rel=1e-9)
    assert np.dot(rel, pe.ext_vel) < 0          # approaching
    # hyperbolic energy: v^2/2 - mu/r = v_inf^2/2
    mu = W.G_SI * W.EARTH_MASS
    e = 0.5 * np.dot(pe.ext_vel, pe.ext_vel) - mu / np.linalg.norm(rel)
    assert e == pytest.approx(0.5 * 3e3 ** 2, rel=1e-9)
    assert math.isfinite(analysis.roche_distance(1.0, 2.0, 3.0))
