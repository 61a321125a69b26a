"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Every comparison runs both on the same seeded inputs.  Aggregate results use
the condition-relative error of parity_util (tolerance 1e-5 mixed, 1e-9 FP64);
contact sets must agree exactly for overlaps above 1e-6 R.
"""
import math

import numpy as np
import pytest

from paper_2311_11322_gb300 import workloads as W
from tests.parity_util import (TOL, agg_errors, contact_set_check, lockstep, resynced_steps,
                               sphere_errors)

pytestmark = pytest.mark.gpu

PRECS = [W.PRECISION_FP64, W.PRECISION_MIXED]


@pytest.fixture(scope="module")
def dem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2311_11322_gb300 import dem as D
    return D


@pytest.fixture(scope="module")
def oracle():
    import oracle as O
    O.build()
    return O


def new_world(dem, **kw):
    return dem.World(**kw)


# ------------------------------------------------------------------ lockstep runs
@pytest.mark.parametrize("prec", PRECS)
def test_random_cluster_lockstep(dem, oracle, prec):
    """Overlapping aggregates of all four shapes, with spin and velocity:
    normal, tangential, rolling and twisting terms live.  10 free steps side by
    side (trajectories of this violent, heavily overlapping cluster separate
    chaotically after that), then 30 steps each taken from the oracle's state."""
    ic, p = W.random_cluster(3, n_agg=70, box=5.0, precision=prec)
    p = p.replace(mu_t=0.05, G=W.G_SI * 1e4)
    pile = oracle.Pile(ic, p, want_scales=True)
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        worst = lockstep(w, pid, pile, 10, TOL[prec], r_ref=1.0)
        assert worst["contacts"] > 20
        assert worst["Fc"] <= 10 * TOL[prec] and worst["Fg"] <= 10 * TOL[prec]
        worst = resynced_steps(w, pid, pile, 30, TOL[prec], p.max_contacts)
        assert worst["contacts"] > 20


@pytest.mark.parametrize("prec", PRECS)
def test_config1_lockstep_100_steps(dem, oracle, prec):
    """The 250-tetrahedron cloud (1,000 spheres), 100 steps, forces every step and
    final COM positions / orientations."""
    ic, p = W.config1(0, precision=prec)
    pile = oracle.Pile(ic, p, want_scales=True)
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        lockstep(w, pid, pile, 100, TOL[prec], r_ref=1.0, every=10)
        r = w.read(pid, "COM")
        q = w.read(pid, "QUAT")
        assert np.max(np.abs(r - pile.r)) < (1e-9 if prec == 0 else 1e-6)
        assert np.max(np.abs(q - pile.q)) < (1e-9 if prec == 0 else 1e-6)


@pytest.mark.parametrize("prec", PRECS)
def test_dense_lattice_lockstep_100_steps(dem, oracle, prec):
    """Contact-stress case: tetrahedra from an FCC lattice overlapping by 0.5% R,
    with random velocities and spins (2,000 spheres, 100 steps)."""
    ic, p = W.dense_lattice(n_spheres=2000, seed=1, precision=prec)
    pile = oracle.Pile(ic, p, want_scales=True)
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        worst = lockstep(w, pid, pile, 100, TOL[prec], r_ref=1.0, every=5)
        assert worst["contacts"] > 3000
        r = w.read(pid, "COM")
        assert np.max(np.abs(r - pile.r)) < (1e-10 if prec == 0 else 1e-6)


@pytest.mark.parametrize("prec", PRECS)
def test_planet_flyby_and_yorp(dem, oracle, prec):
    """External terms: a close planet pass (tidal force on every sphere, planet
    reaction) plus a YORP spin increment, 40 steps."""
    rng = np.random.default_rng(5)
    ic = W.lattice_pile(rng, 150, shapes=("tetra", "rod3"))
    p = W.settled_params(ic, 1.0, precision=prec, eps=0.1)
    com = np.average(ic.pos, axis=0, weights=W.sphere_mass(ic.radius, ic.density))
    p = p.replace(ext_mass=W.EARTH_MASS, ext_pos=tuple(com + np.array([1.2e7, 3.0e6, 0.0])),
                  ext_vel=(-5.0e3, 0.0, 0.0), spin_inc=(0.0, 1e-7, 2e-7), dt=p.dt)
    pile = oracle.Pile(ic, p, want_scales=True)
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        lockstep(w, pid, pile, 40, TOL[prec], r_ref=1.0, every=4)
        pl = w.read(pid, "PLANET")
        assert np.allclose(pl[:3], pile.planet[:3], rtol=0, atol=1e-6)
        assert np.allclose(pl[3:6], pile.planet[3:6], rtol=1e-12, atol=1e-12)
        Fe = w.read(pid, "FORCE_EXT")
        assert np.max(np.abs(Fe)) > 0


# ------------------------------------------------------------------ full size, sampled
def sampled_check(dem, oracle, ic, p, n_agg_sample, tol, seed=0):
    rng = np.random.default_rng(seed)
    A = ic.n_agg
    aggs = np.sort(rng.choice(A, size=min(n_agg_sample, A), replace=False))
    first = np.concatenate([[0], np.cumsum(ic.counts)[:-1]])
    rows = np.concatenate([np.arange(first[a], first[a] + ic.counts[a]) for a in aggs])
    pile = oracle.Pile(ic, p)
    ref = pile.step_sampled(rows)
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        w.step(1)
        Fc = w.read(pid, "SPHERE_FC")[rows]
        Tc = w.read(pid, "SPHERE_TC")[rows]
        Fg = w.read(pid, "SPHERE_FG")[rows]
        F_A = w.read(pid, "FORCE")[aggs]
    scale = ref["Fmag"]
    e_sph = np.linalg.norm(Fc + Fg - ref["Fc"] - ref["Fg"], axis=1) / np.maximum(scale, 1e-300)
    # aggregate totals of the sampled aggregates
    k = 0
    e_agg = []
    for a in aggs:
        c = ic.counts[a]
        Fo = (ref["Fc"][k:k + c] + ref["Fg"][k:k + c] + ref["Fe"][k:k + c]).sum(0)
        sc = scale[k:k + c].sum()
        e_agg.append(np.linalg.norm(F_A[len(e_agg)] - Fo) / max(sc, 1e-300))
        k += c
    et = np.linalg.norm(Tc - ref["Tc"], axis=1) / np.maximum(ref["Tmag"], 1e-300)
    et = np.where(ref["Tmag"] > 0, et, np.linalg.norm(Tc, axis=1))
    return float(e_sph.max()), float(max(e_agg)), float(et.max()), int((ref["Tmag"] > 0).sum())


def test_config2_full_size_sampled(dem, oracle):
    """100,000-sphere collapse cloud (mixed path, as benchmarked): first-step
    gravity and contact forces on 200 sampled aggregates against the oracle."""
    ic, p = W.config2(0)
    es, ea, et, _ = sampled_check(dem, oracle, ic, p, 200, TOL[1])
    assert es <= TOL[1] and ea <= TOL[1] and et <= TOL[1]


@pytest.mark.parametrize("prec", PRECS)
def test_dense_100k_full_size_sampled(dem, oracle, prec):
    """100,000-sphere dense lattice: first-step contacts (9 per sphere) and
    gravity on 150 sampled aggregates."""
    ic, p = W.dense_lattice(n_spheres=100_000, seed=2, precision=prec)
    es, ea, et, ncont = sampled_check(dem, oracle, ic, p, 150, TOL[prec])
    assert ncont > 300
    assert es <= TOL[prec] and ea <= TOL[prec] and et <= TOL[prec]


# ------------------------------------------------------------------ batching
def _three_piles(prec):
    out = []
    for k, n in enumerate((37, 130, 260)):
        rng = np.random.default_rng(10 + k)
        ic = W.lattice_pile(rng, n, shapes=W.SHAPES, spacing_factor=0.95)
        p = W.settled_params(ic, 1.0, precision=prec, eps=0.1)
        out.append((ic, p))
    return out


@pytest.mark.parametrize("prec", PRECS)
def test_batch_alone_equals_mix_bitwise(dem, prec):
    """Each pile stepped alone and stepped inside a batch gives bit-identical
    state: per-pile work never depends on the other piles."""
    piles = _three_piles(prec)
    alone = []
    for ic, p in piles:
        with new_world(dem) as w:
            pid = w.add_pile(ic, p)
            w.step(25)
            alone.append((w.read(pid, "COM"), w.read(pid, "QUAT"), w.read(pid, "FORCE")))
    with new_world(dem) as w:
        ids = [w.add_pile(ic, p) for ic, p in piles]
        w.step(25)
        for pid, ref in zip(ids, alone):
            got = (w.read(pid, "COM"), w.read(pid, "QUAT"), w.read(pid, "FORCE"))
            for g, r in zip(got, ref):
                assert np.array_equal(g, r)


def test_run_twice_bitwise(dem):
    ic, p = W.dense_lattice(n_spheres=4000, seed=3, precision=W.PRECISION_MIXED)
    res = []
    for _ in range(2):
        with new_world(dem) as w:
            pid = w.add_pile(ic, p)
            w.step(20)
            res.append((w.read(pid, "COM"), w.read(pid, "TORQUE"), w.read(pid, "CONTACTS")))
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_remove_pile_keeps_others(dem):
    piles = _three_piles(W.PRECISION_MIXED)
    with new_world(dem) as w:
        ids = [w.add_pile(ic, p) for ic, p in piles]
        w.step(5)
        w.remove(ids[1])
        w.step(10)
        got0, got2 = w.read(ids[0], "COM"), w.read(ids[2], "COM")
    with new_world(dem) as w:
        a = w.add_pile(*piles[0])
        c = w.add_pile(*piles[2])
        w.step(15)
        assert np.array_equal(w.read(a, "COM"), got0)
        assert np.array_equal(w.read(c, "COM"), got2)


def test_step_subset_freezes_others(dem):
    piles = _three_piles(W.PRECISION_MIXED)
    with new_world(dem) as w:
        ids = [w.add_pile(ic, p) for ic, p in piles]
        w.step(3)
        before = w.read(ids[1], "COM")
        w.step(4, piles=[ids[0], ids[2]])
        w.sync()
        assert np.array_equal(w.read(ids[1], "COM"), before)
        assert w.info(ids[0])["steps"] == 7 and w.info(ids[1])["steps"] == 3


@pytest.mark.parametrize("n", [1500, 6000, 20_000])
def test_gravity_split_and_shapes_agree(dem, n):
    """The symmetric form with 512- and (up to 8,192 spheres) 128- and 256-sphere tiles (and 64 up to 2,048),
    and the one-sided form with split j-ranges and other block shapes, only
    reorder sums: the gravity on every sphere agrees to FP32 rounding."""
    ic, p = W.config2(1, n_spheres=n, ball=800.0 * (n / 20_000) ** (1 / 3))
    shapes = [dict(grav_tile=512), dict(grav_sym=0, grav_block=128, grav_ib=2, grav_jchunk=0),
              dict(grav_sym=0, grav_block=64, grav_ib=1, grav_jchunk=n // 4),
              dict(grav_sym=0, grav_block=256, grav_ib=2, grav_jchunk=n // 3)]
    if n <= 8192:
        shapes += [dict(grav_tile=128), dict(grav_tile=256), dict(grav_tile=64)]   # 64: 128 above 2,048
    outs = []
    for kw in shapes:
        with new_world(dem) as w:
            for k, v in kw.items():
                w.set_tuning(k, v)
            pid = w.add_pile(ic, p)
            w.step(1)
            outs.append(w.read(pid, "SPHERE_FG"))
    sc = np.linalg.norm(outs[0], axis=1).max()
    for kw, o in zip(shapes[1:], outs[1:]):
        assert np.max(np.abs(o - outs[0])) < 1e-5 * sc, kw


# ------------------------------------------------------------------ errors and edges
def test_slot_overflow_reported_and_frozen(dem):
    ic, p = W.dense_lattice(n_spheres=800, seed=4, precision=W.PRECISION_MIXED)
    p = p.replace(max_contacts=2)
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        w.step(1)
        with pytest.raises(dem.DemError) as ei:
            w.sync()
        assert ei.value.status == dem.DEM_ERR_SLOTS
        assert w.flags(pid) & dem.DEM_FLAG_SLOTS
        steps = w.info(pid)["steps"]
        w.step(3, check=False)
        w.sync(check=False)
        assert w.info(pid)["steps"] == steps


def test_gravity_range_reported_and_frozen(dem):
    """Mixed direct sum with eps_soft = 0: two aggregates of a 600-sphere pile
    (two 512-sphere tiles, so the integer accumulators are used) put with
    spheres 0.001 s apart, closer than the accumulators' range assumes
    (s_min / 2), raise DEM_FLAG_GRAV_RANGE; the pile is frozen."""
    ic, p = W.config1(0, precision=W.PRECISION_MIXED, n_agg=150)
    p = p.replace(eps=0.0)
    k1 = int(ic.counts[0])
    shift = ic.pos[0] + np.array([1e-3 * ic.radius[0], 0.0, 0.0]) - ic.pos[k1]
    ic.pos[k1:k1 + int(ic.counts[1])] += shift
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        w.step(1)
        with pytest.raises(dem.DemError) as ei:
            w.sync()
        assert ei.value.status == dem.DEM_ERR_NONFINITE
        assert w.flags(pid) & dem.DEM_FLAG_GRAV_RANGE
        steps = w.info(pid)["steps"]
        w.step(2, check=False)
        w.sync(check=False)
        assert w.info(pid)["steps"] == steps


def test_invalid_inputs_rejected(dem):
    ic, p = W.config1(0, n_agg=10, ball=12.0)
    with new_world(dem) as w:
        bad = W.PileIC(ic.counts, ic.pos.copy(), ic.radius, ic.density)
        bad.pos[3, 1] = np.nan
        with pytest.raises(dem.DemError) as ei:
            w.add_pile(bad, p)
        assert ei.value.status == dem.DEM_ERR_ARG and "non-finite" in str(ei.value)
        # a non-positive radius in the last aggregate, and a NaN velocity
        neg = W.PileIC(ic.counts, ic.pos, ic.radius.copy(), ic.density)
        neg.radius[-1] = -1.0
        with pytest.raises(dem.DemError) as ei:
            w.add_pile(neg, p)
        assert ei.value.status == dem.DEM_ERR_ARG and "radius" in str(ei.value)
        vel = np.zeros((len(ic.counts), 3))
        vel[-1, 2] = np.inf
        with pytest.raises(dem.DemError) as ei:
            w.add_pile(W.PileIC(ic.counts, ic.pos, ic.radius, ic.density, vel), p)
        assert ei.value.status == dem.DEM_ERR_ARG and "non-finite" in str(ei.value)
        with pytest.raises(dem.DemError):
            w.add_pile(ic, p.replace(dt=0.0))
        with pytest.raises(dem.DemError):
            w.add_pile(ic, p.replace(max_contacts=0))
        pid = w.add_pile(ic, p)
        with pytest.raises(dem.DemError):
            w.add_pile(ic, p.replace(precision=1 - p.precision))
        with pytest.raises(dem.DemError):
            w.read(pid + 100, "COM")
        w.step(0)


@pytest.mark.parametrize("prec", PRECS)
def test_ragged_and_tiny_piles(dem, oracle, prec):
    """Piles of 1, 2, 3 and 129 spheres (single spheres, one aggregate, ragged
    block tails) in one batch, each against its own oracle."""
    cases = []
    one = W.assemble(["single"], [1.0], np.zeros((1, 3)), np.eye(3)[None], 2500.0)
    one.omega = np.array([[0.01, 0.0, 0.02]])
    cases.append(one)
    cases.append(W.tiny_pair(gap=-0.01, v=0.01))
    tri = W.assemble(["rod3"], [1.0], np.zeros((1, 3)), W.random_rotations(np.random.default_rng(0), 1), 2500.0)
    tri.omega = np.array([[0.003, 0.02, -0.01]])
    cases.append(tri)
    cases.append(W.random_cluster(9, n_agg=43, box=4.0)[0])
    with new_world(dem) as w:
        ids, piles = [], []
        for ic in cases:
            p = W.calibrate(ic, v_max=0.05, r_med=1.0, eps=0.1, precision=prec, overlap_frac=0.05,
                            max_contacts=32)
            p = p.replace(G=W.G_SI * 1e5)
            ids.append(w.add_pile(ic, p))
            piles.append(oracle.Pile(ic, p, want_scales=True))
        for _ in range(20):
            w.step(1)
            for pid, pile in zip(ids, piles):
                pile.step()
        for pid, pile in zip(ids, piles):
            eF, eN = agg_errors(w, pid, pile)
            assert eF.max() <= TOL[prec] and eN.max() <= TOL[prec]
            assert np.max(np.abs(w.read(pid, "COM") - pile.r)) < 1e-6


def test_body_offsets_bit_exact(dem):
    ic, p = W.dense_lattice(n_spheres=2000, seed=5, precision=W.PRECISION_MIXED)
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        b0 = w.read(pid, "BODY_OFFSETS")
        w.step(200)
        assert np.array_equal(w.read(pid, "BODY_OFFSETS"), b0)
        q = w.read(pid, "QUAT")
        assert np.max(np.abs(np.linalg.norm(q, axis=1) - 1.0)) < 1e-14


def test_profiled_step_times_kernel(dem):
    ic, p = W.config2(0, n_spheres=20_000, ball=800.0)
    with new_world(dem) as w:
        w.add_pile(ic, p)
        ms = w.step_profiled(3, "GRAVITY")
        assert ms.shape == (3,) and np.all(ms > 0)


@pytest.mark.parametrize("prec", PRECS)
def test_checkpoint_restore_bitwise(dem, prec):
    """Run 20 steps; separately run 10, checkpoint, restore into a fresh world
    and run 10 more: the final states are bit-identical."""
    ic, p = W.dense_lattice(n_spheres=3000, seed=6, precision=prec)
    p = p.replace(G=W.G_SI * 1e3)
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        w.step(10)
        ck = w.checkpoint(pid)
        w.step(10)
        ref = (w.read(pid, "COM"), w.read(pid, "QUAT"), w.read(pid, "TORQUE"),
               w.read(pid, "CONTACTS"))
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        w.restore(pid, ck)
        w.step(10)
        got = (w.read(pid, "COM"), w.read(pid, "QUAT"), w.read(pid, "TORQUE"),
               w.read(pid, "CONTACTS"))
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)


def test_dense_lattice_resynced_steps_mixed(dem, oracle):
    """Per-step error of the mixed path from identical states (no trajectory
    drift): contacts with friction and rolling on the dense lattice."""
    ic, p = W.dense_lattice(n_spheres=2000, seed=7, precision=W.PRECISION_MIXED)
    pile = oracle.Pile(ic, p, want_scales=True)
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        worst = resynced_steps(w, pid, pile, 20, TOL[1], p.max_contacts)
        assert worst["contacts"] > 3000


def test_config3_full_size_sampled(dem, oracle):
    """200,000-sphere spin-up pile (2-8-sphere clusters in a 3:2:1.5 ellipsoid,
    YORP increment on), mixed path: first-step forces on 100 sampled aggregates."""
    ic, p = W.config3(0)
    assert ic.n_sph == 200_000
    es, ea, et, _ = sampled_check(dem, oracle, ic, p, 100, TOL[1])
    assert es <= TOL[1] and ea <= TOL[1] and et <= TOL[1]


# ------------------------------------------------------------------ free spheres and mixed populations
@pytest.mark.parametrize("prec", PRECS)
def test_free_spheres_and_mixed_population_lockstep(dem, oracle, prec):
    """Free spheres (aggregates of one) alone and mixed with the paper's grain
    shapes (dumbbell, diamond, rod4, tetra, cube8), overlapping: 10 steps side by
    side, then 20 steps each from the oracle's state."""
    for shapes, box in ((("single",), 4.0), (W.E_SHAPES + ("single",), 5.0)):
        ic, p = W.random_cluster(11, n_agg=90, shapes=shapes, box=box, precision=prec)
        pile = oracle.Pile(ic, p, want_scales=True)
        with new_world(dem) as w:
            pid = w.add_pile(ic, p)
            worst = lockstep(w, pid, pile, 10, TOL[prec], r_ref=1.0)
            assert worst["contacts"] > 20
            resynced_steps(w, pid, pile, 20, TOL[prec], p.max_contacts)


def test_e2_collapse_full_size_lockstep(dem, oracle):
    """The paper's profiling collapse (2e4 spheres of 50 m), mixed grain shapes and
    free spheres, mixed path: 3 full steps side by side with the oracle."""
    for kind in ("mixed", "spheres"):
        ic, p = W.e2_collapse(kind, seed=0)
        pile = oracle.Pile(ic, p, want_scales=True)
        with new_world(dem) as w:
            pid = w.add_pile(ic, p)
            lockstep(w, pid, pile, 3, TOL[1], r_ref=50.0)


# ------------------------------------------------------------------ adaptive rotation (Sec. 2.2.1)
@pytest.mark.parametrize("prec", PRECS)
def test_adaptive_rotation_lockstep(dem, oracle, prec):
    """The paper's adaptive fifth-order rotation (rot_tol > 0) on an overlapping
    cluster: side by side with the oracle running the same scheme."""
    ic, p = W.random_cluster(3, n_agg=70, box=5.0, precision=prec)
    p = p.replace(rot_tol=1e-9, mu_t=0.05)
    pile = oracle.Pile(ic, p, want_scales=True)
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        worst = lockstep(w, pid, pile, 10, TOL[prec], r_ref=1.0)
        assert worst["contacts"] > 20
        resynced_steps(w, pid, pile, 10, TOL[prec], p.max_contacts)


@pytest.mark.parametrize("prec", PRECS)
def test_adaptive_rotation_fast_spinners(dem, prec):
    """Isolated asymmetric aggregates spinning fast for the step (|w| h ~ 0.3), no
    gravity, no contacts: with the adaptive scheme the GPU keeps each body's spin
    energy and |L| to ~1e-8 over 200 steps, where one RK4 step per h drifts."""
    rng = np.random.default_rng(4)
    n = 40
    shapes = ["square", "rod3", "tetra", "dumbbell"] * (n // 4)
    coms = np.stack([np.arange(n) * 20.0, np.zeros(n), np.zeros(n)], 1)
    ic = W.assemble(shapes, np.ones(n), coms, W.random_rotations(rng, n), 2500.0)
    ic.omega = rng.standard_normal((n, 3)) * 0.6
    base = W.Params(G=0.0, dt=0.5, kn=0.0, kt=0.0, w0=1.0, eps=0.1, precision=prec, max_contacts=4)
    drift = {}
    for tol in (0.0, 1e-10):
        with new_world(dem) as w:
            pid = w.add_pile(ic, base.replace(rot_tol=tol))
            wb0 = w.read(pid, "OMEGA_BODY")
            w.step(200)
            wb = w.read(pid, "OMEGA_BODY")
            import oracle as O
            agg = O.build_aggregates(ic.counts, ic.pos, ic.radius, ic.density)
            I = agg["I"].reshape(n, 3, 3)
            E0 = np.einsum("ai,aij,aj->a", wb0, I, wb0)
            E1 = np.einsum("ai,aij,aj->a", wb, I, wb)
            L0 = np.linalg.norm(np.einsum("aij,aj->ai", I, wb0), axis=1)
            L1 = np.linalg.norm(np.einsum("aij,aj->ai", I, wb), axis=1)
            drift[tol] = max(np.max(np.abs(E1 / E0 - 1)), np.max(np.abs(L1 / L0 - 1)))
    assert drift[1e-10] < 1e-8
    assert drift[0.0] > 100 * drift[1e-10]


# ------------------------------------------------------------------ tree gravity (the paper's gravity method)
def _fg(dem, ic, p, theta=0.0, steps=1, order=4):
    with new_world(dem) as w:
        if theta:
            w.set_tuning("grav_theta", theta)
            w.set_tuning("grav_order", order)
        pid = w.add_pile(ic, p)
        w.step(steps)
        w.sync()
        return w.read(pid, "SPHERE_FG"), w.flags(pid), w.read(pid, "COM")


# per-sphere relative force error bounds (median, 99th percentile) of the tree
# against the direct sum, about 3x the values measured on the 20,000-sphere cloud
TREE_BOUNDS = {2: ((0.3, 1e-4, 6e-4), (0.5, 6e-4, 4e-3), (0.7, 2e-3, 1.5e-2)),
               4: ((0.3, 3e-6, 2.5e-5), (0.5, 4e-5, 2.5e-4), (0.7, 2.5e-4, 2e-3))}


def test_tree_gravity_error_bound(dem):
    """Tree gravity (opening angle theta; multipoles up to the quadrupole or up
    to the hexadecapole) against the direct sum on a 20,000-sphere collapse
    cloud: per-sphere relative force errors fall with theta within the bounds of
    each expansion, no group of spheres ran out of traversal stack, the
    hexadecapole is several times more accurate at every theta, and its error
    falls faster as theta shrinks (higher order: (theta ratio)^5 vs ^3)."""
    ic, p = W.config2(0, n_spheres=20_000, ball=2000.0 * 0.2 ** (1 / 3))
    ref, _, _ = _fg(dem, ic, p)
    mag = np.linalg.norm(ref, axis=1)
    med = {}
    for order, rows in TREE_BOUNDS.items():
        for theta, p50, p99 in rows:
            fg, flags, _ = _fg(dem, ic, p, theta, order=order)
            assert not flags & dem.DEM_FLAG_TREE
            e = np.linalg.norm(fg - ref, axis=1) / mag
            med[order, theta] = np.median(e)
            assert np.median(e) < p50 and np.quantile(e, 0.99) < p99, (order, theta, np.median(e),
                                                                       np.quantile(e, 0.99))
        assert med[order, 0.3] < med[order, 0.5] < med[order, 0.7]
    for theta in (0.3, 0.5, 0.7):
        assert med[4, theta] < med[2, theta] / 5, theta
    assert med[4, 0.5] / med[4, 0.3] > med[2, 0.5] / med[2, 0.3]


def test_tree_gravity_against_oracle(dem, oracle):
    """The hexadecapole tree against the oracle's direct sum (same positions:
    a cloud at rest, whose first step evaluates gravity where it was built):
    per-sphere relative errors within the tree's bounds for theta 0.5."""
    ic, p = W.config2(2, n_spheres=6000, ball=2000.0 * 0.06 ** (1 / 3))
    agg = oracle.build_aggregates(ic.counts, ic.pos, ic.radius, ic.density)
    ref = oracle.gravity(ic.pos, agg["m"], agg["agg_of"], p.G, p.eps, exclude_same_agg=True)
    fg, flags, _ = _fg(dem, ic, p, 0.5, order=4)
    assert not flags & dem.DEM_FLAG_TREE
    e = np.linalg.norm(fg - ref, axis=1) / np.linalg.norm(ref, axis=1)
    _, p50, p99 = TREE_BOUNDS[4][1]
    assert np.median(e) < p50 and np.quantile(e, 0.99) < p99, (np.median(e), np.quantile(e, 0.99))
    direct, _, _ = _fg(dem, ic, p)
    ed = np.linalg.norm(direct - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert ed.max() < 1e-5          # the direct sum itself: FP32 pair terms only


def test_tree_gravity_deterministic_and_batched(dem):
    """Tree gravity is bitwise reproducible and per pile: a pile alone and in a
    batch with others gives the same state."""
    piles = _three_piles(W.PRECISION_MIXED)
    alone = []
    for ic, p in piles:
        with new_world(dem) as w:
            w.set_tuning("grav_theta", 0.5)
            pid = w.add_pile(ic, p.replace(G=W.G_SI * 1e3))
            w.step(10)
            alone.append((w.read(pid, "COM"), w.read(pid, "SPHERE_FG")))
    with new_world(dem) as w:
        w.set_tuning("grav_theta", 0.5)
        ids = [w.add_pile(ic, p.replace(G=W.G_SI * 1e3)) for ic, p in piles]
        w.step(10)
        for pid, (com, fg) in zip(ids, alone):
            assert np.array_equal(w.read(pid, "COM"), com)
            assert np.array_equal(w.read(pid, "SPHERE_FG"), fg)


@pytest.mark.parametrize("prec", PRECS)
def test_pair_forces_bitwise_opposite(dem, prec):
    """One evaluation of each pair gives both spheres' shares: bitwise opposite
    forces (Newton's third law exactly) and one tangential displacement in the
    contact history (reported from the lower index's side for both rows), with
    unequal radii, an oblique approach, spin and friction."""
    ic = W.tiny_pair(s1=1.0, s2=0.7, gap=-0.02, v=0.05, b=0.2)
    ic.omega = np.array([[0.01, -0.02, 0.03], [-0.03, 0.01, 0.02]])
    p = W.calibrate(ic, v_max=0.05, r_med=0.85, precision=prec, mu_r=0.1, mu_t=0.05).replace(G=0.0)
    with new_world(dem) as w:
        pid = w.add_pile(ic, p)
        for _ in range(6):
            w.step(1)
            fc = w.read(pid, "SPHERE_FC")
            assert np.any(fc != 0)
            assert np.array_equal(fc[0], -fc[1])
            c = w.read(pid, "CONTACTS")
            assert c[0, 0] == 1 and c[1, 0] == 1
            assert np.array_equal(c[0, 2:5], c[1, 2:5])
            assert np.any(c[0, 2:5] != 0)
