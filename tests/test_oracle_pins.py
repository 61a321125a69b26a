"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against a closed form, a symmetry, a library
routine, a hand-worked value or brute force, chosen so that a dropped term, a
wrong sign or index or a transposed operand in the oracle fails at least one.
"""
import math
import os

import numpy as np
import pytest

from paper_2311_11322_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            vals[k] = float(v)
    return vals


def free_params(**kw):
    base = dict(G=0.0, dt=0.01, kn=1e3, kt=2e3 / 7, cn=0.0, ct=0.0, mu_s=0.0, mu_r=0.0,
                mu_t=0.0, w0=1e-9, eps=0.0)
    base.update(kw)
    return W.Params(**base)


# ---------------------------------------------------------------- pin 1
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pair_search_matches_kdtree(oracle_lib, seed):
    """Brute-force contact set == pairs from scipy's k-d tree (library routine)."""
    spatial = pytest.importorskip("scipy.spatial")
    ic, p = W.random_cluster(seed, n_agg=60, box=5.0)
    agg = oracle_lib.build_aggregates(ic.counts, ic.pos, ic.radius, ic.density)
    n = ic.n_sph
    out = oracle_lib.contacts(ic.pos, np.zeros((n, 3)), np.zeros((n, 3)), ic.radius,
                              agg["agg_of"], p)
    got = {tuple(x) for x in out["pairs"].tolist()}
    tree = spatial.cKDTree(ic.pos)
    cand = tree.query_pairs(2.0 * ic.radius.max())
    ref = set()
    for i, j in cand:
        i, j = min(i, j), max(i, j)
        if agg["agg_of"][i] == agg["agg_of"][j]:
            continue
        if np.linalg.norm(ic.pos[i] - ic.pos[j]) < ic.radius[i] + ic.radius[j]:
            ref.add((i, j))
    assert len(ref) > 10
    assert got == ref
    assert np.all(out["x"] > 0)


def test_same_aggregate_pairs_skipped(oracle_lib):
    """Spheres of one aggregate that overlap each other produce no contact."""
    pos = np.array([[0, 0, 0], [1.5, 0, 0], [3.0, 0, 0]], float)
    out = oracle_lib.contacts(pos, np.zeros((3, 3)), np.zeros((3, 3)), np.ones(3),
                              np.array([0, 0, 1], np.int32), free_params())
    assert out["pairs"].tolist() == [[1, 2]]


# ---------------------------------------------------------------- pin 2
def test_gravity_newton_limit(oracle_lib):
    """Two masses far apart: |F| -> G m1 m2 / d^2 (textbook), equal and opposite."""
    G, d = 6.67430e-11, 1000.0
    pos = np.array([[0, 0, 0], [d, 0, 0]], float)
    m = np.array([3.0e6, 5.0e6])
    F = oracle_lib.gravity(pos, m, np.array([0, 1], np.int32), G, eps=1e-3)
    newton = G * m[0] * m[1] / d ** 2
    assert F[0, 0] == pytest.approx(newton, rel=1e-11)
    assert F[1, 0] == pytest.approx(-newton, rel=1e-11)
    assert abs(F[0, 1]) + abs(F[0, 2]) == 0.0


def test_gravity_symmetric_configurations_cancel(oracle_lib):
    """A mass at the centre of an octahedron / cube of equal masses feels no force."""
    rng = np.random.default_rng(3)
    for verts in (np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float),
                  np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], float)):
        R = W.random_rotations(rng, 1)[0]
        pos = np.vstack([[0, 0, 0], verts @ R.T * 7.0]) + 100.0
        m = np.full(len(pos), 2.0e5)
        F = oracle_lib.gravity(pos, m, np.arange(len(pos), dtype=np.int32), 6.67e-11, eps=0.3)
        scale = 6.67e-11 * 2e5 ** 2 / 49.0
        assert np.max(np.abs(F[0])) < 1e-13 * scale


def test_gravity_momentum_and_central(oracle_lib):
    """All-pairs gravity: sum F = 0 and sum r x F = 0 (central pair forces)."""
    rng = np.random.default_rng(5)
    pos = rng.standard_normal((300, 3)) * 50
    m = rng.uniform(1e5, 1e6, 300)
    F, Fm = oracle_lib.gravity(pos, m, np.arange(300, dtype=np.int32), 6.67e-11, eps=0.5,
                               want_mag=True)
    scale = Fm.sum()
    assert np.max(np.abs(F.sum(0))) < 1e-14 * scale
    L = np.cross(pos, F).sum(0)
    assert np.max(np.abs(L)) < 1e-13 * scale * 100


def test_gravity_internal_pairs_cancel_on_aggregates(oracle_lib):
    """Including or excluding pairs inside one aggregate changes F_A and N_A only at
    round-off: internal central forces of a rigid body sum to zero force and torque."""
    ic, p = W.random_cluster(7, n_agg=50, box=30.0)
    agg = oracle_lib.build_aggregates(ic.counts, ic.pos, ic.radius, ic.density)
    Fi, Fm = oracle_lib.gravity(ic.pos, agg["m"], agg["agg_of"], W.G_SI, 0.1, want_mag=True)
    Fx = oracle_lib.gravity(ic.pos, agg["m"], agg["agg_of"], W.G_SI, 0.1, exclude_same_agg=True)
    ao = agg["agg_of"]
    A = ic.n_agg
    for a in range(A):
        sel = ao == a
        rel = ic.pos[sel] - agg["com"][a]
        dF = Fi[sel].sum(0) - Fx[sel].sum(0)
        dN = np.cross(rel, Fi[sel]).sum(0) - np.cross(rel, Fx[sel]).sum(0)
        sc = Fm[sel].sum()
        assert np.max(np.abs(dF)) < 1e-13 * sc
        assert np.max(np.abs(dN)) < 1e-12 * sc * 3.0
    # and the internal pairs are not negligible individually
    assert np.max(np.abs(Fi - Fx)) > 1e-3 * np.max(np.abs(Fx))


# ---------------------------------------------------------------- pin 3
@pytest.mark.parametrize("seed", [0, 1])
def test_contact_pass_conserves_momentum_and_L(oracle_lib, seed):
    """One contact evaluation with friction, rolling and twisting: sum F = 0 and
    sum (r x F + tau) = 0 to round-off."""
    ic, p = W.random_cluster(seed, n_agg=80, box=5.0)
    p = p.replace(mu_r=0.2, mu_t=0.15)
    agg = oracle_lib.build_aggregates(ic.counts, ic.pos, ic.radius, ic.density)
    rng = np.random.default_rng(seed + 10)
    n = ic.n_sph
    vel = rng.standard_normal((n, 3)) * 0.1
    w = rng.standard_normal((n, 3)) * 0.1
    out = oracle_lib.contacts(ic.pos, vel, w, ic.radius, agg["agg_of"], p)
    assert len(out["pairs"]) > 20
    scale = out["Fmag"].sum()
    assert np.max(np.abs(out["Fc"].sum(0))) < 1e-13 * scale
    L = np.cross(ic.pos, out["Fc"]).sum(0) + out["Tc"].sum(0)
    lever = np.max(np.abs(ic.pos)) + 2.0
    assert np.max(np.abs(L)) < 1e-13 * scale * lever
    # friction bound on every contact (F_T <= mu_s |F_N|) is exercised in its own pin


def test_hand_worked_oblique_contact(oracle_lib):
    """Golden: lever arm of Eq. lever_arm and the aggregate torque reading."""
    g = read_golden("two_sphere_oblique.txt")
    # dumbbell (spheres 0, 1, radius 1) along y; free sphere 2 of radius 2
    pos = np.array([[0.0, 1.0, 0.0], [0.0, -1.0, 0.0], [g["dist"], 1.0, 0.0]])
    rad = np.array([g["s_p"], g["s_p"], g["s_n"]])
    ao = np.array([0, 0, 1], np.int32)
    p = free_params(kn=g["kn"])
    out = oracle_lib.contacts(pos, np.zeros((3, 3)), np.zeros((3, 3)), rad, ao, p)
    assert out["pairs"].tolist() == [[0, 2]]
    assert out["x"][0] == pytest.approx(g["overlap"], rel=1e-12)
    assert out["Fc"][0, 0] == pytest.approx(g["force_on_p_x"], rel=1e-12)
    # contact torque about sphere 0's centre is zero (force along the normal) ...
    assert np.max(np.abs(out["Tc"])) < 1e-12
    # ... and the torque on the dumbbell about its COM (0,0,0) is lever x F
    com = pos[:2].mean(0)
    N = np.cross(pos[:2] - com, out["Fc"][:2]).sum(0) + out["Tc"][:2].sum(0)
    lever = np.array([g["l_p"], 1.0, 0.0])
    assert N[2] == pytest.approx(g["torque_dumbbell_z"], rel=1e-12)
    # the hand lever arm gives the same torque directly
    assert np.cross(lever, out["Fc"][0])[2] == pytest.approx(g["torque_dumbbell_z"], rel=1e-12)
    # with a tangential relative velocity the contact point matters: torque about sphere 2
    # equals (-l_n n) x F_2 for the tangential force on it
    vel = np.zeros((3, 3)); vel[2, 1] = 0.01
    p2 = free_params(kn=g["kn"], kt=300.0, ct=0.0, mu_s=10.0, dt=0.5)
    out2 = oracle_lib.contacts(pos, vel, np.zeros((3, 3)), rad, ao, p2)
    F2 = out2["Fc"][2]
    tau2 = np.cross(np.array([-g["l_n"], 0, 0]), F2)
    assert np.allclose(out2["Tc"][2], tau2, rtol=1e-12, atol=1e-14)
    tau0 = np.cross(np.array([g["l_p"], 0, 0]), out2["Fc"][0])
    assert np.allclose(out2["Tc"][0], tau0, rtol=1e-12, atol=1e-14)
    assert abs(F2[1]) > 0


# ---------------------------------------------------------------- friction / rolling
def test_coulomb_cap_and_zero_friction(oracle_lib):
    ic, p = W.random_cluster(4, n_agg=80, box=5.0)
    agg = oracle_lib.build_aggregates(ic.counts, ic.pos, ic.radius, ic.density)
    rng = np.random.default_rng(1)
    n = ic.n_sph
    vel = rng.standard_normal((n, 3))
    w = rng.standard_normal((n, 3))
    for mu in (0.0, 0.3):
        q = p.replace(mu_s=mu, mu_r=0.0, mu_t=0.0)
        out = oracle_lib.contacts(ic.pos, vel, w, ic.radius, agg["agg_of"], q)
        for (i, j), x in zip(out["pairs"], out["x"]):
            d = ic.pos[j] - ic.pos[i]
            nhat = d / np.linalg.norm(d)
            # reconstruct this pair alone
            sub = oracle_lib.contacts(ic.pos[[i, j]], vel[[i, j]], w[[i, j]], ic.radius[[i, j]],
                                      np.array([0, 1], np.int32), q)
            F = sub["Fc"][0]
            FN = np.dot(F, nhat) * nhat
            FT = F - FN
            if mu == 0.0:
                assert np.linalg.norm(FT) <= 1e-12 * np.linalg.norm(F) + 1e-300
            else:
                assert np.linalg.norm(FT) <= mu * np.linalg.norm(FN) * (1 + 1e-12)


def test_sliding_reaches_cap_and_sticking_does_not(oracle_lib):
    """Overlapping pair with a tangential velocity: fast slip saturates at mu_s|F_N|,
    slow slip stays below it (spring k_t S + dashpot below the cap)."""
    pos = np.array([[0, 0, 0], [1.99, 0, 0]], float)
    ao = np.array([0, 1], np.int32)
    for v, expect_cap in ((10.0, True), (1e-6, False)):
        vel = np.array([[0, 0, 0], [0, v, 0]], float)
        p = free_params(kn=1e4, kt=1e3, ct=0.0, mu_s=0.5, dt=0.01)
        out = oracle_lib.contacts(pos, vel, np.zeros((2, 3)), np.ones(2), ao, p)
        F = out["Fc"][0]
        FN, FT = abs(F[0]), math.hypot(F[1], F[2])
        assert FN == pytest.approx(1e4 * 0.01, rel=1e-12)
        if expect_cap:
            assert FT == pytest.approx(0.5 * FN, rel=1e-12)
        else:
            assert FT == pytest.approx(1e3 * v * 0.01, rel=1e-9)
            assert FT < 0.5 * FN


def test_rolling_couple_law(oracle_lib):
    """Normal-only contact (no tangential motion): tau_i is the rolling couple alone.
    |M| = mu_r |F_N| R_red above the regularisation rate, linear in w below it,
    opposite to the relative spin, zero when mu_r = 0."""
    pos = np.array([[0, 0, 0], [2.9, 0, 0]], float)
    rad = np.array([1.0, 2.0])
    ao = np.array([0, 1], np.int32)
    Rred = 2.0 / 3.0
    FN = 1e3 * 0.1
    for wz, regime in ((1.0, "cap"), (1e-4, "lin")):
        w = np.array([[0, 0, wz], [0, 0, 0]], float)
        p = free_params(kn=1e3, mu_r=0.2, w0=1e-2)
        # spin about z makes a tangential contact-point velocity; remove it with mu_s=0
        out = oracle_lib.contacts(pos, np.zeros((2, 3)), w, rad, ao, p)
        M = out["Tc"][0]
        if regime == "cap":
            assert M[2] == pytest.approx(-0.2 * FN * Rred, rel=1e-12)
        else:
            assert M[2] == pytest.approx(-0.2 * FN * Rred * wz / 1e-2, rel=1e-12)
        assert out["Tc"][1][2] == pytest.approx(-M[2], rel=1e-12)
    w = np.array([[0, 0, 1.0], [0, 0, 0]], float)
    out = oracle_lib.contacts(pos, np.zeros((2, 3)), w, rad, ao, free_params(kn=1e3, mu_r=0.0))
    assert np.max(np.abs(out["Tc"])) == 0.0


def test_twisting_couple_law(oracle_lib):
    pos = np.array([[0, 0, 0], [1.95, 0, 0]], float)
    ao = np.array([0, 1], np.int32)
    w = np.array([[0.5, 0, 0], [-0.5, 0, 0]], float)
    p = free_params(kn=2e3, mu_t=0.3, w0=1e-3)
    out = oracle_lib.contacts(pos, np.zeros((2, 3)), w, np.ones(2), ao, p)
    FN = 2e3 * 0.05
    assert out["Tc"][0][0] == pytest.approx(-0.3 * FN * 0.5, rel=1e-12)
    assert out["Tc"][1][0] == pytest.approx(+0.3 * FN * 0.5, rel=1e-12)


# ---------------------------------------------------------------- tangential history
# Sec. 2.1: the tangential displacement of a contact is tracked for as long as the
# two particles stay in contact.  These pins feed the history returned by one
# contact evaluation into the next one, as the step does.
def _hist(n, entries, hcap=None):
    """History arrays with the given (owner, partner, S) entries, in list order."""
    import oracle
    hcap = hcap or oracle.HCAP
    hn = np.zeros(n, np.int32)
    hp = np.zeros(n * hcap, np.int32)
    hS = np.zeros(n * hcap * 3)
    for i, j, S in entries:
        k = i * hcap + hn[i]
        hp[k] = j
        hS[3 * k:3 * k + 3] = S
        hn[i] += 1
    return hn, hp, hS


def _hist_entries(hist, i, hcap=None):
    import oracle
    hcap = hcap or oracle.HCAP
    hn, hp, hS = hist
    return [(int(hp[i * hcap + t]), hS[3 * (i * hcap + t):3 * (i * hcap + t) + 3].copy())
            for t in range(hn[i])]


def test_history_grows_by_ut_h_until_the_cap(oracle_lib):
    """Fixed overlap x = 0.01 along +x (F_N = kn x = 100), constant tangential velocity
    u = 0.3 along +y, k_t = 1e3, c_t = 5, h = 0.01, mu_s = 0.5 (cap 50).  After the
    k-th evaluation S = k u h exactly and F_T = k_t k u h + c_t u = 3 k + 1.5 on
    sphere 0, below the cap for k <= 16; the 17th evaluation is the first capped one
    (3 * 17 + 1.5 = 52.5 > 50): F_T = 50 and S = (50 - c_t u)/k_t = 0.0485, and it
    stays there while the slip goes on."""
    pos = np.array([[0, 0, 0], [1.99, 0, 0]], float)
    vel = np.array([[0, 0, 0], [0, 0.3, 0]], float)
    ao = np.array([0, 1], np.int32)
    p = free_params(kn=1e4, kt=1e3, ct=5.0, mu_s=0.5, dt=0.01)
    hist = None
    for k in range(1, 21):
        out = oracle_lib.contacts(pos, vel, np.zeros((2, 3)), np.ones(2), ao, p, hist=hist)
        hist = out["hist"]
        F0 = out["Fc"][0]
        assert F0[0] == pytest.approx(-100.0, rel=1e-12)
        assert F0[2] == 0.0
        (partner, S), = _hist_entries(hist, 0)
        assert partner == 1
        if k <= 16:
            assert S[1] == pytest.approx(k * 0.003, rel=1e-12)
            assert F0[1] == pytest.approx(3.0 * k + 1.5, rel=1e-12)
        else:
            assert S[1] == pytest.approx(0.0485, rel=1e-12)
            assert F0[1] == pytest.approx(50.0, rel=1e-12)
        assert S[0] == 0.0 and S[2] == 0.0
        # the partner feels the opposite force (Newton's third law)
        assert np.array_equal(out["Fc"][1], -F0)


@pytest.mark.parametrize("axis", ["z", "y"])
def test_history_follows_a_rotating_normal(oracle_lib, axis):
    """At rest, a stored S = (0, s0, 0) on a contact whose normal turns: S is projected
    on the new tangent plane and rescaled to |S_prev|.  Turning the pair about z by
    10 degrees per evaluation carries S rigidly with it, S = s0 (-sin t, cos t, 0) after
    a total turn t (the projection s0 cos(10 deg) (-sin t, cos t, 0) rescaled to s0); turning
    it about y (S along the axis) leaves S unchanged.  F_T = k_t S (no slip velocity,
    below the cap)."""
    s0, kt = 0.01, 1e3
    p = free_params(kn=1e4, kt=kt, ct=0.0, mu_s=0.5)
    ao = np.array([0, 1], np.int32)
    hist = _hist(2, [(0, 1, (0.0, s0, 0.0))])
    step = math.radians(10.0)
    for m in range(1, 9):
        t = m * step
        if axis == "z":
            nrm = np.array([math.cos(t), math.sin(t), 0.0])
            S_expect = s0 * np.array([-math.sin(t), math.cos(t), 0.0])
        else:
            nrm = np.array([math.cos(t), 0.0, -math.sin(t)])
            S_expect = np.array([0.0, s0, 0.0])
        pos = np.array([[0, 0, 0], 1.99 * nrm])
        out = oracle_lib.contacts(pos, np.zeros((2, 3)), np.zeros((2, 3)), np.ones(2), ao, p,
                                  hist=hist)
        hist = out["hist"]
        (partner, S), = _hist_entries(hist, 0)
        assert partner == 1
        assert np.allclose(S, S_expect, rtol=0, atol=1e-15)
        assert np.linalg.norm(S) == pytest.approx(s0, rel=1e-14)
        assert abs(np.dot(S, nrm)) < 1e-16
        F0 = out["Fc"][0]
        FT = F0 - np.dot(F0, nrm) * nrm
        assert np.allclose(FT, kt * S_expect, rtol=0, atol=1e-11)
        assert np.dot(F0, nrm) == pytest.approx(-100.0, rel=1e-12)


def test_history_found_by_partner_not_by_slot(oracle_lib):
    """Sphere 0 touches sphere 1 (normal +x, overlap 0.01) and sphere 2 (normal +y,
    overlap 0.02).  Its stored list holds partner 2 first, partner 1 second and a stale
    partner 3 that no longer touches it.  Each contact must take its own S: sphere 1
    feels +kn 0.01 x - k_t S_1 and sphere 2 feels +kn 0.02 y - k_t S_2 (at rest, S
    already tangent, below the cap).  The new list is in ascending partner order and
    drops partner 3."""
    kn, kt = 1e4, 1e3
    p = free_params(kn=kn, kt=kt, ct=0.0, mu_s=0.9)
    pos = np.array([[0, 0, 0], [1.99, 0, 0], [0, 1.98, 0], [0, 0, -5.0]], float)
    ao = np.array([0, 1, 2, 3], np.int32)
    S1 = np.array([0.0, 0.01, 0.005])
    S2 = np.array([0.02, 0.0, -0.004])
    hist = _hist(4, [(0, 2, S2), (0, 1, S1), (0, 3, (0.0, 0.0, 0.03))])
    out = oracle_lib.contacts(pos, np.zeros((4, 3)), np.zeros((4, 3)), np.ones(4), ao, p,
                              hist=hist)
    assert out["pairs"].tolist() == [[0, 1], [0, 2]]
    F1 = np.array([kn * 0.01, 0, 0]) - kt * S1
    F2 = np.array([0, kn * 0.02, 0]) - kt * S2
    assert np.allclose(out["Fc"][1], F1, rtol=1e-12, atol=1e-12)
    assert np.allclose(out["Fc"][2], F2, rtol=1e-12, atol=1e-12)
    assert np.allclose(out["Fc"][0], -(F1 + F2), rtol=1e-12, atol=1e-12)
    assert np.array_equal(out["Fc"][3], np.zeros(3))
    ent = _hist_entries(out["hist"], 0)
    assert [e[0] for e in ent] == [1, 2]
    assert np.allclose(ent[0][1], S1, rtol=1e-14, atol=0)
    assert np.allclose(ent[1][1], S2, rtol=1e-14, atol=0)


# ---------------------------------------------------------------- Eq. pred-vel spin
def test_predicted_velocity_uses_the_full_step_spin(oracle_lib):
    """Golden (hand-worked step): a dumbbell spinning about a principal axis with a
    stored torque.  The spheres' predicted velocities and spins of the step carry
    w_{n+1} = drifted spin + h/2 I^-1 N_n (0.55), not w_n (0.5) or the drifted 0.525;
    positions follow the RK4 rotation of the quaternion."""
    g = read_golden("spinning_dumbbell_step.txt")
    ic = W.PileIC(counts=np.array([2], np.int32),
                  pos=np.array([[1.0, 0, 0], [-1.0, 0, 0]]), radius=np.ones(2),
                  density=np.full(2, g["density"]), vel=np.zeros((1, 3)),
                  omega=np.array([[0.0, 0.0, g["spin_n"]]]))
    pile = oracle_lib.Pile(ic, free_params(dt=g["h"]))
    assert np.allclose(pile.m, 1.0, rtol=1e-14)
    assert pile.I[0][2, 2] == pytest.approx(2.8, rel=1e-14)
    pile.acc[0] = (g["accel_x"], 0.0, 0.0)
    pile.torque[0] = (0.0, 0.0, g["torque_z"])
    pile.step()
    t = 1e-12
    assert pile.sph_w[0] == pytest.approx([0, 0, g["spin_pred"]], rel=t, abs=t)
    assert pile.sph_w[1] == pytest.approx([0, 0, g["spin_pred"]], rel=t, abs=t)
    assert pile.sph_pos[0] == pytest.approx([g["pos0_x"], g["pos0_y"], 0], rel=t, abs=t)
    assert pile.sph_vel[0] == pytest.approx([g["vel0_x"], g["vel0_y"], 0], rel=t, abs=t)
    assert pile.sph_vel[1] == pytest.approx([g["vel1_x"], g["vel1_y"], 0], rel=t, abs=t)
    assert pile.r[0] == pytest.approx([g["com_x"], 0, 0], rel=t, abs=t)
    assert pile.v[0] == pytest.approx([g["v_half_x"], 0, 0], rel=t, abs=t)
    assert pile.wb[0] == pytest.approx([0, 0, g["spin_half"]], rel=t, abs=t)
    assert pile.q[0] == pytest.approx(
        [math.sqrt(0.5 * (1 + g["cos_t"])), 0, 0, math.sqrt(0.5 * (1 - g["cos_t"]))], rel=t, abs=t)
    assert np.array_equal(pile.torque[0], np.zeros(3))


def test_spin_and_damping_enter_an_oblique_contact(oracle_lib):
    """One step of two free spheres in contact, sphere 0 spinning about z with a stored
    torque, normal and tangential dashpots on: the tangential force is
    c_t u_t + k_t u_t h with the contact-point velocity u_t = -w_{n+1} l_0 y of the
    full-step spin (hand values: l_0 = 0.995 for equal radii at |d| = 1.99)."""
    rho = 3.0 / (4.0 * math.pi)                      # unit sphere mass
    ic = W.PileIC(counts=np.array([1, 1], np.int32),
                  pos=np.array([[0.0, 0, 0], [1.99, 0, 0]]), radius=np.ones(2),
                  density=np.full(2, rho), vel=np.zeros((2, 3)),
                  omega=np.array([[0.0, 0.0, 0.4], [0.0, 0.0, 0.0]]))
    h, kn, kt, cn, ct = 0.01, 1e4, 1e3, 3.0, 2.0
    pile = oracle_lib.Pile(ic, free_params(dt=h, kn=kn, kt=kt, cn=cn, ct=ct, mu_s=10.0))
    # sphere inertia 2/5 m s^2 = 0.4, stored torque 0.2 about z: w_{n+1} = 0.4 + h * 0.5
    pile.torque[0] = (0.0, 0.0, 0.2)
    pile.step()
    w1 = 0.4 + h * 0.2 / 0.4
    assert pile.sph_w[0][2] == pytest.approx(w1, rel=1e-13)
    # the spheres do not move during the drift (no stored accelerations); a free
    # sphere's orientation turns but its centre stays
    assert np.allclose(pile.sph_pos, ic.pos, rtol=0, atol=1e-15)
    l0 = 0.995
    ut_y = -w1 * l0                                  # u = v_1 - (w x l0 x) = -w l0 y
    FT = ct * ut_y + kt * ut_y * h
    F0 = pile.Fc[0]
    assert F0[0] == pytest.approx(-kn * 0.01, rel=1e-12)
    assert F0[1] == pytest.approx(FT, rel=1e-12)
    assert pile.Tc[0][2] == pytest.approx(l0 * FT, rel=1e-12)


# ---------------------------------------------------------------- pin 4
def restitution_run(oracle_lib, e_target, steps_per_contact):
    ic = W.tiny_pair(gap=1e-3, v=0.02)
    m = W.sphere_mass(1.0, 2500.0)
    mu = 0.5 * m
    kn = 1e4
    cn = W.damping_for_restitution(e_target, mu, kn)
    tc = W.contact_time(kn, cn, mu)
    p = free_params(kn=kn, cn=cn, kt=kn * 2 / 7, dt=tc / steps_per_contact)
    pile = oracle_lib.Pile(ic, p)
    v_in = pile.v[1, 0] - pile.v[0, 0]
    steps, touching, t_contact = 0, False, 0
    while steps < 100000:
        pile.step()
        steps += 1
        x = 2.0 - np.linalg.norm(pile.r[1] - pile.r[0])
        if x > 0:
            touching = True
            t_contact += 1
        elif touching:
            break
    v_out = pile.v[1, 0] - pile.v[0, 0]
    return -v_out / v_in, t_contact * p.dt, tc


def test_restitution_closed_form(oracle_lib):
    """Head-on spring-dashpot collision of two free spheres: the coefficient of
    restitution converges to exp(-pi zeta / sqrt(1 - zeta^2)) (damped oscillator),
    first order in h; the contact lasts pi / omega_d."""
    for e in (0.5, 0.8):
        e50, t50, tc = restitution_run(oracle_lib, e, 50)
        e100, _, _ = restitution_run(oracle_lib, e, 100)
        err50, err100 = abs(e50 - e), abs(e100 - e)
        assert err50 < 0.01 * e
        assert err100 < 0.65 * err50          # converges (first order: ratio ~ 0.5)
        assert t50 == pytest.approx(tc, rel=0.05)


# ---------------------------------------------------------------- pin 5
def test_body_offsets_bit_exact_and_rigid(oracle_lib):
    ic, p = W.config1(0, n_agg=40, ball=14.0)
    p = p.replace(dt=p.dt)
    pile = oracle_lib.Pile(ic, p)
    b0 = pile.b.copy()
    d0 = {a: np.linalg.norm(pile.b[pile.first[a]] - pile.b[pile.first[a] + 1]) for a in range(pile.A)}
    pile.step(1000)
    assert np.array_equal(pile.b, b0)
    for a in range(pile.A):
        i = pile.first[a]
        d = np.linalg.norm(pile.sph_pos[i] - pile.sph_pos[i + 1])
        assert d == pytest.approx(d0[a], rel=1e-12)
        assert np.linalg.norm(pile.q[a]) == pytest.approx(1.0, abs=1e-14)


# ---------------------------------------------------------------- pin 6
def torque_free_body(oracle_lib, wb0, h, steps, shape="dumbbell"):
    ic = W.assemble([shape], [1.0], np.zeros((1, 3)), np.eye(3)[None], 2500.0)
    ic.omega = np.array([wb0], float)
    p = free_params(dt=h)
    pile = oracle_lib.Pile(ic, p)
    out = []
    for _ in range(steps):
        pile.step()
        out.append(pile.wb[0].copy())
    return pile, np.array(out)


def test_symmetric_top_precession(oracle_lib):
    """Torque-free symmetric top (dumbbell: I1 = I2 != I3 about the x axis here):
    w_axis constant, w_perp rotates at (I_axis - I_perp) w_axis / I_perp in the body."""
    w = np.array([0.02, 0.01, 0.0])
    h = 0.5
    pile, traj = torque_free_body(oracle_lib, w, h, 400)
    I = pile.I[0]
    Ia, Ip = I[0, 0], I[1, 1]
    assert I[2, 2] == pytest.approx(Ip, rel=1e-14)
    Om = (Ia - Ip) * w[0] / Ip
    t = h * np.arange(1, 401)
    # Euler: I_p dw_y/dt = (I_p - I_a) w_x w_z, I_p dw_z/dt = (I_a - I_p) w_x w_y, so
    # w_y + i w_z = (w_y0 + i w_z0) exp(+i Om t)
    wy = w[1] * np.cos(Om * t)
    wz = w[1] * np.sin(Om * t)
    assert np.max(np.abs(traj[:, 0] - w[0])) < 1e-15
    assert np.max(np.abs(traj[:, 1] - wy)) < 1e-9 * abs(w[1])
    assert np.max(np.abs(traj[:, 2] - wz)) < 1e-9 * abs(w[1])


def test_torque_free_rotor_invariants_and_rk4_order(oracle_lib):
    """Asymmetric body (square): energy and |L| drift < 1e-10 over 1e4 steps; the
    RK4 error against a fine reference falls ~16x when h halves."""
    w = np.array([0.03, 0.02, 0.05])
    pile, _ = torque_free_body(oracle_lib, w, 0.2, 10000, shape="square")
    I = pile.I[0]
    E0 = 0.5 * w @ I @ w
    L0 = np.linalg.norm(I @ w)
    wb = pile.wb[0]
    assert 0.5 * wb @ I @ wb == pytest.approx(E0, rel=1e-10)
    assert np.linalg.norm(I @ wb) == pytest.approx(L0, rel=1e-10)
    # order check on a short interval
    ref = torque_free_body(oracle_lib, w, 0.25 / 16, 16 * 40, shape="square")[1][-1]
    e1 = np.linalg.norm(torque_free_body(oracle_lib, w, 0.25, 40, shape="square")[1][-1] - ref)
    e2 = np.linalg.norm(torque_free_body(oracle_lib, w, 0.125, 80, shape="square")[1][-1] - ref)
    assert e1 > 0
    assert 10.0 < e1 / e2 < 22.0


# ---------------------------------------------------------------- pin 7
def elastic_collision(oracle_lib, h_div, oblique):
    if oblique:
        # two dumbbells, one offset so the contact is off the line of centres
        R1, R2 = np.eye(3), W.random_rotations(np.random.default_rng(2), 1)[0]
        ic = W.assemble(["dumbbell", "dumbbell"], [1.0, 1.0],
                        np.array([[0, 0, 0], [4.5, 0.8, 0.3]]), np.stack([R1, R2]), 2500.0)
        ic.vel = np.array([[0.01, 0, 0], [-0.01, 0, 0]])
        ic.omega = np.array([[0, 0, 0.002], [0.001, 0, 0]])
    else:
        ic = W.tiny_pair(gap=1e-3, v=0.02)
    m = W.sphere_mass(1.0, 2500.0)
    kn = 1e4
    tc = W.contact_time(kn, 0.0, m)
    p = free_params(kn=kn, kt=kn * 2 / 7, dt=tc / (50 * h_div))
    pile = oracle_lib.Pile(ic, p)
    E0, P0, L0 = pile.kinetic_energy(), pile.linear_momentum(), pile.angular_momentum()
    touched, steps = False, 0
    while steps < 200000:
        pile.step()
        steps += 1
        if pile.FA_c.any():
            touched = True
        elif touched:
            break
    assert touched
    return pile, E0, P0, L0


@pytest.mark.parametrize("oblique", [False, True])
def test_elastic_collision_conservation(oracle_lib, oblique):
    """Undamped, frictionless, no gravity: P and L conserved to round-off; kinetic
    energy after separation matches the initial value, error shrinking with h."""
    errs = []
    for h_div in (1, 2):
        pile, E0, P0, L0 = elastic_collision(oracle_lib, h_div, oblique)
        P1, L1 = pile.linear_momentum(), pile.angular_momentum()
        pscale = np.sum(pile.M) * 0.02
        assert np.max(np.abs(P1 - P0)) < 1e-12 * pscale
        assert np.max(np.abs(L1 - L0)) < 1e-10 * (pscale * 5.0 + np.max(np.abs(L0)))
        errs.append(abs(pile.kinetic_energy() - E0) / E0)
    assert errs[0] < 2e-2
    assert errs[1] < 0.7 * errs[0]


# ---------------------------------------------------------------- pin 8
def test_yorp_angular_momentum_increment(oracle_lib):
    """Isolated pile, no contacts or gravity: each step adds exactly I_pile dw to L,
    with I_pile the pile's inertia tensor about its COM (rigid-body textbook sum)."""
    ic, p = W.config1(1, n_agg=30, ball=12.0)
    dw = np.array([1e-4, -2e-4, 3e-4])
    p = p.replace(G=0.0, spin_inc=tuple(dw))
    pile = oracle_lib.Pile(ic, p)
    pile.step(3)
    M = pile.M
    com = np.average(pile.r, axis=0, weights=M)
    L0 = pile.angular_momentum(com)
    pile.step()
    com1 = np.average(pile.r, axis=0, weights=M)
    L1 = pile.angular_momentum(com1)
    # inertia of the pile about its COM at the time of the increment
    Ip = np.zeros((3, 3))
    for a in range(pile.A):
        R = oracle_lib.rotmat(pile.q[a])
        d = pile.r[a] - com1
        Ip += R @ pile.I[a] @ R.T + M[a] * (d @ d * np.eye(3) - np.outer(d, d))
    assert np.allclose(L1 - L0, Ip @ dw, rtol=1e-9, atol=1e-12 * np.linalg.norm(Ip @ dw))


# ---------------------------------------------------------------- aggregates
def test_aggregate_mass_com_inertia(oracle_lib):
    """Eq. agg_mass / agg_position, and the inertia of a dumbbell of touching spheres:
    I_axis = 2 (2/5 m s^2), I_perp = 2 (2/5 m s^2 + m s^2)."""
    pos = np.array([[1.0, 2.0, 3.0], [3.0, 2.0, 3.0], [10, 10, 10]])
    rad = np.array([1.0, 1.0, 0.5])
    rho = np.array([2000.0, 2000.0, 3000.0])
    out = oracle_lib.build_aggregates(np.array([2, 1], np.int32), pos, rad, rho)
    m = 2000 * 4 / 3 * math.pi
    assert out["M"][0] == pytest.approx(2 * m, rel=1e-15)
    assert np.allclose(out["com"][0], [2.0, 2.0, 3.0], rtol=1e-15)
    I = out["I"][0]
    assert I[0, 0] == pytest.approx(2 * 0.4 * m, rel=1e-14)
    assert I[1, 1] == pytest.approx(2 * (0.4 * m + m), rel=1e-14)
    assert np.allclose(I @ out["Iinv"][0], np.eye(3), atol=1e-14)
    # unequal-density spheres weight the COM
    out2 = oracle_lib.build_aggregates(np.array([2], np.int32), pos[:2], rad[:2],
                                       np.array([1000.0, 3000.0]))
    assert out2["com"][0][0] == pytest.approx(1.0 + 2.0 * 3 / 4, rel=1e-15)


def test_rotation_matrix_is_proper(oracle_lib):
    rng = np.random.default_rng(0)
    for _ in range(20):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        R = oracle_lib.rotmat(q)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
        # rotation by angle t about axis u: q = (cos t/2, sin t/2 u)
    t = 0.7
    R = oracle_lib.rotmat(np.array([math.cos(t / 2), 0, 0, math.sin(t / 2)]))
    assert np.allclose(R @ [1, 0, 0], [math.cos(t), math.sin(t), 0], atol=1e-15)


def test_gravity_two_aggregate_tidal_torque_sign(oracle_lib):
    """A dumbbell tilted 45 degrees to the line to a distant mass feels a gravity-gradient
    torque that turns its axis toward that line: N = 3 G M_p / d^3 (I_perp - I_axis) ..."""
    s, rho = 1.0, 2500.0
    m = W.sphere_mass(s, rho)
    d = 500.0
    c45 = math.sqrt(0.5)
    pos = np.array([[c45, c45, 0], [-c45, -c45, 0], [d, 0, 0]]) * np.array([[s], [s], [1.0]])
    big_s = 20.0
    rad = np.array([s, s, big_s])
    dens = np.array([rho, rho, rho])
    agg = oracle_lib.build_aggregates(np.array([2, 1], np.int32), pos, rad, dens)
    F = oracle_lib.gravity(pos, agg["m"], agg["agg_of"], W.G_SI, 0.0)
    N = np.cross(pos[:2] - agg["com"][0], F[:2]).sum(0)
    Mp = agg["m"][2]
    # quadrupole limit: N_z = -3 G Mp / d^3 * (sum m b_x b_y) = -3 G Mp m s^2 / d^3
    expect = -3 * W.G_SI * Mp * m * s * s / d ** 3
    assert N[2] == pytest.approx(expect, rel=1e-2)


def test_free_sphere_has_zero_offset_and_no_gravity_torque(oracle_lib):
    """A one-sphere aggregate (a free sphere) has its COM exactly at the sphere:
    zero body offset, so gravity and the planet exert no torque on it."""
    import oracle as O
    from paper_2311_11322_gb300 import workloads as W
    ic, p = W.random_cluster(2, n_agg=30, shapes=("single",), box=3.0, precision=0)
    ic.pos = ic.pos + 12345.678       # far from the origin: rounding would show
    pile = O.Pile(ic, p.replace(G=W.G_SI * 1e6), want_scales=True)
    pile.step()
    assert np.all(pile.b == 0.0)
    assert np.all(pile.NA_g == 0.0) and np.all(pile.NA_e == 0.0)


# ---------------------------------------------------------------- adaptive RK5 rotation (Sec. 2.2.1)
def _square_body():
    ic = W.assemble(["square"], [1.0], np.zeros((1, 3)), np.eye(3)[None], 2500.0)
    import oracle as O
    agg = O.build_aggregates(ic.counts, ic.pos, ic.radius, ic.density)
    return agg["I"].reshape(3, 3), agg["Iinv"].reshape(3, 3)


def _run_adaptive(oracle_lib, I, Iinv, w0, h, n, tol):
    q, wb, subs = np.array([1.0, 0, 0, 0]), np.array(w0, float), 0
    for _ in range(n):
        q, wb, k = oracle_lib.rotate_adaptive(q, wb, I, Iinv, h, tol)
        subs += k
    return q, wb, subs


def test_adaptive_rotation_fifth_order_and_tolerance(oracle_lib):
    """The embedded RK5(4) of the adaptive integrator: with the tolerance out of
    reach every step is one fifth-order step, and its error against a fine
    reference falls ~32x when h halves; with a tolerance, a coarse step is cut
    into substeps and the error stays near the tolerance."""
    I, Iinv = _square_body()
    w0 = [0.3, 0.2, 0.5]           # |w| h ~ 0.3 at h = 0.5: a hard step for RK4
    T = 8.0
    ref = _run_adaptive(oracle_lib, I, Iinv, w0, T / 2048, 2048, 1e30)[1]
    e = []
    for n in (64, 128, 256):
        q, wb, subs = _run_adaptive(oracle_lib, I, Iinv, w0, T / n, n, 1e30)
        assert subs == n
        e.append(np.linalg.norm(wb - ref))
    assert 24.0 < e[0] / e[1] < 40.0 and 24.0 < e[1] / e[2] < 40.0
    q, wb, subs = _run_adaptive(oracle_lib, I, Iinv, w0, 0.5, 16, 1e-10)
    assert subs > 16
    assert np.linalg.norm(wb - ref) < 1e-8 * np.linalg.norm(ref)


def test_adaptive_rotation_conserves_and_beats_rk4(oracle_lib):
    """Torque-free asymmetric body at a coarse step: the adaptive scheme keeps
    energy and |L| to ~1e-9 where one RK4 step per h drifts by orders more; the
    symmetric top still follows its closed-form precession."""
    I, Iinv = _square_body()
    w0 = np.array([0.3, 0.2, 0.5])
    E0, L0 = 0.5 * w0 @ I @ w0, np.linalg.norm(I @ w0)
    q, wb, _ = _run_adaptive(oracle_lib, I, Iinv, w0, 0.5, 400, 1e-11)
    dE_ad = abs(0.5 * wb @ I @ wb - E0) / E0
    dL_ad = abs(np.linalg.norm(I @ wb) - L0) / L0
    q4, wb4 = np.array([1.0, 0, 0, 0]), w0.copy()
    for _ in range(400):
        q4, wb4 = oracle_lib.rotate(q4, wb4, I, Iinv, np.zeros(3), 0.5)
    dE_rk4 = abs(0.5 * wb4 @ I @ wb4 - E0) / E0
    assert dE_ad < 1e-9 and dL_ad < 1e-9
    assert dE_rk4 > 100 * dE_ad
    # symmetric top (dumbbell about x): closed form
    ic = W.assemble(["dumbbell"], [1.0], np.zeros((1, 3)), np.eye(3)[None], 2500.0)
    import oracle as O
    agg = O.build_aggregates(ic.counts, ic.pos, ic.radius, ic.density)
    Id, Idi = agg["I"].reshape(3, 3), agg["Iinv"].reshape(3, 3)
    w = np.array([0.4, 0.1, 0.0])
    q, wb, _ = _run_adaptive(oracle_lib, Id, Idi, w, 0.5, 200, 1e-11)
    Ia, Ip = Id[0, 0], Id[1, 1]
    Om = (Ia - Ip) * w[0] / Ip
    t = 0.5 * 200
    assert wb[0] == pytest.approx(w[0], abs=1e-14)
    assert wb[1] == pytest.approx(w[1] * np.cos(Om * t), abs=1e-8 * w[1])
    assert wb[2] == pytest.approx(w[1] * np.sin(Om * t), abs=1e-8 * w[1])


# ---------------------------------------------------------------- bulk shape and spin (Sec. 4.1, 4.2)
def _free_spheres(pos, s, rho=2500.0):
    import oracle
    n = len(pos)
    return oracle.build_aggregates(np.ones(n, np.int32), pos, np.full(n, s), np.full(n, rho))


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1)[:, None]


def test_bulk_single_sphere_closed_form(oracle_lib):
    """One sphere: the equal-moment ellipsoid is the sphere itself, so the
    semi-axes and bulk radius are its radius, the bulk density its density,
    and the nominal critical period is sqrt(3 pi / (G rho)) (Sec. 4.1)."""
    import oracle
    s, rho, G = 3.0, 2000.0, W.G_SI
    ag = _free_spheres(np.array([[1.0, -2.0, 5.0]]), s, rho)
    b = oracle.bulk(ag["M"], ag["I"], ag["com"], np.zeros((1, 3)), np.array([[1.0, 0, 0, 0]]),
                    np.zeros((1, 3)), G)
    assert np.allclose(b["axes"], s, rtol=1e-13)
    assert b["radius"] == pytest.approx(s, rel=1e-13)
    assert b["density"] == pytest.approx(rho, rel=1e-13)
    assert b["p_crit"] == pytest.approx(math.sqrt(3 * math.pi / (G * rho)), rel=1e-13)
    assert b["period"] == math.inf and b["planet_dist"] == 0.0


@pytest.mark.parametrize("seed", [0, 1])
def test_bulk_six_sphere_cross_closed_form(oracle_lib, seed):
    """Six equal spheres (radius s) at +-a x, +-b y, +-c z: the principal
    moments are 2 m (b^2 + c^2) + 12/5 m s^2 and cyclic, so the semi-axes are
    sqrt(5/3 a^2 + s^2) etc. (worked by hand); a rigid rotation of the whole
    set changes neither them nor the moments."""
    import oracle
    a, b, c, s = 9.0, 5.0, 2.0, 0.5
    pts = np.array([[a, 0, 0], [-a, 0, 0], [0, b, 0], [0, -b, 0], [0, 0, c], [0, 0, -c]])
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.standard_normal((3, 3)))[0]
    Q *= np.sign(np.linalg.det(Q))
    shift = rng.uniform(-100, 100, 3)
    want = np.sqrt(5.0 / 3.0 * np.array([a, b, c]) ** 2 + s * s)
    m = 2500.0 * 4.0 / 3.0 * math.pi * s ** 3
    mom = np.sort([2 * m * (b * b + c * c), 2 * m * (a * a + c * c), 2 * m * (a * a + b * b)]) + 12 / 5 * m * s * s
    for P in (pts, pts @ Q.T + shift):
        ag = _free_spheres(P, s)
        q = _unit_quats(rng, 6)        # a sphere's orientation changes nothing
        out = oracle.bulk(ag["M"], ag["I"], ag["com"], np.zeros((6, 3)), q, np.zeros((6, 3)), 0.0)
        assert np.allclose(out["axes"], want, rtol=1e-12)
        assert np.allclose(out["moments"], mom, rtol=1e-12)
        assert np.allclose(out["com"], P.mean(0), atol=1e-12)
        assert out["p_crit"] == math.inf


def _rotated_pile(seed):
    import oracle
    ic, _ = W.random_cluster(seed, n_agg=30, box=8.0)
    ag = oracle.build_aggregates(ic.counts, ic.pos, ic.radius, ic.density)
    rng = np.random.default_rng(seed + 100)
    return ic, ag, _unit_quats(rng, len(ic.counts))


@pytest.mark.parametrize("seed", [3, 4])
def test_bulk_inertia_equals_sphere_level_sum(oracle_lib, seed):
    """The pile inertia built from rotated aggregate tensors equals the brute
    sum over spheres (positions r_A + R b_i, own moments 2/5 m s^2): a
    transposed rotation or a missing parallel-axis term fails this."""
    import oracle
    ic, ag, q = _rotated_pile(seed)
    A = len(ic.counts)
    out = oracle.bulk(ag["M"], ag["I"], ag["com"], np.zeros((A, 3)), q, np.zeros((A, 3)), 0.0)
    x = np.array([ag["com"][ag["agg_of"][i]] + oracle.rotmat(q[ag["agg_of"][i]]) @ ag["b"][i]
                  for i in range(len(ic.radius))])
    m = ag["m"]
    c = (m[:, None] * x).sum(0) / m.sum()
    d = x - c
    I = np.zeros((3, 3))
    for i in range(len(m)):
        I += m[i] * (d[i] @ d[i] * np.eye(3) - np.outer(d[i], d[i])) + 0.4 * m[i] * ic.radius[i] ** 2 * np.eye(3)
    assert np.allclose(out["moments"], np.linalg.eigvalsh(I), rtol=1e-11)
    assert np.allclose(out["com"], c, atol=1e-10)


@pytest.mark.parametrize("seed", [5, 6])
def test_bulk_rigid_rotation_recovers_spin(oracle_lib, seed):
    """Every aggregate moving with one rigid rotation Omega (v_A = V + Omega x
    (r_A - c), spin Omega): the pile spin is Omega, the period 2 pi / |Omega|,
    and L = I Omega."""
    import oracle
    ic, ag, q = _rotated_pile(seed)
    A = len(ic.counts)
    rng = np.random.default_rng(seed)
    Om = rng.standard_normal(3) * 1e-3
    V = rng.standard_normal(3)
    c = (ag["M"][:, None] * ag["com"]).sum(0) / ag["M"].sum()
    v = V + np.cross(Om, ag["com"] - c)
    wb = np.array([oracle.rotmat(q[a]).T @ Om for a in range(A)])
    out = oracle.bulk(ag["M"], ag["I"], ag["com"], v, q, wb, 0.0)
    assert np.allclose(out["spin"], Om, rtol=1e-10, atol=1e-16)
    assert out["period"] == pytest.approx(2 * math.pi / np.linalg.norm(Om), rel=1e-10)
    assert np.allclose(out["vcom"], V, atol=1e-12)


def test_bulk_uniform_ball_and_roche(oracle_lib):
    """20,000 small spheres uniform in a ball of radius 10: the equal-moment
    ellipsoid is that ball to sampling accuracy (<x^2> = R^2 / 5), so the bulk
    radius is 10 and the bulk density the mass over the ball's volume.  The
    Roche normalisation reduces to 1.26 R for equal densities (Sec. 4.2)."""
    import oracle
    rng = np.random.default_rng(11)
    n, R = 20000, 10.0
    d = rng.standard_normal((n, 3))
    d *= (R * rng.uniform(0, 1, n) ** (1 / 3) / np.linalg.norm(d, axis=1))[:, None]
    ag = _free_spheres(d, 1e-3)
    out = oracle.bulk(ag["M"], ag["I"], ag["com"], np.zeros((n, 3)), np.tile([1.0, 0, 0, 0], (n, 1)),
                      np.zeros((n, 3)), 0.0, planet_pos=np.array([0.0, 0.0, 500.0]))
    assert np.allclose(out["axes"], R, rtol=0.03)
    assert out["radius"] == pytest.approx(R, rel=0.02)
    assert out["density"] == pytest.approx(ag["M"].sum() / (4 / 3 * math.pi * R ** 3), rel=0.06)
    assert out["planet_dist"] == pytest.approx(np.linalg.norm([0, 0, 500.0] - out["com"]), rel=1e-14)
    assert oracle.roche_distance(7.0, 3000.0, 3000.0) == pytest.approx(1.26 * 7.0)
    assert oracle.roche_distance(7.0, 3000.0, 375.0) == pytest.approx(1.26 * 7.0 * 2.0)
