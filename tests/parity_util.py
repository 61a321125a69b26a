"""Helpers that compare the CUDA library with the FP64 oracle.

Error measure.  F_A and N_A are sums of many sphere terms (contact pairs,
gravity pairs, planet) that largely cancel.  A computed sum in any precision
carries an error bounded by (unit round-off) x (sum of the magnitudes of its
terms), so the error of each aggregate result is reported relative to that
sum of magnitudes, which the oracle computes alongside the result
(`scaleF`, `scaleN`).  The tolerances are then statements about the
arithmetic: 1e-5 for the mixed FP32/FP64 path, 1e-9 for the all-FP64 path.
"""
from __future__ import annotations

import numpy as np

TOL = {0: 1e-9, 1: 1e-5}     # precision id -> relative tolerance


def agg_errors(world, pid, pile):
    """Per-aggregate condition-relative errors of F_A and N_A after the last step."""
    F = world.read(pid, "FORCE")
    N = world.read(pid, "TORQUE")
    Fo = pile.FA_c + pile.FA_g + pile.FA_e
    No = pile.NA_c + pile.NA_g + pile.NA_e
    sF = np.maximum(pile.scaleF, 1e-300)
    sN = np.maximum(pile.scaleN, 1e-300)
    eF = np.linalg.norm(F - Fo, axis=1) / sF
    eN = np.linalg.norm(N - No, axis=1) / sN
    return eF, eN


def sphere_errors(world, pid, pile):
    """Per-sphere condition-relative errors of the contact force, contact torque and gravity."""
    Fc = world.read(pid, "SPHERE_FC")
    Tc = world.read(pid, "SPHERE_TC")
    Fg = world.read(pid, "SPHERE_FG")
    sc = np.maximum(pile.sph_Fmc, 1e-300)
    st = np.maximum(pile.sph_Tmc, 1e-300)
    sg = np.maximum(pile.sph_Fmg, 1e-300)
    ec = np.where(pile.sph_Fmc > 0, np.linalg.norm(Fc - pile.Fc, axis=1) / sc,
                  np.linalg.norm(Fc, axis=1))
    et = np.where(pile.sph_Tmc > 0, np.linalg.norm(Tc - pile.Tc, axis=1) / st,
                  np.linalg.norm(Tc, axis=1))
    eg = np.where(pile.sph_Fmg > 0, np.linalg.norm(Fg - pile.Fg, axis=1) / sg,
                  np.linalg.norm(Fg, axis=1))
    return ec, et, eg


def contact_set_check(world, pid, pile, r_ref):
    """Contact pairs with overlap > 1e-6 R must match exactly; pairs closer to
    touching may differ.  Returns (n_strong, n_gpu, mismatches)."""
    gpu_pairs, _ = world.contacts(pid)
    gset = set(gpu_pairs)
    opairs, ox = pile.contact_pairs()
    thr = 1e-6 * r_ref
    oset = {tuple(p) for p in opairs.tolist()}
    strong = {tuple(p) for p, x in zip(opairs.tolist(), ox) if x > thr}
    bad = [p for p in strong if p not in gset]
    for (i, j) in gset - oset:
        d = np.linalg.norm(pile.sph_pos[i] - pile.sph_pos[j])
        x = pile.s[i] + pile.s[j] - d
        if x > thr or pile.agg_of[i] == pile.agg_of[j]:
            bad.append((i, j))
    return len(strong), len(gset), bad


def lockstep(world, pid, pile, steps, tol, r_ref=1.0, check_contacts=True, every=1):
    """Advance both by `steps`, comparing after each (or every `every`) step.
    Returns the worst errors seen."""
    worst = dict(F=0.0, N=0.0, Fc=0.0, Tc=0.0, Fg=0.0, contacts=0)
    for k in range(steps):
        pile.step()
        world.step(1)
        if (k + 1) % every and k + 1 != steps:
            continue
        eF, eN = agg_errors(world, pid, pile)
        ec, et, eg = sphere_errors(world, pid, pile)
        worst["F"] = max(worst["F"], float(eF.max()))
        worst["N"] = max(worst["N"], float(eN.max()))
        worst["Fc"] = max(worst["Fc"], float(ec.max()))
        worst["Tc"] = max(worst["Tc"], float(et.max()))
        worst["Fg"] = max(worst["Fg"], float(eg.max()))
        if check_contacts:
            ns, ng, bad = contact_set_check(world, pid, pile, r_ref)
            assert not bad, f"step {k + 1}: contact sets differ: {bad[:5]}"
            worst["contacts"] = max(worst["contacts"], ns)
        assert worst["F"] <= tol and worst["N"] <= tol, f"step {k + 1}: {worst}"
    return worst


def oracle_contacts_field(pile, K):
    """The oracle's contact history as the CONTACTS layout of dem_read_state:
    per sphere, count then (partner, Sx, Sy, Sz); both spheres of a pair carry S."""
    N = pile.N
    out = np.zeros((N, 1 + 4 * K))
    hc = pile.h_n
    hp = pile.h_partner.reshape(N, -1)
    hS = pile.h_S.reshape(N, -1, 3)
    for i in range(N):
        for t in range(hc[i]):
            j = hp[i, t]
            for a, b in ((i, j), (j, i)):
                n = int(out[a, 0])
                assert n < K, "too many contacts for the GPU history"
                out[a, 1 + 4 * n:5 + 4 * n] = (b, *hS[i, t])
                out[a, 0] = n + 1
    return out


def resync(world, pid, pile, K):
    """Copy the oracle's full state into the GPU pile (oracle -> GPU only)."""
    world.write(pid, "COM", pile.r)
    world.write(pid, "VEL", pile.v)
    world.write(pid, "QUAT", pile.q)
    world.write(pid, "OMEGA_BODY", pile.wb)
    world.write(pid, "ACC", pile.acc)
    world.write(pid, "TORQUE_STORED", pile.torque)
    world.write(pid, "PLANET", pile.planet)
    world.write(pid, "CONTACTS", oracle_contacts_field(pile, K))


def resynced_steps(world, pid, pile, steps, tol, K, r_ref=1.0):
    """Per-step errors from identical states: before each step the GPU pile is
    overwritten with the oracle's state, then both take one step."""
    worst = dict(F=0.0, N=0.0, contacts=0)
    for k in range(steps):
        resync(world, pid, pile, K)
        pile.step()
        world.step(1)
        eF, eN = agg_errors(world, pid, pile)
        worst["F"] = max(worst["F"], float(eF.max()))
        worst["N"] = max(worst["N"], float(eN.max()))
        ns, ng, bad = contact_set_check(world, pid, pile, r_ref)
        assert not bad, f"step {k + 1}: contact sets differ: {bad[:5]}"
        worst["contacts"] = max(worst["contacts"], ns)
        assert worst["F"] <= tol and worst["N"] <= tol, f"step {k + 1}: {worst}"
    return worst


def same_inputs(ic, gold) -> bool:
    """The initial conditions match the stored run's: shape counts exactly,
    position, radius and density sums within 1e-12 relative (a generator run
    on another machine may differ in the last bit)."""
    import hashlib
    if hashlib.sha256(ic.counts.astype(np.int32).tobytes()).hexdigest() != str(gold["counts_sha256"]):
        return False
    pairs = ((ic.pos.sum(0), gold["pos_sum"]), ((ic.pos ** 2).sum(0), gold["pos_sq_sum"]),
             (ic.radius.sum(), gold["radius_sum"]), (ic.density.sum(), gold["density_sum"]))
    return all(np.allclose(a, b, rtol=1e-12, atol=0) for a, b in pairs)


def trajectory_errors(world, pid, gold, steps=None):
    """Step a GPU pile side by side with a stored oracle trajectory (the npz
    written by tests/golden/make_collapse100k_trajectory.py) and return per-step
    errors of the sampled aggregates: condition-relative (error / sum of the
    magnitudes of the summed terms) and |X|-relative (error / |X_oracle|)
    maxima and 99th percentiles of F_A and N_A, and every `pose_every` steps
    the largest COM deviation (m) and quaternion deviation."""
    idx = gold["sample"]
    n = int(steps or gold["F"].shape[0])
    every = int(gold["pose_every"])
    rows = []
    for k in range(n):
        world.step(1)
        F = world.read(pid, "FORCE")[idx]
        N = world.read(pid, "TORQUE")[idx]
        dF = np.linalg.norm(F - gold["F"][k], axis=1)
        dN = np.linalg.norm(N - gold["N"][k], axis=1)
        cF = dF / np.maximum(gold["scaleF"][k], 1e-300)
        cN = dN / np.maximum(gold["scaleN"][k], 1e-300)
        xF = dF / np.maximum(np.linalg.norm(gold["F"][k], axis=1), 1e-300)
        xN = dN / np.maximum(np.linalg.norm(gold["N"][k], axis=1), 1e-300)
        r = {"step": k + 1, "F_cond_max": float(cF.max()), "F_cond_p99": float(np.quantile(cF, 0.99)),
             "N_cond_max": float(cN.max()), "N_cond_p99": float(np.quantile(cN, 0.99)),
             "F_abs_rel_max": float(xF.max()), "F_abs_rel_p99": float(np.quantile(xF, 0.99)),
             "N_abs_rel_max": float(xN.max()), "N_abs_rel_p99": float(np.quantile(xN, 0.99)),
             "oracle_contacts": int(gold["n_pairs"][k])}
        if (k + 1) % every == 0:
            j = (k + 1) // every - 1
            com = world.read(pid, "COM")[idx]
            q = world.read(pid, "QUAT")[idx]
            r["com_dev_m"] = float(np.abs(com - gold["com"][j]).max())
            r["quat_dev"] = float(np.minimum(np.abs(q - gold["quat"][j]).max(1),
                                             np.abs(q + gold["quat"][j]).max(1)).max())
        rows.append(r)
    return rows


def summarize_trajectory(rows):
    keys = [k for k in rows[0] if k not in ("step", "oracle_contacts")]
    out = {}
    for k in keys + ["com_dev_m", "quat_dev"]:
        vals = [r[k] for r in rows if k in r]
        if vals:
            out[k] = max(vals)
    out["steps"] = len(rows)
    out["oracle_contacts_max"] = max(r["oracle_contacts"] for r in rows)
    return out


def contact_pair_count(world, pid) -> int:
    """Contact pairs of a pile after the last step (each pair is listed by both spheres)."""
    return int(world.read(pid, "CONTACTS")[:, 0].sum()) // 2
