"""Spin-up and tidal-encounter analyses (Sec. 4.1, 4.2) on the device.

A run arms the library's radius-growth watch (``World.watch``): inside every
step graph the device evaluates the pile's bulk record (equal-moment
ellipsoid radius and density, rigid spin, planet distance) every ``every``
steps and latches the first record whose bulk radius has grown by the chosen
fraction.  The host only polls the latch between batches of steps; nothing
else leaves the GPU while the pile evolves.

* critical spin ratio (Sec. 4.1): spin period at the latch (radius grown by
  5%) over the nominal critical period sqrt(3 pi / (G rho)) of the settled
  pile's bulk density;
* disruption ratio (Sec. 4.2): planet distance at the latch (bulk radius grown
  by 0.5%) over the Roche distance 1.26 R (rho_M / rho_m)^(1/3).

Both are ratios of quantities the device computes; the host divides them.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import workloads as W


def settled(world, pile, steps, chunk=10_000):
    """Advance a pile by `steps` and return its state as new initial
    conditions (sphere positions, aggregate velocities and spins): the
    progenitor for the spin-up and encounter runs."""
    done = 0
    while done < steps:
        n = min(chunk, steps - done)
        world.step(n, piles=[pile])
        done += n
    world.sync()
    return world.ic_of(pile)


def run_until_growth(world, pile, growth, every=10, max_steps=1_000_000, chunk=5_000):
    """Arm the watch (growth > 0) and step the pile until it latches or
    `max_steps` have run.  Returns the watch state and the steps taken."""
    world.watch(pile, growth, every)
    taken = 0
    res = world.watch_result(pile)
    while taken < max_steps:
        n = min(chunk, max_steps - taken)
        world.step(n, piles=[pile])
        taken += n
        res = world.watch_result(pile)
        if res["fired_step"] is not None:
            break
    res["steps_run"] = taken
    return res


def critical_spin_ratio(res) -> float | None:
    """Spin period at the latch over the armed pile's nominal critical period."""
    if res["fired_step"] is None:
        return None
    return res["at_fire"]["period"] / res["at_arm"]["p_crit"]


def roche_distance(R_primary, rho_primary, rho_pile):
    """1.26 R (rho_M / rho_m)^(1/3) (Sec. 4.2)."""
    return 1.26 * R_primary * (rho_primary / rho_pile) ** (1.0 / 3.0)


def disruption_ratio(res, R_primary=W.EARTH_RADIUS, rho_primary=5514.0) -> float | None:
    """Planet distance at the latch over the Roche distance of the armed pile."""
    if res["fired_step"] is None:
        return None
    return res["at_fire"]["planet_dist"] / roche_distance(R_primary, rho_primary,
                                                          res["at_arm"]["density"])


def spinup_params(p, ic, omega_target, ramp_steps, axis=(0.0, 0.0, 1.0)):
    """Parameters whose spin increment (Sec. 4.1) adds omega_target to every
    aggregate's spin over ramp_steps steps, about `axis`."""
    ax = np.asarray(axis, np.float64)
    ax = ax / np.linalg.norm(ax)
    return dataclasses.replace(p, spin_inc=tuple(float(x) for x in ax * omega_target / ramp_steps))


def encounter_params(p, ic, periapsis_rp=1.2, v_inf_kms=3.0, start_roche=3.0, rho_primary=5514.0):
    """Parameters with an Earth-mass planet on a hyperbolic flyby of the pile
    (Sec. 4.2): close approach periapsis_rp Earth radii, started start_roche
    Roche distances out on the incoming branch."""
    rng = np.random.default_rng(0)   # ranges collapsed to points: no draws matter
    mP, xP, vP, orb = W.planet_flyby(ic, rng, periapsis_rp=(periapsis_rp, periapsis_rp),
                                     v_inf_kms=(v_inf_kms, v_inf_kms), start_roche=start_roche,
                                     rho_planet=rho_primary)
    m = W.sphere_mass(ic.radius, ic.density)
    com = (m[:, None] * ic.pos).sum(0) / m.sum()
    return dataclasses.replace(p, ext_mass=mP, ext_pos=tuple(com + xP), ext_vel=tuple(vP)), orb
