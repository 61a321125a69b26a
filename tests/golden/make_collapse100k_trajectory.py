"""Write the oracle's 100-step trajectory of the 100,000-sphere collapse.

Test infrastructure: this script calls only the FP64 oracle (``oracle/``) and
the seeded input generator.  It advances the collapse workload (100,000
spheres in rigid dumbbells, 3-rods, tetrahedra and squares, radii lognormal
with median 5 m, at rest in a 2 km ball) by 100 full oracle steps and stores,
for 256 aggregates drawn with a fixed seed, after every step the total force
F_A and torque N_A (Sec. 2.2.3-2.2.4) with the sums of the magnitudes of their
terms (the condition scales), and every 10 steps the COM and quaternion.  A
fingerprint of the initial conditions lets the GPU test refuse a mismatched
generator.

    python tests/golden/make_collapse100k_trajectory.py

takes about 20 minutes on 8 cores and writes collapse100k_100steps.npz here.
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "collapse100k_100steps.npz")
STEPS = 100
N_SAMPLE = 256
POSE_EVERY = 10


def fingerprint(ic) -> str:
    h = hashlib.sha256()
    for a in (ic.counts.astype(np.int32), ic.pos.astype(np.float64), ic.radius.astype(np.float64),
              ic.density.astype(np.float64)):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def describe(ic) -> dict:
    """Descriptors of the initial conditions that survive a change of machine
    (the generator's floating-point results may differ there in the last bit):
    the shape counts exactly, sums of positions, squared positions, radii and
    densities to be compared within 1e-12 relative."""
    return {"counts_sha256": np.array(hashlib.sha256(ic.counts.astype(np.int32).tobytes()).hexdigest()),
            "pos_sum": ic.pos.sum(0), "pos_sq_sum": (ic.pos ** 2).sum(0),
            "radius_sum": np.array(ic.radius.sum()), "density_sum": np.array(ic.density.sum())}


def sample_aggregates(n_agg: int) -> np.ndarray:
    return np.sort(np.random.default_rng(20231120).choice(n_agg, N_SAMPLE, replace=False))


def main():
    import oracle
    from paper_2311_11322_gb300 import workloads as W
    oracle.build()
    ic, p = W.config2(0)
    pile = oracle.Pile(ic, p, want_scales=True)
    idx = sample_aggregates(ic.n_agg)
    F = np.zeros((STEPS, N_SAMPLE, 3))
    N = np.zeros((STEPS, N_SAMPLE, 3))
    sF = np.zeros((STEPS, N_SAMPLE))
    sN = np.zeros((STEPS, N_SAMPLE))
    npairs = np.zeros(STEPS, np.int64)
    n_pose = STEPS // POSE_EVERY
    com = np.zeros((n_pose, N_SAMPLE, 3))
    quat = np.zeros((n_pose, N_SAMPLE, 4))
    t0 = time.time()
    for k in range(STEPS):
        pile.step()
        F[k] = (pile.FA_c + pile.FA_g + pile.FA_e)[idx]
        N[k] = (pile.NA_c + pile.NA_g + pile.NA_e)[idx]
        sF[k] = pile.scaleF[idx]
        sN[k] = pile.scaleN[idx]
        npairs[k] = pile.contact_pairs()[0].shape[0]
        if (k + 1) % POSE_EVERY == 0:
            com[(k + 1) // POSE_EVERY - 1] = pile.r[idx]
            quat[(k + 1) // POSE_EVERY - 1] = pile.q[idx]
        print(f"step {k + 1}: {time.time() - t0:.0f} s", flush=True)
    np.savez_compressed(OUT, fingerprint=np.array(fingerprint(ic)), sample=idx, dt=np.array(p.dt),
                        F=F, N=N, scaleF=sF, scaleN=sN, n_pairs=npairs, com=com, quat=quat,
                        pose_every=np.array(POSE_EVERY), oracle_threads=np.array(oracle.threads()),
                        **describe(ic))
    print("wrote", OUT, flush=True)


def add_descriptors():
    """Add the input descriptors to a stored trajectory written before they
    existed (the oracle's values are kept as they are)."""
    from paper_2311_11322_gb300 import workloads as W
    ic, _ = W.config2(0)
    old = dict(np.load(OUT))
    assert str(old["fingerprint"]) == fingerprint(ic), "stored run is of other inputs"
    old.update(describe(ic))
    np.savez_compressed(OUT, **old)
    print("descriptors added to", OUT, flush=True)


if __name__ == "__main__":
    if "--add-descriptors" in sys.argv:
        add_descriptors()
    else:
        main()
