"""Write the oracle's 30-step trajectory of the pre-settled spin-up pile.

Test infrastructure: this script calls only the FP64 oracle (``oracle/``) and
the seeded input generator.  It advances the pre-settled 3:2:1.5 ellipsoid
(200,000 equal spheres in aggregates of 2-8 face-adjacent spheres of a
face-centred cubic packing, every neighbour pair overlapping by 1e-5 s, at
rest, spin increment 1e-9 rad/s per step about the shortest axis; Sec. 4.1
setting) by 30 full oracle steps and stores, for 256 aggregates drawn with a
fixed seed, after every step the total force F_A and torque N_A (Sec.
2.2.3-2.2.4) with the sums of the magnitudes of their terms (the condition
scales) and the number of contact pairs, and every 10 steps the COM and
quaternion, with descriptors of the initial conditions.

    python tests/golden/make_config3_settled_trajectory.py

takes about 30 minutes on 8 cores and writes config3_settled_30steps.npz here.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for d in (ROOT, HERE):
    if d not in sys.path:
        sys.path.insert(0, d)

from make_collapse100k_trajectory import describe, fingerprint  # noqa: E402

OUT = os.path.join(HERE, "config3_settled_30steps.npz")
STEPS = 30
N_SAMPLE = 256
POSE_EVERY = 10


def sample_aggregates(n_agg: int) -> np.ndarray:
    return np.sort(np.random.default_rng(20231121).choice(n_agg, N_SAMPLE, replace=False))


def main():
    import oracle
    from paper_2311_11322_gb300 import workloads as W
    oracle.build()
    ic, p = W.config3_settled(0)
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
        print(f"step {k + 1}: {time.time() - t0:.0f} s, {npairs[k]} contact pairs", flush=True)
    np.savez_compressed(OUT, fingerprint=np.array(fingerprint(ic)), sample=idx, dt=np.array(p.dt),
                        F=F, N=N, scaleF=sF, scaleN=sN, n_pairs=npairs, com=com, quat=quat,
                        pose_every=np.array(POSE_EVERY), oracle_threads=np.array(oracle.threads()),
                        **describe(ic))
    print("wrote", OUT, flush=True)


if __name__ == "__main__":
    main()
