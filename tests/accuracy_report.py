"""Per-step error report of the CUDA library against the FP64 oracle.

Test infrastructure (it runs the oracle): `python -m tests.accuracy_report
[--out FILE]` on a machine with a GPU.  Both sides start from the same seeded
initial conditions and run side by side; after every step the report takes,
over all aggregates, the maximum and 99th percentile of the condition-relative
force and torque errors (error / sum of the magnitudes of the summed terms),
the number of contacts with overlap above 1e-6 R that the two sides do not
share, and the largest COM and quaternion deviations.

Workloads: the 1,000-sphere tetrahedra cloud (100 steps, both precisions), the
dense contact lattice (2,000 spheres, 100 steps, both precisions), the
100,000-sphere collapse (20 steps, mixed) and the 200,000-sphere spin-up pile
(5 steps, mixed).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from paper_2311_11322_gb300 import workloads as W
from tests.parity_util import agg_errors, contact_set_check


def run_case(dem, oracle, name, ic, p, steps, r_ref):
    pile = oracle.Pile(ic, p, want_scales=True)
    rows = []
    t0 = time.time()
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        for k in range(steps):
            pile.step()
            w.step(1)
            eF, eN = agg_errors(w, pid, pile)
            ns, ng, bad = contact_set_check(w, pid, pile, r_ref)
            dr = np.abs(w.read(pid, "COM") - pile.r).max() / r_ref
            q = w.read(pid, "QUAT")
            dq = np.minimum(np.abs(q - pile.q).max(1), np.abs(q + pile.q).max(1)).max()
            rows.append({"step": k + 1, "F_max": float(eF.max()), "F_p99": float(np.quantile(eF, 0.99)),
                         "N_max": float(eN.max()), "N_p99": float(np.quantile(eN, 0.99)),
                         "contacts": int(ns), "contact_mismatch": len(bad),
                         "com_dev_over_R": float(dr), "quat_dev": float(dq)})
    return {"name": name, "precision": "fp64" if p.precision == W.PRECISION_FP64 else "mixed",
            "n_spheres": ic.n_sph, "n_aggregates": ic.n_agg, "steps": steps,
            "worst": {key: max(r[key] for r in rows) for key in
                      ("F_max", "F_p99", "N_max", "N_p99", "contact_mismatch", "com_dev_over_R", "quat_dev")},
            "max_contacts_seen": max(r["contacts"] for r in rows), "wall_s": time.time() - t0,
            "per_step": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--quick", action="store_true", help="small cases only")
    args = ap.parse_args()
    import __graft_entry__
    import oracle
    __graft_entry__.build()
    oracle.build()
    from paper_2311_11322_gb300 import dem
    cases = []
    for prec in (W.PRECISION_MIXED, W.PRECISION_FP64):
        cases.append(("config1 (250 tetrahedra)", *W.config1(0, precision=prec), 100, 1.0))
        cases.append(("dense lattice (2,000 spheres)",
                      *W.dense_lattice(n_spheres=2000, seed=7, precision=prec), 100, 1.0))
    if not args.quick:
        cases.append(("collapse-100k", *W.config2(0), 20, 5.0))
        cases.append(("spin-up pile 200k", *W.config3(0), 5, 1.0))
    out = [run_case(dem, oracle, name, ic, p, steps, r) for name, ic, p, steps, r in cases]
    text = json.dumps(out)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    for c in out:
        print(c["name"], c["precision"], json.dumps(c["worst"]), "contacts", c["max_contacts_seen"],
              f"{c['wall_s']:.0f} s", flush=True)


if __name__ == "__main__":
    main()
