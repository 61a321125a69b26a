"""100 steps of the 100,000-sphere collapse (the benchmark workload) and 30
steps of the pre-settled 200,000-sphere spin-up pile (every sphere in contact)
on the GPU, mixed and all-FP64, against the FP64 oracle's own trajectories.

The oracle trajectory (every step's total force and torque of 256 sampled
aggregates, with the sums of the magnitudes of the summed terms, and every 10
steps their COM and orientation) is stored in tests/golden/ by
make_collapse100k_trajectory.py and make_config3_settled_trajectory.py, which
call only the oracle; running the oracle here would take 7 and 30 minutes of
host time.  Both sides start from the
same seeded initial conditions (checked by their descriptors) and run side by side
without re-synchronisation.  Bound: condition-relative error 1e-5 (mixed) and
1e-9 (FP64) at every step; the |X|-relative errors are computed alongside.
"""
import os

import numpy as np
import pytest

from paper_2311_11322_gb300 import workloads as W
from tests.parity_util import (TOL, contact_pair_count, same_inputs, summarize_trajectory,
                               trajectory_errors)

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "collapse100k_100steps.npz")
GOLD3 = os.path.join(os.path.dirname(__file__), "golden", "config3_settled_30steps.npz")


@pytest.fixture(scope="module")
def dem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2311_11322_gb300 import dem as D
    return D


@pytest.mark.parametrize("prec", [W.PRECISION_MIXED, W.PRECISION_FP64])
def test_collapse100k_100_steps_against_oracle_trajectory(dem, prec):
    gold = np.load(GOLD)
    ic, p = W.config2(0, precision=prec)
    assert same_inputs(ic, gold), "input generator differs from the stored run"
    assert p.dt == pytest.approx(float(gold["dt"]), rel=1e-12)
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        rows = trajectory_errors(w, pid, gold)
    s = summarize_trajectory(rows)
    tol = TOL[prec]
    assert s["steps"] == 100
    assert s["F_cond_max"] <= tol and s["N_cond_max"] <= tol, s
    # the COMs move ~1e-3 m in these steps; deviations stay at round-off
    assert s["com_dev_m"] <= 1e-6 and s["quat_dev"] <= 1e-6, s


@pytest.mark.parametrize("prec", [W.PRECISION_MIXED, W.PRECISION_FP64])
def test_config3_settled_30_steps_against_oracle_trajectory(dem, prec):
    """The spin-up pile under its spin ramp with ~940,000 contact pairs (friction,
    rolling, history carried between steps) and self-gravity."""
    gold = np.load(GOLD3)
    ic, p = W.config3_settled(0, precision=prec)
    assert same_inputs(ic, gold), "input generator differs from the stored run"
    assert p.dt == pytest.approx(float(gold["dt"]), rel=1e-12)
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        rows = trajectory_errors(w, pid, gold)
        n_pairs = contact_pair_count(w, pid)
    s = summarize_trajectory(rows)
    tol = TOL[prec]
    assert s["steps"] == 30
    assert s["F_cond_max"] <= tol and s["N_cond_max"] <= tol, s
    assert s["com_dev_m"] <= 1e-9 and s["quat_dev"] <= 1e-9, s
    # pairs barely touching (overlap below 1e-6 s) may differ between the two sides
    assert abs(n_pairs - int(gold["n_pairs"][-1])) <= 1e-3 * int(gold["n_pairs"][-1]), n_pairs
