"""The autotuner (dem_autotune) through the C ABI.

It times candidate gravity shapes, cell sizes and the two forms of the
contact pass by stepping the live piles;
the piles must leave it in exactly the state they entered it, the knobs it
keeps must be among its candidates, and the steps after it must still agree
with the FP64 oracle within the tolerance of the precision.
"""
import numpy as np
import pytest

from paper_2311_11322_gb300 import workloads as W
from tests.parity_util import TOL, agg_errors

pytestmark = pytest.mark.gpu

STATE = ("COM", "VEL", "QUAT", "OMEGA_BODY", "ACC", "TORQUE_STORED", "CONTACTS", "PLANET",
         "FRAME", "FORCE", "TORQUE", "SPHERE_POS")


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


@pytest.mark.parametrize("prec", [W.PRECISION_FP64, W.PRECISION_MIXED])
def test_autotune_leaves_state_and_keeps_parity(dem, oracle, prec):
    piles = [W.dense_lattice(n_spheres=1500, seed=11, precision=prec),
             W.random_cluster(5, n_agg=40, box=4.0, precision=prec)]
    piles = [(ic, p.replace(G=W.G_SI * 1e4, max_contacts=32)) for ic, p in piles]
    orc = [oracle.Pile(ic, p, want_scales=True) for ic, p in piles]
    with dem.World() as w:
        ids = [w.add_pile(ic, p) for ic, p in piles]
        w.step(3)
        for o in orc:
            o.step(3)
        before = {pid: {f: w.read(pid, f) for f in STATE} for pid in ids}
        steps0 = [w.info(pid)["steps"] for pid in ids]
        assert any(before[ids[0]]["CONTACTS"][:, 0] > 0)
        best = w.autotune(2)
        assert np.isfinite(best) and best > 0
        for pid, s0 in zip(ids, steps0):
            assert w.info(pid)["steps"] == s0
            for f in STATE:
                assert np.array_equal(w.read(pid, f), before[pid][f]), f
        # the kept shape is one of the candidates
        tile = w.get_tuning("grav_tile")
        sym = w.get_tuning("grav_sym")
        assert w.get_tuning("cell_factor") in (1.0, 1.25, 1.5, 2.0)
        assert w.get_tuning("contact_mode") in (0, 1)
        if sym:
            assert tile in ((0, 512, 64, 128, 256) if prec == W.PRECISION_MIXED else (0, 512))
        else:
            assert w.get_tuning("grav_block") in (64, 128, 256)
            assert w.get_tuning("grav_ib") in (1, 2, 4)
            assert w.get_tuning("grav_item") in (262144.0, 1048576.0, 4194304.0)
        # the tuned steps still follow the oracle
        for _ in range(5):
            w.step(1)
            for pid, o in zip(ids, orc):
                o.step()
                eF, eN = agg_errors(w, pid, o)
                assert eF.max() <= TOL[prec] and eN.max() <= TOL[prec], (eF.max(), eN.max())
        for pid, s0 in zip(ids, steps0):
            assert w.info(pid)["steps"] == s0 + 5


def test_autotune_argument_errors(dem):
    ic, p = W.random_cluster(2, n_agg=10, box=3.0)
    with dem.World() as w:
        w.add_pile(ic, p)
        with pytest.raises(dem.DemError):
            w.autotune(0)
        with pytest.raises(dem.DemError):
            w.get_tuning("no_such_knob")
