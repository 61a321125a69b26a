"""GPU: continuous batching and failure isolation through the C ABI."""
import numpy as np
import pytest

from paper_2311_11322_gb300 import serve
from paper_2311_11322_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2311_11322_gb300 import dem as D
    return D


def small_flyby(seed, n):
    return W.config5_pile(dict(t_arrival=0.0, n_spheres=n, seed=seed, steps=0))


def test_served_results_equal_solo_runs_bitwise(dem):
    """Requests of different sizes and lengths arrive over time, with at most
    two resident piles: each result equals the same request run alone."""
    specs = [(1, 400, 60, 0.0), (2, 900, 25, 0.0), (3, 200, 40, 0.0), (4, 600, 30, 0.05)]
    reqs = []
    for rid, n, steps, t in specs:
        ic, p = small_flyby(rid, n)
        reqs.append(serve.Request(rid=rid, ic=ic, params=p, steps=steps, t_arrival=t))
    with dem.World() as w:
        srv = serve.Server(w, dem.dem_footprint_bytes, budget_bytes=1 << 34, max_piles=2, chunk=16)
        st = srv.run(reqs)
    assert st["completed"] == 4
    got = {r.rid: r.result for r in srv.done}
    for rid, n, steps, t in specs:
        ic, p = small_flyby(rid, n)
        with dem.World() as w:
            pid = w.add_pile(ic, p)
            w.step(steps)
            for f in ("COM", "QUAT", "VEL"):
                assert np.array_equal(w.read(pid, f), got[rid][f]), (rid, f)


def test_exploding_pile_is_frozen_and_others_continue(dem):
    """The host writes an absurd (finite) velocity into one pile; its next
    steps overflow to inf/NaN, it is reported and frozen, and the other pile
    keeps stepping unharmed.  No device fault is involved."""
    ic, p = W.dense_lattice(n_spheres=800, seed=3, precision=W.PRECISION_MIXED)
    good_ic, good_p = W.dense_lattice(n_spheres=800, seed=4, precision=W.PRECISION_MIXED)
    with dem.World() as w:
        pb = w.add_pile(ic, p)
        pg = w.add_pile(good_ic, good_p)
        w.write(pb, "VEL", np.full((ic.n_agg, 3), 1e300))
        seen = None
        for _ in range(60):
            s = w.step(1, check=False)
            if s != dem.DEM_OK:
                seen = s
        s = w.sync(check=False)
        seen = seen if seen is not None else s
        assert seen == dem.DEM_ERR_NONFINITE
        assert w.flags(pb) & dem.DEM_FLAG_NONFINITE
        frozen = w.info(pb)["steps"]
        w.step(5)
        w.sync()
        assert w.info(pb)["steps"] == frozen
        assert w.info(pg)["steps"] == 65
        assert np.all(np.isfinite(w.read(pg, "COM")))
