"""Asynchronous reads (dem_read_state_async / dem_read_wait): the values equal
the synchronous read of the same state bit for bit, a read issued before a
step sees the state before it, pipelined reads (a step in flight while the
previous result is waited for) give every step's result, and misuse is
reported."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2311_11322_gb300 import workloads as W

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


def pinned(shape):
    import torch
    return torch.zeros(shape, dtype=torch.float64).pin_memory().numpy()


@pytest.mark.parametrize("prec", PRECS)
def test_async_equals_sync(dem, prec):
    ic, p = W.random_cluster(5, n_agg=60, box=5.0, precision=prec)
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        w.step(3)
        A = len(ic.counts)
        outs = {}
        for f in dem.World.ASYNC_FIELDS:
            cols = dem.FIELDS[f][2]
            outs[f] = pinned((A, cols) if cols > 1 else (A,))
            w.read_async(pid, f, outs[f])
        w.read_wait()
        for f, o in outs.items():
            assert np.array_equal(o, w.read(pid, f)), f


@pytest.mark.parametrize("prec", PRECS)
def test_pipelined_reads_follow_the_trajectory(dem, prec):
    """Read COM after every step with the next step already issued; compare
    with a second world stepped the same way but read synchronously."""
    ic, p = W.random_cluster(6, n_agg=60, box=5.0, precision=prec)
    steps = 12
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        ref = []
        for _ in range(steps):
            w.step(1)
            ref.append(w.read(pid, "COM"))
    A = len(ic.counts)
    bufs = [pinned((A, 3)) for _ in range(steps)]
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        w.step(1)
        w.read_async(pid, "COM", bufs[0])
        for s in range(1, steps):
            w.step(1)              # in flight while result s-1 is waited for
            w.read_wait()
            w.read_async(pid, "COM", bufs[s])
        w.read_wait()
        w.sync()
    for s in range(steps):
        assert np.array_equal(bufs[s], ref[s]), s
    # a read issued before a step sees the state before it
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        w.step(2)
        before = pinned((A, 3))
        w.read_async(pid, "COM", before)
        w.step(1)
        w.read_wait()
        assert np.array_equal(before, ref[1])
        assert np.array_equal(w.read(pid, "COM"), ref[2])


def test_async_read_misuse_reported(dem):
    ic, p = W.random_cluster(7, n_agg=20, box=4.0, precision=W.PRECISION_MIXED)
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        w.step(1)
        A = len(ic.counts)
        with pytest.raises(dem.DemError) as ei:      # not a per-aggregate state field
            w.read_async(pid, "FORCE", pinned((A, 3)))
        assert ei.value.status == dem.DEM_ERR_ARG
        with pytest.raises(dem.DemError):            # unknown pile
            w.read_async(pid + 7, "COM", pinned((A, 3)))
        w.read_wait()
        bufs = [pinned((A, 3)) for _ in range(9)]
        for b in bufs[:8]:
            w.read_async(pid, "COM", b)
        with pytest.raises(dem.DemError):            # more than 8 pending
            w.read_async(pid, "COM", bufs[8])
        w.read_wait()
        com = w.read(pid, "COM")
        for b in bufs[:8]:
            assert np.array_equal(b, com)
