"""The allocation-free gravity entry point against the world's gravity pass.

dem_gravity_noalloc serves callers that cannot allocate device memory (they
run inside another program's pool or arena, or in a loop that forbids
allocation after start-up) and therefore cannot create a world.  This test
drives it through the C ABI with device buffers owned by the test, twice in a
row, and checks each result against the per-sphere gravity that the world's
step (dem_step, read back with dem_read_state) computed for the same spheres,
within the tests' mixed-precision tolerance.  It lives in a file that pytest
collects last so that, should it fail, every other test has already run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5   # condition-relative, as for every mixed-precision comparison


def test_gravity_noalloc_matches_world_gravity_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2311_11322_gb300 import dem
    from paper_2311_11322_gb300 import workloads as W

    ic, p = W.config2(3, n_spheres=20_000, ball=800.0)
    with dem.World() as w:
        pid = w.add_pile(ic, p)
        w.step(1)
        w.sync()
        fg_world = w.read(pid, "SPHERE_FG")
        pos = w.read(pid, "SPHERE_POS")
    m = W.sphere_mass(ic.radius, ic.density)
    agg = np.repeat(np.arange(ic.n_agg), ic.counts).astype(np.int32)
    origin = np.average(pos, axis=0, weights=m)
    pm = np.concatenate([(pos - origin).astype(np.float32), m.astype(np.float32)[:, None]], 1)
    _, fmag = oracle.gravity(pos, m, agg, p.G, p.eps, exclude_same_agg=True, want_mag=True)

    dev = torch.device("cuda", torch.cuda.current_device())
    t_pm = torch.from_numpy(np.ascontiguousarray(pm)).to(dev)
    t_m = torch.from_numpy(np.ascontiguousarray(m)).to(dev)
    t_a = torch.from_numpy(agg).to(dev)
    out = torch.empty((ic.n_sph, 4), dtype=torch.float64, device=dev)
    assert t_pm.data_ptr() % 16 == 0 and out.data_ptr() % 32 == 0
    L = dem.load()
    msg = C.create_string_buffer(256)
    stream = torch.cuda.current_stream(dev).cuda_stream
    results = []
    for _ in range(2):
        out.fill_(float("nan"))
        rc = L.dem_gravity_noalloc(t_pm.data_ptr(), t_m.data_ptr(), t_a.data_ptr(), ic.n_sph,
                                   p.G, p.eps, out.data_ptr(), stream, msg, len(msg))
        assert rc == dem.DEM_OK, msg.value
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        err = np.linalg.norm(got[:, :3] - fg_world, axis=1) / fmag
        assert err.max() <= TOL, err.max()
        results.append(got)
    assert np.array_equal(results[0], results[1])

    # sizes beyond the fixed scratch are refused without launching anything
    rc = L.dem_gravity_noalloc(t_pm.data_ptr(), t_m.data_ptr(), t_a.data_ptr(), 131073,
                               p.G, p.eps, out.data_ptr(), stream, msg, len(msg))
    assert rc == dem.DEM_ERR_ARG and b"131072" in msg.value
    # so are buffers below their stated alignment (mass 8 B, agg_id 4 B)
    rc = L.dem_gravity_noalloc(t_pm.data_ptr(), t_m.data_ptr() + 4, t_a.data_ptr(), 10,
                               p.G, p.eps, out.data_ptr(), stream, msg, len(msg))
    assert rc == dem.DEM_ERR_ARG and b"aligned" in msg.value
    rc = L.dem_gravity_noalloc(t_pm.data_ptr(), t_m.data_ptr(), t_a.data_ptr() + 2, 10,
                               p.G, p.eps, out.data_ptr(), stream, msg, len(msg))
    assert rc == dem.DEM_ERR_ARG and b"aligned" in msg.value


@pytest.mark.parametrize("n", [1, 3, 131072])
def test_gravity_noalloc_edge_sizes_against_oracle(n):
    """The edges of the fixed scratch: n below the number of j-range parts (the
    empty parts must contribute zeros) and the largest accepted n (the scratch
    filled to its end), each against the oracle's softened direct sum (same
    mixed-precision bound), twice in a row.  n = 1 has no partner: zero force."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2311_11322_gb300 import dem
    from paper_2311_11322_gb300 import workloads as W

    rng = np.random.default_rng(n)
    pos = rng.uniform(-500.0, 500.0, (n, 3))
    rad = rng.uniform(1.0, 3.0, n)
    m = W.sphere_mass(rad, 2500.0)
    agg = (np.arange(n) // 2).astype(np.int32)          # pairs of spheres share an aggregate
    G, eps = W.G_SI, 0.5
    rows = np.arange(n) if n < 5000 else np.sort(rng.choice(n, 2000, replace=False))
    # the entry point takes FP32 positions: the oracle sees the same rounded inputs
    pos = pos.astype(np.float32).astype(np.float64)
    ref, fmag = oracle.gravity(pos, m, agg, G, eps, exclude_same_agg=True, rows=rows, want_mag=True)
    pm = np.concatenate([pos.astype(np.float32), m.astype(np.float32)[:, None]], 1)
    dev = torch.device("cuda", torch.cuda.current_device())
    t_pm = torch.from_numpy(np.ascontiguousarray(pm)).to(dev)
    t_m = torch.from_numpy(np.ascontiguousarray(m)).to(dev)
    t_a = torch.from_numpy(agg).to(dev)
    out = torch.empty((n, 4), dtype=torch.float64, device=dev)
    L = dem.load()
    msg = C.create_string_buffer(256)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for _ in range(2):
        out.fill_(float("nan"))
        rc = L.dem_gravity_noalloc(t_pm.data_ptr(), t_m.data_ptr(), t_a.data_ptr(), n, G, eps,
                                   out.data_ptr(), stream, msg, len(msg))
        assert rc == dem.DEM_OK, msg.value
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        if n <= 2:
            assert np.array_equal(got[:, :3], np.zeros((n, 3)))
        else:
            err = np.linalg.norm(got[rows, :3] - ref, axis=1) / np.maximum(fmag, 1e-300)
            assert err.max() <= TOL, err.max()
