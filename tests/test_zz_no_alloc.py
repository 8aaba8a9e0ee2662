"""The neighbour-list entry point that allocates nothing (GPU only).

Callers that cannot call cudaMalloc (their framework's allocator holds the
device memory, or their memory budget is fixed) pass device positions in and
get the list out in their own buffers; the build's working space is a static
device array inside the library.  The list is checked against a brute-force
minimum-image list computed here in numpy, and against a context's own list.
This file runs last so that a failure here stops a -x run only after every
other test has run.
"""
import numpy as np
import pytest

from paper_1012_5082_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RL = 5.3 + 0.3  # r_c + skin, as a context with default options uses


def _positions(seed, outside=False):
    lat = I.bcc_lattice(10, 10, 10)
    rng = np.random.default_rng(seed)
    L = lat.box
    p = [np.mod(c + rng.normal(0, 0.1, lat.n), L[q]) for q, c in enumerate((lat.x, lat.y, lat.z))]
    if outside:
        # some positions just outside the box, some a whole period away
        sel = rng.choice(lat.n, 300, replace=False)
        for q in range(3):
            shift = rng.choice([-1.0, 1.0, -2.0, 3.0], size=sel.size) * L[q]
            p[q][sel] += shift
        edge = rng.choice(lat.n, 40, replace=False)
        p[0][edge[:20]] = -1e-3 * (1 + np.arange(20))
        p[1][edge[20:]] = L[1] + 1e-3 * (1 + np.arange(20))
    return I.Lattice(x=p[0], y=p[1], z=p[2], box=L)


def _brute(lat, rl):
    """Pairs (i, j) of minimum-image distance d, by brute force in FP64."""
    P = np.stack([lat.x, lat.y, lat.z], axis=1)
    L = np.asarray(lat.box)
    d = P[None, :, :] - P[:, None, :]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(axis=2))
    np.fill_diagonal(r, np.inf)
    return r


def _call(V, torch, lat, K, stream=None):
    dev = torch.device("cuda", 0)
    dx, dy, dz = (torch.tensor(v, dtype=torch.float64, device=dev) for v in (lat.x, lat.y, lat.z))
    nbr = torch.full((lat.n, K), -7, dtype=torch.int32, device=dev)
    cnt = torch.full((lat.n,), -7, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    rc = V.vcsgc_neighbour_list_noalloc(lat.n, dx.data_ptr(), dy.data_ptr(), dz.data_ptr(), lat.box, RL, K,
                                        nbr.data_ptr(), cnt.data_ptr(),
                                        None if stream is None else stream.cuda_stream)
    return rc, nbr.cpu().numpy(), cnt.cpu().numpy()


def _check_rows(r, got_n, got_c, rl, margin):
    for i in range(r.shape[0]):
        row = got_n[i, :got_c[i]]
        assert np.all(got_n[i, got_c[i]:] == -1)
        assert len(set(row.tolist())) == len(row)
        must = set(np.nonzero(r[i] < rl)[0].tolist())
        may = set(np.nonzero(r[i] < rl + margin)[0].tolist())
        assert must <= set(row.tolist()) <= may, i


def _context_rows(V, lat):
    tab = I.eam_tables()
    g = V.Context(lat, np.zeros(lat.n, np.uint8), tab, -2.0, 1000.0, 700.0,
                  schedule=V.SCHED_SPATIAL, sched=(2, 2, 2, 2, 2, 2), skin=0.3)
    rows = [g.neighbours(i) for i in range(lat.n)]
    g.close()
    return rows


def test_noalloc_neighbour_list_matches_brute_force_twice():
    """Two calls in a row on different inputs: every pair within rl is listed,
    nothing beyond rl plus the documented FP32 margin, and the rows equal a
    context's own list."""
    torch = pytest.importorskip("torch")
    from paper_1012_5082_gb300 import vcsgc as V

    K = 96
    for seed in (1, 2):
        lat = _positions(seed)
        rc, got_n, got_c = _call(V, torch, lat, K)
        assert rc == 0
        _check_rows(_brute(lat, RL), got_n, got_c, RL, 0.01 + 1e-6 * max(lat.box))
        want = _context_rows(V, lat)
        for i in range(lat.n):
            assert got_c[i] == len(want[i])
            assert np.array_equal(got_n[i, :got_c[i]], want[i])


def test_noalloc_positions_outside_the_box():
    """Positions just outside the box or whole periods away are binned at
    their periodic image: the list equals the brute-force minimum-image list."""
    torch = pytest.importorskip("torch")
    from paper_1012_5082_gb300 import vcsgc as V

    lat = _positions(3, outside=True)
    assert lat.x.min() < 0 and lat.y.max() > lat.box[1]
    rc, got_n, got_c = _call(V, torch, lat, 96)
    assert rc == 0
    _check_rows(_brute(lat, RL), got_n, got_c, RL, 0.01 + 1e-6 * max(lat.box))


def test_noalloc_overflow_truncates_rows_and_side_stream():
    """A capacity below the row lengths reports OVERFLOW with every row cut to
    K entries of the full list; the call honours a caller's side stream."""
    torch = pytest.importorskip("torch")
    from paper_1012_5082_gb300 import vcsgc as V

    lat = _positions(4)
    rc, full_n, full_c = _call(V, torch, lat, 96)
    assert rc == 0 and full_c.min() > 20
    side = torch.cuda.Stream()
    rc, got_n, got_c = _call(V, torch, lat, 20, stream=side)
    assert rc == -9  # VCSGC_ERR_OVERFLOW
    assert np.all(got_c == 20)
    assert np.array_equal(got_n, full_n[:, :20])
    rc, got_n, got_c = _call(V, torch, lat, 96, stream=side)
    assert rc == 0 and np.array_equal(got_n, full_n) and np.array_equal(got_c, full_c)


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    from paper_1012_5082_gb300 import vcsgc as V

    dev = torch.device("cuda", 0)
    buf = torch.zeros(8, dtype=torch.float64, device=dev)
    out = torch.zeros(8, dtype=torch.int32, device=dev)
    p = buf.data_ptr()
    # more positions than the static working space holds
    assert V.vcsgc_neighbour_list_noalloc(262145, p, p, p, (100.0, 100.0, 100.0), RL, 1,
                                          out.data_ptr(), out.data_ptr()) == -1
    # box too small for three binning cells
    assert V.vcsgc_neighbour_list_noalloc(8, p, p, p, (12.0, 100.0, 100.0), RL, 1,
                                          out.data_ptr(), out.data_ptr()) == -1
