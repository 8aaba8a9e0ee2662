"""The neighbour-list entry point that allocates nothing, against a context's
own list (GPU only).

Callers that cannot call cudaMalloc (their framework's allocator holds the
device memory, or their memory budget is fixed) pass device positions in and
get the list out in their own buffers; the build's working space is a static
device array inside the library.  This file runs last so that a failure here
stops a -x run only after every other test has run.
"""
import numpy as np
import pytest

from paper_1012_5082_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RL = 5.3 + 0.3  # r_c + skin, as a context with default options uses


def _positions(seed):
    lat = I.bcc_lattice(10, 10, 10)
    rng = np.random.default_rng(seed)
    L = lat.box
    x = np.mod(lat.x + rng.normal(0, 0.1, lat.n), L[0])
    y = np.mod(lat.y + rng.normal(0, 0.1, lat.n), L[1])
    z = np.mod(lat.z + rng.normal(0, 0.1, lat.n), L[2])
    return I.Lattice(x=x, y=y, z=z, box=L)


def _context_rows(V, lat):
    tab = I.eam_tables()
    g = V.Context(lat, np.zeros(lat.n, np.uint8), tab, -2.0, 1000.0, 700.0,
                  schedule=V.SCHED_SPATIAL, sched=(2, 2, 2, 2, 2, 2), skin=0.3)
    rows = [g.neighbours(i) for i in range(lat.n)]
    g.close()
    return rows


def test_noalloc_neighbour_list_matches_context_twice():
    torch = pytest.importorskip("torch")
    from paper_1012_5082_gb300 import vcsgc as V

    K = 96
    for seed in (1, 2):  # two calls in a row, different inputs
        lat = _positions(seed)
        want = _context_rows(V, lat)
        dev = torch.device("cuda", 0)
        dx, dy, dz = (torch.tensor(v, dtype=torch.float64, device=dev) for v in (lat.x, lat.y, lat.z))
        nbr = torch.full((lat.n, K), -7, dtype=torch.int32, device=dev)
        cnt = torch.full((lat.n,), -7, dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        rc = V.vcsgc_neighbour_list_noalloc(lat.n, dx.data_ptr(), dy.data_ptr(), dz.data_ptr(),
                                            lat.box, RL, K, nbr.data_ptr(), cnt.data_ptr())
        assert rc == 0
        got_n = nbr.cpu().numpy()
        got_c = cnt.cpu().numpy()
        for i in range(lat.n):
            assert got_c[i] == len(want[i])
            assert np.array_equal(got_n[i, :got_c[i]], want[i])
            assert np.all(got_n[i, got_c[i]:] == -1)


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
