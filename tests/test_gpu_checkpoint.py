"""Checkpoint and resume: the Philox streams are counters, so n sweeps,
vcsgc_save, vcsgc_load into a fresh context built from the same inputs and
m more sweeps reproduce the species (and counters) of n + m uninterrupted
sweeps bit for bit; MD state (positions, velocities, box, Nose-Hoover
variables) resumes to rounding; a checkpoint of another system is refused."""
import numpy as np
import pytest

from paper_1012_5082_gb300 import inputs as I
from _pair import c0_config

pytestmark = pytest.mark.gpu
EXACT = ("n_b", "trials", "local_accepts", "global_trials", "global_accepts", "flips", "steps")


@pytest.fixture(scope="module")
def V():
    from paper_1012_5082_gb300 import vcsgc
    return vcsgc


def _resume(V, make, n, m, tmp_path, R=1):
    a = make()
    a.sweep(n)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.sweep(m)
    b = make()
    b.load(path)
    b.sweep(m)
    for r in range(R):
        assert np.array_equal(a.types(r), b.types(r)), r
        oa, ob = a.observables(r), b.observables(r)
        for k in EXACT:
            assert oa[k] == ob[k], (r, k, oa[k], ob[k])
        assert abs(oa["energy"] - ob["energy"]) <= 1e-9 * abs(oa["energy"])
        assert abs(oa["mean_c"] - ob["mean_c"]) <= 1e-12
    a.close()
    b.close()


def test_resume_blocks_schedule(V, tmp_path):
    """10^3 cells, octant blocks (the parity workload): 50 + 50 sweeps."""
    lat, types, tab = c0_config()
    _resume(V, lambda: V.Context(lat, types, tab, -2.0, 1000.0, 700.0, seed=3, schedule=V.SCHED_BLOCKS,
                                 sched=(5, 5, 5, 2, 2, 2)), 50, 50, tmp_path)


def test_resume_sublattice_replicas(V, tmp_path):
    """16^3 cells x 4 replicas at different phi on the fused sublattice
    step: 30 + 40 sweeps (the step base is not a multiple of the 64-step
    graph)."""
    lat = I.bcc_lattice(16, 16, 16)
    types = I.random_types(lat.n, int(0.05 * lat.n), seed=5)
    phi = np.array([-2.1, -2.0, -1.9, -1.8])
    _resume(V, lambda: V.Context(lat, np.tile(types, 4), I.eam_tables(), 0.0, 100.0, 900.0, n_replicas=4, phi_r=phi,
                                 seed_r=np.arange(4, dtype=np.uint64) + 11, c0=0.05), 30, 40, tmp_path, R=4)


def test_resume_uneven_batch(V, tmp_path):
    """A batch of three lattices of different sizes."""
    cells = [(12, 12, 12), (16, 12, 12), (12, 16, 20)]
    types = [I.random_types(2 * x * y * z, int(0.04 * 2 * x * y * z), seed=20 + q) for q, (x, y, z) in enumerate(cells)]
    _resume(V, lambda: V.Batch(cells, types, I.eam_tables(), -2.0, 100.0, 900.0,
                               seed_r=np.array([7, 8, 9], dtype=np.uint64), c0=0.04), 20, 25, tmp_path, R=3)


def test_resume_md_npt(V, tmp_path):
    """Explicit positions under NPT: 20 steps, save, 20 more; a new context
    loaded from the checkpoint reaches the same positions (1e-9 A), box and
    extended energy after its 20 steps (force sums use atomics, so rounding
    order may differ)."""
    lat0 = I.bcc_lattice(6, 6, 6)
    rng = np.random.default_rng(3)
    lat = I.Lattice(x=(lat0.x + rng.uniform(-0.05, 0.05, lat0.n)) % lat0.box[0],
                    y=(lat0.y + rng.uniform(-0.05, 0.05, lat0.n)) % lat0.box[1],
                    z=(lat0.z + rng.uniform(-0.05, 0.05, lat0.n)) % lat0.box[2], box=lat0.box.copy())
    t = I.random_types(lat.n, 40, seed=9)
    tab = I.eam_tables(I.npt_eam_params())

    def make():
        g = V.Context(lat, t, tab, -2.0, 1000.0, 700.0, schedule=V.SCHED_SPATIAL, sched=(2, 2, 2, 2, 2, 2), dt=1.0,
                      gamma=0.0, T_md=700.0)
        g.set_velocities(I.maxwell_velocities(t, 700.0, seed=4))
        g.set_ensemble("npt", t_damp=50.0, p_damp=200.0, p_ext_bar=1e4)
        return g

    a = make()
    a.md_steps(20)
    path = str(tmp_path / "md.bin")
    a.save(path)
    a.md_steps(20)
    b = make()
    b.load(path)
    b.md_steps(20)
    sa, sb = a.ensemble_state(), b.ensemble_state()
    assert abs(sa["lx"] - sb["lx"]) < 1e-10
    assert abs(sa["conserved"] - sb["conserved"]) <= 1e-10 * abs(sa["conserved"])
    xa, xb = a.md_state(), b.md_state()
    for q in range(3):
        d = np.abs(xa[q] - xb[q])
        assert np.minimum(d, sa["lx"] - d).max() < 1e-9
    a.close()
    b.close()


def test_load_refuses_another_system(V, tmp_path):
    lat, types, tab = c0_config()
    a = V.Context(lat, types, tab, -2.0, 1000.0, 700.0, schedule=V.SCHED_BLOCKS, sched=(5, 5, 5, 2, 2, 2))
    path = str(tmp_path / "x.bin")
    a.save(path)
    lat2 = I.bcc_lattice(12, 12, 12)
    b = V.Context(lat2, I.random_types(lat2.n, 100, seed=1), tab, -2.0, 1000.0, 700.0)
    with pytest.raises(V.VcsgcError):
        b.load(path)
    with pytest.raises(V.VcsgcError):
        b.load(str(tmp_path / "missing.bin"))
    a.close()
    b.close()
