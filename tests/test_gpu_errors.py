"""Error paths of the entry points added for the multicomponent form, the
MD ensemble and conjugate gradients: arguments out of their documented
range and calls in the wrong state come back as error codes with text,
never as device faults, and leave the context usable."""
import numpy as np
import pytest

from paper_1012_5082_gb300 import inputs as I
from _pair import c0_config

pytestmark = pytest.mark.gpu
INVALID, SCHEDULE, STATE = -1, -5, -8


@pytest.fixture(scope="module")
def V():
    from paper_1012_5082_gb300 import vcsgc
    return vcsgc


def test_multi_rejects_bad_input(V):
    tab = I.eam_tables(I.multi_eam_params(3))
    lat = I.bcc_lattice(8, 8, 8)
    t = I.multi_random_types(lat.n, [20, 20], seed=1)
    bad = t.copy()
    bad[5] = 3  # species >= K
    with pytest.raises(V.VcsgcError) as e:
        V.Multi(lat, bad, tab, [-2.0, -2.0], 10.0, 1000.0)
    assert e.value.code == INVALID
    # period 2: same-colour sites 5.7 A apart, not more than 2 r_c
    with pytest.raises(V.VcsgcError) as e:
        V.Multi(lat, t, tab, [-2.0, -2.0], 10.0, 1000.0, period=(2, 2, 2))
    assert e.value.code == SCHEDULE
    # period that does not divide the lattice
    with pytest.raises(V.VcsgcError) as e:
        V.Multi(lat, t, tab, [-2.0, -2.0], 10.0, 1000.0, period=(3, 4, 4))
    assert e.value.code == INVALID
    # a valid context still runs, and rejects out-of-range queries
    g = V.Multi(lat, t, tab, [-2.0, -2.0], 10.0, 1000.0)
    with pytest.raises(V.VcsgcError):
        g.delta_e([lat.n], [1])
    with pytest.raises(V.VcsgcError):
        g.delta_e([0], [3])
    g.sweep(2)
    assert g.observables()["steps"] == 2 * g.steps_per_sweep
    g.close()


def test_ensemble_and_minimize_states(V):
    lat, types, tab = c0_config()
    g = V.Context(lat, types, tab, -2.0, 1000.0, 700.0, schedule=V.SCHED_BLOCKS, sched=(5, 5, 5, 2, 2, 2))
    # rigid lattice: no MD ensemble, no CG
    with pytest.raises(V.VcsgcError) as e:
        g.set_ensemble("nvt", t_damp=100.0)
    assert e.value.code == STATE
    with pytest.raises(V.VcsgcError) as e:
        g.minimize()
    assert e.value.code == STATE
    g.sweep(1)
    g.close()
    rng = np.random.default_rng(2)
    lat0 = I.bcc_lattice(6, 6, 6)
    latp = I.Lattice(x=(lat0.x + rng.uniform(-0.05, 0.05, lat0.n)) % lat0.box[0],
                     y=(lat0.y + rng.uniform(-0.05, 0.05, lat0.n)) % lat0.box[1],
                     z=(lat0.z + rng.uniform(-0.05, 0.05, lat0.n)) % lat0.box[2], box=lat0.box.copy())
    t = I.random_types(latp.n, 40, seed=3)
    m = V.Context(latp, t, tab, -2.0, 1000.0, 700.0, schedule=V.SCHED_SPATIAL, sched=(2, 2, 2, 2, 2, 2),
                  precision=V.PREC_MIXED)
    with pytest.raises(V.VcsgcError) as e:
        m.set_ensemble("npt", t_damp=100.0, p_damp=1000.0)  # the barostat needs the FP64 virial
    assert e.value.code == STATE
    with pytest.raises(V.VcsgcError) as e:
        m.set_ensemble("nvt", t_damp=-1.0)
    assert e.value.code == INVALID
    with pytest.raises(V.VcsgcError) as e:
        m.minimize(ftol=0.0)
    assert e.value.code == INVALID
    m.set_ensemble("nvt", t_damp=100.0)
    m.set_velocities(I.maxwell_velocities(t, 700.0, seed=4))
    m.md_steps(5)
    assert np.isfinite(m.ensemble_state()["conserved"])
    m.close()


def test_checkpoint_of_a_multicomponent_sized_file_is_refused(V, tmp_path):
    """A file that is not a checkpoint is refused without touching the state."""
    lat, types, tab = c0_config()
    g = V.Context(lat, types, tab, -2.0, 1000.0, 700.0, schedule=V.SCHED_BLOCKS, sched=(5, 5, 5, 2, 2, 2))
    path = tmp_path / "junk.bin"
    path.write_bytes(b"not a checkpoint" * 64)
    t0 = g.types().copy()
    with pytest.raises(V.VcsgcError) as e:
        g.load(str(path))
    assert e.value.code == INVALID
    assert np.array_equal(g.types(), t0)
    g.close()
