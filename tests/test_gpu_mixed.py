"""Mixed-precision form (FP32 table evaluation, FP64 sums and embedding
differences) against the FP64 form and the oracle (GPU only).  Tolerances
are set from the FP32 rounding of ~60 interpolated terms per site."""
import numpy as np
import pytest

import oracle as O
from paper_1012_5082_gb300 import inputs as I
from _pair import c0_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_1012_5082_gb300 import vcsgc
    return vcsgc


def _ctx(V, lat, t, tab, prec, sched=(5, 5, 5, 2, 2, 2), kind=None, **kw):
    schedule = V.SCHED_BLOCKS if kind is None else kind
    return V.Context(lat, t, tab, -2.0, 1000.0, 700.0, schedule=schedule, sched=sched,
                     precision=prec, **kw)


@pytest.mark.parametrize("dens_b", [1.0, 1.25])
def test_mixed_rigid_lattice_de_and_energy(V, dens_b):
    lat, _, tab = c0_config(dens_b=dens_b)
    t = I.random_types(lat.n, 600, seed=31)
    orc = O.System(lat, t, tab)
    g64 = _ctx(V, lat, t, tab, V.PREC_FP64)
    g32 = _ctx(V, lat, t, tab, V.PREC_MIXED)
    sites = np.arange(lat.n)
    d64, d32 = g64.delta_e(sites), g32.delta_e(sites)
    d_o = np.array([orc.delta_e(i) for i in sites])
    err = np.abs(d32 - d_o)
    assert err.max() < 2e-5, err.max()
    assert np.sqrt(np.mean(err ** 2)) < 5e-6
    assert np.max(np.abs(d64 - d_o)) < 1e-11
    e_o = orc.energy_full()
    assert abs(g32.energy() - e_o) / lat.n < 2e-6
    assert np.max(np.abs(g32.rho() - orc.rho) / orc.rho) < 1e-6
    g64.close()
    g32.close()


@pytest.mark.parametrize("dens_b", [1.0, 1.25])
def test_mixed_explicit_positions_de_rho_forces(V, dens_b):
    lat, _, tab = c0_config(n_cells=7, dens_b=dens_b)
    rng = np.random.default_rng(8)
    pert = I.Lattice(x=lat.x + rng.normal(0, 0.08, lat.n), y=lat.y + rng.normal(0, 0.08, lat.n),
                     z=lat.z + rng.normal(0, 0.08, lat.n), box=lat.box)
    t = I.random_types(lat.n, 200, seed=32)
    orc = O.System(pert, t, tab)
    g = _ctx(V, pert, t, tab, V.PREC_MIXED, sched=(2, 2, 2, 2, 2, 2), kind=V.SCHED_SPATIAL)
    sites = np.arange(lat.n)
    d32 = g.delta_e(sites)
    d_o = np.array([orc.delta_e(i) for i in sites])
    assert np.max(np.abs(d32 - d_o)) < 2e-5
    assert np.max(np.abs(g.rho() - orc.rho) / orc.rho) < 1e-6
    F32, Fo = g.forces(), orc.forces()
    for a in range(3):
        assert np.max(np.abs(F32[a] - Fo[a])) < 2e-5
    g.close()


def test_mixed_md_energy_behaviour(V):
    """NVE with FP32 force evaluation keeps the total energy within a small
    band (no secular drift beyond the FP32 level)."""
    tab = I.eam_tables()
    lat = I.bcc_lattice(8, 8, 8)
    pos = I.Lattice(x=lat.x.copy(), y=lat.y.copy(), z=lat.z.copy(), box=lat.box)
    t = I.random_types(lat.n, 60, seed=2)
    g = _ctx(V, pos, t, tab, V.PREC_MIXED, sched=(2, 2, 2, 2, 2, 2), kind=V.SCHED_SPATIAL,
             dt=1.0, gamma=0.0)
    g.set_velocities(I.maxwell_velocities(t, 600.0, seed=3))
    e0 = g.energy() + g.kinetic_energy()
    es = []
    for _ in range(10):
        g.md_steps(50)
        es.append(g.energy() + g.kinetic_energy())
    es = np.array(es) - e0
    assert np.max(np.abs(es)) / lat.n < 5e-5
    g.close()


def test_mixed_sweep_concentration_matches_fp64(V):
    """Same start and seed: the mixed-form chain's mean concentration agrees
    with the FP64 chain's within their statistical error."""
    lat, types, tab = c0_config(n_cells=8)
    res = {}
    for prec in (V.PREC_FP64, V.PREC_MIXED):
        g = V.Context(lat, types, tab, -2.45, 20.0, 700.0, seed=2100, c0=0.05,
                      schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4), precision=prec)
        cs = []
        for _ in range(40):
            g.sweep(10)
            cs.append(g.observables()["c"])
        res[prec] = np.array(cs[5:])
        g.close()
    a, b = res[V.PREC_FP64], res[V.PREC_MIXED]
    err = np.sqrt(a.var() / len(a) + b.var() / len(b)) * 3  # correlated samples
    assert abs(a.mean() - b.mean()) < 5 * err + 1e-3
