"""Overlapping, position-weighted domains (Sec. III A) on the GPU: the
weighted site pick of the fused lattice step and of the general per-pair
kernels reproduces the oracle's chain site for site, and a schedule whose
same-colour domains are closer than 2 r_c is refused."""
import numpy as np
import pytest

from paper_1012_5082_gb300 import inputs as I
from _pair import c0_config, compare_obs, lockstep, make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_1012_5082_gb300 import vcsgc
    return vcsgc


@pytest.mark.parametrize("dens_b,sweeps", [(1.0, 60), (1.25, 10)], ids=["fused", "reembed"])
def test_overlap_trajectory_bit_exact(V, dens_b, sweeps):
    """20^3 BCC cells, 5 % B, cells of 10^3 with gap 4 (domains of 6^3 cells,
    13.0 A > 2 r_c apart); phi = -2 eV, kappa = 1000, T = 700 K.  dens_b = 1
    runs the fused bit-packed step, dens_b = 1.25 (re-embedding) the general
    kernels; species agree after every sweep."""
    lat, types, tab = c0_config(n_cells=20, dens_b=dens_b)
    orc, g = make_pair(lat, types, tab, -2.0, 1000.0, 700.0, c0=0.05, seed=515,
                       schedule="overlap", sched=(10, 10, 10, 4, 4, 4))
    spw = g.steps_per_sweep
    assert spw == 2 * 10 ** 3
    resyncs = lockstep(orc, g, sweeps, spw)
    og = g.observables()
    if resyncs == 0:
        compare_obs(orc.obs(), og)
    assert og["trials"] == sweeps * lat.n and og["flips"] > 0
    g.close()


def test_overlap_ising_bit_exact(V):
    """The Ising lattice gas (r_c = 3.5 A) on 12^3 cells, cells of 6^3 with
    gap 2 (7.42 A > 2 r_c): 100 sweeps site for site at c0 = 1/2."""
    tab = I.ising_tables()
    lat = I.bcc_lattice(12, 12, 12)
    types = I.random_types(lat.n, lat.n // 2, seed=616)
    kappa, T = 100.0, 1000.0
    phi = -2.0 * kappa * I.KB_EV * T * 0.5
    orc, g = make_pair(lat, types, tab, phi, kappa, T, c0=0.5, seed=617,
                       schedule="overlap", sched=(6, 6, 6, 2, 2, 2))
    resyncs = lockstep(orc, g, 100, g.steps_per_sweep)
    if resyncs == 0:
        compare_obs(orc.obs(), g.observables())
    assert g.observables()["flips"] > 10000
    g.close()


def test_overlap_separation_refused(V):
    """Gap 3 on the EAM lattice puts same-colour domains 10.19 A apart, less
    than 2 r_c = 10.6 A: vcsgc_init refuses the schedule."""
    lat, types, tab = c0_config(n_cells=18)
    with pytest.raises(V.VcsgcError):
        V.Context(lat, types, tab, -2.0, 1000.0, 700.0, schedule=V.SCHED_OVERLAP, sched=(9, 9, 9, 3, 3, 3))
