"""Multicomponent colour step on the GPU against the multicomponent oracle:
energy changes to every target species and total energies (FP64), and
trajectories site for site over whole sweeps for K = 3 (one density
function) and K = 4 (species-dependent densities: re-embedding), with the
oracle's near-tie flags as the only allowed divergence."""
import numpy as np
import pytest

import oracle as O
from paper_1012_5082_gb300 import inputs as I
from _pair import Lockstep

pytestmark = pytest.mark.gpu

CASES = {
    # K, density scales, phi (eV), kappa, T (K), c0 (per solute)
    3: (None, [-2.3, -2.1], 10.0, 1200.0, 0.05),
    4: ((1.0, 1.25, 0.85, 1.1), [-1.45, -2.45, 0.2], 10.0, 1200.0, 0.05),
}


@pytest.fixture(scope="module")
def V():
    from paper_1012_5082_gb300 import vcsgc
    return vcsgc


def _pair(V, K, cells=(8, 8, 8), seed=3, R=1, phi=None):
    ds, phi0, kappa, T, c0 = CASES[K]
    phi = phi0 if phi is None else phi
    tab = I.eam_tables(I.multi_eam_params(K, dens_scale=ds))
    lat = I.bcc_lattice(*cells)
    t = I.multi_random_types(lat.n, [int(c0 * lat.n)] * (K - 1), seed=seed)
    orc = O.MultiSystem(lat, t, tab)
    orc.set_params(phi, [kappa] * (K - 1), T, c0=[c0] * (K - 1), seed=seed + 100)
    orc.schedule_sublattice(lat.cells, (4, 4, 4))
    g = V.Multi(lat, t, tab, phi, kappa, T, c0=c0, seed_r=np.array([seed + 100] * R, dtype=np.uint64),
                n_replicas=R)
    return lat, tab, orc, g


@pytest.mark.parametrize("K", [3, 4])
def test_multi_delta_e_and_energy(V, K):
    """dE of 300 random (site, target species) pairs within 1e-11 eV of the
    oracle's neighbour-by-neighbour sum, and the energy within 1e-12
    relative."""
    lat, tab, orc, g = _pair(V, K)
    rng = np.random.default_rng(K)
    sites = rng.integers(0, lat.n, 300)
    to = rng.integers(0, K, 300).astype(np.uint8)
    d_gpu = g.delta_e(sites, to)
    d_orc = np.array([orc.delta_e(i, b) for i, b in zip(sites, to)])
    assert np.abs(d_gpu - d_orc).max() < 1e-11, np.abs(d_gpu - d_orc).max()
    assert np.count_nonzero(d_orc) > 200
    e = orc.energy_full()
    assert abs(g.energy() - e) <= 1e-12 * abs(e)
    assert abs(g.observables()["energy"] - e) <= 1e-12 * abs(e)
    g.close()


@pytest.mark.parametrize("K,sweeps", [(3, 60), (4, 30)])
def test_multi_trajectory_bit_exact(V, K, sweeps):
    """8^3 cells, period-4 sublattice (8 trials per colour step): species
    agree after every sweep; counters and counts agree exactly, the tracked
    energy to 1e-9 relative, and it equals the full energy."""
    lat, tab, orc, g = _pair(V, K)
    spw = g.steps_per_sweep
    assert spw == 128
    resyncs = 0
    for s in range(sweeps):
        ties0 = orc.obs()["near_ties"]
        g.sweep(1)
        orc.parallel_steps(spw)
        tg, to = g.types(), orc.types
        if not np.array_equal(tg, to):
            assert orc.obs()["near_ties"] > ties0, f"sweep {s}: species differ without a flagged tie"
            g.set_types(to)
            resyncs += 1
    og, oo = g.observables(), orc.obs()
    if resyncs == 0:
        for k in ("trials", "local_accepts", "global_trials", "global_accepts", "flips"):
            assert og[k] == oo[k], (k, og[k], oo[k])
        assert og["n"] == oo["n"]
        assert abs(og["energy"] - oo["energy"]) <= 1e-9 * abs(oo["energy"])
        for a in range(K):
            assert abs(og["mean_c"][a] * og["steps"] - oo["sum_c"][a]) < 1e-9 * oo["steps"]
    assert og["flips"] > 500
    assert abs(g.energy() - og["energy"]) <= 1e-9 * abs(og["energy"])
    g.close()


def test_multi_replicas_independent(V):
    """Two replicas with the same seed and start evolve identically; a third
    with another seed does not."""
    ds, phi, kappa, T, c0 = CASES[3]
    tab = I.eam_tables(I.multi_eam_params(3, dens_scale=ds))
    lat = I.bcc_lattice(8, 8, 8)
    t = I.multi_random_types(lat.n, [int(c0 * lat.n)] * 2, seed=9)
    g = V.Multi(lat, np.stack([t, t, t]), tab, phi, kappa, T, c0=c0,
                seed_r=np.array([5, 5, 6], dtype=np.uint64))
    g.sweep(20)
    assert np.array_equal(g.types(0), g.types(1))
    assert not np.array_equal(g.types(0), g.types(2))
    assert g.observables(0)["flips"] == g.observables(1)["flips"] > 0
    g.close()


def test_multi_k2_retraces_binary_fused_step(V):
    """K = 2 through the multicomponent kernels and the binary fused step on
    the same 12^3 lattice, period-4 sublattice, seeds and parameters: the same
    species after every sweep (both are the binary chain, up to near-ties)."""
    tab = I.eam_tables(I.multi_eam_params(2))
    lat = I.bcc_lattice(12, 12, 12)
    t = I.random_types(lat.n, int(0.05 * lat.n), seed=77)
    kappa, T, c0, phi = 100.0, 1200.0, 0.05, -3.0
    m = V.Multi(lat, t, tab, [phi], kappa, T, c0=c0, seed_r=np.array([78], dtype=np.uint64))
    b = V.Context(lat, t, tab, phi, kappa, T, seed=78, c0=c0, schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4))
    assert m.steps_per_sweep == b.steps_per_sweep == 128
    same = 0
    for s in range(40):
        m.sweep(1)
        b.sweep(1)
        if np.array_equal(m.types(), b.types()):
            same += 1
        else:
            break
    assert same == 40, same
    om, ob = m.observables(), b.observables()
    assert om["flips"] == ob["flips"] > 500 and om["n"][1] == ob["n_b"]
    m.close()
    b.close()


def test_multi_screened_reembedding_16cubed(V):
    """K = 4 with species-dependent densities on 16^3 cells (64 trials per
    colour step).  The local decision is taken on an FP32 dE inside a proven
    error bound, the open trials and the accepts' energies in FP64: species
    agree with the oracle after every sweep (near-ties aside), counters
    agree, and the tracked energy equals the full energy and the oracle's."""
    # phi where the expected dn of every solute vanishes on the random start
    lat, tab, orc, g = _pair(V, 4, cells=(16, 16, 16), seed=11, phi=[-1.173, -2.037, 0.567])
    spw = g.steps_per_sweep
    resyncs = 0
    for s in range(12):
        ties0 = orc.obs()["near_ties"]
        g.sweep(1)
        orc.parallel_steps(spw)
        if not np.array_equal(g.types(), orc.types):
            assert orc.obs()["near_ties"] > ties0, f"sweep {s}: species differ without a flagged tie"
            g.set_types(orc.types)
            resyncs += 1
    og, oo = g.observables(), orc.obs()
    if resyncs == 0:
        for k in ("trials", "local_accepts", "global_trials", "global_accepts", "flips"):
            assert og[k] == oo[k], (k, og[k], oo[k])
        assert abs(og["energy"] - oo["energy"]) <= 1e-9 * abs(oo["energy"])
    assert og["flips"] > 3000 and og["global_accepts"] > 200
    assert abs(g.energy() - og["energy"]) <= 1e-9 * abs(og["energy"])
    g.close()


@pytest.mark.parametrize("nrho", [5000, 8])
def test_multi_screen_out_of_range_goes_fp64(V, nrho):
    """Embedding grids to rho = 400.  With 5000 points the screen covers
    the densities the five shells can reach (about 12 to 18).  With 8
    points (h = 57) every reachable density lies in the grid's first
    interval, below the screened range, so the context still opens and
    every trial of the re-embedding step takes the FP64 path of the whole
    warp.  Either way the trajectory follows the oracle's site for site."""
    ds, phi, kappa, T, c0 = CASES[4]
    tab = I.eam_tables(I.multi_eam_params(4, dens_scale=ds, rho_max=400.0, nrho=nrho))
    lat = I.bcc_lattice(8, 8, 8)
    t = I.multi_random_types(lat.n, [int(c0 * lat.n)] * 3, seed=5)
    orc = O.MultiSystem(lat, t, tab)
    orc.set_params(phi, [kappa] * 3, T, c0=[c0] * 3, seed=105)
    orc.schedule_sublattice(lat.cells, (4, 4, 4))
    g = V.Multi(lat, t, tab, phi, kappa, T, c0=c0, seed_r=np.array([105], dtype=np.uint64))
    for s in range(10):
        ties0 = orc.obs()["near_ties"]
        g.sweep(1)
        orc.parallel_steps(g.steps_per_sweep)
        if not np.array_equal(g.types(), orc.types):
            assert orc.obs()["near_ties"] > ties0, f"sweep {s}: species differ without a flagged tie"
            g.set_types(orc.types)
    og, oo = g.observables(), orc.obs()
    assert og["flips"] > 100
    assert abs(og["energy"] - orc.energy_full()) <= 1e-9 * abs(og["energy"])
    g.close()


def test_binary_reembedding_sublattice_against_oracle(V):
    """Species-dependent densities (f_B = 1.25 f_A) on the period-4
    sublattice: the binary context advances through the two-species
    multicomponent kernels (FP32-screened decisions, compile-time offsets).
    Lockstep against the binary oracle on a 12^3 lattice, two replicas, 12
    sweeps: species after every sweep, counters and energy; then a save, a
    load into a fresh context and 2 more sweeps retrace an uninterrupted
    chain; the K = 2 multicomponent context runs the same chain."""
    tab = I.eam_tables(I.multi_eam_params(2, dens_scale=(1.0, 1.25)))
    lat = I.bcc_lattice(12, 12, 12)
    t = I.random_types(lat.n, int(0.05 * lat.n), seed=77)
    kappa, T, c0, phis, seeds = 100.0, 1200.0, 0.05, [-2.2, -2.3], [78, 79]
    b = V.Context(lat, np.tile(t, 2), tab, 0.0, kappa, T, c0=c0, schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4),
                  n_replicas=2, phi_r=np.array(phis), seed_r=np.array(seeds, dtype=np.uint64))
    orcs = []
    for phi, seed in zip(phis, seeds):
        o = O.System(lat, t, tab)
        o.set_params(phi, kappa, T, c0=c0, seed=seed)
        o.schedule_sublattice(lat.cells, (4, 4, 4))
        orcs.append(o)
    ls = Lockstep(orcs, b)
    for _ in range(12):
        ls.advance(b.steps_per_sweep)
    assert min(b.observables(r)["flips"] for r in range(2)) > 1000
    ls.close()
    rho_o = orcs[0].rho
    assert np.allclose(b.rho(0), rho_o, rtol=1e-13, atol=0)
    # checkpoint round trip against the uninterrupted chain
    import os
    import tempfile
    path = os.path.join(tempfile.mkdtemp(), "reembed.ck")
    b.save(path)
    b2 = V.Context(lat, np.tile(t, 2), tab, 0.0, kappa, T, c0=c0, schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4),
                   n_replicas=2, phi_r=np.array(phis), seed_r=np.array(seeds, dtype=np.uint64))
    b2.load(path)
    b.sweep(2)
    b2.sweep(2)
    for r in range(2):
        assert np.array_equal(b.types(r), b2.types(r))
        o1, o2 = b.observables(r), b2.observables(r)
        assert o1["flips"] == o2["flips"] and o1["steps"] == o2["steps"]
    b2.close()
    b.close()
    # the multicomponent context with K = 2, replica 0's chain
    m = V.Multi(lat, t, tab, [phis[0]], kappa, T, c0=c0, seed_r=np.array([seeds[0]], dtype=np.uint64))
    o = O.System(lat, t, tab)
    o.set_params(phis[0], kappa, T, c0=c0, seed=seeds[0])
    o.schedule_sublattice(lat.cells, (4, 4, 4))
    m.sweep(6)
    o.parallel_steps(6 * 128)
    assert np.array_equal(m.types(), o.types)
    m.close()

