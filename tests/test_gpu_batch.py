"""Batched replicas of different lattice sizes in one context (one launch
per colour step) against independent oracle chains (GPU only)."""
import numpy as np
import pytest

import oracle as O
from paper_1012_5082_gb300 import inputs as I
from _pair import Lockstep

pytestmark = pytest.mark.gpu

CELLS = [(8, 8, 8), (12, 12, 12), (16, 8, 12)]
PHI = [-2.45, -2.40, -2.50]
T = [700.0, 650.0, 750.0]
SEEDS = [11, 12, 13]


@pytest.fixture(scope="module")
def V():
    from paper_1012_5082_gb300 import vcsgc
    return vcsgc


def _start():
    tab = I.eam_tables()
    lats = [I.bcc_lattice(*c) for c in CELLS]
    types = [I.random_types(l.n, l.n // 20, seed=100 + q) for q, l in enumerate(lats)]
    return tab, lats, types


def _oracles(tab, lats, types, steps=0):
    out = []
    for q, l in enumerate(lats):
        o = O.System(l, types[q], tab)
        o.set_params(PHI[q], 20.0, T[q], c0=0.05, seed=SEEDS[q])
        o.schedule_sublattice(l.cells, (4, 4, 4))
        if steps:
            o.parallel_steps(steps)
        out.append(o)
    return out


def test_batch_of_uneven_lattices_matches_oracles(V):
    tab, lats, types = _start()
    b = V.Batch(CELLS, types, tab, PHI, 20.0, T, seed_r=np.array(SEEDS, np.uint64), c0=0.05)
    ls = Lockstep(_oracles(tab, lats, types), b)
    for _ in range(3):
        ls.advance(5 * 128)
    for q in range(len(CELLS)):
        og = b.observables(q)
        assert og["steps"] == 15 * 128
        assert og["flips"] > 0
    # the batch's own energy evaluation agrees with the tracked energy
    assert abs(b.energy(1) - b.observables(1)["energy"]) <= 1e-9 * abs(b.energy(1))
    ls.close()
    b.close()


def test_autotune_keeps_the_chain_exact(V):
    tab, lats, types = _start()
    b = V.Batch(CELLS, types, tab, PHI, 20.0, T, seed_r=np.array(SEEDS, np.uint64), c0=0.05)
    best = b.autotune(steps=16)
    assert best in (64, 128, 256)
    # every candidate shape (form 0: 3 block sizes x row prefetch on/off;
    # form 1: the cluster sizes x 2 block sizes) runs 1 + 16 steps
    ran = b.observables(0)["steps"]
    assert ran >= 6 * (1 + 16) and ran % (1 + 16) == 0
    orcs = _oracles(tab, lats, types, ran)
    for q, o in enumerate(orcs):
        assert np.array_equal(b.types(q), o.types), q
    ls = Lockstep(orcs, b)
    ls.advance(2 * 128)
    ls.close()
    b.close()


def test_batch_set_types_and_delta_e(V):
    tab, lats, types = _start()
    b = V.Batch(CELLS, types, tab, PHI, 20.0, T, seed_r=np.array(SEEDS, np.uint64), c0=0.05)
    t2 = I.random_types(lats[2].n, lats[2].n // 3, seed=7)
    b.set_types(t2, 2)
    assert np.array_equal(b.types(2), t2)
    o = O.System(lats[2], t2, tab)
    sites = np.arange(0, lats[2].n, 5)
    assert np.max(np.abs(b.delta_e(sites, 2) - np.array([o.delta_e(i) for i in sites]))) < 1e-11
    assert abs(b.observables(2)["energy"] - o.energy_full()) < 1e-9 * abs(o.energy_full())
    b.close()


def test_all_replica_species_and_observables(V):
    """The all-replica calls equal the per-replica ones: species back to back,
    energies and counts against the oracle after set_types_all."""
    tab, lats, types = _start()
    b = V.Batch(CELLS, types, tab, PHI, 20.0, T, seed_r=np.array(SEEDS, np.uint64), c0=0.05)
    b.sweep(2)
    allt = b.types_all()
    off = 0
    for q, l in enumerate(lats):
        assert np.array_equal(allt[off:off + l.n], b.types(q))
        off += l.n
    new = [I.random_types(l.n, l.n // 3 + q, seed=90 + q) for q, l in enumerate(lats)]
    b.set_types_all(np.concatenate(new))
    obs = b.observables_all()
    for q, l in enumerate(lats):
        o = O.System(l, new[q], tab)
        assert obs[q] == b.observables(q)
        assert obs[q]["n_b"] == int(new[q].sum())
        assert abs(obs[q]["energy"] - o.energy_full()) <= 1e-12 * abs(o.energy_full())
        assert np.array_equal(b.types(q), new[q])
    bad = np.concatenate(new)
    bad[3] = 7
    with pytest.raises(V.VcsgcError):
        b.set_types_all(bad)
    assert np.array_equal(b.types_all(), np.concatenate(new))
    b.close()
