"""The colour step at the launch shapes the benchmark times, against the CPU
oracle (GPU only).

Each replica of the benchmark's 80^3 lattice trials 8,000 sites per colour
step, spread over many thread blocks: the dn reduction crosses blocks through
atomics, and the deferred commit of step k-1 runs in every block while other
blocks already read the effective species of step k (Sec. III B 2, the
composite move of Eqs. trans_vcsgc_par1/par2).  These tests step that launch
against the oracle a sweep at a time, species bit for bit and counters
exactly (tests/_pair.py: Lockstep)."""
import numpy as np
import pytest

import oracle as O
from paper_1012_5082_gb300 import inputs as I
from _pair import Lockstep
from test_oracle_pins import PHILOX_KAT

pytestmark = pytest.mark.gpu

KB = I.KB_EV
T_K, KAPPA = 600.0, 1000.0
DMU0 = -2.02  # eV, the benchmark's local driving force
C0 = 0.02 + np.arange(8) * 0.48 / 7
PHI = DMU0 - 2.0 * KAPPA * KB * T_K * C0
SHAPES = [(64, 1), (128, 1), (256, 1), (64, 0), (128, 0), (256, 0)]


@pytest.fixture(scope="module")
def V():
    from paper_1012_5082_gb300 import vcsgc
    return vcsgc


def _pair(V, cells, reps, seed_types, seeds):
    lat = I.bcc_lattice(cells, cells, cells)
    types = I.random_types(lat.n, int(round(0.02 * lat.n)), seed=seed_types)
    tab = I.eam_tables()
    R = len(reps)
    g = V.Context(lat, np.tile(types, R), tab, 0.0, KAPPA, T_K, schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4),
                  n_replicas=R, phi_r=PHI[reps], c0_r=C0[reps], seed_r=np.array(seeds, dtype=np.uint64))
    orcs = []
    for q, r in enumerate(reps):
        o = O.System(lat, types, tab)
        o.set_params(float(PHI[r]), KAPPA, T_K, c0=float(C0[r]), seed=int(seeds[q]))
        o.schedule_sublattice(lat.cells, (4, 4, 4))
        orcs.append(o)
    return lat, g, orcs


def test_device_philox_known_answers(V):
    """The device generator reproduces the published Philox4x32-10
    known-answer vectors (Salmon et al., SC'11), and equals the oracle's on
    a million counters laid out as the colour step draws them."""
    ctr = np.array([c for c, _, _ in PHILOX_KAT], dtype=np.uint32)
    key = np.array([k for _, k, _ in PHILOX_KAT], dtype=np.uint32)
    want = np.array([w for _, _, w in PHILOX_KAT], dtype=np.uint32)
    assert np.array_equal(V.vcsgc_philox(ctr, key), want)
    rng = np.random.default_rng(11)
    n = 1 << 20
    c = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    c[:, 3] = rng.integers(0, 6, size=n)  # the stream tags in use
    k = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    got = V.vcsgc_philox(c, k)
    for q in rng.choice(n, 2000, replace=False):
        assert np.array_equal(got[q], O.philox(c[q], k[q])), q


def test_multiblock_40cubed_8_replicas(V):
    """40^3 cells x 8 replicas at the benchmark's kappa, T and phi grid: 1,000
    trials per replica per colour step (4 to 16 blocks each, by shape), 20
    sweeps.  The launch shape changes every sweep through all six shapes."""
    lat, g, orcs = _pair(V, 40, list(range(8)), 1001, [3000 + r for r in range(8)])
    spw = g.steps_per_sweep
    assert spw == 128 and lat.n // 128 == 1000
    ls = Lockstep(orcs, g)
    for s in range(20):
        g.set_launch(0, *SHAPES[s % len(SHAPES)])
        ls.advance(spw)
    flips = [g.observables(r)["flips"] for r in range(8)]
    assert min(flips) > 0 and sum(flips) > 10000, flips
    assert ls.compared >= 8 * 20 - 8 * ls.max_ties
    ls.close()
    g.close()


def test_full_size_80cubed_every_launch_shape(V):
    """The benchmark's lattice (80^3, 8,000 trials per replica per colour
    step) with its replicas 0 and 1 (c0 = 0.02 and 0.089): one sweep under
    each of the autotuner's six launch shapes, compared after each."""
    lat, g, orcs = _pair(V, 80, [0, 1], 1001, [2001, 2002])
    spw = g.steps_per_sweep
    ls = Lockstep(orcs, g)
    for shape in SHAPES:
        g.set_launch(0, *shape)
        assert g.get_launch() == (0,) + shape
        ls.advance(spw)
    o = [g.observables(r) for r in range(2)]
    assert o[0]["global_accepts"] > 0 and o[1]["flips"] > 1000, o
    ls.close()
    g.close()


def test_autotune_keeps_the_chain_exact_80cubed(V):
    """The autotuner's timed steps are real steps of the chain: after it, the
    species equal the oracle's, and a sweep at the chosen shape stays exact."""
    lat, g, orcs = _pair(V, 80, [1], 1001, [2002])
    steps = 16
    g.autotune(steps)
    ran = g.observables(0)["steps"]  # 1 + 16 steps per candidate shape
    assert ran >= len(SHAPES) * (1 + steps) and ran % (1 + steps) == 0
    orcs[0].parallel_steps(ran)
    assert np.array_equal(g.types(0), orcs[0].types)
    ls = Lockstep(orcs, g)
    ls.advance(g.steps_per_sweep)
    ls.close()
    g.close()


def test_set_launch_rejects_bad_shapes(V):
    lat = I.bcc_lattice(8, 8, 8)
    g = V.Context(lat, I.random_types(lat.n, 20, seed=1), I.eam_tables(), -2.0, KAPPA, T_K,
                  schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4))
    for bad in ((0, 96, 1), (0, 128, 2), (7, 128, 1)):
        with pytest.raises(V.VcsgcError) as e:
            g.set_launch(*bad)
        assert e.value.code == -1
    g.close()


# ----------------------------------------- the cluster-resident form (1)
def _cluster_shapes(g):
    return [(1, b, s) for s in g.cluster_sizes() for b in (512, 256)]


def test_cluster_form_80cubed(V):
    """The benchmark's lattice in the cluster-resident form: one sweep per
    (cluster size, block) the lattice allows, replicas 0 and 1, against the
    oracle after each."""
    lat, g, orcs = _pair(V, 80, [0, 1], 1001, [2001, 2002])
    shapes = _cluster_shapes(g)
    assert (1, 512, 16) in shapes
    ls = Lockstep(orcs, g)
    for shape in shapes:
        g.set_launch(*shape)
        assert g.get_launch() == shape
        ls.advance(g.steps_per_sweep)
    o = [g.observables(r) for r in range(2)]
    assert o[0]["global_accepts"] > 0 and o[1]["flips"] > 1000, o
    ls.close()
    g.close()


def test_cluster_form_40cubed_8_replicas(V):
    """40^3 x 8 replicas: every cluster size from 1 (the whole replica in one
    CTA) to 16, 12 sweeps, against the oracle after each."""
    lat, g, orcs = _pair(V, 40, list(range(8)), 1001, [3000 + r for r in range(8)])
    shapes = _cluster_shapes(g)
    assert {s for _, _, s in shapes} == {1, 2, 4, 8, 16}
    ls = Lockstep(orcs, g)
    for s in range(12):
        g.set_launch(*shapes[s % len(shapes)])
        ls.advance(g.steps_per_sweep)
    assert min(g.observables(r)["flips"] for r in range(8)) > 0
    ls.close()
    g.close()


def test_cluster_form_uneven_batch(V):
    """Replicas of different sizes in one launch, tiles of 2 and 3 rows, tiles
    that are not whole sublattice periods, and (cluster size 1 on 8^3) a tile
    whose halo wraps onto its own rows: every size, 6 sweeps each in turn."""
    cells = [(8, 8, 8), (12, 12, 12), (16, 8, 12)]
    phi, T, seeds = [-2.45, -2.40, -2.50], [700.0, 650.0, 750.0], [11, 12, 13]
    tab = I.eam_tables()
    lats = [I.bcc_lattice(*c) for c in cells]
    types = [I.random_types(l.n, l.n // 20, seed=100 + q) for q, l in enumerate(lats)]
    b = V.Batch(cells, types, tab, phi, 20.0, T, seed_r=np.array(seeds, np.uint64), c0=0.05)
    orcs = []
    for q, l in enumerate(lats):
        o = O.System(l, types[q], tab)
        o.set_params(phi[q], 20.0, T[q], c0=0.05, seed=seeds[q])
        o.schedule_sublattice(l.cells, (4, 4, 4))
        orcs.append(o)
    assert b.cluster_sizes() == [1, 2, 4, 8, 16]
    ls = Lockstep(orcs, b)
    for s in (1, 2, 4, 8, 16):
        b.set_launch(1, 512, s)
        ls.advance(6 * 128)
    assert min(b.observables(q)["flips"] for q in range(3)) > 0
    ls.close()
    b.close()


def test_forms_interleave_mid_sweep(V):
    """The chain passes between the per-step and the cluster-resident forms at
    arbitrary steps (pending commits, step base and colour table handed over):
    13, 70, 45 and 128 steps alternating."""
    lat, g, orcs = _pair(V, 40, [1, 2], 1001, [3001, 3002])
    ls = Lockstep(orcs, g)
    for shape, steps in (((0, 128, 1), 13), ((1, 512, 16), 70), ((0, 256, 0), 45), ((1, 256, 4), 128),
                         ((0, 64, 1), 77)):
        g.set_launch(*shape)
        ls.advance(steps)
    o = g.observables(0)
    assert o["steps"] == 13 + 70 + 45 + 128 + 77
    ls.close()
    g.close()


def test_cluster_form_energy_and_observables(V):
    """After cluster-resident sweeps the tracked energy equals a fresh
    evaluation, the B count equals the species, and <c> sums are the
    oracle's."""
    lat, g, orcs = _pair(V, 40, [3], 1001, [3003])
    g.set_launch(1, 512, 16)
    g.sweep(5)
    orcs[0].parallel_steps(5 * 128)
    og, oo = g.observables(0), orcs[0].obs()
    assert np.array_equal(g.types(0), orcs[0].types)
    assert og["n_b"] == oo["n_b"] == int(g.types(0).sum())
    assert abs(g.energy(0) - og["energy"]) <= 1e-9 * abs(og["energy"])
    assert abs(og["mean_c"] * og["steps"] - oo["sum_c"]) <= 1e-9 * oo["sum_c"]
    g.close()
