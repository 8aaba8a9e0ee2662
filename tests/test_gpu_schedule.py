"""Colour schedules changed mid-chain, and the schedule autotuner, against
the CPU oracle (GPU only).

Each decomposition of Sec. III A (octant blocks, the period-q sublattice,
overlapping position-weighted domains) gives composite moves that keep pi_V
invariant, so a chain may switch between them at any colour step; the step
counter, and with it the random streams, runs on.  The oracle switches at
the same steps and the species must agree after every interval
(tests/_pair.py: Lockstep)."""
import numpy as np
import pytest

import oracle as O
from paper_1012_5082_gb300 import inputs as I
from _pair import Lockstep

pytestmark = pytest.mark.gpu

SCHEDULES = [  # (name, kind, sched, oracle call)
    ("sublattice", 1, (4, 4, 4, 0, 0, 0), lambda o, cells: o.schedule_sublattice(cells, (4, 4, 4))),
    ("blocks", 0, (4, 4, 4, 2, 2, 2), lambda o, cells: o.schedule_blocks(cells, (4, 4, 4), (2, 2, 2))),
    ("overlap", 3, (8, 8, 8, 4, 4, 4), lambda o, cells: o.schedule_overlap(cells, (8, 8, 8), (4, 4, 4))),
]


@pytest.fixture(scope="module")
def V():
    from paper_1012_5082_gb300 import vcsgc
    return vcsgc


def _pair(V, dens_b, first):
    lat = I.bcc_lattice(16, 16, 16)
    tab = I.eam_tables(I.EAMParams(dens_scale=(1.0, dens_b)))
    t = I.random_types(lat.n, int(0.05 * lat.n), seed=91)
    phis, seeds = [-2.45, -2.35], [911, 912]
    name, kind, sched, ocall = first
    g = V.Context(lat, np.tile(t, 2), tab, 0.0, 20.0, 800.0, c0=0.05, schedule=kind, sched=sched, n_replicas=2,
                  phi_r=np.array(phis), seed_r=np.array(seeds, dtype=np.uint64))
    orcs = []
    for phi, seed in zip(phis, seeds):
        o = O.System(lat, t, tab)
        o.set_params(phi, 20.0, 800.0, c0=0.05, seed=seed)
        ocall(o, lat.cells)
        orcs.append(o)
    return lat, g, orcs


@pytest.mark.parametrize("dens_b", [1.0, 1.25], ids=["fused", "reembed"])
def test_schedule_switches_keep_the_chain_exact(V, dens_b):
    """16^3 x 2 replicas: blocks -> sublattice -> overlapping -> blocks ->
    sublattice, a sweep under each (one density: the fused bit-packed form,
    with its per-schedule tables rebuilt; f_B = 1.25 f_A: the general
    re-embedding kernels)."""
    seq = [SCHEDULES[1], SCHEDULES[0], SCHEDULES[2], SCHEDULES[1], SCHEDULES[0]]
    lat, g, orcs = _pair(V, dens_b, seq[0])
    ls = Lockstep(orcs, g)
    for k, (name, kind, sched, ocall) in enumerate(seq):
        if k:
            g.set_schedule(kind, sched)
            for o in orcs:
                ocall(o, lat.cells)
        ls.advance(g.steps_per_sweep)
    assert min(g.observables(r)["flips"] for r in range(2)) > 100
    ls.close()
    g.close()


def test_schedule_autotune_picks_by_accepted_flips(V):
    """Every candidate runs from the chain's state at the call and the chain
    resumes from that state under the winner: afterwards the species and
    counters are those of the call, and the chain then runs in lockstep with
    the oracle under the winning schedule.  Scores are accepted flips per
    second and the winner has the largest.  Here the sublattice's 64
    simultaneous trials per replica carry a dn that the variance constraint
    rejects, while the octant blocks' 8 trials per step are accepted."""
    lat, g, orcs = _pair(V, 1.0, SCHEDULES[0])
    g.sweep(1)
    for o in orcs:
        o.parallel_steps(128)
    before = [(g.types(r).copy(), g.observables(r)) for r in range(2)]
    cand = [(kind, sched) for _, kind, sched, _ in SCHEDULES]
    best, scores = g.autotune_schedule(cand, sweeps=1)
    assert np.all(scores >= 0) and scores.max() > 0 and best == int(np.argmax(scores))
    assert scores[1] > scores[0]
    for r in range(2):
        assert np.array_equal(g.types(r), before[r][0])
        o = g.observables(r)
        for k in ("steps", "trials", "flips", "n_b"):
            assert o[k] == before[r][1][k], (k, o[k], before[r][1][k])
        assert abs(o["energy"] - before[r][1]["energy"]) <= 1e-9 * abs(o["energy"])
    for o in orcs:
        SCHEDULES[best][3](o, lat.cells)
    ls = Lockstep(orcs, g)
    for _ in range(2):
        ls.advance(g.steps_per_sweep)
    ls.close()
    g.close()


def test_schedule_change_refusals(V):
    lat = I.bcc_lattice(12, 12, 12)
    g = V.Context(lat, I.random_types(lat.n, 50, seed=3), I.eam_tables(), -2.0, 20.0, 700.0,
                  schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4))
    with pytest.raises(V.VcsgcError) as e:
        g.set_schedule(0, (3, 3, 3, 2, 2, 2))  # 3-cell blocks: same-colour sites closer than 2 r_c
    assert e.value.code == -5
    g.sweep(1)  # the old schedule still runs
    assert g.steps_per_sweep == 128
    g.close()
