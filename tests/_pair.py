"""Build matched (oracle, CUDA) systems from the same seeded inputs, and step
them in lockstep."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle as O
from paper_1012_5082_gb300 import inputs as I

# Near-tie decisions (|u - p| <= 1e-9 p, where the host's and the device's
# exp may round differently) a lockstep test tolerates before it fails.
MAX_TIES = 3

EXACT = ("n_b", "trials", "local_accepts", "global_trials", "global_accepts", "flips")
COUNTERS = ("trials", "local_accepts", "global_trials", "global_accepts", "flips")


def c0_config(n_cells=10, frac_b=0.05, seed_types=1000, dens_b=1.0):
    """The 10x10x10 BCC parity workload: 5% B placed uniformly at random,
    synthetic Morse/exponential/sqrt EAM tabulated on 5000-point grids."""
    lat = I.bcc_lattice(n_cells, n_cells, n_cells)
    types = I.random_types(lat.n, int(round(frac_b * lat.n)), seed=seed_types)
    tab = I.eam_tables(I.EAMParams(dens_scale=(1.0, dens_b)))
    return lat, types, tab


def make_pair(lat, types, tab, phi, kappa, T, *, c0, seed, schedule, sched, kappa_units=0):
    """schedule: 'blocks' (block, colours), 'sublattice' (period), 'overlap'
    (cell, gap) or 'spatial' (boxes, colours)."""
    from paper_1012_5082_gb300 import vcsgc as V

    orc = O.System(lat, types, tab)
    orc.set_params(phi, kappa, T, kappa_units=kappa_units, c0=c0, seed=seed)
    if schedule == "blocks":
        orc.schedule_blocks(lat.cells, sched[:3], sched[3:])
        kind = V.SCHED_BLOCKS
    elif schedule == "sublattice":
        orc.schedule_sublattice(lat.cells, sched[:3])
        kind = V.SCHED_SUBLATTICE
    elif schedule == "overlap":
        orc.schedule_overlap(lat.cells, sched[:3], sched[3:])
        kind = V.SCHED_OVERLAP
    else:
        orc.schedule_spatial(sched[:3], sched[3:])
        kind = V.SCHED_SPATIAL
    gpu = V.Context(lat, types, tab, phi, kappa, T, seed=seed, c0=c0, kappa_units=kappa_units,
                    schedule=kind, sched=tuple(sched))
    return orc, gpu


def compare_obs(o_orc, o_gpu, exact=EXACT):
    for k in exact:
        assert o_orc[k] == o_gpu[k], (k, o_orc[k], o_gpu[k])
    assert abs(o_orc["energy"] - o_gpu["energy"]) <= 1e-9 * max(1.0, abs(o_orc["energy"]))


class Lockstep:
    """A GPU context (or batch) with R replicas beside R oracle chains started
    from the same species and keys.  advance() runs n colour steps on both
    (the oracles in threads: ctypes releases the GIL) and compares every
    replica: species bit for bit, B count and energy, and the increments of
    the step counters exactly.  A replica whose species differ must have had
    a near tie flagged by its oracle in that interval; it is then re-synced
    (species from the oracle, counters of that interval not compared) and
    the comparison goes on.  More than max_ties flagged ties fail the test."""

    def __init__(self, orcs, g, max_ties=MAX_TIES, on_resync=None):
        self.orcs, self.g, self.max_ties = list(orcs), g, max_ties
        self.on_resync = on_resync
        self.resyncs = 0
        self.compared = 0
        self._synced = [True] * len(self.orcs)  # never re-synced: whole histories equal
        self._prev = [(o.obs(), g.observables(r)) for r, o in enumerate(self.orcs)]
        self._pool = ThreadPoolExecutor(max_workers=min(8, len(self.orcs)))

    def ties(self):
        return sum(o.obs()["near_ties"] for o in self.orcs)

    def advance(self, steps, gpu_run=None):
        (gpu_run or (lambda: self.g.steps(steps)))()
        list(self._pool.map(lambda o: o.parallel_steps(steps), self.orcs))
        for r, o in enumerate(self.orcs):
            oo, og = o.obs(), self.g.observables(r)
            po, pg = self._prev[r]
            to, tg = o.types, self.g.types(r)
            if not np.array_equal(to, tg):
                assert oo["near_ties"] > po["near_ties"], f"replica {r}: species differ without a flagged tie"
                self.g.set_types(to, r)
                if self.on_resync:
                    self.on_resync(r, o)
                self.resyncs += 1
                self._synced[r] = False
                og = self.g.observables(r)
            else:
                assert oo["n_b"] == og["n_b"], (r, oo["n_b"], og["n_b"])
                if oo["near_ties"] == po["near_ties"]:
                    for k in COUNTERS:
                        assert oo[k] - po[k] == og[k] - pg[k], (r, k, oo[k] - po[k], og[k] - pg[k])
                    self.compared += 1
            assert abs(oo["energy"] - og["energy"]) <= 1e-9 * max(1.0, abs(oo["energy"])), \
                (r, oo["energy"], og["energy"])
            if self._synced[r] and og["steps"]:
                # <c> over the steps (Sec. II C observables): the same sum of
                # n / N after every step, up to the summation's rounding
                assert abs(og["mean_c"] * og["steps"] - oo["sum_c"]) <= 1e-12 * max(1.0, oo["sum_c"]), \
                    (r, og["mean_c"] * og["steps"], oo["sum_c"])
            self._prev[r] = (oo, og)
        assert self.ties() <= self.max_ties, f"{self.ties()} near ties (at most {self.max_ties} allowed)"

    def close(self):
        self._pool.shutdown()


def lockstep(orc, g, n_sweeps, steps_per_sweep, max_ties=MAX_TIES):
    """One replica a sweep at a time (see Lockstep); returns the re-syncs."""
    ls = Lockstep([orc], g, max_ties)
    for _ in range(n_sweeps):
        ls.advance(steps_per_sweep)
    ls.close()
    return ls.resyncs
