"""Build matched (oracle, CUDA) systems from the same seeded inputs."""
import numpy as np

import oracle as O
from paper_1012_5082_gb300 import inputs as I


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


def compare_obs(o_orc, o_gpu, exact=("n_b", "trials", "local_accepts", "global_trials",
                                     "global_accepts", "flips")):
    for k in exact:
        assert o_orc[k] == o_gpu[k], (k, o_orc[k], o_gpu[k])
    assert abs(o_orc["energy"] - o_gpu["energy"]) <= 1e-9 * max(1.0, abs(o_orc["energy"]))


def lockstep(orc, g, n_sweeps, steps_per_sweep):
    """Advance both a sweep at a time; species must agree bit for bit unless
    the oracle flagged a near-tie decision in that sweep (then re-sync)."""
    resyncs = 0
    for s in range(n_sweeps):
        ties0 = orc.obs()["near_ties"]
        g.sweep(1)
        orc.parallel_steps(steps_per_sweep)
        tg, to = g.types(), orc.types
        if not np.array_equal(tg, to):
            assert orc.obs()["near_ties"] > ties0, f"sweep {s}: species differ without a flagged tie"
            g.set_types(to)
            resyncs += 1
    return resyncs
