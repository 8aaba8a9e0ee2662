"""The Ising-type lattice gas of Sec. II B through the same CUDA kernels
(a two-shell pair table, no density or embedding): bit-exact trajectories
against the oracle, the parallel acceptance against the oracle's, and the
relation <c> = c0 at dmu0 = dmu (Sec. III C)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1012_5082_gb300 import inputs as I
from _pair import compare_obs, lockstep

pytestmark = pytest.mark.gpu
T_ISING = 1000.0  # k_B T = 0.8617 U, U = 0.1 eV


@pytest.fixture(scope="module")
def V():
    from paper_1012_5082_gb300 import vcsgc
    return vcsgc


@pytest.fixture(scope="module")
def tab():
    return I.ising_tables()


def _pair(V, tab, cells, block, colours, kappa, c0, seed, start_b):
    lat = I.bcc_lattice(*cells)
    types = I.random_types(lat.n, start_b, seed=seed)
    kT = I.KB_EV * T_ISING
    phi = -2.0 * kappa * kT * c0  # dmu0 = 0
    orc = O.System(lat, types, tab)
    orc.set_params(phi, kappa, T_ISING, c0=c0, seed=seed + 1)
    orc.schedule_blocks(cells, block, colours)
    g = V.Context(lat, types, tab, phi, kappa, T_ISING, seed=seed + 1, c0=c0, schedule=V.SCHED_BLOCKS,
                  sched=tuple(block) + tuple(colours))
    return lat, orc, g


def test_ising_trajectory_bit_exact(V, tab):
    """10^3 cells, 5-cell blocks in 8 colours, c0 = 0.5: 100 sweeps agree
    site for site (the two-shell neighbourhood runs the runtime-mask form of
    the fused step)."""
    lat, orc, g = _pair(V, tab, (10, 10, 10), (5, 5, 5), (2, 2, 2), 100.0, 0.5, 40, 1000)
    spw = g.steps_per_sweep
    resyncs = lockstep(orc, g, 100, spw)
    if resyncs == 0:
        compare_obs(orc.obs(), g.observables())
    assert g.observables()["flips"] > 50000
    assert abs(g.energy() - g.observables()["energy"]) <= 1e-9 * abs(g.energy())
    g.close()


def test_ising_parallel_acceptance_matches_oracle(V, tab):
    """The paper's parallel set-up (40^3 cells, 64 domains of 10^3 cells
    split into octants, one trial per domain per step) at kappa = 1000:
    10 sweeps bit-exact, and the acceptance (flips per trial) the same."""
    lat, orc, g = _pair(V, tab, (40, 40, 40), (5, 5, 5), (2, 2, 2), 1000.0, 0.5, 50, 64000)
    spw = g.steps_per_sweep
    assert spw == lat.n // 64
    resyncs = lockstep(orc, g, 10, spw)
    og, oo = g.observables(), orc.obs()
    if resyncs == 0:
        compare_obs(oo, og)
    acc = og["flips"] / og["trials"]
    assert 0.25 < acc < 0.45, acc
    g.close()


def _window_c(V, tab, c0, dmu0, kappa=100.0, R=16, warm=100, sweeps=300, seed=900):
    """Window mean of c per replica (12^3 cells, period-4 sublattice)."""
    lat = I.bcc_lattice(12, 12, 12)
    kT = I.KB_EV * T_ISING
    types = [I.random_types(lat.n, int(round(c0 * lat.n)), seed=700 + q) for q in range(R)]
    b = V.Batch([(12, 12, 12)] * R, types, tab, dmu0 - 2.0 * kappa * kT * c0, kappa, T_ISING,
                seed_r=np.arange(R, dtype=np.uint64) + seed, c0=c0)
    b.sweep(warm)
    s0 = b.observables_all()
    b.sweep(sweeps)
    s1 = b.observables_all()
    b.close()
    c = np.array([(s1[q]["mean_c"] * s1[q]["steps"] - s0[q]["mean_c"] * s0[q]["steps"])
                  / (s1[q]["steps"] - s0[q]["steps"]) for q in range(R)])
    return c.mean(), c.std(ddof=1) / math.sqrt(R)


def test_ising_c_equals_c0_at_dmu(V, tab):
    """Sec. III C (Eq. c0): <c> = c0 exactly when dmu0 equals the driving force
    dmu = phi + 2 kappa_p N <c> (Eq. gforce).  At c0 = 1/2 that force is 0 by
    A <-> B symmetry.  Inside the miscibility gap (c0 = 1/4) the finite
    system's van der Waals loop makes it nonzero: a run at dmu0 = 0 measures
    it, and a run at dmu0 = that value returns <c> = c0.  Near c0, <c> moves
    by -(dmu0 - dmu) / (2 kappa_p N) (kappa_p N = kappa k_B T)."""
    kappa = 100.0
    kT = I.KB_EV * T_ISING
    m, e = _window_c(V, tab, 0.5, 0.0, kappa)
    assert abs(m - 0.5) < 5 * e + 1e-4, (m, e)
    c0 = 0.25
    m0, e0 = _window_c(V, tab, c0, 0.0, kappa)
    dmu = 2.0 * kappa * kT * (m0 - c0)  # phi + 2 kappa_p N <c> at dmu0 = 0
    m1, e1 = _window_c(V, tab, c0, dmu, kappa, seed=1900)
    assert abs(m1 - c0) < 5 * e1 + 0.2 * abs(m0 - c0) + 2e-5, (m0, m1, e1, dmu)
    mp, ep = _window_c(V, tab, c0, dmu + 0.02, kappa, seed=2900)
    shift = -0.02 / (2.0 * kappa * kT)
    assert abs((mp - m1) - shift) < 0.2 * abs(shift) + 5 * math.hypot(ep, e1), (m1, mp, shift)


def test_ising_van_der_waals_loop(V, tab):
    """Inside the miscibility gap the constraint holds the system at any mean
    concentration, so dmu(c) = phi + 2 kappa_p N <c> (Eq. gforce) traces the
    finite system's van der Waals loop instead of jumping across the gap
    (Sec. III C): falling from the dilute side, it overshoots below the
    coexistence value 0 near c = 0.2 and turns back up to 0 at c = 1/2 (A <-> B
    symmetry).  16^3 cells, kappa = 1000, 8 replicas per c0 in one batch."""
    kappa, L, S = 1000.0, 16, 8
    kT = I.KB_EV * T_ISING
    c0s = np.array([0.10, 0.20, 0.40, 0.50])
    c0r = np.repeat(c0s, S)
    R = len(c0r)
    lat = I.bcc_lattice(L, L, L)
    types = [I.random_types(lat.n, int(round(c * lat.n)), seed=3000 + q) for q, c in enumerate(c0r)]
    b = V.Batch([(L, L, L)] * R, types, tab, -2.0 * kappa * kT * c0r, kappa, T_ISING,
                seed_r=np.arange(R, dtype=np.uint64) + 3100, c0_r=c0r)
    b.sweep(500)
    s0 = b.observables_all()
    b.sweep(1000)
    s1 = b.observables_all()
    b.close()
    c = np.array([(s1[q]["mean_c"] * s1[q]["steps"] - s0[q]["mean_c"] * s0[q]["steps"])
                  / (s1[q]["steps"] - s0[q]["steps"]) for q in range(R)]).reshape(-1, S)
    dmu = 2.0 * kappa * kT * (c - c0s[:, None])
    m = dmu.mean(axis=1)
    e = dmu.std(axis=1, ddof=1) / math.sqrt(S)
    assert m[0] > m[1] + 5 * math.hypot(e[0], e[1]), (m, e)   # falling from the dilute side
    assert m[1] < -5 * e[1], (m, e)                            # below coexistence
    assert m[2] > m[1] + 5 * math.hypot(e[1], e[2]), (m, e)   # and back up: the loop
    assert abs(m[3]) < 5 * e[3] + 2e-4, (m, e)                 # 0 at c = 1/2
