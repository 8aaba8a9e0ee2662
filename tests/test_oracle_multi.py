"""Pins of the multicomponent oracle (the K-species generalisation of the
parallel transmutation step, Sec. II and Sec. III B 2 applied per solute):
K = 2 reproduces the binary oracle's chain step for step; pure and dilute
energies match closed forms of the analytic functions; the incremental
energy change equals full recomputation for every target species; and the
sampled joint distribution of the solute counts equals exact enumeration of
an 8-site cell for K = 3 (3^8 states) and K = 4 (4^8 states)."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_1012_5082_gb300 import inputs as I

A = 2.855
KB = I.KB_EV
SHELLS = [(A * math.sqrt(3) / 2, 8), (A, 6), (A * math.sqrt(2), 12), (A * math.sqrt(11) / 2, 24),
          (A * math.sqrt(3), 8)]


@pytest.mark.parametrize("dens_b,phi", [(1.0, -3.0), (1.25, -2.4)])
def test_k2_reduces_to_binary_chain(dens_b, phi):
    """With K = 2 the species draw is not taken and both stages reduce to
    the binary rules: 8^3 cells, period-4 sublattice, phi near the balance of
    the dilute dE at 1200 K (with and without re-embedding), 40 sweeps give
    the same species after every sweep, the same counters and the same
    energy."""
    lat = I.bcc_lattice(8, 8, 8)
    types = I.random_types(lat.n, int(0.05 * lat.n), seed=41)
    p2 = I.multi_eam_params(2, dens_scale=(1.0, dens_b))
    tab = I.eam_tables(p2)
    assert p2.pair_scale == I.EAMParams().pair_scale and p2.A_embed == I.EAMParams().A_embed
    b = O.System(lat, types, tab, brute=True)
    m = O.MultiSystem(lat, types, tab)
    b.set_params(phi, 100.0, 1200.0, kappa_units=0, c0=0.05, seed=99)
    m.set_params([phi], [100.0], 1200.0, c0=[0.05], seed=99)
    b.schedule_sublattice(lat.cells, (4, 4, 4))
    m.schedule_sublattice(lat.cells, (4, 4, 4))
    spw = lat.n // (lat.n // 128)
    for _ in range(40):
        b.parallel_steps(spw)
        m.parallel_steps(spw)
        assert np.array_equal(b.types, m.types)
    ob, om = b.obs(), m.obs()
    for k in ("trials", "local_accepts", "global_trials", "global_accepts", "flips"):
        assert ob[k] == om[k], k
    assert ob["n_b"] == om["n"][1] and om["n"][0] + om["n"][1] == lat.n
    assert ob["energy"] == om["energy"]
    assert ob["flips"] > 1000


def _pure(p, a):
    """E/N of a perfect lattice of species a from the closed forms."""
    q = p.pair_scale and [(x, y) for x in range(len(p.A_embed)) for y in range(x, len(p.A_embed))].index((a, a))
    pair = sum(z * p.pair(q, r)[0] for r, z in SHELLS)
    rho = sum(z * p.dens(a, r)[0] for r, z in SHELLS)
    return 0.5 * pair + p.embed(a, rho)[0], rho


def _pidx(K, a, b):
    a, b = min(a, b), max(a, b)
    return [(x, y) for x in range(K) for y in range(x, K)].index((a, b))


def test_pure_and_dilute_closed_forms():
    """K = 3 with species-dependent densities on 6^3 cells: E/N of each pure
    crystal is 1/2 sum_s z_s phi_aa(r_s) + F_a(rho_a); one site of a pure-a
    crystal becoming b costs sum_s z_s [phi_ab - phi_aa](r_s) + F_b(rho_a) -
    F_a(rho_a) + sum_s z_s [F_a(rho_a + f_b(r_s) - f_a(r_s)) - F_a(rho_a)]
    (re-embedding of the 58 neighbours)."""
    K = 3
    p = I.multi_eam_params(K, dens_scale=(1.0, 1.25, 0.85))
    tab = I.eam_tables(p)
    lat = I.bcc_lattice(6, 6, 6)
    for a in range(K):
        s = O.MultiSystem(lat, np.full(lat.n, a, np.uint8), tab)
        e_pure, rho_a = _pure(p, a)
        assert abs(s.energy_full() / lat.n - e_pure) < 2e-6, (a, s.energy_full() / lat.n, e_pure)
        assert np.allclose(s.rho(), rho_a, rtol=1e-6)
        for b in range(K):
            if b == a:
                assert s.delta_e(0, b) == 0.0
                continue
            de = sum(z * (p.pair(_pidx(K, a, b), r)[0] - p.pair(_pidx(K, a, a), r)[0]) for r, z in SHELLS)
            de += p.embed(b, rho_a)[0] - p.embed(a, rho_a)[0]
            de += sum(z * (p.embed(a, rho_a + p.dens(b, r)[0] - p.dens(a, r)[0])[0] - p.embed(a, rho_a)[0])
                      for r, z in SHELLS)
            assert abs(s.delta_e(0, b) - de) < 2e-5, (a, b, s.delta_e(0, b), de)


@pytest.mark.parametrize("K", [3, 4])
def test_incremental_delta_e_equals_full_recompute(K):
    """Random K-species configurations with species-dependent densities:
    the incremental change equals the difference of two full energies for
    every target species, and applying it keeps the tracked energy."""
    p = I.multi_eam_params(K, dens_scale=(1.0, 1.25, 0.85, 1.1)[:K])
    tab = I.eam_tables(p)
    lat = I.bcc_lattice(4, 4, 4)
    counts = [lat.n // (K + 1)] * (K - 1)
    s = O.MultiSystem(lat, I.multi_random_types(lat.n, counts, seed=5 + K), tab)
    rng = np.random.default_rng(K)
    for i in rng.choice(lat.n, 6, replace=False):
        for b in range(K):
            d1, d2 = s.delta_e(i, b), s.delta_e_full(i, b)
            assert abs(d1 - d2) < 1e-9 * max(1.0, abs(d2)), (i, b, d1, d2)


def _enumerate(s, K, n, beta, phi, kappa_p):
    """Exact joint P(n_1..n_{K-1}) and <E> under the K-species pi_V."""
    states = np.array(list(itertools.product(range(K), repeat=n)), dtype=np.uint8)
    U = np.empty(len(states))
    for k, st in enumerate(states):
        s.set_types(st)
        U[k] = s.energy_full()
    cnt = np.stack([(states == a).sum(1) for a in range(1, K)], 1)
    logw = -beta * (U + cnt @ np.asarray(phi) + (cnt ** 2) @ np.asarray(kappa_p))
    w = np.exp(logw - logw.max())
    w /= w.sum()
    P = np.zeros((n + 1,) * (K - 1))
    np.add.at(P, tuple(cnt.T), w)
    return P, float((w * U).sum())


ENUM = [
    # K, phi, kappa (units of kT/N), c0
    (3, [-1.3, -1.2], [2.0, 1.0], [0.8, 0.1]),
    (4, [-1.3, -1.2, 0.3], [2.0, 1.0, 0.5], [0.1, 0.6, 0.3]),
]


@pytest.mark.parametrize("case", ENUM, ids=["K3", "K4"])
def test_chain_matches_exact_enumeration(case):
    """8 sites (4x1x1 BCC cells, first-shell cutoff, species-dependent
    densities so re-embedding enters), period-2 sublattice along x: two
    simultaneous trials per step 5.7 A > 2 r_c apart.  c0 far from <c> so a
    wrong sign or factor in either stage shifts the result.  Marginals and
    (K = 3) the joint distribution of the solute counts, <n_alpha> and <E>
    agree with the exact pi_V."""
    K, phi, kappa, c0 = case
    p = I.multi_eam_params(K, dens_scale=(1.0, 1.2, 0.9, 1.1)[:K], rc=2.6, r_in=2.55, nr=2000)
    tab = I.eam_tables(p)
    lat = I.bcc_lattice(4, 1, 1)
    n = lat.n
    T = 2000.0
    beta = 1.0 / (KB * T)
    kappa_p = [k * KB * T / n for k in kappa]
    s = O.MultiSystem(lat, np.zeros(n, np.uint8), tab)
    P, Emean = _enumerate(s, K, n, beta, phi, kappa_p)
    s.set_types(np.zeros(n, np.uint8))
    s.set_params(phi, kappa, T, c0=c0, seed=2026)
    s.schedule_sublattice(lat.cells, (2, 1, 1))
    s.run_histogram(5000)
    blocks, e_blocks = [], []
    H = np.zeros_like(P)
    for _ in range(20):
        h, e = s.run_histogram(20000)
        H += h
        ax = np.arange(n + 1)
        blocks.append([(h.sum(axis=tuple(q for q in range(K - 1) if q != a)) * ax).sum() / h.sum()
                       for a in range(K - 1)])
        e_blocks.append(e)
    Pc = H / H.sum()
    blocks = np.array(blocks)
    for a in range(K - 1):
        other = tuple(q for q in range(K - 1) if q != a)
        marg, marg_c = P.sum(axis=other), Pc.sum(axis=other)
        mean_exact = (marg * np.arange(n + 1)).sum()
        err = blocks[:, a].std(ddof=1) / math.sqrt(len(blocks))
        assert abs(blocks[:, a].mean() - mean_exact) < 5 * err + 0.02, (a, blocks[:, a].mean(), mean_exact, err)
        assert 0.5 * np.abs(marg - marg_c).sum() < 0.03, (a, marg, marg_c)
        assert marg.max() < 0.6
    if K == 3:
        assert 0.5 * np.abs(P - Pc).sum() < 0.04
    e_err = float(np.std(e_blocks, ddof=1) / math.sqrt(len(e_blocks)))
    assert abs(np.mean(e_blocks) - Emean) < 5 * e_err + 1e-3, (np.mean(e_blocks), Emean, e_err)
    o = s.obs()
    assert 0.05 * o["trials"] < o["local_accepts"] < o["trials"]
    assert o["global_accepts"] < o["global_trials"]
