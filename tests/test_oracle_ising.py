"""Pins of the oracle on the Ising-type lattice gas of Sec. II B: closed
forms of the model, A <-> B symmetry, and the serial VC-SGC acceptance the
paper prints (Sec. III C)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1012_5082_gb300 import inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ising_acceptance.json")))
T_ISING = 1000.0  # k_B T = 0.8617 U with U = 0.1 eV


@pytest.fixture(scope="module")
def model():
    p = I.IsingParams()
    return p, I.ising_tables(p)


def _first_shell_b(s, t, i, a=2.855):
    r1 = a * np.sqrt(3) / 2
    return sum(int(t[j]) for j, r, _ in s.neighbours(i) if abs(r - r1) < 1e-6)


def test_ising_closed_forms(model):
    """Pure A: E/N = 4 eps_AA(1) + 3 eps_AA(2) = -46 U (8 and 6 neighbours, each
    bond shared); flipping an A site with n B first-shell neighbours changes
    E by (8 - n)(eps_AB - eps_AA)(1) + n (eps_BB - eps_AB)(1) = 0.3 U (8 - 2n),
    the second shell cancelling because eps(2) is the same for all pairs."""
    p, tab = model
    lat = I.bcc_lattice(6, 6, 6)
    s = O.System(lat, np.zeros(lat.n, np.uint8), tab)
    assert abs(s.energy_full() / lat.n - (-46.0 * p.U)) < 1e-12
    t = I.random_types(lat.n, lat.n // 3, seed=5)
    s.set_types(t)
    for i in range(0, lat.n, 37):
        n = _first_shell_b(s, t, i)
        want = 0.3 * p.U * (8 - 2 * n)
        assert abs(s.delta_e(i) - (want if t[i] == 0 else -want)) < 1e-12, (i, n)


def test_ising_ab_symmetry(model):
    """eps_AA = eps_BB: a configuration and its complement have equal energy,
    so the coexistence driving force is 0 and <c> = 1/2 at dmu0 = 0."""
    p, tab = model
    lat = I.bcc_lattice(6, 6, 6)
    t = I.random_types(lat.n, 100, seed=6)
    s1 = O.System(lat, t, tab)
    s2 = O.System(lat, (1 - t).astype(np.uint8), tab)
    assert abs(s1.energy_full() - s2.energy_full()) < 1e-9


def _serial_acceptance(tab, kappa, sweeps=150):
    lat = I.bcc_lattice(10, 10, 10)  # the paper's serial system: 2000 sites
    s = O.System(lat, I.random_types(lat.n, lat.n // 2, seed=1), tab)
    kT = I.KB_EV * T_ISING
    s.set_params(-kappa * kT, kappa, T_ISING, kappa_units=0, c0=0.5, seed=3)  # dmu0 = 0
    s.serial_steps(50 * lat.n, mode=0)
    s.reset_counters()
    s.serial_steps(sweeps * lat.n, mode=0)
    o = s.obs()
    return o["flips"] / o["trials"], o["sum_c"] / o["steps"]


def test_serial_acceptance_matches_paper(model):
    """At c = 50 % and the optimal dmu0 (= 0 by symmetry) the serial method's
    acceptance is about 47 % (Sec. III C) at small kappa and falls linearly
    with kappa (Sec. II C); kappa = 0 is the SGC ensemble, which cannot hold
    c inside the miscibility gap."""
    p, tab = model
    acc_small, c_small = _serial_acceptance(tab, 10.0)
    acc_big, c_big = _serial_acceptance(tab, 1000.0)
    assert abs(acc_small - GOLDEN["serial_max_acceptance_approx"]) < 0.03, acc_small
    assert abs(c_small - 0.5) < 0.01 and abs(c_big - 0.5) < 0.01
    assert acc_big < acc_small - 0.04
    acc_sgc, c_sgc = _serial_acceptance(tab, 0.0, sweeps=100)
    assert abs(c_sgc - 0.5) > 0.2  # phase-separated into one phase
