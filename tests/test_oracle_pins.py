"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
closed form, a brute-force enumeration, an invariant the paper states, or a
special case with a textbook answer.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1012_5082_gb300 import inputs as I

A = 2.855
SHELL_R = np.array([A * math.sqrt(3) / 2, A, A * math.sqrt(2), A * math.sqrt(11) / 2, A * math.sqrt(3)])
SHELL_Z = np.array([8, 6, 12, 24, 8])


# ----------------------------------------------------------------- Philox
# Known-answer values of Philox4x32-10 published with the generator (Salmon,
# Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11;
# the Random123 distribution's known-answer set): (counter, key) -> output.
PHILOX_KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("ctr,key,want", PHILOX_KAT)
def test_philox_known_answers(ctr, key, want):
    """The oracle's generator reproduces the published known-answer vectors
    (a wrong round constant, multiplier, key schedule or word order fails)."""
    assert tuple(int(w) for w in O.philox(ctr, key)) == want


def test_philox_uniformity_and_independence():
    """Statistical pins of the counter-based generator: uniform u01 (chi^2 over
    64 bins), no lag-1 correlation, balanced bits, distinct outputs for
    neighbouring counters and keys."""
    n = 40000
    u = np.empty(n)
    bits = np.zeros(32)
    for k in range(n // 2):
        w = O.philox([k, 0, 7, 0], [12345, 678])
        u[2 * k] = O.u01(w[0], w[1])
        u[2 * k + 1] = O.u01(w[2], w[3])
        for q in range(4):
            bits += (int(w[q]) >> np.arange(32)) & 1
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    chi2 = ((hist - n / 64) ** 2 / (n / 64)).sum()
    assert chi2 < 63 + 5 * math.sqrt(2 * 63)
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 5 / math.sqrt(n)
    frac = bits / (2 * n)
    assert np.all(np.abs(frac - 0.5) < 5 * 0.5 / math.sqrt(2 * n))
    a = O.philox([1, 0, 0, 0], [1, 0])
    assert not np.array_equal(a, O.philox([2, 0, 0, 0], [1, 0]))
    assert not np.array_equal(a, O.philox([1, 0, 0, 0], [2, 0]))
    assert not np.array_equal(a, O.philox([1, 0, 0, 1], [1, 0]))


def test_u01_and_below_maps():
    """u01 keeps the top 53 bits; below(w, m) = floor(w m / 2^64)."""
    assert O.u01(0, 0) == 0.0
    assert O.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert O.u01(0, 0x80000000) == 0.5
    for (lo, hi, m) in [(0, 0, 7), (0xFFFFFFFF, 0xFFFFFFFF, 250), (123, 0x80000000, 1000),
                        (5, 0x40000000, 8)]:
        w = (hi << 32) | lo
        assert O.below(lo, hi, m) == (w * m) >> 64
    assert O.below(0xFFFFFFFF, 0xFFFFFFFF, 1) == 0


# ----------------------------------------------------------------- spline
def _cubic_tables():
    """Tables whose every function is a cubic polynomial with exact knot
    derivatives: cubic Hermite interpolation must reproduce them exactly."""
    rc, nr, nrho, rho_max = 5.3, 200, 300, 50.0
    dr, drho = rc / (nr - 1), rho_max / (nrho - 1)
    r = np.arange(nr) * dr
    rho = np.arange(nrho) * drho
    coef = [(0.3, -0.2, 0.05, -0.004), (1.0, 0.1, -0.03, 0.002), (-0.5, 0.4, 0.0, -0.001),
            (2.0, -0.7, 0.08, -0.003), (1.5, -0.5, 0.06, -0.0025), (-1.0, -0.1, 0.01, 1e-5),
            (-2.0, 0.05, -0.002, 2e-5)]

    def poly(c, x):
        return c[0] + c[1] * x + c[2] * x ** 2 + c[3] * x ** 3, c[1] + 2 * c[2] * x + 3 * c[3] * x ** 2

    vals = [poly(c, r if q < 5 else rho) for q, c in enumerate(coef)]
    tab = I.EAMTables(rc=rc, nr=nr, dr=dr, nrho=nrho, drho=drho,
                      pair=[vals[q][0] for q in range(3)], dpair=[vals[q][1] for q in range(3)],
                      dens=[vals[q][0] for q in (3, 4)], ddens=[vals[q][1] for q in (3, 4)],
                      embed=[vals[q][0] for q in (5, 6)], dembed=[vals[q][1] for q in (5, 6)])
    return tab, coef, poly


def test_spline_reproduces_cubics_exactly():
    tab, coef, poly = _cubic_tables()
    lat = I.bcc_lattice(2, 2, 2)
    s = O.System(lat, np.zeros(lat.n, np.uint8), tab)
    rng = np.random.default_rng(0)
    for which in range(7):
        hi = tab.rc if which < 5 else (tab.nrho - 1) * tab.drho
        for x in np.concatenate([rng.uniform(0, hi, 50), [0.0, hi]]):
            v, dv = s.spline(which, x)
            ev, edv = poly(coef[which], x)
            assert abs(v - ev) <= 1e-12 * max(1.0, abs(ev))
            assert abs(dv - edv) <= 1e-10 * max(1.0, abs(edv))
    with pytest.raises(ValueError):
        s.spline(0, tab.rc * 1.01)
    with pytest.raises(ValueError):
        s.spline(5, -1e-3)


def test_spline_finite_difference_knots_exact_for_quadratics():
    """Without knot derivatives the central-difference slopes are exact for a
    quadratic, so interior intervals reproduce it exactly."""
    tab, _, _ = _cubic_tables()
    r = np.arange(tab.nr) * tab.dr
    q = 0.7 - 0.3 * r + 0.11 * r * r
    tab.pair = [q, q, q]
    tab.dpair = [None, None, None]
    lat = I.bcc_lattice(2, 2, 2)
    s = O.System(lat, np.zeros(lat.n, np.uint8), tab)
    for x in np.linspace(2 * tab.dr, tab.rc - 2 * tab.dr, 37):
        v, dv = s.spline(1, x)
        assert abs(v - (0.7 - 0.3 * x + 0.11 * x * x)) < 1e-12
        assert abs(dv - (-0.3 + 0.22 * x)) < 1e-10


# ----------------------------------------------------------- lattice, EAM
@pytest.fixture(scope="module")
def tables():
    return I.eam_tables()


@pytest.fixture(scope="module")
def params():
    return I.EAMParams()


def test_bcc_neighbour_shells(tables):
    """Rigid BCC within 5.3 A: 58 neighbours in shells of 8/6/12/24/8 at
    a*sqrt(3)/2, a, a*sqrt(2), a*sqrt(11)/2, a*sqrt(3); brute force and
    cell binning give the same list."""
    lat = I.bcc_lattice(6, 6, 6)
    t = np.zeros(lat.n, np.uint8)
    s1 = O.System(lat, t, tables)
    s2 = O.System(lat, t, tables, brute=True)
    for i in (0, 1, 77, lat.n - 1):
        nb1, nb2 = s1.neighbours(i), s2.neighbours(i)
        assert len(nb1) == 58
        assert [e[0] for e in nb1] == [e[0] for e in nb2]
        r = np.array([e[1] for e in nb1])
        counts = [np.sum(np.abs(r - rs) < 1e-9) for rs in SHELL_R]
        assert counts == list(SHELL_Z)
        for j, rr, d in nb1:
            assert abs(np.linalg.norm(d) - rr) < 1e-12


def _closed_form(params, tb):
    """Pure-lattice energy per atom of species tb, and the A->B flip energy in
    pure A, from the closed-form functions at the shell radii."""
    phis = [params.pair(q, SHELL_R)[0] for q in range(3)]
    rho0 = float((SHELL_Z * params.dens(0, SHELL_R)[0]).sum())
    e_pure = 0.5 * float((SHELL_Z * phis[2 * tb]).sum()) + float(params.embed(tb, rho0)[0])
    de = float((SHELL_Z * (phis[1] - phis[0])).sum()) + float(params.embed(1, rho0)[0] - params.embed(0, rho0)[0])
    return e_pure, de, rho0, phis


def test_pure_lattice_energy_closed_form(tables, params):
    lat = I.bcc_lattice(5, 5, 5)
    for tb in (0, 1):
        s = O.System(lat, np.full(lat.n, tb, np.uint8), tables)
        e_pure, _, rho0, _ = _closed_form(params, tb)
        assert abs(s.energy_full() / lat.n - e_pure) < 1e-10
        assert np.allclose(s.rho, rho0, rtol=0, atol=1e-10)
    s = O.System(lat, np.zeros(lat.n, np.uint8), tables)
    _, de, _, _ = _closed_form(params, 0)
    assert abs(s.delta_e(17) - de) < 1e-10


def test_rigid_lattice_delta_e_is_affine_in_shell_counts(tables, params):
    """With one density function for both species, dE of an A->B flip on the
    rigid lattice is sum_s [(z_s - b_s)(phi_AB - phi_AA) + b_s (phi_BB - phi_AB)](r_s)
    + F_B(rho0) - F_A(rho0), and dE(B->A) is its negative."""
    lat = I.bcc_lattice(6, 6, 6)
    t = I.random_types(lat.n, lat.n // 4, seed=3)
    s = O.System(lat, t, tables)
    _, _, rho0, phis = _closed_form(params, 0)
    dF = float(params.embed(1, rho0)[0] - params.embed(0, rho0)[0])
    for i in range(0, lat.n, 37):
        nb = s.neighbours(i)
        b = np.zeros(5)
        for j, r, _ in nb:
            sh = int(np.argmin(np.abs(SHELL_R - r)))
            b[sh] += t[j]
        de_ab = float(((SHELL_Z - b) * (phis[1] - phis[0]) + b * (phis[2] - phis[1])).sum()) + dF
        expect = de_ab if t[i] == 0 else -de_ab
        assert abs(s.delta_e(i) - expect) < 1e-10


@pytest.mark.parametrize("dens_b", [1.0, 1.25])
def test_incremental_delta_e_equals_full_recompute(dens_b):
    """dE from the local formula (pair + own embedding + neighbour re-embedding)
    equals U(after) - U(before); with f_B = 1.25 f the re-embedding term and
    the rho update of a flip are exercised.  Explicit disordered positions."""
    p = I.EAMParams(dens_scale=(1.0, dens_b))
    tab = I.eam_tables(p)
    lat = I.bcc_lattice(4, 4, 4)
    rng = np.random.default_rng(11)
    lat.x = lat.x + rng.normal(0, 0.1, lat.n)
    lat.y = lat.y + rng.normal(0, 0.1, lat.n)
    lat.z = lat.z + rng.normal(0, 0.1, lat.n)
    t = I.random_types(lat.n, 40, seed=5)
    s = O.System(lat, t, tab)
    for i in range(0, lat.n, 9):
        assert abs(s.delta_e(i) - s.delta_e_full(i)) < 1e-9
    # after flips the incrementally updated rho equals a fresh build
    for i in (3, 50, 91):
        s.flip(i)
    t2 = s.types
    fresh = O.System(lat, t2, tab)
    assert np.allclose(s.rho, fresh.rho, rtol=0, atol=1e-12)
    if dens_b != 1.0:
        assert any(abs(s.delta_e(i) - s.delta_e_full(i)) < 1e-9 for i in range(5))


# ---------------------------------------------------------------- schedules
def test_schedule_tables_partition_sites(tables):
    lat = I.bcc_lattice(8, 8, 8)
    s = O.System(lat, np.zeros(lat.n, np.uint8), tables)
    s.schedule_blocks((8, 8, 8), (4, 4, 4))
    col, dom, sites = s.schedule_tables()
    assert len(col) == 9 and len(dom) == 9
    assert sorted(sites.tolist()) == list(range(lat.n))
    s.schedule_sublattice((8, 8, 8), (4, 4, 4))
    col, dom, sites = s.schedule_tables()
    assert len(col) == 129 and np.all(np.diff(col) == lat.n // 128)
    assert sorted(sites.tolist()) == list(range(lat.n))


def test_schedule_separation_against_twice_cutoff(tables):
    """Same-colour trial sites must be more than 2 r_c = 10.6 A apart (the
    many-body independence radius of Sec. III A).  Between blocks of b cells
    the closest pair is a body-centre site and a corner site one block apart,
    a*sqrt((b + 1/2)^2 + 1/2): 13.00 A for b = 4 but only 10.19 A for b = 3;
    the period-4 sublattice gives 4 a = 11.42 A."""
    two_rc = 2 * tables.rc
    lat = I.bcc_lattice(16, 16, 16)
    s = O.System(lat, np.zeros(lat.n, np.uint8), tables)
    s.schedule_blocks((16, 16, 16), (4, 4, 4))
    sep4 = s.schedule_min_separation()
    assert abs(sep4 - A * math.sqrt(4.5 ** 2 + 0.5)) < 1e-9 and sep4 > two_rc
    lat3 = I.bcc_lattice(12, 12, 12)
    s3 = O.System(lat3, np.zeros(lat3.n, np.uint8), tables)
    s3.schedule_blocks((12, 12, 12), (3, 3, 3))
    sep3 = s3.schedule_min_separation()
    assert abs(sep3 - A * math.sqrt(3.5 ** 2 + 0.5)) < 1e-9 and sep3 < two_rc
    lat8 = I.bcc_lattice(8, 8, 8)
    s8 = O.System(lat8, np.zeros(lat8.n, np.uint8), tables)
    s8.schedule_sublattice((8, 8, 8), (4, 4, 4))
    assert abs(s8.schedule_min_separation() - 4 * A) < 1e-9


# ------------------------------------------------ exact enumeration (2^16)
KB = I.KB_EV


def _enumerate(s, n, beta, phi, kappa_p):
    """Exact P(n_B) and <E> under pi_V over all 2^n states (Eq. pi_vcsgc)."""
    states = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    U = np.empty(2 ** n)
    for k in range(2 ** n):
        s.set_types(states[k])
        U[k] = s.energy_full()
    nb = states.sum(axis=1)
    logw = -beta * (U + phi * nb + kappa_p * nb * nb)
    logw -= logw.max()
    w = np.exp(logw)
    w /= w.sum()
    P = np.bincount(nb, weights=w, minlength=n + 1)
    return P, float((w * U).sum())


def _lattice16(kind):
    """Two 16-site cells.  'cube': 2x2x2 BCC cells (every periodic image
    within r_c listed), weak AB mixing energy so that n_B is broadly spread.
    'chain': 8x1x1 cells with a first-shell cutoff, four 2-cell blocks along
    x in two colours, i.e. two simultaneous trial moves per step."""
    if kind == "cube":
        p = I.EAMParams(pair_scale=(1.0, 0.97, 0.95))
        return I.bcc_lattice(2, 2, 2), I.eam_tables(p), dict(cells=(2, 2, 2), block=(2, 2, 2), colours=(1, 1, 1))
    p = I.EAMParams(rc=2.6, r_in=2.55, nr=2000)
    return I.bcc_lattice(8, 1, 1), I.eam_tables(p), dict(cells=(8, 1, 1), block=(2, 1, 1), colours=(2, 1, 1))


@pytest.fixture(scope="module")
def enum_cache():
    return {}


CASES = [
    # kind, T, phi, kappa (units of kT/N), c0, mode
    ("cube", 1500.0, -1.35, 0.0, 0.1, "parallel"),
    ("cube", 1500.0, -1.60, 2.0, 0.1, "parallel"),
    ("cube", 1500.0, -1.40, 0.5, 0.8, "serial"),
    ("cube", 1500.0, -1.60, 2.0, 0.8, "serial2"),
    ("chain", 2000.0, -1.10, 0.5, 0.1, "parallel"),
    ("chain", 2000.0, -1.30, 2.0, 0.8, "parallel"),
    ("chain", 2000.0, -1.30, 2.0, 0.1, "serial2"),
    # delayed acceptance with a random (deliberately poor) surrogate
    ("cube", 1500.0, -1.60, 2.0, 0.1, "parallel-da"),
    ("cube", 1500.0, -1.60, 2.0, 0.8, "serial2-da"),
    ("chain", 2000.0, -1.30, 2.0, 0.8, "parallel-da"),
]


def _random_surrogate(seed):
    """MLP parameters that predict dE badly: random weights around a 1 eV
    offset, so stage 2 has much to correct."""
    rng = np.random.default_rng(seed)
    H, IN = O.MLP_H, O.MLP_IN
    parts = [rng.normal(0, 1.0, H * IN), rng.normal(0, 0.5, H), rng.normal(0, 0.125, H * H),
             rng.normal(0, 0.3, H), rng.normal(0, 0.1, H), [1.0]]
    return np.concatenate(parts)


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[5]}-k{c[3]}" for c in CASES])
def test_chain_matches_exact_enumeration(case, enum_cache):
    """The sampled distribution of n_B (and <E>) equals the exact pi_V of a
    16-site cell.  'chain' is 8x1x1 BCC cells with a first-shell cutoff and
    two domains per colour, so every step proposes two simultaneous moves and
    exercises the global stage with dn in {-2..2}; c0 is set far from <c> so
    a wrong sign or a dropped factor in either stage shifts the result."""
    kind, T, phi, kappa, c0, mode = case
    lat, tab, sch = _lattice16(kind)
    s = O.System(lat, np.zeros(lat.n, np.uint8), tab)
    n = lat.n
    beta = 1.0 / (KB * T)
    kappa_p = kappa * KB * T / n
    key = (kind, T, phi, kappa)
    if key not in enum_cache:
        enum_cache[key] = _enumerate(s, n, beta, phi, kappa_p)
    P, Emean = enum_cache[key]
    s.set_types(np.zeros(n, np.uint8))
    s.set_params(phi, kappa, T, kappa_units=0, c0=c0, seed=2024)
    s.schedule_blocks(sch["cells"], sch["block"], sch["colours"])
    if mode.endswith("-da"):
        s.set_shells(SHELL_R)
        s.set_surrogate("mlp", _random_surrogate(7))
    m = {"parallel": -1, "serial": 0, "serial2": 1, "parallel-da": -1, "serial2-da": 2}[mode]
    s.run_histogram(5000, m)
    blocks = []
    hist_tot = np.zeros(n + 1)
    e_blocks = []
    for _ in range(20):
        h, e = s.run_histogram(20000, m)
        hist_tot += h
        blocks.append((h * np.arange(n + 1)).sum() / h.sum())
        e_blocks.append(e)
    Pc = hist_tot / hist_tot.sum()
    nbar_exact = (P * np.arange(n + 1)).sum()
    nbar = float(np.mean(blocks))
    err = float(np.std(blocks, ddof=1) / math.sqrt(len(blocks)))
    assert abs(nbar - nbar_exact) < 5 * err + 0.02, (nbar, nbar_exact, err)
    assert 0.5 * np.abs(Pc - P).sum() < 0.03, (Pc, P)
    e_err = float(np.std(e_blocks, ddof=1) / math.sqrt(len(e_blocks)))
    assert abs(np.mean(e_blocks) - Emean) < 5 * e_err + 1e-3
    # the distribution is non-degenerate
    assert P.max() < 0.6
    if mode.endswith("-da"):
        o = s.obs()
        # stage 2 both rejects and accepts a real share of the stage-1 passes
        assert 0.05 * o["trials"] < o["stage1_accepts"] < o["trials"]
        assert o["local_accepts"] < 0.95 * o["stage1_accepts"]


def test_kappa_zero_trajectory_independent_of_c0(tables):
    """kappa = 0 is the SGC ensemble with dmu = phi (Sec. II C): the local
    stage uses dmu0 = phi whatever c0 is and the global factor is 1, so the
    trajectory cannot depend on c0 or on the kappa units."""
    lat = I.bcc_lattice(10, 10, 10)
    t0 = I.random_types(lat.n, 100, seed=1000)
    runs = []
    for c0, units in [(0.05, 0), (0.4, 0), (0.9, 1)]:
        s = O.System(lat, t0, tables)
        s.set_params(-2.28, 0.0, 700.0, kappa_units=units, c0=c0, seed=77)
        s.schedule_blocks((10, 10, 10), (5, 5, 5))
        s.parallel_steps(4000)
        runs.append((s.types, s.obs()))
    for t, o in runs[1:]:
        assert np.array_equal(t, runs[0][0])
        assert o["flips"] == runs[0][1]["flips"]
    assert runs[0][1]["flips"] > 10
    assert runs[0][1]["global_accepts"] == runs[0][1]["global_trials"]


def test_incremental_energy_tracks_full_energy(tables):
    """After many composite steps the incrementally tracked energy equals a
    full recomputation."""
    lat = I.bcc_lattice(10, 10, 10)
    s = O.System(lat, I.random_types(lat.n, 100, seed=1000), tables)
    s.set_params(-8.3, 1000.0, 700.0, c0=0.05, seed=2000)
    s.schedule_blocks((10, 10, 10), (5, 5, 5))
    s.parallel_steps(20000)
    o = s.obs()
    assert o["flips"] > 100
    assert abs(o["energy"] - s.energy_full()) < 1e-8


# ---------------------------------------------------------------------- MD
def test_forces_match_finite_differences():
    """F = -dU/dx against central differences (h = 1e-5 A) on a perturbed
    lattice with a species-dependent density."""
    p = I.EAMParams(dens_scale=(1.0, 1.25))
    tab = I.eam_tables(p)
    lat = I.bcc_lattice(5, 5, 5)
    rng = np.random.default_rng(3)
    for c in ("x", "y", "z"):
        setattr(lat, c, getattr(lat, c) + rng.normal(0, 0.1, lat.n))
    t = I.random_types(lat.n, 60, seed=4)
    s = O.System(lat, t, tab)
    F = s.forces()
    h = 1e-5
    for i in rng.choice(lat.n, 10, replace=False):
        for a, c in enumerate(("x", "y", "z")):
            e = []
            for sgn in (1, -1):
                l2 = I.Lattice(x=lat.x.copy(), y=lat.y.copy(), z=lat.z.copy(), box=lat.box)
                getattr(l2, c)[i] += sgn * h
                e.append(O.System(l2, t, tab).energy_full())
            fd = -(e[0] - e[1]) / (2 * h)
            assert abs(F[a][i] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, c, F[a][i], fd)


def test_nve_energy_conservation():
    """gamma = 0 gives velocity Verlet: the total energy error is bounded, has
    no secular drift, and scales as dt^2 (second-order symplectic
    integrator)."""
    tab = I.eam_tables()
    lat = I.bcc_lattice(6, 6, 6)
    t = I.random_types(lat.n, 40, seed=9)
    err = {}
    for dt in (1.0, 0.5):
        s = O.System(lat, t, tab)
        v = I.maxwell_velocities(t, 600.0, seed=10)
        s.set_md(v, (I.MASS_A, I.MASS_B), dt, 0.0, 300.0, 5)
        e0 = s.energy_full() + s.kinetic_energy()
        etot = []
        for _ in range(20):
            s.md_steps(int(10 / dt))
            etot.append(s.energy_full() + s.kinetic_energy())
        etot = np.array(etot) - e0
        err[dt] = np.max(np.abs(etot)) / lat.n
        if dt == 1.0:
            assert err[dt] < 2e-5
            slope = np.polyfit(np.arange(20) * 10.0, etot[:] / lat.n, 1)[0]
            assert abs(slope) * 200 < 1e-5
            # energy moved between the kinetic and potential terms
            assert s.kinetic_energy() / lat.n < 0.9 * 1.5 * I.KB_EV * 600.0
    assert 0.2 < err[0.5] / err[1.0] < 0.3


def test_langevin_thermostat_reaches_target_temperature():
    """BAOAB with friction equilibrates the kinetic temperature to T."""
    tab = I.eam_tables()
    lat = I.bcc_lattice(6, 6, 6)
    t = np.zeros(lat.n, np.uint8)
    s = O.System(lat, t, tab)
    v = I.maxwell_velocities(t, 50.0, seed=1)
    s.set_md(v, (I.MASS_A, I.MASS_B), 2.0, 0.02, 700.0, 6)
    s.md_steps(400)
    temps = []
    for _ in range(20):
        s.md_steps(20)
        temps.append(2 * s.kinetic_energy() / (3 * lat.n * I.KB_EV))
    assert abs(np.mean(temps) - 700.0) < 60.0
