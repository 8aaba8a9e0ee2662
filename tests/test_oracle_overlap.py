"""Oracle pins for overlapping, position-weighted domains (Sec. III A, the
optimal decomposition): each cell of l^3 lattice cells holds eight domains
of edge l - g that overlap in its middle, domains of one colour are g cells
apart, and the sites are picked with weights that make the visiting rate
uniform.  The pins fix the geometry by hand, the exact per-step pick
probability 1 / (sites per cell), the empirical pick frequencies, and the
stationary distribution by exact enumeration."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1012_5082_gb300 import inputs as I

A = 2.855
KB = I.KB_EV


def _cell_coords(site, nx, ny):
    cell = site >> 1
    return cell % nx, (cell // nx) % ny, cell // (nx * ny)


def _system(cells, cell, gap, tables=None):
    lat = I.bcc_lattice(*cells)
    tab = tables if tables is not None else I.eam_tables()
    s = O.System(lat, np.zeros(lat.n, np.uint8), tab)
    s.schedule_overlap(cells, cell, gap)
    return lat, s


def _coverage_1d(x, l, g):
    """Domains of one cell that cover cell-local coordinate x along one axis:
    bit 0 covers [0, l - g), bit 1 covers [g, l)."""
    return int(x < l - g) + int(x >= g)


def test_overlap_geometry_and_exact_pick_probability():
    """12^3 lattice, cells of 6^3, gap 2: eight colours of eight domains, each
    a 4^3-cell cube at offset (bit * gap) inside its cell; every entry's
    weight times the number of the cell's domains that cover the site is 8;
    and the probability that a step trials a given site, sum over colours of
    1/8 * w / W_D, is exactly 1 / (2 * 6^3) for every site."""
    cells, cell, gap = (12, 12, 12), (6, 6, 6), (2, 2, 2)
    lat, s = _system(cells, cell, gap)
    col, dom, sites = s.schedule_tables()
    wt = s.schedule_weights()
    assert wt is not None
    assert len(col) == 9 and np.all(np.diff(col) == 8)
    ld = [l - g for l, g in zip(cell, gap)]
    per_dom = 2 * ld[0] * ld[1] * ld[2]
    assert np.all(np.diff(dom) == per_dom)
    prob = np.zeros(lat.n)
    cover_count = np.zeros(lat.n, dtype=np.int64)
    for c in range(8):
        bits = (c & 1, (c >> 1) & 1, (c >> 2) & 1)
        for d in range(col[c], col[c + 1]):
            ss = sites[dom[d]:dom[d + 1]]
            ww = wt[dom[d]:dom[d + 1]]
            assert len(set(ss.tolist())) == per_dom
            X, Y, Z = _cell_coords(ss, cells[0], cells[1])
            for q, Xq in enumerate((X, Y, Z)):
                local = Xq % cell[q]
                # the domain is the cube [bit * g, bit * g + l - g) of one cell
                assert len(set((Xq // cell[q]).tolist())) == 1
                assert local.min() == bits[q] * gap[q] and local.max() == bits[q] * gap[q] + ld[q] - 1
            cov = np.array([_coverage_1d(x % cell[0], cell[0], gap[0]) * _coverage_1d(y % cell[1], cell[1], gap[1])
                            * _coverage_1d(z % cell[2], cell[2], gap[2]) for x, y, z in zip(X, Y, Z)])
            assert np.all(ww * cov == 8)
            # listed by decreasing weight, ascending index within one weight
            assert np.all(np.diff(ww) <= 0)
            for w in np.unique(ww):
                assert np.all(np.diff(ss[ww == w]) > 0)
            prob[ss] += (1.0 / 8.0) * ww / ww.sum()
            cover_count[ss] += 1
    n_cell = 2 * cell[0] * cell[1] * cell[2]
    assert np.allclose(prob, 1.0 / n_cell, rtol=1e-12, atol=0)
    # every site sits in 1, 2, 4 or 8 of its cell's domains, the middle in all 8
    assert set(np.unique(cover_count).tolist()) == {1, 2, 4, 8}


def test_overlap_same_colour_separation():
    """Domains of one colour in neighbouring cells are gap lattice cells
    apart: the closest pair is a body-centre site and a corner site,
    a * sqrt((gap + 1/2)^2 + 1/2)."""
    for gap in (1, 2):
        cells, cell = (8, 8, 8), (4, 4, 4)
        _, s = _system(cells, cell, (gap,) * 3)
        sep = s.schedule_min_separation()
        assert abs(sep - A * math.sqrt((gap + 0.5) ** 2 + 0.5)) < 1e-9, (gap, sep)


def test_overlap_pick_frequencies_uniform():
    """The oracle's weighted draw visits every site at the same rate: 12^3
    lattice, cells of 6^3, gap 2; 86,400 steps (about 200 trials per site).
    Per-site counts pass a chi-square test against the uniform rate, and the
    four coverage classes (weights 8, 4, 2, 1, which an unweighted pick would
    visit in the ratio 1 : 2 : 4 : 8) agree within 2 %."""
    cells, cell, gap = (12, 12, 12), (6, 6, 6), (2, 2, 2)
    lat, s = _system(cells, cell, gap)
    s.set_params(-1.3, 10.0, 800.0, c0=0.1, seed=77)
    s.track_trials(True)
    n_cell = 2 * cell[0] * cell[1] * cell[2]
    steps = n_cell * 200
    s.parallel_steps(steps)
    cnt = s.trial_counts()
    assert cnt.sum() == steps * 8
    expect = steps / n_cell
    chi2 = float(((cnt - expect) ** 2 / expect).sum())
    dof = lat.n - 1
    assert abs(chi2 / dof - 1.0) < 6 * math.sqrt(2.0 / dof), chi2 / dof
    X, Y, Z = _cell_coords(np.arange(lat.n), cells[0], cells[1])
    cov = np.array([_coverage_1d(x % 6, 6, 2) * _coverage_1d(y % 6, 6, 2) * _coverage_1d(z % 6, 6, 2)
                    for x, y, z in zip(X, Y, Z)])
    for m in (1, 2, 4, 8):
        mean = cnt[cov == m].mean()
        assert abs(mean / expect - 1.0) < 0.02, (m, mean, expect)


def _enumerate(s, n, beta, phi, kappa_p):
    """Exact P(n_B) under pi_V over all 2^n states (Eq. pi_vcsgc)."""
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
    return np.bincount(nb, weights=w, minlength=n + 1), float((w * U).sum())


@pytest.mark.parametrize("mode", ["parallel", "parallel-da"])
def test_overlap_chain_matches_exact_enumeration(mode):
    """8x1x1 BCC cells with a first-shell cutoff (species-independent
    density, so sites more than r_c apart do not interact), cells of 4
    lattice cells along x with gap 1: domains of three lattice cells overlap
    in the middle two, same-colour domains are 4.5 A > r_c apart, and every
    step proposes two simultaneous weighted picks.  The sampled n_B
    distribution and <E> equal the exact pi_V of the 16 sites, also with a
    deliberately poor delayed-acceptance surrogate."""
    p = I.EAMParams(rc=2.6, r_in=2.55, nr=2000)
    tab = I.eam_tables(p)
    lat, s = _system((8, 1, 1), (4, 1, 1), (1, 0, 0), tab)
    assert s.schedule_min_separation() > tab.rc
    n = lat.n
    T, phi, kappa, c0 = 2000.0, -1.30, 2.0, 0.8
    beta = 1.0 / (KB * T)
    kappa_p = kappa * KB * T / n
    P, Emean = _enumerate(s, n, beta, phi, kappa_p)
    s.set_types(np.zeros(n, np.uint8))
    s.set_params(phi, kappa, T, kappa_units=0, c0=c0, seed=4242)
    if mode == "parallel-da":
        from test_oracle_pins import SHELL_R, _random_surrogate
        s.set_shells(SHELL_R)
        s.set_surrogate("mlp", _random_surrogate(11))
    s.run_histogram(5000, -1)
    blocks, e_blocks = [], []
    hist_tot = np.zeros(n + 1)
    for _ in range(20):
        h, e = s.run_histogram(20000, -1)
        hist_tot += h
        blocks.append((h * np.arange(n + 1)).sum() / h.sum())
        e_blocks.append(e)
    Pc = hist_tot / hist_tot.sum()
    nbar_exact = (P * np.arange(n + 1)).sum()
    err = float(np.std(blocks, ddof=1) / math.sqrt(len(blocks)))
    assert abs(np.mean(blocks) - nbar_exact) < 5 * err + 0.02, (np.mean(blocks), nbar_exact, err)
    assert 0.5 * np.abs(Pc - P).sum() < 0.03, (Pc, P)
    e_err = float(np.std(e_blocks, ddof=1) / math.sqrt(len(e_blocks)))
    assert abs(np.mean(e_blocks) - Emean) < 5 * e_err + 1e-3
    assert P.max() < 0.6
