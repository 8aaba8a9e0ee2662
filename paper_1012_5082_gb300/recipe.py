"""Parameter recipe of the parallel VC-SGC method (Sec. III C).

(i)   The chemical driving force Delta mu_S at two-phase coexistence, from SGC
      (kappa = 0) runs of small systems that stay single-phase.
(iii) Delta mu_0 = Delta mu_S, and phi_j = Delta mu_0 - 2 kappa_p N c0_j for
      target concentrations c0_j inside the miscibility gap, so that every
      replica's local stage (Eq. trans_vcsgc_par1) is the SGC move at the
      coexistence driving force.

The SGC ensemble at driving force Delta mu weighs a state by exp[-beta (U +
Delta mu n_B)].  Its grand potential per site, omega(Delta mu) = -k_B T ln Z
/ N, has d omega / d Delta mu = <c>.  Integrated along the A-rich branch from
the top of the scan down (where <c> vanishes, omega_A = e_A, the energy per
site of pure A) and along the B-rich branch from the bottom of the scan up
(omega_B = e_B + Delta mu), the two branches cross at Delta mu_S: the phases
coexist where their grand potentials are equal.

A second driving force is useful away from equilibrium: the Delta mu_0 at
which the first composite move of a given state has no expected drift, sum_i
s_i min{1, exp[-beta (dE_i + s_i Delta mu_0)]} = 0 (s_i = +1 for A -> B).
On a supersaturated random start the local stage at Delta mu_S dissolves
every isolated B site, so its composite moves carry a dn far outside the
variance constraint's width; the balanced Delta mu_0 keeps them small.

The SGC runs go through the library's own colour step; the arithmetic here
(trapezoid integration, crossing, bisection) is host-side bookkeeping.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I


def branch_omegas(dmu, c_a, c_b, e_a, e_b):
    """Grand potential per site along the A-rich and B-rich branches.

    dmu: increasing grid (eV); c_a, c_b: <c> on each branch at those points;
    e_a, e_b: energies per site of pure A and pure B (eV)."""
    dmu = np.asarray(dmu, dtype=np.float64)
    c_a = np.asarray(c_a, dtype=np.float64)
    c_b = np.asarray(c_b, dtype=np.float64)
    assert np.all(np.diff(dmu) > 0)
    seg_a = 0.5 * (c_a[1:] + c_a[:-1]) * np.diff(dmu)
    seg_b = 0.5 * (c_b[1:] + c_b[:-1]) * np.diff(dmu)
    # omega_A(dmu_i) = e_A - int_{dmu_i}^{dmu_max} c_A
    w_a = e_a - np.concatenate([np.cumsum(seg_a[::-1])[::-1], [0.0]])
    # omega_B(dmu_i) = e_B + dmu_min + int_{dmu_min}^{dmu_i} c_B
    w_b = e_b + dmu[0] + np.concatenate([[0.0], np.cumsum(seg_b)])
    return w_a, w_b


def coexistence(dmu, c_a, c_b, e_a, e_b):
    """Delta mu_S where omega_A = omega_B (linear between grid points)."""
    dmu = np.asarray(dmu, dtype=np.float64)
    w_a, w_b = branch_omegas(dmu, c_a, c_b, e_a, e_b)
    d = w_a - w_b
    s = np.nonzero(np.sign(d[1:]) != np.sign(d[:-1]))[0]
    if len(s) != 1:
        raise ValueError("the branches do not cross exactly once on this grid")
    q = s[0]
    return float(dmu[q] - d[q] * (dmu[q + 1] - dmu[q]) / (d[q + 1] - d[q]))


def phi_grid(dmu0, kappa, T, c0):
    """phi_j = dmu0 - 2 kappa_p N c0_j with kappa_p = kappa k_B T / N."""
    return dmu0 - 2.0 * kappa * I.KB_EV * T * np.asarray(c0, dtype=np.float64)


def balanced_dmu0(de, types, T, lo=-5.0, hi=5.0, iters=80):
    """Delta mu_0 at which the expected dn of a composite move on this state
    vanishes: sum_i s_i min{1, exp[-beta (dE_i + s_i Delta mu_0)]} = 0, with
    dE_i the energy change of flipping site i and s_i = +1 (A -> B) or -1."""
    beta = 1.0 / (I.KB_EV * T)
    de = np.asarray(de, dtype=np.float64)
    s = np.where(np.asarray(types) == 0, 1.0, -1.0)

    def drift(m):
        x = np.minimum(beta * (de + s * m), 700.0)
        return float(np.sum(s * np.minimum(1.0, np.exp(-x))))

    a, b = lo, hi
    fa = drift(a)
    if fa * drift(b) > 0:
        raise ValueError("no balanced driving force in the bracket")
    for _ in range(iters):
        m = 0.5 * (a + b)
        fm = drift(m)
        if (fm > 0) == (fa > 0):
            a, fa = m, fm
        else:
            b = m
    return 0.5 * (a + b)


def sgc_branches(V, T, dmu, cells=16, warmup=200, sweeps=400, seed=4100, stream=None, device=None):
    """<c> of the A-rich and B-rich SGC branches at each driving force of the
    grid, from kappa = 0 runs started in pure A and pure B (one replica per
    point and branch, the period-4 sublattice schedule), and the pure
    phases' energies per site.  Returns (c_a, c_b, e_a, e_b)."""
    lat = I.bcc_lattice(cells, cells, cells)
    tab = I.eam_tables()
    dmu = np.asarray(dmu, dtype=np.float64)
    P = len(dmu)
    types = np.concatenate([np.zeros(P * lat.n, np.uint8), np.ones(P * lat.n, np.uint8)])
    phis = np.concatenate([dmu, dmu])
    R = 2 * P
    g = V.Context(lat, types, tab, 0.0, 0.0, T, schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4), n_replicas=R,
                  phi_r=phis, c0=0.0, seed_r=np.arange(R, dtype=np.uint64) + np.uint64(seed), stream=stream,
                  device=device)
    e_a = g.observables(0)["energy_per_atom"]
    e_b = g.observables(P)["energy_per_atom"]
    g.sweep(warmup)
    o0 = g.observables_all()
    g.sweep(sweeps)
    o1 = g.observables_all()
    g.close()
    c = np.array([(o1[r]["mean_c"] * o1[r]["steps"] - o0[r]["mean_c"] * o0[r]["steps"])
                  / (o1[r]["steps"] - o0[r]["steps"]) for r in range(R)])
    return c[:P], c[P:], e_a, e_b
