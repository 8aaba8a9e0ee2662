"""The error bound behind the FP32 screen of the multicomponent step with
re-embedding (multicomponent and binary forms).  For an embedding cubic p_j(t) = c0 + t (c1 + t (c2 + t c3))
evaluated in float (coefficients rounded to float, three FMAs, the
argument rho + f_b(r_s) - f_a(r_s) and x / h carried in float), the
distance from the FP64 evaluation is at most 2^-24 [6 G + 5 P + 3 dmax S]
(G = max sum |c_k|, P = max (j + 2) |dp/dt| near interval j, S = max
|F'|, dmax = max |f_b(r_s) - f_a(r_s)|; over the screened range x >=
max(h, x_max / 20)).  This restates the bound as the device's setup
computes it and checks it against float evaluations emulated in numpy on
the tables of the workloads."""
import numpy as np
import pytest

from paper_1012_5082_gb300 import inputs as I

A = 2.855


def _coefficients(y, m, h):
    """Power-form coefficients of the cubic Hermite interpolant on each
    interval (values y, derivatives m, spacing h)."""
    c0 = y[:-1]
    c1 = h * m[:-1]
    c2 = 3 * (y[1:] - y[:-1]) - h * (2 * m[:-1] + m[1:])
    c3 = 2 * (y[:-1] - y[1:]) + h * (m[:-1] + m[1:])
    return np.stack([c0, c1, c2, c3], 1)


def _fma32(a, b, c):
    # a*b is exact in float64 for float32 operands; one rounding of the sum
    # to float64 then float32 (a rare double rounding is 1 ulp, far inside
    # the margin tested)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


@pytest.mark.parametrize("K,ds", [(4, (1.0, 1.25, 0.85, 1.1)), (2, (1.0, 1.25))])
def test_fp32_embedding_error_within_bound(K, ds):
    """K = 4: the multicomponent workload's tables; K = 2: the binary
    context's re-embedding tables (f_B = 1.25 f_A)."""
    p = I.multi_eam_params(K, dens_scale=ds)
    T = I.eam_tables(p)
    h, n = T.drho, T.nrho - 1
    ih = 1.0 / h
    lo = max(h, (n * h) / 20.0)
    jlo = max(0, int(np.floor(lo / h)) - 1)
    coefs = [_coefficients(np.asarray(T.embed[t]), np.asarray(T.dembed[t]), h) for t in range(K)]
    G = P = S = 0.0
    for C in coefs:
        G = max(G, np.abs(C[jlo:]).sum(1).max())
        D = np.abs(C[:, 1]) + 2 * np.abs(C[:, 2]) + 3 * np.abs(C[:, 3])
        S = max(S, D[jlo:].max() * ih)
        Dn = np.maximum(D, np.maximum(np.r_[0.0, D[:-1]], np.r_[D[1:], 0.0]))
        P = max(P, ((np.arange(n) + 2) * Dn)[jlo + 1:].max())
    rs = A * np.sqrt(np.array([3, 4, 8, 11, 12])) / 2
    Fd = np.array([[p.dens(t, r)[0] for t in range(K)] for r in rs])
    dmax = np.abs(Fd[:, :, None] - Fd[:, None, :]).max()
    E = 2.0 ** -24 * (6 * G + 5 * P + 3 * dmax * S)

    rho0 = (np.array([8, 6, 12, 24, 8]) * Fd[:, 0]).sum()
    rng = np.random.default_rng(7)
    M = 400_000
    t = rng.integers(0, K, M)
    rho = rng.uniform(0.5 * rho0, 1.6 * rho0, M)
    s, a, b = rng.integers(0, 5, M), rng.integers(0, K, M), rng.integers(0, K, M)
    dfs = Fd[s, b] - Fd[s, a]
    Call = np.stack(coefs)                     # [K, n, 4]

    def ev64(x):
        u = x * ih
        j = np.minimum(u.astype(np.int64), n - 1)
        tt = u - j
        c = Call[t, j]
        return c[:, 0] + tt * (c[:, 1] + tt * (c[:, 2] + tt * c[:, 3]))

    def ev32(x32):
        u = (x32 * np.float32(ih)).astype(np.float32)
        j = np.minimum(u.astype(np.int64), n - 1)
        tt = (u - j.astype(np.float32)).astype(np.float32)
        c = Call[t, j].astype(np.float32)
        return _fma32(tt, _fma32(tt, _fma32(tt, c[:, 3], c[:, 2]), c[:, 1]), c[:, 0])

    r32 = rho.astype(np.float32)
    x32 = (r32 + dfs.astype(np.float32)).astype(np.float32)
    err1 = np.abs(ev32(x32).astype(np.float64) - ev64(rho + dfs))
    err0 = np.abs(ev32(r32).astype(np.float64) - ev64(rho))
    worst = max(err1.max(), err0.max())
    assert worst <= E, (worst, E)
    # the bound is not vacuous: within a factor 20 of what float evaluation reaches
    assert worst > E / 20, (worst, E)
    # and small enough that the screen decides nearly every trial: 118
    # evaluations at 1200 K are below 1 % of kT
    assert 118 * E < 0.01 * I.KB_EV * 1200.0


@pytest.mark.parametrize("K,ds", [(4, (1.0, 1.25, 0.85, 1.1)), (2, (1.0, 1.25))])
def test_offset_tables_within_the_reachable_range_bound(K, ds):
    """The multicomponent screen's tables: each species' cubics offset by
    its value at the middle of the densities a rigid five-shell lattice can
    reach (the 58 neighbours' f summed shell by shell, smallest to largest
    species), the bound taken over the intervals reaching [rho_min - dmax,
    rho_max + dmax] only.  Float evaluations of the offset tables stay within
    it, and it is tighter than the full-table bound."""
    p = I.multi_eam_params(K, dens_scale=ds)
    T = I.eam_tables(p)
    h, n = T.drho, T.nrho - 1
    ih = 1.0 / h
    coefs = [_coefficients(np.asarray(T.embed[t]), np.asarray(T.dembed[t]), h) for t in range(K)]
    rs = A * np.sqrt(np.array([3, 4, 8, 11, 12])) / 2
    ns = np.array([8, 6, 12, 24, 8])
    Fd = np.array([[p.dens(t, r)[0] for t in range(K)] for r in rs])
    dmax = np.abs(Fd[:, :, None] - Fd[:, None, :]).max()
    rmin, rmax = (ns * Fd.min(1)).sum(), (ns * Fd.max(1)).sum()
    lo = max(h, (rmin - dmax) * (1 - 1e-5))
    hi = min(n * h * (1 - 1e-6), (rmax + dmax) * (1 + 1e-5))
    rmid = 0.5 * (rmin + rmax)
    jm = min(n - 1, int(rmid / h))
    tm = rmid / h - jm
    fref = np.array([C[jm, 0] + tm * (C[jm, 1] + tm * (C[jm, 2] + tm * C[jm, 3])) for C in coefs])
    shifted = [C - np.array([f, 0.0, 0.0, 0.0]) for C, f in zip(coefs, fref)]
    j0, j1 = max(0, int(np.floor(lo / h)) - 1), min(n - 1, int(np.floor(hi / h)) + 1)
    G = P = S = 0.0
    for C in shifted:
        D = np.abs(C[:, 1]) + 2 * np.abs(C[:, 2]) + 3 * np.abs(C[:, 3])
        Dp = np.r_[0.0, D, 0.0]
        Dn = np.maximum(D, np.maximum(Dp[:-2], Dp[2:]))
        G = max(G, np.abs(C[j0:j1 + 1]).sum(1).max())
        S = max(S, D[j0:j1 + 1].max() * ih)
        P = max(P, ((np.arange(n) + 2) * Dn)[j0:j1 + 1].max())
    E = 2.0 ** -24 * (6 * G + 5 * P + 3 * dmax * S)

    rng = np.random.default_rng(17)
    M = 400_000
    t = rng.integers(0, K, M)
    rho = rng.uniform(rmin, rmax, M)
    s, a, b = rng.integers(0, 5, M), rng.integers(0, K, M), rng.integers(0, K, M)
    dfs = Fd[s, b] - Fd[s, a]
    Call = np.stack(coefs)
    Cs = np.stack(shifted)

    def ev64(x):
        u = x * ih
        j = np.minimum(u.astype(np.int64), n - 1)
        tt = u - j
        c = Call[t, j]
        return c[:, 0] + tt * (c[:, 1] + tt * (c[:, 2] + tt * c[:, 3])) - fref[t]

    def ev32(x32):
        u = (x32 * np.float32(ih)).astype(np.float32)
        j = np.minimum(u.astype(np.int64), n - 1)
        tt = (u - j.astype(np.float32)).astype(np.float32)
        c = Cs[t, j].astype(np.float32)
        return _fma32(tt, _fma32(tt, _fma32(tt, c[:, 3], c[:, 2]), c[:, 1]), c[:, 0])

    r32 = rho.astype(np.float32)
    x32 = (r32 + dfs.astype(np.float32)).astype(np.float32)
    assert np.all((x32 >= lo) & (x32 <= hi))
    err1 = np.abs(ev32(x32).astype(np.float64) - ev64(rho + dfs))
    err0 = np.abs(ev32(r32).astype(np.float64) - ev64(rho))
    worst = max(err1.max(), err0.max())
    assert worst <= E, (worst, E)
    # tighter than the bound over the whole table without offsets
    lo_full = max(h, (n * h) / 20.0)
    jlo = max(0, int(np.floor(lo_full / h)) - 1)
    Gf = Pf = Sf = 0.0
    for C in coefs:
        D = np.abs(C[:, 1]) + 2 * np.abs(C[:, 2]) + 3 * np.abs(C[:, 3])
        Gf = max(Gf, np.abs(C[jlo:]).sum(1).max())
        Sf = max(Sf, D[jlo:].max() * ih)
        Dn = np.maximum(D, np.maximum(np.r_[0.0, D[:-1]], np.r_[D[1:], 0.0]))
        Pf = max(Pf, ((np.arange(n) + 2) * Dn)[jlo + 1:].max())
    E_full = 2.0 ** -24 * (6 * Gf + 5 * Pf + 3 * dmax * Sf)
    print(f"K={K}: offset bound {E:.3g} eV, full-table bound {E_full:.3g} eV, worst {worst:.3g} eV")
    assert E < 0.6 * E_full


def _screen(x32, dx, u53, second_order=True, guard=True):
    """The FP32 screen's rule restated in numpy (float32 arithmetic):
    accept, reject or -1 (undecided) for u = u53 2^-53 against exp(-X),
    given x32 within dx of X.  guard: no decision past dx = 0.5."""
    f = np.float32
    x32, dx = f(x32), f(dx)
    if guard and not dx <= f(0.5):
        return -1
    if x32 <= f(-2.0) * dx:
        return 1
    if u53 == 0:
        return -1
    if x32 >= f(80.0) + dx:
        return 0
    pf = f(np.exp(-np.float64(x32))) * f(2.0 ** 53)
    uf = f(u53)
    m = dx + (dx * dx if second_order else f(0.0)) + f(2.0 ** -20)
    if uf * f(1 + 2.0 ** -22) < pf * (f(1) - m):
        return 1
    if uf * f(1 - 2.0 ** -22) > pf * (f(1) + m):
        return 0
    return -1


def test_screen_margin_covers_the_second_order_term():
    """With x32 at the far end of its bound (x32 = X + dx, so exp(-x32) is
    exp(-X) e^-dx) and u just below exp(-X), a margin of dx alone rejects
    moves the FP64 test accepts once dx exceeds about 1e-3 (as in the
    re-embedding screens, dx ~ 5e-3); the margin dx + dx^2 never decides
    against the FP64 test."""
    rng = np.random.default_rng(11)
    wrong = {True: 0, False: 0}
    for _ in range(20000):
        X = rng.uniform(0.05, 10.0)
        dx = 10 ** rng.uniform(-4, -1.3)
        p = np.exp(-X)
        u53 = int(p * (1 - rng.uniform(0, dx * dx / 4)) * 2 ** 53)
        truth = 1 if u53 * 2.0 ** -53 < p else 0
        for so in (True, False):
            d = _screen(X + 0.999 * dx, dx, u53, so)
            wrong[so] += d >= 0 and d != truth
    assert wrong[True] == 0
    assert wrong[False] > 1000


def test_screen_leaves_large_bounds_to_fp64():
    """For dx beyond 1.79, 1 + dx + dx^2 < e^dx: without the dx <= 0.5 guard
    the rule rejects moves the FP64 test accepts (x32 at X + dx, u just
    below exp(-X)); with it, no bound from 1e-4 to 3 decides wrongly."""
    rng = np.random.default_rng(12)
    wrong = {True: 0, False: 0}
    for _ in range(20000):
        X = rng.uniform(0.05, 10.0)
        dx = 10 ** rng.uniform(-4, np.log10(3.0))
        p = np.exp(-X)
        u53 = int(p * rng.uniform(0.3, 1.0) * 2 ** 53)
        truth = 1 if u53 * 2.0 ** -53 < p else 0
        for g in (True, False):
            for side in (0.999, -0.999):
                d = _screen(X + side * dx, dx, u53, True, guard=g)
                wrong[g] += d >= 0 and d != truth
    assert wrong[True] == 0
    assert wrong[False] > 100
