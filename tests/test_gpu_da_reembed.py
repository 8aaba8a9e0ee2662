"""Delayed acceptance on the re-embedding workload (GPU only).

Species-dependent densities (f_B = 1.25 f_A) on the period-4 sublattice: a
binary context advances through the two-species multicomponent kernels, and
the exact dE of a trial holds 58 neighbour re-embeddings.  The surrogate's
descriptor comes from per-site B counts by shell that the commit keeps up to
date.  Checked here: the two-stage chain bit for bit against the oracle's
with a constant surrogate; the descriptors after those sweeps (kept by the
commits) and after plain sweeps (rebuilt) against the oracle's on every
site; the refusals; and, on the 80^3 x 8 workload itself, that a trained
surrogate samples the plain rule's <c> and <E>."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_1012_5082_gb300 import inputs as I
from _pair import MAX_TIES, Lockstep

pytestmark = pytest.mark.gpu

A = 2.855
SHELL_R = np.array([A * math.sqrt(3) / 2, A, A * math.sqrt(2), A * math.sqrt(11) / 2, A * math.sqrt(3)])
KAPPA, T_K, C0 = 100.0, 1200.0, 0.05


@pytest.fixture(scope="module")
def V():
    from paper_1012_5082_gb300 import vcsgc
    return vcsgc


@pytest.fixture(scope="module")
def torch():
    import torch as T
    return T


@pytest.fixture(scope="module")
def tab():
    return I.eam_tables(I.multi_eam_params(2, dens_scale=(1.0, 1.25)))


def _target(orc, i, t):
    de = orc.delta_e(i)
    return de if t[i] == 0 else -de


def _check_features(X, Y, orcs, n, sample=None):
    for r, o in enumerate(orcs):
        to = o.types
        sites = range(n) if sample is None else sample
        for i in sites:
            assert np.array_equal(X[r * n + i], o.descriptor(i)), (r, i, X[r * n + i], o.descriptor(i))
        for i in list(range(0, n, max(1, n // 300))):
            want = _target(o, i, to)
            assert abs(Y[r * n + i] - want) <= 1.2e-7 * abs(want) + 1e-11, (r, i, Y[r * n + i], want)


def test_constant_surrogate_chain_and_kept_counts(V, torch, tab):
    """A surrogate with all weights zero predicts g = b3 exactly on both
    sides: 10 sweeps of two replicas of a 12^3 lattice equal the oracle's
    two-stage chains (species after every sweep, counters, stage-1 passes).
    The descriptors then equal the oracle's on every site (counts kept by the
    commits); after plain sweeps (counts not kept) they are rebuilt; and the
    two-stage chain goes on in lockstep."""
    lat = I.bcc_lattice(12, 12, 12)
    t = I.random_types(lat.n, int(0.05 * lat.n), seed=91)
    phis, seeds = [-2.2, -2.3], [92, 93]
    orcs = []
    for phi, seed in zip(phis, seeds):
        o = O.System(lat, t, tab)
        o.set_params(phi, KAPPA, T_K, c0=C0, seed=seed)
        o.schedule_sublattice(lat.cells, (4, 4, 4))
        o.set_shells(SHELL_R)
        orcs.append(o)
    # the constant prediction: the mean A -> B change on the start, as a float
    a_sites = np.nonzero(t == 0)[0][:400]
    g0 = float(np.float32(np.mean([orcs[0].delta_e(i) for i in a_sites])))
    p = np.zeros(M.NPARAM, np.float32)
    p[-1] = g0
    s = V.Surrogate(p)
    b = V.Context(lat, np.tile(t, 2), tab, 0.0, KAPPA, T_K, c0=C0, schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4),
                  n_replicas=2, phi_r=np.array(phis), seed_r=np.array(seeds, dtype=np.uint64))
    b.set_surrogate(s)
    for o in orcs:
        o.set_surrogate("mlp", p.astype(np.float64))
    ls = Lockstep(orcs, b)
    for _ in range(10):
        ls.advance(b.steps_per_sweep)
    for r, o in enumerate(orcs):
        og, oo = b.observables(r), o.obs()
        assert og["flips"] > 100, og["flips"]
        assert og["local_accepts"] < og["stage1_accepts"] < og["trials"]
        if ls.resyncs == 0:
            assert og["stage1_accepts"] == oo["stage1_accepts"], (og["stage1_accepts"], oo["stage1_accepts"])
    # per-site counts kept by the commits of the two-stage steps
    X, Y = b.features()
    _check_features(X.cpu().numpy(), Y.cpu().numpy().astype(np.float64), orcs, lat.n)
    # plain steps do not keep the counts: features and the next two-stage
    # steps rebuild them from the species
    b.set_surrogate(None)
    for o in orcs:
        o.set_surrogate("off")
    ls.advance(2 * b.steps_per_sweep)
    X, Y = b.features()
    rng = np.random.default_rng(5)
    _check_features(X.cpu().numpy(), Y.cpu().numpy().astype(np.float64), orcs, lat.n,
                    sample=sorted(rng.choice(lat.n, 500, replace=False)))
    b.set_surrogate(s)
    for o in orcs:
        o.set_surrogate("mlp", p.astype(np.float64))
    for _ in range(3):
        ls.advance(b.steps_per_sweep)
    ls.close()
    b.close()
    s.close()


def test_multiblock_lockstep_plain_then_constant_surrogate(V, torch, tab):
    """40^3 x 2 replicas: 1,000 trials per replica per colour step over 8
    blocks, so the block queues of stage 2, the global decision the commit
    takes from every block's sums and the count words kept across blocks
    all run as at full size.  3 sweeps of the plain rule, then 3 with a
    constant surrogate, in lockstep with the oracle's chains; the
    descriptors of 2,000 sampled sites then equal the oracle's."""
    lat = I.bcc_lattice(40, 40, 40)
    t = I.random_types(lat.n, int(0.05 * lat.n), seed=97)
    phis, seeds = [-2.2, -2.25], [98, 99]
    orcs = []
    for phi, seed in zip(phis, seeds):
        o = O.System(lat, t, tab)
        o.set_params(phi, KAPPA, T_K, c0=C0, seed=seed)
        o.schedule_sublattice(lat.cells, (4, 4, 4))
        o.set_shells(SHELL_R)
        orcs.append(o)
    b = V.Context(lat, np.tile(t, 2), tab, 0.0, KAPPA, T_K, c0=C0, schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4),
                  n_replicas=2, phi_r=np.array(phis), seed_r=np.array(seeds, dtype=np.uint64))
    ls = Lockstep(orcs, b)
    for _ in range(3):
        ls.advance(b.steps_per_sweep)
    a_sites = np.nonzero(orcs[0].types == 0)[0][:400]
    g0 = float(np.float32(np.mean([orcs[0].delta_e(i) for i in a_sites])))
    p = np.zeros(M.NPARAM, np.float32)
    p[-1] = g0
    s = V.Surrogate(p)
    b.set_surrogate(s)
    for o in orcs:
        o.set_surrogate("mlp", p.astype(np.float64))
    for _ in range(3):
        ls.advance(b.steps_per_sweep)
    for r, o in enumerate(orcs):
        og, oo = b.observables(r), o.obs()
        assert og["flips"] > 1000, og["flips"]
        assert 0 < og["stage1_accepts"] < og["trials"]
        if ls.resyncs == 0:
            assert og["stage1_accepts"] == oo["stage1_accepts"]
    X, Y = b.features()
    rng = np.random.default_rng(9)
    _check_features(X.cpu().numpy(), Y.cpu().numpy().astype(np.float64), orcs, lat.n,
                    sample=sorted(rng.choice(lat.n, 1000, replace=False)))
    ls.close()
    b.close()
    s.close()


def test_multicomponent_object_surrogate(V, torch, tab):
    """The K = 2 multicomponent object takes the surrogate directly and runs
    the same two-stage chain as the oracle; K = 3, or no re-embedding, is
    refused with STATE."""
    lat = I.bcc_lattice(12, 12, 12)
    t = I.random_types(lat.n, int(0.05 * lat.n), seed=94)
    p = np.zeros(M.NPARAM, np.float32)
    p[-1] = 2.3
    s = V.Surrogate(p)
    m = V.Multi(lat, t, tab, [-2.2], KAPPA, T_K, c0=C0, seed_r=np.array([95], dtype=np.uint64))
    m.set_surrogate(s)
    o = O.System(lat, t, tab)
    o.set_params(-2.2, KAPPA, T_K, c0=C0, seed=95)
    o.schedule_sublattice(lat.cells, (4, 4, 4))
    o.set_shells(SHELL_R)
    o.set_surrogate("mlp", p.astype(np.float64))
    # a sweep at a time: species bit for bit and the counters' increments
    # exactly; species that differ need a near tie flagged by the oracle in
    # that sweep, and are then re-synced from it
    prev_o, prev_m = o.obs(), m.observables(0)
    compared = 0
    for sw in range(4):
        m.sweep(1)
        o.parallel_steps(m.steps_per_sweep)
        oo, om = o.obs(), m.observables(0)
        if not np.array_equal(m.types(), o.types):
            assert oo["near_ties"] > prev_o["near_ties"], f"sweep {sw}: species differ without a flagged tie"
            m.set_types(o.types)
            om = m.observables(0)
        elif oo["near_ties"] == prev_o["near_ties"]:
            for key in ("stage1_accepts", "local_accepts", "global_accepts", "flips"):
                assert om[key] - prev_m[key] == oo[key] - prev_o[key], (sw, key)
            compared += 1
        prev_o, prev_m = oo, om
    assert oo["near_ties"] <= MAX_TIES and compared >= 1, (oo["near_ties"], compared)
    assert 0 < om["stage1_accepts"] < om["trials"]
    X, Y = m.features()
    assert X.shape == (lat.n, 10)
    m.close()
    for K, ds in ((3, (1.0, 1.25, 0.9)), (2, None)):
        tk = I.multi_eam_params(K, dens_scale=ds)
        tt = I.multi_random_types(lat.n, [int(0.05 * lat.n)] * (K - 1), seed=96)
        m = V.Multi(lat, tt, I.eam_tables(tk), [-2.0] * (K - 1), 10.0, 1200.0, c0=0.05)
        with pytest.raises(V.VcsgcError) as e:
            m.set_surrogate(s)
        assert e.value.code == -8  # VCSGC_ERR_STATE
        with pytest.raises(V.VcsgcError):
            m.features()
        m.close()
    s.close()


def _window(g, R, sweeps):
    o0 = [g.observables(r) for r in range(R)]
    e = np.zeros(R)
    for _ in range(sweeps):
        g.sweep(1)
        e += np.array([g.observables(r)["energy_per_atom"] for r in range(R)])
    o1 = [g.observables(r) for r in range(R)]
    c = np.array([(o1[r]["mean_c"] * o1[r]["steps"] - o0[r]["mean_c"] * o0[r]["steps"])
                  / (o1[r]["steps"] - o0[r]["steps"]) for r in range(R)])
    return c, e / sweeps, o0, o1


def test_trained_surrogate_samples_the_plain_distribution(V, torch, tab):
    """The 80^3 x 8 re-embedding workload: the plain rule equilibrates the
    chains, a surrogate is trained on the descriptors and exact targets of
    that state, and from the same state the plain rule and delayed
    acceptance (fresh random streams) give window means of c and E/N that
    agree within 5 standard errors over the 8 replicas; stage 1 rejects most
    trials and stage 2 confirms most of what passes."""
    R, equil, warm, sweeps = 8, 400, 20, 150
    lat = I.bcc_lattice(80, 80, 80)
    t = np.stack([I.random_types(lat.n, int(C0 * lat.n), seed=8200 + r) for r in range(R)])
    g = V.Context(lat, t.reshape(-1), tab, -2.2, KAPPA, T_K, c0=C0, schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4),
                  n_replicas=R, seed_r=np.arange(R, dtype=np.uint64) + np.uint64(8300))
    g.sweep(equil)
    X, Y = g.features()
    s = V.Surrogate(I.mlp_init(7, out_bias=float(Y.mean())))
    s.train(X, Y, batch=4096, steps=3000, lr=2e-3, seed=19)
    pred = s.forward(X[: 1 << 20])
    rmse = float(torch.sqrt(((pred - Y[: 1 << 20]) ** 2).mean()))
    assert rmse < 0.2 * float(Y.std()), (rmse, float(Y.std()))
    del X, Y, pred
    start = [g.types(r) for r in range(R)]
    g.close()
    out = {}
    for mode, seed0 in (("plain", 9000), ("delayed", 9500)):
        g = V.Context(lat, np.concatenate(start), tab, -2.2, KAPPA, T_K, c0=C0, schedule=V.SCHED_SUBLATTICE,
                      sched=(4, 4, 4), n_replicas=R, seed_r=np.arange(R, dtype=np.uint64) + np.uint64(seed0))
        if mode == "delayed":
            g.set_surrogate(s)
        g.sweep(warm)
        out[mode] = _window(g, R, sweeps)
        g.close()
    (cp, ep, _, _), (cd, ed, o0, o1) = out["plain"], out["delayed"]
    for a, d in ((cp, cd), (ep, ed)):
        se = math.sqrt(a.var(ddof=1) / R + d.var(ddof=1) / R)
        assert abs(a.mean() - d.mean()) < 5 * se, (a.mean(), d.mean(), se)
    trials = sum(o1[r]["trials"] - o0[r]["trials"] for r in range(R))
    s1 = sum(o1[r]["stage1_accepts"] - o0[r]["stage1_accepts"] for r in range(R))
    acc = sum(o1[r]["local_accepts"] - o0[r]["local_accepts"] for r in range(R))
    print(f"re-embedding, trained surrogate: stage-1 pass {s1 / trials:.4f}, stage-2 acceptance {acc / s1:.4f}")
    assert s1 < 0.5 * trials
    assert acc > 0.6 * s1
    s.close()
