"""The learned delayed-acceptance stage on the GPU against the oracle (GPU
only): descriptors and targets, the BF16 tensor-core network (forward and
gradient against the FP64 reference), training on samples drawn by the
method's own sampler, and the two-stage colour step (bit-exact with a
constant surrogate, same distribution as the plain rule with a poor one)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_1012_5082_gb300 import inputs as I
from _pair import Lockstep, c0_config, compare_obs, lockstep, make_pair

pytestmark = pytest.mark.gpu

A = 2.855
SHELL_R = np.array([A * math.sqrt(3) / 2, A, A * math.sqrt(2), A * math.sqrt(11) / 2, A * math.sqrt(3)])


@pytest.fixture(scope="module")
def V():
    from paper_1012_5082_gb300 import vcsgc
    return vcsgc


@pytest.fixture(scope="module")
def torch():
    import torch as T
    return T


def _target(orc, i, t):
    de = orc.delta_e(i)
    return de if t[i] == 0 else -de


# ------------------------------------------------------- descriptors
def test_features_match_oracle(V, torch):
    """Every site of the 10^3 workload at 30% B: the ten counts are equal and
    the FP32 target is the oracle's E(B) - E(A) rounded to FP32."""
    lat, _, tab = c0_config()
    types = I.random_types(lat.n, 600, seed=41)
    g = V.Context(lat, types, tab, -2.0, 1000.0, 700.0, schedule=V.SCHED_BLOCKS, sched=(5, 5, 5, 2, 2, 2))
    X, Y = g.features()
    X, Y = X.cpu().numpy(), Y.cpu().numpy().astype(np.float64)
    orc = O.System(lat, types, tab)
    orc.set_shells(SHELL_R)
    for i in range(lat.n):
        assert np.array_equal(X[i], orc.descriptor(i)), i
        want = _target(orc, i, types)
        assert abs(Y[i] - want) <= 1.2e-7 * abs(want) + 1e-11, (i, Y[i], want)
    g.close()


def test_batch_features_after_sweeps(V, torch):
    """Replicas of uneven sizes after some sweeps: rows are laid out replica
    after replica and match oracle chains run from the same start."""
    tab = I.eam_tables()
    cells = [(8, 8, 8), (12, 8, 8)]
    phi, T, seeds = [-2.45, -2.40], [700.0, 650.0], [21, 22]
    lats = [I.bcc_lattice(*c) for c in cells]
    types = [I.random_types(l.n, l.n // 4, seed=60 + q) for q, l in enumerate(lats)]
    b = V.Batch(cells, types, tab, phi, 20.0, T, seed_r=np.array(seeds, np.uint64), c0=0.25)
    orcs = []
    for q, l in enumerate(lats):
        o = O.System(l, types[q], tab)
        o.set_params(phi[q], 20.0, T[q], c0=0.25, seed=seeds[q])
        o.schedule_sublattice(l.cells, (4, 4, 4))
        o.set_shells(SHELL_R)
        orcs.append(o)
    ls = Lockstep(orcs, b)
    ls.advance(3 * 128)
    ls.close()
    X, Y = b.features()
    X, Y = X.cpu().numpy(), Y.cpu().numpy().astype(np.float64)
    assert X.shape[0] == sum(l.n for l in lats)
    off = 0
    rng = np.random.default_rng(3)
    for q, (l, o) in enumerate(zip(lats, orcs)):
        to = o.types
        assert np.array_equal(b.types(q), to)
        assert o.obs()["flips"] > 0
        for i in list(rng.choice(l.n, 200, replace=False)) + [0, l.n - 1]:
            assert np.array_equal(X[off + i], o.descriptor(i)), (q, i)
            want = _target(o, i, to)
            assert abs(Y[off + i] - want) <= 1.2e-7 * abs(want) + 1e-11
        off += l.n
    b.close()


# --------------------------------------------------------- the network
def _counts(rng, n):
    return np.floor(rng.random((n, 10)) * (M.DESC_MAX + 1)).astype(np.float32)


def test_mlp_forward_matches_reference(V, torch):
    """1000 rows (62 tiles of 16 and a ragged tail of 8).  Against the FP64
    network with the same BF16 rounding of the tensor-core operands the
    remaining difference is the hardware tanh in SiLU (relative error below
    2^-10) and BF16 roundings it tips, a few 1e-4 of the output scale; the
    bound is 2e-3.  Against plain FP64 the BF16 operands add up to ~1%."""
    p = I.mlp_init(3, out_bias=1.5)
    X = _counts(np.random.default_rng(4), 1000)
    s = V.Surrogate(p)
    g = s.forward(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    p64, X64 = p.astype(np.float64), X.astype(np.float64)
    ref_b = M.forward(p64, X64, rnd=M.round_bf16)[0]
    ref = M.forward(p64, X64)[0]
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(g - ref_b).max() <= 2e-3 * scale, np.abs(g - ref_b).max()
    assert np.abs(g - ref).max() <= 1e-2 * scale
    # the network is not trivially constant on these inputs
    assert np.std(ref) > 0.02
    s.close()


def test_mlp_gradient_matches_reference(V, torch):
    """Full-batch gradient of the mean squared error (1000 rows) against the
    FP64 back-propagation with the same BF16 operand rounding: per parameter
    group the relative norm of the difference is below 2e-2 (hardware tanh,
    tipped roundings and FP32 sums), the loss within 1e-3."""
    p = I.mlp_init(5, out_bias=0.5)
    rng = np.random.default_rng(6)
    X = _counts(rng, 1000)
    Y = rng.normal(1.0, 0.5, 1000).astype(np.float32)
    s = V.Surrogate(p)
    grad, loss = s.grad(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
    loss_r, grad_r = M.loss_and_grad(p.astype(np.float64), X.astype(np.float64), Y.astype(np.float64),
                                     rnd=M.round_bf16)
    assert abs(loss - loss_r) <= 1e-3 * loss_r, (loss, loss_r)
    H, IN = 64, 10
    groups = {"W1": slice(0, H * IN), "b1": slice(H * IN, H * IN + H),
              "W2": slice(H * IN + H, H * IN + H + H * H), "b2": slice(H * IN + H + H * H, H * IN + 2 * H + H * H),
              "w3": slice(H * IN + 2 * H + H * H, H * IN + 3 * H + H * H), "b3": slice(M.NPARAM - 1, M.NPARAM)}
    for name, sl in groups.items():
        a, b = grad[sl].astype(np.float64), grad_r[sl]
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-9, (name, np.linalg.norm(a - b),
                                                                          np.linalg.norm(b))
    s.close()


# ------------------------------------------- data from the sampler, training
def _sampler_batch(V, R=16, n=12, seed=300):
    """R replicas of the 10^3 workload's EAM on n^3 lattices, spread over
    concentration by the variance constraint (c0 from 2% to 50%, phi set so
    that the local driving force is the same) and over 600-900 K."""
    tab = I.eam_tables()
    c0 = np.linspace(0.02, 0.5, R)
    T = np.linspace(600.0, 900.0, R)
    kappa = 1000.0
    phi = -2.02 - 2.0 * kappa * I.KB_EV * T * c0
    lat = I.bcc_lattice(n, n, n)
    types = [I.random_types(lat.n, int(round(c * lat.n)), seed=seed + q) for q, c in enumerate(c0)]
    b = V.Batch([(n, n, n)] * R, types, tab, phi, kappa, T, seed_r=np.arange(seed, seed + R, dtype=np.uint64),
                c0_r=c0)
    return b


def _collect(torch, b, snapshots, sweeps_between):
    Xs, Ys = [], []
    for _ in range(snapshots):
        b.sweep(sweeps_between)
        X, Y = b.features()
        Xs.append(X)
        Ys.append(Y)
    return torch.cat(Xs), torch.cat(Ys)


@pytest.fixture(scope="module")
def trained(V, torch):
    b = _sampler_batch(V)
    X, Y = _collect(torch, b, 12, 2)
    Xh, Yh = _collect(torch, b, 2, 5)  # held out
    s = V.Surrogate(I.mlp_init(7, out_bias=float(Y.mean())))
    hist = s.train(X, Y, batch=2048, steps=3000, lr=2e-3, seed=11)
    b.close()
    return s, hist, (X, Y), (Xh, Yh)


def test_training_on_sampler_data(V, torch, trained):
    """Trained by the GPU kernels on dE the sampler produced: the minibatch
    loss falls by two orders of magnitude and the held-out error is a small
    fraction of the spread of dE."""
    s, hist, (X, Y), (Xh, Yh) = trained
    assert np.all(np.isfinite(hist))
    assert hist[-100:].mean() < 0.01 * hist[:10].mean(), (hist[:10].mean(), hist[-100:].mean())
    g = s.forward(Xh)
    rmse = float(torch.sqrt(((g - Yh) ** 2).mean()))
    assert rmse < 0.1 * float(Yh.std()), (rmse, float(Yh.std()))
    # the FP64 network with the trained parameters agrees with the GPU one
    p = s.params.astype(np.float64)
    Xc = Xh[:500].cpu().numpy().astype(np.float64)
    ref = M.forward(p, Xc, rnd=M.round_bf16)[0]
    assert np.abs(g[:500].cpu().numpy() - ref).max() < 2e-3 * max(1.0, np.abs(ref).max())


# --------------------------------------------------- delayed acceptance
def test_constant_surrogate_trajectory_bit_exact(V):
    """A surrogate with all weights zero predicts g = b3 exactly on both
    sides, so the two-stage chain is deterministic given the random streams:
    100 sweeps of the 10^3 workload equal the oracle's two-stage chain."""
    lat, types, tab = c0_config()
    orc, g = make_pair(lat, types, tab, -8.3, 1000.0, 700.0, c0=0.05, seed=2000, schedule="blocks",
                       sched=(5, 5, 5, 2, 2, 2))
    p = np.zeros(M.NPARAM, np.float32)
    p[-1] = 2.2
    s = V.Surrogate(p)
    g.set_surrogate(s)
    orc.set_shells(SHELL_R)
    orc.set_surrogate("mlp", p.astype(np.float64))
    resyncs = lockstep(orc, g, 100, 2000)
    o_g, o_o = g.observables(), orc.obs()
    if resyncs == 0:
        compare_obs(o_o, o_g)
        assert o_g["stage1_accepts"] == o_o["stage1_accepts"]
    assert o_g["flips"] > 100
    assert o_g["local_accepts"] < o_g["stage1_accepts"] < o_g["trials"]
    assert abs(g.energy() - o_g["energy"]) <= 1e-9 * abs(o_g["energy"])
    g.close()
    s.close()


def _window_stats(b, R, warm, sweeps, n_sites):
    b.sweep(warm)
    s0 = [b.observables(q) for q in range(R)]
    e = np.zeros(R)
    for _ in range(sweeps):
        b.sweep(1)
        e += np.array([b.observables(q)["energy"] / n_sites for q in range(R)])
    s1 = [b.observables(q) for q in range(R)]
    c = np.array([(s1[q]["mean_c"] * s1[q]["steps"] - s0[q]["mean_c"] * s0[q]["steps"])
                  / (s1[q]["steps"] - s0[q]["steps"]) for q in range(R)])
    return c, e / sweeps, s1


# single-phase regime where 300 sweeps of the plain rule equilibrate the
# short-range order: 900 K, c0 = 3%, kappa = 1000, dmu0 = -2.02 eV
EQ_T, EQ_KAPPA, EQ_C0 = 900.0, 1000.0, 0.03
EQ_PHI = -2.02 - 2.0 * EQ_KAPPA * I.KB_EV * EQ_T * EQ_C0


def _same_distribution(V, surrogate, R=32, equil=300, warm=20, sweeps=200):
    """Window means of c and E/N over R replicas, plain rule against delayed
    acceptance, both started from the same states equilibrated by the plain
    rule (fresh random streams for each run)."""
    tab = I.eam_tables()
    lat = I.bcc_lattice(12, 12, 12)
    cells = [(12, 12, 12)] * R
    types = [I.random_types(lat.n, int(round(EQ_C0 * lat.n)), seed=900 + q) for q in range(R)]
    b = V.Batch(cells, types, tab, EQ_PHI, EQ_KAPPA, EQ_T, seed_r=np.arange(R, dtype=np.uint64) + 100, c0=EQ_C0)
    b.sweep(equil)
    start = [b.types(q) for q in range(R)]
    b.close()
    out = []
    for mode in ("plain", "da"):
        seeds = np.arange(R, dtype=np.uint64) + (1000 if mode == "plain" else 5000)
        b = V.Batch(cells, start, tab, EQ_PHI, EQ_KAPPA, EQ_T, seed_r=seeds, c0=EQ_C0)
        if mode == "da":
            b.set_surrogate(surrogate)
        out.append(_window_stats(b, R, warm, sweeps, lat.n))
        b.close()
    (cp, ep, _), (cd, ed, sd) = out
    for a, d in ((cp, cd), (ep, ed)):
        se = math.sqrt(a.var(ddof=1) / R + d.var(ddof=1) / R)
        assert abs(a.mean() - d.mean()) < 5 * se, (a.mean(), d.mean(), se)
    return sd


def test_poor_surrogate_keeps_the_distribution(V):
    """A random network (far from dE): stage 2 rejects much of what stage 1
    lets through, yet the window means of c and E/N over 32 replicas equal
    those of the plain rule within statistical error."""
    # random weights, output layer scaled so that g spreads by ~0.03 eV
    # around 2.20 eV, the mean A->B change at a few % B (spread 0.06 eV)
    p = I.mlp_init(13, out_bias=2.20)
    p[-65:-1] *= 3.0
    s = V.Surrogate(p)
    sd = _same_distribution(V, s)
    s1 = sum(o["stage1_accepts"] for o in sd)
    acc = sum(o["local_accepts"] for o in sd)
    print(f"poor surrogate: stage-2 acceptance {acc / s1:.4f}")
    assert acc < 0.8 * s1
    s.close()


def test_trained_surrogate_gain(V, trained):
    """What the trained network buys: the exact dE is skipped for every trial
    stage 1 rejects, stage 2 confirms nearly all that pass, and the sampled
    distribution is the plain rule's."""
    s = trained[0]
    sd = _same_distribution(V, s)
    trials = sum(o["trials"] for o in sd)
    s1 = sum(o["stage1_accepts"] for o in sd)
    acc = sum(o["local_accepts"] for o in sd)
    print(f"trained surrogate: stage-1 rejection {1 - s1 / trials:.4f}, stage-2 acceptance {acc / s1:.4f}")
    assert s1 < 0.5 * trials          # exact dE skipped for over half of the trials
    assert acc > 0.9 * s1             # the surrogate rarely lets a wrong move through
