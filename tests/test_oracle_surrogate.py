"""Pins of the oracle's delayed-acceptance pieces: the environment descriptor,
the surrogate MLP (forward and gradient) and the two-stage local rule.

Each check rests on something other than the oracle itself: the geometry of
the BCC lattice, a closed form, central finite differences, two independent
implementations of one definition, or the reduction of the two-stage rule to
the plain rule when the surrogate is exact.  The distribution test against
exact enumeration of 2^16 states lives with the other enumeration cases.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_1012_5082_gb300 import inputs as I

A = 2.855
SHELL_R = np.array([A * math.sqrt(3) / 2, A, A * math.sqrt(2), A * math.sqrt(11) / 2, A * math.sqrt(3)])


def _site(nx, ny, cx, cy, cz, b):
    return ((cz * ny + cy) * nx + cx) * 2 + b


@pytest.fixture(scope="module")
def lat_sys():
    lat = I.bcc_lattice(6, 6, 6)
    s = O.System(lat, np.zeros(lat.n, np.uint8), I.eam_tables())
    s.set_shells(SHELL_R)
    return lat, s


def test_descriptor_lattice_geometry(lat_sys):
    """Counts fixed by BCC geometry.  Site i at the origin:
    - every other site B: own = shell sizes (8, 6, 12, 24, 8); each of the 8
      first-shell neighbours sees the same shells minus i itself in shell 1,
      so nb = 8 (7, 6, 12, 24, 8);
    - one B at a first-shell site j = (1/2, 1/2, 1/2) a: of the other seven
      first-shell neighbours k, three differ from j in one coordinate sign
      (|j - k| = a, shell 2), three in two (a sqrt 2, shell 3), one in all
      three (a sqrt 3, shell 5): nb = (0, 3, 3, 0, 1);
    - one B at the shell-2 site (a, 0, 0): the four k with k_x = +a/2 see it
      at (a/2, +-a/2, +-a/2) (shell 1), the four with k_x = -a/2 at
      (3a/2, +-a/2, +-a/2), |.| = a sqrt(11)/2 (shell 4): nb = (4, 0, 0, 4, 0);
    - only i itself B: all zero (the descriptor ignores the site's own type)."""
    lat, s = lat_sys
    i = _site(6, 6, 0, 0, 0, 0)
    t = np.ones(lat.n, np.uint8)
    t[i] = 0
    s.set_types(t)
    assert list(s.descriptor(i)) == [8, 6, 12, 24, 8, 56, 48, 96, 192, 64]
    t[:] = 1
    s.set_types(t)
    assert list(s.descriptor(i)) == [8, 6, 12, 24, 8, 56, 48, 96, 192, 64]
    t[:] = 0
    t[_site(6, 6, 0, 0, 0, 1)] = 1
    s.set_types(t)
    assert list(s.descriptor(i)) == [1, 0, 0, 0, 0, 0, 3, 3, 0, 1]
    t[:] = 0
    t[_site(6, 6, 1, 0, 0, 0)] = 1
    s.set_types(t)
    assert list(s.descriptor(i)) == [0, 1, 0, 0, 0, 4, 0, 0, 4, 0]
    t[:] = 0
    t[i] = 1
    s.set_types(t)
    assert list(s.descriptor(i)) == [0] * 10


def test_descriptor_is_linear_in_single_site_contributions(lat_sys):
    """The counts are a sum over B sites of fixed per-offset weights: the
    descriptor of a random configuration equals the sum of the descriptors of
    its single-B configurations (brute force over the B sites)."""
    lat, s = lat_sys
    rng = np.random.default_rng(5)
    t = (rng.random(lat.n) < 0.3).astype(np.uint8)
    i = _site(6, 6, 3, 2, 1, 1)
    s.set_types(t)
    d = s.descriptor(i)
    acc = np.zeros(10)
    for j in np.flatnonzero(t):
        one = np.zeros(lat.n, np.uint8)
        one[j] = 1
        s.set_types(one)
        acc += s.descriptor(i)
    assert np.array_equal(d, acc)


def _random_params(seed, scale=1.0, offset=0.7):
    rng = np.random.default_rng(seed)
    H, IN = M.H, M.IN
    return np.concatenate([rng.normal(0, scale, H * IN), rng.normal(0, 0.3, H),
                           rng.normal(0, scale / 8, H * H), rng.normal(0, 0.3, H),
                           rng.normal(0, 0.2, H), [offset]])


def test_mlp_closed_form_single_path():
    """One active path: W1[0][0] = a, W2[0][0] = b, w3[0] = c, biases zero but
    b3: g = c SiLU(b SiLU(a x0 / 8)) + b3, plus 63 + 63 zero hidden units."""
    p = np.zeros(M.NPARAM)
    W1, b1, W2, b2, w3, _ = M.unpack(p)
    a, b, c, b3 = 1.7, -0.9, 2.5, 0.25
    W1 = W1.copy(); W2 = W2.copy(); w3 = w3.copy()
    W1[0, 0], W2[0, 0], w3[0] = a, b, c
    p = M.pack(W1, b1, W2, b2, w3, b3)
    x = np.array([3, 1, 2, 5, 0, 10, 4, 20, 30, 6], dtype=np.float64)
    sl = lambda z: z / (1.0 + math.exp(-z))
    want = c * sl(b * sl(a * 3 / 8)) + b3
    assert abs(O.mlp_eval(p, x) - want) < 1e-14
    assert abs(M.forward(p, x[None, :])[0][0] - want) < 1e-14


def test_mlp_two_implementations_agree():
    """The C surrogate (used by the delayed-acceptance chain) and the numpy
    network (used to check the GPU training kernels) are written separately;
    on random parameters and counts they agree to rounding."""
    p = _random_params(11)
    rng = np.random.default_rng(12)
    X = rng.integers(0, 9, size=(50, 10)).astype(np.float64) * (M.DESC_MAX / 8)
    g = M.forward(p, X)[0]
    gc = np.array([O.mlp_eval(p, x) for x in X])
    assert np.max(np.abs(g - gc)) < 1e-12 * max(1.0, np.max(np.abs(g)))


def test_mlp_gradient_matches_finite_differences():
    """Back-propagated gradient of the mean squared error against central
    differences of the loss in every one of a random sample of parameters
    (and all output-layer parameters)."""
    p = _random_params(21)
    rng = np.random.default_rng(22)
    X = rng.integers(0, 9, size=(40, 10)).astype(np.float64)
    y = rng.normal(1.0, 0.5, 40)
    loss, grad = M.loss_and_grad(p, X, y)
    idx = np.concatenate([rng.choice(M.NPARAM - 129, 120, replace=False),
                          np.arange(M.NPARAM - 65, M.NPARAM)])
    h = 1e-6
    for q in idx:
        pp, pm = p.copy(), p.copy()
        pp[q] += h
        pm[q] -= h
        fd = (M.loss_and_grad(pp, X, y)[0] - M.loss_and_grad(pm, X, y)[0]) / (2 * h)
        assert abs(grad[q] - fd) <= 1e-6 * max(1.0, abs(fd)), (q, grad[q], fd)


def test_round_bf16_values():
    """BF16 keeps 8 significant bits, rounding to nearest, ties to even."""
    assert M.round_bf16(1.0) == 1.0
    assert M.round_bf16(1.0 + 2 ** -8) == 1.0            # tie -> even
    assert M.round_bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie -> even (up)
    assert M.round_bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7
    assert M.round_bf16(-3.0 - 2 ** -7) == -3.0            # below half an ulp


def _c0_system(tables, seed_types=1000):
    lat = I.bcc_lattice(10, 10, 10)
    s = O.System(lat, I.random_types(lat.n, 100, seed=seed_types), tables)
    s.set_params(-8.3, 1000.0, 700.0, c0=0.05, seed=2000)
    s.schedule_blocks((10, 10, 10), (5, 5, 5))
    s.set_shells(SHELL_R)
    return s


@pytest.fixture(scope="module")
def tables():
    return I.eam_tables()


def test_exact_surrogate_reproduces_plain_chain(tables):
    """With a perfect surrogate (g = the exact E(B) - E(A)) stage 1 is the
    plain local test with the same uniform and stage 2 has exponent 0, so the
    two-stage chain retraces the plain chain move for move."""
    a = _c0_system(tables)
    b = _c0_system(tables)
    b.set_surrogate("exact")
    a.parallel_steps(6000)
    b.parallel_steps(6000)
    oa, ob = a.obs(), b.obs()
    assert np.array_equal(a.types, b.types)
    assert oa["flips"] == ob["flips"] > 50
    assert ob["stage1_accepts"] == ob["local_accepts"] == oa["local_accepts"]
    assert oa["stage1_accepts"] == 0


def test_surrogate_is_antisymmetric(tables):
    """g_i does not depend on the type of site i, so the predicted change of
    the reverse move is exactly the negative one."""
    s = _c0_system(tables)
    s.set_surrogate("mlp", _random_params(3))
    t = s.types
    for i in (0, 17, 555, 1999):
        g0 = s.surrogate(i)
        t2 = t.copy()
        t2[i] ^= 1
        s.set_types(t2)
        assert s.surrogate(i) == g0
        s.set_types(t)


def test_poor_surrogate_changes_path_not_energy_bookkeeping(tables):
    """A poor surrogate changes the trajectory (other moves are tried in
    stage 2) but the tracked energy still equals a full recomputation."""
    a = _c0_system(tables)
    b = _c0_system(tables)
    b.set_surrogate("mlp", _random_params(4, offset=2.2))
    a.parallel_steps(4000)
    b.parallel_steps(4000)
    ob = b.obs()
    assert not np.array_equal(a.types, b.types)
    assert ob["flips"] > 20
    assert abs(ob["energy"] - b.energy_full()) < 1e-8
    assert ob["local_accepts"] <= ob["stage1_accepts"] <= ob["trials"]
