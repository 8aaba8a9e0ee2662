"""Host arithmetic of the parameter recipe (Sec. III C): the coexistence
driving force from two SGC branches and the balanced driving force of a
composite move, against closed forms (no GPU)."""
import math

import numpy as np
import pytest

from paper_1012_5082_gb300 import inputs as I
from paper_1012_5082_gb300 import recipe as R


def test_coexistence_of_pure_phases_is_the_energy_difference():
    """At T -> 0 both branches stay pure (c_A = 0, c_B = 1): omega_A = e_A,
    omega_B = e_B + dmu, equal at dmu = e_A - e_B."""
    dmu = np.linspace(-1.85, -1.25, 13)
    e_a, e_b = -10.489480464, -8.944947203  # the workloads' pure-A and pure-B energies per site
    got = R.coexistence(dmu, np.zeros(13), np.ones(13), e_a, e_b)
    assert abs(got - (e_a - e_b)) < 1e-12


def test_coexistence_with_dilute_branches():
    """Constant dilute concentrations eps_a on the A branch and 1 - eps_b on
    the B branch make both grand potentials linear in dmu (the trapezoid rule
    is exact): e_A - eps_a (dmu_max - dmu) = e_B + dmu_min + (1 - eps_b)(dmu -
    dmu_min)."""
    dmu = np.linspace(-2.0, -1.0, 21)
    e_a, e_b, ea, eb = -10.0, -8.4, 0.01, 0.03
    want = (e_a - ea * dmu[-1] - e_b - dmu[0] + (1 - eb) * dmu[0]) / ((1 - eb) - ea)
    got = R.coexistence(dmu, np.full(21, ea), np.full(21, 1 - eb), e_a, e_b)
    assert abs(got - want) < 1e-12
    with pytest.raises(ValueError):
        R.coexistence(dmu, np.zeros(21), np.ones(21), -10.0, -10.0 + 5.0)  # no crossing on the grid


@pytest.mark.parametrize("na,nb", [(900, 100), (500, 500), (1000, 7)])
def test_balanced_driving_force_closed_form(na, nb):
    """na A sites with dE = +x and nb B sites with dE = -x: the expected dn
    vanishes at dmu0 = -x + k_B T ln(na / nb) (na >= nb)."""
    T, x = 600.0, 2.0
    de = np.concatenate([np.full(na, x), np.full(nb, -x)])
    types = np.concatenate([np.zeros(na, np.uint8), np.ones(nb, np.uint8)])
    want = -x + I.KB_EV * T * math.log(na / nb)
    assert abs(R.balanced_dmu0(de, types, T) - want) < 1e-10


def test_phi_grid():
    c0 = np.array([0.02, 0.5])
    phi = R.phi_grid(-1.5, 1000.0, 600.0, c0)
    assert np.allclose(phi, -1.5 - 2 * 1000.0 * I.KB_EV * 600.0 * c0, rtol=0, atol=1e-15)
