"""The float32 collision's lattice weights (csrc/sc_common.cuh, collide_core)
keep the discrete mass and momentum identities exactly: with the plain
roundings of 1/18, 1/36 and 1/3 the relaxation would add a steady source of
relative size ~3e-8 per step. Checked here in exact rational arithmetic on
the float32 values the kernel forms (CPU only)."""
import os
import re
from fractions import Fraction as Fr

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), 'paper_2003_01490_gb300', 'csrc', 'sc_common.cuh')


def kernel_weights():
    text = open(SRC).read()
    m = re.search(r'const T w2d = sizeof\(T\) == 4 \? T\(([0-9.eE+-]+)\)', text)
    assert m, 'float32 weight literal not found'
    f = np.float32
    w2d = f(float(m.group(1)))
    # the same float32 operations as the kernel
    w2a = f(2) * w2d
    w0 = f(1) - f(12) * w2d
    w6d = f(1) / f(6)
    w6a = f(1) - f(4) * w6d
    return w0, w2a, w2d, w6a, w6d


def F(x):
    return Fr(float(x))


def test_mass_and_momentum_identities_hold_exactly():
    w0, w2a, w2d, w6a, w6d = kernel_weights()
    # mass: the rest weight plus 2w over the 3 axis and 6 diagonal pairs
    assert F(w0) + 3 * F(w2a) + 6 * F(w2d) == 1
    # momentum: the first moment of 6w (c.u) over the pairs with c_x != 0
    assert F(w6a) + 4 * F(w6d) == 1


def test_weights_lie_within_2e7_of_the_lattice_weights():
    w0, w2a, w2d, w6a, w6d = kernel_weights()
    for got, exact in ((w0, Fr(1, 3)), (w2a, Fr(1, 9)), (w2d, Fr(1, 18)), (w6a, Fr(1, 3)), (w6d, Fr(1, 6))):
        assert abs(float((F(got) - exact) / exact)) < 2e-7


def test_plain_roundings_would_break_the_identities():
    # what the fixed weights avoid: 1/18, 1/36, 1/3 rounded to float32
    f = np.float32
    wa, wd, w0 = f(1) / f(18), f(1) / f(36), f(1) / f(3)
    mass = F(w0) + 3 * F(f(2) * wa) + 6 * F(f(2) * wd) - 1
    mom = F(f(6) * wa) + 4 * F(f(6) * wd) - 1
    assert mass != 0 and mom != 0
    assert abs(float(mom)) > 1e-8
