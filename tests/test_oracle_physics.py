"""Pins of the oracle's local physics (Section 2.1 and the Green function of Section 2)."""
import os

import numpy as np
import pytest

from oracle import physics
from oracle.operator import COMPONENTS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_ldr_constants_match_paper():
    vals = {k: float(v) for k, v in _read_golden("ldr_constants.txt")}
    assert physics.LDR_B1 == vals["b1"]
    assert physics.LDR_B2 == vals["b2"]
    assert physics.LDR_B3 == vals["b3"]


def test_alpha_cm_special_values():
    assert physics.alpha_cm(1.0) == 0.0
    assert np.isclose(physics.alpha_cm(4.0), 3.0 / (8.0 * np.pi), rtol=0, atol=1e-15)
    assert np.isclose(physics.alpha_cm(1e12), 3.0 / (4.0 * np.pi), rtol=1e-10)


def test_ldr_tends_to_cm_and_series():
    eps = 1.31 ** 2
    a = physics.alpha_cm(eps)
    for kd in (1e-3, 1e-4):
        S = 0.3
        got = physics.alpha_ldr(eps, kd, 1.0, S)
        # first-order expansion of 1/(1 + a*q),
        # q = (b1 + eps b2 + eps b3 S) kd^2 - (2i/3) kd^3
        q = ((physics.LDR_B1 + eps * physics.LDR_B2 + eps * physics.LDR_B3 * S) * kd ** 2
             - (2j / 3.0) * kd ** 3)
        assert abs(got - a * (1 - a * q)) < 10 * abs(a) * abs(a * q) ** 2 + 1e-15
    assert np.isclose(physics.alpha_ldr(eps, 0.0, 1.0, 0.0), a, rtol=1e-15)


def test_ldr_radiative_reaction_real_eps():
    # Im(1/alpha) = -(2/3)(k dx)^3 exactly when eps is real: the LDR
    # denominator is the only complex term (Section 2.1).
    for eps in (1.31 ** 2, 1.78 ** 2, 4.0):
        for kd in (0.3, 0.625):
            for S in (0.0, 0.5):
                inv = 1.0 / physics.alpha_ldr(eps, kd, 1.0, S)
                assert np.isclose(inv.imag, -(2.0 / 3.0) * kd ** 3, rtol=1e-12)


def test_ldr_S():
    assert physics.ldr_S([0, 0, 1], [1, 0, 0]) == 0.0
    d = np.array([1.0, 1.0, 0.0]) / np.sqrt(2)
    e = np.array([1.0, -1.0, 0.0]) / np.sqrt(2)
    assert np.isclose(physics.ldr_S(d, e), 0.5)


def test_green_on_axis_closed_form():
    k = 1.7
    for r in (0.3, 1.0, 2.5):
        g = physics.green_tensor(np.array([r, 0.0, 0.0]), k)
        ph = np.exp(1j * k * r) / r
        want = ph * (k * k * np.diag([0.0, 1.0, 1.0])
                     + (1j * k * r - 1.0) / r ** 2 * np.diag([-2.0, 1.0, 1.0]))
        assert np.allclose(g, want, rtol=1e-14, atol=0)


def test_green_is_k2_plus_hessian_of_scalar():
    # g = (k^2 I + grad grad) e^{ikr}/r, checked by central differences of
    # the scalar function: independent of the closed form's algebra.
    rng = np.random.default_rng(5)
    k = 2.3
    h = 1e-4
    for _ in range(5):
        R = rng.standard_normal(3) * 1.5
        H = np.zeros((3, 3), dtype=np.complex128)
        f = lambda v: physics.green_scalar(np.linalg.norm(v), k)
        for a in range(3):
            for b in range(3):
                ea = np.eye(3)[a] * h
                eb = np.eye(3)[b] * h
                H[a, b] = (f(R + ea + eb) - f(R + ea - eb) - f(R - ea + eb) + f(R - ea - eb)) / (4 * h * h)
        want = k * k * f(R) * np.eye(3) + H
        got = physics.green_tensor(R, k)
        assert np.allclose(got, want, rtol=1e-5, atol=1e-6 * np.abs(want).max())


def test_green_symmetric_and_even():
    rng = np.random.default_rng(6)
    R = rng.standard_normal((10, 3))
    g = physics.green_tensor(R, 0.9)
    assert np.allclose(g, np.swapaxes(g, -1, -2), rtol=0, atol=1e-15)
    assert np.allclose(g, physics.green_tensor(-R, 0.9), rtol=0, atol=1e-15)


def test_block_parity_against_table1():
    # Parity of each block on each level, found by mirroring the offset
    # along that axis.  Table 1 prints '+' for G_yz on the z level, but
    # g_yz is proportional to r_y r_z, odd in z: that single entry is a
    # misprint and the oracle follows the Green function.
    rows = {r[0]: r[1:] for r in _read_golden("table1_symmetry.txt")}
    names = ["xx", "xy", "xz", "yy", "yz", "zz"]
    R = np.array([0.7, 1.1, 1.9])
    k = 1.3
    g = physics.green_tensor(R, k)
    for c, (a, b) in enumerate(COMPONENTS):
        for ax in range(3):
            Rm = R.copy()
            Rm[ax] = -Rm[ax]
            gm = physics.green_tensor(Rm, k)
            sign = "+" if np.isclose(gm[a, b], g[a, b], rtol=1e-14) else "-"
            if sign == "-":
                assert np.isclose(gm[a, b], -g[a, b], rtol=1e-14)
            if names[c] == "yz" and ax == 2:
                assert rows["yz"][2] == "+" and sign == "-"
            else:
                assert sign == rows[names[c]][ax], (names[c], ax)
