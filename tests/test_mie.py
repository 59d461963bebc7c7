"""Pins for the Mie series used to check the oracle (Bohren & Huffman, cited in Section 3.2):
boundary conditions at the sphere surface between the exterior and interior series, the
Rayleigh limit of the cross sections, the transparent limit and energy conservation."""
import numpy as np
import pytest

from oracle import mie


@pytest.mark.parametrize("eps,x", [(2.25, 1.0), (-8.5 + 0.3j, 0.5), (1.33 ** 2, 5.57 / 1.33), (-10 + 0.4j, 1.5)])
def test_boundary_conditions(eps, x):
    rng = np.random.default_rng(3)
    p = rng.normal(size=(40, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    k, a = x, 1.0
    Eo, Co = mie.fields(p * a, k, a, eps, "outside")
    Ei, Ci = mie.fields(p * a, k, a, eps, "inside")
    n = p
    tang = lambda v: v - np.sum(v * n, 1)[:, None] * n
    scale = np.linalg.norm(Eo)
    assert np.linalg.norm(tang(Eo) - tang(Ei)) < 1e-9 * scale
    assert np.linalg.norm(np.sum(Eo * n, 1) - eps * np.sum(Ei * n, 1)) < 1e-9 * scale
    assert np.linalg.norm(tang(Co) - tang(Ci)) < 1e-9 * np.linalg.norm(Co)


def test_rayleigh_limit():
    k, a = 0.01, 1.0
    for eps in (2.25, -8.5 + 0.3j):
        cext, csca, cabs = mie.cross_sections(k, a, eps)
        al = (eps - 1) / (eps + 2)
        assert abs(csca / (8 * np.pi / 3 * k ** 4 * a ** 6 * abs(al) ** 2) - 1) < 1e-3
        if np.imag(eps) != 0:
            assert abs(cabs / (4 * np.pi * k * a ** 3 * np.imag(al)) - 1) < 1e-3


def test_transparent_and_lossless():
    a_n, b_n, _, _ = mie.coefficients(1.0, 2.0)
    assert np.max(abs(a_n)) < 1e-14 and np.max(abs(b_n)) < 1e-14
    cext, csca, cabs = mie.cross_sections(1.0, 1.0, 2.25)
    assert abs(cabs) < 1e-12 * cext
    cext, csca, cabs = mie.cross_sections(0.5, 1.0, -8.5 + 0.3j)
    assert cabs > 0
