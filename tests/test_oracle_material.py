"""Oracle material laws against closed forms, textbook values and finite differences."""
import numpy as np
import pytest
from scipy import integrate

from oracle.material import (Reduced, carlson_rd, compliance_apply, contract, cubic_stiffness,
                             ellipsoid_demag_factors, h_anisotropy, h_magnetoelastic,
                             spontaneous_strain, voigt_to_tensor)
from paper_2510_09812_gb300 import synth


def test_carlson_rd_against_quadrature_and_equal_arguments():
    assert carlson_rd(2.0, 2.0, 2.0) == pytest.approx(2.0 ** -1.5, rel=1e-14)
    for x, y, z in [(1.0, 2.0, 3.0), (0.3, 4.0, 0.7), (5.0, 0.2, 1.5)]:
        f = lambda t: 1.5 / (np.sqrt(t + x) * np.sqrt(t + y) * (t + z) ** 1.5)
        val, err = integrate.quad(f, 0, np.inf, epsabs=0, epsrel=1e-13, limit=500)
        assert carlson_rd(x, y, z) == pytest.approx(val, rel=1e-10)


def test_demag_factors_sphere_trace_and_spheroids():
    assert np.allclose(ellipsoid_demag_factors(3.0, 3.0, 3.0), 1.0 / 3.0, rtol=1e-13)
    for axes in [(1.0, 2.0, 3.0), (5.0, 1.0, 0.5), (2.0, 2.0, 7.0)]:
        assert ellipsoid_demag_factors(*axes).sum() == pytest.approx(1.0, rel=1e-12)
    # prolate spheroid a > b = c (Osborn 1945): N_a = (1 - e^2)/e^3 (atanh e - e)
    a, c = 3.0, 1.0
    e = np.sqrt(1 - c * c / (a * a))
    Na = (1 - e * e) / e ** 3 * (np.arctanh(e) - e)
    N = ellipsoid_demag_factors(a, c, c)
    assert N[0] == pytest.approx(Na, rel=1e-11)
    assert N[1] == pytest.approx((1 - Na) / 2, rel=1e-11)
    # oblate spheroid a = b > c: N_c = (1/e^2) (1 - sqrt(1 - e^2) arcsin(e) / e)
    a, c = 4.0, 1.5
    e = np.sqrt(1 - c * c / (a * a))
    Nc = (1 - np.sqrt(1 - e * e) * np.arcsin(e) / e) / e ** 2
    assert ellipsoid_demag_factors(a, a, c)[2] == pytest.approx(Nc, rel=1e-11)


def test_spontaneous_strain_defines_lambda100_lambda111():
    l100, l111 = 2.07e-5, -2.12e-5
    # magnetised along [100]: strain lambda100 along the field, -lambda100/2 across (volume kept)
    E = spontaneous_strain(np.array([1.0, 0.0, 0.0]), l100, l111)
    assert np.allclose(E, np.diag([l100, -l100 / 2, -l100 / 2]), rtol=1e-15, atol=0)
    # magnetised along [111]: relative elongation along [111] is lambda111, no normal strains
    n = np.ones(3) / np.sqrt(3)
    E = spontaneous_strain(n, l100, l111)
    assert np.allclose(np.diag(E), 0.0, atol=1e-20)
    assert n @ E @ n == pytest.approx(l111, rel=1e-14)
    # unit magnetisation: magnetostriction conserves volume
    m = synth.random_unit_m(50, 3)
    assert np.abs(np.trace(spontaneous_strain(m, l100, l111), axis1=1, axis2=2)).max() < 1e-15 * l100


def test_compliance_inverts_cubic_stiffness():
    C = cubic_stiffness(243e9, 138e9, 122e9)
    s = voigt_to_tensor([6e6, -2e6, 1e6, 3e5, -4e5, 2e5])
    E = compliance_apply(243e9, 138e9, 122e9, s)
    assert np.allclose(contract(C, E), s, rtol=1e-12, atol=1e-6)


def _fd_grad(fun, m, step=1e-6):
    g = np.zeros(3)
    for i in range(3):
        d = np.zeros(3); d[i] = step
        g[i] = (fun(m + d) - fun(m - d)) / (2 * step)
    return g


def test_local_fields_are_minus_energy_derivatives():
    # h = -(1/(mu0 ms^2)) dPsi/dm for the anisotropy and magnetoelastic densities of Eq. 1,
    # checked by central differences of the densities themselves
    mat = synth.fe_like_material()
    red = Reduced(mat, 1e-12, 0.5)
    C = red.C
    E = np.array([[3e-5, 1e-5, -2e-5], [1e-5, -4e-5, 0.5e-5], [-2e-5, 0.5e-5, 1e-5]])
    for m in synth.random_unit_m(4, 11):
        an = lambda v: mat["K1"] * (v[0] ** 2 * v[1] ** 2 + v[1] ** 2 * v[2] ** 2
                                    + v[2] ** 2 * v[0] ** 2)
        assert np.allclose(h_anisotropy(m[None], red.kappa)[0],
                           -_fd_grad(an, m) / red.scale, rtol=1e-7, atol=1e-12)

        def el(v):
            D = E - spontaneous_strain(v, red.l100, red.l111)
            return 0.5 * np.einsum("ij,ij->", D, contract(C, D))
        sigma = contract(C, E - spontaneous_strain(m, red.l100, red.l111))
        assert np.allclose(h_magnetoelastic(m[None], sigma[None], red)[0],
                           -_fd_grad(el, m, 1e-4) / red.scale, rtol=1e-6, atol=1e-14)


def test_reduced_constants_fe_like():
    red = Reduced(synth.fe_like_material(), 1e-12, 0.5)
    assert red.scale == pytest.approx(3.674528e6, rel=1e-5)       # mu0 ms^2
    assert red.A_star == pytest.approx(11.43003, rel=1e-5)
    assert red.dtau == pytest.approx(0.3783822, rel=1e-6)         # gamma0 ms dt
