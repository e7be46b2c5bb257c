"""Pins of the oracle's cross sections: Rayleigh dipole, optical theorem, Mie series."""
import numpy as np
import pytest
from scipy import special

from dda_inputs import hex_prism_mask, sphere_mask
from oracle import observables, physics
from oracle.problem import Problem


def test_single_voxel_rayleigh():
    k, dx = 0.8, 0.2
    eps = 1.5 + 0.2j
    mat = np.ones((1, 1, 1), dtype=np.uint8)
    d = np.array([0.0, 0.0, 1.0]); e = np.array([1.0, 0.0, 0.0])
    p = Problem(mat=mat, dx=dx, k=k, eps=[eps], d=d, e=e)
    c = p.solve_direct()
    a = physics.alpha_ldr(eps, k, dx, 0.0)
    assert np.allclose(c[:, 0, 0, 0], a * e, rtol=1e-14)
    cext, cabs, csca = p.cross_sections(c, pairs=True)
    assert np.isclose(cext, 4 * np.pi * k * dx ** 3 * a.imag, rtol=1e-12)
    assert np.isclose(csca, 8 * np.pi / 3 * k ** 4 * dx ** 6 * abs(a) ** 2, rtol=1e-12)
    assert np.isclose(cext, cabs + csca, rtol=1e-12)


@pytest.mark.parametrize("m_index", [1.31, 1.31 + 0.05j, 1.78])
def test_optical_theorem_and_csca_routes(m_index):
    l = m = n = 8
    dx, k = 2.0 / 8, 2.5
    mat = hex_prism_mask(l, m, n, dx, 1.0, 2.0)
    d = np.array([0.3, 0.5, 0.81]); d /= np.linalg.norm(d)
    e = np.cross(d, [0, 0, 1.0]); e /= np.linalg.norm(e)
    p = Problem(mat=mat, dx=dx, k=k, eps=[complex(m_index) ** 2], d=d, e=e)
    c = p.solve_direct()
    cext, cabs, csca = p.cross_sections(c, pairs=True)
    assert abs(cext - (cabs + csca)) < 1e-10 * cext
    assert np.isclose(observables.c_sca_fft(c, mat, dx, k), csca, rtol=1e-11)
    assert np.isclose(observables.c_sca_farfield(c, mat, dx, k, 32, 64), csca, rtol=1e-9)
    if complex(m_index).imag == 0:
        assert abs(cabs) < 1e-12 * cext
    else:
        assert cabs > 0


def _mie_q(m, x, nmax=None):
    """Bohren-Huffman Mie series for Q_ext, Q_sca of a homogeneous sphere."""
    if nmax is None:
        nmax = int(x + 4 * x ** (1 / 3) + 2) + 5
    nn = np.arange(1, nmax + 1)
    mx = m * x
    jx = special.spherical_jn(nn, x)
    jxp = special.spherical_jn(nn, x, derivative=True)
    yx = special.spherical_yn(nn, x)
    yxp = special.spherical_yn(nn, x, derivative=True)
    jm = special.spherical_jn(nn, mx)
    jmp = special.spherical_jn(nn, mx, derivative=True)
    psi_x, dpsi_x = x * jx, jx + x * jxp
    xi_x, dxi_x = x * (jx + 1j * yx), (jx + 1j * yx) + x * (jxp + 1j * yxp)
    psi_m, dpsi_m = mx * jm, jm + mx * jmp
    a = (m * psi_m * dpsi_x - psi_x * dpsi_m) / (m * psi_m * dxi_x - xi_x * dpsi_m)
    b = (psi_m * dpsi_x - m * psi_x * dpsi_m) / (psi_m * dxi_x - m * xi_x * dpsi_m)
    qext = 2 / x ** 2 * np.sum((2 * nn + 1) * np.real(a + b))
    qsca = 2 / x ** 2 * np.sum((2 * nn + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    return qext, qsca


def test_mie_small_sphere_textbook_values():
    # Rayleigh limit of the Mie series: Q_sca -> (8/3) x^4 |(m^2-1)/(m^2+2)|^2
    m, x = 1.5, 0.01
    qext, qsca = _mie_q(m, x)
    assert np.isclose(qsca, 8 / 3 * x ** 4 * abs((m * m - 1) / (m * m + 2)) ** 2, rtol=1e-3)


@pytest.mark.parametrize("m_index,x", [(1.31, 1.0), (1.31 + 0.05j, 1.5)])
def test_dda_sphere_close_to_mie(m_index, x):
    # The whole chain (polarizability, Green function, units, cross sections)
    # against the Mie series of an independent textbook solution.  DDA with
    # ~14 voxels across the sphere is accurate to about a percent.
    N = 14
    dx = 1.0
    mat = sphere_mask(N, N, N, dx, N / 2.0 - 1e-9)
    n_ice = int((mat > 0).sum())
    a_eq = (3.0 * n_ice / (4.0 * np.pi)) ** (1.0 / 3.0) * dx
    k = x / a_eq
    p = Problem(mat=mat, dx=dx, k=k, eps=[complex(m_index) ** 2],
                d=np.array([0, 0, 1.0]), e=np.array([1.0, 0, 0]))
    c, info = p.solve_gmres("none", tol=1e-10, restart=100)
    cext, cabs, csca = p.cross_sections(c)
    qext_mie, qsca_mie = _mie_q(complex(m_index), x)
    geo = np.pi * a_eq ** 2
    assert abs(cext / geo - qext_mie) / qext_mie < 0.03
    assert abs(csca / geo - qsca_mie) / qsca_mie < 0.03
