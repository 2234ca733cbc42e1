"""App. D (rotated coordinate system) in the oracle: the rotation and its Voigt (Bond) matrix
against the tensor definitions, the rotated cubic stiffness against closed forms and rotation
invariants, saturation magnetostriction of a free body along <111> and <110> against the
classic direction formula, and the macrospin reduction with rotated anisotropy."""
import numpy as np
import pytest

from oracle.gspm import System
from oracle.material import (bond_matrix, cubic_stiffness, rotation_111, stiffness_from_voigt,
                             tensor_to_voigt, voigt_stiffness, voigt_to_tensor)
from oracle_helpers import periodic
from paper_2510_09812_gb300 import synth

C11, C12, C44 = 243e9, 138e9, 122e9


def test_rotation_111_is_proper_and_along_111():
    R = rotation_111()
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-15)
    assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-15)
    # v_mesh = R v_crystal: the crystal's [111] is the mesh x axis
    assert np.allclose(R @ (np.ones(3) / np.sqrt(3)), [1, 0, 0], atol=1e-15)


def test_bond_matrix_rotates_symmetric_tensors():
    rng = np.random.default_rng(0)
    R = rotation_111()
    M = bond_matrix(R)
    assert np.array_equal(bond_matrix(np.eye(3)), np.eye(6))
    for _ in range(5):
        A = rng.standard_normal((3, 3))
        E = A + A.T
        assert np.allclose(M @ tensor_to_voigt(E), tensor_to_voigt(R @ E @ R.T), atol=1e-14)
    assert np.allclose(np.linalg.inv(M), bond_matrix(R.T), atol=1e-14)


def test_rotated_cubic_stiffness_closed_forms_and_invariants():
    R = rotation_111()
    M = bond_matrix(R)
    D = M @ voigt_stiffness(C11, C12, C44) @ M.T
    C = stiffness_from_voigt(D)
    # the same tensor by rotating C_ijkl index by index
    Cr = np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, cubic_stiffness(C11, C12, C44))
    assert np.abs(C - Cr).max() < 1e-14 * C11
    # longitudinal modulus along <111> = n_i n_j n_k n_l C_ijkl (derived by hand)
    assert D[0, 0] == pytest.approx((C11 + 2 * C12 + 4 * C44) / 3, rel=1e-14)
    # rotation invariants C_iijj = 3 C11 + 6 C12 and C_ijij = 3 C11 + 6 C44
    assert np.einsum("iijj->", C) == pytest.approx(3 * C11 + 6 * C12, rel=1e-14)
    assert np.einsum("ijij->", C) == pytest.approx(3 * C11 + 6 * C44, rel=1e-14)
    # an isotropic stiffness (C11 - C12 = 2 C44) does not change
    Di = voigt_stiffness(2.0e11 + 2 * 0.8e11, 2.0e11, 0.8e11)
    assert np.abs(M @ Di @ M.T - Di).max() < 1e-14 * Di.max()


def _free_body(R, direction):
    mat = synth.fe_like_material()
    mat["R"] = R.reshape(-1).tolist()
    mesh, wm = periodic((2, 2, 2), (8.0, 8.0, 8.0), jitter=0.2, seed=21)
    s = System(wm, mat, 1e-12, 0.5)
    n = np.asarray(direction, float)
    n /= np.linalg.norm(n)
    return mat, s, s.solve_elastic(np.tile(n, (s.n, 1)), np.zeros((s.n, 3))), n


@pytest.mark.parametrize("crystal_dir,expect", [
    ((1, 1, 1), lambda l100, l111: l111),
    ((-1, 1, 0), lambda l100, l111: (l100 + 3 * l111) / 4)])
def test_rotated_free_body_magnetostriction_along_m(crystal_dir, expect):
    """Elongation along a magnetisation direction a of a free cubic body:
    (3/2) l100 (sum a_i^4 - 1/3) + 3 l111 sum_{i<j} a_i^2 a_j^2 -> l111 for <111>,
    (l100 + 3 l111) / 4 for <110>, measured in the mesh axes."""
    R = rotation_111()
    a = np.asarray(crystal_dir, float) / np.linalg.norm(crystal_dir)
    mat, s, el, n = _free_body(R, R @ a)
    assert np.abs(el["u"]).max() < 1e-15
    E_along = np.einsum("i,nij,j->n", n, el["E"], n)
    assert np.allclose(E_along, expect(mat["lambda100"], mat["lambda111"]), rtol=1e-12, atol=0)
    assert np.abs(el["sigma"]).max() < 1e-5            # Pa: stress-free


def test_rotated_uniform_state_reduces_to_rotated_macrospin():
    """No magnetostriction: for uniform m the rotated FEM step equals Algorithm B.1 on one spin
    whose anisotropy field is R h_anis(R^T v)."""
    mat = synth.fe_like_material()
    mat.update(lambda100=0.0, lambda111=0.0, Nd=[0.2, 0, 0, 0, 0.3, 0, 0, 0, 0.5])
    R = rotation_111()
    mat["R"] = R.reshape(-1).tolist()
    mesh, wm = periodic((2, 2, 2), (8.0, 8.0, 8.0), jitter=0.2, seed=21)
    s = System(wm, mat, 2e-12, 0.3)
    red = s.red
    H = np.array([1e4, -3e4, 2e4])

    def hv(v):
        vc = R.T @ v
        vc2 = vc ** 2
        h_an = R @ (-red.kappa * vc * (vc2.sum() - vc2))
        return h_an + H / red.Ms - red.Nd @ v

    m0 = np.array([0.3, -0.5, 0.8]); m0 /= np.linalg.norm(m0)
    m = np.tile(m0, (s.n, 1))
    U, u = np.zeros(s.n), np.zeros((s.n, 3))
    v = m0.copy()
    for _ in range(5):
        m, U, u, _ = s.step(m, U, u, H)
        h0 = hv(v)
        g = v + red.dtau * h0
        a1 = v[0] + g[1] * v[2] - g[2] * v[1]
        gs1 = a1 + red.dtau * h0[0]
        a2 = v[1] + g[2] * a1 - gs1 * v[2]
        gs2 = a2 + red.dtau * h0[1]
        a3 = v[2] + gs1 * a2 - gs2 * a1
        ms = np.array([a1, a2, a3])
        mss = ms + red.alpha * red.dtau * hv(ms)
        v = mss / np.linalg.norm(mss)
        assert np.abs(m - v[None]).max() < 1e-13
