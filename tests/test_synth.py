"""Checks of the synthetic input generators against closed forms (CPU)."""
import numpy as np
import scipy.sparse as sp

import synth


def _rigid_modes(xyz):
    """The six rigid-body displacement fields at points xyz (n x 3), stacked
    node-major as 3n vectors: three translations and three rotations."""
    n = len(xyz)
    R = np.zeros((3 * n, 6))
    for k in range(3):
        R[k::3, k] = 1.0
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    R[0::3, 3], R[1::3, 3] = -y, x   # rotation about z
    R[1::3, 4], R[2::3, 4] = -z, y   # about x
    R[0::3, 5], R[2::3, 5] = z, -x   # about y
    return R


def test_q1_element_kernel_is_rigid_body_modes():
    """A free element stores no energy under a rigid motion, and only then:
    its stiffness has exactly the six rigid-body modes as kernel."""
    Ke = synth._q1_elasticity_stiffness(0.3)
    corners = np.array([[ax, ay, az] for az in (0, 1) for ay in (0, 1) for ax in (0, 1)], float)
    R = _rigid_modes(corners)
    assert np.abs(Ke @ R).max() <= 1e-13
    ev = np.linalg.eigvalsh(Ke)
    assert np.abs(ev[:6]).max() <= 1e-13 and ev[6] > 1e-2
    assert np.allclose(Ke, Ke.T, atol=0)


def test_q1_element_uniform_strain_energy():
    """Patch test: a linear field u = G x has constant strain eps = sym(G);
    the element energy u^T K u / 2 equals the exact volume integral
    (lam/2 tr(eps)^2 + mu eps:eps) over the unit cube."""
    nu = 0.3
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1 / (2 * (1 + nu))
    Ke = synth._q1_elasticity_stiffness(nu)
    corners = np.array([[ax, ay, az] for az in (0, 1) for ay in (0, 1) for ax in (0, 1)], float)
    rng = np.random.default_rng(0)
    for _ in range(3):
        G = rng.standard_normal((3, 3))
        u = (corners @ G.T).ravel()
        eps = 0.5 * (G + G.T)
        exact = 0.5 * lam * np.trace(eps) ** 2 + mu * np.sum(eps * eps)
        assert abs(0.5 * u @ Ke @ u - exact) <= 1e-12 * max(1.0, exact)


def test_elasticity_matrix_spd_and_layers():
    """The assembled, clamped stiffness is symmetric positive definite, and
    the layered modulus enters by element: doubling e_stiff changes A."""
    A, f, xyz = synth.elasticity3d(4, layer=1)
    M = sp.csr_matrix((A.val, A.colind, A.rowptr), shape=(A.n, A.n))
    assert A.n == 3 * (5 ** 3 - 5 ** 2)
    assert abs(M - M.T).max() == 0.0
    assert np.linalg.eigvalsh(M.toarray()).min() > 0
    # unit body force: 1/8 of each element to each node, minus the half of the
    # first element layer's load that sits on the clamped face
    assert np.isclose(f.sum(), -(4 ** 3 - 4 ** 2 / 2))
    A2, _, _ = synth.elasticity3d(4, e_stiff=2e5, layer=1)
    assert not np.allclose(A.val, A2.val)
    part = synth.box_partition_dofs(xyz, (3, 3, 3))
    assert part.min() == 0 and len(np.unique(part)) == part.max() + 1
    # the three dofs of a node stay together
    assert np.all(part[0::3] == part[1::3]) and np.all(part[0::3] == part[2::3])
