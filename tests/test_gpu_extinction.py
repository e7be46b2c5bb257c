"""The differentiable extinction (dda.extinction) on the GPU: C_ext per
incident wave and its gradient in the materials' permittivities (adjoint solve,
per-voxel gradient summed per material) against the oracle's direct solves of
the same two-material prism, with the 3-level and the 2-level preconditioner."""
import numpy as np
import pytest
import torch

from dda_inputs import hex_prism_mask
from gpu_util import dda_module, to_dev
from oracle import adjoint, operator
from oracle.problem import Problem


def _oracle(mat, dx, k, eps, dirs, pols, w):
    cext, grad = [], np.zeros(len(eps), dtype=np.complex128)
    for r, (d, e) in enumerate(zip(dirs, pols)):
        prob = Problem(mat=mat, dx=dx, k=k, eps=list(eps), d=d, e=e)
        A = operator.dense_matrix(prob.mat, prob.alpha_inv_vox, prob.k, prob.dx)
        solve = lambda b: operator.ice_to_box(  # noqa: E731
            np.linalg.solve(A, operator.box_to_ice(b, prob.mat)), prob.mat)
        c, lam = solve(prob.rhs()), solve(adjoint.adjoint_rhs(prob))
        cext.append(adjoint.c_ext_of(prob, c))
        g = adjoint.ext_gradient(prob, c, lam)
        for j in range(len(eps)):
            sel = mat == j + 1
            grad[j] += w[r] * complex(g[0][sel].sum(), g[1][sel].sum())
    return np.array(cext), grad


@pytest.mark.gpu
@pytest.mark.late(3)
@pytest.mark.parametrize("precond", [3, 2])
def test_extinction_and_gradient_vs_oracle(precond):
    dda = dda_module()
    l = m = n = 8
    dx, k = 0.25, 2.2
    mat = hex_prism_mask(l, m, n, dx, 0.75, 1.5)
    mat[mat > 0] = np.where(np.arange(int((mat > 0).sum())) % 3 == 0, 2, 1).astype(np.uint8)
    dirs = [np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])]
    pols = [np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])]
    eps0 = np.array([(1.31 + 0.02j) ** 2, (1.5 + 0.05j) ** 2])
    w = np.array([1.0, 0.7])
    want_c, want_g = _oracle(mat, dx, k, eps0, dirs, pols, w)

    eps = torch.tensor(eps0, dtype=torch.complex128, requires_grad=True)
    c = dda.extinction(eps, to_dev(mat, torch.uint8), dx, k, dirs, pols, tol=1e-12, restart=40,
                       precond=precond, inner_prec=dda.C128)
    assert c.dtype == torch.float64 and c.shape == (2,)
    assert np.abs(c.detach().numpy() - want_c).max() <= 1e-9 * np.abs(want_c).max()
    (torch.tensor(w) * c).sum().backward()
    got = eps.grad.numpy()
    assert np.abs(got - want_g).max() <= 1e-8 * np.abs(want_g).max()
