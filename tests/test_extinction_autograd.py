"""The autograd wrapper of C_ext (dda.extinction): its backward (adjoint solve,
per-voxel gradient, sum per material, PyTorch's complex convention) checked on
the CPU with a stand-in plan whose solves, cross sections and gradients are the
oracle's, against central finite differences of the forward.  The GPU pieces
it calls (solve, dda_adjoint_rhs, dda_ext_gradient) have their own GPU tests."""
import numpy as np
import pytest
import torch

from dda_inputs import hex_prism_mask
from oracle import adjoint, operator
from oracle.problem import Problem


class _Res:
    def __init__(self, x):
        self.x = x


class OraclePlan:
    def __init__(self, mat, eps, dx, k, nrhs, krylov_m, precond2, voxel_eps=None):
        self.mat_np = mat.numpy()
        self.eps, self.dx, self.k = eps, dx, k
        if voxel_eps is not None:
            # one material per scatterer voxel: the oracle's per-material
            # polarizabilities become per-voxel ones
            ve = voxel_eps.numpy()
            idx = np.argwhere(self.mat_np > 0)
            relab = np.zeros_like(self.mat_np)
            for q, (z, y, x) in enumerate(idx):
                relab[z, y, x] = q + 1
            self.mat_np = relab
            self.eps = [complex(ve[z, y, x]) for z, y, x in idx]

    def set_incidence(self, dirs, pols):
        self.probs = [Problem(mat=self.mat_np, dx=self.dx, k=self.k, eps=self.eps, d=np.asarray(d),
                              e=np.asarray(e)) for d, e in zip(dirs, pols)]

    def precond_build(self):
        pass

    def solve(self, b=None, **kw):
        xs = []
        for r, p in enumerate(self.probs):
            A = operator.dense_matrix(p.mat, p.alpha_inv_vox, p.k, p.dx)
            rhs = p.rhs() if b is None else b[r].numpy()
            xs.append(operator.ice_to_box(np.linalg.solve(A, operator.box_to_ice(rhs, p.mat)),
                                          p.mat))
        return _Res(torch.from_numpy(np.stack(xs)))

    def cross_sections(self, x):
        return np.array([list(p.cross_sections(x[r].numpy())) for r, p in enumerate(self.probs)])

    def adjoint_rhs(self, nrhs):
        return torch.from_numpy(np.stack([adjoint.adjoint_rhs(p) for p in self.probs]))

    def ext_gradient_from(self, c, lam):
        return torch.from_numpy(np.stack([adjoint.ext_gradient(p, c[r].numpy(), lam[r].numpy())
                                          for r, p in enumerate(self.probs)]))


def test_extinction_gradient_matches_finite_differences():
    from paper_1903_09802_gb300 import dda
    l = m = n = 4
    dx, k = 0.3, 2.0
    mat = hex_prism_mask(l, m, n, dx, 0.55, 1.2)
    mat[mat > 0] = np.where(np.arange(int((mat > 0).sum())) % 3 == 0, 2, 1).astype(np.uint8)
    mat_t = torch.from_numpy(mat)
    dirs = [np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])]
    pols = [np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])]
    eps0 = np.array([1.7 + 0.05j, 2.2 + 0.1j])
    w = torch.tensor([1.0, 0.7], dtype=torch.float64)

    def loss(e):
        c = dda.extinction(e, mat_t, dx, k, dirs, pols, plan_factory=OraclePlan)
        return (w * c).sum()

    eps = torch.tensor(eps0, dtype=torch.complex128, requires_grad=True)
    loss(eps).backward()
    h = 1e-6
    for j in range(2):
        for part, unit in ((0, 1.0), (1, 1j)):
            ep = eps0.copy(); ep[j] += h * unit
            em = eps0.copy(); em[j] -= h * unit
            fd = (loss(torch.tensor(ep)).item() - loss(torch.tensor(em)).item()) / (2 * h)
            got = eps.grad[j].real.item() if part == 0 else eps.grad[j].imag.item()
            assert got == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_extinction_gradient_per_voxel_matches_finite_differences():
    # eps of shape (n, m, l): one permittivity per voxel, gradient per voxel
    # (zero on air), against central differences of the forward
    from paper_1903_09802_gb300 import dda
    l = m = n = 4
    dx, k = 0.3, 2.0
    mat = hex_prism_mask(l, m, n, dx, 0.55, 1.2)
    mat_t = torch.from_numpy(mat)
    rng = np.random.default_rng(7)
    eps0 = (1.7 + 0.05j) + 0.2 * rng.standard_normal(mat.shape) + 0.02j * rng.random(mat.shape)
    dirs = [np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])]
    pols = [np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])]
    w = torch.tensor([1.0, 0.7], dtype=torch.float64)

    def loss(e):
        return (w * dda.extinction(e, mat_t, dx, k, dirs, pols, plan_factory=OraclePlan)).sum()

    eps = torch.tensor(eps0, dtype=torch.complex128, requires_grad=True)
    loss(eps).backward()
    g = eps.grad.numpy()
    assert np.all(g[mat == 0] == 0)
    h = 1e-6
    ice = np.argwhere(mat > 0)
    for t in rng.choice(len(ice), 5, replace=False):
        z, y, x = ice[t]
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            ep = eps0.copy(); ep[z, y, x] += h * unit
            em = eps0.copy(); em[z, y, x] -= h * unit
            fd = (loss(torch.tensor(ep)).item() - loss(torch.tensor(em)).item()) / (2 * h)
            assert part(g[z, y, x]) == pytest.approx(fd, rel=1e-5, abs=1e-9)
