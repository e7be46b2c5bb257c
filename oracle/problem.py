"""Assemble one scattering problem and solve it (oracle, test infrastructure only).

alpha_tilde (Section 3.1 and eq. 20): the constant diagonal of the
preconditioner is the polarizability of the scatterer's material ("ice").
With several materials this reads as the most frequent non-air material,
ties going to the lowest index.

Preconditioner on the scatterer (reading of Sections 1 and 3.1): the
unknowns live on scatterer voxels only (eq. 8), while P is the matrix of the
whole box "filled in with ice".  P^{-1} acts on an unknown vector by
extending it with zeros over the air voxels, applying the box-level inverse
and keeping the scatterer voxels:  z = M o P^{-1}(M o v),  M the scatterer
mask.  Applying P^{-1} to the full box vector instead (air unknowns kept in
the Krylov space) converges far worse and is not what the paper describes.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import circulant, krylov, observables, operator, physics


@dataclass
class Problem:
    mat: np.ndarray            # (n, m, l) uint8, 0 = air
    dx: float
    k: float
    eps: list                  # permittivity per material 1..K
    d: np.ndarray              # unit incidence direction
    e: np.ndarray              # unit polarisation

    @property
    def dims(self):
        n, m, l = self.mat.shape
        return l, m, n

    @property
    def S(self) -> float:
        return physics.ldr_S(self.d, self.e)

    @property
    def alphas(self) -> np.ndarray:
        return np.array([physics.alpha_ldr(eps, self.k, self.dx, self.S) for eps in self.eps])

    @property
    def alpha_inv_vox(self) -> np.ndarray:
        return operator.alpha_inv_box(self.mat, self.alphas)

    @property
    def alpha_tilde_inv(self) -> complex:
        counts = np.bincount(self.mat.reshape(-1), minlength=len(self.eps) + 1)[1:]
        if counts.sum() == 0:
            return complex(1.0 / self.alphas[0])
        return complex(1.0 / self.alphas[int(np.argmax(counts))])

    def rhs(self) -> np.ndarray:
        return observables.incident_field(self.mat, self.dx, self.k, self.d, self.e)

    def kernel_spectrum(self):
        l, m, n = self.dims
        return operator.kernel_spectrum(l, m, n, self.dx, self.k)

    def matvec(self, c, Ghat=None):
        return operator.fft_matvec(c, self.mat, self.alpha_inv_vox, self.alpha_tilde_inv,
                                   self.k, self.dx, Ghat)

    def precond3(self, restrict: bool = True, kind: str = "chan"):
        """3-level preconditioner; restricted to the scatterer unless restrict=False.

        kind: "chan" (eq. 13) or "strang" (Strang's circulant)."""
        l, m, n = self.dims
        lam = circulant.precond3_lambda(l, m, n, self.dx, self.k, self.alpha_tilde_inv, kind)
        lam_inv = np.linalg.inv(lam)
        ice = (self.mat > 0)[None]
        if not restrict:
            return lambda v: circulant.precond3_apply(v, lam_inv)
        return lambda v: circulant.precond3_apply(v * ice, lam_inv) * ice

    def precond2(self, restrict: bool = True, kind: str = "chan", axis: str = "z"):
        """The paper's 2-level preconditioner; restricted to the scatterer by default.

        axis: the Toeplitz (dense) level, z in the paper; x or y through the
        relabelled frame of circulant.to_toeplitz_frame."""
        l, m, n = circulant.toeplitz_frame_dims(*self.dims, axis)
        blocks = circulant.precond2_blocks(l, m, n, self.dx, self.k, self.alpha_tilde_inv, kind)
        ice = (self.mat > 0)[None] if restrict else True

        def apply(v):
            w = circulant.to_toeplitz_frame(v * ice, axis)
            return circulant.from_toeplitz_frame(circulant.precond2_apply(w, blocks), axis) * ice
        return apply

    def solve_direct(self) -> np.ndarray:
        A = operator.dense_matrix(self.mat, self.alpha_inv_vox, self.k, self.dx)
        b = operator.box_to_ice(self.rhs(), self.mat)
        return operator.ice_to_box(np.linalg.solve(A, b), self.mat)

    def solve_gmres(self, precond: str = "none", tol: float = 1e-6, restart: int = 50,
                    maxiter: int = 2000, side: str = "right"):
        Ghat = self.kernel_spectrum()
        M = {"none": None, "3": self.precond3, "2": self.precond2,
             "3s": lambda: self.precond3(kind="strang"),
             "2s": lambda: self.precond2(kind="strang"),
             "2x": lambda: self.precond2(axis="x"), "2y": lambda: self.precond2(axis="y")}[precond]
        M = M() if M is not None else None
        return krylov.gmres(lambda v: self.matvec(v, Ghat), self.rhs(), tol=tol,
                            restart=restart, maxiter=maxiter, precond=M, side=side)

    def cross_sections(self, c_box, pairs: bool = False):
        b = self.rhs()
        cext = observables.c_ext(c_box, b, self.dx, self.k)
        cabs = observables.c_abs(c_box, self.mat, self.alpha_inv_vox, self.dx, self.k)
        if pairs:
            csca = observables.c_sca_pairs(c_box, self.mat, self.dx, self.k)
        else:
            csca = observables.c_sca_fft(c_box, self.mat, self.dx, self.k)
        return cext, cabs, csca


def from_case(case, rhs: int = 0) -> Problem:
    """Problem for right-hand side ``rhs`` of a dda_inputs.PrismCase."""
    return Problem(mat=case.mask(), dx=case.dx, k=case.k, eps=list(case.eps),
                   d=np.asarray(case.dirs[rhs]), e=np.asarray(case.pols[rhs]))
