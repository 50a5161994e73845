"""Oracle Riesz map (test infrastructure only; see oracle/__init__.py).

Eq. CMCG_PRECONDITIONIER: the representer g~ of the gradient g = J'(v) in the energy inner
product solves (grad g~0, grad phi) = <g0, phi> for all phi in H^1_D and g~1 = c^2-weighted
identity.  Discretely, with K and M of oracle/grid.py:

    K g~0 = g0,      M g~1 = g1.

When the problem has no Dirichlet node, K is singular with kernel = constants (the paper's
coercivity claim needs Gamma_D non-empty).  Then g~0 is the solution with W-weighted mean
zero, sum_j W_j g~0_j = 0, obtained from the bordered system

    [ K   W ] [ s  ]   [ g0 ]
    [ W^T 0 ] [ mu ] = [ 0  ]

which also projects a rounding-level component of g0 along W out of the right-hand side.

Parity: pinned by the closed-form cosine solution of the Neumann Poisson problem on a box
(each cosine mode is an eigenvector of K with a known eigenvalue) and by the residual test.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import Discretization


class RieszSolver:
    """Sparse direct factorisation of K (or of its bordered form when K is singular)."""

    def __init__(self, dz: Discretization):
        self.dz = dz
        Kaa, ia = dz.K_active_sparse()
        self.ia = ia
        self.singular = not dz.has_dirichlet
        if self.singular:
            w = dz.W.ravel()[ia].reshape(-1, 1)
            mat = sp.bmat([[Kaa, sp.csc_matrix(w)], [sp.csc_matrix(w.T), None]], format="csc")
        else:
            mat = Kaa
        self.lu = spla.splu(mat.tocsc())

    def solve(self, g0) -> np.ndarray:
        dz = self.dz
        rhs = np.asarray(g0, dtype=np.float64).ravel()[self.ia]
        if self.singular:
            rhs = np.concatenate([rhs, [0.0]])
        sol = self.lu.solve(rhs)
        out = np.zeros(dz.size)
        out[self.ia] = sol[: len(self.ia)]
        return out.reshape(dz.shape)

    def representer(self, g0, g1):
        """(g~0, g~1) = (K^+ g0, M^-1 g1)."""
        return self.solve(g0), np.asarray(g1).reshape(self.dz.shape) / self.dz.M * self.dz.act
