"""Oracle direct solve (test infrastructure only; see oracle/__init__.py).

The plain definition of the CMCG fixed point.  Substituting y^n = Re(U exp(-i omega t_n))
into the three-level leapfrog scheme of oracle/wave.py (exact because N dt = T) gives the
time-discrete Helmholtz system

    (K - wt^2 M - i wh B) U = F^,   wt = (2/dt) sin(omega dt / 2),   wh = sin(omega dt)/dt,

whose periodic initial state is v0 = Re U, v1 = wh Im U.  This is the "direct solver for
the same discretisation" the paper compares CMCG against in Sec. 4.1 (Eq. discrete_HE),
with the time discretisation folded in so that the agreement is to rounding.

Parity: the direct solve is the library sparse LU of the assembled system; the system itself
is pinned by the continuum plane-wave convergence test and by the manufactured plane wave.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import Discretization


def helmholtz_matrix(dz: Discretization):
    Kaa, ia = dz.K_active_sparse()
    M = dz.M.ravel()[ia]
    B = dz.B.ravel()[ia]
    A = Kaa.astype(np.complex128) + sp.diags(-dz.omega_tilde ** 2 * M - 1j * dz.omega_hat * B)
    return A.tocsc(), ia


def solve(dz: Discretization, F_hat) -> np.ndarray:
    A, ia = helmholtz_matrix(dz)
    rhs = np.asarray(F_hat, dtype=np.complex128).ravel()[ia]
    sol = spla.splu(A).solve(rhs)
    U = np.zeros(dz.size, dtype=np.complex128)
    U[ia] = sol
    return U.reshape(dz.shape)


def periodic_state(dz: Discretization, U):
    """(v0, v1) = (Re U, wh Im U): the initial data of the discrete periodic solution."""
    return np.real(U) * dz.act, dz.omega_hat * np.imag(U) * dz.act

