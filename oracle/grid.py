"""Oracle discretisation (test infrastructure only; see oracle/__init__.py).

The paper discretises in space with mass-lumped P1/P2 finite elements (Sec. 4.1, Sec. 4.3)
and in time with leapfrog and T/dt an integer (Sec. 4.3.1).  On a Cartesian grid the
mass-lumped Q1 element is the vertex-centred finite-difference scheme written out here:

  nodes         x_j = j h, j in {0..n}^d
  axis weight   w(j_a) = 1/2 at j_a in {0, n_a}, else 1
  volume        W_j = h^d prod_a w(j_a)                     (lumped mass of a node)
  stiffness     K = sum over grid links (j, j+e_a) of  h^(d-2) prod_{b!=a} w(j_b) (y_j - y_{j+e_a})^2 / 2
                 differentiated, i.e. (K y)_j = sum_links weight (y_j - y_nbr)   (energy (grad y, grad y))
                 4th order: K = W * (-Lap_h^(4)), per axis [-1/12, 4/3, -5/2, 4/3, -1/12]/h^2
                 with even reflection y_{-m} = y_m, y_{n+m} = y_{n-m}
  ABC area      A_j = sum over absorbing faces through j of h^(d-1) prod_{b!=a} w(j_b)
  mass          M = diag(W / c^2)                             ((1/c^2) y_tt term of Eq. WE)
  damping       B = diag(A / c)                               ((1/c) y_t on Gamma_S, Eq. WE)
  load          F^ = W f^ + A g^,  F^n = Re(F^ exp(-i omega n dt))   (right-hand sides of Eq. WE)
  Dirichlet     nodes on Dirichlet faces or in the obstacle mask are held at 0 and dropped from
                every vector (homogeneous g_D only); their links still enter K rows of active
                neighbours through y_j - 0.
  time          T = 2 pi / omega, N = ceil(T/dt_target - 1e-9), dt = T/N (T/dt integer, Sec. 4.3.1)
  CFL           dt^2 max c^2 rho < 4 with rho = 4d/h^2 (2nd order) or 16d/(3h^2) (4th order)

Parity: K is pinned to the closed-form Neumann eigenpairs (cosine modes, eigenvalues
(4/h^2) sin^2(pi k/(2n)) per axis, and the 4th-order symbol); M, B and F are pinned by the
continuum plane-wave convergence test; the time step by the discrete energy identity.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

ABC, NEUMANN, DIRICHLET = 0, 1, 2


def _axis_weight(m: int) -> np.ndarray:
    w = np.ones(m + 1)
    w[0] = 0.5
    w[-1] = 0.5
    return w


class Discretization:
    """All discrete operators of one problem.  Fields are numpy arrays in grid shape
    (nz+1, ny+1, nx+1) or (ny+1, nx+1); x is the fastest (last) numpy axis."""

    def __init__(self, n, h, c, omega, faces, dt_target, order=2, mask=None):
        self.n = tuple(int(m) for m in n)
        self.dim = len(self.n)
        if self.dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.shape = tuple(m + 1 for m in reversed(self.n))
        self.size = int(np.prod(self.shape))
        self.h = float(h)
        self.c = np.asarray(c, dtype=np.float64).reshape(self.shape)
        self.omega = float(omega)
        self.faces = tuple(int(f) for f in faces)
        self.order = int(order)
        d = self.dim

        # Dirichlet set: Dirichlet faces plus the obstacle mask.
        dir_nodes = np.zeros(self.shape, dtype=bool)
        for a in range(d):
            for side in (0, 1):
                if self.faces[2 * a + side] == DIRICHLET:
                    dir_nodes[self._face_slice(a, side)] = True
        if mask is not None:
            dir_nodes |= np.asarray(mask).reshape(self.shape) != 0
        self.dirichlet = dir_nodes
        self.has_dirichlet = bool(dir_nodes.any())
        self.act = (~dir_nodes).astype(np.float64)

        # Per-axis weights broadcast in numpy order.
        self.axis_w = []
        for a in range(d):
            shp = [1] * d
            shp[d - 1 - a] = self.n[a] + 1
            self.axis_w.append(_axis_weight(self.n[a]).reshape(shp))
        W = np.full(self.shape, self.h ** d)
        for a in range(d):
            W = W * self.axis_w[a]
        self.W = W

        A = np.zeros(self.shape)
        for a in range(d):
            face_w = np.full(self.shape, self.h ** (d - 1))
            for b in range(d):
                if b != a:
                    face_w = face_w * self.axis_w[b]
            for side in (0, 1):
                if self.faces[2 * a + side] == ABC:
                    sl = self._face_slice(a, side)
                    A[sl] += face_w[sl]
        self.A = A * self.act

        self.M = self.W / self.c ** 2
        self.B = self.A / self.c

        self.Kmat = self._build_K()

        # Time discretisation.
        self.T = 2.0 * math.pi / self.omega
        self.N = int(math.ceil(self.T / float(dt_target) - 1e-9))
        self.dt = self.T / self.N
        rho = (4.0 * d if self.order == 2 else 16.0 * d / 3.0) / self.h ** 2
        if self.dt ** 2 * float(np.max(self.c)) ** 2 * rho >= 4.0:
            raise ValueError("CFL violated: dt^2 c_max^2 rho >= 4")
        # Discrete frequencies of the time-discrete Helmholtz problem (see oracle/direct.py).
        self.omega_tilde = 2.0 / self.dt * math.sin(self.omega * self.dt / 2.0)
        self.omega_hat = math.sin(self.omega * self.dt) / self.dt

    # ------------------------------------------------------------------------------------
    def _face_slice(self, a, side):
        sl = [slice(None)] * self.dim
        sl[self.dim - 1 - a] = 0 if side == 0 else self.n[a]
        return tuple(sl)

    def _flat_index(self):
        return np.arange(self.size).reshape(self.shape)

    def _build_K(self):
        d = self.dim
        if self.order == 2:
            # Stiffness written link by link.
            idx = self._flat_index()
            rows, cols, vals = [], [], []
            for a in range(d):
                ax = d - 1 - a
                lo = [slice(None)] * d
                hi = [slice(None)] * d
                lo[ax] = slice(0, self.n[a])
                hi[ax] = slice(1, self.n[a] + 1)
                lo, hi = tuple(lo), tuple(hi)
                wl = np.full(self.shape, self.h ** (d - 2))
                for b in range(d):
                    if b != a:
                        wl = wl * self.axis_w[b]
                wl = wl[lo].ravel()
                i0 = idx[lo].ravel()
                i1 = idx[hi].ravel()
                rows += [i0, i1, i0, i1]
                cols += [i0, i1, i1, i0]
                vals += [wl, wl, -wl, -wl]
            K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                              shape=(self.size, self.size)).tocsr()
        elif self.order == 4:
            stencil = {-2: -1.0 / 12.0, -1: 4.0 / 3.0, 0: -5.0 / 2.0, 1: 4.0 / 3.0, 2: -1.0 / 12.0}
            mats = []
            for a in range(d):
                m = self.n[a]
                L = sp.lil_matrix((m + 1, m + 1))
                for i in range(m + 1):
                    for off, s in stencil.items():
                        k = i + off
                        if k < 0:
                            k = -k
                        if k > m:
                            k = 2 * m - k
                        L[i, k] += -s / self.h ** 2
                mats.append(L.tocsr())
            Lfull = sp.csr_matrix((self.size, self.size))
            for a in range(d):
                term = None
                for b in reversed(range(d)):  # numpy order: z outermost
                    blk = mats[a] if b == a else sp.identity(self.n[b] + 1, format="csr")
                    term = blk if term is None else sp.kron(term, blk, format="csr")
                Lfull = Lfull + term
            K = sp.diags(self.W.ravel()) @ Lfull
            K = K.tocsr()
            if self.has_dirichlet:
                raise ValueError("4th order with Dirichlet nodes is unsupported")
        else:
            raise ValueError("order must be 2 or 4")
        return K

    # ------------------------------------------------------------------------------------
    def K(self, y: np.ndarray) -> np.ndarray:
        """K y restricted to the active nodes (input and output zero on Dirichlet nodes)."""
        return (self.Kmat @ (y * self.act).ravel()).reshape(self.shape) * self.act

    def load(self, f_hat=None, g_hat=None):
        """Complex load amplitude F^ = W f^ + A g^, zero on Dirichlet nodes."""
        F = np.zeros(self.shape, dtype=np.complex128)
        if f_hat is not None:
            F += self.W * np.asarray(f_hat).reshape(self.shape)
        if g_hat is not None:
            F += self.A * np.asarray(g_hat).reshape(self.shape)
        return F * self.act

    def forcing(self, F_hat, n: int) -> np.ndarray:
        """F^n = Re(F^ exp(-i omega t_n)), t_n = n dt (time convention of Eq. WE)."""
        if F_hat is None:
            return np.zeros(self.shape)
        return np.real(F_hat * np.exp(-1j * self.omega * n * self.dt))

    def K_active_sparse(self):
        """K restricted to active rows and columns, with the active index list."""
        ia = np.flatnonzero(self.act.ravel() > 0)
        return self.Kmat[ia][:, ia].tocsc(), ia
