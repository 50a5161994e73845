"""Oracle for the first-order (mixed) formulation of Sec. 3 on a staggered grid (test
infrastructure only; see oracle/__init__.py).

Unknowns (Eq. mixWE, v = y_t and p = grad y):
  v      at the nodes x_j, held at 0 on Dirichlet nodes (sound-soft, homogeneous g_D);
  p_a    on the grid links (j, j + e_a) of axis a, stored at the link's lower node j (the slot
         j_a = n_a holds no link and stays 0).
  W_e    lumped L2 mass of a link of axis a: h^d prod_{b != a} w(j_b) (w = 1/2 at axis ends);
  G      (G v)_a = (v_{j+e_a} - v_j) / h on every link, with v = 0 on Dirichlet nodes.

With these, G^T W_e G is the stiffness K of oracle/grid.py, and the semi-discrete Eq. mixWE
tested against the nodal basis reads
      M v' + B v = -G^T W_e p + F,        p' = G v,
with M, B and F of oracle/grid.py (the boundary term of Eq. mixWE_ABC gives B, g_S enters F).

Time stepping: staggered leapfrog, p at half steps, one step (p^{n-1/2}, v^n) -> (p^{n+1/2}, v^{n+1}):
      p^{n+1/2} = p^{n-1/2} + dt G v^n
      (M + dt/2 B) v^{n+1} = (M - dt/2 B) v^n - dt G^T W_e p^{n+1/2} + dt F^{n+1/2},
with F^{n+1/2} = Re(F^ exp(-i omega (n + 1/2) dt)).  The state is s = (p^{-1/2}, v^0) and the
period map Pi(s) = s^N.

Functional (Eq. mix_cost_functional_J): J^(s) = 1/2 ||Pi(s) - s||_E^2 with the diagonal energy
inner product (a, b)_E = sum_a a.p_a W_e b.p_a + a.v M b.v.  Its gradient (Eq.
mixJ_deriative_2: the backward first-order wave equation from the mismatch) is taken as the
literal transpose of the discrete period; since E is diagonal, the E-representer of J^' is
E^-1 (P - I)^T E (Pi(s) - s) and no elliptic (Riesz) solve is needed.

Fixed point.  Substituting v^n = Re(V e^{-i omega t_n}), p^{n+1/2} = Re(P e^{-i omega t_{n+1/2}})
gives P = (i / wt) G V and, with V = -i wt U,
      (K - wt^2 M - i wh B) U = F^,     wt = (2/dt) sin(omega dt/2),  wh = sin(omega dt)/dt,
the same time-discrete Helmholtz system as the second-order scheme (oracle/direct.py).
Recovery (Eq. mix_solution, discrete): Im U = v^0 / wt, G Re U = Re P with
Re P = (p^{-1/2} + p^{1/2}) / (2 cos(omega dt/2)), and the real part of the Helmholtz system
      Re U = (G^T W_e Re P + wh B Im U - Re F^) / (wt^2 M).
Filter (Eq. TH_FILTERED_MIXED_SOLUTION, rectangle rule, discrete-exact for N >= 3):
      U = (2 i / (N wt)) sum_{n=0}^{N-1} v^n exp(i omega t_n).

Parity: pinned by G^T W_e G = K, by the staggered scheme's conserved energy on closed domains,
by the dot-product test of the transpose, and by the fixed point = the direct solve of the
second-order discrete system (oracle/direct.py) through both recoveries.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .grid import Discretization


class Staggered:
    """Edge weights and difference operators of the staggered grid on top of a Discretization."""

    def __init__(self, dz: Discretization):
        self.dz = dz
        d = dz.dim
        self.edge = []   # 1 where a link of axis a starts at the node
        self.We = []     # lumped link mass, 0 where there is no link
        for a in range(d):
            ax = d - 1 - a
            ex = np.zeros(dz.shape)
            sl = [slice(None)] * d
            sl[ax] = slice(0, dz.n[a])
            ex[tuple(sl)] = 1.0
            w = np.full(dz.shape, dz.h ** d)
            for b in range(d):
                if b != a:
                    w = w * dz.axis_w[b]
            self.edge.append(ex)
            self.We.append(w * ex)

    def G(self, v):
        """Link differences (v_{j+e_a} - v_j)/h of the active field, per axis."""
        dz = self.dz
        d = dz.dim
        va = v * dz.act
        out = []
        for a in range(d):
            ax = d - 1 - a
            g = np.zeros(dz.shape)
            lo = [slice(None)] * d
            hi = [slice(None)] * d
            lo[ax] = slice(0, dz.n[a])
            hi[ax] = slice(1, dz.n[a] + 1)
            g[tuple(lo)] = (va[tuple(hi)] - va[tuple(lo)]) / dz.h
            out.append(g)
        return out

    def GT(self, q):
        """Transpose of G: (G^T q)_j = sum_a (q_a[j - e_a] - q_a[j]) / h, zero on Dirichlet nodes."""
        dz = self.dz
        d = dz.dim
        out = np.zeros(dz.shape)
        for a in range(d):
            ax = d - 1 - a
            qa = q[a] * self.edge[a]
            lo = [slice(None)] * d
            hi = [slice(None)] * d
            lo[ax] = slice(0, dz.n[a])
            hi[ax] = slice(1, dz.n[a] + 1)
            out[tuple(hi)] += qa[tuple(lo)] / dz.h
            out -= qa / dz.h
        return out * dz.act

    def forcing_half(self, F_hat, n: int):
        """F^{n+1/2} = Re(F^ exp(-i omega (n + 1/2) dt))."""
        dz = self.dz
        if F_hat is None:
            return np.zeros(dz.shape)
        return np.real(F_hat * np.exp(-1j * dz.omega * (n + 0.5) * dz.dt))

    # -------------------------------------------------------------------------------------
    def step(self, p, v, n: int, F_hat=None):
        """One staggered leapfrog step (p^{n-1/2}, v^n) -> (p^{n+1/2}, v^{n+1})."""
        dz = self.dz
        dt = dz.dt
        gv = self.G(v)
        p_new = [(p[a] + dt * gv[a]) * self.edge[a] for a in range(dz.dim)]
        rhs = (dz.M - 0.5 * dt * dz.B) * v - dt * self.GT([self.We[a] * p_new[a] for a in range(dz.dim)])
        rhs = rhs + dt * self.forcing_half(F_hat, n)
        v_new = rhs / (dz.M + 0.5 * dt * dz.B) * dz.act
        return p_new, v_new

    def period(self, p0, v0, F_hat=None):
        p = [np.asarray(x, dtype=np.float64).reshape(self.dz.shape) * self.edge[a] for a, x in enumerate(p0)]
        v = np.asarray(v0, dtype=np.float64).reshape(self.dz.shape) * self.dz.act
        for n in range(self.dz.N):
            p, v = self.step(p, v, n, F_hat)
        return p, v

    def transposed_step(self, pb, vb):
        """Transpose of the homogeneous step: cotangents of (p^{n+1/2}, v^{n+1}) -> of (p^{n-1/2}, v^n).
        The v-update is transposed first (it ran last), then the p-update."""
        dz = self.dz
        dt = dz.dt
        u = vb * dz.act / (dz.M + 0.5 * dt * dz.B)
        gu = self.G(u)
        p_mid = [(pb[a] - dt * self.We[a] * gu[a]) * self.edge[a] for a in range(dz.dim)]
        v_out = ((dz.M - 0.5 * dt * dz.B) * u + dt * self.GT(p_mid)) * dz.act
        return p_mid, v_out

    def transposed_period(self, pb, vb):
        p = [np.asarray(x, dtype=np.float64).reshape(self.dz.shape) * self.edge[a] for a, x in enumerate(pb)]
        v = np.asarray(vb, dtype=np.float64).reshape(self.dz.shape) * self.dz.act
        for _ in range(self.dz.N):
            p, v = self.transposed_step(p, v)
        return p, v

    # -------------------------------------------------------------------------------------
    def e_inner(self, a, b) -> float:
        """(a, b)_E for states a = (p, v), b = (p, v)."""
        s = float(np.sum(self.dz.M * a[1] * b[1]))
        for k in range(self.dz.dim):
            s += float(np.sum(self.We[k] * a[0][k] * b[0][k]))
        return s

    def E(self, s):
        return [self.We[a] * s[0][a] for a in range(self.dz.dim)], self.dz.M * s[1] * self.dz.act

    def E_inv(self, s):
        p = [np.where(self.We[a] > 0, s[0][a] / np.where(self.We[a] > 0, self.We[a], 1.0), 0.0)
             for a in range(self.dz.dim)]
        return p, s[1] / self.dz.M * self.dz.act

    def functional(self, s, F_hat=None) -> float:
        """J^(s) = 1/2 ||Pi(s) - s||_E^2 (Eq. mix_cost_functional_J)."""
        e = self.mismatch(s, F_hat)
        return 0.5 * self.e_inner(e, e)

    def mismatch(self, s, F_hat=None):
        pT, vT = self.period(s[0], s[1], F_hat)
        return [pT[a] - s[0][a] * self.edge[a] for a in range(self.dz.dim)], vT - s[1] * self.dz.act

    def gradient(self, s, F_hat=None):
        """E-representer of J^'(s): E^-1 (P - I)^T E e, e = Pi(s) - s; returns (gradient, e)."""
        e = self.mismatch(s, F_hat)
        z = self.E(e)
        q = self.transposed_period(z[0], z[1])
        g = self.E_inv(([q[0][a] - z[0][a] for a in range(self.dz.dim)], q[1] - z[1]))
        return g, e

    # -------------------------------------------------------------------------------------
    def recover(self, s, F_hat):
        """Eq. mix_solution in its discrete-exact form (see the module header)."""
        dz = self.dz
        p, v = s
        im = v * dz.act / dz.omega_tilde
        gv = self.G(v)
        c2 = math.cos(0.5 * dz.omega * dz.dt)
        re_p = [(2.0 * p[a] + dz.dt * gv[a]) * self.edge[a] / (2.0 * c2) for a in range(dz.dim)]
        re_F = np.zeros(dz.shape) if F_hat is None else np.real(F_hat)
        re = (self.GT([self.We[a] * re_p[a] for a in range(dz.dim)]) + dz.omega_hat * dz.B * im - re_F)
        re = re / (dz.omega_tilde ** 2 * dz.M) * dz.act
        return re + 1j * im

    def filtered(self, s, F_hat):
        """Eq. TH_FILTERED_MIXED_SOLUTION: one forced period, U = (2i/(N wt)) sum v^n e^{i omega t_n}."""
        dz = self.dz
        p = [x.copy() for x in s[0]]
        v = s[1].copy()
        acc = np.zeros(dz.shape, dtype=np.complex128)
        for n in range(dz.N):
            acc += v * np.exp(1j * dz.omega * n * dz.dt)
            p, v = self.step(p, v, n, F_hat)
        return 2j / (dz.N * dz.omega_tilde) * acc * dz.act


@dataclasses.dataclass
class FirstOrderResult:
    u: np.ndarray          # recovery by Eq. mix_solution
    u_filtered: np.ndarray  # recovery by Eq. TH_FILTERED_MIXED_SOLUTION
    p0: list
    v0: np.ndarray
    iterations: int
    rel_residual: float
    J_history: list


def solve(dz: Discretization, F_hat, tol=1e-12, max_iter=10000, s_init=None) -> FirstOrderResult:
    """The CMCG Algorithm of Sec. 2.3 on the first-order state (Sec. 3): steps 2 and 5.1 use J^'
    and step 3 (the Riesz map) is the identity, the gradient being formed as an E-representer."""
    st = Staggered(dz)
    d = dz.dim
    # (1)
    if s_init is None:
        s = ([np.zeros(dz.shape) for _ in range(d)], np.zeros(dz.shape))
    else:
        s = ([np.asarray(x, dtype=np.float64).reshape(dz.shape) * st.edge[a] for a, x in enumerate(s_init[0])],
             np.asarray(s_init[1], dtype=np.float64).reshape(dz.shape) * dz.act)
    # (2)-(4)
    g, e = st.gradient(s, F_hat)
    J_hist = [0.5 * st.e_inner(e, e)]
    r = g
    dd = ([x.copy() for x in g[0]], g[1].copy())
    rr = st.e_inner(r, r)
    rr0 = rr
    rel = 1.0 if rr0 > 0 else 0.0
    it = 0
    if rr0 <= 0.0:
        max_iter = 0
    # (5)
    for it in range(1, max_iter + 1):
        gd, ed = st.gradient(dd, None)                                   # 5.1 (and 5.2: E-representer)
        alpha = rr / st.e_inner(gd, dd)                                  # 5.3
        s = ([s[0][a] - alpha * dd[0][a] for a in range(d)], s[1] - alpha * dd[1])          # 5.4
        e = ([e[0][a] - alpha * ed[0][a] for a in range(d)], e[1] - alpha * ed[1])
        J_hist.append(0.5 * st.e_inner(e, e))
        r = ([r[0][a] - alpha * gd[0][a] for a in range(d)], r[1] - alpha * gd[1])          # 5.5
        rr_new = st.e_inner(r, r)
        beta = rr_new / rr                                               # 5.6
        dd = ([r[0][a] + beta * dd[0][a] for a in range(d)], r[1] + beta * dd[1])           # 5.7
        rr = rr_new
        rel = math.sqrt(rr / rr0)
        if rel <= tol:                                                   # 5.8
            break
    # (6)
    return FirstOrderResult(u=st.recover(s, F_hat), u_filtered=st.filtered(s, F_hat), p0=s[0], v0=s[1],
                            iterations=it, rel_residual=rel, J_history=J_hist)
