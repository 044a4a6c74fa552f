"""Stochastic Galerkin system and Newmark-beta time stepping with a direct solve
(Sec. 2 Eqs. K_T, fparts, UmCm; Sec. 4 Eqs. galerproject, stok, K_T_Sto; Rayleigh
appendix C_0 = alpha0 M + alpha1 K_0, C_k = alpha1 K_k).

Unknown ordering: node-major, dof (a, k) -> a * P + k, so a block matrix with blocks
[X]_{jk} = sum_i G_ijk A_i is sum_i kron(A_i, G_i).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, pce

GAMMA = 0.5   # Newmark gamma (Sec. 2)
ZETA = 0.25   # Newmark beta, written zeta in the paper (Sec. 2)


def sg_block(G: np.ndarray, mats) -> sp.csr_matrix:
    """sum_i kron(A_i, G_i): the Galerkin block matrix [.]_{jk} = sum_i G_ijk A_i."""
    out = None
    for i, A in enumerate(mats):
        term = sp.kron(A, sp.csr_matrix(G[i]), format="csr")
        out = term if out is None else out + term
    return out.tocsr()


class SGOperators:
    """Mass, damping, stiffness and transient operators of the SG system for given
    deterministic matrices M (mass, deterministic, Sec. 4) and K_i (PCE coefficients
    of the stiffness)."""

    def __init__(self, M, Ks, G, alpha0, alpha1, dt):
        P = G.shape[1]
        self.P = P
        self.G = G
        I = sp.identity(P, format="csr")
        # [M]_{jk} = <Psi_j Psi_k> delta_jk M = delta_jk M  (orthonormal basis)
        self.Mb = sp.kron(M, I, format="csr")
        # [K]_{jk} = sum_i G_ijk K_i  (Eq. stok)
        self.Kb = sg_block(G, Ks)
        # damping PCE: C_0 = alpha0 M + alpha1 K_0, C_k = alpha1 K_k, then [C]_{jk} = sum_i G_ijk C_i
        Cs = [alpha1 * K for K in Ks]
        Cs[0] = Cs[0] + alpha0 * M
        self.Cb = sg_block(G, Cs)
        self.dt = dt
        # transient stiffness (Eq. K_T_Sto)
        self.Kt = (self.Mb / (ZETA * dt * dt) + self.Cb * (GAMMA / (ZETA * dt)) + self.Kb).tocsr()

    def effective_load(self, F, U, V, A):
        """f~ = f_{n+1} + M u~_m + C u~_c with u~_m, u~_c of Eqs. UmCm."""
        dt = self.dt
        um = (U + dt * V) / (ZETA * dt * dt) + (1.0 - 2.0 * ZETA) * A / (2.0 * ZETA)
        uc = GAMMA * dt * um - V - (1.0 - GAMMA) * A * dt
        return F + self.Mb @ um + self.Cb @ uc, um

    def update(self, Unew, U, V, A, um):
        """a_{n+1} and v_{n+1} from the Newmark relations (Sec. 2)."""
        dt = self.dt
        Anew = Unew / (ZETA * dt * dt) - um
        Vnew = V + dt * ((1.0 - GAMMA) * A + GAMMA * Anew)
        return Vnew, Anew

    def initial_acceleration(self, F0, U0, V0):
        """Consistent a_0 from M a_0 = f_0 - C v_0 - K u_0 (reading: Alg. 1 lists a_0
        without a formula)."""
        rhs = F0 - self.Cb @ V0 - self.Kb @ U0
        return spla.spsolve(self.Mb.tocsc(), rhs)


def galerkin_apply(G: np.ndarray, mats, X: np.ndarray) -> np.ndarray:
    """sg_block(G, mats) @ x without forming the Kronecker products: with x node-major as X (n, P),
    kron(A_i, G_i) x is A_i X G_i^T = A_i X G_i (G_ijk is symmetric in j, k), summed over i.  For
    full-size checks, where the block matrix would not fit in memory."""
    Y = np.zeros_like(X)
    for i, A in enumerate(mats):
        Y += (A @ X) @ G[i]
    return Y


class SGMatrixForm:
    """The operators of SGOperators applied in matrix form (X of shape (n, P), node-major rows), for
    systems too large to assemble as Kronecker block matrices: mass I (x) M, damping with C_0 = alpha0 M +
    alpha1 K_0 and C_k = alpha1 K_k, stiffness sum_i K_i (x) G_i, the transient operator (Eq. K_T_Sto),
    the effective load (Eqs. fparts, UmCm)."""

    def __init__(self, M, Ks, G, alpha0, alpha1, dt):
        self.M, self.Ks, self.G = M, Ks, G
        self.alpha0, self.alpha1, self.dt = alpha0, alpha1, dt

    def stiffness(self, X):
        return galerkin_apply(self.G, self.Ks, X)

    def damping(self, X):
        return self.alpha0 * (self.M @ X) + self.alpha1 * self.stiffness(X)

    def transient(self, X):
        dt = self.dt
        return (self.M @ X) / (ZETA * dt * dt) + self.damping(X) * (GAMMA / (ZETA * dt)) + self.stiffness(X)

    def effective_load(self, F, U, V, A):
        dt = self.dt
        um = (U + dt * V) / (ZETA * dt * dt) + (1.0 - 2.0 * ZETA) * A / (2.0 * ZETA)
        uc = GAMMA * dt * um - V - (1.0 - GAMMA) * A * dt
        return F + self.M @ um + self.damping(uc), um

    def residual(self, F, U, V, A, Unew):
        """||f~_{n+1} - K~ U_{n+1}|| / ||f~_{n+1}||: how well U_{n+1} solves the step's transient system."""
        Ft, _ = self.effective_load(F, U, V, A)
        return np.linalg.norm(Ft - self.transient(Unew)) / np.linalg.norm(Ft)


class SGProblem:
    """Global SG system for a workload on the structured grid (free nodes only).  coef: the PCE
    coefficients of c_s at the element centroids (P_in x 2 N^2) from a KL other than the analytic
    one, or None for fem.element_coefficients(prob)."""

    def __init__(self, prob, coef=None):
        self.prob = prob
        N = prob.N
        self.coef = fem.element_coefficients(prob) if coef is None else coef
        Mfull, Kfull = fem.assemble(N, self.coef)
        self.free = fem.free_nodes(N)
        f = self.free
        self.M = Mfull[f][:, f].tocsr()
        self.Ks = [K[f][:, f].tocsr() for K in Kfull]
        self.G = pce.triple_products(prob.M, prob.p_in, prob.p)
        self.P = self.G.shape[1]
        self.ops = SGOperators(self.M, self.Ks, self.G, prob.alpha0, prob.alpha1, prob.dt)

    def load(self, t: float) -> np.ndarray:
        """[F]_k = <f Psi_k> = f delta_k0 for the deterministic source (Sec. 4)."""
        F = np.zeros((self.free.size, self.P))
        F[:, 0] = fem.point_load(self.prob.N, self.prob.source, t)[self.free]
        return F.ravel()

    def initial_state(self):
        n = self.free.size
        U0 = np.zeros((n, self.P))
        U0[:, 0] = fem.initial_displacement(self.prob.N, self.prob.source)[self.free]
        U0 = U0.ravel()
        V0 = np.zeros_like(U0)
        A0 = self.ops.initial_acceleration(self.load(0.0), U0, V0)
        return U0, V0, A0


def run_direct(sgp: SGProblem, steps: int, callback=None):
    """Newmark time loop with a sparse direct solve of K~ U_{n+1} = f~_{n+1} each step."""
    ops = sgp.ops
    lu = spla.splu(ops.Kt.tocsc())
    U, V, A = sgp.initial_state()
    for n in range(steps):
        t = (n + 1) * sgp.prob.dt
        Ft, um = ops.effective_load(sgp.load(t), U, V, A)
        Unew = lu.solve(Ft)
        V, A = ops.update(Unew, U, V, A, um)
        U = Unew
        if callback is not None:
            callback(n, U, V, A)
    return U, V, A
