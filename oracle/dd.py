"""Non-overlapping domain decomposition of the SG system: interface Schur complement,
probabilistic two-level Neumann-Neumann preconditioner and PCG (Sec. 3 and Sec. 5).

Node classes (Sec. 3): interior nodes belong to one subdomain; interface nodes lie on
internal grid lines x = k H or y = k H; corners are the interface nodes shared by more
than two subdomains (the interior cross points; the end nodes of interface edges lie on
the Dirichlet boundary and are eliminated, a reading of Sec. 3); remaining nodes are the
other interface nodes.  Restrictions R_s, R_s^r, R_s^c, B_c^s act node-wise and are block
diagonal over the PCE modes (Eq. sto_restrict).  D_s is the counting partition of unity
(1 / number of subdomains sharing the node), which satisfies Eq. det_scaling.

Two forms of every operator are provided:
  * explicit dense matrices written literally from Eqs. Sto_Schur, Schur_alphabeta,
    Fcc_2 and NNCP2 (tiny problems only), and
  * the solve-based application (local Dirichlet / Neumann solves), which the tests
    check against the explicit form and which the time loop uses.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, pce
from .sg import SGOperators, GAMMA, ZETA


class Partition:
    """Node classes and restriction maps of an s x s partition of the N x N grid."""

    def __init__(self, N: int, s: int):
        assert N % s == 0
        self.N, self.s, self.H = N, s, N // s
        H = self.H
        self.free = fem.free_nodes(N)                       # global node ids, free order
        self.free_index = {g: k for k, g in enumerate(self.free)}
        iface, corner = [], []
        for g in self.free:
            i, j = g % (N + 1), g // (N + 1)
            on_x, on_y = i % H == 0, j % H == 0
            if on_x or on_y:
                iface.append(g)
            if on_x and on_y:
                corner.append(g)
        self.iface = np.array(iface, dtype=np.int64)        # global interface nodes
        self.iface_index = {g: k for k, g in enumerate(self.iface)}
        self.corner = np.array(corner, dtype=np.int64)
        self.corner_index = {g: k for k, g in enumerate(self.corner)}
        self.mult = np.zeros(self.iface.size)
        self.subs = []
        for sy in range(s):
            for sx in range(s):
                sub = {}
                nodes = [fem.node_id(sx * H + a, sy * H + b, N) for b in range(H + 1) for a in range(H + 1)]
                loc = [g for g in nodes if g in self.free_index]  # local free nodes
                sub["nodes"] = np.array(loc, dtype=np.int64)
                cls = []
                for g in loc:
                    if g in self.corner_index:
                        cls.append("c")
                    elif g in self.iface_index:
                        cls.append("r")
                    else:
                        cls.append("i")
                sub["cls"] = np.array(cls)
                gam = [g for g in loc if g in self.iface_index]
                sub["gamma"] = np.array(gam, dtype=np.int64)     # local interface, global ids
                for g in gam:
                    self.mult[self.iface_index[g]] += 1
                ce = np.zeros(2 * N * N, dtype=bool)
                for b in range(H):
                    for a in range(H):
                        e = 2 * ((sy * H + b) * N + (sx * H + a))
                        ce[e] = ce[e + 1] = True
                sub["elem_mask"] = ce
                self.subs.append(sub)

    def assemble(self, coef, elem_mask=None):
        return fem.assemble(self.N, coef, elem_mask)

    def element_coefficients(self, prob):
        return fem.element_coefficients(prob)


def dofs(node_pos: np.ndarray, P: int) -> np.ndarray:
    """Node positions -> node-major SG dof indices."""
    return (node_pos[:, None] * P + np.arange(P)[None, :]).ravel()


class DDSolver:
    """SG-DD solver for one workload.  Local matrices are assembled from the elements
    of each subdomain only (Eq. ki), so that sum_s R_s^T K_GG^s R_s gives the global
    interface block (Eq. GAssembly_Sto)."""

    def __init__(self, prob, explicit: bool = False, subs=None, coef=None, precond: str = "nn2", partition=None):
        """subs: indices of the only subdomains whose local operators are built (timing samples of
        large workloads); the coarse problem, which needs every subdomain, is then not assembled.
        coef: element PCE coefficients from a KL other than the analytic one (see sg.SGProblem).
        precond: the PCG preconditioner, "nn2" (two-level Neumann-Neumann, Eq. NNCP2), "nn1"
        (one-level Neumann-Neumann) or "lumped" (the one-level comparison of Sec. 6.1).
        partition: node classes of another mesh and partition (umesh.UPartition); None for the
        s x s partition of the structured grid."""
        assert precond in ("nn2", "nn1", "lumped")
        self.pc_kind = precond
        self.prob = prob
        N, s = prob.N, prob.s
        self.part = Partition(N, s) if partition is None else partition
        self.G = pce.triple_products(prob.M, prob.p_in, prob.p)
        P = self.P = self.G.shape[1]
        self.coef = self.part.element_coefficients(prob) if coef is None else coef
        part = self.part
        nG = part.iface.size
        self.nG = nG
        self.nC = part.corner.size
        self.loc = []
        self.sampled = subs is not None
        for si, sub in enumerate(part.subs):
            if subs is not None and si not in subs:
                continue
            Mfull, Kfull = self.part.assemble(self.coef, sub["elem_mask"])
            nd = sub["nodes"]
            M = Mfull[nd][:, nd].tocsr()
            Ks = [K[nd][:, nd].tocsr() for K in Kfull]
            ops = SGOperators(M, Ks, self.G, prob.alpha0, prob.alpha1, prob.dt)
            cls = sub["cls"]
            L = {"ops": ops}
            pos = np.arange(nd.size)
            L["I"] = dofs(pos[cls == "i"], P)
            L["r"] = dofs(pos[cls == "r"], P)
            L["c"] = dofs(pos[cls == "c"], P)
            L["ir"] = dofs(pos[(cls == "i") | (cls == "r")], P)
            gpos = pos[(cls == "r") | (cls == "c")]                 # local interface nodes (local order)
            L["Gam"] = dofs(gpos, P)
            L["free_glob"] = dofs(np.array([part.free_index[g] for g in nd]), P)
            L["R"] = dofs(np.array([part.iface_index[g] for g in nd[gpos]]), P)   # -> global interface dofs
            L["D"] = np.repeat(1.0 / part.mult[[part.iface_index[g] for g in nd[gpos]]], P)
            cnodes = nd[pos[cls == "c"]]
            L["B"] = dofs(np.array([part.corner_index[g] for g in cnodes], dtype=np.int64), P)
            # positions of r / c dofs inside the local interface vector
            gcls = cls[gpos]
            L["Gr"] = dofs(np.nonzero(gcls == "r")[0], P)
            L["Gc"] = dofs(np.nonzero(gcls == "c")[0], P)
            Kt = ops.Kt.tocsc()
            L["Kt"] = ops.Kt
            L["lu_I"] = spla.splu(Kt[L["I"]][:, L["I"]].tocsc(), permc_spec="MMD_AT_PLUS_A") if L["I"].size else None
            L["lu_N"] = spla.splu(Kt[L["ir"]][:, L["ir"]].tocsc(), permc_spec="MMD_AT_PLUS_A")
            # r-dofs inside the ir ordering
            irpos = pos[(cls == "i") | (cls == "r")]
            L["ir_r"] = dofs(np.nonzero(cls[irpos] == "r")[0], P)
            L["ir_i"] = dofs(np.nonzero(cls[irpos] == "i")[0], P)
            self.loc.append(L)
        if subs is not None:
            return
        self._build_coarse()
        if explicit:
            self._build_explicit()

    # ---------------- local solves ----------------
    @staticmethod
    def _blk(L, rows, cols):
        return L["Kt"][L[rows]][:, L[cols]]

    def solve_I(self, L, b):
        return L["lu_I"].solve(b) if L["lu_I"] is not None else b[:0]

    def schur_local(self, L, x):
        """S_s x = K_GG x - K_GI K_II^{-1} K_IG x (Eq. Sto_Schur), x on the local interface."""
        Kt = L["Kt"]
        y = Kt[L["Gam"]][:, L["Gam"]] @ x
        if L["I"].size:
            w = self.solve_I(L, Kt[L["I"]][:, L["Gam"]] @ x)
            y = y - Kt[L["Gam"]][:, L["I"]] @ w
        return y

    def schur(self, p):
        """S p = sum_s R_s^T S_s R_s p."""
        q = np.zeros_like(p)
        for L in self.loc:
            np.add.at(q, L["R"], self.schur_local(L, p[L["R"]]))
        return q

    def neumann(self, L, w_r):
        """Local Neumann problem with corners clamped (Eq. N-NNC2 with the interior row
        driven by 0): returns (y on interior, t on remaining), t = S_rr^{-1} w_r."""
        rhs = np.zeros(L["ir"].size)
        rhs[L["ir_r"]] = w_r
        v = L["lu_N"].solve(rhs)
        return v[L["ir_i"]], v[L["ir_r"]]

    # ---------------- coarse problem ----------------
    def _build_coarse(self):
        """F_cc = sum_s B_c^T (S_cc - S_cr S_rr^{-1} S_rc) B_c (Eq. Fcc_2), assembled column
        by column from Neumann solves: for a local corner dof e, v = -N^{-1} K_[ir],c e
        gives t = -S_rr^{-1} S_rc e (stored as Phi_s) and (K~ (v + e))_c = F^s e."""
        P = self.P
        nCd = self.nC * P
        F = np.zeros((nCd, nCd))
        for L in self.loc:
            nc = L["c"].size
            Kt = L["Kt"]
            Kir_c = Kt[L["ir"]][:, L["c"]].toarray()
            Kc_ir = Kt[L["c"]][:, L["ir"]]
            Kcc = Kt[L["c"]][:, L["c"]].toarray()
            Phi = np.zeros((L["r"].size, nc))
            Fs = np.zeros((nc, nc))
            for col in range(nc):
                v = -L["lu_N"].solve(Kir_c[:, col])
                Phi[:, col] = v[L["ir_r"]]
                Fs[:, col] = Kcc[:, col] + Kc_ir @ v
            L["Phi"] = Phi
            L["Fs"] = Fs
            if nc:
                F[np.ix_(L["B"], L["B"])] += Fs
        self.Fcc = F
        self.Fcc_chol = sla.cho_factor(F) if nCd else None

    def coarse_solve(self, d):
        return sla.cho_solve(self.Fcc_chol, d) if d.size else d

    # ---------------- preconditioner (solve-based) ----------------
    def precond(self, r):
        """z = M_NNC^{-1} r (Eq. NNCP2):
          w_s = D_s R_s r;  t_s = S_rr^{-1} R_s^r w_s  (local Neumann solve)
          d   = R_0 r = sum_s B^T (R_s^c w_s - S_cr t_s),  S_cr t = (K~ [y; t; 0])_c
          u_c = F_cc^{-1} d
          z   = sum_s R_s^T D_s (R_r^T (t_s + Phi_s B u_c) + R_c^T B u_c),  Phi_s = -S_rr^{-1} S_rc."""
        P = self.P
        d = np.zeros(self.nC * P)
        tl = []
        for L in self.loc:
            w = L["D"] * r[L["R"]]
            y, t = self.neumann(L, w[L["Gr"]])
            tl.append(t)
            if L["c"].size:
                Kt = L["Kt"]
                Scr_t = Kt[L["c"]][:, L["ir"]] @ self._ir_vec(L, y, t)
                np.add.at(d, L["B"], w[L["Gc"]] - Scr_t)
        uc = self.coarse_solve(d)
        z = np.zeros_like(r)
        for L, t in zip(self.loc, tl):
            zl = np.zeros(L["Gam"].size)
            ucs = uc[L["B"]] if L["c"].size else np.zeros(0)
            zl[L["Gr"]] = t + (L["Phi"] @ ucs if L["c"].size else 0.0)
            zl[L["Gc"]] = ucs
            np.add.at(z, L["R"], L["D"] * zl)
        return z

    # ---------------- one-level preconditioners of the comparison (Sec. 6.1) ----------------
    # The paper cites the one-level forms without restating them; these are the textbook ones:
    #   lumped: M^{-1} = sum_s R_s^T D_s K~_GG^s D_s R_s
    #   one-level Neumann-Neumann: M^{-1} = sum_s R_s^T D_s S_s^{-1} D_s R_s, with S_s the local Schur
    #   complement on the whole local interface (remaining nodes and corners); S_s^{-1} w is the
    #   interface part of the local Neumann solve K~^s [y; t] = [0; w] (nonsingular: the transient
    #   operator carries the mass term, so no subdomain floats).
    def precond_lumped(self, r):
        z = np.zeros_like(r)
        for L in self.loc:
            w = L["D"] * r[L["R"]]
            np.add.at(z, L["R"], L["D"] * (L["Kt"][L["Gam"]][:, L["Gam"]] @ w))
        return z

    def precond_nn1(self, r):
        z = np.zeros_like(r)
        for L in self.loc:
            if "lu_F" not in L:
                L["lu_F"] = spla.splu(L["Kt"].tocsc(), permc_spec="MMD_AT_PLUS_A")
            rhs = np.zeros(L["Kt"].shape[0])
            rhs[L["Gam"]] = L["D"] * r[L["R"]]
            t = L["lu_F"].solve(rhs)[L["Gam"]]
            np.add.at(z, L["R"], L["D"] * t)
        return z

    def apply_pc(self, r):
        """The PCG preconditioner selected at construction."""
        if self.pc_kind == "lumped":
            return self.precond_lumped(r)
        if self.pc_kind == "nn1":
            return self.precond_nn1(r)
        return self.precond(r)

    @staticmethod
    def _ir_vec(L, y, t):
        v = np.zeros(L["ir"].size)
        v[L["ir_i"]] = y
        v[L["ir_r"]] = t
        return v

    # ---------------- explicit forms (tiny problems) ----------------
    def _build_explicit(self):
        """Dense S, F_cc, R_0 and M_NNC^{-1} written literally from the equations."""
        P, nG = self.P, self.nG
        nGd, nCd = nG * P, self.nC * P
        S = np.zeros((nGd, nGd))
        Minv_local = np.zeros((nGd, nGd))
        R0 = np.zeros((nCd, nGd))
        Fcc = np.zeros((nCd, nCd))
        Mlumped = np.zeros((nGd, nGd))
        Mnn1 = np.zeros((nGd, nGd))
        for L in self.loc:
            Kt = L["Kt"].toarray()
            I, Gm = L["I"], L["Gam"]
            KII = Kt[np.ix_(I, I)]
            Ss = Kt[np.ix_(Gm, Gm)] - Kt[np.ix_(Gm, I)] @ np.linalg.solve(KII, Kt[np.ix_(I, Gm)]) if I.size \
                else Kt[np.ix_(Gm, Gm)]
            Rs = np.zeros((Gm.size, nGd)); Rs[np.arange(Gm.size), L["R"]] = 1.0
            S += Rs.T @ Ss @ Rs
            # Eq. Schur_alphabeta: S_ab = A_ab - A_ai A_ii^{-1} A_ib over the local interface
            Srr = Ss[np.ix_(L["Gr"], L["Gr"])]
            Src = Ss[np.ix_(L["Gr"], L["Gc"])]
            Scr = Ss[np.ix_(L["Gc"], L["Gr"])]
            Scc = Ss[np.ix_(L["Gc"], L["Gc"])]
            Ds = np.diag(L["D"])
            Rr = np.zeros((L["Gr"].size, Gm.size)); Rr[np.arange(L["Gr"].size), L["Gr"]] = 1.0
            Rc = np.zeros((L["Gc"].size, Gm.size)); Rc[np.arange(L["Gc"].size), L["Gc"]] = 1.0
            Srr_inv = np.linalg.inv(Srr)
            Minv_local += Rs.T @ Ds @ (Rr.T @ Srr_inv @ Rr) @ Ds @ Rs
            Mlumped += Rs.T @ Ds @ Kt[np.ix_(Gm, Gm)] @ Ds @ Rs
            Mnn1 += Rs.T @ Ds @ np.linalg.inv(Ss) @ Ds @ Rs
            if L["Gc"].size:
                Bc = np.zeros((L["Gc"].size, nCd)); Bc[np.arange(L["Gc"].size), L["B"]] = 1.0
                Fcc += Bc.T @ (Scc - Scr @ Srr_inv @ Src) @ Bc
                R0 += Bc.T @ (Rc - Scr @ Srr_inv @ Rr) @ Ds @ Rs
        self.S_explicit = S
        self.Mlumped_explicit = Mlumped
        self.Mnn1_explicit = Mnn1
        self.Fcc_explicit = Fcc
        self.R0_explicit = R0
        Minv = Minv_local
        if nCd:
            Minv = Minv + R0.T @ np.linalg.solve(Fcc, R0)
        self.Minv_explicit = Minv

    # ---------------- time step ----------------
    def local_load(self, L, F_glob, um, uc):
        """f~^s = f^s + M^s u~_m + C^s u~_c on the local free nodes, with the external
        load split as f_I^s = f_I and f_G^s = D_s R_s f_G (Alg. 1, force assembly)."""
        ops = L["ops"]
        f = F_glob[L["free_glob"]].copy()
        f[L["Gam"]] *= L["D"]
        return f + ops.Mb @ um[L["free_glob"]] + ops.Cb @ uc[L["free_glob"]]

    def pcg(self, g, x0, tol, max_iter):
        """Preconditioned CG on S u_G = g with M_NNC^{-1}; stops when
        ||r||_2 / ||g||_2 <= tol (reading: RHS-relative residual).  Returns
        (x, iterations, final relative residual)."""
        gn = np.linalg.norm(g)
        if gn == 0.0:
            return np.zeros_like(g), 0, 0.0
        x = x0.copy()
        r = g - self.schur(x)
        rel = np.linalg.norm(r) / gn
        it = 0
        if rel <= tol:
            return x, 0, rel
        z = self.apply_pc(r)
        p = z.copy()
        rz = r @ z
        while it < max_iter:
            q = self.schur(p)
            alpha = rz / (p @ q)
            x = x + alpha * p
            r = r - alpha * q
            it += 1
            rel = np.linalg.norm(r) / gn
            if rel <= tol:
                break
            z = self.apply_pc(r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
        return x, it, rel

    def solve_step(self, F_glob, um, uc, x0, tol, max_iter):
        """One Newmark step's solve (Alg. 1 loop body, stochastic form of Sec. 5):
        condensed RHS, PCG on the interface, interior recovery.  Returns the global
        U_{n+1}, the interface solution, iterations and final relative residual."""
        P = self.P
        g = np.zeros(self.nG * P)
        floc = []
        for L in self.loc:
            f = self.local_load(L, F_glob, um, uc)
            floc.append(f)
            gs = f[L["Gam"]].copy()
            if L["I"].size:
                gs -= L["Kt"][L["Gam"]][:, L["I"]] @ self.solve_I(L, f[L["I"]])
            np.add.at(g, L["R"], gs)
        uG, it, rel = self.pcg(g, x0, tol, max_iter)
        U = np.zeros(self.part.free.size * P)
        for L, f in zip(self.loc, floc):
            xG = uG[L["R"]]
            U[L["free_glob"][L["Gam"]]] = xG
            if L["I"].size:
                uI = self.solve_I(L, f[L["I"]] - L["Kt"][L["I"]][:, L["Gam"]] @ xG)
                U[L["free_glob"][L["I"]]] = uI
        return U, uG, it, rel


def iface_restrict(dd: DDSolver, U: np.ndarray) -> np.ndarray:
    """Global SG vector -> global interface vector."""
    P = dd.P
    pos = np.array([dd.part.free_index[g] for g in dd.part.iface], dtype=np.int64)
    return U[dofs(pos, P)]


def run_dd(sgp, dd: DDSolver, steps: int, tol=None, max_iter=None, callback=None, state=None):
    """Newmark time loop of Alg. 1 with the SG-DD solve; the PCG initial guess is the
    previous step's interface solution (Alg. 1, update of the initial solution)."""
    prob = sgp.prob
    tol = prob.tol if tol is None else tol
    max_iter = prob.max_iter if max_iter is None else max_iter
    ops = sgp.ops
    if state is None:
        U, V, A = sgp.initial_state()
        n0 = 0
    else:
        U, V, A, n0 = state
    x0 = iface_restrict(dd, U)
    iters = []
    for n in range(n0, n0 + steps):
        t = (n + 1) * prob.dt
        dt = prob.dt
        um = (U + dt * V) / (ZETA * dt * dt) + (1.0 - 2.0 * ZETA) * A / (2.0 * ZETA)
        uc = GAMMA * dt * um - V - (1.0 - GAMMA) * A * dt
        Unew, uG, it, rel = dd.solve_step(sgp.load(t), um, uc, x0, tol, max_iter)
        iters.append((it, rel))
        V, A = ops.update(Unew, U, V, A, um)
        U = Unew
        x0 = uG
        if callback is not None:
            callback(n, U, V, A)
    return U, V, A, iters
