"""FP64 CPU oracle of EMU with affine bones and joints (Sec. 3.3 of arXiv 2006.08821).

TEST INFRASTRUCTURE ONLY, like ``emu_oracle``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it, and it shares no code with the CUDA path.

Sec. 3.3 gives the constrained coupling problem (bone rows B_q q = B_F F,
joint rows J q = 0), its KKT system with the slacks eps1 (joints) and eps2
(bones), and the slack schedule; it gives no discretisation of either row
set. The reading taken here:

* Every tet of bone b uses the bone's single deformation gradient F_b, so
  the bone's elastic energy is sum_{i in b} V_i Psi(F_b). A bone whose
  vertices are all pinned keeps F_b = I and is not a variable. The Newton
  variables are the F_i of the other tets and the F_b of the free bones.
* Bone rows: G_i q = F_b for every tet i of bone b. With a slack eps2 < 0
  the KKT system is the stationarity condition of the coupling energy with
  a penalty (1 / |eps2|) |G_i q - F_b|^2 on those rows. The paper's system
  is unweighted (G^T G); the one here carries the ACAP weights w_i = V_i
  (Eq. 3 with the volume measure), so the penalty weight is Vbar / |eps2|
  with Vbar the mean rest volume. A bone tet's ACAP weight thus becomes
  w_i + Vbar / |eps2|. The same weights enter E_C, so E_C(F) is the minimum
  the coupling solve attains and dE/dF keeps the form of Eq. 7.
* Joint rows: at each joint point p, the least-squares affine fits of the
  two bones' vertex positions, evaluated at p, coincide. The fit is linear
  in q and exact when a bone's vertices move affinely. A hinge has the two
  points p0 +- half_length * axis, a ball joint one point.
* Slack schedule: during Newton eps1 = 0 (joints hard, by a KKT solve) and
  eps2 = -1e-3; after convergence the coupling solve is repeated once with
  eps2 = 0 (every bone's vertices follow q_v = F_b Q_v + t_b exactly) and
  eps1 = -1e-4. Joint rows measure a length while bone rows measure a
  gradient, so eps1 is taken relative to l^2, l = Vbar^(1/3): the joint
  penalty per point and coordinate is Vbar / (|eps1| l^2).
* The Newton direction is Eq. 12's Woodbury step in the reduced variables:
  a bone's 9x9 block is the sum of its tets' blocks and its rows of B the
  sum of its tets' rows. The low-rank basis is a Galerkin basis of the
  constrained coupling problem: Eq. 9's lowest eigenvectors of the weighted
  ACAP matrix K, projected onto the null space of the joint rows, plus the
  exact (constrained) responses of q to each entry of each free bone's F_b,
  orthonormalised; Lambda becomes Phi^T K Phi. With the bone tets weighted
  1000x, the lowest modes alone miss how q follows F_b, the bone's block of
  the approximate Hessian is then far too stiff along a hinge rotation, and
  the iteration stalls (measured); with the responses in the basis that
  block is exact. A Galerkin basis keeps Phi (Phi^T K Phi)^-1 Phi^T below
  the constrained inverse of K, so the approximate Hessian stays positive
  definite, and the gradient stays exact.
"""
from __future__ import annotations

import time

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .emu_oracle import EmuOracle, OracleParams, OracleResult, delta_psi, d2psi, dpsi, psd_project, psi


def affine_fit_weights(Q, p):
    """c with sum_v c_v x_v = A p + t for the least-squares affine fit
    x_v ~ A Q_v + t of the points Q (k, 3); exact for affine x."""
    Qt = np.hstack([Q, np.ones((Q.shape[0], 1))])
    return Qt @ np.linalg.solve(Qt.T @ Qt, np.append(p, 1.0))


class BoneOracle:
    """Setup for one assembly; ``solve`` runs Algorithm 1 on the reduced
    variables, then the final coupling solve of Sec. 3.3."""

    def __init__(self, mesh, params: OracleParams | None = None, eps_bone=-1e-3, eps_joint_final=-1e-4,
                 modes: str = "eigsh"):
        if not (eps_bone < 0.0 and eps_joint_final < 0.0):
            raise ValueError("the Newton bone slack and the final joint slack must be negative")
        if getattr(mesh, "f_ext", None) is not None:
            raise ValueError("external forces (Sec. 3.4) are not combined with bones here")
        base = EmuOracle(mesh, params, modes="none", factor=False)
        self.base = base
        self.p = base.p
        self.mesh = mesh
        self.n, self.m = base.n, base.m
        bid = np.full(self.m, -1, dtype=np.int64) if mesh.bone_id is None else np.asarray(mesh.bone_id, np.int64)
        self.bid = bid
        self.nb = int(bid.max()) + 1 if bid.size and bid.max() >= 0 else 0
        is_fixed = np.zeros(self.n, dtype=bool)
        is_fixed[np.asarray(mesh.fixed_verts, dtype=np.int64)] = True
        self.is_fixed = is_fixed
        T = base.T
        self.bone_verts = [np.unique(T[bid == b]) for b in range(self.nb)]
        self.bone_fixed = np.zeros(self.nb, dtype=bool)
        for b, vs in enumerate(self.bone_verts):
            pinned = is_fixed[vs]
            if pinned.all():
                self.bone_fixed[b] = True
            elif pinned.any():
                raise ValueError(f"bone {b} is partly pinned")
        for b in range(self.nb):
            for c in range(b + 1, self.nb):
                if np.intersect1d(self.bone_verts[b], self.bone_verts[c]).size:
                    raise ValueError("bones must not share vertices")
        # reduced variables: one slot per deformable tet, one per free bone
        slot = np.full(self.m, -1, dtype=np.int64)
        dform = np.nonzero(bid < 0)[0]
        slot[dform] = np.arange(dform.size)
        self.bone_slot = np.full(self.nb, -1, dtype=np.int64)
        k = dform.size
        for b in range(self.nb):
            if not self.bone_fixed[b]:
                self.bone_slot[b] = k
                slot[bid == b] = k
                k += 1
        self.slot = slot
        self.nvar = k
        live = slot >= 0
        rows = (9 * np.nonzero(live)[0][:, None] + np.arange(9)).ravel()
        cols = (9 * slot[live][:, None] + np.arange(9)).ravel()
        self.Tmap = sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(9 * self.m, 9 * k))
        self.F_pinned = np.zeros((self.m, 3, 3))  # F of tets of pinned bones (I), 0 elsewhere
        self.F_pinned[~live] = np.eye(3)

        # weights: bone rows as a penalty Vbar / |eps2| on the bone tets
        self.Vbar = float(base.V.mean())
        self.w = base.w + np.where(bid >= 0, self.Vbar / abs(eps_bone), 0.0)
        self.w9 = np.repeat(self.w, 9)
        self.eps_joint_final = eps_joint_final

        # joint rows (vertex level): fit of bone b1 minus fit of bone b2 at each point
        pts = []
        for j in (mesh.joints or []):
            b1, b2 = j["bones"]
            p0 = np.asarray(j["point"], dtype=np.float64)
            if j["type"] == "hinge":
                ax = np.asarray(j["axis"], dtype=np.float64)
                ax = ax / np.linalg.norm(ax)
                pts += [(b1, b2, p0 + j["half_length"] * ax), (b1, b2, p0 - j["half_length"] * ax)]
            elif j["type"] == "ball":
                pts.append((b1, b2, p0))
            else:
                raise ValueError(f"unknown joint type {j['type']}")
        self.joint_points = pts
        jr, jc, jv = [], [], []
        for r, (b1, b2, pt) in enumerate(pts):
            for b, sgn in ((b1, 1.0), (b2, -1.0)):
                vs = self.bone_verts[b]
                cw = affine_fit_weights(base.Q[vs], pt)
                jr += [r] * vs.size
                jc += vs.tolist()
                jv += (sgn * cw).tolist()
        Jv = sp.csr_matrix((jv, (jr, jc)), shape=(len(pts), self.n))
        self.Jv = Jv
        self.J = sp.kron(Jv, sp.eye(3)).tocsr()  # DOF level, rows (point, coordinate)
        self.J_f = self.J[:, base.free_dofs].tocsr()
        self.J_c = self.J[:, base.fixed_dofs].tocsr()

        # Newton-phase coupling matrix (Eq. 4 with the bone penalty) and its KKT system
        G_f = base.G_f
        self.K = (G_f.T @ sp.diags(self.w9) @ G_f).tocsc()
        nj = self.J_f.shape[0]
        if nj:
            kkt = sp.bmat([[self.K, self.J_f.T], [self.J_f, None]], format="csc")
        else:
            kkt = self.K
        self._lu = spla.splu(kkt.tocsc())
        self.nj = nj
        self.j_rhs = -(self.J_c @ base.q_c)
        self.Gc_qc = base.G_c @ base.q_c

        # Eq. 9 basis of the weighted ACAP matrix, restricted to the joints'
        # null space, plus the bones' exact responses; Eq. 11's B in reduced variables
        nf = base.free_dofs.size
        kk = min(self.p.k_modes, nf)
        if modes == "eigsh" and kk < nf - 1 and nf > 600:
            lam_k, Phi = spla.eigsh(self.K, k=kk, sigma=0.0, which="LM")
        else:
            lam_all, vec_all = np.linalg.eigh(self.K.toarray())
            lam_k, Phi = lam_all[:kk], vec_all[:, :kk]
        Phi = Phi[:, np.argsort(lam_k)]
        if nj:
            JJt = (self.J_f @ self.J_f.T).toarray()
            Phi = Phi - self.J_f.T @ np.linalg.solve(JJt, self.J_f @ Phi)
        resp = []
        for bb in range(self.nb):
            if self.bone_fixed[bb]:
                continue
            on = (bid == bb).astype(np.float64)
            for e in range(9):
                d = np.zeros((self.m, 9))
                d[:, e] = on
                resp.append(self._kkt_solve(G_f.T @ (self.w9 * d.reshape(-1)), np.zeros(nj)))
        basis = np.hstack([Phi] + ([np.stack(resp, axis=1)] if resp else []))
        U, sv, _ = np.linalg.svd(basis, full_matrices=False)
        self.Phi = U[:, sv > 1e-10 * sv[0]]
        self.k = self.Phi.shape[1]
        self.Lhat = self.Phi.T @ (self.K @ self.Phi)
        self.Lhat = 0.5 * (self.Lhat + self.Lhat.T)
        self.B = (self.Tmap.T @ (sp.diags(self.w9) @ (G_f @ self.Phi))).T.copy()  # (k, 9 nvar)

    # --- reduced <-> per-tet ---------------------------------------------------
    def full_F(self, X):
        """Per-tet F (m,3,3) from the reduced variables X (nvar,3,3)."""
        return (self.Tmap @ X.reshape(-1)).reshape(self.m, 3, 3) + self.F_pinned

    def full_d(self, dX):
        return (self.Tmap @ dX.reshape(-1)).reshape(self.m, 3, 3)

    def reduce(self, per_tet):
        """Sum of per-tet 9-vectors into the reduced slots (nvar,3,3)."""
        return (self.Tmap.T @ per_tet.reshape(-1)).reshape(self.nvar, 3, 3)

    # --- coupling solves (Sec. 3.3 KKT, Newton phase) ----------------------
    def _kkt_solve(self, rhs_q, rhs_j):
        if self.nj:
            sol = self._lu.solve(np.concatenate([rhs_q, rhs_j]))
            return sol[:rhs_q.size]
        return self._lu.solve(rhs_q)

    def acap_solve(self, F):
        b = self.base
        rhs = b.G_f.T @ (self.w9 * (F.reshape(-1) - self.Gc_qc))
        q = np.empty(3 * self.n)
        q[b.free_dofs] = self._kkt_solve(rhs, self.j_rhs)
        q[b.fixed_dofs] = b.q_c
        return q

    def acap_solve_d(self, d):
        b = self.base
        rhs = b.G_f.T @ (self.w9 * d.reshape(-1))
        dq = np.zeros(3 * self.n)
        dq[b.free_dofs] = self._kkt_solve(rhs, np.zeros(self.nj))
        return dq

    def joint_residual(self, q):
        """x_b1(p) - x_b2(p) at every joint point, (points, 3)."""
        return (self.Jv @ q.reshape(self.n, 3))

    # --- energy and gradient in the reduced variables ------------------------
    def energy(self, X, q, a):
        b = self.base
        F = self.full_F(X)
        ka = b.kappa * a
        P = np.sum(b.V * psi(F, b.mu, b.lam, ka, b.u))
        D = b.deformation_gradients(q) - F
        return P + 0.5 * b.alpha * np.sum(self.w * np.einsum("ijk,ijk->i", D, D))

    def gradient(self, X, q, a):
        """dE/dX: per-tet V Psi'(F) + alpha w (F - G q), summed over each bone."""
        b = self.base
        F = self.full_F(X)
        ka = b.kappa * a
        g = b.V[:, None, None] * dpsi(F, b.mu, b.lam, ka, b.u) + \
            (b.alpha * self.w)[:, None, None] * (F - b.deformation_gradients(q))
        return self.reduce(g)

    def hessian_blocks(self, X, a):
        b = self.base
        F = self.full_F(X)
        ka = b.kappa * a
        Hel = b.V[:, None, None] * d2psi(F, b.mu, b.lam, ka, b.u)
        H = psd_project(Hel) + (b.alpha * self.w)[:, None, None] * np.eye(9)[None]
        Hr = np.zeros((self.nvar, 9, 9))
        live = self.slot >= 0
        np.add.at(Hr, self.slot[live], H[live])
        return Hr

    def woodbury_direction(self, H, g):
        gm = g.reshape(self.nvar, 9)
        Hinv_g = np.linalg.solve(H, gm[..., None])[..., 0].reshape(-1)
        Bt = self.B.T.reshape(self.nvar, 9, self.k)
        Hinv_Bt = np.linalg.solve(H, Bt).reshape(9 * self.nvar, self.k)
        Cap = self.Lhat - self.base.alpha * (self.B @ Hinv_Bt)
        z = sla.solve(0.5 * (Cap + Cap.T), self.B @ Hinv_g, assume_a="pos")
        return -(Hinv_g + self.base.alpha * (Hinv_Bt @ z))

    def delta_energy(self, X, dX, q, dq, a, sigma):
        b = self.base
        F = self.full_F(X)
        d = self.full_d(dX)
        ka = b.kappa * a
        dP = np.sum(b.V * delta_psi(F, d, sigma, b.mu, b.lam, ka, b.u))
        D = (b.deformation_gradients(q) - F).reshape(self.m, 9)
        dD = (b.deformation_gradients(dq) - d).reshape(self.m, 9)
        return dP + 0.5 * b.alpha * np.sum(self.w * (2.0 * sigma * np.einsum("ij,ij->i", D, dD)
                                                     + sigma**2 * np.einsum("ij,ij->i", dD, dD)))

    def identity(self):
        return np.broadcast_to(np.eye(3), (self.nvar, 3, 3)).copy()

    def residual_normaliser(self, a, X_start=None):
        b = self.base
        floor = 1e-12 * np.sqrt(np.sum((b.V * b.mu) ** 2))
        I = self.identity()
        g0 = np.linalg.norm(self.gradient(I, self.acap_solve(self.full_F(I)), a))
        if g0 <= floor:
            g0 = 0.0
            if X_start is not None:
                g0 = np.linalg.norm(self.gradient(X_start, self.acap_solve(self.full_F(X_start)), a))
                if g0 <= floor:
                    g0 = 0.0
        return g0

    # --- final coupling solve (eps2 = 0, eps1 = eps_joint_final) -------------
    def final_solve(self, X):
        """q with every bone's vertices at F_b Q_v + t_b (t_b free for free
        bones) and the joints as a penalty Vbar / |eps1|; deformable vertices
        minimise Eq. 3 with the plain weights."""
        b = self.base
        F = self.full_F(X)
        Q = b.Q
        q0 = Q.copy()
        q0[self.is_fixed] = b.q_c.reshape(-1, 3)
        bone_of_vert = np.full(self.n, -1, dtype=np.int64)
        for bb, vs in enumerate(self.bone_verts):
            bone_of_vert[vs] = bb
        free_def = np.nonzero((~self.is_fixed) & (bone_of_vert < 0))[0]
        free_bones = [bb for bb in range(self.nb) if not self.bone_fixed[bb]]
        nz = 3 * free_def.size + 3 * len(free_bones)
        rows, cols = [], []
        for c in range(3):
            rows += (3 * free_def + c).tolist()
            cols += (3 * np.arange(free_def.size) + c).tolist()
        for kb, bb in enumerate(free_bones):
            vs = self.bone_verts[bb]
            Fb = F[np.nonzero(self.bid == bb)[0][0]]
            q0[vs] = Q[vs] @ Fb.T
            for c in range(3):
                rows += (3 * vs + c).tolist()
                cols += [3 * free_def.size + 3 * kb + c] * vs.size
        P = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(3 * self.n, nz))
        q0 = q0.reshape(-1)
        w9 = np.repeat(b.w, 9)
        GP = b.G @ P
        kj = self.Vbar ** (1.0 / 3.0) / abs(self.eps_joint_final)  # Vbar / (|eps1| l^2)
        JP = self.J @ P
        A = (GP.T @ sp.diags(w9) @ GP + kj * (JP.T @ JP)).tocsc()
        rhs = GP.T @ (w9 * (F.reshape(-1) - b.G @ q0)) - kj * (JP.T @ (self.J @ q0))
        z = spla.spsolve(A, rhs)
        return (P @ z + q0)

    # --- Algorithm 1 (Newton part) on the reduced variables ------------------
    def solve(self, a, X0=None, tol=None, max_newton=None, record=False):
        p = self.p
        tol = p.tol if tol is None else tol
        max_newton = p.max_newton if max_newton is None else max_newton
        a = np.broadcast_to(np.asarray(a, dtype=np.float64), (self.m,)).copy()
        X = self.identity() if X0 is None else np.array(X0, dtype=np.float64)
        t0 = time.perf_counter()
        gnorm0 = self.residual_normaliser(a, X)
        hist, trials_total, it, res = [], 0, 0, 0.0
        while True:
            q = self.acap_solve(self.full_F(X))
            g = self.gradient(X, q, a)
            res = float(np.linalg.norm(g) / gnorm0) if gnorm0 > 0 else 0.0
            if record:
                hist.append(res)
            if res <= tol or it >= max_newton:
                break
            H = self.hessian_blocks(X, a)
            dX = self.woodbury_direction(H, g.reshape(-1)).reshape(self.nvar, 3, 3)
            gtd = float(np.sum(g * dX))
            if gtd >= 0.0:
                raise RuntimeError("quasi-Newton direction is not a descent direction")
            dq = self.acap_solve_d(self.full_d(dX))
            sigma = p.ls_sigma0
            for _ in range(p.ls_max_trials):
                trials_total += 1
                if self.delta_energy(X, dX, q, dq, a, sigma) <= p.ls_c * sigma * gtd:
                    break
                sigma *= p.ls_rho
            else:
                raise RuntimeError("line search failed")
            X = X + sigma * dX
            it += 1
        q_newton = self.acap_solve(self.full_F(X))
        q = self.final_solve(X)
        out = OracleResult(
            q=q.reshape(self.n, 3), F=X, iterations=it, rel_residual=res,
            energy=float(self.energy(X, q_newton, a)), ls_trials=trials_total, history=hist,
            seconds=time.perf_counter() - t0,
        )
        out.q_newton = q_newton.reshape(self.n, 3)
        return out
