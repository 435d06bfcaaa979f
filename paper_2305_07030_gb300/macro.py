"""Synthetic macroscale driver of the FE2 scheme (Section I).

In the FE2 method every material point of a macroscale finite-element model
obtains its constitutive response from a microscale RVE solve: the macroscale
deformation gradient F at a Gauss point drives the RVE to equilibrium, and the
RVE's volume-averaged Cauchy stress is the stress at that point. This module
is a small, self-contained macroscale model around the batched RVE solver:

* a structured mesh of 8-node trilinear hexahedra on a box, 2 x 2 x 2 Gauss
  points per element, one RVE per Gauss point;
* the reference-configuration kinematics F = I + grad_X u at each Gauss point
  and the internal force vector f_a = sum_gp P grad_X N_a w det J with the
  first Piola-Kirchhoff stress P = det(F) sigma F^-T;
* prescribed displacements u = (F_macro - I) X on every boundary node, the
  interior nodes free;
* an outer loop per macro step: solve every Gauss point's RVE (one batched
  solve, warm-started from the previous outer iteration), assemble the
  out-of-balance force on the free nodes, and correct the free displacements
  with a fixed elastic stiffness K0 (modified Newton). The paper does not give
  a consistent tangent; K0 is the small-strain isotropic stiffness fitted to
  the RVEs' own response to two probe strains.

The RVE solve is a function argument (``solve_fn``), so the same driver runs
the GPU batch or, in tests, any other solver of the same problem. Host only
(numpy); every RVE iteration runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

GP = 1.0 / np.sqrt(3.0)
# corner signs of the 8-node hexahedron (xi, eta, zeta), counter-clockwise
# bottom face then top face
CORNERS = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                    [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=float)
GAUSS = CORNERS * GP  # 2 x 2 x 2 points, weights 1


def shape_gradients(xi):
    """d N_a / d xi (8 x 3) of the trilinear shape functions at xi (3,)."""
    s = CORNERS
    one = 1.0 + s * xi[None, :]
    g = np.empty((8, 3))
    g[:, 0] = s[:, 0] * one[:, 1] * one[:, 2] / 8.0
    g[:, 1] = s[:, 1] * one[:, 0] * one[:, 2] / 8.0
    g[:, 2] = s[:, 2] * one[:, 0] * one[:, 1] / 8.0
    return g


class HexMesh:
    """nx x ny x nz trilinear hexahedra on [0, Lx] x [0, Ly] x [0, Lz]."""

    def __init__(self, nx, ny, nz, size=(1.0, 1.0, 1.0)):
        self.shape = (nx, ny, nz)
        xs = [np.linspace(0.0, size[d], n + 1) for d, n in enumerate((nx, ny, nz))]
        # node (i, j, k) -> i + (nx+1) (j + (ny+1) k)
        kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1),
                                 indexing="ij")
        self.X = np.stack([xs[0][ii.ravel()], xs[1][jj.ravel()], xs[2][kk.ravel()]], axis=1)
        nid = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)  # noqa: E731
        conn = []
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    conn.append([nid(i + (c[0] > 0), j + (c[1] > 0), k + (c[2] > 0))
                                 for c in CORNERS])
        self.conn = np.array(conn, dtype=np.int64)
        self.n_nodes = self.X.shape[0]
        self.n_elems = self.conn.shape[0]
        self.n_gp = 8 * self.n_elems
        b = np.zeros(self.n_nodes, bool)
        for d, n in enumerate((nx, ny, nz)):
            b |= np.isclose(self.X[:, d], 0.0) | np.isclose(self.X[:, d], size[d])
        self.boundary = b
        # reference shape-function gradients and weights per Gauss point
        self.dNdX = np.empty((self.n_elems, 8, 8, 3))
        self.wdetJ = np.empty((self.n_elems, 8))
        for e in range(self.n_elems):
            Xe = self.X[self.conn[e]]
            for g, xi in enumerate(GAUSS):
                dN = shape_gradients(xi)
                J = Xe.T @ dN  # dX/dxi
                self.dNdX[e, g] = dN @ np.linalg.inv(J)
                self.wdetJ[e, g] = np.linalg.det(J)

    def deformation_gradients(self, u):
        """F = I + sum_a u_a (x) grad_X N_a at every Gauss point: (n_gp, 3, 3),
        element-major, Gauss points in GAUSS order."""
        ue = u[self.conn]  # (E, 8, 3)
        H = np.einsum("eai,egaj->egij", ue, self.dNdX)
        return (np.eye(3)[None, None] + H).reshape(-1, 3, 3)

    def internal_forces(self, F, sigma):
        """f_a = sum_gp P grad_X N_a w det J, P = det(F) sigma F^-T; (n_nodes, 3)."""
        F = F.reshape(self.n_elems, 8, 3, 3)
        sigma = sigma.reshape(self.n_elems, 8, 3, 3)
        J = np.linalg.det(F)
        P = J[..., None, None] * sigma @ np.transpose(np.linalg.inv(F), (0, 1, 3, 2))
        fe = np.einsum("egij,egaj,eg->eai", P, self.dNdX, self.wdetJ)
        f = np.zeros((self.n_nodes, 3))
        np.add.at(f, self.conn, fe)
        return f

    def stiffness(self, lam, mu):
        """Small-strain stiffness of an isotropic material (lam, mu): the
        3 n_nodes square matrix of sum_gp B^T C B w det J."""
        n = 3 * self.n_nodes
        K = np.zeros((n, n))
        for e in range(self.n_elems):
            dofs = (3 * self.conn[e][:, None] + np.arange(3)[None, :]).ravel()
            Ke = np.zeros((24, 24))
            for g in range(8):
                G = self.dNdX[e, g]  # (8, 3)
                # K_{ai,bk} = lam G_ai G_bk + mu (G_aj G_bj delta_ik + G_ak G_bi)
                GG = G @ G.T
                Kg = (lam * np.einsum("ai,bk->aibk", G, G)
                      + mu * np.einsum("ab,ik->aibk", GG, np.eye(3))
                      + mu * np.einsum("ak,bi->aibk", G, G))
                Ke += Kg.reshape(24, 24) * self.wdetJ[e, g]
            K[np.ix_(dofs, dofs)] += Ke
        return K


def fit_isotropic(solve_fn, eps=1e-3):
    """(lam, mu) of the small-strain response averaged over the Gauss points:
    solve_fn(F (P,3,3), first) -> sigma (P,3,3) at F = I + eps e_x (x) e_x
    gives lam + 2 mu = <s_xx>/eps and lam = <s_yy + s_zz>/(2 eps)."""
    F = np.diag([1.0 + eps, 1.0, 1.0])
    s = solve_fn(None, F)
    sxx = float(np.mean(s[:, 0, 0]))
    slat = float(np.mean(0.5 * (s[:, 1, 1] + s[:, 2, 2])))
    lam = slat / eps
    mu = 0.5 * (sxx / eps - lam)
    return lam, max(mu, 1e-6 * abs(sxx / eps))


class FE2Driver:
    """Quasi-static FE2 loop on a HexMesh with one RVE per Gauss point.

    solve_fn(F, F_uniform) solves every Gauss point's RVE for the given
    deformation gradients (F: (n_gp, 3, 3); or, when F is None, the same
    F_uniform at every point) and returns their Cauchy stresses (n_gp, 3, 3).
    The driver does no RVE arithmetic of its own."""

    def __init__(self, mesh: HexMesh, solve_fn, lam=None, mu=None):
        self.mesh = mesh
        self.solve_fn = solve_fn
        if lam is None or mu is None:
            lam, mu = fit_isotropic(solve_fn)
        self.lam, self.mu = lam, mu
        n = mesh.n_nodes
        self.free = np.repeat(~mesh.boundary, 3)
        K = mesh.stiffness(lam, mu)
        self.K0 = K[np.ix_(self.free, self.free)]
        self.u = np.zeros((n, 3))
        self.history = []

    def step(self, F_macro, tol=1e-6, max_outer=30):
        """One macro step: boundary nodes at u = (F_macro - I) X, free nodes
        relaxed by modified Newton until the out-of-balance force on them is
        at most tol times the largest nodal force. Returns a record of the
        step (outer iterations, residual history, volume-averaged stress)."""
        m = self.mesh
        ub = m.X @ (F_macro - np.eye(3)).T
        u = self.u.copy()
        u[m.boundary] = ub[m.boundary]
        if not np.any(self.u):  # first step: start from the affine field
            u = ub.copy()
        res = []
        for it in range(max_outer):
            F = m.deformation_gradients(u)
            sigma = self.solve_fn(F, None)
            f = m.internal_forces(F, sigma)
            r = f.reshape(-1)[self.free]
            scale = max(np.abs(f).max(), 1e-300)
            res.append(float(np.abs(r).max() / scale))
            if res[-1] <= tol:
                break
            du = np.linalg.solve(self.K0, r)
            uf = u.reshape(-1).copy()
            uf[self.free] -= du
            u = uf.reshape(-1, 3)
        self.u = u
        vol = m.wdetJ.reshape(-1)
        sig_avg = np.einsum("gij,g->ij", sigma, vol) / vol.sum()
        rec = {"outer": len(res), "residuals": res, "converged": res[-1] <= tol,
               "sigma_avg": sig_avg, "F": F, "sigma": sigma}
        self.history.append(rec)
        return rec


class BatchRVEs:
    """solve_fn of FE2Driver on the GPU: one Batch holding every Gauss
    point's RVE; the first solve starts affine, later ones warm from the
    previous solve's converged state (kept on the device)."""

    def __init__(self, nets, damping=None, precision="mixed", tol=1e-8, **opts):
        from . import Batch
        self.batch = Batch(nets, damping=damping)
        self.n = len(nets)
        self.opts = dict(precision=precision, tol=tol, **opts)
        self.solves = 0
        self.iters = []

    def __call__(self, F, F_uniform):
        if F is None:
            F = np.tile(np.asarray(F_uniform, float), (self.n, 1, 1))
        self.batch.solve(F, init="warm" if self.solves else "affine", **self.opts)
        out = self.batch.stress()
        bad = [p for p, s in enumerate(out["status"]) if s != "OK"]
        if bad:
            raise RuntimeError(f"RVEs {bad[:8]} did not converge: {[out['status'][p] for p in bad[:8]]}")
        self.solves += 1
        self.iters.append(np.asarray(out["iters"]).copy())
        return out["sigma"]

    def close(self):
        self.batch.close()
