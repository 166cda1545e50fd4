"""Global operator with constraints, assembly, and reference solvers (FP64).

* Constraints: Dirichlet velocity on walls; constrained rows and columns of
  the Jacobian become identity (source entries zeroed, result equal to the
  source there), and the residual there is u - g (g given on stationary walls,
  zero by default; omega e_z x x on walls moving with the rotor).
* Wall loads (force, torque, power) from the consistent reactions.
* Assembly (path A): element matrices of the volume terms and of every mortar
  cell pair, scattered into a CSR matrix.
* Newton (Eq. Eq-Newton-method) with GMRES (Section 4 uses GMRES) on the
  assembled matrix, pressure mean removed (the operator has the constant
  pressure in its null space).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from .fem import Problem
from .mortar import Mortar


class Operator:
    """Full discrete operator (volume + mortar + constraints) at one angle."""

    def __init__(self, mesh, nu, omega, dt, bdf, theta, F=1.0, source=None, up_star=None,
                 u_n=None, u_nm1=None, stab=True, g=None):
        self.prob = Problem(mesh, nu, omega, dt, bdf, theta, F=F, source=source, stab=stab)
        if u_n is not None:
            self.prob.set_history(u_n, u_nm1)
        self.mortar = Mortar(self.prob)
        self.d = mesh.d
        self.nn = self.prob.nn
        self.ndof = self.nn * (self.d + 1)
        self.wall = self.prob.wall
        self.up_star = None if up_star is None else np.asarray(up_star, dtype=np.float64)
        # constrained DoF mask in the interleaved layout [node][u_1..u_d, p]
        cm = np.zeros((self.nn, self.d + 1), dtype=bool)
        cm[self.wall, :self.d] = True
        self.cmask = cm
        # Dirichlet values g [N_n, d] on wall nodes (zero unless given); walls moving with the
        # rotor (wall = 2) take the rigid-rotation velocity omega e_z x x at the current angle
        self.g = np.zeros((self.nn, self.d)) if g is None else np.array(g, dtype=np.float64)
        mv = np.asarray(mesh.wall) == 2
        if mv.any():
            x = self.prob.x
            self.g[mv, 0] = -self.prob.omega * x[mv, 1]
            self.g[mv, 1] = self.prob.omega * x[mv, 0]

    def set_linearization(self, up_star):
        self.up_star = np.asarray(up_star, dtype=np.float64)

    def apply(self, x):
        """y = J x (matrix-free, path B) with constraints."""
        x = np.asarray(x, dtype=np.float64).reshape(self.nn, self.d + 1)
        xc = np.where(self.cmask, 0.0, x)
        y = self.prob.volume_apply(self.up_star, xc)
        self.mortar.apply(xc, out=y)
        y[self.cmask] = x[self.cmask]
        return y

    def residual(self, up, tau_up=None):
        """R(up) (matrix-free) with r = u - g on constrained DoFs; tau taken at
        tau_up when given (frozen-tau residual)."""
        up = np.asarray(up, dtype=np.float64).reshape(self.nn, self.d + 1)
        r = self.prob.volume_residual(up, tau_up=tau_up)
        self.mortar.apply(up, out=r)
        gg = np.zeros((self.nn, self.d + 1))
        gg[:, :self.d] = self.g
        r[self.cmask] = up[self.cmask] - gg[self.cmask]
        return r

    def wall_loads(self, up, group=None, n_groups=2):
        """Loads of the walls on the fluid from the consistent reactions
        (torque at the impeller, Section 4.4.2; power at the wall in the
        energy balance, Section 4.5.2).  r = the residual rows of the volume and
        mortar terms without the Dirichlet replacement; on a wall node i it
        equals int_wall t . phi_i, t the traction the wall exerts on the fluid.
        Summed over a group of wall nodes: force sum_i r_i, torque about the
        z axis sum_i (x_i x r_i) . e_z (= int x x t since sum_i x_i phi_i = x,
        isoparametric), power sum_i r_i . u_i.  group: [N_n] ints (wall nodes
        whose group is >= n_groups are skipped); None groups by wall type
        (0 = stationary, 1 = moving with the rotor).  Returns [n_groups, d+2]:
        force (d), torque, power."""
        up = np.asarray(up, dtype=np.float64).reshape(self.nn, self.d + 1)
        d = self.d
        r = self.prob.volume_residual(up)
        self.mortar.apply(up, out=r)
        x = self.prob.x
        w = np.asarray(self.prob.mesh.wall)
        grp = (w.astype(np.int64) - 1) if group is None else np.asarray(group, dtype=np.int64)
        out = np.zeros((n_groups, d + 2))
        for gi in range(n_groups):
            sel = (w > 0) & (grp == gi)
            rs = r[sel, :d]
            out[gi, :d] = rs.sum(0)
            out[gi, d] = float((x[sel, 0] * rs[:, 1] - x[sel, 1] * rs[:, 0]).sum())
            out[gi, d + 1] = float((rs * up[sel, :d]).sum())
        return out

    def assemble(self):
        """CSR Jacobian (path A): element matrices + mortar pair matrices, then
        identity rows/columns on constrained DoFs."""
        d, N = self.d, self.prob.N
        nf = d + 1
        rows, cols, vals = [], [], []
        nc = self.prob.cells.shape[0]
        for s0 in range(0, nc, 256):
            cl = np.arange(s0, min(nc, s0 + 256))
            E = self.prob.element_matrices(self.up_star, cl)          # [C,N,nf,N,nf]
            dof = (self.prob.cells[cl][:, :, None] * nf + np.arange(nf)[None, None]).reshape(len(cl), -1)
            E = E.reshape(len(cl), N * nf, N * nf)
            rows.append(np.repeat(dof, N * nf, axis=1).ravel())
            cols.append(np.tile(dof, (1, N * nf)).ravel())
            vals.append(E.ravel())
        for rec in self.mortar.recs:
            M = self.mortar.pair_matrix(rec).reshape(2 * N * nf, 2 * N * nf)
            cc = np.concatenate([self.prob.cells[rec["cells"][0]], self.prob.cells[rec["cells"][1]]])
            dof = (cc[:, None] * nf + np.arange(nf)[None]).ravel()
            rows.append(np.repeat(dof, len(dof)))
            cols.append(np.tile(dof, len(dof)))
            vals.append(M.ravel())
        A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.ndof, self.ndof))
        c = self.cmask.ravel()
        Pf = sp.diags((~c).astype(np.float64))
        Pc = sp.diags(c.astype(np.float64))
        return (Pf @ A @ Pf + Pc).tocsr()

    def diagonal(self):
        """diag(J) of the assembled operator."""
        return self.assemble().diagonal().reshape(self.nn, self.d + 1)


def remove_pressure_mean(v, d):
    v = np.array(v, dtype=np.float64).reshape(-1, d + 1)
    v[:, d] -= v[:, d].mean()
    return v


def gmres_solve(A, b, d, rtol=1e-10, restart=200, maxiter=20):
    """Restarted GMRES on A x = b with the pressure mean removed from b and x."""
    b = remove_pressure_mean(b, d).ravel()
    x, info = spla.gmres(A, b, rtol=rtol, atol=0.0, restart=restart, maxiter=maxiter)
    return remove_pressure_mean(x, d), info


def bordered_solve(A, b, d):
    """Direct solve of A x = b with the extra condition sum(pressure) = 0
    (Lagrange-multiplier border); A is singular in the constant pressure."""
    n = A.shape[0]
    e = np.zeros(n)
    e[d::d + 1] = 1.0
    Ab = sp.bmat([[A, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]]).tocsc()
    x = spla.spsolve(Ab, np.concatenate([b, [0.0]]))
    return x[:n]


def chord_solve(mesh, params, up0, rtol=1e-11, max_iter=200, F=1.0, source=None, g=None, refresh=10):
    """Solve R(u) = 0 with Jacobians assembled at the iterate every `refresh`
    steps and reused in between (chord form of Eq. Eq-Newton-method); direct
    sparse LU solves.  The constant pressure is a null vector only up to the
    interface geometry defect, so the factorised Jacobian is invertible and the
    pressure level follows from it.  Stops at ||R||_2 <= rtol ||R_0||_2."""
    op = Operator(mesh, params["nu"], params["omega"], params["dt"], params["bdf"], params["theta"],
                  F=F, source=source, g=g)
    up = np.array(up0, dtype=np.float64).reshape(op.nn, op.d + 1)
    hist, lu = [], None
    for it in range(max_iter):
        r = op.residual(up)
        nr = np.linalg.norm(r)
        hist.append(nr)
        if nr <= rtol * hist[0] or nr < 1e-14:
            break
        if lu is None or it % refresh == 0:
            op.set_linearization(up)
            A = op.assemble()
            lu = spla.splu(A.tocsc())
        dx = lu.solve(-r.ravel())
        up = up + dx.reshape(up.shape)
    return up, hist


def newton(mesh, params, up0, u_n=None, u_nm1=None, rtol=1e-8, lin_rtol=1e-4, max_newton=20, F=1.0,
           source=None, g=None, direct=False):
    """Newton's method R(u) = 0 with the assembled Jacobian at each iterate;
    stops at ||R||_2 <= rtol ||R_0||_2."""
    op = Operator(mesh, params["nu"], params["omega"], params["dt"], params["bdf"], params["theta"],
                  F=F, source=source, u_n=u_n, u_nm1=u_nm1, g=g)
    up = np.array(up0, dtype=np.float64).reshape(op.nn, op.d + 1)
    r0 = None
    hist = []
    for it in range(max_newton):
        r = op.residual(up)
        nr = np.linalg.norm(r)
        hist.append(nr)
        r0 = nr if r0 is None else r0
        if nr <= rtol * r0 or nr < 1e-13:
            break
        op.set_linearization(up)
        A = op.assemble()
        if direct:
            dx = bordered_solve(A, -r.ravel(), op.d).reshape(up.shape)
        else:
            dx, _ = gmres_solve(A, -r.ravel(), op.d, rtol=lin_rtol)
        up = up + dx
    return up, hist
