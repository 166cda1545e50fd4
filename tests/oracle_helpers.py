"""Shared helpers for the oracle pin tests (test code only)."""
import numpy as np

import synth
from oracle.fem import Problem
from oracle.solve import Operator


def small_case(d=2, k=2, m=2, n_r=1, n_s=2, n_z=2, nu=0.1, omega=1.0, dt=0.01, bdf=1, theta=0.137,
               state="iid", seed=7):
    mesh, prm, f = synth.make_config(d=d, k=k, m=m, n_r=n_r, n_s=n_s, n_z=n_z, nu=nu, omega=omega,
                                     dt=dt, bdf=bdf, theta=theta, state=state, seed=seed)
    return mesh, prm, f


def make_op(mesh, prm, f, **kw):
    return Operator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"],
                    up_star=f["up_star"], u_n=f["u_n"], u_nm1=f["u_nm1"], **kw)


def merge_interface(op):
    """Map every rotor interface node onto the coincident stator node (valid at a
    conforming rotor angle).  Returns (P, conforming mesh-like object) with
    P [N_mortar] -> index in the merged numbering."""
    mesh = op.prob.mesh
    x = op.prob.x
    r = np.linalg.norm(x[:, :2], axis=1)
    on_if = np.abs(r - mesh.R) < 1e-12
    rot_if = np.where(on_if & (mesh.node_side == 0))[0]
    st_if = np.where(on_if & (mesh.node_side == 1))[0]
    target = np.arange(len(x))
    for i in rot_if:
        dist = np.linalg.norm(x[st_if] - x[i], axis=1)
        j = np.argmin(dist)
        assert dist[j] < 1e-12
        target[i] = st_if[j]
    keep = np.unique(target)
    newid = -np.ones(len(x), dtype=np.int64)
    newid[keep] = np.arange(len(keep))
    P = newid[target]

    class M:
        pass
    cm = M()
    cm.d, cm.k = mesh.d, mesh.k
    cm.x0 = x[keep]
    cm.cells = P[np.asarray(mesh.cells)].astype(np.int32)
    cm.cell_side = mesh.cell_side
    cm.node_side = np.ones(len(keep), np.uint8)       # already at the rotated position
    cm.wall = np.zeros(len(keep), np.uint8)
    np.maximum.at(cm.wall, P, np.asarray(mesh.wall))
    return P, cm
