"""Additive Schwarz (ASM) smoother with cell patches, plain FP64 -- test
infrastructure only (the oracle; product code never imports it).

The paper's multigrid smooths with an inverse diagonal (ID) or an additive
Schwarz method (Section 3.4, accelerated by a relaxation scheme), and builds
the local matrices it needs column by column from the matrix-free operator,
mortar terms included (Algorithm 2).  Readings taken here (the paper does not
spell the ASM out):
* patches are the cells; the local matrix of cell K is its own element
  matrix: the volume blocks A-hat..D-hat of Section 2.3 on K plus, for an
  interface cell, the own-side diagonal blocks of every mortar segment it
  meets (the trial and test functions both of K; the blocks coupling the two
  sides of a segment belong to no patch) -- exactly what Algorithm 2
  reconstructs per cell;
* wall velocity DoFs are identity rows and columns of the local matrix, and
  the smoother passes them through (z = r there), like the global Jacobian;
* corrections are averaged over the cells that share a DoF (weight 1/mult):
  z = sum_K R_K^T W_K A_K^{-1} R_K r (weighted additive Schwarz).
"""
import numpy as np


def local_matrices(op):
    """A_K [n_cells, N (d+1), N (d+1)] of an oracle.solve.Operator `op` at
    its linearisation (rows/columns in the cell's tensor node order, fields
    fastest), wall velocity rows/columns replaced by identity."""
    prob = op.prob
    d, N = prob.d, prob.N
    nf = d + 1
    nc = prob.cells.shape[0]
    A = np.zeros((nc, N * nf, N * nf))
    for s0 in range(0, nc, 256):
        cl = np.arange(s0, min(nc, s0 + 256))
        A[cl] = prob.element_matrices(op.up_star, cl).reshape(len(cl), N * nf, N * nf)
    for rec in op.mortar.recs:
        M = op.mortar.pair_matrix(rec)                  # [2, N, nf, 2, N, nf]
        for s in range(2):
            A[rec["cells"][s]] += M[s, :, :, s, :, :].reshape(N * nf, N * nf)
    wall = np.asarray(prob.mesh.wall).astype(bool)
    for K in range(nc):
        dof_wall = np.zeros((N, nf), bool)
        dof_wall[:, :d] = wall[prob.cells[K]][:, None]
        m = dof_wall.ravel()
        A[K][m, :] = 0.0
        A[K][:, m] = 0.0
        A[K][m, m] = 1.0
    return A


def asm_apply(op, r, A=None):
    """z = weighted additive Schwarz of r [N_n, d+1] with cell patches."""
    prob = op.prob
    d, N = prob.d, prob.N
    nf = d + 1
    A = local_matrices(op) if A is None else A
    r = np.asarray(r, dtype=np.float64).reshape(prob.nn, nf)
    wall = np.asarray(prob.mesh.wall).astype(bool)
    mult = np.zeros(prob.nn)
    np.add.at(mult, prob.cells.ravel(), 1.0)
    z = np.zeros_like(r)
    for K in range(prob.cells.shape[0]):
        nodes = prob.cells[K]
        rK = r[nodes].copy()
        rK[wall[nodes], :d] = 0.0
        zK = np.linalg.solve(A[K], rK.ravel()).reshape(N, nf)
        np.add.at(z, nodes, zK / mult[nodes][:, None])
    z[wall, :d] = r[wall, :d]
    return z
