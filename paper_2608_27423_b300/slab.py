"""z-slab partition of the operator over ranks, one GPU per rank (the paper
partitions its mesh over MPI ranks, Section 3.3; here the parts are z-slabs).

Part p owns the z-layers [floor(p n_z / P), floor((p+1) n_z / P)) of a 3D
rotor-stator mesh (mf_mesh_slab).  Every mortar pair lies in one layer, so the
mortar terms never cross parts.  An apply (or residual) on a part leaves
partial rows on the node planes it shares with its neighbours; one exchange
per neighbour and per apply completes them: each part packs its shared-plane
rows (mf_halo_pack), sends them to the neighbour and adds what it receives
(mf_halo_add, which leaves the identity rows of wall velocities alone).  The
exchange uses torch.distributed point-to-point calls (NCCL between GPUs; gloo
for host tensors), so this module holds the protocol and the buffers only:
every arithmetic step of the apply runs in the library.
"""
import math

import numpy as np

from . import RotorStatorOperator, slab_partition, halo_pack, halo_add, vec_dots, vec_maxpy, vec_axpby, vec_mul


def halo_exchange(y, lo, hi, part, n_parts, pack, add, bufs, group=None):
    """Complete the shared-plane rows of y [n_nodes, d+1] on part `part`.

    lo / hi: index tensors of the planes shared with part-1 / part+1 (the
    neighbour's hi / lo list holds the same nodes in the same order);
    pack(y, idx, buf) and add(y, idx, which, buf) move the rows (which = "lo"
    or "hi" selects the wall mask); bufs: dict of send / receive buffers
    ("lo_send", "lo_recv", "hi_send", "hi_recv"), each [n, d+1] like y.
    Non-blocking sends and receives to both neighbours, then the adds."""
    import torch.distributed as dist
    reqs = []
    if part > 0 and lo.numel():
        pack(y, lo, bufs["lo_send"])
    if part + 1 < n_parts and hi.numel():
        pack(y, hi, bufs["hi_send"])
    if part > 0 and lo.numel():
        reqs.append(dist.isend(bufs["lo_send"], part - 1, group=group))
        reqs.append(dist.irecv(bufs["lo_recv"], part - 1, group=group))
    if part + 1 < n_parts and hi.numel():
        reqs.append(dist.isend(bufs["hi_send"], part + 1, group=group))
        reqs.append(dist.irecv(bufs["hi_recv"], part + 1, group=group))
    for r in reqs:
        r.wait()
    if part > 0 and lo.numel():
        add(y, lo, "lo", bufs["lo_recv"])
    if part + 1 < n_parts and hi.numel():
        add(y, hi, "hi", bufs["hi_recv"])


class SlabOperator:
    """The operator on one z-slab of `mesh` (part `part` of n_parts) on the
    current CUDA device, with the halo exchange after every apply and
    residual.  Vectors are the part's local rows [n_local_nodes, d+1] in the
    slab's numbering (plan["node_global"] maps them to the global mesh)."""

    def __init__(self, mesh, nu, omega, dt, bdf, n_parts, part, group=None, penalty_F=1.0):
        import torch
        self.slab, self.plan = slab_partition(mesh, n_parts, part)
        self.part, self.n_parts, self.group = int(part), int(n_parts), group
        self.op = RotorStatorOperator(self.slab, nu, omega, dt, bdf, penalty_F=penalty_F)
        dev = torch.device("cuda", torch.cuda.current_device())
        nf = mesh.d + 1
        self.lo = torch.tensor(self.plan["lo"], dtype=torch.int32, device=dev)
        self.hi = torch.tensor(self.plan["hi"], dtype=torch.int32, device=dev)
        self.walls = {"lo": torch.tensor(self.plan["lo_wall"], dtype=torch.uint8, device=dev),
                      "hi": torch.tensor(self.plan["hi_wall"], dtype=torch.uint8, device=dev)}
        self.bufs = {f"{w}_{k}": torch.empty((len(self.plan[w]), nf), dtype=torch.float64, device=dev)
                     for w in ("lo", "hi") for k in ("send", "recv")}

    @property
    def n_nodes(self):
        return self.slab.n_nodes

    def local(self, global_array):
        """This part's rows of a global per-node array (host numpy)."""
        return np.ascontiguousarray(np.asarray(global_array)[self.plan["node_global"]])

    def _exchange(self, y):
        halo_exchange(y, self.lo, self.hi, self.part, self.n_parts, lambda v, i, b: halo_pack(v, i, b),
                      lambda v, i, which, b: halo_add(v, i, self.walls[which], b), self.bufs, self.group)

    def set_history(self, u_n, u_nm1=None):
        self.op.set_history(u_n, u_nm1)

    def set_linearization(self, up_star, theta):
        self.op.set_linearization(up_star, theta)

    def apply_jacobian(self, x, y):
        """y = J x on this part's rows, shared planes completed (FP64)."""
        self.op.apply_jacobian(x, y)
        self._exchange(y)

    def residual(self, up, r):
        self.op.residual(up, r)
        self._exchange(r)

    def diagonal(self, out):
        """diag(J) on this part's rows (FP64), shared planes completed."""
        self.op.diagonal(out)
        self._exchange(out)

    def owned_weights(self):
        """Weights [n_local_nodes * (d+1)] of this part's rows in global sums:
        0 on the plane shared with the part below (that part counts it), 1
        elsewhere."""
        return owned_weights(self.plan, self.slab.n_nodes, self.slab.d + 1, self.lo.device)


def owned_weights(plan, n_nodes, nf, device=None):
    """1 for the rows a part counts in global sums, 0 for the rows of its lower
    shared plane (owned by the part below): every global row counted once."""
    import torch
    w = torch.ones((n_nodes, nf), dtype=torch.float64, device=device)
    lo = np.asarray(plan["lo"], dtype=np.int64)
    if lo.size:
        w[torch.as_tensor(lo, device=w.device)] = 0.0
    return w.reshape(-1)


class LibVec:
    """The library's Krylov vector kernels (mf_vec_*), for distributed_fgmres
    on device tensors."""

    @staticmethod
    def dots(V, x, w, out):
        vec_dots(V, x, out, w)

    @staticmethod
    def maxpy(V, c, y, sign):
        vec_maxpy(V, c, y, sign)

    @staticmethod
    def axpby(a, x, b, y):
        vec_axpby(a, x, b, y)

    @staticmethod
    def mul(d, v, z):
        vec_mul(d, v, z)


def distributed_fgmres(apply, precond, b, x, weights, vec, m=30, rtol=1e-8, max_iters=300, group=None):
    """Right-preconditioned FGMRES(m) with classical Gram-Schmidt applied
    twice, for A x = b whose rows are spread over the z-slab parts.

    Every part calls it with its own rows (flat FP64 tensors of equal layout):
    apply(v, out) -> A v with the shared-plane rows completed (halo exchange
    inside); precond(v, out) -> a right preconditioner that keeps shared rows
    consistent (e.g. the inverse of the completed diagonal); weights count
    each shared row once (owned_weights; None on a single part); vec does the
    vector arithmetic (LibVec: the library's kernels).  The dot products of
    each Gram-Schmidt pass and each norm are one all_reduce over the group
    (the parts' only collective; skipped without an initialised process
    group).  x is overwritten (zero initial guess).  Returns (iterations,
    relative residual ||b - A x|| / ||b|| as FGMRES estimates it)."""
    import torch
    import torch.distributed as dist
    n = b.numel()
    dev, dt = b.device, b.dtype
    multi = dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1
    V = torch.zeros((m + 1, n), dtype=dt, device=dev)
    Z = torch.zeros((m, n), dtype=dt, device=dev)
    wv = torch.zeros(n, dtype=dt, device=dev)
    r = torch.zeros(n, dtype=dt, device=dev)
    d_out = torch.zeros(m + 1, dtype=dt, device=dev)
    c_dev = torch.zeros(m + 1, dtype=dt, device=dev)

    def dots(Vs, v):
        out = d_out[:Vs.shape[0]]
        vec.dots(Vs, v, weights, out)
        if multi:
            dist.all_reduce(out, group=group)
        return out.cpu().numpy().astype(np.float64)

    def coeffs(vals):
        c_dev[:len(vals)].copy_(torch.as_tensor(np.asarray(vals, dtype=np.float64)))
        return c_dev[:len(vals)]

    vec.mul(Z[0], b, x)                            # x = 0 (Z is zero here; x may hold anything finite or not)
    vec.axpby(1.0, b, 0.0, r)                      # r = b
    beta0 = math.sqrt(max(dots(b[None], b)[0], 0.0))
    if beta0 == 0.0:
        return 0, 0.0
    total, res = 0, 1.0
    while True:
        beta = math.sqrt(max(dots(r[None], r)[0], 0.0))
        if beta <= rtol * beta0 or total >= max_iters:
            return total, beta / beta0
        vec.axpby(1.0 / beta, r, 0.0, V[0])
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        j = 0
        done = False
        while j < m and total < max_iters:
            precond(V[j], Z[j])
            apply(Z[j], wv)
            h1 = dots(V[:j + 1], wv)
            vec.maxpy(V[:j + 1], coeffs(h1), wv, -1.0)
            h2 = dots(V[:j + 1], wv)
            vec.maxpy(V[:j + 1], coeffs(h2), wv, -1.0)
            hn = math.sqrt(max(dots(wv[None], wv)[0], 0.0))
            H[:j + 1, j] = h1 + h2
            H[j + 1, j] = hn
            if hn > 0.0:
                vec.axpby(1.0 / hn, wv, 0.0, V[j + 1])
            for i in range(j):                     # previous rotations
                a, c = H[i, j], H[i + 1, j]
                H[i, j], H[i + 1, j] = cs[i] * a + sn[i] * c, -sn[i] * a + cs[i] * c
            rr = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = (H[j, j] / rr, H[j + 1, j] / rr) if rr > 0 else (1.0, 0.0)
            H[j, j], H[j + 1, j] = rr, 0.0
            g[j + 1], g[j] = -sn[j] * g[j], cs[j] * g[j]
            j += 1
            total += 1
            res = abs(g[j]) / beta0
            if res <= rtol or hn == 0.0:
                done = True
                break
        y = np.zeros(j)
        for i in range(j - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j] @ y[i + 1:j]) / H[i, i]
        vec.maxpy(Z[:j], coeffs(y), x, 1.0)
        if done:
            return total, res
        apply(x, r)                                # true residual for the restart
        vec.axpby(1.0, b, -1.0, r)
