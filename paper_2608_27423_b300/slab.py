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
import numpy as np

from . import RotorStatorOperator, slab_partition, halo_pack, halo_add


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
