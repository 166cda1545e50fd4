"""z-slab partition of the operator (multi-GPU layout; the paper's mesh
decomposition is Section 3.3).  On the CPU: the library's partitioner
(mf_mesh_slab, host code) covers the mesh with disjoint parts whose shared
node planes match, and two gloo ranks that each apply the ORACLE's Jacobian
on their own slab and run the package's halo-exchange protocol reproduce the
oracle's global apply on every row.  The exchange's pack / add run here in
numpy on host tensors; on GPUs the same protocol moves device tensors with
the library's pack / add kernels (tests/test_gpu_slab.py)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth


def _mesh():
    mesh, prm, f = synth.make_config(d=3, k=2, m=2, n_r=1, n_s=2, n_z=5, nu=0.05, omega=1.0, dt=0.01, bdf=2,
                                     theta=0.37, state="smooth", seed=31)
    return mesh, prm, f


@pytest.mark.parametrize("n_parts", [1, 2, 3, 5])
def test_partition_covers_mesh_with_matching_planes(n_parts):
    from paper_2608_27423_b300 import slab_partition
    mesh, prm, f = _mesh()
    parts = [slab_partition(mesh, n_parts, p) for p in range(n_parts)]
    # cells: disjoint cover (counted through the layers' interface rows and the cell totals)
    assert sum(s.n_cells for s, _ in parts) == mesh.n_cells
    assert [pl["layer_begin"] for _, pl in parts] == [int(p * mesh.n_z / n_parts) for p in range(n_parts)]
    covered = np.zeros(mesh.n_nodes, int)
    for s, pl in parts:
        ng = pl["node_global"]
        assert np.all(np.diff(ng) > 0)                      # ascending global ids
        covered[ng] += 1
        # the slab's nodes, cells and interface rows are the global ones
        assert np.array_equal(s.x0, mesh.x0[ng])
        assert np.array_equal(s.wall, mesh.wall[ng])
        gcells = ng[np.asarray(s.cells)]
        l0, l1 = pl["layer_begin"], pl["layer_end"]
        assert s.n_z == l1 - l0
        for lz in range(l0, l1):
            for j in range(mesh.n_R):
                assert np.array_equal(gcells[s.iface_rotor[lz - l0, j]],
                                      np.asarray(mesh.cells)[mesh.iface_rotor[lz, j]])
                assert np.array_equal(gcells[s.iface_stator[lz - l0, j]],
                                      np.asarray(mesh.cells)[mesh.iface_stator[lz, j]])
    assert covered.min() >= 1
    # shared planes: part p's upper plane is part p+1's lower plane, same order
    for p in range(n_parts - 1):
        a, b = parts[p][1], parts[p + 1][1]
        ga, gb = a["node_global"][a["hi"]], b["node_global"][b["lo"]]
        assert len(ga) > 0 and np.array_equal(ga, gb)
        assert np.array_equal(a["hi_wall"], b["lo_wall"])
        # the shared nodes are exactly the nodes both parts use
        assert np.array_equal(np.intersect1d(a["node_global"], b["node_global"]), ga)
        z = mesh.x0[ga, 2]
        assert np.ptp(z) < 1e-12                              # one node plane
    assert len(parts[0][1]["lo"]) == 0 and len(parts[-1][1]["hi"]) == 0
    # nodes counted twice are exactly the shared-plane nodes
    assert (covered == 2).sum() == sum(len(pl["hi"]) for _, pl in parts[:-1])


def test_partition_rejects_bad_arguments():
    from paper_2608_27423_b300 import slab_partition, MfError
    mesh, prm, f = _mesh()
    with pytest.raises(MfError):
        slab_partition(mesh, mesh.n_z + 1, 0)
    with pytest.raises(MfError):
        slab_partition(mesh, 2, 2)
    m2 = synth.rotor_stator_mesh(2, 2, 2, 1, 2)
    with pytest.raises(MfError):
        slab_partition(m2, 1, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _np_pack(y, idx, buf):
    buf.copy_(y[idx.long()])


def _np_add_with(walls):
    def add(y, idx, which, buf):
        w = walls[which].bool()
        b = buf.clone()
        b[w, :-1] = 0.0                                       # wall velocity rows stay identity rows
        y.index_add_(0, idx.long(), b)
    return add


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle.solve import Operator
        from paper_2608_27423_b300 import slab_partition
        from paper_2608_27423_b300.slab import halo_exchange
        mesh, prm, f = _mesh()
        slab, plan = slab_partition(mesh, world, rank)
        ng = plan["node_global"]
        loc = lambda a: None if a is None else np.ascontiguousarray(a[ng])
        op = Operator(slab, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"], up_star=loc(f["up_star"]),
                      u_n=loc(f["u_n"]), u_nm1=loc(f["u_nm1"]))
        results = {}
        for kind in ("jacobian", "residual"):
            vec = f["x"] if kind == "jacobian" else f["up_star"] * 0.6 + 0.05
            y = op.apply(loc(vec)) if kind == "jacobian" else op.residual(loc(vec))
            y = torch.tensor(np.asarray(y).reshape(slab.n_nodes, -1))
            lo = torch.tensor(plan["lo"])
            hi = torch.tensor(plan["hi"])
            walls = {"lo": torch.tensor(plan["lo_wall"]), "hi": torch.tensor(plan["hi_wall"])}
            nf = y.shape[1]
            bufs = {f"{w}_{k}": torch.empty((len(plan[w]), nf), dtype=torch.float64)
                    for w in ("lo", "hi") for k in ("send", "recv")}
            halo_exchange(y, lo, hi, rank, world, _np_pack, _np_add_with(walls), bufs)
            results[kind] = (ng.copy(), y.numpy().copy())
        out[rank] = results
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_with_halo_exchange_reproduce_global_oracle(world):
    """Each gloo rank applies the oracle's Jacobian (and residual) on its own
    slab only; after the halo exchange every local row equals the global
    oracle's row (shared planes and mortar rows included)."""
    from oracle.solve import Operator
    mesh, prm, f = _mesh()
    ref = Operator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"], up_star=f["up_star"],
                   u_n=f["u_n"], u_nm1=f["u_nm1"])
    y_ref = np.asarray(ref.apply(f["x"])).reshape(mesh.n_nodes, -1)
    r_ref = np.asarray(ref.residual(f["up_star"] * 0.6 + 0.05)).reshape(mesh.n_nodes, -1)
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for kind, full in (("jacobian", y_ref), ("residual", r_ref)):
        scale = np.abs(full).max()
        seen = np.zeros(mesh.n_nodes, bool)
        for rank in range(world):
            ng, y = out[rank][kind]
            assert np.abs(y - full[ng]).max() <= 1e-12 * scale, (kind, rank, np.abs(y - full[ng]).max() / scale)
            seen[ng] = True
        assert seen.all()


def test_single_part_needs_no_exchange():
    """n_parts = 1: the slab is the whole mesh with no shared planes."""
    from paper_2608_27423_b300 import slab_partition
    mesh, prm, f = _mesh()
    s, pl = slab_partition(mesh, 1, 0)
    assert s.n_nodes == mesh.n_nodes and s.n_cells == mesh.n_cells
    assert len(pl["lo"]) == 0 and len(pl["hi"]) == 0
    assert np.array_equal(pl["node_global"], np.arange(mesh.n_nodes))


class _TorchVec:
    """Host stand-in for the library's Krylov vector kernels (mf_vec_*)."""

    @staticmethod
    def dots(V, x, w, out):
        out.copy_((V * (x if w is None else w * x)).sum(dim=1))

    @staticmethod
    def maxpy(V, c, y, sign):
        y.add_(sign * (c[:, None] * V).sum(dim=0))

    @staticmethod
    def axpby(a, x, b, y):
        y.copy_(a * x + b * y)

    @staticmethod
    def mul(d, v, z):
        z.copy_(d * v)


def _fgmres_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle.solve import Operator
        from paper_2608_27423_b300 import slab_partition
        from paper_2608_27423_b300.slab import halo_exchange, distributed_fgmres, owned_weights
        mesh, prm, f = _mesh()
        slab, plan = slab_partition(mesh, world, rank)
        ng = plan["node_global"]
        loc = lambda a: None if a is None else np.ascontiguousarray(a[ng])
        op = Operator(slab, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"], up_star=loc(f["up_star"]),
                      u_n=loc(f["u_n"]), u_nm1=loc(f["u_nm1"]))
        nf = mesh.d + 1
        lo, hi = torch.tensor(plan["lo"]), torch.tensor(plan["hi"])
        walls = {"lo": torch.tensor(plan["lo_wall"]), "hi": torch.tensor(plan["hi_wall"])}
        bufs = {f"{w}_{k}": torch.empty((len(plan[w]), nf), dtype=torch.float64)
                for w in ("lo", "hi") for k in ("send", "recv")}

        def complete(y):                       # [n_nodes * nf] -> shared planes summed
            y2 = y.view(slab.n_nodes, nf)
            halo_exchange(y2, lo, hi, rank, world, _np_pack, _np_add_with(walls), bufs)

        def apply(v, o):
            o.copy_(torch.tensor(np.asarray(op.apply(v.numpy().reshape(slab.n_nodes, nf))).reshape(-1)))
            complete(o)

        diag = torch.tensor(np.asarray(op.assemble().diagonal()).copy())
        complete(diag)
        dinv = 1.0 / diag

        def precond(v, o):
            o.copy_(dinv * v)

        b = torch.tensor(loc(f["x"]).reshape(-1).copy())
        x = torch.full_like(b, float("nan"))
        w = owned_weights(plan, slab.n_nodes, nf) if world > 1 else None
        its, res = distributed_fgmres(apply, precond, b, x, w, _TorchVec, m=20, rtol=1e-14, max_iters=40)
        out[rank] = (ng.copy(), x.numpy().reshape(slab.n_nodes, nf).copy(), its, res)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_distributed_fgmres_matches_single_part():
    """FGMRES over the z-slab parts (halo exchange in every apply, one
    all_reduce per Gram-Schmidt pass and per norm, shared rows counted once)
    does the single-part arithmetic up to rounding: after the same 40
    iterations (GMRES(20), one restart: the restart's true residual included)
    on 1, 2 and 3 parts, the assembled iterates agree, both copies of every
    shared row agree, and the residual FGMRES reports is the true residual
    ||b - J x|| / ||b|| of the global oracle's Jacobian."""
    from oracle.solve import Operator
    mesh, prm, f = _mesh()
    ref = Operator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"], up_star=f["up_star"],
                   u_n=f["u_n"], u_nm1=f["u_nm1"])
    J = ref.assemble().tocsr()
    b = np.asarray(f["x"]).reshape(-1)
    xs = {}
    for world in (1, 2, 3):
        mgr = mp.Manager()
        out = mgr.dict()
        mp.spawn(_fgmres_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        assert {out[r][2] for r in range(world)} == {40}
        x_glob = np.full((mesh.n_nodes, mesh.d + 1), np.nan)
        for r in range(world):
            ng, x, _, res = out[r]
            seen = ~np.isnan(x_glob[ng][:, 0])
            if seen.any():                                 # the shared plane: both parts hold the same rows
                assert np.abs(x_glob[ng][seen] - x[seen]).max() <= 1e-12 * np.abs(x).max()
            x_glob[ng] = x
            true_res = np.linalg.norm(b - J @ x_glob.reshape(-1)) / np.linalg.norm(b) if r == world - 1 else None
        assert not np.isnan(x_glob).any()
        assert abs(res - true_res) <= 1e-8 * true_res + 1e-14, (res, true_res)
        xs[world] = x_glob
    scale = np.abs(xs[1]).max()
    for world in (2, 3):
        assert np.abs(xs[world] - xs[1]).max() <= 1e-9 * scale, world


@pytest.mark.parametrize("n_parts", [2, 3, 5])
def test_owned_weights_count_every_global_row_once(n_parts):
    """The weights of the parts' dot products (owned_weights): summed over the
    parts through node_global they are 1 on every global row, so a weighted
    local dot product all-reduced over the parts is the global one."""
    from paper_2608_27423_b300 import slab_partition
    from paper_2608_27423_b300.slab import owned_weights
    mesh, prm, f = _mesh()
    nf = mesh.d + 1
    total = np.zeros((mesh.n_nodes, nf))
    rng = np.random.default_rng(3)
    a, b = rng.uniform(-1, 1, (2, mesh.n_nodes, nf))
    dot = 0.0
    for p in range(n_parts):
        _, plan = slab_partition(mesh, n_parts, p)
        ng = plan["node_global"]
        w = owned_weights(plan, len(ng), nf).numpy().reshape(len(ng), nf)
        np.add.at(total, ng, w)
        dot += float((w * a[ng] * b[ng]).sum())
    assert np.array_equal(total, np.ones_like(total))
    assert abs(dot - float((a * b).sum())) <= 1e-12 * abs(float((a * b).sum()))
