"""z-slab parts on the GPU (the paper's mesh decomposition, Section 3.3).
One GPU holds every part of the partition here, as separate operator
handles; the exchange between neighbours is the library's pack / add
kernels with a device-to-device copy standing in for the send (no
collective: parts that wait on one another never run as separate launches
on one GPU).  After the exchange, every part's rows of the Jacobian apply and
the residual equal the global operator's rows."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_parts", [2, 3])
def test_slab_parts_with_device_exchange_equal_global_apply(n_parts):
    from paper_2608_27423_b300 import RotorStatorOperator, slab_partition, halo_pack, halo_add
    mesh, prm, f = synth.make_config(d=3, k=2, m=4, n_r=2, n_s=2, n_z=6, nu=0.02, omega=1.0, dt=0.01, bdf=2,
                                     theta=0.41, state="smooth", seed=33)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    g.set_history(T(f["u_n"]), T(f["u_nm1"]))
    g.set_linearization(T(f["up_star"]), prm["theta"])
    y_ref = torch.empty_like(T(f["x"]))
    g.apply_jacobian(T(f["x"]), y_ref)
    up = f["up_star"] * 0.6 + 0.05
    r_ref = torch.empty_like(y_ref)
    g.residual(T(up), r_ref)
    parts = []
    for p in range(n_parts):
        slab, plan = slab_partition(mesh, n_parts, p)
        ng = plan["node_global"]
        op = RotorStatorOperator(slab, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
        op.set_history(T(f["u_n"][ng]), T(f["u_nm1"][ng]))
        op.set_linearization(T(f["up_star"][ng]), prm["theta"])
        y = torch.empty((slab.n_nodes, 4), dtype=torch.float64, device="cuda")
        op.apply_jacobian(T(f["x"][ng]), y)
        r = torch.empty_like(y)
        op.residual(T(up[ng]), r)
        dev = lambda a, t=torch.int32: torch.tensor(a, dtype=t, device="cuda")
        parts.append(dict(ng=ng, y=y, r=r, lo=dev(plan["lo"]), hi=dev(plan["hi"]),
                          lo_wall=dev(plan["lo_wall"], torch.uint8), hi_wall=dev(plan["hi_wall"], torch.uint8)))
    for key in ("y", "r"):
        # pack every shared plane first (the sends), then add what the neighbour sent
        sent = {}
        for p in range(n_parts - 1):
            a, b = parts[p], parts[p + 1]
            up_buf = torch.empty((a["hi"].numel(), 4), dtype=torch.float64, device="cuda")
            dn_buf = torch.empty((b["lo"].numel(), 4), dtype=torch.float64, device="cuda")
            halo_pack(a[key], a["hi"], up_buf)
            halo_pack(b[key], b["lo"], dn_buf)
            sent[p] = (up_buf, dn_buf)
        for p in range(n_parts - 1):
            a, b = parts[p], parts[p + 1]
            up_buf, dn_buf = sent[p]
            halo_add(a[key], a["hi"], a["hi_wall"], dn_buf)
            halo_add(b[key], b["lo"], b["lo_wall"], up_buf)
        full = (y_ref if key == "y" else r_ref).cpu().numpy()
        scale = np.abs(full).max()
        for p in parts:
            got = p[key].cpu().numpy()
            err = np.abs(got - full[p["ng"]]).max() / scale
            assert err <= 1e-12, (key, err)


def test_fgmres_with_library_vector_kernels_on_one_part():
    """The z-slab FGMRES (paper_2608_27423_b300.slab.distributed_fgmres) on a
    single part, its vector arithmetic in the library's kernels (mf_vec_*),
    the apply and diagonal of a SlabOperator: after 40 iterations of
    GMRES(20) (one restart) the residual it reports is the true residual of
    the oracle's assembled Jacobian, and the iterate equals the same
    algorithm run on the host with the oracle's apply (tests/test_slab_partition.py
    runs that one over 1, 2 and 3 gloo ranks)."""
    from oracle.solve import Operator
    from paper_2608_27423_b300 import vec_mul
    from paper_2608_27423_b300.slab import SlabOperator, LibVec, distributed_fgmres
    mesh, prm, f = synth.make_config(d=3, k=2, m=2, n_r=1, n_s=2, n_z=5, nu=0.05, omega=1.0, dt=0.01, bdf=2,
                                     theta=0.37, state="smooth", seed=31)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    so = SlabOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], 1, 0)
    so.set_history(T(f["u_n"]), T(f["u_nm1"]))
    so.set_linearization(T(f["up_star"]), prm["theta"])
    n, nf = mesh.n_nodes, mesh.d + 1
    diag = torch.empty((n, nf), dtype=torch.float64, device="cuda")
    so.diagonal(diag)
    dinv = (1.0 / diag).reshape(-1)

    def apply(v, o):
        so.apply_jacobian(v.view(n, nf), o.view(n, nf))

    def precond(v, o):
        vec_mul(dinv, v, o)

    b = T(f["x"]).reshape(-1)
    x = torch.full_like(b, float("nan"))
    its, res = distributed_fgmres(apply, precond, b, x, None, LibVec, m=20, rtol=1e-14, max_iters=40)
    assert its == 40
    ref = Operator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"], up_star=f["up_star"],
                   u_n=f["u_n"], u_nm1=f["u_nm1"])
    J = ref.assemble().tocsr()
    xh = x.cpu().numpy()
    bh = np.asarray(f["x"]).reshape(-1)
    true_res = np.linalg.norm(bh - J @ xh) / np.linalg.norm(bh)
    assert abs(res - true_res) <= 1e-7 * true_res
    # the same algorithm on the host with the oracle's apply and diagonal
    from paper_2608_27423_b300.slab import distributed_fgmres as fg
    from tests.test_slab_partition import _TorchVec
    dref = torch.tensor(np.asarray(J.diagonal()).copy())
    xr = torch.zeros(n * nf, dtype=torch.float64)
    fg(lambda v, o: o.copy_(torch.tensor(J @ v.numpy())), lambda v, o: o.copy_(v / dref),
       torch.tensor(bh.copy()), xr, None, _TorchVec, m=20, rtol=1e-14, max_iters=40)
    assert np.abs(xh - xr.numpy()).max() <= 1e-8 * np.abs(xr.numpy()).max()
