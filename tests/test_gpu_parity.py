"""GPU parity: the CUDA library against the CPU FP64 oracle on the same seeded inputs.

Bars, both checked: normwise ||y_gpu - y_oracle||_2 / ||y_oracle||_2 and
element-wise max_i |y_gpu,i - y_oracle,i| / ||y_oracle||_inf (a localised error
on the few interface rows is not diluted by the interior rows); 1e-12 for FP64
applies, residuals and diagonals; 1e-5 for FP32 applies.
"""
import numpy as np
import pytest

import synth
from tests.oracle_helpers import make_op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def rel(a, b):
    """max(normwise relative error, max-entry error / ||b||_inf)."""
    a, b = np.asarray(a), np.asarray(b)
    nw = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    ew = float(np.abs(a - b).max() / np.abs(b).max())
    return max(nw, ew)


def setup(d, k, m, n_r, n_s, n_z=1, bdf=2, theta=0.137, nu=0.05, omega=1.0, dt=0.01, state="iid", seed=11, blades=0):
    from paper_2608_27423_b300 import RotorStatorOperator
    mesh, prm, f = synth.make_config(d=d, k=k, m=m, n_r=n_r, n_s=n_s, n_z=n_z, nu=nu, omega=omega, dt=dt, bdf=bdf,
                                     theta=theta, state=state, seed=seed, blades=blades)
    op = make_op(mesh, prm, f)
    g = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    dev = torch.device("cuda")
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    g.set_history(T(f["u_n"]), T(f["u_nm1"]) if f["u_nm1"] is not None else None)
    g.set_linearization(T(f["up_star"]), prm["theta"])
    return mesh, prm, f, op, g, T


CASES = [
    dict(d=2, k=2, m=4, n_r=2, n_s=3),
    dict(d=2, k=3, m=2, n_r=2, n_s=2, bdf=1),
    dict(d=2, k=1, m=4, n_r=2, n_s=3),
    dict(d=2, k=4, m=2, n_r=1, n_s=2),
    dict(d=3, k=2, m=2, n_r=1, n_s=2, n_z=3),
    dict(d=3, k=3, m=1, n_r=1, n_s=2, n_z=2, theta=0.9),
    dict(d=3, k=1, m=2, n_r=2, n_s=2, n_z=3),
    dict(d=3, k=2, m=2, n_r=4, n_s=2, n_z=4, theta=0.7, omega=1.3, blades=4),    # blades: walls moving with the rotor
]


def cid(c):
    return f"d{c['d']}k{c['k']}" + ("blades" if c.get("blades") else "")


@pytest.mark.parametrize("c", CASES, ids=cid)
def test_jacobian_fp64_matches_oracle(c):
    mesh, prm, f, op, g, T = setup(**c)
    y_ref = op.apply(f["x"])
    y = torch.empty_like(T(f["x"]))
    g.apply_jacobian(T(f["x"]), y)
    assert rel(y.cpu().numpy(), y_ref) <= TOL64


@pytest.mark.parametrize("c", CASES, ids=cid)
def test_residual_matches_oracle(c):
    mesh, prm, f, op, g, T = setup(**c)
    up = f["up_star"] * 0.7 + 0.1
    r_ref = op.residual(up)
    r = torch.empty_like(T(up))
    g.residual(T(up), r)
    assert rel(r.cpu().numpy(), r_ref) <= TOL64


@pytest.mark.parametrize("c", CASES, ids=cid)
def test_jacobian_fp32_matches_oracle(c):
    mesh, prm, f, op, g, T = setup(**c)
    y_ref = op.apply(f["x"])
    x32 = T(f["x"]).float()
    y = torch.empty_like(x32)
    from paper_2608_27423_b300 import MF_FP32
    g.apply_jacobian(x32, y, prec=MF_FP32)
    assert rel(y.double().cpu().numpy(), y_ref) <= TOL32


@pytest.mark.parametrize("c", [c for c in CASES if c["d"] == 3], ids=cid)
def test_jacobian_fp32_lane_kernel_matches_oracle(c):
    """The one-cell-per-lane FP32 kernel (3D, k <= 3; 32 cells per block,
    ragged last block included).  On these small meshes the default FP32
    variant is the per-point kernel (test_jacobian_fp32_matches_oracle)."""
    mesh, prm, f, op, g, T = setup(**c)
    from paper_2608_27423_b300 import MF_FP32
    g.set_cells_per_block(MF_FP32, 32)
    y_ref = op.apply(f["x"])
    x32 = T(f["x"]).float()
    y = torch.full_like(x32, float("nan"))
    g.apply_jacobian(x32, y, prec=MF_FP32)
    assert rel(y.double().cpu().numpy(), y_ref) <= TOL32


@pytest.mark.parametrize("c", CASES, ids=cid)
def test_jacobian_df64_matches_oracle_at_fp64_bar(c):
    """Double-float applies (FP32 pipes) meet the FP64 bar."""
    mesh, prm, f, op, g, T = setup(**c)
    y_ref = op.apply(f["x"])
    y = torch.empty_like(T(f["x"]))
    from paper_2608_27423_b300 import MF_DF64
    g.apply_jacobian(T(f["x"]), y, prec=MF_DF64)
    assert rel(y.cpu().numpy(), y_ref) <= TOL64


@pytest.mark.parametrize("c", CASES, ids=cid)
def test_diagonal_matches_assembled(c):
    mesh, prm, f, op, g, T = setup(**c)
    dref = op.diagonal()
    dg = torch.empty_like(T(f["x"]))
    g.diagonal(dg)
    assert rel(dg.cpu().numpy(), dref) <= TOL64


@pytest.mark.parametrize("c", CASES, ids=cid)
def test_energy_matches_oracle(c):
    """mf_energy (kinetic energy, both dissipation forms) and mf_kinetic_energy."""
    mesh, prm, f, op, g, T = setup(**c)
    up = f["up_star"] * 0.7 + 0.1
    ref = np.array(op.prob.energy(up))
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    g.energy(T(up), out)
    assert np.abs(out.cpu().numpy() / ref - 1).max() <= TOL64, (out, ref)
    g.kinetic_energy(T(up), out[:1])
    assert abs(float(out[0]) / ref[0] - 1) <= TOL64


@pytest.mark.parametrize("c", CASES, ids=cid)
def test_wall_loads_match_oracle(c):
    """mf_wall_loads: default groups (stationary / moving walls) and caller groups."""
    mesh, prm, f, op, g, T = setup(**c)
    up = f["up_star"] * 0.7 + 0.1
    d = mesh.d
    out = torch.empty((2, d + 2), dtype=torch.float64, device="cuda")
    g.wall_loads(T(up), out)
    ref = op.wall_loads(up)
    assert rel(out.cpu().numpy(), ref) <= TOL64
    # three groups by position, one group (7) skipped
    x = op.prob.x
    grp = np.where(x[:, 0] > 0, 0, np.where(x[:, 1] > 0, 1, 2)).astype(np.uint8)
    grp[::7] = 7
    out3 = torch.empty((3, d + 2), dtype=torch.float64, device="cuda")
    g.wall_loads(T(up), out3, group=torch.tensor(grp, device="cuda"), n_groups=3)
    assert rel(out3.cpu().numpy(), op.wall_loads(up, group=grp, n_groups=3)) <= TOL64


def test_node_coordinates_follow_rotation():
    mesh, prm, f, op, g, T = setup(d=3, k=2, m=2, n_r=1, n_s=2, n_z=2, theta=1.3)
    x = torch.empty((mesh.n_nodes, 3), dtype=torch.float64, device="cuda")
    g.node_coords(x)
    assert np.abs(x.cpu().numpy() - op.prob.x).max() < 1e-14


@pytest.mark.parametrize("theta", [0.0, 1e-9, 2 * np.pi / 8 * 3, 2 * np.pi / 8 * 3 + 1e-11, -0.4, 7.0])
def test_mortar_angles_edge_cases(theta):
    """Conforming angles (zero-length halves), near-conforming, negative and >2pi angles."""
    mesh, prm, f, op, g, T = setup(d=2, k=2, m=2, n_r=1, n_s=2, theta=theta)
    y_ref = op.apply(f["x"])
    y = torch.empty_like(T(f["x"]))
    g.apply_jacobian(T(f["x"]), y)
    assert rel(y.cpu().numpy(), y_ref) <= TOL64


def test_apply_is_deterministic_to_roundoff():
    mesh, prm, f, op, g, T = setup(d=3, k=2, m=2, n_r=1, n_s=2, n_z=3)
    x = T(f["x"])
    y1 = torch.empty_like(x)
    y2 = torch.empty_like(x)
    g.apply_jacobian(x, y1)
    g.apply_jacobian(x, y2)
    assert float((y1 - y2).norm() / y1.norm()) < 1e-14


def test_apply_before_linearization_is_an_error():
    from paper_2608_27423_b300 import RotorStatorOperator, MfError
    mesh, prm, f = synth.make_config(d=2, k=2, m=2, n_r=1, n_s=2, nu=0.1, omega=1.0, dt=0.01, bdf=1, theta=0.1)
    g = RotorStatorOperator(mesh, 0.1, 1.0, 0.01, 1)
    x = torch.zeros(mesh.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(MfError):
        g.apply_jacobian(x, torch.empty_like(x))


@pytest.mark.parametrize("c", CASES, ids=cid)
def test_residual_with_cached_geometry_equals_recomputed(c):
    """After a cache-writing pass at the current angle the state kernel reads
    J^-1, det J w, G and c-tilde from the cache instead of recomputing them;
    the residual must not change (up to the atomic scatter's summation order)
    and must still match the oracle.  set_angle clears the cached geometry,
    so the first residual recomputes it."""
    mesh, prm, f, op, g, T = setup(**c)
    up = T(f["up_star"] * 0.7 + 0.1)
    g.set_angle(prm["theta"])
    r_fresh = torch.empty_like(up)
    g.residual(up, r_fresh)                      # geometry recomputed
    g.set_linearization(T(f["up_star"]), prm["theta"])   # same angle: writes the geometry cache
    r_cached = torch.empty_like(up)
    g.residual(up, r_cached)                     # geometry read from the cache
    a, b = r_cached.cpu().numpy(), r_fresh.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
    assert rel(a, op.residual(f["up_star"] * 0.7 + 0.1)) <= TOL64
