"""Parity at the full workload sizes (2d_q2, 3d_q2: 137k Q2 hexes, 3d_q3: 58k Q3
hexes) in the launch configuration the benchmark times: every output row of a
random sample of nodes (plus whole interface cells on both sides) is computed
by the oracle from all cells and mortar cells that touch it."""
import numpy as np
import pytest

import synth
from oracle.fem import Problem
from oracle.mortar import Mortar

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rows_oracle(mesh, prm, f, nodes, vec, kind):
    prob = Problem(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"])
    prob.set_history(f["u_n"], f["u_nm1"])
    d = mesh.d
    cells = np.asarray(mesh.cells)
    adj = np.where(np.isin(cells, nodes).any(1))[0]
    wall = mesh.wall.astype(bool)
    cmask = np.zeros((mesh.n_nodes, d + 1), bool)
    cmask[wall, :d] = True
    src = np.where(cmask, 0.0, vec) if kind == "jac" else vec
    if kind == "jac":
        out = prob.volume_apply(f["up_star"], src, cl=adj)
    else:
        out = prob.volume_residual(src, cl=adj)
    adjset = set(adj.tolist())
    layers = [lz for lz in range(mesh.n_z)
              if adjset & set(mesh.iface_rotor[lz].tolist()) or adjset & set(mesh.iface_stator[lz].tolist())]
    if layers:
        mt = Mortar(prob, layers=layers)
        recs = [r for r in mt.recs if r["cells"][0] in adjset or r["cells"][1] in adjset]
        mt.apply(src, out=out, recs=recs)
    if kind == "jac":
        out[cmask] = vec[cmask]
    else:
        out[cmask] = vec[cmask]
    return out[nodes]


def _sample_nodes(mesh, rng, n_random=40, n_iface=3):
    nodes = set(rng.choice(mesh.n_nodes, n_random, replace=False).tolist())
    cells = np.asarray(mesh.cells)
    for _ in range(n_iface):
        lz = rng.integers(mesh.n_z)
        j = rng.integers(mesh.n_R)
        nodes |= set(cells[mesh.iface_rotor[lz, j]].tolist()) | set(cells[mesh.iface_stator[lz, j]].tolist())
    return np.array(sorted(nodes))


@pytest.mark.parametrize("name", ["2d_q2", "3d_q2", "3d_q3"])
def test_fullsize_sampled_rows(name):
    from paper_2608_27423_b300 import RotorStatorOperator, MF_FP32
    mesh, prm, f = synth.make_config(name)
    g = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g.set_history(T(f["u_n"]), T(f["u_nm1"]) if f["u_nm1"] is not None else None)
    g.set_linearization(T(f["up_star"]), prm["theta"])
    x = T(f["x"])
    y = torch.empty_like(x)
    g.apply_jacobian(x, y)
    y32 = torch.empty_like(x, dtype=torch.float32)
    g.apply_jacobian(x.float(), y32, prec=MF_FP32)
    y32l = None
    if mesh.d == 3 and mesh.k <= 3:                 # default: one cell per lane; also the per-point kernel
        g.set_cells_per_block(MF_FP32, 9 if mesh.k == 2 else 4)
        y32l = torch.empty_like(x, dtype=torch.float32)
        g.apply_jacobian(x.float(), y32l, prec=MF_FP32)
        g.set_cells_per_block(MF_FP32, 0)
    from paper_2608_27423_b300 import MF_DF64
    ydf = torch.empty_like(x)
    g.apply_jacobian(x, ydf, prec=MF_DF64)
    r = torch.empty_like(x)
    g.residual(T(f["up_star"]), r)
    rng = np.random.default_rng(7)
    nodes = _sample_nodes(mesh, rng)
    yj = _rows_oracle(mesh, prm, f, nodes, f["x"], "jac")
    yr = _rows_oracle(mesh, prm, f, nodes, f["up_star"], "res")
    y = y.cpu().numpy()[nodes]
    ydf = ydf.cpu().numpy()[nodes]
    y32 = y32.double().cpu().numpy()[nodes]
    r = r.cpu().numpy()[nodes]
    checks = [(ydf, yj, 1e-12), (y, yj, 1e-12), (y32, yj, 1e-5), (r, yr, 1e-12)]
    if y32l is not None:
        checks.append((y32l.double().cpu().numpy()[nodes], yj, 1e-5))
    # normwise and element-wise (max-entry error / max entry) on the sampled rows
    for got, ref, tol in checks:
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    # properties at any size: finite everywhere, wall rows copied
    assert np.isfinite(y).all()
