"""Batched apply of several independent instances in one persistent launch per
kernel kind equals the instances' own applies (same kernels, same arithmetic;
only the atomic summation order may differ)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _instances(specs):
    from paper_2608_27423_b300 import RotorStatorOperator
    ops, xs = [], []
    for i, (m, n_r, n_s, n_z, re, theta) in enumerate(specs):
        nu = 1.0 / (2.0 * np.pi * re)
        mesh, prm, f = synth.make_config(d=3, k=2, m=m, n_r=n_r, n_s=n_s, n_z=n_z, nu=nu, omega=1.0, dt=0.005,
                                         bdf=2, theta=theta, seed=100 + 10 * i)
        op = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
        T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        op.set_history(T(f["u_n"]), T(f["u_nm1"]))
        op.set_linearization(T(f["up_star"]), prm["theta"])
        ops.append(op)
        xs.append(T(f["x"]))
    return ops, xs


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_apply_equals_individual_applies(prec):
    from paper_2608_27423_b300 import BatchedOperators, MF_FP64, MF_FP32
    specs = [(4, 1, 2, 3, 1.0, 0.0), (6, 2, 2, 4, 200.0, 0.137), (2, 1, 1, 2, 2000.0, 0.274), (8, 2, 4, 2, 50.0, 1.1)]
    ops, xs = _instances(specs)
    p = MF_FP64 if prec == "fp64" else MF_FP32
    if p == MF_FP32:
        xs = [x.float() for x in xs]
    ys_ref = [torch.empty_like(x) for x in xs]
    for op, x, y in zip(ops, xs, ys_ref):
        op.apply_jacobian(x, y, prec=p)
    batch = BatchedOperators(ops)
    for rep in range(2):
        ys = [torch.full_like(x, float("nan")) for x in xs]
        batch.apply_jacobian(xs, ys, prec=p)
        torch.cuda.synchronize()
        for y, yr in zip(ys, ys_ref):
            tol = 1e-13 if p == MF_FP64 else 1e-5
            assert float((y - yr).norm() / yr.norm()) < tol
