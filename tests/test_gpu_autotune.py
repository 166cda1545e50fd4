"""Launch-shape autotuner of the cell Jacobian (mf_autotune): every compiled
cells-per-block variant gives the oracle's Jacobian apply (FP64 within 1e-12,
FP32 within 1e-5), the tuner keeps the fastest measured variant, and a cache
file reproduces its choice without timing."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,m,n_z", [(2, 4, 3), (3, 2, 2)])
def test_every_variant_matches_oracle(k, m, n_z):
    from oracle.solve import Operator
    from paper_2608_27423_b300 import RotorStatorOperator, MF_FP64, MF_FP32
    mesh, prm, f = synth.make_config(d=3, k=k, m=m, n_r=2, n_s=2, n_z=n_z, nu=0.01, omega=1.0, dt=0.005, bdf=2,
                                     theta=0.3, state="smooth", seed=77)
    ref = Operator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"], up_star=f["up_star"],
                   u_n=f["u_n"], u_nm1=f["u_nm1"])
    yr = ref.apply(f["x"])
    g = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g.set_history(T(f["u_n"]), T(f["u_nm1"]))
    g.set_linearization(T(f["up_star"]), prm["theta"])
    x = T(f["x"])
    res = g.autotune()
    assert len(res["fp64"]["cells_per_block"]) == 3 and len(res["fp32"]["cells_per_block"]) == 3
    for prec, tol, name in ((MF_FP64, 1e-12, "fp64"), (MF_FP32, 1e-5, "fp32")):
        r = res[name]
        assert r["chosen"] in r["cells_per_block"] and not r["from_cache"]
        assert min(r["ms"]) > 0 and r["ms"][r["cells_per_block"].index(r["chosen"])] == min(r["ms"])
        xs = x if prec == MF_FP64 else x.float()
        for cpb in r["cells_per_block"]:
            g.set_cells_per_block(prec, cpb)
            y = torch.full_like(xs, float("nan"))
            g.apply_jacobian(xs, y, prec=prec)
            e = np.linalg.norm(y.double().cpu().numpy() - yr) / np.linalg.norm(yr)
            assert e < tol, (name, cpb, e)


def test_cache_file_reproduces_choice(tmp_path):
    from paper_2608_27423_b300 import RotorStatorOperator, MfError, MF_FP64
    mesh, prm, f = synth.make_config(d=3, k=2, m=4, n_r=2, n_s=2, n_z=3, nu=0.01, omega=1.0, dt=0.005, bdf=2,
                                     theta=0.3, state="smooth", seed=78)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    g.set_history(T(f["u_n"]), T(f["u_nm1"]))
    g.set_linearization(T(f["up_star"]), prm["theta"])
    path = str(tmp_path / "tune.txt")
    a = g.autotune(cache_path=path)
    b = g.autotune(cache_path=path)
    for name in ("fp64", "fp32"):
        assert not a[name]["from_cache"] and b[name]["from_cache"]
        assert a[name]["chosen"] == b[name]["chosen"]
    assert len(open(path).read().strip().splitlines()) == 2
    with pytest.raises(MfError):
        g.set_cells_per_block(MF_FP64, 7)
