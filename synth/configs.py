"""The synthetic rotor-stator workloads (mesh sizes, physics, seeds).

* ``2d_q2``: 2D disk r<0.5 (O-grid m=16, 5 rings: 576 quads) in an annulus
  0.5<r<1 (64 x 12 = 768 quads), interface rotated by 0.137 rad (non-matching),
  Q2, nu=0.01, omega=1, BDF1, dt=0.01; i.i.d. U(-1,1) state.
* ``3d_q2``: cylinder R_out=1, H=1, rotor r<0.5: m=32, n_r=8, n_s=16, n_z=32
  -> 131,072 hexes, Q2 (4.36M DoFs); Re = omega D^2/(2 pi nu) = 200 with D=1,
  omega=1; BDF2, dt=0.005; smooth low-mode state.  Coarsens uniformly three
  times (h-multigrid).
* ``3d_q3``: same cylinder, m=24, n_r=8, n_s=12, n_z=24 -> 59,904 hexes, Q3
  (6.69M DoFs); Re = 200.
* ``3d_q2_mid``: the 3d_q2 physics on m=16, n_r=4, n_s=8, n_z=16 (16,384 hexes,
  0.56M DoFs; per-point cache 124 MB) for profiling and solver checks.
* ``3d_q3_1m``: large cylinder, m=48, n_r=16, n_s=32, n_z=88 -> 1,013,760 Q3 hexes
  (110.8M DoFs), Re = 2000, BDF2 dt = 0.002, four radial blades inside the
  rotor (walls moving with it); apply throughput at scale and transient steps.
* small variants for tests.
"""
import numpy as np
from .mesh import rotor_stator_mesh

SEED = 20260

CONFIGS = {
    "2d_q2": dict(d=2, k=2, m=16, n_r=5, n_s=12, n_z=1, nu=0.01, omega=1.0, dt=0.01, bdf=1,
                  theta=0.137, state="iid"),
    "3d_q2": dict(d=3, k=2, m=32, n_r=8, n_s=16, n_z=32, nu=1.0 / (400.0 * np.pi), omega=1.0,
                  dt=0.005, bdf=2, theta=0.137, state="smooth"),
    "3d_q2_mid": dict(d=3, k=2, m=16, n_r=4, n_s=8, n_z=16, nu=1.0 / (400.0 * np.pi), omega=1.0,
                      dt=0.005, bdf=2, theta=0.137, state="smooth"),
    "3d_q3": dict(d=3, k=3, m=24, n_r=8, n_s=12, n_z=24, nu=1.0 / (400.0 * np.pi), omega=1.0,
                  dt=0.005, bdf=2, theta=0.137, state="smooth"),
    "3d_q3_1m": dict(d=3, k=3, m=48, n_r=16, n_s=32, n_z=88, nu=1.0 / (4000.0 * np.pi), omega=1.0,
                     dt=0.002, bdf=2, theta=0.137, state="smooth", blades=4),
}


def make_config(name=None, seed=SEED, **over):
    """Return (mesh, params, fields) for a named or custom workload.

    fields: up_star [N_n, d+1], u_n [N_n, d], u_nm1 [N_n, d] (or None for BDF1),
    x [N_n, d+1] test vector with zeros on wall velocity DoFs.
    """
    cfg = dict(CONFIGS[name]) if name else {}
    cfg.update(over)
    d, k = cfg["d"], cfg["k"]
    mesh = rotor_stator_mesh(d, k, cfg["m"], cfg["n_r"], cfg["n_s"], cfg.get("n_z", 1), blades=cfg.get("blades", 0))
    N = mesh.n_nodes
    if cfg.get("state", "iid") == "iid":
        up = __import__("synth.fields", fromlist=["x"]).random_nodal_field(N, d + 1, seed)
        un = __import__("synth.fields", fromlist=["x"]).random_nodal_field(N, d, seed + 1)
        unm1 = __import__("synth.fields", fromlist=["x"]).random_nodal_field(N, d, seed + 2)
    else:
        from .fields import smooth_nodal_field
        up = smooth_nodal_field(mesh.x0, d + 1, seed)
        un = smooth_nodal_field(mesh.x0, d, seed + 1)
        unm1 = smooth_nodal_field(mesh.x0, d, seed + 2)
    from .fields import random_nodal_field
    x = random_nodal_field(N, d + 1, seed + 3)
    x[mesh.wall.astype(bool), :d] = 0.0
    if cfg.get("bdf", 1) == 1:
        unm1 = None
    params = dict(nu=cfg["nu"], omega=cfg["omega"], dt=cfg["dt"], bdf=cfg["bdf"], theta=cfg["theta"])
    return mesh, params, dict(up_star=up, u_n=un, u_nm1=unm1, x=x)
