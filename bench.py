"""Benchmark: Jacobian-apply throughput of the rotor-stator operator on B300.

Workload (default, 3d_q2): 3D rotor-stator cylinder, 131,072 Q2 hexes (m=32,
n_r=8, n_s=16, n_z=32), 4,359,940 DoFs, Re=200 (nu = 1/(400 pi), omega = 1),
BDF2, dt = 0.005, rotor at theta = 0.137, smooth low-mode linearisation
state, FP64.  One step = one full Jacobian apply y = J x (cell kernel, mortar
face kernel, Dirichlet rows) with the per-point linearisation already cached.
The working set (1.1 GB cache + vectors) exceeds the 126 MB L2.  Beside the
headline: FP32 and double-float applies, residual, linearisation set-up, the
end-to-end apply from host buffers, and (unless --no-solve) one Newton step
to 1e-8 with the FP32 and the FP64 multigrid; --batched adds the 12-instance
sweep (batched apply and batched Newton step), --transient N the BDF2 driver.

Prints one JSON line.  --impl reference times the CPU FP64 oracle instead
(matrix-free path on a bounded sample of cells and mortar cells).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Jacobian-apply DoFs/s (FP64 vs FP32) at Q2/Q3; time to 1e-8 residual per step"
FP64_NOMINAL_TFLOPS = 1.25       # B300 FP64 (non-tensor) nominal
# DRAM bytes (read + write) per cell of k_cell_jac<3,2,double,9> from one ncu capture on the 16,384-hex
# cylinder (profiles/k_cell_jac_fp64_3d_q2_mid.md: 134.740 MB + 4.888 MB); traffic scales with the cells.
TRAFFIC_BYTES_PER_CELL_Q2_3D_FP64 = (134.739968e6 + 4.887808e6) / 16384


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--workload", default="3d_q2")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--max-newton", type=int, default=20)
    ap.add_argument("--mg-levels", type=int, default=4)
    ap.add_argument("--mg-smooth", type=int, default=5,
                    help="GMRES smoothing steps per level (solve leg; 5 measured fastest on 3d_q2 and 3d_q3 among 3-8)")
    ap.add_argument("--mg-coarse-iters", type=int, default=40, help="coarsest-level GMRES dimension (solve leg)")
    ap.add_argument("--smooth-cgs", type=int, default=1, choices=[1, 2],
                    help="Gram-Schmidt passes of the smoothing GMRES (solve leg; one pass measured 4-6%% faster "
                         "than two on 3d_q2 and 3d_q3 at the same FGMRES iteration counts)")
    ap.add_argument("--batched", action="store_true", help="also time 12 uneven instances, batched vs one by one")
    ap.add_argument("--transient", type=int, default=0, help="also run this many graph-captured BDF2 time steps")
    ap.add_argument("--transient-newton", type=int, default=3, help="Newton iterations per transient step")
    ap.add_argument("--transient-krylov", type=int, default=8, help="FGMRES dimension per Newton iteration")
    ap.add_argument("--transient-rest", action="store_true",
                    help="start the transient from rest (u = 0; the blades and walls drive the flow)")
    ap.add_argument("--transient-no-eager", action="store_true", help="time only the graph-replayed steps")
    ap.add_argument("--transient-step-rtol", type=float, default=0.0,
                    help="per-step convergence control: more Newton iterations while ||R|| > this x ||R_0|| (0: off)")
    ap.add_argument("--transient-max-newton", type=int, default=8, help="Newton iterations per step at most (control)")
    ap.add_argument("--transient-oracle-slab", type=int, default=0,
                    help="compare the final state's energy terms on one z-slab of a partition into this many parts "
                         "(the middle part) with the oracle (0: off)")
    ap.add_argument("--clocks-dir", default=None, help="where the nvidia-smi clock samples are written (default: temp)")
    ap.add_argument("--solve-only", action="store_true",
                    help="profiling aid: run only the Newton-step leg on --workload and print its JSON")
    ap.add_argument("--solve-cold", action="store_true",
                    help="time each solve variant's first call (workspace allocation and graph capture included)")
    ap.add_argument("--solve-variants", default="mixed_fp32_mg,fp64_mg,mixed_fp32_mg_df64_outer",
                    help="comma list of the solve leg's variants")
    ap.add_argument("--q3-workload", default="3d_q3", help="the Q3 workload of the q3 leg")
    ap.add_argument("--no-q3", action="store_true", help="skip the Q3 leg")
    ap.add_argument("--no-tc", action="store_true", help="skip the tensor-core interpolation probe")
    ap.add_argument("--tc-only", action="store_true",
                    help="run only the tensor-core interpolation probe and print its JSON (launch order: 3 checks, "
                         "6 warm-ups, then the timed FMA, TF32 and 3xTF32 launches)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default cells per block (profiling runs: timings under ncu are not representative)")
    return ap.parse_args()


def algorithmic_flops_per_cell(d, k):
    """FP64 operations (FMA = 2) of one cell in the Jacobian kernel, counted from
    its loops: sum factorisation (interpolation, gradients, Hessians, the two
    transposed passes) and the point physics."""
    n = k + 1
    nf = d + 1
    sym = d * (d + 1) // 2
    sumfact_fma = 4 * d * nf * n + sym * d * n
    fma_pt = (nf * d * d) + d * (sym + d) + d * 2 * d + d + d * d * 2 + d * d * d + d * d
    oth_pt = d + d + d * d * 2 + d + 2 * d + 1 + d * d + 1 + d
    per_pt = 2 * (sumfact_fma + fma_pt) + oth_pt
    return per_pt * n ** d


def algorithmic_bytes_per_launch(d, k, n_cells, n_nodes, ncache, prec_bytes=8):
    """Bytes the cell kernel must move once: the per-point cache, the cell->node
    table, src read once per node, dst read+written once per node."""
    nq = (k + 1) ** d
    return n_cells * nq * (ncache * prec_bytes + 4) + n_nodes * (d + 1) * prec_bytes * 3


class ClockSampler:
    def __init__(self, out_path):
        self.path = out_path
        self.p = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.5)
        except Exception:
            self.p = None

    def stop(self, dev_index=0):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != dev_index:
                continue
            rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "samples": len(rows), "reasons": sorted(reasons)}


import synth  # noqa: E402  (seeded input generator: meshes and fields)


def build_inputs(workload):
    mesh, prm, f = synth.make_config(workload)
    return mesh, prm, f


# --------------------------------------------------------------------- ranks
def aggregate_ranks(ms_local, dofs_local, dist=None, device=None):
    """Whole-job timing over replica ranks: the slowest rank's time and the DoFs
    all ranks processed per step (each rank runs its own instance; no data-path
    collective, only this reduction of two scalars)."""
    if dist is None:
        return float(ms_local), float(dofs_local)
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    n = torch.tensor([float(dofs_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


# --------------------------------------------------------------------- solve leg
def build_levels(op, cfg, prm, n_h):
    """Multigrid levels below `op`: one polynomial level (k -> k-1) when k >= 3,
    then geometric halvings of the mesh (n_h levels in all below the finest).
    cfg: the mesh parameters d, k, m, n_r, n_s, n_z of `op`."""
    from paper_2608_27423_b300 import RotorStatorOperator
    base = dict(d=cfg["d"], k=cfg["k"], m=cfg["m"], n_r=cfg["n_r"], n_s=cfg["n_s"], n_z=cfg["n_z"])
    levels = [op]
    if cfg["k"] >= 3:
        pm = synth.rotor_stator_mesh(cfg["d"], cfg["k"] - 1, cfg["m"], cfg["n_r"], cfg["n_s"], cfg["n_z"])
        lp = RotorStatorOperator(pm, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
        op.mg_attach(lp)
        levels.append(lp)
        base = dict(base, k=cfg["k"] - 1)
    p = base
    for _ in range(n_h):
        try:
            cp, parent, child = synth.mesh.coarsen(p)
        except ValueError:
            break
        cm = synth.rotor_stator_mesh(cp["d"], cp["k"], cp["m"], cp["n_r"], cp["n_s"], cp["n_z"])
        lc = RotorStatorOperator(cm, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
        levels[-1].mg_attach(lc, parent, child)
        levels.append(lc)
        p = cp
    return levels


def solve_leg(args, op, mesh, prm, f, T, workload=None):
    """Newton + FGMRES(30) (FP64 residual, Jacobian applies and CGS2)
    preconditioned by one V-cycle of the global-coarsening multigrid (GMRES-Jacobi
    smoothing, --mg-smooth steps per level, --mg-coarse-iters on the coarsest),
    with the V-cycle's operator applies in FP32 (mixed) or FP64.
    Initial guess: u^n with p = 0 and zero wall velocity."""
    import torch
    from paper_2608_27423_b300 import MF_PC_MG, MF_FP32, MF_FP64, solver_defaults, MF_SMOOTH_ASM, MF_SMOOTH_JACOBI
    from synth.configs import CONFIGS
    d = mesh.d
    cfg = CONFIGS[workload or args.workload]
    levels = build_levels(op, cfg, prm, args.mg_levels - 1)
    u0 = np.zeros_like(f["up_star"])
    u0[:, :d] = f["u_n"]
    u0[mesh.wall.astype(bool), :d] = 0.0
    U0 = T(u0)
    res = {"levels": [f"Q{lv.k}:{lv.n_cells}" for lv in levels]}
    sols = {}
    from paper_2608_27423_b300 import MF_DF64
    wanted = set(args.solve_variants.split(","))
    for name, pcp, outer, smoother in (("mixed_fp32_mg", MF_FP32, MF_FP64, MF_SMOOTH_JACOBI),
                                       ("fp64_mg", MF_FP64, MF_FP64, MF_SMOOTH_JACOBI),
                                       ("mixed_fp32_mg_df64_outer", MF_FP32, MF_DF64, MF_SMOOTH_JACOBI),
                                       ("mixed_fp32_mg_asm", MF_FP32, MF_FP64, MF_SMOOTH_ASM)):
        if name not in wanted:
            continue
        o = solver_defaults(theta=prm["theta"], pc=MF_PC_MG, pc_precision=pcp, newton_rtol=1e-8,
                            max_newton=args.max_newton, lin_rtol=1e-2, restart=30, max_lin_iters=150,
                            mg_smooth=args.mg_smooth, mg_coarse_iters=args.mg_coarse_iters, outer_precision=outer,
                            mg_smoother=smoother, smooth_cgs_passes=args.smooth_cgs)
        # the first solve of a variant also allocates its workspaces and
        # captures its V-cycle graph; the timed one is the next, from the
        # same initial guess (as every later time step would run)
        first = None
        if not args.solve_cold:
            up = U0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            op.solve_step(up, o)
            torch.cuda.synchronize()
            first = round(time.perf_counter() - t0, 4)
        up = U0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, rep = op.solve_step(up, o)
        torch.cuda.synchronize()
        dt_s = time.perf_counter() - t0
        n_it = rep.newton_iters
        res[name] = {"status": int(st), "seconds": round(dt_s, 4), "first_solve_seconds": first, "newton_iters": n_it,
                     "lin_iters": list(rep.lin_iters[:n_it]), "fgmres_iters": int(rep.lin_iters_total),
                     "res_reduction": (rep.res_norm[n_it] / rep.res_norm[0]) if rep.res_norm[0] > 0 else None}
        print(f"solve {name}: status {st} {dt_s:.2f}s newton {n_it} "
              f"res {rep.res_norm[0]:.3e} -> {rep.res_norm[n_it]:.3e}", file=sys.stderr, flush=True)
        sols[name] = up
    if "fp64_mg" not in sols or "mixed_fp32_mg" not in sols:
        return res
    a, b = sols["fp64_mg"], sols["mixed_fp32_mg"]
    va, vb = a[:, :d], b[:, :d]
    pa, pb = a[:, d] - a[:, d].mean(), b[:, d] - b[:, d].mean()
    res["rel_velocity_diff_mixed_vs_fp64"] = float((va - vb).norm() / va.norm())
    res["rel_pressure_diff_mixed_vs_fp64_mean_removed"] = float((pa - pb).norm() / pa.norm())
    if res["mixed_fp32_mg"]["seconds"] > 0:
        res["speedup_mixed_vs_fp64"] = res["fp64_mg"]["seconds"] / res["mixed_fp32_mg"]["seconds"]
    return res


# --------------------------------------------------------------------- transient leg
def transient_leg(args, op, mesh, prm, f, T):
    """BDF2 time steps with the rotor turning at omega (remap every step), each
    step a fixed number of Newton iterations x FGMRES(m) (default 3 x 8)
    preconditioned by the FP32 multigrid V-cycle; the step is captured once as
    a CUDA graph and replayed.  Reports
    the time per step (graph vs eager), DoFs/s over the steps, the histories
    of kinetic energy, viscous dissipation, impeller torque and wall power,
    and the per-step residual reductions."""
    import torch
    from paper_2608_27423_b300 import MF_PC_MG, MF_FP32, solver_defaults
    from synth.configs import CONFIGS
    d = mesh.d
    cfg = CONFIGS[args.workload]
    if op.__dict__.get("_coarse") is None:
        build_levels(op, cfg, prm, args.mg_levels - 1)
    u0 = np.zeros_like(f["up_star"])
    if not args.transient_rest:
        u0[:, :d] = f["u_n"]
        u0[mesh.wall.astype(bool), :d] = 0.0
    o = solver_defaults(pc=MF_PC_MG, pc_precision=MF_FP32, mg_smooth=4, mg_coarse_iters=40,
                        step_rtol=args.transient_step_rtol, max_newton=args.transient_max_newton)
    nn, nk = args.transient_newton, args.transient_krylov
    out = {"steps": args.transient, "newton_per_step": nn, "fgmres_per_newton": nk,
           "start": "rest" if args.transient_rest else "smooth random u^n (walls zero)",
           "step_rtol": args.transient_step_rtol, "max_newton_per_step": args.transient_max_newton}
    modes = (("graph", True),) if args.transient_no_eager else (("graph", True), ("eager", False))
    for label, graph in modes:
        un, unm1 = T(u0), T(u0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rec = op.run_transient(un, unm1, args.transient, prm["theta"], newton_iters=nn, krylov_iters=nk, opts=o,
                               use_graph=graph)
        torch.cuda.synchronize()
        dt_s = time.perf_counter() - t0
        out[label] = {"seconds": round(dt_s, 4), "ms_per_step": 1e3 * dt_s / args.transient,
                      "dofs_steps_per_s": op.n_dofs * args.transient / dt_s}
        if graph:
            for key in ("kinetic_energy", "dissipation_sym", "torque_moving", "power"):
                out[key] = [float(x) for x in rec[key]]
            out["residual_reduction_per_step"] = [float(x) for x in rec["residual_reduction"][1:]]
            out["newton_iters_per_step"] = [int(x) for x in rec["newton_iters"][1:]]
            ke = np.asarray(rec["kinetic_energy"])
            # energy balance of each step (Section 4.5.2): numerical dissipation rate = wall power -
            # viscous dissipation - dE/dt (BDF1 difference of the recorded kinetic energies)
            out["numerical_dissipation_rate"] = [float(rec["power"][i] - rec["dissipation_sym"][i]
                                                       - (ke[i] - ke[i - 1]) / prm["dt"]) for i in range(1, len(ke))]
            final = (un, unm1)
    out["dofs_steps_per_s"] = out["graph"]["dofs_steps_per_s"]
    if args.transient_oracle_slab > 0:
        theta_end = prm["theta"] + args.transient * prm["omega"] * prm["dt"]
        out["oracle_slab"] = energy_on_slab(mesh, prm, final[0].cpu().numpy(), theta_end,
                                            args.transient_oracle_slab, T)
    return out


def energy_on_slab(mesh, prm, up, theta, n_parts, T):
    """Energy terms (kinetic energy, both dissipation forms) of the state `up`
    restricted to the middle z-slab of an n_parts partition, by the library
    (an operator on the slab mesh, mf_energy) and by the oracle
    (Problem.energy on the same slab), at rotor angle theta."""
    import torch
    from oracle.fem import Problem
    from paper_2608_27423_b300 import RotorStatorOperator, slab_partition
    part = n_parts // 2
    slab, plan = slab_partition(mesh, n_parts, part)
    ups = np.ascontiguousarray(up[plan["node_global"]])
    op = RotorStatorOperator(slab, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    op.set_linearization(T(ups), theta)
    e = torch.empty(3, dtype=torch.float64, device=T(ups[:1]).device)
    op.energy(T(ups), e)
    gpu = [float(v) for v in e.cpu().numpy()]
    t0 = time.perf_counter()
    ref = list(Problem(slab, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], theta).energy(ups))
    return {"parts": n_parts, "part": part, "layers": [plan["layer_begin"], plan["layer_end"]],
            "cells": slab.n_cells, "fraction_of_cells": slab.n_cells / mesh.n_cells,
            "gpu": gpu, "oracle": ref, "oracle_seconds": time.perf_counter() - t0,
            "max_rel_diff": max(abs(a - b) / abs(b) for a, b in zip(gpu, ref) if b != 0.0)}


# --------------------------------------------------------------------- batched sweep
BATCH_RE = [1, 2, 5, 10, 20, 50, 100, 200, 500, 1000, 1500, 2000]


def batched_leg(args, T, dev):
    """12 independent cylinders (Re in BATCH_RE, omega = 1, Q2, BDF2 dt = 0.005,
    rotor angle 0.137 i, m = 16 .. 32 -> ~16k .. ~131k hexes): FP64 Jacobian
    applies of all instances, one persistent launch per kernel kind against
    the instances applied one after another; then one nonlinear step of all
    12 to ||R|| <= 1e-8 ||R_0|| (mf_batch_solve_step: Newton with FGMRES(8),
    FP64 outer applies, FP32 multigrid V-cycle per instance, one Newton
    iteration of the batch as a CUDA graph), batched against sequential."""
    import torch
    from paper_2608_27423_b300 import RotorStatorOperator, BatchedOperators
    ops, xs, cfgs, fields, meshes, prms = [], [], [], [], [], []
    for i, re in enumerate(BATCH_RE):
        m = 16 + (16 * i) // 11
        m -= m % 2
        nu = 1.0 / (2.0 * np.pi * re)
        cfg = dict(d=3, k=2, m=m, n_r=2 * max(1, m // 8), n_s=2 * (m // 4), n_z=m)   # even: coarsens
        mesh, prm, f = synth.make_config(**cfg, nu=nu, omega=1.0, dt=0.005, bdf=2, theta=0.137 * i, state="smooth",
                                         seed=20260 + 10 * i)
        op = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
        op.set_history(T(f["u_n"]), T(f["u_nm1"]))
        op.set_linearization(T(f["up_star"]), prm["theta"])
        ops.append(op)
        xs.append(T(f["x"]))
        cfgs.append(cfg)
        fields.append(f)
        meshes.append(mesh)
        prms.append(prm)
    ys = [torch.empty_like(x) for x in xs]
    batch = BatchedOperators(ops)
    stream = torch.cuda.current_stream()
    steps = max(10, args.steps // 5)

    def run(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def seq():
        for op, x, y in zip(ops, xs, ys):
            op.apply_jacobian(x, y)
    ms_seq = run(seq)
    ms_bat = run(lambda: batch.apply_jacobian(xs, ys))
    dofs = sum(op.n_dofs for op in ops)
    out = {"instances": len(ops), "cells": [op.n_cells for op in ops], "total_dofs": dofs,
           "ms_one_by_one": ms_seq, "ms_batched": ms_bat, "dofs_per_s_batched": dofs / (ms_bat * 1e-3),
           "speedup": ms_seq / ms_bat}
    if args.no_solve:
        return out
    # ---- one nonlinear step of all instances
    from paper_2608_27423_b300 import MF_PC_MG, MF_FP32, solver_defaults
    for op, cfg, prm in zip(ops, cfgs, prms):
        build_levels(op, cfg, prm, args.mg_levels - 1)
    u0s = []
    for mesh, f in zip(meshes, fields):
        u0 = np.zeros_like(f["up_star"])
        u0[:, :3] = f["u_n"]
        u0[mesh.wall.astype(bool), :3] = 0.0
        u0s.append(u0)
    o = solver_defaults(pc=MF_PC_MG, pc_precision=MF_FP32, newton_rtol=1e-8, max_newton=20, mg_smooth=4,
                        mg_coarse_iters=40)
    thetas = [p["theta"] for p in prms]
    sols = {}
    for label, batched in (("batched", True), ("one_by_one", False)):
        ups = [T(u) for u in u0s]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, reps = batch.solve_step(ups, thetas, o, krylov_iters=8, batched=batched, use_graph=True)
        torch.cuda.synchronize()
        dt_s = time.perf_counter() - t0
        its = [r.newton_iters for r in reps]
        out[f"solve_{label}"] = {"status": int(st), "seconds": round(dt_s, 4), "fgmres_per_newton": 8,
                                 "newton_iters": its, "statuses": [int(r.status) for r in reps],
                                 "fallback_newton_iters": [int(r.fallback_newton_iters) for r in reps],
                                 "fallback_restarted": [int(r.fallback_restarted) for r in reps],
                                 "res_reduction": [float(r.res_norm[r.newton_iters] / r.res_norm[0]) for r in reps]}
        print(f"batched solve {label}: status {st} {dt_s:.2f}s newton {its} statuses "
              f"{[int(r.status) for r in reps]}", file=sys.stderr, flush=True)
        sols[label] = ups
    out["solve_speedup"] = out["solve_one_by_one"]["seconds"] / out["solve_batched"]["seconds"]
    out["solve_rel_diff_batched_vs_one_by_one"] = [float((a[:, :3] - b[:, :3]).norm() / b[:, :3].norm())
                                                   for a, b in zip(sols["batched"], sols["one_by_one"])]
    return out


# --------------------------------------------------------------------- end to end
def e2e_pipelined(op, x, steps, stream):
    """Milliseconds for `steps` end-to-end applies through the public API:
    step i copies its input from pinned host memory (two host / device
    buffers used in turn), applies the Jacobian and copies the result back;
    the host-to-device copy of step i+1 and the device-to-host copy of step
    i-1 run on their own streams while step i computes.  Timed with CUDA
    events from before the first copy to after the last result is on the
    host."""
    import torch
    xh = [torch.empty(x.shape, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    yh = [torch.empty(x.shape, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    for b in xh:
        b.copy_(x.cpu())
    xd = [torch.empty_like(x) for _ in range(2)]
    yd = [torch.empty_like(x) for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()
    applied = [ev(), ev()]
    copied_in = [ev(), ev()]
    copied_out = [ev(), ev()]

    def run(n):
        used = [False, False]
        for i in range(n):
            b = i % 2
            if used[b]:
                s_in.wait_event(applied[b])
            with torch.cuda.stream(s_in):
                xd[b].copy_(xh[b], non_blocking=True)
            copied_in[b].record(s_in)
            stream.wait_event(copied_in[b])
            if used[b]:
                stream.wait_event(copied_out[b])
            op.apply_jacobian(xd[b], yd[b], stream=stream)
            applied[b].record(stream)
            s_out.wait_event(applied[b])
            with torch.cuda.stream(s_out):
                yh[b].copy_(yd[b], non_blocking=True)
            copied_out[b].record(s_out)
            used[b] = True
        stream.wait_stream(s_out)
    run(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_in.wait_stream(stream)
    run(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


# --------------------------------------------------------------------- Q3 leg
def q3_leg(args, T, timed):
    """The Q3 cylinder (59,904 Q3 hexes, 6,685,924 DoFs, Re = 200, BDF2): FP64,
    FP32 and double-float Jacobian-apply DoFs/s with the autotuned launch
    shape, and (unless --no-solve) the Newton step to 1e-8 with the FP32
    p-multigrid (Q3 -> Q2 -> geometric Q2 levels) against the all-FP64
    multigrid, with the relative solution difference."""
    import torch
    from paper_2608_27423_b300 import RotorStatorOperator, MF_FP32, MF_DF64
    name = args.q3_workload
    mesh, prm, f = build_inputs(name)
    op = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    up_star = T(f["up_star"])
    op.set_history(T(f["u_n"]), T(f["u_nm1"]))
    op.set_linearization(up_star, prm["theta"])
    out = {"workload": name, "n_cells": op.n_cells, "n_dofs": op.n_dofs, "k": mesh.k}
    if not args.no_autotune:
        tune = op.autotune()
        out["cells_per_block"] = {p: tune[p]["chosen"] for p in ("fp64", "fp32")}
    x = T(f["x"])
    y = torch.empty_like(x)
    steps = max(20, args.steps // 3)
    ms = timed(lambda: op.apply_jacobian(x, y), steps, 3)
    op.profile(True)                       # kernel durations: separate, serialised pass
    timed(lambda: op.apply_jacobian(x, y), steps, 0)
    prof = op.profile_read()
    op.profile(False)
    nl, kms = prof["cell_jac_fp64"]
    out["fp64_apply_dofs_per_s"] = op.n_dofs / (ms / steps * 1e-3)
    out["fp64_cell_kernel_ms"] = kms / max(nl, 1)
    out["fp64_cell_kernel_tflops"] = algorithmic_flops_per_cell(mesh.d, mesh.k) * op.n_cells / (
        out["fp64_cell_kernel_ms"] * 1e-3) / 1e12
    x32 = x.float()
    y32 = torch.empty_like(x32)
    ms32 = timed(lambda: op.apply_jacobian(x32, y32, prec=MF_FP32), steps, 3)
    out["fp32_apply_dofs_per_s"] = op.n_dofs / (ms32 / steps * 1e-3)
    ydf = torch.empty_like(x)
    msdf = timed(lambda: op.apply_jacobian(x, ydf, prec=MF_DF64), steps, 3)
    out["df64_apply_dofs_per_s"] = op.n_dofs / (msdf / steps * 1e-3)
    out["df64_vs_fp64_rel_diff"] = float((ydf - y).norm() / y.norm())
    out["fp32_vs_fp64_rel_diff"] = float((y32.double() - y).norm() / y.norm())
    if not args.no_solve:
        out["solve_to_1e-8"] = solve_leg(args, op, mesh, prm, f, T, workload=name)
    return out


def peaks_leg(clocks_path, local):
    """Measured FMA rates of this GPU (mf_fma_peak: a hand-written kernel of
    independent FMA chains on every SM, CUDA events) in FP64 and FP32, with the
    SM clock sampled while they run."""
    from paper_2608_27423_b300 import fma_peak, MF_FP64, MF_FP32
    sampler = ClockSampler(clocks_path)
    sampler.start()
    f64, ms64 = fma_peak(MF_FP64)
    f32, ms32 = fma_peak(MF_FP32)
    clocks = sampler.stop(local)
    return {"fp64_tflops": f64, "fp32_tflops": f32, "fp64_probe_ms": ms64, "fp32_probe_ms": ms32,
            "fp64_nominal_tflops": FP64_NOMINAL_TFLOPS, "clocks": clocks,
            "how": "mf_fma_peak: 8 independent FMA chains per thread, 2048 threads per SM on every SM, "
                   "2 warm-up + 5 timed launches (CUDA events)"}


# --------------------------------------------------------------------- tensor-core measurement
def tc_leg(args):
    """Interpolation stage of the Q2 cell kernel (nodal values of 4 fields ->
    values + first derivatives at 27 Gauss points) as a compute-only probe
    (mf_contract_probe), one tile of 32 cells per CTA on every SM, repeated:
    FP32 FMA sum factorisation against tcgen05 TF32 and 3xTF32 dense Kronecker
    products.  Reports cells/s, the time the stage would take for the 3d_q2
    cylinder at that rate, and each variant's deviation from the FMA result."""
    import torch
    from paper_2608_27423_b300 import contract_probe
    # the tensor-core kernel runs one CTA (4 warps) per SM; the FMA kernel gets
    # 8 CTAs per SM (32 warps) for the same total work
    launch = {0: (148 * 8, 512), 1: (148, 4096), 2: (148, 4096)}
    g = torch.Generator(device="cuda").manual_seed(7)
    u = torch.rand((148 * 8, 27, 4, 32), generator=g, device="cuda", dtype=torch.float32) * 2 - 1
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    outs = {v: torch.empty((148, 108, 4, 32), dtype=torch.float32, device="cuda") for v in (0, 1, 2)}
    sums = torch.empty((148 * 8, 4, 32), dtype=torch.float32, device="cuda")
    res = {"launch_blocks_reps": launch, "cells_per_tile": 32, "fields": 4, "outputs_per_field": 108}
    names = {0: "fp32_fma_sum_factorised", 1: "tcgen05_tf32", 2: "tcgen05_3xtf32"}
    for v in (0, 1, 2):
        contract_probe(v, u[:148], outs[v], reps=1, err=err)
    for v in (0, 1, 2):                     # warm-up: every variant twice, then one timed launch of each
        blocks, reps = launch[v]
        for _ in range(2):
            contract_probe(v, u[:blocks], sums[:blocks], reps=reps, err=err)
    torch.cuda.synchronize()
    for v in (0, 1, 2):
        blocks, reps = launch[v]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        contract_probe(v, u[:blocks], sums[:blocks], reps=reps, err=err)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        cells = blocks * 32 * reps
        macs = {0: 729, 1: 2916, 2: 3 * 2916}[v] * 4      # useful multiply-adds per cell (4 fields)
        res[names[v]] = {"ms": ms, "cells_per_s": cells / (ms * 1e-3),
                         "us_for_131072_cells": 131072 / (cells / (ms * 1e-3)) * 1e6,
                         "useful_tflops": 2 * macs * cells / (ms * 1e-3) / 1e12,
                         "max_rel_diff_vs_fma": float((outs[v] - outs[0]).abs().max() / outs[0].abs().max())}
    res["tensor_core_error_flag"] = int(err.item())
    return res


# --------------------------------------------------------------------- CPU oracle
def cpu_oracle_rate(mesh, prm, f, seconds):
    """Oracle matrix-free Jacobian apply on a bounded sample (cells and mortar
    cells of the first z-layers), scaled to whole-operator DoFs/s."""
    from oracle.fem import Problem
    from oracle.mortar import Mortar
    prob = Problem(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"])
    prob.set_history(f["u_n"], f["u_nm1"])
    d = mesh.d
    cmask = np.zeros((mesh.n_nodes, d + 1), bool)
    cmask[mesh.wall.astype(bool), :d] = True
    xc = np.where(cmask, 0.0, f["x"])
    nc = mesh.n_cells
    # volume: grow the sample until the time budget is used
    t_vol, cells_done, chunk = 0.0, 0, 512
    out = np.zeros((mesh.n_nodes, d + 1))
    while t_vol < 0.8 * seconds and cells_done < nc:
        cl = np.arange(cells_done, min(nc, cells_done + chunk))
        t0 = time.perf_counter()
        prob.volume_apply(f["up_star"], xc, cl=cl, out=out)
        t_vol += time.perf_counter() - t0
        cells_done += len(cl)
    # mortar: one z-layer of mortar cells (whole mortar in 2D); its set-up is the counterpart of the GPU's
    # set_linearization and is not timed, like the GPU's
    mt = _layer_mortar(prob, mesh, 0) if mesh.d == 3 else Mortar(prob)
    t0 = time.perf_counter()
    mt.apply(xc, out=out)
    t_mort = time.perf_counter() - t0
    n_layers = mesh.n_z
    t_full = t_vol * nc / cells_done + t_mort * n_layers
    rate = mesh.n_dofs / t_full
    sample = (f"volume apply on {cells_done} of {nc} cells ({t_vol:.1f} s) + mortar apply on 1 of "
              f"{n_layers} z-layers ({t_mort:.2f} s; its set-up untimed), scaled to the whole operator")
    return rate, sample, t_full


def _layer_mortar(prob, mesh, layer):
    """The oracle's mortar of one z-layer of a 3D mesh (the same code path as a
    whole-mesh Mortar with n_z = 1), built on `prob`; prob.mesh is restored."""
    from oracle.mortar import Mortar

    class OneLayer:
        pass
    m1 = OneLayer()
    for key in ("d", "k", "x0", "cells", "cell_side", "node_side", "wall", "R", "n_R", "phi0"):
        setattr(m1, key, getattr(mesh, key))
    m1.n_z, m1.H = 1, mesh.H / mesh.n_z
    m1.iface_rotor = mesh.iface_rotor[layer:layer + 1]
    m1.iface_stator = mesh.iface_stator[layer:layer + 1]
    vol_mesh, prob.mesh = prob.mesh, m1
    try:
        mt = Mortar.__new__(Mortar)
        Mortar.__init__(mt, prob)
    finally:
        prob.mesh = vol_mesh
    return mt


_ORACLE_STATE = {}      # per worker process: workload -> (mesh, prm, fields, oracle problem, x, out, mortar s)
_WORKLOAD_SIZES = {}    # parent process: workload -> (n_cells, n_z, d, n_dofs)


def _oracle_state(name, layer):
    """The worker's oracle set-up for `name`, built once per process: mesh and
    fields, the volume problem, the test vector with zero wall velocities, and
    the time to build and apply the mortar of z-layer `layer` (measured once)."""
    if name not in _ORACLE_STATE:
        mesh, prm, f = synth.make_config(name)
        from oracle.fem import Problem
        from oracle.mortar import Mortar
        prob = Problem(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"])
        prob.set_history(f["u_n"], f["u_nm1"])
        d = mesh.d
        xc = f["x"].copy()
        xc[mesh.wall.astype(bool), :d] = 0.0
        out = np.zeros((mesh.n_nodes, d + 1))
        t_mort = 0.0
        if d == 2:                      # one interface ring: the whole mortar (set-up untimed, like the GPU's)
            mt = Mortar(prob)
            t0 = time.perf_counter()
            mt.apply(xc, out=out)
            t_mort = time.perf_counter() - t0
        elif layer is not None:
            mt = _layer_mortar(prob, mesh, layer)    # set-up of the layer's mortar points: untimed, like the GPU's
            t0 = time.perf_counter()
            mt.apply(xc, out=out)
            t_mort = time.perf_counter() - t0
        _ORACLE_STATE[name] = (mesh, prm, f, prob, xc, out, t_mort)
    return _ORACLE_STATE[name]


def _oracle_worker(job):
    """One host process of the all-cores oracle timing: the oracle's
    matrix-free volume apply on cells from [lo, hi) for about `budget`
    seconds (one BLAS thread, from the environment the process was spawned
    with).  Returns (cells done, volume seconds, mortar seconds per layer)."""
    name, lo, hi, layer, budget = job
    mesh, prm, f, prob, xc, out, t_mort = _oracle_state(name, layer)
    t_vol, done = 0.0, lo
    while t_vol < budget and done < hi:
        cl = np.arange(done, min(hi, done + 64))
        t0 = time.perf_counter()
        prob.volume_apply(f["up_star"], xc, cl=cl, out=out)
        t_vol += time.perf_counter() - t0
        done += len(cl)
    return done - lo, t_vol, t_mort


def oracle_pool(procs=None):
    """A pool of spawned oracle processes (one per core, at most 32 and at most
    one per 3 GB of free host memory), each with one BLAS thread."""
    import concurrent.futures as cf
    import multiprocessing as mp
    if not procs:
        procs = min(os.cpu_count() or 1, 32)
        try:
            import psutil
            procs = max(1, min(procs, int(psutil.virtual_memory().available // (3 << 30))))
        except Exception:
            pass
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})          # read by numpy as each worker starts
    try:
        ex = cf.ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn"))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return ex, procs


def cpu_oracle_rate_all_cores(name, seconds, pool=None):
    """The oracle's matrix-free apply on the host cores: every process of the
    pool applies the volume terms to its own contiguous slice of cells for
    about `seconds` (the first call per process also builds its workload and
    times one z-layer's mortar).  Aggregate rate = processes x (cells / volume
    seconds, summed over processes); whole-operator time = all cells at that
    rate + the z-layers' mortar work spread over the processes."""
    own = pool is None
    ex, procs = oracle_pool() if own else pool
    try:
        if name not in _WORKLOAD_SIZES:
            mesh = synth.make_config(name)[0]
            _WORKLOAD_SIZES[name] = (mesh.n_cells, mesh.n_z, mesh.d, mesh.n_dofs)
        nc, n_z, d, n_dofs = _WORKLOAD_SIZES[name]
        edges = np.linspace(0, nc, procs + 1).astype(int)
        jobs = [(name, int(edges[i]), int(edges[i + 1]), i % n_z, seconds) for i in range(procs)]
        res = list(ex.map(_oracle_worker, jobs))
    finally:
        if own:
            ex.shutdown()
    cells = sum(r[0] for r in res)
    t_sum = sum(r[1] for r in res)
    rate_cells = procs * cells / t_sum
    t_layer = float(np.mean([r[2] for r in res]))
    t_full = nc / rate_cells + -(-n_z // procs) * t_layer
    sample = (f"{procs} processes x 1 thread: volume apply on {cells} of {nc} cells ({t_sum:.1f} process-seconds), "
              f"mortar apply of one z-layer per process ({t_layer:.3f} s; its set-up untimed), scaled to the whole operator")
    return n_dofs / t_full, sample, procs


def cpu_model():
    """The host CPU's model string (/proc/cpuinfo) and logical core count."""
    name = "unknown"
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.startswith("model name"):
                    name = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"model": name, "logical_cores": os.cpu_count()}


def cpu_oracle_2d():
    """The oracle's two evaluation paths on the whole 2D workload (576 + 768 Q2
    quads): (A) element matrices assembled to CSR, then SpMV; (B) the
    matrix-free per-point apply.  Returns DoFs/s of each (median of 5, B of 3)
    and the assembly time."""
    from oracle.solve import Operator
    mesh, prm, f = synth.make_config("2d_q2")
    op = Operator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"], up_star=f["up_star"],
                  u_n=f["u_n"], u_nm1=f["u_nm1"])
    tb = []
    for _ in range(3):
        t0 = time.perf_counter()
        op.apply(f["x"])
        tb.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    A = op.assemble().tocsr()
    t_asm = time.perf_counter() - t0
    xv = f["x"].ravel()
    ta = []
    for _ in range(5):
        t0 = time.perf_counter()
        A @ xv
        ta.append(time.perf_counter() - t0)
    return {"workload": "2d_q2", "n_dofs": mesh.n_dofs, "path_A_csr_spmv_dofs_per_s": mesh.n_dofs / np.median(ta),
            "path_A_assembly_s": t_asm, "path_B_matrix_free_dofs_per_s": mesh.n_dofs / np.median(tb)}


def cpu_cores_used():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([1] + [i.get("num_threads", 1) for i in info if i.get("user_api") == "blas"])
    except Exception:
        return 1


# --------------------------------------------------------------------- main
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return main_reference(args, rank, world)
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2608_27423_b300 import RotorStatorOperator, MF_FP32, MF_FP64, solver_defaults, MF_PC_JACOBI, \
        MF_PC_CHEBYSHEV
    from paper_2608_27423_b300 import build as _b
    if args.tc_only:
        print(json.dumps({"interpolation_tensor_cores": tc_leg(args)}), flush=True)
        return
    mesh, prm, f = build_inputs(args.workload)
    dev = torch.device("cuda", local)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    op = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    up_star = T(f["up_star"])
    op.set_history(T(f["u_n"]), T(f["u_nm1"]) if f["u_nm1"] is not None else None)
    op.set_linearization(up_star, prm["theta"])
    if args.solve_only:
        if not args.no_autotune:
            op.autotune()
        print(json.dumps({"workload": args.workload, "solve": solve_leg(args, op, mesh, prm, f, T)}), flush=True)
        return
    x = T(f["x"])
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    n_dofs = op.n_dofs
    d, k = mesh.d, mesh.k
    # launch shape of the cell Jacobian picked by measurement (cells per block, FP64 and FP32)
    default_tune = {"fp64": {"cells_per_block": [], "ms": [], "chosen": 9 if k == 2 else 4, "from_cache": False},
                    "fp32": {"cells_per_block": [], "ms": [], "chosen": 32 if d == 3 and k <= 3 else
                             (9 if k == 2 else 4), "from_cache": False}}
    if args.no_autotune:
        tune = default_tune
    else:
        try:
            tune = op.autotune()
        except Exception as exc:         # keep the defaults and the bench line
            tune = dict(default_tune, error=repr(exc))

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # ---- FP64 apply: the headline
    import tempfile
    clocks_dir = args.clocks_dir or tempfile.gettempdir()
    sampler = ClockSampler(os.path.join(clocks_dir, f"clocks_rank{rank}.csv"))
    for _ in range(args.warmup):
        op.apply_jacobian(x, y)
    torch.cuda.synchronize()
    sampler.start()
    ms = timed(lambda: op.apply_jacobian(x, y), args.steps, 0)
    # per-kernel CUDA-event durations in a separate pass (profiling serialises
    # the apply's mortar kernel behind the cell kernel so that each is timed alone)
    op.profile(True)
    timed(lambda: op.apply_jacobian(x, y), min(args.steps, 100), 0)
    prof = op.profile_read()
    op.profile(False)
    clocks = sampler.stop(local)
    t_max, dofs_all = aggregate_ranks(ms, n_dofs, dist, dev)
    ms_step = t_max / args.steps
    value = dofs_all / (ms_step * 1e-3)

    # measured FMA peaks of this GPU (the ALU roofline's denominators)
    try:
        peaks = peaks_leg(os.path.join(clocks_dir, f"clocks_peaks_rank{rank}.csv"), local)
    except Exception as exc:
        peaks = {"error": repr(exc)}
    fp64_peak = peaks.get("fp64_tflops") or FP64_NOMINAL_TFLOPS
    peak_source = ("measured in this run: mf_fma_peak FP64 FMA chains (nominal 1.25 TFLOP/s beside it)"
                   if peaks.get("fp64_tflops") else "recipe nominal FP64 1.25 TFLOP/s (probe failed)")

    # dominant kernel roofline (FP64 cell Jacobian, bound by the FP64 pipe)
    nl, kms = prof["cell_jac_fp64"]
    k_ms = kms / max(nl, 1)
    flops = algorithmic_flops_per_cell(d, k) * op.n_cells
    ncache = (d * d + 1 + d * (d + 1) // 2 + d + d + d * d + d + 1)
    byts = algorithmic_bytes_per_launch(d, k, op.n_cells, op.n_nodes, ncache)
    achieved_tf = flops / (k_ms * 1e-3) / 1e12
    traffic = (TRAFFIC_BYTES_PER_CELL_Q2_3D_FP64 * op.n_cells
               if (d, k) == (3, 2) and tune["fp64"]["chosen"] == 9 else None)
    roofline = {"bound": "alu", "achieved": round(achieved_tf, 4), "peak": round(fp64_peak, 4),
                "unit": "TFLOP/s", "frac": round(achieved_tf / fp64_peak, 4), "traffic": traffic,
                "kernel": f"k_cell_jac<{d},{k},double,{tune['fp64']['chosen']}>", "kernel_ms": round(k_ms, 4),
                "flops_per_launch": flops, "peak_source": peak_source,
                "frac_of_nominal": round(achieved_tf / FP64_NOMINAL_TFLOPS, 4),
                "hbm": {"achieved_gbs": round(byts / (k_ms * 1e-3) / 1e9, 1),
                        "algorithmic_bytes": byts}}
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        pk = json.load(open(peaks_path))
        roofline["hbm"]["peak_gbs"] = pk.get("hbm_gbs")
        roofline["hbm"]["frac"] = round(roofline["hbm"]["achieved_gbs"] / pk["hbm_gbs"], 4)
    shares = {kk: {"launches": v[0], "ms": round(v[1], 3)} for kk, v in prof.items() if v[0]}

    extra = {"autotune": tune, "peaks": peaks}
    # ---- FP32 apply
    x32 = x.float()
    y32 = torch.empty_like(x32)
    ms32 = timed(lambda: op.apply_jacobian(x32, y32, prec=MF_FP32), args.steps, 3)
    extra["fp32_apply_dofs_per_s"] = n_dofs / (ms32 / args.steps * 1e-3)
    # ---- FP64-accurate apply in double-float arithmetic on the FP32 pipes
    from paper_2608_27423_b300 import MF_DF64
    ydf = torch.empty_like(x)
    msdf = timed(lambda: op.apply_jacobian(x, ydf, prec=MF_DF64), args.steps, 3)
    extra["df64_apply_dofs_per_s"] = n_dofs / (msdf / args.steps * 1e-3)
    extra["df64_vs_fp64_rel_diff"] = float((ydf - y).norm() / y.norm())
    # ---- residual and linearisation set-up
    r = torch.empty_like(x)
    msr = timed(lambda: op.residual(up_star, r), max(10, args.steps // 10), 2)
    extra["residual_dofs_per_s"] = n_dofs / (msr / max(10, args.steps // 10) * 1e-3)
    msl = timed(lambda: op.set_linearization(up_star, prm["theta"]), 10, 1)
    extra["set_linearization_ms"] = msl / 10

    # ---- e2e: host buffers, H2D + apply + D2H per step
    xh = torch.empty(x.shape, dtype=torch.float64, pin_memory=True)
    xh.copy_(x.cpu())
    yh = torch.empty(x.shape, dtype=torch.float64, pin_memory=True)
    xd = torch.empty_like(x)

    def e2e_step():
        xd.copy_(xh, non_blocking=True)
        op.apply_jacobian(xd, y)
        yh.copy_(y, non_blocking=True)
    e2e_steps = max(20, args.steps // 5)
    ms_e2e = timed(e2e_step, e2e_steps, 2)
    serial = n_dofs * world / (ms_e2e / e2e_steps * 1e-3)
    ms_pipe = e2e_pipelined(op, x, e2e_steps, stream)
    e2e = {"value": n_dofs * world / (ms_pipe / e2e_steps * 1e-3), "unit": "DoFs/s",
           "h2d_bytes_per_step": int(xh.numel() * 8), "d2h_bytes_per_step": int(yh.numel() * 8),
           "mode": "every step copies its input host->device and its result device->host (pinned host buffers); "
                   "copies run on two copy streams, overlapped with the neighbouring steps' applies",
           "serial_value": serial}

    # ---- nonlinear step to 1e-8: all-FP64 vs mixed precision (same algorithm)
    # optional legs: a failure is reported in the line instead of losing the line
    def leg(key, fn):
        try:
            extra[key] = fn()
        except Exception as exc:
            extra[key] = {"error": repr(exc)}
            print(f"{key} failed: {exc!r}", file=sys.stderr, flush=True)

    if not args.no_solve:
        leg("solve_to_1e-8", lambda: solve_leg(args, op, mesh, prm, f, T))
        op.set_linearization(up_star, prm["theta"])
    if not args.no_q3:
        leg("q3", lambda: q3_leg(args, T, timed))
    if not args.no_tc:
        leg("interpolation_tensor_cores", lambda: tc_leg(args))
    if args.batched:
        leg("batched_12", lambda: batched_leg(args, T, dev))
    if args.transient > 0:
        leg("transient", lambda: transient_leg(args, op, mesh, prm, f, T))

    line = {"metric": METRIC, "value": value, "unit": "DoFs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {d}D rotor-stator, {op.n_cells} Q{k} cells, "
                                   f"{n_dofs} DoFs, nu={prm['nu']:.4g}, omega={prm['omega']}, BDF{prm['bdf']} "
                                   f"dt={prm['dt']}, theta={prm['theta']}, FP64 Jacobian apply",
                       "n_cells": op.n_cells, "n_dofs": n_dofs, "k": k, "d": d,
                       "l2": "inputs larger than L2 (per-point cache ~1.1 GB)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": roofline, "kernel_shares": shares, "gpu_launches": 3 * args.steps,
            "e2e": e2e, "clocks": clocks, **extra}
    if rank == 0 and world == 1 and not args.no_cpu:
        rate1, sample1, _ = cpu_oracle_rate(mesh, prm, f, args.cpu_seconds)
        try:
            pool = oracle_pool()
            try:
                cpu_oracle_rate_all_cores(args.workload, 0.5, pool)        # workers build the workload
                rate, sample, procs = cpu_oracle_rate_all_cores(args.workload, args.cpu_seconds, pool)
            finally:
                pool[0].shutdown()
        except Exception as exc:     # keep the bench line: report the single-process timing
            rate, sample, procs = rate1, f"{sample1} (all-cores timing failed: {exc!r})", cpu_cores_used()
        line["cpu_baseline"] = {"value": rate, "unit": "DoFs/s", "cores": procs, "kind": "oracle",
                                "sample": sample,
                                "single_process": {"value": rate1, "threads": cpu_cores_used(), "sample": sample1},
                                "oracle_2d": cpu_oracle_2d(), "cpu_model": cpu_model()}
        if not args.no_q3:
            try:       # config 3: the Q3 cylinder, one process on a bounded sample
                mq, pq, fq = build_inputs(args.q3_workload)
                rq, sq, _ = cpu_oracle_rate(mq, pq, fq, max(4.0, args.cpu_seconds / 2))
                line["cpu_baseline"]["single_process_q3"] = {"workload": args.q3_workload, "value": rq,
                                                             "threads": cpu_cores_used(), "sample": sq}
            except Exception as exc:
                line["cpu_baseline"]["single_process_q3"] = {"error": repr(exc)}
    if rank == 0:
        print(json.dumps(line, default=float), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main_reference(args, rank, world):
    if rank != 0:
        return
    mesh, prm, f = build_inputs(args.workload)
    # one pool for the whole run: the workers build the workload once (first warm-up step), then every step
    # is a bounded sample; the run stays within a few minutes for any --steps
    budget = max(0.2, 120.0 / max(1, args.steps + args.warmup))
    rates = []
    sample = ""
    pool = oracle_pool()
    cores = pool[1]
    try:
        for i in range(max(1, args.warmup) + args.steps):
            rate, sample, cores = cpu_oracle_rate_all_cores(args.workload, budget, pool)
            if i >= max(1, args.warmup):
                rates.append(rate)
    finally:
        pool[0].shutdown()
    value = float(np.median(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DoFs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mesh.n_dofs / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: CPU FP64 oracle, matrix-free path", "n_dofs": mesh.n_dofs},
            "cpu_baseline": {"value": value, "unit": "DoFs/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "DoFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
