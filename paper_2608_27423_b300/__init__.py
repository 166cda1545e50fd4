"""B300 matrix-free rotor-stator operator (stabilised ALE Navier-Stokes + Nitsche/SIPG mortar).

Thin Python binding over ``libmf.so`` (C ABI in ``include/mf.h``).  Device
memory and streams come from PyTorch; every arithmetic step runs in the CUDA
library.  There is no CPU fallback: calls raise if the library is missing.
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import MF_FP64, MF_FP32, MF_DF64, MF_PC_JACOBI, MF_PC_CHEBYSHEV, MF_PC_GMRES, MF_PC_MG, MfError, \
    MfSolverOpts, MfSolveReport

__all__ = ["RotorStatorOperator", "BatchedOperators", "MF_FP64", "MF_FP32", "MF_DF64", "MF_PC_JACOBI", "MF_PC_CHEBYSHEV", "MF_PC_GMRES", "MF_PC_MG", "MfError",
           "solver_defaults"]


def _check(status, h=None, what=""):
    if status != 0:
        lib = _lib.load()
        msg = lib.mf_last_error(h).decode() if h else ""
        name = _lib.STATUS_NAMES[status] if 0 <= status < len(_lib.STATUS_NAMES) else str(status)
        err = MfError(f"{what}: {name} {msg}")
        err.status = status
        raise err


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def solver_defaults(**over):
    o = MfSolverOpts()
    _lib.load().mf_solver_defaults(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


class RotorStatorOperator:
    """One operator instance on the current CUDA device.

    mesh: object with d, k, x0, node_side, wall, cells, cell_side, R, n_R, n_z,
    H, phi0, iface_rotor, iface_stator (e.g. synth.RotorStatorMesh).
    """

    def __init__(self, mesh, nu, omega, dt, bdf, penalty_F=1.0):
        lib = _lib.load()
        self.lib = lib
        self.d, self.k = int(mesh.d), int(mesh.k)
        x0 = np.ascontiguousarray(mesh.x0, dtype=np.float64)
        ns = np.ascontiguousarray(mesh.node_side, dtype=np.uint8)
        wall = np.ascontiguousarray(mesh.wall, dtype=np.uint8)
        cells = np.ascontiguousarray(mesh.cells, dtype=np.int32)
        cs = np.ascontiguousarray(mesh.cell_side, dtype=np.uint8)
        ifr = np.ascontiguousarray(mesh.iface_rotor, dtype=np.int32)
        ifs = np.ascontiguousarray(mesh.iface_stator, dtype=np.int32)
        mp = C.c_void_p()
        _check(lib.mf_mesh_from_arrays(self.d, self.k, x0.shape[0], _np_ptr(x0), _np_ptr(ns), _np_ptr(wall),
                                       cells.shape[0], _np_ptr(cells), _np_ptr(cs), float(mesh.R), int(mesh.n_R),
                                       int(mesh.n_z), float(mesh.H), float(mesh.phi0), _np_ptr(ifr), _np_ptr(ifs),
                                       C.byref(mp)), None, "mf_mesh_from_arrays")
        opt = _lib.MfOptions()
        opt.penalty_F = penalty_F
        hp = C.c_void_p()
        st = lib.mf_create(mp, self.k, float(nu), float(omega), float(dt), int(bdf), C.byref(opt), C.byref(hp))
        lib.mf_mesh_free(mp)
        _check(st, None, "mf_create")
        self.h = hp
        nn, nd, nc, nm = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib.mf_sizes(hp, C.byref(nn), C.byref(nd), C.byref(nc), C.byref(nm)), hp, "mf_sizes")
        self.n_nodes, self.n_dofs, self.n_cells, self.n_mortar = nn.value, nd.value, nc.value, nm.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.mf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st, what):
        _check(st, self.h, what)

    def set_angle(self, theta, stream=None):
        self._chk(self.lib.mf_set_angle(self.h, float(theta), _stream(stream)), "mf_set_angle")

    def node_coords(self, out, stream=None):
        self._chk(self.lib.mf_node_coords(self.h, _ptr(out), _stream(stream)), "mf_node_coords")

    def set_dirichlet(self, g=None, stream=None):
        self._chk(self.lib.mf_dirichlet(self.h, _ptr(g) if g is not None else None, _stream(stream)),
                  "mf_dirichlet")

    def set_history(self, u_n, u_nm1=None, stream=None):
        self._chk(self.lib.mf_set_history(self.h, _ptr(u_n), _ptr(u_nm1) if u_nm1 is not None else None,
                                          _stream(stream)), "mf_set_history")

    def set_linearization(self, up_star, theta, stream=None):
        self._chk(self.lib.mf_set_linearization(self.h, _ptr(up_star), float(theta), _stream(stream)),
                  "mf_set_linearization")

    def residual(self, up, r, stream=None):
        self._chk(self.lib.mf_residual(self.h, _ptr(up), _ptr(r), _stream(stream)), "mf_residual")

    def apply_jacobian(self, x, y, prec=MF_FP64, stream=None):
        self._chk(self.lib.mf_apply_jacobian(self.h, _ptr(x), _ptr(y), int(prec), _stream(stream)),
                  "mf_apply_jacobian")

    def diagonal(self, out, prec=MF_FP64, stream=None):
        self._chk(self.lib.mf_diagonal(self.h, _ptr(out), int(prec), _stream(stream)), "mf_diagonal")

    def mg_attach(self, coarse, parent=None, child=None):
        """Link `coarse` as the next multigrid level below this operator (h-coarsening
        when parent/child maps are given, else p-coarsening k -> k-1)."""
        if parent is None:
            st = self.lib.mf_mg_attach(self.h, coarse.h, None, None)
        else:
            par = np.ascontiguousarray(parent, dtype=np.int32)
            chd = np.ascontiguousarray(child, dtype=np.uint8)
            st = self.lib.mf_mg_attach(self.h, coarse.h, _np_ptr(par), _np_ptr(chd))
        self._chk(st, "mf_mg_attach")
        self._coarse = coarse          # keep the coarse level alive while linked

    def mg_prolongate(self, x_coarse, x_fine, stream=None):
        self._chk(self.lib.mf_mg_prolongate(self.h, _ptr(x_coarse), _ptr(x_fine), _stream(stream)), "mf_mg_prolongate")

    def mg_restrict(self, r_fine, r_coarse, stream=None):
        self._chk(self.lib.mf_mg_restrict(self.h, _ptr(r_fine), _ptr(r_coarse), _stream(stream)), "mf_mg_restrict")

    def mg_interpolate(self, u_fine, u_coarse, stream=None):
        self._chk(self.lib.mf_mg_interpolate(self.h, _ptr(u_fine), _ptr(u_coarse), _stream(stream)),
                  "mf_mg_interpolate")

    def profile(self, enable=True):
        """Enable (and reset) or disable the per-kernel CUDA-event timers."""
        self._chk(self.lib.mf_profile(self.h, int(bool(enable))), "mf_profile")

    def profile_read(self):
        """{kernel kind: (launches, total device ms)} since the last reset (synchronising)."""
        pr = _lib.MfProfile()
        self._chk(self.lib.mf_profile_read(self.h, C.byref(pr)), "mf_profile_read")
        return {k: (pr.launches[i], pr.ms[i]) for i, k in enumerate(_lib.PROF_KINDS)}

    def kinetic_energy(self, up, out, stream=None):
        """out (1-element device FP64 tensor) = 1/2 int |u|^2."""
        self._chk(self.lib.mf_kinetic_energy(self.h, _ptr(up), _ptr(out), _stream(stream)), "mf_kinetic_energy")

    def energy(self, up, out, stream=None):
        """out (3-element device FP64 tensor) = (1/2 int |u|^2, nu int grad u : grad u,
        nu int (grad u + grad u^T) : grad u)."""
        self._chk(self.lib.mf_energy(self.h, _ptr(up), _ptr(out), _stream(stream)), "mf_energy")

    def wall_loads(self, up, out, group=None, n_groups=2, stream=None):
        """out (device FP64 [n_groups, d+2]) = per wall group: force on the fluid (d),
        torque about e_z, power (see mf_wall_loads).  group: device uint8 [n_nodes]
        or None (0 = stationary walls, 1 = walls moving with the rotor)."""
        self._chk(self.lib.mf_wall_loads(self.h, _ptr(up), _ptr(group) if group is not None else None,
                                         int(n_groups), _ptr(out), _stream(stream)), "mf_wall_loads")

    def run_transient(self, u_n, u_nm1, n_steps, theta0, newton_iters=3, krylov_iters=6, opts=None,
                      use_graph=True, stream=None):
        """n_steps BDF steps with the rotor turning (see mf_run_transient); returns
        {field: array [n_steps+1]} for the fields of mf_step_record (record 0 is the
        initial state)."""
        recs = (_lib.MfStepRecord * (n_steps + 1))()
        o = opts if opts is not None else solver_defaults()
        st = self.lib.mf_run_transient(self.h, _ptr(u_n), _ptr(u_nm1) if u_nm1 is not None else None, int(n_steps),
                                       float(theta0), int(newton_iters), int(krylov_iters), C.byref(o),
                                       int(bool(use_graph)), recs, _stream(stream))
        self._chk(st, "mf_run_transient")
        return {f: np.array([getattr(r, f) for r in recs]) for f in _lib.STEP_RECORD_FIELDS}

    def last_error(self):
        return self.lib.mf_last_error(self.h).decode()

    def solve_step(self, up, opts=None, stream=None):
        rep = MfSolveReport()
        o = opts if opts is not None else solver_defaults()
        st = self.lib.mf_solve_step(self.h, _ptr(up), C.byref(o), C.byref(rep), _stream(stream))
        return st, rep


class BatchedOperators:
    """Several RotorStatorOperator instances (same d, k) applied in one persistent
    launch per kernel kind (mf_batch_apply_jacobian)."""

    def __init__(self, ops):
        lib = _lib.load()
        self.lib = lib
        self.ops = list(ops)
        arr = (C.c_void_p * len(self.ops))(*[o.h.value for o in self.ops])
        bp = C.c_void_p()
        _check(lib.mf_batch_create(arr, len(self.ops), C.byref(bp)), None, "mf_batch_create")
        self.b = bp

    def apply_jacobian(self, xs, ys, prec=MF_FP64, stream=None):
        n = len(self.ops)
        xa = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
        ya = (C.c_void_p * n)(*[y.data_ptr() for y in ys])
        st = self.lib.mf_batch_apply_jacobian(self.b, xa, ya, int(prec), _stream(stream))
        _check(st, None, "mf_batch_apply_jacobian")

    def close(self):
        if getattr(self, "b", None):
            self.lib.mf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
