"""B300 matrix-free rotor-stator operator (stabilised ALE Navier-Stokes + Nitsche/SIPG mortar).

Thin Python binding over ``libmf.so`` (C ABI in ``include/mf.h``).  Device
memory and streams come from PyTorch; every arithmetic step runs in the CUDA
library.  There is no CPU fallback: calls raise if the library is missing.
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import MF_FP64, MF_FP32, MF_DF64, MF_PC_JACOBI, MF_PC_CHEBYSHEV, MF_PC_GMRES, MF_PC_MG, MfError, \
    MF_SMOOTH_JACOBI, MF_SMOOTH_ASM, \
    MfSolverOpts, MfSolveReport

__all__ = ["RotorStatorOperator", "BatchedOperators", "Mesh", "rotor_stator_mesh", "coarsen_map", "save_checkpoint", "load_checkpoint", "log_open", "fma_peak", "mortar_segments", "slab_partition", "halo_pack", "halo_add", "MF_FP64", "MF_FP32", "MF_DF64", "MF_PC_JACOBI", "MF_PC_CHEBYSHEV", "MF_PC_GMRES", "MF_PC_MG", "MF_SMOOTH_JACOBI", "MF_SMOOTH_ASM", "MfError",
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


class Mesh:
    """A rotor-stator mesh generated by the library (mf_mesh_rotor_stator), as
    host arrays: x0 [N_n, d], cells [N_c, (k+1)^d] int32, cell_side,
    node_side, wall (uint8), iface_rotor / iface_stator [n_z, n_R] int32,
    and R, n_R, n_z, H, phi0; `params` holds the generator parameters."""

    def __init__(self, **kw):
        self.__dict__.update(kw)

    @property
    def n_nodes(self):
        return self.x0.shape[0]

    @property
    def n_cells(self):
        return self.cells.shape[0]

    @property
    def n_dofs(self):
        return self.n_nodes * (self.d + 1)


def _mesh_params(params):
    p = _lib.MfMeshParams()
    _lib.load().mf_mesh_params_defaults(C.byref(p))
    for key, v in params.items():
        if key not in dict(_lib.MfMeshParams._fields_):
            raise TypeError(f"unknown mesh parameter {key}")
        setattr(p, key, v)
    return p


def rotor_stator_mesh(**params):
    """Generate a rotor-stator mesh in the library (parameters of
    mf_mesh_params: d, k, m, n_r, n_s, n_z, R, R_out, H, sq, phi0, blades;
    the rest default) and return it as a Mesh."""
    lib = _lib.load()
    p = _mesh_params(params)
    mp = C.c_void_p()
    _check(lib.mf_mesh_rotor_stator(C.byref(p), C.byref(mp)), None, "mf_mesh_rotor_stator")
    try:
        m = _read_mesh(mp, R=p.R, H=p.H, phi0=p.phi0)
    finally:
        lib.mf_mesh_free(mp)
    m.params = {f: getattr(p, f) for f, _ in _lib.MfMeshParams._fields_}
    return m


def _read_mesh(mp, R, H, phi0):
    """Host arrays of an mf_mesh (mf_mesh_sizes, mf_mesh_interface, mf_mesh_read) as a Mesh."""
    lib = _lib.load()
    d, k, n_R, n_z = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    nn, nc = C.c_int64(), C.c_int64()
    _check(lib.mf_mesh_sizes(mp, C.byref(d), C.byref(k), C.byref(nn), C.byref(nc), C.byref(n_R), C.byref(n_z)),
           None, "mf_mesh_sizes")
    d, k, nn, nc, n_R, n_z = d.value, k.value, nn.value, nc.value, n_R.value, n_z.value
    nrs = C.c_int()
    _check(lib.mf_mesh_interface(mp, None, C.byref(nrs), None), None, "mf_mesh_interface")
    n_Rs = nrs.value
    x0 = np.empty((nn, d))
    ns, wall = np.empty(nn, np.uint8), np.empty(nn, np.uint8)
    cells = np.empty((nc, (k + 1) ** d), np.int32)
    cs = np.empty(nc, np.uint8)
    ifr, ifs = np.empty((n_z, n_R), np.int32), np.empty((n_z, n_Rs), np.int32)
    _check(lib.mf_mesh_read(mp, _np_ptr(x0), _np_ptr(ns), _np_ptr(wall), _np_ptr(cells), _np_ptr(cs),
                            _np_ptr(ifr), _np_ptr(ifs)), None, "mf_mesh_read")
    return Mesh(d=d, k=k, x0=x0, cells=cells, cell_side=cs, node_side=ns, wall=wall, iface_rotor=ifr,
                iface_stator=ifs, R=R, n_R=n_R, n_z=n_z, H=(H if d == 3 else 1.0), phi0=phi0, params=None,
                n_R_stator=n_Rs)


def slab_partition(mesh, n_parts, part):
    """Part `part` of the z-slab partition of a 3D mesh into n_parts parts
    (mf_mesh_slab).  Returns (slab Mesh, plan) with plan = dict(node_global
    [n_nodes] int64, lo / hi [n] int32 local ids of the nodes shared with the
    part below / above (ascending global id), lo_wall / hi_wall uint8,
    layer_begin, layer_end)."""
    lib = _lib.load()
    gm = _mesh_handle(mesh)
    sm = C.c_void_p()
    try:
        info = _lib.MfSlabInfo()
        _check(lib.mf_mesh_slab(gm, int(n_parts), int(part), None, C.byref(info), None, None, None, None, None),
               None, "mf_mesh_slab")
        ng = np.empty(info.n_nodes, np.int64)
        lo, hi = np.empty(info.n_lo, np.int32), np.empty(info.n_hi, np.int32)
        lw, hw = np.empty(info.n_lo, np.uint8), np.empty(info.n_hi, np.uint8)
        _check(lib.mf_mesh_slab(gm, int(n_parts), int(part), C.byref(sm), C.byref(info), _np_ptr(ng), _np_ptr(lo),
                                _np_ptr(hi), _np_ptr(lw), _np_ptr(hw)), None, "mf_mesh_slab")
        H = float(mesh.H) * (info.layer_end - info.layer_begin) / int(mesh.n_z)
        slab = _read_mesh(sm, R=float(mesh.R), H=H, phi0=float(mesh.phi0))
    finally:
        lib.mf_mesh_free(gm)
        if sm.value:
            lib.mf_mesh_free(sm)
    plan = dict(node_global=ng, lo=lo, hi=hi, lo_wall=lw, hi_wall=hw, layer_begin=info.layer_begin,
                layer_end=info.layer_end)
    return slab, plan


def halo_pack(y, idx, buf, stream=None):
    """buf[i, :] = y[idx[i], :] (mf_halo_pack; device FP64 tensors, idx int32)."""
    _check(_lib.load().mf_halo_pack(_ptr(y), _ptr(idx), int(idx.numel()), int(y.shape[-1]), _ptr(buf),
                                    _stream(stream)), None, "mf_halo_pack")


def halo_add(y, idx, wall, buf, stream=None):
    """y[idx[i], :] += buf[i, :] except wall velocity rows (mf_halo_add)."""
    _check(_lib.load().mf_halo_add(_ptr(y), _ptr(idx), _ptr(wall) if wall is not None else None, int(idx.numel()),
                                   int(y.shape[-1]), _ptr(buf), _stream(stream)), None, "mf_halo_add")


def mortar_segments(n_R, n_Rs, theta):
    """Mortar segments of an interface with n_R rotor and n_Rs stator cells at
    rotor angle theta (mf_mortar_segments): arrays start, length, rotor cell,
    stator cell."""
    lib = _lib.load()
    cap = int(n_R) + int(n_Rs)
    a, L = np.empty(cap), np.empty(cap)
    jr, js = np.empty(cap, np.int32), np.empty(cap, np.int32)
    cnt = C.c_int()
    _check(lib.mf_mortar_segments(int(n_R), int(n_Rs), float(theta), cap, _np_ptr(a), _np_ptr(L), _np_ptr(jr),
                                  _np_ptr(js), C.byref(cnt)), None, "mf_mortar_segments")
    c = cnt.value
    return a[:c], L[:c], jr[:c], js[:c]


def coarsen_map(**params):
    """Uniform coarsening of a generated mesh (mf_mesh_coarsen_map): returns
    (coarse parameters as a dict, parent [N_c] int32, child [N_c] uint8) for
    RotorStatorOperator.mg_attach."""
    lib = _lib.load()
    p = _mesh_params(params)
    fine = rotor_stator_mesh(**params)
    cp = _lib.MfMeshParams()
    parent = np.empty(fine.n_cells, np.int32)
    child = np.empty(fine.n_cells, np.uint8)
    _check(lib.mf_mesh_coarsen_map(C.byref(p), C.byref(cp), _np_ptr(parent), _np_ptr(child)), None,
           "mf_mesh_coarsen_map")
    return {f: getattr(cp, f) for f, _ in _lib.MfMeshParams._fields_}, parent, child


def _mesh_handle(mesh):
    """An mf_mesh (host copy) of a mesh object; free it with mf_mesh_free."""
    lib = _lib.load()
    x0 = np.ascontiguousarray(mesh.x0, dtype=np.float64)
    ns = np.ascontiguousarray(mesh.node_side, dtype=np.uint8)
    wall = np.ascontiguousarray(mesh.wall, dtype=np.uint8)
    cells = np.ascontiguousarray(mesh.cells, dtype=np.int32)
    cs = np.ascontiguousarray(mesh.cell_side, dtype=np.uint8)
    ifr = np.ascontiguousarray(mesh.iface_rotor, dtype=np.int32)
    ifs = np.ascontiguousarray(mesh.iface_stator, dtype=np.int32)
    mp = C.c_void_p()
    n_Rs = int(ifs.shape[1]) if ifs.ndim == 2 else int(mesh.n_R)
    _check(lib.mf_mesh_from_arrays_ex(int(mesh.d), int(mesh.k), x0.shape[0], _np_ptr(x0), _np_ptr(ns), _np_ptr(wall),
                                      cells.shape[0], _np_ptr(cells), _np_ptr(cs), float(mesh.R), int(mesh.n_R), n_Rs,
                                      int(mesh.n_z), float(mesh.H), float(mesh.phi0), _np_ptr(ifr), _np_ptr(ifs),
                                      C.byref(mp)), None, "mf_mesh_from_arrays_ex")
    return mp


def log_open(path):
    """Append one JSON line per library call (solves, transient runs, mesh
    generation, autotuning, checkpoints) to `path`; None turns the log off."""
    _check(_lib.load().mf_log_open(str(path).encode() if path else None), None, "mf_log_open")


def fma_peak(prec=MF_FP64, stream=None):
    """Measured FMA rate of the current device (mf_fma_peak): (TFLOP/s, ms per
    probe launch) in FP64 or FP32."""
    tf, ms = C.c_double(), C.c_double()
    _check(_lib.load().mf_fma_peak(int(prec), C.byref(tf), C.byref(ms), _stream(stream)), None, "mf_fma_peak")
    return tf.value, ms.value


def contract_probe(variant, u, out, reps=1, err=None, stream=None):
    """Interpolation-stage probe (mf_contract_probe): variant 0 FP32 FMA sum
    factorisation, 1 tcgen05 TF32, 2 tcgen05 3xTF32.  u: device float32
    [blocks, 27, 4, 32]; out: device float32 [blocks, 108, 4, 32] (reps == 1)
    or [blocks, 4, 32] (sums over reps > 1); err: device int32 [1] (variants
    1, 2).  Asynchronous on `stream`."""
    blocks = int(u.shape[0])
    _check(_lib.load().mf_contract_probe(int(variant), blocks, int(reps), _ptr(u), _ptr(out),
                                         _ptr(err) if err is not None else None, _stream(stream)),
           None, "mf_contract_probe")


def vec_dots(V, x, out, w=None, stream=None):
    """out[i] = sum_j w[j] V[i, j] x[j] (mf_vec_dots): V a device float64
    [m, n] tensor (rows are the vectors), x [n], w [n] or None, out [m]."""
    m, n = int(V.shape[0]), int(V.shape[1])
    _check(_lib.load().mf_vec_dots(n, _ptr(V), int(V.stride(0)), m, _ptr(x), _ptr(w) if w is not None else None,
                                   _ptr(out), _stream(stream)), None, "mf_vec_dots")


def vec_maxpy(V, c, y, sign=1.0, stream=None):
    """y += sign sum_i c[i] V[i] (mf_vec_maxpy): V device float64 [m, n], c [m] device."""
    m, n = int(V.shape[0]), int(V.shape[1])
    _check(_lib.load().mf_vec_maxpy(n, _ptr(V), int(V.stride(0)), m, _ptr(c), float(sign), _ptr(y),
                                    _stream(stream)), None, "mf_vec_maxpy")


def vec_axpby(a, x, b, y, stream=None):
    """y = a x + b y (mf_vec_axpby), float64 device vectors."""
    _check(_lib.load().mf_vec_axpby(int(x.numel()), float(a), _ptr(x), float(b), _ptr(y), _stream(stream)),
           None, "mf_vec_axpby")


def vec_mul(d, v, z, stream=None):
    """z = d * v entrywise (mf_vec_mul), float64 device vectors."""
    _check(_lib.load().mf_vec_mul(int(v.numel()), _ptr(d), _ptr(v), _ptr(z), _stream(stream)), None, "mf_vec_mul")


def _host_f64(a):
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


def save_checkpoint(path, mesh, u_n, u_nm1=None, *, step, t, theta, dt, nu, omega):
    """Write a checkpoint of a time-dependent run (mf_checkpoint_write): u_n
    and, for BDF2, u_nm1 ([n_nodes, d+1], numpy arrays or tensors on any
    device; copied to the host), step, time, rotor angle and parameters."""
    lib = _lib.load()
    info = _lib.MfCheckpointInfo(bdf=2 if u_nm1 is not None else 1, step=int(step), t=float(t), theta=float(theta),
                                 dt=float(dt), nu=float(nu), omega=float(omega))
    a = _host_f64(u_n)
    b = _host_f64(u_nm1) if u_nm1 is not None else None
    for arr in (a, b):
        if arr is not None and arr.size != mesh.n_nodes * (mesh.d + 1):
            raise MfError("save_checkpoint: state size does not match the mesh")
    mp = _mesh_handle(mesh)
    try:
        st = lib.mf_checkpoint_write(str(path).encode(), mp, C.byref(info), _np_ptr(a),
                                     _np_ptr(b) if b is not None else None)
    finally:
        lib.mf_mesh_free(mp)
    _check(st, None, "mf_checkpoint_write")


def load_checkpoint(path, mesh):
    """Read a checkpoint written for `mesh` (mf_checkpoint_read).  Returns
    (info dict, u_n, u_nm1 or None) with host numpy arrays [n_nodes, d+1]."""
    lib = _lib.load()
    info = _lib.MfCheckpointInfo()
    shape = (mesh.n_nodes, mesh.d + 1)
    a, b = np.empty(shape), np.empty(shape)
    mp = _mesh_handle(mesh)
    try:
        st = lib.mf_checkpoint_read(str(path).encode(), mp, C.byref(info), _np_ptr(a), _np_ptr(b))
    finally:
        lib.mf_mesh_free(mp)
    _check(st, None, "mf_checkpoint_read")
    d = {f: getattr(info, f) for f, _ in _lib.MfCheckpointInfo._fields_}
    return d, a, (b if info.bdf == 2 else None)


class RotorStatorOperator:
    """One operator instance on the current CUDA device.

    mesh: object with d, k, x0, node_side, wall, cells, cell_side, R, n_R, n_z,
    H, phi0, iface_rotor, iface_stator (e.g. synth.RotorStatorMesh).
    """

    def __init__(self, mesh, nu, omega, dt, bdf, penalty_F=1.0):
        lib = _lib.load()
        self.lib = lib
        self.d, self.k = int(mesh.d), int(mesh.k)
        mp = _mesh_handle(mesh)
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

    def autotune(self, cache_path=None, stream=None):
        """Time the cells-per-block variants of the FP64 and FP32 cell Jacobian
        kernels (mf_autotune) and keep the fastest.  Returns one dict per
        precision: variants, ms, chosen cells per block, from_cache."""
        res = (_lib.MfTuneResult * 2)()
        cp = cache_path.encode() if cache_path else None
        self._chk(self.lib.mf_autotune(self.h, cp, res, _stream(stream)), "mf_autotune")
        out = {}
        for name, r in zip(("fp64", "fp32"), res):
            n = r.n_variants
            out[name] = {"cells_per_block": list(r.cells_per_block[:n]), "ms": list(r.ms[:n]),
                         "chosen": r.cells_per_block[r.chosen], "from_cache": bool(r.from_cache)}
        return out

    def asm_setup(self, stream=None):
        """Additive Schwarz local matrices and FP32 inverses (mf_asm_setup);
        returns the number of replaced pivots."""
        bad = C.c_int()
        self._chk(self.lib.mf_asm_setup(self.h, C.byref(bad), _stream(stream)), "mf_asm_setup")
        return bad.value

    def asm_apply(self, r, z, stream=None):
        """z = ASM(r), FP32 device tensors (mf_asm_apply)."""
        self._chk(self.lib.mf_asm_apply(self.h, _ptr(r), _ptr(z), _stream(stream)), "mf_asm_apply")

    def set_cells_per_block(self, prec, cpb):
        self._chk(self.lib.mf_set_cells_per_block(self.h, int(prec), int(cpb)), "mf_set_cells_per_block")

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

    def solve_step(self, ups, thetas, opts=None, krylov_iters=8, batched=True, use_graph=True, stream=None):
        """One Newton step of every instance (mf_batch_solve_step); ups are
        overwritten.  Returns (status, [MfSolveReport per instance])."""
        n = len(self.ops)
        ua = (C.c_void_p * n)(*[u.data_ptr() for u in ups])
        ta = (C.c_double * n)(*[float(t) for t in thetas])
        reps = (MfSolveReport * n)()
        o = opts if opts is not None else solver_defaults()
        st = self.lib.mf_batch_solve_step(self.b, ua, ta, C.byref(o), int(krylov_iters), int(bool(batched)),
                                          int(bool(use_graph)), reps, _stream(stream))
        if st not in (_lib.MF_OK, _lib.MF_ERR_NOT_CONVERGED, _lib.MF_ERR_NAN):
            raise MfError(f"mf_batch_solve_step: {_lib.STATUS_NAMES[st]} ({self.last_error()})")
        return st, list(reps)

    def last_error(self):
        return self.lib.mf_batch_last_error(self.b).decode()

    def close(self):
        if getattr(self, "b", None):
            self.lib.mf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
