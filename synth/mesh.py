"""Structured rotor-stator meshes with a circular sliding interface.

Layout (Section 3.1 of the paper: rotor and stator grids are generated
separately and merged; both sides of the interface carry the same number of
equally sized cells):

* rotor disk r < R: an O-grid made of an m x m centre square (half width
  ``sq * R``) and four ring blocks of m x n_r cells blending the square's sides
  into the circle r = R; the interface therefore has n_R = 4 m cells;
* stator annulus R < r < R_out: a polar grid of n_Rs x n_s cells, n_Rs = n_R
  unless n_R_stator is given (unequal interface partitions, beyond the
  paper's equal-partition restriction);
* 3D: both are extruded along z in n_z layers over [0, H].

Geometry nodes are the Q_k nodes of every cell (Gauss-Lobatto points in
the cell's parameter square/cube), placed on the parametric map of the block,
so the interface nodes sit exactly on the circle at angles linear in the
cell's angular coordinate.  Nodes on the interface are duplicated: the rotor
copy and the stator copy are different nodes (their values are independent
unknowns).

Cell-local node order is tensor order with xi_0 fastest.  Ring and stator
cells are oriented with xi_0 = radial (outward), xi_1 = angular
(counter-clockwise), xi_2 = z, so every cell map has a positive Jacobian and
the interface face is xi_0 = 1 on rotor cells and xi_0 = 0 on stator cells.

Interface cell tables: ``iface_rotor[l, j]`` / ``iface_stator[l, j]`` is the
cell at z-layer l whose angular span, in the reference configuration, is
[phi0 + j*D, phi0 + (j+1)*D], D = 2*pi/n_R.
"""
from dataclasses import dataclass, field
import numpy as np


def _gll01(k):
    """Gauss-Lobatto points on [0, 1] (k+1 of them), symmetric to roundoff."""
    if k < 1:
        raise ValueError("k >= 1 required")
    from numpy.polynomial import legendre as L
    c = np.zeros(k + 1)
    c[k] = 1.0
    inner = np.sort(np.real(L.legroots(L.legder(c)))) if k >= 2 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    x = 0.5 * (x - x[::-1])
    return 0.5 * (x + 1.0)


def _param(ncell, k, g):
    """Parameter in [0,1] of node index i = 0..ncell*k along a block side."""
    i = np.arange(ncell * k + 1)
    c = np.minimum(i // k, ncell - 1)
    a = i - c * k
    return (c + g[a]) / ncell


@dataclass
class RotorStatorMesh:
    d: int
    k: int
    x0: np.ndarray            # [N_n, d] reference-configuration coordinates
    cells: np.ndarray         # [N_c, (k+1)^d] int32, tensor order, xi_0 fastest
    cell_side: np.ndarray     # [N_c] uint8, 0 rotor, 1 stator
    node_side: np.ndarray     # [N_n] uint8, 0 rotor, 1 stator
    wall: np.ndarray          # [N_n] uint8, 1 = stationary wall, 2 = wall moving with the rotor (blade)
    iface_rotor: np.ndarray   # [n_z, n_R] int32
    iface_stator: np.ndarray  # [n_z, n_R_stator] int32
    R: float
    n_R: int
    n_z: int
    H: float
    phi0: float
    params: dict = field(default_factory=dict)
    n_R_stator: int = 0       # stator interface cells per layer; 0: equal to n_R

    @property
    def n_nodes(self):
        return self.x0.shape[0]

    @property
    def n_cells(self):
        return self.cells.shape[0]

    @property
    def n_dofs(self):
        return self.n_nodes * (self.d + 1)


def rotor_stator_mesh(d, k, m, n_r, n_s, n_z=1, R=0.5, R_out=1.0, H=1.0, sq=0.55,
                      phi0=-0.25 * np.pi, blades=0, n_R_stator=None):
    """Generate the merged rotor/stator mesh (see module docstring).

    blades > 0 (3D): that many radial blades inside the rotor, each the ring
    cells of one angular index (equally spaced), the inner three quarters of
    the rings and the middle half of the height; their nodes are walls moving
    with the rotor (wall = 2, velocity omega e_z x x)."""
    if d not in (2, 3):
        raise ValueError("d must be 2 or 3")
    g = _gll01(k)
    n = k + 1
    mk = m * k
    n_R = 4 * m
    n_Rs = n_R if n_R_stator is None else int(n_R_stator)
    if n_Rs < 1:
        raise ValueError("n_R_stator >= 1 required")
    nRk = n_Rs * k                                        # stator nodes per ring
    s = sq * R

    # ---- 2D rotor: centre square nodes
    tq = _param(m, k, g)
    sx = -s + 2.0 * s * tq
    SX, SY = np.meshgrid(sx, sx, indexing="xy")           # [iy, ix]
    sq_xy = np.stack([SX.ravel(), SY.ravel()], axis=1)    # id = iy*(mk+1)+ix
    n_sq = (mk + 1) ** 2

    def sq_id(ix, iy):
        return iy * (mk + 1) + ix

    # perimeter index ia in [0, 4mk): block b = ia // mk, it = ia % mk
    ia = np.arange(4 * mk)
    b = ia // mk
    it = ia % mk
    per_ix = np.select([b == 0, b == 1, b == 2, b == 3], [np.full_like(it, mk), mk - it, np.zeros_like(it), it])
    per_iy = np.select([b == 0, b == 1, b == 2, b == 3], [it, np.full_like(it, mk), mk - it, np.zeros_like(it)])
    per_id = sq_id(per_ix, per_iy)
    tb = tq[it]
    per_xy = sq_xy[per_id]
    ang = phi0 + (b + tb) * (0.5 * np.pi)
    circ = np.stack([R * np.cos(ang), R * np.sin(ang)], axis=1)

    rho = _param(n_r, k, g)                               # ir = 0..n_r*k
    n_ring = n_r * k * 4 * mk
    ring_xy = np.empty((n_r * k, 4 * mk, 2))
    for ir in range(1, n_r * k + 1):
        r_ = rho[ir]
        ring_xy[ir - 1] = (1.0 - r_) * per_xy + r_ * circ
    ring_xy[-1] = circ                                    # interface ring exactly on the circle
    rotor_xy = np.concatenate([sq_xy, ring_xy.reshape(-1, 2)], axis=0)
    n_rot2 = n_sq + n_ring

    def ring_id(ir, ia_):
        ia_ = ia_ % (4 * mk)
        return np.where(ir == 0, per_id[ia_], n_sq + (np.maximum(ir, 1) - 1) * (4 * mk) + ia_)

    li = np.arange(n)
    I0, I1 = np.meshgrid(li, li, indexing="xy")           # I0 fastest after ravel
    I0 = I0.ravel()
    I1 = I1.ravel()
    cells2 = []
    # centre square cells (xi_0 = x, xi_1 = y)
    for cy in range(m):
        for cx in range(m):
            cells2.append(sq_id(cx * k + I0, cy * k + I1))
    n_sq_cells = len(cells2)
    # ring cells: angular cell j = 0..n_R-1, radial jr = 0..n_r-1 (xi_0 radial, xi_1 angular)
    ring_cell_index = np.empty((n_R, n_r), dtype=np.int64)
    for jr in range(n_r):
        for j in range(n_R):
            ring_cell_index[j, jr] = len(cells2)
            cells2.append(ring_id(jr * k + I0, j * k + I1))
    n_rot_cells2 = len(cells2)

    # ---- 2D stator annulus
    rr = R + (R_out - R) * _param(n_s, k, g)
    angp = _param(n_Rs, k, g)[:-1]                        # ia = 0..nRk-1
    phis = phi0 + 2.0 * np.pi * angp
    RR, PP = np.meshgrid(rr, phis, indexing="ij")         # [ir, ia]
    st_xy = np.stack([RR * np.cos(PP), RR * np.sin(PP)], axis=-1).reshape(-1, 2)
    # the interface copy of the stator uses the same angles as the rotor circle
    st_xy[:nRk] = circ_all = np.stack([R * np.cos(phis), R * np.sin(phis)], axis=1)
    del circ_all
    n_st2 = st_xy.shape[0]

    def st_id(ir, ia_):
        return n_rot2 + ir * nRk + (ia_ % nRk)

    st_cell_index = np.empty((n_Rs, n_s), dtype=np.int64)
    for jr in range(n_s):
        for j in range(n_Rs):
            st_cell_index[j, jr] = len(cells2)
            cells2.append(st_id(jr * k + I0, j * k + I1))
    cells2 = np.asarray(cells2, dtype=np.int64)
    n_c2 = cells2.shape[0]
    xy = np.concatenate([rotor_xy, st_xy], axis=0)
    n2 = xy.shape[0]
    node_side2 = np.concatenate([np.zeros(n_rot2, np.uint8), np.ones(n_st2, np.uint8)])
    wall2 = np.zeros(n2, np.uint8)
    wall2[n_rot2 + n_s * k * nRk: n_rot2 + (n_s * k + 1) * nRk] = 1   # r = R_out
    cell_side2 = np.concatenate([np.zeros(n_rot_cells2, np.uint8), np.ones(n_c2 - n_rot_cells2, np.uint8)])
    ifr2 = ring_cell_index[:, n_r - 1]
    ifs2 = st_cell_index[:, 0]

    params = dict(d=d, k=k, m=m, n_r=n_r, n_s=n_s, n_z=n_z, R=R, R_out=R_out, H=H, sq=sq, phi0=phi0, blades=blades,
                  n_R_stator=n_Rs)
    if d == 2:
        return RotorStatorMesh(d=2, k=k, x0=xy.copy(), cells=cells2.astype(np.int32),
                               cell_side=cell_side2, node_side=node_side2, wall=wall2,
                               iface_rotor=ifr2[None, :].astype(np.int32),
                               iface_stator=ifs2[None, :].astype(np.int32),
                               R=R, n_R=n_R, n_z=1, H=1.0, phi0=phi0, params=params, n_R_stator=n_Rs)

    # ---- 3D extrusion: node id = iz * n2 + id2, cell id = lz * n_c2 + c2
    blade_cells2 = []
    if blades > 0:
        for b in range(blades):
            j = (b * n_R) // blades
            for jr in range(0, max(1, (3 * n_r) // 4)):
                blade_cells2.append(ring_cell_index[j, jr])
    zs = H * _param(n_z, k, g)
    nz_nodes = n_z * k + 1
    x3 = np.empty((nz_nodes, n2, 3))
    x3[:, :, 0:2] = xy[None]
    x3[:, :, 2] = zs[:, None]
    x3 = x3.reshape(-1, 3)
    wall3 = np.tile(wall2, nz_nodes)
    if blade_cells2:
        bnodes2 = np.unique(cells2[blade_cells2].ravel())
        for iz in range((n_z // 4) * k, (3 * n_z // 4) * k + 1):
            wall3[iz * n2 + bnodes2] = 2
    wall3[:n2] = 1
    wall3[(nz_nodes - 1) * n2:] = 1
    node_side3 = np.tile(node_side2, nz_nodes)
    cells3 = np.empty((n_z, n_c2, n ** 3), dtype=np.int64)
    for i2 in range(n):
        cells3[:, :, i2 * n * n:(i2 + 1) * n * n] = (np.arange(n_z)[:, None, None] * k + i2) * n2 + cells2[None]
    cells3 = cells3.reshape(-1, n ** 3)
    cell_side3 = np.tile(cell_side2, n_z)
    ifr3 = np.arange(n_z)[:, None] * n_c2 + ifr2[None, :]
    ifs3 = np.arange(n_z)[:, None] * n_c2 + ifs2[None, :]
    return RotorStatorMesh(d=3, k=k, x0=x3, cells=cells3.astype(np.int32), cell_side=cell_side3,
                           node_side=node_side3, wall=wall3, iface_rotor=ifr3.astype(np.int32),
                           iface_stator=ifs3.astype(np.int32), R=R, n_R=n_R, n_z=n_z, H=H,
                           phi0=phi0, params=params, n_R_stator=n_Rs)


def coarsen(params):
    """Parameters of the uniformly coarsened mesh (every block halved in each of
    its cell directions) and the parent map of the fine cells.

    Returns (coarse_params, parent [N_c fine] int32, child [N_c fine] uint8):
    parent[c] is the coarse cell containing fine cell c, bit r of child[c] is 1
    when c is the upper half of its parent along xi_r.  Requires m, n_r, n_s
    (and n_z in 3D) even.  Both meshes use the same parametric block maps, so
    the fine cells subdivide the coarse cells in parameter space.
    """
    d, m, n_r, n_s, n_z = params["d"], params["m"], params["n_r"], params["n_s"], params["n_z"]
    if params.get("n_R_stator") not in (None, 4 * m):
        raise ValueError("coarsen: unequal interface partitions are not supported")
    if m % 2 or n_r % 2 or n_s % 2 or (d == 3 and n_z % 2):
        raise ValueError("m, n_r, n_s (and n_z in 3D) must be even to coarsen")
    cp = dict(params, m=m // 2, n_r=n_r // 2, n_s=n_s // 2, n_z=(n_z // 2 if d == 3 else n_z))
    if "n_R_stator" in params:
        cp["n_R_stator"] = 2 * m          # equal partitions on the coarse mesh too
    mc, n_R, n_Rc = m // 2, 4 * m, 2 * m
    parent, child = [], []
    # centre square (xi_0 = x, xi_1 = y), index cy*m + cx
    for cy in range(m):
        for cx in range(m):
            parent.append((cy // 2) * mc + cx // 2)
            child.append((cx % 2) | ((cy % 2) << 1))
    nsq_c = mc * mc
    # ring cells (xi_0 radial, xi_1 angular), index n_sq + jr*n_R + j
    for jr in range(n_r):
        for j in range(n_R):
            parent.append(nsq_c + (jr // 2) * n_Rc + j // 2)
            child.append((jr % 2) | ((j % 2) << 1))
    nrot_c = nsq_c + (n_r // 2) * n_Rc
    for jr in range(n_s):
        for j in range(n_R):
            parent.append(nrot_c + (jr // 2) * n_Rc + j // 2)
            child.append((jr % 2) | ((j % 2) << 1))
    parent = np.array(parent, dtype=np.int64)
    child = np.array(child, dtype=np.uint8)
    if d == 3:
        nc2, nc2c = len(parent), nrot_c + (n_s // 2) * n_Rc
        lz = np.arange(n_z)
        parent = ((lz[:, None] // 2) * nc2c + parent[None, :]).ravel()
        child = (child[None, :] | ((lz[:, None] % 2) << 2).astype(np.uint8)).ravel()
    return cp, parent.astype(np.int32), child.astype(np.uint8)


def hierarchy(params, levels):
    """Meshes of an h-hierarchy: [(mesh, parent, child)] from fine to coarse;
    parent/child of the coarsest level are None."""
    out = []
    p = dict(params)
    for lev in range(levels):
        mesh = rotor_stator_mesh(p["d"], p["k"], p["m"], p["n_r"], p["n_s"], p.get("n_z", 1))
        if lev + 1 < levels:
            cp, parent, child = coarsen(dict(p, n_z=p.get("n_z", 1)))
            out.append((mesh, parent, child))
            p = cp
        else:
            out.append((mesh, None, None))
    return out
