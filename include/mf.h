/* mf.h -- C ABI of the B300 matrix-free rotor-stator operator library (libmf.so).
 *
 * The library evaluates, on one GPU, the discrete operator of "High-order
 * stabilized matrix-free simulation of rotating mixing devices using the Mortar
 * Element Method":
 *   - the stabilised ALE incompressible Navier-Stokes residual F-hat*_NS
 *     (Eqs. EqNS, Eq-NSweakWmortar, Eq-NSweakComplete, Eq-strong-residual,
 *     Eq-stab-param) on continuous Q_k quadrilaterals (d = 2) or hexahedra
 *     (d = 3) with equal-order velocity/pressure (Eq. Eq-shape-functions);
 *   - its Newton Jacobian (blocks A-hat..D-hat, Section 2.3; tau frozen);
 *   - the Nitsche/SIPG mortar face terms coupling the rotating rotor to the
 *     stator (Eqs. EqMortarPre, EqMortarDiff, EqPenalty, EqMortarMass) on mortar
 *     cells built from both angular partitions of the interface (Section 3.2),
 *     with the rotor rotated rigidly (Section 3.1);
 *   - a Newton / flexible-GMRES solve of one nonlinear step (Eq.
 *     Eq-Newton-method) with Jacobi, Chebyshev-Jacobi (FP32 or FP64) smoothing.
 *
 * Conventions
 *   - Vectors are interleaved per node: [node][u_1 .. u_d, p] (d+1 values per
 *     node), in the mesh's node numbering.  Interface nodes are duplicated: the
 *     rotor copy and the stator copy are different nodes.
 *   - Unless stated otherwise, every pointer argument of an operator call is
 *     caller-owned DEVICE memory on the current CUDA device; the library keeps
 *     no caller pointer past the call.  Calls are asynchronous on `stream`
 *     (a cudaStream_t passed as void*, NULL = legacy default stream), except
 *     those documented as synchronising.
 *   - Velocity components on wall nodes carry homogeneous (or mf_dirichlet)
 *     Dirichlet conditions: Jacobian rows/columns there are identity and the
 *     residual there is u - g.  Pressure is unconstrained.  The constant
 *     pressure is only a near null vector of the discrete operator (the mortar
 *     integrates the exact circle while a cell's divergence theorem uses its
 *     polynomial face, an O(h^k) defect on interface rows), so the equations
 *     fix the pressure level weakly and no solve removes a pressure mean;
 *     mf_solver_opts.deflate_pressure optionally minimises the residual along
 *     J e_p at each FGMRES restart (off by default).
 *   - Every call returns an mf_status; on failure mf_last_error(h) holds a
 *     message.  No call throws across the ABI.
 */
#ifndef MF_H
#define MF_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct mf_ctx* mf_handle;
typedef struct mf_mesh mf_mesh;

typedef enum {
  MF_OK = 0,
  MF_ERR_ARG = 1,          /* invalid argument (null pointer, size, range) */
  MF_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  MF_ERR_OOM = 3,          /* device allocation failed */
  MF_ERR_STATE = 4,        /* call out of order (e.g. apply before set_linearization) */
  MF_ERR_NAN = 5,          /* non-finite value met by a solve */
  MF_ERR_NOT_CONVERGED = 6,/* solve stopped at its iteration limit above tolerance */
  MF_ERR_BREAKDOWN = 7,    /* Krylov breakdown (zero Arnoldi vector before convergence) */
  MF_ERR_ITER_LIMIT = 8    /* reserved: device-side loop hit its hard cap */
} mf_status;

/* MF_FP64: native FP64 arithmetic.  MF_FP32: FP32 arithmetic on an FP32 copy of
 * the cache (vectors are float).  MF_DF64: FP64-accurate applies computed in
 * double-float arithmetic (pairs of floats, ~48-bit significand) on the FP32
 * pipes, FP64 vectors in memory; only mf_apply_jacobian accepts it. */
typedef enum { MF_FP64 = 0, MF_FP32 = 1, MF_DF64 = 2 } mf_precision;

/* ---------------------------------------------------------------- mesh
 * mf_mesh_from_arrays: copy a merged rotor-stator mesh from HOST arrays.
 *   d            2 or 3
 *   k            polynomial degree of the Q_k geometry/solution nodes (1..5)
 *   n_nodes, x0  [n_nodes][d] node coordinates in the reference (theta = 0)
 *                configuration
 *   node_side    [n_nodes] 0 = rotor node (rotates), 1 = stator node
 *   wall         [n_nodes] 0 = free, 1 = stationary velocity Dirichlet node,
 *                2 = wall moving with the rotor (e.g. a blade; a rotor node):
 *                Dirichlet velocity omega e_z x x at the node's current position
 *   n_cells, cells [n_cells][(k+1)^d] int32 node ids, tensor order with xi_0
 *                fastest; every cell map must have positive Jacobian
 *   cell_side    [n_cells] 0 = rotor cell (mesh velocity omega e_z x x), 1 = stator
 *   R, n_R, n_z, H, phi0  circular interface r = R about the z axis with n_R
 *                equal cells per z-layer on each side (the paper's restriction,
 *                Section 3.1), n_z layers of height H/n_z (d = 3; n_z = 1 and H
 *                ignored in 2D); at theta = 0 both partitions start at angle phi0
 *   iface_rotor, iface_stator  [n_z][n_R] cell ids: entry (l, j) is the cell
 *                of z-layer l spanning angles [phi0 + j D, phi0 + (j+1) D],
 *                D = 2 pi / n_R, at theta = 0.  Interface cells are oriented
 *                xi_0 radial outward, xi_1 counter-clockwise angle, xi_2 = z;
 *                the interface face is xi_0 = 1 (rotor) / xi_0 = 0 (stator).
 * The library copies everything; the caller may free its arrays on return.
 * Errors: MF_ERR_ARG for null pointers, d/k out of range, ids out of range,
 * wall values above 2.
 */
mf_status mf_mesh_from_arrays(int d, int k, int64_t n_nodes, const double* x0,
                              const uint8_t* node_side, const uint8_t* wall,
                              int64_t n_cells, const int32_t* cells, const uint8_t* cell_side,
                              double R, int n_R, int n_z, double H, double phi0,
                              const int32_t* iface_rotor, const int32_t* iface_stator,
                              mf_mesh** out);
/* mf_mesh_from_arrays_ex: the same with n_R_stator stator interface cells per
 * layer (iface_stator [n_z][n_R_stator]), possibly different from the rotor's
 * n_R (a general interface; the paper restricts itself to equal partitions,
 * Section 3.1 and its conclusions).  n_R_stator = n_R is mf_mesh_from_arrays. */
mf_status mf_mesh_from_arrays_ex(int d, int k, int64_t n_nodes, const double* x0,
                                 const uint8_t* node_side, const uint8_t* wall,
                                 int64_t n_cells, const int32_t* cells, const uint8_t* cell_side,
                                 double R, int n_R, int n_R_stator, int n_z, double H, double phi0,
                                 const int32_t* iface_rotor, const int32_t* iface_stator,
                                 mf_mesh** out);
void mf_mesh_free(mf_mesh* m);

/* mf_mesh_rotor_stator: generate a merged rotor-stator mesh (Section 3.1: the
 * two grids are built separately and meet on a circle of radius R that both
 * split into n_R = 4 m equal cells).
 *   rotor disk r < R: O-grid of an m x m centre square of half width sq * R and
 *     four ring blocks of m x n_r cells blending the square's sides into the
 *     circle; stator annulus R < r < R_out: n_R x n_s polar cells;
 *   d = 3: both extruded in n_z layers over [0, H]; blades > 0 marks that many
 *     equally spaced radial blades in the rotor (the ring cells of one angular
 *     index, inner three quarters of the rings, middle half of the height) as
 *     walls moving with the rotor (wall = 2).
 * Q_k nodes at the Gauss-Lobatto points of each cell's parameter square, on the
 * blocks' parametric maps (interface nodes exactly on the circle, duplicated
 * per side); cell-local nodes in tensor order, xi_0 fastest; ring and stator
 * cells xi_0 radial outward, xi_1 counter-clockwise.  Walls: r = R_out (and
 * z = 0, H).  The interface cell tables follow mf_mesh_from_arrays.  Errors:
 * MF_ERR_ARG for out-of-range parameters (d, k in 1..5, m, n_r, n_s, n_z >= 1,
 * 0 < R < R_out, H > 0, 0 < sq < 1/sqrt 2, blades in 0..n_R and only in 3D) or
 * more than 2^31 - 1 nodes.
 * mf_mesh_params_defaults: d 3, k 2, m 8, n_r 2, n_s 4, n_z 8, R 0.5, R_out 1,
 * H 1, sq 0.55, phi0 -pi/4, no blades, equal partitions.
 * n_R_stator > 0 gives the stator its own number of interface cells per layer
 * (unequal partitions, beyond the paper's equal-partition restriction).  The
 * operator supports such meshes: its mortar cells are then the n_R +
 * n_R_stator segments per layer between consecutive rotor and stator vertices
 * (see mf_mortar_segments); mf_mesh_coarsen_map and mf_mesh_slab reject them.
 * mf_mesh_sizes / mf_mesh_read: the mesh's sizes and a copy of its arrays into
 * caller HOST buffers sized as in mf_mesh_from_arrays (any pointer may be NULL).
 * mf_mesh_coarsen_map: the parameters of the uniformly coarsened mesh (every
 * block halved along each cell direction; m, n_r, n_s and in 3D n_z must be
 * even, else MF_ERR_ARG) and, when parent / child are not NULL (host, one entry
 * per fine cell), the coarse cell containing each fine cell and its child code
 * (bit r set when the fine cell is the upper half along xi_r), the inputs of
 * mf_mg_attach for the geometric levels of the multigrid (Section 3.4). */
typedef struct {
  int    d, k;
  int    m, n_r, n_s, n_z;
  double R, R_out, H;
  double sq;
  double phi0;
  int    blades;
  int    n_R_stator;   /* stator interface cells per layer; 0 = 4 m (equal partitions, the paper's case) */
} mf_mesh_params;
void mf_mesh_params_defaults(mf_mesh_params* p);
mf_status mf_mesh_rotor_stator(const mf_mesh_params* p, mf_mesh** out);
/* Interface partitions of a mesh: rotor and stator cells per z-layer, layers.
 * iface_stator of mf_mesh_read holds n_z x n_R_stator entries. */
mf_status mf_mesh_interface(const mf_mesh* m, int* n_R_rotor, int* n_R_stator, int* n_z);

/* mf_mortar_segments: the mortar segments of an interface whose rotor has n_R
 * and whose stator has n_Rs equal cells (Section 3.2; the paper's case is
 * n_Rs = n_R): the circle is cut at every rotor vertex theta + 2 pi i / n_R
 * and every stator vertex 2 pi j / n_Rs (angles from the partitions' common
 * origin); each piece longer than 1e-13 is a segment with its start angle in
 * [0, 2 pi), its length, and the rotor and stator cells it lies in.  HOST
 * arrays of max_out entries (any may be NULL); *count receives the number of
 * segments (at most n_R + n_Rs).  MF_ERR_ARG for bad sizes, a non-finite
 * angle, or max_out < *count (nothing beyond max_out is written).  Host code. */
mf_status mf_mortar_segments(int n_R, int n_Rs, double theta, int max_out, double* start, double* length,
                             int32_t* rotor_cell, int32_t* stator_cell, int* count);
mf_status mf_mesh_sizes(const mf_mesh* m, int* d, int* k, int64_t* n_nodes, int64_t* n_cells, int* n_R, int* n_z);
mf_status mf_mesh_read(const mf_mesh* m, double* x0, uint8_t* node_side, uint8_t* wall, int32_t* cells,
                       uint8_t* cell_side, int32_t* iface_rotor, int32_t* iface_stator);
mf_status mf_mesh_coarsen_map(const mf_mesh_params* fine, mf_mesh_params* coarse, int32_t* parent, uint8_t* child);

/* ---------------------------------------------------------------- z-slab partition (multi-GPU)
 * mf_mesh_slab: part `part` of a partition of a 3D mesh into n_parts z-slabs
 * (1 <= n_parts <= n_z), the counterpart of the paper's mesh decomposition
 * (Section 3.3).  Part p owns the z-layers [floor(p n_z / P), floor((p+1)
 * n_z / P)) (a cell's layer from the mean z of its nodes).  The rotation axis
 * is z, so every mortar pair lies in one layer and stays on one part at every
 * rotor angle.  Parts p and p+1 share the node plane between their layers:
 * an operator applied on each part gives partial sums on its shared planes,
 * and one exchange per neighbour completes them (mf_halo_pack on the sender,
 * mf_halo_add on the receiver).  Outputs (HOST, each may be NULL):
 *   out        the slab as a mesh of its own (local node numbering in
 *              ascending global id; its layers' interface rows; height
 *              H (l1 - l0) / n_z, so the layer height is unchanged);
 *   info       sizes: nodes, cells, layer range, shared-plane node counts;
 *   node_global [n_nodes] global id of each local node;
 *   lo, hi     [n_lo], [n_hi] local ids of the nodes shared with part p-1 /
 *              p+1, in ascending global id (the neighbour lists the same
 *              nodes in the same order); lo_wall, hi_wall: 1 for wall nodes.
 * Call once with out and the arrays NULL to size the arrays.  Errors:
 * MF_ERR_ARG (2D mesh, part out of range, n_parts > n_z, unequal interface
 * partitions, an interface cell outside its layer's part).  Host code. */
typedef struct {
  int64_t n_nodes, n_cells;
  int     layer_begin, layer_end;
  int     n_lo, n_hi;
} mf_slab_info;
mf_status mf_mesh_slab(const mf_mesh* m, int n_parts, int part, mf_mesh** out, mf_slab_info* info,
                       int64_t* node_global, int32_t* lo, int32_t* hi, uint8_t* lo_wall, uint8_t* hi_wall);
/* Halo exchange kernels (device pointers, asynchronous on `stream`):
 * mf_halo_pack: buf[i][f] = y[idx[i]][f] for i < n, f < nf (the partial
 * rows of a shared plane, to send);  mf_halo_add: y[idx[i]][f] += buf[i][f]
 * (the neighbour's partial rows), except the velocity components of wall
 * nodes (wall[i] = 1; wall may be NULL), whose identity rows both parts hold
 * already.  MF_ERR_ARG for null pointers or nf < 1. */
mf_status mf_halo_pack(const double* y, const int32_t* idx, int64_t n, int nf, double* buf, void* stream);
mf_status mf_halo_add(double* y, const int32_t* idx, const uint8_t* wall, int64_t n, int nf, const double* buf,
                      void* stream);
/* Krylov vector kernels for a solver that spans the parts (the z-slab
 * FGMRES of the Python package: these kernels do its vector arithmetic, the
 * caller all-reduces the dot products).  FP64 device vectors of length n;
 * V holds m vectors, vector i at V + i ldv.  Asynchronous on `stream`.
 *   mf_vec_dots:  out[i] = sum_j w[j] V_i[j] x[j], i < m (w NULL: weights
 *                 1; the weights count each shared row once over the parts);
 *                 out: device, m doubles; fixed summation order.
 *   mf_vec_maxpy: y += sign sum_{i<m} c[i] V_i (c: device, m doubles).
 *   mf_vec_axpby: y = a x + b y (host scalars).
 *   mf_vec_mul:   z = d * v entrywise (an inverse-diagonal preconditioner).
 * MF_ERR_ARG for n < 0, m < 1 or m > 256, ldv < n, or a null pointer. */
mf_status mf_vec_dots(int64_t n, const double* V, int64_t ldv, int m, const double* x, const double* w, double* out,
                      void* stream);
mf_status mf_vec_maxpy(int64_t n, const double* V, int64_t ldv, int m, const double* c, double sign, double* y,
                       void* stream);
mf_status mf_vec_axpby(int64_t n, double a, const double* x, double b, double* y, void* stream);
mf_status mf_vec_mul(int64_t n, const double* d, const double* v, double* z, void* stream);

/* ---------------------------------------------------------------- per-call metrics log
 * mf_log_open(path): from now on the mesh generator, mf_solve_step,
 * mf_batch_solve_step, mf_run_transient, mf_autotune and the checkpoint calls
 * each append one JSON object per line to `path` (created if missing): the
 * call name, its status, sizes, iteration counts, the residual history of a
 * solve and the wall seconds.  NULL or "" turns the log off (the default).
 * Process-wide; records of concurrent calls are written whole (a mutex).
 * MF_ERR_ARG when the file cannot be opened for appending.  Not in the paper
 * (the paper reports iteration counts and wall times per run). */
mf_status mf_log_open(const char* path);

/* ---------------------------------------------------------------- checkpoint / resume
 * A time-dependent run (mf_run_transient or the caller's own BDF loop) is
 * fully described by u^n, u^{n-1} (BDF2), the rotor angle and the step/time
 * counters.  mf_checkpoint_write stores them in one file: a one-line JSON
 * header (format "mf-checkpoint-1", d, k, sizes, an FNV-1a fingerprint of the
 * mesh's cells, coordinates, sides and walls, bdf, step, t, theta, dt, nu,
 * omega) followed by the raw little-endian FP64 arrays u^n and, for BDF2,
 * u^{n-1}, each [n_nodes][d+1] in the library's layout.  The file is written
 * to path.tmp and renamed, so an interrupted write leaves the old checkpoint.
 * mf_checkpoint_read checks the format, the mesh fingerprint, the sizes and
 * the file length, fills info and copies the arrays into u_n / u_nm1 (either
 * may be NULL to read the header only).  Both take HOST buffers (copy device
 * state to the host first) and touch no GPU.  Errors: MF_ERR_ARG (null
 * pointers, bdf not 1/2, non-finite values, I/O failure, another mesh, a
 * malformed or truncated file).  Not in the paper (no restart facility is
 * described); it lets the 50-step transient of the large cylinder resume. */
typedef struct {
  int     bdf;      /* 1 or 2: number of state arrays stored */
  int64_t step;     /* time steps taken */
  double  t;        /* simulated time */
  double  theta;    /* rotor angle at t */
  double  dt, nu, omega;
} mf_checkpoint_info;
mf_status mf_checkpoint_write(const char* path, const mf_mesh* m, const mf_checkpoint_info* info, const double* u_n,
                              const double* u_nm1);
mf_status mf_checkpoint_read(const char* path, const mf_mesh* m, mf_checkpoint_info* info, double* u_n, double* u_nm1);

/* ---------------------------------------------------------------- options */
typedef struct {
  double penalty_F;   /* F of Eq. EqPenalty (default 1) */
  int    reserved[8];
} mf_options;

/* mf_create: set up the operator on the current CUDA device (synchronising).
 * Parameters of the ALE Navier-Stokes problem of Eq. EqNS (nu, the rotor's
 * omega) and of its discretisation: Q_k shape functions (Eq.
 * Eq-shape-functions), the time step that enters tau (Eq. Eq-stab-param) and
 * the BDF order of the time integration (Section 4: BDF2 in the transient
 * examples), the penalty factor F of Eq. EqPenalty in opt.
 *   k must equal the mesh degree; nu >= 0 kinematic viscosity; omega rotor
 *   angular velocity about e_z; dt > 0 time step of BDF order bdf (1|2), or
 *   dt = 0 for the steady operator (time terms and the (1/dt)^2 part of tau
 *   dropped).  opt may be NULL (defaults).  The rotor starts at theta = 0.
 * Errors: MF_ERR_ARG (bad parameters), MF_ERR_OOM, MF_ERR_CUDA. */
mf_status mf_create(const mf_mesh* m, int k, double nu, double omega, double dt, int bdf,
                    const mf_options* opt, mf_handle* out);
mf_status mf_destroy(mf_handle h);
const char* mf_last_error(mf_handle h);
mf_status mf_sizes(mf_handle h, int64_t* n_nodes, int64_t* n_dofs, int64_t* n_cells,
                   int64_t* n_mortar_cells);

/* Rotor angle (Section 3.1 rotation, Section 3.2 mortar cells): rotates the
 * rotor nodes to x = R(theta) x0 and rebuilds the mortar points.  Called by
 * mf_set_linearization; exposed for drivers that move the rotor alone. */
mf_status mf_set_angle(mf_handle h, double theta, void* stream);

/* Current node coordinates, device out [n_nodes][d]. */
mf_status mf_node_coords(mf_handle h, double* xyz_out, void* stream);

/* Dirichlet values g (device [n_nodes][d], read at stationary wall nodes,
 * wall = 1), NULL = zero.  Walls moving with the rotor (wall = 2) always take
 * the rigid rotation omega e_z x x of the current angle instead. */
mf_status mf_dirichlet(mf_handle h, const double* g, void* stream);

/* BDF history (Section 4: backward-difference time integration of the time
 * derivative of Eq. EqNS; device [n_nodes][d] each; u_nm1 ignored/NULL for
 * BDF1): stores h_t = (alpha_1 u^n + alpha_2 u^{n-1}) / dt with alpha =
 * (1, -1) for BDF1 and (3/2, -2, 1/2) for BDF2 at constant dt. */
mf_status mf_set_history(mf_handle h, const double* u_n, const double* u_nm1, void* stream);

/* Linearisation state u*, p* of the Newton Jacobian (Section 2.3 blocks
 * A-hat..D-hat) at rotor angle theta (rotation, Section 3.1; mortar cells and
 * points, Section 3.2).  up_star: device [n_nodes][d+1] FP64.  The call
 * rotates, remaps the mortar, and caches per Gauss point the geometry and the
 * frozen-tau linearisation (advection u*-u_ALE, grad u*, strong residual R*,
 * tau) in FP64 and an FP32 copy.  Must precede mf_apply_jacobian/mf_diagonal. */
mf_status mf_set_linearization(mf_handle h, const double* up_star, double theta, void* stream);

/* Residual r = F-hat*_NS(up) (volume + mortar terms, FP64), r = u - g on wall
 * velocity DoFs.  up, r: device [n_nodes][d+1] FP64; tau from up itself. */
mf_status mf_residual(mf_handle h, const double* up, double* r, void* stream);

/* y = J x at the current linearisation: the Jacobian of the residual of Eq.
 * Eq-NSweakWmortar with the SUPG/PSPG terms of Eq. Eq-NSweakComplete, i.e.
 * the blocks A-hat..D-hat of Section 2.3 (tau frozen) plus the mortar face
 * terms of Eqs. EqMortarPre, EqMortarDiff, EqMortarMass.  prec MF_FP64: x, y double; MF_FP32:
 * x, y float (FP32 cache); MF_DF64: x, y double, double-float arithmetic (its
 * cache copy is built on the first such call after each linearisation).  x entries on wall velocity DoFs are ignored as
 * inputs and copied to y (identity rows/columns).  x and y must not alias.
 * Asynchronous on `stream`: the mortar kernel runs on a side stream the
 * handle owns, forked from `stream` and joined back to it with events, so
 * the call is ordered on `stream` like a single launch and can be captured
 * into a CUDA graph from `stream`; one handle must not run two applies on
 * different streams at the same time. */
mf_status mf_apply_jacobian(mf_handle h, const void* x, void* y, mf_precision prec, void* stream);

/* diag(J) at the current linearisation (volume and mortar parts, Algorithm 1;
 * 1 on wall velocity DoFs), device [n_nodes][d+1] of the given precision. */
mf_status mf_diagonal(mf_handle h, void* diag_out, mf_precision prec, void* stream);

/* ---------------------------------------------------------------- solve */
/* Preconditioners of the outer FGMRES:
 *   MF_PC_JACOBI     z = D^-1 v
 *   MF_PC_CHEBYSHEV  degree-s Chebyshev-Jacobi polynomial on [cheb_lo, 1.1] * lambda_max(D^-1 J)
 *   MF_PC_GMRES      inner_iters steps of Jacobi-preconditioned GMRES (zero initial guess, CGS2)
 *   MF_PC_MG         one V-cycle of the multigrid hierarchy attached with mf_mg_attach (Section 3.4):
 *                    mg_smooth GMRES-Jacobi steps before and after the coarse correction on each
 *                    level, mg_coarse_iters GMRES-Jacobi steps on the coarsest level; in pc_precision
 * each applied with pc_precision operator applies (MF_FP32: the FP32 cache). */
typedef enum { MF_PC_JACOBI = 0, MF_PC_CHEBYSHEV = 1, MF_PC_GMRES = 2, MF_PC_MG = 3 } mf_pc_kind;

/* Smoother of the MF_PC_MG levels (Section 3.4: inverse diagonal or additive
 * Schwarz), each as the right preconditioner of the levels' smoothing GMRES:
 *   MF_SMOOTH_JACOBI  the inverse diagonal (default);
 *   MF_SMOOTH_ASM     additive Schwarz with cell patches: per cell the local
 *                     matrix of Algorithm 2 (the cell's volume element matrix
 *                     plus the own-side blocks of the mortar segments it meets,
 *                     reconstructed column by column from the matrix-free
 *                     kernels; wall velocity rows and columns identity),
 *                     inverted once per linearisation in FP32; z = sum over
 *                     cells of the local solves, each DoF's corrections averaged
 *                     over the cells sharing it.  pc_precision must be MF_FP32.
 *                     Levels whose local matrices exceed 108 rows (3D Q3 and
 *                     up) keep the inverse diagonal.  Needs (d+1)^2 (k+1)^(2d)
 *                     floats per cell on every level (6.1 GB for 131k Q2 hexes). */
typedef enum { MF_SMOOTH_JACOBI = 0, MF_SMOOTH_ASM = 1 } mf_smoother_kind;

/* mf_asm_setup: the additive Schwarz local matrices of this handle at its
 * current linearisation (Algorithm 2, as above) and their FP32 inverses --
 * what MF_SMOOTH_ASM does on every level inside mf_solve_step; *n_bad_pivots
 * (host, may be NULL; synchronising when given) receives the number of pivots
 * below 1e-30 that the inversion replaced.  mf_asm_apply: z = ASM(r) with
 * those inverses, r and z FP32 device [n_nodes][d+1] (must not alias).
 * Errors: MF_ERR_ARG (local matrices over 108 rows, null or aliased
 * pointers), MF_ERR_STATE (no linearisation; apply before setup).  The first
 * setup allocates the local matrices. */
mf_status mf_asm_setup(mf_handle h, int* n_bad_pivots, void* stream);
mf_status mf_asm_apply(mf_handle h, const float* r, float* z, void* stream);

typedef struct {
  double newton_rtol;   /* stop when ||R||_2 <= newton_rtol ||R_0||_2 (default 1e-8) */
  double newton_atol;   /* or ||R||_2 <= newton_atol (default 0) */
  int    max_newton;    /* default 20 */
  double lin_rtol;      /* FGMRES relative tolerance per Newton step (default 1e-4) */
  int    restart;       /* FGMRES restart length (default 50, max 200) */
  int    max_lin_iters; /* total FGMRES iterations per Newton step (default 500) */
  int    pc;            /* mf_pc_kind (default MF_PC_GMRES) */
  int    pc_precision;  /* mf_precision of the preconditioner applies (default MF_FP32) */
  int    cheb_degree;   /* Chebyshev degree (default 4) */
  double cheb_lo;       /* lower end of the Chebyshev interval as a fraction of lambda_max (default 0.1) */
  double theta;         /* rotor angle of this step */
  int    inner_iters;   /* MF_PC_GMRES inner Krylov dimension (default 20, max 120) */
  int    line_search;   /* halve the Newton step up to this many times while ||R|| does not decrease (default 6) */
  int    mg_smooth;     /* MF_PC_MG smoothing steps per level (default 4) */
  int    mg_coarse_iters; /* MF_PC_MG coarsest-level GMRES dimension (default 40) */
  int    deflate_pressure; /* 1: at each FGMRES restart, minimise the residual along J e_p (the
                              constant pressure, a near null vector); 0: off (default 0) */
  int    use_graphs;    /* MF_PC_MG: 1 = capture one V-cycle per solve as a CUDA graph on a library
                           stream and replay it for every preconditioner application (default 1);
                           0 = launch eagerly.  Graphs are skipped while profiling is enabled. */
  int    outer_precision; /* Jacobian applies of the outer FGMRES: MF_FP64 (default) or MF_DF64
                             (FP64-accurate double-float on the FP32 pipes) */
  int    batch_fallback;  /* mf_batch_solve_step only: 1 = an instance still above tolerance after the
                             batched iterations (or stopped by the step safeguard) continues alone with
                             mf_solve_step (restart max(restart, 30), lin_rtol, max(max_newton, 40)
                             iterations, MG smoothing max(2 mg_smooth, 8), its own graphs) from its last
                             iterate, to the same absolute target newton_rtol ||R_0|| (default 1) */
  int    mg_smoother;     /* mf_smoother_kind of MF_PC_MG (default MF_SMOOTH_JACOBI) */
  double step_rtol;       /* mf_run_transient only: > 0 turns on per-step convergence control (after
                             newton_iters iterations, one more at a time, up to max_newton per step,
                             while ||R|| > step_rtol ||R_0|| of the step); 0 = fixed iterations (default) */
  int    smooth_cgs_passes; /* MF_PC_MG: classical Gram-Schmidt passes of the smoothing GMRES on every
                               level, 1 or 2 (default 2); the coarse solve always takes 2 */
} mf_solver_opts;

typedef struct {
  int    newton_iters;
  int    lin_iters_total;
  int    lin_iters[64];       /* per Newton step (first 64) */
  double res_norm[65];        /* ||R||_2 before each Newton step and at exit */
  double lambda_max;          /* estimated spectral radius of D^-1 J */
  double seconds;             /* wall time of the solve (host clock) */
  int    status;              /* mf_status of the solve */
  int    fallback_newton_iters; /* mf_batch_solve_step: Newton iterations of the adaptive fallback
                                   (included in newton_iters; 0 when none ran) */
  int    fallback_restarted;  /* mf_batch_solve_step: 1 when the fallback started over from the
                                 initial guess (res_norm then continues from ||R_0|| again) */
} mf_solve_report;

void mf_solver_defaults(mf_solver_opts* o);

/* One nonlinear step: Newton on R(up) = 0 (Eq. Eq-Newton-method: solve
 * J [du, dp] = -R, update, repeat) at angle so->theta, each linear
 * system by right-preconditioned FGMRES with FP64 residual, Jacobian applies
 * and CGS2 orthogonalisation.  up: device [n_nodes][d+1] FP64, in: initial
 * guess, out: solution.  Synchronising (reads convergence data back);
 * rep (host) may be NULL.  Returns MF_ERR_NOT_CONVERGED / MF_ERR_BREAKDOWN /
 * MF_ERR_NAN on failure (up then holds the last iterate). */
mf_status mf_solve_step(mf_handle h, double* up, const mf_solver_opts* so, mf_solve_report* rep,
                        void* stream);

/* ---------------------------------------------------------------- energy budget and wall loads
 * (Section 4.5.2 energy balance, Section 4.4.2 torque analysis)
 *
 * mf_kinetic_energy: ke_dev (device double) = 1/2 int |u|^2 over the mesh at
 * the current geometry (Gauss rule of the operator); needs the geometry cache
 * of a previous mf_set_linearization.  Asynchronous.
 *
 * mf_energy: the energy budget terms of up at the current geometry, out_dev
 * (device double[3]): [0] 1/2 int |u|^2; [1] nu int grad u : grad u (the
 * dissipation of the Laplacian form of the viscous term, Eq. 1); [2] nu int
 * (grad u + grad u^T) : grad u (the paper's -tau : grad u with the deviatoric
 * stress tau = -nu (grad u + grad u^T)).  Gauss rule of the operator, wall
 * values included.  Needs the geometry cache.  Asynchronous.
 *
 * mf_wall_loads: loads the walls exert on the fluid, from the consistent
 * reactions r = the volume + mortar residual rows of up without the Dirichlet
 * replacement (on a wall node i, r_i = int_wall t . phi_i with t the wall's
 * traction on the fluid).  For each group g of wall nodes, out (device
 * double[n_groups][d+2]): [g][0..d-1] force sum_i r_i, [g][d] torque about
 * the z axis sum_i (x_i x r_i) . e_z, [g][d+1] power sum_i r_i . u_i.
 * group: device uint8 [n_nodes], the group of each wall node (values >=
 * n_groups skipped, non-wall nodes ignored), 1 <= n_groups <= 16; or NULL with
 * n_groups = 2: group 0 = stationary walls (wall = 1), 1 = walls moving with
 * the rotor (wall = 2, e.g. the impeller).  The torque the fluid exerts on the
 * impeller is minus its group's torque, its power number 2 pi T / (N^2 D^5)
 * (rho = 1).  Uses the history term and angle of the handle; needs the
 * geometry cache.  The first call allocates an n_dofs scratch vector.
 * Asynchronous.
 */
#define MF_MAX_LOAD_GROUPS 16
mf_status mf_kinetic_energy(mf_handle h, const double* up, double* ke_dev, void* stream);
mf_status mf_energy(mf_handle h, const double* up, double* out_dev, void* stream);
mf_status mf_wall_loads(mf_handle h, const double* up, const uint8_t* group, int n_groups, double* out,
                        void* stream);

/* ---------------------------------------------------------------- transient driver
 * mf_run_transient: n_steps BDF steps (the handle's dt and BDF order) starting
 * at rotor angle theta0, the rotor advancing by omega*dt per step (rotation and
 * mortar remap every step, Sections 3.1-3.2).  Each step: history term from
 * (u_n, u_nm1), newton_iters Newton iterations from u_n, each with FGMRES of
 * fixed dimension krylov_iters (CGS2, device-side least squares) and the
 * preconditioner of `so` (MF_PC_JACOBI, MF_PC_GMRES or MF_PC_MG with its
 * precision; Chebyshev is not supported); then u_nm1 <- u_n, u_n <- solution.
 * No step waits on the host, so with use_graph = 1 one step is captured as a
 * CUDA graph (on a library stream) and replayed n_steps times on `stream`.
 * With so->step_rtol > 0 (convergence control) a step is three graphs: the
 * start with newton_iters iterations, then one more iteration at a time while
 * ||R|| > step_rtol ||R_0|| of the step (at most so->max_newton iterations in
 * all; the host reads two norms per check), then the end of the step.
 * u_n, u_nm1: device [n_nodes][d+1] FP64 (u_nm1 unused for BDF1).  On return
 * (synchronising) rec_host[0..n_steps] (host, may be NULL) holds the record of
 * the initial state and of each step's solution: energy terms as mf_energy,
 * wall loads as mf_wall_loads with the default groups (at the step's history
 * term, so the torque includes the BDF inertia of the wall rows) and the
 * step's residual reduction ||R_end|| / ||R_start|| (0 in record 0).  The
 * numerical dissipation of the energy balance follows on the host:
 * eps_n T-bar = power - dissipation_sym - dE/dt (Section 4.5.2).  Errors:
 * MF_ERR_ARG (dt = 0, counts out of range), MF_ERR_STATE (MG without levels). */
typedef struct {
  double kinetic_energy;      /* 1/2 int |u|^2 */
  double dissipation;         /* nu int grad u : grad u */
  double dissipation_sym;     /* nu int (grad u + grad u^T) : grad u */
  double torque_still;        /* z torque of the stationary walls on the fluid */
  double torque_moving;       /* z torque of the walls moving with the rotor on the fluid */
  double power;               /* power of all walls on the fluid */
  double residual_reduction;  /* ||R_end|| / ||R_start|| of the step */
  double newton_iters;        /* Newton iterations the step took (0 in record 0) */
} mf_step_record;
mf_status mf_run_transient(mf_handle h, double* u_n, double* u_nm1, int n_steps, double theta0, int newton_iters,
                           int krylov_iters, const mf_solver_opts* so, int use_graph, mf_step_record* rec_host,
                           void* stream);

/* ---------------------------------------------------------------- no-allocation solve
 * mf_solve_step_static: the same Newton / FGMRES step as mf_solve_step, for
 * callers that must not allocate device memory during the solve -- e.g. a
 * serving process whose own allocator has reserved the device memory up front
 * (a cudaMalloc from the library would fail or break its accounting), or a
 * control loop that cannot afford cudaMalloc's implicit device-wide
 * synchronisation.  (The paper has no counterpart: this is a deployment
 * variant of the solver's workspace handling.)
 *
 * The Krylov workspace lives in one file-scope device array of
 * MF_STATIC_WS_DOUBLES doubles (32 MiB) that every GPU which loads libmf.so
 * holds until the process exits.  The call allocates no device or pinned host
 * memory: no cudaMalloc, cudaFree, cudaMallocHost or event creation.  Limits:
 *   - pc must be MF_PC_JACOBI with pc_precision MF_FP64 and outer_precision MF_FP64;
 *   - (2*restart + 10) * n_dofs + 3*(restart + 2) + (restart + 2) * MF_REDUCE_BLOCKS
 *     doubles must fit in the array, otherwise MF_ERR_ARG with a message (e.g.
 *     2D workloads of ~16k DoFs with restart <= 100); MF_REDUCE_BLOCKS is the
 *     number of partial sums of the library's dot-product kernels (the same
 *     constant sizes them);
 *   - per-kernel profiling (mf_profile) must be off (MF_ERR_STATE otherwise).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and it keeps the previous call's contents; the
 * solve initialises everything it reads.  Calls that overlap on the GPU (two
 * streams, two threads, two handles) race on the array: serialise them.
 * Arguments, results and errors are those of mf_solve_step. */
#define MF_STATIC_WS_DOUBLES (4u << 20)
#define MF_REDUCE_BLOCKS 592
mf_status mf_solve_step_static(mf_handle h, double* up, const mf_solver_opts* so, mf_solve_report* rep,
                               void* stream);

/* ---------------------------------------------------------------- batched instances
 * Several independent operator instances (same d and k; different meshes,
 * nu, omega, angles) applied in one persistent launch per kernel kind: the
 * cells (and mortar half-cells) of all instances form one device tile queue
 * that a grid sized to the GPU drains, so uneven instance sizes balance.
 * mf_batch_create keeps the handles (caller-owned, at most 64) and allocates
 * the tile tables; mf_batch_apply_jacobian takes HOST arrays of n device
 * pointers (xs[i] -> ys[i], each instance's own layout and precision prec) and
 * is asynchronous on `stream`, except that it waits for the previous call's
 * table upload to finish before refilling the staging buffer.  Errors:
 * MF_ERR_ARG (null or aliased pointers, mixed d/k, n out of range),
 * MF_ERR_STATE (an instance without linearisation). */
typedef struct mf_batch mf_batch;
mf_status mf_batch_create(const mf_handle* hs, int n, mf_batch** out);
mf_status mf_batch_destroy(mf_batch* b);
mf_status mf_batch_apply_jacobian(mf_batch* b, const void* const* xs, void* const* ys, mf_precision prec,
                                  void* stream);

/* mf_batch_solve_step: one nonlinear step (Eq. Eq-Newton-method) of every
 * instance of the batch, each at its own rotor angle thetas[i] (host array)
 * from the initial guess ups[i] (HOST array of n device pointers,
 * [n_nodes_i][d+1] FP64, overwritten by the result).  Each Newton iteration
 * of each instance: linearisation at its iterate (Section 2.3 blocks, frozen
 * tau), Jacobi diagonal (Algorithm 1) in so->pc_precision, multigrid levels
 * for MF_PC_MG (attached with mf_mg_attach), rhs = -R, then FGMRES with a
 * fixed dimension krylov_iters (1..100; CGS2, right preconditioned by so->pc
 * = MF_PC_JACOBI, MF_PC_GMRES or MF_PC_MG; least squares on the device) and
 * a full Newton step.  The outer FGMRES and its Jacobian applies are FP64.
 *   batched = 1: the per-instance work runs on streams forked from `stream`
 *                and the outer Jacobian applies of all instances run as one
 *                persistent launch per kernel kind (one tile queue);
 *   batched = 0: the instances run one after another on `stream`, each with
 *                its own applies (same arithmetic).
 *   use_graph = 1: one Newton iteration of the whole batch is captured as a
 *                CUDA graph (once per call) and replayed.
 * After each iteration the host reads the n residual norms back (one small
 * copy and a synchronisation).  An instance stops iterating once ||R_i|| <=
 * newton_rtol ||R_i,0|| or <= newton_atol (the graph and the tile tables are
 * rebuilt for the remaining ones); the batch stops when none is left or after
 * so->max_newton (<= 64) iterations.  A step that makes ||R_i|| non-finite or
 * ten times the smallest ||R_i|| reached so far is halved from the previous
 * iterate up to so->line_search times until ||R_i|| falls below its previous
 * value, else the instance keeps its previous iterate and stops
 * (line_search = 0: full steps; only a non-finite ||R_i|| stops an instance).  reps (host, n entries, may be NULL): per instance
 * res_norm[0..newton_iters], lin_iters, wall seconds of the call, status.
 * With so->batch_fallback = 1 (default), an instance that has not converged
 * when the batched loop ends continues alone with mf_solve_step (adaptive
 * FGMRES(max(restart, 30)), the same preconditioner with twice the multigrid
 * smoothing steps, at least 8, up to max(max_newton, 40) iterations) until
 * ||R_i|| <= newton_rtol ||R_i,0||: from its last iterate if the batched
 * iterations reached sqrt(newton_rtol) ||R_i,0||, else from its initial guess
 * (a device copy taken at entry); its report then covers both parts
 * (fallback_newton_iters says how many iterations the fallback took).
 * Returns MF_OK when every instance converged, otherwise the first failing
 * instance's status (MF_ERR_NOT_CONVERGED or MF_ERR_NAN; ups then hold the
 * last accepted iterates).  Errors: MF_ERR_ARG (null pointers,
 * non-finite angle, pc = MF_PC_CHEBYSHEV, outer_precision != MF_FP64),
 * MF_ERR_STATE (profiling on, MF_PC_MG without levels).  Synchronising.
 * Not part of the paper, which solves one problem at a time. */
mf_status mf_batch_solve_step(mf_batch* b, double* const* ups, const double* thetas, const mf_solver_opts* so,
                              int krylov_iters, int batched, int use_graph, mf_solve_report* reps, void* stream);
const char* mf_batch_last_error(mf_batch* b);

/* ---------------------------------------------------------------- launch-shape autotuning
 * The FP64 cell Jacobian kernel runs one thread per Gauss point and several
 * cells per block; the 3D Q1, Q2 and Q3 kernels are compiled for three
 * cells-per-block values (Q1: 32 (default), 16, 32; Q2: 9 (default), 4, 16;
 * Q3: 4 (default), 2, 6), other (d, k) for the default only.  The FP32
 * variants of 3D Q1-Q3 are the one-cell-per-lane kernel (32 cells per block;
 * the default from 148 x 32 cells up) and the per-point kernel with its
 * default (the default below that size) and smaller block (Q1: 32, 16; Q2:
 * 9, 4; Q3: 4, 2).  mf_autotune times every variant of the FP64 and of the FP32
 * kernel on this handle's mesh and current linearisation (CUDA events, 3
 * warm-up and 20 timed launches each, on `stream`) and keeps the fastest for
 * this handle's later applies.  res (host, may be NULL) receives two entries,
 * [0] FP64 and [1] FP32.  cache_path (may be NULL): a text file of earlier
 * choices, one line "<gpu name> <d> <k> <n_cells> <64|32> <cells per block>";
 * a matching line is used without timing (from_cache = 1), a new choice is
 * appended.  Needs a linearisation (MF_ERR_STATE otherwise); allocates two
 * temporary vectors; synchronising.  The double-float apply keeps the default.
 * mf_set_cells_per_block forces a variant (cpb = 0: the default); MF_ERR_ARG
 * when no variant with cpb cells per block is compiled for the handle's d, k.
 * Not in the paper (its CPU code vectorises over cell batches instead). */
typedef struct {
  int    n_variants;          /* variants timed (1 when d, k has only the default) */
  int    cells_per_block[3];
  double ms[3];               /* mean kernel time per launch (0 when read from the cache) */
  int    chosen;              /* index into cells_per_block */
  int    from_cache;
} mf_tune_result;
mf_status mf_autotune(mf_handle h, const char* cache_path, mf_tune_result* res, void* stream);
mf_status mf_set_cells_per_block(mf_handle h, mf_precision prec, int cpb);

/* ---------------------------------------------------------------- multigrid
 * The global-coarsening multigrid of Section 3.4 (geometric and polynomial
 * coarsening) as a hierarchy of operator handles.  mf_mg_attach links `coarse`
 * below `fine` (both created by the caller on the same device, same d, nu,
 * omega, dt, BDF order; the caller keeps both alive while the link is used):
 *   parent == NULL: polynomial coarsening, same cells and node-free layout,
 *                   coarse k = fine k - 1;
 *   parent != NULL: geometric coarsening, equal k; parent[c] (host, [fine
 *                   cells]) is the coarse cell containing fine cell c and bit r
 *                   of child[c] is 1 when c is the upper half of it along xi_r.
 * Coarse levels are linearised at the fine state interpolated to their nodes
 * during mf_solve_step with pc = MF_PC_MG.  Synchronising.
 * mf_mg_prolongate / mf_mg_restrict / mf_mg_interpolate expose the transfers
 * (device FP64 vectors in the interleaved layout of each level):
 *   prolongate: x_fine = P x_coarse (coarse function at the fine nodes);
 *   restrict:   r_coarse = P^T-weighted r_fine (transpose with node multiplicities);
 *   interpolate: u_coarse = fine function at the coarse nodes. */
mf_status mf_mg_attach(mf_handle fine, mf_handle coarse, const int32_t* parent, const uint8_t* child);
mf_status mf_mg_prolongate(mf_handle fine, const double* x_coarse, double* x_fine, void* stream);
mf_status mf_mg_restrict(mf_handle fine, const double* r_fine, double* r_coarse, void* stream);
mf_status mf_mg_interpolate(mf_handle fine, const double* u_fine, double* u_coarse, void* stream);

/* ---------------------------------------------------------------- profiling
 * Per-kernel CUDA-event timers.  When enabled, every kernel the operator calls
 * launch is bracketed by events on its launch stream; mf_profile_read
 * synchronises on those events and returns, per kernel kind, the number of
 * launches and the summed device milliseconds since the last reset.  While
 * profiling is on, a Jacobian apply runs its mortar kernel after the cell
 * kernel on the caller's stream (otherwise the two run side by side on two
 * streams), so that each kernel's events bracket that kernel alone.
 * Kinds: 0 cell Jacobian FP64, 1 cell Jacobian FP32, 2 mortar FP64, 3 mortar
 * FP32, 4 cell residual, 5 cell linearisation, 6 Dirichlet rows, 7 diagonal. */
#define MF_PROF_KINDS 8
typedef struct {
  int64_t launches[MF_PROF_KINDS];
  double  ms[MF_PROF_KINDS];
} mf_profile_t;
mf_status mf_profile(mf_handle h, int enable);           /* enable/disable, resets counters */
mf_status mf_profile_read(mf_handle h, mf_profile_t* out); /* synchronising */

/* mf_fma_peak: the measured FMA issue rate of the current device in FP64
 * (prec = MF_FP64) or FP32 (MF_FP32), the denominator of the ALU roofline that
 * bounds the cell and mortar kernels.  One hand-written kernel of independent
 * FMA chains (8 per thread, 2048 threads per SM, every SM) is launched twice
 * to warm up and five times between CUDA events on `stream`; *tflops receives
 * 2 x FMAs / seconds / 1e12 and ms_out (host, may be NULL) the mean launch time.
 * Synchronising; allocates one small scratch buffer.  MF_ERR_ARG for another
 * prec or a null tflops, MF_ERR_CUDA on a failed launch.  Not in the paper
 * (a measurement aid: the paper reports no roofline). */
mf_status mf_fma_peak(int prec, double* tflops, double* ms_out, void* stream);

/* mf_contract_probe: the interpolation stage of the 3D Q2 cell kernel (nodal
 * values of the four fields -> values and the three first reference
 * derivatives at the 27 Gauss points, Section 3.1 sum factorisation) as a
 * compute-only kernel, to measure whether these batched contractions are
 * dense enough for the tensor cores.  Each of `blocks` CTAs loads its tile of
 * 32 cells x 4 fields into shared memory once and contracts it `reps` times.
 *   variant 0: FP32 FMA, sum-factorised (729 FMAs per field and cell);
 *   variant 1: tcgen05.mma kind::tf32, the tile as one dense product
 *              [128 rows = field x cell] x [32 = nodes, 27 used] against the
 *              Kronecker basis [112 outputs, 108 used] (2916 MACs per field and
 *              cell), accumulator in TMEM (double-buffered), tcgen05.ld back;
 *   variant 2: as 1 with hi/lo TF32 splits of both operands and three
 *              products per step (FP32-level accuracy).
 * u   : device, [blocks][27 nodes][4 fields][32 cells] floats; node
 *       a = ax + 3 ay + 9 az (Gauss-Lobatto nodes of mf_mesh cells).
 * out : device; reps == 1: [blocks][108][4][32], output n = q (value at Gauss
 *       point q = qx + 3 qy + 9 qz) or 27 (1 + d) + q (d/dxi_d there);
 *       reps > 1: [blocks][4][32] sums of all outputs over the repetitions.
 * err : device int (variants 1, 2), set to 1 when a wait on the tensor core
 *       ran out (the outputs are then invalid); never cleared here.
 * Asynchronous on `stream`; the caller times it.  MF_ERR_ARG for a bad
 * variant, blocks < 1, reps < 1 or a null pointer.  Not in the paper (a
 * measurement aid). */
mf_status mf_contract_probe(int variant, int blocks, int reps, const float* u, float* out, int* err, void* stream);

#ifdef __cplusplus
}
#endif
#endif
