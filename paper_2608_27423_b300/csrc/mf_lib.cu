// C ABI of the rotor-stator operator library: context set-up, operator calls
// and the Newton / FGMRES solve.  See include/mf.h for the contract.
#include <cuda_runtime.h>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>
#include <algorithm>

#include "../../include/mf.h"
#include "mf_cell.cuh"
#include "mf_lane.cuh"
#include "mf_mortar.cuh"
#include "mf_small.cuh"
#include "mf_pmg.cuh"

using namespace mf;

#ifndef MF_OVERLAP_MORTAR
#define MF_OVERLAP_MORTAR 7   // precisions whose apply runs the mortar beside the cell kernel: 1 FP64, 2 FP32, 4 DF64
#endif
#ifndef MF_OVERLAP_ORDER
// 1: the cell kernel is launched first and the mortar on a low-priority side
//    stream fills the room its blocks leave on each SM; 0: the mortar first, on
//    a high-priority side stream
#define MF_OVERLAP_ORDER 1
#endif

#include "mf_log.inc"

struct mf_mesh {
  int d, k;
  int64_t nn, nc;
  std::vector<double> x0;
  std::vector<uint8_t> node_side, wall, cell_side;
  std::vector<int32_t> cells;
  double R, H, phi0;
  int n_R, n_z;
  int n_Rs = 0;            // stator interface cells per layer (0: equal to n_R)
  std::vector<int32_t> ifr, ifs;
};

struct Workspace {
  int m = 0;                 // restart length allocated
  double* V = nullptr;       // [m+1][n]
  double* Z = nullptr;       // [m][n]
  double* w = nullptr;       // [n]
  double* r = nullptr;       // [n] residual / rhs
  double* dx = nullptr;      // [n]
  double* hcol = nullptr;    // [m+2] device column of H (and scratch)
  double* part = nullptr;    // [m+2][nb] partial sums
  double* diag64 = nullptr;  // [n]
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  float* f_v = nullptr;      // FP32 Chebyshev vectors
  float* f_x = nullptr;
  float* f_r = nullptr;
  float* f_d = nullptr;
  float* f_t = nullptr;
  float* f_w = nullptr;
  double* c_x = nullptr;     // FP64 Chebyshev vectors
  double* c_r = nullptr;
  double* c_d = nullptr;
  double* c_t = nullptr;
  double* c_v = nullptr;
  double* c_w = nullptr;
  double* pinned = nullptr;  // host [m+2]
  double* utrial = nullptr;  // [n] Newton line-search trial state
  double* ep = nullptr;      // [n] normalised constant-pressure vector
  double* jep = nullptr;     // [n] J e_p
  int mi32 = 0, mi64 = 0;    // inner GMRES dimensions allocated
  int part_cap = 0;          // rows of the partial-sum buffer
  double* hout = nullptr;    // transient driver: outer Hessenberg columns and scalars (65536 doubles)
  double* rec = nullptr;     // per-step records (mf_step_record layout)
  int* rec_count = nullptr;
  int rec_cap = 0;
  float* f_Vin = nullptr;    // [(mi+1) n] inner FP32 Krylov basis
  double* c_Vin = nullptr;   // [(mi+1) n] inner FP64 Krylov basis
  double* hin = nullptr;     // device inner Hessenberg columns
  bool is_static = false;    // a view into mf_solve_step_static's device array: never allocated, grown or freed
};

struct mf_ctx;
struct MgLink {
  mf_ctx* coarse = nullptr;      // next coarser level (caller-owned handle)
  bool hcoarse = false;          // geometric (true) or polynomial coarsening
  int32_t* parent = nullptr;     // [fine cells] coarse cell (h-coarsening)
  uint8_t* child = nullptr;      // [fine cells] upper-half bits
  double* inv_mult64 = nullptr;  // [fine nodes] 1 / number of cells sharing the node
  float* inv_mult32 = nullptr;
  XferTab tab;
};

struct ProfEvent {
  cudaEvent_t a, b;
  int kind;
};

struct mf_ctx {
  bool prof = false;
  int cpb_sel[2] = {0, 0};             // cell Jacobian variant per precision (FP64, FP32); 0 = default
  std::vector<ProfEvent> prof_ev;      // pending event pairs
  std::vector<cudaEvent_t> ev_pool;    // reusable events
  mf_profile_t prof_acc;
  int d = 0, k = 0;
  int64_t nn = 0, nc = 0, ndof = 0;
  double nu = 0, omega = 0, dt = 0, a0dt = 0, inv_dt2 = 0, alpha[3] = {0, 0, 0}, F = 1.0;
  int bdf = 1;
  double R = 0, H = 1, phi0 = 0, theta = 0;
  int n_R = 0, n_z = 1;
  int n_Rs = 0;                        // stator interface cells per layer (equal to n_R in the paper's case)
  int64_t nm = 0, nwall = 0, nif = 0, nif_s = 0;
  SegTable seg{nullptr, nullptr, nullptr, nullptr, nullptr};   // unequal partitions: segments of one layer
  int64_t nmwall = 0;  // the last nmwall entries of `wall` move with the rotor (blade walls)
  bool have_lin = false;
  bool geo_valid = false;              // the cache's geometry fields match the current coordinates
  int smooth_passes = 2;               // Gram-Schmidt passes of this level's smoothing GMRES (solver option)
  bool angle_set = false;              // coordinates, mortar map and face geometry are at the host angle `theta`
  int ncache = 0;
  int nb = 0;  // blocks for reductions
  // device
  double *x0 = nullptr, *x = nullptr;
  uint8_t *node_side = nullptr, *cell_side = nullptr;
  int32_t *cells = nullptr, *wall = nullptr, *ifr = nullptr, *ifs = nullptr;
  double *tau_r = nullptr, *tau_s = nullptr;
  int32_t* mc_cell = nullptr;
  double *mc_tau = nullptr, *mc_xi = nullptr, *mc_cs = nullptr, *mc_w = nullptr;
  double* mg_jinv64 = nullptr;   // face geometry J^-1 at the mortar points [M][2][NP][d][d]
  float* mg_jinv32 = nullptr;
  df* mg_jinvdf = nullptr;       // double-float copies for MF_DF64 (built on demand)
  df* cachedf = nullptr;
  bool df_valid = false;
  double *ht = nullptr, *g = nullptr;
  double* react = nullptr;             // reaction rows scratch of mf_wall_loads [n_dofs]
  double* cache64 = nullptr;
  float* cache32 = nullptr;
  float* asm_E = nullptr;              // additive Schwarz: inverted local matrices [nc][NL][NL] (FP32)
  int* asm_bad = nullptr;              // pivots replaced during the last inversion
  float* inv_mult32 = nullptr;         // 1 / (cells sharing the node)
  bool asm_on = false;                 // the level's smoother uses the local inverses
  float* lcache32 = nullptr;           // 3D, k <= 3: FP32 cache in the lane layout (k_cell_jac_lane)
  int32_t* lcells = nullptr;           // 3D, k <= 3: lane-interleaved cell table
  Workspace ws;
  MgLink mg;
  cudaStream_t cap_stream = nullptr;   // library stream for graph capture
  cudaStream_t side = nullptr;         // high-priority stream the mortar apply runs on beside the cell kernel
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double* d_theta = nullptr;           // device copy of the rotor angle (transient driver)
  bool own_theta = false;              // d_theta allocated by this handle
  bool theta_on_dev = false;           // kernels read the angle from d_theta
  cudaGraphExec_t mg_exec = nullptr;   // captured V-cycle of the current solve
  std::string err;
};

static bool g_tabs_ready[64] = {false};

// Profiling: a scope that records an event pair around one launch when enabled.
static cudaEvent_t pool_get(mf_ctx* h) {
  if (!h->ev_pool.empty()) { cudaEvent_t e = h->ev_pool.back(); h->ev_pool.pop_back(); return e; }
  cudaEvent_t e; cudaEventCreate(&e); return e;
}
struct ProfScope {
  mf_ctx* h; int kind; cudaStream_t st; cudaEvent_t a = nullptr;
  ProfScope(mf_ctx* h_, int kind_, cudaStream_t st_) : h(h_), kind(kind_), st(st_) {
    if (h->prof) { a = pool_get(h); cudaEventRecord(a, st); }
  }
  ~ProfScope() {
    if (h->prof && a) { cudaEvent_t b = pool_get(h); cudaEventRecord(b, st); h->prof_ev.push_back({a, b, kind}); }
  }
};

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      if (h) h->err = std::string(#call) + ": " + cudaGetErrorString(e_);             \
      return e_ == cudaErrorMemoryAllocation ? MF_ERR_OOM : MF_ERR_CUDA;               \
    }                                                                                  \
  } while (0)

static inline cudaStream_t S(void* s) { return (cudaStream_t)s; }
static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
// grid of the grid-stride vector kernels (256 threads): one entry per thread
// up to 8 blocks per SM (short coarse-level vectors are latency-bound: spread
// them over as many SMs as they fill), grid-stride beyond
static inline unsigned vgrid(int64_t n) { return (unsigned)std::min<int64_t>(148 * 8, std::max<int64_t>(1, (n + 255) / 256)); }

static mf_status upload_tables(mf_ctx* h) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 64 && g_tabs_ready[dev]) return MF_OK;
  MfTab<double> t64[MF_KMAX + 1];
  MfTab<float> t32[MF_KMAX + 1];
  MfTab<df> tdf[MF_KMAX + 1];
  std::memset(t64, 0, sizeof(t64));
  std::memset(t32, 0, sizeof(t32));
  std::memset(tdf, 0, sizeof(tdf));
  for (int k = 1; k <= MF_KMAX; ++k) {
    mfhost::build_tab(k, t64[k]);
    mfhost::cast_tab(t64[k], t32[k]);
    mfhost::cast_tab(t64[k], tdf[k]);
  }
  CK(cudaMemcpyToSymbol(c_tab64, t64, sizeof(t64)));
  CK(cudaMemcpyToSymbol(c_tab32, t32, sizeof(t32)));
  CK(cudaMemcpyToSymbol(c_tabdf, tdf, sizeof(tdf)));
  if (dev < 64) g_tabs_ready[dev] = true;
  return MF_OK;
}

// ------------------------------------------------------------------ dispatch
#define MF_DISPATCH(D_, K_, CALL)                                              \
  switch ((D_) * 10 + (K_)) {                                                  \
    case 21: { constexpr int D = 2, K = 1; CALL; } break;                      \
    case 22: { constexpr int D = 2, K = 2; CALL; } break;                      \
    case 23: { constexpr int D = 2, K = 3; CALL; } break;                      \
    case 24: { constexpr int D = 2, K = 4; CALL; } break;                      \
    case 25: { constexpr int D = 2, K = 5; CALL; } break;                      \
    case 31: { constexpr int D = 3, K = 1; CALL; } break;                      \
    case 32: { constexpr int D = 3, K = 2; CALL; } break;                      \
    case 33: { constexpr int D = 3, K = 3; CALL; } break;                      \
    case 34: { constexpr int D = 3, K = 4; CALL; } break;                      \
    case 35: { constexpr int D = 3, K = 5; CALL; } break;                      \
    default: break;                                                            \
  }

template <int D, int K>
static void launch_state(mf_ctx* h, int mode, const double* up, double* dst, cudaStream_t st) {
  StateArgs A;
  A.cells = h->cells; A.nc = h->nc; A.x = h->x; A.cell_side = h->cell_side; A.up = up; A.ht = h->ht;
  A.cache = h->cache64; A.dst = dst; A.nu = h->nu; A.omega = h->omega; A.a0dt = h->a0dt; A.inv_dt2 = h->inv_dt2;
  using C = CellCfg<D, K>;
  const unsigned g = nblk(h->nc, C::CPB);
  ProfScope ps(h, mode == 0 ? 5 : 4, st);
  // the cached geometry is reused while the coordinates have not moved since
  // a cache-writing pass (apply_angle clears geo_valid)
  if (h->geo_valid) {
    if (mode == 0) k_cell_state<D, K, 0, true><<<g, C::THREADS, 0, st>>>(A);
    else if (mode == 1) k_cell_state<D, K, 1, true><<<g, C::THREADS, 0, st>>>(A);
    else k_cell_state<D, K, 2, true><<<g, C::THREADS, 0, st>>>(A);
  } else {
    if (mode == 0) k_cell_state<D, K, 0, false><<<g, C::THREADS, 0, st>>>(A);
    else if (mode == 1) k_cell_state<D, K, 1, false><<<g, C::THREADS, 0, st>>>(A);
    else k_cell_state<D, K, 2, false><<<g, C::THREADS, 0, st>>>(A);
    if (mode != 1) h->geo_valid = true;
  }
}

// The one-cell-per-lane FP32 kernel (mf_lane.cuh) exists for 3D, k = 1..3;
// for those it is the default FP32 variant (index 0, 32 cells per block), and
// the per-point kernel's default and smaller blocks are variants 1 and 2.
static constexpr bool lane_kernel_available(int d, int k) { return d == 3 && k >= 1 && k <= 3; }

// Cells-per-block variants of the cell Jacobian that mf_autotune times, per
// (D, K): index 0 is the default CellCfg<D, K>::CPB (about 256 threads), 1 and
// 2 a smaller and a larger block.  (D, K) without own variants repeat the
// default, so only the 3D Q2 and Q3 kernels are compiled three times.
template <int D, int K> struct CpbVariants {
  static constexpr int n = 1, v1 = CellCfg<D, K>::CPB, v2 = CellCfg<D, K>::CPB;
};
template <> struct CpbVariants<3, 2> { static constexpr int n = 3, v1 = 4, v2 = 16; };   // 108 / 243 / 432 threads
template <> struct CpbVariants<3, 3> { static constexpr int n = 3, v1 = 2, v2 = 6; };    // 128 / 256 / 384 threads
template <> struct CpbVariants<3, 1> { static constexpr int n = 3, v1 = 16, v2 = 32; };  // 128 / 256 / 256 threads
template <int D, int K> static int cpb_variant(int i, bool fp32 = false) {
  if (fp32 && lane_kernel_available(D, K))
    return i == 0 ? LaneCfg<K <= 3 ? K : 1>::CB : i == 1 ? CellCfg<D, K>::CPB : CpbVariants<D, K>::v1;
  return i == 1 ? CpbVariants<D, K>::v1 : i == 2 ? CpbVariants<D, K>::v2 : CellCfg<D, K>::CPB;
}

template <int D, int K, typename T, int CPB>
static void launch_jac_cpb(mf_ctx* h, const T* cache, const typename IO<T>::type* x, typename IO<T>::type* y,
                           cudaStream_t st) {
  k_cell_jac<D, K, T, CPB><<<nblk(h->nc, CPB), CPB * CellCfg<D, K>::NQ, 0, st>>>(h->cells, h->nc, cache, x, y,
                                                                                (T)h->nu, (T)h->a0dt);
}

// Default FP32 variant: the one-cell-per-lane kernel where it exists and the
// mesh gives every SM at least one of its 32-cell blocks, else the per-point
// kernel (small coarse multigrid levels launch faster with its smaller blocks).
static int default_fp32_variant(int d, int k, int64_t nc) {
  return lane_kernel_available(d, k) && nc < 148 * 32 ? 1 : 0;
}

template <int D, int K>
static void launch_lane_cells(mf_ctx* h, cudaStream_t st) {
  if constexpr (D == 3 && K <= 3) {
    const int64_t total = (h->nc + 31) / 32 * LaneCfg<K>::NQ * 32;
    k_lane_cells<K><<<std::min<int64_t>(nblk(total, 256), 148 * 16), 256, 0, st>>>(h->cells, h->nc, h->lcells);
  }
}

template <int D, int K>
static void launch_lane_cache(mf_ctx* h, cudaStream_t st) {
  if constexpr (D == 3 && K <= 3) {
    const int64_t total = (h->nc + 31) / 32 * LaneCache::NF * LaneCfg<K>::NQ * 32;
    k_lane_cache<K><<<std::min<int64_t>(nblk(total, 256), 148 * 16), 256, 0, st>>>(h->cache64, h->nc, h->lcache32);
  }
}

template <int K>
static void launch_jac_lane(mf_ctx* h, const float* x, float* y, cudaStream_t st) {
  using L = LaneCfg<K>;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaFuncSetAttribute(k_cell_jac_lane<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM);
    attr_set[dev] = true;
  }
  k_cell_jac_lane<K><<<nblk(h->nc, L::CB), L::THREADS, L::SMEM, st>>>(h->lcells, h->nc, h->lcache32,
                                                                      reinterpret_cast<const float4*>(x), y,
                                                                      (float)h->nu, (float)h->a0dt);
}

template <int D, int K, typename T>
static void launch_jac(mf_ctx* h, const T* cache, const typename IO<T>::type* x, typename IO<T>::type* y,
                       cudaStream_t st) {
  ProfScope ps(h, std::is_same<T, double>::value ? 0 : 1, st);
  if constexpr (std::is_same<T, df>::value) {
    launch_jac_cpb<D, K, T, CellCfg<D, K>::CPB>(h, cache, x, y, st);    // double-float: default only
  } else {
    int sel = h->cpb_sel[std::is_same<T, double>::value ? 0 : 1];
    if constexpr (std::is_same<T, float>::value && D == 3 && K <= 3) {
      if (sel == 0) { launch_jac_lane<K>(h, x, y, st); return; }
      sel = sel == 1 ? 0 : 1;                  // per-point kernel: default, then the smaller block
    }
    switch (sel) {
      case 1: launch_jac_cpb<D, K, T, CpbVariants<D, K>::v1>(h, cache, x, y, st); break;
      case 2: launch_jac_cpb<D, K, T, CpbVariants<D, K>::v2>(h, cache, x, y, st); break;
      default: launch_jac_cpb<D, K, T, CellCfg<D, K>::CPB>(h, cache, x, y, st); break;
    }
  }
}

template <int D, int K, typename T>
static void launch_mortar(mf_ctx* h, int mode, const typename IO<T>::type* src, typename IO<T>::type* dst,
                          int zero_wall, cudaStream_t st) {
  MortarArgs<T> A;
  A.cells = h->cells; A.mc_cell = h->mc_cell; A.mc_tau = h->mc_tau; A.mc_xi = h->mc_xi;
  A.jinv = std::is_same<T, double>::value ? (const T*)h->mg_jinv64
         : std::is_same<T, float>::value ? (const T*)h->mg_jinv32 : (const T*)h->mg_jinvdf;
  A.mc_cs = h->mc_cs; A.mc_w = h->mc_w; A.nm = h->nm; A.src = src; A.dst = dst; A.nu = (T)h->nu;
  A.dz = h->H / h->n_z; A.zero_wall = zero_wall;
  using C = MortarCfg<D, K>;
  const unsigned g = nblk(h->nm, C::MPB);
  ProfScope ps(h, mode == 1 ? 7 : (std::is_same<T, double>::value ? 2 : 3), st);
  if (mode == 0) k_mortar<D, K, T, 0><<<g, C::THREADS, 0, st>>>(A);
  else k_mortar<D, K, T, 1><<<g, C::THREADS, 0, st>>>(A);
}

template <int D, int K, typename T>
static void launch_cell_diag(mf_ctx* h, const T* cache, T* diag, cudaStream_t st) {
  using C = CellCfg<D, K>;
  ProfScope ps(h, 7, st);
  k_cell_diag<D, K, T><<<nblk(h->nc, C::CPB), C::THREADS, 0, st>>>(h->cells, h->nc, cache, diag, (T)h->nu, (T)h->a0dt);
}

template <int D, int K>
static void launch_penalty(mf_ctx* h, cudaStream_t st) {
  const int64_t nif = (int64_t)h->n_z * h->n_R, nifs = (int64_t)h->n_z * h->n_Rs;
  k_penalty<D, K><<<nblk(nif, 64), 64, 0, st>>>(h->cells, h->x, h->ifr, nif, 0, h->F, h->tau_r);
  k_penalty<D, K><<<nblk(nifs, 64), 64, 0, st>>>(h->cells, h->x, h->ifs, nifs, 1, h->F, h->tau_s);
}

template <int K>
static void launch_map(mf_ctx* h, cudaStream_t st) {
  MortarMap A;
  A.mc_cell = h->mc_cell; A.mc_tau = h->mc_tau; A.mc_xi = h->mc_xi; A.mc_cs = h->mc_cs; A.mc_w = h->mc_w;
  A.ifr = h->ifr; A.ifs = h->ifs; A.tau_r = h->tau_r; A.tau_s = h->tau_s; A.n_R = h->n_R; A.n_z = h->n_z;
  A.R = h->R; A.phi0 = h->phi0; A.theta = h->theta; A.theta_dev = h->theta_on_dev ? h->d_theta : nullptr;
  if (h->n_Rs != h->n_R) {
    k_mortar_segments<<<1, 1, 0, st>>>(h->seg, h->n_R, h->n_Rs, h->theta, A.theta_dev);
    k_mortar_map_general<K><<<nblk(h->nm, 128), 128, 0, st>>>(A, h->seg, h->n_Rs);
    return;
  }
  k_mortar_map<K><<<nblk(h->nm, 128), 128, 0, st>>>(A);
}

template <int D, int K>
static void launch_mortar_geom(mf_ctx* h, cudaStream_t st) {
  const int64_t nt = h->nm * 2 * ipow(K + 1, D - 1);
  k_mortar_geom<D, K><<<nblk(nt, 128), 128, 0, st>>>(h->cells, h->x, h->mc_cell, h->mc_xi, h->nm, h->mg_jinv64,
                                                     h->mg_jinv32);
}

// ------------------------------------------------------------------ mesh
extern "C" mf_status mf_mesh_from_arrays(int d, int k, int64_t n_nodes, const double* x0, const uint8_t* node_side,
                                         const uint8_t* wall, int64_t n_cells, const int32_t* cells,
                                         const uint8_t* cell_side, double R, int n_R, int n_z, double H, double phi0,
                                         const int32_t* iface_rotor, const int32_t* iface_stator, mf_mesh** out) {
  return mf_mesh_from_arrays_ex(d, k, n_nodes, x0, node_side, wall, n_cells, cells, cell_side, R, n_R, n_R, n_z, H,
                                phi0, iface_rotor, iface_stator, out);
}

extern "C" mf_status mf_mesh_from_arrays_ex(int d, int k, int64_t n_nodes, const double* x0, const uint8_t* node_side,
                                            const uint8_t* wall, int64_t n_cells, const int32_t* cells,
                                            const uint8_t* cell_side, double R, int n_R, int n_R_stator, int n_z,
                                            double H, double phi0, const int32_t* iface_rotor,
                                            const int32_t* iface_stator, mf_mesh** out) {
  if (!out || !x0 || !node_side || !wall || !cells || !cell_side || !iface_rotor || !iface_stator) return MF_ERR_ARG;
  if ((d != 2 && d != 3) || k < 1 || k > MF_KMAX || n_nodes <= 0 || n_cells <= 0 || n_R < 1 || n_R_stator < 1 ||
      n_z < 1 || !(R > 0) || (d == 3 && !(H > 0)))
    return MF_ERR_ARG;
  if (n_nodes >= (int64_t)1 << 31) return MF_ERR_ARG;
  if (d == 2) n_z = 1;
  const int npc = ipow(k + 1, d);
  mf_mesh* m = new mf_mesh();
  m->d = d; m->k = k; m->nn = n_nodes; m->nc = n_cells; m->R = R; m->H = (d == 2 ? 1.0 : H); m->phi0 = phi0;
  m->n_R = n_R; m->n_z = n_z;
  m->n_Rs = n_R_stator == n_R ? 0 : n_R_stator;
  m->x0.assign(x0, x0 + n_nodes * d);
  m->node_side.assign(node_side, node_side + n_nodes);
  m->wall.assign(wall, wall + n_nodes);
  for (uint8_t w : m->wall)
    if (w > 2) { delete m; return MF_ERR_ARG; }
  m->cells.assign(cells, cells + n_cells * npc);
  m->cell_side.assign(cell_side, cell_side + n_cells);
  m->ifr.assign(iface_rotor, iface_rotor + (int64_t)n_z * n_R);
  m->ifs.assign(iface_stator, iface_stator + (int64_t)n_z * n_R_stator);
  for (int32_t c : m->cells)
    if (c < 0 || c >= n_nodes) { delete m; return MF_ERR_ARG; }
  for (int64_t i = 0; i < (int64_t)n_z * n_R; ++i)
    if (m->ifr[i] < 0 || m->ifr[i] >= n_cells) { delete m; return MF_ERR_ARG; }
  for (int64_t i = 0; i < (int64_t)n_z * n_R_stator; ++i)
    if (m->ifs[i] < 0 || m->ifs[i] >= n_cells) { delete m; return MF_ERR_ARG; }
  *out = m;
  return MF_OK;
}

extern "C" void mf_mesh_free(mf_mesh* m) { delete m; }

#include "mf_meshgen.inc"
#include "mf_checkpoint.inc"
#include "mf_slab.inc"

// ------------------------------------------------------------------ create
static void free_ws(Workspace& w) {
  if (w.is_static) { w = Workspace(); return; }   // symbol memory: nothing to free
  void* ptrs[] = {w.V, w.Z, w.w, w.r, w.dx, w.hcol, w.part, w.diag64, w.dinv64, w.dinv32, w.f_v, w.f_x, w.f_r,
                  w.f_d, w.f_t, w.f_w, w.c_x, w.c_r, w.c_d, w.c_t, w.c_v, w.c_w, w.utrial, w.f_Vin, w.c_Vin, w.hin, w.ep, w.jep,
                  w.hout, w.rec, w.rec_count};
  for (void* p : ptrs) if (p) cudaFree(p);
  if (w.pinned) cudaFreeHost(w.pinned);
  w = Workspace();
}

extern "C" mf_status mf_destroy(mf_handle h) {
  if (!h) return MF_ERR_ARG;
  for (auto& e : h->prof_ev) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  if (h->mg_exec) cudaGraphExecDestroy(h->mg_exec);
  if (h->d_theta && h->own_theta) cudaFree(h->d_theta);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  void* ptrs[] = {h->x0, h->x, h->node_side, h->cell_side, h->cells, h->wall, h->ifr, h->ifs, h->tau_r, h->tau_s,
                  h->mc_cell, h->mc_tau, h->mc_xi, h->mc_cs, h->mc_w, h->ht, h->g, h->cache64, h->cache32,
                  h->mg_jinv64, h->mg_jinv32, h->mg_jinvdf, h->cachedf, h->react, h->mg.parent, h->mg.child, h->mg.inv_mult64, h->mg.inv_mult32,
                  h->lcache32, h->lcells, h->asm_E, h->asm_bad, h->inv_mult32, h->seg.start, h->seg.len, h->seg.rstart, h->seg.jr, h->seg.js};
  for (void* p : ptrs) if (p) cudaFree(p);
  free_ws(h->ws);
  delete h;
  return MF_OK;
}

extern "C" const char* mf_last_error(mf_handle h) { return h ? h->err.c_str() : "null handle"; }

static mf_status apply_angle(mf_ctx* h, double theta, cudaStream_t st) {
  h->theta = theta;
  h->angle_set = !h->theta_on_dev;
  h->df_valid = false;
  h->geo_valid = false;
  const double ct = cos(theta), sn = sin(theta);
  const double* td = h->theta_on_dev ? h->d_theta : nullptr;
  if (h->d == 2) k_rotate<2><<<nblk(h->nn, 256), 256, 0, st>>>(h->x0, h->node_side, h->x, h->nn, ct, sn, td);
  else k_rotate<3><<<nblk(h->nn, 256), 256, 0, st>>>(h->x0, h->node_side, h->x, h->nn, ct, sn, td);
  switch (h->k) {
    case 1: launch_map<1>(h, st); break;
    case 2: launch_map<2>(h, st); break;
    case 3: launch_map<3>(h, st); break;
    case 4: launch_map<4>(h, st); break;
    case 5: launch_map<5>(h, st); break;
  }
  MF_DISPATCH(h->d, h->k, (launch_mortar_geom<D, K>(h, st)));
  CK(cudaGetLastError());
  return MF_OK;
}

extern "C" mf_status mf_create(const mf_mesh* m, int k, double nu, double omega, double dt, int bdf,
                               const mf_options* opt, mf_handle* out) {
  if (!m || !out) return MF_ERR_ARG;
  if (k != m->k || !(nu >= 0) || !std::isfinite(omega) || !(dt >= 0) || (bdf != 1 && bdf != 2)) return MF_ERR_ARG;
  mf_ctx* h = new mf_ctx();
  h->d = m->d; h->k = k; h->nn = m->nn; h->nc = m->nc; h->ndof = m->nn * (m->d + 1);
  h->nu = nu; h->omega = omega; h->dt = dt; h->bdf = bdf;
  h->F = (opt && opt->penalty_F > 0) ? opt->penalty_F : 1.0;
  const double al1[3] = {1.0, -1.0, 0.0}, al2[3] = {1.5, -2.0, 0.5};
  for (int i = 0; i < 3; ++i) h->alpha[i] = bdf == 1 ? al1[i] : al2[i];
  h->a0dt = dt > 0 ? h->alpha[0] / dt : 0.0;
  h->inv_dt2 = dt > 0 ? 1.0 / (dt * dt) : 0.0;
  h->R = m->R; h->H = m->H; h->phi0 = m->phi0; h->n_R = m->n_R; h->n_z = m->n_z;
  h->n_Rs = m->n_Rs > 0 ? m->n_Rs : m->n_R;
  h->nm = (int64_t)m->n_z * (m->n_R + h->n_Rs);      // equal partitions: two halves per stator cell
  h->nif = (int64_t)m->n_z * m->n_R;
  h->nif_s = (int64_t)m->n_z * h->n_Rs;
  h->ncache = (m->d == 2) ? Cache<2>::NF : Cache<3>::NF;
  h->cpb_sel[1] = default_fp32_variant(m->d, k, m->nc);
  h->nb = MF_REDUCE_BLOCKS;
  mf_status s = upload_tables(h);
  if (s != MF_OK) { mf_destroy(h); return s; }
  const int npc = ipow(k + 1, m->d);
  // cell table with wall nodes encoded as ~id
  std::vector<int32_t> cells(m->cells);
  for (auto& c : cells) if (m->wall[c]) c = ~c;
  // wall list: stationary walls first, then the walls moving with the rotor
  std::vector<int32_t> wl;
  for (int64_t i = 0; i < m->nn; ++i) if (m->wall[i] == 1) wl.push_back((int32_t)i);
  for (int64_t i = 0; i < m->nn; ++i) if (m->wall[i] == 2) wl.push_back((int32_t)i);
  h->nwall = (int64_t)wl.size();
  h->nmwall = h->nwall - (int64_t)std::count(m->wall.begin(), m->wall.end(), (uint8_t)1);
  const size_t nn = m->nn, nc = m->nc, d = m->d;
#define ALLOC(p, cnt) CK(cudaMalloc((void**)&(p), sizeof(*(p)) * std::max<size_t>(1, (size_t)(cnt))))
  auto fail = [&](mf_status st) { std::string e = h->err; mf_destroy(h); (void)e; return st; };
  do {
#define ALLOC2(p, cnt)                                                                          \
  if (cudaMalloc((void**)&(p), sizeof(*(p)) * std::max<size_t>(1, (size_t)(cnt))) != cudaSuccess) \
    return fail(MF_ERR_OOM);
    ALLOC2(h->x0, nn * d); ALLOC2(h->x, nn * d); ALLOC2(h->node_side, nn); ALLOC2(h->cell_side, nc);
    ALLOC2(h->cells, nc * npc); ALLOC2(h->wall, wl.size()); ALLOC2(h->ifr, h->nif); ALLOC2(h->ifs, h->nif_s);
    ALLOC2(h->tau_r, h->nif); ALLOC2(h->tau_s, h->nif_s);
    if (h->n_Rs != h->n_R) {
      const size_t ns = (size_t)h->n_R + h->n_Rs;
      ALLOC2(h->seg.start, ns); ALLOC2(h->seg.len, ns); ALLOC2(h->seg.rstart, ns); ALLOC2(h->seg.jr, ns);
      ALLOC2(h->seg.js, ns);
    }
    ALLOC2(h->mc_cell, h->nm * 2); ALLOC2(h->mc_tau, h->nm); ALLOC2(h->mc_xi, h->nm * 2 * (k + 1));
    ALLOC2(h->mc_cs, h->nm * (k + 1) * 2); ALLOC2(h->mc_w, h->nm * (k + 1));
    ALLOC2(h->mg_jinv64, h->nm * 2 * ipow(k + 1, m->d - 1) * m->d * m->d);
    ALLOC2(h->mg_jinv32, h->nm * 2 * ipow(k + 1, m->d - 1) * m->d * m->d);
    ALLOC2(h->ht, nn * d); ALLOC2(h->cache64, (size_t)h->ncache * nc * npc); ALLOC2(h->cache32, (size_t)h->ncache * nc * npc);
    if (lane_kernel_available(h->d, h->k)) {
      const size_t padded = (nc + 31) / 32 * 32;
      ALLOC2(h->lcells, padded * npc); ALLOC2(h->lcache32, (size_t)LaneCache::NF * padded * npc);
    }
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, MF_OVERLAP_ORDER == 1 ? prio_lo : prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess)
      return fail(MF_ERR_CUDA);
  } while (0);
#undef ALLOC2
  if (cudaMemcpy(h->x0, m->x0.data(), nn * d * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->node_side, m->node_side.data(), nn, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->cell_side, m->cell_side.data(), nc, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->cells, cells.data(), nc * npc * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      (wl.size() && cudaMemcpy(h->wall, wl.data(), wl.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(h->ifr, m->ifr.data(), h->nif * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->ifs, m->ifs.data(), h->nif_s * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(h->ht, 0, nn * d * 8) != cudaSuccess)
    return fail(MF_ERR_CUDA);
  if (h->lcells) MF_DISPATCH(h->d, h->k, (launch_lane_cells<D, K>(h, 0)));
  // geometry at theta = 0, penalties (rotation-invariant), mortar cells
  if (h->d == 2) k_rotate<2><<<nblk(h->nn, 256), 256>>>(h->x0, h->node_side, h->x, h->nn, 1.0, 0.0, nullptr);
  else k_rotate<3><<<nblk(h->nn, 256), 256>>>(h->x0, h->node_side, h->x, h->nn, 1.0, 0.0, nullptr);
  MF_DISPATCH(h->d, h->k, (launch_penalty<D, K>(h, 0)));
  if (apply_angle(h, 0.0, 0) != MF_OK) return fail(MF_ERR_CUDA);
  if (cudaDeviceSynchronize() != cudaSuccess) { h->err = cudaGetErrorString(cudaGetLastError()); return fail(MF_ERR_CUDA); }
  *out = h;
  return MF_OK;
#undef ALLOC
}

extern "C" mf_status mf_sizes(mf_handle h, int64_t* n_nodes, int64_t* n_dofs, int64_t* n_cells, int64_t* n_mortar) {
  if (!h) return MF_ERR_ARG;
  if (n_nodes) *n_nodes = h->nn;
  if (n_dofs) *n_dofs = h->ndof;
  if (n_cells) *n_cells = h->nc;
  if (n_mortar) *n_mortar = h->nm;
  return MF_OK;
}

extern "C" mf_status mf_set_angle(mf_handle h, double theta, void* stream) {
  if (!h) return MF_ERR_ARG;
  if (!std::isfinite(theta)) { h->err = "theta must be finite"; return MF_ERR_ARG; }
  h->have_lin = false;
  return apply_angle(h, theta, S(stream));
}

extern "C" mf_status mf_node_coords(mf_handle h, double* xyz, void* stream) {
  if (!h || !xyz) return MF_ERR_ARG;
  CK(cudaMemcpyAsync(xyz, h->x, h->nn * h->d * 8, cudaMemcpyDeviceToDevice, S(stream)));
  return MF_OK;
}

extern "C" mf_status mf_dirichlet(mf_handle h, const double* g, void* stream) {
  if (!h) return MF_ERR_ARG;
  if (!g) { if (h->g) { cudaFree(h->g); h->g = nullptr; } return MF_OK; }
  if (!h->g) CK(cudaMalloc((void**)&h->g, h->nn * h->d * 8));
  CK(cudaMemcpyAsync(h->g, g, h->nn * h->d * 8, cudaMemcpyDeviceToDevice, S(stream)));
  return MF_OK;
}

extern "C" mf_status mf_set_history(mf_handle h, const double* u_n, const double* u_nm1, void* stream) {
  if (!h || !u_n || (h->bdf == 2 && !u_nm1)) return MF_ERR_ARG;
  if (h->dt <= 0) { CK(cudaMemsetAsync(h->ht, 0, h->nn * h->d * 8, S(stream))); return MF_OK; }
  const int64_t n = h->nn * h->d;
  k_history<<<nblk(n, 256), 256, 0, S(stream)>>>(u_n, h->bdf == 2 ? u_nm1 : nullptr, h->ht, n, h->alpha[1] / h->dt,
                                                 h->alpha[2] / h->dt);
  CK(cudaGetLastError());
  return MF_OK;
}

extern "C" mf_status mf_set_linearization(mf_handle h, const double* up_star, double theta, void* stream) {
  if (!h || !up_star) return MF_ERR_ARG;
  if (!std::isfinite(theta)) { h->err = "theta must be finite"; return MF_ERR_ARG; }
  cudaStream_t st = S(stream);
  // the rotation, mortar map and face geometry depend on the angle only: a
  // relinearisation at the angle already applied (the Newton loop's levels)
  // keeps them, and the state pass keeps the cached cell geometry too
  if (!(h->angle_set && !h->theta_on_dev && theta == h->theta)) {
    mf_status s = apply_angle(h, theta, st);
    if (s != MF_OK) return s;
  }
  MF_DISPATCH(h->d, h->k, (launch_state<D, K>(h, 0, up_star, nullptr, st)));
  const int64_t ncv = (int64_t)h->ncache * h->nc * ipow(h->k + 1, h->d);
  k_cast<double, float><<<nblk(ncv, 256), 256, 0, st>>>(h->cache64, h->cache32, ncv);
  if (h->lcache32) MF_DISPATCH(h->d, h->k, (launch_lane_cache<D, K>(h, st)));
  CK(cudaGetLastError());
  h->have_lin = true;
  h->df_valid = false;
  return MF_OK;
}

// Residual r = F-hat*_NS(up) (as mf_residual) and, from the same pass over the
// cells, the linearisation cache at up (as mf_set_linearization at the
// handle's current angle): the Newton loop needs both at every new iterate.
static mf_status residual_rows(mf_ctx* h, const double* up, double* r, cudaStream_t st);
static mf_status residual_constrain(mf_ctx* h, const double* up, double* r, cudaStream_t st);
static mf_status residual_and_linearize(mf_ctx* h, const double* up, double* r, cudaStream_t st) {
  CK(cudaMemsetAsync(r, 0, h->ndof * 8, st));
  MF_DISPATCH(h->d, h->k, (launch_state<D, K>(h, 2, up, r, st)));
  MF_DISPATCH(h->d, h->k, (launch_mortar<D, K, double>(h, 0, up, r, 0, st)));
  const int64_t ncv = (int64_t)h->ncache * h->nc * ipow(h->k + 1, h->d);
  k_cast<double, float><<<nblk(ncv, 256), 256, 0, st>>>(h->cache64, h->cache32, ncv);
  if (h->lcache32) MF_DISPATCH(h->d, h->k, (launch_lane_cache<D, K>(h, st)));
  CK(cudaGetLastError());
  h->have_lin = true;
  h->df_valid = false;
  return residual_constrain(h, up, r, st);
}

// Volume + mortar residual rows without the Dirichlet replacement (on wall
// nodes these are the consistent reactions).
static mf_status residual_rows(mf_ctx* h, const double* up, double* r, cudaStream_t st) {
  CK(cudaMemsetAsync(r, 0, h->ndof * 8, st));
  MF_DISPATCH(h->d, h->k, (launch_state<D, K>(h, 1, up, r, st)));
  MF_DISPATCH(h->d, h->k, (launch_mortar<D, K, double>(h, 0, up, r, 0, st)));
  CK(cudaGetLastError());
  return MF_OK;
}

// r = u - g on the wall velocity rows
static mf_status residual_constrain(mf_ctx* h, const double* up, double* r, cudaStream_t st) {
  if (h->nwall) {
    const int64_t m0 = h->nwall - h->nmwall;
    if (h->d == 2) k_dirichlet_res<2><<<nblk(h->nwall, 256), 256, 0, st>>>(h->wall, h->nwall, m0, up, h->g, h->x, h->omega, r);
    else k_dirichlet_res<3><<<nblk(h->nwall, 256), 256, 0, st>>>(h->wall, h->nwall, m0, up, h->g, h->x, h->omega, r);
  }
  CK(cudaGetLastError());
  return MF_OK;
}

extern "C" mf_status mf_residual(mf_handle h, const double* up, double* r, void* stream) {
  if (!h || !up || !r) return MF_ERR_ARG;
  cudaStream_t st = S(stream);
  mf_status e = residual_rows(h, up, r, st);
  if (e != MF_OK) return e;
  return residual_constrain(h, up, r, st);
}

// Wall loads from reaction rows r: out[g][0..d-1] force, [d] torque about e_z,
// [d+1] power, summed over the wall nodes of group g (zeroed first).
static mf_status wall_loads_from_rows(mf_ctx* h, const double* up, const double* r, const uint8_t* group, int n_groups,
                                      double* out, cudaStream_t st) {
  CK(cudaMemsetAsync(out, 0, sizeof(double) * n_groups * (h->d + 2), st));
  if (h->nwall) {
    const int64_t m0 = h->nwall - h->nmwall;
    const unsigned nb = std::min<unsigned>(nblk(h->nwall, 256), 148 * 2);
    if (h->d == 2) k_wall_loads<2><<<nb, 256, 0, st>>>(h->wall, h->nwall, m0, group, n_groups, h->x, up, r, out);
    else k_wall_loads<3><<<nb, 256, 0, st>>>(h->wall, h->nwall, m0, group, n_groups, h->x, up, r, out);
  }
  CK(cudaGetLastError());
  return MF_OK;
}

extern "C" mf_status mf_wall_loads(mf_handle h, const double* up, const uint8_t* group, int n_groups, double* out,
                                   void* stream) {
  if (!h || !up || !out || n_groups < 1 || n_groups > MF_MAX_LOAD_GROUPS || (!group && n_groups != 2)) return MF_ERR_ARG;
  cudaStream_t st = S(stream);
  if (!h->react) CK(cudaMalloc((void**)&h->react, h->ndof * sizeof(double)));
  mf_status e = residual_rows(h, up, h->react, st);
  if (e != MF_OK) return e;
  return wall_loads_from_rows(h, up, h->react, group, n_groups, out, st);
}

template <typename T>
static mf_status apply_t(mf_ctx* h, const typename IO<T>::type* x, typename IO<T>::type* y, cudaStream_t st) {
  using TI = typename IO<T>::type;
  const T* cache = std::is_same<T, double>::value ? (const T*)h->cache64
                 : std::is_same<T, float>::value ? (const T*)h->cache32 : (const T*)h->cachedf;
  CK(cudaMemsetAsync(y, 0, h->ndof * sizeof(TI), st));
  if (!h->prof && (MF_OVERLAP_MORTAR & (std::is_same<T, double>::value ? 1 : std::is_same<T, float>::value ? 2 : 4))) {
    // Both kernels scatter with atomics into the zeroed y: the mortar blocks
    // run on the side stream, beside the cell kernel's waves (serialised
    // while profiling, so that each kernel's events time it alone).
    CK(cudaEventRecord(h->ev_fork, st));
    CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
    if (MF_OVERLAP_ORDER == 1) {
      MF_DISPATCH(h->d, h->k, (launch_jac<D, K, T>(h, cache, x, y, st)));
      MF_DISPATCH(h->d, h->k, (launch_mortar<D, K, T>(h, 0, x, y, 1, h->side)));
    } else {
      MF_DISPATCH(h->d, h->k, (launch_mortar<D, K, T>(h, 0, x, y, 1, h->side)));
      MF_DISPATCH(h->d, h->k, (launch_jac<D, K, T>(h, cache, x, y, st)));
    }
    CK(cudaEventRecord(h->ev_join, h->side));
    CK(cudaStreamWaitEvent(st, h->ev_join, 0));
  } else {
    MF_DISPATCH(h->d, h->k, (launch_jac<D, K, T>(h, cache, x, y, st)));
    MF_DISPATCH(h->d, h->k, (launch_mortar<D, K, T>(h, 0, x, y, 1, st)));
  }
  if (h->nwall) {
    ProfScope ps(h, 6, st);
    if (h->d == 2) k_dirichlet_copy<2, TI><<<nblk(h->nwall, 256), 256, 0, st>>>(h->wall, h->nwall, x, y);
    else k_dirichlet_copy<3, TI><<<nblk(h->nwall, 256), 256, 0, st>>>(h->wall, h->nwall, x, y);
  }
  CK(cudaGetLastError());
  return MF_OK;
}

// double-float copies of the linearisation cache and the face geometry
static mf_status ensure_df(mf_ctx* h, cudaStream_t st) {
  const int64_t ncv = (int64_t)h->ncache * h->nc * ipow(h->k + 1, h->d);
  const int64_t njv = h->nm * 2 * ipow(h->k + 1, h->d - 1) * h->d * h->d;
  if (!h->cachedf) CK(cudaMalloc((void**)&h->cachedf, sizeof(df) * ncv));
  if (!h->mg_jinvdf) CK(cudaMalloc((void**)&h->mg_jinvdf, sizeof(df) * njv));
  if (h->df_valid) return MF_OK;
  k_split_df<<<nblk(ncv, 256), 256, 0, st>>>(h->cache64, h->cachedf, ncv);
  k_split_df<<<nblk(njv, 256), 256, 0, st>>>(h->mg_jinv64, h->mg_jinvdf, njv);
  CK(cudaGetLastError());
  h->df_valid = true;
  return MF_OK;
}

extern "C" mf_status mf_apply_jacobian(mf_handle h, const void* x, void* y, mf_precision prec, void* stream) {
  if (!h || !x || !y || x == y) return MF_ERR_ARG;
  if (!h->have_lin) { h->err = "mf_apply_jacobian before mf_set_linearization"; return MF_ERR_STATE; }
  if (prec == MF_FP64) return apply_t<double>(h, (const double*)x, (double*)y, S(stream));
  if (prec == MF_FP32) return apply_t<float>(h, (const float*)x, (float*)y, S(stream));
  if (prec == MF_DF64) {
    mf_status e = ensure_df(h, S(stream));
    if (e != MF_OK) return e;
    return apply_t<df>(h, (const double*)x, (double*)y, S(stream));
  }
  return MF_ERR_ARG;
}

template <typename T>
static mf_status diag_t(mf_ctx* h, T* dg, cudaStream_t st) {
  const T* cache = std::is_same<T, double>::value ? (const T*)h->cache64 : (const T*)h->cache32;
  CK(cudaMemsetAsync(dg, 0, h->ndof * sizeof(T), st));
  MF_DISPATCH(h->d, h->k, (launch_cell_diag<D, K, T>(h, cache, dg, st)));
  MF_DISPATCH(h->d, h->k, (launch_mortar<D, K, T>(h, 1, (const T*)nullptr, dg, 1, st)));
  if (h->nwall) {
    if (h->d == 2) k_dirichlet_one<2, T><<<nblk(h->nwall, 256), 256, 0, st>>>(h->wall, h->nwall, dg);
    else k_dirichlet_one<3, T><<<nblk(h->nwall, 256), 256, 0, st>>>(h->wall, h->nwall, dg);
  }
  CK(cudaGetLastError());
  return MF_OK;
}

extern "C" mf_status mf_diagonal(mf_handle h, void* diag_out, mf_precision prec, void* stream) {
  if (!h || !diag_out) return MF_ERR_ARG;
  if (!h->have_lin) { h->err = "mf_diagonal before mf_set_linearization"; return MF_ERR_STATE; }
  if (prec == MF_FP64) return diag_t<double>(h, (double*)diag_out, S(stream));
  if (prec == MF_FP32) return diag_t<float>(h, (float*)diag_out, S(stream));
  return MF_ERR_ARG;
}

extern "C" mf_status mf_profile(mf_handle h, int enable) {
  if (!h) return MF_ERR_ARG;
  for (auto& e : h->prof_ev) { h->ev_pool.push_back(e.a); h->ev_pool.push_back(e.b); }
  h->prof_ev.clear();
  std::memset(&h->prof_acc, 0, sizeof(h->prof_acc));
  h->prof = enable != 0;
  return MF_OK;
}

extern "C" mf_status mf_profile_read(mf_handle h, mf_profile_t* out) {
  if (!h || !out) return MF_ERR_ARG;
  for (auto& e : h->prof_ev) {
    CK(cudaEventSynchronize(e.b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e.a, e.b));
    h->prof_acc.launches[e.kind] += 1;
    h->prof_acc.ms[e.kind] += ms;
    h->ev_pool.push_back(e.a);
    h->ev_pool.push_back(e.b);
  }
  h->prof_ev.clear();
  *out = h->prof_acc;
  return MF_OK;
}

#include "mf_asm.inc"
#include "mf_solve.inc"
#include "mf_mg.inc"
#include "mf_transient.inc"
#include "mf_autotune.inc"
#include "mf_probe.inc"
#include "mf_tc.inc"
#include "mf_vec.inc"

// ---------------------------------------------------------------- batched instances
struct mf_batch {
  std::vector<mf_ctx*> hs;
  int d = 0, k = 0;
  BatchTable<double>* tab64 = nullptr;         // device
  BatchTable<float>* tab32 = nullptr;
  MortarBatchTable<double>* mtab64 = nullptr;
  MortarBatchTable<float>* mtab32 = nullptr;
  unsigned long long* counters = nullptr;      // device [2]
  BatchTable<double>* h_tab64 = nullptr;       // pinned host staging
  BatchTable<float>* h_tab32 = nullptr;
  MortarBatchTable<double>* h_mtab64 = nullptr;
  MortarBatchTable<float>* h_mtab32 = nullptr;
  cudaEvent_t staged = nullptr;                // staging buffers free again
  int grid_cell = 0, grid_mortar = 0;          // persistent grid sizes
  std::string err;
  // batched solve (mf_batch_solve_step): per-instance streams forked from the
  // caller's stream, a capture stream, one device table pair per FGMRES
  // column (Z_j -> w of every instance) and the residual norms read back
  std::vector<cudaStream_t> ist;
  std::vector<cudaEvent_t> iev;
  cudaEvent_t fork_ev = nullptr;
  cudaStream_t cap = nullptr;
  BatchTable<double>* sol_tab = nullptr;       // device [sol_m]
  MortarBatchTable<double>* sol_mtab = nullptr;
  std::vector<BatchTable<double>> sol_htab;    // host copies (launch parameters)
  std::vector<MortarBatchTable<double>> sol_hmtab;
  int sol_m = 0;
  double* norms2 = nullptr;                    // device [n] ||R_i||^2
  double* h_norms2 = nullptr;                  // pinned [n]
  std::vector<double*> u_start;                // device copies of the initial guesses (fallback restarts)
  std::vector<int64_t> u_start_n;
};

template <int D, int K>
static void batch_grids(mf_batch* b) {
  int dev = 0, sms = 148, occ_c = 1, occ_m = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, k_cell_jac_batched<D, K, double>, CellCfg<D, K>::THREADS, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_m, k_mortar_batched<D, K, double>, MortarCfg<D, K>::THREADS, 0);
  b->grid_cell = sms * std::max(occ_c, 1);
  b->grid_mortar = sms * std::max(occ_m, 1);
}

extern "C" mf_status mf_batch_create(const mf_handle* hs, int n, mf_batch** out) {
  if (!hs || !out || n < 1 || n > MF_BATCH_MAX) return MF_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!hs[i] || hs[i]->d != hs[0]->d || hs[i]->k != hs[0]->k) return MF_ERR_ARG;
  mf_batch* b = new mf_batch();
  b->hs.assign(hs, hs + n);
  b->d = hs[0]->d; b->k = hs[0]->k;
  bool ok = cudaMalloc((void**)&b->tab64, sizeof(BatchTable<double>)) == cudaSuccess &&
            cudaMalloc((void**)&b->tab32, sizeof(BatchTable<float>)) == cudaSuccess &&
            cudaMalloc((void**)&b->mtab64, sizeof(MortarBatchTable<double>)) == cudaSuccess &&
            cudaMalloc((void**)&b->mtab32, sizeof(MortarBatchTable<float>)) == cudaSuccess &&
            cudaMalloc((void**)&b->counters, 2 * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMallocHost((void**)&b->h_tab64, sizeof(BatchTable<double>)) == cudaSuccess &&
            cudaMallocHost((void**)&b->h_tab32, sizeof(BatchTable<float>)) == cudaSuccess &&
            cudaMallocHost((void**)&b->h_mtab64, sizeof(MortarBatchTable<double>)) == cudaSuccess &&
            cudaMallocHost((void**)&b->h_mtab32, sizeof(MortarBatchTable<float>)) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    mf_batch_destroy(b);
    return MF_ERR_OOM;
  }
  MF_DISPATCH(b->d, b->k, (batch_grids<D, K>(b)));
  *out = b;
  return MF_OK;
}

extern "C" const char* mf_batch_last_error(mf_batch* b) {
  if (!b) return "null batch";
  if (!b->err.empty()) return b->err.c_str();
  for (mf_ctx* c : b->hs)
    if (!c->err.empty()) return c->err.c_str();
  return "";
}

extern "C" mf_status mf_batch_destroy(mf_batch* b) {
  if (!b) return MF_ERR_ARG;
  void* dp[] = {b->tab64, b->tab32, b->mtab64, b->mtab32, b->counters};
  for (void* p : dp) if (p) cudaFree(p);
  void* hp[] = {b->h_tab64, b->h_tab32, b->h_mtab64, b->h_mtab32};
  for (void* p : hp) if (p) cudaFreeHost(p);
  if (b->staged) cudaEventDestroy(b->staged);
  for (cudaStream_t q : b->ist) cudaStreamDestroy(q);
  for (cudaEvent_t q : b->iev) cudaEventDestroy(q);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->sol_tab) cudaFree(b->sol_tab);
  if (b->sol_mtab) cudaFree(b->sol_mtab);
  if (b->norms2) cudaFree(b->norms2);
  for (double* p : b->u_start) if (p) cudaFree(p);
  if (b->h_norms2) cudaFreeHost(b->h_norms2);
  delete b;
  return MF_OK;
}

// Tile tables of one batched apply xs[i] -> ys[i] (host copies ht, hm).
// sel (optional): the instances (indices into b->hs) that form the table, in
// order; xs/ys are indexed like sel.  NULL: every instance.
template <typename T>
static mf_status fill_batch_tables(mf_batch* b, const void* const* xs, void* const* ys, BatchTable<T>* ht,
                                   MortarBatchTable<T>* hm, bool need_lin = true, const int* sel = nullptr,
                                   int nsel = 0) {
  const bool f64 = std::is_same<T, double>::value;
  const int n = sel ? nsel : (int)b->hs.size();
  int cpb = 1, mpb = 1;
  switch (b->d * 10 + b->k) {
#define CASE(D_, K_) case D_ * 10 + K_: cpb = CellCfg<D_, K_>::CPB; mpb = MortarCfg<D_, K_>::MPB; break;
    CASE(2, 1) CASE(2, 2) CASE(2, 3) CASE(2, 4) CASE(2, 5) CASE(3, 1) CASE(3, 2) CASE(3, 3) CASE(3, 4) CASE(3, 5)
#undef CASE
  }
  ht->ninst = n; hm->ninst = n;
  ht->first_tile[0] = 0; hm->first_tile[0] = 0;
  for (int i = 0; i < n; ++i) {
    mf_ctx* c = b->hs[sel ? sel[i] : i];
    if (need_lin && !c->have_lin) { b->err = "batched apply: an instance has no linearisation"; return MF_ERR_STATE; }
    if (!xs[i] || !ys[i] || xs[i] == ys[i]) return MF_ERR_ARG;
    BatchInst<T>& in = ht->inst[i];
    in.cells = c->cells; in.nc = c->nc; in.cache = f64 ? (const T*)c->cache64 : (const T*)c->cache32;
    in.src = (const T*)xs[i]; in.dst = (T*)ys[i]; in.nu = (T)c->nu; in.a0dt = (T)c->a0dt;
    ht->first_tile[i + 1] = ht->first_tile[i] + (c->nc + cpb - 1) / cpb;
    MortarArgs<T>& A = hm->inst[i];
    A.cells = c->cells; A.mc_cell = c->mc_cell; A.mc_tau = c->mc_tau; A.mc_xi = c->mc_xi;
    A.jinv = f64 ? (const T*)c->mg_jinv64 : (const T*)c->mg_jinv32;
    A.mc_cs = c->mc_cs; A.mc_w = c->mc_w; A.nm = c->nm; A.src = (const T*)xs[i]; A.dst = (T*)ys[i];
    A.nu = (T)c->nu; A.dz = c->H / c->n_z; A.zero_wall = 1;
    hm->first_tile[i + 1] = hm->first_tile[i] + (c->nm + mpb - 1) / mpb;
  }
  return MF_OK;
}

// The launches of one batched apply from device tables dt, dm whose host
// copies are ht, hm: zero every ys[i], one persistent cell launch and one
// persistent mortar launch over all instances, then the Dirichlet rows.
template <typename T>
static mf_status launch_batch(mf_batch* b, const BatchTable<T>* ht, const MortarBatchTable<T>* hm,
                              const BatchTable<T>* dt, const MortarBatchTable<T>* dm, cudaStream_t st,
                              const int* sel = nullptr) {
  using TI = typename IO<T>::type;
  mf_ctx* h = b->hs[0];     // CUDA errors are reported on the first instance
  const int n = ht->ninst;
  for (int i = 0; i < n; ++i) CK(cudaMemsetAsync(ht->inst[i].dst, 0, b->hs[sel ? sel[i] : i]->ndof * sizeof(TI), st));
  CK(cudaMemsetAsync(b->counters, 0, 2 * sizeof(unsigned long long), st));
  const int64_t tc = ht->first_tile[n], tm = hm->first_tile[n];
  switch (b->d * 10 + b->k) {
#define CASE(D_, K_)                                                                                          \
  case D_ * 10 + K_:                                                                                          \
    k_cell_jac_batched<D_, K_, T><<<(unsigned)std::min<int64_t>(tc, b->grid_cell), CellCfg<D_, K_>::THREADS, 0,  \
                                    st>>>(dt, b->counters);                                                   \
    k_mortar_batched<D_, K_, T><<<(unsigned)std::min<int64_t>(std::max<int64_t>(tm, 1), b->grid_mortar),        \
                                  MortarCfg<D_, K_>::THREADS, 0, st>>>(dm, b->counters + 1);                  \
    break;
    CASE(2, 1) CASE(2, 2) CASE(2, 3) CASE(2, 4) CASE(2, 5) CASE(3, 1) CASE(3, 2) CASE(3, 3) CASE(3, 4) CASE(3, 5)
#undef CASE
  }
  for (int i = 0; i < n; ++i) {
    mf_ctx* c = b->hs[sel ? sel[i] : i];
    if (!c->nwall) continue;
    const TI* x = (const TI*)ht->inst[i].src;
    TI* y = (TI*)ht->inst[i].dst;
    if (c->d == 2) k_dirichlet_copy<2, TI><<<nblk(c->nwall, 256), 256, 0, st>>>(c->wall, c->nwall, x, y);
    else k_dirichlet_copy<3, TI><<<nblk(c->nwall, 256), 256, 0, st>>>(c->wall, c->nwall, x, y);
  }
  CK(cudaGetLastError());
  return MF_OK;
}

template <typename T>
static mf_status batch_apply_t(mf_batch* b, const void* const* xs, void* const* ys, cudaStream_t st) {
  mf_ctx* h = b->hs[0];     // CUDA errors are reported on the first instance
  const bool f64 = std::is_same<T, double>::value;
  BatchTable<T>* ht = f64 ? (BatchTable<T>*)b->h_tab64 : (BatchTable<T>*)b->h_tab32;
  BatchTable<T>* dt = f64 ? (BatchTable<T>*)b->tab64 : (BatchTable<T>*)b->tab32;
  MortarBatchTable<T>* hm = f64 ? (MortarBatchTable<T>*)b->h_mtab64 : (MortarBatchTable<T>*)b->h_mtab32;
  MortarBatchTable<T>* dm = f64 ? (MortarBatchTable<T>*)b->mtab64 : (MortarBatchTable<T>*)b->mtab32;
  CK(cudaEventSynchronize(b->staged));    // the previous call's table copies have completed
  mf_status e = fill_batch_tables<T>(b, xs, ys, ht, hm);
  if (e != MF_OK) return e;
  CK(cudaMemcpyAsync(dt, ht, sizeof(BatchTable<T>), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dm, hm, sizeof(MortarBatchTable<T>), cudaMemcpyHostToDevice, st));
  CK(cudaEventRecord(b->staged, st));
  return launch_batch<T>(b, ht, hm, dt, dm, st);
}

extern "C" mf_status mf_batch_apply_jacobian(mf_batch* b, const void* const* xs, void* const* ys, mf_precision prec,
                                             void* stream) {
  if (!b || !xs || !ys) return MF_ERR_ARG;
  mf_status s = prec == MF_FP64 ? batch_apply_t<double>(b, xs, ys, S(stream))
              : prec == MF_FP32 ? batch_apply_t<float>(b, xs, ys, S(stream)) : MF_ERR_ARG;
  return s;
}

#include "mf_batch_solve.inc"

// ---------------------------------------------------------------- no-allocation solve
// Workspace of mf_solve_step_static: a file-scope device array.  In host code
// the name is only a host-side stand-in; kernels get the device address looked
// up with cudaGetSymbolAddress (once per device, on the first call).
static __device__ __align__(256) double mf_static_ws[MF_STATIC_WS_DOUBLES];
static double* g_static_ws_dev[64] = {nullptr};
static double g_static_host[3 * (200 + 2)];      // host staging for the small read-backs

extern "C" mf_status mf_solve_step_static(mf_handle h, double* up, const mf_solver_opts* so_in, mf_solve_report* rep,
                                          void* stream) {
  if (!h || !up) return MF_ERR_ARG;
  mf_solver_opts so;
  if (so_in) so = *so_in; else mf_solver_defaults(&so);
  if (so.pc != MF_PC_JACOBI || so.pc_precision != MF_FP64 || so.outer_precision != MF_FP64) {
    h->err = "mf_solve_step_static: only pc = MF_PC_JACOBI with pc_precision = MF_FP64 (FP64 outer applies)";
    return MF_ERR_ARG;
  }
  if (h->prof) { h->err = "mf_solve_step_static: disable profiling (it creates events)"; return MF_ERR_STATE; }
  const int m = std::min(std::max(so.restart, 1), 200);
  const int64_t n = h->ndof;
  const int part_cap = m + 2;
  const int64_t need = (int64_t)(2 * m + 10) * n + 3 * (m + 2) + (int64_t)part_cap * h->nb;
  if (need > (int64_t)MF_STATIC_WS_DOUBLES) {
    char buf[256];
    std::snprintf(buf, sizeof(buf),
                  "mf_solve_step_static: needs %lld doubles for %lld DoFs with restart %d, the static workspace "
                  "holds %u",
                  (long long)need, (long long)n, m, (unsigned)MF_STATIC_WS_DOUBLES);
    h->err = buf;
    return MF_ERR_ARG;
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) { h->err = "mf_solve_step_static: device index out of range"; return MF_ERR_ARG; }
  if (!g_static_ws_dev[dev]) {
    double* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, mf_static_ws);
    if (e != cudaSuccess || !p) {
      h->err = std::string("mf_solve_step_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return MF_ERR_CUDA;
    }
    g_static_ws_dev[dev] = p;
  }
  // carve the view: V (m+1)n, Z m n, then w r dx diag64 dinv64 utrial ep jep dinv32, hcol, part
  double* p = g_static_ws_dev[dev];
  Workspace view;
  view.m = m;
  view.V = p; p += (size_t)(m + 1) * n;
  view.Z = p; p += (size_t)m * n;
  view.w = p; p += n;
  view.r = p; p += n;
  view.dx = p; p += n;
  view.diag64 = p; p += n;
  view.dinv64 = p; p += n;
  view.utrial = p; p += n;
  view.ep = p; p += n;
  view.jep = p; p += n;
  view.dinv32 = (float*)p; p += n;      // n floats (half of this slot is spare)
  view.hcol = p; p += 3 * (m + 2);
  view.part = p; p += (size_t)part_cap * h->nb;
  view.part_cap = part_cap;
  view.pinned = g_static_host;
  // The Jacobi / FP64 Newton-FGMRES path reads and writes only the fields set
  // above (V, Z, w, r, dx, diag64, dinv64, dinv32, utrial, ep, jep, hcol, part,
  // pinned).  The FP32 / Chebyshev vectors, the inner GMRES bases and the
  // transient buffers stay null; a solver path that asks for them (or for a
  // larger workspace) gets MF_ERR_STATE from ensure_ws / ensure_inner instead of
  // an allocation, because the view is marked static.
  view.is_static = true;
  // the small scalars start at zero on every call
  CK(cudaMemsetAsync(view.hcol, 0, sizeof(double) * (3 * (m + 2) + (size_t)part_cap * h->nb), S(stream)));
  Workspace saved = h->ws;
  h->ws = view;
  so.restart = m;
  const mf_status st = mf_solve_step(h, up, &so, rep, stream);
  h->ws = saved;
  return st;
}
