// Multigrid transfers between a fine level and a coarser level of the global-
// coarsening multigrid (Section 3.4): polynomial coarsening (same cells,
// degree KC < KF) or geometric coarsening (each coarse cell split into 2^d
// fine cells; parent[c] and child[c] bit r = upper half along xi_r).
// In the parent's reference coordinates a fine node at xi_f sits at
//   s(xi_f) = xi_f (p), xi_f / 2 (lower half), (1 + xi_f) / 2 (upper half).
//   prolongation  u_f(a) = sum_b prod_r l^KC_{b_r}(s_r(x^KF_{a_r})) u_c(b)
//   restriction   r_c(b) += sum_a [same weights] r_f(a) / mult(a)   (transpose)
//   state interpolation u_c(b) = fine field at the coarse node, evaluated in
//                 the fine cell that contains it
// mult(a) = number of fine cells sharing node a.  Prolongation and
// interpolation write node values (continuous fields: every cell writes the
// same value); restriction accumulates.
#pragma once
#include "mf_cell.cuh"

namespace mf {

struct XferTab {
  double icf[3][MF_NMAX][MF_NMAX];   // [code][fine node a][coarse node b]
  double ifc[3][MF_NMAX][MF_NMAX];   // [code][coarse node b][fine node a]
  float icf32[3][MF_NMAX][MF_NMAX];  // FP32 copies (FP32 transfers multiply their weights in FP32)
  float ifc32[3][MF_NMAX][MF_NMAX];
  unsigned char in_child[3][MF_NMAX];  // coarse node b lies in the child's half (code 1, 2) or always (code 0)
};

template <typename T> struct XferW;
template <> struct XferW<double> {
  __device__ static double icf(const XferTab& t, int c, int a, int b) { return t.icf[c][a][b]; }
  __device__ static double ifc(const XferTab& t, int c, int b, int a) { return t.ifc[c][b][a]; }
};
template <> struct XferW<float> {
  __device__ static float icf(const XferTab& t, int c, int a, int b) { return t.icf32[c][a][b]; }
  __device__ static float ifc(const XferTab& t, int c, int b, int a) { return t.ifc32[c][b][a]; }
};

__host__ __device__ constexpr int xmax(int a, int b) { return a > b ? a : b; }

// Launch shape of k_transfer: 32 threads per cell, CPB cells per block (fewer
// for the largest tiles, so that the two stage buffers stay in 40 KB).
template <int D, int KF, int KC, int NFLD, typename T> struct XferCfg {
  static constexpr int NB = ipow(xmax(KF, KC) + 1, D);            // largest stage tile
  static constexpr int CPB = 2 * 4 * NB * NFLD * (int)sizeof(T) <= 40 * 1024 ? 4 : 2;
};

// The weights are tensor products of one 1D matrix per direction (chosen by
// the child code of that direction), so the transfer is sum-factorised: D
// contractions of the cell's tile, one direction at a time, through two
// shared buffers (nin^D -> nout nin^(D-1) -> ... -> nout^D).
template <int D, int KF, int KC, int NFLD, int MODE, typename T>
__global__ void k_transfer(const int32_t* __restrict__ cells_f, const int32_t* __restrict__ cells_c,
                           const int32_t* __restrict__ parent, const uint8_t* __restrict__ child, int64_t ncf,
                           const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ inv_mult,
                           int in_stride, int out_stride, const XferTab tb) {
  constexpr int NFN = KF + 1, NCN = KC + 1;
  constexpr int NPF = ipow(NFN, D), NPC = ipow(NCN, D);
  constexpr int nin = (MODE == 1) ? NCN : NFN, nout = (MODE == 1) ? NFN : NCN;   // 1D sizes
  constexpr int NIN = ipow(nin, D), NOUT = ipow(nout, D);
  constexpr int CPB = XferCfg<D, KF, KC, NFLD, T>::CPB, NB = XferCfg<D, KF, KC, NFLD, T>::NB;
  __shared__ T sa[CPB][NB][NFLD], sb[CPB][NB][NFLD];
  __shared__ T sm[CPB][D][nout][nin];              // the cell's 1D matrices, output x input
  const int cl = threadIdx.y;
  const int64_t cell = (int64_t)blockIdx.x * CPB + cl;
  const bool active = cell < ncf;
  const int64_t pcell = active ? (parent ? (int64_t)parent[cell] : cell) : 0;
  int code[3] = {0, 0, 0};
  if (active && parent) {
    const int bits = child[cell];
#pragma unroll
    for (int r = 0; r < D; ++r) code[r] = 1 + ((bits >> r) & 1);
  }
  for (int e = threadIdx.x; e < D * nout * nin; e += blockDim.x) {
    const int r = e / (nout * nin), o = (e / nin) % nout, i = e % nin;
    T w;
    if (MODE == 0) w = XferW<T>::ifc(tb, code[r], o, i);
    else if (MODE == 1) w = XferW<T>::icf(tb, code[r], o, i);
    else w = XferW<T>::icf(tb, code[r], i, o);
    sm[cl][r][o][i] = w;
  }
  for (int i = threadIdx.x; i < NIN; i += blockDim.x) {
    if (active) {
      int id = (MODE == 1) ? cells_c[pcell * NPC + i] : cells_f[cell * NPF + i];
      id = id < 0 ? ~id : id;
      const T sc = (MODE == 2) ? inv_mult[id] : T(1);
#pragma unroll
      for (int f = 0; f < NFLD; ++f) sa[cl][i][f] = in[(int64_t)id * in_stride + f] * sc;
    } else {
#pragma unroll
      for (int f = 0; f < NFLD; ++f) sa[cl][i][f] = T(0);
    }
  }
  __syncthreads();
  // direction r: sizes nout along directions < r, nin along directions >= r
  T (*cur)[NFLD] = sa[cl];
  T (*nxt)[NFLD] = sb[cl];
#pragma unroll
  for (int r = 0; r < D; ++r) {
    int sz[3] = {1, 1, 1};
#pragma unroll
    for (int q = 0; q < D; ++q) sz[q] = q <= r ? nout : nin;     // sizes after this contraction
    const int total = sz[0] * sz[1] * sz[2];
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      int x[3] = {e % sz[0], (e / sz[0]) % sz[1], e / (sz[0] * sz[1])};
      // input index with x_r running over nin: strides of the current layout
      int st0 = 1, str = 1, base = 0;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const int n = q < r ? nout : nin;
        if (q == r) str = st0;
        else base += x[q] * st0;
        st0 *= n;
      }
      T acc[NFLD];
#pragma unroll
      for (int f = 0; f < NFLD; ++f) acc[f] = T(0);
#pragma unroll
      for (int j = 0; j < nin; ++j) {
        const T w = sm[cl][r][x[r]][j];
#pragma unroll
        for (int f = 0; f < NFLD; ++f) acc[f] = fma(w, cur[base + j * str][f], acc[f]);
      }
#pragma unroll
      for (int f = 0; f < NFLD; ++f) nxt[e][f] = acc[f];
    }
    __syncthreads();
    T (*t)[NFLD] = cur; cur = nxt; nxt = t;
  }
  if (!active) return;
  for (int o = threadIdx.x; o < NOUT; o += blockDim.x) {
    if (MODE == 0) {
      const int oi[3] = {o % nout, (o / nout) % nout, o / (nout * nout)};
      bool inside = true;
#pragma unroll
      for (int r = 0; r < D; ++r) inside = inside && tb.in_child[code[r]][oi[r]];
      if (!inside) continue;
    }
    int id = (MODE == 1) ? cells_f[cell * NPF + o] : cells_c[pcell * NPC + o];
    id = id < 0 ? ~id : id;
#pragma unroll
    for (int f = 0; f < NFLD; ++f) {
      if (MODE == 2) atomicAdd(&out[(int64_t)id * out_stride + f], cur[o][f]);
      else out[(int64_t)id * out_stride + f] = cur[o][f];
    }
  }
}

// number of cells sharing each node (as T), then its reciprocal
template <typename T>
__global__ void k_count_nodes(const int32_t* __restrict__ cells, int64_t n, T* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int id = cells[i];
  id = id < 0 ? ~id : id;
  atomicAdd(&cnt[id], T(1));
}

// zero the velocity components of wall rows
template <int D, typename T>
__global__ void k_dirichlet_zero(const int32_t* __restrict__ wall, int64_t nw, T* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nw) return;
  const int64_t n = wall[i];
#pragma unroll
  for (int c = 0; c < D; ++c) y[n * (D + 1) + c] = T(0);
}

}  // namespace mf
