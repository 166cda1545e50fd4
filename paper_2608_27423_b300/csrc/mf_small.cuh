// Element-wise and reduction kernels: history term, Dirichlet rows, casts,
// the cell part of diag(J) (Algorithm 1 written as a direct sum per local DoF),
// and the vector kernels of the Krylov solver (FP64 dots/axpys for CGS2).
#pragma once
#include "mf_cell.cuh"

namespace mf {

// h_t = (alpha_1 u^n + alpha_2 u^{n-1}) / dt
__global__ void k_history(const double* __restrict__ un, const double* __restrict__ unm1, double* __restrict__ ht,
                          int64_t n, double c1, double c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ht[i] = c1 * un[i] + (unm1 ? c2 * unm1[i] : 0.0);
}

// Jacobian: identity rows on wall velocity DoFs (y = x there).
template <int D, typename T>
__global__ void k_dirichlet_copy(const int32_t* __restrict__ wall, int64_t nw, const T* __restrict__ x, T* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nw) return;
  const int64_t n = wall[i];
#pragma unroll
  for (int c = 0; c < D; ++c) y[n * (D + 1) + c] = x[n * (D + 1) + c];
}
// Residual: r = u - g on wall velocity DoFs.  Entries i >= m0 of the wall
// list move with the rotor: there g is the rigid rotation omega e_z x x at
// the current node position x (the mesh velocity of Section 3.1).
template <int D>
__global__ void k_dirichlet_res(const int32_t* __restrict__ wall, int64_t nw, int64_t m0, const double* __restrict__ up,
                                const double* __restrict__ g, const double* __restrict__ x, double omega,
                                double* __restrict__ r) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nw) return;
  const int64_t n = wall[i];
  double gv[D];
  if (i >= m0) {
    gv[0] = -omega * x[n * D + 1];
    gv[1] = omega * x[n * D + 0];
    if (D == 3) gv[D - 1] = 0.0;
  } else {
#pragma unroll
    for (int c = 0; c < D; ++c) gv[c] = g ? g[n * D + c] : 0.0;
  }
#pragma unroll
  for (int c = 0; c < D; ++c) r[n * (D + 1) + c] = up[n * (D + 1) + c] - gv[c];
}
// Wall loads from the reaction rows r (volume + mortar residual without the
// Dirichlet replacement): per group g, out[g][0..D-1] += r_i (force on the
// fluid), out[g][D] += (x_i x r_i) . e_z (torque), out[g][D+1] += r_i . u_i
// (power).  Group of wall-list entry i: group[node] if group is given (values
// >= n_groups skipped), else 0 for stationary walls (i < m0) and 1 for walls
// moving with the rotor.  Block partial sums in shared memory, one global
// atomic per block and value.
template <int D>
__global__ void __launch_bounds__(256) k_wall_loads(const int32_t* __restrict__ wall, int64_t nw, int64_t m0,
                                                    const uint8_t* __restrict__ group, int n_groups,
                                                    const double* __restrict__ x, const double* __restrict__ up,
                                                    const double* __restrict__ r, double* __restrict__ out) {
  constexpr int NV = D + 2;
  __shared__ double acc[MF_MAX_LOAD_GROUPS * NV];
  for (int j = threadIdx.x; j < n_groups * NV; j += blockDim.x) acc[j] = 0.0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = wall[i];
    const int gi = group ? (int)group[n] : (i >= m0 ? 1 : 0);
    if (gi >= n_groups) continue;
    double v[NV];
    double pw = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      v[c] = r[n * (D + 1) + c];
      pw = fma(v[c], up[n * (D + 1) + c], pw);
    }
    v[D] = x[n * D] * v[1] - x[n * D + 1] * v[0];
    v[D + 1] = pw;
#pragma unroll
    for (int j = 0; j < NV; ++j) atomicAdd(&acc[gi * NV + j], v[j]);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n_groups * NV; j += blockDim.x)
    if (acc[j] != 0.0) atomicAdd(&out[j], acc[j]);
}

// diag = 1 on wall velocity DoFs.
template <int D, typename T>
__global__ void k_dirichlet_one(const int32_t* __restrict__ wall, int64_t nw, T* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nw) return;
  const int64_t n = wall[i];
#pragma unroll
  for (int c = 0; c < D; ++c) y[n * (D + 1) + c] = T(1);
}

template <typename A, typename B>
__global__ void k_cast(const A* __restrict__ a, B* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (B)a[i];
}

// ---------------------------------------------------------------------------
// Cell part of diag(J): for each local DoF (node a, field f) the entry of the
// element matrix of blocks A-hat (velocity) and D-hat (pressure) on the
// diagonal, summed over the Gauss points from the linearisation cache.
// The cache fields the diagonal reads at each point (slot order: J^-1, W, G,
// ctil, a, the diagonal of grad u*, tau, R*) and their count.
template <int D> struct DiagSlots {
  static constexpr int n = D * D + 1 + Sym<D>::n + 3 * D + 1 + D;
  __device__ static int field(int s) {
    using CF = Cache<D>;
    if (s < D * D) return CF::JINV + s;
    s -= D * D;
    if (s == 0) return CF::W;
    s -= 1;
    if (s < Sym<D>::n) return CF::G + s;
    s -= Sym<D>::n;
    if (s < D) return CF::CT + s;
    s -= D;
    if (s < D) return CF::A + s;
    s -= D;
    if (s < D) return CF::GU + s * D + s;
    s -= D;
    if (s == 0) return CF::TAU;
    return CF::RS + (s - 1);
  }
};
// Every node's thread needs every point's coefficients of its cell: where the
// block's share fits (FP32, and FP64 at small k) they are staged in shared
// memory once, coalesced, instead of re-read NQ times per cell from L1/L2.
template <int D, int K, typename T> struct DiagCfg {
  static constexpr int BYTES = CellCfg<D, K>::CPB * DiagSlots<D>::n * CellCfg<D, K>::NQ * (int)sizeof(T);
  static constexpr bool STAGE = BYTES <= 40 * 1024;
  static constexpr int CPB_S = STAGE ? CellCfg<D, K>::CPB : 1, NQ_S = STAGE ? CellCfg<D, K>::NQ : 1;
};

template <int D, int K, typename T>
__global__ void __launch_bounds__(CellCfg<D, K>::THREADS)
k_cell_diag(const int32_t* __restrict__ cells, int64_t nc, const T* __restrict__ cache, T* __restrict__ diag,
            T nu, T a0dt) {
  using C = CellCfg<D, K>;
  constexpr int N = C::N, NQ = C::NQ, NF = D + 1;
  using CF = Cache<D>;
  using DS = DiagSlots<D>;
  using G = DiagCfg<D, K, T>;
  __shared__ SmTab<N, T> st;
  __shared__ T sc[G::CPB_S][DS::n][G::NQ_S];
  load_tab<K, T>(st);
  const int64_t P = nc * NQ;
  if constexpr (G::STAGE) {
    const int64_t c0 = (int64_t)blockIdx.x * C::CPB;
    for (int i = threadIdx.x; i < C::CPB * NQ * DS::n; i += blockDim.x) {
      const int s = i / (C::CPB * NQ), rem = i % (C::CPB * NQ);
      const int c = rem / NQ, q = rem % NQ;
      sc[c][s][q] = (c0 + c < nc) ? cache[(int64_t)DS::field(s) * P + c0 * NQ + rem] : T(0);
    }
  }
  __syncthreads();
  const int cl = threadIdx.x / NQ, t = threadIdx.x % NQ;
  const int64_t cell = (int64_t)blockIdx.x * C::CPB + cl;
  if (cell >= nc) return;
  const int ai[3] = {t % N, (t / N) % N, t / (N * N)};
  T dsum[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) dsum[f] = T(0);
  for (int q = 0; q < NQ; ++q) {
    const int qi[3] = {q % N, (q / N) % N, q / (N * N)};
    T bv[3], dvv[3], hv[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      bv[u] = u < D ? st.B[qi[u]][ai[u]] : T(1);
      dvv[u] = u < D ? st.Dn[qi[u]][ai[u]] : T(0);
      hv[u] = u < D ? st.Hn[qi[u]][ai[u]] : T(0);
    }
    const T phi = bv[0] * bv[1] * bv[2];
    T dphi[D], Hphi[Sym<D>::n];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      T p = T(1);
#pragma unroll
      for (int u = 0; u < D; ++u) p *= (u == r) ? dvv[u] : bv[u];
      dphi[r] = p;
    }
#pragma unroll
    for (int e = 0; e < Sym<D>::n; ++e) {
      const int r = sym_r(D, e), s = sym_s(D, e);
      T p = T(1);
#pragma unroll
      for (int u = 0; u < D; ++u) p *= (r == s) ? (u == r ? hv[u] : bv[u]) : ((u == r || u == s) ? dvv[u] : bv[u]);
      Hphi[e] = p;
    }
    // slot s of this point: the staged copy, else the cache itself
    auto fv = [&](int s) -> T {
      if constexpr (G::STAGE) return sc[cl][s][q];
      else return cache[(int64_t)DS::field(s) * P + cell * NQ + q];
    };
    constexpr int SW = D * D, SG = SW + 1, SCT = SG + Sym<D>::n, SA = SCT + D, SGU = SA + D, STAU = SGU + D,
                  SRS = STAU + 1;
    T Ji[D][D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int m = 0; m < D; ++m) Ji[r][m] = fv(r * D + m);
    const T Wq = fv(SW);
    T gphi[D];
#pragma unroll
    for (int m = 0; m < D; ++m) {
      T s = T(0);
#pragma unroll
      for (int r = 0; r < D; ++r) s = fma(dphi[r], Ji[r][m], s);
      gphi[m] = s;
    }
    T lap = T(0);
#pragma unroll
    for (int e = 0; e < Sym<D>::n; ++e) lap = fma(fv(SG + e), Hphi[e], lap);
#pragma unroll
    for (int r = 0; r < D; ++r) lap = fma(-fv(SCT + r), dphi[r], lap);
    T sa = T(0), g2 = T(0);
#pragma unroll
    for (int m = 0; m < D; ++m) { sa = fma(fv(SA + m), gphi[m], sa); g2 = fma(gphi[m], gphi[m], g2); }
    const T tau = fv(STAU);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const T guc = fv(SGU + c);
      const T lb = a0dt * phi + sa + guc * phi;
      T e = phi * lb + nu * g2 + tau * sa * (lb - nu * lap) + tau * phi * gphi[c] * fv(SRS + c);
      dsum[c] = fma(Wq, e, dsum[c]);
    }
    dsum[D] = fma(Wq * tau, g2, dsum[D]);
  }
  int id = cells[cell * NQ + t];
  const int64_t node = id < 0 ? ~id : id;
#pragma unroll
  for (int f = 0; f < NF; ++f) atomicAdd(&diag[node * NF + f], dsum[f]);
}

// ---------------------------------------------------------------------------
// Krylov vector kernels (grid-stride).
template <typename T>
__global__ void k_axpby(int64_t n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
// y = x / sqrt(*nrm2)  (norm read on the device: no host round trip); a zero
// norm gives y = 0 instead of a division by zero.
template <typename T>
__global__ void k_scale_by(int64_t n, const T* __restrict__ x, T* __restrict__ y, const double* __restrict__ nrm2) {
  const double nn = *nrm2;
  const T inv = nn > 1e-300 ? (T)(1.0 / sqrt(nn)) : T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = x[i] * inv;
}
template <typename T>
__global__ void k_mul(int64_t n, const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a[i] * b[i];
}
template <typename T>
__global__ void k_recip(int64_t n, const T* __restrict__ a, T* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = T(1) / a[i];
}

// Partial dot products: part[i][blockIdx.x] = sum over the block's range of V_i . w
// (V_i = V + i * ldv), one grid row per vector (blockIdx.y = i).
// Thread-level accumulation in T (FP32 vectors accumulate a few dozen terms per
// thread in FP32), block and final reductions in FP64.
template <typename T>
__global__ void k_mdot_part(int64_t n, const T* __restrict__ V, int64_t ldv, const T* __restrict__ w,
                            double* __restrict__ part) {
  const int i = blockIdx.y;
  const T* v = V + (int64_t)i * ldv;
  T st = T(0);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    st = fma(v[j], w[j], st);
  double s = (double)st;
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[(int64_t)i * gridDim.x + blockIdx.x] = s;
  }
}
// Weighted partial dot products: part[i][blockIdx.x] = sum over the block's
// range of wt[j] V_i[j] x[j] (wt may be null: weights 1); FP64 throughout.
__global__ void k_wdot_part(int64_t n, const double* __restrict__ V, int64_t ldv, const double* __restrict__ x,
                            const double* __restrict__ wt, double* __restrict__ part) {
  const int i = blockIdx.y;
  const double* v = V + (int64_t)i * ldv;
  double s = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    s = fma(wt ? wt[j] * v[j] : v[j], x[j], s);
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[(int64_t)i * gridDim.x + blockIdx.x] = s;
  }
}

// Short vectors: out[i] = V_i . w with one block per vector (no second pass);
// four independent accumulators per thread keep four loads in flight.  Any
// block size that is a multiple of 32, up to 1024.
template <typename T>
__global__ void k_mdot_block(int64_t n, const T* __restrict__ V, int64_t ldv, const T* __restrict__ w,
                             double* __restrict__ out) {
  const int i = blockIdx.x;
  const T* v = V + (int64_t)i * ldv;
  T a[4] = {T(0), T(0), T(0), T(0)};
  const int64_t stride = blockDim.x;
  int64_t j = threadIdx.x;
  for (; j + 3 * stride < n; j += 4 * stride) {
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = fma(v[j + u * stride], w[j + u * stride], a[u]);
  }
  for (; j < n; j += stride) a[0] = fma(v[j], w[j], a[0]);
  double s = ((double)a[0] + (double)a[1]) + ((double)a[2] + (double)a[3]);
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[i] = s;
  }
}
// y = x / sqrt(*nrm2) and z = d * y in one pass (the next Arnoldi column and
// its inverse-diagonal preconditioning)
template <typename T>
__global__ void k_scale_by_mul(int64_t n, const T* __restrict__ x, T* __restrict__ y, const double* __restrict__ nrm2,
                               const T* __restrict__ d, T* __restrict__ z) {
  const double nn = *nrm2;
  const T inv = nn > 1e-300 ? (T)(1.0 / sqrt(nn)) : T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T v = x[i] * inv;
    y[i] = v;
    z[i] = d[i] * v;
  }
}
// out[i] (+)= sum_b part[i][b]  (one block per vector, fixed order: deterministic)
__global__ void k_mdot_final(const double* __restrict__ part, int nb, double* __restrict__ out, int accumulate) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(int64_t)i * nb + b];
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[i] = accumulate ? out[i] + s : s;
  }
}
// w += sign * sum_{i<m} h[i] V_i  (h in FP64 on the device)
template <typename T>
__global__ void k_maxpy(int64_t n, int m, const T* __restrict__ V, int64_t ldv, const double* __restrict__ h,
                        double sign, T* __restrict__ w) {
  // the m coefficients, scaled and rounded to T once per block (m <= 256:
  // restart lengths and inner dimensions are capped below that)
  __shared__ T c[256];
  for (int i = threadIdx.x; i < m; i += blockDim.x) c[i] = (T)(sign * h[i]);
  __syncthreads();
  // eight independent partial sums: eight loads in flight per thread (the
  // coarse levels' GMRES has up to 40 short vectors, where one dependent
  // chain of loads and FMAs set the time)
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    T s[8] = {w[j], T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    int i = 0;
    for (; i + 8 <= m; i += 8) {
      T a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = V[(int64_t)(i + u) * ldv + j];
#pragma unroll
      for (int u = 0; u < 8; ++u) s[u] = fma(c[i + u], a[u], s[u]);
    }
    // the remainder on two fixed accumulators (a dynamic index would put s in local memory)
    for (; i + 2 <= m; i += 2) {
      const T a0 = V[(int64_t)i * ldv + j], a1 = V[(int64_t)(i + 1) * ldv + j];
      s[0] = fma(c[i], a0, s[0]);
      s[1] = fma(c[i + 1], a1, s[1]);
    }
    if (i < m) s[2] = fma(c[i], V[(int64_t)i * ldv + j], s[2]);
    w[j] = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
  }
}
// subtract the mean of the pressure component (stride d+1) given its sum
__global__ void k_sub_pmean(int64_t nn, int nf, double* __restrict__ v, const double* __restrict__ psum) {
  const double mean = *psum / (double)nn;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x)
    v[i * nf + nf - 1] -= mean;
}
// sum of the pressure component, partials per block
__global__ void k_psum_part(int64_t nn, int nf, const double* __restrict__ v, double* __restrict__ part) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x)
    s += v[i * nf + nf - 1];
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

}  // namespace mf
