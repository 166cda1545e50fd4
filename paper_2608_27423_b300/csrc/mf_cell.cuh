// Cell kernels of the stabilised ALE Navier-Stokes operator on Q_k cells.
//
// One thread per Gauss point (= per node: q = k+1 points and k+1 nodes per
// direction), CPB cells per block.  Sum factorisation (tensor-product 1D
// contractions) runs as line sweeps through shared memory:
//   nodal values --B (d sweeps)--> Gauss values --Dg--> reference gradients
//   --Dg--> reference Hessians;  fluxes --Dg^T--> --B^T (d sweeps)--> nodal.
// B[q][a] = l_a(s_q) (Gauss-Lobatto Lagrange basis at Gauss points), Dg is the
// collocation derivative on the Gauss points.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>
#include "mf_tables.h"
#include "mf_df64.cuh"

#ifndef MF_DF_MINB
#define MF_DF_MINB 2
#endif
#ifndef MF_F32_MINB
#define MF_F32_MINB 5
#endif

namespace mf {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <int D> struct Sym { static constexpr int n = D * (D + 1) / 2; };
// Symmetric pair order: (0,0),(1,1)[,(2,2)],(0,1)[,(0,2),(1,2)]
__host__ __device__ constexpr int sym_r(int D, int e) {
  return D == 2 ? (e == 0 ? 0 : e == 1 ? 1 : 0) : (e < 3 ? e : e == 3 ? 0 : e == 4 ? 0 : 1);
}
__host__ __device__ constexpr int sym_s(int D, int e) {
  return D == 2 ? (e == 0 ? 0 : 1) : (e < 3 ? e : e == 3 ? 1 : 2);
}

// Per-Gauss-point linearisation cache, field offsets (each field is a plane of
// n_cells * NQ values, point-fastest so a warp reads contiguous memory).
template <int D> struct Cache {
  static constexpr int JINV = 0;                    // Jinv[r][m] = d xi_r / d x_m   (D*D)
  static constexpr int W = D * D;                   // det J * Gauss weight          (1)
  static constexpr int G = W + 1;                   // G = Jinv Jinv^T, sym, off-diagonals doubled
  static constexpr int CT = G + Sym<D>::n;          // ctil_r = sum_m Jinv[r][m] tr(G H_xi x_m)
  static constexpr int A = CT + D;                  // a = u* - u_ALE (physical)
  static constexpr int GU = A + D;                  // grad u*: GU[c][m] = d u*_c / d x_m
  static constexpr int RS = GU + D * D;             // strong residual R* (Eq. Eq-strong-residual)
  static constexpr int TAU = RS + D;                // tau (Eq. Eq-stab-param)
  static constexpr int NF = TAU + 1;
};

template <int D, int K> struct CellCfg {
  static constexpr int N = K + 1;
  static constexpr int NQ = ipow(N, D);
  static constexpr int CPB = NQ >= 128 ? 1 : (256 / NQ);
  static constexpr int THREADS = CPB * NQ;
};

template <typename T> struct TabSel;
// Defined once: the library is a single translation unit.
__constant__ MfTab<double> c_tab64[MF_KMAX + 1];
__constant__ MfTab<float> c_tab32[MF_KMAX + 1];
__constant__ MfTab<df> c_tabdf[MF_KMAX + 1];
template <> struct TabSel<double> { __device__ static const MfTab<double>& get(int k) { return c_tab64[k]; } };
template <> struct TabSel<float> { __device__ static const MfTab<float>& get(int k) { return c_tab32[k]; } };
template <> struct TabSel<df> { __device__ static const MfTab<df>& get(int k) { return c_tabdf[k]; } };

// Shared copies of the 1D matrices for degree K.
template <int N, typename T> struct SmTab {
  T B[N][N], Dg[N][N], Dn[N][N], Hn[N][N], w[N];
};

template <int K, typename T>
__device__ __forceinline__ void load_tab(SmTab<K + 1, T>& st) {
  constexpr int N = K + 1;
  const MfTab<T>& t = TabSel<T>::get(K);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    int q = i / N, a = i % N;
    st.B[q][a] = t.B[q][a]; st.Dg[q][a] = t.Dg[q][a]; st.Dn[q][a] = t.Dn[q][a]; st.Hn[q][a] = t.Hn[q][a];
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) st.w[i] = t.w[i];
}

// Apply a 1D matrix along direction r to NFLD planes of the cell's shared
// tile: out[f] = sum_j M[i_r][j] * tile[f][t with i_r := j]  (TRANS: M[j][i_r]).
template <int D, int N, int NFLD, bool TRANS, typename T>
__device__ __forceinline__ void line(const T* __restrict__ tile, int NQ, int t, int ir, int stride,
                                     const T (*M)[N], T* out) {
  const int base = t - ir * stride;
#pragma unroll
  for (int f = 0; f < NFLD; ++f) out[f] = T(0);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const T m = TRANS ? M[j][ir] : M[ir][j];
#pragma unroll
    for (int f = 0; f < NFLD; ++f) out[f] = fma(m, tile[f * NQ + base + j * stride], out[f]);
  }
}

template <typename T> __device__ __forceinline__ void atomic_add(typename IO<T>::type* p, T v) { atomicAdd(p, to_io<T>(v)); }

// ---------------------------------------------------------------------------
// Jacobian apply, volume part (blocks A-hat .. D-hat of Section 2.3, tau frozen).
// dst += J_cell src.  src entries on wall nodes (negative ids in `cells`) are
// taken as zero for the velocity components.
// FP32 applies stage the block's slice of the per-point cache in shared
// memory with asynchronous copies issued at kernel entry, so the loads overlap
// the gather and the sum-factorisation sweeps instead of stalling the point
// physics (the FP32 kernel is latency-bound on them; the FP64 kernel is bound
// by the FP64 pipe and keeps direct loads).  On when the block's shared
// memory stays within the 48 KB static limit.
template <int D, int K, typename T, int CPB> struct StageCfg {
  static constexpr int NQ = ipow(K + 1, D), NS = (D + 1) * D, THREADS = CPB * NQ;
  static constexpr size_t bytes = sizeof(T) * ((size_t)THREADS * Cache<D>::NF + (size_t)CPB * NS * NQ + 5 * (K + 1) * (K + 1));
  static constexpr bool on = std::is_same<T, float>::value && bytes <= 48 * 1024;
};

template <int D, int K, typename T, int CPB = CellCfg<D, K>::CPB>
struct JacSmem {
  static constexpr int N = K + 1, NQ = ipow(N, D), NS = (D + 1) * D;
  SmTab<N, T> st;
  T tile[CPB][NS * NQ];
  T stage[StageCfg<D, K, T, CPB>::on ? Cache<D>::NF * CPB * NQ : 1];
};

// 4-byte asynchronous global -> shared copy (completes at cp_async_wait_all,
// visible to the issuing thread).
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Point physics of the Jacobian (blocks A-hat..D-hat of Section 2.3, tau
// frozen) at one Gauss point.  In: reference values v (u_1..u_D, p),
// reference gradients dv[f][r], reference Hessians of the velocity H[c][e]
// (symmetric pair order), and the point's coefficients: Ji = J^-1, Wq = det J
// times the Gauss weight, G = Ji Ji^T (off-diagonals doubled), ct (Laplacian
// mapping correction), a = u* - u_ALE, gU = grad u*, Rs = R*, tau.  Out: value
// fluxes fv and reference gradient fluxes Fx, quadrature weight folded in, so
// that the cell vector is B^T (fv + sum_r Dg_r^T Fx[.][r]).
template <int D, typename T>
__device__ __forceinline__ void jac_point(const T (&v)[D + 1], const T (&dv)[D + 1][D], const T (&H)[D][Sym<D>::n],
                                          const T (&Ji)[D][D], T Wq, const T (&G)[Sym<D>::n], const T (&ct)[D],
                                          const T (&a)[D], const T (&gU)[D][D], const T (&Rs)[D], T tau, T nu, T a0dt,
                                          T (&fv)[D + 1], T (&Fx)[D + 1][D]) {
  T gw[D][D], gr[D], lap[D], gal[D], Rl[D];
#pragma unroll
  for (int c = 0; c <= D; ++c)
#pragma unroll
    for (int m = 0; m < D; ++m) {
      T s = T(0);
#pragma unroll
      for (int r = 0; r < D; ++r) s = fma(dv[c][r], Ji[r][m], s);
      if (c < D) gw[c][m] = s; else gr[m] = s;
    }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    T l = T(0);
#pragma unroll
    for (int e = 0; e < Sym<D>::n; ++e) l = fma(G[e], H[c][e], l);
#pragma unroll
    for (int r = 0; r < D; ++r) l = fma(-ct[r], dv[c][r], l);
    lap[c] = l;
    T cv = a0dt * v[c];
#pragma unroll
    for (int m = 0; m < D; ++m) cv = fma(a[m], gw[c][m], fma(v[m], gU[c][m], cv));
    gal[c] = cv;
    Rl[c] = fma(-nu, l, cv + gr[c]);
  }
  // physical flux of grad v: nu grad w - r I + tau (R' (x) a + R* (x) w),
  // with the quadrature weight W folded into its coefficients before the
  // J^-1 contraction (W nu, W tau R', W tau R*, W r: fewer FP64 multiplies)
  const T Wnu = Wq * nu, Wtau = Wq * tau, Wp = Wq * v[D];
  T WRl[D], WRs[D];
#pragma unroll
  for (int c = 0; c < D; ++c) { WRl[c] = Wtau * Rl[c]; WRs[c] = Wtau * Rs[c]; }
  T Fp[D][D];
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int m = 0; m < D; ++m)
      Fp[c][m] = fma(Wnu, gw[c][m], fma(WRl[c], a[m], WRs[c] * v[m])) - (c == m ? Wp : T(0));
  T divw = T(0);
#pragma unroll
  for (int c = 0; c < D; ++c) { fv[c] = Wq * gal[c]; divw += gw[c][c]; }
  fv[D] = Wq * divw;
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int r = 0; r < D; ++r) {
      T s = Ji[r][0] * Fp[c][0];
#pragma unroll
      for (int m = 1; m < D; ++m) s = fma(Ji[r][m], Fp[c][m], s);
      Fx[c][r] = s;
    }
#pragma unroll
  for (int r = 0; r < D; ++r) {
    T s = Ji[r][0] * WRl[0];
#pragma unroll
    for (int m = 1; m < D; ++m) s = fma(Ji[r][m], WRl[m], s);
    Fx[D][r] = s;
  }
}

// One block's worth of cells (block index `blk`) of the cell Jacobian.  The
// tables in sm.st must be loaded and visible to the block.
// ELEM = true: element-matrix columns (the volume part of the local matrix of
// Algorithm 2): every sub-block of NQ threads works on cell `blk` with the
// unit input vector of local DoF col = col0 + sub-block (node col / (D+1),
// field col % (D+1); wall velocities stay zero) and writes the resulting
// local vector to column col of E (column-major [NL][NL] per cell, NL =
// NQ (D+1)) instead of scattering it.
template <int D, int K, typename T, int CPB = CellCfg<D, K>::CPB, bool ELEM = false>
__device__ __forceinline__ void cell_jac_block(JacSmem<D, K, T, CPB>& sm, int64_t blk, const int32_t* __restrict__ cells,
                                               int64_t nc, const T* __restrict__ cache,
                                               const typename IO<T>::type* __restrict__ src,
                                               typename IO<T>::type* __restrict__ dst, T nu, T a0dt,
                                               int col0 = 0, T* __restrict__ E = nullptr) {
  using C = CellCfg<D, K>;
  constexpr int N = C::N, NQ = C::NQ, NF = D + 1, NL = NQ * (D + 1);
  using CF = Cache<D>;
  SmTab<N, T>& st = sm.st;
  const int cl = threadIdx.x / NQ, t = threadIdx.x % NQ;
  const int64_t cell = ELEM ? blk : blk * CPB + cl;
  const int col = col0 + cl;
  const bool active = ELEM ? (col < NL && cell < nc) : cell < nc;
  T* tile = sm.tile[cl];
  int ii[3] = {t % N, (t / N) % N, t / (N * N)};
  const int strd[3] = {1, N, N * N};
  constexpr bool STAGE = StageCfg<D, K, T, CPB>::on;
  constexpr int THREADS = CPB * NQ;
  if constexpr (STAGE) {
    // this point's cache entries -> stage[f][threadIdx.x]; a point past the
    // last cell stages zeros (its results are never scattered)
    if (active) {
      const int64_t P = nc * NQ;
      const T* cp = cache + cell * NQ + t;
#pragma unroll
      for (int f = 0; f < CF::NF; ++f) cp_async4(&sm.stage[f * THREADS + threadIdx.x], cp + f * P);
    } else {
#pragma unroll
      for (int f = 0; f < CF::NF; ++f) sm.stage[f * THREADS + threadIdx.x] = T(0);
    }
    cp_async_commit();
  }

  T v[NF];
  int node = 0;
  if (active) {
    const int id = cells[cell * NQ + t];
    const bool wall = id < 0;
    node = wall ? ~id : id;
#pragma unroll
    for (int f = 0; f < NF; ++f)
      v[f] = ELEM ? T(t * NF + f == col ? 1 : 0) : from_io<T>(src[(int64_t)node * NF + f]);
    if (wall) {
#pragma unroll
      for (int c = 0; c < D; ++c) v[c] = T(0);
    }
  } else {
#pragma unroll
    for (int f = 0; f < NF; ++f) v[f] = T(0);
  }
  __syncthreads();
  // nodal -> Gauss values
#pragma unroll
  for (int r = 0; r < D; ++r) {
#pragma unroll
    for (int f = 0; f < NF; ++f) tile[f * NQ + t] = v[f];
    __syncthreads();
    line<D, N, NF, false>(tile, NQ, t, ii[r], strd[r], st.B, v);
    __syncthreads();
  }
  // reference gradients of all fields
  T dv[NF][D];
#pragma unroll
  for (int f = 0; f < NF; ++f) tile[f * NQ + t] = v[f];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < D; ++r) {
    T o[NF];
    line<D, N, NF, false>(tile, NQ, t, ii[r], strd[r], st.Dg, o);
#pragma unroll
    for (int f = 0; f < NF; ++f) dv[f][r] = o[f];
  }
  __syncthreads();
  // reference Hessians of the velocity components
  T H[D][Sym<D>::n];
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int r = 0; r < D; ++r) tile[(c * D + r) * NQ + t] = dv[c][r];
  __syncthreads();
#pragma unroll
  for (int e = 0; e < Sym<D>::n; ++e) {
    const int r = sym_r(D, e), s = sym_s(D, e);
    T o[D];
    // d/ds of (d w_c / d xi_r): planes c*D + r
    const int base = t - ii[s] * strd[s];
#pragma unroll
    for (int c = 0; c < D; ++c) o[c] = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const T m = st.Dg[ii[s]][j];
#pragma unroll
      for (int c = 0; c < D; ++c) o[c] = fma(m, tile[(c * D + r) * NQ + base + j * strd[s]], o[c]);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) H[c][e] = o[c];
  }
  __syncthreads();

  // ---- point physics
  T fv[NF], Fx[NF][D];
  {
    const int64_t P = nc * NQ;
    const T* cp = cache + (active ? cell * NQ + t : 0);
    if constexpr (STAGE) cp_async_wait_all();
    // cache entry f of this point: staged copy or direct load
    auto ld = [&](int f) -> T {
      if constexpr (STAGE) return sm.stage[f * THREADS + threadIdx.x];
      else return cp[f * P];
    };
    T Ji[D][D], a[D], gU[D][D], Rs[D], G[Sym<D>::n], ct[D];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int m = 0; m < D; ++m) Ji[r][m] = ld(CF::JINV + r * D + m);
    const T Wq = ld(CF::W);
#pragma unroll
    for (int e = 0; e < Sym<D>::n; ++e) G[e] = ld(CF::G + e);
#pragma unroll
    for (int r = 0; r < D; ++r) ct[r] = ld(CF::CT + r);
#pragma unroll
    for (int m = 0; m < D; ++m) a[m] = ld(CF::A + m);
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int m = 0; m < D; ++m) gU[c][m] = ld(CF::GU + c * D + m);
#pragma unroll
    for (int c = 0; c < D; ++c) Rs[c] = ld(CF::RS + c);
    const T tau = ld(CF::TAU);

    jac_point<D, T>(v, dv, H, Ji, Wq, G, ct, a, gU, Rs, tau, nu, a0dt, fv, Fx);
  }
  // ---- integrate: gradient fluxes through Dg^T, then B^T to the nodes
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int r = 0; r < D; ++r) tile[(f * D + r) * NQ + t] = Fx[f][r];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < D; ++r) {
    const int base = t - ii[r] * strd[r];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const T m = st.Dg[j][ii[r]];
#pragma unroll
      for (int f = 0; f < NF; ++f) fv[f] = fma(m, tile[(f * D + r) * NQ + base + j * strd[r]], fv[f]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < D; ++r) {
#pragma unroll
    for (int f = 0; f < NF; ++f) tile[f * NQ + t] = fv[f];
    __syncthreads();
    line<D, N, NF, true>(tile, NQ, t, ii[r], strd[r], st.B, fv);
    __syncthreads();
  }
  if (active) {
    if constexpr (ELEM) {
#pragma unroll
      for (int f = 0; f < NF; ++f) E[((int64_t)cell * NL + col) * NL + t * NF + f] = fv[f];
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f) atomic_add(&dst[(int64_t)node * NF + f], fv[f]);
    }
  }
}

// Minimum resident blocks requested from the register allocator: the
// double-float variant is latency-bound at one block per SM otherwise.
template <typename T> struct MinBlocks { static constexpr int value = 1; };
template <> struct MinBlocks<df> { static constexpr int value = MF_DF_MINB; };
template <> struct MinBlocks<float> { static constexpr int value = MF_F32_MINB; };

// Launch shape of the cell Jacobian with CPB cells per block: resident blocks
// requested per SM = MinBlocks<T>, lowered so that the blocks fit the SM's
// 2048 threads and 228 KB of shared memory and keep at least 48 registers per
// thread (fewer spill).
template <int D, int K, typename T, int CPB> struct JacLaunch {
  static constexpr int THREADS = CPB * CellCfg<D, K>::NQ;
  static constexpr int by_threads = 2048 / THREADS;
  static constexpr int by_smem = (int)(233472 / (sizeof(JacSmem<D, K, T, CPB>) + 1024));
  static constexpr int by_regs = 65536 / (THREADS * 48);
  static constexpr int m0 = MinBlocks<T>::value < by_threads ? MinBlocks<T>::value : by_threads;
  static constexpr int m1 = m0 < by_smem ? m0 : by_smem;
  static constexpr int m2 = m1 < by_regs ? m1 : by_regs;
  static constexpr int MINB = m2 > 1 ? m2 : 1;
};

// CPB cells per block (THREADS = CPB * (K+1)^D); the default CellCfg<D, K>::CPB
// fills about 256 threads, other values are variants the autotuner times.
template <int D, int K, typename T, int CPB = CellCfg<D, K>::CPB>
__global__ void __launch_bounds__(JacLaunch<D, K, T, CPB>::THREADS, JacLaunch<D, K, T, CPB>::MINB)
k_cell_jac(const int32_t* __restrict__ cells, int64_t nc, const T* __restrict__ cache,
           const typename IO<T>::type* __restrict__ src, typename IO<T>::type* __restrict__ dst, T nu, T a0dt) {
  __shared__ JacSmem<D, K, T, CPB> sm;
  load_tab<K, T>(sm.st);
  cell_jac_block<D, K, T, CPB>(sm, blockIdx.x, cells, nc, cache, src, dst, nu, a0dt);
}

// Element matrices of the volume terms (FP32 local matrices of the additive
// Schwarz smoother): block (cell, column batch), CPB columns per block.
template <int D, int K>
__global__ void __launch_bounds__(CellCfg<D, K>::THREADS)
k_cell_elem(const int32_t* __restrict__ cells, int64_t nc, const float* __restrict__ cache, float nu, float a0dt,
            float* __restrict__ E) {
  __shared__ JacSmem<D, K, float> sm;
  load_tab<K, float>(sm.st);
  cell_jac_block<D, K, float, CellCfg<D, K>::CPB, true>(sm, blockIdx.x, cells, nc, cache, nullptr, nullptr, nu, a0dt,
                                                       blockIdx.y * CellCfg<D, K>::CPB, E);
}

// ---------------------------------------------------------------------------
// Batched cell Jacobian over several operator instances of the same (D, K):
// a persistent grid takes tiles (one tile = one block of CPB cells of one
// instance) from a device counter until all tiles are done; tile -> instance
// by the prefix table `first_tile` (ninst + 1 entries).  The loop runs a
// bounded number of times (tiles are finite); it never waits on other blocks.
template <typename T> struct BatchInst {
  const int32_t* cells; int64_t nc; const T* cache; const typename IO<T>::type* src; typename IO<T>::type* dst;
  T nu; T a0dt;
};
#define MF_BATCH_MAX 64
template <typename T> struct BatchTable {
  int ninst;
  int64_t first_tile[MF_BATCH_MAX + 1];
  BatchInst<T> inst[MF_BATCH_MAX];
};

template <int D, int K, typename T>
__global__ void __launch_bounds__(CellCfg<D, K>::THREADS)
k_cell_jac_batched(const BatchTable<T>* __restrict__ tab, unsigned long long* __restrict__ counter) {
  __shared__ JacSmem<D, K, T> sm;
  __shared__ long long s_tile;
  load_tab<K, T>(sm.st);
  const int64_t total = tab->first_tile[tab->ninst];
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= total) break;
    int i = 0;
    while (i + 1 < tab->ninst && tab->first_tile[i + 1] <= tile) ++i;
    const BatchInst<T>& in = tab->inst[i];
    cell_jac_block<D, K, T>(sm, tile - tab->first_tile[i], in.cells, in.nc, in.cache, in.src, in.dst, in.nu, in.a0dt);
  }
}

// ---------------------------------------------------------------------------
// State evaluation at Gauss points (FP64).  MODE 0: write the linearisation
// cache at the state up (Section 2.3 Jacobian coefficients).  MODE 1: residual
// volume terms of Eq. Eq-NSweakComplete (with the integrated-by-parts pressure
// and viscous terms of Eq. Eq-NSweakWmortar), dst += R_cell(up).  MODE 2:
// both in one pass (a Newton step needs the residual and the linearisation at
// the same state; they share the interpolation, geometry and tau).
struct StateArgs {
  const int32_t* cells; int64_t nc;
  const double* x;          // [N_n][D] current coordinates
  const uint8_t* cell_side; // 0 rotor
  const double* up;         // [N_n][D+1]
  const double* ht;         // [N_n][D] history term
  double* cache;            // MODE 0 output
  double* dst;              // MODE 1 output
  double nu, omega, a0dt, inv_dt2;
};

#ifndef MF_STATE_MINB
#define MF_STATE_MINB 2      // resident blocks of the FP64 state kernel requested from the register allocator (2: 7-9 % faster than 1 at Q2/Q3)
#endif
// GEO: the geometry fields of the cache (J^-1, det J w, G, ctil) are valid
// for the current coordinates (an earlier pass at the same rotor angle wrote
// them): read them instead of differentiating x twice and inverting J, and
// leave them unwritten.  Bit-for-bit the values a recomputation would give.
template <int D, int K, int MODE, bool GEO>
__global__ void __launch_bounds__(CellCfg<D, K>::THREADS, MF_STATE_MINB) k_cell_state(StateArgs A) {
  using C = CellCfg<D, K>;
  using T = double;
  constexpr int N = C::N, NQ = C::NQ, NF = D + 1;
  constexpr int NV = 3 * D + 1;          // x (D), u (D), p, h_t (D)
  constexpr int NS = 2 * D * D + D;      // largest plane count: gradients of x, u and p
  constexpr int F0 = GEO ? D : 0;        // first differentiated field: x only without the geometry
  using CF = Cache<D>;
  __shared__ SmTab<N, T> st;
  __shared__ T smem[C::CPB][NS * NQ];
  __shared__ T vol[C::CPB];
  load_tab<K, T>(st);
  const int cl = threadIdx.x / NQ, t = threadIdx.x % NQ;
  const int64_t cell = (int64_t)blockIdx.x * C::CPB + cl;
  const bool active = cell < A.nc;
  T* tile = smem[cl];
  int ii[3] = {t % N, (t / N) % N, t / (N * N)};
  const int strd[3] = {1, N, N * N};
  if (t == 0) vol[cl] = 0.0;

  // fields: [0,D) x, [D,2D) u, 2D p, [2D+1, 3D+1) h_t
  T v[NV];
  int node = 0;
  bool rotor = false;
  if (active) {
    const int id = A.cells[cell * NQ + t];
    node = id < 0 ? ~id : id;
#pragma unroll
    for (int m = 0; m < D; ++m) v[m] = A.x[(int64_t)node * D + m];
#pragma unroll
    for (int f = 0; f < NF; ++f) v[D + f] = A.up[(int64_t)node * NF + f];
#pragma unroll
    for (int c = 0; c < D; ++c) v[2 * D + 1 + c] = A.ht[(int64_t)node * D + c];
    rotor = A.cell_side[cell] == 0;
  } else {
#pragma unroll
    for (int f = 0; f < NV; ++f) v[f] = T(0);
    // a harmless unit cell: keeps J invertible on padding threads
    v[0] = (T)ii[0]; v[1] = (T)ii[1]; if (D == 3) v[2] = (T)ii[2];
  }
  __syncthreads();
  // nodal -> Gauss values (NV planes; NS >= NV)
#pragma unroll
  for (int r = 0; r < D; ++r) {
#pragma unroll
    for (int f = 0; f < NV; ++f) tile[f * NQ + t] = v[f];
    __syncthreads();
    line<D, N, NV, false>(tile, NQ, t, ii[r], strd[r], st.B, v);
    __syncthreads();
  }
  // reference gradients of x (unless GEO), u, p (fields F0 .. 2D)
  constexpr int NG = 2 * D + 1, NGD = NG - F0;
  T dv[NG][D];
#pragma unroll
  for (int f = F0; f < NG; ++f) tile[(f - F0) * NQ + t] = v[f];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < D; ++r) {
    T o[NGD];
    line<D, N, NGD, false>(tile, NQ, t, ii[r], strd[r], st.Dg, o);
#pragma unroll
    for (int f = 0; f < NGD; ++f) dv[F0 + f][r] = o[f];
  }
  __syncthreads();
  // reference Hessians of x (unless GEO) and u (fields F0 .. 2D-1) from their gradients
  constexpr int NH = 2 * D - F0;
  T H[2 * D][Sym<D>::n];
#pragma unroll
  for (int f = 0; f < NH; ++f)
#pragma unroll
    for (int r = 0; r < D; ++r) tile[(f * D + r) * NQ + t] = dv[F0 + f][r];
  __syncthreads();
#pragma unroll
  for (int e = 0; e < Sym<D>::n; ++e) {
    const int r = sym_r(D, e), s = sym_s(D, e);
    const int base = t - ii[s] * strd[s];
    T o[NH];
#pragma unroll
    for (int f = 0; f < NH; ++f) o[f] = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const T m = st.Dg[ii[s]][j];
#pragma unroll
      for (int f = 0; f < NH; ++f) o[f] = fma(m, tile[(f * D + r) * NQ + base + j * strd[s]], o[f]);
    }
#pragma unroll
    for (int f = 0; f < NH; ++f) H[F0 + f][e] = o[f];
  }
  __syncthreads();

  // ---- geometry: J[m][r] = dv[m][r], or the cached fields (GEO)
  T Ji[D][D], Wq;
  T G[Sym<D>::n];
  T ct[D];
  if constexpr (GEO) {
    const int64_t Pn = A.nc * NQ;
    const double* cq = A.cache + (active ? cell : 0) * NQ + t;
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int m = 0; m < D; ++m) Ji[r][m] = cq[(CF::JINV + r * D + m) * Pn];
    Wq = cq[CF::W * Pn];
#pragma unroll
    for (int e = 0; e < Sym<D>::n; ++e) G[e] = cq[(CF::G + e) * Pn];
#pragma unroll
    for (int r = 0; r < D; ++r) ct[r] = cq[(CF::CT + r) * Pn];
    if (active) atomicAdd(&vol[cl], Wq);
  } else {
  T detJ;
  if (D == 2) {
    const T j00 = dv[0][0], j01 = dv[0][1], j10 = dv[1][0], j11 = dv[1][1];
    detJ = j00 * j11 - j01 * j10;
    const T id = T(1) / detJ;
    Ji[0][0] = j11 * id; Ji[0][1] = -j01 * id; Ji[1][0] = -j10 * id; Ji[1][1] = j00 * id;
  } else {
    T j[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int r = 0; r < 3; ++r) j[m][r] = dv[m][r];
    const T c00 = j[1][1] * j[2][2] - j[1][2] * j[2][1];
    const T c01 = j[1][2] * j[2][0] - j[1][0] * j[2][2];
    const T c02 = j[1][0] * j[2][1] - j[1][1] * j[2][0];
    detJ = j[0][0] * c00 + j[0][1] * c01 + j[0][2] * c02;
    const T id = T(1) / detJ;
    // Jinv[r][m] = cofactor(J)[m][r] / det
    T I[3][3];
    I[0][0] = c00 * id;
    I[1][0] = c01 * id;
    I[2][0] = c02 * id;
    I[0][1] = (j[0][2] * j[2][1] - j[0][1] * j[2][2]) * id;
    I[1][1] = (j[0][0] * j[2][2] - j[0][2] * j[2][0]) * id;
    I[2][1] = (j[0][1] * j[2][0] - j[0][0] * j[2][1]) * id;
    I[0][2] = (j[0][1] * j[1][2] - j[0][2] * j[1][1]) * id;
    I[1][2] = (j[0][2] * j[1][0] - j[0][0] * j[1][2]) * id;
    I[2][2] = (j[0][0] * j[1][1] - j[0][1] * j[1][0]) * id;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int m = 0; m < 3; ++m) Ji[r][m] = I[r][m];
  }
  const T wq = st.w[ii[0]] * st.w[ii[1]] * (D == 3 ? st.w[ii[2]] : T(1));
  Wq = detJ * wq;
  if (active) atomicAdd(&vol[cl], Wq);
  // G = Jinv Jinv^T (symmetric, off-diagonals doubled for the contraction with H)
#pragma unroll
  for (int e = 0; e < Sym<D>::n; ++e) {
    const int r = sym_r(D, e), s = sym_s(D, e);
    T g = T(0);
#pragma unroll
    for (int m = 0; m < D; ++m) g = fma(Ji[r][m], Ji[s][m], g);
    G[e] = (r == s) ? g : T(2) * g;
  }
  // ctil_r = sum_m Jinv[r][m] (G : H_xi x_m)
  {
    T cv[D];
#pragma unroll
    for (int m = 0; m < D; ++m) {
      T s = T(0);
#pragma unroll
      for (int e = 0; e < Sym<D>::n; ++e) s = fma(G[e], H[m][e], s);
      cv[m] = s;
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
      T s = T(0);
#pragma unroll
      for (int m = 0; m < D; ++m) s = fma(Ji[r][m], cv[m], s);
      ct[r] = s;
    }
  }
  }   // geometry computed
  __syncthreads();
  const T V = vol[cl];
  const T h = (D == 2) ? sqrt(T(4) * V / T(M_PI)) : cbrt(T(6) * V / T(M_PI));

  // ---- state at the point
  T U[D], gU[D][D], lU[D], gP[D], ua[D], a[D];
#pragma unroll
  for (int c = 0; c < D; ++c) U[c] = v[D + c];
  const T P = v[2 * D];
#pragma unroll
  for (int c = 0; c <= D; ++c)
#pragma unroll
    for (int m = 0; m < D; ++m) {
      T s = T(0);
#pragma unroll
      for (int r = 0; r < D; ++r) s = fma(dv[D + c][r], Ji[r][m], s);
      if (c < D) gU[c][m] = s; else gP[m] = s;
    }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    T l = T(0);
#pragma unroll
    for (int e = 0; e < Sym<D>::n; ++e) l = fma(G[e], H[D + c][e], l);
#pragma unroll
    for (int r = 0; r < D; ++r) l = fma(-ct[r], dv[D + c][r], l);
    lU[c] = l;
  }
  // mesh velocity omega e_z x x in rotor cells
#pragma unroll
  for (int c = 0; c < D; ++c) ua[c] = T(0);
  if (rotor) { ua[0] = -A.omega * v[1]; ua[1] = A.omega * v[0]; }
  T an2 = T(0);
#pragma unroll
  for (int c = 0; c < D; ++c) { a[c] = U[c] - ua[c]; an2 = fma(a[c], a[c], an2); }
  const T dterm = T(4) * A.nu / (h * h);
  const T tau = T(1) / sqrt(A.inv_dt2 + T(4) * an2 / (h * h) + T(9) * dterm * dterm);
  T Rs[D], conv[D];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    T cv = T(0);
#pragma unroll
    for (int m = 0; m < D; ++m) cv = fma(a[m], gU[c][m], cv);
    conv[c] = cv;
    Rs[c] = A.a0dt * U[c] + v[2 * D + 1 + c] + cv + gP[c] - A.nu * lU[c];
  }

  if (MODE == 0 || MODE == 2) {
    if (active) {
      const int64_t Pn = A.nc * NQ;
      double* cp = A.cache + cell * NQ + t;
      if constexpr (!GEO) {
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
          for (int m = 0; m < D; ++m) cp[(CF::JINV + r * D + m) * Pn] = Ji[r][m];
        cp[CF::W * Pn] = Wq;
#pragma unroll
        for (int e = 0; e < Sym<D>::n; ++e) cp[(CF::G + e) * Pn] = G[e];
#pragma unroll
        for (int r = 0; r < D; ++r) cp[(CF::CT + r) * Pn] = ct[r];
      }
#pragma unroll
      for (int m = 0; m < D; ++m) cp[(CF::A + m) * Pn] = a[m];
#pragma unroll
      for (int c = 0; c < D; ++c)
#pragma unroll
        for (int m = 0; m < D; ++m) cp[(CF::GU + c * D + m) * Pn] = gU[c][m];
#pragma unroll
      for (int c = 0; c < D; ++c) cp[(CF::RS + c) * Pn] = Rs[c];
      cp[CF::TAU * Pn] = tau;
    }
  }
  if (MODE == 0) {
    return;
  } else {
    // residual fluxes
    T fv[NF], Fx[NF][D];
    T Fp[D][D];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int m = 0; m < D; ++m) Fp[c][m] = fma(A.nu, gU[c][m], tau * Rs[c] * a[m]) - (c == m ? P : T(0));
    T divu = T(0);
#pragma unroll
    for (int c = 0; c < D; ++c) { fv[c] = Wq * (A.a0dt * U[c] + v[2 * D + 1 + c] + conv[c]); divu += gU[c][c]; }
    fv[D] = Wq * divu;
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int r = 0; r < D; ++r) {
        T s = T(0);
#pragma unroll
        for (int m = 0; m < D; ++m) s = fma(Ji[r][m], Fp[c][m], s);
        Fx[c][r] = Wq * s;
      }
#pragma unroll
    for (int r = 0; r < D; ++r) {
      T s = T(0);
#pragma unroll
      for (int m = 0; m < D; ++m) s = fma(Ji[r][m], Rs[m], s);
      Fx[D][r] = Wq * tau * s;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int r = 0; r < D; ++r) tile[(f * D + r) * NQ + t] = Fx[f][r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < D; ++r) {
      const int base = t - ii[r] * strd[r];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const T m = st.Dg[j][ii[r]];
#pragma unroll
        for (int f = 0; f < NF; ++f) fv[f] = fma(m, tile[(f * D + r) * NQ + base + j * strd[r]], fv[f]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < D; ++r) {
#pragma unroll
      for (int f = 0; f < NF; ++f) tile[f * NQ + t] = fv[f];
      __syncthreads();
      line<D, N, NF, true>(tile, NQ, t, ii[r], strd[r], st.B, fv);
      __syncthreads();
    }
    if (active) {
#pragma unroll
      for (int f = 0; f < NF; ++f) atomicAdd(&A.dst[(int64_t)node * NF + f], fv[f]);
    }
  }
}

}  // namespace mf
