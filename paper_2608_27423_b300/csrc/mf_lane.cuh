// FP32 cell Jacobian of the 3D operator with one cell per lane.
//
// The FP32 apply (the multigrid smoother's operator and the mixed solve's
// inner workhorse) has FMA headroom that the one-thread-per-point kernel of
// mf_cell.cuh cannot use: its line sweeps re-read every tile value N times
// from shared memory, so the shared-memory pipe saturates first.  Here a block
// holds 32 cells, lane l of every warp works on cell l, and warp w takes one
// position t = w of the N x N cross-section of the cell:
//   pencil   (i, j) = (t % N, t / N): the z-line of points (i, j, 0..N-1),
//   x-line   (j, k) = (t % N, t / N): the points (0..N-1, j, k),
//   y-line   (i, k) = (t % N, t / N): the points (i, 0..N-1, k).
// Contractions along a thread's own line run in registers (N loads give N
// outputs, not one), and shared memory is laid out [plane][point][lane] so
// every access of a warp touches 32 consecutive words (no bank conflicts
// whatever the point pattern).  The
// per-point coefficients come from an FP32 copy of the linearisation cache in
// the same lane-interleaved layout, [block][field][point][lane], so each warp
// load is one 128-byte line; G = J^-1 J^-T is recomputed instead of read
// (29 of the 35 cached fields).  Same arithmetic as k_cell_jac (Section 2.3
// blocks, tau frozen), different summation order.
#pragma once
#include "mf_cell.cuh"

#ifndef MF_LANE_MINB_Q2
#define MF_LANE_MINB_Q2 2     // Q2: two 288-thread blocks per SM (96 registers, no spills)
#endif

namespace mf {

template <int K> struct LaneCfg {
  static constexpr int N = K + 1, N2 = N * N, NQ = N2 * N;
  static constexpr int CB = 32;                 // cells per block: one per lane
  static constexpr int THREADS = N2 * CB;       // one warp per cross-section position
  static constexpr int PLANES = 21;             // shared planes of NQ x CB floats
  static constexpr int MINB = THREADS <= 128 ? 4 : THREADS <= 288 ? MF_LANE_MINB_Q2 : 1;   // resident blocks asked of ptxas
  static constexpr size_t SMEM = sizeof(float) * (size_t)PLANES * NQ * CB + sizeof(float) * 3 * N * N;
};

// Fields of the lane-layout FP32 cache (a subset of Cache<3>; G recomputed).
struct LaneCache {
  static constexpr int JINV = 0, W = 9, CT = 10, A = 13, GU = 16, RS = 25, TAU = 28, NF = 29;
  // field of Cache<3> that lane field f copies
  __host__ __device__ static constexpr int src(int f) { return f < 10 ? f : f + Sym<3>::n; }
};

// FP32 lane cache from the FP64 point-fastest cache: out index
// ((blk * NF + f) * NQ + p) * 32 + lane for cell blk * 32 + lane (zero past nc).
template <int K>
__global__ void k_lane_cache(const double* __restrict__ c64, int64_t nc, float* __restrict__ lc) {
  constexpr int NQ = LaneCfg<K>::NQ, NF = LaneCache::NF;
  const int64_t nb = (nc + 31) / 32, total = nb * NF * NQ * 32, P = nc * NQ;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    const int lane = (int)(o & 31);
    const int64_t r = o >> 5;
    const int p = (int)(r % NQ);
    const int f = (int)((r / NQ) % NF);
    const int64_t cell = (r / NQ / NF) * 32 + lane;
    lc[o] = cell < nc ? (float)c64[(int64_t)LaneCache::src(f) * P + cell * NQ + p] : 0.f;
  }
}

// Lane-interleaved cell table: out[(blk * NQ + p) * 32 + lane] = cells[cell * NQ + p]
// (wall nodes keep their ~id encoding; 0 past nc, never read).
template <int K>
__global__ void k_lane_cells(const int32_t* __restrict__ cells, int64_t nc, int32_t* __restrict__ lcells) {
  constexpr int NQ = LaneCfg<K>::NQ;
  const int64_t total = (nc + 31) / 32 * NQ * 32;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    const int lane = (int)(o & 31);
    const int64_t r = o >> 5;
    const int p = (int)(r % NQ);
    const int64_t cell = (r / NQ) * 32 + lane;
    lcells[o] = cell < nc ? cells[cell * NQ + p] : 0;
  }
}

template <int K>
__global__ void __launch_bounds__(LaneCfg<K>::THREADS, LaneCfg<K>::MINB)
k_cell_jac_lane(const int32_t* __restrict__ lcells, int64_t nc, const float* __restrict__ lc,
                const float4* __restrict__ src, float* __restrict__ dst, float nu, float a0dt) {
  using L = LaneCfg<K>;
  constexpr int N = L::N, N2 = L::N2, NQ = L::NQ, CB = L::CB;
  using LC = LaneCache;
  extern __shared__ float smem[];
  float* S = smem;                                          // [PLANES][NQ][CB]
  float (*sB)[N] = reinterpret_cast<float (*)[N]>(smem + L::PLANES * NQ * CB);
  float (*sDg)[N] = sB + N;
  float (*sD2)[N] = sB + 2 * N;
  {
    const MfTab<float>& tb = c_tab32[K];
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
      const int q = e / N, a = e % N;
      sB[q][a] = tb.B[q][a];
      sDg[q][a] = tb.Dg[q][a];
      float s = 0.f;
      for (int j = 0; j < N; ++j) s = fmaf(tb.Dg[q][j], tb.Dg[j][a], s);
      sD2[q][a] = s;                                        // second collocation derivative Dg Dg
    }
  }
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5;
  const int64_t cell = (int64_t)blockIdx.x * CB + lane;
  const bool active = cell < nc;
  const int u0 = t % N, u1 = t / N;                         // (i, j) pencil / (j, k) x-line / (i, k) y-line
  auto sp = [&](int pl, int p) -> float& { return S[(pl * NQ + p) * CB + lane]; };
  const float* lcb = lc + (int64_t)blockIdx.x * LC::NF * NQ * CB + lane;
  const int32_t* lcl = lcells + (int64_t)blockIdx.x * NQ * CB + lane;

  // ---- gather the pencil's nodal values (wall velocities as zero)
  int node[N];
  float nv[N][4];
#pragma unroll
  for (int c = 0; c < N; ++c) {
    const int p = u0 + N * u1 + N2 * c;
    float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
    node[c] = -1;
    if (active) {
      const int id = lcl[p * CB];
      const bool wall = id < 0;
      node[c] = wall ? ~id : id;
      s4 = src[node[c]];
      if (wall) { s4.x = 0.f; s4.y = 0.f; s4.z = 0.f; }
    }
    nv[c][0] = s4.x; nv[c][1] = s4.y; nv[c][2] = s4.z; nv[c][3] = s4.w;
  }
  __syncthreads();                                          // tables visible
  // ---- nodal -> Gauss values: z in registers, then x and y through shared memory
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < N; ++c) {
      const float b = sB[k][c];
#pragma unroll
      for (int f = 0; f < 4; ++f) o[f] = fmaf(b, nv[c][f], o[f]);
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) sp(f, u0 + N * u1 + N2 * k) = o[f];
  }
  __syncthreads();
  {  // x-line (j, k) = (u0, u1)
    float xv[N][4];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int f = 0; f < 4; ++f) xv[a][f] = sp(f, a + N * u0 + N2 * u1);
#pragma unroll
    for (int q = 0; q < N; ++q) {
      float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const float b = sB[q][a];
#pragma unroll
        for (int f = 0; f < 4; ++f) o[f] = fmaf(b, xv[a][f], o[f]);
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) sp(f, q + N * u0 + N2 * u1) = o[f];
    }
  }
  __syncthreads();
  {  // y-line (i, k) = (u0, u1): Gauss values V, d/dy (all fields), d2/dy2 (velocity)
    float yv[N][4], V[N][4];
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int f = 0; f < 4; ++f) yv[b][f] = sp(f, u0 + N * b + N2 * u1);
#pragma unroll
    for (int q = 0; q < N; ++q) {
#pragma unroll
      for (int f = 0; f < 4; ++f) V[q][f] = 0.f;
#pragma unroll
      for (int b = 0; b < N; ++b) {
        const float m = sB[q][b];
#pragma unroll
        for (int f = 0; f < 4; ++f) V[q][f] = fmaf(m, yv[b][f], V[q][f]);
      }
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
      float gy[4] = {0.f, 0.f, 0.f, 0.f}, hy[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int b = 0; b < N; ++b) {
        const float m = sDg[q][b], m2 = sD2[q][b];
#pragma unroll
        for (int f = 0; f < 4; ++f) gy[f] = fmaf(m, V[b][f], gy[f]);
#pragma unroll
        for (int c = 0; c < 3; ++c) hy[c] = fmaf(m2, V[b][c], hy[c]);
      }
      const int p = u0 + N * q + N2 * u1;
#pragma unroll
      for (int f = 0; f < 4; ++f) { sp(f, p) = V[q][f]; sp(4 + f, p) = gy[f]; }
#pragma unroll
      for (int c = 0; c < 3; ++c) sp(8 + c, p) = hy[c];
    }
  }
  __syncthreads();
  {  // x-line (j, k): d/dx (all fields), d2/dx2 and d2/dxdy (velocity) -> planes 11..20
    float xv[N][4], xy[N][3];
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const int p = a + N * u0 + N2 * u1;
#pragma unroll
      for (int f = 0; f < 4; ++f) xv[a][f] = sp(f, p);
#pragma unroll
      for (int c = 0; c < 3; ++c) xy[a][c] = sp(4 + c, p);
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
      float gx[4] = {0.f, 0.f, 0.f, 0.f}, hxx[3] = {0.f, 0.f, 0.f}, hxy[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const float m = sDg[q][a], m2 = sD2[q][a];
#pragma unroll
        for (int f = 0; f < 4; ++f) gx[f] = fmaf(m, xv[a][f], gx[f]);
#pragma unroll
        for (int c = 0; c < 3; ++c) { hxx[c] = fmaf(m2, xv[a][c], hxx[c]); hxy[c] = fmaf(m, xy[a][c], hxy[c]); }
      }
      const int p = q + N * u0 + N2 * u1;
#pragma unroll
      for (int f = 0; f < 4; ++f) sp(11 + f, p) = gx[f];
#pragma unroll
      for (int c = 0; c < 3; ++c) { sp(15 + c, p) = hxx[c]; sp(18 + c, p) = hxy[c]; }
    }
  }
  __syncthreads();
  // ---- pencil (i, j): point physics, z-transpose.  The pencil's values and
  // x/y-derivatives stay in shared memory and are read per point (the thread
  // owns every entry of its pencil, so nothing else touches them in this
  // phase); the outputs of point k go to its own Hessian slots, which no
  // later point reads: Fx[.][0] -> planes 15..18, Fx[.][1] -> planes 19, 20,
  // 8, 9; the z-transposed sums g -> planes 0..3 after the last point.
  {
    float gz[N][4];
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
      for (int f = 0; f < 4; ++f) gz[c][f] = 0.f;
    const int p0 = u0 + N * u1;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int p = p0 + N2 * k;
      float v[4], dv[4][3], H[3][6];
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        float gzf = 0.f;
#pragma unroll
        for (int c = 0; c < N; ++c) gzf = fmaf(sDg[k][c], sp(f, p0 + N2 * c), gzf);
        v[f] = sp(f, p);
        dv[f][0] = sp(11 + f, p);
        dv[f][1] = sp(4 + f, p);
        dv[f][2] = gzf;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float hzz = 0.f, hxz = 0.f, hyz = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const int pj = p0 + N2 * j;
          hzz = fmaf(sD2[k][j], sp(c, pj), hzz);
          hxz = fmaf(sDg[k][j], sp(11 + c, pj), hxz);
          hyz = fmaf(sDg[k][j], sp(4 + c, pj), hyz);
        }
        H[c][0] = sp(15 + c, p);
        H[c][1] = sp(8 + c, p);
        H[c][2] = hzz;
        H[c][3] = sp(18 + c, p);
        H[c][4] = hxz;
        H[c][5] = hyz;
      }
      // coefficients of this point (coalesced: one 128-byte line per field)
      float Ji[3][3], a[3], gU[3][3], Rs[3], G[6], ct[3];
      const float* cq = lcb + p * CB;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int m = 0; m < 3; ++m) Ji[r][m] = cq[(LC::JINV + r * 3 + m) * NQ * CB];
      const float Wq = cq[LC::W * NQ * CB];
#pragma unroll
      for (int r = 0; r < 3; ++r) ct[r] = cq[(LC::CT + r) * NQ * CB];
#pragma unroll
      for (int m = 0; m < 3; ++m) a[m] = cq[(LC::A + m) * NQ * CB];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < 3; ++m) gU[c][m] = cq[(LC::GU + c * 3 + m) * NQ * CB];
#pragma unroll
      for (int c = 0; c < 3; ++c) Rs[c] = cq[(LC::RS + c) * NQ * CB];
      const float tau = cq[LC::TAU * NQ * CB];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const int r = sym_r(3, e), s2 = sym_s(3, e);
        float g = 0.f;
#pragma unroll
        for (int m = 0; m < 3; ++m) g = fmaf(Ji[r][m], Ji[s2][m], g);
        G[e] = (r == s2) ? g : 2.f * g;
      }
      float fv[4], Fx[4][3];
      jac_point<3, float>(v, dv, H, Ji, Wq, G, ct, a, gU, Rs, tau, nu, a0dt, fv, Fx);
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        gz[k][f] += fv[f];
#pragma unroll
        for (int c = 0; c < N; ++c) gz[c][f] = fmaf(sDg[k][c], Fx[f][2], gz[c][f]);
        sp(15 + f, p) = Fx[f][0];
      }
      sp(19, p) = Fx[0][1];
      sp(20, p) = Fx[1][1];
      sp(8, p) = Fx[2][1];
      sp(9, p) = Fx[3][1];
    }
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
      for (int f = 0; f < 4; ++f) sp(f, p0 + N2 * c) = gz[c][f];
  }
  __syncthreads();
  {  // x-line: g += Dg_x^T Fx[.][0]   (Fx0 in planes 15..18, g in planes 0..3)
    float fx[N][4], g[N][4];
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const int p = a + N * u0 + N2 * u1;
#pragma unroll
      for (int f = 0; f < 4; ++f) { fx[a][f] = sp(15 + f, p); g[a][f] = sp(f, p); }
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const int p = a + N * u0 + N2 * u1;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        float s = g[a][f];
#pragma unroll
        for (int q = 0; q < N; ++q) s = fmaf(sDg[q][a], fx[q][f], s);
        sp(f, p) = s;
      }
    }
  }
  __syncthreads();
  {  // y-line: g += Dg_y^T Fx[.][1] (planes 19, 20, 8, 9), then B^T along y -> planes 0..3
    constexpr int FY[4] = {19, 20, 8, 9};
    float fy[N][4], g[N][4];
#pragma unroll
    for (int b = 0; b < N; ++b) {
      const int p = u0 + N * b + N2 * u1;
#pragma unroll
      for (int f = 0; f < 4; ++f) { fy[b][f] = sp(FY[f], p); g[b][f] = sp(f, p); }
    }
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        float s = g[b][f];
#pragma unroll
        for (int q = 0; q < N; ++q) s = fmaf(sDg[q][b], fy[q][f], s);
        g[b][f] = s;
      }
#pragma unroll
    for (int c = 0; c < N; ++c) {
      float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int b = 0; b < N; ++b) {
        const float m = sB[b][c];
#pragma unroll
        for (int f = 0; f < 4; ++f) o[f] = fmaf(m, g[b][f], o[f]);
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) sp(f, u0 + N * c + N2 * u1) = o[f];
    }
  }
  __syncthreads();
  {  // x-line: B^T along x (planes 0..3)
    float h[N][4];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int f = 0; f < 4; ++f) h[a][f] = sp(f, a + N * u0 + N2 * u1);
#pragma unroll
    for (int c = 0; c < N; ++c) {
      float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const float m = sB[a][c];
#pragma unroll
        for (int f = 0; f < 4; ++f) o[f] = fmaf(m, h[a][f], o[f]);
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) sp(f, c + N * u0 + N2 * u1) = o[f];
    }
  }
  __syncthreads();
  // ---- pencil: B^T along z, scatter-add to the nodes
  {
    float h[N][4];
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
      for (int f = 0; f < 4; ++f) h[k][f] = sp(f, u0 + N * u1 + N2 * k);
    if (active) {
#pragma unroll
      for (int c = 0; c < N; ++c) {
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const float m = sB[k][c];
#pragma unroll
          for (int f = 0; f < 4; ++f) o[f] = fmaf(m, h[k][f], o[f]);
        }
        atomicAdd(reinterpret_cast<float4*>(dst) + node[c], make_float4(o[0], o[1], o[2], o[3]));
      }
    }
  }
}

}  // namespace mf
