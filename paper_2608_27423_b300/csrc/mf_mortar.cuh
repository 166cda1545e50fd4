// Mortar interface kernels: rotor rotation (Section 3.1), mortar-cell mapping
// (Section 3.2), Hillewaert penalty (Eq. EqPenalty) and the Nitsche/SIPG face
// terms of Eq. Eq-NSweakWmortar (pressure central flux, SIPG consistency,
// symmetry and penalty terms, strong-DG mass term).
#pragma once
#include "mf_cell.cuh"

namespace mf {

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// 1D Lagrange values/derivatives on the Gauss-Lobatto nodes at an arbitrary t.
template <int N, typename T>
__device__ __forceinline__ void lagrange_at(const MfTab<T>& tb, T t, T* L, T* dL) {
#pragma unroll
  for (int b = 0; b < N; ++b) {
    T v = T(1), d = T(0);
#pragma unroll
    for (int c = 0; c < N; ++c) {
      if (c == b) continue;
      d = d * (t - tb.gll[c]) + v;     // product rule, accumulated left to right
      v = v * (t - tb.gll[c]);
    }
    L[b] = v * tb.bw[b];
    dL[b] = d * tb.bw[b];
  }
}

// ---------------------------------------------------------------------------
// x = R(theta) x0 for rotor nodes (2D rotation matrix; 3D
// R = cos I + sin W + (1 - cos) r (x) r with axis r = e_z), x = x0 otherwise.
template <int D>
__global__ void k_rotate(const double* __restrict__ x0, const uint8_t* __restrict__ side, double* __restrict__ x,
                         int64_t nn, double ct, double st, const double* __restrict__ theta_dev) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  if (theta_dev) { ct = cos(*theta_dev); st = sin(*theta_dev); }   // angle kept on the device (graph replays)
  double p[3] = {x0[i * D], x0[i * D + 1], D == 3 ? x0[i * D + 2] : 0.0};
  if (side[i] == 0) {
    const double r[3] = {0.0, 0.0, 1.0};
    double Rm[3][3];
    const double W[3][3] = {{0.0, -r[2], r[1]}, {r[2], 0.0, -r[0]}, {-r[1], r[0], 0.0}};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Rm[a][b] = (a == b ? ct : 0.0) + st * W[a][b] + (1.0 - ct) * r[a] * r[b];
    double q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) q[a] = Rm[a][0] * p[0] + Rm[a][1] * p[1] + Rm[a][2] * p[2];
    p[0] = q[0]; p[1] = q[1]; p[2] = q[2];
  }
#pragma unroll
  for (int m = 0; m < D; ++m) x[i * D + m] = p[m];
}

// ---------------------------------------------------------------------------
// Mortar cells at rotor angle theta.  With D = 2 pi / n_R, theta = s D + th
// (0 <= th < D), stator cell js of layer lz is cut by one rotor vertex into
//   half 0: angles [js D, js D + th], covered by rotor cell js - s - 1,
//   half 1: angles [js D + th, (js+1) D], covered by rotor cell js - s,
// (angles relative to phi0; a half of zero length gets zero weights).
// Gauss rule mapped into each half: weight w_g R L, point on the exact circle,
// each side's face coordinate linear in the angle.
struct MortarMap {
  int32_t* mc_cell;   // [M][2] rotor, stator cell
  double* mc_tau;     // [M] face penalty max(tau_rotor, tau_stator)
  double* mc_xi;      // [M][2][N] face coordinate on each side
  double* mc_cs;      // [M][N][2] cos and sin of the point's absolute angle (outward stator normal)
  double* mc_w;       // [M][N] angular weight w_g R L
  const int32_t* ifr; // [n_z][n_R]
  const int32_t* ifs;
  const double* tau_r; // [n_z][n_R] tau_k of rotor interface cells
  const double* tau_s;
  int n_R, n_z;
  double R, phi0, theta;
  const double* theta_dev;   // if set, the angle is read from device memory
};

template <int K>
__global__ void k_mortar_map(MortarMap A) {
  constexpr int N = K + 1;
  const int64_t M = (int64_t)A.n_z * A.n_R * 2;
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int h = (int)(m & 1);
  const int js = (int)((m >> 1) % A.n_R);
  const int lz = (int)((m >> 1) / A.n_R);
  const double Dl = 2.0 * M_PI / A.n_R;
  const double theta = A.theta_dev ? *A.theta_dev : A.theta;
  const double sf = floor(theta / Dl);
  double th = theta - sf * Dl;
  if (th < 0.0) th = 0.0;
  if (th > Dl) th = Dl;
  long long si = (long long)sf % A.n_R;
  if (si < 0) si += A.n_R;
  int jr = (int)(((long long)js - si - (h == 0 ? 1 : 0)) % A.n_R);
  if (jr < 0) jr += A.n_R;
  const double L = (h == 0) ? th : Dl - th;
  const double start = js * Dl + (h == 0 ? 0.0 : th);
  const MfTab<double>& tb = c_tab64[K];
  A.mc_cell[2 * m] = A.ifr[(int64_t)lz * A.n_R + jr];
  A.mc_cell[2 * m + 1] = A.ifs[(int64_t)lz * A.n_R + js];
  A.mc_tau[m] = fmax(A.tau_r[(int64_t)lz * A.n_R + jr], A.tau_s[(int64_t)lz * A.n_R + js]);
#pragma unroll
  for (int g = 0; g < N; ++g) {
    const double sg = tb.s[g];
    // stator: (phi - js D)/D ; rotor: (phi - start of rotor cell)/D
    const double xs = (h == 0) ? sg * th / Dl : (th + sg * (Dl - th)) / Dl;
    const double xr = (h == 0) ? 1.0 - (1.0 - sg) * th / Dl : sg * (Dl - th) / Dl;
    A.mc_xi[(m * 2 + 0) * N + g] = xr;
    A.mc_xi[(m * 2 + 1) * N + g] = xs;
    const double ang = A.phi0 + start + sg * L;
    A.mc_cs[(m * N + g) * 2 + 0] = cos(ang);
    A.mc_cs[(m * N + g) * 2 + 1] = sin(ang);
    A.mc_w[m * N + g] = tb.w[g] * A.R * L;
  }
}

// ---------------------------------------------------------------------------
// General interfaces (n_R rotor and n_Rs stator cells per layer, Section 3.2's
// mortar cells with the paper's equal-partition restriction lifted): the
// circle is cut at every rotor vertex theta + 2 pi i / n_R and every stator
// vertex 2 pi j / n_Rs (angles from phi0), giving n_R + n_Rs segments per
// layer, of zero length where a rotor and a stator vertex coincide (their
// points get zero weights).  One thread merges the two sorted vertex
// sequences (stator first on ties) into the segment table: start angle,
// length, rotor cell, stator cell and the rotor cell's start angle.  The
// angle comes from theta_dev when set (graph replays).
struct SegTable {
  double* start; double* len; double* rstart; int32_t* jr; int32_t* js;
};

__global__ void k_mortar_segments(SegTable S, int n_R, int n_Rs, double theta, const double* __restrict__ theta_dev) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const double two_pi = 2.0 * M_PI, Dr = two_pi / n_R, Ds = two_pi / n_Rs;
  const double th = theta_dev ? *theta_dev : theta;
  const double sf = floor(th / Dr);
  double tp = th - sf * Dr;                         // first rotor vertex in [0, Dr)
  if (tp < 0.0) tp = 0.0;
  if (tp >= Dr) tp = 0.0;
  long long si = (long long)sf % n_R;
  if (si < 0) si += n_R;
  auto rcell = [&](int rank) { int c = (int)(((long long)rank - si) % n_R); return c < 0 ? c + n_R : c; };
  // the rotor cell covering angle 0 starts at the last rotor vertex, wrapped below 0
  int cur_r = rcell(n_R - 1), cur_s = n_Rs - 1;
  double cur_rstart = tp + (n_R - 1) * Dr - two_pi;
  int i = 0, j = 0;
  const int nseg = n_R + n_Rs;
  for (int t = 0; t < nseg; ++t) {
    const double ar = tp + i * Dr, as = j * Ds;
    double a;
    if (j < n_Rs && (i >= n_R || as <= ar)) { a = as; cur_s = j; ++j; }
    else { a = ar; cur_r = rcell(i); cur_rstart = ar; ++i; }
    S.start[t] = a; S.jr[t] = cur_r; S.js[t] = cur_s; S.rstart[t] = cur_rstart;
  }
  for (int t = 0; t < nseg; ++t) {
    const double end = (t + 1 < nseg) ? S.start[t + 1] : two_pi;
    const double L = end - S.start[t];
    S.len[t] = L > 0.0 ? L : 0.0;
  }
}

// Mortar cells of a general interface from the segment table: m = layer *
// (n_R + n_Rs) + segment; Gauss rule mapped into the segment, point on the
// exact circle, face coordinates linear in the angle on each side.
template <int K>
__global__ void k_mortar_map_general(MortarMap A, SegTable S, int n_Rs) {
  constexpr int N = K + 1;
  const int nseg = A.n_R + n_Rs;
  const int64_t M = (int64_t)A.n_z * nseg;
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int t = (int)(m % nseg);
  const int lz = (int)(m / nseg);
  const double Dr = 2.0 * M_PI / A.n_R, Ds = 2.0 * M_PI / n_Rs;
  const int jr = S.jr[t], js = S.js[t];
  const double st = S.start[t], L = S.len[t], rs = S.rstart[t], ss = js * Ds;
  const MfTab<double>& tb = c_tab64[K];
  A.mc_cell[2 * m] = A.ifr[(int64_t)lz * A.n_R + jr];
  A.mc_cell[2 * m + 1] = A.ifs[(int64_t)lz * n_Rs + js];
  A.mc_tau[m] = fmax(A.tau_r[(int64_t)lz * A.n_R + jr], A.tau_s[(int64_t)lz * n_Rs + js]);
#pragma unroll
  for (int g = 0; g < N; ++g) {
    const double phi = st + tb.s[g] * L;
    A.mc_xi[(m * 2 + 0) * N + g] = (phi - rs) / Dr;
    A.mc_xi[(m * 2 + 1) * N + g] = (phi - ss) / Ds;
    const double ang = A.phi0 + phi;
    A.mc_cs[(m * N + g) * 2 + 0] = cos(ang);
    A.mc_cs[(m * N + g) * 2 + 1] = sin(ang);
    A.mc_w[m * N + g] = tb.w[g] * A.R * L;
  }
}

// ---------------------------------------------------------------------------
// Penalty tau_k = F (k+1)^2 (A(other faces)/2 + A(interface face)) / V of each
// interface cell (Eq. EqPenalty; all non-interface faces halved).  Face areas
// and the volume by the (k+1)-point Gauss rule on the isoparametric map.
// Interface face: xi_0 = 1 (rotor, side 0) or xi_0 = 0 (stator, side 1).
template <int D, int K>
__global__ void k_penalty(const int32_t* __restrict__ cells, const double* __restrict__ x,
                          const int32_t* __restrict__ iface, int64_t ncell_if, int side, double F,
                          double* __restrict__ tau_out) {
  constexpr int N = K + 1, NPC = ipow(N, D);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncell_if) return;
  const MfTab<double>& tb = c_tab64[K];
  const int64_t cell = iface[i];
  double X[NPC][D];
  for (int b = 0; b < NPC; ++b) {
    int id = cells[cell * NPC + b];
    id = id < 0 ? ~id : id;
    for (int m = 0; m < D; ++m) X[b][m] = x[(int64_t)id * D + m];
  }
  double area_if = 0.0, area_other = 0.0, vol = 0.0;
  double L0[N], dL0[N], L1[N], dL1[N], L2[N], dL2[N];
  // volume
  const int nq = ipow(N, D);
  for (int q = 0; q < nq; ++q) {
    int qi[3] = {q % N, (q / N) % N, q / (N * N)};
    double J[3][3] = {{0}};
    for (int b = 0; b < NPC; ++b) {
      int bi[3] = {b % N, (b / N) % N, b / (N * N)};
      double dphi[3];
      for (int r = 0; r < D; ++r) {
        double p = 1.0;
        for (int u = 0; u < D; ++u) p *= (u == r) ? tb.Dn[qi[u]][bi[u]] : tb.B[qi[u]][bi[u]];
        dphi[r] = p;
      }
      for (int m = 0; m < D; ++m)
        for (int r = 0; r < D; ++r) J[m][r] += X[b][m] * dphi[r];
    }
    double det = (D == 2) ? J[0][0] * J[1][1] - J[0][1] * J[1][0]
                          : J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double wq = 1.0;
    for (int u = 0; u < D; ++u) wq *= tb.w[qi[u]];
    vol += det * wq;
  }
  // faces xi_r = sd
  for (int r = 0; r < D; ++r)
    for (int sd = 0; sd < 2; ++sd) {
      double fa = 0.0;
      const int nfq = ipow(N, D - 1);
      for (int fq = 0; fq < nfq; ++fq) {
        // tangential directions t0 < t1 (3D) or t0 (2D)
        int tdir[2], k2 = 0;
        for (int u = 0; u < D; ++u) if (u != r) tdir[k2++] = u;
        double xi[3];
        xi[r] = (double)sd;
        xi[tdir[0]] = tb.s[fq % N];
        if (D == 3) xi[tdir[1]] = tb.s[fq / N];
        double wf = tb.w[fq % N] * (D == 3 ? tb.w[fq / N] : 1.0);
        lagrange_at<N, double>(tb, xi[0], L0, dL0);
        lagrange_at<N, double>(tb, xi[1], L1, dL1);
        if (D == 3) lagrange_at<N, double>(tb, xi[2], L2, dL2);
        double J[3][3] = {{0}};
        for (int b = 0; b < NPC; ++b) {
          int b0 = b % N, b1 = (b / N) % N, b2 = b / (N * N);
          double l2 = D == 3 ? L2[b2] : 1.0, d2 = D == 3 ? dL2[b2] : 0.0;
          double dphi[3] = {dL0[b0] * L1[b1] * l2, L0[b0] * dL1[b1] * l2, L0[b0] * L1[b1] * d2};
          for (int m = 0; m < D; ++m)
            for (int u = 0; u < D; ++u) J[m][u] += X[b][m] * dphi[u];
        }
        double da;
        if (D == 2) {
          da = sqrt(J[0][tdir[0]] * J[0][tdir[0]] + J[1][tdir[0]] * J[1][tdir[0]]);
        } else {
          double t0[3] = {J[0][tdir[0]], J[1][tdir[0]], J[2][tdir[0]]};
          double t1[3] = {J[0][tdir[1]], J[1][tdir[1]], J[2][tdir[1]]};
          double c0 = t0[1] * t1[2] - t0[2] * t1[1];
          double c1 = t0[2] * t1[0] - t0[0] * t1[2];
          double c2 = t0[0] * t1[1] - t0[1] * t1[0];
          da = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
        }
        fa += da * wf;
      }
      const int face_if_sd = (side == 0) ? 1 : 0;
      if (r == 0 && sd == face_if_sd) area_if += fa; else area_other += fa;
    }
  tau_out[i] = F * (double)(N * N) * (0.5 * area_other + area_if) / vol;
}

// ---------------------------------------------------------------------------
// Face geometry at the mortar points (set-up, once per rotor angle): J^-1 of
// each side's cell map at its face point, FP64 and an FP32 copy.
// Layout [M][2][NP][D][D], point index p = ia + (k+1) * iz.
template <int D, int K>
__global__ void k_mortar_geom(const int32_t* __restrict__ cells, const double* __restrict__ x,
                              const int32_t* __restrict__ mc_cell, const double* __restrict__ mc_xi, int64_t nm,
                              double* __restrict__ jinv64, float* __restrict__ jinv32) {
  constexpr int N = K + 1, NPC = ipow(N, D), NP = ipow(N, D - 1);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nm * 2 * NP) return;
  const int p = (int)(t % NP);
  const int s = (int)((t / NP) % 2);
  const int64_t mc = t / (2 * NP);
  const MfTab<double>& tb = c_tab64[K];
  const int ia = p % N, iz = (D == 3) ? p / N : 0;
  double L0[N], dL0[N], L1[N], dL1[N];
  lagrange_at<N, double>(tb, s == 0 ? 1.0 : 0.0, L0, dL0);
  lagrange_at<N, double>(tb, mc_xi[(mc * 2 + s) * N + ia], L1, dL1);
  const int64_t cell = mc_cell[2 * mc + s];
  double J[D][D];
#pragma unroll
  for (int m = 0; m < D; ++m)
#pragma unroll
    for (int r = 0; r < D; ++r) J[m][r] = 0.0;
  for (int b = 0; b < NPC; ++b) {
    const int b0 = b % N, b1 = (b / N) % N, b2 = b / (N * N);
    const double l2 = (D == 3) ? tb.B[iz][b2] : 1.0, d2 = (D == 3) ? tb.Dn[iz][b2] : 0.0;
    const double dphi[3] = {dL0[b0] * L1[b1] * l2, L0[b0] * dL1[b1] * l2, L0[b0] * L1[b1] * d2};
    int id = cells[cell * NPC + b];
    id = id < 0 ? ~id : id;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      const double xm = x[(int64_t)id * D + m];
#pragma unroll
      for (int r = 0; r < D; ++r) J[m][r] = fma(dphi[r], xm, J[m][r]);
    }
  }
  double Ji[D][D];
  if (D == 2) {
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det; Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
  } else {
    double c[3][3];
    c[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    c[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    c[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    c[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    c[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    c[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    c[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    c[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    c[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double det = J[0][0] * c[0][0] + J[0][1] * c[0][1] + J[0][2] * c[0][2];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int m = 0; m < 3; ++m) Ji[r][m] = c[m][r] / det;
  }
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int m = 0; m < D; ++m) {
      jinv64[t * D * D + r * D + m] = Ji[r][m];
      jinv32[t * D * D + r * D + m] = (float)Ji[r][m];
    }
}

// ---------------------------------------------------------------------------
// Face terms.  MODE 0: dst += M src (Jacobian / residual, linear in src);
// MODE 1: diag += diagonal of the face operator.  Per mortar cell and side s
// (own = s, other = 1-s; jump = own - other; n_s own outward normal):
//   -(q, 1/2 [[u]].n) + (v, {p} n) - (grad v : nu/2 [[u]] (x) n)
//   - (v, nu {grad u} n) + (v, nu tau [[u]])
// Traces by sum factorisation: the face-normal direction xi_0 is contracted
// first (value = face layer of the nodes since l_b(face) is a Kronecker delta;
// normal derivative with l_b'(face)), then the face directions with the 1D
// tables at the point's angular coordinate and the Gauss z-points.  The test
// side is integrated the same way in reverse.
template <int D, int K> struct MortarCfg {
  static constexpr int N = K + 1, NPC = ipow(N, D), NP = ipow(N, D - 1);
  static constexpr int MPB = (2 * NPC >= 128) ? 1 : (256 / (2 * NPC));
  static constexpr int THREADS = MPB * 2 * NPC;
};

template <typename T> struct MortarArgs {
  const int32_t* cells;
  const int32_t* mc_cell; const double* mc_tau; const double* mc_xi; const double* mc_cs; const double* mc_w;
  const T* jinv;      // [M][2][NP][D][D]
  int64_t nm;
  const typename IO<T>::type* src; typename IO<T>::type* dst;
  T nu; double dz; int zero_wall;
};

template <int D, int K, typename T> struct MortarSmem {
  static constexpr int N = K + 1, NPC = ipow(N, D), NP = ipow(N, D - 1), NF = D + 1,
                       MPB = MortarCfg<D, K>::MPB;
  T val[MPB][2][NPC][NF];     // gathered nodal values
  T fa[MPB][2][NP][NF];       // face-layer values (b1,b2)
  T fn[MPB][2][NP][NF];       // normal derivative per (b1,b2)
  T U[MPB][2][NP][NF];        // traces at the points
  T GU[MPB][2][NP][D][D];     // physical velocity gradients at the points
  T L1[MPB][2][N][N];         // l_b(xi1 of angular point ia)  [ia][b]
  T dL1[MPB][2][N][N];
  T fv[MPB][2][NP][NF];       // value fluxes
  T Fx[MPB][2][NP][D][D];     // reference gradient fluxes of v
  T G[MPB][2][NP][NF];        // integrated against face-layer test functions
  T H[MPB][2][NP][D];         // integrated against normal derivatives
};

// One block's worth of mortar half-cells (block index `blk`).
template <int D, int K, typename T, int MODE>
__device__ __forceinline__ void mortar_block(MortarSmem<D, K, T>& S, int64_t blk, const MortarArgs<T>& A) {
  using C = MortarCfg<D, K>;
  constexpr int N = C::N, NPC = C::NPC, NP = C::NP, NF = D + 1;
  auto& s_val = S.val; auto& s_fa = S.fa; auto& s_fn = S.fn; auto& s_U = S.U; auto& s_GU = S.GU;
  auto& s_L1 = S.L1; auto& s_dL1 = S.dL1; auto& s_fv = S.fv; auto& s_Fx = S.Fx; auto& s_G = S.G; auto& s_H = S.H;
  const MfTab<T>& tb = TabSel<T>::get(K);
  const int lm = threadIdx.x / (2 * NPC);
  const int loc = threadIdx.x % (2 * NPC);
  const int s = loc / NPC, a = loc % NPC;
  const int64_t mc = blk * C::MPB + lm;
  const bool active = mc < A.nm;
  const int fc = (s == 0) ? K : 0;         // index of the face layer along xi_0
  T L0[N], dL0[N];
  lagrange_at<N, T>(tb, (s == 0) ? T(1) : T(0), L0, dL0);
  // ---- phase 1: gather, and 1D tables along the face
  int node = 0;
  if (active) {
    const int cell = A.mc_cell[2 * mc + s];
    const int id = A.cells[(int64_t)cell * NPC + a];
    const bool wall = id < 0;
    node = wall ? ~id : id;
    if (MODE == 0) {
#pragma unroll
      for (int f = 0; f < NF; ++f) s_val[lm][s][a][f] = from_io<T>(A.src[(int64_t)node * NF + f]);
      if (wall && A.zero_wall) {
#pragma unroll
        for (int c = 0; c < D; ++c) s_val[lm][s][a][c] = T(0);
      }
    }
    if (a < N) {
      T L1[N], dL1[N];
      lagrange_at<N, T>(tb, (T)A.mc_xi[(mc * 2 + s) * N + a], L1, dL1);
#pragma unroll
      for (int b = 0; b < N; ++b) { s_L1[lm][s][a][b] = L1[b]; s_dL1[lm][s][a][b] = dL1[b]; }
    }
  } else {
    if (MODE == 0) {
#pragma unroll
      for (int f = 0; f < NF; ++f) s_val[lm][s][a][f] = T(0);
    }
    if (a < N) {
#pragma unroll
      for (int b = 0; b < N; ++b) { s_L1[lm][s][a][b] = T(0); s_dL1[lm][s][a][b] = T(0); }
    }
  }
  __syncthreads();
  const T tau_f = active ? (T)A.mc_tau[mc] : T(0);
  {
    // ---- diagonal: w nu [tau phi^2 - phi (grad phi . n_s)] on face nodes, per velocity component
    if (!active) return;
    const int a0 = a % N, a1 = (a / N) % N, a2 = a / (N * N);
    if (a0 != fc) return;
    T dv = T(0);
    const T sg = (s == 0) ? T(1) : T(-1);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int ia = p % N, iz = (D == 3) ? p / N : 0;
      double wd = A.mc_w[mc * N + ia];
      if (D == 3) wd *= TabSel<double>::get(K).w[iz] * A.dz;
      const T w = (T)wd;
      const T n[3] = {sg * (T)A.mc_cs[(mc * N + ia) * 2], sg * (T)A.mc_cs[(mc * N + ia) * 2 + 1], T(0)};
      const T l1 = s_L1[lm][s][ia][a1], d1 = s_dL1[lm][s][ia][a1];
      const T l2 = (D == 3) ? tb.B[iz][a2] : T(1), d2 = (D == 3) ? tb.Dn[iz][a2] : T(0);
      const T phi = l1 * l2;
      const T dphi[3] = {dL0[a0] * l1 * l2, d1 * l2, l1 * d2};
      const T* Ji = A.jinv + ((mc * 2 + s) * NP + p) * D * D;
      T gn = T(0);
#pragma unroll
      for (int m = 0; m < D; ++m) {
        T g = T(0);
#pragma unroll
        for (int r = 0; r < D; ++r) g = fma(dphi[r], Ji[r * D + m], g);
        gn = fma(g, n[m], gn);
      }
      dv += w * A.nu * (tau_f * phi * phi - phi * gn);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) atomic_add(&A.dst[(int64_t)node * NF + c], dv);
  }
}


// ---------------------------------------------------------------------------
// Face terms, MODE 0 (dst += M src), every phase spread over all threads of
// the half-cell.  Same terms and tables as mortar_block, with the traces and
// the test-side integration sum-factorised over the two face directions
// (angular first, then z) and the point data precomputed per rotor angle
// (cos / sin of the point's angle; the nodal basis is a Kronecker delta on
// the face and its normal derivative there is the table dLe).  Per side:
//   2a  face layer fa (all fields) and normal derivative fn (velocity)
//   2b  traces u and reference velocity gradients du at the points
//   2c  physical velocity gradients GU = du J^-1
//   3   fluxes fv, Fx of the face terms at the points
//   4a  integration against the face test functions: G (values), H (normal
//       derivative)
//   4b  node a = a0 + N q: l_a0(face) G_q + l_a0'(face) H_q, scatter-add.
template <int D, int K, typename T> struct MortarApplySmem {
  static constexpr int N = K + 1, NPC = ipow(N, D), NP = ipow(N, D - 1), NF = D + 1, MPB = MortarCfg<D, K>::MPB;
  // three regions reused across phases (lifetimes do not overlap within a region)
  static constexpr int NV3 = 10, NZ3 = 13;                        // 3D intermediate variants
  static constexpr int R1 = cmax(cmax(NPC * NF, N * N * NV3), cmax(NP * (NF + D * D), NP * (NF + D)));
  static constexpr int R2 = cmax(NP * (NF + D) + NP * D * D, N * N * NZ3);
  static constexpr int R3 = NP * NF + NP * D * D;
  T r1[MPB][2][R1];   // val | Y | fv, Fx | G, H
  T r2[MPB][2][R2];   // fa, fn, DU | Z
  T r3[MPB][2][R3];   // U, GU
  T L1[MPB][2][N][N];
  T dL1[MPB][2][N][N];
};

// ELEM = true (Algorithm 2, mortar part of the local matrices): slot lm of
// the block is (mortar cell mc, column side sc, local DoF column j), slot =
// blk * MPB + lm = (mc * 2 + sc) * NL + j; the input is the unit vector of DoF
// j on side sc (zero on the other side, wall velocities zero) and side sc's
// rows of the result, the own-side block's column j, are added to E[cell]
// (column-major [NL][NL]); the other side's rows (the coupling block) belong
// to no local matrix and are dropped.
template <int D, int K, typename T, bool ELEM = false>
__device__ __forceinline__ void mortar_apply_block(MortarApplySmem<D, K, T>& S, int64_t blk, const MortarArgs<T>& A,
                                                   T* __restrict__ E = nullptr) {
  using C = MortarCfg<D, K>;
  using SM = MortarApplySmem<D, K, T>;
  constexpr int N = C::N, NPC = C::NPC, NP = C::NP, NF = D + 1, TPM = 2 * NPC, NL = NPC * NF;
  const MfTab<T>& tb = TabSel<T>::get(K);
  const int lm = threadIdx.x / TPM;
  const int loc = threadIdx.x % TPM;
  const int64_t slot = blk * C::MPB + lm;
  const int64_t mc = ELEM ? slot / (2 * NL) : slot;
  const int sc = ELEM ? (int)((slot / NL) % 2) : 0;
  const int jcol = ELEM ? (int)(slot % NL) : 0;
  const bool active = mc < A.nm;
  // region views, per side
  auto val = [&](int s, int a, int f) -> T& { return S.r1[lm][s][a * NF + f]; };
  auto fa = [&](int s, int q, int f) -> T& { return S.r2[lm][s][q * NF + f]; };
  auto fn = [&](int s, int q, int c) -> T& { return S.r2[lm][s][NP * NF + q * D + c]; };
  auto DU = [&](int s, int p, int c, int r) -> T& { return S.r2[lm][s][NP * (NF + D) + (p * D + c) * D + r]; };
  auto Y = [&](int s, int ia, int b2, int v) -> T& { return S.r1[lm][s][(ia * N + b2) * SM::NV3 + v]; };
  auto U = [&](int s, int p, int f) -> T& { return S.r3[lm][s][p * NF + f]; };
  auto GU = [&](int s, int p, int c, int m) -> T& { return S.r3[lm][s][NP * NF + (p * D + c) * D + m]; };
  auto FV = [&](int s, int p, int f) -> T& { return S.r1[lm][s][p * NF + f]; };
  auto FX = [&](int s, int p, int c, int r) -> T& { return S.r1[lm][s][NP * NF + (p * D + c) * D + r]; };
  auto Z = [&](int s, int ia, int a2, int v) -> T& { return S.r2[lm][s][(ia * N + a2) * SM::NZ3 + v]; };
  // G, H: in 3D read Z (r2) and go to r1; in 2D they read fv, Fx (r1) and go to r2
  auto GH = [&](int s) -> T* { return D == 3 ? S.r1[lm][s] : S.r2[lm][s]; };
  auto G = [&](int s, int q, int f) -> T& { return GH(s)[q * NF + f]; };
  auto H = [&](int s, int q, int c) -> T& { return GH(s)[NP * NF + q * D + c]; };

  // ---- phase 1: gather both sides (node a of side s per thread), 1D tables along the face
  int node = 0;
  {
    const int s = loc / NPC, a = loc % NPC;
    if (active) {
      const int cell = A.mc_cell[2 * mc + s];
      const int id = A.cells[(int64_t)cell * NPC + a];
      const bool wall = id < 0;
      node = wall ? ~id : id;
#pragma unroll
      for (int f = 0; f < NF; ++f)
        val(s, a, f) = ELEM ? T(s == sc && a * NF + f == jcol ? 1 : 0) : from_io<T>(A.src[(int64_t)node * NF + f]);
      if (wall && (ELEM || A.zero_wall)) {
#pragma unroll
        for (int c = 0; c < D; ++c) val(s, a, c) = T(0);
      }
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f) val(s, a, f) = T(0);
    }
    if (a < N) {
      T L1[N], dL1[N];
      lagrange_at<N, T>(tb, active ? (T)A.mc_xi[(mc * 2 + s) * N + a] : T(0), L1, dL1);
#pragma unroll
      for (int b = 0; b < N; ++b) { S.L1[lm][s][a][b] = L1[b]; S.dL1[lm][s][a][b] = dL1[b]; }
    }
  }
  __syncthreads();
  // ---- 2a: face layer (xi_0 = 1 rotor, 0 stator) and its normal derivative
  for (int it = loc; it < 2 * NP * NF; it += TPM) {
    const int s = it / (NP * NF), q = (it / NF) % NP, f = it % NF;
    const int fc = (s == 0) ? K : 0;
    const T v = val(s, fc + N * q, f);
    T dn = T(0);
    if (f < D) {
#pragma unroll
      for (int b0 = 0; b0 < N; ++b0) dn = fma(tb.dLe[s == 0 ? 1 : 0][b0], val(s, b0 + N * q, f), dn);
    }
    fa(s, q, f) = v;
    if (f < D) fn(s, q, f) = dn;
  }
  __syncthreads();
  if constexpr (D == 3) {
    // ---- 2b (angular): Y[ia][b2] = {L1 fa (4), dL1 fa (3), L1 fn (3)}
    for (int it = loc; it < 2 * N * N * SM::NV3; it += TPM) {
      const int s = it / (N * N * SM::NV3), r = it % (N * N * SM::NV3);
      const int ia = r / (N * SM::NV3), b2 = (r / SM::NV3) % N, v = r % SM::NV3;
      T acc = T(0);
#pragma unroll
      for (int b1 = 0; b1 < N; ++b1) {
        const int q = b1 + N * b2;
        const T x = v < NF ? fa(s, q, v) : v < NF + D ? fa(s, q, v - NF) : fn(s, q, v - NF - D);
        const T m = (v >= NF && v < NF + D) ? S.dL1[lm][s][ia][b1] : S.L1[lm][s][ia][b1];
        acc = fma(m, x, acc);
      }
      Y(s, ia, b2, v) = acc;
    }
    __syncthreads();
    // ---- 2b (z): u (4), du_0 (3, normal), du_1 (3, angular), du_2 (3, z) at p = ia + N iz
    for (int it = loc; it < 2 * NP * SM::NZ3; it += TPM) {
      const int s = it / (NP * SM::NZ3), p = (it / SM::NZ3) % NP, o = it % SM::NZ3;
      const int ia = p % N, iz = p / N;
      const int v = o < NF ? o : o < NF + D ? NF + D + (o - NF) : o < NF + 2 * D ? NF + (o - NF - D) : o - NF - 2 * D;
      T acc = T(0);
#pragma unroll
      for (int b2 = 0; b2 < N; ++b2) acc = fma(o < NF + 2 * D ? tb.B[iz][b2] : tb.Dn[iz][b2], Y(s, ia, b2, v), acc);
      if (o < NF) U(s, p, o) = acc;
      else DU(s, p, (o - NF) % D, (o - NF) / D) = acc;
    }
  } else {
    // ---- 2b (2D, one face direction): u (3), du_0 (2), du_1 (2) at p = ia
    constexpr int NO = NF + 2 * D;
    for (int it = loc; it < 2 * NP * NO; it += TPM) {
      const int s = it / (NP * NO), p = (it / NO) % NP, o = it % NO;
      T acc = T(0);
#pragma unroll
      for (int b1 = 0; b1 < N; ++b1) {
        const T x = o < NF ? fa(s, b1, o) : o < NF + D ? fn(s, b1, o - NF) : fa(s, b1, o - NF - D);
        const T m = o < NF + D ? S.L1[lm][s][p][b1] : S.dL1[lm][s][p][b1];
        acc = fma(m, x, acc);
      }
      if (o < NF) U(s, p, o) = acc;
      else DU(s, p, (o - NF) % D, (o - NF) / D) = acc;
    }
  }
  __syncthreads();
  // ---- 2c: physical velocity gradients
  for (int it = loc; it < 2 * NP * D * D; it += TPM) {
    const int s = it / (NP * D * D), p = (it / (D * D)) % NP, c = (it / D) % D, m = it % D;
    const T* Ji = A.jinv + ((mc * 2 + s) * NP + p) * D * D;
    T g = T(0);
#pragma unroll
    for (int r = 0; r < D; ++r) g = fma(DU(s, p, c, r), active ? Ji[r * D + m] : T(0), g);
    GU(s, p, c, m) = g;
  }
  __syncthreads();
  // ---- 3: fluxes of side s at point p
  for (int it = loc; it < 2 * NP; it += TPM) {
    const int s = it / NP, p = it % NP, ia = p % N, iz = (D == 3) ? p / N : 0;
    const int o = 1 - s;
    double wd = active ? A.mc_w[mc * N + ia] : 0.0;
    if (D == 3) wd *= TabSel<double>::get(K).w[iz] * A.dz;
    const T w = (T)wd;
    const T sg = (s == 0) ? T(1) : T(-1);
    const T n[3] = {active ? sg * (T)A.mc_cs[(mc * N + ia) * 2] : T(0),
                    active ? sg * (T)A.mc_cs[(mc * N + ia) * 2 + 1] : T(0), T(0)};
    const T tau_f = active ? (T)A.mc_tau[mc] : T(0);
    T jump[D];
#pragma unroll
    for (int c = 0; c < D; ++c) jump[c] = U(s, p, c) - U(o, p, c);
    const T pavg = T(0.5) * (U(s, p, D) + U(o, p, D));
    T jn = T(0);
#pragma unroll
    for (int c = 0; c < D; ++c) jn = fma(jump[c], n[c], jn);
    T fvl[NF];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T gn = T(0);
#pragma unroll
      for (int m = 0; m < D; ++m) gn = fma(GU(s, p, c, m) + GU(o, p, c, m), n[m], gn);
      fvl[c] = w * (pavg * n[c] - T(0.5) * A.nu * gn + A.nu * tau_f * jump[c]);
    }
    fvl[D] = -T(0.5) * w * jn;
    const T* Ji = A.jinv + ((mc * 2 + s) * NP + p) * D * D;
    T jin[D];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      T t = T(0);
#pragma unroll
      for (int m = 0; m < D; ++m) t = fma(active ? Ji[r * D + m] : T(0), n[m], t);
      jin[r] = t;
    }
    const T hw = -T(0.5) * w * A.nu;
#pragma unroll
    for (int f = 0; f < NF; ++f) FV(s, p, f) = fvl[f];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int r = 0; r < D; ++r) FX(s, p, c, r) = hw * jump[c] * jin[r];
  }
  __syncthreads();
  if constexpr (D == 3) {
    // ---- 4a (z): Z[ia][a2] = {B fv (4), B Fx_.1 (3), Dn Fx_.2 (3), B Fx_.0 (3)}
    for (int it = loc; it < 2 * N * N * SM::NZ3; it += TPM) {
      const int s = it / (N * N * SM::NZ3), r = it % (N * N * SM::NZ3);
      const int ia = r / (N * SM::NZ3), a2 = (r / SM::NZ3) % N, v = r % SM::NZ3;
      T acc = T(0);
#pragma unroll
      for (int iz = 0; iz < N; ++iz) {
        const int p = ia + N * iz;
        const T x = v < NF ? FV(s, p, v)
                  : v < NF + D ? FX(s, p, v - NF, 1)
                  : v < NF + 2 * D ? FX(s, p, v - NF - D, 2) : FX(s, p, v - NF - 2 * D, 0);
        const T m = (v >= NF + D && v < NF + 2 * D) ? tb.Dn[iz][a2] : tb.B[iz][a2];
        acc = fma(m, x, acc);
      }
      Z(s, ia, a2, v) = acc;
    }
    __syncthreads();
    // ---- 4a (angular): G_q (4), H_q (3) at q = a1 + N a2
    for (int it = loc; it < 2 * NP * (NF + D); it += TPM) {
      const int s = it / (NP * (NF + D)), q = (it / (NF + D)) % NP, o = it % (NF + D);
      const int a1 = q % N, a2 = q / N;
      T acc = T(0);
#pragma unroll
      for (int ia = 0; ia < N; ++ia) {
        const T l1 = S.L1[lm][s][ia][a1];
        if (o < D) {
          acc = fma(l1, Z(s, ia, a2, o) + Z(s, ia, a2, NF + D + o), acc);
          acc = fma(S.dL1[lm][s][ia][a1], Z(s, ia, a2, NF + o), acc);
        } else if (o == D) {
          acc = fma(l1, Z(s, ia, a2, D), acc);
        } else {
          acc = fma(l1, Z(s, ia, a2, NF + 2 * D + (o - NF)), acc);
        }
      }
      if (o < NF) G(s, q, o) = acc;
      else H(s, q, o - NF) = acc;
    }
  } else {
    // ---- 4a (2D): G_q (3), H_q (2) at q = a1
    for (int it = loc; it < 2 * NP * (NF + D); it += TPM) {
      const int s = it / (NP * (NF + D)), q = (it / (NF + D)) % NP, o = it % (NF + D);
      T acc = T(0);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const T l1 = S.L1[lm][s][p][q];
        if (o < D) acc = fma(S.dL1[lm][s][p][q], FX(s, p, o, 1), fma(l1, FV(s, p, o), acc));
        else if (o == D) acc = fma(l1, FV(s, p, D), acc);
        else acc = fma(l1, FX(s, p, o - NF, 0), acc);
      }
      if (o < NF) G(s, q, o) = acc;
      else H(s, q, o - NF) = acc;
    }
  }
  __syncthreads();
  if (!active) return;
  // ---- 4b: node a = a0 + N q of side s
  {
    const int s = loc / NPC, a = loc % NPC;
    const int a0 = a % N, q = a / N, fc = (s == 0) ? K : 0;
    const T dl = tb.dLe[s == 0 ? 1 : 0][a0];
    T out[NF];
#pragma unroll
    for (int c = 0; c < D; ++c) out[c] = (a0 == fc) ? fma(dl, H(s, q, c), G(s, q, c)) : dl * H(s, q, c);
    out[D] = (a0 == fc) ? G(s, q, D) : T(0);
    if constexpr (ELEM) {
      if (s == sc) {
        T* col = E + ((int64_t)A.mc_cell[2 * mc + s] * NL + jcol) * NL + a * NF;
#pragma unroll
        for (int f = 0; f < NF; ++f) atomicAdd(col + f, out[f]);
      }
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f) atomic_add(&A.dst[(int64_t)node * NF + f], out[f]);
    }
  }
}

// Mortar own-side blocks of the local matrices (FP32): nm * 2 * NL slots.
template <int D, int K>
__global__ void __launch_bounds__(MortarCfg<D, K>::THREADS) k_mortar_elem(MortarArgs<float> A, float* __restrict__ E) {
  __shared__ MortarApplySmem<D, K, float> S;
  mortar_apply_block<D, K, float, true>(S, blockIdx.x, A, E);
}

template <int D, int K, typename T, int MODE>
__global__ void __launch_bounds__(MortarCfg<D, K>::THREADS) k_mortar(MortarArgs<T> A) {
  if constexpr (MODE == 0) {
    __shared__ MortarApplySmem<D, K, T> S;
    mortar_apply_block<D, K, T>(S, blockIdx.x, A);
  } else {
    __shared__ MortarSmem<D, K, T> S;
    mortar_block<D, K, T, MODE>(S, blockIdx.x, A);
  }
}

// Batched mortar terms (MODE 0) over several instances: persistent grid,
// tiles from a device counter, tile -> instance by the prefix table.
template <typename T> struct MortarBatchTable {
  int ninst;
  int64_t first_tile[MF_BATCH_MAX + 1];
  MortarArgs<T> inst[MF_BATCH_MAX];
};

template <int D, int K, typename T>
__global__ void __launch_bounds__(MortarCfg<D, K>::THREADS)
k_mortar_batched(const MortarBatchTable<T>* __restrict__ tab, unsigned long long* __restrict__ counter) {
  __shared__ MortarApplySmem<D, K, T> S;
  __shared__ long long s_tile;
  const int64_t total = tab->first_tile[tab->ninst];
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= total) break;
    int i = 0;
    while (i + 1 < tab->ninst && tab->first_tile[i + 1] <= tile) ++i;
    mortar_apply_block<D, K, T>(S, tile - tab->first_tile[i], tab->inst[i]);
  }
}

}  // namespace mf
