// Batched periodic-RVE Newton solver for 3D (Hex8, 2x2x2 Gauss), one thread block per RVE,
// persistent over a work queue of macro quadrature points (uneven grid sizes in one launch,
// largest first).
//
// Method (paper Sec. 3.2-3.3): identical to the 2D kernel — R_a = sum wt detJ P(Fbar + Grad w)
// Grad N_a (Eq. f_I^int, micro), Newton corrections K_T dw = -R (Eq. Saddlepoint-problem-Set-
// of-eqs with periodic elimination, ch_3_eq_22), Pbar = <P> (Eq. Average-of-P-and-F) and the
// tangent transfer Abar = <A> - L^T K^-1 L with L = dR/dFbar (the condensed form of the paper's
// omega/|K_delta| T^T K T, Eq. k-mac-element-6; the two are checked equal in the oracle tests).
//
// GB300 layout:
//  * 512 threads per block, one block per SM.  Elements are processed thread-strided; the
//    nodal unknowns live in per-block global scratch (L2 resident), except the vector the
//    tangent is applied to and its product, which live in shared memory.
//  * Residual in FP64 per element (edge differences of the fluctuation; P = mu F + hb F^-T),
//    element forces staged in global scratch and gathered per node (deterministic sums).
//  * Tangent apply matrix-free in TA (FP32 in mixed mode): per Gauss point the kernel stores
//    F^-T, hb and lam J^2 (11 values); the apply computes dF = Grad p from edge differences,
//    dP = mu dF - hb Fit dF^T Fit + gm (Fit:dF) Fit and adds the element's nodal results to
//    shared memory with float atomics.
//  * Preconditioner: geometric multigrid V(1,1)-cycle with Galerkin coarse levels where the
//    grid halves down to 2 or 3 nodes per axis, else block-Jacobi with the 3x3 nodal diagonal
//    blocks; PCG in the single-reduction form of Chronopoulos and Gear; truncated on negative
//    curvature for Newton corrections.
//  * Tangent transfer: L_c = apply of the element operator to the constant gradient E_c (the
//    affine field), 9 PCG solves X_c = -K^-1 L_c, Abar = <A> + sym(L^T X), all sums in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "fehmm_device.cuh"
#include "rve_args.h"

namespace fehmm {
namespace {

constexpr int kThreads3D = 512;
// Gauss-point data per law: neo-Hookean Fit (9), hb, gm, padding (12); St. Venant-Kirchhoff F (9),
// S (6: 00, 01, 02, 11, 12, 22), padding (16).  Scratch is sized for the larger.
constexpr int kLawNH = 0, kLawSVK = 1;
template <int LAW>
__host__ __device__ constexpr int qp_vals() { return LAW == kLawNH ? 12 : 16; }
constexpr int kQp3Max = 16;

// Pinned nodes of the fluctuation: node 0 (periodic coupling) or every node on the lattice
// planes i = 0, j = 0 or k = 0 (KUBC: the cell boundary).
__device__ __forceinline__ bool pinned3(int v, int n, int bc) {
  if (!bc) return v == 0;
  const int i = v % n, j = (v / n) % n, k = v / (n * n);
  return i == 0 || j == 0 || k == 0;
}

// Gauss-point data layout [8 qp][NQ values][NE] grouped into 4-wide vectors so that a thread
// loads its element's data with NQ/4 float4 (FP32) or NQ/2 double2 (FP64) loads, coalesced over e.
template <int NQ>
__device__ __forceinline__ void load_qp(const float* qpd, int NE, int q, int e, float (&d)[NQ]) {
  const float4* b = reinterpret_cast<const float4*>(qpd) + (size_t)(q * (NQ / 4)) * NE + e;
#pragma unroll
  for (int j = 0; j < NQ / 4; ++j) {
    const float4 v = b[(size_t)j * NE];
    d[4 * j] = v.x;
    d[4 * j + 1] = v.y;
    d[4 * j + 2] = v.z;
    d[4 * j + 3] = v.w;
  }
}
template <int NQ>
__device__ __forceinline__ void load_qp(const double* qpd, int NE, int q, int e, double (&d)[NQ]) {
  const double2* b = reinterpret_cast<const double2*>(qpd) + (size_t)(q * (NQ / 2)) * NE + e;
#pragma unroll
  for (int j = 0; j < NQ / 2; ++j) {
    const double2 v = b[(size_t)j * NE];
    d[2 * j] = v.x;
    d[2 * j + 1] = v.y;
  }
}
template <int NQ>
__device__ __forceinline__ void store_qp(float* qpd, int NE, int q, int e, const float (&d)[NQ]) {
  float4* b = reinterpret_cast<float4*>(qpd) + (size_t)(q * (NQ / 4)) * NE + e;
#pragma unroll
  for (int j = 0; j < NQ / 4; ++j) b[(size_t)j * NE] = make_float4(d[4 * j], d[4 * j + 1], d[4 * j + 2], d[4 * j + 3]);
}
template <int NQ>
__device__ __forceinline__ void store_qp(double* qpd, int NE, int q, int e, const double (&d)[NQ]) {
  double2* b = reinterpret_cast<double2*>(qpd) + (size_t)(q * (NQ / 2)) * NE + e;
#pragma unroll
  for (int j = 0; j < NQ / 2; ++j) b[(size_t)j * NE] = make_double2(d[2 * j], d[2 * j + 1]);
}

__device__ __forceinline__ double g01(int g) { return g == 0 ? 0.21132486540518711775 : 0.78867513459481288225; }

template <typename T>
__device__ __forceinline__ T phi(int o, T t) { return o ? t : T(1) - t; }

// 3x3 helpers (row-major, index 3*i + J)
template <typename T>
struct NH3 {
  T Fit[9];
  T J, hb, gm;
};

template <typename T>
__device__ __forceinline__ NH3<T> nh3_eval(const T (&F)[9], T lam, T mu) {
  NH3<T> r;
  // cofactor matrix cof_iJ = dJ/dF_iJ; F^-T = cof / J
  const T c00 = F[4] * F[8] - F[5] * F[7], c01 = F[5] * F[6] - F[3] * F[8], c02 = F[3] * F[7] - F[4] * F[6];
  const T c10 = F[2] * F[7] - F[1] * F[8], c11 = F[0] * F[8] - F[2] * F[6], c12 = F[1] * F[6] - F[0] * F[7];
  const T c20 = F[1] * F[5] - F[2] * F[4], c21 = F[2] * F[3] - F[0] * F[5], c22 = F[0] * F[4] - F[1] * F[3];
  r.J = F[0] * c00 + F[1] * c01 + F[2] * c02;
  const T iJ = recip_T(r.J);
  r.Fit[0] = c00 * iJ;
  r.Fit[1] = c01 * iJ;
  r.Fit[2] = c02 * iJ;
  r.Fit[3] = c10 * iJ;
  r.Fit[4] = c11 * iJ;
  r.Fit[5] = c12 * iJ;
  r.Fit[6] = c20 * iJ;
  r.Fit[7] = c21 * iJ;
  r.Fit[8] = c22 * iJ;
  const T J2 = r.J * r.J;
  r.hb = T(0.5) * lam * (J2 - T(1)) - mu;
  r.gm = lam * J2;
  return r;
}

// dP = mu dF - hb Fit dF^T Fit + gm (Fit:dF) Fit
template <typename T>
__device__ __forceinline__ void tangent_action(const T* Fit, T hb, T gm, T mu, const T (&dF)[9], T (&dP)[9]) {
  T U[9];  // U = dF^T Fit : U_LJ = sum_k dF_kL Fit_kJ
#pragma unroll
  for (int L = 0; L < 3; ++L)
#pragma unroll
    for (int J = 0; J < 3; ++J) U[3 * L + J] = dF[L] * Fit[J] + dF[3 + L] * Fit[3 + J] + dF[6 + L] * Fit[6 + J];
  T a = T(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) a += Fit[k] * dF[k];
  const T ga = gm * a;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int J = 0; J < 3; ++J) {
      const T t = Fit[3 * i + 0] * U[0 * 3 + J] + Fit[3 * i + 1] * U[1 * 3 + J] + Fit[3 * i + 2] * U[2 * 3 + J];
      dP[3 * i + J] = mu * dF[3 * i + J] - hb * t + ga * Fit[3 * i + J];
    }
}

// St. Venant-Kirchhoff (S = lam tr(E) I + 2 mu E, E = (F^T F - I)/2): S as 6 values (00, 01, 02,
// 11, 12, 22).
template <typename T>
__device__ __forceinline__ void svk3_S(const T* F, T lam, T mu, T (&S6)[6]) {
  T C[6];  // C = F^T F, same order
  const int I6[6] = {0, 0, 0, 1, 1, 2}, J6[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int k = 0; k < 6; ++k) C[k] = F[I6[k]] * F[J6[k]] + F[3 + I6[k]] * F[3 + J6[k]] + F[6 + I6[k]] * F[6 + J6[k]];
  const T trE = T(0.5) * (C[0] + C[3] + C[5]) - T(1.5);
  S6[0] = lam * trE + mu * (C[0] - T(1));
  S6[3] = lam * trE + mu * (C[3] - T(1));
  S6[5] = lam * trE + mu * (C[5] - T(1));
  S6[1] = mu * C[1];
  S6[2] = mu * C[2];
  S6[4] = mu * C[4];
}

// symmetric 3x3 entry (I, J) of 6 stored values
template <typename T>
__device__ __forceinline__ T sym6(const T (&S6)[6], int I, int J) {
  const int a = I < J ? I : J, b = I < J ? J : I;
  return S6[a == 0 ? b : (a == 1 ? 2 + b : 5)];
}

// St. Venant-Kirchhoff tangent action: dP = dF S + F dS, dS = lam tr(U) I + mu (U + U^T), U = F^T dF.
template <typename T>
__device__ __forceinline__ void svk_tangent_action(const T* F, const T* S6p, T lam, T mu, const T (&dF)[9],
                                                   T (&dP)[9]) {
  T S6[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) S6[k] = S6p[k];
  T U[9];
#pragma unroll
  for (int I = 0; I < 3; ++I)
#pragma unroll
    for (int J = 0; J < 3; ++J) U[3 * I + J] = F[I] * dF[J] + F[3 + I] * dF[3 + J] + F[6 + I] * dF[6 + J];
  const T lt = lam * (U[0] + U[4] + U[8]);
  T dS[9];
#pragma unroll
  for (int I = 0; I < 3; ++I)
#pragma unroll
    for (int J = 0; J < 3; ++J) dS[3 * I + J] = mu * (U[3 * I + J] + U[3 * J + I]) + (I == J ? lt : T(0));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int J = 0; J < 3; ++J) {
      T v = T(0);
#pragma unroll
      for (int K = 0; K < 3; ++K) v += dF[3 * i + K] * sym6(S6, K, J) + F[3 * i + K] * dS[3 * K + J];
      dP[3 * i + J] = v;
    }
}

struct Geo3 {
  int n, NN;
  __device__ __forceinline__ int node(int i, int j, int k) const {
    return (i % n) + n * ((j % n) + n * (k % n));
  }
  // corner a = ox + 2 oy + 4 oz of element e
  __device__ __forceinline__ void corners(int e, int (&nd)[8]) const {
    const int i = e % n, j = (e / n) % n, k = e / (n * n);
#pragma unroll
    for (int a = 0; a < 8; ++a) nd[a] = node(i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
  }
};

// natural-coordinate gradient of a nodal field u[8][3] at (s,t,r): G[3*i + J] = du_i/dxi_J
template <typename T>
__device__ __forceinline__ void nat_grad(const T (&u)[8][3], T s, T t, T r, T (&G)[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
    for (int oy = 0; oy < 2; ++oy)
#pragma unroll
      for (int oz = 0; oz < 2; ++oz) {
        const int a0 = 2 * oy + 4 * oz;
        gx += (u[a0 + 1][i] - u[a0][i]) * phi(oy, t) * phi(oz, r);
      }
#pragma unroll
    for (int ox = 0; ox < 2; ++ox)
#pragma unroll
      for (int oz = 0; oz < 2; ++oz) {
        const int a0 = ox + 4 * oz;
        gy += (u[a0 + 2][i] - u[a0][i]) * phi(ox, s) * phi(oz, r);
      }
#pragma unroll
    for (int ox = 0; ox < 2; ++ox)
#pragma unroll
      for (int oy = 0; oy < 2; ++oy) {
        const int a0 = ox + 2 * oy;
        gz += (u[a0 + 4][i] - u[a0][i]) * phi(ox, s) * phi(oy, t);
      }
    G[3 * i + 0] = gx;
    G[3 * i + 1] = gy;
    G[3 * i + 2] = gz;
  }
}

// y_a += c * sum_J S_iJ dN_a/dxi_J at (s,t,r) for the 8 corners
template <typename T>
__device__ __forceinline__ void nat_scatter(const T (&S)[9], T c, T s, T t, T r, T (&y)[8][3]) {
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int ox = a & 1, oy = (a >> 1) & 1, oz = (a >> 2) & 1;
    const T dx = (ox ? T(1) : T(-1)) * phi(oy, t) * phi(oz, r);
    const T dy = (oy ? T(1) : T(-1)) * phi(ox, s) * phi(oz, r);
    const T dz = (oz ? T(1) : T(-1)) * phi(ox, s) * phi(oy, t);
#pragma unroll
    for (int i = 0; i < 3; ++i) y[a][i] += c * (S[3 * i] * dx + S[3 * i + 1] * dy + S[3 * i + 2] * dz);
  }
}

template <typename TA>
struct Scratch3 {
  // per-block global scratch, layout set by scratch3_layout
  double* Rf;   // [24][NE] element forces (FP64)
  TA* qpd;      // [8][qp_vals][NE] Gauss-point material data (4-wide groups, see load_qp)
  TA* x;        // [3][NN] PCG solution
  TA* r;        // [3][NN]
  TA* p;        // [3][NN]
  TA* s;        // [3][NN]
  TA* mi;       // [6][NN] inverted diagonal blocks (xx, xy, xz, yy, yz, zz)
  TA* L;        // [9][3][NN] transfer right-hand sides
  TA* mg;       // multigrid levels (mg3_elems)
};

// ------------------------------------------------------------ multigrid sizes (3D)
// Coarse levels: halve while the grid is even and above 3 (16 -> 8, 4, 2; 12 -> 6, 3; 8 -> 4, 2);
// 0 when the hierarchy does not end at 2 or 3 nodes per axis.
__host__ __device__ inline int mg3_levels(int n) {
  int l = 0, m = n;
  while (m > 3 && (m & 1) == 0) {
    m >>= 1;
    ++l;
  }
  return (m <= 3 && l >= 1) ? l : 0;
}
// Elements (TA) of the multigrid region for grid n: per coarse level the element blocks
// [36][9][NE], the inverted nodal blocks [6][NN] and r, z, t [3][NN]; then the coarsest
// inverse (two buffers of D x (D + 1), D = 3 NN_c).
__host__ __device__ inline long long mg3_elems(int n) {
  const int L = mg3_levels(n);
  if (!L) return 0;
  long long e = 0;
  for (int l = 1; l <= L; ++l) {
    const long long m = n >> l, nn = m * m * m;
    e += 324 * nn + 6 * nn + 9 * nn;
  }
  const long long m = n >> L, D = 3 * m * m * m;
  return e + 2 * D * (D + 1);
}
__host__ __device__ inline long long mg3_elems_max(int nn_max) {
  long long mx = 0;
  for (int n = 2; n * n * n <= nn_max; ++n) mx = mg3_elems(n) > mx ? mg3_elems(n) : mx;
  return mx;
}

template <typename TA>
__host__ __device__ inline size_t scratch3_base_bytes(int NN) {
  const size_t b = sizeof(double) * 24 * (size_t)NN +
                   sizeof(TA) * ((size_t)kQp3Max * 8 * NN + 4 * 3 * (size_t)NN + 6 * (size_t)NN + 27 * (size_t)NN);
  return (b + 255) & ~size_t(255);
}

template <typename TA>
__host__ __device__ inline size_t scratch3_bytes(int NN) {
  const size_t b = scratch3_base_bytes<TA>(NN) + sizeof(TA) * (size_t)mg3_elems_max(NN);
  return (b + 255) & ~size_t(255);  // every block's scratch starts 256-byte aligned
}

template <typename TA>
__device__ inline Scratch3<TA> scratch3_layout(unsigned char* base, int NN) {
  Scratch3<TA> s;
  s.Rf = reinterpret_cast<double*>(base);
  TA* t = reinterpret_cast<TA*>(base + sizeof(double) * 24 * (size_t)NN);
  s.qpd = t;
  t += (size_t)kQp3Max * 8 * NN;
  s.x = t;
  t += 3 * (size_t)NN;
  s.r = t;
  t += 3 * (size_t)NN;
  s.p = t;
  t += 3 * (size_t)NN;
  s.s = t;
  t += 3 * (size_t)NN;
  s.mi = t;
  t += 6 * (size_t)NN;
  s.L = t;
  s.mg = reinterpret_cast<TA*>(base + scratch3_base_bytes<TA>(NN));
  return s;
}

// shared memory: vin [3][NN], vout [3][NN] (TA), reductions, lame, misc
template <typename TA>
__host__ __device__ inline size_t smem3_bytes(int NN) {
  return sizeof(TA) * 6 * (size_t)NN + sizeof(double) * (2 * 512 + 2 * kMaxPhase + 128);
}

template <typename T>
__device__ __forceinline__ void block_sum_n(T* v, int nv, T* buf) {
  // nv <= 16 values; buf >= 32*16
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < nv; ++k) {
    T x = warp_sum(v[k]);
    if (lane == 0) buf[k * 32 + warp] = x;
  }
  __syncthreads();
  for (int k = 0; k < nv; ++k) v[k] = warp_sum(lane < nw ? buf[k * 32 + lane] : T(0));
  __syncthreads();
}

template <typename TA>
struct Mg3Level {
  int n, NN, bc;
  TA* kb;  // [36 block pairs a <= b][9][NN] element blocks (row-major 3x3)
  TA* mi;  // [6][NN] inverted nodal diagonal blocks (zero at node 0)
  TA* r;   // [3][NN]
  TA* z;   // [3][NN]
  TA* t;   // [3][NN]
};

template <typename TA>
struct Mg3 {
  int levels = 0;  // coarse levels, 0 = block-Jacobi
  int n = 0;       // fine grid
  int bc = 0;      // pinned nodes of every level as on the fine grid (pinned3)
  TA omega = TA(0.6);  // smoother damping
  TA* base = nullptr;
  __device__ __forceinline__ Mg3Level<TA> level(int l) const {
    TA* p = base;
    for (int q = 1; q < l; ++q) {
      const int m = n >> q;
      p += 339 * m * m * m;
    }
    Mg3Level<TA> v;
    v.n = n >> l;
    v.NN = v.n * v.n * v.n;
    v.bc = bc;
    v.kb = p;
    v.mi = p + 324 * v.NN;
    v.r = v.mi + 6 * v.NN;
    v.z = v.r + 3 * v.NN;
    v.t = v.z + 3 * v.NN;
    return v;
  }
  __device__ __forceinline__ TA* inverse() const {
    const Mg3Level<TA> c = level(levels);
    return c.t + 3 * c.NN;
  }
};

template <typename TA>
struct Ctx3 {
  Geo3 g;
  int NE;
  Mg3<TA> mg;
  const uint8_t* phase;
  const double* lame;  // shared [kMaxPhase][2]
  Scratch3<TA> sc;
  TA* vin;   // shared [3][NN]
  TA* vout;  // shared [3][NN]
  double* red;  // shared 2*512
  int bc;       // 0 periodic, 1 KUBC (pinned3)
  double Fb[9];
};

// ---------------------------------------------------------------- FP64 residual
template <typename TA, int LAW>
__device__ __noinline__ void residual3(const Ctx3<TA>& c, const double* w, double (&Psum)[9], double& bad) {
  const int n = c.g.n;
  const double ih = (double)n, cw = 0.125 / (ih * ih);  // wq / h = h^2 / 8
  for (int e = threadIdx.x; e < c.NE; e += blockDim.x) {
    int nd[8];
    c.g.corners(e, nd);
    double u[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) u[a][i] = w[3 * nd[a] + i];
    const int ph = c.phase[e];
    const double lam = c.lame[2 * ph], mu = c.lame[2 * ph + 1];
    double y[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a) y[a][0] = y[a][1] = y[a][2] = 0.0;
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      const double s = g01(q & 1), t = g01((q >> 1) & 1), r = g01(q >> 2);
      double G[9], F[9];
      nat_grad(u, s, t, r, G);
#pragma unroll
      for (int k = 0; k < 9; ++k) F[k] = c.Fb[k] + ih * G[k];
      double P[9];
      if constexpr (LAW == kLawNH) {
        // P = mu F + hb F^-T = mu F + (hb / J) cof(F), the reciprocal refined in FP64
        double cof[9];
        cof[0] = F[4] * F[8] - F[5] * F[7];
        cof[1] = F[5] * F[6] - F[3] * F[8];
        cof[2] = F[3] * F[7] - F[4] * F[6];
        cof[3] = F[2] * F[7] - F[1] * F[8];
        cof[4] = F[0] * F[8] - F[2] * F[6];
        cof[5] = F[1] * F[6] - F[0] * F[7];
        cof[6] = F[1] * F[5] - F[2] * F[4];
        cof[7] = F[2] * F[3] - F[0] * F[5];
        cof[8] = F[0] * F[4] - F[1] * F[3];
        const double J = F[0] * cof[0] + F[1] * cof[1] + F[2] * cof[2];
        bad += J > 0.0 ? 0.0 : 1.0;
        const double c = (0.5 * lam * (J * J - 1.0) - mu) * recip_fp64(J);
#pragma unroll
        for (int k = 0; k < 9; ++k) P[k] = fma(mu, F[k], c * cof[k]);
      } else {
        const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                         F[2] * (F[3] * F[7] - F[4] * F[6]);
        bad += J > 0.0 ? 0.0 : 1.0;
        double S6[6];
        svk3_S(F, lam, mu, S6);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int J2 = 0; J2 < 3; ++J2)
            P[3 * i + J2] = F[3 * i] * sym6(S6, 0, J2) + F[3 * i + 1] * sym6(S6, 1, J2) + F[3 * i + 2] * sym6(S6, 2, J2);
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) Psum[k] += P[k];
      nat_scatter(P, cw, s, t, r, y);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) c.sc.Rf[(size_t)(3 * a + i) * c.NE + e] = y[a][i];
  }
}

// sum over this thread's elements of psi at the Gauss points (FP64; Eq. NH-free-energy)
template <typename TA, int LAW>
__device__ __noinline__ double energy3(const Ctx3<TA>& c, const double* w) {
  const int n = c.g.n;
  const double ih = (double)n;
  double acc = 0.0;
  for (int e = threadIdx.x; e < c.NE; e += blockDim.x) {
    int nd[8];
    c.g.corners(e, nd);
    double u[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) u[a][i] = w[3 * nd[a] + i];
    const int ph = c.phase[e];
    const double lam = c.lame[2 * ph], mu = c.lame[2 * ph + 1];
    for (int q = 0; q < 8; ++q) {
      const double s = g01(q & 1), t = g01((q >> 1) & 1), r = g01(q >> 2);
      double G[9], F[9];
      nat_grad(u, s, t, r, G);
#pragma unroll
      for (int k = 0; k < 9; ++k) F[k] = c.Fb[k] + ih * G[k];
      if constexpr (LAW == kLawNH) {
        const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                         F[2] * (F[3] * F[7] - F[4] * F[6]);
        double trC = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) trC += F[k] * F[k];
        acc += 0.25 * lam * (J * J - 1.0) - (0.5 * lam + mu) * log(J) + 0.5 * mu * (trC - 3.0);
      } else {  // lam/2 (tr E)^2 + mu E:E, E = (F^T F - I)/2
        double E[9];
#pragma unroll
        for (int I = 0; I < 3; ++I)
#pragma unroll
          for (int J2 = 0; J2 < 3; ++J2)
            E[3 * I + J2] = 0.5 * (F[I] * F[J2] + F[3 + I] * F[3 + J2] + F[6 + I] * F[6 + J2] - (I == J2 ? 1.0 : 0.0));
        const double trE = E[0] + E[4] + E[8];
        double ee = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) ee += E[k] * E[k];
        acc += 0.5 * lam * trE * trE + mu * ee;
      }
    }
  }
  return acc;
}

// gather element forces of node v: corner a of element (node - offset(a))
template <typename TA>
__device__ __forceinline__ void gather_R(const Ctx3<TA>& c, int v, double (&R)[3]) {
  const int n = c.g.n;
  const int i = v % n, j = (v / n) % n, k = v / (n * n);
  R[0] = R[1] = R[2] = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int e = c.g.node(i + n - (a & 1), j + n - ((a >> 1) & 1), k + n - ((a >> 2) & 1));
#pragma unroll
    for (int d = 0; d < 3; ++d) R[d] += c.sc.Rf[(size_t)(3 * a + d) * c.NE + e];
  }
}

// ------------------------------------------------------- tangent data (TA)
// Gauss-point data and nodal diagonal blocks (accumulated in shared memory vin|vout as
// [6][NN]); optional FP64 accumulation of <A> (45 symmetric entries) for the transfer.
template <typename TA, int LAW, bool withA>
__device__ __noinline__ void tangent3(const Ctx3<TA>& c, const double* w, double* Asum /*[45] per thread, withA only*/) {
  const int n = c.g.n, NN = c.g.NN;
  TA* diag = c.vin;  // [6][NN] spans vin and vout
  for (int v = threadIdx.x; v < 6 * NN; v += blockDim.x) diag[v] = TA(0);
  __syncthreads();
  const TA ih = (TA)n, wq = TA(0.125) / (ih * ih * ih);
  for (int e = threadIdx.x; e < c.NE; e += blockDim.x) {
    int nd[8];
    c.g.corners(e, nd);
    TA u[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) u[a][i] = (TA)w[3 * nd[a] + i];
    const int ph = c.phase[e];
    const TA lam = (TA)c.lame[2 * ph], mu = (TA)c.lame[2 * ph + 1];
    TA D[8][6];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int k = 0; k < 6; ++k) D[a][k] = TA(0);
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
      const TA s = (TA)g01(q & 1), t = (TA)g01((q >> 1) & 1), r = (TA)g01(q >> 2);
      TA G[9], F[9];
      nat_grad(u, s, t, r, G);
#pragma unroll
      for (int k = 0; k < 9; ++k) F[k] = (TA)c.Fb[k] + ih * G[k];
      if constexpr (LAW == kLawNH) {
        const NH3<TA> m = nh3_eval(F, lam, mu);
        TA qv[12];
#pragma unroll
        for (int k = 0; k < 9; ++k) qv[k] = m.Fit[k];
        qv[9] = m.hb;
        qv[10] = m.gm;
        qv[11] = TA(0);
        store_qp<12>(c.sc.qpd, c.NE, q, e, qv);
        // diagonal blocks: K_aa,ik = wq [mu |g_a|^2 d_ik + (gm - hb) v_a,i v_a,k], v_a = Fit g_a
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int ox = a & 1, oy = (a >> 1) & 1, oz = (a >> 2) & 1;
          const TA gx = ih * (ox ? TA(1) : TA(-1)) * phi(oy, t) * phi(oz, r);
          const TA gy = ih * (oy ? TA(1) : TA(-1)) * phi(ox, s) * phi(oz, r);
          const TA gz = ih * (oz ? TA(1) : TA(-1)) * phi(ox, s) * phi(oy, t);
          const TA v0 = m.Fit[0] * gx + m.Fit[1] * gy + m.Fit[2] * gz;
          const TA v1 = m.Fit[3] * gx + m.Fit[4] * gy + m.Fit[5] * gz;
          const TA v2 = m.Fit[6] * gx + m.Fit[7] * gy + m.Fit[8] * gz;
          const TA mg = wq * mu * (gx * gx + gy * gy + gz * gz), cc = wq * (m.gm - m.hb);
          D[a][0] += mg + cc * v0 * v0;
          D[a][1] += cc * v0 * v1;
          D[a][2] += cc * v0 * v2;
          D[a][3] += mg + cc * v1 * v1;
          D[a][4] += cc * v1 * v2;
          D[a][5] += mg + cc * v2 * v2;
        }
        if constexpr (withA) {  // <A>_(iJ)(kL), upper triangle of the 9x9 major-symmetric matrix
          int idx = 0;
#pragma unroll
          for (int p = 0; p < 9; ++p)
#pragma unroll
            for (int qq = p; qq < 9; ++qq) {
              const int i = p / 3, J = p % 3, k = qq / 3, L = qq % 3;
              TA val = -m.hb * m.Fit[3 * i + L] * m.Fit[3 * k + J] + m.gm * m.Fit[3 * i + J] * m.Fit[3 * k + L];
              if (i == k && J == L) val += mu;
              Asum[idx++] += (double)(wq * val);
            }
        }
      } else {
        TA S6[6];
        svk3_S(F, lam, mu, S6);
        TA qv[16];
#pragma unroll
        for (int k = 0; k < 9; ++k) qv[k] = F[k];
#pragma unroll
        for (int k = 0; k < 6; ++k) qv[9 + k] = S6[k];
        qv[15] = TA(0);
        store_qp<16>(c.sc.qpd, c.NE, q, e, qv);
        TA b6[6];  // b = F F^T (00, 01, 02, 11, 12, 22)
        {
          const int I6[6] = {0, 0, 0, 1, 1, 2}, J6[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
          for (int k = 0; k < 6; ++k)
            b6[k] = F[3 * I6[k]] * F[3 * J6[k]] + F[3 * I6[k] + 1] * F[3 * J6[k] + 1] + F[3 * I6[k] + 2] * F[3 * J6[k] + 2];
        }
        // diagonal blocks: K_aa,ik = wq [d_ik g_a.S.g_a + lam v_a,i v_a,k + mu (|g_a|^2 b_ik + v_a,i v_a,k)],
        // v_a = F g_a
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int ox = a & 1, oy = (a >> 1) & 1, oz = (a >> 2) & 1;
          const TA g[3] = {ih * (ox ? TA(1) : TA(-1)) * phi(oy, t) * phi(oz, r),
                           ih * (oy ? TA(1) : TA(-1)) * phi(ox, s) * phi(oz, r),
                           ih * (oz ? TA(1) : TA(-1)) * phi(ox, s) * phi(oy, t)};
          TA v[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) v[i] = F[3 * i] * g[0] + F[3 * i + 1] * g[1] + F[3 * i + 2] * g[2];
          TA gSg = TA(0);
#pragma unroll
          for (int I = 0; I < 3; ++I)
#pragma unroll
            for (int J = 0; J < 3; ++J) gSg += g[I] * sym6(S6, I, J) * g[J];
          const TA gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
          const int I6[6] = {0, 0, 0, 1, 1, 2}, J6[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            TA val = (lam + mu) * v[I6[k]] * v[J6[k]] + mu * gg * b6[k];
            if (I6[k] == J6[k]) val += gSg;
            D[a][k] += wq * val;
          }
        }
        if constexpr (withA) {  // A_iJkL = d_ik S_JL + lam F_iJ F_kL + mu b_ik d_JL + mu F_iL F_kJ
          int idx = 0;
#pragma unroll
          for (int p = 0; p < 9; ++p)
#pragma unroll
            for (int qq = p; qq < 9; ++qq) {
              const int i = p / 3, J = p % 3, k = qq / 3, L = qq % 3;
              TA val = lam * F[3 * i + J] * F[3 * k + L] + mu * F[3 * i + L] * F[3 * k + J];
              if (i == k) val += sym6(S6, J, L);
              if (J == L) val += mu * sym6(b6, i, k);
              Asum[idx++] += (double)(wq * val);
            }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int k = 0; k < 6; ++k) atomicAdd(&diag[k * NN + nd[a]], D[a][k]);
  }
  __syncthreads();
  // invert the diagonal blocks (node 0 pinned: zero)
  for (int v = threadIdx.x; v < NN; v += blockDim.x) {
    const TA a00 = diag[v], a01 = diag[NN + v], a02 = diag[2 * NN + v];
    const TA a11 = diag[3 * NN + v], a12 = diag[4 * NN + v], a22 = diag[5 * NN + v];
    const TA c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
    const TA c11 = a00 * a22 - a02 * a02, c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
    const TA det = a00 * c00 + a01 * c01 + a02 * c02;
    const TA id = pinned3(v, n, c.bc) ? TA(0) : TA(1) / det;
    c.sc.mi[v] = c00 * id;
    c.sc.mi[NN + v] = c01 * id;
    c.sc.mi[2 * NN + v] = c02 * id;
    c.sc.mi[3 * NN + v] = c11 * id;
    c.sc.mi[4 * NN + v] = c12 * id;
    c.sc.mi[5 * NN + v] = c22 * id;
  }
  __syncthreads();
}

// Kept out of line so the element loop gets its own register allocation (no spills).
// vout = K vin (mode 0) or vout = L_c: the element operator applied to the constant
// gradient E_c (mode 1, c = 3k + L).  Pinned node 0 row zeroed.
template <typename TA, int LAW>
__device__ __noinline__ void apply3(const Ctx3<TA>& c, int mode, int cidx) {
  const int n = c.g.n, NN = c.g.NN;
  for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) c.vout[v] = TA(0);
  __syncthreads();
  const TA ih = (TA)n, cw = TA(0.125) / (ih * ih);
  for (int e = threadIdx.x; e < c.NE; e += blockDim.x) {
    int nd[8];
    c.g.corners(e, nd);
    TA u[8][3];
    if (mode == 0) {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) u[a][i] = c.vin[i * NN + nd[a]];
    }
    const int ph = c.phase[e];
    const TA mu = (TA)c.lame[2 * ph + 1];
    TA y[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a) y[a][0] = y[a][1] = y[a][2] = TA(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {  // fully unrolled: the shape-function weights fold to constants
      const TA s = (TA)g01(q & 1), t = (TA)g01((q >> 1) & 1), r = (TA)g01(q >> 2);
      TA dF[9];
      if (mode == 0) {
        TA G[9];
        nat_grad(u, s, t, r, G);
#pragma unroll
        for (int k = 0; k < 9; ++k) dF[k] = ih * G[k];
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) dF[k] = k == cidx ? TA(1) : TA(0);
      }
      TA dP[9];
      if constexpr (LAW == kLawNH) {
        TA qv[12];
        load_qp<12>(c.sc.qpd, c.NE, q, e, qv);
        tangent_action(qv, qv[9], qv[10], mu, dF, dP);
      } else {
        TA qv[16];
        load_qp<16>(c.sc.qpd, c.NE, q, e, qv);
        svk_tangent_action(qv, qv + 9, (TA)c.lame[2 * ph], mu, dF, dP);
      }
      nat_scatter(dP, cw, s, t, r, y);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      if (pinned3(nd[a], n, c.bc)) continue;
#pragma unroll
      for (int i = 0; i < 3; ++i) atomicAdd(&c.vout[i * NN + nd[a]], y[a][i]);
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ multigrid (3D)
// Geometric V(1,1)-cycle used as the PCG preconditioner (same construction as in 2D): Galerkin
// coarse operators stored as element blocks, coarse node 0 without a basis function (every
// level pinned at node 0), damped 3x3 block-Jacobi smoothing (omega = 0.6), coarsest level
// (2^3 or 3^3 nodes) solved through its dense inverse.  The first coarse level is integrated
// directly from the fine Gauss-point data (Fit, hb, gm): its element blocks are
//   K_E(a,b)_ik = sum over the 64 fine Gauss points of E of
//                 w [mu d_ik g_a.g_b + gm v_a,i v_b,k - hb v_b,i v_a,k],  v = Fit g,
// with g the gradients of E's trilinear shape functions — the fine bilinear form evaluated on
// the coarse functions, i.e. P^T K P.  Deeper levels follow from the element blocks with the
// trilinear weights.  All multigrid data live in the block's global scratch; coarse applies
// gather per node (no atomics).
// The smoother must contract in the energy norm for the V-cycle to stay positive definite:
// omega < 2 / lambda_max(D^-1 K).  For Hex8 elasticity lambda_max is about 3.0 (measured on the
// 8^3 two-sphere RVE), so omega = 0.7 (used in 2D, where lambda_max is about 2.3) is too large
// here; 0.6 keeps a margin.

__host__ __device__ constexpr int pair8(int a, int b) {  // a <= b
  return a * 8 - (a * (a - 1)) / 2 + (b - a);
}

// block (a, b) entry (i, k) of element E (any order of a, b: symmetric storage)
template <typename TA>
__device__ __forceinline__ TA mg3_kb(const Mg3Level<TA>& L, int E, int a, int b, int i, int k) {
  return a <= b ? L.kb[(size_t)(pair8(a, b) * 9 + 3 * i + k) * L.NN + E]
                : L.kb[(size_t)(pair8(b, a) * 9 + 3 * k + i) * L.NN + E];
}

__device__ __forceinline__ int node3(int n, int i, int j, int k) { return i + n * (j + n * k); }

// level 1 element blocks, task (E, a): row block a, b >= a, from the fine Gauss-point data
template <typename TA, int LAW>
__device__ __noinline__ void mg3_build_level1(const Ctx3<TA>& c) {
  const Mg3Level<TA> L = c.mg.level(1);
  const int n = c.g.n, nc = L.n;
  const TA ihc = (TA)nc, wq = TA(0.125) / ((TA)n * (TA)n * (TA)n);
  for (int task = threadIdx.x; task < 8 * L.NN; task += blockDim.x) {
    const int E = task >> 3, a = task & 7;
    const int I = E % nc, J = (E / nc) % nc, K = E / (nc * nc);
    const int ax = a & 1, ay = (a >> 1) & 1, az = (a >> 2) & 1;
    TA acc[8][9];
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int q = 0; q < 9; ++q) acc[b][q] = TA(0);
    for (int sub = 0; sub < 8; ++sub) {
      const int sx = sub & 1, sy = (sub >> 1) & 1, sz = sub >> 2;
      const int e = node3(n, 2 * I + sx, 2 * J + sy, 2 * K + sz);
      const TA mu = (TA)c.lame[2 * c.phase[e] + 1];
      const TA lam = (TA)c.lame[2 * c.phase[e]];
#pragma unroll 1
      for (int q = 0; q < 8; ++q) {
        const TA xi = TA(0.5) * ((TA)sx + (TA)g01(q & 1)), et = TA(0.5) * ((TA)sy + (TA)g01((q >> 1) & 1)),
                 ze = TA(0.5) * ((TA)sz + (TA)g01(q >> 2));
        const TA gax = ihc * (ax ? TA(1) : TA(-1)) * phi(ay, et) * phi(az, ze);
        const TA gay = ihc * (ay ? TA(1) : TA(-1)) * phi(ax, xi) * phi(az, ze);
        const TA gaz = ihc * (az ? TA(1) : TA(-1)) * phi(ax, xi) * phi(ay, et);
        // neo-Hookean: K = mu d_ik g_a.g_b + gm v_a,i v_b,k - hb v_b,i v_a,k, v = Fit g
        // St. Venant-Kirchhoff: K = d_ik g_a.S.g_b + lam v_a,i v_b,k + mu ((g_a.g_b) b_ik + v_b,i v_a,k),
        // v = F g, b = F F^T
        TA qv[qp_vals<LAW>()];
        load_qp<qp_vals<LAW>()>(c.sc.qpd, c.NE, q, e, qv);
        TA va[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) va[i] = qv[3 * i] * gax + qv[3 * i + 1] * gay + qv[3 * i + 2] * gaz;
        TA c_vv, c_sw, wm;  // coefficients of v_a,i v_b,k and of v_b,i v_a,k, and of d_ik g_a.g_b
        TA Sa[3] = {TA(0), TA(0), TA(0)}, b6[6];  // SVK: S g_a (weighted) and b = F F^T
        if constexpr (LAW == kLawNH) {
          c_vv = wq * qv[10];
          c_sw = -wq * qv[9];
          wm = wq * mu;
        } else {
          c_vv = wq * lam;
          c_sw = wq * mu;
          wm = TA(0);
          const TA S6[6] = {qv[9], qv[10], qv[11], qv[12], qv[13], qv[14]};
          const TA ga[3] = {gax, gay, gaz};
#pragma unroll
          for (int I = 0; I < 3; ++I) Sa[I] = wq * (sym6(S6, I, 0) * ga[0] + sym6(S6, I, 1) * ga[1] + sym6(S6, I, 2) * ga[2]);
          const int I6[6] = {0, 0, 0, 1, 1, 2}, J6[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
          for (int k = 0; k < 6; ++k)
            b6[k] = wq * mu * (qv[3 * I6[k]] * qv[3 * J6[k]] + qv[3 * I6[k] + 1] * qv[3 * J6[k] + 1] +
                               qv[3 * I6[k] + 2] * qv[3 * J6[k] + 2]);
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          if (b < a) continue;
          const int bx = b & 1, by = (b >> 1) & 1, bz = (b >> 2) & 1;
          const TA gbx = ihc * (bx ? TA(1) : TA(-1)) * phi(by, et) * phi(bz, ze);
          const TA gby = ihc * (by ? TA(1) : TA(-1)) * phi(bx, xi) * phi(bz, ze);
          const TA gbz = ihc * (bz ? TA(1) : TA(-1)) * phi(bx, xi) * phi(by, et);
          TA vb[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) vb[i] = qv[3 * i] * gbx + qv[3 * i + 1] * gby + qv[3 * i + 2] * gbz;
          const TA gab = gax * gbx + gay * gby + gaz * gbz;
          TA dterm = wm * gab;  // the d_ik part
          if constexpr (LAW == kLawSVK) dterm = Sa[0] * gbx + Sa[1] * gby + Sa[2] * gbz;
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              TA val = c_vv * va[i] * vb[k] + c_sw * vb[i] * va[k] + (i == k ? dterm : TA(0));
              if constexpr (LAW == kLawSVK) val += gab * sym6(b6, i, k);
              acc[b][3 * i + k] += val;
            }
        }
      }
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      if (b < a) continue;
#pragma unroll
      for (int q = 0; q < 9; ++q) L.kb[(size_t)(pair8(a, b) * 9 + q) * L.NN + E] = acc[b][q];
    }
  }
}

// trilinear weight of coarse corner a at fine corner c of sub-element sub
__device__ __forceinline__ float mg3_w(int sub, int c, int a) {
  float w = 1.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int p = ((sub >> d) & 1) + ((c >> d) & 1);  // position in halves: 0, 1, 2
    w *= ((a >> d) & 1) ? 0.5f * p : 1.0f - 0.5f * p;
  }
  return w;
}

// level l + 1 element blocks from level l, task (E, a)
template <typename TA>
__device__ __noinline__ void mg3_build_next(const Mg3<TA>& mg, int l) {
  const Mg3Level<TA> F = mg.level(l), C = mg.level(l + 1);
  const int nf = F.n, nc = C.n;
  for (int task = threadIdx.x; task < 8 * C.NN; task += blockDim.x) {
    const int E = task >> 3, a = task & 7;
    const int I = E % nc, J = (E / nc) % nc, K = E / (nc * nc);
    TA acc[8][9];
#pragma unroll
    for (int b = 0; b < 8; ++b)
#pragma unroll
      for (int q = 0; q < 9; ++q) acc[b][q] = TA(0);
    for (int sub = 0; sub < 8; ++sub) {
      const int e = node3(nf, 2 * I + (sub & 1), 2 * J + ((sub >> 1) & 1), 2 * K + (sub >> 2));
      for (int cc = 0; cc < 8; ++cc) {
        const float wca = mg3_w(sub, cc, a);
        if (wca == 0.0f) continue;
        for (int d = 0; d < 8; ++d) {
          TA blk[9];
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) blk[3 * i + k] = mg3_kb<TA>(F, e, cc, d, i, k);
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            if (b < a) continue;
            const float w = wca * mg3_w(sub, d, b);
            if (w == 0.0f) continue;
#pragma unroll
            for (int q = 0; q < 9; ++q) acc[b][q] += (TA)w * blk[q];
          }
        }
      }
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      if (b < a) continue;
#pragma unroll
      for (int q = 0; q < 9; ++q) C.kb[(size_t)(pair8(a, b) * 9 + q) * C.NN + E] = acc[b][q];
    }
  }
}

// inverted nodal diagonal blocks of a smoothing level
template <typename TA>
__device__ __noinline__ void mg3_build_diag(const Mg3<TA>& mg, int l) {
  const Mg3Level<TA> L = mg.level(l);
  const int n = L.n;
  for (int v = threadIdx.x; v < L.NN; v += blockDim.x) {
    const int i = v % n, j = (v / n) % n, k = v / (n * n);
    TA d[6] = {TA(0), TA(0), TA(0), TA(0), TA(0), TA(0)};
    for (int a = 0; a < 8; ++a) {
      const int E = node3(n, (i - (a & 1) + n) % n, (j - ((a >> 1) & 1) + n) % n, (k - (a >> 2) + n) % n);
      d[0] += mg3_kb<TA>(L, E, a, a, 0, 0);
      d[1] += mg3_kb<TA>(L, E, a, a, 0, 1);
      d[2] += mg3_kb<TA>(L, E, a, a, 0, 2);
      d[3] += mg3_kb<TA>(L, E, a, a, 1, 1);
      d[4] += mg3_kb<TA>(L, E, a, a, 1, 2);
      d[5] += mg3_kb<TA>(L, E, a, a, 2, 2);
    }
    const TA c00 = d[3] * d[5] - d[4] * d[4], c01 = d[2] * d[4] - d[1] * d[5], c02 = d[1] * d[4] - d[2] * d[3];
    const TA c11 = d[0] * d[5] - d[2] * d[2], c12 = d[1] * d[2] - d[0] * d[4], c22 = d[0] * d[3] - d[1] * d[1];
    const TA det = d[0] * c00 + d[1] * c01 + d[2] * c02;
    const TA id = pinned3(v, n, L.bc) ? TA(0) : TA(1) / det;
    L.mi[v] = c00 * id;
    L.mi[L.NN + v] = c01 * id;
    L.mi[2 * L.NN + v] = c02 * id;
    L.mi[3 * L.NN + v] = c11 * id;
    L.mi[4 * L.NN + v] = c12 * id;
    L.mi[5 * L.NN + v] = c22 * id;
  }
}

// coarsest: dense pinned matrix (dof = comp * NN + node, one row per thread), then its inverse
// by Gauss-Jordan over the block, one pivot per step, alternating between two buffers
template <typename TA>
__device__ __noinline__ void mg3_build_coarsest(const Mg3<TA>& mg) {
  const Mg3Level<TA> L = mg.level(mg.levels);
  const int n = L.n, NN = L.NN, D = 3 * NN, ld = D + 1;
  TA* A = mg.inverse();
  TA* B = A + (size_t)D * ld;
  for (int row = threadIdx.x; row < D; row += blockDim.x) {
    const int ii = row / NN, v = row % NN, i = v % n, j = (v / n) % n, k = v / (n * n);
    for (int q = 0; q < D; ++q) A[(size_t)row * ld + q] = TA(0);
    for (int a = 0; a < 8; ++a) {
      const int ei = (i - (a & 1) + n) % n, ej = (j - ((a >> 1) & 1) + n) % n, ek = (k - (a >> 2) + n) % n;
      const int E = node3(n, ei, ej, ek);
      for (int b = 0; b < 8; ++b) {
        const int nb = node3(n, (ei + (b & 1)) % n, (ej + ((b >> 1) & 1)) % n, (ek + (b >> 2)) % n);
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) A[(size_t)row * ld + kk * NN + nb] += mg3_kb<TA>(L, E, a, b, ii, kk);
      }
    }
    if (pinned3(v, n, L.bc)) {  // pinned rows: identity; pinned columns of the other rows: zero
      for (int q = 0; q < D; ++q) A[(size_t)row * ld + q] = q == row ? TA(1) : TA(0);
    } else {
      for (int q = 0; q < D; ++q)
        if (pinned3(q % NN, n, L.bc)) A[(size_t)row * ld + q] = TA(0);
    }
  }
  __syncthreads();
  for (int kp = 0; kp < D; ++kp) {  // SPD: no pivoting
    const TA* Ao = (kp & 1) ? B : A;
    TA* An = (kp & 1) ? A : B;
    const TA ip = TA(1) / Ao[(size_t)kp * ld + kp];
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
      const int i = e / D, j = e % D;
      const TA aik = Ao[(size_t)i * ld + kp], akj = Ao[(size_t)kp * ld + j];
      TA v;
      if (i == kp) v = (j == kp) ? ip : akj * ip;
      else v = (j == kp) ? -aik * ip : Ao[(size_t)i * ld + j] - aik * akj * ip;
      An[(size_t)i * ld + j] = v;
    }
    __syncthreads();
  }
  if (D & 1) {  // odd number of steps: the inverse ended in B
    for (int e = threadIdx.x; e < D * D; e += blockDim.x) A[(size_t)(e / D) * ld + e % D] = B[(size_t)(e / D) * ld + e % D];
    __syncthreads();
  }
}

// After tangent3: all coarse levels of the current tangent.
template <typename TA, int LAW>
__device__ void mg3_build(const Ctx3<TA>& c) {
  mg3_build_level1<TA, LAW>(c);
  for (int l = 1; l < c.mg.levels; ++l) {
    __syncthreads();
    mg3_build_next<TA>(c.mg, l);
  }
  __syncthreads();
  for (int l = 1; l < c.mg.levels; ++l) mg3_build_diag<TA>(c.mg, l);
  mg3_build_coarsest<TA>(c.mg);  // ends with a barrier
  __syncthreads();
}

// y = K_l z at node v (gathered from the 8 elements around v; zero at the pinned node)
template <typename TA>
__device__ __forceinline__ void mg3_apply(const Mg3Level<TA>& L, const TA* z, int v, TA (&y)[3]) {
  const int n = L.n, NN = L.NN, i = v % n, j = (v / n) % n, k = v / (n * n);
  y[0] = y[1] = y[2] = TA(0);
  if (pinned3(v, n, L.bc)) return;
  for (int a = 0; a < 8; ++a) {
    const int ei = (i - (a & 1) + n) % n, ej = (j - ((a >> 1) & 1) + n) % n, ek = (k - (a >> 2) + n) % n;
    const int E = node3(n, ei, ej, ek);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int nb = node3(n, (ei + (b & 1)) % n, (ej + ((b >> 1) & 1)) % n, (ek + (b >> 2)) % n);
      const TA z0 = z[nb], z1 = z[NN + nb], z2 = z[2 * NN + nb];
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
        y[ii] += mg3_kb<TA>(L, E, a, b, ii, 0) * z0 + mg3_kb<TA>(L, E, a, b, ii, 1) * z1 +
                 mg3_kb<TA>(L, E, a, b, ii, 2) * z2;
    }
  }
}

template <typename TA>
__device__ __forceinline__ void mg3_smooth(const TA* mi, int NN, int v, const TA (&r)[3], TA om, TA (&z)[3]) {
  const TA m00 = mi[v], m01 = mi[NN + v], m02 = mi[2 * NN + v], m11 = mi[3 * NN + v], m12 = mi[4 * NN + v],
           m22 = mi[5 * NN + v];
  z[0] = om * (m00 * r[0] + m01 * r[1] + m02 * r[2]);
  z[1] = om * (m01 * r[0] + m11 * r[1] + m12 * r[2]);
  z[2] = om * (m02 * r[0] + m12 * r[1] + m22 * r[2]);
}

// Full-weighting restriction to coarse node I of grid nc of the fine residual t(v) = ta[v] -
// tb[v] (tb may be null) on grid 2 nc; zero at the pinned node.  Stores r and, for a smoothing
// level, the pre-smoothed z.
template <typename TA>
__device__ __forceinline__ void mg3_restrict_smooth(const Mg3<TA>& mg, int l, const TA* ta, const TA* tb, int I) {
  const Mg3Level<TA> C = mg.level(l);
  const int nc = C.n, nf = 2 * nc, NNf = nf * nf * nf;
  const int ci = I % nc, cj = (I / nc) % nc, ck = I / (nc * nc);
  TA r[3] = {TA(0), TA(0), TA(0)};
  if (!pinned3(I, nc, mg.bc)) {
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const TA w = TA((dx ? 0.5f : 1.0f) * (dy ? 0.5f : 1.0f) * (dz ? 0.5f : 1.0f));
          const int f = node3(nf, (2 * ci + dx + nf) % nf, (2 * cj + dy + nf) % nf, (2 * ck + dz + nf) % nf);
#pragma unroll
          for (int d = 0; d < 3; ++d) r[d] += w * (tb ? ta[d * NNf + f] - tb[d * NNf + f] : ta[d * NNf + f]);
        }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) C.r[d * C.NN + I] = r[d];
  if (l < mg.levels) {
    TA z[3];
    mg3_smooth<TA>(C.mi, C.NN, I, r, mg.omega, z);
#pragma unroll
    for (int d = 0; d < 3; ++d) C.z[d * C.NN + I] = z[d];
  }
}

// Trilinear prolongation of the coarse vector zc (grid nf/2) to fine node v of grid nf.
template <typename TA>
__device__ __forceinline__ void mg3_prolong(const TA* zc, int nf, int v, TA (&z)[3]) {
  const int nc = nf >> 1, NNc = nc * nc * nc;
  const int i = v % nf, j = (v / nf) % nf, k = v / (nf * nf);
  z[0] = z[1] = z[2] = TA(0);
  for (int p = 0; p < 8; ++p) {
    const int px = p & 1, py = (p >> 1) & 1, pz = p >> 2;
    if ((px && !(i & 1)) || (py && !(j & 1)) || (pz && !(k & 1))) continue;
    const TA w = TA(((i & 1) ? 0.5f : 1.0f) * ((j & 1) ? 0.5f : 1.0f) * ((k & 1) ? 0.5f : 1.0f));
    const int c = node3(nc, ((i >> 1) + px) % nc, ((j >> 1) + py) % nc, ((k >> 1) + pz) % nc);
#pragma unroll
    for (int d = 0; d < 3; ++d) z[d] += w * zc[d * NNc + c];
  }
}

// where the corrected z of level l ends: t of a smoothing level, z of the coarsest
template <typename TA>
__device__ __forceinline__ const TA* mg3_result(const Mg3<TA>& mg, int l) {
  const Mg3Level<TA> v = mg.level(l);
  return l == mg.levels ? v.z : v.t;
}

// Coarse part of the V-cycle (level 1 holds the restricted residual and, for a smoothing level,
// its pre-smoothed z); result in mg3_result(mg, 1).  Two block barriers per level each way.
template <typename TA>
__device__ __noinline__ void mg3_coarse_cycle(const Mg3<TA>& mg) {
  const int tid = threadIdx.x;
  const TA om = mg.omega;
  for (int l = 1; l < mg.levels; ++l) {  // descend
    const Mg3Level<TA> v = mg.level(l);
    for (int x = tid; x < v.NN; x += blockDim.x) {
      TA kz[3];
      mg3_apply<TA>(v, v.z, x, kz);
#pragma unroll
      for (int d = 0; d < 3; ++d) v.t[d * v.NN + x] = v.r[d * v.NN + x] - kz[d];
    }
    __syncthreads();
    const Mg3Level<TA> cn = mg.level(l + 1);
    for (int x = tid; x < cn.NN; x += blockDim.x) mg3_restrict_smooth<TA>(mg, l + 1, v.t, nullptr, x);
    __syncthreads();
  }
  {  // coarsest: z = A^-1 r (rows of the pinned node: identity, z = 0 there)
    const Mg3Level<TA> C = mg.level(mg.levels);
    const int D = 3 * C.NN, ld = D + 1;
    const TA* A = mg.inverse();
    for (int row = tid; row < D; row += blockDim.x) {
      TA zz = TA(0);
      for (int q = 0; q < D; ++q) zz += A[(size_t)row * ld + q] * C.r[q];
      C.z[row] = pinned3(row % C.NN, C.n, mg.bc) ? TA(0) : zz;
    }
    __syncthreads();
  }
  for (int l = mg.levels - 1; l >= 1; --l) {  // ascend
    const Mg3Level<TA> v = mg.level(l);
    const TA* zc = mg3_result<TA>(mg, l + 1);
    for (int x = tid; x < v.NN; x += blockDim.x) {
      TA zp[3];
      mg3_prolong<TA>(zc, v.n, x, zp);
#pragma unroll
      for (int d = 0; d < 3; ++d) v.z[d * v.NN + x] += zp[d];
    }
    __syncthreads();
    for (int x = tid; x < v.NN; x += blockDim.x) {
      TA kz[3], rr[3], dz[3];
      mg3_apply<TA>(v, v.z, x, kz);
#pragma unroll
      for (int d = 0; d < 3; ++d) rr[d] = v.r[d * v.NN + x] - kz[d];
      mg3_smooth<TA>(v.mi, v.NN, x, rr, om, dz);
#pragma unroll
      for (int d = 0; d < 3; ++d) v.t[d * v.NN + x] = v.z[d * v.NN + x] + dz[d];
    }
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ T div3(T a, T b) {
  if constexpr (sizeof(T) == 4) {
    return __fdividef(a, b);
  } else {
    return a / b;
  }
}

// Fine-level part of the V-cycle: vin holds the pre-smoothed omega M^-1 r on entry and the
// preconditioned residual on return (three fine applies per PCG iteration with the caller's).
template <typename TA, int LAW>
__device__ __noinline__ void mg3_vcycle_fine(const Ctx3<TA>& c, const TA* r) {
  const Mg3<TA>& mg = c.mg;
  const int NN = c.g.NN;
  apply3<TA, LAW>(c, 0, 0);  // vout = K vin
  const Mg3Level<TA> L1 = mg.level(1);
  for (int I = threadIdx.x; I < L1.NN; I += blockDim.x) mg3_restrict_smooth<TA>(mg, 1, r, c.vout, I);
  __syncthreads();
  mg3_coarse_cycle<TA>(mg);
  const TA* zc = mg3_result<TA>(mg, 1);
  for (int v = threadIdx.x; v < NN; v += blockDim.x) {
    TA zp[3];
    mg3_prolong<TA>(zc, c.g.n, v, zp);
#pragma unroll
    for (int d = 0; d < 3; ++d) c.vin[d * NN + v] += zp[d];
  }
  __syncthreads();
  apply3<TA, LAW>(c, 0, 0);  // vout = K vin
  for (int v = threadIdx.x; v < NN; v += blockDim.x) {
    TA rr[3], dz[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) rr[d] = r[d * NN + v] - c.vout[d * NN + v];
    mg3_smooth<TA>(c.sc.mi, NN, v, rr, mg.omega, dz);
#pragma unroll
    for (int d = 0; d < 3; ++d) c.vin[d * NN + v] += dz[d];
  }
  __syncthreads();
}

// Chronopoulos-Gear PCG for K x = b; b given in sc.r on entry (overwritten), x in sc.x.
template <typename TA, int LAW>
__device__ int pcg3(const Ctx3<TA>& c, TA rtol, int max_it, bool truncate, int* status, bool warm = false) {
  const int NN = c.g.NN;
  TA* x = c.sc.x;
  TA* r = c.sc.r;
  TA* p = c.sc.p;
  TA* s = c.sc.s;
  const TA* mi = c.sc.mi;
  auto precond_to_vin = [&]() {  // u = M^-1 r -> vin: block-Jacobi, or the multigrid V-cycle
    const TA om = c.mg.levels ? c.mg.omega : TA(1);
    for (int v = threadIdx.x; v < NN; v += blockDim.x) {
      const TA r0 = r[v], r1 = r[NN + v], r2 = r[2 * NN + v];
      const TA m00 = mi[v], m01 = mi[NN + v], m02 = mi[2 * NN + v], m11 = mi[3 * NN + v], m12 = mi[4 * NN + v],
               m22 = mi[5 * NN + v];
      c.vin[v] = om * (m00 * r0 + m01 * r1 + m02 * r2);
      c.vin[NN + v] = om * (m01 * r0 + m11 * r1 + m12 * r2);
      c.vin[2 * NN + v] = om * (m02 * r0 + m12 * r1 + m22 * r2);
    }
    __syncthreads();
    if (c.mg.levels) mg3_vcycle_fine<TA, LAW>(c, r);
  };
  // inner products: per thread and per warp in TA, over the block in FP64 (block_dot2_fp64); the
  // stopping test compares the FP64 sums, the step scalars are formed in TA from them
  auto dots = [&](double& gam, double& del) {
    TA g = TA(0), d = TA(0);
    for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) {
      g += r[v] * c.vin[v];
      d += c.vout[v] * c.vin[v];
    }
    block_dot2_fp64<TA>(g, d, c.red + 2 * 512 - 64, gam, del);
  };
  *status = kStatusOk;
  double gref = -1.0;  // stopping reference b^T M^-1 b of a warm start
  int it = 0;
  if (!warm) {
    for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) x[v] = TA(0);
  } else {
    // x holds the start value x0 (the previous solve's solution): iterate on r = b - K x0 with
    // the stopping reference of b (one more preconditioner application and apply, counted)
    precond_to_vin();
    {
      TA g = TA(0);
      for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) g += r[v] * c.vin[v];
      double unused;
      block_dot2_fp64<TA>(g, TA(0), c.red + 2 * 512 - 64, gref, unused);
    }
    for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) c.vin[v] = x[v];
    __syncthreads();
    apply3<TA, LAW>(c, 0, 0);
    for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) r[v] -= c.vout[v];
    __syncthreads();
    it = 1;
  }
  precond_to_vin();
  apply3<TA, LAW>(c, 0, 0);
  double gd, dd;
  dots(gd, dd);
  TA gamma = (TA)gd, delta = (TA)dd;
  const double gamma0 = gd;
  const double stop = (double)rtol * (double)rtol * (warm ? gref : gamma0);
  // a non-finite or negative preconditioned residual norm r^T M^-1 r (the preconditioner is not
  // positive definite) is a breakdown
  if (!isfinite(gamma0) || gamma0 < 0.0 || (warm && !(gref >= 0.0))) {
    *status = kStatusPcgBreakdown;
    __syncthreads();
    return it;
  }
  if (warm && gamma0 <= stop) {  // the start value already meets the tolerance
    __syncthreads();
    return it;
  }
  if (!(gamma0 > 0.0)) return 0;
  if (!(dd > 0.0)) {
    if (truncate && delta < TA(0)) {
      const TA a0 = div3(gamma, -delta);
      for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) x[v] = a0 * c.vin[v];
      *status = kStatusNegCurv;
    } else {
      *status = kStatusPcgBreakdown;
    }
    __syncthreads();
    return 0;
  }
  TA alpha = div3(gamma, delta), beta = TA(0);
  for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) {
    p[v] = c.vin[v];
    s[v] = c.vout[v];
  }
  for (;;) {
    if (it >= max_it) {
      *status = kStatusPcgCap;
      break;
    }
    for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) {
      x[v] += alpha * p[v];
      r[v] -= alpha * s[v];
    }
    __syncthreads();
    precond_to_vin();
    apply3<TA, LAW>(c, 0, 0);
    double gnd, dnd;
    dots(gnd, dnd);
    const TA gn = (TA)gnd, dn = (TA)dnd;
    ++it;
    if (!(gnd >= 0.0)) {  // preconditioner not positive definite (or non-finite)
      *status = kStatusPcgBreakdown;
      break;
    }
    if (gnd <= stop) break;
    beta = div3(gn, gamma);
    const TA den = dn - beta * div3(gn, alpha);
    if (!(den > TA(0))) {
      *status = (truncate && den < TA(0)) ? kStatusNegCurv : kStatusPcgBreakdown;
      break;
    }
    alpha = div3(gn, den);
    gamma = gn;
    for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) {
      p[v] = c.vin[v] + beta * p[v];
      s[v] = c.vout[v] + beta * s[v];
    }
    __syncthreads();
  }
  __syncthreads();
  return it;
}

template <typename TA, int LAW>
__device__ void solve_item_3d(const Rve2dArgs& a, int qp, unsigned char* smem, unsigned char* gscr) {
  const int rv = a.qp_rve[qp];
  const int n = a.rve_n[rv];
  const int NN = n * n * n;
  Ctx3<TA> c;
  c.g.n = n;
  c.g.NN = NN;
  c.NE = NN;
  c.phase = a.phase + a.rve_phase_off[rv];
  c.vin = reinterpret_cast<TA*>(smem);
  c.vout = c.vin + 3 * NN;
  c.red = reinterpret_cast<double*>(smem + sizeof(TA) * 6 * (size_t)a.nn_max);
  double* lame_s = c.red + 2 * 512;
  double* misc = lame_s + 2 * kMaxPhase;
  c.lame = lame_s;
  c.sc = scratch3_layout<TA>(gscr, NN);
  c.mg.levels = a.mg ? mg3_levels(n) : 0;
  c.mg.n = n;
  c.mg.bc = a.bc;
  c.mg.omega = (TA)a.mg_omega;
  c.bc = a.bc;
  c.mg.base = c.sc.mg;
  if (threadIdx.x < 2 * kMaxPhase) lame_s[threadIdx.x] = a.rve_lame[(size_t)rv * 2 * kMaxPhase + threadIdx.x];
#pragma unroll
  for (int k = 0; k < 9; ++k) c.Fb[k] = a.F[(size_t)qp * 9 + k];
  const double* w_in = a.w_in + a.qp_w_off[qp];
  double* w = a.w_out + a.qp_w_off[qp];
  // the current fluctuation is kept in w_out (FP64, global); node 0 pinned to zero
  for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) w[v] = pinned3(v / 3, n, a.bc) ? 0.0 : w_in[v];
  __syncthreads();

  // Load continuation on failure: a Newton solve that ends in J <= 0, a non-finite residual or a
  // PCG breakdown is restarted from w = 0 and Fbar is reached in retry_stages equal increments
  // of Fbar - I, each increment a Newton solve warm-started from the previous one.
  int status = kStatusNewtonCap, it_total = 0, cg_total = 0, stages = 1, stage = 1;
  double Psum[9];
  for (;;) {
    int it = 0, nhalf = 0;
    double r0 = 0.0, step = 1.0;
    status = kStatusNewtonCap;
    for (;;) {
      double bad = 0.0;
#pragma unroll
      for (int k = 0; k < 9; ++k) Psum[k] = 0.0;
      residual3<TA, LAW>(c, w, Psum, bad);
      __syncthreads();
      double rr = 0.0;
      for (int v = threadIdx.x; v < NN; v += blockDim.x) {
        double R[3];
        gather_R(c, v, R);
        if (pinned3(v, n, a.bc)) R[0] = R[1] = R[2] = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          rr += R[d] * R[d];
          c.sc.r[d * NN + v] = (TA)(-R[d]);  // right-hand side of the Newton correction
        }
      }
      double v2[2] = {rr, bad};
      block_sum_n<double>(v2, 2, c.red);
      const double rn = sqrt(v2[0]);
      if (it == 0) r0 = rn;
      if ((v2[1] > 0.0 || !isfinite(rn)) && it > 0 && nhalf < kMaxStepHalvings) {
        // backtrack: w = w_prev + step x  ->  w_prev + (step/2) x
        ++nhalf;
        step *= 0.5;
        for (int v = threadIdx.x; v < NN; v += blockDim.x) {
          if (pinned3(v, n, a.bc)) continue;
#pragma unroll
          for (int d = 0; d < 3; ++d) w[3 * v + d] -= step * (double)c.sc.x[d * NN + v];
        }
        __syncthreads();
        continue;
      }
      if (v2[1] > 0.0) {
        status = kStatusJNonPos;
        break;
      }
      if (!isfinite(rn)) {
        status = kStatusNonFinite;
        break;
      }
      if (rn <= fmax(a.newton_rtol * r0, a.newton_atol)) {
        status = kStatusOk;
        break;
      }
      if (it >= (stages > 1 ? max(a.max_newton, kRetryNewtonCap) : a.max_newton)) {
        status = kStatusNewtonCap;
        break;
      }
      tangent3<TA, LAW, false>(c, w, nullptr);
      // The coarse levels are built on the first Newton iteration of a solve (or continuation
      // stage) and reused by the later ones, with the current fine operator, smoother and
      // residual.  The V-cycle stays symmetric; it stays positive definite as long as the reused
      // Galerkin operators are positive definite and the damped smoother still contracts at the
      // current tangent, which holds for nearby tangents but is not guaranteed under large
      // stretch and stiffness contrast.  So a PCG that breaks down, hits its cap or sees negative
      // curvature (which an indefinite V-cycle can fake) with reused levels is run again once
      // with levels rebuilt at the current tangent (its right-hand side
      // is kept in the transfer area, unused during Newton).  The tangent transfer keeps them
      // too (rebuilding them only after a breakdown or cap).
      // A V-cycle whose fresh levels still break down (its damped smoother no longer contracts at
      // this tangent) is retried with half the damping, down to omega / 8.
      bool reused = c.mg.levels && it > 0 && a.mg_reuse;
      if (c.mg.levels && !reused) mg3_build<TA, LAW>(c);
      if (c.mg.levels)
        for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) c.sc.L[v] = c.sc.r[v];
      int pst = kStatusOk;
      const TA omega0 = c.mg.omega;
      for (;;) {
        cg_total += pcg3<TA, LAW>(c, (TA)a.cg_rtol, a.max_cg, true, &pst);
        if (reused && (pst == kStatusPcgBreakdown || pst == kStatusPcgCap || pst == kStatusNegCurv)) {
          mg3_build<TA, LAW>(c);
          reused = false;
        } else if (c.mg.levels && (pst == kStatusPcgBreakdown || pst == kStatusPcgCap) &&
                   c.mg.omega > TA(0.2) * omega0) {
          c.mg.omega *= TA(0.5);
        } else {
          break;
        }
        for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) c.sc.r[v] = c.sc.L[v];
        __syncthreads();
        pst = kStatusOk;
      }
      c.mg.omega = omega0;
      if (pst == kStatusPcgBreakdown) {
        status = kStatusPcgBreakdown;
        break;
      }
      step = 1.0;
      nhalf = 0;
      for (int v = threadIdx.x; v < NN; v += blockDim.x) {
        if (pinned3(v, n, a.bc)) continue;
#pragma unroll
        for (int d = 0; d < 3; ++d) w[3 * v + d] += (double)c.sc.x[d * NN + v];
      }
      __syncthreads();
      ++it;
    }
    it_total += it;
    const bool failed = !(status == kStatusOk || status == kStatusNewtonCap);
    if (failed && stages == 1 && a.retry_stages > 1) {
      stages = a.retry_stages;
      stage = 0;
      for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) w[v] = 0.0;
    } else if (failed || stage >= stages) {
      break;
    }
    ++stage;
    const double* Ft = a.F + (size_t)qp * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k)
      c.Fb[k] = stage == stages ? Ft[k] : (k % 4 == 0 ? 1.0 : 0.0) + (Ft[k] - (k % 4 == 0 ? 1.0 : 0.0)) * stage / stages;
    __syncthreads();
  }
  const int it = it_total;

  const bool usable = (status == kStatusOk || status == kStatusNewtonCap);
  double Pv[10];
#pragma unroll
  for (int k = 0; k < 9; ++k) Pv[k] = Psum[k];
  const bool want_W = usable && (a.flags & kFlagEnergy) && a.W != nullptr;
  Pv[9] = want_W ? energy3<TA, LAW>(c, w) : 0.0;
  block_sum_n<double>(Pv, 10, c.red);
  if (threadIdx.x == 0)
    for (int k = 0; k < 10; ++k) misc[k] = Pv[k];

  int cond_total = 0, cond_max = 0;
  const bool want_A = usable && !(a.flags & kFlagNoTangent) && a.A != nullptr;
  if (want_A) {
    double As[45];
#pragma unroll
    for (int k = 0; k < 45; ++k) As[k] = 0.0;
    tangent3<TA, LAW, true>(c, w, As);
    // the coarse levels of this solve's last tangent (when its Newton loop iterated at all) are
    // kept for the transfer as for the later Newton iterations; a transfer PCG that breaks down or
    // hits its cap with them is run again with levels rebuilt at the converged state
    bool reuse_t = c.mg.levels && a.mg_reuse && it > 0;
    if (c.mg.levels && !reuse_t) mg3_build<TA, LAW>(c);
    // <A>: 45 FP64 sums in three reductions of 15
    for (int part = 0; part < 3; ++part) block_sum_n<double>(As + 15 * part, 15, c.red);
    // right-hand sides L_c (c = 3k + L) stored [c][3][NN]
    for (int cc = 0; cc < 9; ++cc) {
      apply3<TA, LAW>(c, 1, cc);
      for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) c.sc.L[(size_t)cc * 3 * NN + v] = c.vout[v];
    }
    __syncthreads();
    // LX[c][c'] = L_c . X_c', X_c' = -K^-1 L_c'  (kept in shared memory: misc[16 + 9c + c'])
    double* LX = misc + 16;
    // kept solutions of this point's previous transfer solves ([9][3][NN], zero at first) start
    // the PCG and receive the new ones
    const bool warm = a.X_in != nullptr;
    const TA* X0 = warm ? reinterpret_cast<const TA*>(a.X_in) + 9 * (size_t)a.qp_w_off[qp] : nullptr;
    TA* X1 = a.X_out ? reinterpret_cast<TA*>(a.X_out) + 9 * (size_t)a.qp_w_off[qp] : nullptr;
    const TA omega0 = c.mg.omega;
    for (int cp = 0; cp < 9; ++cp) {
      int pst = kStatusOk, ci = 0;
      for (;;) {  // as for the Newton corrections: a breakdown is retried with half the damping
        for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) {
          c.sc.r[v] = -c.sc.L[(size_t)cp * 3 * NN + v];
          if (warm) c.sc.x[v] = X0[(size_t)cp * 3 * NN + v];
        }
        __syncthreads();
        ci += pcg3<TA, LAW>(c, (TA)a.cond_rtol, a.max_cond_cg, false, &pst, warm);
        if (reuse_t && (pst == kStatusPcgBreakdown || pst == kStatusPcgCap)) {
          mg3_build<TA, LAW>(c);
          reuse_t = false;
          pst = kStatusOk;
          continue;
        }
        if (!(c.mg.levels && (pst == kStatusPcgBreakdown || pst == kStatusPcgCap) && c.mg.omega > TA(0.2) * omega0))
          break;
        c.mg.omega *= TA(0.5);
        pst = kStatusOk;
      }
      c.mg.omega = omega0;
      if (X1)
        for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) X1[(size_t)cp * 3 * NN + v] = c.sc.x[v];
      cond_total += ci;
      cond_max = ci > cond_max ? ci : cond_max;
      if (pst != kStatusOk && status == kStatusOk) status = pst;
      double col[9];
#pragma unroll
      for (int cc = 0; cc < 9; ++cc) col[cc] = 0.0;
      for (int v = threadIdx.x; v < 3 * NN; v += blockDim.x) {
        const double xv = (double)c.sc.x[v];
#pragma unroll
        for (int cc = 0; cc < 9; ++cc) col[cc] += (double)c.sc.L[(size_t)cc * 3 * NN + v] * xv;
      }
      block_sum_n<double>(col, 9, c.red);
      if (threadIdx.x == 0)
        for (int cc = 0; cc < 9; ++cc) LX[9 * cc + cp] = col[cc];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int idx = 0;
      for (int p = 0; p < 9; ++p)
        for (int q = p; q < 9; ++q) {
          const double v = As[idx++] + 0.5 * (LX[9 * p + q] + LX[9 * q + p]);
          a.A[(size_t)qp * 81 + p * 9 + q] = v;
          a.A[(size_t)qp * 81 + q * 9 + p] = v;
        }
    }
  }
  if (threadIdx.x == 0) {
    a.status[qp] = status;
    if (a.iters) {
      a.iters[(size_t)qp * 4 + 0] = it;
      a.iters[(size_t)qp * 4 + 1] = cg_total;
      a.iters[(size_t)qp * 4 + 2] = cond_total;
      a.iters[(size_t)qp * 4 + 3] = cond_max;
    }
    if (usable) {
      const double wq = 0.125 / ((double)n * n * n);
      for (int k = 0; k < 9; ++k) a.P[(size_t)qp * 9 + k] = misc[k] * wq;
      if (want_W) a.W[qp] = misc[9] * wq;
    }
  }
  __syncthreads();
}

template <typename TA, int LAW>
__global__ void __launch_bounds__(kThreads3D, 1) rve3d_kernel(const Rve2dArgs a) {
  extern __shared__ __align__(16) unsigned char smem3[];
  __shared__ int s_item;
  unsigned char* gscr = reinterpret_cast<unsigned char*>(a.scratch) + (size_t)blockIdx.x * scratch3_bytes<TA>(a.nn_max);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= (a.n_dev ? *a.n_dev : a.n_qp)) break;
    solve_item_3d<TA, LAW>(a, a.order[item], smem3, gscr);
  }
}

}  // namespace

size_t rve3d_smem_bytes(int nn_max, bool mixed) {
  return mixed ? smem3_bytes<float>(nn_max) : smem3_bytes<double>(nn_max);
}

size_t rve3d_scratch_bytes(int nn_max, bool mixed, int n_blocks) {
  return (mixed ? scratch3_bytes<float>(nn_max) : scratch3_bytes<double>(nn_max)) * (size_t)n_blocks;
}

template <typename TA, int LAW>
cudaError_t rve3d_launch_instance(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream) {
  const cudaError_t err =
      cudaFuncSetAttribute(rve3d_kernel<TA, LAW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  rve3d_kernel<TA, LAW><<<n_blocks, kThreads3D, smem, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t rve3d_launch(const Rve2dArgs& a, bool mixed, int n_blocks, cudaStream_t stream) {
  const size_t smem = rve3d_smem_bytes(a.nn_max, mixed);
  if (mixed)
    return a.law == kLawSVK ? rve3d_launch_instance<float, kLawSVK>(a, n_blocks, smem, stream)
                            : rve3d_launch_instance<float, kLawNH>(a, n_blocks, smem, stream);
  return a.law == kLawSVK ? rve3d_launch_instance<double, kLawSVK>(a, n_blocks, smem, stream)
                          : rve3d_launch_instance<double, kLawNH>(a, n_blocks, smem, stream);
}

}  // namespace fehmm
