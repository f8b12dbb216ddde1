// Device code of the batched periodic-RVE Newton solver for 2D plane strain (Q1, 2x2 Gauss), one thread
// block per RVE, persistent over a work queue of macro quadrature points.
//
// Method (paper Sec. 3.2-3.3): for each macro quadrature point the fluctuation w of the
// periodic RVE solves R(w) = 0 with R_a = sum_e sum_qp wt detJ P(Fbar + Grad w) Grad N_a
// (Eq. f_I^int on the micro scale); Newton corrections solve K_T dw = -R (Eq.
// Saddlepoint-problem-Set-of-eqs with the periodic constraints eliminated, ch_3_eq_19-1,
// ch_3_eq_22).  The outputs are Pbar = <P> (Eq. Average-of-P-and-F) and the tangent
// transfer Abar_(c)(c') = <(E_c + Grad X_c) : A : (E_c' + Grad X_c')>, where X_c are the
// periodic responses to the unit macro gradients E_c; this is the paper's
// k^H = omega/|K_delta| T^T K_T T (Eq. k-mac-element-6/7) written per unit gradient.
//
// GB300 layout (one RVE per SM, everything on chip):
//  * 512 threads; thread (col, strip) owns the node pair (col, 2*strip), (col, 2*strip+1)
//    and the two elements whose lower-left corners are those nodes.
//  * w (FP64) lives in shared memory; the residual is evaluated per element in FP64 and the
//    element forces are staged in shared memory, then gathered per node (no atomics).
//  * Mixed precision (TA = float): element tangents are staged in the block's global scratch
//    (L2 resident) and the assembled 9-point block stencil of each owned node (9 x 2x2 floats)
//    is gathered into REGISTERS, where it stays for the whole PCG; the PCG exchanges only the
//    search direction through shared memory, which also holds the multigrid's coarse levels
//    (kept over the Newton iterations of a solve).  FP64 mode (TA = double) keeps the staged element
//    tangents and the stencil in a per-block global scratch area (L2 resident).
//  * Preconditioner: geometric multigrid V(1,1)-cycle with Galerkin coarse levels (grids
//    n = 2^k m, m <= 4; a separate kernel instantiation), else block-Jacobi (inverted 2x2
//    nodal diagonal blocks).
//  * Newton iterations stop on the FP64 2-norm of the residual; PCG inner products are summed
//    per thread and per warp in TA and over the block in FP64 by one warp (at GB300's FP64:FP32
//    rate of about 1:62 an FP64 sum in every thread would cost more than the stencil apply).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "fehmm_device.cuh"
#include "rve_args.h"

namespace fehmm {

namespace {

constexpr int kThreads2D = 512;

__host__ __device__ constexpr int offx(int a) { return (a == 1 || a == 2) ? 1 : 0; }
__host__ __device__ constexpr int offy(int a) { return a >= 2 ? 1 : 0; }
// upper-triangle index of a symmetric 8x8 element matrix
__host__ __device__ constexpr int tri8(int r, int c) {
  return r <= c ? r * 8 - (r * (r - 1)) / 2 + (c - r) : c * 8 - (c * (c - 1)) / 2 + (r - c);
}

__device__ __forceinline__ double gauss01(int g) {
  // Gauss points of [0,1]: 1/2 -+ 1/(2 sqrt 3)
  return g == 0 ? 0.21132486540518711775 : 0.78867513459481288225;
}

// Multigrid level counts and region sizes (the preconditioner itself is further below).  The
// damping omega of its block-Jacobi smoother is a run-time option (default 0.7); the V-cycle
// stays positive definite for omega < 2 / lambda_max(D^-1 K), about 0.86 for Q1 elasticity
// (lambda_max about 2.3, measured).
constexpr int kMgMaxLevels = 4;  // coarse levels: 32 -> 16, 8, 4

// Number of coarse levels (0: no multigrid for this grid).
__host__ __device__ inline int mg_levels(int n) {
  int l = 0, m = n;
  while (m > 4 && (m & 1) == 0) {
    m >>= 1;
    ++l;
  }
  return (m <= 4 && l >= 1 && l <= kMgMaxLevels) ? l : 0;
}

// Element counts (TA) of the fast region (stencils, inverted blocks, vectors, coarsest inverse)
// and of the slow region (coarse element matrices) for grid n.
__host__ __device__ inline long long mg_fast_elems(int n) {
  const int L = mg_levels(n);
  if (!L) return 0;
  long long e = 0;
  for (int l = 1; l < L; ++l) {
    const long long nn = (long long)(n >> l) * (n >> l);
    e += 36 * nn + 4 * nn + 3 * 2 * nn;  // stencil, Minv, r/z/t
  }
  const long long nc = (long long)(n >> L) * (n >> L), D = 2 * nc;
  // fine-level residual, coarsest r/z and its inverse (row stride D + 1; two buffers for the
  // out-of-place Gauss-Jordan steps)
  return 2LL * n * n + e + 2 * 2 * nc + 2 * D * (D + 1);
}
__host__ __device__ inline long long mg_slow_elems(int n) {
  const int L = mg_levels(n);
  long long e = 0;
  for (int l = 1; l <= L; ++l) e += 36LL * (n >> l) * (n >> l);
  return e;
}
// Largest region sizes over the grids a batch with n^2 <= nn_max may hold.
__host__ __device__ inline long long mg_fast_max(int nn_max) {
  long long m = 0;
  for (int n = 2; n * n <= nn_max; n += 2) m = mg_fast_elems(n) > m ? mg_fast_elems(n) : m;
  return m;
}
__host__ __device__ inline long long mg_slow_max(int nn_max) {
  long long m = 0;
  for (int n = 2; n * n <= nn_max; n += 2) m = mg_slow_elems(n) > m ? mg_slow_elems(n) : m;
  return m;
}

template <typename TA>
struct Smem2D {
  double2* w;        // [NN] fluctuation (FP64)
  float2* w32;       // [NN] FP32 copy (mixed mode only)
  vec2_t<TA>* p;     // [2][NN] PCG exchange vector (u = M^-1 r), two alternating buffers
  vec2_t<TA>* x;     // [NN] PCG solution (owned nodes written by their thread)
  unsigned char* stage;  // element forces / element tangents / condensation solutions
  double* red;       // 2 x 512 doubles of reduction buffers
  double* lame;      // [kMaxPhase][2]
  double* misc;      // [16]: Fbar (0..3), homogenised P and W (4..8)
};

template <typename TA>
__host__ __device__ inline size_t smem2d_layout(int NN, Smem2D<TA>* s, unsigned char* base) {
  constexpr bool REG = std::is_same<TA, float>::value;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 15) & ~size_t(15);
    return o;
  };
  size_t o_w = take(sizeof(double2) * NN);
  size_t o_w32 = REG ? take(sizeof(float2) * NN) : 0;
  size_t o_p = take(2 * sizeof(vec2_t<TA>) * NN);
  size_t o_x = take(sizeof(vec2_t<TA>) * NN);
  size_t stage_bytes = sizeof(double) * 8 * NN;                               // element forces
  // condensation solutions X[4][NN] and right-hand sides L[4][NN]; in mixed mode followed by
  // the multigrid fast region of the RVE's grid (largest over the grids up to NN)
  if (sizeof(vec2_t<TA>) * 8 * NN > stage_bytes) stage_bytes = sizeof(vec2_t<TA>) * 8 * NN;
  if (REG)
    for (int m = 2; m * m <= NN; m += 2) {
      const size_t need = sizeof(vec2_t<TA>) * 8 * (size_t)m * m + sizeof(TA) * (size_t)mg_fast_elems(m);
      if (need > stage_bytes) stage_bytes = need;
    }
  size_t o_stage = take(stage_bytes);
  size_t o_red = take(sizeof(double) * 2 * 512);
  size_t o_lame = take(sizeof(double) * 2 * kMaxPhase);
  size_t o_misc = take(sizeof(double) * 16);
  if (s) {
    s->w = reinterpret_cast<double2*>(base + o_w);
    s->w32 = REG ? reinterpret_cast<float2*>(base + o_w32) : nullptr;
    s->p = reinterpret_cast<vec2_t<TA>*>(base + o_p);
    s->x = reinterpret_cast<vec2_t<TA>*>(base + o_x);
    s->stage = base + o_stage;
    s->red = reinterpret_cast<double*>(base + o_red);
    s->lame = reinterpret_cast<double*>(base + o_lame);
    s->misc = reinterpret_cast<double*>(base + o_misc);
  }
  return off;
}

// Per-thread geometry of the owned node pair.
// Pinned nodes of the fluctuation field: node 0 for periodic coupling (translation), every node
// on the lattice lines i = 0 or j = 0 for KUBC (the cell boundary, where the fluctuation vanishes).
__device__ __forceinline__ bool pinned2(int i, int j, int bc) { return bc ? (i == 0 || j == 0) : (i == 0 && j == 0); }

struct Own2D {
  int n, NN, col, strip;
  bool active;
  bool pin[2];   // owned nodes pinned (zero fluctuation)
  int node[2];   // (col, 2*strip), (col, 2*strip+1)
  int rows[4];   // (2s-1, 2s, 2s+1, 2s+2 periodic) * n: row offsets
  int cols[3];   // col-1, col, col+1 (periodic)
};

__device__ __forceinline__ Own2D make_own(int n, int bc) {
  Own2D o;
  o.n = n;
  o.NN = n * n;
  const int t = threadIdx.x;
  o.col = t % n;
  o.strip = t / n;
  o.active = o.strip < n / 2;
  if (!o.active) o.col = o.strip = 0;  // idle threads: every derived index stays inside the RVE
  const int r0 = 2 * o.strip;
  o.node[0] = o.col + n * r0;
  o.node[1] = o.node[0] + n;
  o.pin[0] = pinned2(o.col, r0, bc);
  o.pin[1] = pinned2(o.col, r0 + 1, bc);
  o.rows[0] = ((r0 - 1 + n) % n) * n;
  o.rows[1] = r0 * n;
  o.rows[2] = ((r0 + 1) % n) * n;
  o.rows[3] = ((r0 + 2) % n) * n;
  o.cols[0] = (o.col - 1 + n) % n;
  o.cols[1] = o.col;
  o.cols[2] = (o.col + 1) % n;
  return o;
}

// Stencil storage.  REG (FP32): registers, block nb of owned node s as two row pairs
// K2[s][nb][0] = (K_xx, K_xy), K2[s][nb][1] = (K_yx, K_yy), consumed by paired FP32 FMAs
// (FFMA2).  Otherwise (FP64): global scratch [36][NN] in row-major block order.
template <typename TA, bool REG>
struct Stencil {
  float2 K2[2][9][2];
  TA* g;  // global stencil base (FP64 mode)
  int NN;
  __device__ __forceinline__ TA get(int nb, int c, int node) const { return g[(size_t)(nb * 4 + c) * NN + node]; }
};

// ------------------------------------------------------------------ constitutive laws (2D)
// kLawNH: the paper's neo-Hookean law (factored form in fehmm_device.cuh).  kLawSVK: St.
// Venant-Kirchhoff, S = lam tr(E) I + 2 mu E with E = (F^T F - I)/2 (plane strain: E_33 = 0).
constexpr int kLawNH = 0, kLawSVK = 1;

// First Piola-Kirchhoff stress at one point; returns J = det F.
template <int LAW, typename T>
__device__ __forceinline__ T law2_P(T F00, T F01, T F10, T F11, T lam, T mu, T& P00, T& P01, T& P10, T& P11) {
  if constexpr (LAW == kLawNH) {
    // P = mu F + hb F^-T with F^-T = cof(F) / J, i.e. P = mu F + c cof(F),
    // c = hb / J = lam J / 2 - (lam / 2 + mu) / J (cof(F) = [[F11, -F10], [-F01, F00]])
    const T J = F00 * F11 - F01 * F10;
    const T c = fma(T(0.5) * lam, J, -(T(0.5) * lam + mu) * recip_T(J));
    P00 = fma(mu, F00, c * F11);
    P01 = fma(mu, F01, -c * F10);
    P10 = fma(mu, F10, -c * F01);
    P11 = fma(mu, F11, c * F00);
    return J;
  } else {
    const T c00 = F00 * F00 + F10 * F10, c01 = F00 * F01 + F10 * F11, c11 = F01 * F01 + F11 * F11;
    const T trE = T(0.5) * (c00 + c11) - T(1);
    const T S00 = lam * trE + mu * (c00 - T(1)), S11 = lam * trE + mu * (c11 - T(1)), S01 = mu * c01;
    P00 = F00 * S00 + F01 * S01;
    P01 = F00 * S01 + F01 * S11;
    P10 = F10 * S00 + F11 * S01;
    P11 = F10 * S01 + F11 * S11;
    return F00 * F11 - F01 * F10;
  }
}

// ------------------------------------------------------------------ residual (FP64)
// FP64 first Piola-Kirchhoff stress at one Gauss point (the residual's law; same factored forms
// as law2_P, with the reciprocal above in place of a division).
template <int LAW>
__device__ __forceinline__ double law2_P_fp64(double F00, double F01, double F10, double F11, double hl, double hk,
                                              double lam, double mu, double& P00, double& P01, double& P10,
                                              double& P11) {
  if constexpr (LAW == kLawNH) {
    // c = lam J / 2 - (lam / 2 + mu) / J with hl = lam / 2, hk = lam / 2 + mu
    const double J = fma(F00, F11, -F01 * F10);
    const double c = fma(hl, J, -hk * recip_fp64(J));
    P00 = fma(mu, F00, c * F11);
    P01 = fma(mu, F01, -c * F10);
    P10 = fma(mu, F10, -c * F01);
    P11 = fma(mu, F11, c * F00);
    return J;
  } else {
    return law2_P<LAW, double>(F00, F01, F10, F11, lam, mu, P00, P01, P10, P11);
  }
}

// Element e's nodal forces into stage[k][e] (k = 2*local_node + comp) and this thread's
// contributions to sum wt P and to the J <= 0 flag.
//
// With natural coordinates (s, t) in [0,1]^2 the displacement gradient is bilinear: the first
// column of F depends on t only, the second on s only.  The nodal forces are (wq / h) P G_a with
// wq = h^2 / 4 and G_a the natural-coordinate shape gradients, i.e. sums of P's first column
// weighted by (1 - t) or t and of its second column weighted by (1 - s) or s.  The stress is
// therefore summed over the Gauss points of equal t (first column) or equal s (second column)
// first, and the two Gauss abscissae g0 and g1 = 1 - g0 give both weights.
template <int LAW>
__device__ __forceinline__ void element_residual(int e, int n, const double2* w, const double* Fb,
                                                 double lam, double mu, double* stage_f, double (&Psum)[4],
                                                 double& bad) {
  const int i = e % n, j = e / n, ip = (i + 1) % n, jp = (j + 1) % n;
  const double2 w0 = w[e], w1 = w[ip + n * j], w2 = w[ip + n * jp], w3 = w[i + n * jp];
  const double ih = (double)n;
  const double2 d10 = make_double2(w1.x - w0.x, w1.y - w0.y);
  const double2 d30 = make_double2(w3.x - w0.x, w3.y - w0.y);
  const double2 e1 = make_double2((w2.x - w3.x) - d10.x, (w2.y - w3.y) - d10.y);
  const double2 e2 = make_double2((w2.x - w1.x) - d30.x, (w2.y - w1.y) - d30.y);
  const double hl = 0.5 * lam, hk = hl + mu;
  // F's first column at t = g0, g1; second column at s = g0, g1
  double Fc0[2][2], Fc1[2][2];
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const double t = gauss01(g);
    Fc0[g][0] = fma(ih, fma(t, e1.x, d10.x), Fb[0]);
    Fc0[g][1] = fma(ih, fma(t, e1.y, d10.y), Fb[2]);
    Fc1[g][0] = fma(ih, fma(t, e2.x, d30.x), Fb[1]);
    Fc1[g][1] = fma(ih, fma(t, e2.y, d30.y), Fb[3]);
  }
  double q0x[2], q0y[2], q1x[2], q1y[2];  // P's first column summed over s (per t), second over t (per s)
  int nbad = 0;
#pragma unroll
  for (int gy = 0; gy < 2; ++gy) {
#pragma unroll
    for (int gx = 0; gx < 2; ++gx) {
      double P00, P01, P10, P11;
      const double J = law2_P_fp64<LAW>(Fc0[gy][0], Fc1[gx][0], Fc0[gy][1], Fc1[gx][1], hl, hk, lam, mu, P00, P01,
                                        P10, P11);
      nbad += (J > 0.0) ? 0 : 1;
      if (gx == 0) {
        q0x[gy] = P00;
        q0y[gy] = P10;
      } else {
        q0x[gy] += P00;
        q0y[gy] += P10;
      }
      if (gy == 0) {
        q1x[gx] = P01;
        q1y[gx] = P11;
      } else {
        q1x[gx] += P01;
        q1y[gx] += P11;
      }
    }
  }
  if (nbad) bad += (double)nbad;
  Psum[0] += q0x[0] + q0x[1];
  Psum[1] += q1x[0] + q1x[1];
  Psum[2] += q0y[0] + q0y[1];
  Psum[3] += q1y[0] + q1y[1];
  const double k = 0.25 / ih, kg0 = k * gauss01(0), kg1 = k * gauss01(1);
  // weight 1 - t is g1 at t = g0 and g0 at t = g1
  const double Sa0x = fma(kg1, q0x[0], kg0 * q0x[1]), Sa1x = fma(kg0, q0x[0], kg1 * q0x[1]);
  const double Sa0y = fma(kg1, q0y[0], kg0 * q0y[1]), Sa1y = fma(kg0, q0y[0], kg1 * q0y[1]);
  const double Sb0x = fma(kg1, q1x[0], kg0 * q1x[1]), Sb1x = fma(kg0, q1x[0], kg1 * q1x[1]);
  const double Sb0y = fma(kg1, q1y[0], kg0 * q1y[1]), Sb1y = fma(kg0, q1y[0], kg1 * q1y[1]);
  const int NN = n * n;
  stage_f[0 * NN + e] = -Sa0x - Sb0x;
  stage_f[1 * NN + e] = -Sa0y - Sb0y;
  stage_f[2 * NN + e] = Sa0x - Sb1x;
  stage_f[3 * NN + e] = Sa0y - Sb1y;
  stage_f[4 * NN + e] = Sa1x + Sb1x;
  stage_f[5 * NN + e] = Sa1y + Sb1y;
  stage_f[6 * NN + e] = -Sa1x + Sb0x;
  stage_f[7 * NN + e] = -Sa1y + Sb0y;
}

// Psi summed over the element's Gauss points: neo-Hookean lam/4 (J^2-1) - (lam/2+mu) ln J +
// mu/2 (|F|^2 - 2), or St. Venant-Kirchhoff lam/2 (tr E)^2 + mu E:E.
template <int LAW>
__device__ __forceinline__ double element_energy(int e, int n, const double2* w, const double* Fb, double lam,
                                                 double mu) {
  const int i = e % n, j = e / n, ip = (i + 1) % n, jp = (j + 1) % n;
  const double2 w0 = w[e], w1 = w[ip + n * j], w2 = w[ip + n * jp], w3 = w[i + n * jp];
  const double ih = (double)n;
  double acc = 0.0;
#pragma unroll
  for (int gy = 0; gy < 2; ++gy) {
    const double t = gauss01(gy);
#pragma unroll
    for (int gx = 0; gx < 2; ++gx) {
      const double s = gauss01(gx);
      const double F00 = Fb[0] + ih * ((1 - t) * (w1.x - w0.x) + t * (w2.x - w3.x));
      const double F10 = Fb[2] + ih * ((1 - t) * (w1.y - w0.y) + t * (w2.y - w3.y));
      const double F01 = Fb[1] + ih * ((1 - s) * (w3.x - w0.x) + s * (w2.x - w1.x));
      const double F11 = Fb[3] + ih * ((1 - s) * (w3.y - w0.y) + s * (w2.y - w1.y));
      if constexpr (LAW == kLawNH) {
        const double J = F00 * F11 - F01 * F10;
        const double trC = F00 * F00 + F01 * F01 + F10 * F10 + F11 * F11;
        acc += 0.25 * lam * (J * J - 1.0) - (0.5 * lam + mu) * log(J) + 0.5 * mu * (trC - 2.0);
      } else {
        const double E00 = 0.5 * (F00 * F00 + F10 * F10 - 1.0), E11 = 0.5 * (F01 * F01 + F11 * F11 - 1.0);
        const double E01 = 0.5 * (F00 * F01 + F10 * F11), trE = E00 + E11;
        acc += 0.5 * lam * trE * trE + mu * (E00 * E00 + E11 * E11 + 2.0 * E01 * E01);
      }
    }
  }
  return acc;
}

// ------------------------------------------------------------------ tangent (TA)
// Element tangent Ke (36 upper-triangle entries) into stage[tri][slot]:
//   K_(a,i)(b,k) = sum_qp wq g_a,J A_iJkL g_b,L.
// Neo-Hookean: mu d_ik g_a.g_b + gm v_a,i v_b,k - hb v_b,i v_a,k with v = F^-T g.
// St. Venant-Kirchhoff (A = d_ik S_JL + F_iI F_kK CC_IJKL, CC = lam 1(x)1 + 2 mu I^sym):
//   d_ik g_a.S.g_b + lam v_a,i v_b,k + mu [(g_a.g_b) (F F^T)_ik + v_b,i v_a,k] with v = F g.
template <typename TA, int LAW>
__device__ __forceinline__ void element_tangent(int e, int n, const vec2_t<TA>* w, const TA* Fb, TA lam, TA mu,
                                                TA* stage_k, int slot, int NN) {
  const int i = e % n, j = e / n, ip = (i + 1) % n, jp = (j + 1) % n;
  const vec2_t<TA> w0 = w[e], w1 = w[ip + n * j], w2 = w[ip + n * jp], w3 = w[i + n * jp];
  const TA ih = (TA)n;
  const TA d10x = w1.x - w0.x, d10y = w1.y - w0.y, d30x = w3.x - w0.x, d30y = w3.y - w0.y;
  const TA e1x = (w2.x - w3.x) - d10x, e1y = (w2.y - w3.y) - d10y;
  const TA e2x = (w2.x - w1.x) - d30x, e2y = (w2.y - w1.y) - d30y;
  TA Ke[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) Ke[k] = TA(0);
  const TA wq = TA(0.25) / (ih * ih);
#pragma unroll
  for (int gy = 0; gy < 2; ++gy) {
    const TA t = (TA)gauss01(gy);
#pragma unroll
    for (int gx = 0; gx < 2; ++gx) {
      const TA s = (TA)gauss01(gx);
      const TA F00 = Fb[0] + ih * (d10x + t * e1x);
      const TA F10 = Fb[2] + ih * (d10y + t * e1y);
      const TA F01 = Fb[1] + ih * (d30x + s * e2x);
      const TA F11 = Fb[3] + ih * (d30y + s * e2y);
      // physical shape gradients g_a
      TA gx_[4] = {-(1 - t) * ih, (1 - t) * ih, t * ih, -t * ih};
      TA gy_[4] = {-(1 - s) * ih, -s * ih, s * ih, (1 - s) * ih};
      TA vx[4], vy[4];
      if constexpr (LAW == kLawNH) {
        const NH2<TA> q = nh2_eval(F00, F01, F10, F11, lam, mu);
#pragma unroll
        for (int a = 0; a < 4; ++a) {  // v_a = Fit g_a
          vx[a] = q.f00 * gx_[a] + q.f01 * gy_[a];
          vy[a] = q.f10 * gx_[a] + q.f11 * gy_[a];
        }
        const TA cm = wq * mu, cg = wq * q.gm, ch = wq * q.hb;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
          for (int c = r; c < 8; ++c) {
            const int a = r >> 1, ii = r & 1, b = c >> 1, kk = c & 1;
            const TA va_i = ii ? vy[a] : vx[a], va_k = kk ? vy[a] : vx[a];
            const TA vb_i = ii ? vy[b] : vx[b], vb_k = kk ? vy[b] : vx[b];
            TA val = cg * va_i * vb_k - ch * vb_i * va_k;
            if (ii == kk) val += cm * (gx_[a] * gx_[b] + gy_[a] * gy_[b]);
            Ke[tri8(r, c)] += val;
          }
        }
      } else {
#pragma unroll
        for (int a = 0; a < 4; ++a) {  // v_a = F g_a
          vx[a] = F00 * gx_[a] + F01 * gy_[a];
          vy[a] = F10 * gx_[a] + F11 * gy_[a];
        }
        const TA c00 = F00 * F00 + F10 * F10, c01 = F00 * F01 + F10 * F11, c11 = F01 * F01 + F11 * F11;
        const TA trE = TA(0.5) * (c00 + c11) - TA(1);
        const TA S00 = wq * (lam * trE + mu * (c00 - TA(1))), S11 = wq * (lam * trE + mu * (c11 - TA(1)));
        const TA S01 = wq * mu * c01;
        const TA b00 = F00 * F00 + F01 * F01, b01 = F00 * F10 + F01 * F11, b11 = F10 * F10 + F11 * F11;
        const TA cl = wq * lam, cm = wq * mu;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
#pragma unroll
          for (int c = r; c < 8; ++c) {
            const int a = r >> 1, ii = r & 1, b = c >> 1, kk = c & 1;
            const TA va_i = ii ? vy[a] : vx[a], va_k = kk ? vy[a] : vx[a];
            const TA vb_i = ii ? vy[b] : vx[b], vb_k = kk ? vy[b] : vx[b];
            const TA gg = gx_[a] * gx_[b] + gy_[a] * gy_[b];
            const TA bik = (ii == kk) ? (ii ? b11 : b00) : b01;
            TA val = cl * va_i * vb_k + cm * (gg * bik + vb_i * va_k);
            if (ii == kk)
              val += gx_[a] * (S00 * gx_[b] + S01 * gy_[b]) + gy_[a] * (S01 * gx_[b] + S11 * gy_[b]);
            Ke[tri8(r, c)] += val;
          }
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 36; ++k) stage_k[(size_t)k * NN + slot] = Ke[k];
}

// Gather the 9-point stencil row of node (i,j) from the staged element tangents of the
// four elements around it; optionally also L = dR/dFbar (rows of K times the affine field).
template <typename TA>
__device__ __forceinline__ void gather_stencil(int node, int n, const TA* stage_k, TA (&K)[9][4], bool withL,
                                               TA (&L)[2][4]) {
  const int NN = n * n, i = node % n, j = node / n;
  const TA h = TA(1) / (TA)n;
#pragma unroll
  for (int nb = 0; nb < 9; ++nb)
#pragma unroll
    for (int c = 0; c < 4; ++c) K[nb][c] = TA(0);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) L[a][c] = TA(0);
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int ei = (i - offx(l) + n) % n, ej = (j - offy(l) + n) % n;
    const int slot = ei + n * ej;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int nb = (offy(m) - offy(l) + 1) * 3 + (offx(m) - offx(l) + 1);
#pragma unroll
      for (int ii = 0; ii < 2; ++ii)
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const TA v = stage_k[(size_t)tri8(2 * l + ii, 2 * m + kk) * NN + slot];
          K[nb][2 * ii + kk] += v;
          if (withL) {
            if (offx(m)) L[ii][2 * kk + 0] += v * h;
            if (offy(m)) L[ii][2 * kk + 1] += v * h;
          }
        }
    }
  }
}

// y = K p for the owned node pair; p of neighbours from shared memory.  The four
// neighbour rows (2s-1 .. 2s+2) are streamed one at a time: row r feeds the lower node
// (row offset r-1) and the upper node (row offset r-2), so only one row is live.
template <typename TA, bool REG>
__device__ __forceinline__ void apply_pair(const Stencil<TA, REG>& S, const Own2D& o, const vec2_t<TA>* ps,
                                           const TA (&pown)[4], TA (&y)[4]) {
  if constexpr (REG) {
    // acc[s][i] accumulates (K_i0 p_x, K_i1 p_y) pairs; y_i = acc.x + acc.y at the end
    float2 acc[2][2] = {{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float2 P[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (c == 1 && r == 1) {
          P[c] = make_float2(pown[0], pown[1]);
        } else if (c == 1 && r == 2) {
          P[c] = make_float2(pown[2], pown[3]);
        } else {
          P[c] = ps[o.rows[r] + o.cols[c]];
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (r <= 2) {
          const int nb = r * 3 + c;
          acc[0][0] = __ffma2_rn(S.K2[0][nb][0], P[c], acc[0][0]);
          acc[0][1] = __ffma2_rn(S.K2[0][nb][1], P[c], acc[0][1]);
        }
        if (r >= 1) {
          const int nb = (r - 1) * 3 + c;
          acc[1][0] = __ffma2_rn(S.K2[1][nb][0], P[c], acc[1][0]);
          acc[1][1] = __ffma2_rn(S.K2[1][nb][1], P[c], acc[1][1]);
        }
      }
    }
    y[0] = acc[0][0].x + acc[0][0].y;
    y[1] = acc[0][1].x + acc[0][1].y;
    y[2] = acc[1][0].x + acc[1][0].y;
    y[3] = acc[1][1].x + acc[1][1].y;
  } else {
    TA y0x = TA(0), y0y = TA(0), y1x = TA(0), y1y = TA(0);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      vec2_t<TA> P[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (c == 1 && r == 1) {
          P[c] = mk2<TA>(pown[0], pown[1]);
        } else if (c == 1 && r == 2) {
          P[c] = mk2<TA>(pown[2], pown[3]);
        } else {
          P[c] = ps[o.rows[r] + o.cols[c]];
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (r <= 2) {
          const int nb = r * 3 + c;
          y0x += S.get(nb, 0, o.node[0]) * P[c].x + S.get(nb, 1, o.node[0]) * P[c].y;
          y0y += S.get(nb, 2, o.node[0]) * P[c].x + S.get(nb, 3, o.node[0]) * P[c].y;
        }
        if (r >= 1) {
          const int nb = (r - 1) * 3 + c;
          y1x += S.get(nb, 0, o.node[1]) * P[c].x + S.get(nb, 1, o.node[1]) * P[c].y;
          y1y += S.get(nb, 2, o.node[1]) * P[c].x + S.get(nb, 3, o.node[1]) * P[c].y;
        }
      }
    }
    y[0] = y0x;
    y[1] = y0y;
    y[2] = y1x;
    y[3] = y1y;
  }
}

// Quotient for the CG step scalars: fast reciprocal-based division in FP32 (a few ulp,
// irrelevant for the step lengths), IEEE division in FP64 mode.
template <typename T>
__device__ __forceinline__ T cg_div(T a, T b) {
  if constexpr (sizeof(T) == 4) {
    return __fdividef(a, b);
  } else {
    return a / b;
  }
}

template <typename TA>
__device__ __forceinline__ void invert_block(const TA (&Kself)[4], bool pinned, TA (&Mi)[4]) {
  const TA det = Kself[0] * Kself[3] - Kself[1] * Kself[2];
  const TA id = pinned ? TA(0) : TA(1) / det;
  Mi[0] = Kself[3] * id;
  Mi[1] = -Kself[1] * id;
  Mi[2] = -Kself[2] * id;
  Mi[3] = Kself[0] * id;
}

// ------------------------------------------------------------------ multigrid preconditioner
// Geometric V(1,1)-cycle over the periodic grid hierarchy n, n/2, ..., n_c (n_c <= 4), used as
// the PCG preconditioner in place of block-Jacobi where n = 2^k m with m <= 4.
//  * Galerkin coarse operators, built element by element: K_E = sum over the four fine elements
//    e of the coarse element E of W_e^T K_e W_e, W_e the bilinear weights of E's corners at e's
//    corners.  Bilinear prolongation P restricted to E depends only on E's corners, so the
//    assembled K_E equal P^T K P exactly, and they are again element matrices, which gives the
//    next level the same way.
//  * The fine node 0 is pinned; the coarse node 0 (the same point) carries no basis function,
//    so every level is pinned at node 0 and P^T K P stays the exact Galerkin operator.
//  * Smoother: damped block-Jacobi (omega = 0.7) with the inverted nodal 2x2 blocks, one sweep
//    before and one after the coarse correction (symmetric, so the V-cycle is an SPD
//    preconditioner for CG).  Coarsest level (at most 16 nodes, 32 dofs): exact, through its
//    dense inverse, computed by Gauss-Jordan elimination in one warp.
//  * Fine level: the stencil of the PCG.  Coarse levels: stencil, inverted blocks and vectors
//    in the fast region (shared memory in mixed mode, block scratch in FP64 mode); coarse
//    element matrices (needed only while building) in the block's global scratch.
template <typename TA>
struct MgLevel {
  int n, NN, bc;
  TA* st;          // [36][NN]
  TA* mi;          // [4][NN]
  vec2_t<TA>* r;   // [NN]
  vec2_t<TA>* z;   // [NN]
  vec2_t<TA>* t;   // [NN]
  TA* ke;          // [36][NN] coarse element matrices (slow region)
};

template <typename TA>
struct MgCtx {
  int levels;  // coarse levels, 0 = off
  int n;       // fine grid
  int bc;      // pinned nodes of every level: as on the fine grid (pinned2)
  TA omega;    // smoother damping
  TA* fast;
  TA* slow;
  // fine-level residual (restriction input), at the start of the fast region
  __device__ __forceinline__ vec2_t<TA>* fine_t() const { return reinterpret_cast<vec2_t<TA>*>(fast); }
  // view of coarse level l (1..levels); the coarsest has no st/mi/t, its inverse follows r, z
  __device__ __forceinline__ MgLevel<TA> level(int l) const {
    MgLevel<TA> v;
    TA* f = fast + 2 * n * n;
    TA* k = slow;
    for (int q = 1; q < l; ++q) {
      const int nn = (n >> q) * (n >> q);
      f += 46 * nn;
      k += 36 * nn;
    }
    v.n = n >> l;
    v.NN = v.n * v.n;
    v.bc = bc;
    v.ke = k;
    if (l < levels) {
      v.st = f;
      v.mi = f + 36 * v.NN;
      v.r = reinterpret_cast<vec2_t<TA>*>(f + 40 * v.NN);
      v.z = v.r + v.NN;
      v.t = v.z + v.NN;
    } else {
      v.st = v.mi = nullptr;
      v.r = reinterpret_cast<vec2_t<TA>*>(f);
      v.z = v.r + v.NN;
      v.t = nullptr;
    }
    return v;
  }
  __device__ __forceinline__ TA* coarsest_inverse() const {
    const MgLevel<TA> v = level(levels);
    return reinterpret_cast<TA*>(v.z + v.NN);
  }
};

// Galerkin element matrix of coarse element E (grid nc = nf/2) from the four fine element
// matrices in kf ([36][nf*nf], upper triangle of each 8x8): K_E = sum over the fine elements e of
// E of W_e^T K_e W_e, W_e the bilinear weights of E's corners at e's corners.  Per fine element,
// one column of K_e W_e at a time (8 values) and its product with W_e^T into the upper triangle
// (400 FMA per fine element; the runtime loop over the four fine elements keeps the code small).
template <typename TA>
__device__ __forceinline__ void mg_coarse_element(const TA* kf, int nf, int E, TA* kc, int nnc) {
  const int nc = nf >> 1, I = E % nc, J = E / nc, NNf = nf * nf;
  TA acc[36];
#pragma unroll
  for (int q = 0; q < 36; ++q) acc[q] = TA(0);
#pragma unroll 1
  for (int ab = 0; ab < 4; ++ab) {
    const int a = ab & 1, b = ab >> 1;
    const int e = (2 * I + a) + nf * (2 * J + b);
    TA k8[36];
#pragma unroll
    for (int q = 0; q < 36; ++q) k8[q] = kf[(size_t)q * NNf + e];
    // W[k][c]: weight of coarse corner c at fine corner k (positions in halves of E)
    TA W[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const TA x2 = (TA)(a + offx(k)), y2 = (TA)(b + offy(k));
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const TA fx = offx(c) ? TA(0.5) * x2 : TA(1) - TA(0.5) * x2;
        const TA fy = offy(c) ? TA(0.5) * y2 : TA(1) - TA(0.5) * y2;
        W[k][c] = fx * fy;
      }
    }
#pragma unroll
    for (int col = 0; col < 8; ++col) {
      TA t[8];  // column col of K_e W_e
#pragma unroll
      for (int row = 0; row < 8; ++row) {
        TA v = TA(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) v += k8[tri8(row, 2 * m + (col & 1))] * W[m][col >> 1];
        t[row] = v;
      }
#pragma unroll
      for (int r = 0; r <= col; ++r) {
        TA v = TA(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) v += W[k][r >> 1] * t[2 * k + (r & 1)];
        acc[tri8(r, col)] += v;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 36; ++q) kc[(size_t)q * nnc + E] = acc[q];
}

// Periodic neighbours without integer division.
__device__ __forceinline__ int wrap_dec(int i, int n) { return i == 0 ? n - 1 : i - 1; }
__device__ __forceinline__ int wrap_inc(int i, int n) { return i == n - 1 ? 0 : i + 1; }

// y = K_l z at node v = (i, j) of a coarse level (zero at the pinned node).
template <typename TA>
__device__ __forceinline__ vec2_t<TA> mg_apply(const MgLevel<TA>& L, const vec2_t<TA>* z, int i, int j) {
  const int n = L.n, v = i + n * j;
  const int cols[3] = {wrap_dec(i, n), i, wrap_inc(i, n)};
  const int rows[3] = {wrap_dec(j, n) * n, j * n, wrap_inc(j, n) * n};
  TA yx = TA(0), yy = TA(0);
#pragma unroll
  for (int nb = 0; nb < 9; ++nb) {
    const vec2_t<TA> zn = z[rows[nb / 3] + cols[nb % 3]];
    yx += L.st[(size_t)(nb * 4 + 0) * L.NN + v] * zn.x + L.st[(size_t)(nb * 4 + 1) * L.NN + v] * zn.y;
    yy += L.st[(size_t)(nb * 4 + 2) * L.NN + v] * zn.x + L.st[(size_t)(nb * 4 + 3) * L.NN + v] * zn.y;
  }
  return pinned2(i, j, L.bc) ? mk2<TA>(TA(0), TA(0)) : mk2<TA>(yx, yy);
}

template <typename TA>
__device__ __forceinline__ vec2_t<TA> mg_smooth(const TA* mi, int NN, int v, vec2_t<TA> r, TA omega) {
  const TA m0 = mi[v], m1 = mi[NN + v], m2 = mi[2 * NN + v], m3 = mi[3 * NN + v];
  return mk2<TA>(omega * (m0 * r.x + m1 * r.y), omega * (m2 * r.x + m3 * r.y));
}

// Full-weighting restriction (the transpose of bilinear prolongation) of the fine vector t
// (grid nf) to coarse node (I, J); zero at the pinned node.
template <typename TA>
__device__ __forceinline__ vec2_t<TA> mg_restrict(const vec2_t<TA>* t, int nf, int I, int J, int bc) {
  const int ix = 2 * I, jy = 2 * J;
  const int cols[3] = {wrap_dec(ix, nf), ix, ix + 1};
  const int rows[3] = {wrap_dec(jy, nf) * nf, jy * nf, (jy + 1) * nf};
  TA sx = TA(0), sy = TA(0);
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
      const TA wgt = TA((dx == 1 ? 1.0f : 0.5f) * (dy == 1 ? 1.0f : 0.5f));
      const vec2_t<TA> v = t[rows[dy] + cols[dx]];
      sx += wgt * v.x;
      sy += wgt * v.y;
    }
  return pinned2(I, J, bc) ? mk2<TA>(TA(0), TA(0)) : mk2<TA>(sx, sy);
}

// Bilinear prolongation of the coarse vector zc (grid nf/2) to fine node (i, j) of grid nf.
template <typename TA>
__device__ __forceinline__ vec2_t<TA> mg_prolong(const vec2_t<TA>* zc, int nf, int i, int j) {
  const int nc = nf >> 1;
  const int i0 = i >> 1, j0 = j >> 1, i1 = wrap_inc(i0, nc), j1 = wrap_inc(j0, nc);
  const vec2_t<TA> a = zc[i0 + nc * j0];
  if (!(i & 1) && !(j & 1)) return a;
  if (!(i & 1)) {  // between two coarse rows
    const vec2_t<TA> c = zc[i0 + nc * j1];
    return mk2<TA>(TA(0.5f) * (a.x + c.x), TA(0.5f) * (a.y + c.y));
  }
  const vec2_t<TA> b = zc[i1 + nc * j0];
  if (!(j & 1)) return mk2<TA>(TA(0.5f) * (a.x + b.x), TA(0.5f) * (a.y + b.y));
  const vec2_t<TA> c = zc[i0 + nc * j1], d = zc[i1 + nc * j1];
  return mk2<TA>(TA(0.25f) * ((a.x + b.x) + (c.x + d.x)), TA(0.25f) * ((a.y + b.y) + (c.y + d.y)));
}

// Build the coarse levels below the fine element matrices kf0 (grid n, [36][n*n]).  Part 1 (the
// Galerkin element matrices of every coarse level, slow region) runs while kf0 is intact and
// before the fine stencil is gathered into registers, so its many live values do not compete
// with the stencil; part 2 (coarse stencils, inverted blocks and the coarsest inverse, fast
// region) runs after the fine gather and keeps only a few values live at a time.
template <typename TA>
__device__ __forceinline__ void mg_build_part1(const MgCtx<TA>& mg, const TA* kf0) {
  const MgLevel<TA> L1 = mg.level(1);
  for (int E = threadIdx.x; E < L1.NN; E += blockDim.x) mg_coarse_element<TA>(kf0, mg.n, E, L1.ke, L1.NN);
  for (int l = 1; l < mg.levels; ++l) {
    __syncthreads();
    const MgLevel<TA> f = mg.level(l), c = mg.level(l + 1);
    for (int E = threadIdx.x; E < c.NN; E += blockDim.x) mg_coarse_element<TA>(f.ke, f.n, E, c.ke, c.NN);
  }
}

// Stencil block nb of node (i, j) summed from the element matrices ke ([36][n*n]) as it is
// needed: one 2x2 block live at a time.
template <typename TA>
__device__ __forceinline__ void mg_stencil_block(const TA* ke, int n, int i, int j, int nb, TA (&blk)[4]) {
  const int NN = n * n;
#pragma unroll
  for (int q = 0; q < 4; ++q) blk[q] = TA(0);
#pragma unroll
  for (int l = 0; l < 4; ++l)
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if ((offy(m) - offy(l) + 1) * 3 + (offx(m) - offx(l) + 1) != nb) continue;
      const int slot = (i - offx(l) + n) % n + n * ((j - offy(l) + n) % n);
#pragma unroll
      for (int ii = 0; ii < 2; ++ii)
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) blk[2 * ii + kk] += ke[(size_t)tri8(2 * l + ii, 2 * m + kk) * NN + slot];
    }
}

template <typename TA>
__device__ __forceinline__ void mg_build_part2(const MgCtx<TA>& mg) {
  const int tid = threadIdx.x;
  __syncthreads();  // part 1's element matrices complete
  for (int l = 1; l < mg.levels; ++l) {  // stencils and inverted blocks of the smoothing levels
    const MgLevel<TA> v = mg.level(l);
    for (int node = tid; node < v.NN; node += blockDim.x) {
      const int i = node % v.n, j = node / v.n;
#pragma unroll 1
      for (int nb = 0; nb < 9; ++nb) {
        TA blk[4];
        mg_stencil_block<TA>(v.ke, v.n, i, j, nb, blk);
#pragma unroll
        for (int q = 0; q < 4; ++q) v.st[(size_t)(nb * 4 + q) * v.NN + node] = blk[q];
        if (nb == 4) {
          TA m[4];
          invert_block<TA>(blk, pinned2(i, j, v.bc), m);
#pragma unroll
          for (int q = 0; q < 4; ++q) v.mi[(size_t)q * v.NN + node] = m[q];
        }
      }
    }
  }
  // coarsest: dense pinned matrix (one row per thread), then its inverse by Gauss-Jordan
  // elimination, one pivot per step over the whole block, alternating between two buffers
  const MgLevel<TA> c = mg.level(mg.levels);
  const int D = 2 * c.NN, ld = D + 1;
  TA* A = mg.coarsest_inverse();
  TA* B = A + (size_t)D * ld;
  if (tid < D) {
    const int node = tid >> 1, ii = tid & 1, ni = node % c.n, nj = node / c.n;
    for (int q = 0; q < D; ++q) A[(size_t)tid * ld + q] = TA(0);
#pragma unroll
    for (int l = 0; l < 4; ++l) {  // the four elements with this node as corner l
      const int ei = (ni - offx(l) + c.n) % c.n, ej = (nj - offy(l) + c.n) % c.n, slot = ei + c.n * ej;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int nm = (ei + offx(m)) % c.n + c.n * ((ej + offy(m)) % c.n);
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
          A[(size_t)tid * ld + 2 * nm + kk] += c.ke[(size_t)tri8(2 * l + ii, 2 * m + kk) * c.NN + slot];
      }
    }
    // pinned rows: identity; pinned columns of the other rows: zero
    if (pinned2(ni, nj, c.bc)) {
      for (int q = 0; q < D; ++q) A[(size_t)tid * ld + q] = q == tid ? TA(1) : TA(0);
    } else {
      for (int q = 0; q < D; q += 2)
        if (pinned2((q >> 1) % c.n, (q >> 1) / c.n, c.bc)) A[(size_t)tid * ld + q] = A[(size_t)tid * ld + q + 1] = TA(0);
    }
  }
  __syncthreads();
  // entries (i, j) of this thread: e and e + blockDim.x (D*D <= 1024 = 2 x 512)
  const int e0 = tid, e1 = tid + blockDim.x;
  const int i0 = e0 / D, j0 = e0 % D, i1 = e1 / D, j1 = e1 % D;
  for (int k = 0; k < D; ++k) {  // SPD: no pivoting; D is even, so the result ends in A
    const TA* Ao = (k & 1) ? B : A;
    TA* An = (k & 1) ? A : B;
    const TA ip = TA(1) / Ao[(size_t)k * ld + k];
    auto step = [&](int i, int j) {
      const TA aik = Ao[(size_t)i * ld + k], akj = Ao[(size_t)k * ld + j];
      TA v;
      if (i == k) v = (j == k) ? ip : akj * ip;
      else v = (j == k) ? -aik * ip : Ao[(size_t)i * ld + j] - aik * akj * ip;
      An[(size_t)i * ld + j] = v;
    };
    if (e0 < D * D) step(i0, j0);
    if (e1 < D * D) step(i1, j1);
    __syncthreads();
  }
}

// Restricted residual of coarse node t of level l (from the residual t_f of the finer grid nf),
// stored with its pre-smoothed correction when level l is a smoothing level: the smoothing is
// local to the node, so it needs no barrier of its own.
template <typename TA>
__device__ __forceinline__ void mg_restrict_smooth(const MgCtx<TA>& mg, int l, const vec2_t<TA>* tf, int nf, int t) {
  const MgLevel<TA> c = mg.level(l);
  const vec2_t<TA> r = mg_restrict<TA>(tf, nf, t % c.n, t / c.n, mg.bc);
  c.r[t] = r;
  if (l < mg.levels) c.z[t] = mg_smooth<TA>(c.mi, c.NN, t, r, mg.omega);
}

// Where the corrected z of level l ends: the t vector of a smoothing level (free on the way
// up), the z vector of the coarsest.
template <typename TA>
__device__ __forceinline__ const vec2_t<TA>* mg_result(const MgCtx<TA>& mg, int l) {
  const MgLevel<TA> v = mg.level(l);
  return l == mg.levels ? v.z : v.t;
}

// Coarse part of the V-cycle.  On entry level(1) holds the restricted residual (and, for a
// smoothing level, its pre-smoothed z); on return mg_result(mg, 1) holds the coarse
// correction.  Two block barriers per level each way.  All threads call it; ends with a barrier.
// (Running the small levels in one warp with warp barriers was measured slower: the other warps
// idle while one warp walks the level's nodes serially.)
template <typename TA>
__device__ void mg_coarse_cycle(const MgCtx<TA>& mg) {
  const int tid = threadIdx.x;
  const TA om = mg.omega;
  for (int l = 1; l < mg.levels; ++l) {  // descend: residual, restrict (+ next pre-smoothing)
    const MgLevel<TA> v = mg.level(l);
    if (tid < v.NN) {
      const vec2_t<TA> kz = mg_apply<TA>(v, v.z, tid % v.n, tid / v.n), rr = v.r[tid];
      v.t[tid] = mk2<TA>(rr.x - kz.x, rr.y - kz.y);
    }
    __syncthreads();
    if (tid < mg.level(l + 1).NN) mg_restrict_smooth<TA>(mg, l + 1, v.t, v.n, tid);
    __syncthreads();
  }
  {  // coarsest: z = A^-1 r, 16 lanes per row (rows 0, 1 of the inverse: the pinned identity)
    const MgLevel<TA> c = mg.level(mg.levels);
    const int D = 2 * c.NN, ld = D + 1, row = tid >> 4, l16 = tid & 15;
    const TA* A = mg.coarsest_inverse();
    const TA* r = reinterpret_cast<const TA*>(c.r);
    TA zz = TA(0);
    if (row < D)
      for (int q = l16; q < D; q += 16) zz += A[(size_t)row * ld + q] * r[q];
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) zz += __shfl_xor_sync(0xffffffffu, zz, o);
    if (row < D && l16 == 0)
      reinterpret_cast<TA*>(c.z)[row] = pinned2((row >> 1) % c.n, (row >> 1) / c.n, c.bc) ? TA(0) : zz;
    __syncthreads();
  }
  for (int l = mg.levels - 1; l >= 1; --l) {  // ascend: prolong, post-smooth into t
    const MgLevel<TA> v = mg.level(l);
    const vec2_t<TA>* zc = mg_result<TA>(mg, l + 1);
    const int i = tid % v.n, j = tid / v.n;
    if (tid < v.NN) {
      const vec2_t<TA> zo = v.z[tid], zp = mg_prolong<TA>(zc, v.n, i, j);
      v.z[tid] = mk2<TA>(zo.x + zp.x, zo.y + zp.y);
    }
    __syncthreads();
    if (tid < v.NN) {
      const vec2_t<TA> kz = mg_apply<TA>(v, v.z, i, j), rr = v.r[tid], z = v.z[tid];
      const vec2_t<TA> dz = mg_smooth<TA>(v.mi, v.NN, tid, mk2<TA>(rr.x - kz.x, rr.y - kz.y), om);
      v.t[tid] = mk2<TA>(z.x + dz.x, z.y + dz.y);
    }
    __syncthreads();
  }
}

// Block-Jacobi preconditioned CG for K x = b on the pinned periodic space, in the
// single-reduction form of Chronopoulos and Gear (one fused block reduction of
// gamma = r.u and delta = u.Ku per iteration, u = M^-1 r; p and s = K p follow by
// recurrence).  All threads call it.  x is accumulated in shared memory (xs, the owned
// nodes only).  Returns the iteration count; *status receives kStatusPcgCap /
// kStatusPcgBreakdown / kStatusNegCurv.
// truncate: for Newton corrections away from equilibrium the tangent may be indefinite; on
// negative curvature (p^T K p <= 0) the iteration stops with the step built so far
// (Steihaug's truncated CG; on the first iteration the preconditioned residual direction with
// |p^T K p| as curvature) and reports kStatusNegCurv, which the Newton loop accepts.
// warm: xs holds a start value x0 at the owned nodes (the previous solve's solution); the
// iteration runs on r = b - K x0 and stops at the same rtol relative to b^T M^-1 b as a start
// from zero (one more preconditioner application and apply, counted as one iteration).
template <typename TA, bool REG, bool kMG>
__device__ __forceinline__ int pcg_pair(const Stencil<TA, REG>& S, const Own2D& o, const TA (&Minv)[2][4],
                                        const MgCtx<TA>& mg, const TA (&b)[4],
                        vec2_t<TA>* xs, TA rtol, int max_it, vec2_t<TA>* ps, double* red, int* status,
                        bool truncate, bool warm = false) {
  // x: registers on the block-Jacobi path; accumulated in xs on the multigrid path, where the
  // V-cycle needs the registers
  TA r[4], u[4], w[4], p[4], s[4], x[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    r[k] = o.active ? b[k] : TA(0);
    x[k] = TA(0);
    u[k] = TA(0);
  }
  auto x_axpy = [&](TA a, const TA (&v)[4]) {  // x += a v
    if constexpr (kMG) {
      if (o.active) {
        const vec2_t<TA> x0 = xs[o.node[0]], x1 = xs[o.node[1]];
        xs[o.node[0]] = mk2<TA>(x0.x + a * v[0], x0.y + a * v[1]);
        xs[o.node[1]] = mk2<TA>(x1.x + a * v[2], x1.y + a * v[3]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] += a * v[k];
    }
  };
  if constexpr (kMG) {
    if (o.active && !warm) {
      xs[o.node[0]] = mk2<TA>(TA(0), TA(0));
      xs[o.node[1]] = mk2<TA>(TA(0), TA(0));
    }
  }
  // The exchange alternates between two buffers: the barrier of exchange k + 1 orders every read of
  // exchange k before the writes of exchange k + 2, so no barrier is needed after the reads.
  int pb = 0;
  auto exchange_apply = [&]() {  // w = K u
    vec2_t<TA>* pbuf = ps + (pb ? o.NN : 0);
    pb ^= 1;
    if (o.active) {
      pbuf[o.node[0]] = mk2<TA>(u[0], u[1]);
      pbuf[o.node[1]] = mk2<TA>(u[2], u[3]);
    }
    __syncthreads();
    if (o.active) {
      apply_pair<TA, REG>(S, o, pbuf, u, w);
      if (o.pin[0]) w[0] = w[1] = TA(0);  // pinned nodes
      if (o.pin[1]) w[2] = w[3] = TA(0);
    } else {
      w[0] = w[1] = w[2] = w[3] = TA(0);
    }
  };
  auto jacobi = [&](const TA (&v)[4], TA om) {  // u += om M^-1 v (inverted nodal 2x2 blocks)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      u[2 * q] += om * (Minv[q][0] * v[2 * q] + Minv[q][1] * v[2 * q + 1]);
      u[2 * q + 1] += om * (Minv[q][2] * v[2 * q] + Minv[q][3] * v[2 * q + 1]);
    }
  };
  auto precond = [&]() {  // u = M^-1 r: block-Jacobi, or the multigrid V-cycle
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = TA(0);
    if (!kMG || !mg.levels) {
      jacobi(r, TA(1));
      return;
    }
    const TA om = mg.omega;
    jacobi(r, om);     // pre-smoothing from zero
    exchange_apply();  // w = K u
    vec2_t<TA>* ft = mg.fine_t();
    if (o.active) {
      ft[o.node[0]] = mk2<TA>(r[0] - w[0], r[1] - w[1]);
      ft[o.node[1]] = mk2<TA>(r[2] - w[2], r[3] - w[3]);
    }
    __syncthreads();
    {
      const MgLevel<TA> c = mg.level(1);
      for (int I = threadIdx.x; I < c.NN; I += blockDim.x) mg_restrict_smooth<TA>(mg, 1, ft, o.n, I);
    }
    __syncthreads();
    mg_coarse_cycle<TA>(mg);
    if (o.active) {
      const vec2_t<TA>* zc = mg_result<TA>(mg, 1);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const vec2_t<TA> zp = mg_prolong<TA>(zc, o.n, o.col, 2 * o.strip + q);
        u[2 * q] += zp.x;
        u[2 * q + 1] += zp.y;
      }
    }
    exchange_apply();  // w = K u
    const TA t[4] = {r[0] - w[0], r[1] - w[1], r[2] - w[2], r[3] - w[3]};
    jacobi(t, om);     // post-smoothing
  };
  *status = kStatusOk;
  double gref = -1.0;  // stopping reference b^T M^-1 b of a warm start
  int it = 0;
  if (warm) {
    precond();  // u = M^-1 b
    double unused;
    block_dot2_fp64<TA>(r[0] * u[0] + r[1] * u[1] + r[2] * u[2] + r[3] * u[3], TA(0), red, gref, unused);
    if (o.active) {  // u = x0, w = K x0, r = b - K x0
      const vec2_t<TA> x0 = xs[o.node[0]], x1 = xs[o.node[1]];
      u[0] = x0.x;
      u[1] = x0.y;
      u[2] = x1.x;
      u[3] = x1.y;
    } else {
      u[0] = u[1] = u[2] = u[3] = TA(0);
    }
    if constexpr (!kMG) {
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] = u[k];
    }
    exchange_apply();
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k] -= w[k];
    it = 1;
  }
  precond();
  exchange_apply();
  // inner products: per thread and per warp in TA, over the block in FP64 (block_dot2_fp64); the
  // stopping test compares FP64 sums, the step scalars are formed in TA from them
  double gd, dd;
  block_dot2_fp64<TA>(r[0] * u[0] + r[1] * u[1] + r[2] * u[2] + r[3] * u[3],
                      w[0] * u[0] + w[1] * u[1] + w[2] * u[2] + w[3] * u[3], red, gd, dd);
  TA gamma = (TA)gd, delta = (TA)dd;
  const double gamma0 = gd;
  const double stop = (double)rtol * (double)rtol * (warm ? gref : gamma0);
  // a non-finite or negative preconditioned residual norm r^T M^-1 r (a multigrid coarse inverse of
  // an indefinite tangent, or a V-cycle that is not positive definite) is a breakdown, not a
  // converged zero correction
  if (!isfinite(gamma0) || gamma0 < 0.0 || (warm && !(gref >= 0.0))) *status = kStatusPcgBreakdown;
  if (*status == kStatusOk && gamma0 > 0.0 && !(warm && gamma0 <= stop)) {
    if (!(dd > 0.0)) {
      if (truncate && delta < TA(0)) {
        const TA a0 = cg_div<TA>(gamma, -delta);
        x_axpy(a0, u);
        *status = kStatusNegCurv;
      } else {
        *status = kStatusPcgBreakdown;
      }
    } else {
      TA alpha = cg_div<TA>(gamma, delta);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        p[k] = u[k];
        s[k] = w[k];
      }
      for (;;) {
        if (it >= max_it) {
          *status = kStatusPcgCap;
          break;
        }
        x_axpy(alpha, p);
#pragma unroll
        for (int k = 0; k < 4; ++k) r[k] -= alpha * s[k];
        precond();
        exchange_apply();
        double gnd, dnd;
        block_dot2_fp64<TA>(r[0] * u[0] + r[1] * u[1] + r[2] * u[2] + r[3] * u[3],
                            w[0] * u[0] + w[1] * u[1] + w[2] * u[2] + w[3] * u[3], red, gnd, dnd);
        const TA gn = (TA)gnd, dn = (TA)dnd;
        ++it;
        if (!(gnd >= 0.0)) {  // preconditioner not positive definite (or non-finite)
          *status = kStatusPcgBreakdown;
          break;
        }
        if (gnd <= stop) break;
        const TA beta = cg_div<TA>(gn, gamma);
        const TA den = dn - beta * cg_div<TA>(gn, alpha);  // p_new^T K p_new
        if (!(den > TA(0))) {
          *status = (truncate && den < TA(0)) ? kStatusNegCurv : kStatusPcgBreakdown;
          break;
        }
        alpha = cg_div<TA>(gn, den);
        gamma = gn;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          p[k] = u[k] + beta * p[k];
          s[k] = w[k] + beta * s[k];
        }
      }
    }
  }
  if (!kMG && o.active) {
    xs[o.node[0]] = mk2<TA>(x[0], x[1]);
    xs[o.node[1]] = mk2<TA>(x[2], x[3]);
  }
  return it;
}


// Assemble the tangent at the current w: element tangents -> stage, stencil gather, Minv.
// Minv (inverted nodal blocks, zero on idle threads and the pinned node) stays in
// registers; with withL the condensation right-hand sides go to shared memory,
// Lb[c][NN] = -L_c of each owned node.
template <typename TA, bool REG, bool kMG, int LAW>
__device__ __forceinline__ void build_tangent(const Own2D& o, const Smem2D<TA>& sm, TA* stage_k,
                                              const TA (&Fb)[4], const uint8_t* phase, Stencil<TA, REG>& S,
                                              TA (&Minv)[2][4], bool withL, vec2_t<TA>* Lb, const MgCtx<TA>& mg,
                                              bool build_mg = true) {
  TA L[2][2][4];
  const int n = o.n, NN = o.NN;
  const vec2_t<TA>* wsrc;
  if constexpr (REG) {
    wsrc = reinterpret_cast<const vec2_t<TA>*>(sm.w32);
  } else {
    wsrc = reinterpret_cast<const vec2_t<TA>*>(sm.w);
  }
  if (o.active) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int e = o.node[s];
      const int ph = phase[e];
      element_tangent<TA, LAW>(e, n, wsrc, Fb, (TA)sm.lame[2 * ph], (TA)sm.lame[2 * ph + 1], stage_k, e, NN);
    }
  }
  __syncthreads();
  if (kMG && mg.levels && build_mg) mg_build_part1<TA>(mg, stage_k);  // reads the staged element tangents
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    TA Kn[9][4];
    TA Ln[2][4];
    if (o.active) {
      gather_stencil<TA>(o.node[s], n, stage_k, Kn, withL, Ln);
    } else {
#pragma unroll
      for (int nb = 0; nb < 9; ++nb)
#pragma unroll
        for (int c = 0; c < 4; ++c) Kn[nb][c] = TA(0);
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) Ln[a][c] = TA(0);
    }
    if constexpr (REG) {
#pragma unroll
      for (int nb = 0; nb < 9; ++nb) {
        S.K2[s][nb][0] = make_float2(Kn[nb][0], Kn[nb][1]);
        S.K2[s][nb][1] = make_float2(Kn[nb][2], Kn[nb][3]);
      }
    } else {
      if (o.active) {
#pragma unroll
        for (int nb = 0; nb < 9; ++nb)
#pragma unroll
          for (int c = 0; c < 4; ++c) S.g[(size_t)(nb * 4 + c) * NN + o.node[s]] = Kn[nb][c];
      }
    }
    TA self[4] = {Kn[4][0], Kn[4][1], Kn[4][2], Kn[4][3]};
    TA mi[4];
    invert_block<TA>(self, !o.active || o.pin[s], mi);
#pragma unroll
    for (int c = 0; c < 4; ++c) Minv[s][c] = mi[c];
    if (withL) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) L[s][a][c] = Ln[a][c];
    }
  }
  __syncthreads();  // stage reads done; global stencil writes visible
  if (o.active && withL) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const bool pinned = o.pin[s];
          Lb[c * o.NN + o.node[s]] = mk2<TA>(pinned ? TA(0) : -L[s][0][c], pinned ? TA(0) : -L[s][1][c]);
        }
      }
    }
  }
  if (kMG && mg.levels && build_mg) mg_build_part2<TA>(mg);  // ends with a barrier
}

// Energy form of the tangent transfer over this thread's two elements (FP64 sums of
// per-element TA partials).  X: [4][NN] periodic responses to the unit gradients.
// G_c : A : G_d with M_c = Fit^T G_c (neo-Hookean): mu G_c:G_d - hb tr(M_c M_d) + gm tr M_c tr M_d;
// with M_c = F^T G_c (St. Venant-Kirchhoff): tr(G_c S G_d^T) + lam tr M_c tr M_d
// + mu [M_c:M_d + tr(M_c M_d)].
template <typename TA, int LAW>
__device__ __forceinline__ void element_transfer(int e, int n, const vec2_t<TA>* wsrc, const vec2_t<TA>* X,
                                                 const TA (&Fb)[4], TA lam, TA mu, double (&Q)[10]) {
  const int NN = n * n;
  const int i = e % n, j = e / n, ip = (i + 1) % n, jp = (j + 1) % n;
  const int nd[4] = {e, ip + n * j, ip + n * jp, i + n * jp};
  const TA ih = (TA)n;
  const vec2_t<TA> w0 = wsrc[nd[0]], w1 = wsrc[nd[1]], w2 = wsrc[nd[2]], w3 = wsrc[nd[3]];
  vec2_t<TA> x[4][4];  // [rhs][local node]
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int a = 0; a < 4; ++a) x[c][a] = X[c * NN + nd[a]];
  TA q[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) q[k] = TA(0);
  const TA wq = TA(0.25) / (ih * ih);
#pragma unroll
  for (int gy = 0; gy < 2; ++gy) {
    const TA t = (TA)gauss01(gy);
#pragma unroll
    for (int gx = 0; gx < 2; ++gx) {
      const TA s = (TA)gauss01(gx);
      const TA F00 = Fb[0] + ih * ((1 - t) * (w1.x - w0.x) + t * (w2.x - w3.x));
      const TA F10 = Fb[2] + ih * ((1 - t) * (w1.y - w0.y) + t * (w2.y - w3.y));
      const TA F01 = Fb[1] + ih * ((1 - s) * (w3.x - w0.x) + s * (w2.x - w1.x));
      const TA F11 = Fb[3] + ih * ((1 - s) * (w3.y - w0.y) + s * (w2.y - w1.y));
      // K = Fit (neo-Hookean) or F (St. Venant-Kirchhoff) for M_c = K^T G_c
      TA k00, k01, k10, k11, hb = TA(0), gm = TA(0), S00 = TA(0), S01 = TA(0), S11 = TA(0);
      if constexpr (LAW == kLawNH) {
        const NH2<TA> nh = nh2_eval(F00, F01, F10, F11, lam, mu);
        k00 = nh.f00;
        k01 = nh.f01;
        k10 = nh.f10;
        k11 = nh.f11;
        hb = nh.hb;
        gm = nh.gm;
      } else {
        k00 = F00;
        k01 = F01;
        k10 = F10;
        k11 = F11;
        const TA c00 = F00 * F00 + F10 * F10, c01 = F00 * F01 + F10 * F11, c11 = F01 * F01 + F11 * F11;
        const TA trE = TA(0.5) * (c00 + c11) - TA(1);
        S00 = lam * trE + mu * (c00 - TA(1));
        S11 = lam * trE + mu * (c11 - TA(1));
        S01 = mu * c01;
      }
      TA G[4][4];  // G_c = E_c + Grad X_c, row-major 2x2
      TA M[4][4];  // M_c = K^T G_c
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const vec2_t<TA> a0 = x[c][0], a1 = x[c][1], a2 = x[c][2], a3 = x[c][3];
        G[c][0] = ih * ((1 - t) * (a1.x - a0.x) + t * (a2.x - a3.x));
        G[c][2] = ih * ((1 - t) * (a1.y - a0.y) + t * (a2.y - a3.y));
        G[c][1] = ih * ((1 - s) * (a3.x - a0.x) + s * (a2.x - a1.x));
        G[c][3] = ih * ((1 - s) * (a3.y - a0.y) + s * (a2.y - a1.y));
        G[c][c] += TA(1);
        // M_LJ = sum_i K_iL G_iJ
        M[c][0] = k00 * G[c][0] + k10 * G[c][2];
        M[c][1] = k00 * G[c][1] + k10 * G[c][3];
        M[c][2] = k01 * G[c][0] + k11 * G[c][2];
        M[c][3] = k01 * G[c][1] + k11 * G[c][3];
      }
      int k = 0;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int d = c; d < 4; ++d) {
          // tr(M_c M_d)
          const TA tm = M[c][0] * M[d][0] + M[c][1] * M[d][2] + M[c][2] * M[d][1] + M[c][3] * M[d][3];
          const TA ac = M[c][0] + M[c][3], ad = M[d][0] + M[d][3];
          if constexpr (LAW == kLawNH) {
            const TA gg = G[c][0] * G[d][0] + G[c][1] * G[d][1] + G[c][2] * G[d][2] + G[c][3] * G[d][3];
            q[k++] += wq * (mu * gg - hb * tm + gm * ac * ad);
          } else {
            const TA mm = M[c][0] * M[d][0] + M[c][1] * M[d][1] + M[c][2] * M[d][2] + M[c][3] * M[d][3];
            // tr(G_c S G_d^T) = sum_i (G_c S)_iL G_d,iL
            const TA gs = (G[c][0] * S00 + G[c][1] * S01) * G[d][0] + (G[c][0] * S01 + G[c][1] * S11) * G[d][1] +
                          (G[c][2] * S00 + G[c][3] * S01) * G[d][2] + (G[c][2] * S01 + G[c][3] * S11) * G[d][3];
            q[k++] += wq * (gs + lam * ac * ad + mu * (mm + tm));
          }
        }
    }
  }
#pragma unroll
  for (int k = 0; k < 10; ++k) Q[k] += (double)q[k];
}

// kFixed: one grid size for the whole batch, arrays indexed arithmetically (qp -> RVE qp or 0,
// fluctuation of qp at qp*2*n*n) instead of through the context's index tables.
template <typename TA, bool kFixed, bool kMG, int LAW>
__device__ void solve_item_2d(const Rve2dArgs& a, int qp, const Smem2D<TA>& sm, TA* gscr) {
  constexpr bool REG = std::is_same<TA, float>::value;
  const int tid = threadIdx.x;
  const int rv = kFixed ? (a.phase_per_qp ? qp : 0) : a.qp_rve[qp];
  const int n = kFixed ? a.fixed_n : a.rve_n[rv];
  const int NN = n * n;
  const Own2D o = make_own(n, a.bc);
  const uint8_t* phase = a.phase + (kFixed ? (size_t)rv * n * n : (size_t)a.rve_phase_off[rv]);
  const size_t w_off = kFixed ? (size_t)qp * 2 * n * n : (size_t)a.qp_w_off[qp];
  const double* w_in = a.w_in + w_off;
  double* w_out = a.w_out + w_off;
  if constexpr (kFixed) {
    // the fixed-layout entry takes its phase maps as device data that the host never sees:
    // a phase id outside the material table is reported (status kStatusBadPhase) before any
    // table read
    int badp = 0;
    for (int e = tid; e < NN; e += blockDim.x) badp |= phase[e] >= kMaxPhase;
    if (__syncthreads_or(badp)) {
      if (tid == 0) a.status[qp] = kStatusBadPhase;
      return;
    }
  }
  // Fbar of the current continuation stage, in shared memory (misc[0..3]); read where used
  if (tid < 4) sm.misc[tid] = a.F[(size_t)qp * 4 + tid];
  if (tid < 2 * kMaxPhase) sm.lame[tid] = a.rve_lame[(size_t)rv * 2 * kMaxPhase + tid];
  for (int v = tid; v < NN; v += blockDim.x) {
    double2 wv = make_double2(w_in[2 * v], w_in[2 * v + 1]);
    if (pinned2(v % n, v / n, a.bc)) wv = make_double2(0.0, 0.0);
    sm.w[v] = wv;
    if constexpr (REG) sm.w32[v] = make_float2((float)wv.x, (float)wv.y);
  }
  __syncthreads();

  double* stage_f = reinterpret_cast<double*>(sm.stage);
  // staged element tangents [36][NN]: the block's global scratch in both modes
  TA* stage_k = REG ? reinterpret_cast<TA*>(a.scratch) + (size_t)blockIdx.x * a.scratch_stride
                    : gscr + (size_t)36 * NN;
  Stencil<TA, REG> S;
  S.g = gscr;
  S.NN = NN;
  // multigrid levels: fast region after the condensation arrays in the stage area (mixed) or
  // after the staged tangents and stencil in the block scratch (FP64); slow region in the
  // block scratch
  MgCtx<TA> mg;
  mg.n = n;
  mg.levels = (kMG && a.mg) ? mg_levels(n) : 0;
  mg.bc = a.bc;
  mg.omega = (TA)a.mg_omega;
  if constexpr (REG) {
    mg.fast = reinterpret_cast<TA*>(sm.stage + 8 * (size_t)NN * sizeof(vec2_t<TA>));
    mg.slow = reinterpret_cast<TA*>(a.scratch) + (size_t)blockIdx.x * a.scratch_stride + (size_t)36 * a.nn_max;
  } else {
    mg.fast = gscr + (size_t)72 * a.nn_max;
    mg.slow = mg.fast + mg_fast_max(a.nn_max);
  }
  double* redD = sm.red + 2 * 512 - 64;  // the PCG's FP64 dot buffer (34 doubles) at the end of red
  vec2_t<TA>* Xs = reinterpret_cast<vec2_t<TA>*>(sm.stage);  // [4][NN]
  vec2_t<TA>* Lb = Xs + 4 * NN;                               // [4][NN]
  TA Minv[2][4];

  // Load continuation on failure (as in the 3D kernel): a Newton solve ending in J <= 0, a
  // non-finite residual or a PCG breakdown restarts from w = 0 and reaches Fbar in retry_stages
  // equal increments of Fbar - I.
  // The stage counters live in shared memory (block-uniform) to keep them out of the registers
  // of the PCG loop.
  __shared__ int s_ctl[3];  // stages, stage, Newton iterations of the earlier stages
  if (tid == 0) {
    s_ctl[0] = 1;
    s_ctl[1] = 1;
    s_ctl[2] = 0;
  }
  __syncthreads();
  int status = kStatusNewtonCap, it = 0, cg_total = 0;
  double Psum[4];
  for (;;) {
    int nhalf = 0;
    double r0 = 0.0, step = 1.0;
    it = 0;
    status = kStatusNewtonCap;
    for (;;) {
      // ---- FP64 residual
      Psum[0] = Psum[1] = Psum[2] = Psum[3] = 0.0;
      double bad = 0.0;
      if (o.active) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int e = o.node[s];
          const int ph = phase[e];
          element_residual<LAW>(e, n, sm.w, sm.misc, sm.lame[2 * ph], sm.lame[2 * ph + 1], stage_f, Psum, bad);
        }
      }
      __syncthreads();
      double R[4] = {0, 0, 0, 0};
      if (o.active) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int nd = o.node[s], i = nd % n, j = nd / n;
          const int im = (i - 1 + n) % n, jm = (j - 1 + n) % n;
          const int eA = nd, eB = im + n * j, eC = im + n * jm, eD = i + n * jm;
          R[2 * s] = stage_f[0 * NN + eA] + stage_f[2 * NN + eB] + stage_f[4 * NN + eC] + stage_f[6 * NN + eD];
          R[2 * s + 1] = stage_f[1 * NN + eA] + stage_f[3 * NN + eB] + stage_f[5 * NN + eC] + stage_f[7 * NN + eD];
        }
        if (o.pin[0]) R[0] = R[1] = 0.0;
        if (o.pin[1]) R[2] = R[3] = 0.0;
      }
      double v2[2] = {R[0] * R[0] + R[1] * R[1] + R[2] * R[2] + R[3] * R[3], bad};
      block_sum<2, double>(v2, sm.red + (it & 1) * 512);
      const double rn = sqrt(v2[0]);
      if (it == 0) r0 = rn;
      if ((v2[1] > 0.0 || !isfinite(rn)) && it > 0 && nhalf < kMaxStepHalvings) {
        // backtrack: w = w_prev + step x  ->  w_prev + (step/2) x
        ++nhalf;
        step *= 0.5;
        if (o.active) {
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const int nd = o.node[s];
            double2 wv = sm.w[nd];
            const vec2_t<TA> dx = sm.x[nd];
            wv.x -= step * (double)dx.x;
            wv.y -= step * (double)dx.y;
            sm.w[nd] = wv;
            if constexpr (REG) sm.w32[nd] = make_float2((float)wv.x, (float)wv.y);
          }
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
      if (it >= (s_ctl[0] > 1 ? max(a.max_newton, kRetryNewtonCap) : a.max_newton)) {
        status = kStatusNewtonCap;
        break;
      }
      // ---- tangent and PCG correction.  The multigrid's coarse levels are built at the first
      // Newton iteration of a solve (or continuation stage) and, with mg_reuse, kept for the later
      // ones (the fine level is always the current tangent).  The V-cycle stays symmetric; it stays
      // positive definite while the kept Galerkin operators are and the damped smoother still
      // contracts at the current tangent, true for nearby tangents but not guaranteed under large
      // stretch and contrast, so a PCG that breaks down, hits its cap or sees negative curvature
      // (which an indefinite V-cycle can fake) with kept levels is run once more with levels
      // rebuilt from the current element tangents.
      // (The retry rebuilds the whole tangent: the coarse build must not run while the fine
      // stencil occupies the registers, and one call site of each keeps the code from spilling.)
      // A V-cycle whose fresh levels still break down (its damped smoother no longer contracts at
      // this tangent, e.g. St. Venant-Kirchhoff under compression) is retried with half the
      // damping, down to omega / 8.
      bool reuse = kMG && mg.levels && a.mg_reuse && it > 0;
      TA b[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) b[k] = (TA)(-R[k]);
      int pst = kStatusOk;
      const TA omega0 = mg.omega;
      for (int attempt = 0;; ++attempt) {
        {
          const TA Fb[4] = {(TA)sm.misc[0], (TA)sm.misc[1], (TA)sm.misc[2], (TA)sm.misc[3]};
          build_tangent<TA, REG, kMG, LAW>(o, sm, stage_k, Fb, phase, S, Minv, false, Lb, mg, !reuse);
        }
        cg_total += pcg_pair<TA, REG, kMG>(S, o, Minv, mg, b, sm.x, (TA)a.cg_rtol, a.max_cg, sm.p, redD, &pst, true);
        __syncthreads();
        if (reuse && (pst == kStatusPcgBreakdown || pst == kStatusPcgCap || pst == kStatusNegCurv)) {
          reuse = false;  // once more with levels of the current tangent
        } else if (kMG && mg.levels && (pst == kStatusPcgBreakdown || pst == kStatusPcgCap) &&
                   mg.omega > TA(0.2) * omega0) {
          mg.omega *= TA(0.5);
        } else {
          break;
        }
        pst = kStatusOk;
      }
      mg.omega = omega0;
      if (pst == kStatusPcgBreakdown) {
        status = kStatusPcgBreakdown;
        break;
      }
      step = 1.0;
      nhalf = 0;
      if (o.active) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const int nd = o.node[s];
          double2 wv = sm.w[nd];
          const vec2_t<TA> dx = sm.x[nd];
          wv.x += (double)dx.x;
          wv.y += (double)dx.y;
          sm.w[nd] = wv;
          if constexpr (REG) sm.w32[nd] = make_float2((float)wv.x, (float)wv.y);
        }
      }
      __syncthreads();
      ++it;
    }
    const bool failed = !(status == kStatusOk || status == kStatusNewtonCap);
    int stages = s_ctl[0], stage = s_ctl[1];
    if (failed && stages == 1 && a.retry_stages > 1) {
      stages = a.retry_stages;
      stage = 0;
      for (int v = tid; v < NN; v += blockDim.x) {
        sm.w[v] = make_double2(0.0, 0.0);
        if constexpr (REG) sm.w32[v] = make_float2(0.f, 0.f);
      }
    } else if (failed || stage >= stages) {
      break;
    }
    ++stage;
    __syncthreads();  // every thread has read s_ctl and finished with this stage's Fbar
    if (tid < 4) {
      const double Ft = a.F[(size_t)qp * 4 + tid], id = (tid == 0 || tid == 3) ? 1.0 : 0.0;
      sm.misc[tid] = stage == stages ? Ft : id + (Ft - id) * stage / stages;
    }
    if (tid == 0) {
      s_ctl[0] = stages;
      s_ctl[1] = stage;
      s_ctl[2] += it;
    }
    __syncthreads();
  }
  const int it_total = s_ctl[2] + it;

  // ---- homogenised stress (and energy) at the final state
  double Pv[5] = {Psum[0], Psum[1], Psum[2], Psum[3], 0.0};
  const bool usable = (status == kStatusOk || status == kStatusNewtonCap);
  const bool want_W = usable && (a.flags & kFlagEnergy) && a.W != nullptr;
  if (want_W && o.active) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int e = o.node[s];
      const int ph = phase[e];
      Pv[4] += element_energy<LAW>(e, n, sm.w, sm.misc, sm.lame[2 * ph], sm.lame[2 * ph + 1]);
    }
  }
  // the last residual norm used buffer (it & 1) and may still be read: use the other one
  block_sum<5, double>(Pv, sm.red + ((it + 1) & 1) * 512);
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) sm.misc[4 + k] = Pv[k];
  }

  // ---- tangent transfer (condensation) at the converged state
  int cond_total = 0, cond_max = 0;
  double Q[10];
  const bool want_A = usable && !(a.flags & kFlagNoTangent) && a.A != nullptr;
  if (want_A) {
    const TA Fb[4] = {(TA)sm.misc[0], (TA)sm.misc[1], (TA)sm.misc[2], (TA)sm.misc[3]};
    vec2_t<TA>* X = Xs;
    // kept solutions of this point's previous transfer solves ([4][NN] vec2, zero at first)
    const bool warm = a.X_in != nullptr;
    const vec2_t<TA>* X0 = warm ? reinterpret_cast<const vec2_t<TA>*>(a.X_in) + 2 * w_off : nullptr;
    const TA omega0 = mg.omega;
    // The coarse levels the final Newton stage built (at its first iteration, when it iterated at
    // all) are kept for the transfer too, as for the later Newton iterations: its fine level is
    // the converged tangent.  A transfer PCG that breaks down or hits its cap with kept levels
    // rebuilds the whole tangent with fresh levels and starts the transfer again.
    bool reuse_t = kMG && mg.levels && a.mg_reuse && it > 0;
    for (;;) {
      build_tangent<TA, REG, kMG, LAW>(o, sm, stage_k, Fb, phase, S, Minv, true, Lb, mg, !reuse_t);
      bool redo = false;
      int t_total = 0, t_max = 0, t_status = kStatusOk;
      for (int c = 0; c < 4; ++c) {
        TA b[4] = {TA(0), TA(0), TA(0), TA(0)};
        if (o.active) {
          const vec2_t<TA> b0 = Lb[c * NN + o.node[0]], b1 = Lb[c * NN + o.node[1]];
          b[0] = b0.x;
          b[1] = b0.y;
          b[2] = b1.x;
          b[3] = b1.y;
        }
        int pst = kStatusOk, ci = 0;
        for (;;) {  // as for the Newton corrections: a breakdown is retried with half the damping
          if (warm && o.active) {
#pragma unroll
            for (int s = 0; s < 2; ++s)
              X[c * NN + o.node[s]] = o.pin[s] ? mk2<TA>(TA(0), TA(0)) : X0[c * NN + o.node[s]];
          }
          ci += pcg_pair<TA, REG, kMG>(S, o, Minv, mg, b, X + c * NN, (TA)a.cond_rtol, a.max_cond_cg, sm.p, redD,
                                       &pst, false, warm);
          __syncthreads();
          if (reuse_t && (pst == kStatusPcgBreakdown || pst == kStatusPcgCap)) {
            redo = true;
            break;
          }
          if (!(kMG && mg.levels && (pst == kStatusPcgBreakdown || pst == kStatusPcgCap) &&
                mg.omega > TA(0.2) * omega0))
            break;
          mg.omega *= TA(0.5);
          pst = kStatusOk;
        }
        mg.omega = omega0;
        t_total += ci;
        t_max = ci > t_max ? ci : t_max;
        if (redo) break;
        if (pst != kStatusOk && t_status == kStatusOk) t_status = pst;
      }
      cond_total += t_total;
      cond_max = t_max > cond_max ? t_max : cond_max;
      if (!redo) {
        if (t_status != kStatusOk && status == kStatusOk) status = t_status;
        break;
      }
      reuse_t = false;
    }
    __syncthreads();
    const vec2_t<TA>* wsrc;
    if constexpr (REG) {
      wsrc = reinterpret_cast<const vec2_t<TA>*>(sm.w32);
    } else {
      wsrc = reinterpret_cast<const vec2_t<TA>*>(sm.w);
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) Q[k] = 0.0;
    if (o.active) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int e = o.node[s];
        const int ph = phase[e];
        element_transfer<TA, LAW>(e, n, wsrc, X, Fb, (TA)sm.lame[2 * ph], (TA)sm.lame[2 * ph + 1], Q);
      }
    }
    block_sum<10, double>(Q, sm.red + (it & 1) * 512);
  }

  // ---- outputs
  for (int v = tid; v < NN; v += blockDim.x) {
    const double2 wv = sm.w[v];
    w_out[2 * v] = wv.x;
    w_out[2 * v + 1] = wv.y;
  }
  if (want_A && a.X_out) {  // the transfer solutions, kept as the next solve's start values
    vec2_t<TA>* Xo = reinterpret_cast<vec2_t<TA>*>(a.X_out) + 2 * w_off;
    for (int v = tid; v < 4 * NN; v += blockDim.x) Xo[v] = Xs[v];
  }
  if (tid == 0) {
    a.status[qp] = status;
    if (a.iters) {
      a.iters[(size_t)qp * 4 + 0] = it_total;
      a.iters[(size_t)qp * 4 + 1] = cg_total;
      a.iters[(size_t)qp * 4 + 2] = cond_total;
      a.iters[(size_t)qp * 4 + 3] = cond_max;
    }
    if (usable) {
      const double wq = 0.25 / ((double)n * n);  // Gauss weight x det J; |Omega| = 1
#pragma unroll
      for (int k = 0; k < 4; ++k) a.P[(size_t)qp * 4 + k] = sm.misc[4 + k] * wq;
      if (want_W) a.W[qp] = sm.misc[8] * wq;
      if (want_A) {
        int k = 0;
        for (int c = 0; c < 4; ++c)
          for (int d = c; d < 4; ++d) {
            a.A[(size_t)qp * 16 + c * 4 + d] = Q[k];
            a.A[(size_t)qp * 16 + d * 4 + c] = Q[k];
            ++k;
          }
      }
    }
  }
  __syncthreads();
}

template <typename TA, bool kFixed, bool kMG, int LAW>
__global__ void __launch_bounds__(kThreads2D, 1) rve2d_kernel(const Rve2dArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem2D<TA> sm;
  smem2d_layout<TA>(a.nn_max, &sm, smem_raw);
  __shared__ int s_item;
  constexpr bool REG = std::is_same<TA, float>::value;
  TA* gscr = REG ? nullptr : reinterpret_cast<TA*>(a.scratch) + (size_t)blockIdx.x * a.scratch_stride;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= (a.n_dev ? *a.n_dev : a.n_qp)) break;
    solve_item_2d<TA, kFixed, kMG, LAW>(a, kFixed ? item : a.order[item], sm, gscr);
  }
}

}  // namespace

// Launch of one instantiation (grid of n_blocks persistent blocks, smem dynamic shared bytes).
template <typename TA, bool kFixed, bool kMG, int LAW>
inline cudaError_t rve2d_launch_instance(const Rve2dArgs& a, int n_blocks, size_t smem, cudaStream_t stream) {
  const cudaError_t err = cudaFuncSetAttribute(rve2d_kernel<TA, kFixed, kMG, LAW>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  rve2d_kernel<TA, kFixed, kMG, LAW><<<n_blocks, kThreads2D, smem, stream>>>(a);
  return cudaGetLastError();
}

}  // namespace fehmm
