// Energy surrogate at the macro quadrature points (the learned part of the workload; the paper
// has no counterpart).  For each macro deformation gradient F:
//   C = F^T F, E = (C - I)/2, right stretch U = C^(1/2);
//   trust region: |U - I|_F <= radius, with |U - I|_F^2 = sum_i (sqrt(l_i) - 1)^2 over the
//     eigenvalues l_i of C (closed-form eigenvalues of a symmetric 3x3 matrix, trigonometric
//     method of O. K. Smith, Comm. ACM 4 (1961) 168);
//   energy W(E) = W_base(E) + sg * y(x), x = Mandel(E) / sx, y the MLP;
//   W_base = neo-Hookean(lam0, mu0) + 1/2 m(E).Ca.m(E), m(E) = Mandel(E) (the anisotropic
//     small-strain remainder of the RVE's homogenised elasticity tensor);
//   S = dW/dE, CC = d2W/dEdE, P = F S, A_iJkL = d_ik S_JL + F_iI F_kK CC_IJKL.
// W_base is the compressible neo-Hookean law of the paper's Sec. 6 (Eq. NH-free-energy and the
// closed forms for S and CC) with effective Lame constants (lam0, mu0); the network learns the
// remainder.  Mandel order (11, 22, 33, 23, 13, 12) with sqrt(2) on the shear entries, so that
// S_IJ = (sg/sx) g_p / w_p and CC_IJKL = (sg/sx^2) H_pq / (w_p w_q), w = 1 or sqrt(2).
// The correction y is the sum of a fitted polynomial of degree 3 to 5 in x (weighted linear
// least squares on the training targets, fehmm_surrogate_fit_poly) and the network, which learns
// what the polynomial leaves; both vanish to third order at x = 0.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "fehmm.h"

namespace fehmm {
namespace {

__constant__ int kMandelI[6] = {0, 1, 2, 1, 0, 0};
__constant__ int kMandelJ[6] = {0, 1, 2, 2, 2, 1};

struct BaseAniso {
  double Ca[36];
  double y0, g0[6], H0[36];
};

// m = Mandel(E), s = Ca m  (base stress contribution in Mandel form), e = 1/2 m.Ca.m
__device__ __forceinline__ void aniso_base(const BaseAniso& b, const double (&C)[9], double (&sm)[6], double& e) {
  double m[6];
  for (int p = 0; p < 6; ++p) {
    const int I = kMandelI[p], J = kMandelJ[p];
    m[p] = (I == J ? 1.0 : 1.4142135623730950488) * 0.5 * (C[3 * I + J] - (I == J ? 1.0 : 0.0));
  }
  e = 0.0;
  for (int p = 0; p < 6; ++p) {
    double t = 0.0;
    for (int q = 0; q < 6; ++q) t += b.Ca[6 * p + q] * m[q];
    sm[p] = t;
    e += 0.5 * m[p] * t;
  }
}

__device__ __forceinline__ int mandel_index(int I, int J) {
  if (I == J) return I;
  const int a = I < J ? I : J, b = I < J ? J : I;
  return (a == 1 && b == 2) ? 3 : (a == 0 && b == 2) ? 4 : 5;
}

// ------------------------------------------------------------------ polynomial part
constexpr int kPolyTerms = FEHMM_POLY_TERMS;
constexpr int kPolyMaxDeg = 6;

// Index tuples of the monomials: degree 3, 4, 5, 6, each in lexicographic order of the
// nondecreasing tuples (i1 <= ... <= id); unused positions hold 6 (the factor 1).
struct MonoTable {
  unsigned char idx[kPolyTerms][kPolyMaxDeg];
  unsigned char deg[kPolyTerms];
  int count;
};

constexpr MonoTable make_monomials() {
  MonoTable t{};
  int c = 0;
  for (int d = 3; d <= kPolyMaxDeg; ++d) {
    int a[kPolyMaxDeg] = {0, 0, 0, 0, 0, 0};
    for (;;) {
      if (c < kPolyTerms) {
        for (int k = 0; k < kPolyMaxDeg; ++k) t.idx[c][k] = (unsigned char)(k < d ? a[k] : 6);
        t.deg[c] = (unsigned char)d;
      }
      ++c;
      int k = d - 1;
      while (k >= 0 && a[k] == 5) --k;
      if (k < 0) break;
      ++a[k];
      for (int m = k + 1; m < d; ++m) a[m] = a[k];
    }
  }
  t.count = c;
  return t;
}

constexpr MonoTable kMonoHost = make_monomials();
static_assert(kMonoHost.count == kPolyTerms, "56 + 126 + 252 + 462 monomials of degree 3..6 in 6 variables");

// terms of degree <= d (the coefficients are ordered by degree)
__host__ __device__ constexpr int poly_terms_upto(int d) {
  return d <= 2 ? 0 : d == 3 ? 56 : d == 4 ? 182 : d == 5 ? 434 : 896;
}
__constant__ MonoTable kMono = make_monomials();

// Factors of monomial c at x (padded with ones) and the products of all factors but one.
__device__ __forceinline__ void mono_factors(int c, const double (&x7)[7], double (&v)[kPolyMaxDeg],
                                             int (&id)[kPolyMaxDeg]) {
#pragma unroll
  for (int k = 0; k < kPolyMaxDeg; ++k) {
    id[k] = kMono.idx[c][k];
    v[k] = x7[id[k]];
  }
}

// y_poly, its gradient and (H != null) Hessian at x (FP64), coefficients coef[kPolyTerms].
__device__ void poly_eval(const double* coef, const double (&x)[6], double& y, double (&g)[6], double* H) {
  double x7[7];
#pragma unroll
  for (int k = 0; k < 6; ++k) x7[k] = x[k];
  x7[6] = 1.0;
  y = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) g[k] = 0.0;
  if (H)
    for (int k = 0; k < 36; ++k) H[k] = 0.0;
  for (int c = 0; c < kPolyTerms; ++c) {
    const double a = coef[c];
    if (a == 0.0) continue;
    double v[kPolyMaxDeg];
    int id[kPolyMaxDeg];
    mono_factors(c, x7, v, id);
    const int d = kMono.deg[c];
    y += a * (v[0] * v[1] * v[2] * v[3] * v[4] * v[5]);
#pragma unroll
    for (int i = 0; i < kPolyMaxDeg; ++i) {
      if (i >= d) break;
      double pe = a;
#pragma unroll
      for (int k = 0; k < kPolyMaxDeg; ++k)
        if (k != i) pe *= v[k];
      g[id[i]] += pe;
      if (H) {
#pragma unroll
        for (int j = i + 1; j < kPolyMaxDeg; ++j) {
          if (j >= d) break;
          double pij = a;
#pragma unroll
          for (int k = 0; k < kPolyMaxDeg; ++k)
            if (k != i && k != j) pij *= v[k];
          H[6 * id[i] + id[j]] += pij;
          H[6 * id[j] + id[i]] += pij;
        }
      }
    }
  }
}

// eigenvalues of a symmetric 3x3 matrix (trigonometric closed form)
__device__ void sym3_eigenvalues(const double (&C)[9], double (&l)[3]) {
  const double p1 = C[1] * C[1] + C[2] * C[2] + C[5] * C[5];
  const double q = (C[0] + C[4] + C[8]) / 3.0;
  if (p1 < 1e-300) {
    l[0] = C[0];
    l[1] = C[4];
    l[2] = C[8];
    return;
  }
  const double p2 = (C[0] - q) * (C[0] - q) + (C[4] - q) * (C[4] - q) + (C[8] - q) * (C[8] - q) + 2.0 * p1;
  const double p = sqrt(p2 / 6.0);
  double B[9];
  for (int k = 0; k < 9; ++k) B[k] = (C[k] - (k % 4 == 0 ? q : 0.0)) / p;
  const double detB = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                      B[2] * (B[3] * B[7] - B[4] * B[6]);
  double r = 0.5 * detB;
  r = r < -1.0 ? -1.0 : (r > 1.0 ? 1.0 : r);
  const double phi = acos(r) / 3.0;
  l[0] = q + 2.0 * p * cos(phi);
  l[2] = q + 2.0 * p * cos(phi + 2.0943951023931954923);
  l[1] = 3.0 * q - l[0] - l[2];
}

__global__ void features_kernel(const double* F, int n, double sx, double radius, float* x, int32_t* inside) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double* f = F + (size_t)q * 9;
  double C[9];
  for (int I = 0; I < 3; ++I)
    for (int J = 0; J < 3; ++J) C[3 * I + J] = f[I] * f[J] + f[3 + I] * f[3 + J] + f[6 + I] * f[6 + J];
  double l[3];
  sym3_eigenvalues(C, l);
  double r2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double s = sqrt(l[k] > 0.0 ? l[k] : 0.0) - 1.0;
    r2 += s * s;
  }
  inside[q] = (r2 <= radius * radius) ? 1 : 0;
  for (int p = 0; p < 6; ++p) {
    const int I = kMandelI[p], J = kMandelJ[p];
    const double E = 0.5 * (C[3 * I + J] - (I == J ? 1.0 : 0.0));
    x[(size_t)q * 6 + p] = (float)((I == J ? 1.0 : 1.4142135623730950488) * E / sx);
  }
}

__global__ void combine_kernel(const double* F, int n, double lam0, double mu0, double sx, double sg, const BaseAniso ba,
                               const double* coef, const float* y, const float* g, const float* H, double* P, double* A,
                               double* Wout) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double* f = F + (size_t)q * 9;
  double C[9];
  for (int I = 0; I < 3; ++I)
    for (int J = 0; J < 3; ++J) C[3 * I + J] = f[I] * f[J] + f[3 + I] * f[3 + J] + f[6 + I] * f[6 + J];
  // base law: S = lam/2 (J^2-1) C^-1 + mu (I - C^-1), CC = [lam(J^2-1) - 2mu] dC^-1/dC + lam J^2 C^-1 x C^-1
  const double c00 = C[4] * C[8] - C[5] * C[7], c01 = C[5] * C[6] - C[3] * C[8], c02 = C[3] * C[7] - C[4] * C[6];
  const double c11 = C[0] * C[8] - C[2] * C[6], c12 = C[2] * C[3] - C[0] * C[5], c22 = C[0] * C[4] - C[1] * C[3];
  const double J2 = C[0] * c00 + C[1] * c01 + C[2] * c02;
  const double Ci[9] = {c00 / J2, c01 / J2, c02 / J2, c01 / J2, c11 / J2, c12 / J2, c02 / J2, c12 / J2, c22 / J2};
  double S[9];
  for (int k = 0; k < 9; ++k) S[k] = 0.5 * lam0 * (J2 - 1.0) * Ci[k] + mu0 * ((k % 4 == 0 ? 1.0 : 0.0) - Ci[k]);
  const double sq2 = 1.4142135623730950488;
  double sa[6], ea;
  aniso_base(ba, C, sa, ea);
  // network correction with its Taylor terms at x = 0 removed
  double xs[6], gs[6], ys;
  for (int p = 0; p < 6; ++p) {
    const int I = kMandelI[p], J = kMandelJ[p];
    xs[p] = (I == J ? 1.0 : sq2) * 0.5 * (C[3 * I + J] - (I == J ? 1.0 : 0.0)) / sx;
  }
  double yp, gp[6], Hp[36];
  poly_eval(coef, xs, yp, gp, A ? Hp : nullptr);
  ys = (double)y[q] - ba.y0 + yp;
  for (int p = 0; p < 6; ++p) {
    double hx = 0.0;
    for (int r = 0; r < 6; ++r) hx += ba.H0[6 * p + r] * xs[r];
    gs[p] = (double)g[(size_t)q * 6 + p] - ba.g0[p] - hx + gp[p];
    ys -= (ba.g0[p] + 0.5 * hx) * xs[p];
  }
  for (int I = 0; I < 3; ++I)
    for (int J = 0; J < 3; ++J) {
      const int p = mandel_index(I, J);
      S[3 * I + J] += (sg / sx * gs[p] + sa[p]) / (I == J ? 1.0 : sq2);
    }
  const double Jd = sqrt(J2);
  if (Wout) {
    const double trC = C[0] + C[4] + C[8];
    Wout[q] = 0.25 * lam0 * (J2 - 1.0) - (0.5 * lam0 + mu0) * log(Jd) + 0.5 * mu0 * (trC - 3.0) + ea + sg * ys;
  }
  for (int i = 0; i < 3; ++i)
    for (int J = 0; J < 3; ++J) P[(size_t)q * 9 + 3 * i + J] = f[3 * i] * S[J] + f[3 * i + 1] * S[3 + J] + f[3 * i + 2] * S[6 + J];
  if (!A) return;
  const double beta = lam0 * (J2 - 1.0) - 2.0 * mu0, gam = lam0 * J2;
  const float* Hq = H + (size_t)q * 36;
  for (int i = 0; i < 3; ++i)
    for (int Jj = 0; Jj < 3; ++Jj)
      for (int k = 0; k < 3; ++k)
        for (int L = 0; L < 3; ++L) {
          double acc = (i == k) ? S[3 * Jj + L] : 0.0;
          for (int I = 0; I < 3; ++I)
            for (int K = 0; K < 3; ++K) {
              const double cc_base = beta * (-0.5) * (Ci[3 * I + K] * Ci[3 * Jj + L] + Ci[3 * Jj + K] * Ci[3 * I + L]) +
                                     gam * Ci[3 * I + Jj] * Ci[3 * K + L];
              const int pp = mandel_index(I, Jj), qq = mandel_index(K, L);
              const double wp = (I == Jj) ? 1.0 : sq2, wq = (K == L) ? 1.0 : sq2;
              const double hn = (double)Hq[pp * 6 + qq] - ba.H0[6 * pp + qq] + Hp[6 * pp + qq];
              const double cc = cc_base + (sg / (sx * sx) * hn + ba.Ca[6 * pp + qq]) / (wp * wq);
              acc += f[3 * i + I] * f[3 * k + K] * cc;
            }
          A[(size_t)q * 81 + (3 * i + Jj) * 9 + 3 * k + L] = acc;
        }
}

// Training targets from full RVE solves at F (= U): features x = Mandel(E)/sx, value target
// ty = (Wbar - W_base)/sg and input-gradient target tg_p = (sx/sg) w_p (Sbar - S_base)_p with
// Sbar = sym(F^-1 Pbar).
__global__ void targets_kernel(const double* F, const double* Pbar, const double* Wbar, int n, double lam0, double mu0,
                               double sx, double sg, const BaseAniso ba, float* x, float* ty, float* tg) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double* f = F + (size_t)q * 9;
  const double* pb = Pbar + (size_t)q * 9;
  double C[9];
  for (int I = 0; I < 3; ++I)
    for (int J = 0; J < 3; ++J) C[3 * I + J] = f[I] * f[J] + f[3 + I] * f[3 + J] + f[6 + I] * f[6 + J];
  // F^-1 = cof(F)^T / det F
  const double c00 = f[4] * f[8] - f[5] * f[7], c01 = f[5] * f[6] - f[3] * f[8], c02 = f[3] * f[7] - f[4] * f[6];
  const double c10 = f[2] * f[7] - f[1] * f[8], c11 = f[0] * f[8] - f[2] * f[6], c12 = f[1] * f[6] - f[0] * f[7];
  const double c20 = f[1] * f[5] - f[2] * f[4], c21 = f[2] * f[3] - f[0] * f[5], c22 = f[0] * f[4] - f[1] * f[3];
  const double det = f[0] * c00 + f[1] * c01 + f[2] * c02;
  const double Fi[9] = {c00 / det, c10 / det, c20 / det, c01 / det, c11 / det, c21 / det, c02 / det, c12 / det, c22 / det};
  double Sb[9];
  for (int I = 0; I < 3; ++I)
    for (int J = 0; J < 3; ++J) Sb[3 * I + J] = Fi[3 * I] * pb[J] + Fi[3 * I + 1] * pb[3 + J] + Fi[3 * I + 2] * pb[6 + J];
  const double k00 = C[4] * C[8] - C[5] * C[7], k01 = C[5] * C[6] - C[3] * C[8], k02 = C[3] * C[7] - C[4] * C[6];
  const double k11 = C[0] * C[8] - C[2] * C[6], k12 = C[2] * C[3] - C[0] * C[5], k22 = C[0] * C[4] - C[1] * C[3];
  const double J2 = C[0] * k00 + C[1] * k01 + C[2] * k02;
  const double Ci[9] = {k00 / J2, k01 / J2, k02 / J2, k01 / J2, k11 / J2, k12 / J2, k02 / J2, k12 / J2, k22 / J2};
  double sa[6], ea;
  aniso_base(ba, C, sa, ea);
  const double Wb =
      0.25 * lam0 * (J2 - 1.0) - (0.5 * lam0 + mu0) * 0.5 * log(J2) + 0.5 * mu0 * (C[0] + C[4] + C[8] - 3.0) + ea;
  ty[q] = (float)((Wbar[q] - Wb) / sg);
  for (int p = 0; p < 6; ++p) {
    const int I = kMandelI[p], J = kMandelJ[p];
    const double w = I == J ? 1.0 : 1.4142135623730950488;
    const double sbase = 0.5 * lam0 * (J2 - 1.0) * Ci[3 * I + J] + mu0 * ((I == J ? 1.0 : 0.0) - Ci[3 * I + J]) +
                         sa[p] / w;
    const double ssym = 0.5 * (Sb[3 * I + J] + Sb[3 * J + I]);
    tg[(size_t)q * 6 + p] = (float)(sx / sg * w * (ssym - sbase));
    x[(size_t)q * 6 + p] = (float)(w * 0.5 * (C[3 * I + J] - (I == J ? 1.0 : 0.0)) / sx);
  }
}

// list of the indices q with mask[q] == value (stable order), count in *count
__global__ void compact_kernel(const int32_t* mask, int n, int value, int stride, int32_t* list, int32_t* count) {
  // one block: prefix count in chunks of blockDim
  __shared__ int32_t base;
  __shared__ int32_t warp_tot[32];
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int start = 0; start < n; start += blockDim.x) {
    const int q = start + threadIdx.x;
    const int flag = (q < n && mask[q] == value && (q % stride) == 0) ? 1 : 0;
    const unsigned ballot = __ballot_sync(0xffffffffu, flag);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int before = __popc(ballot & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[warp] = __popc(ballot);
    __syncthreads();
    int off = 0;
    for (int w = 0; w < warp; ++w) off += warp_tot[w];
    if (flag) list[base + off + before] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += warp_tot[w];
      base += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}


// ------------------------------------------------------------------ polynomial fit
constexpr int kFitTile = 32;
constexpr int kFitChunk = 12;              // samples per shared-memory chunk (7 rows each)
constexpr int kFitRows = 7 * kFitChunk;
constexpr int kFitMaxSamples = 65536;

// sums of ty^2 and |tg|^2 over the fit samples (the loss normalisation)
__global__ void fit_norms_kernel(const float* ty, const float* tg, int n, double* out) {
  double a = 0.0, b = 0.0;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    a += (double)ty[q] * ty[q];
    for (int k = 0; k < 6; ++k) b += (double)tg[(size_t)q * 6 + k] * tg[(size_t)q * 6 + k];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], a);
    atomicAdd(&out[1], b);
  }
}

// The 7 rows (value, 6 partial derivatives) of column col for a sample at features x, each
// scaled by the square root of its weight; the target column holds ty, tg.
__device__ __forceinline__ void fit_column(int col, int nt, const double (&x7)[7], float tyv, const float* tgv,
                                           double ry, double rg, double (&r)[7]) {
  if (col > nt) {
#pragma unroll
    for (int k = 0; k < 7; ++k) r[k] = 0.0;
    return;
  }
  if (col == nt) {
    r[0] = ry * tyv;
#pragma unroll
    for (int k = 0; k < 6; ++k) r[1 + k] = rg * tgv[k];
    return;
  }
  double v[kPolyMaxDeg];
  int id[kPolyMaxDeg];
  mono_factors(col, x7, v, id);
  const int d = kMono.deg[col];
  r[0] = ry * (v[0] * v[1] * v[2] * v[3] * v[4] * v[5]);
#pragma unroll
  for (int k = 0; k < 6; ++k) r[1 + k] = 0.0;
#pragma unroll
  for (int i = 0; i < kPolyMaxDeg; ++i) {
    if (i >= d) break;
    double pe = rg;
#pragma unroll
    for (int k = 0; k < kPolyMaxDeg; ++k)
      if (k != i) pe *= v[k];
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (id[i] == k) r[1 + k] += pe;
  }
}

// G[i][j] += sum over rows of phi_i phi_j (nt monomial columns and the target column nt, G is
// (nt + 1)^2) for the column tiles (ti <= tj) of blockIdx.x, over the sample slice blockIdx.y.
// FP64 throughout; block partials added to G atomically.
__global__ void __launch_bounds__(256) fit_normal_kernel(const float* x, const float* ty, const float* tg, int n,
                                                         int nt, const double* norms, double* G) {
  __shared__ double Pi[kFitRows][kFitTile + 1], Pj[kFitRows][kFitTile + 1];
  const int cols = nt + 1, tiles = (cols + kFitTile - 1) / kFitTile;
  int ti = 0, rem = blockIdx.x;
  while (rem >= tiles - ti) {
    rem -= tiles - ti;
    ++ti;
  }
  const int tj = ti + rem;
  const double ry = sqrt((double)n / fmax(norms[0], 1e-300)), rg = sqrt((double)n / fmax(norms[1], 1e-300));
  const int per = (n + gridDim.y - 1) / gridDim.y;
  const int s_begin = blockIdx.y * per, s_end = min(n, s_begin + per);
  const int t = threadIdx.x, cc = t & 31, r0 = t >> 5;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int s0 = s_begin; s0 < s_end; s0 += kFitChunk) {
    for (int item = t; item < 2 * kFitChunk * kFitTile; item += blockDim.x) {
      const int which = item / (kFitChunk * kFitTile), rest = item % (kFitChunk * kFitTile);
      const int ls = rest / kFitTile, col = rest % kFitTile, sidx = s0 + ls;
      double r[7];
      if (sidx < s_end) {
        double x7[7];
#pragma unroll
        for (int k = 0; k < 6; ++k) x7[k] = (double)x[(size_t)sidx * 6 + k];
        x7[6] = 1.0;
        fit_column((which ? tj : ti) * kFitTile + col, nt, x7, ty[sidx], tg + (size_t)sidx * 6, ry, rg, r);
      } else {
#pragma unroll
        for (int k = 0; k < 7; ++k) r[k] = 0.0;
      }
      double(*Pd)[kFitTile + 1] = which ? Pj : Pi;
#pragma unroll
      for (int k = 0; k < 7; ++k) Pd[7 * ls + k][col] = r[k];
    }
    __syncthreads();
    for (int row = 0; row < kFitRows; ++row) {
      const double bj = Pj[row][cc];
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[m] = fma(Pi[row][r0 + 8 * m], bj, acc[m]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int gi = ti * kFitTile + r0 + 8 * m, gj = tj * kFitTile + cc;
    if (gi < cols && gj < cols) atomicAdd(&G[(size_t)gi * cols + gj], acc[m]);
  }
}

// ty -= y_poly(x), tg -= grad y_poly(x) for every sample
__global__ void fit_subtract_kernel(const double* coef, const float* x, int n, float* ty, float* tg) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  double xs[6], y, g[6];
  for (int k = 0; k < 6; ++k) xs[k] = (double)x[(size_t)q * 6 + k];
  poly_eval(coef, xs, y, g, nullptr);
  ty[q] = (float)((double)ty[q] - y);
  for (int k = 0; k < 6; ++k) tg[(size_t)q * 6 + k] = (float)((double)tg[(size_t)q * 6 + k] - g[k]);
}

// Cholesky solve of the symmetric positive definite system A c = b (host, in place on a copy)
bool cholesky_solve(std::vector<double>& A, int N, std::vector<double>& b) {
  for (int j = 0; j < N; ++j) {
    double d = A[(size_t)j * N + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * N + k] * A[(size_t)j * N + k];
    if (!(d > 0.0)) return false;
    const double ljj = sqrt(d);
    A[(size_t)j * N + j] = ljj;
    for (int i = j + 1; i < N; ++i) {
      double v = A[(size_t)i * N + j];
      for (int k = 0; k < j; ++k) v -= A[(size_t)i * N + k] * A[(size_t)j * N + k];
      A[(size_t)i * N + j] = v / ljj;
    }
  }
  for (int i = 0; i < N; ++i) {  // L z = b
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= A[(size_t)i * N + k] * b[k];
    b[i] = v / A[(size_t)i * N + i];
  }
  for (int i = N - 1; i >= 0; --i) {  // L^T c = z
    double v = b[i];
    for (int k = i + 1; k < N; ++k) v -= A[(size_t)k * N + i] * b[k];
    b[i] = v / A[(size_t)i * N + i];
  }
  return true;
}

}  // namespace
}  // namespace fehmm

using namespace fehmm;

extern "C" int fehmm_mlp_eval(fehmm_mlp* m, const float* x, int B, float* y, float* g, float* H, void* stream);

extern "C" int fehmm_surrogate_eval(fehmm_mlp* mlp, const fehmm_surrogate_params* sp, const double* F, int n,
                                    double* P, double* A, double* W, int32_t* inside, float* work, void* stream) {
  if (!mlp || !sp || !F || !P || !inside || !work || n <= 0) return FEHMM_ERR_ARG;
  if (!(sp->sx > 0) || !(sp->sg > 0) || !(sp->radius >= 0)) return FEHMM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  double* coef = reinterpret_cast<double*>(work);  // [kPolyTerms], then the float arrays
  float* x = work + 2 * kPolyTerms;                 // [n][6]
  float* y = x + (size_t)n * 6;                     // [n]
  float* g = y + n;                // [n][6]
  float* H = g + (size_t)n * 6;    // [n][36]
  const int blocks = (n + 127) / 128;
  if (reinterpret_cast<uintptr_t>(work) % 8 != 0) return FEHMM_ERR_ARG;
  if (cudaMemcpyAsync(coef, sp->poly, sizeof(double) * kPolyTerms, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return FEHMM_ERR_CUDA;
  features_kernel<<<blocks, 128, 0, s>>>(F, n, sp->sx, sp->radius, x, inside);
  int rc = fehmm_mlp_eval(mlp, x, n, y, g, A ? H : nullptr, stream);
  if (rc != FEHMM_OK) return rc;
  BaseAniso ba;
  for (int k = 0; k < 36; ++k) {
    ba.Ca[k] = sp->Ca[k];
    ba.H0[k] = sp->H0[k];
  }
  for (int k = 0; k < 6; ++k) ba.g0[k] = sp->g0[k];
  ba.y0 = sp->y0;
  combine_kernel<<<blocks, 128, 0, s>>>(F, n, sp->lam0, sp->mu0, sp->sx, sp->sg, ba, coef, y, g, H, P, A, W);
  return cudaGetLastError() == cudaSuccess ? FEHMM_OK : FEHMM_ERR_CUDA;
}

extern "C" size_t fehmm_surrogate_work_floats(int n) { return 2 * (size_t)kPolyTerms + (size_t)n * (6 + 1 + 6 + 36); }

extern "C" int fehmm_select(const int32_t* mask, int n, int value, int stride, int32_t* list, int32_t* count,
                            void* stream) {
  if (!mask || !list || !count || n <= 0 || stride < 1) return FEHMM_ERR_ARG;
  compact_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(mask, n, value, stride, list, count);
  return cudaGetLastError() == cudaSuccess ? FEHMM_OK : FEHMM_ERR_CUDA;
}

extern "C" int fehmm_surrogate_targets(const fehmm_surrogate_params* sp, const double* F, const double* P,
                                       const double* W, int n, float* x, float* ty, float* tg, void* stream) {
  if (!sp || !F || !P || !W || !x || !ty || !tg || n <= 0 || !(sp->sx > 0) || !(sp->sg > 0)) return FEHMM_ERR_ARG;
  BaseAniso ba{};
  for (int k = 0; k < 36; ++k) ba.Ca[k] = sp->Ca[k];
  targets_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(F, P, W, n, sp->lam0, sp->mu0, sp->sx, sp->sg, ba, x,
                                                                    ty, tg);
  return cudaGetLastError() == cudaSuccess ? FEHMM_OK : FEHMM_ERR_CUDA;
}

// Base law of the surrogate from the small-strain homogenised tangent (host set-up arithmetic on
// 81 numbers; see include/fehmm.h).
extern "C" int fehmm_surrogate_base_law(const double* A0, fehmm_surrogate_params* sp) {
  if (!A0 || !sp) return FEHMM_ERR_ARG;
  double S[81];  // minor-symmetric part
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l)
          S[((i * 3 + j) * 3 + k) * 3 + l] =
              0.25 * (A0[((i * 3 + j) * 3 + k) * 3 + l] + A0[((j * 3 + i) * 3 + k) * 3 + l] +
                      A0[((i * 3 + j) * 3 + l) * 3 + k] + A0[((j * 3 + i) * 3 + l) * 3 + k]);
  double iijj = 0.0, ijij = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      iijj += S[((i * 3 + i) * 3 + j) * 3 + j];
      ijij += S[((i * 3 + j) * 3 + i) * 3 + j];
    }
  const double K = iijj / 9.0, mu = (ijij - iijj / 3.0) / 10.0, lam = K - 2.0 * mu / 3.0;
  if (!(mu > 0.0) || !(lam + 2.0 * mu / 3.0 > 0.0)) return FEHMM_ERR_ARG;
  const int I6[6] = {0, 1, 2, 1, 0, 0}, J6[6] = {0, 1, 2, 2, 2, 1};
  const double r2 = 1.4142135623730951;
  for (int p = 0; p < 6; ++p)
    for (int q = 0; q < 6; ++q) {
      const int i = I6[p], j = J6[p], k = I6[q], l = J6[q];
      const double iso = lam * (i == j) * (k == l) + mu * ((i == k) * (j == l) + (i == l) * (j == k));
      const double wp = p < 3 ? 1.0 : r2, wq = q < 3 ? 1.0 : r2;
      sp->Ca[6 * p + q] = wp * wq * (S[((i * 3 + j) * 3 + k) * 3 + l] - iso);
    }
  sp->lam0 = lam;
  sp->mu0 = mu;
  return FEHMM_OK;
}

extern "C" int fehmm_surrogate_fit_poly(fehmm_surrogate_params* sp, const float* x, float* ty, float* tg, int n,
                                        int max_degree, void* stream) {
  if (!sp || !x || !ty || !tg || n <= 0 || max_degree < 3 || max_degree > kPolyMaxDeg) return FEHMM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int nf = n < kFitMaxSamples ? n : kFitMaxSamples;
  const int N = poly_terms_upto(max_degree), cols = N + 1, tiles = (cols + kFitTile - 1) / kFitTile;
  double* d = nullptr;  // norms [2], G [cols^2], coefficients [kPolyTerms]
  const size_t nG = (size_t)cols * cols;
  if (cudaMalloc(&d, sizeof(double) * (2 + nG + kPolyTerms)) != cudaSuccess) {
    cudaGetLastError();
    return FEHMM_ERR_OOM;
  }
  double* norms = d;
  double* G = d + 2;
  double* coef = G + nG;
  int rc = FEHMM_OK;
  std::vector<double> Gh(nG);
  if (cudaMemsetAsync(d, 0, sizeof(double) * (2 + nG), s) != cudaSuccess) rc = FEHMM_ERR_CUDA;
  if (rc == FEHMM_OK) {
    fit_norms_kernel<<<64, 256, 0, s>>>(ty, tg, nf, norms);
    const int pairs = tiles * (tiles + 1) / 2;
    fit_normal_kernel<<<dim3(pairs, 8), 256, 0, s>>>(x, ty, tg, nf, N, norms, G);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(Gh.data(), G, sizeof(double) * nG, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = FEHMM_ERR_CUDA;
  }
  std::vector<double> c(kPolyTerms, 0.0);
  if (rc == FEHMM_OK) {
    // entry (i, j) was accumulated where tile(i) <= tile(j): take it from there
    std::vector<double> A((size_t)N * N), b(N);
    double tr = 0.0;
    for (int i = 0; i < N; ++i) {
      for (int j = 0; j < N; ++j) {
        const bool up = (i / kFitTile) <= (j / kFitTile);
        A[(size_t)i * N + j] = up ? Gh[(size_t)i * cols + j] : Gh[(size_t)j * cols + i];
      }
      b[i] = Gh[(size_t)i * cols + N];
      tr += A[(size_t)i * N + i];
    }
    for (int i = 0; i < N; ++i) A[(size_t)i * N + i] += 1e-12 * tr / N;
    if (!cholesky_solve(A, N, b)) rc = FEHMM_ERR_ARG;
    for (int i = 0; i < N; ++i) c[i] = b[i];
  }
  if (rc == FEHMM_OK) {
    if (cudaMemcpyAsync(coef, c.data(), sizeof(double) * kPolyTerms, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      rc = FEHMM_ERR_CUDA;
    } else {
      fit_subtract_kernel<<<(n + 127) / 128, 128, 0, s>>>(coef, x, n, ty, tg);
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) rc = FEHMM_ERR_CUDA;
    }
  }
  cudaFree(d);
  if (rc == FEHMM_OK)
    for (int k = 0; k < kPolyTerms; ++k) sp->poly[k] = c[k];
  return rc;
}
