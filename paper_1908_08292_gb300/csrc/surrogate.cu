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
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

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
                               const float* y, const float* g, const float* H, double* P, double* A, double* Wout) {
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
  ys = (double)y[q] - ba.y0;
  for (int p = 0; p < 6; ++p) {
    double hx = 0.0;
    for (int r = 0; r < 6; ++r) hx += ba.H0[6 * p + r] * xs[r];
    gs[p] = (double)g[(size_t)q * 6 + p] - ba.g0[p] - hx;
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
              const double hn = (double)Hq[pp * 6 + qq] - ba.H0[6 * pp + qq];
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

}  // namespace
}  // namespace fehmm

using namespace fehmm;

extern "C" int fehmm_mlp_eval(fehmm_mlp* m, const float* x, int B, float* y, float* g, float* H, void* stream);

extern "C" int fehmm_surrogate_eval(fehmm_mlp* mlp, const fehmm_surrogate_params* sp, const double* F, int n,
                                    double* P, double* A, double* W, int32_t* inside, float* work, void* stream) {
  if (!mlp || !sp || !F || !P || !inside || !work || n <= 0) return FEHMM_ERR_ARG;
  if (!(sp->sx > 0) || !(sp->sg > 0) || !(sp->radius >= 0)) return FEHMM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  float* x = work;                 // [n][6]
  float* y = x + (size_t)n * 6;    // [n]
  float* g = y + n;                // [n][6]
  float* H = g + (size_t)n * 6;    // [n][36]
  const int blocks = (n + 127) / 128;
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
  combine_kernel<<<blocks, 128, 0, s>>>(F, n, sp->lam0, sp->mu0, sp->sx, sp->sg, ba, y, g, H, P, A, W);
  return cudaGetLastError() == cudaSuccess ? FEHMM_OK : FEHMM_ERR_CUDA;
}

extern "C" size_t fehmm_surrogate_work_floats(int n) { return (size_t)n * (6 + 1 + 6 + 36); }

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
