// Device-side helpers shared by the fehmm kernels: vector traits, warp/block reductions
// and the compressible neo-Hookean law of the paper's Sec. 6 in the factored form used by
// the kernels.
//
// Neo-Hookean law (Eq. NH-free-energy and the closed forms for S and CC that follow it):
//   psi = lam/4 (J^2 - 1) - (lam/2 + mu) ln J + mu/2 (tr C - 3)
//   S   = lam/2 (J^2 - 1) C^-1 + mu (I - C^-1)
// With F C^-1 = F^-T (written Fit) and F C^-1 F^T = I these give, exactly,
//   P = F S = mu F + hb Fit,                       hb = lam (J^2 - 1)/2 - mu
//   A_iJkL = dP_iJ/dF_kL = mu d_ik d_JL - hb Fit_iL Fit_kJ + gm Fit_iJ Fit_kL,  gm = lam J^2
// which is delta_ik S_JL + F_iI F_kK CC_IJKL with CC = [lam (J^2-1) - 2 mu] dC^-1/dC
// + lam J^2 C^-1 (x) C^-1 (Eq. Aijkl-NeoHook) after contracting with F.  2D is plane strain
// (F_33 = 1): the same formulas hold for the in-plane 2x2 blocks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fehmm {

constexpr int kMaxPhase = 4;
constexpr int kStatusOk = 0, kStatusNewtonCap = 1, kStatusJNonPos = 2, kStatusPcgBreakdown = 3,
              kStatusNonFinite = 4, kStatusPcgCap = 5,
              kStatusNegCurv = 6,  // internal: truncated Newton-correction PCG
              kStatusBadPhase = 7;  // a device-supplied phase id >= kMaxPhase (nothing solved)
constexpr int kFlagNoTangent = 1, kFlagFromCommitted = 2, kFlagEnergy = 4;
// Newton globalisation: after an update that makes det F <= 0 somewhere (or the residual
// non-finite) the step is halved, up to this many times, before the RVE is reported failed.
constexpr int kMaxStepHalvings = 8;
// Newton cap of each load-continuation stage of a retried solve (at least max_newton): a retry
// recovers a usable state even when max_newton = 1 (the alternating scheme).
constexpr int kRetryNewtonCap = 25;

template <typename T> struct vec2_of;
template <> struct vec2_of<float> { using type = float2; };
template <> struct vec2_of<double> { using type = double2; };
template <typename T> using vec2_t = typename vec2_of<T>::type;

template <typename T>
__device__ __forceinline__ vec2_t<T> mk2(T x, T y) {
  vec2_t<T> v;
  v.x = x;
  v.y = y;
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of NV values over the whole block; every thread receives the totals.
// buf: shared memory with room for 32*NV values; blockDim.x must be a multiple of 32.
// Contains one __syncthreads(); callers alternate buffers between consecutive calls.
template <int NV, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NV], T* buf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) buf[k * 32 + warp] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(lane < nw ? buf[k * 32 + lane] : T(0));
}

// Two inner products summed over a block of 16 warps, the block-level sum in FP64: each thread's
// partial and the warp's shuffle tree stay in T (FP32 in mixed mode), lane 0 of every warp
// stores its warp sum as a double, and warp 0 adds the 16 warp sums of each product in FP64
// (lanes 0-15 the first, lanes 16-31 the second, a 4-level shuffle tree in a fixed order, so
// every launch sums identically) and broadcasts them.  Two barriers.  buf: 34 doubles of shared
// memory; consecutive calls may reuse it (the second barrier orders every read of a call before
// the next call's writes).
template <typename T>
__device__ __forceinline__ void block_dot2_fp64(T a, T b, double* buf, double& sa, double& sb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) {
    buf[warp] = (double)a;
    buf[16 + warp] = (double)b;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    double v = (lane & 15) < nw ? buf[lane] : 0.0;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((lane & 15) == 0) buf[32 + (lane >> 4)] = v;
  }
  __syncthreads();
  sa = buf[32];
  sb = buf[33];
}

// 1/J for the FP64 neo-Hookean stress of the residuals: the FP32 approximate reciprocal (rcp.approx, relative error
// below 2^-22) refined by two Newton-Raphson steps x <- x + x (1 - J x) in FP64, each of which
// squares the relative error (2^-44, then below FP64 rounding), so the result is within an ulp
// or so of the rounded quotient.  J below FP32's normal range (a collapsed element) gives a
// non-finite result, which the Newton loop treats like J <= 0.
__device__ __forceinline__ double recip_fp64(double J) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"((float)J));
  double x = (double)r;
  double e = fma(-J, x, 1.0);
  x = fma(x, e, x);
  e = fma(-J, x, 1.0);
  return fma(x, e, x);
}

// 1/J at the tangent's precision: FP32 through the hardware approximate reciprocal (about one
// FP32 ulp, ample for an FP32 tangent), FP64 as a plain division.
template <typename T>
__device__ __forceinline__ T recip_T(T J) {
  if constexpr (sizeof(T) == 4) {
    return __fdividef(1.f, J);
  } else {
    return 1.0 / J;
  }
}

// Lame constants from (E, nu), as in the paper's material table (Sec. 6).
__host__ __device__ inline void lame_from_E_nu(double E, double nu, double& lam, double& mu) {
  lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  mu = E / (2.0 * (1.0 + nu));
}

// 2D plane-strain point quantities: J, Fit = F^-T, hb, gm (see header comment).
template <typename T>
struct NH2 {
  T J, f00, f01, f10, f11;  // Fit
  T hb, gm;
};

template <typename T>
__device__ __forceinline__ NH2<T> nh2_eval(T F00, T F01, T F10, T F11, T lam, T mu) {
  NH2<T> r;
  r.J = F00 * F11 - F01 * F10;
  const T iJ = recip_T(r.J);
  r.f00 = F11 * iJ;
  r.f01 = -F10 * iJ;
  r.f10 = -F01 * iJ;
  r.f11 = F00 * iJ;
  const T J2 = r.J * r.J;
  r.hb = T(0.5) * lam * (J2 - T(1)) - mu;
  r.gm = lam * J2;
  return r;
}

}  // namespace fehmm
