// Energy-surrogate MLP on BF16 tensor cores (the learned part of the workload; the paper has
// no counterpart).  x in R^6 -> 4 hidden layers of 128 SiLU units -> scalar y.
//   z1 = W1 x + b1, a_l = silu(z_l), z_{l+1} = W_{l+1} a_l + b_{l+1}, y = w5 . a4 + b5
// Provided: forward, input gradient dy/dx (reverse mode), input Hessian (forward mode over the
// reverse pass, the 6 input directions batched as extra rows), the Sobolev training loss
// L = 1/2 sum_b [cy (y_b - ty_b)^2 + cg |dy/dx_b - tg_b|^2] with its exact parameter gradient
// (reverse mode through both the forward and the input-gradient pass), and a fused AdamW step
// on FP32 master weights that refreshes the BF16 copies.
//
// Every matrix product runs in one hand-written kernel: BF16 operands staged in shared memory,
// fragments loaded with ldmatrix, mma.sync.m16n8k16 with FP32 accumulation (64x64 block tile,
// 4 warps of 32x32), optional split-K with FP32 atomics for the weight gradients.  Activations
// are stored sample-major ([batch][128]), so the forward product is A_act(K-major) x W^T with W
// itself as the column-major B operand; transposed operands (batch-reductions) are transposed
// while staging.  BF16 rounding happens exactly where an operand of a product is stored.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include "fehmm.h"
#include "tc_gemm.cuh"

namespace fehmm {
namespace {

using bf16 = __nv_bfloat16;

constexpr int W = 128;   // hidden width
constexpr int NIN = 6;   // inputs
constexpr int NINP = 8;  // inputs padded to a 16-byte row
constexpr int BM = 64, BN = 64, BK = 32, LDS = BK + 8;

// packed FP32 parameter layout
constexpr int OFF_W1 = 0;                     // [128][8]
constexpr int OFF_B1 = OFF_W1 + W * NINP;     // [128]
constexpr int OFF_W2 = OFF_B1 + W;            // [128][128]
constexpr int OFF_B2 = OFF_W2 + W * W;
constexpr int OFF_W3 = OFF_B2 + W;
constexpr int OFF_B3 = OFF_W3 + W * W;
constexpr int OFF_W4 = OFF_B3 + W;
constexpr int OFF_B4 = OFF_W4 + W * W;
constexpr int OFF_W5 = OFF_B4 + W;            // [128]
constexpr int OFF_B5 = OFF_W5 + W;            // [1]
constexpr int N_PARAMS = OFF_B5 + 4;          // padded

__host__ __device__ constexpr int off_W(int l) { return l == 1 ? OFF_W1 : l == 2 ? OFF_W2 : l == 3 ? OFF_W3 : OFF_W4; }
__host__ __device__ constexpr int off_b(int l) { return l == 1 ? OFF_B1 : l == 2 ? OFF_B2 : l == 3 ? OFF_B3 : OFF_B4; }
__host__ __device__ constexpr int fan_in(int l) { return l == 1 ? NINP : W; }

// ------------------------------------------------------------------------- GEMM
struct GemmArgs {
  int M, N, K;
  const bf16* A;
  int lda;
  const bf16* B;
  int ldb;
  float* C;
  int ldc;
  const float* bias;  // per column, or null
  int atomic;         // accumulate into C with atomics (split-K)
  int k_split;        // K range per blockIdx.z (multiple of BK)
};

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const bf16* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Stage a 64 (rows) x 32 (k) tile in shared memory, k contiguous.  MMAJ: the source is stored
// [k][row] (row contiguous) and is transposed while staging.  Out-of-range entries are zero.
template <bool MMAJ>
__device__ __forceinline__ void stage_tile(bf16 (*S)[LDS], const bf16* src, int ld, int r0, int k0, int R, int kend) {
  const uint4 zero = make_uint4(0, 0, 0, 0);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int c = threadIdx.x + i * 128;
    if constexpr (!MMAJ) {
      const int row = c >> 2, kc = (c & 3) * 8;
      const int gr = r0 + row, gk = k0 + kc;
      uint4 v = zero;
      if (gr < R && gk < kend) v = *reinterpret_cast<const uint4*>(src + (size_t)gr * ld + gk);
      *reinterpret_cast<uint4*>(&S[row][kc]) = v;
    } else {
      const int kr = c >> 3, rc = (c & 7) * 8;
      const int gk = k0 + kr, gr = r0 + rc;
      uint4 v = zero;
      if (gk < kend && gr < R) v = *reinterpret_cast<const uint4*>(src + (size_t)gk * ld + gr);
      const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
      for (int j = 0; j < 8; ++j) S[rc + j][kr] = e[j];
    }
  }
}

// C[m][n] (+)= sum_k A(m,k) B(k,n); A(m,k) = AM ? A[k*lda+m] : A[m*lda+k];
// B(k,n) = BNM ? B[k*ldb+n] : B[n*ldb+k].
template <bool AM, bool BNM>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g) {
  __shared__ __align__(16) bf16 As[BM][LDS];
  __shared__ __align__(16) bf16 Bs[BN][LDS];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kb = blockIdx.z * g.k_split, ke = min(g.K, kb + g.k_split);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += BK) {
    stage_tile<AM>(As, g.A, g.lda, m0, k0, g.M, ke);
    stage_tile<BNM>(Bs, g.B, g.ldb, n0, k0, g.N, ke);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) ldmatrix_x4(a[mi], &As[wm + mi * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
      for (int nj = 0; nj < 2; ++nj) {
        uint32_t r[4];
        ldmatrix_x4(r, &Bs[wn + nj * 16 + (lane & 7) + ((lane >> 4) << 3)][kk + ((lane >> 3) & 1) * 8]);
        b[2 * nj][0] = r[0];
        b[2 * nj][1] = r[1];
        b[2 * nj + 1][0] = r[2];
        b[2 * nj + 1][1] = r[3];
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni][0], b[ni][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = m0 + wm + mi * 16 + (lane >> 2) + 8 * h;
        const int c = n0 + wn + ni * 8 + (lane & 3) * 2;
        if (r >= g.M) continue;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (c + e >= g.N) continue;
          float v = acc[mi][ni][2 * h + e];
          float* dst = g.C + (size_t)r * g.ldc + c + e;
          if (g.atomic) {
            atomicAdd(dst, v);
          } else {
            if (g.bias) v += g.bias[c + e];
            *dst = v;
          }
        }
      }
}

// --------------------------------------------------------------- elementwise
__device__ __forceinline__ float sig(float z) { return 1.f / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_f(float z) { return z * sig(z); }
__device__ __forceinline__ float silu_d(float z) {
  const float s = sig(z);
  return s * (1.f + z * (1.f - s));
}
__device__ __forceinline__ float silu_dd(float z) {
  const float s = sig(z);
  return s * (1.f - s) * (2.f + z * (1.f - 2.f * s));
}

#define GRID_STRIDE(i, n) for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)(n); i += (size_t)gridDim.x * blockDim.x)

__global__ void pack_x_kernel(const float* x, int B, bf16* X) {  // [B][6] -> bf16 [B][8]
  GRID_STRIDE(i, (size_t)B * NINP) {
    const int b = i / NINP, k = i % NINP;
    X[i] = __float2bfloat16(k < NIN ? x[(size_t)b * NIN + k] : 0.f);
  }
}

__global__ void silu_kernel(const float* Z, size_t n, bf16* A) {
  GRID_STRIDE(i, n) A[i] = __float2bfloat16(silu_f(Z[i]));
}

// y_b = sum_j w5_j a4_bj + b5 (one warp per sample); bf16 operands, FP32 accumulation
__global__ void output_kernel(const bf16* A4, const bf16* w5, const float* b5, int B, float* y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= B) return;
  float s = 0.f;
  for (int j = lane; j < W; j += 32) s += __bfloat162float(w5[j]) * __bfloat162float(A4[(size_t)warp * W + j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[warp] = s + b5[0];
}

// D4 = w5 * silu'(Z4) (bf16)
__global__ void d4_kernel(const float* Z4, const bf16* w5, int B, bf16* D4) {
  GRID_STRIDE(i, (size_t)B * W) D4[i] = __float2bfloat16(__bfloat162float(w5[i % W]) * silu_d(Z4[i]));
}

// D = C * silu'(Z) (bf16)
__global__ void dmul_kernel(const float* C, const float* Z, size_t n, bf16* D) {
  GRID_STRIDE(i, n) D[i] = __float2bfloat16(C[i] * silu_d(Z[i]));
}

// loss residuals: ry = cy (y - ty), rg = cg (g - tg) (bf16, padded); loss accumulated
__global__ void residual_kernel(const float* y, const float* g, const float* ty, const float* tg, int B, float cy,
                                float cg, float* ry, bf16* rg, float* loss) {
  float l = 0.f;
  GRID_STRIDE(b, B) {
    const float e = y[b] - ty[b];
    ry[b] = cy * e;
    l += cy * e * e;
#pragma unroll
    for (int k = 0; k < NINP; ++k) {
      float v = 0.f;
      if (k < NIN) {
        const float eg = g[(size_t)b * NINP + k] - tg[(size_t)b * NIN + k];
        v = cg * eg;
        l += cg * eg * eg;
      }
      rg[(size_t)b * NINP + k] = __float2bfloat16(v);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, 0.5f * l);
}

// QZ = E * C * silu''(Z) (fp32), ES = E * silu'(Z) (bf16)
__global__ void dbl_kernel(const float* E, const float* C, const float* Z, size_t n, float* QZ, bf16* ES) {
  GRID_STRIDE(i, n) {
    const float z = Z[i];
    QZ[i] = E[i] * C[i] * silu_dd(z);
    ES[i] = __float2bfloat16(E[i] * silu_d(z));
  }
}

// top layer: QZ4 = E4 w5 silu''(Z4); DZ4 = ry w5 silu'(Z4) + QZ4 (fp32 and bf16 copies)
__global__ void top_kernel(const float* E4, const float* Z4, const bf16* w5, const float* ry, int B, float* QZ4,
                           float* DZf, bf16* DZ) {
  GRID_STRIDE(i, (size_t)B * W) {
    const int b = i / W, j = i % W;
    const float w = __bfloat162float(w5[j]), z = Z4[i];
    const float q = E4[i] * w * silu_dd(z);
    QZ4[i] = q;
    const float d = ry[b] * w * silu_d(z) + q;
    DZf[i] = d;
    DZ[i] = __float2bfloat16(d);
  }
}

// DZ_{l-1} = T * silu'(Z_{l-1}) + QZ_{l-1}
__global__ void dz_kernel(const float* T, const float* Z, const float* QZ, size_t n, float* DZf, bf16* DZ) {
  GRID_STRIDE(i, n) {
    const float d = T[i] * silu_d(Z[i]) + QZ[i];
    DZf[i] = d;
    DZ[i] = __float2bfloat16(d);
  }
}

// out[j] += sum_b (X[b][j] * (Y ? Y[b][j] : 1) * (s ? s[b] : 1)) over a batch slice (column sums)
template <typename TX>
__global__ void colsum_kernel(const TX* X, const float* Y, const float* s, int B, int ncol, float* out, int zfun) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncol) return;
  float acc = 0.f;
  for (int b = blockIdx.y; b < B; b += gridDim.y) {
    float v = (float)X[(size_t)b * ncol + j];
    if (Y) v *= zfun ? silu_d(Y[(size_t)b * ncol + j]) : Y[(size_t)b * ncol + j];
    if (s) v *= s[b];
    acc += v;
  }
  atomicAdd(&out[j], acc);
}

// ---------------------------------------------- input Hessian (6 directions)
// ZD1[k*B + b][:] = W1[:, k]
__global__ void hess_init_kernel(const bf16* W1, int B, float* ZD) {
  GRID_STRIDE(i, (size_t)NIN * B * W) {
    const int j = i % W;
    const int k = i / ((size_t)B * W);
    ZD[i] = __bfloat162float(W1[j * NINP + k]);
  }
}

// AD = silu'(Z) * ZD (Z broadcast over the 6 directions) -> bf16
__global__ void hess_fwd_kernel(const float* ZD, const float* Z, int B, bf16* AD) {
  GRID_STRIDE(i, (size_t)NIN * B * W) AD[i] = __float2bfloat16(ZD[i] * silu_d(Z[i % ((size_t)B * W)]));
}

// DD4 = w5 * silu''(Z4) * ZD4
__global__ void hess_top_kernel(const float* ZD, const float* Z4, const bf16* w5, int B, bf16* DD) {
  GRID_STRIDE(i, (size_t)NIN * B * W) {
    const size_t bi = i % ((size_t)B * W);
    DD[i] = __float2bfloat16(__bfloat162float(w5[i % W]) * silu_dd(Z4[bi]) * ZD[i]);
  }
}

// DD_l = T * silu'(Z_l) + C_l * silu''(Z_l) * ZD_l
__global__ void hess_back_kernel(const float* T, const float* Z, const float* C, const float* ZD, int B, bf16* DD) {
  GRID_STRIDE(i, (size_t)NIN * B * W) {
    const size_t bi = i % ((size_t)B * W);
    const float z = Z[bi];
    DD[i] = __float2bfloat16(T[i] * silu_d(z) + C[bi] * silu_dd(z) * ZD[i]);
  }
}

// H[b][j][k] = HK[k*B + b][j]
__global__ void hess_out_kernel(const float* HK, int B, float* H) {
  GRID_STRIDE(i, (size_t)B * NIN * NIN) {
    const int b = i / (NIN * NIN), j = (i / NIN) % NIN, k = i % NIN;
    H[i] = HK[((size_t)k * B + b) * NINP + j];
  }
}

__global__ void copy_g_kernel(const float* G8, int B, float* g) {
  GRID_STRIDE(i, (size_t)B * NIN) g[i] = G8[(i / NIN) * NINP + (i % NIN)];
}

// ------------------------------------------------------------ parameters
// bf16 copies: Wb_l row-major [out][in] and WTb_l = W_l^T row-major [in][out]; W1T padded [8][128]
__global__ void refresh_bf16_kernel(const float* P, bf16* Wb) {
  GRID_STRIDE(i, N_PARAMS) Wb[i] = __float2bfloat16(P[i]);
}
__global__ void transpose_bf16_kernel(const float* P, bf16* WT, int rows, int cols, int ld_out) {
  GRID_STRIDE(i, (size_t)rows * cols) {
    const int r = i / cols, c = i % cols;
    WT[(size_t)c * ld_out + r] = __float2bfloat16(P[i]);
  }
}

// AdamW (decoupled weight decay on weight matrices only); padded input columns of W1 stay zero
__global__ void adamw_kernel(float* P, const float* G, float* m, float* v, int n, float lr, float b1, float b2,
                             float eps, float wd, float bc1, float bc2) {
  GRID_STRIDE(i, n) {
    const int ii = (int)i;
    if (ii < OFF_B1 && (ii % NINP) >= NIN) continue;
    if (ii >= OFF_B5 + 1) continue;
    const bool is_weight = (ii < OFF_B1) || (ii >= OFF_W2 && ii < OFF_B2) || (ii >= OFF_W3 && ii < OFF_B3) ||
                           (ii >= OFF_W4 && ii < OFF_B4) || (ii >= OFF_W5 && ii < OFF_B5);
    const float g = G[i];
    const float mm = b1 * m[i] + (1.f - b1) * g;
    const float vv = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mm;
    v[i] = vv;
    float p = P[i];
    if (is_weight) p -= lr * wd * p;
    p -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    P[i] = p;
  }
}

}  // namespace
}  // namespace fehmm

using namespace fehmm;

struct fehmm_mlp {
  int max_batch = 0;
  float* P = nullptr;   // FP32 masters [N_PARAMS]
  float* G = nullptr;   // gradient
  float* m = nullptr;
  float* v = nullptr;
  bf16* Wb = nullptr;   // bf16 copy of P (row-major weights)
  bf16* WTb = nullptr;  // transposed copies: W1T [8][128], W2T..W4T [128][128]
  float* loss = nullptr;
  // workspace
  bf16* X = nullptr;
  float* Z[5] = {};
  bf16* A[5] = {};
  bf16* D[5] = {};
  float* Cc[5] = {};
  float* QZ[5] = {};
  float* E = nullptr;
  bf16* ES = nullptr;
  float* T = nullptr;
  float* DZf = nullptr;
  bf16* DZ = nullptr;
  float* y = nullptr;
  float* g8 = nullptr;
  float* ry = nullptr;
  bf16* rg = nullptr;
  float* ZD[5] = {};     // forward tangents of z_1..z_4 along the 6 inputs: [6 B][128] each
  bf16* AD = nullptr;
  float* TD = nullptr;
  float* HK = nullptr;   // [6 B][8]
  int step = 0;
  int* err = nullptr;     // set by a tensor-core GEMM whose mbarrier wait ran out
  std::vector<void*> allocs;
  long long launches = 0;
};

namespace {

template <typename T>
int alloc(fehmm_mlp* m, T*& p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    return FEHMM_ERR_OOM;
  }
  m->allocs.push_back(q);
  p = static_cast<T*>(q);
  return FEHMM_OK;
}

int blocks_for(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 4096) b = 4096;
  return (int)(b ? b : 1);
}

template <bool AM, bool BNM, int BN>
cudaError_t launch_tc_bn(const tc::Args& a, dim3 grid, cudaStream_t s) {
  using C = tc::Cfg<BN>;
  // the shared-memory attribute belongs to a device: set once per device for this instantiation
  static std::atomic<uint64_t> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (1ull << dev) : 0ull;
  if (!bit || !(done.load(std::memory_order_relaxed) & bit)) {
    e = cudaFuncSetAttribute(tc::gemm_tc_kernel<AM, BNM, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             C::kSmemBytes);
    if (e != cudaSuccess) return e;
    done.fetch_or(bit, std::memory_order_relaxed);
  }
  tc::gemm_tc_kernel<AM, BNM, BN><<<grid, 128, C::kSmemBytes, s>>>(a);
  return cudaSuccess;
}

template <bool AM, bool BNM>
cudaError_t launch_tc(const tc::Args& a, int bn, dim3 grid, cudaStream_t s) {
  if (bn == 32) return launch_tc_bn<AM, BNM, 32>(a, grid, s);
  if (bn == 64) return launch_tc_bn<AM, BNM, 64>(a, grid, s);
  return launch_tc_bn<AM, BNM, 128>(a, grid, s);
}

// Products with 64 < N <= 128 and K >= 64 (every 128 x 128 layer product, forward, backward and
// weight gradient) run on tcgen05, 128-row tiles of C split into column tiles of 32 or 64 when
// there are too few row tiles to fill the GPU; the narrow ones (the 6-wide input layer, N or K =
// 8) on the mma.sync kernel.
cudaError_t gemm(fehmm_mlp* mm, bool am, bool bnm, int M, int N, int K, const bf16* A, int lda, const bf16* B,
                 int ldb, float* C, int ldc, const float* bias, bool atomic, cudaStream_t s) {
  if (N > 64 && N <= tc::kBNMax && K >= tc::kBK) {
    tc::Args a{M, N, K, A, lda, B, ldb, C, ldc, bias, atomic ? 1 : 0, K, mm->err};
    const int tiles = (M + tc::kBM - 1) / tc::kBM;
    int splits = 1, bn = tc::kBNMax;
    if (atomic) {  // split the batch reduction: chunks of >= 256, at most one CTA per SM in all
      splits = (K + 255) / 256;
      if (splits * tiles > 148) splits = 148 / tiles;
      if (splits < 1) splits = 1;
      a.k_split = ((K + splits - 1) / splits + tc::kBK - 1) / tc::kBK * tc::kBK;
      splits = (K + a.k_split - 1) / a.k_split;
    } else {
      a.k_split = (K + tc::kBK - 1) / tc::kBK * tc::kBK;
      bn = tiles >= 112 ? 128 : (tiles >= 56 ? 64 : 32);  // about 112+ CTAs on the 152 SMs
    }
    const dim3 grid(tiles, (N + bn - 1) / bn, splits);
    cudaError_t e;
    if (!am && !bnm)
      e = launch_tc<false, false>(a, bn, grid, s);
    else if (am && bnm)
      e = launch_tc<true, true>(a, bn, grid, s);
    else if (am)
      e = launch_tc<true, false>(a, bn, grid, s);
    else
      e = launch_tc<false, true>(a, bn, grid, s);
    mm->launches += 1;
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  GemmArgs g{M, N, K, A, lda, B, ldb, C, ldc, bias, atomic ? 1 : 0, K};
  int splits = 1;
  if (atomic) {  // split the batch reduction across blocks
    const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    splits = (K + 511) / 512;
    if (splits * tiles > 1024) splits = 1024 / tiles;
    if (splits < 1) splits = 1;
    g.k_split = ((K + splits - 1) / splits + BK - 1) / BK * BK;
    splits = (K + g.k_split - 1) / g.k_split;
  }
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN, splits);
  if (!am && !bnm)
    gemm_bf16_kernel<false, false><<<grid, 128, 0, s>>>(g);
  else if (am && bnm)
    gemm_bf16_kernel<true, true><<<grid, 128, 0, s>>>(g);
  else if (am)
    gemm_bf16_kernel<true, false><<<grid, 128, 0, s>>>(g);
  else
    gemm_bf16_kernel<false, true><<<grid, 128, 0, s>>>(g);
  mm->launches += 1;
  return cudaGetLastError();
}

const bf16* Wl(fehmm_mlp* m, int l) { return m->Wb + off_W(l); }
const bf16* WTl(fehmm_mlp* m, int l) { return m->WTb + (l == 1 ? 0 : NINP * W + (size_t)(l - 2) * W * W); }

void refresh(fehmm_mlp* m, cudaStream_t s) {
  refresh_bf16_kernel<<<blocks_for(N_PARAMS), 256, 0, s>>>(m->P, m->Wb);
  transpose_bf16_kernel<<<blocks_for(W * NINP), 256, 0, s>>>(m->P + OFF_W1, m->WTb, W, NINP, W);
  for (int l = 2; l <= 4; ++l)
    transpose_bf16_kernel<<<blocks_for(W * W), 256, 0, s>>>(m->P + off_W(l), const_cast<bf16*>(WTl(m, l)), W, W, W);
  m->launches += 5;
}

// forward + input gradient for B samples (x: device [B][6]); leaves Z, A, D, C, y, g8 set
int forward_grad(fehmm_mlp* m, const float* x, int B, cudaStream_t s) {
  const size_t nBW = (size_t)B * W;
  pack_x_kernel<<<blocks_for((size_t)B * NINP), 256, 0, s>>>(x, B, m->X);
  const bf16* a_prev = m->X;
  for (int l = 1; l <= 4; ++l) {
    gemm(m, false, false, B, W, fan_in(l), a_prev, fan_in(l), Wl(m, l), fan_in(l), m->Z[l], W, m->P + off_b(l),
         false, s);
    silu_kernel<<<blocks_for(nBW), 256, 0, s>>>(m->Z[l], nBW, m->A[l]);
    a_prev = m->A[l];
  }
  output_kernel<<<(B * 32 + 255) / 256, 256, 0, s>>>(m->A[4], m->Wb + OFF_W5, m->P + OFF_B5, B, m->y);
  d4_kernel<<<blocks_for(nBW), 256, 0, s>>>(m->Z[4], m->Wb + OFF_W5, B, m->D[4]);
  for (int l = 3; l >= 1; --l) {  // C_l = D_{l+1} W_{l+1}; D_l = C_l silu'(Z_l)
    gemm(m, false, false, B, W, W, m->D[l + 1], W, WTl(m, l + 1), W, m->Cc[l], W, nullptr, false, s);
    dmul_kernel<<<blocks_for(nBW), 256, 0, s>>>(m->Cc[l], m->Z[l], nBW, m->D[l]);
  }
  gemm(m, false, false, B, NINP, W, m->D[1], W, WTl(m, 1), W, m->g8, NINP, nullptr, false, s);
  m->launches += 3 + 2 * 3 + 1 + 4;
  return cudaGetLastError() == cudaSuccess ? FEHMM_OK : FEHMM_ERR_CUDA;
}

}  // namespace

extern "C" {

int fehmm_mlp_num_params(void) { return N_PARAMS; }

int fehmm_mlp_create(fehmm_mlp** out, int max_batch) {
  if (!out || max_batch <= 0) return FEHMM_ERR_ARG;
  *out = nullptr;
  fehmm_mlp* m = new (std::nothrow) fehmm_mlp();
  if (!m) return FEHMM_ERR_OOM;
  m->max_batch = max_batch;
  const size_t B = (size_t)max_batch, BW = B * W;
  int rc = FEHMM_OK;
  rc |= alloc(m, m->P, N_PARAMS);
  rc |= alloc(m, m->G, N_PARAMS);
  rc |= alloc(m, m->m, N_PARAMS);
  rc |= alloc(m, m->v, N_PARAMS);
  rc |= alloc(m, m->Wb, N_PARAMS);
  rc |= alloc(m, m->WTb, (size_t)NINP * W + 3 * (size_t)W * W);
  rc |= alloc(m, m->loss, 4);
  rc |= alloc(m, m->X, B * NINP);
  for (int l = 1; l <= 4; ++l) {
    rc |= alloc(m, m->Z[l], BW);
    rc |= alloc(m, m->A[l], BW);
    rc |= alloc(m, m->D[l], BW);
    rc |= alloc(m, m->QZ[l], BW);
    if (l <= 3) rc |= alloc(m, m->Cc[l], BW);
  }
  rc |= alloc(m, m->E, BW);
  rc |= alloc(m, m->ES, BW);
  rc |= alloc(m, m->T, 6 * BW);
  rc |= alloc(m, m->DZf, BW);
  rc |= alloc(m, m->DZ, BW);
  rc |= alloc(m, m->y, B);
  rc |= alloc(m, m->g8, B * NINP);
  rc |= alloc(m, m->ry, B);
  rc |= alloc(m, m->rg, B * NINP);
  for (int l = 1; l <= 4; ++l) rc |= alloc(m, m->ZD[l], 6 * BW);
  rc |= alloc(m, m->AD, 6 * BW);
  rc |= alloc(m, m->HK, 6 * B * NINP);
  rc |= alloc(m, m->err, 1);
  if (rc != FEHMM_OK) {
    for (void* p : m->allocs) cudaFree(p);
    delete m;
    return FEHMM_ERR_OOM;
  }
  cudaMemset(m->P, 0, sizeof(float) * N_PARAMS);
  cudaMemset(m->err, 0, sizeof(int));
  cudaMemset(m->m, 0, sizeof(float) * N_PARAMS);
  cudaMemset(m->v, 0, sizeof(float) * N_PARAMS);
  *out = m;
  return FEHMM_OK;
}

int fehmm_mlp_destroy(fehmm_mlp* m) {
  if (!m) return FEHMM_ERR_ARG;
  for (void* p : m->allocs) cudaFree(p);
  delete m;
  return FEHMM_OK;
}

int fehmm_mlp_set_params(fehmm_mlp* m, const float* host_params) {
  if (!m || !host_params) return FEHMM_ERR_ARG;
  if (cudaMemcpy(m->P, host_params, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice) != cudaSuccess)
    return FEHMM_ERR_CUDA;
  cudaMemset(m->m, 0, sizeof(float) * N_PARAMS);
  cudaMemset(m->v, 0, sizeof(float) * N_PARAMS);
  m->step = 0;
  refresh(m, 0);
  return cudaDeviceSynchronize() == cudaSuccess ? FEHMM_OK : FEHMM_ERR_CUDA;
}

int fehmm_mlp_get_params(fehmm_mlp* m, float* host_params, float* host_grad) {
  if (!m || (!host_params && !host_grad)) return FEHMM_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return FEHMM_ERR_CUDA;
  if (host_params && cudaMemcpy(host_params, m->P, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost) != cudaSuccess)
    return FEHMM_ERR_CUDA;
  if (host_grad && cudaMemcpy(host_grad, m->G, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost) != cudaSuccess)
    return FEHMM_ERR_CUDA;
  return FEHMM_OK;
}

int fehmm_mlp_eval(fehmm_mlp* m, const float* x, int B, float* y, float* g, float* H, void* stream) {
  if (!m || !x || B <= 0 || B > m->max_batch) return FEHMM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = forward_grad(m, x, B, s);
  if (rc != FEHMM_OK) return rc;
  const size_t nBW = (size_t)B * W, n6 = 6 * nBW;
  if (y && cudaMemcpyAsync(y, m->y, sizeof(float) * B, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return FEHMM_ERR_CUDA;
  if (g) copy_g_kernel<<<blocks_for((size_t)B * NIN), 256, 0, s>>>(m->g8, B, g);
  if (H) {  // forward mode over the reverse pass, the 6 directions stacked as 6B rows
    hess_init_kernel<<<blocks_for(n6), 256, 0, s>>>(m->Wb + OFF_W1, B, m->ZD[1]);
    for (int l = 1; l <= 3; ++l) {  // ZD_{l+1} = (silu'(Z_l) ZD_l) W_{l+1}^T
      hess_fwd_kernel<<<blocks_for(n6), 256, 0, s>>>(m->ZD[l], m->Z[l], B, m->AD);
      gemm(m, false, false, 6 * B, W, W, m->AD, W, Wl(m, l + 1), W, m->ZD[l + 1], W, nullptr, false, s);
    }
    hess_top_kernel<<<blocks_for(n6), 256, 0, s>>>(m->ZD[4], m->Z[4], m->Wb + OFF_W5, B, m->AD);
    for (int l = 3; l >= 1; --l) {  // DD_l = (DD_{l+1} W_{l+1}) silu'(Z_l) + C_l silu''(Z_l) ZD_l
      gemm(m, false, false, 6 * B, W, W, m->AD, W, WTl(m, l + 1), W, m->T, W, nullptr, false, s);
      hess_back_kernel<<<blocks_for(n6), 256, 0, s>>>(m->T, m->Z[l], m->Cc[l], m->ZD[l], B, m->AD);
    }
    gemm(m, false, false, 6 * B, NINP, W, m->AD, W, WTl(m, 1), W, m->HK, NINP, nullptr, false, s);
    hess_out_kernel<<<blocks_for((size_t)B * 36), 256, 0, s>>>(m->HK, B, H);
    m->launches += 1 + 3 + 1 + 3 + 1;
  }
  return cudaGetLastError() == cudaSuccess ? FEHMM_OK : FEHMM_ERR_CUDA;
}

int fehmm_mlp_loss_grad(fehmm_mlp* m, const float* x, const float* ty, const float* tg, int B, float cy, float cg,
                        float* loss_out, void* stream) {
  if (!m || !x || !ty || !tg || B <= 0 || B > m->max_batch) return FEHMM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = forward_grad(m, x, B, s);
  if (rc != FEHMM_OK) return rc;
  const size_t nBW = (size_t)B * W;
  cudaMemsetAsync(m->G, 0, sizeof(float) * N_PARAMS, s);
  cudaMemsetAsync(m->loss, 0, sizeof(float), s);
  residual_kernel<<<blocks_for(B), 256, 0, s>>>(m->y, m->g8, ty, tg, B, cy, cg, m->ry, m->rg, m->loss);
  // reverse through the input-gradient pass
  gemm(m, false, false, B, W, NINP, m->rg, NINP, Wl(m, 1), NINP, m->E, W, nullptr, false, s);     // E1 = rg W1^T
  gemm(m, true, true, W, NINP, B, m->D[1], W, m->rg, NINP, m->G + OFF_W1, NINP, nullptr, true, s);  // GW1 += D1^T rg
  for (int l = 1; l <= 3; ++l) {
    dbl_kernel<<<blocks_for(nBW), 256, 0, s>>>(m->E, m->Cc[l], m->Z[l], nBW, m->QZ[l], m->ES);
    gemm(m, true, true, W, W, B, m->D[l + 1], W, m->ES, W, m->G + off_W(l + 1), W, nullptr, true, s);  // GW_{l+1}
    gemm(m, false, false, B, W, W, m->ES, W, Wl(m, l + 1), W, m->E, W, nullptr, false, s);  // E_{l+1} = ES W^T
  }
  // d4 = w5 silu'(z4): gw5 += sum_b E4 silu'(Z4)
  {
    dim3 grid(1, 64);
    colsum_kernel<float><<<grid, W, 0, s>>>(m->E, m->Z[4], nullptr, B, W, m->G + OFF_W5, 1);
  }
  top_kernel<<<blocks_for(nBW), 256, 0, s>>>(m->E, m->Z[4], m->Wb + OFF_W5, m->ry, B, m->QZ[4], m->DZf, m->DZ);
  {
    dim3 grid(1, 64);
    colsum_kernel<bf16><<<grid, W, 0, s>>>(m->A[4], nullptr, m->ry, B, W, m->G + OFF_W5, 0);  // gw5 += A4^T ry
    colsum_kernel<float><<<dim3(1, 64), 1, 0, s>>>(m->ry, nullptr, nullptr, B, 1, m->G + OFF_B5, 0);
  }
  for (int l = 4; l >= 1; --l) {
    const bf16* a_prev = l == 1 ? m->X : m->A[l - 1];
    gemm(m, true, true, W, fan_in(l), B, m->DZ, W, a_prev, fan_in(l), m->G + off_W(l), fan_in(l), nullptr, true, s);
    colsum_kernel<float><<<dim3(1, 64), W, 0, s>>>(m->DZf, nullptr, nullptr, B, W, m->G + off_b(l), 0);
    if (l > 1) {
      gemm(m, false, false, B, W, W, m->DZ, W, WTl(m, l), W, m->T, W, nullptr, false, s);
      dz_kernel<<<blocks_for(nBW), 256, 0, s>>>(m->T, m->Z[l - 1], m->QZ[l - 1], nBW, m->DZf, m->DZ);
    }
  }
  if (loss_out && cudaMemcpyAsync(loss_out, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return FEHMM_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? FEHMM_OK : FEHMM_ERR_CUDA;
}

int fehmm_mlp_adamw(fehmm_mlp* m, float lr, float beta1, float beta2, float eps, float weight_decay, void* stream) {
  if (!m || !(lr > 0)) return FEHMM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  m->step += 1;
  const float bc1 = 1.f - powf(beta1, (float)m->step), bc2 = 1.f - powf(beta2, (float)m->step);
  adamw_kernel<<<blocks_for(N_PARAMS), 256, 0, s>>>(m->P, m->G, m->m, m->v, N_PARAMS, lr, beta1, beta2, eps,
                                                   weight_decay, bc1, bc2);
  refresh(m, s);
  return cudaGetLastError() == cudaSuccess ? FEHMM_OK : FEHMM_ERR_CUDA;
}

long long fehmm_mlp_launch_count(const fehmm_mlp* m) { return m ? m->launches : -1; }

int fehmm_mlp_check(fehmm_mlp* m, int* flag) {
  if (!m || !flag) return FEHMM_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return FEHMM_ERR_CUDA;
  if (cudaMemcpy(flag, m->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FEHMM_ERR_CUDA;
  if (*flag != 0 && cudaMemset(m->err, 0, sizeof(int)) != cudaSuccess) return FEHMM_ERR_CUDA;
  return FEHMM_OK;
}

int fehmm_mlp_grad_buffer(fehmm_mlp* m, float** dev_ptr, int* n) {
  if (!m || !dev_ptr) return FEHMM_ERR_ARG;
  *dev_ptr = m->G;
  if (n) *n = N_PARAMS;
  return FEHMM_OK;
}

// Surrogate file: magic, format version, parameter count, the packed FP32 parameters, then the
// fehmm_surrogate_params fields as little-endian doubles in declaration order (every double of
// the struct is written, so a load reproduces the evaluation exactly).
namespace {
constexpr char kMagic[8] = {'F', 'E', 'H', 'M', 'M', 'S', 'U', 'R'};
constexpr int32_t kFormat = 2;  // 2: with the polynomial part
constexpr size_t kSpDoubles = sizeof(fehmm_surrogate_params) / sizeof(double);
static_assert(sizeof(fehmm_surrogate_params) == kSpDoubles * sizeof(double), "surrogate params are all doubles");
}  // namespace

int fehmm_surrogate_save(fehmm_mlp* m, const fehmm_surrogate_params* sp, const char* path) {
  if (!m || !sp || !path) return FEHMM_ERR_ARG;
  std::vector<float> params(N_PARAMS);
  const int rc = fehmm_mlp_get_params(m, params.data(), nullptr);
  if (rc != FEHMM_OK) return rc;
  FILE* f = fopen(path, "wb");
  if (!f) return FEHMM_ERR_ARG;
  const int32_t np = N_PARAMS, nsp = (int32_t)kSpDoubles;
  bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(&kFormat, sizeof(kFormat), 1, f) == 1 &&
            fwrite(&np, sizeof(np), 1, f) == 1 && fwrite(&nsp, sizeof(nsp), 1, f) == 1 &&
            fwrite(params.data(), sizeof(float), N_PARAMS, f) == (size_t)N_PARAMS &&
            fwrite(sp, sizeof(double), kSpDoubles, f) == kSpDoubles;
  ok = (fclose(f) == 0) && ok;
  return ok ? FEHMM_OK : FEHMM_ERR_ARG;
}

int fehmm_surrogate_load(fehmm_mlp* m, fehmm_surrogate_params* sp, const char* path) {
  if (!m || !sp || !path) return FEHMM_ERR_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return FEHMM_ERR_ARG;
  char magic[8];
  int32_t fmt = 0, np = 0, nsp = 0;
  std::vector<float> params(N_PARAMS);
  fehmm_surrogate_params tmp;
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 && fread(&fmt, sizeof(fmt), 1, f) == 1 &&
            fmt == kFormat && fread(&np, sizeof(np), 1, f) == 1 && np == N_PARAMS &&
            fread(&nsp, sizeof(nsp), 1, f) == 1 && nsp == (int32_t)kSpDoubles &&
            fread(params.data(), sizeof(float), N_PARAMS, f) == (size_t)N_PARAMS &&
            fread(&tmp, sizeof(double), kSpDoubles, f) == kSpDoubles;
  fclose(f);
  if (!ok) return FEHMM_ERR_ARG;
  const int rc = fehmm_mlp_set_params(m, params.data());
  if (rc != FEHMM_OK) return rc;
  *sp = tmp;
  return FEHMM_OK;
}

}  // extern "C"
