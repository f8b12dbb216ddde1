// BF16 x BF16 -> FP32 matrix product on the 5th-generation tensor cores (tcgen05.mma, accumulator
// in tensor memory), for the surrogate network's 128-wide layers.
//
//   C[m][n] (+)= sum_k A(m,k) B(k,n),  m < M, n < N <= 128, k in [kb, ke)
//   A(m,k) = AM ? A[k*lda + m] : A[m*lda + k];  B(k,n) = BNM ? B[k*ldb + n] : B[n*ldb + k]
//
// One CTA of 128 threads per 128-row x BN-column tile of C (BN = 32, 64 or 128, chosen so that
// small products still fill the GPU) and K slice (blockIdx.z; split-K with FP32 atomics).  K is
// walked in chunks of 64 through two shared-memory stages: the chunk of A (128 x 64) and B
// (BN x 64) is staged in the canonical K-major layout without swizzle (8-row x 16-byte core
// matrices, the two core matrices along K of one MMA 128 bytes apart, 8-row groups 1024 bytes
// apart).  K-contiguous operands go straight to shared memory with cp.async (16-byte pieces of a
// row, zero-filled outside the matrix); operands stored M- or N-major in global memory are
// transposed in registers (8 x 8 blocks) on the way.  Both stages are loaded up front; one thread
// issues four 128 x BN x 16 MMAs per chunk and commits them to the stage's mbarrier, whose
// completion releases the stage for the chunk after next.  The epilogue reads the 128 x BN FP32
// accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows), adds the bias and
// stores (or atomically adds) the rows.
//
// Every mbarrier wait is bounded (about 2 s of SM clock); a wait that runs out sets *err = 1,
// the CTA stops issuing work, frees its tensor memory and returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fehmm {
namespace tc {

constexpr int kBM = 128, kBNMax = 128, kBK = 64;
constexpr int kATileBytes = kBM * kBK * 2;  // one A chunk: 16 KB
constexpr int kStages = 2;
constexpr uint32_t kCoreBytes = 128;        // 8 rows x 16 bytes
constexpr uint32_t kLBO = kCoreBytes;       // next core matrix along K
constexpr uint32_t kSBO = (kBK / 8) * kCoreBytes;  // next 8-row group: 1024 bytes
constexpr long long kWaitCycles = 1ll << 32;

template <int BN>
struct Cfg {
  static_assert(BN == 32 || BN == 64 || BN == 128, "tile width");
  static constexpr int kBTileBytes = BN * kBK * 2;
  static constexpr int kStageBytes = kATileBytes + kBTileBytes;
  static constexpr int kSmemBytes = kStages * kStageBytes + 64;  // + mbarriers and the TMEM slot
  static constexpr uint32_t kTmemCols = BN;                        // FP32 accumulator 128 x BN
};

struct Args {
  int M, N, K;
  const __nv_bfloat16* A;
  int lda;
  const __nv_bfloat16* B;
  int ldb;
  float* C;
  int ldc;
  const float* bias;  // per column, or null
  int atomic;
  int k_split;        // K range per blockIdx.z, a multiple of kBK
  int* err;
};

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading-dimension byte offset
// >> 4 (bits 16-29), stride-dimension byte offset >> 4 (bits 32-45), the fixed value 1 at bit 46,
// base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(kSBO >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 16 bytes global -> shared, the bytes past src_bytes (0 or 16) zero-filled
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 8 x 8 transpose of 16-bit elements: in[k] holds row k (8 values along m); out[m] holds column m
// (8 values along k).  Word j of out[m] = (in[2j][m], in[2j+1][m]).
__device__ __forceinline__ void transpose8x8(const uint4 (&in)[8], uint4 (&out)[8]) {
  const uint32_t* w[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) w[k] = reinterpret_cast<const uint32_t*>(&in[k]);
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const uint32_t sel = (m & 1) ? 0x7632u : 0x5410u;
    uint32_t o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = __byte_perm(w[2 * j][m >> 1], w[2 * j + 1][m >> 1], sel);
    out[m] = make_uint4(o[0], o[1], o[2], o[3]);
  }
}

union Pack8 {
  uint4 v;
  __nv_bfloat16 e[8];
};

// Stage rows [r0, r0 + ROWS) x k [k0, k0 + 64) of an operand into the K-major core-matrix layout
// at S; entries outside rows < R, k < kend are zero.  MN: the source is stored [k][ld] (rows
// contiguous), else [row][ld] (k contiguous; cp.async where a piece is 16-byte aligned and whole
// or empty).
template <bool MN, int ROWS>
__device__ __forceinline__ void stage(uint8_t* S, const __nv_bfloat16* src, int ld, int r0, int R, int k0, int kend) {
  const int t = threadIdx.x;
  if constexpr (!MN) {
    const bool vec_ok = (ld % 8) == 0 && (k0 % 8) == 0 && ((uintptr_t)src % 16) == 0;
#pragma unroll
    for (int i = 0; i < ROWS / 16; ++i) {
      const int c = t + i * 128;
      const int r8 = c & 7, kg = (c >> 3) & 7, rg = c >> 6;
      const int row = r0 + rg * 8 + r8, k = k0 + kg * 8;
      uint8_t* dst = S + rg * kSBO + kg * kLBO + r8 * 16;
      const bool none = row >= R || k >= kend;
      const __nv_bfloat16* p = src + (size_t)row * ld + k;
      if (vec_ok && (none || k + 8 <= kend)) {
        cp_async16(smem_u32(dst), none ? (const void*)src : (const void*)p, none ? 0u : 16u);
      } else {
        Pack8 u;
#pragma unroll
        for (int j = 0; j < 8; ++j) u.e[j] = (!none && k + j < kend) ? p[j] : __float2bfloat16(0.f);
        *reinterpret_cast<uint4*>(dst) = u.v;
      }
    }
  } else {
    const bool vec_ok = (ld % 8) == 0 && (r0 % 8) == 0 && ((uintptr_t)src % 16) == 0;
    if (t < ROWS) {  // ROWS / 8 row blocks x 8 k blocks of 8 x 8
      const int kb = t & 7, rb = t >> 3;
      const int row = r0 + rb * 8;
      uint4 in[8];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const int k = k0 + kb * 8 + kk;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (k < kend && row < R) {
          const __nv_bfloat16* p = src + (size_t)k * ld + row;
          if (vec_ok && row + 8 <= R) {
            v = *reinterpret_cast<const uint4*>(p);
          } else {
            Pack8 u;
#pragma unroll
            for (int j = 0; j < 8; ++j) u.e[j] = (row + j < R) ? p[j] : __float2bfloat16(0.f);
            v = u.v;
          }
        }
        in[kk] = v;
      }
      uint4 out[8];
      transpose8x8(in, out);
#pragma unroll
      for (int m = 0; m < 8; ++m) *reinterpret_cast<uint4*>(S + rb * kSBO + kb * kLBO + m * 16) = out[m];
    }
  }
}

template <bool AM, bool BNM, int BN>
__global__ void __launch_bounds__(128) gemm_tc_kernel(const Args g) {
  using C = Cfg<BN>;
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * C::kStageBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kStages * C::kStageBytes + 32);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int kb = blockIdx.z * g.k_split, ke = min(g.K, kb + g.k_split);
  const int nch = ke > kb ? (ke - kb + kBK - 1) / kBK : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&bars[s]));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(C::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = idesc_bf16_f32(kBM, BN);

  // stage chunk c into buffer c & 1 (one cp.async group per chunk and thread)
  auto load_chunk = [&](int c) {
    uint8_t* SA = smem + (c & 1) * C::kStageBytes;
    const int k0 = kb + c * kBK;
    stage<AM, kBM>(SA, g.A, g.lda, m0, g.M, k0, ke);
    stage<BNM, BN>(SA + kATileBytes, g.B, g.ldb, n0, g.N, k0, ke);
    cp_async_commit();
  };
  if (nch > 0) load_chunk(0);
  if (nch > 1) load_chunk(1);
  bool failed = false;
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch)
      cp_async_wait<1>();  // chunk c landed (c + 1 may still be in flight)
    else
      cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    const int s = c & 1;
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(smem + s * C::kStageBytes), b0 = a0 + kATileBytes;
#pragma unroll
      for (int j = 0; j < kBK / 16; ++j)  // K = 16 per MMA: two core matrices along K
        mma_bf16(tmem, smem_desc(a0 + j * 2 * kLBO), smem_desc(b0 + j * 2 * kLBO), idesc, (c > 0 || j > 0) ? 1u : 0u);
      mma_commit(smem_u32(&bars[s]));
    }
    if (c + 2 < nch) {  // the stage is free once the MMAs of chunk c have read it
      failed = !mbar_wait(smem_u32(&bars[s]), (c >> 1) & 1);
      if (!failed) load_chunk(c + 2);
    }
  }
  cp_async_wait<0>();
  if (!failed && nch > 0) {
    const int last = nch - 1;
    failed = !mbar_wait(smem_u32(&bars[last & 1]), (last >> 1) & 1);
  }
  failed = __syncthreads_or(failed);
  if (failed) {
    if (threadIdx.x == 0 && g.err) atomicExch(g.err, 1);
  } else if (nch > 0 || !g.atomic) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int r = m0 + warp * 32 + lane;
    const bool vec = !g.atomic && n0 + BN <= g.N && (g.ldc % 4) == 0 && ((uintptr_t)g.C % 16) == 0;
#pragma unroll
    for (int cc = 0; cc < BN / 32; ++cc) {
      uint32_t v[32];
      if (nch > 0) {
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
              "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
              "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0u;
      }
      if (r < g.M) {
        const int c0 = n0 + cc * 32;
        float* dst = g.C + (size_t)r * g.ldc + c0;
        if (vec) {
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            float4 o = make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]), __uint_as_float(v[j + 2]),
                                   __uint_as_float(v[j + 3]));
            if (g.bias) {
              o.x += g.bias[c0 + j];
              o.y += g.bias[c0 + j + 1];
              o.z += g.bias[c0 + j + 2];
              o.w += g.bias[c0 + j + 3];
            }
            *reinterpret_cast<float4*>(dst + j) = o;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = c0 + j;
            if (col >= g.N) continue;
            float o = __uint_as_float(v[j]);
            if (g.atomic) {
              atomicAdd(dst + j, o);
            } else {
              if (g.bias) o += g.bias[col];
              dst[j] = o;
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kTmemCols) : "memory");
  }
}

}  // namespace tc
}  // namespace fehmm
