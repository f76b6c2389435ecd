// 5th-generation tensor-core (tcgen05) GEMM for the surrogate MLP on sm_103a:
// C[M x N] = A[M x K] . Bt[N x K]^T with BF16 operands and an FP32 accumulator
// in tensor memory (TMEM), the same three epilogues as the mma.sync kernel.
//
// One CTA (4 warps) computes a 128 x BN tile (BN = 64 or 256): it allocates BN
// TMEM columns, walks K in chunks of 64, copies the chunk of A (128 x 64) and
// of Bt (BN x 64) into shared memory in the canonical no-swizzle K-major layout
// (8-row x 16-byte core matrices; core matrices adjacent in K are 128 bytes
// apart, adjacent 8-row groups 1024 bytes apart), and one thread issues four
// tcgen05.mma (M = 128, N = BN, K = 16) and commits them to an mbarrier.  The
// wait on that mbarrier is bounded (0.5 s of %globaltimer): on timeout the
// kernel records an error code, and still waits (bounded) before it frees TMEM.  After the last chunk
// every thread reads its accumulator row (warp w owns TMEM lanes 32w..32w+31)
// with tcgen05.ld and runs the epilogue.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace drt {
namespace mlp {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;
constexpr unsigned long long TC_WAIT_NS = 500000000ull;   // give up waiting after 0.5 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of the tcgen05 family: start address,
// leading (K-direction) and stride (M/N-direction) byte offsets, descriptor
// version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = BN.
template <int BN>
__device__ __forceinline__ constexpr uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
}

// byte offset of element (r, k) of a [rows x 64] chunk in the core-matrix layout
__device__ __forceinline__ uint32_t tc_off(int r, int k) {
  return (uint32_t)((((r >> 3) * (TC_BK / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint64_t tc_now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Polls the mbarrier phase without blocking; gives up after TC_WAIT_NS.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase) {
  const uint64_t t0 = tc_now_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
    if (tc_now_ns() - t0 > TC_WAIT_NS) return false;
    __nanosleep(64);
  }
}

// skip_mma != 0 (test knob): no MMA and no commit is issued, so the bounded
// wait runs out with nothing in flight; the kernel must then report the
// timeout, skip its epilogue and still free its tensor memory.
template <int EPI, int BN>
__global__ void __launch_bounds__(128, 1) tc_gemm_nt_kernel(const GemmArgs g, int* status,
                                                            int skip_mma) {
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  uint8_t* sA = tc_smem;                                  // 128 x 64 bf16 = 16 KB
  uint8_t* sB = tc_smem + TC_BM * TC_BK * 2;              // BN x 64 bf16
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * BN;
  const uint32_t mbar_a = smem_u32(&mbar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t IDESC = tc_idesc<BN>();

  uint32_t phase = 0;
  const int n_chunks = g.K / TC_BK;
  for (int kc = 0; kc < n_chunks; ++kc) {
    const int k0 = kc * TC_BK;
    // A chunk: 128 rows x 8 pieces of 16 bytes; Bt chunk: BN rows x 8 pieces
    for (int i = tid; i < TC_BM * 8; i += 128) {
      const int r = i >> 3, c = (i & 7) * 8;
      const uint4 v = *reinterpret_cast<const uint4*>(g.A + (size_t)(m0 + r) * g.lda + k0 + c);
      *reinterpret_cast<uint4*>(sA + tc_off(r, c)) = v;
    }
    for (int i = tid; i < BN * 8; i += 128) {
      const int r = i >> 3, c = (i & 7) * 8;
      const uint4 v = *reinterpret_cast<const uint4*>(g.Bt + (size_t)(n0 + r) * g.ldb + k0 + c);
      *reinterpret_cast<uint4*>(sB + tc_off(r, c)) = v;
    }
    // make the generic-proxy stores visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && !skip_mma) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < TC_BK; kk += 16) {
        const uint64_t da = tc_smem_desc(smem_u32(sA) + kk * 16, 128, 1024);
        const uint64_t db = tc_smem_desc(smem_u32(sB) + kk * 16, 128, 1024);
        const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(IDESC), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              mbar_a)
          : "memory");
    }
    // every thread waits: the chunk buffers are reused by the next iteration
    if (!tc_wait(mbar_a, phase)) {
      s_fail = 1;
      if (status) atomicExch(status, 1);
    }
    __syncthreads();
    if (s_fail) break;   // `phase` stays the one still pending
    phase ^= 1u;
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (!s_fail) {
    const int row = m0 + tid;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(lane_addr + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = n0 + c0 + j;
        const float acc = __uint_as_float(v[j]);
        if (EPI == EPI_FWD) {
          const float z = acc + g.bias[col];
          if (g.Z) g.Z[(size_t)row * g.ldz + col] = z;
          const bf16 h = __float2bfloat16(z * sigm(z));
          g.H[(size_t)row * g.ldh + col] = h;
          if (g.HT) g.HT[(size_t)col * g.ldht + row] = h;
        } else if (EPI == EPI_DH) {
          const float zp = g.Z[(size_t)row * g.ldz + col];
          const float s = sigm(zp);
          const bf16 dz = __float2bfloat16(acc * s * (1.f + zp * (1.f - s)));
          g.H[(size_t)row * g.ldh + col] = dz;
          g.HT[(size_t)col * g.ldht + row] = dz;
        } else {
          g.C[(size_t)row * g.ldc + col] = acc;
        }
      }
    }
  } else if (!skip_mma) {
    // give an MMA that may still be running a last bounded chance to finish
    tc_wait(mbar_a, phase);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)BN)
                 : "memory");
  }
}

}  // namespace mlp
}  // namespace drt
