// 5th-generation tensor-core (tcgen05) GEMM for the surrogate MLP on sm_103a:
// C[M x N] = A[M x K] . Bt[N x K]^T with BF16 operands and an FP32 accumulator
// in tensor memory (TMEM), the same three epilogues as the mma.sync kernel.
//
// One CTA (4 warps) computes a 128 x BN tile (BN = 64 or 128): it allocates BN
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
//
// Pipeline: two shared-memory stages; the copy of chunk k+1 overlaps the MMAs of
// chunk k, and a stage is refilled only after the commit of the MMAs that read it.
// Epilogue: the accumulator goes TMEM -> registers (tcgen05.ld, one row per
// thread) -> a shared-memory tile, from which the outputs are written with
// consecutive threads on consecutive columns (row-major outputs) or rows (the
// transposed copy), i.e. coalesced.
template <int BN>
struct TcSmem {
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;
  static constexpr int B_BYTES = BN * TC_BK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int TILE_LD = BN + 1;   // padded row of the FP32 tile
  static constexpr int TILE = TC_BM * TILE_LD * 4;
  static constexpr int BYTES = (2 * STAGE > TILE ? 2 * STAGE : TILE);
};

template <int EPI, int BN>
__global__ void __launch_bounds__(128, 1) tc_gemm_nt_kernel(const GemmArgs g, int* status,
                                                            int skip_mma) {
  using SM = TcSmem<BN>;
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * BN;
  const uint32_t mb0 = smem_u32(&mbar[0]), mb1 = smem_u32(&mbar[1]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    s_fail = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t IDESC = tc_idesc<BN>();

  const int kz = g.K / (g.k_splits > 0 ? g.k_splits : 1);   // this CTA's K slice (split-K)
  const int kbase = blockIdx.z * kz;
  const int n_chunks = kz / TC_BK;
  int last_issued = -1;
  for (int kc = 0; kc < n_chunks; ++kc) {
    const int st = kc & 1;
    const uint32_t mb = st ? mb1 : mb0;
    uint8_t* sA = tc_smem + st * SM::STAGE;
    uint8_t* sB = sA + SM::A_BYTES;
    if (kc >= 2) {
      // the MMAs of chunk kc-2 read this stage: wait for their commit
      if (!tc_wait(mb, ((kc - 2) >> 1) & 1)) {
        s_fail = 1;
        if (status) atomicExch(status, 1);
      }
      __syncthreads();
      if (s_fail) break;
    }
    const int k0 = kbase + kc * TC_BK;
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
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb)
          : "memory");
    }
    last_issued = kc;
  }
  // the last commit covers every MMA issued before it
  if (!s_fail && last_issued >= 0) {
    const uint32_t mb = (last_issued & 1) ? mb1 : mb0;
    if (!tc_wait(mb, (last_issued >> 1) & 1)) {
      s_fail = 1;
      if (status) atomicExch(status, 1);
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

  if (!s_fail) {
    float* tile = reinterpret_cast<float*>(tc_smem);   // [128][BN + 1], the stages are free now
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
      for (int j = 0; j < 16; ++j) tile[tid * SM::TILE_LD + c0 + j] = __uint_as_float(v[j]);
    }
    __syncthreads();
    // row-major outputs: consecutive threads on consecutive columns
    for (int idx = tid; idx < TC_BM * BN; idx += 128) {
      const int r = idx / BN, c = idx % BN;
      const int row = m0 + r, col = n0 + c;
      const float acc = tile[r * SM::TILE_LD + c];
      if (EPI == EPI_FWD) {
        const float z = acc + g.bias[col];
        if (g.Z) g.Z[(size_t)row * g.ldz + col] = z;
        const float h = z * sigm(z);
        g.H[(size_t)row * g.ldh + col] = __float2bfloat16(h);
        tile[r * SM::TILE_LD + c] = h;
      } else if (EPI == EPI_DH) {
        const float zp = g.Z[(size_t)row * g.ldz + col];
        const float s = sigm(zp);
        const float dz = acc * s * (1.f + zp * (1.f - s));
        g.H[(size_t)row * g.ldh + col] = __float2bfloat16(dz);
        tile[r * SM::TILE_LD + c] = dz;
      } else {
        g.C[(size_t)blockIdx.z * g.M * g.ldc + (size_t)row * g.ldc + col] = acc;
      }
    }
    if (EPI != EPI_DW && g.HT) {
      __syncthreads();
      // transposed copy: consecutive threads on consecutive rows
      for (int idx = tid; idx < TC_BM * BN; idx += 128) {
        const int c = idx / TC_BM, r = idx % TC_BM;
        g.HT[(size_t)(n0 + c) * g.ldht + m0 + r] = __float2bfloat16(tile[r * SM::TILE_LD + c]);
      }
    }
  } else if (!skip_mma && last_issued >= 0) {
    // give MMAs that may still be running a last bounded chance to finish
    tc_wait((last_issued & 1) ? mb1 : mb0, (last_issued >> 1) & 1);
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
