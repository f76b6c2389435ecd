// Fused inference pass of the surrogate MLP on the 5th-generation tensor cores
// (sm_103a): Fourier features, the four Linear(256) + SiLU layers and the
// Linear(1) output for 256 rows per CTA, with the activations kept on chip.
//
// Per CTA (one per SM, all 512 TMEM columns, 192 KB of shared memory): 256
// rows in two 128-row tiles, 16 epilogue warps (8 per tile: each row is shared
// by two threads, one per half of the 256 columns; warp w reads TMEM lanes
// 32 (w % 4) .. + 31 of accumulator w / 8) and one issuing warp:
//   * the epilogue warps compute the Fourier features into the activation
//     buffer (shared memory: per tile four 128 x 64 BF16 chunks in the
//     canonical no-swizzle K-major layout of the tcgen05 operands);
//   * each layer is, per tile, one 128 x 256 x K GEMM into that tile's 256 TMEM
//     columns.  The weights stream through a ring of four 16 KB shared-memory
//     stages in 256 x 32 chunks, stored pre-arranged in the operand layout in
//     global memory (the shadow's chunked copy), one bulk copy (cp.async.bulk,
//     completion on the stage's mbarrier with a byte count) per chunk;
//   * the tiles are software-pipelined: the issuing thread runs a layer's MMAs
//     for tile 0, then for tile 1, while the warps of tile 0 run that layer's
//     epilogue (the tensor pipe on one tile, the XU/FMA pipes on the other), so
//     each layer's weights stream once per tile.  Per tile, mbarriers carry the
//     hand-offs: "accumulator full" (an MMA commit) to the epilogue warps, and
//     "activations ready" (256 arrivals, two per row, after the BF16 rows are
//     in shared memory and the accumulator has been read) back to the issuing
//     thread; biases and w5 are staged in shared memory once per CTA;
//   * the epilogue reads its half row back (tcgen05.ld, 32 columns at a time), adds
//     the bias, applies SiLU z / (1 + 2^(-z log2 e)) (ex2.approx, rcp.approx),
//     rounds to BF16 and writes the row over the activation buffer as the next
//     layer's A operand; after the last layer it takes the dot product with w5
//     instead (the two halves meet through shared memory at a per-tile named
//     barrier), and only y leaves the chip.
// BF16 rounding points are those of the layer-by-layer path.  Every wait is
// bounded (TC_WAIT_NS) and also ends once another thread of the CTA has given
// up: the CTA then records an error code, drains its bulk copies and MMAs in
// flight (bounded) and frees its tensor memory.
#pragma once

#include "drt_mlp_tc.cuh"

namespace drt {
namespace mlp {

constexpr int FZ_TILE = 128;                        // rows per MMA (M), TMEM lanes
constexpr int FZ_TILES = 2;                         // row tiles per CTA
constexpr int FZ_ROWS = FZ_TILE * FZ_TILES;         // 256 rows
constexpr int FZ_EPI = 2 * FZ_ROWS;                 // epilogue threads: two per row
constexpr int FZ_THREADS = FZ_EPI + 32;             // + the issuing warp
constexpr int FZ_N = 256;                           // layer width = MMA N
constexpr int FZ_STAGES = 4;
constexpr int FZ_A_CHUNK = FZ_TILE * 64 * 2;        // 128 x 64 BF16
constexpr int FZ_A_TILE = 4 * FZ_A_CHUNK;           // 128 x 256 BF16
constexpr int FZ_A_BYTES = FZ_TILES * FZ_A_TILE;    // 128 KB
constexpr int FZ_W_STAGE = FZ_N * WCHUNK_K * 2;     // 16 KB
constexpr int FZ_SMEM = FZ_A_BYTES + FZ_STAGES * FZ_W_STAGE;   // 192 KB
constexpr int FZ_CHUNKS = (NFEAT + (NL - 1) * WID) / WCHUNK_K; // weight chunks of all layers
constexpr int FZ_SEQ = FZ_TILES * FZ_CHUNKS;        // chunk copies: each layer once per tile

// instruction descriptor: FP32 accumulator, BF16 A and B (K-major), M = 128, N = 256
__device__ __forceinline__ constexpr uint32_t fz_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(FZ_N >> 3) << 17) |
         ((uint32_t)(FZ_TILE >> 4) << 24);
}

// byte offset of element (r, k) of row tile t of the activation buffer
__device__ __forceinline__ uint32_t fz_aoff(int t, int r, int k) {
  return (uint32_t)(t * FZ_A_TILE + (k >> 6) * FZ_A_CHUNK) + tc_off(r, k & 63);
}

__device__ __forceinline__ float fz_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float fz_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

struct FusedArgs {
  const float* params;     // FP32 parameters (biases, b5)
  const bf16* shadow;      // BF16 weights: chunked W_l, w5
  const float* freqs;      // [32][2]
  const float* x;          // [batch][2]
  float* y;                // [batch]
  int batch;
  long long swc[NL], b[NL], sw5, b5;
};

// (layer, tile, K chunk) of entry q of the copy sequence: per layer, the
// layer's chunks for tile 0, then again for tile 1
__device__ __forceinline__ void fz_seq(int q, int& layer, int& tile, int& kc) {
  constexpr int C0 = NFEAT / WCHUNK_K, CL = WID / WCHUNK_K;
  if (q < FZ_TILES * C0) {
    layer = 0;
    tile = q / C0;
    kc = q % C0;
  } else {
    const int u = q - FZ_TILES * C0;
    layer = 1 + u / (FZ_TILES * CL);
    const int v = u % (FZ_TILES * CL);
    tile = v / CL;
    kc = v % CL;
  }
}

// bulk copy of the weight chunk of sequence entry q into stage st (issuing thread)
__device__ __forceinline__ void fz_issue_copy(const FusedArgs& a, int q, uint8_t* stage,
                                              uint64_t* full_st) {
  int l, t, kc;
  fz_seq(q, l, t, kc);
  const bf16* src = a.shadow + a.swc[l] + (long long)kc * FZ_N * WCHUNK_K;
  const uint32_t mb = smem_u32(full_st);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb),
               "r"((uint32_t)FZ_W_STAGE)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(smem_u32(stage)),
      "l"(src), "r"((uint32_t)FZ_W_STAGE), "r"(mb)
      : "memory");
}

// Bounded wait that also gives up once another thread has set *fail; a timeout
// sets *fail and the status flag.
__device__ __forceinline__ bool fz_wait(uint32_t mbar, uint32_t parity, volatile int* fail,
                                        int* status) {
  const uint64_t t0 = tc_now_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (*fail) return false;
    if (tc_now_ns() - t0 > TC_WAIT_NS) {
      *fail = 1;
      if (status) atomicExch(status, 1);
      return false;
    }
    __nanosleep(32);
  }
}

__global__ void __launch_bounds__(FZ_THREADS, 1) tc_mlp_forward_kernel(const FusedArgs a, int* status,
                                                                       int skip_mma) {
  extern __shared__ __align__(1024) uint8_t fz_smem[];
  __shared__ __align__(8) uint64_t full[FZ_STAGES], empt[FZ_STAGES];
  __shared__ __align__(8) uint64_t accf[FZ_TILES], actr[FZ_TILES];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  __shared__ __align__(16) float s_bias[NL][FZ_N];
  __shared__ float s_w5[FZ_N];
  __shared__ float s_y[FZ_ROWS];
  volatile int* fail = &s_fail;
  uint8_t* sA = fz_smem;
  uint8_t* sW = fz_smem + FZ_A_BYTES;
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool issuer_warp = tid >= FZ_EPI;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"((uint32_t)(FZ_TILES * FZ_N))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  int issued = 0;   // issuing thread: chunk copies issued
  // biases and output weights, read by every epilogue thread, into shared memory
  for (int i = tid; i < NL * FZ_N; i += FZ_THREADS)
    s_bias[i / FZ_N][i % FZ_N] = a.params[a.b[i / FZ_N] + i % FZ_N];
  for (int i = tid; i < FZ_N; i += FZ_THREADS) s_w5[i] = __bfloat162float(a.shadow[a.sw5 + i]);
  if (tid == FZ_EPI) {
    s_fail = 0;
    for (int s = 0; s < FZ_STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empt[s])) : "memory");
    }
    for (int t = 0; t < FZ_TILES; ++t) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&accf[t])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&actr[t])),
                   "r"(2 * FZ_TILE)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    // the first chunks arrive while the features are computed
    for (; issued < FZ_STAGES; ++issued)
      fz_issue_copy(a, issued, sW + issued * FZ_W_STAGE, &full[issued]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t IDESC = fz_idesc();

  if (issuer_warp) {
    if (tid == FZ_EPI) {
      // ------------------------------------------------ issuing thread
      int q = 0, last_committed = -1;
      for (int l = 0; l < NL && !*fail; ++l) {
        const int n_chunks = (l == 0 ? NFEAT : WID) / WCHUNK_K;
        for (int t = 0; t < FZ_TILES && !*fail; ++t) {
          // the tile's activations for this layer are in shared memory and its
          // accumulator has been read out
          if (!fz_wait(smem_u32(&actr[t]), l & 1, fail, status)) break;
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          for (int kc = 0; kc < n_chunks; ++kc, ++q) {
            const int st = q % FZ_STAGES;
            if (!fz_wait(smem_u32(&full[st]), (q / FZ_STAGES) & 1, fail, status)) break;
            if (skip_mma) {   // test knob: nothing is multiplied, the stage is never released
              *fail = 1;
              if (status) atomicExch(status, 1);
              ++q;
              break;
            }
            const uint32_t wst = smem_u32(sW + st * FZ_W_STAGE);
#pragma unroll
            for (int kk = 0; kk < WCHUNK_K; kk += 16) {
              const int k = kc * WCHUNK_K + kk;
              const uint64_t da = tc_smem_desc(
                  smem_u32(sA) + t * FZ_A_TILE + (k >> 6) * FZ_A_CHUNK + (k & 63) * 16, 128, 1024);
              const uint64_t db = tc_smem_desc(wst + kk * 16, 128, 512);
              const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                      tmem + (uint32_t)(t * FZ_N)),
                  "l"(da), "l"(db), "r"(IDESC), "r"(acc)
                  : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(&empt[st]))
                : "memory");
            last_committed = q;
            // refill the previous entry's stage once its MMAs are done
            const int prev = q - 1;
            if (prev >= 0 && issued < FZ_SEQ && issued == prev + FZ_STAGES) {
              const int ps = prev % FZ_STAGES;
              if (!fz_wait(smem_u32(&empt[ps]), (prev / FZ_STAGES) & 1, fail, status)) {
                ++q;
                break;
              }
              fz_issue_copy(a, issued, sW + ps * FZ_W_STAGE, &full[ps]);
              ++issued;
            }
          }
          if (*fail) break;
          // the tile's accumulator is complete once these MMAs are
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                  smem_u32(&accf[t]))
              : "memory");
        }
      }
      if (*fail) {
        // let what is still in flight land before the memory is released:
        // the copies not yet consumed, then the last committed MMAs
        for (int c = q; c < issued; ++c)
          tc_wait(smem_u32(&full[c % FZ_STAGES]), (c / FZ_STAGES) & 1);
        if (last_committed >= 0)
          tc_wait(smem_u32(&empt[last_committed % FZ_STAGES]), (last_committed / FZ_STAGES) & 1);
      }
    }
  } else {
    // ------------------------------------------------ epilogue warps
    const int tile = warp >> 3, half = (warp >> 2) & 1;
    const int r = (warp & 3) * 32 + (tid & 31);
    const int row = blockIdx.x * FZ_ROWS + tile * FZ_TILE + r;
    const bool live = row < a.batch;
    const uint32_t row_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                              (uint32_t)(tile * FZ_N + half * (FZ_N / 2));
    const uint32_t actr_t = smem_u32(&actr[tile]);
    // Fourier features of this thread's row (its half of the frequencies) into
    // the first K chunk of its tile
    {
      const float x0 = live ? a.x[2 * row] : 0.f, x1 = live ? a.x[2 * row + 1] : 0.f;
#pragma unroll 1
      for (int j0 = half * (NFREQ / 2); j0 < (half + 1) * (NFREQ / 2); j0 += 8) {
        float s[8], c[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = j0 + q;
          const float v = 2.f * fmaf(a.freqs[2 * j], x0, a.freqs[2 * j + 1] * x1);
          sincospif(v, &s[q], &c[q]);
        }
        uint4 ps, pc;
        ps.x = pack_bf16x2(s[0], s[1]);
        ps.y = pack_bf16x2(s[2], s[3]);
        ps.z = pack_bf16x2(s[4], s[5]);
        ps.w = pack_bf16x2(s[6], s[7]);
        pc.x = pack_bf16x2(c[0], c[1]);
        pc.y = pack_bf16x2(c[2], c[3]);
        pc.z = pack_bf16x2(c[4], c[5]);
        pc.w = pack_bf16x2(c[6], c[7]);
        *reinterpret_cast<uint4*>(sA + fz_aoff(tile, r, j0)) = ps;
        *reinterpret_cast<uint4*>(sA + fz_aoff(tile, r, NFREQ + j0)) = pc;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(actr_t) : "memory");
    float yacc = 0.f;
    bool ok = true;
    for (int l = 0; l < NL; ++l) {
      if (!fz_wait(smem_u32(&accf[tile]), l & 1, fail, status)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      // z = acc + bias, h = SiLU(z) in BF16 -> next layer's A (or the output dot)
      const float* bias = s_bias[l];
#pragma unroll 1
      for (int cc = 0; cc < FZ_N / 2; cc += 32) {
        const int c0 = half * (FZ_N / 2) + cc;
        uint32_t v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
              "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
              "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
              "=r"(v[31])
            : "r"(row_addr + (uint32_t)cc));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        float h[32];
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const float4 b4 = *reinterpret_cast<const float4*>(bias + c0 + j);
          const float bb[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            // SiLU: z / (1 + 2^(-z log2 e)); the reciprocal of +inf is +0
            const float z = __uint_as_float(v[j + q]) + bb[q];
            h[j + q] = z * fz_rcp(1.f + fz_ex2(-1.4426950408889634f * z));
          }
        }
        if (l + 1 < NL) {
#pragma unroll
          for (int q = 0; q < 32; q += 8) {
            uint4 p;
            p.x = pack_bf16x2(h[q], h[q + 1]);
            p.y = pack_bf16x2(h[q + 2], h[q + 3]);
            p.z = pack_bf16x2(h[q + 4], h[q + 5]);
            p.w = pack_bf16x2(h[q + 6], h[q + 7]);
            *reinterpret_cast<uint4*>(sA + fz_aoff(tile, r, c0 + q)) = p;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            yacc = fmaf(__bfloat162float(__float2bfloat16(h[j])), s_w5[c0 + j], yacc);
        }
      }
      if (l + 1 < NL) {
        // hand the new activations (and the read-out accumulator) to the MMAs
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(actr_t) : "memory");
      }
    }
    // the two halves of each row's output dot product (the tile's 8 warps meet at
    // a named barrier; the bounded waits above end on every thread alike)
    if (half == 1) s_y[tile * FZ_TILE + r] = yacc;
    asm volatile("bar.sync %0, %1;\n" ::"r"(1 + tile), "r"(2 * FZ_TILE) : "memory");
    if (half == 0 && ok && !*fail && live)
      a.y[row] = (yacc + s_y[tile * FZ_TILE + r]) + a.params[a.b5];
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)(FZ_TILES * FZ_N))
                 : "memory");
  }
}

}  // namespace mlp
}  // namespace drt
