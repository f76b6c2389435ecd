// Forward pass of the smoothed image-method objective: received power per
// receiver (Sec. V, Eq. 7) and the min-power loss (Eq. 8).
//
// Mapping on the GPU: the 32 lanes of a warp hold 32 receivers; the warp walks
// one path candidate at a time, so the candidate's wall sequence, its TX image
// chain and every branch are warp-uniform, and the walls are read from shared
// memory as broadcasts.  A work unit is (32 receivers) x (a chunk of
// candidates); the warps of a persistent grid take units from a counter (work
// stealing, next_unit_of) and write one partial sum per (chunk, receiver), which
// a second kernel adds up in chunk order.  The result is therefore deterministic
// whichever warp took which unit.
//
// Hot loop (obstruction, Sec. V-A with the comparison rule x0 > x1 -> s(x0 - x1)):
// for every wall, the smoothed side of each path vertex is computed once and
// shared by the two legs that meet there; each leg then needs only the sides of
// the wall's two end points w.r.t. the leg's line.
#include <cuda_runtime.h>

#include "drt_common.cuh"
#include "drt_internal.h"
#include "drt_path.cuh"
#include "drt_path_pair.cuh"

namespace drt {

namespace {

// GLOBAL: the wall records were written to a.staged by stage_global_kernel (scenes
// with more walls than shared memory holds) and are read through the L1 / L2
// caches instead of shared memory.  SAVE: every path's leg visibilities are also
// written to a.saved (for the sigmoid's adjoint).
template <int MODE, bool GLOBAL = false, bool SAVE = false>
__global__ void __launch_bounds__(256, MODE == MODE_SIGMOID ? 3 : 4) forward_kernel(const FwdArgs a) {
  extern __shared__ float4 smem[];
  float4* base = GLOBAL ? a.staged : smem;
  SmemWalls s{base, base + a.W, base + 2 * a.W, base + 3 * a.W};
  const float2 tx = make_float2(__ldg(a.tx), __ldg(a.tx + 1));
  if (!GLOBAL) stage_walls<MODE>(a.walls, a.W, tx, a.alpha, s);
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const long long warps_per_cta = blockDim.x >> 5;
  const long long nwarps = (long long)gridDim.x * warps_per_cta;
  for (long long u = (long long)blockIdx.x * warps_per_cta + (threadIdx.x >> 5); u < a.n_units;
       u = next_unit_of(a.unit_counter, u, nwarps, lane)) {
    const long long tile = u % a.n_tiles;
    const long long chunk = u / a.n_tiles;
    long long r = tile * 32 + lane;
    const bool live = r < a.R;
    if (!live) r = a.R - 1;
    const float2 q = __ldg(reinterpret_cast<const float2*>(a.rx) + r);
    // N_K < 2^31 for every supported (W, K): candidate indices fit in 32 bits
    const int c0 = (int)(chunk * a.chunk);
    const int nc = (int)(min(c0 + (long long)a.chunk, a.n_cand) - c0);
    float acc = 0.f;
    const bool masked = a.alpha > FAST_SKIP_MAX_ALPHA;
    float vbuf[KMAX + 1];   // the path's leg visibilities when they are saved
    float* vo = SAVE ? vbuf : nullptr;
    Cand cd = decode_candidate(c0, a.W, a.K);
    for (int i = 0; i < nc; ++i) {
      if (i > 0) next_candidate(cd, a.W);
      float p;
      if (vo) {
#pragma unroll
        for (int j = 0; j <= KMAX; ++j) vbuf[j] = 0.f;
      }
      if (!masked) {
        switch (cd.k) {
          case 0: p = path_power<MODE, 0>(s, a.W, tx, q, cd, a.alpha, a.gk[0], a.cull, vo); break;
          case 1: p = path_power<MODE, 1>(s, a.W, tx, q, cd, a.alpha, a.gk[1], a.cull, vo); break;
          case 2: p = path_power<MODE, 2>(s, a.W, tx, q, cd, a.alpha, a.gk[2], a.cull, vo); break;
          default: p = path_power<MODE, 3>(s, a.W, tx, q, cd, a.alpha, a.gk[3], a.cull, vo); break;
        }
      } else {
        switch (cd.k) {
          case 0: p = path_power<MODE, 0, true>(s, a.W, tx, q, cd, a.alpha, a.gk[0], a.cull, vo); break;
          case 1: p = path_power<MODE, 1, true>(s, a.W, tx, q, cd, a.alpha, a.gk[1], a.cull, vo); break;
          case 2: p = path_power<MODE, 2, true>(s, a.W, tx, q, cd, a.alpha, a.gk[2], a.cull, vo); break;
          default: p = path_power<MODE, 3, true>(s, a.W, tx, q, cd, a.alpha, a.gk[3], a.cull, vo); break;
        }
      }
      acc += p;
      if (vo && live) {   // [n_cand][K + 1][R]: consecutive lanes write consecutive floats
        float* dst = a.saved + (long long)(c0 + i) * (a.K + 1) * a.R + r;
        for (int j = 0; j <= cd.k; ++j) dst[j * a.R] = vbuf[j];
      }
    }
    if (live) a.partial[chunk * a.R + r] = acc;
  }
}

// Hard sigmoid and sigmoid, two receivers per lane (tiles of 64 receivers:
// lane l holds receivers l and l + 32 of its tile); the walls' paired records
// follow the four single-receiver arrays in shared memory.
// EXIT (hard sigmoid): the obstruction loop's exit for warps whose 64 paths are
// all blocked (DRT_TILE_EXIT_BLOCKED).
template <int MODE, bool GLOBAL = false, bool SAVE = false, bool EXIT = false>
__global__ void __launch_bounds__(256, 2) forward_pair_kernel(const FwdArgs a) {
  extern __shared__ float4 smem[];
  float4* base = GLOBAL ? a.staged : smem;
  SmemWalls s{base, base + a.W, base + 2 * a.W, base + 3 * a.W};
  SmemPairs pr{base + 4 * a.W, base + 5 * a.W, base + 6 * a.W, base + 7 * a.W};
  const float2 tx = make_float2(__ldg(a.tx), __ldg(a.tx + 1));
  if (!GLOBAL) {
    stage_walls<MODE>(a.walls, a.W, tx, a.alpha, s);
    __syncthreads();
    stage_pairs<MODE>(s, a.W, pr);
    __syncthreads();
  }

  const int lane = threadIdx.x & 31;
  const long long warps_per_cta = blockDim.x >> 5;
  const long long nwarps = (long long)gridDim.x * warps_per_cta;
  for (long long u = (long long)blockIdx.x * warps_per_cta + (threadIdx.x >> 5); u < a.n_units;
       u = next_unit_of(a.unit_counter, u, nwarps, lane)) {
    const long long tile = u % a.n_tiles;
    const long long chunk = u / a.n_tiles;
    const long long r0 = tile * 64 + lane, r1 = r0 + 32;
    const bool live0 = r0 < a.R, live1 = r1 < a.R;
    const float2 q0 = __ldg(reinterpret_cast<const float2*>(a.rx) + (live0 ? r0 : a.R - 1));
    const float2 q1 = __ldg(reinterpret_cast<const float2*>(a.rx) + (live1 ? r1 : a.R - 1));
    const int c0 = (int)(chunk * a.chunk);
    const int nc = (int)(min(c0 + (long long)a.chunk, a.n_cand) - c0);
    float acc0 = 0.f, acc1 = 0.f;
    float2 vbuf[KMAX + 1];   // the path's leg visibilities when they are saved
    float2* vo = SAVE ? vbuf : nullptr;
    Cand cd = decode_candidate(c0, a.W, a.K);
    for (int i = 0; i < nc; ++i) {
      if (i > 0) next_candidate(cd, a.W);
      float2 p;
      if (vo) {
#pragma unroll
        for (int j = 0; j <= KMAX; ++j) vbuf[j] = make_float2(0.f, 0.f);
      }
      switch (cd.k) {
        case 0: p = path_power_pair<MODE, 0, EXIT>(s, pr, a.W, tx, q0, q1, cd, a.alpha, a.gk[0], a.cull, vo); break;
        case 1: p = path_power_pair<MODE, 1, EXIT>(s, pr, a.W, tx, q0, q1, cd, a.alpha, a.gk[1], a.cull, vo); break;
        case 2: p = path_power_pair<MODE, 2, EXIT>(s, pr, a.W, tx, q0, q1, cd, a.alpha, a.gk[2], a.cull, vo); break;
        default: p = path_power_pair<MODE, 3, EXIT>(s, pr, a.W, tx, q0, q1, cd, a.alpha, a.gk[3], a.cull, vo); break;
      }
      acc0 += p.x;
      acc1 += p.y;
      if (vo) {   // [n_cand][K + 1][R]: consecutive lanes write consecutive floats
        float* dst = a.saved + (long long)(c0 + i) * (a.K + 1) * a.R;
        for (int j = 0; j <= cd.k; ++j) {
          if (live0) dst[j * a.R + r0] = vbuf[j].x;
          if (live1) dst[j * a.R + r1] = vbuf[j].y;
        }
      }
    }
    if (live0) a.partial[chunk * a.R + r0] = acc0;
    if (live1) a.partial[chunk * a.R + r1] = acc1;
  }
}

// Writes the wall records of forward_kernel / forward_pair_kernel (4 or 8
// float4 per wall, the shared-memory layout) to a global buffer, for scenes with
// more walls than shared memory holds.  One CTA: the records are a few float4 per
// wall, written once per launch.
template <int MODE>
__global__ void __launch_bounds__(1024) stage_global_kernel(const FwdArgs a) {
  float4* base = a.staged;
  SmemWalls s{base, base + a.W, base + 2 * a.W, base + 3 * a.W};
  const float2 tx = make_float2(__ldg(a.tx), __ldg(a.tx + 1));
  stage_walls<MODE>(a.walls, a.W, tx, a.alpha, s);
  if (a.pairs) {
    __syncthreads();   // the block's own global writes are visible to it after the barrier
    stage_pairs<MODE>(s, a.W, SmemPairs{base + 4 * a.W, base + 5 * a.W, base + 6 * a.W,
                                        base + 7 * a.W});
  }
}

// power[r] = sum over chunks of partial[chunk][r], in chunk order.
__global__ void reduce_chunks_kernel(const float* __restrict__ partial, long long n_chunks,
                                     long long R, float* __restrict__ power) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < R;
       r += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (long long c = 0; c < n_chunks; ++c) acc += partial[c * R + r];
    power[r] = acc;
  }
}

// loss = -min_r power[r], argmin = lowest index attaining it (Eq. 8, Sec. III).
__global__ void __launch_bounds__(1024) loss_kernel(const float* __restrict__ power, int R,
                                                    float* __restrict__ loss,
                                                    int32_t* __restrict__ argmin) {
  float best = INFINITY;
  int bi = 0x7fffffff;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const float v = power[r];
    if (v < best || (v == best && r < bi)) {
      best = v;
      bi = r;
    }
  }
  __shared__ float sv[32];
  __shared__ int si[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov < best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sv[wid] = best;
    si[wid] = bi;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    best = lane < nw ? sv[lane] : INFINITY;
    bi = lane < nw ? si[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov < best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      // every power is finite and >= 0 for validated input; bi < R always holds here
      loss[0] = -best;
      argmin[0] = bi < R ? bi : 0;
    }
  }
}

__global__ void loss_backward_kernel(const int32_t* __restrict__ argmin,
                                     const float* __restrict__ grad_loss, int R,
                                     float* __restrict__ grad_power) {
  const int am = argmin[0];
  const float g = grad_loss ? grad_loss[0] : 1.0f;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x)
    grad_power[r] = (r == am) ? -g : 0.f;
}

}  // namespace

size_t forward_smem_bytes(int W, bool pairs) { return (size_t)(pairs ? 8 : 4) * W * sizeof(float4); }

bool forward_streams_walls(int W) { return W > DRT_MAX_WALLS; }

bool forward_uses_pairs(int mode, float alpha, int flags) {
  return (mode == MODE_HARD || mode == MODE_SIGMOID) && !(alpha > FAST_SKIP_MAX_ALPHA) &&
         !(flags & DRT_TILE_SINGLE_RX);
}

cudaError_t launch_forward(const FwdArgs& a, int mode, int ctas, int threads, cudaStream_t st) {
  if (a.unit_counter && a.n_units > 0) {
    cudaError_t e = cudaMemsetAsync(a.unit_counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  if (forward_streams_walls(a.W)) {
    if (a.n_units > 0) {
      switch (mode) {
        case MODE_SIGMOID: stage_global_kernel<MODE_SIGMOID><<<1, 1024, 0, st>>>(a); break;
        case MODE_HARD: stage_global_kernel<MODE_HARD><<<1, 1024, 0, st>>>(a); break;
        default: stage_global_kernel<MODE_STEP><<<1, 1024, 0, st>>>(a); break;
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      if (a.pairs) {
        if (mode == MODE_SIGMOID)
          forward_pair_kernel<MODE_SIGMOID, true><<<ctas, threads, 0, st>>>(a);
        else if (a.exit_blocked)
          forward_pair_kernel<MODE_HARD, true, false, true><<<ctas, threads, 0, st>>>(a);
        else
          forward_pair_kernel<MODE_HARD, true><<<ctas, threads, 0, st>>>(a);
      } else {
        switch (mode) {
          case MODE_SIGMOID: forward_kernel<MODE_SIGMOID, true><<<ctas, threads, 0, st>>>(a); break;
          case MODE_HARD: forward_kernel<MODE_HARD, true><<<ctas, threads, 0, st>>>(a); break;
          default: forward_kernel<MODE_STEP, true><<<ctas, threads, 0, st>>>(a); break;
        }
      }
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return launch_reduce_chunks(a.partial, a.n_chunks, a.R, a.power, st);
  }
  const size_t smem = forward_smem_bytes(a.W, a.pairs);
  if (a.n_units > 0 && a.saved && mode == MODE_SIGMOID) {
    if (a.pairs)
      forward_pair_kernel<MODE_SIGMOID, false, true><<<ctas, threads, smem, st>>>(a);
    else
      forward_kernel<MODE_SIGMOID, false, true><<<ctas, threads, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else if (a.n_units > 0 && a.pairs) {
    if (mode == MODE_SIGMOID)
      forward_pair_kernel<MODE_SIGMOID><<<ctas, threads, smem, st>>>(a);
    else if (a.exit_blocked)
      forward_pair_kernel<MODE_HARD, false, false, true><<<ctas, threads, smem, st>>>(a);
    else
      forward_pair_kernel<MODE_HARD><<<ctas, threads, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else if (a.n_units > 0) {
    switch (mode) {
      case MODE_SIGMOID:
        forward_kernel<MODE_SIGMOID><<<ctas, threads, smem, st>>>(a);
        break;
      case MODE_HARD:
        forward_kernel<MODE_HARD><<<ctas, threads, smem, st>>>(a);
        break;
      default:
        forward_kernel<MODE_STEP><<<ctas, threads, smem, st>>>(a);
        break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (a.R > 0) {
    const long long nb = (a.R + 255) / 256;
    const int rb = (int)(nb < 4096 ? nb : 4096);
    reduce_chunks_kernel<<<rb, 256, 0, st>>>(a.partial, a.n_chunks, a.R, a.power);
  }
  return cudaGetLastError();
}

cudaError_t forward_occupancy(int mode, bool pairs, int threads, int W, int* ctas_per_sm) {
  if (forward_streams_walls(W)) {
    if (pairs)
      return mode == MODE_SIGMOID
                 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                       ctas_per_sm, forward_pair_kernel<MODE_SIGMOID, true>, threads, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                       ctas_per_sm, forward_pair_kernel<MODE_HARD, true>, threads, 0);
    switch (mode) {
      case MODE_SIGMOID:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            ctas_per_sm, forward_kernel<MODE_SIGMOID, true>, threads, 0);
      case MODE_HARD:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            ctas_per_sm, forward_kernel<MODE_HARD, true>, threads, 0);
      default:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            ctas_per_sm, forward_kernel<MODE_STEP, true>, threads, 0);
    }
  }
  const size_t smem = forward_smem_bytes(W, pairs);
  if (pairs)
    return mode == MODE_SIGMOID
               ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     ctas_per_sm, forward_pair_kernel<MODE_SIGMOID>, threads, smem)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     ctas_per_sm, forward_pair_kernel<MODE_HARD>, threads, smem);
  switch (mode) {
    case MODE_SIGMOID:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm,
                                                           forward_kernel<MODE_SIGMOID>, threads, smem);
    case MODE_HARD:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm,
                                                           forward_kernel<MODE_HARD>, threads, smem);
    default:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm,
                                                           forward_kernel<MODE_STEP>, threads, smem);
  }
}

cudaError_t forward_set_smem_limit(int W) {
  const int smem = (int)forward_smem_bytes(W, false);
  cudaError_t e;
  const int psmem = (int)forward_smem_bytes(W, true);
  e = cudaFuncSetAttribute(forward_pair_kernel<MODE_HARD>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(forward_pair_kernel<MODE_HARD, false, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(forward_pair_kernel<MODE_SIGMOID>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(forward_pair_kernel<MODE_SIGMOID, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(forward_kernel<MODE_SIGMOID>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(forward_kernel<MODE_SIGMOID, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(forward_kernel<MODE_HARD>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(forward_kernel<MODE_STEP>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_reduce_chunks(const float* partial, long long n_chunks, long long R,
                                 float* power, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  const long long nb = (R + 255) / 256;
  const int rb = (int)(nb < 4096 ? nb : 4096);
  reduce_chunks_kernel<<<rb, 256, 0, st>>>(partial, n_chunks, R, power);
  return cudaGetLastError();
}

cudaError_t launch_loss(const float* power, int R, float* loss, int32_t* argmin,
                        cudaStream_t st) {
  loss_kernel<<<1, 1024, 0, st>>>(power, R, loss, argmin);
  return cudaGetLastError();
}

cudaError_t launch_loss_backward(const int32_t* argmin, const float* grad_loss, int R,
                                 float* grad_power, cudaStream_t st) {
  const int b = (R + 255) / 256;
  loss_backward_kernel<<<b < 1024 ? (b > 0 ? b : 1) : 1024, 256, 0, st>>>(argmin, grad_loss, R,
                                                                          grad_power);
  return cudaGetLastError();
}

}  // namespace drt
