// Coherent field per receiver: Eq. 7 read as a sum of complex path fields,
//   E_r = sum over candidates of  prod_j C_j * V * vis * exp(-2 pi i L / lambda) / L,
// with the field normal to the scene plane, C_j the Fresnel reflection
// coefficient for that polarisation (TE) at the angle of incidence of the leg
// arriving at reflection j, or a constant amplitude coefficient, and the
// coherent power |E_r|^2.
//
// The geometry, validity and obstruction of each (receiver, candidate) are the
// forward pass's (path_geometry, leg_visibility): the obstruction loop is the
// cost and is unchanged.  Only the per-path epilogue differs: it recomputes the
// path length with correctly rounded leg lengths (the phase 2 pi L / lambda
// magnifies any error in L by L / lambda), takes 1/lambda as a float pair so
// the cycle count's only rounding is L's own, and reduces the cycle count to
// [-1/2, 1/2] before sincospi.  Work decomposition, determinism and the chunk
// reduction follow drt_forward.cu with (re, im) partial sums, including its two
// receivers per lane (packed FP32 obstruction loop) for the hard sigmoid and the
// sigmoid at alpha <= 1e4; the visibilities are the same, bit for bit, either way.
#include <cuda_runtime.h>

#include "drt_common.cuh"
#include "drt_internal.h"
#include "drt_path.cuh"
#include "drt_path_pair.cuh"

namespace drt {

namespace {

// Field (re, im) of one path from its geometry and its legs' visibilities.
template <int MODE, int K>
__device__ __forceinline__ float2 field_of_path(const SmemWalls& s, const FieldArgs& a,
                                                const PathGeom<MODE, K>& g, const float* vis,
                                                const Cand& cd) {
  // Only L needs correctly rounded arithmetic (the phase); the amplitude's factors
  // take the approximate reciprocal square root and division (a few ulps each,
  // far inside the amplitude's tolerance).
  float L = 0.f, coef = 1.f, amp = g.V;
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    const float dx = g.Qx[j + 1] - g.Qx[j], dy = g.Qy[j + 1] - g.Qy[j];
    const float len2 = fmaf(dx, dx, dy * dy);
    L += __fsqrt_rn(len2);
    amp *= vis[j];
    if (j < K) {
      // leg j arrives at reflection j + 1 on wall w_{j+1}: cosine of incidence
      // |n . d| / |d| with n the wall's unit normal
      const float4 G = s.G[cd.w[j]];
      const float c = fminf(fabsf(fmaf(G.x, dx, G.y * dy)) * rsqrtf(len2), 1.f);
      float r = a.refl_amp;
      if (a.eps_r > 0.f) {
        const float x = fmaf(c, c, a.eps_r - 1.f);
        const float root = x > 0.f ? x * rsqrtf(x) : 0.f;
        const float den = c + root;
        r = den > 0.f ? __fdividef(c - root, den) : 0.f;   // den >= sqrt(eps_r - 1) > 0
      }
      coef *= r;
    }
  }
  // cycles L / lambda = L * (hi + lo): the product's rounding error is recovered
  // by an FMA, so the fractional part carries only L's own error
  const float p = L * a.inv_lambda_hi;
  const float e = fmaf(L, a.inv_lambda_hi, -p);
  const float frac = (p - rintf(p)) + fmaf(L, a.inv_lambda_lo, e);
  float sn, cs;
  sincospif(2.f * frac, &sn, &cs);
  const float m = __fdividef(amp * coef, L);
  return g.degenerate ? make_float2(0.f, 0.f) : make_float2(m * cs, -m * sn);
}

// Field of one path candidate of order K for this lane's receiver.
template <int MODE, int K, bool MASKED>
__device__ __forceinline__ float2 path_field(const SmemWalls& s, const FieldArgs& a, float2 tx,
                                             float2 rx, const Cand& cd,
                                             float* vis_out = nullptr) {
  float Ix[K + 1], Iy[K + 1];
  tx_images<K>(s, tx, cd, Ix, Iy);
  PathGeom<MODE, K> g;
  path_geometry<MODE, K>(s, Ix, Iy, tx, rx, cd, a.alpha, g);
  if (a.cull && __all_sync(0xffffffffu, g.V == 0.f || g.degenerate)) return make_float2(0.f, 0.f);
  float vis[K + 1];
  const float min_div =
      leg_visibility<MODE, K, MASKED>(s, a.W, cd, g.Qx, g.Qy, g.mx, g.my, g.mc, vis);
  if constexpr (!MASKED && MODE != MODE_STEP) {
    // as in path_power: an unreliable divided-out factor recomputes with masking
    const bool bad = !g.degenerate && !(min_div >= 0.25f);
    if (__any_sync(0xffffffffu, bad))
      leg_visibility<MODE, K, true>(s, a.W, cd, g.Qx, g.Qy, g.mx, g.my, g.mc, vis);
  }
  if (vis_out) {
#pragma unroll
    for (int j = 0; j <= K; ++j) vis_out[j] = vis[j];
  }
  return field_of_path<MODE, K>(s, a, g, vis, cd);
}

// Fields of one path candidate of order K for the receivers rx0 and rx1 (hard
// sigmoid or sigmoid): the packed obstruction loop of path_power_pair.
template <int MODE, int K>
__device__ __forceinline__ void path_field_pair(const SmemWalls& s, const SmemPairs& p,
                                                const FieldArgs& a, float2 tx, float2 rx0,
                                                float2 rx1, const Cand& cd, float2& f0,
                                                float2& f1, float2* vis_out = nullptr) {
  float Ix[K + 1], Iy[K + 1];
  tx_images<K>(s, tx, cd, Ix, Iy);
  PathGeom<MODE, K> g0, g1;
  path_geometry<MODE, K>(s, Ix, Iy, tx, rx0, cd, a.alpha, g0);
  path_geometry<MODE, K>(s, Ix, Iy, tx, rx1, cd, a.alpha, g1);
  if (a.cull && __all_sync(0xffffffffu, (g0.V == 0.f || g0.degenerate) &&
                                            (g1.V == 0.f || g1.degenerate))) {
    f0 = f1 = make_float2(0.f, 0.f);
    return;
  }
  float2 Qx[K + 2], Qy[K + 2], mx[K + 1], my[K + 1], mc[K + 1], vis2[K + 1];
#pragma unroll
  for (int i = 0; i <= K + 1; ++i) {
    Qx[i] = f2(g0.Qx[i], g1.Qx[i]);
    Qy[i] = f2(g0.Qy[i], g1.Qy[i]);
  }
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    mx[j] = f2(g0.mx[j], g1.mx[j]);
    my[j] = f2(g0.my[j], g1.my[j]);
    mc[j] = f2(g0.mc[j], g1.mc[j]);
  }
  if (MODE == MODE_HARD)
    hard_visibility_pair<K>(s, p, a.W, Qx, Qy, mx, my, mc, vis2);
  else
    sigmoid_visibility_pair<K>(s, p, a.W, Qx, Qy, mx, my, mc, vis2);
  float vis0[K + 1], vis1[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    vis0[j] = vis2[j].x;
    vis1[j] = vis2[j].y;
  }
  float d0, d1;
  if (MODE == MODE_HARD) {
    d0 = hard_skip_divide<K>(s, cd, g0.Qx, g0.Qy, g0.mx, g0.my, g0.mc, vis0);
    d1 = hard_skip_divide<K>(s, cd, g1.Qx, g1.Qy, g1.mx, g1.my, g1.mc, vis1);
  } else {
    d0 = sigmoid_skip_divide<K>(s, cd, g0.Qx, g0.Qy, g0.mx, g0.my, g0.mc, vis0);
    d1 = sigmoid_skip_divide<K>(s, cd, g1.Qx, g1.Qy, g1.mx, g1.my, g1.mc, vis1);
  }
  if (__any_sync(0xffffffffu, !g0.degenerate && !(d0 >= 0.25f)))
    leg_visibility<MODE, K, true>(s, a.W, cd, g0.Qx, g0.Qy, g0.mx, g0.my, g0.mc, vis0);
  if (__any_sync(0xffffffffu, !g1.degenerate && !(d1 >= 0.25f)))
    leg_visibility<MODE, K, true>(s, a.W, cd, g1.Qx, g1.Qy, g1.mx, g1.my, g1.mc, vis1);
  if (vis_out) {
#pragma unroll
    for (int j = 0; j <= K; ++j) vis_out[j] = f2(vis0[j], vis1[j]);
  }
  f0 = field_of_path<MODE, K>(s, a, g0, vis0, cd);
  f1 = field_of_path<MODE, K>(s, a, g1, vis1, cd);
}

template <int MODE, bool MASKED>
__device__ __forceinline__ float2 field_of(const SmemWalls& s, const FieldArgs& a, float2 tx,
                                           float2 q, const Cand& cd, float* vis_out) {
  switch (cd.k) {
    case 0: return path_field<MODE, 0, MASKED>(s, a, tx, q, cd, vis_out);
    case 1: return path_field<MODE, 1, MASKED>(s, a, tx, q, cd, vis_out);
    case 2: return path_field<MODE, 2, MASKED>(s, a, tx, q, cd, vis_out);
    default: return path_field<MODE, 3, MASKED>(s, a, tx, q, cd, vis_out);
  }
}

// One receiver per lane; a unit is (32 receivers) x (a chunk of candidates), as in
// the forward kernel, with one (re, im) partial sum per (chunk, receiver).  SAVE
// (sigmoid): every path's leg visibilities also go to a.saved, as drt_forward_save
// writes them (the same values: the same obstruction loops).
template <int MODE, bool SAVE = false>
__global__ void __launch_bounds__(256, MODE == MODE_SIGMOID ? 2 : 3) field_kernel(const FieldArgs a) {
  extern __shared__ float4 smem[];
  SmemWalls s{smem, smem + a.W, smem + 2 * a.W, smem + 3 * a.W};
  const float2 tx = make_float2(__ldg(a.tx), __ldg(a.tx + 1));
  stage_walls<MODE>(a.walls, a.W, tx, a.alpha, s);
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const long long warps_per_cta = blockDim.x >> 5;
  const long long nwarps = (long long)gridDim.x * warps_per_cta;
  const bool masked = a.alpha > FAST_SKIP_MAX_ALPHA;
  for (long long u = (long long)blockIdx.x * warps_per_cta + (threadIdx.x >> 5); u < a.n_units;
       u = next_unit_of(a.unit_counter, u, nwarps, lane)) {
    const long long tile = u % a.n_tiles;
    const long long chunk = u / a.n_tiles;
    long long r = tile * 32 + lane;
    const bool live = r < a.R;
    if (!live) r = a.R - 1;
    const float2 q = __ldg(reinterpret_cast<const float2*>(a.rx) + r);
    const int c0 = (int)(chunk * a.chunk);
    const int nc = (int)(min(c0 + (long long)a.chunk, a.n_cand) - c0);
    float2 acc = make_float2(0.f, 0.f);
    float vbuf[KMAX + 1];   // the path's leg visibilities when they are saved
    float* vo = SAVE ? vbuf : nullptr;
    Cand cd = decode_candidate(c0, a.W, a.K);
    for (int i = 0; i < nc; ++i) {
      if (i > 0) next_candidate(cd, a.W);
      if (vo) {
#pragma unroll
        for (int j = 0; j <= KMAX; ++j) vbuf[j] = 0.f;
      }
      const float2 f = masked ? field_of<MODE, true>(s, a, tx, q, cd, vo)
                              : field_of<MODE, false>(s, a, tx, q, cd, vo);
      acc.x += f.x;
      acc.y += f.y;
      if (vo && live) {   // [n_cand][K + 1][R]
        float* dst = a.saved + (long long)(c0 + i) * (a.K + 1) * a.R + r;
        for (int j = 0; j <= cd.k; ++j) dst[j * a.R] = vbuf[j];
      }
    }
    if (live) a.partial[chunk * a.R + r] = acc;
  }
}

// Hard sigmoid and sigmoid, two receivers per lane: lane l holds receivers l and
// l + 32 of its 64-receiver tile; the walls' paired records follow the four
// single-receiver arrays in shared memory.
template <int MODE, bool SAVE = false>
__global__ void __launch_bounds__(256, 2) field_pair_kernel(const FieldArgs a) {
  extern __shared__ float4 smem[];
  SmemWalls s{smem, smem + a.W, smem + 2 * a.W, smem + 3 * a.W};
  SmemPairs pr{smem + 4 * a.W, smem + 5 * a.W, smem + 6 * a.W, smem + 7 * a.W};
  const float2 tx = make_float2(__ldg(a.tx), __ldg(a.tx + 1));
  stage_walls<MODE>(a.walls, a.W, tx, a.alpha, s);
  __syncthreads();
  stage_pairs<MODE>(s, a.W, pr);
  __syncthreads();

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
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    float2 vbuf[KMAX + 1];   // the path's leg visibilities when they are saved
    float2* vo = SAVE ? vbuf : nullptr;
    Cand cd = decode_candidate(c0, a.W, a.K);
    for (int i = 0; i < nc; ++i) {
      if (i > 0) next_candidate(cd, a.W);
      if (vo) {
#pragma unroll
        for (int j = 0; j <= KMAX; ++j) vbuf[j] = make_float2(0.f, 0.f);
      }
      float2 f0, f1;
      switch (cd.k) {
        case 0: path_field_pair<MODE, 0>(s, pr, a, tx, q0, q1, cd, f0, f1, vo); break;
        case 1: path_field_pair<MODE, 1>(s, pr, a, tx, q0, q1, cd, f0, f1, vo); break;
        case 2: path_field_pair<MODE, 2>(s, pr, a, tx, q0, q1, cd, f0, f1, vo); break;
        default: path_field_pair<MODE, 3>(s, pr, a, tx, q0, q1, cd, f0, f1, vo); break;
      }
      acc0.x += f0.x;
      acc0.y += f0.y;
      acc1.x += f1.x;
      acc1.y += f1.y;
      if (vo) {   // [n_cand][K + 1][R]
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

// field[r] = sum over chunks of partial[chunk][r] in chunk order; power[r] = |field[r]|^2.
__global__ void reduce_field_kernel(const float2* __restrict__ partial, long long n_chunks,
                                    long long R, float2* __restrict__ field,
                                    float* __restrict__ power) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < R;
       r += (long long)gridDim.x * blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (long long c = 0; c < n_chunks; ++c) {
      const float2 v = partial[c * R + r];
      acc.x += v.x;
      acc.y += v.y;
    }
    field[r] = acc;
    if (power) power[r] = fmaf(acc.x, acc.x, acc.y * acc.y);
  }
}

}  // namespace

cudaError_t launch_field(const FieldArgs& a, int mode, int ctas, int threads, cudaStream_t st) {
  const size_t smem = forward_smem_bytes(a.W, a.pairs);
  if (a.unit_counter && a.n_units > 0) {
    cudaError_t e = cudaMemsetAsync(a.unit_counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  const bool save = a.saved && mode == MODE_SIGMOID;
  if (a.n_units > 0 && a.pairs) {
    if (mode == MODE_SIGMOID && save)
      field_pair_kernel<MODE_SIGMOID, true><<<ctas, threads, smem, st>>>(a);
    else if (mode == MODE_SIGMOID)
      field_pair_kernel<MODE_SIGMOID><<<ctas, threads, smem, st>>>(a);
    else
      field_pair_kernel<MODE_HARD><<<ctas, threads, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else if (a.n_units > 0) {
    switch (mode) {
      case MODE_SIGMOID:
        if (save)
          field_kernel<MODE_SIGMOID, true><<<ctas, threads, smem, st>>>(a);
        else
          field_kernel<MODE_SIGMOID><<<ctas, threads, smem, st>>>(a);
        break;
      case MODE_HARD: field_kernel<MODE_HARD><<<ctas, threads, smem, st>>>(a); break;
      default: field_kernel<MODE_STEP><<<ctas, threads, smem, st>>>(a); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (a.R > 0) {
    const long long nb = (a.R + 255) / 256;
    const int rb = (int)(nb < 4096 ? nb : 4096);
    reduce_field_kernel<<<rb, 256, 0, st>>>(a.partial, a.n_chunks, a.R, a.field, a.power);
  }
  return cudaGetLastError();
}

cudaError_t field_occupancy(int mode, bool pairs, int threads, int W, int* ctas_per_sm) {
  const size_t smem = forward_smem_bytes(W, pairs);
  if (pairs)
    return mode == MODE_SIGMOID
               ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     ctas_per_sm, field_pair_kernel<MODE_SIGMOID>, threads, smem)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     ctas_per_sm, field_pair_kernel<MODE_HARD>, threads, smem);
  switch (mode) {
    case MODE_SIGMOID:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, field_kernel<MODE_SIGMOID>,
                                                           threads, smem);
    case MODE_HARD:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, field_kernel<MODE_HARD>,
                                                           threads, smem);
    default:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, field_kernel<MODE_STEP>,
                                                           threads, smem);
  }
}

cudaError_t field_set_smem_limit(int W) {
  const int smem = (int)forward_smem_bytes(W, false);
  const int psmem = (int)forward_smem_bytes(W, true);
  cudaError_t e = cudaFuncSetAttribute(field_pair_kernel<MODE_HARD>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(field_pair_kernel<MODE_SIGMOID>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(field_pair_kernel<MODE_SIGMOID, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(field_kernel<MODE_SIGMOID>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(field_kernel<MODE_SIGMOID, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(field_kernel<MODE_HARD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(field_kernel<MODE_STEP>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace drt
