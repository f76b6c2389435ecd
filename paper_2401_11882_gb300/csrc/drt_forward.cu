// Forward pass of the smoothed image-method objective: received power per
// receiver (Sec. V, Eq. 7) and the min-power loss (Eq. 8).
//
// Mapping on the GPU: the 32 lanes of a warp hold 32 receivers; the warp walks
// one path candidate at a time, so the candidate's wall sequence, its TX image
// chain and every branch are warp-uniform, and the walls are read from shared
// memory as broadcasts.  A work unit is (32 receivers) x (a chunk of
// candidates); a persistent grid strides over the units in a fixed order and
// writes one partial sum per (chunk, receiver), which a second kernel adds up in
// chunk order.  The result is therefore deterministic.
//
// Hot loop (obstruction, Sec. V-A with the comparison rule x0 > x1 -> s(x0 - x1)):
// for every wall, the smoothed side of each path vertex is computed once and
// shared by the two legs that meet there; each leg then needs only the sides of
// the wall's two end points w.r.t. the leg's line.
#include <cuda_runtime.h>

#include "drt_common.cuh"
#include "drt_internal.h"

namespace drt {

namespace {

// Shared-memory layout: 4 float4 per wall, as separate arrays.
//   sG, sE, sT: wall_geometry() records.
//   sH: smoothing-ready record for the obstruction loop:
//     hard    {a6 nx, a6 ny, 1/2 - a6 c, s(d(TX))}            a6 = alpha/6
//     step    {nx, ny, -c, theta(d(TX))}
//     sigmoid {k nx, k ny, -k c, sign(z_TX) * 2^-|z_TX|}      k = alpha log2(e)
struct SmemWalls {
  float4 *G, *E, *T, *H;
};

template <int MODE>
__device__ void stage_walls(const float4* __restrict__ walls, int W, float2 tx, float alpha,
                            SmemWalls s) {
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    const WallGeom g = wall_geometry(walls[w]);
    s.G[w] = g.G;
    s.E[w] = g.E;
    s.T[w] = g.T;
    float4 h;
    if (MODE == MODE_HARD) {
      const float a6 = alpha * (1.0f / 6.0f);
      h = make_float4(g.G.x * a6, g.G.y * a6, fmaf(-g.G.z, a6, 0.5f), 0.f);
      h.w = __saturatef(fmaf(h.x, tx.x, fmaf(h.y, tx.y, h.z)));
    } else if (MODE == MODE_STEP) {
      h = make_float4(g.G.x, g.G.y, -g.G.z, 0.f);
      h.w = fmaf(h.x, tx.x, fmaf(h.y, tx.y, h.z)) > 0.f ? 1.f : 0.f;
    } else {
      const float kap = alpha * LOG2E;
      h = make_float4(g.G.x * kap, g.G.y * kap, -g.G.z * kap, 0.f);
      const float z = fmaf(h.x, tx.x, fmaf(h.y, tx.y, h.z));
      h.w = copysignf(ex2_approx(-fabsf(z)), z);
    }
    s.H[w] = h;
  }
}

// s() of an argument already scaled and offset by the H record (hard: sat; step: theta).
template <int MODE>
__device__ __forceinline__ float side(float z) {
  if (MODE == MODE_HARD) return __saturatef(z);
  return z > 0.f ? 1.f : 0.f;
}

// Power of one path candidate of order K for this lane's receiver (Eq. 7 term).
template <int MODE, int K>
__device__ __forceinline__ float path_power(const SmemWalls& s, int W, float2 tx, float2 rx,
                                            const Cand& cd, float alpha, float gk, int cull) {
  // --- image method (Sec. V-B): TX images in the walls of the sequence.
  float Ix[K + 1], Iy[K + 1];
  Ix[0] = tx.x;
  Iy[0] = tx.y;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const float4 G = s.G[cd.w[j - 1]];
    const float d = line_dist(G, Ix[j - 1], Iy[j - 1]);
    Ix[j] = fmaf(-2.f * d, G.x, Ix[j - 1]);
    Iy[j] = fmaf(-2.f * d, G.y, Iy[j - 1]);
  }
  // --- backtrace on the infinite lines: Q_{K+1} = RX, Q_j = line(Q_{j+1}, I_j) x wall j.
  float Qx[K + 2], Qy[K + 2];
  Qx[0] = tx.x;
  Qy[0] = tx.y;
  Qx[K + 1] = rx.x;
  Qy[K + 1] = rx.y;
  bool degenerate = false;
#pragma unroll
  for (int j = K; j >= 1; --j) {
    const float4 G = s.G[cd.w[j - 1]];
    const float a = line_dist(G, Ix[j], Iy[j]);
    const float b = line_dist(G, Qx[j + 1], Qy[j + 1]);
    // parallel lines (or a reflection point absurdly far away): no path
    float t = __fdiv_rn(b, b - a);
    if (!(fabsf(t) <= 1e8f)) {
      degenerate = true;
      t = 0.f;
    }
    Qx[j] = fmaf(t, Ix[j] - Qx[j + 1], Qx[j + 1]);
    Qy[j] = fmaf(t, Iy[j] - Qy[j + 1], Qy[j + 1]);
  }
  // --- legs: length and the smoothing-ready normal form of each leg's line.
  float L = 0.f;
  float mx[K + 1], my[K + 1], mc[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    const float dx = Qx[j + 1] - Qx[j], dy = Qy[j + 1] - Qy[j];
    const float len2 = fmaf(dx, dx, dy * dy);
    degenerate |= !(len2 > 0.f);
    const float inv = rsqrtf(len2);
    L = fmaf(len2, inv, L);
    const float nx = -dy * inv, ny = dx * inv;
    const float nq = fmaf(nx, Qx[j], ny * Qy[j]);
    if (MODE == MODE_HARD) {
      const float a6 = alpha * (1.0f / 6.0f);
      mx[j] = nx * a6;
      my[j] = ny * a6;
      mc[j] = fmaf(-nq, a6, 0.5f);
    } else if (MODE == MODE_STEP) {
      mx[j] = nx;
      my[j] = ny;
      mc[j] = -nq;
    } else {
      const float kap = alpha * LOG2E;
      mx[j] = nx * kap;
      my[j] = ny * kap;
      mc[j] = -nq * kap;
    }
  }
  // --- continuous validity of each reflection (Sec. V-A): on the segment, and the
  //     previous and next vertices on the same side of the wall's line.
  float V = 1.f;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const int w = cd.w[j - 1];
    const float4 G = s.G[w];
    const float t0 = s.T[w].x;
    const float tau = fmaf(G.y, Qx[j], fmaf(-G.x, Qy[j], -t0));   // u = (ny, -nx)
    const Smooth3 s1 = smooth3<MODE>(tau, alpha);
    const Smooth3 s2 = smooth3<MODE>(G.w - tau, alpha);
    const Smooth3 sp = smooth3<MODE>(line_dist(G, Qx[j - 1], Qy[j - 1]), alpha);
    const Smooth3 sq = smooth3<MODE>(line_dist(G, Qx[j + 1], Qy[j + 1]), alpha);
    V *= s1.s * s2.s * fmaf(sp.s, sq.s, sp.sb * sq.sb);
  }
  // optional: skip the obstruction loop when the whole warp's validity is exactly 0
  if (cull && __all_sync(0xffffffffu, V == 0.f || degenerate)) return 0.f;
  // --- obstruction of every leg by every wall except the ones its end points lie on.
  float vis[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) vis[j] = 1.f;

  if constexpr (MODE != MODE_SIGMOID) {
    // blocked = X(x1, y1) X(x2, y2) with X(x, y) = s(x) s(-y) + s(-x) s(y) = s_x + s_y (1 - 2 s_x).
#pragma unroll 2
    for (int w = 0; w < W; ++w) {
      const float4 h = s.H[w];
      const float4 e = s.E[w];
      float sv[K + 2], uv[K + 1];
      sv[0] = h.w;
      uv[0] = fmaf(-2.f, h.w, 1.f);
#pragma unroll
      for (int i = 1; i <= K + 1; ++i) sv[i] = side<MODE>(fmaf(h.x, Qx[i], fmaf(h.y, Qy[i], h.z)));
#pragma unroll
      for (int i = 1; i <= K; ++i) uv[i] = fmaf(-2.f, sv[i], 1.f);
#pragma unroll
      for (int j = 0; j <= K; ++j) {
        const float sa = side<MODE>(fmaf(mx[j], e.x, fmaf(my[j], e.y, mc[j])));
        const float sb = side<MODE>(fmaf(mx[j], e.z, fmaf(my[j], e.w, mc[j])));
        const float x2 = fmaf(sb, fmaf(-2.f, sa, 1.f), sa);
        const float x1 = fmaf(sv[j + 1], uv[j], sv[j]);
        float bl = x1 * x2;
        const bool skip = (j >= 1 && w == cd.w[j - 1]) || (j < K && w == cd.w[j]);
        bl = skip ? 0.f : bl;
        vis[j] = fmaf(-vis[j], bl, vis[j]);
      }
    }
  } else {
    // Sigmoid: with e = 2^-|z| <= 1 per argument, for a pair (x, y)
    //   Ns = e_x + e_y, No = 1 + e_x e_y, D = (1 + e_x)(1 + e_y) = Ns + No,
    //   X = (same sign ? Ns : No) / D and 1 - X = (same sign ? No : Ns) / D,
    // and 1 - X1 X2 = (Xb1 D2 + X1 Xb2) / (D1 D2) in numerators: every term is a
    // sum of non-negative products, so a nearly blocked leg keeps its relative
    // accuracy.  Numerator and denominator products are folded into vis every 8 walls.
    float vn[K + 1], vd[K + 1];
#pragma unroll
    for (int j = 0; j <= K; ++j) vn[j] = vd[j] = 1.f;
    for (int w0 = 0; w0 < W; w0 += 8) {
      const int w1 = min(w0 + 8, W);
      for (int w = w0; w < w1; ++w) {
        const float4 h = s.H[w];
        const float4 e = s.E[w];
        float ze[K + 2], ee[K + 2];
        ze[0] = h.w;
        ee[0] = fabsf(h.w);
#pragma unroll
        for (int i = 1; i <= K + 1; ++i) {
          ze[i] = fmaf(h.x, Qx[i], fmaf(h.y, Qy[i], h.z));
          ee[i] = ex2_approx(-fabsf(ze[i]));
        }
#pragma unroll
        for (int j = 0; j <= K; ++j) {
          const float za = fmaf(mx[j], e.x, fmaf(my[j], e.y, mc[j]));
          const float zb = fmaf(mx[j], e.z, fmaf(my[j], e.w, mc[j]));
          const float ea = ex2_approx(-fabsf(za));
          const float eb = ex2_approx(-fabsf(zb));
          // pair 1: the leg's end points w.r.t. the wall's line
          const float ns1 = ee[j] + ee[j + 1];
          const float no1 = fmaf(ee[j], ee[j + 1], 1.f);
          const bool same1 = (__float_as_int(ze[j]) ^ __float_as_int(ze[j + 1])) >= 0;
          const float x1 = same1 ? ns1 : no1, xb1 = same1 ? no1 : ns1;
          // pair 2: the wall's end points w.r.t. the leg's line
          const float ns2 = ea + eb;
          const float no2 = fmaf(ea, eb, 1.f);
          const bool same2 = (__float_as_int(za) ^ __float_as_int(zb)) >= 0;
          const float x2 = same2 ? ns2 : no2, xb2 = same2 ? no2 : ns2;
          const float den = (ns1 + no1) * (ns2 + no2);
          float num = fmaf(xb1, ns2 + no2, x1 * xb2);
          const bool skip = (j >= 1 && w == cd.w[j - 1]) || (j < K && w == cd.w[j]);
          num = skip ? den : num;
          vn[j] *= num;
          vd[j] *= den;
        }
      }
#pragma unroll
      for (int j = 0; j <= K; ++j) {
        vis[j] *= __fdividef(vn[j], vd[j]);
        vn[j] = vd[j] = 1.f;
      }
    }
  }
  float p = V * gk;
#pragma unroll
  for (int j = 0; j <= K; ++j) p *= vis[j];
  p = __fdiv_rn(p, L * L);
  return degenerate ? 0.f : p;
}

template <int MODE>
__global__ void __launch_bounds__(256, MODE == MODE_SIGMOID ? 3 : 4) forward_kernel(const FwdArgs a) {
  extern __shared__ float4 smem[];
  SmemWalls s{smem, smem + a.W, smem + 2 * a.W, smem + 3 * a.W};
  const float2 tx = make_float2(__ldg(a.tx), __ldg(a.tx + 1));
  stage_walls<MODE>(a.walls, a.W, tx, a.alpha, s);
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const long long warps_per_cta = blockDim.x >> 5;
  const long long nwarps = (long long)gridDim.x * warps_per_cta;
  for (long long u = (long long)blockIdx.x * warps_per_cta + (threadIdx.x >> 5); u < a.n_units;
       u += nwarps) {
    const long long tile = u % a.n_tiles;
    const long long chunk = u / a.n_tiles;
    long long r = tile * 32 + lane;
    const bool live = r < a.R;
    if (!live) r = a.R - 1;
    const float2 q = __ldg(reinterpret_cast<const float2*>(a.rx) + r);
    const long long c0 = chunk * a.chunk;
    const long long c1 = min(c0 + (long long)a.chunk, a.n_cand);
    float acc = 0.f;
    for (long long c = c0; c < c1; ++c) {
      const Cand cd = decode_candidate(c, a.W, a.K);
      float p;
      switch (cd.k) {
        case 0: p = path_power<MODE, 0>(s, a.W, tx, q, cd, a.alpha, a.gk[0], a.cull); break;
        case 1: p = path_power<MODE, 1>(s, a.W, tx, q, cd, a.alpha, a.gk[1], a.cull); break;
        case 2: p = path_power<MODE, 2>(s, a.W, tx, q, cd, a.alpha, a.gk[2], a.cull); break;
        default: p = path_power<MODE, 3>(s, a.W, tx, q, cd, a.alpha, a.gk[3], a.cull); break;
      }
      acc += p;
    }
    if (live) a.partial[chunk * a.R + r] = acc;
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

size_t forward_smem_bytes(int W) { return (size_t)4 * W * sizeof(float4); }

cudaError_t launch_forward(const FwdArgs& a, int mode, int ctas, int threads, cudaStream_t st) {
  const size_t smem = forward_smem_bytes(a.W);
  if (a.n_units > 0) {
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

cudaError_t forward_occupancy(int mode, int threads, int W, int* ctas_per_sm) {
  const size_t smem = forward_smem_bytes(W);
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
  const int smem = (int)forward_smem_bytes(W);
  cudaError_t e;
  e = cudaFuncSetAttribute(forward_kernel<MODE_SIGMOID>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(forward_kernel<MODE_HARD>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(forward_kernel<MODE_STEP>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
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
