// Hand-written adjoint (reverse mode) of the forward pass: the vector-Jacobian
// product  sum_r g_r dP_r / d(tx, walls)  (Sec. III: gradient of the loss with
// respect to the scene parameters).
//
// Each (receiver, candidate) recomputes its image chain, reflection points, legs
// and validity, then runs two sweeps over the walls.  Sweep 1 rebuilds each
// leg's visibility as a product of non-zero factors plus a count of exact zeros,
// so that the derivative of the product w.r.t. one factor never divides by zero
// (for the sigmoid the forward can keep these visibilities instead, and the
// SAVED variants read them in place of sweep 1).  Sweep 2 recomputes each
// factor and pushes its adjoint into the vertices, the leg normals and the
// wall.  The vertex and leg adjoints then flow back through the leg lengths,
// the validity, the backtrace and the image chain to the transmitter.
//
// The mapping is the forward's: 32 receivers per warp, one warp-uniform
// candidate at a time; warps take their units from a counter (work stealing)
// and store each unit's TX adjoint.  Per-wall adjoints are summed over the warp
// with shuffles (only when a lane has a non-zero one), added into a per-CTA
// shared-memory table, and written per CTA; a last kernel adds the CTA tables
// in a fixed order, adds the units' TX adjoints in unit order, and chains the
// per-wall quantities (n, c, t0, len) back to the end points.
#include <cuda_runtime.h>

#include "drt_common.cuh"
#include "drt_internal.h"
#include "drt_path_vjp.cuh"
#include "drt_path_vjp_pair.cuh"

namespace drt {

namespace {

// Work stealing of the receiver-tile adjoints: a warp's first unit is its own
// index, later ones come from a global counter (zeroed before the launch), so a
// warp whose units end early (tiles at weight 0, paths skipped as exactly zero)
// takes more.
__device__ __forceinline__ long long next_unit(const VjpArgs& a, long long nwarps, int lane) {
  unsigned long long v = 0;
  if (lane == 0) v = atomicAdd(a.unit_counter, 1ULL);
  return nwarps + (long long)__shfl_sync(FULL, v, 0);
}

// The TX adjoint of one unit, summed over the warp and stored per unit: the
// finalize kernel adds the units in index order, so the TX gradient does not
// depend on which warp took which unit.
__device__ __forceinline__ void unit_tx_done(const VjpArgs& a, long long u, int lane, float ux,
                                             float uy) {
  ux = warp_sum(ux);
  uy = warp_sum(uy);
  if (lane == 0) {
    a.unit_tx[2 * u] = ux;
    a.unit_tx[2 * u + 1] = uy;
  }
}

// SAVED: the sigmoid's leg visibilities come from a.saved (the forward's) instead
// of the first wall sweep.
template <int MODE, bool WG, bool SAVED = false>
__global__ void __launch_bounds__(256) vjp_kernel(const VjpArgs a) {
  extern __shared__ float4 smem[];
  const float2 tx = make_float2(__ldg(a.tx), __ldg(a.tx + 1));
  VSmem s;
  s.G = smem;
  s.E = smem + a.W;
  s.T = smem + 2 * a.W;
  s.H = smem + 3 * a.W;
  s.acc = reinterpret_cast<float*>(smem + 4 * a.W);
  stage_walls<MODE>(a.walls, a.W, tx, a.alpha, SmemWalls{s.G, s.E, s.T, s.H});
  if (WG)
    for (int i = threadIdx.x; i < a.W * VJP_SLOTS; i += blockDim.x) s.acc[i] = 0.f;
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const long long warps_per_cta = blockDim.x >> 5;
  const long long gwarp = (long long)blockIdx.x * warps_per_cta + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * warps_per_cta;
  for (long long u = gwarp; u < a.n_units; u = next_unit(a, nwarps, lane)) {
    const long long tile = u % a.n_tiles;
    const long long chunk = u / a.n_tiles;
    long long r = tile * 32 + lane;
    const bool live = r < a.R;
    if (!live) r = a.R - 1;
    const float g = live ? __ldg(a.grad_power + r) : 0.f;
    float ux = 0.f, uy = 0.f;
    if (!__all_sync(FULL, g == 0.f)) {
      const float2 q = __ldg(reinterpret_cast<const float2*>(a.rx) + r);
      const long long c0 = chunk * a.chunk;
      const long long c1 = min(c0 + (long long)a.chunk, a.n_cand);
      for (long long c = c0; c < c1; ++c) {
        const Cand cd = decode_candidate(c, a.W, a.K);
        // the forward's saved visibilities, [n_cand][K + 1][R] (or none)
        const float* sv = SAVED ? a.saved + c * (a.K + 1) * a.R + r : nullptr;
        switch (cd.k) {
          case 0: path_vjp<MODE, 0, WG, true>(s, a.W, tx, q, cd, a.alpha, a.gk[0], g, ux, uy, nullptr, sv, a.R); break;
          case 1: path_vjp<MODE, 1, WG, true>(s, a.W, tx, q, cd, a.alpha, a.gk[1], g, ux, uy, nullptr, sv, a.R); break;
          case 2: path_vjp<MODE, 2, WG, true>(s, a.W, tx, q, cd, a.alpha, a.gk[2], g, ux, uy, nullptr, sv, a.R); break;
          default: path_vjp<MODE, 3, WG, true>(s, a.W, tx, q, cd, a.alpha, a.gk[3], g, ux, uy, nullptr, sv, a.R); break;
        }
      }
    }
    unit_tx_done(a, u, lane, ux, uy);
  }
  if (WG) {
    __syncthreads();
    float* out = a.cta_walls + (size_t)blockIdx.x * a.W * VJP_SLOTS;
    for (int i = threadIdx.x; i < a.W * VJP_SLOTS; i += blockDim.x) out[i] = s.acc[i];
  }
}

// Sigmoid with the wall gradient, two receivers per lane: units are (64
// receivers) x (a chunk of candidates); lane l holds receivers l and l + 32 of
// its tile.  The paired wall
// records follow the four single-receiver arrays, the per-CTA wall table follows
// those.
// Resident CTAs per SM the paired kernel is compiled for (registers per thread
// follow: 65536 / (256 threads x this)).  Two CTAs (128 registers, a few hundred
// bytes of spills) measured faster than one (227 registers, no spills, 8 warps
// per SM: dependency stalls dominate).
#ifndef DRT_VJP_PAIR_MIN_CTAS
#define DRT_VJP_PAIR_MIN_CTAS 2
#endif
#ifndef DRT_VJP_PAIR_MAX_THREADS
#define DRT_VJP_PAIR_MAX_THREADS 256
#endif

template <bool WG, bool SAVED = false>
__global__ void __launch_bounds__(DRT_VJP_PAIR_MAX_THREADS, DRT_VJP_PAIR_MIN_CTAS)
    vjp_pair_kernel(const VjpArgs a) {
  extern __shared__ float4 smem[];
  const float2 tx = make_float2(__ldg(a.tx), __ldg(a.tx + 1));
  VSmem s;
  s.G = smem;
  s.E = smem + a.W;
  s.T = smem + 2 * a.W;
  s.H = smem + 3 * a.W;
  const SmemPairsVjp pr{smem + 4 * a.W, smem + 5 * a.W, smem + 6 * a.W, smem + 7 * a.W,
                        smem + 8 * a.W};
  s.acc = reinterpret_cast<float*>(smem + 9 * a.W);
  stage_walls<MODE_SIGMOID>(a.walls, a.W, tx, a.alpha, SmemWalls{s.G, s.E, s.T, s.H});
  if (WG)
    for (int i = threadIdx.x; i < a.W * VJP_SLOTS; i += blockDim.x) s.acc[i] = 0.f;
  __syncthreads();
  stage_pairs_vjp(s, a.W, pr);
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const long long warps_per_cta = blockDim.x >> 5;
  const long long gwarp = (long long)blockIdx.x * warps_per_cta + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * warps_per_cta;
  for (long long u = gwarp; u < a.n_units; u = next_unit(a, nwarps, lane)) {
    const long long tile = u % a.n_tiles;
    const long long chunk = u / a.n_tiles;
    const long long r0 = tile * 64 + lane, r1 = r0 + 32;
    const bool live0 = r0 < a.R, live1 = r1 < a.R;
    const float g0 = live0 ? __ldg(a.grad_power + r0) : 0.f;
    const float g1 = live1 ? __ldg(a.grad_power + r1) : 0.f;
    float ux = 0.f, uy = 0.f;
    if (!__all_sync(FULL, g0 == 0.f && g1 == 0.f)) {
      const float2 q0 = __ldg(reinterpret_cast<const float2*>(a.rx) + (live0 ? r0 : a.R - 1));
      const float2 q1 = __ldg(reinterpret_cast<const float2*>(a.rx) + (live1 ? r1 : a.R - 1));
      const long long c0 = chunk * a.chunk;
      const long long c1 = min(c0 + (long long)a.chunk, a.n_cand);
      // the forward's saved visibilities, [n_cand][K + 1][R] (or none)
      const long long rr0 = live0 ? r0 : a.R - 1, rr1 = live1 ? r1 : a.R - 1;
      for (long long c = c0; c < c1; ++c) {
        const Cand cd = decode_candidate(c, a.W, a.K);
        const float* sv0 = SAVED ? a.saved + c * (a.K + 1) * a.R + rr0 : nullptr;
        const float* sv1 = SAVED ? a.saved + c * (a.K + 1) * a.R + rr1 : nullptr;
        switch (cd.k) {
          case 0: path_vjp_pair<0, WG>(s, pr, a.W, tx, q0, q1, cd, a.alpha, a.gk[0], g0, g1, ux, uy, sv0, sv1, a.R); break;
          case 1: path_vjp_pair<1, WG>(s, pr, a.W, tx, q0, q1, cd, a.alpha, a.gk[1], g0, g1, ux, uy, sv0, sv1, a.R); break;
          case 2: path_vjp_pair<2, WG>(s, pr, a.W, tx, q0, q1, cd, a.alpha, a.gk[2], g0, g1, ux, uy, sv0, sv1, a.R); break;
          default: path_vjp_pair<3, WG>(s, pr, a.W, tx, q0, q1, cd, a.alpha, a.gk[3], g0, g1, ux, uy, sv0, sv1, a.R); break;
        }
      }
    }
    unit_tx_done(a, u, lane, ux, uy);
  }
  if (WG) {
    __syncthreads();
    float* out = a.cta_walls + (size_t)blockIdx.x * a.W * VJP_SLOTS;
    for (int i = threadIdx.x; i < a.W * VJP_SLOTS; i += blockDim.x) out[i] = s.acc[i];
  }
}

// Adjoint of the coherent field's power |E_r|^2 with cotangent g_r: the same
// mapping as vjp_kernel, each lane weighing its paths' fields by w = 2 g_r conj(E_r)
// (E_r from drt_field, one load per unit).  SAVED: the sigmoid's leg visibilities
// come from a.saved (drt_field_save's or drt_forward_save's) instead of the first
// wall sweep.
template <int MODE, bool WG, bool SAVED = false>
__global__ void __launch_bounds__(256, WG ? 2 : 1) field_vjp_kernel(const VjpArgs a) {
  extern __shared__ float4 smem[];
  const float2 tx = make_float2(__ldg(a.tx), __ldg(a.tx + 1));
  VSmem s;
  s.G = smem;
  s.E = smem + a.W;
  s.T = smem + 2 * a.W;
  s.H = smem + 3 * a.W;
  s.acc = reinterpret_cast<float*>(smem + 4 * a.W);
  stage_walls<MODE>(a.walls, a.W, tx, a.alpha, SmemWalls{s.G, s.E, s.T, s.H});
  if (WG)
    for (int i = threadIdx.x; i < a.W * VJP_SLOTS; i += blockDim.x) s.acc[i] = 0.f;
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const long long warps_per_cta = blockDim.x >> 5;
  const long long gwarp = (long long)blockIdx.x * warps_per_cta + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * warps_per_cta;
  FieldW fw;
  fw.inv_lambda_hi = a.inv_lambda_hi;
  fw.inv_lambda_lo = a.inv_lambda_lo;
  fw.k2pi = a.k2pi;
  fw.eps_r = a.eps_r;
  fw.refl_amp = a.refl_amp;
  for (long long u = gwarp; u < a.n_units; u = next_unit(a, nwarps, lane)) {
    const long long tile = u % a.n_tiles;
    const long long chunk = u / a.n_tiles;
    long long r = tile * 32 + lane;
    const bool live = r < a.R;
    if (!live) r = a.R - 1;
    const float gp = live ? __ldg(a.grad_power + r) : 0.f;
    const float2 E = __ldg(a.field + r);
    fw.wre = 2.f * gp * E.x;
    fw.wim = -2.f * gp * E.y;
    const float g = (fw.wre != 0.f || fw.wim != 0.f) ? 1.f : 0.f;
    float ux = 0.f, uy = 0.f;
    if (!__all_sync(FULL, g == 0.f)) {
      const float2 q = __ldg(reinterpret_cast<const float2*>(a.rx) + r);
      const long long c0 = chunk * a.chunk;
      const long long c1 = min(c0 + (long long)a.chunk, a.n_cand);
      for (long long c = c0; c < c1; ++c) {
        const Cand cd = decode_candidate(c, a.W, a.K);
        const float* sv = SAVED ? a.saved + c * (a.K + 1) * a.R + r : nullptr;
        switch (cd.k) {
          case 0: path_vjp<MODE, 0, WG, true, true>(s, a.W, tx, q, cd, a.alpha, 1.f, g, ux, uy, &fw, sv, a.R); break;
          case 1: path_vjp<MODE, 1, WG, true, true>(s, a.W, tx, q, cd, a.alpha, 1.f, g, ux, uy, &fw, sv, a.R); break;
          case 2: path_vjp<MODE, 2, WG, true, true>(s, a.W, tx, q, cd, a.alpha, 1.f, g, ux, uy, &fw, sv, a.R); break;
          default: path_vjp<MODE, 3, WG, true, true>(s, a.W, tx, q, cd, a.alpha, 1.f, g, ux, uy, &fw, sv, a.R); break;
        }
      }
    }
    unit_tx_done(a, u, lane, ux, uy);
  }
  if (WG) {
    __syncthreads();
    float* out = a.cta_walls + (size_t)blockIdx.x * a.W * VJP_SLOTS;
    for (int i = threadIdx.x; i < a.W * VJP_SLOTS; i += blockDim.x) out[i] = s.acc[i];
  }
}

// Adjoint of the min-power loss: loss = -P[argmin], so the gradient is
// -grad_loss * dP[argmin]/d(tx, walls) for one receiver.  Here the lanes of a
// warp hold 32 consecutive candidates of that receiver (one unit = 32
// candidates); candidates are ordered by reflection count, so a unit spans at
// most a few orders, and the warp runs each order present with the lanes of
// other orders idle (weight 0 on a stand-in candidate of that order).
template <int MODE, bool WG>
__global__ void __launch_bounds__(256) vjp_rx_kernel(const VjpArgs a) {
  extern __shared__ float4 smem[];
  const float2 tx = make_float2(__ldg(a.tx), __ldg(a.tx + 1));
  VSmem s;
  s.G = smem;
  s.E = smem + a.W;
  s.T = smem + 2 * a.W;
  s.H = smem + 3 * a.W;
  s.acc = reinterpret_cast<float*>(smem + 4 * a.W);
  stage_walls<MODE>(a.walls, a.W, tx, a.alpha, SmemWalls{s.G, s.E, s.T, s.H});
  if (WG)
    for (int i = threadIdx.x; i < a.W * VJP_SLOTS; i += blockDim.x) s.acc[i] = 0.f;
  __syncthreads();

  int ri = __ldg(a.rx_index);
  ri = ri < 0 ? 0 : (ri >= a.R ? (int)a.R - 1 : ri);
  const float2 q = __ldg(reinterpret_cast<const float2*>(a.rx) + ri);
  const float g = -(a.grad_loss ? __ldg(a.grad_loss) : 1.0f);
  const int lane = threadIdx.x & 31;
  const long long warps_per_cta = blockDim.x >> 5;
  const long long gwarp = (long long)blockIdx.x * warps_per_cta + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * warps_per_cta;
  const long long n_units = (a.n_cand + 31) / 32;
  float txb_x = 0.f, txb_y = 0.f;
  for (long long u = gwarp; u < n_units; u += nwarps) {
    const long long c = u * 32 + lane;
    const bool live = c < a.n_cand;
    const Cand mine = decode_candidate(live ? c : a.n_cand - 1, a.W, a.K);
    const int k_lo = decode_candidate(u * 32, a.W, a.K).k;
    const int k_hi = decode_candidate(min(u * 32 + 31, a.n_cand - 1), a.W, a.K).k;
    for (int k = k_lo; k <= k_hi; ++k) {
      const bool use = live && mine.k == k;
      Cand cd = mine;
      if (!use) {   // stand-in of order k: walls 0, 1, 0, ... (never two equal in a row)
        cd.k = k;
#pragma unroll
        for (int j = 0; j < KMAX; ++j) cd.w[j] = (j & 1) ? (a.W > 1 ? 1 : 0) : 0;
      }
      const float gl = use ? g : 0.f;
      switch (k) {
        case 0: path_vjp<MODE, 0, WG, false>(s, a.W, tx, q, cd, a.alpha, a.gk[0], gl, txb_x, txb_y); break;
        case 1: path_vjp<MODE, 1, WG, false>(s, a.W, tx, q, cd, a.alpha, a.gk[1], gl, txb_x, txb_y); break;
        case 2: path_vjp<MODE, 2, WG, false>(s, a.W, tx, q, cd, a.alpha, a.gk[2], gl, txb_x, txb_y); break;
        default: path_vjp<MODE, 3, WG, false>(s, a.W, tx, q, cd, a.alpha, a.gk[3], gl, txb_x, txb_y); break;
      }
    }
  }
  txb_x = warp_sum(txb_x);
  txb_y = warp_sum(txb_y);
  if (lane == 0) {
    a.warp_tx[2 * gwarp] = txb_x;
    a.warp_tx[2 * gwarp + 1] = txb_y;
  }
  if (WG) {
    __syncthreads();
    float* out = a.cta_walls + (size_t)blockIdx.x * a.W * VJP_SLOTS;
    for (int i = threadIdx.x; i < a.W * VJP_SLOTS; i += blockDim.x) out[i] = s.acc[i];
  }
}

// Sums the per-CTA wall tables and the per-warp TX partials in a fixed order
// and chains (n, c, t0, len) back to the end points A, B of each wall:
//   u = (B - A)/|B - A|, n = (-u_y, u_x), c = n . A, t0 = u . A.
__global__ void __launch_bounds__(256) vjp_finalize_kernel(const VjpArgs a, int n_ctas,
                                                           int n_warps, int wall_grad) {
  if (wall_grad) {
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < a.W; w += gridDim.x * blockDim.x) {
      float acc[VJP_SLOTS];
#pragma unroll
      for (int k = 0; k < VJP_SLOTS; ++k) acc[k] = 0.f;
      for (int c = 0; c < n_ctas; ++c) {
        const float* src = a.cta_walls + ((size_t)c * a.W + w) * VJP_SLOTS;
#pragma unroll
        for (int k = 0; k < VJP_SLOTS; ++k) acc[k] += src[k];
      }
      const float4 ab = a.walls[w];
      const WallGeom g = wall_geometry(ab);
      const float nx = g.G.x, ny = g.G.y, len = g.G.w;
      const float ux = ny, uy = -nx;
      float nbx = acc[S_NX], nby = acc[S_NY];
      float Abx = acc[S_AX], Aby = acc[S_AY], Bbx = acc[S_BX], Bby = acc[S_BY];
      // c = n . A
      nbx = fmaf(acc[S_C], ab.x, nbx);
      nby = fmaf(acc[S_C], ab.y, nby);
      Abx = fmaf(acc[S_C], nx, Abx);
      Aby = fmaf(acc[S_C], ny, Aby);
      // t0 = u . A
      float ubx = acc[S_T0] * ab.x, uby = acc[S_T0] * ab.y;
      Abx = fmaf(acc[S_T0], ux, Abx);
      Aby = fmaf(acc[S_T0], uy, Aby);
      // n = (-u_y, u_x)
      ubx += nby;
      uby -= nbx;
      // u = e / len, len = |e|, e = B - A
      const float uu = fmaf(ubx, ux, uby * uy);
      const float ebx = fmaf(acc[S_LEN], ux, (ubx - uu * ux) / len);
      const float eby = fmaf(acc[S_LEN], uy, (uby - uu * uy) / len);
      Abx -= ebx;
      Aby -= eby;
      Bbx += ebx;
      Bby += eby;
      reinterpret_cast<float4*>(a.grad_walls)[w] = make_float4(Abx, Aby, Bbx, Bby);
    }
  }
  if (blockIdx.x == 0) {
    __shared__ float sx[256], sy[256];
    float x = 0.f, y = 0.f;
    // per-unit TX adjoints (the receiver-tile kernels) or per-warp ones
    const float* parts = a.unit_tx ? a.unit_tx : a.warp_tx;
    const long long n_parts = a.unit_tx ? a.n_units : n_warps;
    for (long long i = threadIdx.x; i < n_parts; i += blockDim.x) {
      x += parts[2 * i];
      y += parts[2 * i + 1];
    }
    sx[threadIdx.x] = x;
    sy[threadIdx.x] = y;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) {
        sx[threadIdx.x] += sx[threadIdx.x + o];
        sy[threadIdx.x] += sy[threadIdx.x + o];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      a.grad_tx[0] = sx[0];
      a.grad_tx[1] = sy[0];
    }
  }
}

template <int MODE, bool WG>
void launch_vjp_t(const VjpArgs& a, int ctas, int threads, size_t smem, cudaStream_t st) {
  if (a.rx_index)
    vjp_rx_kernel<MODE, WG><<<ctas, threads, smem, st>>>(a);
  else if (MODE == MODE_SIGMOID && a.saved)
    vjp_kernel<MODE, WG, true><<<ctas, threads, smem, st>>>(a);
  else
    vjp_kernel<MODE, WG><<<ctas, threads, smem, st>>>(a);
}

}  // namespace

size_t vjp_smem_bytes(int W, bool wall_grad, bool pairs) {
  return (size_t)(pairs ? 9 : 4) * W * sizeof(float4) +
         (wall_grad ? (size_t)W * VJP_SLOTS * sizeof(float) : 0);
}

bool vjp_uses_pairs(int mode, int flags) {
  return mode == MODE_SIGMOID && !(flags & DRT_TILE_SINGLE_RX);
}

cudaError_t launch_vjp(const VjpArgs& a, int mode, int ctas, int threads, cudaStream_t st) {
  const bool wg = a.grad_walls != nullptr;
  const size_t smem = vjp_smem_bytes(a.W, wg, a.pairs && !a.rx_index && wg);
  if (!a.rx_index) {   // the receiver-tile kernels steal work: zero their counter
    cudaError_t e = cudaMemsetAsync(a.unit_counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  if (a.pairs && !a.rx_index && mode == MODE_SIGMOID && wg) {
    if (a.saved)
      vjp_pair_kernel<true, true><<<ctas, threads, smem, st>>>(a);
    else
      vjp_pair_kernel<true><<<ctas, threads, smem, st>>>(a);
  } else
  switch (mode * 2 + (wg ? 1 : 0)) {
    case MODE_SIGMOID * 2: launch_vjp_t<MODE_SIGMOID, false>(a, ctas, threads, smem, st); break;
    case MODE_SIGMOID * 2 + 1: launch_vjp_t<MODE_SIGMOID, true>(a, ctas, threads, smem, st); break;
    case MODE_HARD * 2: launch_vjp_t<MODE_HARD, false>(a, ctas, threads, smem, st); break;
    case MODE_HARD * 2 + 1: launch_vjp_t<MODE_HARD, true>(a, ctas, threads, smem, st); break;
    case MODE_STEP * 2: launch_vjp_t<MODE_STEP, false>(a, ctas, threads, smem, st); break;
    default: launch_vjp_t<MODE_STEP, true>(a, ctas, threads, smem, st); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n_warps = ctas * (threads / 32);
  const int fb = wg ? (a.W + 255) / 256 : 1;
  vjp_finalize_kernel<<<fb, 256, 0, st>>>(a, ctas, n_warps, wg ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_field_vjp(const VjpArgs& a, int mode, int ctas, int threads, cudaStream_t st) {
  const bool wg = a.grad_walls != nullptr;
  const size_t smem = vjp_smem_bytes(a.W, wg, false);
  {   // the field adjoint steals work like the receiver-tile adjoints
    cudaError_t e = cudaMemsetAsync(a.unit_counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
  const bool saved = a.saved && mode == MODE_SIGMOID;
  switch (mode * 2 + (wg ? 1 : 0)) {
    case MODE_SIGMOID * 2:
      if (saved)
        field_vjp_kernel<MODE_SIGMOID, false, true><<<ctas, threads, smem, st>>>(a);
      else
        field_vjp_kernel<MODE_SIGMOID, false><<<ctas, threads, smem, st>>>(a);
      break;
    case MODE_SIGMOID * 2 + 1:
      if (saved)
        field_vjp_kernel<MODE_SIGMOID, true, true><<<ctas, threads, smem, st>>>(a);
      else
        field_vjp_kernel<MODE_SIGMOID, true><<<ctas, threads, smem, st>>>(a);
      break;
    case MODE_HARD * 2: field_vjp_kernel<MODE_HARD, false><<<ctas, threads, smem, st>>>(a); break;
    case MODE_HARD * 2 + 1: field_vjp_kernel<MODE_HARD, true><<<ctas, threads, smem, st>>>(a); break;
    case MODE_STEP * 2: field_vjp_kernel<MODE_STEP, false><<<ctas, threads, smem, st>>>(a); break;
    default: field_vjp_kernel<MODE_STEP, true><<<ctas, threads, smem, st>>>(a); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n_warps = ctas * (threads / 32);
  const int fb = wg ? (a.W + 255) / 256 : 1;
  vjp_finalize_kernel<<<fb, 256, 0, st>>>(a, ctas, n_warps, wg ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t field_vjp_occupancy(int mode, bool wg, int threads, int W, int* ctas_per_sm) {
  const size_t smem = vjp_smem_bytes(W, wg, false);
  switch (mode * 2 + (wg ? 1 : 0)) {
    case MODE_SIGMOID * 2:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, field_vjp_kernel<MODE_SIGMOID, false>, threads, smem);
    case MODE_SIGMOID * 2 + 1:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, field_vjp_kernel<MODE_SIGMOID, true>, threads, smem);
    case MODE_HARD * 2:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, field_vjp_kernel<MODE_HARD, false>, threads, smem);
    case MODE_HARD * 2 + 1:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, field_vjp_kernel<MODE_HARD, true>, threads, smem);
    case MODE_STEP * 2:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, field_vjp_kernel<MODE_STEP, false>, threads, smem);
    default:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, field_vjp_kernel<MODE_STEP, true>, threads, smem);
  }
}

cudaError_t vjp_occupancy(int mode, bool wg, bool pairs, int threads, int W, int* ctas_per_sm) {
  const size_t smem = vjp_smem_bytes(W, wg, pairs);
  if (pairs && mode == MODE_SIGMOID && wg)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp_pair_kernel<true>,
                                                         threads, smem);
  switch (mode * 2 + (wg ? 1 : 0)) {
    case MODE_SIGMOID * 2:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp_kernel<MODE_SIGMOID, false>, threads, smem);
    case MODE_SIGMOID * 2 + 1:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp_kernel<MODE_SIGMOID, true>, threads, smem);
    case MODE_HARD * 2:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp_kernel<MODE_HARD, false>, threads, smem);
    case MODE_HARD * 2 + 1:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp_kernel<MODE_HARD, true>, threads, smem);
    case MODE_STEP * 2:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp_kernel<MODE_STEP, false>, threads, smem);
    default:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp_kernel<MODE_STEP, true>, threads, smem);
  }
}

cudaError_t vjp_set_smem_limit(int W) {
  const int s0 = (int)vjp_smem_bytes(W, false, false), s1 = (int)vjp_smem_bytes(W, true, false);
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(vjp_pair_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)vjp_smem_bytes(W, true, true));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(vjp_pair_kernel<true, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)vjp_smem_bytes(W, true, true));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(vjp_kernel<MODE_SIGMOID, true, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, s1);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(vjp_kernel<MODE_SIGMOID, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, s0);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(field_vjp_kernel<MODE_SIGMOID, true, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, s1);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(field_vjp_kernel<MODE_SIGMOID, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, s0);
  if (e != cudaSuccess) return e;
#define DRT_SET(M, B, S)                                                                    \
  e = cudaFuncSetAttribute(vjp_kernel<M, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, S); \
  if (e != cudaSuccess) return e;                                                           \
  e = cudaFuncSetAttribute(vjp_rx_kernel<M, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, S); \
  if (e != cudaSuccess) return e;                                                           \
  e = cudaFuncSetAttribute(field_vjp_kernel<M, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, S); \
  if (e != cudaSuccess) return e;
  DRT_SET(MODE_SIGMOID, false, s0)
  DRT_SET(MODE_SIGMOID, true, s1)
  DRT_SET(MODE_HARD, false, s0)
  DRT_SET(MODE_HARD, true, s1)
  DRT_SET(MODE_STEP, false, s0)
  DRT_SET(MODE_STEP, true, s1)
#undef DRT_SET
  return e;
}

}  // namespace drt
