// Iterative path finder with the smoothed convergence check (Sec. V-B,
// "Continuous Path Finding"): the reflection points of every path candidate are
// found by Min-Path-Tracing (MPT) steps instead of the image method, and the
// path carries the check s(eps - C) on its MPT cost C.
//
// For a candidate (w_1..w_k) the unknowns are the coordinates tau_j of the
// reflection points X_j = A_j + tau_j u_j along the walls' lines (X_0 = TX,
// X_{k+1} = RX).  With h_j the unit direction of leg j and R_j the mirror of
// wall j, the residuals r_j = h_j - R_j h_{j-1} vanish exactly where the
// reflection law holds, and C = sum_j |r_j|^2.  From the walls' midpoints,
// each step solves the Gauss-Newton system (J^T J + mu) delta = -J^T r
// (mu = 1e-6 of the diagonal), clamps delta_j to [-len_j, len_j] and
// backtracks: it takes the largest fraction 2^-m (m < 12) of delta that lowers
// C by 1e-4 of its slope, up to 8 units of FP32 rounding of C (no step if none
// does).  The path's validity is prod_j s(tau_j) s(len_j - tau_j) times
// kappa = s(eps - C); the obstruction loop and the power are the forward's.  A
// leg of zero length at any step, or shorter than 1e-3 at the final points
// (an iteration running into the corner where two walls meet), makes the path
// degenerate: it contributes 0.
//
// Fermat path tracing (FPT) runs the same loop with the total length L = sum_j l_j
// as the objective: Newton steps (H + mu) delta = -grad L with
// dL/dtau_j = u_j . (h_{j-1} - h_j) and H's entries (1 - (h . u)^2) / l on the
// diagonal, -(u_j . u_{j+1} - (h_j . u_j)(h_j . u_{j+1})) / l_j beside it, the
// backtracking on L; the check is still s(eps - C) with the MPT cost C.
//
// Mapping: the forward's (one receiver per lane, a warp-uniform candidate,
// units of 32 receivers x a chunk of candidates, chunk sums added in order).
// The iterations diverge only where lanes take different numbers of
// backtracking halvings.
#include <cuda_runtime.h>

#include "drt_common.cuh"
#include "drt_internal.h"
#include "drt_path.cuh"

namespace drt {
namespace {

constexpr int MPT_HALVINGS = 12;
constexpr float MPT_MU = 1e-6f;
constexpr float MPT_ROUNDING = 8.f * 1.1920929e-7f;   // 8 units of FP32 rounding
constexpr float MPT_MIN_LEG = 1e-3f;   // a shorter leg at the final points: degenerate path

// Vertices, unit leg directions and leg lengths of a candidate at tau.
template <int K>
struct MptLegs {
  float X[K + 2], Y[K + 2];
  float hx[K + 1], hy[K + 1], l[K + 1];
  bool degenerate;
};

template <int K>
__device__ __forceinline__ void mpt_legs(const SmemWalls& s, const Cand& cd, float2 tx, float2 rx,
                                         const float* tau, MptLegs<K>& f) {
  f.X[0] = tx.x;
  f.Y[0] = tx.y;
  f.X[K + 1] = rx.x;
  f.Y[K + 1] = rx.y;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const float4 G = s.G[cd.w[j - 1]];
    const float4 E = s.E[cd.w[j - 1]];
    // u = (n_y, -n_x): the wall's unit direction from A to B
    f.X[j] = fmaf(tau[j - 1], G.y, E.x);
    f.Y[j] = fmaf(tau[j - 1], -G.x, E.y);
  }
  f.degenerate = false;
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    const float dx = f.X[j + 1] - f.X[j], dy = f.Y[j + 1] - f.Y[j];
    const float l2 = fmaf(dx, dx, dy * dy);
    f.degenerate |= !(l2 > 0.f);
    const float l = __fsqrt_rn(l2);
    const float inv = l2 > 0.f ? __frcp_rn(l) : 0.f;
    f.l[j] = l;
    f.hx[j] = dx * inv;
    f.hy[j] = dy * inv;
  }
}

// reflection law residual at point j: h_j - R_j h_{j-1}
template <int K>
__device__ __forceinline__ float2 mpt_residual(const float4& G, const MptLegs<K>& f, int j) {
  const float in = fmaf(G.x, f.hx[j - 1], G.y * f.hy[j - 1]);
  return make_float2(f.hx[j] - fmaf(-2.f * in, G.x, f.hx[j - 1]),
                     f.hy[j] - fmaf(-2.f * in, G.y, f.hy[j - 1]));
}

template <int K>
__device__ __forceinline__ float mpt_cost(const SmemWalls& s, const Cand& cd, const MptLegs<K>& f) {
  float C = 0.f;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const float2 r = mpt_residual<K>(s.G[cd.w[j - 1]], f, j);
    C = fmaf(r.x, r.x, fmaf(r.y, r.y, C));
  }
  return C;
}

// (I - h h^T) v / l for leg `leg`
template <int K>
__device__ __forceinline__ float2 mpt_proj(const MptLegs<K>& f, int leg, float vx, float vy) {
  const float c = fmaf(f.hx[leg], vx, f.hy[leg] * vy);
  const float il = __frcp_rn(f.l[leg]);
  return make_float2(fmaf(-c, f.hx[leg], vx) * il, fmaf(-c, f.hy[leg], vy) * il);
}

// mirror of a direction in the wall with unit normal (G.x, G.y)
__device__ __forceinline__ float2 mpt_mirror(const float4& G, float2 v) {
  const float c = fmaf(G.x, v.x, G.y * v.y);
  return make_float2(fmaf(-2.f * c, G.x, v.x), fmaf(-2.f * c, G.y, v.y));
}

template <int K>
__device__ __forceinline__ float fpt_length(const MptLegs<K>& f) {
  float L = 0.f;
#pragma unroll
  for (int j = 0; j <= K; ++j) L += f.l[j];
  return L;
}

// The finder's objective: the MPT cost C, or the path length L for FPT.
template <int FINDER, int K>
__device__ __forceinline__ float finder_objective(const SmemWalls& s, const Cand& cd,
                                                  const MptLegs<K>& f) {
  if (FINDER == FINDER_FPT) return fpt_length<K>(f);
  return mpt_cost<K>(s, cd, f);
}

// Result of the path finder for one path: tau, the final cost, degeneracy.
template <int K>
struct MptResult {
  float tau[K > 0 ? K : 1];
  float C;
  bool degenerate;
};

template <int FINDER, int K>
__device__ __forceinline__ void finder_points(const SmemWalls& s, const Cand& cd, float2 tx,
                                              float2 rx, int n_iter, MptResult<K>& res) {
  float tau[K > 0 ? K : 1];
#pragma unroll
  for (int j = 0; j < K; ++j) tau[j] = 0.5f * s.G[cd.w[j]].w;
  MptLegs<K> f;
  mpt_legs<K>(s, cd, tx, rx, tau, f);
  bool dead = f.degenerate;
  for (int it = 0; it < n_iter && K > 0 && !dead; ++it) {
    float A[K + 1][K + 1], b[K + 1], g0[K + 1];
    if (FINDER == FINDER_FPT) {
      // b = -grad L, A = the Hessian of L (tridiagonal)
#pragma unroll
      for (int j = 1; j <= K; ++j) {
        const float4 G = s.G[cd.w[j - 1]];
        const float ux = G.y, uy = -G.x;   // the wall's unit direction
        const float gin = fmaf(ux, f.hx[j - 1], uy * f.hy[j - 1]);
        const float gout = fmaf(ux, f.hx[j], uy * f.hy[j]);
        b[j] = gout - gin;
#pragma unroll
        for (int q = 1; q <= K; ++q) A[j][q] = 0.f;
        A[j][j] = fmaf(-gin, gin, 1.f) * __frcp_rn(f.l[j - 1]) +
                  fmaf(-gout, gout, 1.f) * __frcp_rn(f.l[j]);
      }
#pragma unroll
      for (int j = 1; j < K; ++j) {
        const float4 G = s.G[cd.w[j - 1]], Gn = s.G[cd.w[j]];
        const float ux = G.y, uy = -G.x, vx = Gn.y, vy = -Gn.x;
        const float hu = fmaf(ux, f.hx[j], uy * f.hy[j]);
        const float hv = fmaf(vx, f.hx[j], vy * f.hy[j]);
        const float c = -fmaf(-hu, hv, fmaf(ux, vx, uy * vy)) * __frcp_rn(f.l[j]);
        A[j][j + 1] = c;
        A[j + 1][j] = c;
      }
#pragma unroll
      for (int p = 1; p <= K; ++p) {
        g0[p] = b[p];
        A[p][p] *= 1.f + MPT_MU;
      }
    } else {
    // Jacobian: J[j][i] = dr_j / dtau_i (2-vectors), nonzero for |i - j| <= 1
    float2 J[K + 1][K + 1];
    float2 r[K + 1];
#pragma unroll
    for (int j = 1; j <= K; ++j) {
      const float4 G = s.G[cd.w[j - 1]];
      r[j] = mpt_residual<K>(G, f, j);
#pragma unroll
      for (int i = 1; i <= K; ++i) J[j][i] = make_float2(0.f, 0.f);
      // tau_j moves the end of leg j - 1 and the start of leg j
      const float2 a = mpt_proj<K>(f, j, G.y, -G.x);
      const float2 c = mpt_mirror(G, mpt_proj<K>(f, j - 1, G.y, -G.x));
      J[j][j] = make_float2(-a.x - c.x, -a.y - c.y);
      if (j < K) {   // the end of leg j
        const float4 Gn = s.G[cd.w[j]];
        J[j][j + 1] = mpt_proj<K>(f, j, Gn.y, -Gn.x);
      }
      if (j > 1) {   // the start of leg j - 1
        const float4 Gp = s.G[cd.w[j - 2]];
        J[j][j - 1] = mpt_mirror(G, mpt_proj<K>(f, j - 1, Gp.y, -Gp.x));
      }
    }
    // normal equations (J^T J + mu) delta = -J^T r
#pragma unroll
    for (int p = 1; p <= K; ++p) {
#pragma unroll
      for (int q = 1; q <= K; ++q) {
        float v = 0.f;
#pragma unroll
        for (int j = 1; j <= K; ++j) v = fmaf(J[j][p].x, J[j][q].x, fmaf(J[j][p].y, J[j][q].y, v));
        A[p][q] = v;
      }
      float v = 0.f;
#pragma unroll
      for (int j = 1; j <= K; ++j) v = fmaf(J[j][p].x, r[j].x, fmaf(J[j][p].y, r[j].y, v));
      b[p] = -v;
      g0[p] = b[p];
      A[p][p] *= 1.f + MPT_MU;
    }
    }
    // Cholesky: A = L L^T (lower triangle in place), then L y = b, L^T x = y
#pragma unroll
    for (int c = 1; c <= K; ++c) {
      float d = A[c][c];
#pragma unroll
      for (int p = 1; p < c; ++p) d = fmaf(-A[c][p], A[c][p], d);
      d = d > 0.f ? __fsqrt_rn(d) : 0.f;
      A[c][c] = d;
      const float id = d > 0.f ? __frcp_rn(d) : 0.f;
#pragma unroll
      for (int q = c + 1; q <= K; ++q) {
        float v = A[q][c];
#pragma unroll
        for (int p = 1; p < c; ++p) v = fmaf(-A[q][p], A[c][p], v);
        A[q][c] = v * id;
      }
    }
#pragma unroll
    for (int q = 1; q <= K; ++q) {
      float v = b[q];
#pragma unroll
      for (int p = 1; p < q; ++p) v = fmaf(-A[q][p], b[p], v);
      b[q] = A[q][q] > 0.f ? v * __frcp_rn(A[q][q]) : 0.f;
    }
#pragma unroll
    for (int q = K; q >= 1; --q) {
      float v = b[q];
#pragma unroll
      for (int p = q + 1; p <= K; ++p) v = fmaf(-A[p][q], b[p], v);
      b[q] = A[q][q] > 0.f ? v * __frcp_rn(A[q][q]) : 0.f;
    }
    // clamp, slope of the objective along the step (grad C = 2 J^T r = -2 g0 for
    // MPT, grad L = -g0 for FPT)
    float slope = 0.f;
#pragma unroll
    for (int q = 1; q <= K; ++q) {
      const float lim = s.G[cd.w[q - 1]].w;
      b[q] = fminf(fmaxf(b[q], -lim), lim);
      slope = fmaf((FINDER == FINDER_FPT ? -1.f : -2.f) * g0[q], b[q], slope);
    }
    const float C0 = finder_objective<FINDER, K>(s, cd, f);
    const float tol = MPT_ROUNDING * C0;
    float t = 1.f;
    bool moved = false;
    for (int m = 0; m < MPT_HALVINGS; ++m, t *= 0.5f) {
      float trial[K > 0 ? K : 1];
#pragma unroll
      for (int q = 0; q < K; ++q) trial[q] = fmaf(t, b[q + 1], tau[q]);
      MptLegs<K> ft;
      mpt_legs<K>(s, cd, tx, rx, trial, ft);
      if (ft.degenerate) continue;
      if (finder_objective<FINDER, K>(s, cd, ft) <= fmaf(1e-4f * t, slope, C0) + tol) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
          moved |= !(trial[q] == tau[q]);
          tau[q] = trial[q];
        }
        f = ft;
        break;
      }
    }
    // a step that leaves every tau as it was (no step taken, or one below the
    // rounding of tau) leaves the whole state as it was: the remaining steps would
    // repeat it exactly, so the points are final (the result is the same bit for bit)
    if (!moved) break;
  }
  res.degenerate = dead || f.degenerate;
#pragma unroll
  for (int j = 0; j <= K; ++j) res.degenerate |= !(f.l[j] >= MPT_MIN_LEG);
#pragma unroll
  for (int q = 0; q < K; ++q) res.tau[q] = tau[q];
  res.C = res.degenerate ? 0.f : mpt_cost<K>(s, cd, f);
}

// Power of one candidate of order K with MPT reflection points.  When `out` is
// not null it receives the per-path record of a scene of maximum order KS:
// tau_1..tau_KS (NaN past K, or for a degenerate path), C, kappa.
template <int MODE, int FINDER, int K>
__device__ __forceinline__ float path_power_mpt(const SmemWalls& s, int W, float2 tx, float2 rx,
                                                const Cand& cd, float alpha, float gk, int n_iter,
                                                float eps, float* out, int KS) {
  MptResult<K> m;
  finder_points<FINDER, K>(s, cd, tx, rx, n_iter, m);
  const float kappa = m.degenerate ? 0.f : smooth3<MODE>(eps - m.C, alpha).s;
  if (out) {
    const float nan = __int_as_float(0x7fc00000);
    for (int q = 0; q < KS; ++q) out[q] = (q < K && !m.degenerate) ? m.tau[q < K ? q : 0] : nan;
    out[KS] = m.C;
    out[KS + 1] = kappa;
  }
  // --- the path's geometry in the forward's form: vertices, leg lines, length
  PathGeom<MODE, K> g;
  MptLegs<K> f;
  mpt_legs<K>(s, cd, tx, rx, m.tau, f);
  g.degenerate = m.degenerate || f.degenerate;
  g.L = 0.f;
#pragma unroll
  for (int i = 0; i <= K + 1; ++i) {
    g.Qx[i] = f.X[i];
    g.Qy[i] = f.Y[i];
  }
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    g.L += f.l[j];
    const float nx = -f.hy[j], ny = f.hx[j];
    const float nq = fmaf(nx, f.X[j], ny * f.Y[j]);
    if (MODE == MODE_HARD) {
      const float a6 = alpha * (1.0f / 6.0f);
      g.mx[j] = nx * a6;
      g.my[j] = ny * a6;
      g.mc[j] = fmaf(-nq, a6, 0.5f);
    } else if (MODE == MODE_STEP) {
      g.mx[j] = nx;
      g.my[j] = ny;
      g.mc[j] = -nq;
    } else {
      const float kap = alpha * LOG2E;
      g.mx[j] = nx * kap;
      g.my[j] = ny * kap;
      g.mc[j] = -nq * kap;
    }
  }
  // validity: on the segments, times the convergence check
  g.V = kappa;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const float len = s.G[cd.w[q]].w;
    g.V *= smooth3<MODE>(m.tau[q], alpha).s * smooth3<MODE>(len - m.tau[q], alpha).s;
  }
  if (__all_sync(0xffffffffu, g.degenerate || g.V == 0.f)) return 0.f;
  float vis[K + 1];
  if (MODE == MODE_STEP || alpha > FAST_SKIP_MAX_ALPHA) {
    leg_visibility<MODE, K, true>(s, W, cd, g.Qx, g.Qy, g.mx, g.my, g.mc, vis);
  } else {
    const float min_div = leg_visibility<MODE, K, false>(s, W, cd, g.Qx, g.Qy, g.mx, g.my, g.mc, vis);
    const bool bad = !g.degenerate && !(min_div >= 0.25f);
    if (__any_sync(0xffffffffu, bad))
      leg_visibility<MODE, K, true>(s, W, cd, g.Qx, g.Qy, g.mx, g.my, g.mc, vis);
  }
  return path_power_of<MODE, K>(g, vis, gk);
}

template <int MODE, int FINDER>
__global__ void __launch_bounds__(256, 2) forward_mpt_kernel(const MptArgs m) {
  const FwdArgs& a = m.f;
  extern __shared__ float4 smem[];
  SmemWalls s{smem, smem + a.W, smem + 2 * a.W, smem + 3 * a.W};
  const float2 tx = make_float2(__ldg(a.tx), __ldg(a.tx + 1));
  stage_walls<MODE>(a.walls, a.W, tx, a.alpha, s);
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
    const int c0 = (int)(chunk * a.chunk);
    const int nc = (int)(min(c0 + (long long)a.chunk, a.n_cand) - c0);
    float acc = 0.f;
    Cand cd = decode_candidate(c0, a.W, a.K);
    for (int i = 0; i < nc; ++i) {
      if (i > 0) next_candidate(cd, a.W);
      const int c = c0 + i;
      float* out = (m.paths && live) ? m.paths + ((long long)r * a.n_cand + c) * (a.K + 2)
                                     : nullptr;
      float p;
      switch (cd.k) {
        case 0: p = path_power_mpt<MODE, FINDER, 0>(s, a.W, tx, q, cd, a.alpha, a.gk[0], m.n_iter, m.check_eps, out, a.K); break;
        case 1: p = path_power_mpt<MODE, FINDER, 1>(s, a.W, tx, q, cd, a.alpha, a.gk[1], m.n_iter, m.check_eps, out, a.K); break;
        case 2: p = path_power_mpt<MODE, FINDER, 2>(s, a.W, tx, q, cd, a.alpha, a.gk[2], m.n_iter, m.check_eps, out, a.K); break;
        default: p = path_power_mpt<MODE, FINDER, 3>(s, a.W, tx, q, cd, a.alpha, a.gk[3], m.n_iter, m.check_eps, out, a.K); break;
      }
      acc += p;
    }
    if (live && a.partial) a.partial[chunk * a.R + r] = acc;
  }
}

template <typename F>
cudaError_t launch_mpt_t(F kern, const MptArgs& a, int ctas, int threads, cudaStream_t st) {
  const size_t smem = forward_smem_bytes(a.f.W, false);
  kern<<<ctas, threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_forward_mpt(const MptArgs& a, int mode, int ctas, int threads, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (a.f.n_units > 0) {
    if (a.f.unit_counter) {
      e = cudaMemsetAsync(a.f.unit_counter, 0, sizeof(unsigned long long), st);
      if (e != cudaSuccess) return e;
    }
    if (a.finder == FINDER_FPT) {
      switch (mode) {
        case MODE_SIGMOID: e = launch_mpt_t(forward_mpt_kernel<MODE_SIGMOID, FINDER_FPT>, a, ctas, threads, st); break;
        case MODE_HARD: e = launch_mpt_t(forward_mpt_kernel<MODE_HARD, FINDER_FPT>, a, ctas, threads, st); break;
        default: e = launch_mpt_t(forward_mpt_kernel<MODE_STEP, FINDER_FPT>, a, ctas, threads, st); break;
      }
    } else {
      switch (mode) {
        case MODE_SIGMOID: e = launch_mpt_t(forward_mpt_kernel<MODE_SIGMOID, FINDER_MPT>, a, ctas, threads, st); break;
        case MODE_HARD: e = launch_mpt_t(forward_mpt_kernel<MODE_HARD, FINDER_MPT>, a, ctas, threads, st); break;
        default: e = launch_mpt_t(forward_mpt_kernel<MODE_STEP, FINDER_MPT>, a, ctas, threads, st); break;
      }
    }
    if (e != cudaSuccess) return e;
  }
  if (a.f.power) return launch_reduce_chunks(a.f.partial, a.f.n_chunks, a.f.R, a.f.power, st);
  return cudaSuccess;
}

cudaError_t launch_mpt_paths(const MptArgs& a, int mode, int ctas, int threads, cudaStream_t st) {
  return launch_forward_mpt(a, mode, ctas, threads, st);
}

cudaError_t forward_mpt_occupancy(int mode, int finder, int threads, int W, int* ctas_per_sm) {
  const size_t smem = forward_smem_bytes(W, false);
  if (finder == FINDER_FPT) {
    switch (mode) {
      case MODE_SIGMOID:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, forward_mpt_kernel<MODE_SIGMOID, FINDER_FPT>, threads, smem);
      case MODE_HARD:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, forward_mpt_kernel<MODE_HARD, FINDER_FPT>, threads, smem);
      default:
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, forward_mpt_kernel<MODE_STEP, FINDER_FPT>, threads, smem);
    }
  }
  switch (mode) {
    case MODE_SIGMOID:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, forward_mpt_kernel<MODE_SIGMOID, FINDER_MPT>, threads, smem);
    case MODE_HARD:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, forward_mpt_kernel<MODE_HARD, FINDER_MPT>, threads, smem);
    default:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, forward_mpt_kernel<MODE_STEP, FINDER_MPT>, threads, smem);
  }
}

cudaError_t forward_mpt_set_smem_limit(int W) {
  const int smem = (int)forward_smem_bytes(W, false);
  const void* kernels[] = {
      (const void*)forward_mpt_kernel<MODE_SIGMOID, FINDER_MPT>,
      (const void*)forward_mpt_kernel<MODE_HARD, FINDER_MPT>,
      (const void*)forward_mpt_kernel<MODE_STEP, FINDER_MPT>,
      (const void*)forward_mpt_kernel<MODE_SIGMOID, FINDER_FPT>,
      (const void*)forward_mpt_kernel<MODE_HARD, FINDER_FPT>,
      (const void*)forward_mpt_kernel<MODE_STEP, FINDER_FPT>};
  for (const void* k : kernels) {
    const cudaError_t e =
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace drt
