// Per-path forward evaluation shared by the single-scene and batched kernels:
// wall staging into shared memory and the power of one path candidate for one
// receiver (Sec. V, Eq. 7 term).
#pragma once

#include "drt_common.cuh"

namespace drt {

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

// s() of (a b + c) for the H-record forms: one saturating FMA for the hard sigmoid
template <int MODE>
__device__ __forceinline__ float side_fma(float a, float b, float c) {
  if (MODE == MODE_HARD) return fma_sat(a, b, c);
  return fmaf(a, b, c) > 0.f ? 1.f : 0.f;
}

// Largest alpha for which the hard-sigmoid and sigmoid loops test every (leg,
// wall) pair and divide the skipped pairs out afterwards: there a point lying on
// a wall's line has s within 1/4 of 1/2 even after FP32 rounding of its
// distance, so a skipped pair's factor is >= 1/2.  Above it (and for the unit
// step) the skipped pairs are masked inside the loop.
constexpr float FAST_SKIP_MAX_ALPHA = 1e4f;

// Hard sigmoid: divides out of vis[0..K] the factors of the (leg, wall) pairs a
// leg must skip (the walls its own end points lie on), which the wall loop
// multiplied in; returns the smallest factor divided out.
template <int K>
__device__ __forceinline__ float hard_skip_divide(const SmemWalls& s, const Cand& cd,
                                                  const float* Qx, const float* Qy, const float* mx,
                                                  const float* my, const float* mc, float* vis) {
  float min_div = 1.f;
#pragma unroll
  for (int j = 0; j <= K; ++j) {
#pragma unroll
    for (int side_ = 0; side_ < 2; ++side_) {
      // leg j skips w_j (side 0, j >= 1) and w_{j+1} (side 1, j < K)
      if ((side_ == 0 && j >= 1) || (side_ == 1 && j < K)) {
        const int w = cd.w[side_ == 0 ? j - 1 : j];
        const float4 h = s.H[w];
        const float4 e = s.E[w];
        const float s0 = (j == 0) ? h.w : fma_sat(h.x, Qx[j], fmaf(h.y, Qy[j], h.z));
        const float s1 = fma_sat(h.x, Qx[j + 1], fmaf(h.y, Qy[j + 1], h.z));
        const float sa = fma_sat(mx[j], e.x, fmaf(my[j], e.y, mc[j]));
        const float sb = fma_sat(mx[j], e.z, fmaf(my[j], e.w, mc[j]));
        const float x2 = fmaf(sb, fmaf(-2.f, sa, 1.f), sa);
        const float x1 = (j == 0) ? fmaf(s0, fmaf(-2.f, s1, 1.f), s1) : fmaf(s1, fmaf(-2.f, s0, 1.f), s0);
        const float f = fmaf(-x1, x2, 1.f);
        min_div = fminf(min_div, f);
        vis[j] = __fdividef(vis[j], f);
      }
    }
  }
  return min_div;
}

// Sigmoid: the factor 1 - X1 X2 of leg j and one wall as (numerator,
// denominator), in the product form of the sigmoid loop below.
template <int K>
__device__ __forceinline__ void sigmoid_pair_factor(const float4& h, const float4& e, int j,
                                                    const float* Qx, const float* Qy,
                                                    const float* mx, const float* my,
                                                    const float* mc, float& num, float& den) {
  float ze0, ee0, ze1, ee1;
  if (j == 0) {
    ze0 = copysignf(1.f, h.w);   // the TX side: only the sign is used
    ee0 = fabsf(h.w);
  } else {
    ze0 = fmaf(h.x, Qx[j], fmaf(h.y, Qy[j], h.z));
    ee0 = ex2_approx(-fabsf(ze0));
  }
  ze1 = fmaf(h.x, Qx[j + 1], fmaf(h.y, Qy[j + 1], h.z));
  ee1 = ex2_approx(-fabsf(ze1));
  const float za = fmaf(mx[j], e.x, fmaf(my[j], e.y, mc[j]));
  const float zb = fmaf(mx[j], e.z, fmaf(my[j], e.w, mc[j]));
  const float ea = ex2_approx(-fabsf(za));
  const float eb = ex2_approx(-fabsf(zb));
  const float ns1 = ee0 + ee1, no1 = fmaf(ee0, ee1, 1.f);
  const bool same1 = same_side(ze0, ze1);
  const float x1 = same1 ? ns1 : no1, xb1 = same1 ? no1 : ns1;
  const float ns2 = ea + eb, no2 = fmaf(ea, eb, 1.f);
  const bool same2 = same_side(za, zb);
  const float x2 = same2 ? ns2 : no2, xb2 = same2 ? no2 : ns2;
  den = (ns1 + no1) * (ns2 + no2);
  num = fmaf(xb1, ns2 + no2, x1 * xb2);
}

// Sigmoid counterpart of hard_skip_divide.
template <int K>
__device__ __forceinline__ float sigmoid_skip_divide(const SmemWalls& s, const Cand& cd,
                                                     const float* Qx, const float* Qy,
                                                     const float* mx, const float* my,
                                                     const float* mc, float* vis) {
  float min_div = 1.f;
#pragma unroll
  for (int j = 0; j <= K; ++j) {
#pragma unroll
    for (int side_ = 0; side_ < 2; ++side_) {
      if ((side_ == 0 && j >= 1) || (side_ == 1 && j < K)) {
        const int w = cd.w[side_ == 0 ? j - 1 : j];
        float num, den;
        sigmoid_pair_factor<K>(s.H[w], s.E[w], j, Qx, Qy, mx, my, mc, num, den);
        min_div = fminf(min_div, __fdividef(num, den));
        vis[j] *= __fdividef(den, num);
      }
    }
  }
  return min_div;
}

// Visibility of each leg (obstruction by every wall except the ones its end points
// lie on), written to vis[0..K].  Returns the smallest factor divided out for the
// skipped (leg, wall) pairs (1 when they are masked instead).
template <int MODE, int K, bool MASKED>
__device__ __forceinline__ float leg_visibility(const SmemWalls& s, int W, const Cand& cd,
                                                const float* Qx, const float* Qy, const float* mx,
                                                const float* my, const float* mc, float* vis) {
#pragma unroll
  for (int j = 0; j <= K; ++j) vis[j] = 1.f;
  float min_div = 1.f;

  if constexpr (MODE == MODE_HARD && !MASKED) {
    // blocked = X(x1, y1) X(x2, y2) with X(a, b) = s(a) s(-b) + s(-a) s(b) = s_a + s_b (1 - 2 s_a).
    // Every wall is tested against every leg here; the (leg, wall) pairs a leg must skip
    // (the walls its own end points lie on) are divided out after the loop: one end point
    // of such a pair lies on the wall's line, s = 1/2 there (C3), so its factor is >= 1/2.
#pragma unroll 2
    for (int w = 0; w < W; ++w) {
      const float4 h = s.H[w];
      const float4 e = s.E[w];
      float sv[K + 2], uv[K + 2];
      sv[0] = h.w;
#pragma unroll
      for (int i = 1; i <= K + 1; ++i) sv[i] = fma_sat(h.x, Qx[i], fmaf(h.y, Qy[i], h.z));
#pragma unroll
      for (int i = 1; i <= (K > 0 ? K : 1); ++i) uv[i] = fmaf(-2.f, sv[i], 1.f);
#pragma unroll
      for (int j = 0; j <= K; ++j) {
        const float sa = fma_sat(mx[j], e.x, fmaf(my[j], e.y, mc[j]));
        const float sb = fma_sat(mx[j], e.z, fmaf(my[j], e.w, mc[j]));
        const float x2 = fmaf(sb, fmaf(-2.f, sa, 1.f), sa);
        const float x1 = (j == 0) ? fmaf(sv[0], uv[1], sv[1]) : fmaf(sv[j + 1], uv[j], sv[j]);
        vis[j] = fmaf(-vis[j], x1 * x2, vis[j]);
      }
    }
    min_div = hard_skip_divide<K>(s, cd, Qx, Qy, mx, my, mc, vis);
  } else if constexpr (MODE != MODE_SIGMOID) {
    // unit step (no 1/2 at 0), or a large alpha: the skipped pairs are masked inside the loop.
#pragma unroll 2
    for (int w = 0; w < W; ++w) {
      const float4 h = s.H[w];
      const float4 e = s.E[w];
      float sv[K + 2], uv[K + 1];
      sv[0] = h.w;
      uv[0] = fmaf(-2.f, h.w, 1.f);
#pragma unroll
      for (int i = 1; i <= K + 1; ++i) sv[i] = side_fma<MODE>(h.x, Qx[i], fmaf(h.y, Qy[i], h.z));
#pragma unroll
      for (int i = 1; i <= K; ++i) uv[i] = fmaf(-2.f, sv[i], 1.f);
#pragma unroll
      for (int j = 0; j <= K; ++j) {
        const float sa = side_fma<MODE>(mx[j], e.x, fmaf(my[j], e.y, mc[j]));
        const float sb = side_fma<MODE>(mx[j], e.z, fmaf(my[j], e.w, mc[j]));
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
    // accuracy.  Numerator and denominator products are folded into vis every 8
    // walls.  Skipped (leg, wall) pairs are divided out after the loop, as for the
    // hard sigmoid (their factor is >= 1/2).
    float vn[K + 1], vd[K + 1];
#pragma unroll
    for (int j = 0; j <= K; ++j) vn[j] = vd[j] = 1.f;
    for (int w0 = 0; w0 < W; w0 += 8) {
      const int w1 = min(w0 + 8, W);
      for (int w = w0; w < w1; ++w) {
        const float4 h = s.H[w];
        const float4 e = s.E[w];
        float ze[K + 2], ee[K + 2];
        ze[0] = copysignf(1.f, h.w);   // the TX side: only the sign is used
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
          const bool same1 = same_side(ze[j], ze[j + 1]);
          const float x1 = same1 ? ns1 : no1, xb1 = same1 ? no1 : ns1;
          // pair 2: the wall's end points w.r.t. the leg's line
          const float ns2 = ea + eb;
          const float no2 = fmaf(ea, eb, 1.f);
          const bool same2 = same_side(za, zb);
          const float x2 = same2 ? ns2 : no2, xb2 = same2 ? no2 : ns2;
          const float den = (ns1 + no1) * (ns2 + no2);
          float num = fmaf(xb1, ns2 + no2, x1 * xb2);
          if constexpr (MASKED) {
            const bool skip = (j >= 1 && w == cd.w[j - 1]) || (j < K && w == cd.w[j]);
            num = skip ? den : num;
          }
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
    if constexpr (!MASKED) min_div = sigmoid_skip_divide<K>(s, cd, Qx, Qy, mx, my, mc, vis);
  }
  return min_div;
}

// TX image chain of a candidate (Sec. V-B): I_0 = TX, I_j = mirror of I_{j-1} in
// the line of wall w_j.  Independent of the receiver.
template <int K>
__device__ __forceinline__ void tx_images(const SmemWalls& s, float2 tx, const Cand& cd, float* Ix,
                                          float* Iy) {
  Ix[0] = tx.x;
  Iy[0] = tx.y;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const float4 G = s.G[cd.w[j - 1]];
    const float d = line_dist(G, Ix[j - 1], Iy[j - 1]);
    Ix[j] = fmaf(-2.f * d, G.x, Ix[j - 1]);
    Iy[j] = fmaf(-2.f * d, G.y, Iy[j - 1]);
  }
}

// Receiver-dependent geometry of one path: the reflection points (backtrace on
// the walls' infinite lines), each leg's line in smoothing-ready normal form,
// the path length L and the product V of the reflections' validities.
template <int MODE, int K>
struct PathGeom {
  float Qx[K + 2], Qy[K + 2];
  float mx[K + 1], my[K + 1], mc[K + 1];
  float L, V;
  bool degenerate;
};

template <int MODE, int K>
__device__ __forceinline__ void path_geometry(const SmemWalls& s, const float* Ix, const float* Iy,
                                              float2 tx, float2 rx, const Cand& cd, float alpha,
                                              PathGeom<MODE, K>& g) {
  // --- backtrace on the infinite lines: Q_{K+1} = RX, Q_j = line(Q_{j+1}, I_j) x wall j.
  g.Qx[0] = tx.x;
  g.Qy[0] = tx.y;
  g.Qx[K + 1] = rx.x;
  g.Qy[K + 1] = rx.y;
  g.degenerate = false;
#pragma unroll
  for (int j = K; j >= 1; --j) {
    const float4 G = s.G[cd.w[j - 1]];
    const float a = line_dist(G, Ix[j], Iy[j]);
    const float b = line_dist(G, g.Qx[j + 1], g.Qy[j + 1]);
    // parallel lines (or a reflection point absurdly far away): no path
    float t = __fdividef(b, b - a);
    if (!(fabsf(t) <= 1e8f)) {
      g.degenerate = true;
      t = 0.f;
    }
    g.Qx[j] = fmaf(t, Ix[j] - g.Qx[j + 1], g.Qx[j + 1]);
    g.Qy[j] = fmaf(t, Iy[j] - g.Qy[j + 1], g.Qy[j + 1]);
  }
  // --- legs: length and the smoothing-ready normal form of each leg's line.
  g.L = 0.f;
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    const float dx = g.Qx[j + 1] - g.Qx[j], dy = g.Qy[j + 1] - g.Qy[j];
    const float len2 = fmaf(dx, dx, dy * dy);
    g.degenerate |= !(len2 > 0.f);
    const float inv = rsqrtf(len2);
    g.L = fmaf(len2, inv, g.L);
    const float nx = -dy * inv, ny = dx * inv;
    const float nq = fmaf(nx, g.Qx[j], ny * g.Qy[j]);
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
  // --- continuous validity of each reflection (Sec. V-A): on the segment, and the
  //     previous and next vertices on the same side of the wall's line.
  g.V = 1.f;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const int w = cd.w[j - 1];
    const float4 G = s.G[w];
    const float t0 = s.T[w].x;
    const float tau = fmaf(G.y, g.Qx[j], fmaf(-G.x, g.Qy[j], -t0));   // u = (ny, -nx)
    const Smooth3 s1 = smooth3<MODE>(tau, alpha);
    const Smooth3 s2 = smooth3<MODE>(G.w - tau, alpha);
    const Smooth3 sp = smooth3<MODE>(line_dist(G, g.Qx[j - 1], g.Qy[j - 1]), alpha);
    const Smooth3 sq = smooth3<MODE>(line_dist(G, g.Qx[j + 1], g.Qy[j + 1]), alpha);
    g.V *= s1.s * s2.s * fmaf(sp.s, sq.s, sp.sb * sq.sb);
  }
}

// Path power from the geometry and the legs' visibilities (Eq. 7 term).
template <int MODE, int K>
__device__ __forceinline__ float path_power_of(const PathGeom<MODE, K>& g, const float* vis,
                                               float gk) {
  float p = g.V * gk;
#pragma unroll
  for (int j = 0; j <= K; ++j) p *= vis[j];
  p = __fdividef(p, g.L * g.L);
  return g.degenerate ? 0.f : p;
}

// Power of one path candidate of order K for this lane's receiver (Eq. 7 term).
template <int MODE, int K, bool MASKED = false>
__device__ __forceinline__ float path_power(const SmemWalls& s, int W, float2 tx, float2 rx,
                                            const Cand& cd, float alpha, float gk, int cull,
                                            float* vis_out = nullptr) {
  float Ix[K + 1], Iy[K + 1];
  tx_images<K>(s, tx, cd, Ix, Iy);
  PathGeom<MODE, K> g;
  path_geometry<MODE, K>(s, Ix, Iy, tx, rx, cd, alpha, g);
  // optional: skip the obstruction loop when the whole warp's validity is exactly 0
  if (cull && __all_sync(0xffffffffu, g.V == 0.f || g.degenerate)) return 0.f;
  // --- obstruction of every leg by every wall except the ones its end points lie on.
  float vis[K + 1];
  const float min_div = leg_visibility<MODE, K, MASKED>(s, W, cd, g.Qx, g.Qy, g.mx, g.my, g.mc, vis);
  if constexpr (!MASKED && MODE != MODE_STEP) {
    // A skipped pair's factor is >= 1/2 when its end point's distance to the wall's
    // line is accurate; a relaxed reflection point far along the line (large
    // backtrace ratio) can break that.  A warp with such a lane recomputes the
    // candidate with the skipped pairs masked (same function up to rounding).
    const bool bad = !g.degenerate && !(min_div >= 0.25f);
    if (__any_sync(0xffffffffu, bad))
      leg_visibility<MODE, K, true>(s, W, cd, g.Qx, g.Qy, g.mx, g.my, g.mc, vis);
  }
  if (vis_out) {
#pragma unroll
    for (int j = 0; j <= K; ++j) vis_out[j] = vis[j];
  }
  return path_power_of<MODE, K>(g, vis, gk);
}

}  // namespace drt
