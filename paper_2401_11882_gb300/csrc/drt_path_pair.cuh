// Path power for two receivers per lane (hard sigmoid and sigmoid).  The
// obstruction loop does the same operations on both receivers, so every
// floating-point operation that has a packed form (fma/add/mul.f32x2, without
// saturation) runs as one instruction on the pair; saturating FMAs, ex2, the
// sign tests and selects stay per receiver.  The loop issues far fewer
// instructions than two single-receiver loops for the same arithmetic, and the
// FMA pipe, not the issue rate, becomes the limit.  Results are those of
// path_power<MODE> bit for bit: the same operations in the same order, each
// rounded once (a packed FMA rounds each half like the scalar FMA).
#pragma once

#include "drt_path.cuh"

namespace drt {

// Wall records of the paired loop, each value duplicated into both halves of a
// register pair where the loop uses it as a packed operand; (hx, hy, hz, hw) is
// the mode's H record and (ax, ay, bx, by) the end points.
//   hard:     A = {hy, hy, hz, hz}   B = {hw, hw, ay, ay}   C = {by, by, ax, bx}
//   sigmoid:  A = {hx, hx, hy, hy}   B = {hz, hz, |hw|, |hw|}
//             C = {ax, ax, ay, ay}   D = {bx, bx, by, by}
struct SmemPairs {
  float4 *A, *B, *C, *D;
};

template <int MODE>
__device__ __forceinline__ void stage_pairs(const SmemWalls& s, int W, SmemPairs p) {
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    const float4 h = s.H[w], e = s.E[w];
    if (MODE == MODE_HARD) {
      p.A[w] = make_float4(h.y, h.y, h.z, h.z);
      p.B[w] = make_float4(h.w, h.w, e.y, e.y);
      p.C[w] = make_float4(e.w, e.w, e.x, e.z);
    } else {
      p.A[w] = make_float4(h.x, h.x, h.y, h.y);
      p.B[w] = make_float4(h.z, h.z, fabsf(h.w), fabsf(h.w));
      p.C[w] = make_float4(e.x, e.x, e.y, e.y);
      p.D[w] = make_float4(e.z, e.z, e.w, e.w);
    }
  }
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 ex2_pair(float2 z) {
  return f2(ex2_approx(-fabsf(z.x)), ex2_approx(-fabsf(z.y)));
}
// same_side for both receivers: one packed multiply, two compares
__device__ __forceinline__ void same_side2(float2 a, float2 b, bool& sx, bool& sy) {
  const float2 p = __fmul2_rn(a, b);
  sx = p.x > 0.f;
  sy = p.y > 0.f;
}

// Hard sigmoid: visibility of each leg of both receivers' paths, every wall
// tested (the skipped pairs are divided out by the caller).
// EXIT: once some leg of each of the warp's 64 paths has a visibility of exactly 0
// (a wall the hard sigmoid saturates to a full block), every power is 0 whatever
// the remaining walls do (0 stays 0 under each factor), so the warp leaves the
// wall loop; checked between blocks of 8 walls (a block has no exit inside, so it
// keeps the plain loop's schedule).
template <int K, bool EXIT = false>
__device__ __forceinline__ void hard_visibility_pair(const SmemWalls& s, const SmemPairs& p, int W,
                                                     const float2* Qx, const float2* Qy,
                                                     const float2* mx, const float2* my,
                                                     const float2* mc, float2* vis) {
  const float2 one = f2(1.f, 1.f), m2 = f2(-2.f, -2.f);
#pragma unroll
  for (int j = 0; j <= K; ++j) vis[j] = one;
  auto wall = [&](int w) {
    const float4 A = p.A[w], B = p.B[w], C = p.C[w];
    const float hx = s.H[w].x;
    const float2 hy = f2(A.x, A.y), hz = f2(A.z, A.w);
    const float2 ay = f2(B.z, B.w), by = f2(C.x, C.y);
    const float ax = C.z, bx = C.w;
    float2 sv[K + 2], uv[K + 2];
    sv[0] = f2(B.x, B.y);
#pragma unroll
    for (int i = 1; i <= K + 1; ++i) {
      const float2 t = fma2(hy, Qy[i], hz);
      sv[i] = f2(fma_sat(hx, Qx[i].x, t.x), fma_sat(hx, Qx[i].y, t.y));
    }
#pragma unroll
    for (int i = 1; i <= (K > 0 ? K : 1); ++i) uv[i] = fma2(m2, sv[i], one);
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      const float2 ta = fma2(my[j], ay, mc[j]);
      const float2 tb = fma2(my[j], by, mc[j]);
      const float2 sa = f2(fma_sat(mx[j].x, ax, ta.x), fma_sat(mx[j].y, ax, ta.y));
      const float2 sb = f2(fma_sat(mx[j].x, bx, tb.x), fma_sat(mx[j].y, bx, tb.y));
      const float2 x2 = fma2(sb, fma2(m2, sa, one), sa);
      const float2 x1 = (j == 0) ? fma2(sv[0], uv[1], sv[1]) : fma2(sv[j + 1], uv[j], sv[j]);
      vis[j] = fma2(f2(-vis[j].x, -vis[j].y), mul2(x1, x2), vis[j]);
    }
  };
  if (!EXIT) {
#pragma unroll 2
    for (int w = 0; w < W; ++w) wall(w);
    return;
  }
  for (int w0 = 0; w0 < W; w0 += 8) {
    if (w0 > 0) {
      bool z0 = false, z1 = false;
#pragma unroll
      for (int j = 0; j <= K; ++j) {
        z0 |= vis[j].x == 0.f;
        z1 |= vis[j].y == 0.f;
      }
      if (__all_sync(0xffffffffu, z0 && z1)) break;
    }
    const int we = min(w0 + 8, W);
#pragma unroll 2
    for (int w = w0; w < we; ++w) wall(w);
  }
}

// Sigmoid: the product form of leg_visibility<MODE_SIGMOID> on both receivers
// (numerator and denominator products folded into vis every 8 walls).
template <int K>
__device__ __forceinline__ void sigmoid_visibility_pair(const SmemWalls& s, const SmemPairs& p,
                                                        int W, const float2* Qx, const float2* Qy,
                                                        const float2* mx, const float2* my,
                                                        const float2* mc, float2* vis) {
  const float2 one = f2(1.f, 1.f);
  float2 vn[K + 1], vd[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) vis[j] = vn[j] = vd[j] = one;
  // one wall's factors for every leg, folded into vn, vd
  auto wall = [&](int w) {
    const float4 A = p.A[w], B = p.B[w], C = p.C[w], D = p.D[w];
    // the TX side: only the sign of H.w is used (as +-1, so that the same-side
    // product cannot underflow)
    const float zt = copysignf(1.f, s.H[w].w);
    const float2 hx = f2(A.x, A.y), hy = f2(A.z, A.w), hz = f2(B.x, B.y);
    const float2 ax = f2(C.x, C.y), ay = f2(C.z, C.w), bx = f2(D.x, D.y), by = f2(D.z, D.w);
    float2 ze[K + 2], ee[K + 2];
    ze[0] = f2(zt, zt);
    ee[0] = f2(B.z, B.w);
#pragma unroll
    for (int i = 1; i <= K + 1; ++i) {
      ze[i] = fma2(hx, Qx[i], fma2(hy, Qy[i], hz));
      ee[i] = ex2_pair(ze[i]);
    }
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      const float2 za = fma2(mx[j], ax, fma2(my[j], ay, mc[j]));
      const float2 zb = fma2(mx[j], bx, fma2(my[j], by, mc[j]));
      const float2 ea = ex2_pair(za), eb = ex2_pair(zb);
      const float2 ns1 = add2(ee[j], ee[j + 1]);
      const float2 no1 = fma2(ee[j], ee[j + 1], one);
      bool s1x, s1y;
      same_side2(ze[j], ze[j + 1], s1x, s1y);
      const float2 x1 = f2(s1x ? ns1.x : no1.x, s1y ? ns1.y : no1.y);
      const float2 xb1 = f2(s1x ? no1.x : ns1.x, s1y ? no1.y : ns1.y);
      const float2 ns2 = add2(ea, eb);
      const float2 no2 = fma2(ea, eb, one);
      bool s2x, s2y;
      same_side2(za, zb, s2x, s2y);
      const float2 x2 = f2(s2x ? ns2.x : no2.x, s2y ? ns2.y : no2.y);
      const float2 xb2 = f2(s2x ? no2.x : ns2.x, s2y ? no2.y : ns2.y);
      const float2 d2 = add2(ns2, no2);
      const float2 den = mul2(add2(ns1, no1), d2);
      const float2 num = fma2(xb1, d2, mul2(x1, xb2));
      vn[j] = mul2(vn[j], num);
      vd[j] = mul2(vd[j], den);
    }
  };
  for (int w0 = 0; w0 < W; w0 += 8) {
    if (w0 + 8 <= W) {   // a full block of 8 walls: unrolled, for independent work
#pragma unroll
      for (int i = 0; i < 8; ++i) wall(w0 + i);
    } else {
      for (int w = w0; w < W; ++w) wall(w);
    }
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      vis[j] = mul2(vis[j], f2(__fdividef(vn[j].x, vd[j].x), __fdividef(vn[j].y, vd[j].y)));
      vn[j] = vd[j] = one;
    }
  }
}

// Powers of one path candidate of order K for the receivers rx0 and rx1.
template <int MODE, int K, bool EXIT = false>
__device__ __forceinline__ float2 path_power_pair(const SmemWalls& s, const SmemPairs& p, int W,
                                                  float2 tx, float2 rx0, float2 rx1, const Cand& cd,
                                                  float alpha, float gk, int cull,
                                                  float2* vis_out = nullptr) {
  float Ix[K + 1], Iy[K + 1];
  tx_images<K>(s, tx, cd, Ix, Iy);
  PathGeom<MODE, K> g0, g1;
  path_geometry<MODE, K>(s, Ix, Iy, tx, rx0, cd, alpha, g0);
  path_geometry<MODE, K>(s, Ix, Iy, tx, rx1, cd, alpha, g1);
  if (cull && __all_sync(0xffffffffu, (g0.V == 0.f || g0.degenerate) &&
                                          (g1.V == 0.f || g1.degenerate)))
    return f2(0.f, 0.f);
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
    hard_visibility_pair<K, EXIT>(s, p, W, Qx, Qy, mx, my, mc, vis2);
  else
    sigmoid_visibility_pair<K>(s, p, W, Qx, Qy, mx, my, mc, vis2);
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
  // as in path_power: a lane whose divided-out factor is unreliably small
  // recomputes with the skipped pairs masked
  if (__any_sync(0xffffffffu, !g0.degenerate && !(d0 >= 0.25f)))
    leg_visibility<MODE, K, true>(s, W, cd, g0.Qx, g0.Qy, g0.mx, g0.my, g0.mc, vis0);
  if (__any_sync(0xffffffffu, !g1.degenerate && !(d1 >= 0.25f)))
    leg_visibility<MODE, K, true>(s, W, cd, g1.Qx, g1.Qy, g1.mx, g1.my, g1.mc, vis1);
  if (vis_out) {
#pragma unroll
    for (int j = 0; j <= K; ++j) vis_out[j] = f2(vis0[j], vis1[j]);
  }
  return f2(path_power_of<MODE, K>(g0, vis0, gk), path_power_of<MODE, K>(g1, vis1, gk));
}

}  // namespace drt
