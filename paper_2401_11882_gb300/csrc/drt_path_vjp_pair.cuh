// Sigmoid adjoint with two receivers per lane (tiles of 64 receivers: lane l
// holds receivers l and l + 32 of its tile, for the same warp-uniform path
// candidate).  The per-path O(K) work (recompute, factor adjoints, the reverse
// of the backtrace and image chain) runs once per receiver as in path_vjp; the
// two O(K W) sweeps over the walls run both receivers in packed FP32 pairs
// (fma/mul/add.f32x2), so each of their floating-point operations issues once
// for the pair; ex2, rcp, the sign tests and selects stay per receiver.  The
// per-wall adjoints of the two receivers are added in the lane before the warp
// reduction, which is then shared by 64 receivers.
//
// Sweep 1 is sigmoid_vis_sweep's product form without the zero count: a factor
// that is exactly 0 (an FP32 underflow of the sigmoid) or a product that
// underflows makes the leg's visibility 0, and such a path has an exactly-zero
// gradient either way (see path_vjp), so the lane only needs to know that it is
// dead.  Sweep 2 is path_vjp's rational form, with the two denominators taken as
// D = Ns + No (the forward's form) and each vertex's e factored out of its
// accumulated adjoint.
#pragma once

#include "drt_path_pair.cuh"
#include "drt_path_vjp.cuh"

namespace drt {

// Paired wall records of the adjoint, each value duplicated into both halves of a
// register pair: the forward's sigmoid records (A = {hx, hx, hy, hy}, B = {hz, hz,
// |hw|, |hw|}, C = {ax, ax, ay, ay}, D = {bx, bx, by, by}) and the unit normal
// N = {nx, nx, ny, ny}.
struct SmemPairsVjp {
  float4 *A, *B, *C, *D, *N;
};

__device__ __forceinline__ void stage_pairs_vjp(const VSmem& s, int W, SmemPairsVjp p) {
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    const float4 h = s.H[w], e = s.E[w], g = s.G[w];
    p.A[w] = make_float4(h.x, h.x, h.y, h.y);
    p.B[w] = make_float4(h.z, h.z, fabsf(h.w), fabsf(h.w));
    p.C[w] = make_float4(e.x, e.x, e.y, e.y);
    p.D[w] = make_float4(e.z, e.z, e.w, e.w);
    p.N[w] = make_float4(g.x, g.x, g.y, g.y);
  }
}

__device__ __forceinline__ float2 copysign2(float2 v, float2 sgn) {
  return f2(copysignf(v.x, sgn.x), copysignf(v.y, sgn.y));
}

// Both smoothed pairs of one (leg, wall) factor in the product form, per
// receiver: x = X, xb = 1 - X, times D (see leg_visibility's sigmoid loop).
struct PairTerms {
  float2 x1, xb1, x2, xb2, D1, D2;
};

__device__ __forceinline__ PairTerms pair_terms(float2 e0, float2 e1, float2 z0, float2 z1,
                                                float2 ea, float2 eb, float2 za, float2 zb) {
  const float2 one = f2(1.f, 1.f);
  PairTerms t;
  const float2 ns1 = add2(e0, e1), no1 = fma2(e0, e1, one);
  bool s1x, s1y;
  same_side2(z0, z1, s1x, s1y);
  t.x1 = f2(s1x ? ns1.x : no1.x, s1y ? ns1.y : no1.y);
  t.xb1 = f2(s1x ? no1.x : ns1.x, s1y ? no1.y : ns1.y);
  const float2 ns2 = add2(ea, eb), no2 = fma2(ea, eb, one);
  bool s2x, s2y;
  same_side2(za, zb, s2x, s2y);
  t.x2 = f2(s2x ? ns2.x : no2.x, s2y ? ns2.y : no2.y);
  t.xb2 = f2(s2x ? no2.x : ns2.x, s2y ? no2.y : ns2.y);
  t.D1 = add2(ns1, no1);
  t.D2 = add2(ns2, no2);
  return t;
}

// Sweep 1, both receivers: each leg's visibility (the leg's own walls masked),
// numerator and denominator products folded every 8 walls.
template <int K>
__device__ __forceinline__ void sigmoid_vis_sweep_pair(const VSmem& s, const SmemPairsVjp& p,
                                                       int W, const Cand& cd, const float2* Qx,
                                                       const float2* Qy, const float2* mxk,
                                                       const float2* myk, const float2* mck,
                                                       float2* vis) {
  const float2 one = f2(1.f, 1.f);
  float2 vn[K + 1], vd[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) vis[j] = vn[j] = vd[j] = one;
  auto wall = [&](int w) {
    const float4 A = p.A[w], B = p.B[w], C = p.C[w], D = p.D[w];
    const float zt = copysignf(1.f, s.H[w].w);   // the TX side: only the sign is used
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
      const bool skip = (j >= 1 && w == cd.w[j - 1]) || (j < K && w == cd.w[j]);
      if (skip) continue;
      const float2 za = fma2(mxk[j], ax, fma2(myk[j], ay, mck[j]));
      const float2 zb = fma2(mxk[j], bx, fma2(myk[j], by, mck[j]));
      const PairTerms t = pair_terms(ee[j], ee[j + 1], ze[j], ze[j + 1], ex2_pair(za),
                                     ex2_pair(zb), za, zb);
      const float2 num = fma2(t.xb1, t.D2, mul2(t.x1, t.xb2));
      vn[j] = mul2(vn[j], num);
      vd[j] = mul2(vd[j], mul2(t.D1, t.D2));
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

// Sweep 2, both receivers: the adjoint of every (leg, wall) factor f = 1 - X1 X2
// in rational form.  With e = 2^-|z| per smoothed distance, F = 1 - e^2 and
// D = Ns + No = (1 + e_x)(1 + e_y) per pair,
//   dX/dx = -alpha sign(y) e_x F_y / D^2   (and symmetrically in y),
// so with t = Wa / (num D1 D2) (Wa = the leg's visibility adjoint times its
// visibility and alpha) the two vertex distances of the leg get
// t X2 D2 e F of the other vertex, and the wall's end points t X1 D1 e F of the
// other end point.  Wa = 0 in a dead lane; the guard keeps t finite there.
template <int K, bool WG>
__device__ __forceinline__ void sigmoid_adjoint_sweep_pair(
    const VSmem& s, const SmemPairsVjp& p, int W, const Cand& cd, const float2* Qx,
    const float2* Qy, const float2* mxk, const float2* myk, const float2* mck, float inv_kap,
    const float2* Wa, float2* Qbx, float2* Qby, float2* mAx, float2* mAy, float2* sm) {
  const float2 one = f2(1.f, 1.f);
  const float2 tiny = f2(SIGMOID_VJP_TINY, SIGMOID_VJP_TINY);
  for (int w = 0; w < W; ++w) {
    const float4 A = p.A[w], B = p.B[w], C = p.C[w], D = p.D[w], N = p.N[w];
    const float zt = copysignf(1.f, s.H[w].w);
    const float2 hx = f2(A.x, A.y), hy = f2(A.z, A.w), hz = f2(B.x, B.y);
    const float2 ax = f2(C.x, C.y), ay = f2(C.z, C.w), bx = f2(D.x, D.y), by = f2(D.z, D.w);
    const float2 nx = f2(N.x, N.y), ny = f2(N.z, N.w);
    float2 ze[K + 2], ev[K + 2], sF[K + 2], vb[K + 2];
    ze[0] = f2(zt, zt);
    ev[0] = f2(B.z, B.w);
#pragma unroll
    for (int i = 1; i <= K + 1; ++i) {
      ze[i] = fma2(hx, Qx[i], fma2(hy, Qy[i], hz));
      ev[i] = ex2_pair(ze[i]);
    }
#pragma unroll
    for (int i = 0; i <= K + 1; ++i) {
      sF[i] = copysign2(fma2(f2(-ev[i].x, -ev[i].y), ev[i], one), ze[i]);
      vb[i] = f2(0.f, 0.f);
    }
    float2 Abx = f2(0.f, 0.f), Aby = Abx, Bbx = Abx, Bby = Abx;
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      const bool skip = (j >= 1 && w == cd.w[j - 1]) || (j < K && w == cd.w[j]);
      if (skip) continue;
      const float2 za = fma2(mxk[j], ax, fma2(myk[j], ay, mck[j]));
      const float2 zb = fma2(mxk[j], bx, fma2(myk[j], by, mck[j]));
      const float2 ea = ex2_pair(za), eb = ex2_pair(zb);
      const PairTerms t = pair_terms(ev[j], ev[j + 1], ze[j], ze[j + 1], ea, eb, za, zb);
      const float2 num = fma2(t.xb1, t.D2, mul2(t.x1, t.xb2));
      const float2 q = fma2(num, mul2(t.D1, t.D2), tiny);
      const float2 tw = mul2(Wa[j], f2(rcp_approx(q.x), rcp_approx(q.y)));
      const float2 c1 = mul2(mul2(tw, t.x2), t.D2);
      const float2 c2 = mul2(mul2(tw, t.x1), t.D1);
      // vertex distances d(Q_j), d(Q_{j+1}); each vertex's own e is applied below
      vb[j] = fma2(c1, sF[j + 1], vb[j]);
      vb[j + 1] = fma2(c1, sF[j], vb[j + 1]);
      const float2 sFa = copysign2(fma2(f2(-ea.x, -ea.y), ea, one), za);
      const float2 sFb = copysign2(fma2(f2(-eb.x, -eb.y), eb, one), zb);
      const float2 x2b = mul2(mul2(c2, ea), sFb), y2b = mul2(mul2(c2, eb), sFa);
      // x2 = m . (A - Q_j), y2 = m . (B - Q_j)
      mAx[j] = fma2(x2b, ax, fma2(y2b, bx, mAx[j]));
      mAy[j] = fma2(x2b, ay, fma2(y2b, by, mAy[j]));
      sm[j] = add2(sm[j], add2(x2b, y2b));
      if (WG) {   // against the scaled normal: times 1 / (alpha log2 e) below
        Abx = fma2(x2b, mxk[j], Abx);
        Aby = fma2(x2b, myk[j], Aby);
        Bbx = fma2(y2b, mxk[j], Bbx);
        Bby = fma2(y2b, myk[j], Bby);
      }
    }
    // vertex distances d(Q_i) = n . Q_i - c
    float2 nbx = f2(0.f, 0.f), nby = nbx, cb = nbx;
#pragma unroll
    for (int i = 0; i <= K + 1; ++i) {
      const float2 v = mul2(vb[i], ev[i]);
      Qbx[i] = fma2(v, nx, Qbx[i]);
      Qby[i] = fma2(v, ny, Qby[i]);
      if (WG) {
        nbx = fma2(v, Qx[i], nbx);
        nby = fma2(v, Qy[i], nby);
        cb = add2(cb, v);
      }
    }
    if (WG)
      add_wall_adjoint(s, w, nbx.x + nbx.y, nby.x + nby.y, -(cb.x + cb.y),
                       (Abx.x + Abx.y) * inv_kap, (Aby.x + Aby.y) * inv_kap,
                       (Bbx.x + Bbx.y) * inv_kap, (Bby.x + Bby.y) * inv_kap);
  }
}

// Adjoint of one path candidate of order K for the receivers rx0 and rx1 (weights
// g0, g1) of this lane; adds both receivers' TX adjoints to (txb_x, txb_y).
template <int K, bool WG>
__device__ __forceinline__ void path_vjp_pair(const VSmem& s, const SmemPairsVjp& p, int W,
                                              float2 tx, float2 rx0, float2 rx1, const Cand& cd,
                                              float alpha, float gk, float g0, float g1,
                                              float& txb_x, float& txb_y,
                                              const float* saved0 = nullptr,
                                              const float* saved1 = nullptr,
                                              long long saved_stride = 0) {
  float2 Qx[K + 2], Qy[K + 2], mxk[K + 1], myk[K + 1], mck[K + 1];
  float V0[K + 1], V1[K + 1];
  float L0, L1;
  bool dead0, dead1;
  {
    VjpPath<K> P0, P1;
    vjp_recompute<MODE_SIGMOID, K>(s, tx, rx0, cd, alpha, P0);
    vjp_recompute<MODE_SIGMOID, K>(s, tx, rx1, cd, alpha, P1);
    dead0 = P0.degenerate || g0 == 0.f;
    dead1 = P1.degenerate || g1 == 0.f;
#pragma unroll
    for (int j = 1; j <= K; ++j) {
      dead0 |= (P0.V[j] == 0.f);
      dead1 |= (P1.V[j] == 0.f);
    }
    if (__all_sync(FULL, dead0 && dead1)) return;
    const float kap = alpha * LOG2E;
#pragma unroll
    for (int i = 0; i <= K + 1; ++i) {
      Qx[i] = f2(P0.Qx[i], P1.Qx[i]);
      Qy[i] = f2(P0.Qy[i], P1.Qy[i]);
    }
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      mxk[j] = f2(P0.mx[j] * kap, P1.mx[j] * kap);
      myk[j] = f2(P0.my[j] * kap, P1.my[j] * kap);
      mck[j] = f2(-P0.mq[j] * kap, -P1.mq[j] * kap);
      V0[j] = P0.V[j];
      V1[j] = P1.V[j];
    }
    L0 = P0.L;
    L1 = P1.L;
  }
  // ------------------------------------------------ sweep 1: visibilities
  float2 vis[K + 1];
  if (saved0) {   // the forward's visibilities of this path (sweep 1 done there)
    // a path the forward found degenerate has no finite visibilities there: such
    // lanes, and lanes already at weight 0, take 1 (their weight stays an exact 0)
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      vis[j] = f2(__ldg(saved0 + j * saved_stride), __ldg(saved1 + j * saved_stride));
      dead0 |= (vis[j].x != vis[j].x);
      dead1 |= (vis[j].y != vis[j].y);
    }
#pragma unroll
    for (int j = 0; j <= K; ++j) vis[j] = f2(dead0 ? 1.f : vis[j].x, dead1 ? 1.f : vis[j].y);
  } else {
    sigmoid_vis_sweep_pair<K>(s, p, W, cd, Qx, Qy, mxk, myk, mck, vis);
  }
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    dead0 |= (vis[j].x == 0.f);
    dead1 |= (vis[j].y == 0.f);
  }
  if (__all_sync(FULL, dead0 && dead1)) return;
  // ------------------------------------------------ factor adjoints (per receiver)
  float2 Wa[K + 1];
  float Vb0[K + 1], Vb1[K + 1], Lb0, Lb1;
  {
    float nz0[K + 1], nz1[K + 1];
    int zc[K + 1];
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      nz0[j] = vis[j].x;
      nz1[j] = vis[j].y;
      zc[j] = 0;
    }
    VjpPath<K> P;   // only V and L are read by the power's factor adjoints
#pragma unroll
    for (int j = 0; j <= K; ++j) P.V[j] = V0[j];
    P.L = L0;
    VjpFactorAdj<K> A0, A1;
    vjp_factor_adjoints<K, false>(s, cd, P, nz0, zc, dead0 ? 0.f : g0, gk, nullptr, A0);
#pragma unroll
    for (int j = 0; j <= K; ++j) P.V[j] = V1[j];
    P.L = L1;
    vjp_factor_adjoints<K, false>(s, cd, P, nz1, zc, dead1 ? 0.f : g1, gk, nullptr, A1);
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      Wa[j] = f2(A0.visb[j] * nz0[j] * alpha, A1.visb[j] * nz1[j] * alpha);
      Vb0[j] = A0.Vb[j];
      Vb1[j] = A1.Vb[j];
    }
    Lb0 = A0.Lb;
    Lb1 = A1.Lb;
  }
  // ------------------------------------------------ sweep 2: obstruction adjoint
  float2 Qbx[K + 2], Qby[K + 2], mAx[K + 1], mAy[K + 1], sm[K + 1];
#pragma unroll
  for (int i = 0; i <= K + 1; ++i) Qbx[i] = Qby[i] = f2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j <= K; ++j) mAx[j] = mAy[j] = sm[j] = f2(0.f, 0.f);
  // (at alpha = 0 every weight is 0 and the scaled normals are 0: no rescale)
  const float inv_kap = alpha > 0.f ? 1.f / (alpha * LOG2E) : 0.f;
  sigmoid_adjoint_sweep_pair<K, WG>(s, p, W, cd, Qx, Qy, mxk, myk, mck, inv_kap, Wa, Qbx, Qby,
                                    mAx, mAy, sm);
  // ------------------------------------------------ legs, validity, backtrace, images
  // (the path is recomputed per receiver: O(K) work, fewer live registers)
  VjpReflAdj<K> R0, R1;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    VjpPath<K> P;
    vjp_recompute<MODE_SIGMOID, K>(s, tx, h ? rx1 : rx0, cd, alpha, P);
    VjpFactorAdj<K> A;
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      A.Vb[j] = h ? Vb1[j] : Vb0[j];
      A.visb[j] = A.cosb[j] = 0.f;
    }
    A.Lb = h ? Lb1 : Lb0;
    float qbx[K + 2], qby[K + 2], max_[K + 1], may_[K + 1], sm_[K + 1];
#pragma unroll
    for (int i = 0; i <= K + 1; ++i) {
      qbx[i] = h ? Qbx[i].y : Qbx[i].x;
      qby[i] = h ? Qby[i].y : Qby[i].x;
    }
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      max_[j] = h ? mAx[j].y : mAx[j].x;
      may_[j] = h ? mAy[j].y : mAy[j].x;
      sm_[j] = h ? sm[j].y : sm[j].x;
    }
    vjp_backprop<MODE_SIGMOID, K, false>(s, cd, P, alpha, A, qbx, qby, max_, may_, sm_, txb_x,
                                         txb_y, h ? R1 : R0);
  }
  if (WG) {
#pragma unroll
    for (int j = 1; j <= K; ++j) {
      R0.nx[j] += R1.nx[j];
      R0.ny[j] += R1.ny[j];
      R0.c[j] += R1.c[j];
      R0.t0[j] += R1.t0[j];
      R0.len[j] += R1.len[j];
    }
    vjp_emit_reflections<K, true>(s, cd, R0);
  }
}

}  // namespace drt
