// Per-path adjoint shared by the single-scene and batched adjoint kernels:
// recompute one path candidate for one receiver and push the adjoint of its
// power into the transmitter, the path vertices and the walls (Sec. III:
// gradient of the loss with respect to the scene parameters).
#pragma once

#include "drt_common.cuh"
#include "drt_internal.h"
#include "drt_path.cuh"

namespace drt {

constexpr unsigned FULL = 0xffffffffu;

// Added to the sigmoid adjoint's denominators (the smallest normal FP32 value,
// rounded up): keeps the reciprocal finite in a lane whose weight is 0.
constexpr float SIGMOID_VJP_TINY = 1.2e-38f;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Slots of the per-wall accumulator.
enum : int { S_NX = 0, S_NY, S_C, S_AX, S_AY, S_BX, S_BY, S_T0, S_LEN };

// Staged walls (the forward's records: G, E, T and the mode's H record, see
// stage_walls) and the per-CTA wall-gradient accumulator.
struct VSmem {
  float4 *G, *E, *T, *H;
  float* acc;   // [W][VJP_SLOTS] (wall gradient only)
};

// Sums v[0..7] over the warp by recursive halving: lane l ends with the warp
// total of v[(l >> 2) & 7] (each total held by 4 lanes); 9 shuffles instead of
// 40 for eight separate butterfly sums.
__device__ __forceinline__ float warp_reduce_scatter8(const float* v) {
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float a[4], c[2];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float keep = b4 ? v[k + 4] : v[k], send = b4 ? v[k] : v[k + 4];
    a[k] = keep + __shfl_xor_sync(FULL, send, 16);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float keep = b3 ? a[k + 2] : a[k], send = b3 ? a[k] : a[k + 2];
    c[k] = keep + __shfl_xor_sync(FULL, send, 8);
  }
  float d = (b2 ? c[1] : c[0]) + __shfl_xor_sync(FULL, b2 ? c[0] : c[1], 4);
  d += __shfl_xor_sync(FULL, d, 2);
  d += __shfl_xor_sync(FULL, d, 1);
  return d;
}

// Adds the warp's adjoints of one wall's (n, c, A, B) into the CTA table (the
// wall is the same in every lane, whatever candidate each lane holds).
__device__ __forceinline__ void add_wall_adjoint(const VSmem& s, int w, float nbx, float nby,
                                                 float cb, float Abx, float Aby, float Bbx,
                                                 float Bby) {
  const float v[8] = {nbx, nby, cb, Abx, Aby, Bbx, Bby, 0.f};   // slots S_NX .. S_BY
  const float t = warp_reduce_scatter8(v);
  const int lane = threadIdx.x & 31, slot = (lane >> 2) & 7;
  if ((lane & 3) == 0 && slot <= S_BY) atomicAdd(&s.acc[w * VJP_SLOTS + slot], t);
}

// Sigmoid, sweep 1 of the adjoint: each leg's visibility in the forward's
// product form (e = 2^-|z|, numerator and denominator products folded every 8
// walls), the leg's own walls masked.  A factor that is exactly 0 (an FP32
// underflow) makes the visibility 0, and so does a product that underflows; either
// way the path's gradient is exactly 0 (see path_vjp), so no zero count is kept
// (zc stays 0).  mxk, myk, mck: the leg's line scaled by alpha log2(e), as the
// forward's.
template <int K>
__device__ __forceinline__ void sigmoid_vis_sweep(const VSmem& s, int W, const Cand& cd,
                                                  const float* Qx, const float* Qy,
                                                  const float* mxk, const float* myk,
                                                  const float* mck, float* nz, int* zc) {
  float vn[K + 1], vd[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    nz[j] = vn[j] = vd[j] = 1.f;
    zc[j] = 0;
  }
  // one wall's factors for every leg (the leg's own walls masked)
  auto wall = [&](int w) {
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
      const bool skip = (j >= 1 && w == cd.w[j - 1]) || (j < K && w == cd.w[j]);
      if (skip) continue;
      const float za = fmaf(mxk[j], e.x, fmaf(myk[j], e.y, mck[j]));
      const float zb = fmaf(mxk[j], e.z, fmaf(myk[j], e.w, mck[j]));
      const float ea = ex2_approx(-fabsf(za)), eb = ex2_approx(-fabsf(zb));
      const float ns1 = ee[j] + ee[j + 1], no1 = fmaf(ee[j], ee[j + 1], 1.f);
      const bool same1 = same_side(ze[j], ze[j + 1]);
      const float x1 = same1 ? ns1 : no1, xb1 = same1 ? no1 : ns1;
      const float ns2 = ea + eb, no2 = fmaf(ea, eb, 1.f);
      const bool same2 = same_side(za, zb);
      const float xb2 = same2 ? no2 : ns2;
      const float d2 = ns2 + no2;
      vn[j] *= fmaf(xb1, d2, x1 * xb2);
      vd[j] *= (ns1 + no1) * d2;
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
      nz[j] *= __fdividef(vn[j], vd[j]);
      vn[j] = vd[j] = 1.f;
    }
  }
}

// One leg x wall factor f = 1 - X(x1, y1) X(x2, y2), written as
// Xb1 + X1 Xb2 with Xb = 1 - X = s(x) s(y) + s(-x) s(-y), and its partials.
struct LegWall {
  float f, dx1, dy1, dx2, dy2;
};

template <int MODE, bool GRAD>
__device__ __forceinline__ LegWall leg_wall(float x1, float y1, float x2, float y2, float alpha) {
  const Smooth3 a = smooth3<MODE>(x1, alpha), b = smooth3<MODE>(y1, alpha);
  const Smooth3 c = smooth3<MODE>(x2, alpha), d = smooth3<MODE>(y2, alpha);
  const float X1 = fmaf(a.s, b.sb, a.sb * b.s), Xb1 = fmaf(a.s, b.s, a.sb * b.sb);
  const float X2 = fmaf(c.s, d.sb, c.sb * d.s), Xb2 = fmaf(c.s, d.s, c.sb * d.sb);
  LegWall r;
  r.f = fmaf(X1, Xb2, Xb1);
  if (GRAD) {
    // df/dX1 = -X2, df/dX2 = -X1; dX/dx = s'(x) (s(-y) - s(y)), dX/dy = s'(y) (s(-x) - s(x))
    r.dx1 = -X2 * a.ds * (b.sb - b.s);
    r.dy1 = -X2 * b.ds * (a.sb - a.s);
    r.dx2 = -X1 * c.ds * (d.sb - d.s);
    r.dy2 = -X1 * d.ds * (c.sb - c.s);
  } else {
    r.dx1 = r.dy1 = r.dx2 = r.dy2 = 0.f;
  }
  return r;
}

// Coherent field (FIELD): this lane's weight w = 2 g conj(E) on the path fields
// a = prod_j C_j V vis exp(-i 2 pi L / lambda) / L (the adjoint of |E|^2 with
// cotangent g is Re(w da)), and the field's constants.
struct FieldW {
  float wre, wim;                        // w = wre + i wim
  float inv_lambda_hi, inv_lambda_lo;    // 1 / lambda as a float pair
  float k2pi;                            // 2 pi / lambda
  float eps_r;                           // > 1: Fresnel TE; 0: the constant refl_amp
  float refl_amp;
};

// Forward values of one path, recomputed for its adjoint: image chain, reflection
// points, legs and the validity of each reflection.
template <int K>
struct VjpPath {
  float Ix[K + 1], Iy[K + 1], dimg[K + 1];       // images and their distances to the walls
  float Qx[K + 2], Qy[K + 2];                    // vertices TX, X_1..X_K, RX
  float ta[K + 1], tb[K + 1], tt[K + 1];         // backtrace: a, b and t = b / (b - a)
  float mx[K + 1], my[K + 1], mq[K + 1], len[K + 1];   // leg normals, offsets, lengths
  float L;                                       // path length (1 for a degenerate path)
  float V[K + 1];                                // V_1..V_K
  bool degenerate;
};

template <int MODE, int K>
__device__ __forceinline__ void vjp_recompute(const VSmem& s, float2 tx, float2 rx, const Cand& cd,
                                              float alpha, VjpPath<K>& P) {
  P.Ix[0] = tx.x;
  P.Iy[0] = tx.y;
  P.dimg[0] = 0.f;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const float4 G = s.G[cd.w[j - 1]];
    P.dimg[j] = line_dist(G, P.Ix[j - 1], P.Iy[j - 1]);
    P.Ix[j] = fmaf(-2.f * P.dimg[j], G.x, P.Ix[j - 1]);
    P.Iy[j] = fmaf(-2.f * P.dimg[j], G.y, P.Iy[j - 1]);
  }
  P.Qx[0] = tx.x;
  P.Qy[0] = tx.y;
  P.Qx[K + 1] = rx.x;
  P.Qy[K + 1] = rx.y;
  P.degenerate = false;
#pragma unroll
  for (int j = K; j >= 1; --j) {
    const float4 G = s.G[cd.w[j - 1]];
    P.ta[j] = line_dist(G, P.Ix[j], P.Iy[j]);
    P.tb[j] = line_dist(G, P.Qx[j + 1], P.Qy[j + 1]);
    float t = __fdiv_rn(P.tb[j], P.tb[j] - P.ta[j]);
    if (!(fabsf(t) <= 1e8f)) {
      P.degenerate = true;
      t = 0.f;
    }
    P.tt[j] = t;
    P.Qx[j] = fmaf(t, P.Ix[j] - P.Qx[j + 1], P.Qx[j + 1]);
    P.Qy[j] = fmaf(t, P.Iy[j] - P.Qy[j + 1], P.Qy[j + 1]);
  }
  P.L = 0.f;
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    const float dx = P.Qx[j + 1] - P.Qx[j], dy = P.Qy[j + 1] - P.Qy[j];
    const float len2 = fmaf(dx, dx, dy * dy);
    float inv = 0.f;
    if (len2 > 0.f) {
      inv = rsqrtf(len2);
    } else {
      P.degenerate = true;
    }
    P.len[j] = len2 * inv;
    P.L += P.len[j];
    P.mx[j] = -dy * inv;
    P.my[j] = dx * inv;
    P.mq[j] = fmaf(P.mx[j], P.Qx[j], P.my[j] * P.Qy[j]);
  }
  if (P.degenerate) P.L = 1.f;
  P.V[0] = 1.f;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const int w = cd.w[j - 1];
    const float4 G = s.G[w];
    const float tau = fmaf(G.y, P.Qx[j], fmaf(-G.x, P.Qy[j], -s.T[w].x));
    const Smooth3 s1 = smooth3<MODE>(tau, alpha), s2 = smooth3<MODE>(G.w - tau, alpha);
    const Smooth3 sp = smooth3<MODE>(line_dist(G, P.Qx[j - 1], P.Qy[j - 1]), alpha);
    const Smooth3 sq = smooth3<MODE>(line_dist(G, P.Qx[j + 1], P.Qy[j + 1]), alpha);
    P.V[j] = s1.s * s2.s * fmaf(sp.s, sq.s, sp.sb * sq.sb);
  }
}

// Adjoints of the path's factors (p = C prod(F), C = Gamma^k / L^2, F = {V_1..V_K,
// vis_0..vis_K}; for FIELD the path field's amplitude and phase): Vb, visb, the
// path length's Lb and, for FIELD, the incidence cosines' cosb.
template <int K>
struct VjpFactorAdj {
  float Vb[K + 1], visb[K + 1], cosb[K + 1];
  float Lb;
};

template <int K, bool FIELD>
__device__ __forceinline__ void vjp_factor_adjoints(const VSmem& s, const Cand& cd,
                                                    const VjpPath<K>& P, const float* nz,
                                                    const int* zc, float g, float gk,
                                                    const FieldW* fw, VjpFactorAdj<K>& A) {
  constexpr int NF = 2 * K + 1;
  float F[NF];
#pragma unroll
  for (int j = 1; j <= K; ++j) F[j - 1] = P.V[j];
#pragma unroll
  for (int j = 0; j <= K; ++j) F[K + j] = zc[j] ? 0.f : nz[j];
  float pre[NF + 1], suf[NF + 1];
  pre[0] = 1.f;
#pragma unroll
  for (int i = 0; i < NF; ++i) pre[i + 1] = pre[i] * F[i];
  suf[NF] = 1.f;
#pragma unroll
  for (int i = NF - 1; i >= 0; --i) suf[i] = suf[i + 1] * F[i];
  float gC, p = 0.f;
  const float L = P.L;
#pragma unroll
  for (int j = 0; j <= K; ++j) A.cosb[j] = 0.f;
  if constexpr (!FIELD) {
    const float C = __fdiv_rn(gk, L * L);
    p = C * pre[NF];
    gC = g * C;
  } else {
    // a = A exp(-i phi), A = prod_j C_j(c_j) prod(F) / L, phi = 2 pi L / lambda:
    // Re(w da) = A_bar dA + phi_bar dphi with A_bar = Re(w e^{-i phi}) and
    // phi_bar = A Im(w e^{-i phi}).  c_j = |n_j . d| / |d| for the leg d arriving
    // at reflection j; C_j the Fresnel TE coefficient, dC/dc = 2 (eps - 1) / (r (c + r)^2)
    // with r = sqrt(eps - 1 + c^2), or the constant (dC/dc = 0).
    float Cj[K + 1], dC[K + 1];
    float Cf = 1.f;
#pragma unroll
    for (int j = 1; j <= K; ++j) {
      const float4 G = s.G[cd.w[j - 1]];
      const float dx = P.Qx[j] - P.Qx[j - 1], dy = P.Qy[j] - P.Qy[j - 1];
      const float il = P.len[j - 1] > 0.f ? __frcp_rn(P.len[j - 1]) : 0.f;
      const float c = fminf(fabsf(fmaf(G.x, dx, G.y * dy)) * il, 1.f);
      Cj[j] = fw->refl_amp;
      dC[j] = 0.f;
      if (fw->eps_r > 0.f) {
        const float x = fmaf(c, c, fw->eps_r - 1.f);
        const float root = x > 0.f ? x * rsqrtf(x) : 0.f;
        const float den = c + root;
        Cj[j] = den > 0.f ? __fdividef(c - root, den) : 0.f;
        dC[j] = root > 0.f ? __fdividef(2.f * (fw->eps_r - 1.f), root * den * den) : 0.f;
      }
      Cf *= Cj[j];
    }
    const float iL = __frcp_rn(L);
    const float Am = Cf * pre[NF] * iL;
    const float cyc = L * fw->inv_lambda_hi;
    const float cer = fmaf(L, fw->inv_lambda_hi, -cyc);
    const float frac = (cyc - rintf(cyc)) + fmaf(L, fw->inv_lambda_lo, cer);
    float sph, cph;
    sincospif(2.f * frac, &sph, &cph);
    const float Ab = g * fmaf(fw->wre, cph, fw->wim * sph);
    const float phb = g * Am * fmaf(fw->wim, cph, -fw->wre * sph);
    gC = Ab * Cf * iL;
    A.Lb = fmaf(-Ab, Am * iL, phb * fw->k2pi);
#pragma unroll
    for (int j = 1; j <= K; ++j) {
      float others = 1.f;
#pragma unroll
      for (int i = 1; i <= K; ++i)
        if (i != j) others *= Cj[i];
      A.cosb[j] = Ab * others * pre[NF] * iL * dC[j];
    }
  }
  A.Vb[0] = 0.f;
#pragma unroll
  for (int j = 1; j <= K; ++j) A.Vb[j] = gC * pre[j - 1] * suf[j];
#pragma unroll
  for (int j = 0; j <= K; ++j) A.visb[j] = gC * pre[K + j] * suf[K + j + 1];
  if constexpr (!FIELD) A.Lb = -2.f * g * __fdiv_rn(p, L);
}

// Adjoints of each reflection's wall quantities (n, c, t0, len) from the
// back-propagation below.
template <int K>
struct VjpReflAdj {
  float nx[K + 1], ny[K + 1], c[K + 1], t0[K + 1], len[K + 1];
};

// Reverse of the leg normals and lengths, the validity, the backtrace and the
// image chain, given the vertex adjoints (Qbx, Qby) and the leg-normal adjoints
// (mAx, mAy, sm) of the sweeps: adds the TX adjoint to (txb_x, txb_y) and returns
// the per-reflection wall adjoints in R.
template <int MODE, int K, bool FIELD>
__device__ __forceinline__ void vjp_backprop(const VSmem& s, const Cand& cd, const VjpPath<K>& P,
                                             float alpha, const VjpFactorAdj<K>& A, float* Qbx,
                                             float* Qby, const float* mAx, const float* mAy,
                                             const float* sm, float& txb_x, float& txb_y,
                                             VjpReflAdj<K>& R) {
  const float* Qx = P.Qx;
  const float* Qy = P.Qy;
  // ------------------------------------------------ legs: normals and lengths
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    // m_bar = sum x2b (A - Q_j) + y2b (B - Q_j); the -Q_j part and dx2/dQ_j = -m
    const float mbx = mAx[j] - sm[j] * Qx[j];
    const float mby = mAy[j] - sm[j] * Qy[j];
    Qbx[j] -= sm[j] * P.mx[j];
    Qby[j] -= sm[j] * P.my[j];
    // m = (-D_y, D_x)/len: D_bar = (mb_y, -mb_x)/len - (mb . m) D/len^2 ; len_bar = Lb
    const float dx = Qx[j + 1] - Qx[j], dy = Qy[j + 1] - Qy[j];
    const float il = P.len[j] > 0.f ? 1.f / P.len[j] : 0.f;
    const float mm = fmaf(mbx, P.mx[j], mby * P.my[j]);
    const float Dbx = fmaf(mby, il, fmaf(-mm * il * il, dx, A.Lb * dx * il));
    const float Dby = fmaf(-mbx, il, fmaf(-mm * il * il, dy, A.Lb * dy * il));
    Qbx[j + 1] += Dbx;
    Qby[j + 1] += Dby;
    Qbx[j] -= Dbx;
    Qby[j] -= Dby;
  }

  // ------------------------------------------------ validity, backtrace, images
#pragma unroll
  for (int j = 0; j <= K; ++j) R.nx[j] = R.ny[j] = R.c[j] = R.t0[j] = R.len[j] = 0.f;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const int w = cd.w[j - 1];
    const float4 G = s.G[w];
    const float tau = fmaf(G.y, Qx[j], fmaf(-G.x, Qy[j], -s.T[w].x));
    const float pv = line_dist(G, Qx[j - 1], Qy[j - 1]);
    const float qv = line_dist(G, Qx[j + 1], Qy[j + 1]);
    const Smooth3 s1 = smooth3<MODE>(tau, alpha), s2 = smooth3<MODE>(G.w - tau, alpha);
    const Smooth3 sp = smooth3<MODE>(pv, alpha), sq = smooth3<MODE>(qv, alpha);
    const float S = fmaf(sp.s, sq.s, sp.sb * sq.sb);
    const float a1 = A.Vb[j] * s2.s * S, a2 = A.Vb[j] * s1.s * S, aS = A.Vb[j] * s1.s * s2.s;
    const float taub = a1 * s1.ds - a2 * s2.ds;
    const float pb = aS * sp.ds * (sq.s - sq.sb);
    const float qb = aS * sq.ds * (sp.s - sp.sb);
    R.len[j] = a2 * s2.ds;
    R.t0[j] = -taub;
    // tau = n_y Qx - n_x Qy - t0
    Qbx[j] = fmaf(taub, G.y, Qbx[j]);
    Qby[j] = fmaf(-taub, G.x, Qby[j]);
    R.nx[j] = -taub * Qy[j];
    R.ny[j] = taub * Qx[j];
    // p = n . Q_{j-1} - c ; q = n . Q_{j+1} - c
    Qbx[j - 1] = fmaf(pb, G.x, Qbx[j - 1]);
    Qby[j - 1] = fmaf(pb, G.y, Qby[j - 1]);
    Qbx[j + 1] = fmaf(qb, G.x, Qbx[j + 1]);
    Qby[j + 1] = fmaf(qb, G.y, Qby[j + 1]);
    R.nx[j] = fmaf(pb, Qx[j - 1], fmaf(qb, Qx[j + 1], R.nx[j]));
    R.ny[j] = fmaf(pb, Qy[j - 1], fmaf(qb, Qy[j + 1], R.ny[j]));
    R.c[j] = -(pb + qb);
  }
  if constexpr (FIELD) {
    // c_j = |n . d| / |d|, d = Q_j - Q_{j-1}:
    //   dc/dd = sign(n . d) (n - (n . d) d / |d|^2) / |d|,  dc/dn = sign(n . d) d / |d|
#pragma unroll
    for (int j = 1; j <= K; ++j) {
      const float4 G = s.G[cd.w[j - 1]];
      const float dx = Qx[j] - Qx[j - 1], dy = Qy[j] - Qy[j - 1];
      const float il = P.len[j - 1] > 0.f ? __frcp_rn(P.len[j - 1]) : 0.f;
      const float sd = fmaf(G.x, dx, G.y * dy);
      const float k = A.cosb[j] * il * copysignf(1.f, sd);
      const float proj = sd * il * il;
      const float Dbx = k * fmaf(-proj, dx, G.x);
      const float Dby = k * fmaf(-proj, dy, G.y);
      Qbx[j] += Dbx;
      Qby[j] += Dby;
      Qbx[j - 1] -= Dbx;
      Qby[j - 1] -= Dby;
      R.nx[j] = fmaf(k, dx, R.nx[j]);
      R.ny[j] = fmaf(k, dy, R.ny[j]);
    }
  }
  float Ibx[K + 1], Iby[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) Ibx[j] = Iby[j] = 0.f;
  // backtrace, reversed: Q_j = Q_{j+1} + t (I_j - Q_{j+1}), t = b / (b - a)
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const float4 G = s.G[cd.w[j - 1]];
    const float t = P.tt[j];
    const float ex = P.Ix[j] - Qx[j + 1], ey = P.Iy[j] - Qy[j + 1];
    Qbx[j + 1] = fmaf(1.f - t, Qbx[j], Qbx[j + 1]);
    Qby[j + 1] = fmaf(1.f - t, Qby[j], Qby[j + 1]);
    Ibx[j] = fmaf(t, Qbx[j], Ibx[j]);
    Iby[j] = fmaf(t, Qby[j], Iby[j]);
    const float tbar = fmaf(Qbx[j], ex, Qby[j] * ey);
    const float den = P.tb[j] - P.ta[j];
    const float id2 = (den != 0.f && !P.degenerate) ? 1.f / (den * den) : 0.f;
    const float abar = tbar * P.tb[j] * id2;
    const float bbar = -tbar * P.ta[j] * id2;
    Ibx[j] = fmaf(abar, G.x, Ibx[j]);
    Iby[j] = fmaf(abar, G.y, Iby[j]);
    Qbx[j + 1] = fmaf(bbar, G.x, Qbx[j + 1]);
    Qby[j + 1] = fmaf(bbar, G.y, Qby[j + 1]);
    R.nx[j] = fmaf(abar, P.Ix[j], fmaf(bbar, Qx[j + 1], R.nx[j]));
    R.ny[j] = fmaf(abar, P.Iy[j], fmaf(bbar, Qy[j + 1], R.ny[j]));
    R.c[j] -= abar + bbar;
  }
  // image chain, reversed: I_j = I_{j-1} - 2 d n, d = n . I_{j-1} - c
#pragma unroll
  for (int j = K; j >= 1; --j) {
    const float4 G = s.G[cd.w[j - 1]];
    const float dbar = -2.f * fmaf(Ibx[j], G.x, Iby[j] * G.y);
    Ibx[j - 1] += fmaf(dbar, G.x, Ibx[j]);
    Iby[j - 1] += fmaf(dbar, G.y, Iby[j]);
    R.nx[j] = fmaf(-2.f * P.dimg[j], Ibx[j], fmaf(dbar, P.Ix[j - 1], R.nx[j]));
    R.ny[j] = fmaf(-2.f * P.dimg[j], Iby[j], fmaf(dbar, P.Iy[j - 1], R.ny[j]));
    R.c[j] -= dbar;
  }
  txb_x += Qbx[0] + Ibx[0];
  txb_y += Qby[0] + Iby[0];
}

// Adds the per-reflection wall adjoints to the CTA table.  UNI: the candidate is the
// same in all 32 lanes, so each reflection's adjoints are summed over the warp
// first; otherwise each lane adds its own.
template <int K, bool UNI>
__device__ __forceinline__ void vjp_emit_reflections(const VSmem& s, const Cand& cd,
                                                     const VjpReflAdj<K>& R) {
  if (!UNI) {
#pragma unroll
    for (int j = 1; j <= K; ++j) {
      const bool any = (R.nx[j] != 0.f) | (R.ny[j] != 0.f) | (R.c[j] != 0.f) |
                       (R.t0[j] != 0.f) | (R.len[j] != 0.f);
      if (any) {
        float* dst = &s.acc[cd.w[j - 1] * VJP_SLOTS];
        atomicAdd(dst + S_NX, R.nx[j]);
        atomicAdd(dst + S_NY, R.ny[j]);
        atomicAdd(dst + S_C, R.c[j]);
        atomicAdd(dst + S_T0, R.t0[j]);
        atomicAdd(dst + S_LEN, R.len[j]);
      }
    }
  } else {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 1; j <= K; ++j) {
      const bool any = (R.nx[j] != 0.f) | (R.ny[j] != 0.f) | (R.c[j] != 0.f) |
                       (R.t0[j] != 0.f) | (R.len[j] != 0.f);
      if (__any_sync(FULL, any)) {
        const float a0 = warp_sum(R.nx[j]), a1 = warp_sum(R.ny[j]), a2 = warp_sum(R.c[j]);
        const float a3 = warp_sum(R.t0[j]), a4 = warp_sum(R.len[j]);
        float v = a0;
        int slot = S_NX;
        if (lane == 1) { v = a1; slot = S_NY; }
        if (lane == 2) { v = a2; slot = S_C; }
        if (lane == 3) { v = a3; slot = S_T0; }
        if (lane == 4) { v = a4; slot = S_LEN; }
        if (lane < 5) atomicAdd(&s.acc[cd.w[j - 1] * VJP_SLOTS + slot], v);
      }
    }
  }
}

// One path candidate's adjoint for this lane's receiver: recompute, two sweeps
// over the walls, back-propagation.
// UNI: the candidate is the same in all 32 lanes (lanes hold receivers), so the
// adjoints of the reflecting walls can be summed over the warp; otherwise (lanes
// hold different candidates of one receiver) each lane adds its own.
// FIELD: the adjoint of the coherent field's |E|^2 instead of the power (fw
// holds the lane's weight; g is 1 or 0).
template <int MODE, int K, bool WG, bool UNI, bool FIELD = false>
__device__ __forceinline__ void path_vjp(const VSmem& s, int W, float2 tx, float2 rx,
                                         const Cand& cd, float alpha, float gk, float g,
                                         float& txb_x, float& txb_y,
                                         const FieldW* fw = nullptr,
                                         const float* saved = nullptr,
                                         long long saved_stride = 0) {
  // ------------------------------------------------ forward recompute (guarded)
  VjpPath<K> P;
  vjp_recompute<MODE, K>(s, tx, rx, cd, alpha, P);
  const float* Qx = P.Qx;
  const float* Qy = P.Qy;
  const float* mx = P.mx;
  const float* my = P.my;
  const float* mq = P.mq;
  if (P.degenerate) g = 0.f;
  // A path with an exactly-zero factor has an exactly-zero gradient: a zero
  // validity or visibility factor is a saturated smoothing (derivative 0, also
  // at the hard sigmoid's kinks by convention) or an FP32 underflow of the
  // sigmoid, and every other factor's adjoint carries the zero.  Such lanes get
  // weight 0, and a warp whose lanes are all such skips the rest.
  bool dead = P.degenerate || g == 0.f;
#pragma unroll
  for (int j = 1; j <= K; ++j) dead |= (P.V[j] == 0.f);
  if (__all_sync(FULL, dead)) return;
  // sweep 1: visibility as (product of non-zero factors, number of zero factors)
  float nz[K + 1];
  int zc[K + 1];
  float mxk[K + 1], myk[K + 1], mck[K + 1];   // sigmoid: the leg lines scaled by alpha log2(e)
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    nz[j] = 1.f;
    zc[j] = 0;
    const float kap = alpha * LOG2E;
    mxk[j] = mx[j] * kap;
    myk[j] = my[j] * kap;
    mck[j] = -mq[j] * kap;
  }
  if constexpr (MODE == MODE_SIGMOID) {
    if (saved) {   // the forward's visibilities of this path (sweep 1 done there)
      // A path the forward found degenerate (a zero-length leg) has no finite
      // visibilities there and contributes nothing: such lanes, and lanes already
      // at weight 0, take 1 so that their zero weight stays an exact zero.
#pragma unroll
      for (int j = 0; j <= K; ++j) {
        const float v = __ldg(saved + j * saved_stride);
        dead |= (v != v);
        nz[j] = v;
      }
#pragma unroll
      for (int j = 0; j <= K; ++j) nz[j] = dead ? 1.f : nz[j];
    } else {
      sigmoid_vis_sweep<K>(s, W, cd, Qx, Qy, mxk, myk, mck, nz, zc);
    }
  } else {
  for (int w = 0; w < W; ++w) {
    const float4 G = s.G[w];
    const float4 E = s.E[w];
    float dv[K + 2];
#pragma unroll
    for (int i = 0; i <= K + 1; ++i) dv[i] = line_dist(G, Qx[i], Qy[i]);
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      const bool skip = (j >= 1 && w == cd.w[j - 1]) || (j < K && w == cd.w[j]);
      if (skip) continue;
      const float x2 = fmaf(mx[j], E.x, fmaf(my[j], E.y, -mq[j]));
      const float y2 = fmaf(mx[j], E.z, fmaf(my[j], E.w, -mq[j]));
      const float f = leg_wall<MODE, false>(dv[j], dv[j + 1], x2, y2, alpha).f;
      if (f == 0.f) {
        zc[j] += 1;
      } else {
        nz[j] *= f;
      }
    }
  }
  }
#pragma unroll
  for (int j = 0; j <= K; ++j) dead |= (zc[j] != 0) | (MODE == MODE_SIGMOID && nz[j] == 0.f);
  if (__all_sync(FULL, dead)) return;
  if (dead) g = 0.f;
  // ------------------------------------------------ factor adjoints
  VjpFactorAdj<K> A;
  vjp_factor_adjoints<K, FIELD>(s, cd, P, nz, zc, g, gk, fw, A);
  const float* visb = A.visb;

  // ------------------------------------------------ sweep 2: obstruction adjoint
  // legs whose visibility adjoint is zero in every lane contribute nothing here
  // (hard sigmoid and step; the sigmoid's legs carry a weight of 0 instead)
  bool live_leg[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j)
    live_leg[j] = MODE != MODE_SIGMOID && __any_sync(FULL, visb[j] != 0.f);
  float Qbx[K + 2], Qby[K + 2], mAx[K + 1], mAy[K + 1], sm[K + 1];
#pragma unroll
  for (int i = 0; i <= K + 1; ++i) Qbx[i] = Qby[i] = 0.f;
#pragma unroll
  for (int j = 0; j <= K; ++j) mAx[j] = mAy[j] = sm[j] = 0.f;
  if constexpr (MODE == MODE_SIGMOID) {
    // Rational form of each factor's derivatives: with e = 2^-|z| per smoothed
    // distance, F = 1 - e^2 and D = Ns + No = (1 + e_x)(1 + e_y) per pair,
    //   dX/dx = -alpha sign(y) e_x F_y / D^2   (and symmetrically in y),
    // so the adjoint of factor f = 1 - X1 X2 = num / (D1 D2) reaches the four
    // distances through one reciprocal 1 / (num D1 D2) and the per-vertex e, F
    // (each vertex's own e is applied once per wall, after the legs).  A lane
    // with an exactly-zero factor has weight 0; the tiny addend keeps its
    // reciprocal finite.
    float Wa[K + 1];
#pragma unroll
    for (int j = 0; j <= K; ++j) Wa[j] = (zc[j] == 0) ? visb[j] * nz[j] * alpha : 0.f;
#pragma unroll 2
    for (int w = 0; w < W; ++w) {
      const float4 G = s.G[w];
      const float4 E = s.E[w];
      const float4 h = s.H[w];
      float ze[K + 2], ev[K + 2], sF[K + 2], vb[K + 2];
      ze[0] = copysignf(1.f, h.w);   // the TX side: only the sign is used
      ev[0] = fabsf(h.w);
#pragma unroll
      for (int i = 1; i <= K + 1; ++i) {
        ze[i] = fmaf(h.x, Qx[i], fmaf(h.y, Qy[i], h.z));
        ev[i] = ex2_approx(-fabsf(ze[i]));
      }
#pragma unroll
      for (int i = 0; i <= K + 1; ++i) {
        sF[i] = copysignf(fmaf(-ev[i], ev[i], 1.f), ze[i]);
        vb[i] = 0.f;
      }
      float Abx = 0.f, Aby = 0.f, Bbx = 0.f, Bby = 0.f;
#pragma unroll
      for (int j = 0; j <= K; ++j) {
        const bool skip = (j >= 1 && w == cd.w[j - 1]) || (j < K && w == cd.w[j]);
        if (skip) continue;
        const float za = fmaf(mxk[j], E.x, fmaf(myk[j], E.y, mck[j]));
        const float zb = fmaf(mxk[j], E.z, fmaf(myk[j], E.w, mck[j]));
        const float ea = ex2_approx(-fabsf(za)), eb = ex2_approx(-fabsf(zb));
        const float ns1 = ev[j] + ev[j + 1], no1 = fmaf(ev[j], ev[j + 1], 1.f);
        const bool same1 = same_side(ze[j], ze[j + 1]);
        const float x1 = same1 ? ns1 : no1, xb1 = same1 ? no1 : ns1;
        const float ns2 = ea + eb, no2 = fmaf(ea, eb, 1.f);
        const bool same2 = same_side(za, zb);
        const float x2 = same2 ? ns2 : no2, xb2 = same2 ? no2 : ns2;
        const float D1 = ns1 + no1, D2 = ns2 + no2;
        const float num = fmaf(xb1, D2, x1 * xb2);
        const float t = Wa[j] * rcp_approx(fmaf(num, D1 * D2, SIGMOID_VJP_TINY));
        const float c1 = t * x2 * D2, c2 = t * x1 * D1;
        vb[j] = fmaf(c1, sF[j + 1], vb[j]);
        vb[j + 1] = fmaf(c1, sF[j], vb[j + 1]);
        const float sFa = copysignf(fmaf(-ea, ea, 1.f), za);
        const float sFb = copysignf(fmaf(-eb, eb, 1.f), zb);
        const float x2b = c2 * ea * sFb, y2b = c2 * eb * sFa;
        // x2 = m . (A - Q_j), y2 = m . (B - Q_j)
        mAx[j] = fmaf(x2b, E.x, fmaf(y2b, E.z, mAx[j]));
        mAy[j] = fmaf(x2b, E.y, fmaf(y2b, E.w, mAy[j]));
        sm[j] += x2b + y2b;
        if (WG) {
          Abx = fmaf(x2b, mx[j], Abx);
          Aby = fmaf(x2b, my[j], Aby);
          Bbx = fmaf(y2b, mx[j], Bbx);
          Bby = fmaf(y2b, my[j], Bby);
        }
      }
      // vertex distances d(Q_i) = n . Q_i - c
      float nbx = 0.f, nby = 0.f, cb = 0.f;
#pragma unroll
      for (int i = 0; i <= K + 1; ++i) {
        const float v = vb[i] * ev[i];
        Qbx[i] = fmaf(v, G.x, Qbx[i]);
        Qby[i] = fmaf(v, G.y, Qby[i]);
        if (WG) {
          nbx = fmaf(v, Qx[i], nbx);
          nby = fmaf(v, Qy[i], nby);
          cb -= v;
        }
      }
      if (WG) add_wall_adjoint(s, w, nbx, nby, cb, Abx, Aby, Bbx, Bby);
    }
  } else {
  for (int w = 0; w < W; ++w) {
    const float4 G = s.G[w];
    const float4 E = s.E[w];
    float dv[K + 2], vb[K + 2];
#pragma unroll
    for (int i = 0; i <= K + 1; ++i) {
      dv[i] = line_dist(G, Qx[i], Qy[i]);
      vb[i] = 0.f;
    }
    float Abx = 0.f, Aby = 0.f, Bbx = 0.f, Bby = 0.f;
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      const bool skip = (j >= 1 && w == cd.w[j - 1]) || (j < K && w == cd.w[j]);
      if (skip || !live_leg[j]) continue;
      const float x2 = fmaf(mx[j], E.x, fmaf(my[j], E.y, -mq[j]));
      const float y2 = fmaf(mx[j], E.z, fmaf(my[j], E.w, -mq[j]));
      const LegWall lw = leg_wall<MODE, true>(dv[j], dv[j + 1], x2, y2, alpha);
      // d vis / d f = product of the other factors
      float dvis;
      if (zc[j] == 0) {
        dvis = __fdividef(nz[j], lw.f);
      } else {
        dvis = (zc[j] == 1 && lw.f == 0.f) ? nz[j] : 0.f;
      }
      const float fb = visb[j] * dvis;
      vb[j] = fmaf(fb, lw.dx1, vb[j]);
      vb[j + 1] = fmaf(fb, lw.dy1, vb[j + 1]);
      const float x2b = fb * lw.dx2, y2b = fb * lw.dy2;
      // x2 = m . (A - Q_j), y2 = m . (B - Q_j)
      mAx[j] = fmaf(x2b, E.x, fmaf(y2b, E.z, mAx[j]));
      mAy[j] = fmaf(x2b, E.y, fmaf(y2b, E.w, mAy[j]));
      sm[j] += x2b + y2b;
      if (WG) {
        Abx = fmaf(x2b, mx[j], Abx);
        Aby = fmaf(x2b, my[j], Aby);
        Bbx = fmaf(y2b, mx[j], Bbx);
        Bby = fmaf(y2b, my[j], Bby);
      }
    }
    // vertex distances d(Q_i) = n . Q_i - c
    float nbx = 0.f, nby = 0.f, cb = 0.f;
#pragma unroll
    for (int i = 0; i <= K + 1; ++i) {
      Qbx[i] = fmaf(vb[i], G.x, Qbx[i]);
      Qby[i] = fmaf(vb[i], G.y, Qby[i]);
      if (WG) {
        nbx = fmaf(vb[i], Qx[i], nbx);
        nby = fmaf(vb[i], Qy[i], nby);
        cb -= vb[i];
      }
    }
    if (WG) {
      const bool any = (nbx != 0.f) | (nby != 0.f) | (cb != 0.f) | (Abx != 0.f) |
                       (Aby != 0.f) | (Bbx != 0.f) | (Bby != 0.f);
      if (__any_sync(FULL, any)) add_wall_adjoint(s, w, nbx, nby, cb, Abx, Aby, Bbx, Bby);
    }
  }

  }

  VjpReflAdj<K> R;
  vjp_backprop<MODE, K, FIELD>(s, cd, P, alpha, A, Qbx, Qby, mAx, mAy, sm, txb_x, txb_y, R);
  if (WG) vjp_emit_reflections<K, UNI>(s, cd, R);
}

}  // namespace drt
