// Forward pass of the method in 3D (Sec. VI: the framework does not depend on the
// dimension): walls are triangles, lines become planes, and a point lies on an
// object when its three in-plane edge distances pass the smoothed comparison.
//
//   plane of triangle (A, B, C): unit normal n along (B - A) x (C - A), c = n . A,
//   d(p) = n . p - c; edge k (A->B, B->C, C->A): in-plane unit normal
//   m_k = n x e_k / |e_k| (pointing inside), delta_k(p) = m_k . p - m_k . (start of k);
//   image method and backtrace as in 2D with planes for lines;
//   validity of reflection j: prod_k s(delta_k(Q_j)) (s(p) s(q) + s(-p) s(-q));
//   obstruction of leg Q_j -> Q_{j+1} by triangle w (not one in the plane of a
//   triangle its end points lie on, which the leg meets only at that end point):
//   X(x, y) prod_k s(delta_k(P)), x, y the end points' plane distances and P
//   the point where the leg's line meets the plane, whose edge distances are the
//   end points' ones interpolated at t = x / (x - y) (delta_k is affine);
//   path power Gamma^k V vis / L^2, summed over the candidates;
//   two consecutive reflections on triangles of one plane make a degenerate path:
//   the leg between them has zero length, and in floating point its rounding-sized
//   length would make the path's power an arbitrary function of the rounding.
//   "One plane": normals parallel and offsets equal, both to 1e-5.
//
// Mapping as in drt_forward.cu: lanes are receivers, the candidate is
// warp-uniform, the triangles' plane and edge records sit in shared memory and
// are read as broadcasts; per triangle, the plane and edge distances of every
// path vertex are computed once and shared by the two legs meeting there.  Units
// of (32 receivers) x (a chunk of candidates), per-chunk partial sums added in
// chunk order: deterministic.
#include <cuda_runtime.h>

#include "drt_common.cuh"
#include "drt_internal.h"

namespace drt {

namespace {

// Triangle records in shared memory, 4 float4 per triangle:
//   P  {nx, ny, nz, c}            plane: d(p) = n . p - c
//   Mk {mx, my, mz, o_k}, k=0..2  edge k: delta_k(p) = m_k . p - o_k
struct SmemTris {
  float4 *P, *M0, *M1, *M2;
};

__device__ __forceinline__ float dot3(float4 r, float3 p) {
  return fmaf(r.x, p.x, fmaf(r.y, p.y, r.z * p.z));
}

__device__ void stage_tris(const float* __restrict__ tris, int W, SmemTris s) {
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    const float* t = tris + 9 * (size_t)w;
    const float3 a = make_float3(t[0], t[1], t[2]);
    const float3 b = make_float3(t[3], t[4], t[5]);
    const float3 c = make_float3(t[6], t[7], t[8]);
    const float3 e1 = make_float3(b.x - a.x, b.y - a.y, b.z - a.z);
    const float3 e2 = make_float3(c.x - a.x, c.y - a.y, c.z - a.z);
    float3 n = make_float3(fmaf(e1.y, e2.z, -e1.z * e2.y), fmaf(e1.z, e2.x, -e1.x * e2.z),
                           fmaf(e1.x, e2.y, -e1.y * e2.x));
    const float nl = __fsqrt_rn(fmaf(n.x, n.x, fmaf(n.y, n.y, n.z * n.z)));
    n = make_float3(__fdiv_rn(n.x, nl), __fdiv_rn(n.y, nl), __fdiv_rn(n.z, nl));
    const float4 P = make_float4(n.x, n.y, n.z, fmaf(n.x, a.x, fmaf(n.y, a.y, n.z * a.z)));
    s.P[w] = P;
    const float3 v[3] = {a, b, c};
    float4* M[3] = {s.M0, s.M1, s.M2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float3 p = v[k], q = v[(k + 1) % 3];
      const float3 e = make_float3(q.x - p.x, q.y - p.y, q.z - p.z);
      float3 m = make_float3(fmaf(n.y, e.z, -n.z * e.y), fmaf(n.z, e.x, -n.x * e.z),
                             fmaf(n.x, e.y, -n.y * e.x));
      const float ml = __fsqrt_rn(fmaf(m.x, m.x, fmaf(m.y, m.y, m.z * m.z)));
      m = make_float3(__fdiv_rn(m.x, ml), __fdiv_rn(m.y, ml), __fdiv_rn(m.z, ml));
      M[k][w] = make_float4(m.x, m.y, m.z, fmaf(m.x, p.x, fmaf(m.y, p.y, m.z * p.z)));
    }
  }
}

// Sigmoid obstruction of every leg by every triangle (the forward's loop; the
// adjoint keeps its own).  With e = 2^-|z| for the smoothed distances of a leg's
// end points to the triangle's plane, the straddle term is X = x1 / D1 with
// Ns = e_j + e_{j+1}, No = 1 + e_j e_{j+1}, D1 = Ns + No and x1 = Ns when both
// lie on one side, No otherwise (xb1 the other one), as in 2D.  The on-triangle
// factor at the crossing point is in = 1 / Pin with Pin = prod_k (1 + u_k),
// u_k = 2^-a_k for the three scaled in-plane edge distances a_k (u_k capped at
// 2^24, where s < 6e-8 already rounds the product); Pin - 1 is expanded as a sum
// of products of the u_k.  Then
//   1 - X in = (xb1 + x1 (1 - in)) / D1,   1 - in = (Pin - 1) / Pin,
// a sum of non-negative terms: a leg nearly blocked by a triangle keeps its
// relative accuracy, and one reciprocal gives the three edge factors (four MUFU
// operations per test and one per vertex, against seven and two for three
// separate sigmoids).  Numerators and D1 are multiplied up separately and folded
// into vis every 8 triangles (D1 <= 4).
template <int K>
__device__ __forceinline__ void sigmoid_visibility3(const SmemTris& s, int W, const float3* Q,
                                                    const float4* Pr, float alpha, float* vis) {
  const float kap = alpha * LOG2E;
  float vn[K + 1], vd[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) vn[j] = vd[j] = 1.f;
  for (int w0 = 0; w0 < W; w0 += 8) {
    const int w1 = min(w0 + 8, W);
    for (int w = w0; w < w1; ++w) {
      const float4 P = s.P[w], M0 = s.M0[w], M1 = s.M1[w], M2 = s.M2[w];
      bool cop[K + 2];   // w in the plane of reflection j's triangle (warp-uniform)
      cop[0] = cop[K + 1] = false;
#pragma unroll
      for (int j = 1; j <= K; ++j) {
        const float nn = fmaf(P.x, Pr[j].x, fmaf(P.y, Pr[j].y, P.z * Pr[j].z));
        cop[j] = fabsf(nn) >= 1.f - 1e-5f &&
                 fabsf(fmaf(-nn, Pr[j].w, P.w)) <= 1e-5f * (1.f + fabsf(P.w));
      }
      float d[K + 2], ee[K + 2], e0[K + 2], e1[K + 2], e2[K + 2];
#pragma unroll
      for (int i = 0; i <= K + 1; ++i) {
        d[i] = dot3(P, Q[i]) - P.w;
        ee[i] = ex2_approx(-fabsf(d[i] * kap));
        e0[i] = (dot3(M0, Q[i]) - M0.w) * kap;
        e1[i] = (dot3(M1, Q[i]) - M1.w) * kap;
        e2[i] = (dot3(M2, Q[i]) - M2.w) * kap;
      }
#pragma unroll
      for (int j = 0; j <= K; ++j) {
        if (cop[j] || cop[j + 1]) continue;
        const float t = __fdividef(d[j], d[j] - d[j + 1]);
        // the leg's line misses the plane (or meets it absurdly far): not blocked
        if (!(fabsf(t) <= 1e8f)) continue;
        const float ns = ee[j] + ee[j + 1];
        const float no = fmaf(ee[j], ee[j + 1], 1.f);
        const bool same = same_side(d[j], d[j + 1]);
        const float x1 = same ? ns : no, xb1 = same ? no : ns;
        const float u0 = ex2_approx(fminf(-fmaf(t, e0[j + 1] - e0[j], e0[j]), 24.f));
        const float u1 = ex2_approx(fminf(-fmaf(t, e1[j + 1] - e1[j], e1[j]), 24.f));
        const float u2 = ex2_approx(fminf(-fmaf(t, e2[j + 1] - e2[j], e2[j]), 24.f));
        const float a01 = fmaf(u0, u1, u0 + u1);
        const float pm1 = fmaf(u2, 1.f + a01, a01);
        const float omi = pm1 * rcp_approx(1.f + pm1);
        vn[j] *= fmaf(x1, omi, xb1);
        vd[j] *= ns + no;
      }
    }
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      vis[j] *= __fdividef(vn[j], vd[j]);
      vn[j] = vd[j] = 1.f;
    }
  }
}

// Power of one candidate of order K for this lane's receiver.
template <int MODE, int K>
__device__ __forceinline__ float path_power3(const SmemTris& s, int W, float3 tx, float3 rx,
                                             const Cand& cd, float alpha, float gk) {
  // images (warp-uniform)
  float3 I[K + 1];
  I[0] = tx;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const float4 P = s.P[cd.w[j - 1]];
    const float d2 = 2.f * (dot3(P, I[j - 1]) - P.w);
    I[j] = make_float3(fmaf(-d2, P.x, I[j - 1].x), fmaf(-d2, P.y, I[j - 1].y),
                       fmaf(-d2, P.z, I[j - 1].z));
  }
  // two consecutive reflections in one plane (two triangles of one flat face): the
  // leg between them has zero length, the path is degenerate (warp-uniform test)
  bool degenerate = false;
#pragma unroll
  for (int j = 1; j < K; ++j) {
    const float4 Pa = s.P[cd.w[j - 1]], Pb = s.P[cd.w[j]];
    const float nn = fmaf(Pa.x, Pb.x, fmaf(Pa.y, Pb.y, Pa.z * Pb.z));
    if (fabsf(nn) >= 1.f - 1e-5f && fabsf(fmaf(-nn, Pb.w, Pa.w)) <= 1e-5f * (1.f + fabsf(Pa.w)))
      degenerate = true;
  }
  // backtrace on the planes: Q_{K+1} = RX, Q_j = line(Q_{j+1}, I_j) x plane j
  float3 Q[K + 2];
  Q[0] = tx;
  Q[K + 1] = rx;
#pragma unroll
  for (int j = K; j >= 1; --j) {
    const float4 P = s.P[cd.w[j - 1]];
    const float a = dot3(P, I[j]) - P.w;
    const float b = dot3(P, Q[j + 1]) - P.w;
    float t = __fdividef(b, b - a);
    if (!(fabsf(t) <= 1e8f)) {
      degenerate = true;
      t = 0.f;
    }
    Q[j] = make_float3(fmaf(t, I[j].x - Q[j + 1].x, Q[j + 1].x),
                       fmaf(t, I[j].y - Q[j + 1].y, Q[j + 1].y),
                       fmaf(t, I[j].z - Q[j + 1].z, Q[j + 1].z));
  }
  float L = 0.f;
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    const float dx = Q[j + 1].x - Q[j].x, dy = Q[j + 1].y - Q[j].y, dz = Q[j + 1].z - Q[j].z;
    const float len2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    degenerate |= !(len2 > 0.f);
    L += __fsqrt_rn(len2);
  }
  // validity: on the triangle, and the neighbours on the same side of its plane
  float V = 1.f;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const int w = cd.w[j - 1];
    const float4 P = s.P[w];
    const Smooth3 sp = smooth3<MODE>(dot3(P, Q[j - 1]) - P.w, alpha);
    const Smooth3 sq = smooth3<MODE>(dot3(P, Q[j + 1]) - P.w, alpha);
    const float4 M0 = s.M0[w], M1 = s.M1[w], M2 = s.M2[w];
    const float in = smooth3<MODE>(dot3(M0, Q[j]) - M0.w, alpha).s *
                     smooth3<MODE>(dot3(M1, Q[j]) - M1.w, alpha).s *
                     smooth3<MODE>(dot3(M2, Q[j]) - M2.w, alpha).s;
    V *= in * fmaf(sp.s, sq.s, sp.sb * sq.sb);
  }
  if (__all_sync(0xffffffffu, V == 0.f || degenerate)) return 0.f;
  // obstruction: every triangle against every leg, except the triangles in the plane
  // of a triangle the leg's end points lie on (the leg meets that plane only there)
  float vis[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) vis[j] = 1.f;
  float4 Pr[K + 1];
#pragma unroll
  for (int j = 1; j <= K; ++j) Pr[j] = s.P[cd.w[j - 1]];
  if constexpr (MODE == MODE_SIGMOID) {
    sigmoid_visibility3<K>(s, W, Q, Pr, alpha, vis);
  } else {
  for (int w = 0; w < W; ++w) {
    const float4 P = s.P[w], M0 = s.M0[w], M1 = s.M1[w], M2 = s.M2[w];
    bool cop[K + 2];   // w in the plane of reflection j's triangle (warp-uniform)
    cop[0] = cop[K + 1] = false;
#pragma unroll
    for (int j = 1; j <= K; ++j) {
      const float nn = fmaf(P.x, Pr[j].x, fmaf(P.y, Pr[j].y, P.z * Pr[j].z));
      cop[j] = fabsf(nn) >= 1.f - 1e-5f &&
               fabsf(fmaf(-nn, Pr[j].w, P.w)) <= 1e-5f * (1.f + fabsf(P.w));
    }
    float d[K + 2], e0[K + 2], e1[K + 2], e2[K + 2];
    Smooth3 sd[K + 2];
#pragma unroll
    for (int i = 0; i <= K + 1; ++i) {
      d[i] = dot3(P, Q[i]) - P.w;
      sd[i] = smooth3<MODE>(d[i], alpha);
      e0[i] = dot3(M0, Q[i]) - M0.w;
      e1[i] = dot3(M1, Q[i]) - M1.w;
      e2[i] = dot3(M2, Q[i]) - M2.w;
    }
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      if (cop[j] || cop[j + 1]) continue;
      const float X = fmaf(sd[j].s, sd[j + 1].sb, sd[j].sb * sd[j + 1].s);
      const float den = d[j] - d[j + 1];
      const float t = __fdividef(d[j], den);
      // the leg's line misses the plane (or meets it absurdly far): not blocked
      if (!(fabsf(t) <= 1e8f)) continue;
      const float in = smooth3<MODE>(fmaf(t, e0[j + 1] - e0[j], e0[j]), alpha).s *
                       smooth3<MODE>(fmaf(t, e1[j + 1] - e1[j], e1[j]), alpha).s *
                       smooth3<MODE>(fmaf(t, e2[j + 1] - e2[j], e2[j]), alpha).s;
      vis[j] = fmaf(-X, in * vis[j], vis[j]);
    }
  }
  }
  float p = V * gk;
#pragma unroll
  for (int j = 0; j <= K; ++j) p *= vis[j];
  p = __fdividef(p, L * L);
  return degenerate ? 0.f : p;
}

template <int MODE>
__global__ void __launch_bounds__(256, 2) forward3_kernel(const Fwd3Args a) {
  extern __shared__ float4 smem[];
  SmemTris s{smem, smem + a.W, smem + 2 * a.W, smem + 3 * a.W};
  stage_tris(a.tris, a.W, s);
  __syncthreads();
  const float3 tx = make_float3(__ldg(a.tx), __ldg(a.tx + 1), __ldg(a.tx + 2));
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
    const float3 q = make_float3(__ldg(a.rx + 3 * r), __ldg(a.rx + 3 * r + 1),
                                 __ldg(a.rx + 3 * r + 2));
    const int c0 = (int)(chunk * a.chunk);
    const int nc = (int)(min(c0 + (long long)a.chunk, a.n_cand) - c0);
    float acc = 0.f;
    Cand cd = decode_candidate(c0, a.W, a.K);
    for (int i = 0; i < nc; ++i) {
      if (i > 0) next_candidate(cd, a.W);
      switch (cd.k) {
        case 0: acc += path_power3<MODE, 0>(s, a.W, tx, q, cd, a.alpha, a.gk[0]); break;
        case 1: acc += path_power3<MODE, 1>(s, a.W, tx, q, cd, a.alpha, a.gk[1]); break;
        case 2: acc += path_power3<MODE, 2>(s, a.W, tx, q, cd, a.alpha, a.gk[2]); break;
        default: acc += path_power3<MODE, 3>(s, a.W, tx, q, cd, a.alpha, a.gk[3]); break;
      }
    }
    if (live) a.partial[chunk * a.R + r] = acc;
  }
}

// ------------------------------------------------------------ TX adjoint
// Reverse mode of path_power3 for the transmitter only (the gradient the antenna
// placement of Sec. VII needs): recompute the path, sweep the triangles once for
// each leg's visibility as (product of the non-zero factors, number of zero
// factors), then once more pushing each factor's adjoint into the path vertices;
// the vertex adjoints flow back through the leg lengths, the validity, the
// backtrace and the image chain to the transmitter.  A path with an exactly-zero
// factor has an exactly-zero gradient (a saturated smoothing), as in 2D.
struct LegTri {
  float x, y, X, t, ins, f;
  Smooth3 sx, sy, sd[3];
  float e0[3], e1[3];
};

template <int MODE>
__device__ __forceinline__ bool leg_tri(const float4& P, const float4* M, float3 a, float3 b,
                                        float alpha, LegTri& r) {
  r.x = dot3(P, a) - P.w;
  r.y = dot3(P, b) - P.w;
  r.sx = smooth3<MODE>(r.x, alpha);
  r.sy = smooth3<MODE>(r.y, alpha);
  r.X = fmaf(r.sx.s, r.sy.sb, r.sx.sb * r.sy.s);
  r.t = __fdividef(r.x, r.x - r.y);
  if (!(fabsf(r.t) <= 1e8f)) return false;
  r.ins = 1.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.e0[k] = dot3(M[k], a) - M[k].w;
    r.e1[k] = dot3(M[k], b) - M[k].w;
    r.sd[k] = smooth3<MODE>(fmaf(r.t, r.e1[k] - r.e0[k], r.e0[k]), alpha);
    r.ins *= r.sd[k].s;
  }
  if (MODE == MODE_SIGMOID) {
    // f = 1 - X ins as sums of non-negative terms (s + sb = 1 for each smoothed
    // value): 1 - X = s_x s_y + sb_x sb_y and 1 - ins = sb_0 + s_0 (sb_1 + s_1 sb_2),
    // so f = (1 - X) + X (1 - ins) keeps its relative accuracy where a triangle
    // nearly blocks the leg (1 - X ins there cancels to a few ulps of 1)
    const float omx = fmaf(r.sx.s, r.sy.s, r.sx.sb * r.sy.sb);
    const float omi = fmaf(r.sd[0].s, fmaf(r.sd[1].s, r.sd[2].sb, r.sd[1].sb), r.sd[0].sb);
    r.f = fmaf(r.X, omi, omx);
  } else {
    r.f = fmaf(-r.X, r.ins, 1.f);
  }
  return true;
}

// Per-triangle adjoint slots of the wall gradient (the four records' values):
// P = {n, c} in 0..3, M_k = {m_k, o_k} in 4 + 4k .. 7 + 4k.
constexpr int TRI_SLOTS = 16;

// Sums v[0..15] over the warp by recursive halving: lane l ends with the warp
// total of v[(l >> 1) & 15] (each total held by 2 lanes); 16 shuffles.
__device__ __forceinline__ float warp_reduce_scatter16(const float* v) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float a[8], b[4], c[2];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    a[k] = (b4 ? v[k + 8] : v[k]) + __shfl_xor_sync(full, b4 ? v[k] : v[k + 8], 16);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    b[k] = (b3 ? a[k + 4] : a[k]) + __shfl_xor_sync(full, b3 ? a[k] : a[k + 4], 8);
#pragma unroll
  for (int k = 0; k < 2; ++k)
    c[k] = (b2 ? b[k + 2] : b[k]) + __shfl_xor_sync(full, b2 ? b[k] : b[k + 2], 4);
  float d = (b1 ? c[1] : c[0]) + __shfl_xor_sync(full, b1 ? c[0] : c[1], 2);
  return d + __shfl_xor_sync(full, d, 1);
}

// Adds the warp's 16 adjoint slots of triangle w into the CTA table (the
// triangle is the same in every lane).
__device__ __forceinline__ void add_tri_adjoint(float* acc, int w, const float* v) {
  const float t = warp_reduce_scatter16(v);
  const int lane = threadIdx.x & 31;
  if ((lane & 1) == 0) atomicAdd(&acc[w * TRI_SLOTS + ((lane >> 1) & 15)], t);
}

__device__ __forceinline__ void axpy3(float a, float4 v, float3& acc) {
  acc.x = fmaf(a, v.x, acc.x);
  acc.y = fmaf(a, v.y, acc.y);
  acc.z = fmaf(a, v.z, acc.z);
}

// WG: also the adjoints of every triangle's records (plane {n, c}, edges
// {m_k, o_k}) into the CTA table acc [W][TRI_SLOTS], summed over the warp (the
// candidate is the same in all lanes).
template <int MODE, int K, bool WG>
__device__ __forceinline__ void path_vjp3(const SmemTris& s, int W, float3 tx, float3 rx,
                                          const Cand& cd, float alpha, float gk, float g,
                                          float3& txb, float* acc) {
  bool degenerate = false;
#pragma unroll
  for (int j = 1; j < K; ++j) {
    const float4 Pa = s.P[cd.w[j - 1]], Pb = s.P[cd.w[j]];
    const float nn = fmaf(Pa.x, Pb.x, fmaf(Pa.y, Pb.y, Pa.z * Pb.z));
    if (fabsf(nn) >= 1.f - 1e-5f && fabsf(fmaf(-nn, Pb.w, Pa.w)) <= 1e-5f * (1.f + fabsf(Pa.w)))
      degenerate = true;
  }
  float3 I[K + 1];
  float dimg[K + 1];   // d = n . I_{j-1} - c of each image step
  I[0] = tx;
  dimg[0] = 0.f;
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const float4 P = s.P[cd.w[j - 1]];
    dimg[j] = dot3(P, I[j - 1]) - P.w;
    const float d2 = 2.f * dimg[j];
    I[j] = make_float3(fmaf(-d2, P.x, I[j - 1].x), fmaf(-d2, P.y, I[j - 1].y),
                       fmaf(-d2, P.z, I[j - 1].z));
  }
  float3 Q[K + 2];
  float ta[K + 1], tb[K + 1], tt[K + 1];
  Q[0] = tx;
  Q[K + 1] = rx;
#pragma unroll
  for (int j = K; j >= 1; --j) {
    const float4 P = s.P[cd.w[j - 1]];
    ta[j] = dot3(P, I[j]) - P.w;
    tb[j] = dot3(P, Q[j + 1]) - P.w;
    float t = __fdiv_rn(tb[j], tb[j] - ta[j]);
    if (!(fabsf(t) <= 1e8f)) {
      degenerate = true;
      t = 0.f;
    }
    tt[j] = t;
    Q[j] = make_float3(fmaf(t, I[j].x - Q[j + 1].x, Q[j + 1].x),
                       fmaf(t, I[j].y - Q[j + 1].y, Q[j + 1].y),
                       fmaf(t, I[j].z - Q[j + 1].z, Q[j + 1].z));
  }
  float len[K + 1], L = 0.f;
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    const float dx = Q[j + 1].x - Q[j].x, dy = Q[j + 1].y - Q[j].y, dz = Q[j + 1].z - Q[j].z;
    const float len2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    degenerate |= !(len2 > 0.f);
    len[j] = __fsqrt_rn(len2);
    L += len[j];
  }
  if (degenerate) {
    g = 0.f;
    L = 1.f;
  }
  float V[K + 1];
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const int w = cd.w[j - 1];
    const float4 P = s.P[w];
    const Smooth3 sp = smooth3<MODE>(dot3(P, Q[j - 1]) - P.w, alpha);
    const Smooth3 sq = smooth3<MODE>(dot3(P, Q[j + 1]) - P.w, alpha);
    const float4 M0 = s.M0[w], M1 = s.M1[w], M2 = s.M2[w];
    const float in = smooth3<MODE>(dot3(M0, Q[j]) - M0.w, alpha).s *
                     smooth3<MODE>(dot3(M1, Q[j]) - M1.w, alpha).s *
                     smooth3<MODE>(dot3(M2, Q[j]) - M2.w, alpha).s;
    V[j] = in * fmaf(sp.s, sq.s, sp.sb * sq.sb);
  }
  bool dead = degenerate || g == 0.f;
#pragma unroll
  for (int j = 1; j <= K; ++j) dead |= (V[j] == 0.f);
  if (__all_sync(0xffffffffu, dead)) return;
  float4 Pr[K + 1];
#pragma unroll
  for (int j = 1; j <= K; ++j) Pr[j] = s.P[cd.w[j - 1]];
  // sweep 1: each leg's visibility as (product of non-zero factors, zero count)
  float nz[K + 1];
  int zc[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    nz[j] = 1.f;
    zc[j] = 0;
  }
  for (int w = 0; w < W; ++w) {
    const float4 P = s.P[w];
    const float4 M[3] = {s.M0[w], s.M1[w], s.M2[w]};
    bool cop[K + 2];
    cop[0] = cop[K + 1] = false;
#pragma unroll
    for (int j = 1; j <= K; ++j) {
      const float nn = fmaf(P.x, Pr[j].x, fmaf(P.y, Pr[j].y, P.z * Pr[j].z));
      cop[j] = fabsf(nn) >= 1.f - 1e-5f &&
               fabsf(fmaf(-nn, Pr[j].w, P.w)) <= 1e-5f * (1.f + fabsf(P.w));
    }
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      if (cop[j] || cop[j + 1]) continue;
      LegTri r;
      if (!leg_tri<MODE>(P, M, Q[j], Q[j + 1], alpha, r)) continue;
      if (r.f == 0.f) zc[j] += 1;
      else nz[j] *= r.f;
    }
  }
#pragma unroll
  for (int j = 0; j <= K; ++j) dead |= (zc[j] != 0);
  if (__all_sync(0xffffffffu, dead)) return;
  if (dead) g = 0.f;
  // factor adjoints: p = C prod(F), C = Gamma^k / L^2, F = {V_1..V_K, vis_0..vis_K}
  constexpr int NF = 2 * K + 1;
  float F[NF];
#pragma unroll
  for (int j = 1; j <= K; ++j) F[j - 1] = V[j];
#pragma unroll
  for (int j = 0; j <= K; ++j) F[K + j] = zc[j] ? 0.f : nz[j];
  float pre[NF + 1], suf[NF + 1];
  pre[0] = 1.f;
#pragma unroll
  for (int i = 0; i < NF; ++i) pre[i + 1] = pre[i] * F[i];
  suf[NF] = 1.f;
#pragma unroll
  for (int i = NF - 1; i >= 0; --i) suf[i] = suf[i + 1] * F[i];
  const float C = __fdiv_rn(gk, L * L);
  const float p = C * pre[NF];
  const float gC = g * C;
  float Vb[K + 1], visb[K + 1];
#pragma unroll
  for (int j = 1; j <= K; ++j) Vb[j] = gC * pre[j - 1] * suf[j];
#pragma unroll
  for (int j = 0; j <= K; ++j) visb[j] = gC * pre[K + j] * suf[K + j + 1];
  const float Lb = -2.f * g * __fdiv_rn(p, L);
  float3 Qb[K + 2];
#pragma unroll
  for (int i = 0; i <= K + 1; ++i) Qb[i] = make_float3(0.f, 0.f, 0.f);
  // sweep 2: each factor f = 1 - X ins pushes its adjoint into the leg's end points
  // (and, WG, into the triangle's records: x = n . Q_j - c, y = n . Q_{j+1} - c,
  // delta_k = (1 - t) e0_k + t e1_k with e_k = m_k . Q - o_k)
  for (int w = 0; w < W; ++w) {
    const float4 P = s.P[w];
    const float4 M[3] = {s.M0[w], s.M1[w], s.M2[w]};
    bool cop[K + 2];
    cop[0] = cop[K + 1] = false;
#pragma unroll
    for (int j = 1; j <= K; ++j) {
      const float nn = fmaf(P.x, Pr[j].x, fmaf(P.y, Pr[j].y, P.z * Pr[j].z));
      cop[j] = fabsf(nn) >= 1.f - 1e-5f &&
               fabsf(fmaf(-nn, Pr[j].w, P.w)) <= 1e-5f * (1.f + fabsf(P.w));
    }
    float wa[TRI_SLOTS];
    bool any = false;
    if (WG) {
#pragma unroll
      for (int i = 0; i < TRI_SLOTS; ++i) wa[i] = 0.f;
    }
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      if (cop[j] || cop[j + 1]) continue;
      LegTri r;
      if (!leg_tri<MODE>(P, M, Q[j], Q[j + 1], alpha, r)) continue;
      float dvis;
      if (zc[j] == 0) dvis = __fdiv_rn(nz[j], r.f);
      else dvis = (zc[j] == 1 && r.f == 0.f) ? nz[j] : 0.f;
      const float fb = visb[j] * dvis;
      if (fb == 0.f) continue;
      const float Xb = -fb * r.ins, inb = -fb * r.X;
      float xb = Xb * r.sx.ds * (r.sy.sb - r.sy.s);
      float yb = Xb * r.sy.ds * (r.sx.sb - r.sx.s);
      float tbar = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float others = r.sd[(k + 1) % 3].s * r.sd[(k + 2) % 3].s;
        const float db = inb * r.sd[k].ds * others;
        axpy3(db * (1.f - r.t), M[k], Qb[j]);
        axpy3(db * r.t, M[k], Qb[j + 1]);
        tbar = fmaf(db, r.e1[k] - r.e0[k], tbar);
        if (WG) {
          const float b0 = db * (1.f - r.t), b1 = db * r.t;
          float* m = wa + 4 + 4 * k;
          m[0] = fmaf(b0, Q[j].x, fmaf(b1, Q[j + 1].x, m[0]));
          m[1] = fmaf(b0, Q[j].y, fmaf(b1, Q[j + 1].y, m[1]));
          m[2] = fmaf(b0, Q[j].z, fmaf(b1, Q[j + 1].z, m[2]));
          m[3] -= b0 + b1;
        }
      }
      const float den = r.x - r.y;
      const float id2 = __frcp_rn(den * den);
      xb = fmaf(tbar * -r.y, id2, xb);
      yb = fmaf(tbar * r.x, id2, yb);
      axpy3(xb, P, Qb[j]);
      axpy3(yb, P, Qb[j + 1]);
      if (WG) {
        wa[0] = fmaf(xb, Q[j].x, fmaf(yb, Q[j + 1].x, wa[0]));
        wa[1] = fmaf(xb, Q[j].y, fmaf(yb, Q[j + 1].y, wa[1]));
        wa[2] = fmaf(xb, Q[j].z, fmaf(yb, Q[j + 1].z, wa[2]));
        wa[3] -= xb + yb;
        any = true;
      }
    }
    if (WG && __any_sync(0xffffffffu, any)) add_tri_adjoint(acc, w, wa);
  }
  // legs: L = sum |Q_{j+1} - Q_j|
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    const float il = len[j] > 0.f ? __frcp_rn(len[j]) : 0.f;
    const float4 u = make_float4((Q[j + 1].x - Q[j].x) * il, (Q[j + 1].y - Q[j].y) * il,
                                 (Q[j + 1].z - Q[j].z) * il, 0.f);
    axpy3(Lb, u, Qb[j + 1]);
    axpy3(-Lb, u, Qb[j]);
  }
  // validity: on the triangle (three edge tests) and the same-side test
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const int w = cd.w[j - 1];
    const float4 P = s.P[w];
    const float4 M[3] = {s.M0[w], s.M1[w], s.M2[w]};
    const Smooth3 sp = smooth3<MODE>(dot3(P, Q[j - 1]) - P.w, alpha);
    const Smooth3 sq = smooth3<MODE>(dot3(P, Q[j + 1]) - P.w, alpha);
    const float S = fmaf(sp.s, sq.s, sp.sb * sq.sb);
    Smooth3 sdl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) sdl[k] = smooth3<MODE>(dot3(M[k], Q[j]) - M[k].w, alpha);
    const float ins = sdl[0].s * sdl[1].s * sdl[2].s;
    const float insb = Vb[j] * S, Sb = Vb[j] * ins;
    float wa[TRI_SLOTS];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float dk = insb * sdl[k].ds * sdl[(k + 1) % 3].s * sdl[(k + 2) % 3].s;
      axpy3(dk, M[k], Qb[j]);
      wa[4 + 4 * k] = dk * Q[j].x;   // delta_k = m_k . Q_j - o_k
      wa[5 + 4 * k] = dk * Q[j].y;
      wa[6 + 4 * k] = dk * Q[j].z;
      wa[7 + 4 * k] = -dk;
    }
    const float pb = Sb * sp.ds * (sq.s - sq.sb), qb = Sb * sq.ds * (sp.s - sp.sb);
    axpy3(pb, P, Qb[j - 1]);
    axpy3(qb, P, Qb[j + 1]);
    if (WG) {   // p = n . Q_{j-1} - c, q = n . Q_{j+1} - c
      wa[0] = fmaf(pb, Q[j - 1].x, qb * Q[j + 1].x);
      wa[1] = fmaf(pb, Q[j - 1].y, qb * Q[j + 1].y);
      wa[2] = fmaf(pb, Q[j - 1].z, qb * Q[j + 1].z);
      wa[3] = -(pb + qb);
      add_tri_adjoint(acc, w, wa);
    }
  }
  // backtrace, reversed: Q_j = Q_{j+1} + t (I_j - Q_{j+1}), t = b / (b - a)
  float3 Ib[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) Ib[j] = make_float3(0.f, 0.f, 0.f);
#pragma unroll
  for (int j = 1; j <= K; ++j) {
    const float4 P = s.P[cd.w[j - 1]];
    const float t = tt[j];
    const float4 q = make_float4(Qb[j].x, Qb[j].y, Qb[j].z, 0.f);
    axpy3(1.f - t, q, Qb[j + 1]);
    axpy3(t, q, Ib[j]);
    const float tbar = fmaf(Qb[j].x, I[j].x - Q[j + 1].x,
                            fmaf(Qb[j].y, I[j].y - Q[j + 1].y, Qb[j].z * (I[j].z - Q[j + 1].z)));
    const float den = tb[j] - ta[j];
    const float id2 = (den != 0.f && !degenerate) ? __frcp_rn(den * den) : 0.f;
    const float abar = tbar * tb[j] * id2, bbar = -tbar * ta[j] * id2;
    axpy3(abar, P, Ib[j]);
    axpy3(bbar, P, Qb[j + 1]);
    if (WG) {   // a = n . I_j - c, b = n . Q_{j+1} - c
      float wa[TRI_SLOTS];
#pragma unroll
      for (int i = 4; i < TRI_SLOTS; ++i) wa[i] = 0.f;
      wa[0] = fmaf(abar, I[j].x, bbar * Q[j + 1].x);
      wa[1] = fmaf(abar, I[j].y, bbar * Q[j + 1].y);
      wa[2] = fmaf(abar, I[j].z, bbar * Q[j + 1].z);
      wa[3] = -(abar + bbar);
      add_tri_adjoint(acc, cd.w[j - 1], wa);
    }
  }
  // image chain, reversed: I_j = I_{j-1} - 2 d n, d = n . I_{j-1} - c
#pragma unroll
  for (int j = K; j >= 1; --j) {
    const float4 P = s.P[cd.w[j - 1]];
    const float dbar = -2.f * fmaf(Ib[j].x, P.x, fmaf(Ib[j].y, P.y, Ib[j].z * P.z));
    if (WG) {   // n_bar = -2 d I_bar_j + d_bar I_{j-1}, c_bar = -d_bar
      float wa[TRI_SLOTS];
#pragma unroll
      for (int i = 4; i < TRI_SLOTS; ++i) wa[i] = 0.f;
      wa[0] = fmaf(-2.f * dimg[j], Ib[j].x, dbar * I[j - 1].x);
      wa[1] = fmaf(-2.f * dimg[j], Ib[j].y, dbar * I[j - 1].y);
      wa[2] = fmaf(-2.f * dimg[j], Ib[j].z, dbar * I[j - 1].z);
      wa[3] = -dbar;
      add_tri_adjoint(acc, cd.w[j - 1], wa);
    }
    Ib[j - 1].x += fmaf(dbar, P.x, Ib[j].x);
    Ib[j - 1].y += fmaf(dbar, P.y, Ib[j].y);
    Ib[j - 1].z += fmaf(dbar, P.z, Ib[j].z);
  }
  txb.x += Qb[0].x + Ib[0].x;
  txb.y += Qb[0].y + Ib[0].y;
  txb.z += Qb[0].z + Ib[0].z;
}

__device__ __forceinline__ float warp_sum3(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// grad_tx += sum_r g_r dP_r / dTX (and, WG, the per-CTA table of the triangles'
// record adjoints): lanes are receivers, as in the forward
template <int MODE, bool WG>
__global__ void __launch_bounds__(256, 1) vjp3_kernel(const Vjp3Args a) {
  extern __shared__ float4 smem[];
  SmemTris s{smem, smem + a.W, smem + 2 * a.W, smem + 3 * a.W};
  float* acc = reinterpret_cast<float*>(smem + 4 * a.W);
  stage_tris(a.tris, a.W, s);
  if (WG)
    for (int i = threadIdx.x; i < a.W * TRI_SLOTS; i += blockDim.x) acc[i] = 0.f;
  __syncthreads();
  const float3 tx = make_float3(__ldg(a.tx), __ldg(a.tx + 1), __ldg(a.tx + 2));
  const int lane = threadIdx.x & 31;
  const long long warps_per_cta = blockDim.x >> 5;
  const long long gwarp = (long long)blockIdx.x * warps_per_cta + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * warps_per_cta;
  // work stealing (next_unit_of): each unit's TX adjoint is summed over the warp and
  // stored per unit; the finalize kernel adds the units in index order, so the TX
  // gradient does not depend on which warp took which unit
  for (long long u = gwarp; u < a.n_units; u = next_unit_of(a.unit_counter, u, nwarps, lane)) {
    const long long tile = u % a.n_tiles;
    const long long chunk = u / a.n_tiles;
    long long r = tile * 32 + lane;
    const bool live = r < a.R;
    if (!live) r = a.R - 1;
    const float g = live ? __ldg(a.grad_power + r) : 0.f;
    float3 txb = make_float3(0.f, 0.f, 0.f);
    if (!__all_sync(0xffffffffu, g == 0.f)) {
      const float3 q = make_float3(__ldg(a.rx + 3 * r), __ldg(a.rx + 3 * r + 1),
                                   __ldg(a.rx + 3 * r + 2));
      const long long c0 = chunk * a.chunk;
      const long long c1 = min(c0 + (long long)a.chunk, a.n_cand);
      for (long long c = c0; c < c1; ++c) {
        const Cand cd = decode_candidate(c, a.W, a.K);
        switch (cd.k) {
          case 0: path_vjp3<MODE, 0, WG>(s, a.W, tx, q, cd, a.alpha, a.gk[0], g, txb, acc); break;
          case 1: path_vjp3<MODE, 1, WG>(s, a.W, tx, q, cd, a.alpha, a.gk[1], g, txb, acc); break;
          case 2: path_vjp3<MODE, 2, WG>(s, a.W, tx, q, cd, a.alpha, a.gk[2], g, txb, acc); break;
          default: path_vjp3<MODE, 3, WG>(s, a.W, tx, q, cd, a.alpha, a.gk[3], g, txb, acc); break;
        }
      }
    }
    txb.x = warp_sum3(txb.x);
    txb.y = warp_sum3(txb.y);
    txb.z = warp_sum3(txb.z);
    if (lane == 0) {
      a.unit_tx[3 * u] = txb.x;
      a.unit_tx[3 * u + 1] = txb.y;
      a.unit_tx[3 * u + 2] = txb.z;
    }
  }
  if (WG) {
    __syncthreads();
    float* out = a.cta_tris + (size_t)blockIdx.x * a.W * TRI_SLOTS;
    for (int i = threadIdx.x; i < a.W * TRI_SLOTS; i += blockDim.x) out[i] = acc[i];
  }
}

__device__ __forceinline__ float3 sub3(float3 a, float3 b) {
  return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z),
                     fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float dot3f(float3 a, float3 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}
__device__ __forceinline__ float3 axpy3f(float a, float3 x, float3 y) {
  return make_float3(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z));
}
// adjoint of u = v / |v| (|v| = len): (u_bar - (u_bar . u) u) / len
__device__ __forceinline__ float3 unit_adjoint(float3 ub, float3 u, float len) {
  const float il = __frcp_rn(len);
  const float c = dot3f(ub, u);
  return make_float3(fmaf(-c, u.x, ub.x) * il, fmaf(-c, u.y, ub.y) * il, fmaf(-c, u.z, ub.z) * il);
}

// Per triangle: adds the per-CTA tables of the records' adjoints in a fixed order
// and chains them back to the corners A, B, C (the records of stage_tris):
//   N = (B - A) x (C - A), n = N / |N|, c = n . A;
//   edge k from p to q: M_k = n x (q - p), m_k = M_k / |M_k|, o_k = m_k . p.
__global__ void __launch_bounds__(256) vjp3_tris_finalize_kernel(const Vjp3Args a, int n_ctas) {
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < a.W; w += gridDim.x * blockDim.x) {
    float v[TRI_SLOTS];
#pragma unroll
    for (int i = 0; i < TRI_SLOTS; ++i) v[i] = 0.f;
    for (int c = 0; c < n_ctas; ++c) {
      const float* src = a.cta_tris + ((size_t)c * a.W + w) * TRI_SLOTS;
#pragma unroll
      for (int i = 0; i < TRI_SLOTS; ++i) v[i] += src[i];
    }
    const float* t = a.tris + 9 * (size_t)w;
    const float3 P3[3] = {make_float3(t[0], t[1], t[2]), make_float3(t[3], t[4], t[5]),
                          make_float3(t[6], t[7], t[8])};
    const float3 e1 = sub3(P3[1], P3[0]), e2 = sub3(P3[2], P3[0]);
    const float3 N = cross3(e1, e2);
    const float nl = __fsqrt_rn(dot3f(N, N));
    const float3 n = make_float3(__fdiv_rn(N.x, nl), __fdiv_rn(N.y, nl), __fdiv_rn(N.z, nl));
    float3 cb[3] = {make_float3(0.f, 0.f, 0.f), make_float3(0.f, 0.f, 0.f),
                    make_float3(0.f, 0.f, 0.f)};
    float3 nb = make_float3(v[0], v[1], v[2]);
    // c = n . A
    nb = axpy3f(v[3], P3[0], nb);
    cb[0] = axpy3f(v[3], n, cb[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float3 p = P3[k], q = P3[(k + 1) % 3];
      const float3 e = sub3(q, p);
      const float3 Mv = cross3(n, e);
      const float ml = __fsqrt_rn(dot3f(Mv, Mv));
      const float3 m = make_float3(__fdiv_rn(Mv.x, ml), __fdiv_rn(Mv.y, ml), __fdiv_rn(Mv.z, ml));
      float3 mb = make_float3(v[4 + 4 * k], v[5 + 4 * k], v[6 + 4 * k]);
      const float ob = v[7 + 4 * k];
      // o = m . p
      mb = axpy3f(ob, p, mb);
      cb[k] = axpy3f(ob, m, cb[k]);
      // m = M / |M|, M = n x e: n_bar += e x M_bar, e_bar = M_bar x n
      const float3 Mb = unit_adjoint(mb, m, ml);
      nb = make_float3(nb.x + cross3(e, Mb).x, nb.y + cross3(e, Mb).y, nb.z + cross3(e, Mb).z);
      const float3 eb = cross3(Mb, n);
      cb[(k + 1) % 3] = make_float3(cb[(k + 1) % 3].x + eb.x, cb[(k + 1) % 3].y + eb.y,
                                    cb[(k + 1) % 3].z + eb.z);
      cb[k] = make_float3(cb[k].x - eb.x, cb[k].y - eb.y, cb[k].z - eb.z);
    }
    // n = N / |N|, N = e1 x e2: e1_bar = e2 x N_bar, e2_bar = N_bar x e1
    const float3 Nb = unit_adjoint(nb, n, nl);
    const float3 e1b = cross3(e2, Nb), e2b = cross3(Nb, e1);
    cb[1] = make_float3(cb[1].x + e1b.x, cb[1].y + e1b.y, cb[1].z + e1b.z);
    cb[2] = make_float3(cb[2].x + e2b.x, cb[2].y + e2b.y, cb[2].z + e2b.z);
    cb[0] = make_float3(cb[0].x - e1b.x - e2b.x, cb[0].y - e1b.y - e2b.y,
                        cb[0].z - e1b.z - e2b.z);
    float* out = a.grad_tris + 9 * (size_t)w;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      out[3 * k] = cb[k].x;
      out[3 * k + 1] = cb[k].y;
      out[3 * k + 2] = cb[k].z;
    }
  }
}

// grad_tx = sum of the per-warp partials, in warp order (one thread per component)
// grad_tx = the sum of the per-unit TX adjoints, in a fixed order (one CTA of 256:
// strided partial sums, then a tree)
__global__ void __launch_bounds__(256) vjp3_finalize_kernel(const float* __restrict__ unit_tx,
                                                            long long n_units,
                                                            float* __restrict__ grad_tx) {
  __shared__ float part[3][256];
  float x = 0.f, y = 0.f, z = 0.f;
  for (long long u = threadIdx.x; u < n_units; u += blockDim.x) {
    x += unit_tx[3 * u];
    y += unit_tx[3 * u + 1];
    z += unit_tx[3 * u + 2];
  }
  part[0][threadIdx.x] = x;
  part[1][threadIdx.x] = y;
  part[2][threadIdx.x] = z;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int c = 0; c < 3; ++c) part[c][threadIdx.x] += part[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) grad_tx[threadIdx.x] = part[threadIdx.x][0];
}

__global__ void reduce3_kernel(const float* __restrict__ partial, long long n_chunks, long long R,
                               float* __restrict__ power) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < R;
       r += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (long long c = 0; c < n_chunks; ++c) acc += partial[c * R + r];
    power[r] = acc;
  }
}

// ------------------------------------------------------- batched descent (3D)
// The 2D batched descent's phases for triangle scenes (Sec. VI with Sec. VII's
// antenna placement): a problem is (scene, start); a forward unit is (problem,
// 32-receiver tile) with the scene's candidates split over the CTA's warps,
// taken from a global counter longest first; an adjoint unit is (problem, a block
// of warps x 32 candidates) of the argmin receiver, lanes holding candidates.
constexpr int BATCH3_MAX_WARPS = 8;

__device__ __forceinline__ long long batch3_n_candidates(int W, int K) {
  long long n = 1, level = 1;
  for (int k = 1; k <= K; ++k) {
    level = (k == 1) ? W : level * (W - 1);
    n += level;
  }
  return n;
}

__device__ __forceinline__ float batch3_alpha(const Batch3Args& a) {
  int st = *a.step;
  st = st < 0 ? 0 : (st >= a.n_alpha ? a.n_alpha - 1 : st);
  return a.alpha_sched[st];
}

__device__ __forceinline__ float3 batch3_tx(const Batch3Args& a, int p) {
  return make_float3(a.tx[3 * p], a.tx[3 * p + 1], a.tx[3 * p + 2]);
}

template <int MODE>
__global__ void __launch_bounds__(256, 2) batch3_forward_kernel(const Batch3Args a) {
  extern __shared__ float4 smem[];
  __shared__ long long s_unit;
  __shared__ int s_info[2];   // problem, sorted index
  __shared__ float s_part[BATCH3_MAX_WARPS][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const float alpha = batch3_alpha(a);
  for (;;) {
    if (threadIdx.x == 0) {
      const long long u = (long long)atomicAdd(a.counter, 1ULL);
      s_unit = u;
      if (u < a.n_fwd_units) {
        const int i = a.fwd_unit[u];
        s_info[0] = a.fwd_prob[i];
        s_info[1] = i;
      }
    }
    __syncthreads();
    const long long u = s_unit;
    if (u >= a.n_fwd_units) break;
    const int p = s_info[0];
    const long long tile = u - a.fwd_prefix[s_info[1]];
    const int s = p / a.T;
    const int woff = a.tri_off[s], W = a.tri_off[s + 1] - woff;
    const int roff = a.rx_off[s], R = a.rx_off[s + 1] - roff;
    const int K = a.order[s];
    const float3 tx = batch3_tx(a, p);
    SmemTris st{smem, smem + W, smem + 2 * W, smem + 3 * W};
    stage_tris(a.tris + 9 * (size_t)woff, W, st);
    __syncthreads();
    const int r = (int)(tile * 32) + lane;
    const bool live = r < R;
    const size_t ri = 3 * (size_t)(roff + (live ? r : R - 1));
    const float3 q = make_float3(__ldg(a.rx + ri), __ldg(a.rx + ri + 1), __ldg(a.rx + ri + 2));
    const long long nc = batch3_n_candidates(W, K);
    float acc = 0.f;
    // each warp takes a contiguous block of candidates and steps through it
    const long long cb = nc * warp / nwarps, ce = nc * (warp + 1) / nwarps;
    Cand cd;
    if (cb < ce) cd = decode_candidate(cb, W, K);
    for (long long c = cb; c < ce; ++c) {
      if (c > cb) next_candidate(cd, W);
      switch (cd.k) {
        case 0: acc += path_power3<MODE, 0>(st, W, tx, q, cd, alpha, a.gk[0]); break;
        case 1: acc += path_power3<MODE, 1>(st, W, tx, q, cd, alpha, a.gk[1]); break;
        case 2: acc += path_power3<MODE, 2>(st, W, tx, q, cd, alpha, a.gk[2]); break;
        default: acc += path_power3<MODE, 3>(st, W, tx, q, cd, alpha, a.gk[3]); break;
      }
    }
    s_part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
      float sum = 0.f;
      for (int w2 = 0; w2 < nwarps; ++w2) sum += s_part[w2][lane];
      if (live) a.power[a.pw_off[p] + r] = sum;
    }
    __syncthreads();
  }
}

// loss = -min_r P_r and its argmin (lowest index among ties) per problem
__global__ void batch3_argmin_kernel(const Batch3Args a) {
  const int lane = threadIdx.x & 31;
  const int P = a.S * a.T;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const int step = *a.step;
  for (long long p = gw; p < P; p += nw) {
    const int s = (int)(p / a.T);
    const int R = a.rx_off[s + 1] - a.rx_off[s];
    const float* pw = a.power + a.pw_off[p];
    float best = INFINITY;
    int bi = 0x7fffffff;
    for (int r = lane; r < R; r += 32) {
      const float val = pw[r];
      if (val < best || (val == best && r < bi)) {
        best = val;
        bi = r;
      }
    }
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
      a.loss[p] = -best;
      a.argmin[p] = (bi < R) ? bi : 0;
      if (a.loss_hist && step >= 0 && step < a.hist_len) a.loss_hist[(long long)step * P + p] = -best;
    }
  }
}

// largest i with prefix[i] <= u (prefix[0] = 0, prefix[n] > u)
__device__ __forceinline__ int batch3_find(const long long* prefix, int n, long long u) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= u) lo = mid; else hi = mid;
  }
  return lo;
}

template <int MODE>
__global__ void __launch_bounds__(256, 1) batch3_adjoint_kernel(const Batch3Args a) {
  extern __shared__ float4 smem[];
  __shared__ long long s_unit;
  __shared__ int s_prob;
  __shared__ float s_part[BATCH3_MAX_WARPS][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const float alpha = batch3_alpha(a);
  const int P = a.S * a.T;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long u = (long long)atomicAdd(a.counter + 1, 1ULL);
      s_unit = u;
      if (u < a.n_adj_units) s_prob = batch3_find(a.adj_prefix, P, u);
    }
    __syncthreads();
    const long long u = s_unit;
    if (u >= a.n_adj_units) break;
    const int p = s_prob;
    const long long chunk = u - a.adj_prefix[p];
    const int s = p / a.T;
    const int woff = a.tri_off[s], W = a.tri_off[s + 1] - woff;
    const int roff = a.rx_off[s];
    const int K = a.order[s];
    const float3 tx = batch3_tx(a, p);
    SmemTris st{smem, smem + W, smem + 2 * W, smem + 3 * W};
    stage_tris(a.tris + 9 * (size_t)woff, W, st);
    __syncthreads();
    const size_t ri = 3 * (size_t)(roff + a.argmin[p]);
    const float3 q = make_float3(__ldg(a.rx + ri), __ldg(a.rx + ri + 1), __ldg(a.rx + ri + 2));
    const long long nc = batch3_n_candidates(W, K);
    const long long base = chunk * nwarps * 32 + (long long)warp * 32;
    float3 txb = make_float3(0.f, 0.f, 0.f);
    if (base < nc) {
      const long long c = base + lane;
      const bool livec = c < nc;
      const Cand mine = decode_candidate(livec ? c : nc - 1, W, K);
      const int k_lo = decode_candidate(base, W, K).k;
      const int k_hi = decode_candidate(min(base + 31, nc - 1), W, K).k;
      // candidates are ordered by reflection count: the warp runs each order present,
      // the lanes of other orders with weight 0 on a placeholder sequence
      for (int k = k_lo; k <= k_hi; ++k) {
        const bool use = livec && mine.k == k;
        Cand cd = mine;
        if (!use) {
          cd.k = k;
#pragma unroll
          for (int j = 0; j < KMAX; ++j) cd.w[j] = (j & 1) ? (W > 1 ? 1 : 0) : 0;
        }
        const float g = use ? -1.f : 0.f;   // loss = -P[argmin]
        switch (k) {
          case 0: path_vjp3<MODE, 0, false>(st, W, tx, q, cd, alpha, a.gk[0], g, txb, nullptr); break;
          case 1: path_vjp3<MODE, 1, false>(st, W, tx, q, cd, alpha, a.gk[1], g, txb, nullptr); break;
          case 2: path_vjp3<MODE, 2, false>(st, W, tx, q, cd, alpha, a.gk[2], g, txb, nullptr); break;
          default: path_vjp3<MODE, 3, false>(st, W, tx, q, cd, alpha, a.gk[3], g, txb, nullptr); break;
        }
      }
      txb.x = warp_sum3(txb.x);
      txb.y = warp_sum3(txb.y);
      txb.z = warp_sum3(txb.z);
    }
    if (lane == 0) {
      s_part[warp][0] = txb.x;
      s_part[warp][1] = txb.y;
      s_part[warp][2] = txb.z;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float g3[3] = {0.f, 0.f, 0.f};
      for (int w2 = 0; w2 < nwarps; ++w2)
        for (int i = 0; i < 3; ++i) g3[i] += s_part[w2][i];
      for (int i = 0; i < 3; ++i) a.adj_partial[3 * u + i] = g3[i];
    }
    __syncthreads();
  }
}

// Adam on the TX (three coordinates), the problem's adjoint partials added in unit order
__global__ void batch3_adam_kernel(const Batch3Args a) {
  const int P = a.S * a.T;
  const int t = *a.step + 1;   // Adam's 1-based step
  const float c1 = 1.f - powf(a.b1, (float)t), c2 = 1.f - powf(a.b2, (float)t);
  const float lr = a.lr * powf(a.lr_decay, (float)(t - 1));
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    float g[3] = {0.f, 0.f, 0.f};
    for (long long u = a.adj_prefix[p]; u < a.adj_prefix[p + 1]; ++u)
      for (int i = 0; i < 3; ++i) g[i] += a.adj_partial[3 * u + i];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float m = fmaf(a.b1, a.m[3 * p + i], (1.f - a.b1) * g[i]);
      const float v = fmaf(a.b2, a.v[3 * p + i], (1.f - a.b2) * g[i] * g[i]);
      a.m[3 * p + i] = m;
      a.v[3 * p + i] = v;
      const float mh = m / c1, vh = v / c2;
      float x = a.tx[3 * p + i] - lr * mh / (sqrtf(vh) + a.eps);
      x = fminf(fmaxf(x, a.lo[i]), a.hi[i]);
      a.tx[3 * p + i] = x;
    }
  }
}

__global__ void batch3_step_end_kernel(int32_t* step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

}  // namespace

size_t batch3_smem_bytes(int Wmax) { return (size_t)4 * (Wmax > 1 ? Wmax : 1) * sizeof(float4); }

cudaError_t batch3_set_smem_limits(int Wmax) {
  const int smem = (int)batch3_smem_bytes(Wmax);
  const void* kernels[] = {(const void*)batch3_forward_kernel<MODE_SIGMOID>,
                           (const void*)batch3_forward_kernel<MODE_HARD>,
                           (const void*)batch3_forward_kernel<MODE_STEP>,
                           (const void*)batch3_adjoint_kernel<MODE_SIGMOID>,
                           (const void*)batch3_adjoint_kernel<MODE_HARD>,
                           (const void*)batch3_adjoint_kernel<MODE_STEP>};
  for (const void* k : kernels) {
    const cudaError_t e =
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t batch3_occupancy(int mode, int threads, int Wmax, int* fwd_per_sm, int* adj_per_sm) {
  const size_t smem = batch3_smem_bytes(Wmax);
  cudaError_t e;
  switch (mode) {
    case MODE_SIGMOID:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(fwd_per_sm, batch3_forward_kernel<MODE_SIGMOID>, threads, smem);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(adj_per_sm, batch3_adjoint_kernel<MODE_SIGMOID>, threads, smem);
      return e;
    case MODE_HARD:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(fwd_per_sm, batch3_forward_kernel<MODE_HARD>, threads, smem);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(adj_per_sm, batch3_adjoint_kernel<MODE_HARD>, threads, smem);
      return e;
    default:
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(fwd_per_sm, batch3_forward_kernel<MODE_STEP>, threads, smem);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(adj_per_sm, batch3_adjoint_kernel<MODE_STEP>, threads, smem);
      return e;
  }
}

cudaError_t launch_batch3(const Batch3Args& a, int mode, int ctas_fwd, int ctas_adj, int threads,
                          int Wmax, bool full_step, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.counter, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const size_t smem = batch3_smem_bytes(Wmax);
  switch (mode) {
    case MODE_SIGMOID: batch3_forward_kernel<MODE_SIGMOID><<<ctas_fwd, threads, smem, st>>>(a); break;
    case MODE_HARD: batch3_forward_kernel<MODE_HARD><<<ctas_fwd, threads, smem, st>>>(a); break;
    default: batch3_forward_kernel<MODE_STEP><<<ctas_fwd, threads, smem, st>>>(a); break;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int P = a.S * a.T;
  const long long nb = ((long long)P * 32 + 255) / 256;
  batch3_argmin_kernel<<<(int)(nb < 1 ? 1 : (nb > 4096 ? 4096 : nb)), 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess || !full_step) return e;
  switch (mode) {
    case MODE_SIGMOID: batch3_adjoint_kernel<MODE_SIGMOID><<<ctas_adj, threads, smem, st>>>(a); break;
    case MODE_HARD: batch3_adjoint_kernel<MODE_HARD><<<ctas_adj, threads, smem, st>>>(a); break;
    default: batch3_adjoint_kernel<MODE_STEP><<<ctas_adj, threads, smem, st>>>(a); break;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int pb = (P + 255) / 256;
  batch3_adam_kernel<<<pb < 1 ? 1 : (pb > 4096 ? 4096 : pb), 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  batch3_step_end_kernel<<<1, 32, 0, st>>>(a.step);
  return cudaGetLastError();
}

size_t forward3_smem_bytes(int W) { return (size_t)4 * W * sizeof(float4); }

size_t vjp3_smem_bytes(int W, bool tri_grad) {
  return forward3_smem_bytes(W) + (tri_grad ? (size_t)W * TRI_SLOTS * sizeof(float) : 0);
}

size_t vjp3_workspace_floats(int W, int ctas, long long n_units, bool tri_grad) {
  // 4 floats for the 8-byte-aligned work-stealing counter, [n_units][3] TX adjoints,
  // then the per-CTA triangle tables
  return 4 + (size_t)n_units * 3 + (tri_grad ? (size_t)ctas * W * TRI_SLOTS : 0);
}

cudaError_t launch_forward3(const Fwd3Args& a, int mode, int ctas, int threads, cudaStream_t st) {
  const size_t smem = forward3_smem_bytes(a.W);
  if (a.n_units > 0) {
    if (a.unit_counter) {
      cudaError_t e = cudaMemsetAsync(a.unit_counter, 0, sizeof(unsigned long long), st);
      if (e != cudaSuccess) return e;
    }
    switch (mode) {
      case MODE_SIGMOID: forward3_kernel<MODE_SIGMOID><<<ctas, threads, smem, st>>>(a); break;
      case MODE_HARD: forward3_kernel<MODE_HARD><<<ctas, threads, smem, st>>>(a); break;
      default: forward3_kernel<MODE_STEP><<<ctas, threads, smem, st>>>(a); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (a.R > 0) {
    const long long nb = (a.R + 255) / 256;
    reduce3_kernel<<<(int)(nb < 4096 ? nb : 4096), 256, 0, st>>>(a.partial, a.n_chunks, a.R,
                                                                 a.power);
  }
  return cudaGetLastError();
}

cudaError_t launch_vjp3(const Vjp3Args& a, int mode, int ctas, int threads, cudaStream_t st) {
  const bool wg = a.grad_tris != nullptr;
  const size_t smem = vjp3_smem_bytes(a.W, wg);
  if (a.n_units > 0) {
    cudaError_t e0 = cudaMemsetAsync(a.unit_counter, 0, sizeof(unsigned long long), st);
    if (e0 != cudaSuccess) return e0;
    switch (mode * 2 + (wg ? 1 : 0)) {
      case MODE_SIGMOID * 2: vjp3_kernel<MODE_SIGMOID, false><<<ctas, threads, smem, st>>>(a); break;
      case MODE_SIGMOID * 2 + 1: vjp3_kernel<MODE_SIGMOID, true><<<ctas, threads, smem, st>>>(a); break;
      case MODE_HARD * 2: vjp3_kernel<MODE_HARD, false><<<ctas, threads, smem, st>>>(a); break;
      case MODE_HARD * 2 + 1: vjp3_kernel<MODE_HARD, true><<<ctas, threads, smem, st>>>(a); break;
      case MODE_STEP * 2: vjp3_kernel<MODE_STEP, false><<<ctas, threads, smem, st>>>(a); break;
      default: vjp3_kernel<MODE_STEP, true><<<ctas, threads, smem, st>>>(a); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    vjp3_finalize_kernel<<<1, 256, 0, st>>>(a.unit_tx, a.n_units, a.grad_tx);
    if (wg) {
      vjp3_tris_finalize_kernel<<<(a.W + 255) / 256, 256, 0, st>>>(a, ctas);
    }
  } else {
    cudaError_t e = cudaMemsetAsync(a.grad_tx, 0, 3 * sizeof(float), st);
    if (e != cudaSuccess) return e;
    if (wg) e = cudaMemsetAsync(a.grad_tris, 0, (size_t)a.W * 9 * sizeof(float), st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t vjp3_occupancy(int mode, bool tri_grad, int threads, int W, int* ctas_per_sm) {
  const size_t smem = vjp3_smem_bytes(W, tri_grad);
  switch (mode * 2 + (tri_grad ? 1 : 0)) {
    case MODE_SIGMOID * 2:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp3_kernel<MODE_SIGMOID, false>, threads, smem);
    case MODE_SIGMOID * 2 + 1:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp3_kernel<MODE_SIGMOID, true>, threads, smem);
    case MODE_HARD * 2:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp3_kernel<MODE_HARD, false>, threads, smem);
    case MODE_HARD * 2 + 1:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp3_kernel<MODE_HARD, true>, threads, smem);
    case MODE_STEP * 2:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp3_kernel<MODE_STEP, false>, threads, smem);
    default:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, vjp3_kernel<MODE_STEP, true>, threads, smem);
  }
}

cudaError_t forward3_occupancy(int mode, int threads, int W, int* ctas_per_sm) {
  const size_t smem = forward3_smem_bytes(W);
  switch (mode) {
    case MODE_SIGMOID:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, forward3_kernel<MODE_SIGMOID>,
                                                           threads, smem);
    case MODE_HARD:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, forward3_kernel<MODE_HARD>,
                                                           threads, smem);
    default:
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, forward3_kernel<MODE_STEP>,
                                                           threads, smem);
  }
}

cudaError_t forward3_set_smem_limit(int W) {
  const int smem = (int)forward3_smem_bytes(W);
  cudaError_t e = cudaFuncSetAttribute(forward3_kernel<MODE_SIGMOID>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(forward3_kernel<MODE_HARD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(forward3_kernel<MODE_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           smem);
  if (e != cudaSuccess) return e;
  const int s1 = (int)vjp3_smem_bytes(W, true);
#define DRT_SET3(M)                                                                           \
  e = cudaFuncSetAttribute(vjp3_kernel<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
  if (e != cudaSuccess) return e;                                                             \
  e = cudaFuncSetAttribute(vjp3_kernel<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s1); \
  if (e != cudaSuccess) return e;
  DRT_SET3(MODE_SIGMOID)
  DRT_SET3(MODE_HARD)
  DRT_SET3(MODE_STEP)
#undef DRT_SET3
  return e;
}

}  // namespace drt
