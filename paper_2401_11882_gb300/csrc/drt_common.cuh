// Device-side building blocks shared by the forward and adjoint kernels:
// per-wall records staged in shared memory, the smoothing functions, and the
// path-candidate decoder.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "drt.h"

namespace drt {

constexpr int KMAX = DRT_MAX_ORDER;
constexpr int WMAX = DRT_MAX_WALLS;
constexpr float LOG2E = 1.4426950408889634f;

enum : int { MODE_SIGMOID = 0, MODE_HARD = 1, MODE_STEP = 2 };

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// a * b + c clamped to [0, 1] in one rounding (PTX fma with the .sat modifier)
__device__ __forceinline__ float fma_sat(float a, float b, float c) {
  float y;
  asm("fma.rn.sat.f32 %0, %1, %2, %3;" : "=f"(y) : "f"(a), "f"(b), "f"(c));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Whether two scaled signed distances lie on the same side of a line, for the
// smoothed straddle pair X(x, y): their product is positive.  A product that
// underflows to 0 counts as opposite sides; one distance is then below 2^-74 of
// alpha's scale, its e = 2^-|z| rounds to 1, and the pair's two forms (e_x + e_y
// and 1 + e_x e_y) agree.  (A side known only through a tiny signed e, as the
// transmitter's in the wall records, is passed as +-1.)  One multiply on the FMA
// pipe and one compare.
__device__ __forceinline__ bool same_side(float a, float b) { return a * b > 0.f; }

// Work stealing of the persistent path kernels: a warp's first unit is its own
// index; the next one is the static split's (counter == nullptr) or one taken from
// a 64-bit counter that was zeroed before the launch, so no SM idles through a
// ragged last wave.  Every unit writes its own partial sums: results do not depend
// on which warp took which unit.  Warp-uniform; every lane must call it.
__device__ __forceinline__ long long next_unit_of(unsigned long long* counter, long long u,
                                                  long long nwarps, int lane) {
  if (!counter) return u + nwarps;
  unsigned long long v = 0;
  if (lane == 0) v = atomicAdd(counter, 1ULL);
  return nwarps + (long long)__shfl_sync(0xffffffffu, v, 0);
}

// ------------------------------------------------------------ smoothing
// s(x; alpha) = s(alpha x) (Eq. 3) for the three functions of Sec. IV:
// the value s(x), the complement s(-x) (by C4 equal to 1 - s(x), but
// evaluated directly so that it keeps its relative accuracy when small), and
// the derivative ds/dx.
struct Smooth3 {
  float s, sb, ds;
};

template <int MODE>
__device__ __forceinline__ Smooth3 smooth3(float x, float alpha) {
  Smooth3 r;
  if (MODE == MODE_HARD) {
    // Eqs. 5-6: relu6(alpha x + 3) / 6 = sat(alpha/6 x + 1/2); slope alpha/6 on the
    // open interval (-3/alpha, 3/alpha), 0 elsewhere (the kinks get 0).
    const float a6 = alpha * (1.0f / 6.0f);
    const float t = fmaf(x, a6, 0.5f);
    r.s = __saturatef(t);
    r.sb = __saturatef(fmaf(-x, a6, 0.5f));
    r.ds = (t > 0.0f && t < 1.0f) ? a6 : 0.0f;
  } else if (MODE == MODE_STEP) {
    // Eq. 1: theta(x) = [x > 0]; theta(0) = 0 on both sides.
    r.s = x > 0.0f ? 1.0f : 0.0f;
    r.sb = x < 0.0f ? 1.0f : 0.0f;
    r.ds = 0.0f;
  } else {
    // Eq. 4 with e = exp(-alpha |x|) in (0, 1]: s(|x|) = 1/(1+e), s(-|x|) = e/(1+e).
    const float z = x * (alpha * LOG2E);
    const float e = ex2_approx(-fabsf(z));
    const float q = rcp_approx(1.0f + e);   // 1 + e in (1, 2]: no special cases
    const float big = q, small = e * q;
    r.s = z >= 0.0f ? big : small;
    r.sb = z >= 0.0f ? small : big;
    r.ds = alpha * small * q;
  }
  return r;
}

// ------------------------------------------------------------ candidates
// Path candidate c of the list of every wall sequence of length 0..K with no
// wall twice in a row (Sec. V), ordered by length, then lexicographically.
struct Cand {
  int k;
  int w[KMAX > 0 ? KMAX : 1];
};

__device__ __forceinline__ Cand decode_candidate(long long c_in, int W, int K) {
  // N_K < 2^31 for every supported (W, K), so 32-bit unsigned arithmetic suffices
  unsigned c = (unsigned)c_in;
  Cand cd;
  cd.k = 0;
#pragma unroll
  for (int j = 0; j < KMAX; ++j) cd.w[j] = -1;
  if (c == 0) return cd;
  c -= 1;
  const unsigned Wm1 = (unsigned)(W - 1);
  unsigned block = (unsigned)W;   // number of candidates of order k: W (W-1)^(k-1)
  unsigned stride = 1;            // (W-1)^(k-1)
  int k = 1;
  while (k < K && c >= block) {
    c -= block;
    block *= Wm1;
    stride *= Wm1;
    ++k;
  }
  cd.k = k;
  // first wall: c / (W-1)^(k-1); every later digit d in [0, W-2] skips the previous wall
  int prev = (int)(c / stride);
  cd.w[0] = prev;
  unsigned rem = c - (unsigned)prev * stride;
#pragma unroll
  for (int j = 1; j < KMAX; ++j) {
    if (j < k) {
      stride /= Wm1;
      const int d = (int)(rem / stride);
      rem -= (unsigned)d * stride;
      prev = d < prev ? d : d + 1;
      cd.w[j] = prev;
    }
  }
  return cd;
}

// The candidate after cd in the same order (lexicographic increment of the wall
// sequence, each position skipping the wall before it), or the first candidate
// of the next order (0, 1, 0, 1, ...).  Only called while a next one exists.
__device__ __forceinline__ void next_candidate(Cand& cd, int W) {
  const int k = cd.k;
  int jstar = -1;   // position incremented (positions after it are reset)
#pragma unroll
  for (int j = KMAX - 1; j >= 0; --j) {
    if (jstar < 0 && j < k) {
      const int prevw = (j > 0) ? cd.w[j > 0 ? j - 1 : 0] : -1;
      int v = cd.w[j] + 1;
      if (v == prevw) ++v;
      if (v < W) {
        cd.w[j] = v;
        jstar = j;
      }
    }
  }
  if (jstar < 0) {   // order k exhausted: first sequence of order k + 1
    cd.k = k + 1;
#pragma unroll
    for (int i = 0; i < KMAX; ++i) cd.w[i] = (i < k + 1) ? (i & 1) : -1;
    return;
  }
#pragma unroll
  for (int i = 1; i < KMAX; ++i)
    if (i > jstar && i < k) cd.w[i] = (cd.w[i - 1] == 0) ? 1 : 0;
}

// ------------------------------------------------------------ wall records
// Per wall (Sec. V, relaxed geometry on the wall's infinite line):
//   G = {nx, ny, c, len}: unit normal n = (-u_y, u_x) of the unit direction
//       u = (B - A)/|B - A|, offset c = n . A (signed distance d(p) = n . p - c),
//       segment length.
//   E = {ax, ay, bx, by}: the end points.
//   T = {t0, 0, 0, 0}: t0 = u . A (coordinate along the wall: u . p - t0).
struct WallGeom {
  float4 G, E, T;
};

__device__ __forceinline__ WallGeom wall_geometry(float4 ab) {
  WallGeom g;
  const float ex = ab.z - ab.x, ey = ab.w - ab.y;
  const float len = __fsqrt_rn(fmaf(ex, ex, ey * ey));
  const float ux = __fdiv_rn(ex, len), uy = __fdiv_rn(ey, len);
  const float nx = -uy, ny = ux;
  g.G = make_float4(nx, ny, fmaf(nx, ab.x, ny * ab.y), len);
  g.E = ab;
  g.T = make_float4(fmaf(ux, ab.x, uy * ab.y), 0.f, 0.f, 0.f);
  return g;
}

// signed distance of p to the line of a wall record
__device__ __forceinline__ float line_dist(const float4& G, float px, float py) {
  return fmaf(G.x, px, fmaf(G.y, py, -G.z));
}

}  // namespace drt
