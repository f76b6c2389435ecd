// Batched gradient descent on the transmitter position (Sec. VII: antenna
// placement by gradient steps on the loss of Eq. 8) for many scenes of uneven
// size at once, each with several starting positions.
//
// A "problem" is (scene s, start t).  One descent step is five kernels:
//   1. batch_forward_kernel: received power of every receiver of every problem.
//      Persistent CTAs take work units from a global counter; a unit is
//      (problem, 64-receiver tile, two receivers per lane with the packed
//      wall loop of drt_path_pair.cuh; 32 receivers for the unit step) with all
//      of the scene's path candidates split over the CTA's warps, and units are
//      ordered longest first.
//      The CTA stages the scene's walls in shared memory for each unit and
//      adds the warps' partial sums in warp order (deterministic).
//   2. batch_argmin_kernel: loss = -min_r P_r and its argmin per problem.
//   3. batch_adjoint_kernel: d loss / d tx for the argmin receiver of every
//      problem; a unit is (problem, a block of warps x 32 candidates), lanes
//      hold candidates (as in the one-receiver adjoint).
//   4. batch_adam_kernel: Adam on the TX position, clamped to a box.
//   5. batch_step_end_kernel: advances the device-side step counter, which
//      also selects the step's alpha from a schedule.
// Kernel boundaries order the phases, so no kernel waits on another CTA.
// The host captures one step into a CUDA graph once and replays it.  A batch of
// 3D scenes (dim 3) takes the same plan with the 3D phases of drt_forward3d.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "drt_common.cuh"
#include "drt_internal.h"
#include "drt_path.cuh"
#include "drt_path_pair.cuh"
#include "drt_path_vjp.cuh"

namespace drt {
namespace {

constexpr int BATCH_MAX_WARPS = 8;

struct BatchArgs {
  const float4* walls;
  const int32_t* wall_off;
  const float* rx;
  const int32_t* rx_off;
  const int32_t* order;      // K per scene
  int S, T;
  float gk[DRT_MAX_ORDER + 1];
  const float* alpha_sched;
  int n_alpha;
  int32_t* step;
  float* tx;                 // [S*T][2]
  float* m;                  // [S*T][2]
  float* v;                  // [S*T][2]
  float* loss;               // [S*T]
  float* loss_hist;          // [hist_len][S*T] or null
  int hist_len;
  float lr, b1, b2, eps, lo_x, lo_y, hi_x, hi_y, lr_decay;
  int cull;                      // skip the obstruction loop of warp-wide invalid paths (exact)
  // workspace
  unsigned long long* counter;   // [2]
  const int32_t* fwd_prob;       // [P] problems, longest forward first
  const long long* fwd_prefix;   // [P+1] tiles, in that order
  const int32_t* fwd_unit;       // [n_fwd_units] position in that order of each unit's problem
  long long n_fwd_units;
  const long long* adj_prefix;   // [P+1] adjoint units per problem (natural order)
  long long n_adj_units;
  const long long* pw_off;       // [P] offset of each problem's power array
  float* power;
  int32_t* argmin;               // [P]
  float* adj_partial;            // [n_adj_units][2]
};

__device__ __forceinline__ long long n_candidates(int W, int K) {
  long long n = 1, level = 1;
  for (int k = 1; k <= K; ++k) {
    level = (k == 1) ? W : level * (W - 1);
    n += level;
  }
  return n;
}

__device__ __forceinline__ float step_alpha(const BatchArgs& a) {
  int st = *a.step;
  st = st < 0 ? 0 : (st >= a.n_alpha ? a.n_alpha - 1 : st);
  return a.alpha_sched[st];
}

// largest i with prefix[i] <= u (prefix[0] = 0, prefix[n] > u)
__device__ __forceinline__ int find_unit(const long long* prefix, int n, long long u) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= u) lo = mid; else hi = mid;
  }
  return lo;
}

template <int MODE, int K>
__device__ __forceinline__ float batch_path_power(const SmemWalls& sw, int W, float2 txy, float2 q,
                                                  const Cand& cd, float alpha, float gk, int cull,
                                                  bool masked) {
  return masked ? path_power<MODE, K, true>(sw, W, txy, q, cd, alpha, gk, cull)
                : path_power<MODE, K>(sw, W, txy, q, cd, alpha, gk, cull);
}

template <int MODE, int K, bool EXIT>
__device__ __forceinline__ float2 batch_path_power2(const SmemWalls& sw, const SmemPairs& pr, int W,
                                                    float2 txy, float2 q0, float2 q1,
                                                    const Cand& cd, float alpha, float gk,
                                                    int cull, bool masked) {
  if (masked)   // alpha above the packed loop's range: one receiver at a time, masked
    return make_float2(path_power<MODE, K, true>(sw, W, txy, q0, cd, alpha, gk, cull),
                       path_power<MODE, K, true>(sw, W, txy, q1, cd, alpha, gk, cull));
  return path_power_pair<MODE, K, EXIT>(sw, pr, W, txy, q0, q1, cd, alpha, gk, cull);
}

// PAIRS: lane l holds receivers l and l + 32 of a 64-receiver tile.
// EXIT (hard sigmoid, PAIRS): the exact exit of warps whose paths are all blocked
// (DRT_TILE_EXIT_BLOCKED).
template <int MODE, bool PAIRS, bool EXIT = false>
__global__ void __launch_bounds__(256, PAIRS ? 2 : 1) batch_forward_kernel(const BatchArgs a) {
  extern __shared__ float4 smem[];
  __shared__ long long s_unit;
  __shared__ int s_info[2];   // problem, sorted index
  __shared__ float s_part[BATCH_MAX_WARPS][PAIRS ? 64 : 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const float alpha = step_alpha(a);
  constexpr int TILE = PAIRS ? 64 : 32;
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
    const int woff = a.wall_off[s], W = a.wall_off[s + 1] - woff;
    const int roff = a.rx_off[s], R = a.rx_off[s + 1] - roff;
    const int K = a.order[s];
    const float2 txy = reinterpret_cast<const float2*>(a.tx)[p];
    SmemWalls sw{smem, smem + W, smem + 2 * W, smem + 3 * W};
    SmemPairs pr{smem + 4 * W, smem + 5 * W, smem + 6 * W, smem + 7 * W};
    stage_walls<MODE>(a.walls + woff, W, txy, alpha, sw);
    __syncthreads();
    if (PAIRS) {
      stage_pairs<MODE>(sw, W, pr);
      __syncthreads();
    }
    const int r0 = (int)(tile * TILE) + lane, r1 = r0 + 32;
    const bool live0 = r0 < R, live1 = PAIRS && r1 < R;
    const float2 q0 = __ldg(reinterpret_cast<const float2*>(a.rx) + roff + (live0 ? r0 : R - 1));
    const float2 q1 = __ldg(reinterpret_cast<const float2*>(a.rx) + roff + (live1 ? r1 : R - 1));
    const long long nc = n_candidates(W, K);
    float acc0 = 0.f, acc1 = 0.f;
    const bool masked = alpha > FAST_SKIP_MAX_ALPHA;
    // each warp takes a contiguous block of candidates and steps through it
    const long long cb = nc * warp / nwarps, ce = nc * (warp + 1) / nwarps;
    Cand cd;
    if (cb < ce) cd = decode_candidate(cb, W, K);
    for (long long c = cb; c < ce; ++c) {
      if (c > cb) next_candidate(cd, W);
      if (PAIRS) {
        float2 pp;
        switch (cd.k) {
          case 0: pp = batch_path_power2<MODE, 0, EXIT>(sw, pr, W, txy, q0, q1, cd, alpha, a.gk[0], a.cull, masked); break;
          case 1: pp = batch_path_power2<MODE, 1, EXIT>(sw, pr, W, txy, q0, q1, cd, alpha, a.gk[1], a.cull, masked); break;
          case 2: pp = batch_path_power2<MODE, 2, EXIT>(sw, pr, W, txy, q0, q1, cd, alpha, a.gk[2], a.cull, masked); break;
          default: pp = batch_path_power2<MODE, 3, EXIT>(sw, pr, W, txy, q0, q1, cd, alpha, a.gk[3], a.cull, masked); break;
        }
        acc0 += pp.x;
        acc1 += pp.y;
      } else {
        switch (cd.k) {
          case 0: acc0 += batch_path_power<MODE, 0>(sw, W, txy, q0, cd, alpha, a.gk[0], a.cull, masked); break;
          case 1: acc0 += batch_path_power<MODE, 1>(sw, W, txy, q0, cd, alpha, a.gk[1], a.cull, masked); break;
          case 2: acc0 += batch_path_power<MODE, 2>(sw, W, txy, q0, cd, alpha, a.gk[2], a.cull, masked); break;
          default: acc0 += batch_path_power<MODE, 3>(sw, W, txy, q0, cd, alpha, a.gk[3], a.cull, masked); break;
        }
      }
    }
    s_part[warp][lane] = acc0;
    if (PAIRS) s_part[warp][lane + 32 * PAIRS] = acc1;
    __syncthreads();
    if (warp == 0) {
      float sum0 = 0.f, sum1 = 0.f;
      for (int w2 = 0; w2 < nwarps; ++w2) {
        sum0 += s_part[w2][lane];
        if (PAIRS) sum1 += s_part[w2][lane + 32 * PAIRS];
      }
      if (live0) a.power[a.pw_off[p] + r0] = sum0;
      if (live1) a.power[a.pw_off[p] + r1] = sum1;
    }
    __syncthreads();
  }
}

__global__ void batch_argmin_kernel(const BatchArgs a) {
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

template <int MODE>
__global__ void __launch_bounds__(256) batch_adjoint_kernel(const BatchArgs a) {
  extern __shared__ float4 smem[];
  __shared__ long long s_unit;
  __shared__ int s_prob;
  __shared__ float s_part[BATCH_MAX_WARPS][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const float alpha = step_alpha(a);
  const int P = a.S * a.T;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long u = (long long)atomicAdd(a.counter + 1, 1ULL);
      s_unit = u;
      if (u < a.n_adj_units) s_prob = find_unit(a.adj_prefix, P, u);
    }
    __syncthreads();
    const long long u = s_unit;
    if (u >= a.n_adj_units) break;
    const int p = s_prob;
    const long long chunk = u - a.adj_prefix[p];
    const int s = p / a.T;
    const int woff = a.wall_off[s], W = a.wall_off[s + 1] - woff;
    const int roff = a.rx_off[s];
    const int K = a.order[s];
    const float2 txy = reinterpret_cast<const float2*>(a.tx)[p];
    VSmem vs;
    vs.G = smem;
    vs.E = smem + W;
    vs.T = smem + 2 * W;
    vs.H = smem + 3 * W;
    vs.acc = nullptr;
    stage_walls<MODE>(a.walls + woff, W, txy, alpha, SmemWalls{vs.G, vs.E, vs.T, vs.H});
    __syncthreads();
    const float2 q = __ldg(reinterpret_cast<const float2*>(a.rx) + roff + a.argmin[p]);
    const long long nc = n_candidates(W, K);
    const long long base = chunk * nwarps * 32 + (long long)warp * 32;
    float tbx = 0.f, tby = 0.f;
    if (base < nc) {
      const long long c = base + lane;
      const bool livec = c < nc;
      const Cand mine = decode_candidate(livec ? c : nc - 1, W, K);
      const int k_lo = decode_candidate(base, W, K).k;
      const int k_hi = decode_candidate(min(base + 31, nc - 1), W, K).k;
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
          case 0: path_vjp<MODE, 0, false, false>(vs, W, txy, q, cd, alpha, a.gk[0], g, tbx, tby); break;
          case 1: path_vjp<MODE, 1, false, false>(vs, W, txy, q, cd, alpha, a.gk[1], g, tbx, tby); break;
          case 2: path_vjp<MODE, 2, false, false>(vs, W, txy, q, cd, alpha, a.gk[2], g, tbx, tby); break;
          default: path_vjp<MODE, 3, false, false>(vs, W, txy, q, cd, alpha, a.gk[3], g, tbx, tby); break;
        }
      }
      tbx = warp_sum(tbx);
      tby = warp_sum(tby);
    }
    if (lane == 0) {
      s_part[warp][0] = tbx;
      s_part[warp][1] = tby;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float gx = 0.f, gy = 0.f;
      for (int w2 = 0; w2 < nwarps; ++w2) {
        gx += s_part[w2][0];
        gy += s_part[w2][1];
      }
      a.adj_partial[2 * u] = gx;
      a.adj_partial[2 * u + 1] = gy;
    }
    __syncthreads();
  }
}

__global__ void batch_adam_kernel(const BatchArgs a) {
  const int P = a.S * a.T;
  const int t = *a.step + 1;   // Adam's 1-based step
  const float c1 = 1.f - powf(a.b1, (float)t), c2 = 1.f - powf(a.b2, (float)t);
  const float lr = a.lr * powf(a.lr_decay, (float)(t - 1));
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    float gx = 0.f, gy = 0.f;
    for (long long u = a.adj_prefix[p]; u < a.adj_prefix[p + 1]; ++u) {
      gx += a.adj_partial[2 * u];
      gy += a.adj_partial[2 * u + 1];
    }
    float g[2] = {gx, gy};
    const float lo[2] = {a.lo_x, a.lo_y}, hi[2] = {a.hi_x, a.hi_y};
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float m = fmaf(a.b1, a.m[2 * p + i], (1.f - a.b1) * g[i]);
      const float v = fmaf(a.b2, a.v[2 * p + i], (1.f - a.b2) * g[i] * g[i]);
      a.m[2 * p + i] = m;
      a.v[2 * p + i] = v;
      const float mh = m / c1, vh = v / c2;
      float x = a.tx[2 * p + i] - lr * mh / (sqrtf(vh) + a.eps);
      x = fminf(fmaxf(x, lo[i]), hi[i]);
      a.tx[2 * p + i] = x;
    }
  }
}

__global__ void batch_step_end_kernel(int32_t* step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

template <typename F>
cudaError_t occupancy(F kern, int threads, size_t smem, int* n) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, threads, smem);
}

}  // namespace

// ------------------------------------------------------------------ host side
struct BatchPlan {
  int dim = 2;   // 2D segments or 3D triangles
  int S = 0, T = 0, P = 0, mode = 0, Wmax = 0, threads = 256, warps = 8;
  float gamma = 0.5f;
  const float* walls = nullptr;
  const int32_t* wall_off = nullptr;
  const float* rx = nullptr;
  const int32_t* rx_off = nullptr;
  const int32_t* order = nullptr;
  std::vector<int32_t> fwd_prob, fwd_unit;
  std::vector<long long> fwd_prefix, adj_prefix, pw_off;
  long long n_fwd_units = 0, n_adj_units = 0, n_power = 0;
  int ctas_fwd = 1, ctas_adj = 1, per_sm_req = 0, cull = 0, exit_blocked = 0;
  bool pairs = false;   // forward with two receivers per lane (64-receiver tiles)
  size_t off_funit = 0;
  size_t off_counter = 0, off_prob = 0, off_fprefix = 0, off_aprefix = 0, off_pwoff = 0,
         off_power = 0, off_argmin = 0, off_partial = 0, ws_bytes = 0;
  bool bound = false;
  BatchArgs args{};
  Batch3Args args3{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture_stream = nullptr;
};

namespace {

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

long long host_n_candidates(int W, int K) {
  long long n = 1, level = 1;
  for (int k = 1; k <= K; ++k) {
    level = (k == 1) ? W : level * (W - 1);
    n += level;
  }
  return n;
}

double host_forward_cost(int W, int K, int R) {
  double c = W, level = 1;
  for (int k = 1; k <= K; ++k) {
    level = (k == 1) ? W : level * (W - 1);
    c += level * ((k + 1.0) * W - 2.0 * k);
  }
  return c * R;
}

size_t batch_fwd_smem(int Wmax, bool pairs) { return (size_t)(pairs ? 8 : 4) * Wmax * sizeof(float4); }
size_t batch_adj_smem(int Wmax) { return (size_t)4 * Wmax * sizeof(float4); }

cudaError_t set_smem_limits(int Wmax) {
  const int s1 = (int)batch_fwd_smem(std::max(Wmax, 1), true), s2 = (int)batch_adj_smem(std::max(Wmax, 1));
  cudaError_t e;
#define DRT_B(K_, S_)                                                                     \
  e = cudaFuncSetAttribute(K_, cudaFuncAttributeMaxDynamicSharedMemorySize, S_);         \
  if (e != cudaSuccess) return e;
  DRT_B((batch_forward_kernel<MODE_SIGMOID, true>), s1)
  DRT_B((batch_forward_kernel<MODE_HARD, true>), s1)
  DRT_B((batch_forward_kernel<MODE_HARD, true, true>), s1)
  DRT_B((batch_forward_kernel<MODE_SIGMOID, false>), s1)
  DRT_B((batch_forward_kernel<MODE_HARD, false>), s1)
  DRT_B((batch_forward_kernel<MODE_STEP, false>), s1)
  DRT_B(batch_adjoint_kernel<MODE_SIGMOID>, s2)
  DRT_B(batch_adjoint_kernel<MODE_HARD>, s2)
  DRT_B(batch_adjoint_kernel<MODE_STEP>, s2)
#undef DRT_B
  return cudaSuccess;
}

void launch_batch_forward(BatchPlan* pl, size_t sf, cudaStream_t st) {
  const BatchArgs& a = pl->args;
  if (pl->pairs && pl->mode == MODE_SIGMOID)
    batch_forward_kernel<MODE_SIGMOID, true><<<pl->ctas_fwd, pl->threads, sf, st>>>(a);
  else if (pl->pairs && pl->exit_blocked)
    batch_forward_kernel<MODE_HARD, true, true><<<pl->ctas_fwd, pl->threads, sf, st>>>(a);
  else if (pl->pairs)
    batch_forward_kernel<MODE_HARD, true><<<pl->ctas_fwd, pl->threads, sf, st>>>(a);
  else if (pl->mode == MODE_SIGMOID)
    batch_forward_kernel<MODE_SIGMOID, false><<<pl->ctas_fwd, pl->threads, sf, st>>>(a);
  else if (pl->mode == MODE_HARD)
    batch_forward_kernel<MODE_HARD, false><<<pl->ctas_fwd, pl->threads, sf, st>>>(a);
  else
    batch_forward_kernel<MODE_STEP, false><<<pl->ctas_fwd, pl->threads, sf, st>>>(a);
}

cudaError_t launch_evaluate(BatchPlan* pl, cudaStream_t st) {
  if (pl->dim == 3)
    return launch_batch3(pl->args3, pl->mode, pl->ctas_fwd, pl->ctas_adj, pl->threads, pl->Wmax,
                         false, st);
  BatchArgs& a = pl->args;
  cudaError_t e = cudaMemsetAsync(a.counter, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const size_t sf = batch_fwd_smem(pl->Wmax, pl->pairs);
  launch_batch_forward(pl, sf, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int ab = (int)std::min<long long>(((long long)pl->P * 32 + 255) / 256, 4096);
  batch_argmin_kernel<<<std::max(ab, 1), 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_step(BatchPlan* pl, cudaStream_t st) {
  if (pl->dim == 3)
    return launch_batch3(pl->args3, pl->mode, pl->ctas_fwd, pl->ctas_adj, pl->threads, pl->Wmax,
                         true, st);
  BatchArgs& a = pl->args;
  cudaError_t e = cudaMemsetAsync(a.counter, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const size_t sf = batch_fwd_smem(pl->Wmax, pl->pairs), sa = batch_adj_smem(pl->Wmax);
  launch_batch_forward(pl, sf, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int ab = (int)std::min<long long>(((long long)pl->P * 32 + 255) / 256, 4096);
  batch_argmin_kernel<<<std::max(ab, 1), 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  switch (pl->mode) {
    case MODE_SIGMOID: batch_adjoint_kernel<MODE_SIGMOID><<<pl->ctas_adj, pl->threads, sa, st>>>(a); break;
    case MODE_HARD: batch_adjoint_kernel<MODE_HARD><<<pl->ctas_adj, pl->threads, sa, st>>>(a); break;
    default: batch_adjoint_kernel<MODE_STEP><<<pl->ctas_adj, pl->threads, sa, st>>>(a); break;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int pb = std::max(1, std::min((pl->P + 255) / 256, 4096));
  batch_adam_kernel<<<pb, 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  batch_step_end_kernel<<<1, 32, 0, st>>>(a.step);
  return cudaGetLastError();
}

}  // namespace

drt_status batch_plan_create(const drt_batch* b, const drt_tile* tile, BatchPlan** out,
                             std::string* err) {
  if (b->dim != 0 && b->dim != 2 && b->dim != 3) {
    *err = "dim must be 2 or 3";
    return DRT_ERR_INVALID_ARG;
  }
  BatchPlan* pl = new BatchPlan();
  pl->dim = b->dim == 3 ? 3 : 2;
  pl->S = b->n_scenes;
  pl->T = b->n_tx;
  pl->P = pl->S * pl->T;
  pl->mode = b->smoothing;
  pl->gamma = b->refl_coef;
  pl->walls = b->walls;
  pl->wall_off = b->wall_off;
  pl->rx = b->rx;
  pl->rx_off = b->rx_off;
  pl->order = b->max_order;
  pl->warps = (tile && tile->warps_per_cta) ? tile->warps_per_cta : 8;
  pl->threads = pl->warps * 32;
  pl->per_sm_req = tile ? tile->ctas_per_sm : 0;
  pl->cull = (tile && (tile->flags & DRT_TILE_CULL_INVALID)) ? 1 : 0;
  pl->exit_blocked = (tile && (tile->flags & DRT_TILE_EXIT_BLOCKED)) ? 1 : 0;
  pl->pairs = pl->dim == 2 && (pl->mode == MODE_HARD || pl->mode == MODE_SIGMOID) &&
              !(tile && (tile->flags & DRT_TILE_SINGLE_RX));
  std::vector<double> cost(pl->P);
  std::vector<long long> tiles(pl->P), adj_units(pl->P);
  pl->pw_off.resize(pl->P);
  long long pw = 0;
  for (int s = 0; s < pl->S; ++s) {
    const int W = b->wall_off_host[s + 1] - b->wall_off_host[s];
    const int R = b->rx_off_host[s + 1] - b->rx_off_host[s];
    const int K = b->max_order_host[s];
    if (W < 1 || W > DRT_MAX_WALLS || R < 1 || K < 0 || K > DRT_MAX_ORDER) {
      *err = "scene " + std::to_string(s) + ": need 1 <= W <= " + std::to_string(DRT_MAX_WALLS) +
             ", R >= 1, 0 <= K <= " + std::to_string(DRT_MAX_ORDER);
      delete pl;
      return DRT_ERR_INVALID_ARG;
    }
    if (b->wall_off_host[s] < 0 || b->rx_off_host[s] < 0) {
      *err = "negative offset";
      delete pl;
      return DRT_ERR_INVALID_ARG;
    }
    pl->Wmax = std::max(pl->Wmax, W);
    const long long nc = host_n_candidates(W, K);
    for (int t = 0; t < pl->T; ++t) {
      const int p = s * pl->T + t;
      cost[p] = host_forward_cost(W, K, R);
      tiles[p] = pl->pairs ? (R + 63) / 64 : (R + 31) / 32;
      adj_units[p] = (nc + pl->threads - 1) / pl->threads;
      pl->pw_off[p] = pw;
      pw += R;
    }
  }
  pl->n_power = pw;
  pl->fwd_prob.resize(pl->P);
  for (int p = 0; p < pl->P; ++p) pl->fwd_prob[p] = p;
  std::stable_sort(pl->fwd_prob.begin(), pl->fwd_prob.end(),
                   [&](int x, int y) { return cost[x] / tiles[x] > cost[y] / tiles[y]; });
  pl->fwd_prefix.assign(pl->P + 1, 0);
  for (int i = 0; i < pl->P; ++i) pl->fwd_prefix[i + 1] = pl->fwd_prefix[i] + tiles[pl->fwd_prob[i]];
  pl->adj_prefix.assign(pl->P + 1, 0);
  for (int p = 0; p < pl->P; ++p) pl->adj_prefix[p + 1] = pl->adj_prefix[p] + adj_units[p];
  pl->n_fwd_units = pl->fwd_prefix[pl->P];
  // unit -> its problem's position in the sorted order (one load per unit fetch
  // instead of a binary search over the prefix sums)
  pl->fwd_unit.resize(pl->n_fwd_units);
  for (int i = 0; i < pl->P; ++i)
    std::fill(pl->fwd_unit.begin() + pl->fwd_prefix[i], pl->fwd_unit.begin() + pl->fwd_prefix[i + 1], i);
  pl->n_adj_units = pl->adj_prefix[pl->P];
  size_t off = 0;
  pl->off_counter = off; off = align_up(off + 2 * sizeof(unsigned long long));
  pl->off_prob = off; off = align_up(off + (size_t)pl->P * sizeof(int32_t));
  pl->off_fprefix = off; off = align_up(off + (size_t)(pl->P + 1) * sizeof(long long));
  pl->off_funit = off; off = align_up(off + (size_t)pl->n_fwd_units * sizeof(int32_t));
  pl->off_aprefix = off; off = align_up(off + (size_t)(pl->P + 1) * sizeof(long long));
  pl->off_pwoff = off; off = align_up(off + (size_t)pl->P * sizeof(long long));
  pl->off_power = off; off = align_up(off + (size_t)pl->n_power * sizeof(float));
  pl->off_argmin = off; off = align_up(off + (size_t)pl->P * sizeof(int32_t));
  pl->off_partial = off;
  off = align_up(off + (size_t)pl->n_adj_units * pl->dim * sizeof(float));
  pl->ws_bytes = off;
  *out = pl;
  return DRT_OK;
}

drt_status batch_bind(BatchPlan* pl, const drt_descent_state* d, void* ws, size_t ws_bytes,
                      cudaStream_t st, std::string* err) {
  if (!ws || ws_bytes < pl->ws_bytes || (reinterpret_cast<uintptr_t>(ws) & 255)) {
    *err = "workspace must be 256-byte aligned and >= " + std::to_string(pl->ws_bytes) + " bytes";
    return DRT_ERR_WORKSPACE;
  }
  cudaError_t e = pl->dim == 3 ? batch3_set_smem_limits(pl->Wmax) : set_smem_limits(pl->Wmax);
  if (e != cudaSuccess) { *err = cudaGetErrorString(e); return DRT_ERR_CUDA; }
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return DRT_ERR_CUDA;
  }
  int occ_f = 0, occ_a = 0;
  const size_t sf = batch_fwd_smem(pl->Wmax, pl->pairs), sa = batch_adj_smem(pl->Wmax);
  if (pl->dim == 3) e = batch3_occupancy(pl->mode, pl->threads, pl->Wmax, &occ_f, &occ_a);
  else switch (pl->mode) {
    case MODE_SIGMOID:
      e = pl->pairs ? occupancy(batch_forward_kernel<MODE_SIGMOID, true>, pl->threads, sf, &occ_f)
                    : occupancy(batch_forward_kernel<MODE_SIGMOID, false>, pl->threads, sf, &occ_f);
      if (e == cudaSuccess) e = occupancy(batch_adjoint_kernel<MODE_SIGMOID>, pl->threads, sa, &occ_a);
      break;
    case MODE_HARD:
      e = pl->pairs ? occupancy(batch_forward_kernel<MODE_HARD, true>, pl->threads, sf, &occ_f)
                    : occupancy(batch_forward_kernel<MODE_HARD, false>, pl->threads, sf, &occ_f);
      if (e == cudaSuccess) e = occupancy(batch_adjoint_kernel<MODE_HARD>, pl->threads, sa, &occ_a);
      break;
    default:
      e = occupancy(batch_forward_kernel<MODE_STEP, false>, pl->threads, sf, &occ_f);
      if (e == cudaSuccess) e = occupancy(batch_adjoint_kernel<MODE_STEP>, pl->threads, sa, &occ_a);
      break;
  }
  if (e != cudaSuccess || occ_f < 1 || occ_a < 1) {
    *err = "batched kernels do not fit on an SM";
    return DRT_ERR_UNSUPPORTED;
  }
  if (pl->per_sm_req > 0) {
    occ_f = std::min(occ_f, pl->per_sm_req);
    occ_a = std::min(occ_a, pl->per_sm_req);
  }
  pl->ctas_fwd = (int)std::max(1LL, std::min((long long)sms * occ_f, pl->n_fwd_units));
  pl->ctas_adj = (int)std::max(1LL, std::min((long long)sms * occ_a, pl->n_adj_units));
  char* base = static_cast<char*>(ws);
  // tables
  if ((e = cudaMemcpyAsync(base + pl->off_prob, pl->fwd_prob.data(), pl->P * sizeof(int32_t),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + pl->off_fprefix, pl->fwd_prefix.data(),
                           (pl->P + 1) * sizeof(long long), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + pl->off_funit, pl->fwd_unit.data(),
                           pl->n_fwd_units * sizeof(int32_t), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + pl->off_aprefix, pl->adj_prefix.data(),
                           (pl->P + 1) * sizeof(long long), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(base + pl->off_pwoff, pl->pw_off.data(), pl->P * sizeof(long long),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return DRT_ERR_CUDA;
  }
  if (pl->dim == 3) {
    Batch3Args& b3 = pl->args3;
    b3.tris = pl->walls;
    b3.tri_off = pl->wall_off;
    b3.rx = pl->rx;
    b3.rx_off = pl->rx_off;
    b3.order = pl->order;
    b3.S = pl->S;
    b3.T = pl->T;
    b3.gk[0] = 1.f;
    for (int k = 1; k <= DRT_MAX_ORDER; ++k) b3.gk[k] = b3.gk[k - 1] * pl->gamma;
    b3.alpha_sched = d->alpha_schedule;
    b3.n_alpha = d->n_alpha;
    b3.step = d->step;
    b3.tx = d->tx;
    b3.m = d->adam_m;
    b3.v = d->adam_v;
    b3.loss = d->loss;
    b3.loss_hist = d->loss_history;
    b3.hist_len = d->history_len;
    b3.lr = d->lr;
    b3.b1 = d->beta1;
    b3.b2 = d->beta2;
    b3.eps = d->eps;
    b3.lr_decay = d->lr_decay;
    b3.lo[0] = d->lo_x;
    b3.lo[1] = d->lo_y;
    b3.lo[2] = d->lo_z;
    b3.hi[0] = d->hi_x;
    b3.hi[1] = d->hi_y;
    b3.hi[2] = d->hi_z;
    b3.counter = reinterpret_cast<unsigned long long*>(base + pl->off_counter);
    b3.fwd_prob = reinterpret_cast<const int32_t*>(base + pl->off_prob);
    b3.fwd_prefix = reinterpret_cast<const long long*>(base + pl->off_fprefix);
    b3.fwd_unit = reinterpret_cast<const int32_t*>(base + pl->off_funit);
    b3.n_fwd_units = pl->n_fwd_units;
    b3.adj_prefix = reinterpret_cast<const long long*>(base + pl->off_aprefix);
    b3.n_adj_units = pl->n_adj_units;
    b3.pw_off = reinterpret_cast<const long long*>(base + pl->off_pwoff);
    b3.power = reinterpret_cast<float*>(base + pl->off_power);
    b3.argmin = reinterpret_cast<int32_t*>(base + pl->off_argmin);
    b3.adj_partial = reinterpret_cast<float*>(base + pl->off_partial);
  }
  BatchArgs& a = pl->args;
  a.walls = reinterpret_cast<const float4*>(pl->walls);
  a.wall_off = pl->wall_off;
  a.rx = pl->rx;
  a.rx_off = pl->rx_off;
  a.order = pl->order;
  a.S = pl->S;
  a.T = pl->T;
  a.gk[0] = 1.f;
  for (int k = 1; k <= DRT_MAX_ORDER; ++k) a.gk[k] = a.gk[k - 1] * pl->gamma;
  a.alpha_sched = d->alpha_schedule;
  a.n_alpha = d->n_alpha;
  a.step = d->step;
  a.tx = d->tx;
  a.m = d->adam_m;
  a.v = d->adam_v;
  a.loss = d->loss;
  a.loss_hist = d->loss_history;
  a.hist_len = d->history_len;
  a.lr = d->lr;
  a.b1 = d->beta1;
  a.b2 = d->beta2;
  a.eps = d->eps;
  a.lo_x = d->lo_x;
  a.lo_y = d->lo_y;
  a.hi_x = d->hi_x;
  a.hi_y = d->hi_y;
  a.lr_decay = d->lr_decay;
  a.cull = pl->cull;
  a.counter = reinterpret_cast<unsigned long long*>(base + pl->off_counter);
  a.fwd_prob = reinterpret_cast<const int32_t*>(base + pl->off_prob);
  a.fwd_prefix = reinterpret_cast<const long long*>(base + pl->off_fprefix);
  a.fwd_unit = reinterpret_cast<const int32_t*>(base + pl->off_funit);
  a.n_fwd_units = pl->n_fwd_units;
  a.adj_prefix = reinterpret_cast<const long long*>(base + pl->off_aprefix);
  a.n_adj_units = pl->n_adj_units;
  a.pw_off = reinterpret_cast<const long long*>(base + pl->off_pwoff);
  a.power = reinterpret_cast<float*>(base + pl->off_power);
  a.argmin = reinterpret_cast<int32_t*>(base + pl->off_argmin);
  a.adj_partial = reinterpret_cast<float*>(base + pl->off_partial);
  // capture one step on a private stream, once
  if (pl->exec) {
    cudaGraphExecDestroy(pl->exec);
    pl->exec = nullptr;
  }
  if (pl->graph) {
    cudaGraphDestroy(pl->graph);
    pl->graph = nullptr;
  }
  if (!pl->capture_stream &&
      (e = cudaStreamCreateWithFlags(&pl->capture_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return DRT_ERR_CUDA;
  }
  if ((e = cudaStreamBeginCapture(pl->capture_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
    *err = std::string("begin capture: ") + cudaGetErrorString(e);
    return DRT_ERR_CUDA;
  }
  cudaError_t le = launch_step(pl, pl->capture_stream);
  e = cudaStreamEndCapture(pl->capture_stream, &pl->graph);
  if (le != cudaSuccess || e != cudaSuccess) {
    *err = std::string("capture: ") + cudaGetErrorString(le != cudaSuccess ? le : e);
    return DRT_ERR_CUDA;
  }
  if ((e = cudaGraphInstantiate(&pl->exec, pl->graph, 0)) != cudaSuccess) {
    *err = std::string("instantiate: ") + cudaGetErrorString(e);
    return DRT_ERR_CUDA;
  }
  pl->bound = true;
  return DRT_OK;
}

drt_status batch_evaluate(BatchPlan* pl, cudaStream_t st, std::string* err) {
  if (!pl->bound) {
    *err = "plan is not bound";
    return DRT_ERR_INVALID_ARG;
  }
  cudaError_t e = launch_evaluate(pl, st);
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return DRT_ERR_CUDA;
  }
  return DRT_OK;
}

drt_status batch_run(BatchPlan* pl, int n_steps, int use_graph, cudaStream_t st, std::string* err) {
  if (!pl->bound) {
    *err = "plan is not bound";
    return DRT_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n_steps; ++i) {
    cudaError_t e = use_graph ? cudaGraphLaunch(pl->exec, st) : launch_step(pl, st);
    if (e != cudaSuccess) {
      *err = cudaGetErrorString(e);
      return DRT_ERR_CUDA;
    }
  }
  return DRT_OK;
}

void batch_destroy(BatchPlan* pl) {
  if (!pl) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  if (pl->capture_stream) cudaStreamDestroy(pl->capture_stream);
  delete pl;
}

size_t batch_workspace_bytes(const BatchPlan* pl) { return pl->ws_bytes; }

void batch_info(const BatchPlan* pl, long long* out) {
  out[0] = pl->P;
  out[1] = pl->n_fwd_units;
  out[2] = pl->n_adj_units;
  out[3] = pl->ctas_fwd;
  out[4] = pl->ctas_adj;
  out[5] = pl->Wmax;
  out[6] = pl->n_power;
  out[7] = pl->threads;
}

}  // namespace drt

struct drt_batch_plan {
  drt::BatchPlan impl;
};

namespace {

bool al(const void* p, size_t a) { return p && (reinterpret_cast<uintptr_t>(p) % a) == 0; }

drt_status bad(drt_status st, const std::string& msg) {
  drt::set_error_message(msg.c_str());
  return st;
}

}  // namespace

extern "C" {

drt_status drt_batch_plan_create(const drt_batch* b, const drt_tile* tile, drt_batch_plan** plan) {
  if (!b || !plan) return bad(DRT_ERR_INVALID_ARG, "batch or plan is NULL");
  if (b->n_scenes < 1 || b->n_tx < 1) return bad(DRT_ERR_INVALID_ARG, "n_scenes and n_tx must be >= 1");
  if (b->smoothing < 0 || b->smoothing > 2) return bad(DRT_ERR_INVALID_ARG, "unknown smoothing");
  if (!std::isfinite(b->refl_coef)) return bad(DRT_ERR_INVALID_ARG, "refl_coef must be finite");
  const bool d3 = b->dim == 3;
  if (!al(b->walls, d3 ? 4 : 16) || !al(b->rx, d3 ? 4 : 8) || !al(b->wall_off, 4) ||
      !al(b->rx_off, 4) || !al(b->max_order, 4))
    return bad(DRT_ERR_INVALID_ARG,
               "device arrays must be non-NULL and aligned (2D: walls 16, rx 8; 3D: 4)");
  if (!b->wall_off_host || !b->rx_off_host || !b->max_order_host)
    return bad(DRT_ERR_INVALID_ARG, "host copies of the offsets are required");
  if ((long long)b->n_scenes * b->n_tx > (1LL << 30)) return bad(DRT_ERR_UNSUPPORTED, "too many problems");
  if (tile && (tile->warps_per_cta < 0 || tile->warps_per_cta > 8 || tile->ctas_per_sm < 0))
    return bad(DRT_ERR_INVALID_ARG, "tile: warps_per_cta 0..8, ctas_per_sm >= 0");
  std::string err;
  drt::BatchPlan* p = nullptr;
  drt_status st = drt::batch_plan_create(b, tile, &p, &err);
  if (st != DRT_OK) return bad(st, err);
  drt_batch_plan* h = new drt_batch_plan();
  h->impl = std::move(*p);
  delete p;
  *plan = h;
  return DRT_OK;
}

drt_status drt_batch_workspace_size(const drt_batch_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return bad(DRT_ERR_INVALID_ARG, "NULL argument");
  *bytes = drt::batch_workspace_bytes(&plan->impl);
  return DRT_OK;
}

drt_status drt_batch_bind(drt_batch_plan* plan, const drt_descent_state* d, void* workspace,
                          size_t workspace_bytes, void* stream) {
  if (!plan || !d) return bad(DRT_ERR_INVALID_ARG, "NULL argument");
  const bool d3 = plan->impl.dim == 3;
  const size_t ta = d3 ? 4 : 8;
  if (!al(d->tx, ta) || !al(d->adam_m, ta) || !al(d->adam_v, ta) || !al(d->step, 4) ||
      !al(d->loss, 4) || !al(d->alpha_schedule, 4))
    return bad(DRT_ERR_INVALID_ARG, "state arrays must be non-NULL and aligned (tx, m, v: 8 in 2D)");
  if (d3 && !(d->lo_z <= d->hi_z)) return bad(DRT_ERR_INVALID_ARG, "clamp box: lo_z > hi_z");
  if (d->n_alpha < 1) return bad(DRT_ERR_INVALID_ARG, "n_alpha must be >= 1");
  if (d->loss_history && d->history_len < 0) return bad(DRT_ERR_INVALID_ARG, "history_len < 0");
  if (!(d->lr >= 0.f) || !std::isfinite(d->lr) || !(d->beta1 >= 0.f && d->beta1 < 1.f) ||
      !(d->beta2 >= 0.f && d->beta2 < 1.f) || !(d->eps > 0.f) || !(d->lo_x <= d->hi_x) ||
      !(d->lo_y <= d->hi_y) || !(d->lr_decay > 0.f && d->lr_decay <= 1.f))
    return bad(DRT_ERR_INVALID_ARG, "Adam parameters or clamp box out of range");
  std::string err;
  drt_status st = drt::batch_bind(&plan->impl, d, workspace, workspace_bytes,
                                  static_cast<cudaStream_t>(stream), &err);
  return st == DRT_OK ? st : bad(st, err);
}

drt_status drt_batch_run(drt_batch_plan* plan, int32_t n_steps, int32_t use_graph, void* stream) {
  if (!plan) return bad(DRT_ERR_INVALID_ARG, "plan is NULL");
  if (n_steps < 0) return bad(DRT_ERR_INVALID_ARG, "n_steps < 0");
  std::string err;
  drt_status st = drt::batch_run(&plan->impl, n_steps, use_graph, static_cast<cudaStream_t>(stream), &err);
  return st == DRT_OK ? st : bad(st, err);
}

drt_status drt_batch_evaluate(drt_batch_plan* plan, void* stream) {
  if (!plan) return bad(DRT_ERR_INVALID_ARG, "plan is NULL");
  std::string err;
  drt_status st = drt::batch_evaluate(&plan->impl, static_cast<cudaStream_t>(stream), &err);
  return st == DRT_OK ? st : bad(st, err);
}

drt_status drt_batch_plan_info(const drt_batch_plan* plan, int64_t* info) {
  if (!plan || !info) return bad(DRT_ERR_INVALID_ARG, "NULL argument");
  long long v[8];
  drt::batch_info(&plan->impl, v);
  for (int i = 0; i < 8; ++i) info[i] = v[i];
  return DRT_OK;
}

drt_status drt_batch_plan_destroy(drt_batch_plan* plan) {
  if (!plan) return DRT_OK;
  drt::BatchPlan& p = plan->impl;
  if (p.exec) cudaGraphExecDestroy(p.exec);
  if (p.graph) cudaGraphDestroy(p.graph);
  if (p.capture_stream) cudaStreamDestroy(p.capture_stream);
  p.exec = nullptr;
  p.graph = nullptr;
  p.capture_stream = nullptr;
  delete plan;
  return DRT_OK;
}

}  // extern "C"
