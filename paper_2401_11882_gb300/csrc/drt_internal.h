// Host <-> kernel argument blocks and launchers (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "drt.h"

namespace drt {

// Work decomposition shared by the forward and adjoint kernels: a unit is
// (32 receivers, or 64 for the two-receivers-per-lane forward) x (`chunk`
// consecutive candidates); unit u covers receiver tile u % n_tiles and candidate
// chunk u / n_tiles.
struct Decomp {
  bool pairs;   // forward with two receivers per lane (64-receiver tiles)
  long long n_cand;
  int chunk;
  long long n_chunks, n_tiles, n_units;
  int threads;   // threads per CTA
  int ctas;      // persistent grid size
};

struct FwdArgs {
  const float4* walls;
  int W;
  const float* rx;
  long long R;
  const float* tx;
  int K;
  float alpha;
  float gk[DRT_MAX_ORDER + 1];   // Gamma^k
  long long n_cand;
  int chunk;
  long long n_chunks, n_tiles, n_units;
  int cull;
  int exit_blocked;   // hard sigmoid, pairs: leave the wall loop of fully blocked warps
  bool pairs;       // two receivers per lane (n_tiles counts 64-receiver tiles)
  float* partial;   // [n_chunks][R]
  float* power;     // [R]
  float4* staged;   // [8 or 4][W] wall records in global memory (W > DRT_MAX_WALLS), or null
  float* saved;     // sigmoid: every path's leg visibilities [n_cand][K + 1][R], or null
  // work-stealing counter (zeroed by launch_forward), or null for a static split;
  // drt_forward points it at the first 8 bytes of `power`, which only the chunk-sum
  // kernel writes, after the forward kernel has finished
  unsigned long long* unit_counter;
};

// Coherent field (drt_field.cu): the forward's decomposition (one or two
// receivers per lane) with (re, im) partial sums.
struct FieldArgs {
  const float4* walls;
  int W;
  const float* rx;
  long long R;
  const float* tx;
  int K;
  float alpha;
  float refl_amp;        // constant amplitude coefficient per reflection (eps_r == 0)
  float eps_r;           // > 1: Fresnel TE coefficient of this relative permittivity; 0: refl_amp
  float inv_lambda_hi;   // 1/lambda = hi + lo
  float inv_lambda_lo;
  long long n_cand;
  int chunk;
  long long n_chunks, n_tiles, n_units;
  int cull;
  bool pairs;        // two receivers per lane (n_tiles counts 64-receiver tiles)
  float2* partial;   // [n_chunks][R]
  float2* field;     // [R]
  float* power;      // [R] or null
  float* saved;      // sigmoid: every path's leg visibilities [n_cand][K + 1][R], or null
  // work-stealing counter (zeroed by launch_field; drt_field points it at `field`,
  // which only the chunk-sum kernel writes), or null for a static split
  unsigned long long* unit_counter;
};

// 3D forward (drt_forward3d.cu): triangle walls, 3D receivers, one receiver per lane.
struct Fwd3Args {
  const float* tris;   // [W][9]
  int W;
  const float* rx;     // [R][3]
  long long R;
  const float* tx;     // [3]
  int K;
  float alpha;
  float gk[DRT_MAX_ORDER + 1];
  long long n_cand;
  int chunk;
  long long n_chunks, n_tiles, n_units;
  float* partial;      // [n_chunks][R]
  float* power;        // [R]
  // work-stealing counter (zeroed by launch_forward3; drt3_forward points it at
  // `power`, which only the chunk-sum kernel writes), or null for a static split
  unsigned long long* unit_counter;
};

// 3D transmitter adjoint (drt_forward3d.cu): lanes are receivers; per-warp partials.
struct Vjp3Args {
  const float* tris;
  int W;
  const float* rx;
  long long R;
  const float* tx;
  int K;
  float alpha;
  float gk[DRT_MAX_ORDER + 1];
  long long n_cand;
  int chunk;
  long long n_chunks, n_tiles, n_units;
  const float* grad_power;   // [R]
  unsigned long long* unit_counter;   // work stealing, zeroed by launch_vjp3
  float* unit_tx;            // [n_units][3] per-unit TX adjoints
  float* grad_tx;            // [3]
  float* cta_tris;           // [ctas][W][16] per-CTA record adjoints (triangle gradient only)
  float* grad_tris;          // [W][9] or null
};

struct VjpArgs {
  const float4* walls;
  int W;
  const float* rx;
  long long R;
  const float* tx;
  int K;
  float alpha;
  float gk[DRT_MAX_ORDER + 1];
  long long n_cand;
  int chunk;
  long long n_chunks, n_tiles, n_units;
  bool pairs;                // sigmoid receiver-tile kernel: two receivers per lane (64-receiver tiles)
  const float* grad_power;   // [R] (receiver-tile kernel)
  const int32_t* rx_index;   // [1]: one-receiver kernel (min-loss adjoint) when non-null
  const float* grad_loss;    // [1] or null (one-receiver kernel)
  float* cta_walls;          // [ctas][W][9] per-CTA wall-gradient partials (wall gradient only)
  float* warp_tx;            // [ctas * warps_per_cta][2]
  // receiver-tile kernels (drt_vjp, drt_field_vjp): the work-stealing counter
  // (zeroed by launch_vjp / launch_field_vjp) and the per-unit TX adjoints
  // [n_units][2]; null for the min-loss kernel (per-warp TX adjoints in warp_tx)
  unsigned long long* unit_counter;
  float* unit_tx;
  float* grad_tx;            // [2]
  float* grad_walls;         // [W][4] or null
  // sigmoid: the forward's leg visibilities [n_cand][K + 1][R] (drt_forward_save), read
  // instead of the first wall sweep; or null
  const float* saved;
  // coherent-field adjoint only (drt_field_vjp): the field E [R] from drt_field and
  // the field's constants; grad_power then weighs |E_r|^2
  const float2* field;
  float inv_lambda_hi, inv_lambda_lo, k2pi, eps_r, refl_amp;
};

// number of float slots per wall in the adjoint's accumulators:
// d/d{nx, ny, c, ax, ay, bx, by, t0, len}
constexpr int VJP_SLOTS = 9;

// Sets the message drt_last_error() returns on this host thread.
void set_error_message(const char* msg);

size_t forward_smem_bytes(int W, bool pairs);
// whether the forward reads its wall records from a global staging buffer (more
// walls than its shared memory holds)
bool forward_streams_walls(int W);
// whether the forward runs two receivers per lane for this smoothing, alpha and tile flags
bool forward_uses_pairs(int mode, float alpha, int flags);
cudaError_t launch_forward(const FwdArgs& a, int mode, int ctas, int threads, cudaStream_t st);
cudaError_t forward_occupancy(int mode, bool pairs, int threads, int W, int* ctas_per_sm);
cudaError_t forward_set_smem_limit(int W);
// power[r] = sum over chunks of partial[chunk][r], in chunk order
cudaError_t launch_reduce_chunks(const float* partial, long long n_chunks, long long R,
                                 float* power, cudaStream_t st);
cudaError_t launch_loss(const float* power, int R, float* loss, int32_t* argmin, cudaStream_t st);
cudaError_t launch_loss_backward(const int32_t* argmin, const float* grad_loss, int R,
                                 float* grad_power, cudaStream_t st);

// Path-finder forward (drt_mpt.cu): the forward's decomposition (one receiver per
// lane) with the reflection points found by Min-Path-Tracing steps.
enum : int { FINDER_MPT = 0, FINDER_FPT = 1 };   // the path finder (Sec. V-B)
struct MptArgs {
  FwdArgs f;          // scene, decomposition, partial sums and power (pairs = false)
  int n_iter;         // finder steps from the walls' midpoints
  int finder;         // FINDER_MPT or FINDER_FPT
  float check_eps;    // the convergence check is s(check_eps - C)
  float* paths;       // drt_mpt_paths: [R][n_cand][K + 2] (tau_1..tau_K, C, kappa) or null
};
cudaError_t launch_forward_mpt(const MptArgs& a, int mode, int ctas, int threads, cudaStream_t st);
cudaError_t launch_mpt_paths(const MptArgs& a, int mode, int ctas, int threads, cudaStream_t st);
cudaError_t forward_mpt_occupancy(int mode, int finder, int threads, int W, int* ctas_per_sm);
cudaError_t forward_mpt_set_smem_limit(int W);

size_t forward3_smem_bytes(int W);
// Batched descent on 3D scenes (drt_forward3d.cu; the host plan is drt_batched.cu's):
// the 2D batched descent's five phases for triangle walls, one receiver per lane.
struct Batch3Args {
  const float* tris;          // [sum_s W_s][9]
  const int32_t* tri_off;     // [S + 1]
  const float* rx;            // [sum_s R_s][3]
  const int32_t* rx_off;      // [S + 1]
  const int32_t* order;       // K per scene
  int S, T;
  float gk[DRT_MAX_ORDER + 1];
  const float* alpha_sched;
  int n_alpha;
  int32_t* step;
  float* tx;                  // [S*T][3]
  float* m;                   // [S*T][3]
  float* v;                   // [S*T][3]
  float* loss;                // [S*T]
  float* loss_hist;           // [hist_len][S*T] or null
  int hist_len;
  float lr, b1, b2, eps, lr_decay;
  float lo[3], hi[3];         // the box the TX is clamped to
  unsigned long long* counter;   // [2]
  const int32_t* fwd_prob;
  const long long* fwd_prefix;
  const int32_t* fwd_unit;
  long long n_fwd_units;
  const long long* adj_prefix;
  long long n_adj_units;
  const long long* pw_off;
  float* power;
  int32_t* argmin;
  float* adj_partial;         // [n_adj_units][3]
};
size_t batch3_smem_bytes(int Wmax);
cudaError_t batch3_set_smem_limits(int Wmax);
cudaError_t batch3_occupancy(int mode, int threads, int Wmax, int* fwd_per_sm, int* adj_per_sm);
// the whole step (forward, argmin, adjoint, Adam, step counter), or the forward
// and argmin alone (evaluate)
cudaError_t launch_batch3(const Batch3Args& a, int mode, int ctas_fwd, int ctas_adj, int threads,
                          int Wmax, bool full_step, cudaStream_t st);

cudaError_t launch_forward3(const Fwd3Args& a, int mode, int ctas, int threads, cudaStream_t st);
cudaError_t forward3_occupancy(int mode, int threads, int W, int* ctas_per_sm);
cudaError_t forward3_set_smem_limit(int W);
cudaError_t launch_vjp3(const Vjp3Args& a, int mode, int ctas, int threads, cudaStream_t st);
cudaError_t vjp3_occupancy(int mode, bool tri_grad, int threads, int W, int* ctas_per_sm);
size_t vjp3_workspace_floats(int W, int ctas, long long n_units, bool tri_grad);

cudaError_t launch_field(const FieldArgs& a, int mode, int ctas, int threads, cudaStream_t st);
cudaError_t field_occupancy(int mode, bool pairs, int threads, int W, int* ctas_per_sm);
cudaError_t field_set_smem_limit(int W);

size_t vjp_smem_bytes(int W, bool wall_grad, bool pairs);
// whether drt_vjp's receiver-tile kernel holds two receivers per lane for this smoothing and flags
bool vjp_uses_pairs(int mode, int flags);
cudaError_t launch_vjp(const VjpArgs& a, int mode, int ctas, int threads, cudaStream_t st);
cudaError_t vjp_occupancy(int mode, bool wall_grad, bool pairs, int threads, int W,
                          int* ctas_per_sm);
cudaError_t vjp_set_smem_limit(int W);
cudaError_t launch_field_vjp(const VjpArgs& a, int mode, int ctas, int threads, cudaStream_t st);
cudaError_t field_vjp_occupancy(int mode, bool wall_grad, int threads, int W, int* ctas_per_sm);

}  // namespace drt
