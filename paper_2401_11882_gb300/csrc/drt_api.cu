// C ABI of the library (include/drt.h): argument validation, work
// decomposition, workspace sizing and kernel launches.  No entry point
// allocates device memory or synchronises the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "drt.h"
#include "drt_internal.h"

namespace drt {
namespace {

thread_local std::string g_last_error;

drt_status fail(drt_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
drt_status fail(drt_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

drt_status cuda_fail(cudaError_t e, const char* where) {
  return fail(DRT_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Per-device facts, cached: SM count, and whether the kernels' dynamic shared
// memory limit has been raised on that device.
struct DeviceInfo {
  int sms = 0;
  bool smem_set = false;
};
std::mutex g_dev_mu;
DeviceInfo g_dev[64];

drt_status device_info(int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(DRT_ERR_UNSUPPORTED, "device index %d", dev);
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DeviceInfo& d = g_dev[dev];
  if (d.sms == 0) {
    e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  }
  if (!d.smem_set) {
    e = forward_set_smem_limit(DRT_MAX_WALLS);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(forward)");
    e = vjp_set_smem_limit(DRT_MAX_WALLS);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(vjp)");
    e = field_set_smem_limit(DRT_MAX_WALLS);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(field)");
    e = forward3_set_smem_limit(DRT_MAX_WALLS);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(forward3)");
    e = forward_mpt_set_smem_limit(DRT_MAX_WALLS);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(forward_mpt)");
    d.smem_set = true;
  }
  *sms = d.sms;
  return DRT_OK;
}

long long num_candidates(int W, int K) {
  long long n = 1, level = 1;
  for (int k = 1; k <= K; ++k) {
    level = (k == 1) ? W : level * (W - 1);
    n += level;
  }
  return n;
}

// max_walls: DRT_MAX_WALLS for the kernels that hold every wall in shared memory,
// DRT_MAX_WALLS_STREAMED for drt_forward (global staging above DRT_MAX_WALLS)
drt_status check_scene(const drt_scene* sc, int max_walls = DRT_MAX_WALLS) {
  if (!sc) return fail(DRT_ERR_INVALID_ARG, "scene is NULL");
  if (sc->n_walls < 1 || sc->n_walls > max_walls)
    return fail(sc->n_walls > max_walls ? DRT_ERR_UNSUPPORTED : DRT_ERR_INVALID_ARG,
                "n_walls = %d outside 1..%d", sc->n_walls, max_walls);
  if (sc->n_rx < 0) return fail(DRT_ERR_INVALID_ARG, "n_rx = %d < 0", sc->n_rx);
  if (sc->max_order < 0 || sc->max_order > DRT_MAX_ORDER)
    return fail(sc->max_order > DRT_MAX_ORDER ? DRT_ERR_UNSUPPORTED : DRT_ERR_INVALID_ARG,
                "max_order = %d outside 0..%d", sc->max_order, DRT_MAX_ORDER);
  // the kernels index the candidates with 32-bit integers
  if (num_candidates(sc->n_walls, sc->max_order) > 0x7fffffffLL)
    return fail(DRT_ERR_UNSUPPORTED, "%d walls with max_order %d: more than 2^31 - 1 candidates",
                sc->n_walls, sc->max_order);
  if (!(sc->alpha >= 0.f) || !std::isfinite(sc->alpha))
    return fail(DRT_ERR_INVALID_ARG, "alpha must be finite and >= 0");
  if (!std::isfinite(sc->refl_coef)) return fail(DRT_ERR_INVALID_ARG, "refl_coef must be finite");
  if (sc->smoothing < 0 || sc->smoothing > 2)
    return fail(DRT_ERR_INVALID_ARG, "unknown smoothing %d", sc->smoothing);
  if (!sc->walls || !aligned(sc->walls, 16))
    return fail(DRT_ERR_INVALID_ARG, "walls must be a 16-byte aligned device pointer");
  if (!sc->tx || !aligned(sc->tx, 4)) return fail(DRT_ERR_INVALID_ARG, "tx pointer");
  if (sc->n_rx > 0 && (!sc->rx || !aligned(sc->rx, 8)))
    return fail(DRT_ERR_INVALID_ARG, "rx must be an 8-byte aligned device pointer");
  return DRT_OK;
}

drt_status check_tile(const drt_tile* t) {
  if (!t) return DRT_OK;
  if (t->warps_per_cta < 0 || t->warps_per_cta > 8)
    return fail(DRT_ERR_INVALID_ARG, "warps_per_cta = %d outside 0..8", t->warps_per_cta);
  if (t->cands_per_unit < 0) return fail(DRT_ERR_INVALID_ARG, "cands_per_unit < 0");
  if (t->ctas_per_sm < 0 || t->ctas_per_sm > 32)
    return fail(DRT_ERR_INVALID_ARG, "ctas_per_sm = %d outside 0..32", t->ctas_per_sm);
  return DRT_OK;
}

// Largest number of (chunk, receiver) partial sums the forward keeps.
constexpr long long MAX_PARTIALS = 1LL << 26;
// Most (receiver tile, candidate chunk) units the dense adjoints (drt_vjp,
// drt_field_vjp, drt3_vjp) split their work into: they keep one TX adjoint per unit
// (8 or 12 bytes); more tiles than this make one unit per tile.
constexpr long long MAX_VJP_UNITS = 1LL << 22;

// VJP_RX: the min-loss adjoint's one-receiver kernel (lanes = candidates)
// VJP_TX: drt_vjp without the wall gradient (one receiver per lane)
// VJP3_TX: drt3_vjp without the triangle gradient
enum Kernel { FWD, VJP, VJP_TX, VJP_RX, FIELD, FIELD_VJP, FWD3, VJP3, VJP3_TX, FWD_MPT, FWD_FPT };

drt_status decompose(const drt_scene* sc, const drt_tile* t, Kernel kern, Decomp* d) {
  int sms = 0;
  drt_status st = device_info(&sms);
  if (st != DRT_OK) return st;
  const int W = sc->n_walls, K = sc->max_order;
  const long long R = sc->n_rx;
  const int warps = (t && t->warps_per_cta) ? t->warps_per_cta : 8;
  d->threads = warps * 32;
  d->n_cand = num_candidates(W, K);
  // default candidates per unit: 32 for the power and field forwards (finer units
  // balance the work-stealing grid's tail: 1% faster on the benchmark launch than
  // 64), 64 elsewhere
  const long long default_chunk = (kern == FWD || kern == FIELD) ? 32 : 64;
  long long chunk = (t && t->cands_per_unit) ? t->cands_per_unit : default_chunk;
  const bool finder = kern == FWD_MPT || kern == FWD_FPT;
  if ((kern == FWD || kern == FIELD || kern == FWD3 || finder) && R > 0) {
    const long long max_chunks = std::max(1LL, MAX_PARTIALS / R);
    chunk = std::max(chunk, (d->n_cand + max_chunks - 1) / max_chunks);
  }
  if (chunk > (1LL << 30)) chunk = 1LL << 30;
  d->chunk = (int)chunk;
  d->n_chunks = (d->n_cand + chunk - 1) / chunk;
  d->pairs = ((kern == FWD || kern == FIELD) &&
              forward_uses_pairs(sc->smoothing, sc->alpha, t ? t->flags : 0)) ||
             (kern == VJP && vjp_uses_pairs(sc->smoothing, t ? t->flags : 0));
  d->n_tiles = d->pairs ? (R + 63) / 64 : (R + 31) / 32;
  if ((kern == VJP || kern == VJP_TX || kern == FIELD_VJP || kern == VJP3 || kern == VJP3_TX) &&
      d->n_tiles * d->n_chunks > MAX_VJP_UNITS) {
    // larger chunks keep drt_vjp's per-unit TX table within MAX_VJP_UNITS entries
    const long long max_chunks = std::max(1LL, MAX_VJP_UNITS / std::max(1LL, d->n_tiles));
    d->chunk = (int)std::min((d->n_cand + max_chunks - 1) / max_chunks, 1LL << 30);
    d->n_chunks = (d->n_cand + d->chunk - 1) / d->chunk;
  }
  d->n_units = d->n_tiles * d->n_chunks;
  int per_sm = (t && t->ctas_per_sm) ? t->ctas_per_sm : 0;
  if (per_sm == 0) {
    const int mode = sc->smoothing;
    cudaError_t e = (kern == FWD)         ? forward_occupancy(mode, d->pairs, d->threads, W, &per_sm)
                    : (kern == FIELD)     ? field_occupancy(mode, d->pairs, d->threads, W, &per_sm)
                    : (kern == FIELD_VJP) ? field_vjp_occupancy(mode, true, d->threads, W, &per_sm)
                    : (kern == FWD3)      ? forward3_occupancy(mode, d->threads, W, &per_sm)
                    : (kern == VJP3)      ? vjp3_occupancy(mode, true, d->threads, W, &per_sm)
                    : (kern == VJP3_TX)   ? vjp3_occupancy(mode, false, d->threads, W, &per_sm)
                    : finder              ? forward_mpt_occupancy(
                                                mode, kern == FWD_FPT ? FINDER_FPT : FINDER_MPT,
                                                d->threads, W, &per_sm)
                                          : vjp_occupancy(mode, true, d->pairs, d->threads, W,
                                                          &per_sm);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (per_sm < 1) return fail(DRT_ERR_UNSUPPORTED, "kernel does not fit on an SM");
  }
  long long ctas = (long long)sms * per_sm;
  const long long needed = (d->n_units + warps - 1) / warps;
  if (kern == FWD || kern == FIELD || kern == FWD3 || finder)
    ctas = std::min(ctas, std::max(1LL, needed));
  d->ctas = (int)std::max(1LL, ctas);
  return DRT_OK;
}

void gamma_powers(float gamma, float* gk) {
  gk[0] = 1.f;
  for (int k = 1; k <= DRT_MAX_ORDER; ++k) gk[k] = gk[k - 1] * gamma;
}

// drt_vjp's workspace: [16 bytes: the work-stealing counter][ctas][W][VJP_SLOTS]
// wall partials, [warps][2] TX partials, then [n_units][2] per-unit TX adjoints
// (n_units <= max(MAX_VJP_UNITS, receiver tiles)).  The other adjoints use the
// same size from offset 0.
size_t vjp_workspace(const drt_scene* sc, const Decomp& d) {
  const size_t warps = (size_t)d.ctas * (d.threads / 32);
  return 16 + (size_t)d.ctas * sc->n_walls * VJP_SLOTS * sizeof(float) +
         warps * 2 * sizeof(float) + (size_t)d.n_units * 2 * sizeof(float);
}

}  // namespace

void set_error_message(const char* msg) { g_last_error = msg ? msg : ""; }

}  // namespace drt

using namespace drt;

extern "C" {

const char* drt_status_string(drt_status s) {
  switch (s) {
    case DRT_OK: return "ok";
    case DRT_ERR_INVALID_ARG: return "invalid argument";
    case DRT_ERR_UNSUPPORTED: return "unsupported configuration";
    case DRT_ERR_CUDA: return "CUDA error";
    case DRT_ERR_TIMEOUT: return "device wait timed out";
    case DRT_ERR_WORKSPACE: return "workspace too small";
  }
  return "unknown status";
}

const char* drt_last_error(void) { return g_last_error.c_str(); }

drt_status drt_num_candidates(int32_t n_walls, int32_t max_order, int64_t* count) {
  if (!count) return fail(DRT_ERR_INVALID_ARG, "count is NULL");
  if (n_walls < 1 || max_order < 0) return fail(DRT_ERR_INVALID_ARG, "n_walls/max_order");
  if (max_order > DRT_MAX_ORDER) return fail(DRT_ERR_UNSUPPORTED, "max_order > %d", DRT_MAX_ORDER);
  *count = num_candidates(n_walls, max_order);
  return DRT_OK;
}

// drt_forward's workspace: the per-chunk partial sums, then (more walls than
// shared memory holds) the staged wall records, 16-byte aligned
// The partial sums; rounded up to 16 bytes when the staged wall records follow them.
size_t forward_partials_bytes(const drt_scene* sc, const Decomp& d) {
  const size_t b = (size_t)d.n_chunks * (size_t)sc->n_rx * sizeof(float);
  return forward_streams_walls(sc->n_walls) ? (b + 15) & ~(size_t)15 : b;
}
size_t forward_workspace(const drt_scene* sc, const Decomp& d) {
  const size_t staged =
      forward_streams_walls(sc->n_walls) ? (d.pairs ? 8 : 4) * (size_t)sc->n_walls * 16 : 0;
  return forward_partials_bytes(sc, d) + staged;
}

drt_status drt_forward_workspace_size(const drt_scene* scene, const drt_tile* tile, size_t* bytes) {
  drt_status st = check_scene(scene, DRT_MAX_WALLS_STREAMED);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!bytes) return fail(DRT_ERR_INVALID_ARG, "bytes is NULL");
  Decomp d;
  if ((st = decompose(scene, tile, FWD, &d)) != DRT_OK) return st;
  *bytes = forward_workspace(scene, d);
  return DRT_OK;
}

namespace {
drt_status forward_impl(const drt_scene* scene, const drt_tile* tile, float* power, float* saved,
                        void* workspace, size_t workspace_bytes, void* stream) {
  drt_status st = check_scene(scene, DRT_MAX_WALLS_STREAMED);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (scene->n_rx > 0 && !power) return fail(DRT_ERR_INVALID_ARG, "power is NULL");
  if (scene->n_rx == 0) return DRT_OK;
  Decomp d;
  if ((st = decompose(scene, tile, FWD, &d)) != DRT_OK) return st;
  const size_t need = forward_workspace(scene, d);
  const bool streamed = forward_streams_walls(scene->n_walls);
  if (!workspace || workspace_bytes < need || (streamed && !aligned(workspace, 16)))
    return fail(DRT_ERR_WORKSPACE, "forward needs %zu workspace bytes, got %zu", need,
                workspace_bytes);
  FwdArgs a{};
  a.walls = reinterpret_cast<const float4*>(scene->walls);
  a.W = scene->n_walls;
  a.rx = scene->rx;
  a.R = scene->n_rx;
  a.tx = scene->tx;
  a.K = scene->max_order;
  a.alpha = scene->alpha;
  gamma_powers(scene->refl_coef, a.gk);
  a.n_cand = d.n_cand;
  a.chunk = d.chunk;
  a.n_chunks = d.n_chunks;
  a.n_tiles = d.n_tiles;
  a.n_units = d.n_units;
  a.cull = (tile && (tile->flags & DRT_TILE_CULL_INVALID)) ? 1 : 0;
  a.exit_blocked = (tile && (tile->flags & DRT_TILE_EXIT_BLOCKED)) ? 1 : 0;
  a.pairs = d.pairs;
  a.partial = static_cast<float*>(workspace);
  a.power = power;
  a.staged = streamed ? reinterpret_cast<float4*>(static_cast<char*>(workspace) +
                                                  forward_partials_bytes(scene, d))
                      : nullptr;
  a.saved = saved;
  // the work-stealing counter borrows power's first 8 bytes: the forward kernel
  // never touches power, and the chunk-sum kernel overwrites all of it afterwards
  if (scene->n_rx >= 2 && aligned(power, 8))
    a.unit_counter = reinterpret_cast<unsigned long long*>(power);
  cudaError_t e = launch_forward(a, scene->smoothing, d.ctas, d.threads,
                                 static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "forward launch");
  return DRT_OK;
}

// The saved visibilities' size, and the cases that can save them: the sigmoid
// (whose adjoint's first sweep they replace), walls in shared memory.
drt_status check_saved(const drt_scene* scene, const float* saved, long long* floats) {
  if (scene->smoothing != DRT_SMOOTH_SIGMOID)
    return fail(DRT_ERR_UNSUPPORTED, "saved visibilities are kept for the sigmoid only");
  if (scene->n_walls > DRT_MAX_WALLS)
    return fail(DRT_ERR_UNSUPPORTED, "saved visibilities need n_walls <= %d", DRT_MAX_WALLS);
  const long long n = num_candidates(scene->n_walls, scene->max_order) *
                      (scene->max_order + 1) * (long long)scene->n_rx;
  if (floats) *floats = n;
  if (n > 0 && (!saved || !aligned(saved, 4)))
    return fail(DRT_ERR_INVALID_ARG, "saved must be a 4-byte aligned device pointer");
  return DRT_OK;
}
}  // namespace

drt_status drt_forward(const drt_scene* scene, const drt_tile* tile, float* power,
                       void* workspace, size_t workspace_bytes, void* stream) {
  return forward_impl(scene, tile, power, nullptr, workspace, workspace_bytes, stream);
}

drt_status drt_saved_vis_size(const drt_scene* scene, int64_t* floats) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if (!floats) return fail(DRT_ERR_INVALID_ARG, "floats is NULL");
  long long n = 0;
  static const float dummy = 0.f;
  if ((st = check_saved(scene, &dummy, &n)) != DRT_OK) return st;
  *floats = n;
  return DRT_OK;
}

drt_status drt_forward_save(const drt_scene* scene, const drt_tile* tile, float* power,
                            float* saved, void* workspace, size_t workspace_bytes, void* stream) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_saved(scene, saved, nullptr)) != DRT_OK) return st;
  return forward_impl(scene, tile, power, saved, workspace, workspace_bytes, stream);
}

namespace {
drt_status check_mpt_args(int32_t n_iter, float check_eps) {
  if (n_iter < 0 || n_iter > DRT_MPT_MAX_ITER)
    return fail(DRT_ERR_INVALID_ARG, "n_iter = %d outside 0..%d", n_iter, DRT_MPT_MAX_ITER);
  if (!std::isfinite(check_eps)) return fail(DRT_ERR_INVALID_ARG, "check_eps must be finite");
  return DRT_OK;
}

MptArgs mpt_args(const drt_scene* scene, const drt_tile* tile, const Decomp& d, int32_t n_iter,
                 float check_eps) {
  MptArgs m{};
  FwdArgs& a = m.f;
  a.walls = reinterpret_cast<const float4*>(scene->walls);
  a.W = scene->n_walls;
  a.rx = scene->rx;
  a.R = scene->n_rx;
  a.tx = scene->tx;
  a.K = scene->max_order;
  a.alpha = scene->alpha;
  gamma_powers(scene->refl_coef, a.gk);
  a.n_cand = d.n_cand;
  a.chunk = d.chunk;
  a.n_chunks = d.n_chunks;
  a.n_tiles = d.n_tiles;
  a.n_units = d.n_units;
  a.cull = 0;
  a.pairs = false;
  (void)tile;
  m.n_iter = n_iter;
  m.check_eps = check_eps;
  return m;
}
}  // namespace

namespace {
drt_status finder_workspace_size(int finder, const drt_scene* scene, const drt_tile* tile,
                                  size_t* bytes) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!bytes) return fail(DRT_ERR_INVALID_ARG, "bytes is NULL");
  Decomp d;
  if ((st = decompose(scene, tile, finder == FINDER_FPT ? FWD_FPT : FWD_MPT, &d)) != DRT_OK)
    return st;
  *bytes = (size_t)d.n_chunks * (size_t)scene->n_rx * sizeof(float);
  return DRT_OK;
}

drt_status finder_forward(int finder, const drt_scene* scene, const drt_tile* tile,
                          int32_t n_iter, float check_eps, float* power, void* workspace,
                          size_t workspace_bytes, void* stream) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if ((st = check_mpt_args(n_iter, check_eps)) != DRT_OK) return st;
  if (scene->n_rx > 0 && !power) return fail(DRT_ERR_INVALID_ARG, "power is NULL");
  if (scene->n_rx == 0) return DRT_OK;
  Decomp d;
  if ((st = decompose(scene, tile, finder == FINDER_FPT ? FWD_FPT : FWD_MPT, &d)) != DRT_OK)
    return st;
  const size_t need = (size_t)d.n_chunks * (size_t)scene->n_rx * sizeof(float);
  if (!workspace || workspace_bytes < need)
    return fail(DRT_ERR_WORKSPACE, "path-finder forward needs %zu workspace bytes, got %zu",
                need, workspace_bytes);
  MptArgs m = mpt_args(scene, tile, d, n_iter, check_eps);
  m.finder = finder;
  m.f.partial = static_cast<float*>(workspace);
  m.f.power = power;
  m.paths = nullptr;
  // work stealing, the counter in power's first 8 bytes (as drt_forward)
  if (scene->n_rx >= 2 && aligned(power, 8))
    m.f.unit_counter = reinterpret_cast<unsigned long long*>(power);
  cudaError_t e = launch_forward_mpt(m, scene->smoothing, d.ctas, d.threads,
                                     static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "path-finder forward launch");
  return DRT_OK;
}

drt_status finder_paths(int finder, const drt_scene* scene, int32_t n_iter, float check_eps,
                        float* paths, void* stream) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_mpt_args(n_iter, check_eps)) != DRT_OK) return st;
  if (scene->n_rx > 0 && (!paths || !aligned(paths, 4)))
    return fail(DRT_ERR_INVALID_ARG, "paths must be a 4-byte aligned device pointer");
  if (scene->n_rx == 0) return DRT_OK;
  const long long n_cand = num_candidates(scene->n_walls, scene->max_order);
  if ((long long)scene->n_rx * n_cand * (scene->max_order + 2) > (1LL << 40))
    return fail(DRT_ERR_UNSUPPORTED, "paths output of %lld records is too large",
                (long long)scene->n_rx * n_cand);
  Decomp d;
  if ((st = decompose(scene, nullptr, finder == FINDER_FPT ? FWD_FPT : FWD_MPT, &d)) != DRT_OK)
    return st;
  MptArgs m = mpt_args(scene, nullptr, d, n_iter, check_eps);
  m.finder = finder;
  m.f.partial = nullptr;
  m.f.power = nullptr;
  m.paths = paths;
  cudaError_t e = launch_mpt_paths(m, scene->smoothing, d.ctas, d.threads,
                                   static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "path-finder paths launch");
  return DRT_OK;
}
}  // namespace

drt_status drt_forward_mpt_workspace_size(const drt_scene* scene, const drt_tile* tile,
                                          size_t* bytes) {
  return finder_workspace_size(FINDER_MPT, scene, tile, bytes);
}

drt_status drt_forward_mpt(const drt_scene* scene, const drt_tile* tile, int32_t n_iter,
                           float check_eps, float* power, void* workspace,
                           size_t workspace_bytes, void* stream) {
  return finder_forward(FINDER_MPT, scene, tile, n_iter, check_eps, power, workspace,
                        workspace_bytes, stream);
}

drt_status drt_mpt_paths(const drt_scene* scene, int32_t n_iter, float check_eps, float* paths,
                         void* stream) {
  return finder_paths(FINDER_MPT, scene, n_iter, check_eps, paths, stream);
}

drt_status drt_forward_fpt_workspace_size(const drt_scene* scene, const drt_tile* tile,
                                          size_t* bytes) {
  return finder_workspace_size(FINDER_FPT, scene, tile, bytes);
}

drt_status drt_forward_fpt(const drt_scene* scene, const drt_tile* tile, int32_t n_iter,
                           float check_eps, float* power, void* workspace,
                           size_t workspace_bytes, void* stream) {
  return finder_forward(FINDER_FPT, scene, tile, n_iter, check_eps, power, workspace,
                        workspace_bytes, stream);
}

drt_status drt_fpt_paths(const drt_scene* scene, int32_t n_iter, float check_eps, float* paths,
                         void* stream) {
  return finder_paths(FINDER_FPT, scene, n_iter, check_eps, paths, stream);
}

drt_status drt_field_workspace_size(const drt_scene* scene, const drt_tile* tile, size_t* bytes) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!bytes) return fail(DRT_ERR_INVALID_ARG, "bytes is NULL");
  Decomp d;
  if ((st = decompose(scene, tile, FIELD, &d)) != DRT_OK) return st;
  *bytes = (size_t)d.n_chunks * (size_t)scene->n_rx * 2 * sizeof(float);
  return DRT_OK;
}

namespace {
drt_status field_impl(const drt_scene* scene, const drt_tile* tile, float wavelength, float eps_r,
                      float* field, float* power, float* saved, void* workspace,
                      size_t workspace_bytes, void* stream) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!(wavelength > 0.f) || !std::isfinite(wavelength))
    return fail(DRT_ERR_INVALID_ARG, "wavelength must be finite and > 0");
  if (!(eps_r == 0.f || eps_r >= 1.f) || !std::isfinite(eps_r))
    return fail(DRT_ERR_INVALID_ARG, "eps_r must be 0 (constant coefficient) or finite and >= 1");
  if (eps_r == 0.f && !(scene->refl_coef >= 0.f))
    return fail(DRT_ERR_INVALID_ARG, "refl_coef must be >= 0 for the constant coefficient");
  if (scene->n_rx > 0 && (!field || !aligned(field, 8)))
    return fail(DRT_ERR_INVALID_ARG, "field must be an 8-byte aligned device pointer");
  if (scene->n_rx == 0) return DRT_OK;
  Decomp d;
  if ((st = decompose(scene, tile, FIELD, &d)) != DRT_OK) return st;
  const size_t need = (size_t)d.n_chunks * (size_t)scene->n_rx * 2 * sizeof(float);
  if (!workspace || workspace_bytes < need || !aligned(workspace, 8))
    return fail(DRT_ERR_WORKSPACE, "field needs %zu 8-byte aligned workspace bytes, got %zu",
                need, workspace_bytes);
  FieldArgs a{};
  a.walls = reinterpret_cast<const float4*>(scene->walls);
  a.W = scene->n_walls;
  a.rx = scene->rx;
  a.R = scene->n_rx;
  a.tx = scene->tx;
  a.K = scene->max_order;
  a.alpha = scene->alpha;
  // eps_r = 1: the Fresnel coefficient is 0 at every angle; pass it as that constant
  a.refl_amp = eps_r == 0.f ? -(float)std::sqrt((double)scene->refl_coef) : 0.f;
  a.eps_r = eps_r == 1.f ? 0.f : eps_r;
  const double inv = 1.0 / (double)wavelength;
  a.inv_lambda_hi = (float)inv;
  a.inv_lambda_lo = (float)(inv - (double)a.inv_lambda_hi);
  a.n_cand = d.n_cand;
  a.chunk = d.chunk;
  a.n_chunks = d.n_chunks;
  a.n_tiles = d.n_tiles;
  a.n_units = d.n_units;
  a.cull = (tile && (tile->flags & DRT_TILE_CULL_INVALID)) ? 1 : 0;
  a.pairs = d.pairs;
  a.partial = static_cast<float2*>(workspace);
  a.field = reinterpret_cast<float2*>(field);
  a.power = power;
  // work stealing, the counter in field's first 8 bytes until the chunk sums land
  if (aligned(field, 8)) a.unit_counter = reinterpret_cast<unsigned long long*>(field);
  a.saved = saved;
  cudaError_t e = launch_field(a, scene->smoothing, d.ctas, d.threads,
                               static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "field launch");
  return DRT_OK;
}
}  // namespace

drt_status drt_field(const drt_scene* scene, const drt_tile* tile, float wavelength, float eps_r,
                     float* field, float* power, void* workspace, size_t workspace_bytes,
                     void* stream) {
  return field_impl(scene, tile, wavelength, eps_r, field, power, nullptr, workspace,
                    workspace_bytes, stream);
}

drt_status drt_field_save(const drt_scene* scene, const drt_tile* tile, float wavelength,
                          float eps_r, float* field, float* power, float* saved,
                          void* workspace, size_t workspace_bytes, void* stream) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_saved(scene, saved, nullptr)) != DRT_OK) return st;
  return field_impl(scene, tile, wavelength, eps_r, field, power, saved, workspace,
                    workspace_bytes, stream);
}

// The 3D scene's counts and options in a drt_scene, for the shared decomposition.
drt_status check_scene3(const drt3_scene* sc, drt_scene* flat) {
  if (!sc) return fail(DRT_ERR_INVALID_ARG, "scene is NULL");
  if (sc->n_tris < 1 || sc->n_tris > DRT_MAX_WALLS)
    return fail(sc->n_tris > DRT_MAX_WALLS ? DRT_ERR_UNSUPPORTED : DRT_ERR_INVALID_ARG,
                "n_tris = %d outside 1..%d", sc->n_tris, DRT_MAX_WALLS);
  if (sc->n_rx < 0) return fail(DRT_ERR_INVALID_ARG, "n_rx = %d < 0", sc->n_rx);
  if (sc->max_order < 0 || sc->max_order > DRT_MAX_ORDER)
    return fail(sc->max_order > DRT_MAX_ORDER ? DRT_ERR_UNSUPPORTED : DRT_ERR_INVALID_ARG,
                "max_order = %d outside 0..%d", sc->max_order, DRT_MAX_ORDER);
  if (!(sc->alpha >= 0.f) || !std::isfinite(sc->alpha))
    return fail(DRT_ERR_INVALID_ARG, "alpha must be finite and >= 0");
  if (!std::isfinite(sc->refl_coef)) return fail(DRT_ERR_INVALID_ARG, "refl_coef must be finite");
  if (sc->smoothing < 0 || sc->smoothing > 2)
    return fail(DRT_ERR_INVALID_ARG, "unknown smoothing %d", sc->smoothing);
  if (!sc->tris || !aligned(sc->tris, 4))
    return fail(DRT_ERR_INVALID_ARG, "tris must be a 4-byte aligned device pointer");
  if (!sc->tx || !aligned(sc->tx, 4)) return fail(DRT_ERR_INVALID_ARG, "tx pointer");
  if (sc->n_rx > 0 && (!sc->rx || !aligned(sc->rx, 4)))
    return fail(DRT_ERR_INVALID_ARG, "rx must be a 4-byte aligned device pointer");
  *flat = drt_scene{};
  flat->n_walls = sc->n_tris;
  flat->n_rx = sc->n_rx;
  flat->max_order = sc->max_order;
  flat->alpha = sc->alpha;
  flat->smoothing = sc->smoothing;
  flat->refl_coef = sc->refl_coef;
  return DRT_OK;
}

drt_status drt3_forward_workspace_size(const drt3_scene* scene, const drt_tile* tile,
                                       size_t* bytes) {
  drt_scene flat;
  drt_status st = check_scene3(scene, &flat);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!bytes) return fail(DRT_ERR_INVALID_ARG, "bytes is NULL");
  Decomp d;
  if ((st = decompose(&flat, tile, FWD3, &d)) != DRT_OK) return st;
  *bytes = (size_t)d.n_chunks * (size_t)scene->n_rx * sizeof(float);
  return DRT_OK;
}

drt_status drt3_forward(const drt3_scene* scene, const drt_tile* tile, float* power,
                        void* workspace, size_t workspace_bytes, void* stream) {
  drt_scene flat;
  drt_status st = check_scene3(scene, &flat);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (scene->n_rx > 0 && !power) return fail(DRT_ERR_INVALID_ARG, "power is NULL");
  if (scene->n_rx == 0) return DRT_OK;
  Decomp d;
  if ((st = decompose(&flat, tile, FWD3, &d)) != DRT_OK) return st;
  const size_t need = (size_t)d.n_chunks * (size_t)scene->n_rx * sizeof(float);
  if (!workspace || workspace_bytes < need)
    return fail(DRT_ERR_WORKSPACE, "3D forward needs %zu workspace bytes, got %zu", need,
                workspace_bytes);
  Fwd3Args a{};
  a.tris = scene->tris;
  a.W = scene->n_tris;
  a.rx = scene->rx;
  a.R = scene->n_rx;
  a.tx = scene->tx;
  a.K = scene->max_order;
  a.alpha = scene->alpha;
  gamma_powers(scene->refl_coef, a.gk);
  a.n_cand = d.n_cand;
  a.chunk = d.chunk;
  a.n_chunks = d.n_chunks;
  a.n_tiles = d.n_tiles;
  a.n_units = d.n_units;
  a.partial = static_cast<float*>(workspace);
  a.power = power;
  // work stealing, the counter in power's first 8 bytes (as drt_forward)
  a.unit_counter = (scene->n_rx >= 2 && aligned(power, 8))
                       ? reinterpret_cast<unsigned long long*>(power)
                       : nullptr;
  cudaError_t e = launch_forward3(a, scene->smoothing, d.ctas, d.threads,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "3D forward launch");
  return DRT_OK;
}

drt_status drt3_vjp_workspace_size(const drt3_scene* scene, const drt_tile* tile, size_t* bytes) {
  drt_scene flat;
  drt_status st = check_scene3(scene, &flat);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!bytes) return fail(DRT_ERR_INVALID_ARG, "bytes is NULL");
  // enough for either variant (with or without the triangle gradient)
  Decomp d, dt;
  if ((st = decompose(&flat, tile, VJP3, &d)) != DRT_OK) return st;
  if ((st = decompose(&flat, tile, VJP3_TX, &dt)) != DRT_OK) return st;
  *bytes = std::max(vjp3_workspace_floats(scene->n_tris, d.ctas, d.n_units, true),
                    vjp3_workspace_floats(scene->n_tris, dt.ctas, dt.n_units, false)) *
           sizeof(float);
  return DRT_OK;
}

drt_status drt3_vjp(const drt3_scene* scene, const drt_tile* tile, const float* grad_power,
                    float* grad_tx, float* grad_tris, void* workspace, size_t workspace_bytes,
                    void* stream) {
  drt_scene flat;
  drt_status st = check_scene3(scene, &flat);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!grad_tx || (scene->n_rx > 0 && !grad_power))
    return fail(DRT_ERR_INVALID_ARG, "NULL pointer");
  if (grad_tris && !aligned(grad_tris, 4))
    return fail(DRT_ERR_INVALID_ARG, "grad_tris must be 4-byte aligned");
  Decomp d;
  if ((st = decompose(&flat, tile, grad_tris ? VJP3 : VJP3_TX, &d)) != DRT_OK) return st;
  const size_t need =
      vjp3_workspace_floats(scene->n_tris, d.ctas, d.n_units, grad_tris != nullptr) *
      sizeof(float);
  if (!workspace || workspace_bytes < need || !aligned(workspace, 4))
    return fail(DRT_ERR_WORKSPACE, "3D vjp needs %zu workspace bytes, got %zu", need,
                workspace_bytes);
  Vjp3Args a{};
  a.tris = scene->tris;
  a.W = scene->n_tris;
  a.rx = scene->rx;
  a.R = scene->n_rx;
  a.tx = scene->tx;
  a.K = scene->max_order;
  a.alpha = scene->alpha;
  gamma_powers(scene->refl_coef, a.gk);
  a.n_cand = d.n_cand;
  a.chunk = d.chunk;
  a.n_chunks = d.n_chunks;
  a.n_tiles = d.n_tiles;
  a.n_units = d.n_units;
  a.grad_power = grad_power;
  float* ws = static_cast<float*>(workspace);
  // the counter on the first 8-byte boundary of the 4 leading floats
  a.unit_counter = reinterpret_cast<unsigned long long*>(aligned(ws, 8) ? ws : ws + 1);
  a.unit_tx = ws + 4;
  a.cta_tris = grad_tris ? a.unit_tx + (size_t)d.n_units * 3 : nullptr;
  a.grad_tx = grad_tx;
  a.grad_tris = grad_tris;
  cudaError_t e = launch_vjp3(a, scene->smoothing, d.ctas, d.threads,
                              static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "3D vjp launch");
  return DRT_OK;
}

drt_status drt3_vjp_tx_workspace_size(const drt3_scene* scene, const drt_tile* tile,
                                      size_t* bytes) {
  drt_scene flat;
  drt_status st = check_scene3(scene, &flat);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!bytes) return fail(DRT_ERR_INVALID_ARG, "bytes is NULL");
  Decomp d;
  if ((st = decompose(&flat, tile, VJP3_TX, &d)) != DRT_OK) return st;
  *bytes = vjp3_workspace_floats(scene->n_tris, d.ctas, d.n_units, false) * sizeof(float);
  return DRT_OK;
}

drt_status drt3_vjp_tx(const drt3_scene* scene, const drt_tile* tile, const float* grad_power,
                       float* grad_tx, void* workspace, size_t workspace_bytes, void* stream) {
  return drt3_vjp(scene, tile, grad_power, grad_tx, nullptr, workspace, workspace_bytes, stream);
}

drt_status drt_tune_forward(const drt_scene* scene, const drt_tile* cands, int32_t n_cand,
                            int32_t reps, float* power, void* workspace, size_t workspace_bytes,
                            drt_tile* best, float* ms_out, void* stream) {
  drt_status st = check_scene(scene, DRT_MAX_WALLS_STREAMED);
  if (st != DRT_OK) return st;
  if (!cands || n_cand < 1 || !best || !power)
    return fail(DRT_ERR_INVALID_ARG, "cands, n_cand >= 1, best and power are required");
  if (reps < 1) return fail(DRT_ERR_INVALID_ARG, "reps = %d < 1", reps);
  if (scene->n_rx < 1) return fail(DRT_ERR_INVALID_ARG, "n_rx must be >= 1 to time the forward");
  for (int i = 0; i < n_cand; ++i)
    if ((st = check_tile(&cands[i])) != DRT_OK) return st;
  cudaStream_t strm = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  if (e != cudaSuccess) {
    if (ev[0]) cudaEventDestroy(ev[0]);
    return cuda_fail(e, "cudaEventCreate");
  }
  float best_ms = INFINITY;
  int bi = -1;
  st = DRT_OK;
  for (int i = 0; i < n_cand && st == DRT_OK; ++i) {
    float ms = INFINITY;
    size_t need = 0;
    if ((st = drt_forward_workspace_size(scene, &cands[i], &need)) != DRT_OK) break;
    if (workspace && need <= workspace_bytes) {
      if ((st = drt_forward(scene, &cands[i], power, workspace, workspace_bytes, stream)) != DRT_OK)
        break;
      if ((e = cudaEventRecord(ev[0], strm)) != cudaSuccess) {
        st = cuda_fail(e, "cudaEventRecord");
        break;
      }
      for (int r = 0; r < reps && st == DRT_OK; ++r)
        st = drt_forward(scene, &cands[i], power, workspace, workspace_bytes, stream);
      if (st != DRT_OK) break;
      if ((e = cudaEventRecord(ev[1], strm)) != cudaSuccess ||
          (e = cudaEventSynchronize(ev[1])) != cudaSuccess ||
          (e = cudaEventElapsedTime(&ms, ev[0], ev[1])) != cudaSuccess) {
        st = cuda_fail(e, "timing events");
        break;
      }
      ms /= (float)reps;
      if (ms < best_ms) {
        best_ms = ms;
        bi = i;
      }
    }
    if (ms_out) ms_out[i] = ms;
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (st != DRT_OK) return st;
  if (bi < 0) return fail(DRT_ERR_WORKSPACE, "no candidate tile fits %zu workspace bytes",
                          workspace_bytes);
  *best = cands[bi];
  return DRT_OK;
}

drt_status drt_loss(const float* power, int32_t n_rx, float* loss, int32_t* argmin,
                    void* stream) {
  if (!power || !loss || !argmin) return fail(DRT_ERR_INVALID_ARG, "NULL pointer");
  if (n_rx < 1) return fail(DRT_ERR_INVALID_ARG, "n_rx = %d < 1", n_rx);
  cudaError_t e = launch_loss(power, n_rx, loss, argmin, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "loss launch");
  return DRT_OK;
}

drt_status drt_loss_backward(const int32_t* argmin, const float* grad_loss, int32_t n_rx,
                             float* grad_power, void* stream) {
  if (!argmin || !grad_power) return fail(DRT_ERR_INVALID_ARG, "NULL pointer");
  if (n_rx < 1) return fail(DRT_ERR_INVALID_ARG, "n_rx = %d < 1", n_rx);
  cudaError_t e = launch_loss_backward(argmin, grad_loss, n_rx, grad_power,
                                       static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "loss backward launch");
  return DRT_OK;
}

drt_status drt_vjp_workspace_size(const drt_scene* scene, const drt_tile* tile, size_t* bytes) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!bytes) return fail(DRT_ERR_INVALID_ARG, "bytes is NULL");
  // enough for either mapping (with or without the wall gradient)
  Decomp d, dt;
  if ((st = decompose(scene, tile, VJP, &d)) != DRT_OK) return st;
  if ((st = decompose(scene, tile, VJP_TX, &dt)) != DRT_OK) return st;
  *bytes = std::max(vjp_workspace(scene, d), vjp_workspace(scene, dt));
  return DRT_OK;
}

namespace {
drt_status vjp_impl(const drt_scene* scene, const drt_tile* tile, const float* grad_power,
                    const float* saved, float* grad_tx, float* grad_walls, void* workspace,
                    size_t workspace_bytes, void* stream) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!grad_tx || (scene->n_rx > 0 && !grad_power))
    return fail(DRT_ERR_INVALID_ARG, "NULL pointer");
  if (grad_walls && !aligned(grad_walls, 16))
    return fail(DRT_ERR_INVALID_ARG, "grad_walls must be 16-byte aligned");
  Decomp d;
  if ((st = decompose(scene, tile, grad_walls ? VJP : VJP_TX, &d)) != DRT_OK) return st;
  const size_t need = vjp_workspace(scene, d);
  if (!workspace || workspace_bytes < need || !aligned(workspace, 16))
    return fail(DRT_ERR_WORKSPACE, "vjp needs %zu aligned workspace bytes, got %zu", need,
                workspace_bytes);
  VjpArgs a{};
  a.rx_index = nullptr;
  a.grad_loss = nullptr;
  a.walls = reinterpret_cast<const float4*>(scene->walls);
  a.W = scene->n_walls;
  a.rx = scene->rx;
  a.R = scene->n_rx;
  a.tx = scene->tx;
  a.K = scene->max_order;
  a.alpha = scene->alpha;
  gamma_powers(scene->refl_coef, a.gk);
  a.n_cand = d.n_cand;
  a.chunk = d.chunk;
  a.n_chunks = d.n_chunks;
  a.n_tiles = d.n_tiles;
  a.n_units = d.n_units;
  a.pairs = d.pairs;
  a.grad_power = grad_power;
  float* ws = static_cast<float*>(workspace);
  a.cta_walls = ws + 4;
  a.warp_tx = a.cta_walls + (size_t)d.ctas * scene->n_walls * VJP_SLOTS;
  a.unit_counter = static_cast<unsigned long long*>(workspace);
  a.unit_tx = a.warp_tx + (size_t)d.ctas * (d.threads / 32) * 2;
  a.grad_tx = grad_tx;
  a.grad_walls = grad_walls;
  a.saved = saved;
  cudaError_t e = launch_vjp(a, scene->smoothing, d.ctas, d.threads,
                             static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "vjp launch");
  return DRT_OK;
}
}  // namespace

drt_status drt_vjp(const drt_scene* scene, const drt_tile* tile, const float* grad_power,
                   float* grad_tx, float* grad_walls, void* workspace, size_t workspace_bytes,
                   void* stream) {
  return vjp_impl(scene, tile, grad_power, nullptr, grad_tx, grad_walls, workspace,
                  workspace_bytes, stream);
}

drt_status drt_vjp_saved(const drt_scene* scene, const drt_tile* tile, const float* grad_power,
                         const float* saved, float* grad_tx, float* grad_walls, void* workspace,
                         size_t workspace_bytes, void* stream) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_saved(scene, saved, nullptr)) != DRT_OK) return st;
  return vjp_impl(scene, tile, grad_power, saved, grad_tx, grad_walls, workspace,
                  workspace_bytes, stream);
}

drt_status drt_field_vjp_workspace_size(const drt_scene* scene, const drt_tile* tile,
                                        size_t* bytes) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!bytes) return fail(DRT_ERR_INVALID_ARG, "bytes is NULL");
  Decomp d;
  if ((st = decompose(scene, tile, FIELD_VJP, &d)) != DRT_OK) return st;
  *bytes = vjp_workspace(scene, d);
  return DRT_OK;
}

namespace {
drt_status field_vjp_impl(const drt_scene* scene, const drt_tile* tile, float wavelength,
                          float eps_r, const float* field, const float* grad_power,
                          const float* saved, float* grad_tx, float* grad_walls,
                          void* workspace, size_t workspace_bytes, void* stream) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!(wavelength > 0.f) || !std::isfinite(wavelength))
    return fail(DRT_ERR_INVALID_ARG, "wavelength must be finite and > 0");
  if (!(eps_r == 0.f || eps_r >= 1.f) || !std::isfinite(eps_r))
    return fail(DRT_ERR_INVALID_ARG, "eps_r must be 0 (constant coefficient) or finite and >= 1");
  if (eps_r == 0.f && !(scene->refl_coef >= 0.f))
    return fail(DRT_ERR_INVALID_ARG, "refl_coef must be >= 0 for the constant coefficient");
  if (!grad_tx || (scene->n_rx > 0 && (!grad_power || !field)))
    return fail(DRT_ERR_INVALID_ARG, "NULL pointer");
  if (field && !aligned(field, 8)) return fail(DRT_ERR_INVALID_ARG, "field must be 8-byte aligned");
  if (grad_walls && !aligned(grad_walls, 16))
    return fail(DRT_ERR_INVALID_ARG, "grad_walls must be 16-byte aligned");
  Decomp d;
  if ((st = decompose(scene, tile, FIELD_VJP, &d)) != DRT_OK) return st;
  const size_t need = vjp_workspace(scene, d);
  if (!workspace || workspace_bytes < need || !aligned(workspace, 16))
    return fail(DRT_ERR_WORKSPACE, "field vjp needs %zu aligned workspace bytes, got %zu", need,
                workspace_bytes);
  VjpArgs a{};
  a.rx_index = nullptr;
  a.grad_loss = nullptr;
  a.walls = reinterpret_cast<const float4*>(scene->walls);
  a.W = scene->n_walls;
  a.rx = scene->rx;
  a.R = scene->n_rx;
  a.tx = scene->tx;
  a.K = scene->max_order;
  a.alpha = scene->alpha;
  gamma_powers(scene->refl_coef, a.gk);
  a.n_cand = d.n_cand;
  a.chunk = d.chunk;
  a.n_chunks = d.n_chunks;
  a.n_tiles = d.n_tiles;
  a.n_units = d.n_units;
  a.grad_power = grad_power;
  float* ws = static_cast<float*>(workspace);
  a.cta_walls = ws + 4;
  a.warp_tx = a.cta_walls + (size_t)d.ctas * scene->n_walls * VJP_SLOTS;
  a.unit_counter = static_cast<unsigned long long*>(workspace);
  a.unit_tx = a.warp_tx + (size_t)d.ctas * (d.threads / 32) * 2;
  a.grad_tx = grad_tx;
  a.grad_walls = grad_walls;
  a.field = reinterpret_cast<const float2*>(field);
  const double inv = 1.0 / (double)wavelength;
  a.inv_lambda_hi = (float)inv;
  a.inv_lambda_lo = (float)(inv - (double)a.inv_lambda_hi);
  a.k2pi = (float)(2.0 * M_PI * inv);
  // as in drt_field: eps_r = 1 is the zero coefficient
  a.refl_amp = eps_r == 0.f ? -(float)std::sqrt((double)scene->refl_coef) : 0.f;
  a.eps_r = eps_r == 1.f ? 0.f : eps_r;
  a.saved = saved;
  cudaError_t e = launch_field_vjp(a, scene->smoothing, d.ctas, d.threads,
                                   static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "field vjp launch");
  return DRT_OK;
}
}  // namespace

drt_status drt_field_vjp(const drt_scene* scene, const drt_tile* tile, float wavelength,
                         float eps_r, const float* field, const float* grad_power,
                         float* grad_tx, float* grad_walls, void* workspace,
                         size_t workspace_bytes, void* stream) {
  return field_vjp_impl(scene, tile, wavelength, eps_r, field, grad_power, nullptr, grad_tx,
                        grad_walls, workspace, workspace_bytes, stream);
}

drt_status drt_field_vjp_saved(const drt_scene* scene, const drt_tile* tile, float wavelength,
                               float eps_r, const float* field, const float* grad_power,
                               const float* saved, float* grad_tx, float* grad_walls,
                               void* workspace, size_t workspace_bytes, void* stream) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_saved(scene, saved, nullptr)) != DRT_OK) return st;
  return field_vjp_impl(scene, tile, wavelength, eps_r, field, grad_power, saved, grad_tx,
                        grad_walls, workspace, workspace_bytes, stream);
}

drt_status drt_min_loss_vjp(const drt_scene* scene, const drt_tile* tile, const int32_t* argmin,
                            const float* grad_loss, float* grad_tx, float* grad_walls,
                            void* workspace, size_t workspace_bytes, void* stream) {
  drt_status st = check_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!argmin || !grad_tx) return fail(DRT_ERR_INVALID_ARG, "NULL pointer");
  if (scene->n_rx < 1) return fail(DRT_ERR_INVALID_ARG, "n_rx = %d < 1", scene->n_rx);
  if (grad_walls && !aligned(grad_walls, 16))
    return fail(DRT_ERR_INVALID_ARG, "grad_walls must be 16-byte aligned");
  Decomp d, drx;
  if ((st = decompose(scene, tile, VJP, &d)) != DRT_OK) return st;
  if ((st = decompose(scene, tile, VJP_RX, &drx)) != DRT_OK) return st;
  const size_t need = vjp_workspace(scene, d);
  if (!workspace || workspace_bytes < need || !aligned(workspace, 16))
    return fail(DRT_ERR_WORKSPACE, "min-loss vjp needs %zu aligned workspace bytes, got %zu",
                need, workspace_bytes);
  VjpArgs a{};
  a.walls = reinterpret_cast<const float4*>(scene->walls);
  a.W = scene->n_walls;
  a.rx = scene->rx;
  a.R = scene->n_rx;
  a.tx = scene->tx;
  a.K = scene->max_order;
  a.alpha = scene->alpha;
  gamma_powers(scene->refl_coef, a.gk);
  a.n_cand = d.n_cand;
  a.chunk = 32;
  a.n_chunks = (d.n_cand + 31) / 32;
  a.n_tiles = 1;
  a.n_units = a.n_chunks;
  a.grad_power = nullptr;
  a.rx_index = argmin;
  a.grad_loss = grad_loss;
  float* ws = static_cast<float*>(workspace);
  a.cta_walls = ws;
  a.warp_tx = ws + (size_t)d.ctas * scene->n_walls * VJP_SLOTS;
  a.grad_tx = grad_tx;
  a.grad_walls = grad_walls;
  // one receiver: only ceil(N_K / 32) warps have work, so launch no more CTAs than
  // that (fewer per-CTA tables for the final reduction to add up)
  // (and no more than the receiver-tile decomposition the workspace is sized for)
  const long long busy = (a.n_units + d.threads / 32 - 1) / (d.threads / 32);
  const int ctas = (int)std::max(
      1LL, std::min({(long long)d.ctas, (long long)drx.ctas, busy}));
  cudaError_t e = launch_vjp(a, scene->smoothing, ctas, d.threads,
                             static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "min-loss vjp launch");
  return DRT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ end to end
// Layout of drt_objective_host's device workspace: the copied inputs, the
// intermediate power, loss and argmin, the gradients, then the forward's and
// the adjoint's own workspaces; every section starts on a 256-byte boundary.
namespace {
struct HostObjLayout {
  size_t walls, tx, rx, power, loss, argmin, gtx, gw, fws, vws, total;
  size_t fws_bytes, vws_bytes;
};

size_t round256(size_t n) { return (n + 255) & ~(size_t)255; }

drt_status host_obj_layout(const drt_scene* sc, const drt_tile* tile, HostObjLayout* L) {
  Decomp df, dv;
  drt_status st = decompose(sc, tile, FWD, &df);
  if (st != DRT_OK) return st;
  if ((st = decompose(sc, tile, VJP, &dv)) != DRT_OK) return st;
  const size_t W = (size_t)sc->n_walls, R = (size_t)sc->n_rx;
  L->fws_bytes = forward_workspace(sc, df);
  L->vws_bytes = vjp_workspace(sc, dv);
  size_t off = 0;
  auto take = [&](size_t n) { const size_t o = off; off += round256(n); return o; };
  L->walls = take(W * 4 * sizeof(float));
  L->tx = take(2 * sizeof(float));
  L->rx = take(R * 2 * sizeof(float));
  L->power = take(R * sizeof(float));
  L->loss = take(sizeof(float));
  L->argmin = take(sizeof(int32_t));
  L->gtx = take(2 * sizeof(float));
  L->gw = take(W * 4 * sizeof(float));
  L->fws = take(L->fws_bytes);
  L->vws = take(L->vws_bytes);
  L->total = off;
  return DRT_OK;
}

// The scene with its arrays checked as host arrays (drt_objective_host): the
// same rules as check_scene except alignment, which only device arrays need.
drt_status check_host_scene(const drt_scene* sc) {
  if (!sc) return fail(DRT_ERR_INVALID_ARG, "scene is NULL");
  if (!sc->walls || !sc->tx || !sc->rx)
    return fail(DRT_ERR_INVALID_ARG, "walls, tx and rx host pointers are required");
  if (sc->n_rx < 1) return fail(DRT_ERR_INVALID_ARG, "n_rx = %d < 1", sc->n_rx);
  drt_scene probe = *sc;
  // any 256-aligned non-null value passes the pointer checks of check_scene
  probe.walls = probe.tx = probe.rx = reinterpret_cast<const float*>(256);
  return check_scene(&probe);
}
}  // namespace

extern "C" {

drt_status drt_objective_host_workspace_size(const drt_scene* scene, const drt_tile* tile,
                                             size_t* bytes) {
  drt_status st = check_host_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!bytes) return fail(DRT_ERR_INVALID_ARG, "bytes is NULL");
  HostObjLayout L;
  if ((st = host_obj_layout(scene, tile, &L)) != DRT_OK) return st;
  *bytes = L.total;
  return DRT_OK;
}

drt_status drt_objective_host(const drt_scene* scene, const drt_tile* tile, float* loss,
                              int32_t* argmin, float* power, float* grad_tx, float* grad_walls,
                              void* workspace, size_t workspace_bytes, void* stream) {
  drt_status st = check_host_scene(scene);
  if (st != DRT_OK) return st;
  if ((st = check_tile(tile)) != DRT_OK) return st;
  if (!loss || !grad_tx) return fail(DRT_ERR_INVALID_ARG, "loss and grad_tx are required");
  HostObjLayout L;
  if ((st = host_obj_layout(scene, tile, &L)) != DRT_OK) return st;
  if (!workspace || workspace_bytes < L.total || !aligned(workspace, 256))
    return fail(DRT_ERR_WORKSPACE, "objective needs %zu 256-byte aligned workspace bytes, got %zu",
                L.total, workspace_bytes);
  char* ws = static_cast<char*>(workspace);
  cudaStream_t strm = static_cast<cudaStream_t>(stream);
  const size_t W = (size_t)scene->n_walls, R = (size_t)scene->n_rx;
  drt_scene dev = *scene;
  dev.walls = reinterpret_cast<const float*>(ws + L.walls);
  dev.tx = reinterpret_cast<const float*>(ws + L.tx);
  dev.rx = reinterpret_cast<const float*>(ws + L.rx);
  float* d_power = reinterpret_cast<float*>(ws + L.power);
  float* d_loss = reinterpret_cast<float*>(ws + L.loss);
  int32_t* d_arg = reinterpret_cast<int32_t*>(ws + L.argmin);
  float* d_gtx = reinterpret_cast<float*>(ws + L.gtx);
  float* d_gw = grad_walls ? reinterpret_cast<float*>(ws + L.gw) : nullptr;
  // inputs: one copy per array
  cudaError_t e = cudaMemcpyAsync(const_cast<float*>(dev.walls), scene->walls, W * 16,
                                  cudaMemcpyHostToDevice, strm);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<float*>(dev.tx), scene->tx, 8, cudaMemcpyHostToDevice, strm);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<float*>(dev.rx), scene->rx, R * 8, cudaMemcpyHostToDevice,
                        strm);
  if (e != cudaSuccess) return cuda_fail(e, "objective input copies");
  // power, loss = -min power (lowest-index argmin), gradient of the loss
  if ((st = drt_forward(&dev, tile, d_power, ws + L.fws, L.fws_bytes, stream)) != DRT_OK)
    return st;
  if ((st = drt_loss(d_power, scene->n_rx, d_loss, d_arg, stream)) != DRT_OK) return st;
  if ((st = drt_min_loss_vjp(&dev, tile, d_arg, nullptr, d_gtx, d_gw, ws + L.vws, L.vws_bytes,
                             stream)) != DRT_OK)
    return st;
  // outputs: one copy per array
  e = cudaMemcpyAsync(loss, d_loss, 4, cudaMemcpyDeviceToHost, strm);
  if (e == cudaSuccess && argmin) e = cudaMemcpyAsync(argmin, d_arg, 4, cudaMemcpyDeviceToHost, strm);
  if (e == cudaSuccess && power)
    e = cudaMemcpyAsync(power, d_power, R * 4, cudaMemcpyDeviceToHost, strm);
  if (e == cudaSuccess) e = cudaMemcpyAsync(grad_tx, d_gtx, 8, cudaMemcpyDeviceToHost, strm);
  if (e == cudaSuccess && grad_walls)
    e = cudaMemcpyAsync(grad_walls, d_gw, W * 16, cudaMemcpyDeviceToHost, strm);
  if (e != cudaSuccess) return cuda_fail(e, "objective output copies");
  return DRT_OK;
}

}  // extern "C"
