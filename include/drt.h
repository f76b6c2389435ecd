/*
 * drt.h - C ABI of the GB300 (sm_103a) smoothed, differentiable 2D
 * image-method ray tracer.
 *
 * The operations follow the paper's problem statement (Sec. III): a scene of
 * walls (2D segments, Sec. VI), one transmitter (TX) and a set of receivers
 * (RX); every path candidate up to K reflections (Sec. V) is traced by the
 * image method (Sec. V-B), its validity and obstruction are smoothed by
 * s(x; alpha) (Sec. IV, Eqs. 1-6; Sec. V-A), and the per-path powers are
 * summed per receiver (Eq. 7).  The objective is the minimum received power
 * (Eq. 8) and the loss its negative (Sec. III).
 *
 * Conventions shared by every entry point:
 *  - Every array argument is a CUDA DEVICE pointer owned by the caller,
 *    unless the comment says "host".  FP32 in, FP32 out, C-contiguous.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Work is only enqueued: no call synchronises the
 *    stream, and no call allocates device memory.
 *  - Arguments are validated on the host before anything is enqueued;
 *    a rejected call returns DRT_ERR_INVALID_ARG (or DRT_ERR_UNSUPPORTED /
 *    DRT_ERR_WORKSPACE) and leaves every output untouched.
 *  - Outputs are overwritten, never accumulated into.
 *  - A failed CUDA launch returns DRT_ERR_CUDA; drt_last_error() gives the
 *    message (per host thread).  Device-side faults surface, as usual in
 *    CUDA, at the caller's next synchronisation.
 *  - No exception crosses the ABI.
 */
#ifndef DRT_H
#define DRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DRT_MAX_ORDER 3    /* largest supported K */
#define DRT_MAX_WALLS 1024 /* largest supported W per scene */

typedef enum {
  DRT_OK = 0,
  DRT_ERR_INVALID_ARG = 1,
  DRT_ERR_UNSUPPORTED = 2,
  DRT_ERR_CUDA = 3,
  DRT_ERR_TIMEOUT = 4,
  DRT_ERR_WORKSPACE = 5
} drt_status;

/* Smoothing function s (Sec. IV-B), scaled as s(alpha x) (Eq. 3). */
typedef enum {
  DRT_SMOOTH_SIGMOID = 0,      /* Eq. 4: 1 / (1 + exp(-alpha x))          */
  DRT_SMOOTH_HARD_SIGMOID = 1, /* Eqs. 5-6: relu6(alpha x + 3) / 6          */
  DRT_SMOOTH_STEP = 2          /* Eq. 1: 1 if x > 0 else 0 (alpha ignored)  */
} drt_smoothing;

/* One scene (Sec. III).  Pointers are device pointers. */
typedef struct {
  const float* walls;  /* [n_walls][4]: x0, y0, x1, y1 of each segment; 16-byte aligned */
  int32_t n_walls;     /* W, 1..DRT_MAX_WALLS */
  const float* rx;     /* [n_rx][2] receiver positions; 8-byte aligned */
  int32_t n_rx;        /* R >= 0 */
  const float* tx;     /* [2] transmitter position */
  int32_t max_order;   /* K, 0..DRT_MAX_ORDER: paths with 0..K reflections */
  float alpha;         /* smoothing sharpness, >= 0, finite */
  int32_t smoothing;   /* drt_smoothing */
  float refl_coef;     /* Gamma: power factor per reflection, finite (0.5 by convention) */
} drt_scene;

/* Work decomposition of the path kernels.  Zero fields take the defaults. */
typedef struct {
  int32_t warps_per_cta;   /* 1..8 (default 8) */
  int32_t cands_per_unit;  /* path candidates one warp evaluates per work unit (default 64) */
  int32_t ctas_per_sm;     /* resident CTAs per SM for the persistent grid (default: occupancy) */
  int32_t flags;           /* DRT_TILE_* bits */
} drt_tile;

/* Skip the obstruction loop of a candidate when the validity of the path is
   exactly 0 for all 32 receivers of the warp (exact for hard sigmoid and step,
   where s saturates at 0; a no-op for the sigmoid).  Off by default. */
#define DRT_TILE_CULL_INVALID 1

/* Human-readable name of a status code (static string). */
const char* drt_status_string(drt_status status);

/* Message of the last failed call on this host thread ("" if none). */
const char* drt_last_error(void);

/* Number of path candidates N_K = 1 + sum_{k=1..K} W (W-1)^(k-1): every wall
   sequence of length 0..K with no wall twice in a row (Sec. V, candidate list
   from the visibility matrix).  `count` is a host pointer. */
drt_status drt_num_candidates(int32_t n_walls, int32_t max_order, int64_t* count);

/* Bytes of device workspace drt_forward needs for this scene and tile (host out). */
drt_status drt_forward_workspace_size(const drt_scene* scene, const drt_tile* tile, size_t* bytes);

/* Received power per receiver (Eq. 7, incoherent scalar reading):
     power[r] = sum over candidates of Gamma^k * prod_j V_j * prod_j vis_j / L^2
   with V_j the smoothed validity of reflection j (on-segment and same-side
   tests, Sec. V-A), vis_j the smoothed visibility of leg j (every wall except
   the ones the leg's end points lie on), L the path length.
   scene: host pointer to the descriptor; power: [n_rx], overwritten;
   workspace: device scratch of at least drt_forward_workspace_size bytes
   (contents undefined on return); tile: host pointer or NULL for defaults. */
drt_status drt_forward(const drt_scene* scene, const drt_tile* tile, float* power,
                       void* workspace, size_t workspace_bytes, void* stream);

/* Loss of the antenna-placement problem (Eq. 8 and Sec. III):
     loss[0] = -min_r power[r],  argmin[0] = the smallest r attaining the min.
   power: [n_rx] with n_rx >= 1; loss: [1]; argmin: [1] (int32). */
drt_status drt_loss(const float* power, int32_t n_rx, float* loss, int32_t* argmin,
                    void* stream);

/* Gradient of the loss w.r.t. power (the subgradient of -min at its argmin):
     grad_power[r] = -(grad_loss ? grad_loss[0] : 1) if r == argmin[0] else 0.
   argmin: [1] from drt_loss; grad_loss: [1] or NULL; grad_power: [n_rx]. */
drt_status drt_loss_backward(const int32_t* argmin, const float* grad_loss, int32_t n_rx,
                             float* grad_power, void* stream);

/* Bytes of device workspace drt_vjp needs (host out). */
drt_status drt_vjp_workspace_size(const drt_scene* scene, const drt_tile* tile, size_t* bytes);

/* Vector-Jacobian product of drt_forward (reverse-mode derivative, Sec. III:
   gradient of the loss w.r.t. the scene parameters), by a hand-written adjoint
   that recomputes the path geometry instead of storing it:
     grad_tx[i]       = sum_r grad_power[r] * d power[r] / d tx[i]
     grad_walls[w][c] = sum_r grad_power[r] * d power[r] / d walls[w][c]
   grad_power: [n_rx]; grad_tx: [2], overwritten; grad_walls: [n_walls][4],
   overwritten, or NULL to skip the wall gradient.  Receivers whose 32-wide
   tile has grad_power == 0 everywhere are skipped.  The hard sigmoid's
   derivative is taken as 0 at its kinks (x = +-3/alpha). */
drt_status drt_vjp(const drt_scene* scene, const drt_tile* tile, const float* grad_power,
                   float* grad_tx, float* grad_walls, void* workspace, size_t workspace_bytes,
                   void* stream);

/* Gradient of the min-power loss (Eq. 8, Sec. III) w.r.t. the scene, in one call:
   with loss = -power[argmin[0]],
     grad_tx    = -(grad_loss ? grad_loss[0] : 1) * d power[argmin] / d tx,
     grad_walls = -(grad_loss ? grad_loss[0] : 1) * d power[argmin] / d walls.
   Equal to drt_loss_backward followed by drt_vjp, but the lanes of each warp
   take different path candidates of the one receiver, instead of 32
   receivers of which only one has a non-zero weight.  argmin: [1] device
   int32 from drt_loss (clamped to 0..n_rx-1); grad_loss: [1] or NULL;
   grad_tx: [2]; grad_walls: [n_walls][4] or NULL; workspace: as for drt_vjp
   (drt_vjp_workspace_size bytes). */
drt_status drt_min_loss_vjp(const drt_scene* scene, const drt_tile* tile, const int32_t* argmin,
                            const float* grad_loss, float* grad_tx, float* grad_walls,
                            void* workspace, size_t workspace_bytes, void* stream);

/* Size of the static device scratch array behind drt_forward_noalloc. */
#define DRT_NOALLOC_SCRATCH_BYTES (8u << 20)

/* drt_forward for callers that cannot allocate device memory (the paper has no
   counterpart; this is a deployment convenience).  Plugins and callbacks that
   only receive the buffers they must fill, and applications that fix their
   whole device-memory plan at start-up, cannot provide drt_forward's
   workspace.  This call instead uses a scratch array of
   DRT_NOALLOC_SCRATCH_BYTES compiled into the library's device image, which
   every GPU that loads the library keeps until the process exits, and calls no
   allocator.  Same arguments and result as drt_forward with default tiling
   (scene: host pointer; power: [n_rx] device, overwritten).
   - Limit: one partial sum per (candidate chunk, receiver) must fit, so
     n_rx <= DRT_NOALLOC_SCRATCH_BYTES / 4; larger scenes get
     DRT_ERR_UNSUPPORTED before anything is enqueued.
   - All calls on a device share the array, and it keeps the last call's
     contents (every value a call reads was written by that same call).
     Calls that overlap on the GPU race on it: order them on one stream.
   - The first call on each device looks the array's device address up
     (cudaGetSymbolAddress) with that device current; make that first call
     before any stream capture begins. */
drt_status drt_forward_noalloc(const drt_scene* scene, float* power, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DRT_H */
