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
 *  - The first call on each device caches per-device settings (SM count,
 *    the kernels' shared-memory limits); they are not re-applied after
 *    cudaDeviceReset, so a device must not be used through this library
 *    after it has been reset in the same process.
 */
#ifndef DRT_H
#define DRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DRT_MAX_ORDER 3    /* largest supported K */
#define DRT_MAX_WALLS 1024 /* largest supported W per scene (see DRT_MAX_WALLS_STREAMED) */
/* Largest W of drt_forward (and its workspace query and tuner): above
   DRT_MAX_WALLS it reads the walls' records from a staging area in its workspace
   instead of shared memory.  Every other entry point takes at most DRT_MAX_WALLS.
   Every entry point also needs fewer than 2^31 path candidates (N_K below);
   larger (n_walls, max_order) pairs get DRT_ERR_UNSUPPORTED. */
#define DRT_MAX_WALLS_STREAMED 65536

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
  int32_t cands_per_unit;  /* path candidates one warp evaluates per work unit (default 32
                              for drt_forward and drt_field, 64 for the other kernels) */
  int32_t ctas_per_sm;     /* resident CTAs per SM for the persistent grid (default: occupancy) */
  int32_t flags;           /* DRT_TILE_* bits */
} drt_tile;

/* Skip the obstruction loop of a candidate when the validity of the path is
   exactly 0 for all 32 receivers of the warp (exact for hard sigmoid and step,
   where s saturates at 0; a no-op for the sigmoid).  Off by default. */
#define DRT_TILE_CULL_INVALID 1

/* Hard sigmoid and sigmoid with alpha <= 1e4: the forward holds two receivers
   per lane (tiles of 64 receivers) and runs its obstruction loop in packed FP32
   pairs; the powers are the same, bit for bit.  This flag selects one receiver
   per lane (tiles of 32) instead.  The unit step and alpha > 1e4 always use one
   receiver per lane. */
#define DRT_TILE_SINGLE_RX 2

/* Hard sigmoid forward of drt_forward and of the 2D batched descent, with two
   receivers per lane (the default):
   every 8 walls the warp leaves its obstruction loop once some leg of each of its
   64 paths has a visibility of exactly 0, since no later wall can change a power
   of 0 (exact: the powers are the same, bit for bit).  Ignored by the other kernels
   and smoothings.  Off by default. */
#define DRT_TILE_EXIT_BLOCKED 4

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
   scene: host pointer to the descriptor (n_walls up to DRT_MAX_WALLS_STREAMED);
   power: [n_rx], overwritten; workspace: device scratch of at least
   drt_forward_workspace_size bytes (contents undefined on return; 16-byte aligned
   when n_walls > DRT_MAX_WALLS: it then also holds the walls' records, which the
   kernels read through the caches instead of shared memory); tile: host pointer
   or NULL for defaults.  Warps take their (receiver tile, candidate chunk) units
   from a counter that lives in power's first 8 bytes until the last kernel of the
   call writes the powers (when n_rx >= 2 and power is 8-byte aligned; otherwise
   the split is static); the powers do not depend on the split. */
drt_status drt_forward(const drt_scene* scene, const drt_tile* tile, float* power,
                       void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------
   Iterative path finder with the smoothed convergence check (Sec. V-B,
   "Continuous Path Finding": the path finders check convergence with the
   Min-Path-Tracing cost, which is zero on a valid path, the comparison with
   zero smoothed by s).  For every candidate (w_1..w_k) the reflection points
   X_j = A_j + tau_j u_j on the walls' lines are found by Min-Path-Tracing
   steps instead of the image method:
     residuals  r_j = h_j - R_j h_{j-1}, h_j the unit direction of leg j, R_j the
                mirror of wall j (zero iff the reflection law holds at X_j);
     cost       C = sum_j |r_j|^2;
     start      tau_j = |B_j - A_j| / 2 (the walls' midpoints);
     each step  a Gauss-Newton step (J^T J + 1e-6 diag) delta = -J^T r, every
                delta_j clamped to [-len_j, len_j], then the largest fraction
                2^-m (m < 12) of delta that lowers C by 1e-4 of its slope (up to
                8 units of FP32 rounding of C), or no step;
     validity   prod_j s(tau_j) s(len_j - tau_j) * kappa with the convergence
                check kappa = s(check_eps - C); the same-side test of drt_forward
                is not applied (a converged reflection has its neighbours on one
                side);
   obstruction, Gamma^k and 1 / L^2 as in drt_forward.  A path with a leg of
   zero length at any step, or shorter than 1e-3 (scene units) at the final
   points, contributes 0.  n_iter: 0..DRT_MPT_MAX_ITER steps.
   check_eps: finite, in the units of C (which is dimensionless, 0 to 4 per
   reflection).  With the hard sigmoid, check_eps >= 3 / alpha makes kappa = 1 on
   converged paths.  One receiver per lane; tile as for drt_forward (the flags
   are ignored). */
#define DRT_MPT_MAX_ITER 64
drt_status drt_forward_mpt_workspace_size(const drt_scene* scene, const drt_tile* tile,
                                          size_t* bytes);
drt_status drt_forward_mpt(const drt_scene* scene, const drt_tile* tile, int32_t n_iter,
                           float check_eps, float* power, void* workspace,
                           size_t workspace_bytes, void* stream);

/* Per path record of the path finder for every (receiver, candidate):
   paths [n_rx][N_K][K + 2] device floats, overwritten: tau_1..tau_K (NaN past the
   path's order and for a degenerate path), C, kappa (0 for a degenerate path).
   For inspection and tests of small scenes: the output holds n_rx * N_K * (K + 2)
   floats.  Needs no workspace.  Enqueued on `stream`. */
drt_status drt_mpt_paths(const drt_scene* scene, int32_t n_iter, float check_eps, float* paths,
                         void* stream);

/* The same three calls with Fermat path tracing (Sec. V-B) as the finder: from the
   walls' midpoints, n_iter Newton steps on the total path length L = sum_j l_j
   along the walls' lines, (H + 1e-6 diag H) delta = -grad L with
     dL/dtau_j = u_j . (h_{j-1} - h_j),
     H_jj = (1 - (h_{j-1} . u_j)^2) / l_{j-1} + (1 - (h_j . u_j)^2) / l_j,
     H_{j,j+1} = -(u_j . u_{j+1} - (h_j . u_j)(h_j . u_{j+1})) / l_j
   (u_j the wall's unit direction, h_j and l_j leg j's unit direction and length),
   the same clamp, backtracking (on L), convergence check s(check_eps - C) with the
   MPT cost C at the final points, validity and degenerate rule as the MPT finder.
   L is convex in tau, so every accepted step shortens the path; where a wall's line
   separates a path's neighbours the minimum is the straight crossing, whose C is
   4 (i . n)^2 and which the check rejects.  Where two walls meet in a corner the
   iteration can run into it (the leg between them vanishing, L losing its
   derivative) and end degenerate where the MPT finder converges.  Arguments,
   layouts and errors as for drt_forward_mpt / drt_mpt_paths; the paths record's C
   is the MPT cost. */
drt_status drt_forward_fpt_workspace_size(const drt_scene* scene, const drt_tile* tile,
                                          size_t* bytes);
drt_status drt_forward_fpt(const drt_scene* scene, const drt_tile* tile, int32_t n_iter,
                           float check_eps, float* power, void* workspace,
                           size_t workspace_bytes, void* stream);
drt_status drt_fpt_paths(const drt_scene* scene, int32_t n_iter, float check_eps, float* paths,
                         void* stream);

/* Coherent field per receiver: Eq. 7 read as a sum of complex path fields (the
   field normal to the scene plane, free-space spreading 1/L of the unfolded path):
     E_r = sum over the candidates of  prod_j C_j * V * vis * exp(-2 pi i L / wavelength) / L
   with V, vis and L as in drt_forward (Sec. V-A smoothing, same candidates) and
   C_j the reflection coefficient at reflection j:
     eps_r >= 1: Fresnel TE (c - sqrt(eps_r - 1 + c^2)) / (c + sqrt(eps_r - 1 + c^2)),
                 c the cosine of the angle between the arriving leg and the wall's
                 normal (0 at eps_r = 1 and grazing incidence);
     eps_r == 0: the constant -sqrt(scene->refl_coef) (refl_coef >= 0), whose square
                 is drt_forward's power coefficient.
   wavelength: > 0, in the scene's length unit.  The phase carries the FP32 path
   length's rounding: its error grows as 2 pi (L / wavelength) times a few units
   of 2^-24.
   field: [n_rx][2] device (re, im; 8-byte aligned), overwritten.
   power: [n_rx] device receiving |E_r|^2, or NULL.
   workspace: device scratch of at least drt_field_workspace_size bytes.
   tile: as for drt_forward, including two receivers per lane for the hard
   sigmoid and the sigmoid at alpha <= 1e4 unless DRT_TILE_SINGLE_RX is set.
   Enqueued on `stream`; never synchronises. */
drt_status drt_field_workspace_size(const drt_scene* scene, const drt_tile* tile, size_t* bytes);
drt_status drt_field(const drt_scene* scene, const drt_tile* tile, float wavelength, float eps_r,
                     float* field, float* power, void* workspace, size_t workspace_bytes,
                     void* stream);

/* Vector-Jacobian product of drt_field's power: grad_power^T d|E|^2 / d(tx, walls)
   = sum_r grad_power[r] 2 Re(conj(E_r) dE_r / d(tx, walls)) (reverse mode through
   the path fields' amplitude, phase, Fresnel coefficients and the geometry; the
   geometry is recomputed, nothing is stored).
   field: [n_rx][2] device, the E drt_field returned for the same scene, wavelength
   and eps_r (8-byte aligned).  grad_power: [n_rx] device.
   grad_tx: [2] device, overwritten.  grad_walls: [n_walls][4] device (16-byte
   aligned), overwritten, or NULL to skip the wall gradient.
   workspace: at least drt_field_vjp_workspace_size bytes, 16-byte aligned.
   Arguments and errors as for drt_field and drt_vjp. */
drt_status drt_field_vjp_workspace_size(const drt_scene* scene, const drt_tile* tile,
                                        size_t* bytes);
drt_status drt_field_vjp(const drt_scene* scene, const drt_tile* tile, float wavelength,
                         float eps_r, const float* field, const float* grad_power,
                         float* grad_tx, float* grad_walls, void* workspace,
                         size_t workspace_bytes, void* stream);

/* The coherent field with the leg visibilities kept for its adjoint (sigmoid):
   drt_field_save is drt_field (same arguments and workspace) that also fills
   `saved` in drt_forward_save's layout (drt_saved_vis_size floats, device, 4-byte
   aligned, caller-owned); the values are drt_forward_save's, bit for bit (the
   same obstruction loops).  drt_field_vjp_saved is drt_field_vjp given such a
   `saved` for the same scene: its first wall sweep reads them instead; gradients
   equal drt_field_vjp's within FP32 rounding.  Both need smoothing
   DRT_SMOOTH_SIGMOID and n_walls <= DRT_MAX_WALLS (DRT_ERR_UNSUPPORTED otherwise);
   a NULL or misaligned `saved` is DRT_ERR_INVALID_ARG. */
drt_status drt_field_save(const drt_scene* scene, const drt_tile* tile, float wavelength,
                          float eps_r, float* field, float* power, float* saved,
                          void* workspace, size_t workspace_bytes, void* stream);
drt_status drt_field_vjp_saved(const drt_scene* scene, const drt_tile* tile, float wavelength,
                               float eps_r, const float* field, const float* grad_power,
                               const float* saved, float* grad_tx, float* grad_walls,
                               void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------
   3D scenes (Sec. VI: the method does not depend on the dimension).  Walls are
   triangles; planes replace lines, and a point lies on a triangle when its three
   in-plane edge distances pass the smoothed comparison:
     plane of (A, B, C): unit normal n along (B - A) x (C - A), d(p) = n . (p - A);
     edge k (A->B, B->C, C->A): delta_k(p) = m_k . (p - start of k), m_k = n x e_k / |e_k|;
     reflection j valid: prod_k s(delta_k(Q_j)) (s(p) s(q) + s(-p) s(-q)) with p, q the
       plane distances of the neighbouring vertices;
     leg Q_j -> Q_{j+1} blocked by triangle w (not one in the plane of a triangle
       its end points lie on: the leg meets that plane only at the end point):
       X(x, y) prod_k s(delta_k(P)), X(x, y) = s(x) s(-y) + s(-x) s(y), x, y the end
       points' plane distances, P where the leg's line meets w's plane (a line
       parallel to the plane, or meeting it more than 1e8 leg lengths away, is not
       blocked);
     path power Gamma^k V vis / L^2 over the same candidates as in 2D; two
       consecutive reflections on triangles of one plane (normals parallel and
       offsets equal to within 1e-5) make a degenerate path, which contributes 0.
   ------------------------------------------------------------------------ */
typedef struct {
  const float* tris;      /* [n_tris][9] device: corners A, B, C as x, y, z (4-byte aligned) */
  int32_t n_tris;         /* W, 1..DRT_MAX_WALLS; no zero-area triangle */
  const float* rx;        /* [n_rx][3] device */
  int32_t n_rx;           /* R >= 0 */
  const float* tx;        /* [3] device */
  int32_t max_order;      /* K, 0..DRT_MAX_ORDER */
  float alpha;            /* >= 0 */
  drt_smoothing smoothing;
  float refl_coef;        /* Gamma */
} drt3_scene;

/* Bytes of device workspace drt3_forward needs (host out). */
drt_status drt3_forward_workspace_size(const drt3_scene* scene, const drt_tile* tile,
                                       size_t* bytes);

/* Received power per receiver of a 3D scene: power [n_rx] device, overwritten.
   Paths with an exactly-zero validity in all 32 receivers of a warp skip their
   obstruction loop (their power is exactly 0 either way).  tile: as for
   drt_forward (one receiver per lane; the cull flag is implied).  Enqueued on
   `stream`; never synchronises. */
drt_status drt3_forward(const drt3_scene* scene, const drt_tile* tile, float* power,
                        void* workspace, size_t workspace_bytes, void* stream);

/* Transmitter gradient of drt3_forward: grad_tx = sum_r grad_power[r] dP_r / dTX
   (reverse mode with the path recomputed, as drt_vjp; the gradient the antenna
   placement of Sec. VII needs).  grad_power: [n_rx] device; grad_tx: [3] device,
   overwritten; workspace: at least drt3_vjp_tx_workspace_size bytes (warps take
   their units from a counter there; per-unit partials, added in unit order:
   deterministic). */
drt_status drt3_vjp_tx_workspace_size(const drt3_scene* scene, const drt_tile* tile,
                                      size_t* bytes);
drt_status drt3_vjp_tx(const drt3_scene* scene, const drt_tile* tile, const float* grad_power,
                       float* grad_tx, void* workspace, size_t workspace_bytes, void* stream);

/* Vector-Jacobian product of drt3_forward with respect to the transmitter and,
   when grad_tris is not NULL, every triangle corner (Sec. III: the gradient of
   the loss w.r.t. the scene parameters, in 3D):
     grad_tx[i]      = sum_r grad_power[r] dP_r / dTX[i],
     grad_tris[w][c] = sum_r grad_power[r] dP_r / dtris[w][c].
   Reverse mode with the path recomputed, as drt3_vjp_tx; the adjoints of each
   triangle's plane (n, c = n . A) and in-plane edge records (m_k, m_k . start)
   are summed per CTA (warp reductions, shared-memory atomics: the order of those
   additions varies between runs) and chained back to the corners in a fixed
   order by a last kernel.  grad_power: [n_rx]; grad_tx: [3], overwritten;
   grad_tris: [n_tris][9] (4-byte aligned), overwritten, or NULL; workspace: at
   least drt3_vjp_workspace_size bytes (either variant). */
drt_status drt3_vjp_workspace_size(const drt3_scene* scene, const drt_tile* tile, size_t* bytes);
drt_status drt3_vjp(const drt3_scene* scene, const drt_tile* tile, const float* grad_power,
                    float* grad_tx, float* grad_tris, void* workspace, size_t workspace_bytes,
                    void* stream);

/* Autotuner probe for drt_forward (the work decomposition does not change the
   result beyond the order of the per-chunk sums): runs drt_forward on `scene`
   with each of the n_cand tiles of `cands` (host array), one untimed launch
   then `reps` launches timed with CUDA events on `stream`, and writes the
   fastest tile to *best (host; ties go to the earlier candidate) and, when
   ms_out is not NULL, each candidate's mean milliseconds per launch to
   ms_out[0..n_cand) (host; +inf for a candidate whose workspace need exceeds
   workspace_bytes, which is skipped).  power: [n_rx] device, receives the last
   timed candidate's result.  Requires n_rx >= 1 and reps >= 1.  Waits for the
   stream (it reads the events), so it is not for hot paths or stream capture;
   DRT_ERR_WORKSPACE if no candidate fits. */
drt_status drt_tune_forward(const drt_scene* scene, const drt_tile* cands, int32_t n_cand,
                            int32_t reps, float* power, void* workspace, size_t workspace_bytes,
                            drt_tile* best, float* ms_out, void* stream);

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
   derivative is taken as 0 at its kinks (x = +-3/alpha).  Warps take their
   (receiver tile, candidate chunk) units from a counter in the workspace, which
   drt_vjp zeroes on `stream` first (a 16-byte memset), so one workspace serves
   one call in flight at a time.  grad_tx is the same bit for bit from run to
   run; grad_walls varies in the last bits (shared-memory atomics). */
drt_status drt_vjp(const drt_scene* scene, const drt_tile* tile, const float* grad_power,
                   float* grad_tx, float* grad_walls, void* workspace, size_t workspace_bytes,
                   void* stream);

/* The forward's leg visibilities kept for the adjoint (sigmoid).  The sigmoid's
   adjoint spends about a quarter of its time rebuilding every leg's visibility
   (its first wall sweep); drt_forward_save writes them while computing the power,
   and drt_vjp_saved reads them instead.  Layout: saved[(c (K + 1) + j) n_rx + r]
   = the visibility of leg j of candidate c (the candidate order of
   drt_num_candidates) for receiver r, for j <= the candidate's order (the other
   slots are not written).
   drt_saved_vis_size: *floats = N_K (K + 1) n_rx (host out).
   drt_forward_save: drt_forward (same arguments and workspace) that also fills
   `saved` (device, 4-byte aligned, caller-owned, drt_saved_vis_size floats).
   drt_vjp_saved: drt_vjp (same arguments and workspace) given the `saved` of a
   drt_forward_save on the same scene; gradients equal drt_vjp's within FP32
   rounding (the forward's visibilities and the adjoint's sweep differ in the
   order of their products).
   All three need smoothing DRT_SMOOTH_SIGMOID and n_walls <= DRT_MAX_WALLS
   (DRT_ERR_UNSUPPORTED otherwise: the other smoothings' first sweep is cheap). */
drt_status drt_saved_vis_size(const drt_scene* scene, int64_t* floats);
drt_status drt_forward_save(const drt_scene* scene, const drt_tile* tile, float* power,
                            float* saved, void* workspace, size_t workspace_bytes, void* stream);
drt_status drt_vjp_saved(const drt_scene* scene, const drt_tile* tile, const float* grad_power,
                         const float* saved, float* grad_tx, float* grad_walls, void* workspace,
                         size_t workspace_bytes, void* stream);

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

/* The whole objective of Sec. III end to end, from HOST arrays to HOST arrays:
   copies the scene's walls, tx and rx to the device (one cudaMemcpyAsync per
   array), computes the received power (drt_forward), the loss -min_r power[r]
   with its lowest-index argmin (drt_loss, Eq. 8) and the gradient of the loss
   w.r.t. the TX and, when grad_walls is not NULL, the walls (drt_min_loss_vjp),
   and copies the results back (one cudaMemcpyAsync per array), all enqueued on
   `stream`.  For a caller that holds its scene in host memory and has no
   device arrays of its own.
   scene: host pointer whose walls [n_walls][4], tx [2] and rx [n_rx][2] are
   HOST arrays (no alignment needed), n_rx >= 1; other fields as for drt_scene.
   Outputs, all HOST pointers, overwritten: loss [1]; argmin [1] int32 or NULL;
   power [n_rx] or NULL; grad_tx [2]; grad_walls [n_walls][4] or NULL.
   workspace: DEVICE scratch of at least drt_objective_host_workspace_size
   bytes, 256-byte aligned (it holds the device copies of the inputs, the
   power, the loss and the gradients, and the forward's and adjoint's
   workspaces; contents undefined on return).
   The copies are asynchronous with respect to the host when the host arrays
   are pinned (page-locked); the outputs are valid once the stream has been
   synchronised.  Errors as for the calls it makes; a rejected call enqueues
   nothing. */
drt_status drt_objective_host_workspace_size(const drt_scene* scene, const drt_tile* tile,
                                             size_t* bytes);
drt_status drt_objective_host(const drt_scene* scene, const drt_tile* tile, float* loss,
                              int32_t* argmin, float* power, float* grad_tx, float* grad_walls,
                              void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------
   Batched gradient descent on the TX position (Sec. VII, antenna placement),
   for many scenes of uneven size, each with several starting positions.
   A problem is (scene s, start t); each step evaluates the received power of
   every receiver of every problem, the loss -min_r P_r (Eq. 8), its gradient
   w.r.t. the TX by the adjoint of the argmin receiver, and one Adam update of
   the TX, clamped to a box.  One step is captured once into a CUDA graph and
   replayed.  Usage: drt_batch_plan_create -> drt_batch_workspace_size ->
   drt_batch_bind -> drt_batch_run (any number of times) ->
   drt_batch_plan_destroy.  Results are deterministic (fixed summation order).
   With dim = 3 the scenes are 3D (Sec. VI: triangle walls as in drt3_scene,
   receivers and TX in 3D), and the same calls run the same five phases with
   one receiver per lane.
   ------------------------------------------------------------------------ */
typedef struct {
  const float* walls;            /* device [sum_s W_s][4], 16-byte aligned, scene after scene
                                    (dim 3: triangles [sum_s W_s][9], 4-byte aligned) */
  const int32_t* wall_off;       /* device [n_scenes + 1]: scene s owns walls wall_off[s] .. wall_off[s+1]-1 */
  const float* rx;               /* device [sum_s R_s][2], 8-byte aligned (dim 3: [sum_s R_s][3]) */
  const int32_t* rx_off;         /* device [n_scenes + 1] */
  const int32_t* max_order;      /* device [n_scenes]: K of each scene, 0..DRT_MAX_ORDER */
  const int32_t* wall_off_host;  /* host copies of the three arrays above, used to plan the work */
  const int32_t* rx_off_host;
  const int32_t* max_order_host;
  int32_t n_scenes;              /* S >= 1; each scene needs 1 <= W <= DRT_MAX_WALLS, R >= 1 */
  int32_t n_tx;                  /* T >= 1 starting positions per scene */
  int32_t smoothing;             /* drt_smoothing */
  float refl_coef;               /* Gamma */
  int32_t dim;                   /* 2 (or 0) for 2D scenes, 3 for 3D scenes */
} drt_batch;

typedef struct {
  float* tx;                     /* device [S][T][2] ([S][T][3] for 3D), in/out: TX positions */
  float* adam_m;                 /* device, as tx, in/out: Adam first moments (start at 0) */
  float* adam_v;                 /* device, as tx, in/out: Adam second moments (start at 0) */
  int32_t* step;                 /* device [1], in/out: steps taken so far (Adam's t - 1) */
  float* loss;                   /* device [S][T], out: loss of the latest step, before its update */
  float* loss_history;           /* device [history_len][S][T] or NULL: row i = loss of step i */
  int32_t history_len;
  const float* alpha_schedule;   /* device [n_alpha]: alpha of step i = schedule[min(i, n_alpha - 1)] */
  int32_t n_alpha;               /* >= 1 */
  float lr, beta1, beta2, eps;   /* Adam; the learning rate of step i is lr * lr_decay^i */
  float lo_x, lo_y, hi_x, hi_y;  /* the TX is clamped to this box after every update */
  float lr_decay;                /* per-step factor of the learning rate, in (0, 1] */
  float lo_z, hi_z;              /* 3D: the box's z range */
} drt_descent_state;

typedef struct drt_batch_plan drt_batch_plan;

/* Plans the work of a batch (host memory only): validates the host copies of
   the offsets, orders the forward work longest first, sizes the workspace.
   tile: warps_per_cta (1..8), ctas_per_sm and the DRT_TILE_CULL_INVALID,
   DRT_TILE_SINGLE_RX and DRT_TILE_EXIT_BLOCKED flags (the last two for 2D
   batches) are used; NULL for defaults.
   *plan receives a handle owned by the caller (drt_batch_plan_destroy). */
drt_status drt_batch_plan_create(const drt_batch* batch, const drt_tile* tile,
                                 drt_batch_plan** plan);

/* Device workspace the plan needs (bytes, 256-byte aligned). */
drt_status drt_batch_workspace_size(const drt_batch_plan* plan, size_t* bytes);

/* Binds the descent state and workspace to the plan: copies the work tables
   into the workspace (on `stream`) and captures one step into a CUDA graph on
   a stream the plan owns.  The batch's and the state's arrays and the
   workspace must stay valid while the plan is used. */
drt_status drt_batch_bind(drt_batch_plan* plan, const drt_descent_state* state, void* workspace,
                          size_t workspace_bytes, void* stream);

/* Enqueues n_steps descent steps on `stream`: graph replays when use_graph is
   non-zero, direct kernel launches otherwise (same results). */
drt_status drt_batch_run(drt_batch_plan* plan, int32_t n_steps, int32_t use_graph, void* stream);

/* Evaluates the loss of every problem at its current TX (forward + min over
   receivers, written to state->loss) without any update or step count.  With
   tile flag DRT_TILE_CULL_INVALID the obstruction loop of paths whose validity
   is exactly 0 for a whole warp is skipped (exact for hard sigmoid and step). */
drt_status drt_batch_evaluate(drt_batch_plan* plan, void* stream);

/* Plan facts (host out, 8 values): problems, forward units, adjoint units,
   forward CTAs, adjoint CTAs, largest W, receivers x starts, threads per CTA. */
drt_status drt_batch_plan_info(const drt_batch_plan* plan, int64_t* info);

/* Releases the plan (its graph and stream); NULL is accepted. */
drt_status drt_batch_plan_destroy(drt_batch_plan* plan);

/* ------------------------------------------------------------------------
   Surrogate MLP of the objective over the TX position (no counterpart in the
   paper; used to propose starting points for the exact descent).
   x in [0,1]^2 -> Fourier features [sin(2 pi B x), cos(2 pi B x)] (B:
   DRT_MLP_FREQS x 2) -> DRT_MLP_LAYERS x (Linear(DRT_MLP_WIDTH) + SiLU) ->
   Linear(1).  BF16 weights and activations on the tensor cores, FP32
   accumulation, FP32 master weights.  Flat FP32 parameter vector: W1
   [256][64], b1 [256], W2..W4 [256][256], b2..b4 [256], w5 [256], b5 [1].
   The BF16 "shadow" holds each W and its transpose, and w5.  batch must be a
   positive multiple of 64.
   ------------------------------------------------------------------------ */
#define DRT_MLP_FREQS 32
#define DRT_MLP_WIDTH 256
#define DRT_MLP_LAYERS 4

/* Parameter count, shadow bytes, and workspace bytes for `batch` (any NULL out is skipped). */
drt_status drt_mlp_sizes(int32_t batch, int64_t* n_params, size_t* shadow_bytes,
                         size_t* workspace_bytes);

/* shadow <- BF16 copies of the weights of params (16-byte aligned shadow). */
drt_status drt_mlp_shadow(const float* params, void* shadow, void* stream);

/* y[b] = MLP(x[b]) for b < batch (x: [batch][2], freqs: [DRT_MLP_FREQS][2]);
   params supplies the FP32 biases, shadow the BF16 weights (kept in sync by
   drt_mlp_shadow / drt_mlp_adam).  workspace: 256-byte aligned, size from
   drt_mlp_sizes. */
drt_status drt_mlp_forward(const float* params, const void* shadow, const float* freqs,
                           const float* x, int32_t batch, float* y, void* workspace,
                           size_t workspace_bytes, void* stream);

/* loss[0] = mean_b (MLP(x[b]) - target[b])^2 and grad = d loss / d params
   (flat, FP32, overwritten).  Deterministic. */
drt_status drt_mlp_loss_grad(const float* params, const void* shadow, const float* freqs,
                             const float* x, const float* target, int32_t batch, float* loss,
                             float* grad, void* workspace, size_t workspace_bytes, void* stream);

/* Selects the tensor-core path of the MLP's dense layers for this process:
   1 (default) = inference (drt_mlp_forward) by the fused tcgen05.mma kernel
   (accumulators in tensor memory), the training GEMMs of drt_mlp_loss_grad by
   mma.sync (warp-level MMA), which is the faster of the two for them (batch
   8192: 0.35 against 0.47 ms);
   2 = tcgen05.mma for inference and for the training GEMMs whose batch is a
   multiple of 128 (other shapes use mma.sync);
   0 = mma.sync everywhere.
   All give the same function up to FP32 summation order. */
drt_status drt_mlp_set_tensor_core_path(int32_t use_tcgen05);

/* Synchronous: *timed_out = 1 if a tcgen05 kernel gave up waiting for its
   MMAs since the last call (its outputs are then invalid), else 0; clears the
   flag.  Returns DRT_ERR_TIMEOUT in the first case. */
drt_status drt_mlp_tc_status(int32_t* timed_out);

/* Test knob for the timeout path: while skip != 0, the tcgen05 kernels issue no
   MMA and no commit, so their bounded mbarrier wait runs out with nothing in
   flight; they then set the flag read by drt_mlp_tc_status, skip their
   epilogue, free their tensor memory and return (outputs undefined). */
drt_status drt_mlp_test_skip_mma(int32_t skip);

/* One Adam step on the FP32 master params with moments m, v and the device
   step counter (incremented); refreshes the shadow when it is non-NULL. */
drt_status drt_mlp_adam(float* params, float* m, float* v, const float* grad, int32_t* step,
                        float lr, float beta1, float beta2, float eps, void* shadow, void* stream);

/* Size of the static device scratch array behind drt_forward_noalloc. */
#define DRT_NOALLOC_SCRATCH_BYTES (8u << 20)

/* drt_forward for callers that cannot allocate device memory (the paper has no
   counterpart; this is a deployment convenience).  Plugins and callbacks that
   only receive the buffers they must fill, and applications that fix their
   whole device-memory plan at start-up, cannot provide drt_forward's
   workspace.  This call instead uses a scratch array of
   DRT_NOALLOC_SCRATCH_BYTES compiled into the library's device image, which
   every GPU that loads the library keeps until the process exits, and calls no
   allocator.  Same arguments as drt_forward with default tiling (scene: host
   pointer; power: [n_rx] device, overwritten); the result equals drt_forward's
   within FP32 rounding: for large n_rx the candidate chunk is larger than the
   default one, so the per-chunk partial sums are grouped differently.  Two
   calls with the same arguments give the same bits.
   - Limit: one partial sum per (candidate chunk, receiver) must fit, so
     n_rx <= DRT_NOALLOC_SCRATCH_BYTES / 4; above DRT_MAX_WALLS walls the
     staged wall records (128 bytes per wall) share the array and lower that
     bound accordingly.  Larger scenes get DRT_ERR_UNSUPPORTED before anything
     is enqueued.  Scenes that drt_forward rejects are rejected with the same
     status.
   - All calls on a device share the array, and it keeps the last call's
     contents (every value a call reads was written by that same call).
     Calls that overlap on the GPU race on it: order them on one stream.
   - The first call on each device looks the array's device address up
     (cudaGetSymbolAddress) with that device current; make that first call
     before any stream capture begins.  The address is kept until the process
     exits: do not call this entry point on a device after cudaDeviceReset. */
drt_status drt_forward_noalloc(const drt_scene* scene, float* power, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DRT_H */
