/* sph.h — C ABI of the B300 weakly-compressible SPH library (libsph_b300.so).
 *
 * The library advances particle states with the delta-SPH scheme described in diffSPH
 * (Winchenbach & Thuerey, arXiv 2507.21684) and differentiates rollouts with a hand-written
 * adjoint.  Every step of the method runs in CUDA kernels for sm_103a; there is no CPU path.
 *
 * Method summary (paper sections in brackets):
 *   state u = (x, v, rho) per particle, global parameters sigma, u_{n+1} = P(u_n)   [Sec. 2.2]
 *   kernel W(r, H) = C_d / H^d w(|r|/H), Wendland C4 (2D/3D) or C2, support H     [App. A.1]
 *   neighbours: cell list (cell key, radix sort, cell ranges), periodic minimum image [Sec. 3.2, App. B]
 *   drho_i/dt = -rho_i sum_j V_j (v_j - v_i) . grad_i W_ij
 *               + delta h c0 sum_j V_j psi_ij . grad_i W_ij                         [Sec. 2.3, Eq. continuity]
 *   dv_i/dt   = -(1/rho_i) sum_j V_j (p_i + p_j) grad_i W_ij
 *               + 2(d+2) nu (rho0/rho_i) sum_j V_j pi_ij grad_i W_ij + g            [Sec. 2.3, Eq. NS, viscosity]
 *   p = rho0 c0^2 / gamma [(rho/rho0)^gamma - 1]  (Tait)                           [Sec. 2.3, Eq. EOS]
 *   v' = v + dt a, rho' = rho + dt drho, x' = x + dt v'  (symplectic Euler)       [Sec. 3.4]
 *   psi_ij = 2 (rho_j - rho_i)(x_j - x_i)/(|x_ij|^2 + eps h^2),
 *   pi_ij  = (v_i - v_j).(x_i - x_j)/(|x_ij|^2 + eps h^2),  V_j = m_j / rho_j
 *   H is the kernel support; h = H/2 is the smoothing length used in delta h c0 and eps h^2
 *   (the paper's common choice H/h = 2, App. A.1).
 *
 * Conventions shared by all calls:
 *   - Every function returns an int status (SPH_OK = 0).  Nothing throws across the ABI.
 *     sph_last_error() returns a thread-local message for the last failing call.
 *   - Particle arrays are packed row-major: x and v hold n*dim floats (x0 y0 [z0] x1 ...),
 *     rho and mass hold n floats.  Fluid particles come first, then wall particles.
 *   - "ptr_is_device" = 1 means the pointers are CUDA device pointers (for example torch
 *     tensors' data_ptr()); 0 means host memory (pageable or pinned).  Inputs are copied;
 *     the caller keeps ownership of everything it passes.  Outputs are caller-allocated.
 *   - Results are always returned in the caller's original particle order.
 *   - A scene is bound to one CUDA stream (0 = legacy default stream).  Calls on one scene
 *     are not thread-safe; different scenes may be used from different threads.
 *   - Device memory of scenes comes from the allocator set with sph_set_allocator (default: the
 *     device's stream-ordered pool, cudaMallocAsync).  The serving loop's scenes always use the
 *     stream-ordered pool (see sph_server_create).
 *   - A scene bound to stream 0 runs on a private non-blocking stream that is ordered after the
 *     legacy default stream at every call and before it when device outputs are returned.
 */
#ifndef SPH_B300_H
#define SPH_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPH_ABI_VERSION 2

#if defined(__GNUC__)
#define SPH_API __attribute__((visibility("default")))
#else
#define SPH_API
#endif

/* status codes */
#define SPH_OK 0
#define SPH_EINVAL 1      /* bad argument or unsupported combination */
#define SPH_ENOMEM 2      /* device allocation failed */
#define SPH_ECUDA 3       /* a CUDA runtime call failed */
#define SPH_EUNSTABLE 4   /* non-finite state or density out of [0.5, 2] rho0 */
#define SPH_ETIMEOUT 5    /* a bounded wait ran out */
#define SPH_EBUSY 6       /* resource temporarily unavailable (admission) */
#define SPH_EINTERNAL 7   /* internal consistency check failed (e.g. a cell overflow) */

#define SPH_KERNEL_WENDLAND4 0   /* Wendland C4, 2D and 3D (App. A.1) */
#define SPH_KERNEL_WENDLAND2 1   /* Wendland C2, 2D and 3D */
#define SPH_DENSITY_CONTINUITY 0 /* integrate drho/dt with delta diffusion (Sec. 2.3) */
#define SPH_DENSITY_SUMMATION 1  /* rho_i = sum_j m_j W_ij each step, no diffusion (Sec. 2.3) */
/* delta-SPH density diffusion of the continuity mode, delta h c0 sum_j V_j psi_ij . grad_i W_ij
 * (Sec. 2.3 cites the delta-SPH model without printing the term):
 *   MC      psi_ij = 2 (rho_j - rho_i) (x_j - x_i) / (|x_ij|^2 + eps h^2)   (Molteni-Colagrossi)
 *   RENORM  psi_ij = 2 [(rho_j - rho_i) - (g_i + g_j) . (x_j - x_i) / 2] (x_j - x_i) / (|x_ij|^2 + eps h^2)
 *           with g_i = <grad rho>_i^L = sum_j V_j (rho_j - rho_i) L_i grad_i W_ij and
 *           L_i = pinv(sum_j V_j (x_j - x_i) (x) grad_i W_ij) over all neighbours, walls included
 *           (the kernel renormalisation of App. A; the pseudo-inverse drops eigen-directions with
 *           |lambda| <= 1e-3 max|lambda|).  The term then vanishes for a linear density, also at a
 *           free surface.  One extra neighbour pass per step; no adjoint (sph_rollout rejects it). */
#define SPH_DIFFUSION_MC 0
#define SPH_DIFFUSION_RENORM 1
/* Wall treatment (Sec. "Boundary Conditions"):
 *   SHEPARD  p_w = (sum_f p_f W + g . sum_f rho_f r_wf W) / sum_f W over fluid neighbours f,
 *            rho_w by the inverse Tait law (the default);
 *   MDBC     each wall particle b has a ghost node g inside the fluid (its mirror image across the
 *            wall surface, sph_set_ghosts); the SPH interpolation at g of a first-order expansion
 *            of q = rho - rho0 in the fluid gives the (d+1) x (d+1) system
 *              [<1> <x_jg>^T; <grad 1> <grad (x) x_jg>] [f; f'] = [<q>; <grad q>],
 *            x_jg = x_j - x_g over fluid j within H of g, solved by a pseudo-inverse in units of H
 *            (singular values <= 1e-3 of the largest dropped); rho_b = rho0 + f + (x_b - x_g) . f',
 *            rho0 when no fluid is in range; p_b by the Tait law.  Walls keep v = 0.  No adjoint. */
#define SPH_BOUNDARY_SHEPARD 0
#define SPH_BOUNDARY_MDBC 1

/* Global parameters sigma of one scene (Sec. 2.2; App. C "global state dictionary").
 * The support radius H is the kernel's cut-off (the paper stores the support and calls it h).
 * Box: [box_lo, box_hi) per axis; periodic axes (bit k of periodic_mask) use the minimum
 * image on absolute, unwrapped positions (Sec. 3.2); open axes clamp particles into the edge
 * cells.  Cells have edge >= H + skin; a periodic axis needs at least 3 cells.
 * The cell structure is rebuilt every step when skin == 0.  With skin > 0 (a Verlet list in the
 * sense of App. B) a captured step rebuilds only when rebuild_interval sweeps have used the
 * current cells or when some particle has moved farther than skin/2 since the last build (the
 * sweep measures the displacement; in 2D its last CTA decides and the rebuild is a cooperative
 * launch in the step's CUDA graph that returns at once unless a rebuild is due; in 3D a one-thread
 * kernel decides and a conditional node of the graph runs the rebuild kernels).  Steps run without
 * graphs rebuild every step; the adjoint's replay rebuilds on its own schedule (sph_adjoint_info). */
typedef struct sph_params {
  int32_t dim;            /* 2 or 3 */
  int32_t kernel;         /* SPH_KERNEL_* */
  int32_t density_mode;   /* SPH_DENSITY_* */
  int32_t periodic_mask;  /* bit k: axis k periodic */
  double box_lo[3];
  double box_hi[3];
  float H;                /* support radius (> 0) */
  float dt;               /* fixed time step (> 0) */
  float rho0;             /* rest density */
  float c0;               /* numerical speed of sound */
  float gamma;            /* Tait exponent (7) */
  float nu;               /* kinematic viscosity (>= 0) */
  float delta;            /* delta-SPH diffusion coefficient (term delta h c0, h = H/2) */
  float eps;              /* regulariser: denominators use |x_ij|^2 + eps h^2, h = H/2 */
  float g[3];             /* body acceleration */
  int32_t rebuild_interval; /* >= 1, used when skin > 0 */
  float skin;             /* Verlet skin (absolute length, >= 0) */
  int32_t diffusion;      /* SPH_DIFFUSION_* (continuity mode; no effect with summation density) */
  float shift;            /* explicit particle shifting at the end of each step, coefficient C >= 0
                           * (0: off).  The paper shifts in a post-processing step after each time
                           * step, citing the explicit scheme of Sun et al. (not printed); here the
                           * delta+-SPH form dx_i = -C H^2 sum_j V_j [1 + 0.2 (W_ij/W(dp))^4] grad_i W_ij,
                           * dp = (m_i/rho0)^(1/d), over the neighbours at the swept positions, in
                           * the bulk (lambda_i >= 0.75, lambda_i the smallest eigenvalue of the
                           * renormalisation matrix), tangential to the outward normal
                           * -sum_j V_j grad_i W_ij in the free-surface band (0.4 <= lambda_i < 0.75),
                           * none for isolated particles.  Positions only; walls stay.  C is the
                           * product CFL * Mach of Sun et al.  No adjoint (sph_rollout rejects it).
                           * The shift needs cells valid for the swept positions: eager steps rebuild
                           * twice per step, captured steps check the skin again before the shift. */
  int32_t boundary;       /* SPH_BOUNDARY_* (shared by the scenes of a batch) */
} sph_params;

typedef struct sph_scene sph_scene;

/* Allocator hooks: alloc(bytes, stream, ctx) returns a device pointer or NULL; free(ptr, bytes,
 * stream, ctx).  Passing NULL restores the default (cudaMallocAsync / cudaFreeAsync).  Applies to scenes created after
 * the call.  The hooks must stay valid until every scene using them is destroyed. */
typedef void* (*sph_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*sph_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
SPH_API int sph_set_allocator(sph_alloc_fn alloc_fn, sph_free_fn free_fn, void* ctx);

SPH_API int sph_abi_version(void);
SPH_API const char* sph_last_error(void);

/* Create a scene from an initial state u_0 = (x, v, rho) with per-particle masses.
 * n_fluid fluid particles followed by n_wall fixed wall particles (walls keep v = 0; their
 * pressure and density are extrapolated from the fluid every step).  Returns SPH_EINVAL for
 * inconsistent parameters (dim, H <= 0, fewer than 3 cells on a periodic axis, ...). */
SPH_API int sph_init(const sph_params* params, int n_fluid, int n_wall, const float* x, const float* v,
             const float* rho, const float* mass, int ptr_is_device, void* cuda_stream, sph_scene** out);

/* Batched scenes: n_scenes independent problems packed into one scene object (segments), advanced
 * by the same launches (one launch per stage for all of them; the paper's batched merging of
 * scenes, Sec. 4.1 "Computational Scaling").  All scenes must share dim, kernel, density mode and
 * rebuild_interval, and either all or none have a Verlet skin (the skins may differ); every other
 * parameter is per scene.  Arrays are given per scene.
 * The other calls then act on the whole batch: particle rows of get_state / rates / adjoint are
 * the scenes' rows concatenated in scene order (sph_batch_info gives each scene's first row and
 * row count), and sph_adjoint writes one viscosity adjoint per scene.  Each scene's results are
 * identical (bitwise) to running it alone when the cells are rebuilt every step (no skin, or
 * steps without graphs); with a Verlet skin the batch rebuilds all its scenes whenever one of them
 * needs it, so a scene may be re-sorted at other steps than alone: the same neighbours, its sums
 * taken in another order (float rounding). */
SPH_API int sph_init_batch(int n_scenes, const sph_params* params, const int* n_fluid, const int* n_wall,
                           const float* const* x, const float* const* v, const float* const* rho,
                           const float* const* mass, int ptr_is_device, void* cuda_stream, sph_scene** out);
SPH_API int sph_batch_info(const sph_scene* scene, int* n_scenes, int32_t* first_row, int32_t* n_rows);

/* Advance the scene by n_steps steps of the scheme above (no tape kept).  Asynchronous with
 * respect to the host; errors detected on the device surface at the next synchronising call. */
SPH_API int sph_step(sph_scene* scene, int n_steps);

/* Copy the current state out (original order).  Any pointer may be NULL to skip that field.
 * Synchronises the scene's stream; returns SPH_EUNSTABLE if the state is not finite. */
SPH_API int sph_get_state(const sph_scene* scene, float* x, float* v, float* rho, int ptr_is_device);

/* Evaluate the right-hand side at the current state without advancing it: a (n_fluid*dim)
 * and drho/dt (n_fluid), plus the density used (n_fluid; differs from the state only in
 * summation mode).  Original order, fluid particles only.  Any output may be NULL. */
SPH_API int sph_rates(sph_scene* scene, float* a, float* drho, float* rho_used, int ptr_is_device);

/* Shifting by optimisation (Sec. "New Applications: Differentiable Particle Shifting"): particle
 * positions are optimised against
 *   L = (1/n) sum_i [ w_color (1 - c_i)^2 + w_grad |g_i|^2 + w_density (rho_i - t(x_i))^2
 *                     + w_reg sum_{j: |x_ij| < a dp_i} (a dp_i - |x_ij|)^2 ]
 * over the n fluid particles of each scene (walls are fixed neighbours), with the summation density
 * rho_i = sum_j m_j W_ij (self included, every particle), the colour field c_i = sum_j (m_j/rho_j) W_ij
 * (self included), its gradient g_i = sum_j (m_j/rho_j) grad_i W_ij, the target density t (a
 * sinusoid t_base + t_amp sin(t_k . x + t_phase), or a step: t_lo where t_n . x < t_c, else t_hi),
 * and a pair penalty below a = reg_fraction times the spacing dp_i = (m_i/rho0)^(1/d).  The
 * neighbour set is that of the current positions, held fixed under differentiation.  Only the
 * positions are used (velocities and the state's densities are ignored). */
typedef struct sph_shift_objective {
  float w_color, w_grad, w_density, w_reg, reg_fraction;
  int32_t target_kind;   /* 0 sinusoid, 1 step */
  float t_base, t_amp, t_k[3], t_phase;
  float t_lo, t_hi, t_n[3], t_c;
} sph_shift_objective;

/* L per scene (host doubles, may be NULL) and dL/dx of every particle row ((n_fluid + n_wall) * dim
 * floats, original order, walls 0; may be NULL) at the current positions. */
SPH_API int sph_shift_gradient(sph_scene* scene, const sph_shift_objective* objective, double* loss, float* grad,
                               int ptr_is_device);
/* n_iters steps of gradient descent x <- x - step dL/dx on the fluid positions (walls fixed);
 * loss_hist (host, n_iters * n_scenes doubles, may be NULL) receives L before each step. */
SPH_API int sph_shift_descend(sph_scene* scene, const sph_shift_objective* objective, int n_iters, float step,
                              double* loss_hist);

/* Variable support radius (the paper's symmetric neighbour search for per-particle radii): radii
 * H_i of every particle row ((n_fluid + n_wall) floats, original order), 0 < H_i <= the scene's H
 * (which sizes the cells).  Kept with the particles; the time step itself keeps the uniform H.
 * With radii set, sph_debug_pairs returns the pairs with |x_ij| < max(H_i, H_j) (FP64 decision).
 * Single scenes. */
SPH_API int sph_set_support(sph_scene* scene, const float* H, int ptr_is_device);
/* At the current positions, per particle row (any output may be NULL; radii H_i, or the scene's H
 * where none were set):
 *   search_radius  s_i = max(H_i, max{H_k : |x_ik| < H_k})   (the neighbour search's radius: every
 *                  j with |x_ij| < max(H_i, H_j) lies within s_i; exact, FP64 decisions)
 *   rho_super      sum_j m_j (W(|x_ij|, H_i) + W(|x_ij|, H_j)) / 2 over |x_ij| < max(H_i, H_j)
 *   rho_gather     sum_j m_j W(|x_ij|, H_i) over |x_ij| < H_i
 * (self terms included; W(r, h) = C_d / h^d w(r / h)). */
SPH_API int sph_support_query(sph_scene* scene, float* search_radius, float* rho_super, float* rho_gather,
                              int ptr_is_device);

/* Ghost nodes of the wall particles for SPH_BOUNDARY_MDBC: n_wall * dim floats per scene (the
 * walls in their input order; a batch's scenes one after another).  Copied; required before the
 * first step, rate evaluation or rollout of an mDBC scene with walls (SPH_EINVAL otherwise). */
SPH_API int sph_set_ghosts(sph_scene* scene, const float* ghost, int ptr_is_device);

/* Renormalised density gradient <grad rho>^L (see SPH_DIFFUSION_RENORM) at the current state,
 * after the wall extrapolation a step applies: (n_fluid + n_wall) * dim floats, original order
 * (fluid rows, then wall rows; per scene for a batch, n_rows of sph_batch_info plus the walls).
 * Any diffusion mode; synchronises the scene's stream. */
SPH_API int sph_density_gradient(sph_scene* scene, float* grad, int ptr_is_device);

/* Forward rollout of n_steps that keeps what the adjoint needs: the state every ckpt_every
 * steps (gradient checkpointing, Sec. 3.3).  Replaces any previous tape of this scene.
 * SPH_EINVAL with SPH_DIFFUSION_RENORM in continuity mode or particle shifting (no reverse pass of
 * those terms); sph_adjoint needs a scene without walls. */
SPH_API int sph_rollout(sph_scene* scene, int n_steps, int ckpt_every);

/* Reverse pass of the last sph_rollout (vector-Jacobian product, Sec. 2.2): given the adjoints
 * of the final state (xbar_T, vbar_T, rhobar_T; NULL = zero) return those of the initial state
 * (xbar_0, vbar_0, rhobar_0; NULL = skip) and of the viscosity (nubar: host doubles, one per
 * scene of a batch; may be NULL).
 * Segments between checkpoints are recomputed forward and replayed backwards; the forward replay
 * of the next segment runs on a second stream of the library's beside the reverse pass of the
 * current one (two tapes of ckpt_every + 1 steps are kept).  Continuity or
 * summation density (Sec. 2.3); in summation mode each step's density sum_j m_j W_ij of the
 * step's positions is differentiated too (its adjoint passes to the positions, and rhobar_0 is
 * zero: the step overwrites the density it is given).  Scenes without wall particles only
 * (SPH_EINVAL otherwise, or without a preceding rollout).
 * The scene's state is left at the end of the rollout. */
SPH_API int sph_adjoint(sph_scene* scene, const float* xbar_T, const float* vbar_T, const float* rhobar_T,
                float* xbar_0, float* vbar_0, float* rhobar_0, double* nubar, int ptr_is_device);

/* The adjoint's forward replay of each segment rebuilds the cells at its first step and then
 * every replay_interval steps when the scene has a Verlet skin (every step without one; the
 * interval starts at three quarters of the rollout's mean rebuild interval, at most 16); a segment
 * whose displacements outgrow the skin is replayed again with a rebuild every step, and the
 * interval is halved for the segments that follow.  Reports the current interval and how many
 * segments fell back (cumulative). */
SPH_API int sph_adjoint_info(sph_scene* scene, int32_t* replay_interval, int64_t* replay_fallbacks);
/* Fix the replay's starting interval (taken at the next sph_rollout; 0 restores the automatic
 * choice).  Results do not depend on it: an interval the skin cannot sustain falls back. */
SPH_API int sph_set_adjoint_replay(sph_scene* scene, int replay_interval);

/* Scene geometry: cells per axis (3 ints), total particles. */
SPH_API int sph_scene_info(const sph_scene* scene, int32_t* ncell3, int32_t* n_particles);

/* Cell structure of the current state (host outputs): CSR offsets cell_start[n_cells + 1] over
 * the linear cell index ((cz * ny + cy) * nx + cx), and sorted_ids[n] = original particle index
 * in sorted order (stable by cell; ties keep the previous storage order, which is ascending
 * original index for a freshly initialised scene).  Builds the cells if needed. */
SPH_API int sph_debug_cells(sph_scene* scene, int64_t* cell_start, int32_t* sorted_ids);

/* All ordered neighbour pairs (i, j), i != j, |mimg(x_i - x_j)|^2 < H^2 with the squared
 * distance evaluated in FP64 from the float32 positions, as original indices (host outputs,
 * unordered).  *n_pairs receives the total; at most cap pairs are written. */
SPH_API int sph_debug_pairs(sph_scene* scene, int64_t* n_pairs, int32_t* pi, int32_t* pj, int64_t cap);

/* Test of the device-side bounded waits on the current device: a sweep tile's wait on a gate that
 * no wall task opens, and a cooperative grid barrier that one CTA never reaches.  Each gives up
 * after its poll limit (a fraction of a second) and reports status bit 1 (2) in *gate_status and
 * *barrier_status; the context stays usable.  No fault is involved. */
SPH_API int sph_debug_bounded_waits(int* gate_status, int* barrier_status);

/* Per-kernel device timing.  When enabled, the scene records CUDA events around its launches
 * on its stream; sph_timing returns the accumulated milliseconds and launch count of one
 * kernel class (0 = fused sweep, 1 = rebuild (keys+sort+ranges+permute), 2 = walls,
 * 3 = density, 4 = adjoint sweep, 5 = renormalised density gradient, 6 = particle shifting,
 * 7 = shifting-by-optimisation objective, 8 = its gradient) and resets it.  Synchronises the stream. */
SPH_API int sph_profile(sph_scene* scene, int enable);
SPH_API int sph_timing(sph_scene* scene, int kernel_class, double* ms, int64_t* launches);

/* How sph_step issues its work: use_graphs = 1 (default) captures chunks of graph_chunk steps
 * (default 8) into CUDA graphs and replays them; 0 launches every kernel from the host, one step
 * at a time, and then rebuilds the cell structure every step (the device-side skin check lives in
 * the captured steps).  Results do not depend on the choice, except through the
 * summation order that the rebuild schedule sets.  SPH_EINVAL for graph_chunk outside [1, 4096]. */
SPH_API int sph_set_execution(sph_scene* scene, int use_graphs, int graph_chunk);

/* Counters of the last sph_step/sph_rollout/sph_adjoint call: in-radius ordered pairs per step
 * (fluid i), kernel launches executed (conditional rebuilds included).  Synchronises. */
SPH_API int sph_counters(sph_scene* scene, int64_t* pairs_per_step, int64_t* launches);

/* Cumulative counters since sph_init: forward steps, cell-structure rebuilds (host-launched and
 * those decided on the device under a Verlet skin), kernel launches executed.  Synchronises.
 * Any output may be NULL. */
SPH_API int sph_stats(sph_scene* scene, int64_t* steps, int64_t* rebuilds, int64_t* launches);

SPH_API void sph_destroy(sph_scene* scene);

/* ------------------------------------------------------------------------------------------
 * Serving: continuous batching of rollout requests on one GPU (no counterpart in the paper;
 * it serves many independent scenes the way the paper batches them, Sec. 4.1).
 *
 * A server owns a stream and a host thread for the forward batch and one of each per adjoint
 * worker (three), so it takes no caller stream: requests arrive from host memory and sph_wait
 * returns results to host memory.  sph_submit copies the request and queues it;
 * requests are admitted in arrival order while the estimated device bytes of all admitted
 * requests stay within hbm_budget_bytes and at most max_active run at once.  Admitted forward
 * rollouts keep their particle state resident in one packed batch that is advanced with shared
 * launches; arrivals join and finished requests leave at step-chunk boundaries (the batch is
 * re-packed on the device).  Adjoint requests (forward rollout with checkpoints, then the reverse
 * pass for the loss L = (1/N) sum_i |x_i^T - x~_i|^2 with target positions x~, Sec. 4.1) run on
 * a pool of adjoint workers (one stream each) concurrently.  The server launches the batch's steps
 * without graphs; without a Verlet skin every step rebuilds the cells, so a served result is
 * bitwise the result of the scene alone; with a skin the batch rebuilds all its scenes when the
 * device finds that one of them needs it, so a served scene may be re-sorted at other steps than
 * alone (the same neighbours, its sums in another order: float rounding).
 * Forward requests share the batch only with requests of the same dim, kernel, density mode,
 * diffusion form, shifting on or off, wall treatment, rebuild_interval and with a skin or without
 * (the skins may differ); one of another kind waits, in arrival order, until the running batch has
 * drained.
 * A scene of the batch that becomes unstable fails alone (SPH_EUNSTABLE from sph_wait); the others
 * continue.  Results stay with the server until sph_wait returns them (once per ticket). */
#define SPH_REQ_FORWARD 0
#define SPH_REQ_ADJOINT 1

typedef struct sph_request {
  sph_params params;
  int n_fluid, n_wall;
  const float *x, *v, *rho, *mass;  /* host arrays, copied by sph_submit */
  int n_steps;                      /* >= 1 */
  int mode;                         /* SPH_REQ_FORWARD or SPH_REQ_ADJOINT */
  int ckpt_every;                   /* adjoint: checkpoint interval (0: 20) */
  const float* x_target;            /* adjoint: target final positions (NULL: the initial positions) */
  const float* ghost;               /* SPH_BOUNDARY_MDBC with walls: ghost nodes (n_wall * dim), copied */
} sph_request;

typedef struct sph_result {
  float *x, *v, *rho;               /* caller buffers for the final state (or NULL) */
  float *xbar0, *vbar0, *rhobar0;   /* adjoint: caller buffers for dL/d(x0, v0, rho0) (or NULL) */
  double nubar;                     /* adjoint: dL/dnu */
  double loss;                      /* adjoint: L */
  double t_submit, t_admit, t_done; /* server clock, seconds */
} sph_result;

typedef struct sph_server_info {
  double particle_steps_fwd;        /* fluid particle-steps done by the forward batch */
  double particle_steps_adj;        /* forward particle-steps of finished adjoint requests */
  int queued, active, max_batch;
  size_t bytes_in_use;
  long long repacks, iterations;
} sph_server_info;

typedef struct sph_server sph_server;
/* The server's threads create and destroy scenes at a high rate (every re-pack of the batch,
 * every adjoint request); they allocate from the CUDA stream-ordered pool of the server's streams
 * (cudaMallocAsync / cudaFreeAsync), never through the sph_set_allocator hooks, which may call
 * back into an interpreter whose lock those threads would contend for.  hbm_budget_bytes bounds
 * what the admitted requests may hold; max_active the number of requests admitted at once. */
SPH_API int sph_server_create(size_t hbm_budget_bytes, int max_active, sph_server** out);
/* SPH_EINVAL for malformed requests or one that alone exceeds the budget. */
SPH_API int sph_submit(sph_server* server, const sph_request* request, uint64_t* ticket);
SPH_API int sph_poll(sph_server* server, uint64_t ticket, int* done);
/* Bounded wait: SPH_ETIMEOUT if the request is not done within timeout_ms (it stays queued or
 * running and can be waited on again); otherwise copies the results and forgets the ticket. */
SPH_API int sph_wait(sph_server* server, uint64_t ticket, int timeout_ms, sph_result* result);
SPH_API int sph_server_stats(sph_server* server, sph_server_info* stats);
/* Stops the loops after the current chunk; unfinished requests are dropped. */
SPH_API void sph_server_destroy(sph_server* server);

#ifdef __cplusplus
}
#endif
#endif /* SPH_B300_H */
