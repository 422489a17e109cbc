/*
 * pdmts.h -- C ABI of the GB300 library for multi-time-step (MTS) coupling of
 * bond-based peridynamics (PD) and classical continuum mechanics (CCM)
 * following arXiv 2403.03605 ("Multi-time-step coupling of peridynamics and
 * classical continuum mechanics for dynamic brittle fracture").
 *
 * Conventions (apply to every call below):
 *  - Every call returns int: PDMTS_OK (0) on success, a negative PDMTS_ERR_*
 *    code otherwise. pdmts_last_error() returns a message for the calling
 *    thread's most recent failure.
 *  - Handles are opaque and owned by the library; each *_destroy frees one.
 *  - Input arrays are caller-owned and are copied in during the call; nothing
 *    is retained after the call returns. A pointer may address host memory
 *    (pageable or pinned) or device memory of the context's device (UVA).
 *  - Output arrays are caller-owned buffers of the stated size, host or device.
 *  - Vector fields are structure-of-arrays: component d of node i is at
 *    [d * n + i]. Units are SI. Indices are int32 within one subdomain.
 *  - All device work is ordered after work already queued on the stream given
 *    to pdmts_ctx_create, and work queued on that stream afterwards is ordered
 *    after it. Read-back calls block until their data is on the caller side.
 *  - Failure: arguments are validated before any device work; a failed call
 *    leaves the handle's state unchanged unless stated otherwise.
 */
#ifndef PDMTS_H
#define PDMTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PDMTS_OK 0
#define PDMTS_ERR_ARG (-1)         /* null pointer, size mismatch, NaN, out-of-range value   */
#define PDMTS_ERR_MASS (-2)        /* a PD node with (1 - alpha_i) rho <= 0                 */
#define PDMTS_ERR_STABILITY (-3)   /* dt above the explicit stability bound of the PD model */
#define PDMTS_ERR_CUDA (-4)        /* a CUDA runtime call or kernel failed                  */
#define PDMTS_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up                    */
#define PDMTS_ERR_STATE (-6)       /* call out of order (e.g. advance before set-up)        */
#define PDMTS_ERR_NOMEM (-7)       /* host or device allocation failed                      */
#define PDMTS_ERR_UNSUPPORTED (-8) /* valid request this library does not implement          */

/* ---- enumerations -------------------------------------------------------- */
#define PDMTS_FP64 0      /* all PD arithmetic in IEEE FP64, fixed summation order, no FMA  */
#define PDMTS_FP32_BULK 1 /* bond stretch/force in FP32 from displacement differences;
                             u, v carried as compensated FP32 pairs (needs lattice nodes).
                             On a full 2D rectangle with 3 h <= delta < sqrt(10) h the
                             family is stored as one 28-bit word per node (lattice kernel);
                             otherwise as a sliced-ELL neighbour list                      */
#define PDMTS_FP32_BULK_SELL 2 /* FP32 bulk arithmetic, always on the sliced-ELL list     */

#define PDMTS_MICRO_POWER 0 /* c(|xi|) = c / |xi|^3  (linearised PMB constant)           */
#define PDMTS_MICRO_EXP 1   /* c(|xi|) = c exp(-|xi| / l)                                 */

#define PDMTS_FORCE_LINEAR 0 /* f = c(|xi|) (xi (x) xi) eta                     (Eq. 2)  */
#define PDMTS_FORCE_PMB 1    /* f = c(|xi|) |xi|^3 s (xi + eta) / |xi + eta|   (variant) */

#define PDMTS_WEIGHT_CONSTANT 0 /* alpha = 1/2 in the overlap                     (Sec. 3.2) */
#define PDMTS_WEIGHT_LINEAR 1   /* alpha = l1 / l_O                                (Sec. 3.2) */
#define PDMTS_WEIGHT_CUBIC 2    /* alpha = (l1 / l_O)^3                            (Sec. 3.2) */

typedef struct pdmts_ctx pdmts_ctx;
typedef struct pdmts_pd pdmts_pd;
typedef struct pdmts_fem pdmts_fem;
typedef struct pdmts_arl pdmts_arl;
typedef struct pdmts_batch pdmts_batch;

/* ---- context ------------------------------------------------------------- */

/* Create a context on CUDA device `device`. `cuda_stream` is a cudaStream_t
 * (e.g. torch.cuda.current_stream().cuda_stream) or NULL for the legacy
 * default stream; the library orders its own stream against it. */
int pdmts_ctx_create(pdmts_ctx **ctx, int device, void *cuda_stream);
int pdmts_ctx_destroy(pdmts_ctx *ctx);

/* Message for the calling thread's last failed call ("" if none). The
 * pointer stays valid until the next failing call on the same thread. */
const char *pdmts_last_error(void);

/* Optional device allocator (e.g. PyTorch's caching allocator). alloc must
 * return device memory of the context's device, aligned to 256 bytes, or NULL.
 * Must be set before any subdomain is created. NULL restores cudaMalloc. */
typedef void *(*pdmts_alloc_fn)(size_t bytes, void *user);
typedef void (*pdmts_free_fn)(void *ptr, void *user);
int pdmts_set_allocator(pdmts_ctx *ctx, pdmts_alloc_fn alloc, pdmts_free_fn free_fn, void *user);

/* Block the host until all work queued by the library has finished. */
int pdmts_ctx_synchronize(pdmts_ctx *ctx);

/* ---- PD subdomain (Sec. 2.1: Eq. 1-5; Sec. 2.3: Eq. 34 weights) ---------- */

/* Create the PD subdomain of `ctx` (one per context).
 *   dim            2 (plane stress, per-unit-thickness volumes) or 3
 *   n              number of PD nodes (material points), 0 < n < 2^31
 *   X              reference positions, dim * n doubles (SoA)
 *   vol            nodal volumes V_i (n doubles) or NULL to use vol_uniform
 *   horizon        delta > 0; the family is H_delta(x) = {x' : |x' - x| <= delta}
 *   micro_kind     PDMTS_MICRO_POWER or PDMTS_MICRO_EXP; c, l its constants (Eq. 2,
 *                  Sec. 3.2 / Sec. 3.3 exponential form)
 *   s0             critical stretch s_crit of Eq. 4 (> 0)
 *   rho            mass density (> 0)
 *   precision      PDMTS_FP64 or PDMTS_FP32_BULK
 * The family (CSR, each row ascending) is built here. FP32_BULK requires the
 * nodes to lie on a regular lattice x = x0 + k h (k integer, |k| < 32768);
 * otherwise PDMTS_ERR_UNSUPPORTED. Initial state: u = v = 0, all bonds intact,
 * no body force, breaking enabled, force law PDMTS_FORCE_LINEAR. */
int pd_create(pdmts_ctx *ctx, int dim, int64_t n, const double *X, const double *vol,
              double vol_uniform, double horizon, int micro_kind, double c, double l,
              double s0, double rho, int precision, pdmts_pd **pd);
/* Release the subdomain and its device memory (waits for the context's
 * work). A coupling bound to it must be destroyed first. NULL is a no-op. */
int pd_destroy(pdmts_pd *pd);

/* Pre-crack: each cut is 5 doubles {normal axis, level, along axis, lo, hi}:
 * the plane x[normal] = level, restricted to lo <= x[along] < hi (in 3D the
 * third axis is unrestricted). A bond is broken (mu = 0, Eq. 4) when its end
 * points lie strictly on opposite sides of the plane and its crossing point
 * is inside [lo, hi). On a lattice the test is exact (half-spacing units). */
int pd_set_precrack(pdmts_pd *pd, int n_cuts, const double *cuts);

/* External body force density b (Eq. 1), dim * n doubles [N/m^3]; NULL clears. */
int pd_set_body_force(pdmts_pd *pd, const double *b);

/* Displacement u and velocity v (dim * n doubles each; NULL means zero). The
 * acceleration is recomputed from u (Eq. 1) at the start of the next advance. */
int pd_set_state(pdmts_pd *pd, const double *u, const double *v);

/* Arlequin weights alpha_i of the PD nodes (Eq. 17-18, Eq. 34), n doubles in
 * [0, 1) or NULL (all zero). The PD node mass becomes (1 - alpha_i) rho V_i,
 * its body force (1 - alpha_i) b_i, and bond (i, j) is weighted by
 * 1 - (alpha_i + alpha_j) / 2. PDMTS_ERR_MASS if some 1 - alpha_i <= 0.
 * arlequin_bind sets these from the overlap geometry. */
int pd_set_weights(pdmts_pd *pd, const double *alpha);

/* Enable (1) or freeze (0) bond breaking (Eq. 4). */
int pd_set_breaking(pdmts_pd *pd, int enabled);

/* PDMTS_FORCE_LINEAR (Eq. 2, default) or PDMTS_FORCE_PMB. */
int pd_set_force_law(pdmts_pd *pd, int kind);

/* Tile configuration of the FP32-bulk 2D lattice kernel (a performance
 * setting; results do not depend on it: every configuration evaluates each
 * node's bonds in the same order). 0 .. PDMTS_LATTICE_TILES - 1 fixes one
 * for every chain; PDMTS_LATTICE_TILE_AUTO (the default) times every
 * configuration once, on scratch copies of the state, before the next
 * substep chain and keeps the fastest, and for a coupled subdomain also
 * times one chain of the link run's growing windows (a few hundred tiles per
 * launch) and keeps the fastest configuration for link chains separately. Configurations: 0: one CTA per 32 x 16 tile, strips of 2 nodes
 * per thread, registers for 3 CTAs per SM; 1: the same for 4 CTAs per SM;
 * 2: a persistent grid that stages each CTA's next tile while it computes
 * the current one, 2 nodes per thread; 3: the same with 1 node per thread;
 * 4: configuration 0 where a tile whose nodes all hold
 * their bonds evaluates each bond once (f_ji = -f_ij) and exchanges the
 * reactions through shared memory (linear force law; PMB as configuration 0);
 * 5 and 6: configurations 1 and 0 with every input of a tile staged by
 * tensor copies; 7 and 8: persistent grids with two tensor-copy stages (the
 * next tiles in flight while the CTA computes), 2 and 1 nodes per thread;
 * 9: tensor copies, one CTA per 32 x 32 tile, strips of 4 nodes per thread,
 * registers for 2 CTAs per SM. Lattices with nx % 4 != 0 take the
 * asynchronous-copy kernel of the same shape for 5 to 9 (1, 0, 0, 1 and
 * 4-node strips). The 3D lattice layout has three configurations of its own
 * (0, 1: blocks of 32 x 4 and 32 x 8 nodes of one z plane; AUTO times them the
 * same way). Other layouts and precisions ignore the setting. PDMTS_ERR_ARG
 * if out of range. */
#define PDMTS_LATTICE_TILES 10
#define PDMTS_LATTICE_TILE_AUTO (-1)
int pd_set_lattice_tile(pdmts_pd *pd, int tile);

typedef struct {
    int32_t dim;
    int32_t precision;
    int64_t n;             /* nodes                                        */
    int64_t n_bonds;       /* directed bonds (CSR entries)                 */
    int64_t n_slots;       /* stored slots of the sliced-ELL layout        */
    int32_t max_degree;    /* largest family                               */
    int32_t on_lattice;    /* 1 if the nodes lie on a regular lattice      */
    int32_t layout;        /* 0: sliced-ELL list; 1: 2D lattice bond words;
                              2: 3D lattice bond words (4 per node)        */
    int32_t lattice_nx;    /* lattice layout: nodes along x                */
    int32_t lattice_ny;    /* lattice layout: nodes along y                */
    int32_t lattice_tile;  /* lattice kernel tile configuration in use,
                              PDMTS_LATTICE_TILE_AUTO until it is tuned    */
    double lattice_h;      /* lattice spacing (0 if not on a lattice)      */
    int64_t steps_done;    /* PD substeps advanced since creation          */
    int64_t device_bytes;  /* device memory held by this subdomain         */
    int32_t lattice_nz;    /* 3D lattice layout: nodes along z (else 0)    */
    int32_t link_tile;     /* tile configuration of the link chains (the
                              coupled subdomain's link runs, Eq. 48b)      */
} pdmts_pd_info;
int pd_info(const pdmts_pd *pd, pdmts_pd_info *info);

/* Read-back (blocking). u, v, a: dim * n doubles at the current time. */
int pd_read_displacement(pdmts_pd *pd, double *u);
int pd_read_velocity(pdmts_pd *pd, double *v);
int pd_read_acceleration(pdmts_pd *pd, double *a);
/* Damage phi_i (Eq. 5), n doubles. */
int pd_read_damage(pdmts_pd *pd, double *phi);
/* Damage like pd_read_damage, for callers that cannot let the library
 * allocate device memory at this point: an application whose device memory is
 * wholly reserved by its own pool allocator, or a time-critical loop where an
 * allocation is forbidden because cudaMalloc/cudaFree may synchronise the
 * device. The paper has no counterpart; it is a library facility. The
 * per-node result is staged in a device array that is part of the library
 * image (2^20 doubles, 8 MiB, held by every GPU that loads the library until
 * exit); no cudaMalloc/cudaFree or other allocating routine is called. The
 * first call on a device looks the array's address up (once per device). The
 * call is blocking: it synchronises the context's stream and copies the
 * result into phi (host or device memory, n doubles) before it returns. PD
 * subdomains with more than 2^20 nodes are rejected with
 * PDMTS_ERR_UNSUPPORTED. All calls share the one array, which keeps the last
 * call's contents: calls whose work overlaps on the same GPU (different
 * contexts or threads) race and must be serialised by the caller. On failure
 * only the host-side error message is recorded. */
int pd_read_damage_static(pdmts_pd *pd, double *phi);
/* Bond status mu (Eq. 4) in CSR order (n_bonds bytes, 1 = intact); n_intact
 * may be NULL. */
int pd_read_bond_status(pdmts_pd *pd, uint8_t *mu, int64_t *n_intact);
/* The family in CSR form: row_ptr (n + 1 int64), col (n_bonds int32). */
int pd_read_family(pdmts_pd *pd, int64_t *row_ptr, int32_t *col);

/* ---- time integration (Sec. 2.4 Eq. 38; Sec. 2.5 Eq. 39-49, Alg. 1) ------- */

/* dt_pd: PD time step; m_ratio: dt_fe = m dt_pd (Sec. 2.5); (gamma_fe, beta_fe):
 * Newmark parameters of the FE subdomain. The PD subdomain always uses
 * velocity Verlet (gamma, beta) = (1/2, 0). With check_stability != 0 a dt_pd
 * above the PD stability bound returns PDMTS_ERR_STABILITY. */
int mts_set_time(pdmts_ctx *ctx, double dt_pd, int m_ratio, double gamma_fe, double beta_fe,
                 int check_stability);

/* Advance n_coarse coarse steps. Without an Arlequin coupling bound, a coarse
 * step is m_ratio plain PD velocity-Verlet steps (pure PD). With a coupling,
 * each coarse step is Alg. 1 (FE free step, m PD free substeps with the
 * interpolated multiplier, multiplier solve, correction). */
int mts_advance(pdmts_ctx *ctx, int64_t n_coarse);

/* Kernel timing. While enabled, every chain of PD substeps is bracketed by
 * CUDA events on the library's own stream (the stream the substep kernels run
 * on). pdmts_get_timing blocks, returns the summed chain time in milliseconds
 * and the number of substeps inside those chains, and resets both. */
int pdmts_set_timing(pdmts_ctx *ctx, int enabled);
int pdmts_get_timing(pdmts_ctx *ctx, double *substep_ms, int64_t *substeps);
/* Phase times of the coupled coarse steps run while timing was enabled,
 * summed in milliseconds since the last call (blocks): phase_ms[0] PD free
 * substeps with the FE free step alongside, up to their join; [1] interface
 * problem (constraint residual and lambda_m, Eq. 49); [2] PD link run (Eq.
 * 48b) with the FE correction alongside; [3] PD correction and the rebuild
 * flag, up to the end of the FE correction; [4] whole steps. n_steps receives
 * the number of steps timed. phase_ms holds 5 doubles. */
int mts_get_phase_timing(pdmts_ctx *ctx, double *phase_ms, int64_t *n_steps);

/* ---- CCM subdomain and Arlequin coupling (Sec. 2.2-2.5, Eq. 33-49, Alg. 1) -- */

/* Finite-element subdomain of `ctx` (one per context): linear elastic,
 * isotropic (Eq. 8-9). dim = 2: bilinear quadrilaterals (nodes_per_elem = 4,
 * counter-clockwise, axis-aligned rectangles), plane stress with thickness
 * `thickness`. dim = 3: trilinear hexahedra (nodes_per_elem = 8, axis-aligned
 * boxes; bottom face counter-clockwise seen from +z, then the top face in
 * the same order), `thickness` unused. Xn: dim * n_nodes (SoA); conn:
 * n_elems * nodes_per_elem int32 node ids. 2 x 2 (x 2) Gauss points.
 * PDMTS_ERR_UNSUPPORTED for other element kinds. */
int fem_create(pdmts_ctx *ctx, int dim, int64_t n_nodes, const double *Xn, int64_t n_elems,
               int nodes_per_elem, const int32_t *conn, double E, double nu, double rho,
               double thickness, pdmts_fem **fe);
/* Uniform traction on boundary faces: face_nodes n_faces * 2 node ids (2D
 * edges) or n_faces * 4 (3D planar quadrilaterals, in order around the face),
 * traction n_faces * dim [Pa]; the load of a face is shared equally by its
 * nodes (the consistent load on these straight edges and parallelograms,
 * Eq. 8). Call before arlequin_bind. */
int fem_set_traction(pdmts_fem *fe, int64_t n_faces, const int32_t *face_nodes, const double *traction);
/* Dirichlet boundary (Sec. 3.2: the beam's fixed end): dofs[n_fixed] are dof
 * ids d * n_nodes + node (SoA, host or device memory) held at zero
 * displacement, velocity and acceleration; n_fixed = 0 clears the set.
 * Elimination keeps each fixed row and column only its diagonal, and the
 * fixed dofs' loads are dropped. Call before arlequin_bind; arlequin_bind
 * fails with PDMTS_ERR_ARG when a fixed dof belongs to an overlap element.
 * PDMTS_ERR_ARG for an id out of range, PDMTS_ERR_STATE after binding. */
int fem_set_fixed(pdmts_fem *fe, int64_t n_fixed, const int64_t *dofs);
int fem_destroy(pdmts_fem *fe);
/* Initial FE displacement and velocity (dim * n_nodes each, NULL = zero); the
 * acceleration follows from M a = P - K u; entries at fixed dofs are taken
 * as zero. Call after arlequin_bind. */
int fem_set_state(pdmts_fem *fe, const double *u, const double *v);
/* FE displacement, velocity, acceleration (dim * n_nodes doubles, SoA). */
int fem_read_displacement(pdmts_fem *fe, double *u);
int fem_read_velocity(pdmts_fem *fe, double *v);
int fem_read_acceleration(pdmts_fem *fe, double *a);

/* Couple the PD and FE subdomains over overlap bands (Eq. 17-23, Eq. 33).
 * bands: n_bands * 5 doubles {axis, lo, hi, fe_side, 0}: the overlap is
 * lo <= x[axis] <= hi; the FE-only region lies below lo (fe_side = -1) or
 * above hi (+1). weight_kind: PDMTS_WEIGHT_CONSTANT | LINEAR | CUBIC (Sec. 3.2),
 * alpha = 1 on the FE-only side, 0 on the PD-only side. This sets the PD
 * weights (pd_set_weights), assembles the alpha-weighted FE stiffness, lumped
 * mass and loads (Eq. 34), and builds the constraint operators: the
 * multiplier lives on the FE nodes of the overlap, G_FE = int_O N_k N_I dV,
 * G_PD = N_k(x_p) V_p. Both subdomains have the same dim (2 or 3; axis <
 * dim). Afterwards mts_advance runs Algorithm 1. */
int arlequin_bind(pdmts_ctx *ctx, pdmts_pd *pd, pdmts_fem *fe, int weight_kind, int n_bands,
                  const double *bands, pdmts_arl **arl);
int arlequin_destroy(pdmts_arl *arl);
/* The multiplier lambda of the last completed coarse step (n_lambda doubles,
 * component-major over the multiplier nodes). */
int arlequin_read_lambda(pdmts_arl *arl, double *lambda, int64_t *n_lambda);
/* |G_FE v_FE - G_PD v_PD| (Eq. 41) at the current time and |G_FE v_FE|. */
int arlequin_constraint_residual(pdmts_arl *arl, double *residual, double *reference);
/* How lambda_m = (-H)^-1 y (Eq. 49) is multiplied out each coarse step. AUTO:
 * in the FP64 precision an FP64 product; in FP32-bulk (even n_lambda) the
 * inverse kept as FP32 pairs (hi + lo, scaled by a power of two) and
 * multiplied with error-free FP32 products and compensated sums: FP64-level
 * accuracy (about 2^-40 of sum |a_j y_j|) at the FP32 rate, since GB300 runs
 * FP64 FMAs at a small fraction of its FP32 rate. FP64: the FP64 product in
 * every precision. Takes effect at the next coarse step; PDMTS_ERR_ARG for an
 * unknown kind. */
#define PDMTS_PRODUCT_AUTO 0
#define PDMTS_PRODUCT_FP64 1
int arlequin_set_multiplier_product(pdmts_arl *arl, int kind);

typedef struct {
    int64_t n_lambda;        /* multiplier components                     */
    int64_t n_overlap_pd;    /* PD nodes inside overlap elements          */
    int64_t fe_dofs;         /* finite-element degrees of freedom         */
    int64_t colors;          /* link runs per interface-operator build    */
    int64_t rebuilds;        /* interface-operator builds so far          */
    int64_t cheb_iterations; /* Chebyshev iterations per FE solve         */
    int64_t device_bytes;    /* device memory of the coupling and FE      */
} pdmts_arl_info;
int arlequin_info(pdmts_arl *arl, pdmts_arl_info *info);

/* ---- batches of coupled problems (many specimens, one launch per substep) ---- */

/* A batch of n_members coupled problems advanced together. Every member is a
 * context with a PD subdomain in PDMTS_FP32_BULK on a 2D lattice, an FE
 * subdomain, an Arlequin coupling and mts_set_time called; all on one device
 * and with one force law; no context twice; none already in a batch. The
 * members keep their own sizes, loads, cracks and ratios m and may still be
 * advanced or read alone between batch calls. The batch does not own them; a
 * member destroyed first leaves the batch. PDMTS_ERR_STATE / _UNSUPPORTED /
 * _ARG otherwise. */
int mts_batch_create(int n_members, pdmts_ctx *const *members, pdmts_batch **batch);
/* Advance every member by n_rounds of its own coarse steps (Algorithm 1,
 * m_i PD substeps each in the free and in the link problem). The PD substeps
 * of all members in the same substep slot run as one launch over a work list
 * of (member, tile) of the batch's lattice tile configuration (tuned at the
 * first call among the one-CTA-per-tile configurations). Each member's state
 * afterwards equals, bit for bit, what n_rounds calls of mts_advance(member, 1)
 * would give with the same tile configuration. Work for each member is
 * ordered after its user stream and before it afterwards. */
int mts_batch_advance(pdmts_batch *batch, int64_t n_rounds);
typedef struct {
    int32_t n_members;
    int32_t lattice_tile;      /* tile configuration of the batched substeps */
    int64_t rounds;            /* rounds advanced                            */
    int64_t work_items;        /* (member, tile) items launched              */
    int64_t batched_launches;  /* batched substep launches                   */
    int64_t kernel_launches;   /* all kernels the batch launched (batched PD
                                  substeps, batched FE solves, per-member
                                  coupling kernels)                          */
    /* phases of the last round on the batch stream (ms; blocks until it ends):
     * [0] interface forces of lambda_0, [1] free PD substeps (the FE free
     * steps run beside them), [2] lambda_m and link-problem start, [3] link
     * PD substeps (the FE corrections beside them), [4] corrections, flags
     * and the end of the FE corrections */
    double last_round_ms[5];
} pdmts_batch_info;
int mts_batch_info(const pdmts_batch *batch, pdmts_batch_info *info);
/* Release the batch (waits for its last round); the members stay usable
 * alone. NULL is a no-op. */
int mts_batch_destroy(pdmts_batch *batch);

/* Test facility for the failure path of the bounded device-side waits. The
 * lattice kernels that stage a tile's inputs by tensor copies wait on
 * mbarriers with a poll limit (2^21 polls of at most ~1 us each); a wait that
 * gives up makes its tile skip all writes and raises a device flag. This call
 * sets the limit of each tile's first wait to `polls` (0: give up at once;
 * negative: restore the default); the waits that drain the tile's copies
 * before it returns keep the full limit, so no copy is in flight when a tile
 * ends. After a give-up the substep's result is undefined: mts_advance,
 * mts_batch_advance, the read-backs, pdmts_get_stats and mts_state_save of
 * that context return PDMTS_ERR_TIMEOUT (the advance once the flag has
 * reached the host, at the latest after the next blocking call) until
 * mts_state_load loads a checkpoint image. Not part of the method; for tests. */
int pdmts_set_debug_poll_limit(pdmts_ctx *ctx, int64_t polls);

/* Counters since context creation. */
typedef struct {
    int64_t pd_substeps;      /* PD substeps (free + link)                */
    int64_t bond_updates;     /* directed-bond evaluations                */
    int64_t coarse_steps;     /* coarse steps completed                   */
    int64_t bonds_broken;     /* bonds broken by the dynamics             */
    int64_t kernel_launches;  /* kernels launched by the library          */
    int64_t graph_launches;   /* CUDA graph launches                      */
} pdmts_stats;
int pdmts_get_stats(pdmts_ctx *ctx, pdmts_stats *stats);

/* Checkpoint / resume (the paper has no counterpart; a long run can be
 * stopped and continued). mts_state_size gives the size in bytes of the
 * context's time-stepping state; mts_state_save copies it into `image` (host
 * or device memory, caller-owned, exactly that many bytes); mts_state_load
 * restores an image into a context set up by the same calls (same subdomains,
 * precision, coupling and time settings; the PD step counter comes from the
 * image, the context's statistics do not). The image holds the PD state in its working precision and layout
 * (both displacement buffers, velocity, acceleration), the bond words, the FE
 * state and the last multiplier; continuing after a load gives the same bits
 * as continuing the saved context. A load makes the next coarse step rebuild
 * the interface operator. Blocking (waits for the context's work, and for a
 * batch round it takes part in). PDMTS_ERR_ARG for a wrong size or an image
 * from another set-up, PDMTS_ERR_STATE without a PD subdomain. */
int mts_state_size(pdmts_ctx *ctx, int64_t *bytes);
int mts_state_save(pdmts_ctx *ctx, void *image, int64_t bytes);
int mts_state_load(pdmts_ctx *ctx, const void *image, int64_t bytes);

#ifdef __cplusplus
}
#endif
#endif /* PDMTS_H */
