// internal.h -- shared internal declarations of the pdmts library (host + device).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "pdmts.h"

namespace pdmts {

// Poll limit of a bounded device-side wait on an mbarrier (each poll suspends
// for at most ~1 us): 2^21 polls, about two seconds.
constexpr unsigned kWaitPolls = 1u << 21;

// ---------------------------------------------------------------- errors ---
int fail(int code, const char *fmt, ...);  // records a thread-local message, returns code
void clear_error();

#define PDMTS_CUDA_TRY(call)                                                              \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return ::pdmts::fail(PDMTS_ERR_CUDA, "%s failed: %s (%s:%d)", #call,          \
                                 cudaGetErrorString(e_), __FILE__, __LINE__);             \
    } while (0)

#define PDMTS_TRY(expr)         \
    do {                        \
        int r_ = (expr);        \
        if (r_ != PDMTS_OK)     \
            return r_;          \
    } while (0)

// --------------------------------------------------------- kernel views ---
// Sliced-ELL family with slice height 32 (one warp = one tile of 32 nodes).
// Node i = 32 t + lane of tile t owns slots k = 0..deg_i-1 at
// col[tile_ptr[t] + 32 k + lane] in ascending neighbour order; slots
// deg_i..tile_k[t]-1 are padding (bit 0 in the mask). Bond status bit k of
// node i is bit (k % 32) of mask[mask_ptr[t] + 32 (k / 32) + lane].
struct SellView {
    const int64_t *tile_ptr;  // [ntiles + 1]
    const int32_t *tile_k;    // [ntiles]
    const int64_t *mask_ptr;  // [ntiles]
    const int32_t *col;       // FP64 path: neighbour index; FP32 path: (j << 8) | stencil id
    uint32_t *mask;
    const int32_t *deg;       // [n]
    int64_t n;
    int64_t ntiles;
};

struct F64StepArgs {
    SellView fam;
    const double *X;      // dim * n
    const double *V;      // n
    const double *cb;     // per slot: c(|xi|)
    const double *alpha;  // n (null when no weights)
    const double *mass;   // n: (1 - alpha) rho
    const double *wb;     // dim * n: (1 - alpha) b (null when no body force)
    const double *g;      // dim * n: interface force per volume (null when none)
    const double *u_in;   // dim * n: displacement at the evaluated time
    double *u_out;        // dim * n: predicted displacement for the next step
    double *v;            // dim * n, in place
    double *a;            // dim * n, in place
    double s0p2;          // (1 + s0)^2
    double dt, hdt, hdt2; // dt, dt/2, dt^2/2
    double theta;         // interface-force factor of this substep
    int breaking;
    int pmb;              // PMB force law instead of the linearised one
    unsigned long long *broken;  // running count of broken bonds (may be null)
};

// Stencil entry of the lattice (FP32) path: offset d = (x_j - x_i) / h in
// lattice units, coef = c(|xi|) h^2 V, thr = s0 (2 + s0) |d|^2, rd = |d|,
// r2 = |d|^2.
struct StencilEntry {
    float d[3];
    float coef;
    float thr;
    float rd;
    float r2;
    float pad;
};
constexpr int kMaxStencil = 256;

// Per-node arrays and constants of the FP32-bulk update (shared by the
// sliced-ELL and the lattice kernels).
struct F32NodeArgs {
    int64_t n;
    const float *inv_m;         // n: 1 / ((1 - alpha) rho)
    const float *wb;            // dim * n: (1 - alpha) b / h (null when none)
    const float *g;             // dim * n: interface force per volume / h (null when none)
    // state in lattice units (u / h) as compensated pairs hi + lo, packed per
    // node: 2D u4 = {hx, hy, lx, ly}; 3D u4 = {hx, hy, hz, lx}, u2 = {ly, lz}
    const float4 *u4_in;
    const float2 *u2_in;
    float4 *u4_out;
    float2 *u2_out;
    float4 *v4;                 // in place, same packing
    float2 *v2;
    float *a;                   // 2D: float2 {ax, ay}; 3D: float4 {ax, ay, az, 0}; in place
    float dt, hdt, hdt2, theta;
    int breaking;
    int pmb;
    unsigned long long *broken;
};

struct F32StepArgs {
    SellView fam;               // col = (j << 8) | stencil id
    const StencilEntry *stencil;// [n_stencil]
    int n_stencil;
    const float *alpha;         // n (null when no weights)
    F32NodeArgs nd;
};

// The 28-offset family of a 2D lattice with 3 h <= delta < sqrt(10) h, in
// ascending neighbour-index order for row-major (x fastest) numbering, i.e.
// sorted by (dy, dx). Bit k of a node's bond word is offset k.
namespace lat2d {
constexpr int NS = 28;
constexpr int R = 3;
constexpr int TX = 32, TY = 8;  // CTA node tile of the lattice kernel
__host__ __device__ constexpr int DX(int k)
{
    constexpr int t[NS] = {0, -2, -1, 0, 1, 2, -2, -1, 0, 1, 2, -3, -2, -1, 1, 2, 3, -2, -1, 0, 1, 2, -2, -1, 0, 1, 2, 0};
    return t[k];
}
__host__ __device__ constexpr int DY(int k)
{
    constexpr int t[NS] = {-3, -2, -2, -2, -2, -2, -1, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 3};
    return t[k];
}
}  // namespace lat2d

// Lattice kernel: nodes form a full nx * ny rectangle numbered i = x + nx y;
// the bond word mask[i] has bit k set while the bond to (x + DX[k], y + DY[k])
// exists and is intact. Coefficients are indexed by |d|^2 (0..9).
struct Lat2DArgs {
    int nx, ny;
    uint32_t *mask;
    const float *alpha;         // n (null when no weights)
    const int32_t *alpha_rows;  // ny + 1: rows y' < y with a weighted node (null when no weights)
    float clin[10];             // linear law: c(|xi|) h^2 V |d|^2 / 2
    float cpmb[10];             // PMB: c(|xi|) h^2 V |d|^4
    float qthr;                 // s0 (2 + s0)
    float qfast;                // qthr (1 - 2^-12): threshold of the fast path's conservative break watch
    int tile;                   // tile configuration, 0 .. kLatTiles - 1
    int num_sms;                // SMs of the device (persistent grids)
    int win_lo[2], win_n[2];    // optional windows in units of TY node rows (win_n[0] == 0: whole lattice)
    int pdl;                    // launch as a programmatic dependent of the previous substep kernel
    unsigned first_polls = kWaitPolls;  // poll limit of each tile's first tensor-copy wait (tests lower it)
    F32NodeArgs nd;
};

// 3D lattice kernel: nodes form a full nx * ny * nz box numbered
// i = x + nx (y + ny z); the family is the 122-offset stencil |d|^2 <= 9
// (lattice units) clipped to the box, offsets in ascending neighbour-index
// order, (dz, dy, dx) lexicographic; a node's bond forces are summed in that
// order. Bond bits: word w of node i at mask[w * n + i], offset k at bit k % 32
// of word k / 32. Per |d|^2 (0..9): coef = c(|xi|) h^2 V, thr = s0 (2 + s0)
// |d|^2, rd = |d|, r2 = |d|^2, ir2 = 1 / |d|^2.
namespace lat3d {
constexpr int NS = 122, W = 4;
// reach of a plane |dz| = a in dy: dy^2 <= 9 - a^2
__host__ __device__ constexpr int reach_y(const int a) { return a == 0 ? 3 : a == 3 ? 0 : 2; }
// reach of row dy of plane |dz| = a in dx: floor(sqrt(9 - a^2 - dy^2))
__host__ __device__ constexpr int reach_x(const int a, const int dy)
{
    const int rem = 9 - a * a - dy * dy;
    return rem < 0 ? -1 : rem >= 9 ? 3 : rem >= 4 ? 2 : rem >= 1 ? 1 : 0;
}
// The 29 stencil rows (dz, dy) in lexicographic order and their reach in dx.
constexpr int NR = 29;
struct RowTab {
    signed char dy[NR], dz[NR], rx[NR];
};
__host__ __device__ constexpr RowTab make_row_tab()
{
    RowTab t{};
    int r = 0;
    for (int dz = -3; dz <= 3; ++dz) {
        const int a = dz < 0 ? -dz : dz;
        for (int dy = -reach_y(a); dy <= reach_y(a); ++dy) {
            t.dy[r] = (signed char)dy;
            t.dz[r] = (signed char)dz;
            t.rx[r] = (signed char)reach_x(a, dy);
            ++r;
        }
    }
    return t;
}
}  // namespace lat3d
// One stencil row of the 3D lattice kernel (a table of NR rows in device
// memory, built once per PD body): per |dx| = 0..3 the coefficient
// c(|xi|) h^2 V, 1/|d|^2, |d|^2 and |d| of the bond (dx, dy, dz) (zeros past
// |d|^2 = 9), the row's offset dz nx ny + dy nx in the node numbering, dy and
// dz as floats and its reach in dx.
struct alignas(16) Row3DEnt {
    float4 coef, ir2, rr, rd;
    int off;
    float fdy, fdz;
    int rx;
};
struct Lat3DArgs {
    int nx, ny, nz;
    uint32_t *mask;
    const uint32_t *exists;     // bond words of the bonds that exist (all intact)
    const float *alpha;         // n (null when no weights)
    const int32_t *alpha_rows;  // ny + 1: rows y' < y with a weighted node (null when no weights)
    const Row3DEnt *rows;       // the NR stencil rows (device)
    // indexed by |d|^2 up to 18 = 9 + 3^2 (a row's dy^2 + dz^2 plus dx^2); 0 past 9
    float coef[19], thr[10], rd[19], r2[19], ir2[19];
    float qfast;                // s0 (2 + s0) (1 - 2^-16): a bond at or past the critical stretch exceeds it
    int tile;                   // 3D tile configuration: blocks of 32 x (4 << tile) nodes in x, y
    int pdl;                    // launch as a programmatic dependent of the previous substep kernel
    F32NodeArgs nd;
};
constexpr int kLat3DTiles = 2;
cudaError_t launch_pd_step_lattice3d(const Lat3DArgs &A, bool init, cudaStream_t s);

// Tensor maps of the lattice kernel's inputs for the tensor-copy staging
// (tile configurations with `tma`): u halo, weight halo, bond words, v, a,
// 1/m and the two planes of the loads wb and g. Built per launch from the
// pointers of a Lat2DArgs; needs nx % 4 == 0 (16-byte row pitch of the FP32
// planes).
struct LatMaps {
    CUtensorMap u, al, mk, v, a, im, wb, g;
};

// Launchers (pd_kernels.cu). `init` computes a_0 from u_0 and predicts u_1
// without touching v.
cudaError_t launch_pd_step_f64(int dim, const F64StepArgs &A, bool init, cudaStream_t s);
cudaError_t launch_pd_step_f32(int dim, const F32StepArgs &A, bool init, cudaStream_t s);
cudaError_t launch_pd_step_lattice2d(const Lat2DArgs &A, bool init, cudaStream_t s);
// Lattice tile configurations: strip height KR (nodes per thread, CTA tile
// 32 x 8 KR), the resident CTAs per SM the registers are limited for,
// whether the persistent pipelined kernel (asynchronous staging of the next
// tiles) is used, and whether clean tiles evaluate each bond once (pair).
struct LatTile {
    int kr, min_blocks, pipelined, pair, tma;
};
constexpr int kLatTiles = 10;
constexpr LatTile kLatTile[kLatTiles] = {{2, 3, 0, 0, 0}, {2, 4, 0, 0, 0}, {2, 2, 1, 0, 0}, {1, 4, 1, 0, 0},
                                         {2, 3, 0, 1, 0}, {2, 4, 0, 0, 1}, {2, 3, 0, 0, 1}, {2, 2, 1, 0, 1},
                                         {1, 4, 1, 0, 1}, {4, 2, 0, 0, 1}};
cudaError_t launch_lattice2d_t0(const Lat2DArgs &A, bool init, cudaStream_t s);
cudaError_t launch_lattice2d_t1(const Lat2DArgs &A, bool init, cudaStream_t s);
cudaError_t launch_lattice2d_t2(const Lat2DArgs &A, bool init, cudaStream_t s);
cudaError_t launch_lattice2d_t3(const Lat2DArgs &A, bool init, cudaStream_t s);
cudaError_t launch_lattice2d_t4(const Lat2DArgs &A, bool init, cudaStream_t s);
cudaError_t launch_lattice2d_t5(const Lat2DArgs &A, bool init, cudaStream_t s);
cudaError_t launch_lattice2d_t6(const Lat2DArgs &A, bool init, cudaStream_t s);
cudaError_t launch_lattice2d_t7(const Lat2DArgs &A, bool init, cudaStream_t s);
cudaError_t launch_lattice2d_t8(const Lat2DArgs &A, bool init, cudaStream_t s);
cudaError_t launch_lattice2d_t9(const Lat2DArgs &A, bool init, cudaStream_t s);
// Batched substeps (tile configurations 0 and 1): lattice2d_batch_prepare
// converts A's windows to the configuration's tile rows and returns the
// instance's tile count (-1 for another configuration); the launch runs one
// CTA per work item {instance index into d_args, tile}.
constexpr int kLatBatchTiles = 2;
int lattice2d_batch_prepare(Lat2DArgs &A, int tile);
cudaError_t launch_lattice2d_batch(const Lat2DArgs *d_args, const int2 *d_work, int nwork, int tile, bool pmb,
                                   cudaStream_t s);
// Damage of the lattice layout (uniform volume): 1 - popc(intact) / popc(exists).
cudaError_t launch_damage_lattice(int64_t n, const uint32_t *mask, const uint32_t *exists, int words,
                                  double *phi, cudaStream_t s);
cudaError_t launch_damage(const SellView &fam, int packed, const double *V, double *phi, cudaStream_t s);
// Unpack a packed FP32 state field (u4/u2 or v4/v2 pairs, or a with u2 ==
// null and `accel`) into dim * n doubles scaled by h.
cudaError_t launch_unpack_f32(int dim, int64_t n, const float4 *p4, const float2 *p2, int accel,
                              double h, double *out, cudaStream_t s);
// Weighted body force from a staged dim * n FP64 field b on the device:
// FP64: wb64 = (1 - alpha) b ; FP32: wb32 = (1 - alpha) b / h. Sets
// flag[0] = 1 if b holds a non-finite value.
cudaError_t launch_weighted_load(int dim, int64_t n, const double *b, const double *alpha64,
                                 const float *alpha32, double inv_h, double *wb64, float *wb32,
                                 unsigned long long *flag, cudaStream_t s);

// ---- MTS coupling helpers (pd_kernels.cu) ----
// Interface force density of the PD overlap nodes, g_p = sum_a N_a(x_p)
// lambda[k_a] per component (= (G_PD^T lambda)_p / V_p); nodes outside the
// overlap are not written. g64 (FP64, dim * n) or g32 (FP32 lattice units,
// scaled by inv_h); lam is dim * nl (component-major). g64b / g32b, if not
// null, receive the same values (a second force field from the same lam).
cudaError_t launch_interface_force(int dim, int64_t n, int64_t n_ov, const int32_t *ov_node, const int32_t *ov_k,
                                   const double *ov_N, int corners, const double *lam, int64_t nl, double inv_h,
                                   double *g64, float *g32, cudaStream_t s, double *g64b = nullptr,
                                   float *g32b = nullptr);
// y[c * nl + k] = sign * sum_p G_PD[k, p] v_p[c] over CSR rows (row k, per
// component) plus, if gfe_col != null, sum_I G_FE[k, I] vfe[c * nfe + I]
// (ELL rows of width gfe_w). v is the PD velocity (FP64 v64, or the FP32
// packed pairs v4/v2 scaled by h). yf, if not null, also receives each y as
// an FP32 pair (hi = y rounded to FP32, lo = the rest rounded to FP32).
cudaError_t launch_constraint(int dim, int64_t nl, const int64_t *gpd_ptr, const int32_t *gpd_col,
                              const double *gpd_val, int64_t npd, const double *v64, const float4 *v4,
                              const float2 *v2, double h, const int32_t *gfe_col, const double *gfe_val, int gfe_w,
                              int64_t nfe, const double *vfe, double sign_pd, double sign_fe, double *y,
                              cudaStream_t s, float2 *yf = nullptr);
// The PD part of launch_constraint (2D, sign_pd, no FE term) for nv FP32
// velocity fields v4 + j v4_stride at once, into y + j y_stride.
cudaError_t launch_constraint_pd_many(int64_t nl, const int64_t *gpd_ptr, const int32_t *gpd_col,
                                      const double *gpd_val, int64_t npd, const float4 *v4, int64_t v4_stride,
                                      int nv, double h, double sign_pd, double *y, int64_t y_stride, cudaStream_t s);
// U_PD += W (u, v, a of the link state), then the prediction for the next
// substep u + dt v + dt^2/2 a.
struct PDAddLink {
    int dim;
    int64_t n;
    int64_t seg_lo[2], seg_n[2];  // node ranges to correct (the link state is zero elsewhere)
    double dt, hdt2;
    // FP64
    double *u, *u_pred, *v, *a;
    const double *wu, *wv, *wa;
    // FP32 (lattice units)
    float4 *u4, *u4_pred, *v4;
    float2 *u2, *u2_pred, *v2;
    float *af;
    const float4 *wu4, *wv4;
    const float2 *wu2, *wv2;
    const float *waf;
};
// End of a coarse step in one launch: U_PD += W on L's link segments,
// count[0] += the changed bits of the `flag`ged words of a against b
// (lattice layout: words indexed by node; sliced ELL: per tile), b = a,
// lam0 = lam (nlam doubles).
cudaError_t launch_finish_step(const PDAddLink &L, int64_t nwords, const uint32_t *a, uint32_t *b,
                               const uint8_t *word_flag, unsigned long long *count, int64_t nlam,
                               const double *lam, double *lam0, cudaStream_t s);

}  // namespace pdmts

// --------------------------------------------------------------- handles ---
struct pdmts_ctx {
    int device = 0;
    int num_sms = 1;                                       // SMs of the device
    cudaStream_t user_stream = nullptr;  // caller's stream (may be legacy default)
    cudaStream_t stream = nullptr;       // library's own non-blocking stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    pdmts_alloc_fn alloc = nullptr;
    pdmts_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    pdmts_pd *pd = nullptr;
    pdmts_fem *fem = nullptr;
    pdmts_arl *arl = nullptr;
    double dt_pd = 0.0;
    int m_ratio = 1;
    double gamma_fe = 0.5, beta_fe = 0.25;
    bool time_set = false;
    pdmts_stats stats{};
    unsigned long long *d_counter = nullptr;  // [0] broken bonds, [1] non-finite input flag,
                                              // [2] a tensor-copy wait of the lattice kernel gave up
    // Give-up watch: h_watch (pinned host) receives d_counter[2] by a copy
    // queued behind each advance and before each read-back's synchronisation;
    // once a give-up is seen the state is undefined and `gave_up` latches
    // until a checkpoint image is loaded.
    unsigned long long *h_watch = nullptr;
    bool gave_up = false;
    unsigned first_wait_polls = pdmts::kWaitPolls;  // pdmts_set_debug_poll_limit
    int watch_enqueue(cudaStream_t s);   // queue the copy of d_counter[2] to h_watch on s
    int watch_check(const char *who);    // PDMTS_ERR_TIMEOUT once a give-up has been seen
    int sync_checked(const char *who);   // watch_enqueue + synchronise `stream` + watch_check
    int64_t device_bytes = 0;
    // substep-chain timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_marks;
    std::vector<int64_t> ev_counts;
    int time_begin(cudaEvent_t *start);                    // record a start mark (if timing)
    int time_end(cudaEvent_t start, int64_t substeps);     // record the matching stop mark
    // coupled coarse steps while timing: start, free phase joined, lambda
    // solved, link run done, end
    std::vector<std::array<cudaEvent_t, 5>> phase_marks;
    int pool_event(cudaEvent_t *e);                        // an event from the pool
    int mark(cudaEvent_t *e);                              // record one on `stream` if timing

    void *dalloc(size_t bytes);
    void dfree(void *p);
    int begin();  // order own stream after the user stream
    int end();    // order the user stream after own stream
};
