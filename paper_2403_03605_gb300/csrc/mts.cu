// mts.cu -- multi-time-step Arlequin coupling of PD and finite elements
// (arXiv 2403.03605, Sec. 2.2-2.5, Eq. 33-49, Algorithm 1).
//
// Per coarse step t_0 -> t_m = t_0 + m dt_PD:
//   stream B: finite-element free step (Eq. 47a with Newmark, Eq. 39): predictor,
//             K_eff a = P - K u~ by Chebyshev iteration (no reductions), update;
//   stream A: interface force G_PD^T lambda_0 / V on the PD overlap nodes, then
//             the m PD free substeps (Eq. 48a) with factor (1 - j/m), one graph;
//   join;     y = G_FE v_FE - G_PD v_PD, lambda_m = (-H)^-1 y (Eq. 49);
//             stream B: FE correction a += a_W with K_eff a_W = -G_FE^T lambda_m
//             (Eq. 47b, the same Chebyshev solve as the free step); stream A:
//             PD correction U += W from the link problem (Eq. 48b, zero start,
//             factor j/m, bond words of the step start, no breaking); rebuild
//             flag if a bond near an overlap band broke.
// Stream B has the higher priority: its short kernels take SMs as soon as a
// PD kernel's blocks retire, so the FE work hides under the PD chains. Both FE
// sequences run as CUDA graphs captured once per schedule.
// Conventions follow Eq. 33: FE carries +G_FE^T lambda, PD -G_PD^T lambda and
// the constraint is G_FE v_FE - G_PD v_PD = 0. All coupling arithmetic is FP64.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

#include <cusolverDn.h>
#include <map>
#include <new>

#include "pd.h"

using namespace pdmts;

// A captured launch sequence, replayed while the launch arguments it was
// captured with (pointers and scalars, packed into key) are unchanged.
struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    std::vector<uint64_t> key;
    int64_t launches = 0;
    void reset()
    {
        if (exec)
            cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
        launches = 0;
    }
};

static uint64_t key_bits(double x)
{
    uint64_t b;
    std::memcpy(&b, &x, sizeof b);
    return b;
}
static uint64_t key_bits(const void *p) { return (uint64_t)(uintptr_t)p; }

// Replay g on s, capturing enqueue(&launches) first if g is empty or was
// captured under another key.
template <class F>
static int run_graph(pdmts_ctx *ctx, GraphSlot &g, const std::vector<uint64_t> &key, cudaStream_t s, F &&enqueue,
                     int64_t *launches)
{
    if (!g.exec || g.key != key) {
        g.reset();
        cudaGraph_t graph = nullptr;
        PDMTS_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int64_t n = 0;
        const int r = enqueue(&n);
        const cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (r != PDMTS_OK) {
            if (graph)
                cudaGraphDestroy(graph);
            return r;
        }
        if (ce != cudaSuccess)
            return fail(PDMTS_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            g.exec = nullptr;
            return fail(PDMTS_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
        }
        g.key = key;
        g.launches = n;
    }
    PDMTS_CUDA_TRY(cudaGraphLaunch(g.exec, s));
    *launches += g.launches;
    ctx->stats.graph_launches += 1;
    return PDMTS_OK;
}

// ------------------------------------------------------------ FE handle --
struct pdmts_fem {
    pdmts_ctx *ctx = nullptr;
    int dim = 2, npe = 4;
    int64_t n = 0, ne = 0;
    std::vector<double> X;      // dim * n
    std::vector<int32_t> conn;  // ne * npe
    double E = 0, nu = 0, rho = 0, thick = 1;
    std::vector<int32_t> faces;       // nf * 2
    std::vector<double> face_tr;      // nf * dim
    std::vector<char> fixed;          // ndof flags (empty: no Dirichlet dof)
    // assembled operators (host copies of the alpha-weighted matrices)
    int W = 18;                       // ELL width (2D Q4: 9 nodes x 2 components)
    std::vector<int32_t> col;         // ndof * W
    std::vector<double> kval;         // ndof * W, stiffness K
    std::vector<double> mass;         // ndof, lumped mass
    std::vector<double> load;         // ndof, loads P
    double gersh = 0;                 // upper bound on the spectrum of M^-1 K
    // device; the ELL arrays are stored transposed (entry e of row i at
    // e * ndof + i) so that a warp's 32 rows read consecutive words
    DevArr<int32_t> d_col;
    DevArr<double> d_K, d_Keff, d_Minv, d_P;
    DevArr<double> d_u, d_v, d_a, d_ut, d_vt, d_b, d_r, d_d[2];
    DevArr<double> d_aw, d_bw;        // link correction: a_W and -G_FE^T lambda
    int64_t device_bytes = 0;
    // Chebyshev schedule for K_eff (depends on dt_FE); version counts changes
    double keff_dt = -1, cheb_theta = 0, cheb_delta = 0;
    std::vector<double> cheb_c1, cheb_c2;
    DevArr<double> d_cheb;            // the schedule on the device: c1[it], then c2[it]
    int64_t keff_version = 0;
    bool paired_rows = false;         // x and y rows of every node share one column list
    GraphSlot g_free, g_link;         // captured free step and link correction
    bool assembled = false;
    int64_t ndof() const { return (int64_t)dim * n; }

    template <typename T>
    int alloc(DevArr<T> &a, int64_t count)
    {
        release(a);
        a.p = (T *)ctx->dalloc(sizeof(T) * (size_t)std::max<int64_t>(count, 1));
        if (!a.p)
            return fail(PDMTS_ERR_NOMEM, "FE: device allocation of %lld bytes failed", (long long)(sizeof(T) * count));
        a.count = count;
        device_bytes += (int64_t)(sizeof(T) * std::max<int64_t>(count, 1));
        return PDMTS_OK;
    }
    template <typename T>
    void release(DevArr<T> &a)
    {
        if (a.p)
            ctx->dfree(a.p);
        a.p = nullptr;
        a.count = 0;
    }
    void release_all()
    {
        g_free.reset();
        g_link.reset();
        release(d_col); release(d_K); release(d_Keff); release(d_Minv); release(d_P);
        release(d_u); release(d_v); release(d_a); release(d_ut); release(d_vt); release(d_b); release(d_r);
        release(d_d[0]); release(d_d[1]); release(d_cheb); release(d_aw); release(d_bw);
    }
};

struct BandDesc {
    int axis;
    double lo, hi;
    int fe_side;
};

// Arlequin weight (Sec. 3.2) at a point: t = normalised distance to the FE
// boundary of the band; linear t, cubic t^3, constant 1/2; `outside` elsewhere.
static double arlequin_alpha(const std::vector<BandDesc> &bands, int kind, const double *x, double outside)
{
    for (const BandDesc &b : bands) {
        const double c = x[b.axis];
        if (c >= b.lo && c <= b.hi) {
            const double t = b.fe_side < 0 ? (b.hi - c) / (b.hi - b.lo) : (c - b.lo) / (b.hi - b.lo);
            if (kind == PDMTS_WEIGHT_CONSTANT)
                return 0.5;
            if (kind == PDMTS_WEIGHT_CUBIC)
                return t * t * t;
            return t;
        }
    }
    return outside;
}

// ------------------------------------------------------- arlequin handle --
struct pdmts_arl {
    pdmts_ctx *ctx = nullptr;
    pdmts_pd *pd = nullptr;
    pdmts_fem *fe = nullptr;
    int kind = PDMTS_WEIGHT_LINEAR;
    std::vector<BandDesc> bands;
    int64_t nl = 0, nlam = 0;        // multiplier nodes, multiplier components (dim * nl)
    std::vector<int32_t> lam_node;   // FE node of each multiplier node
    // G_FE rows (ELL, width 9 in 2D) per multiplier node; G_PD rows (CSR)
    int gfe_w = 9;
    std::vector<int32_t> gfe_col;
    std::vector<double> gfe_val;
    std::vector<int64_t> gpd_ptr;
    std::vector<int32_t> gpd_col;
    std::vector<double> gpd_val;
    // PD overlap nodes: element corners (multiplier ids) and shape values
    std::vector<int32_t> ov_node, ov_k;
    std::vector<double> ov_N;
    int64_t n_ov = 0;
    int corners = 4;                 // FE element corners per overlap PD node (4 in 2D, 8 in 3D)
    // device
    // G_FE^T by FE node (CSR): multiplier node and weight of each entry
    std::vector<int64_t> gfeT_ptr;
    std::vector<int32_t> gfeT_k;
    std::vector<double> gfeT_val;
    DevArr<int32_t> d_gfe_col, d_gpd_col, d_ov_node, d_ov_k, d_gfeT_k;
    DevArr<int64_t> d_gfeT_ptr;
    DevArr<double> d_gfe_val, d_gpd_val, d_ov_N, d_gfeT_val, d_Hfe, d_Hneg_inv, d_colbuf, d_lam0, d_lam, d_y;
    DevArr<double> d_B[4];          // block Chebyshev work (x, r, d0, d1)
    // FP32-bulk precision, even n_lambda: (-H)^-1 scaled by 2^-e (e = exponent
    // of its largest entry) as FP32 pairs, 2^e, and y as FP32 pairs
    int product_kind = PDMTS_PRODUCT_AUTO;
    DevArr<float2> d_Hinv_df, d_ydf;
    DevArr<double> d_df_scale;
    DevArr<unsigned long long> d_absmax;
    DevArr<int64_t> d_gpd_ptr;
    DevArr<uint8_t> d_near;         // bond words of nodes within (m + 1) delta of a band
    DevArr<unsigned long long> d_changed;
    // the PD free-chain interface force already holds G_PD^T lambda_0 (written
    // beside the link force of the lambda_m that becomes lambda_0)
    bool g0_ready = false;
    unsigned long long *h_changed = nullptr;  // pinned
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_flag = nullptr;
    cudaStream_t fe_stream = nullptr;
    bool H_valid = false, Hfe_valid = false, flag_pending = false;
    struct pdmts_batch *batch = nullptr;  // the batch this coupling belongs to, if any
    cusolverDnHandle_t solver = nullptr;  // dense Cholesky (or LU) for (-H)^-1
    int64_t lu_inverses = 0;              // inverses by LU
    // colouring of the multiplier columns for the link runs of build_H (per m):
    // colour c's unit multipliers and, per constraint row, the column it measures
    int colors_m = 0;
    std::vector<std::vector<int64_t>> color_cols;
    DevArr<double> d_units;           // colours x nlam
    DevArr<int32_t> d_owners;         // colours x nlam
    int64_t rebuilds = 0, colors = 0;
    int built_m = 0;
    std::vector<double> theta_free, theta_link;
    int64_t device_bytes = 0;

    template <typename T>
    int alloc(DevArr<T> &a, int64_t count)
    {
        release(a);
        a.p = (T *)ctx->dalloc(sizeof(T) * (size_t)std::max<int64_t>(count, 1));
        if (!a.p)
            return fail(PDMTS_ERR_NOMEM, "coupling: device allocation of %lld bytes failed",
                        (long long)(sizeof(T) * count));
        a.count = count;
        device_bytes += (int64_t)(sizeof(T) * std::max<int64_t>(count, 1));
        return PDMTS_OK;
    }
    template <typename T>
    void release(DevArr<T> &a)
    {
        if (a.p)
            ctx->dfree(a.p);
        a.p = nullptr;
        a.count = 0;
    }
    void release_all()
    {
        release(d_gfe_col); release(d_gpd_col); release(d_ov_node); release(d_ov_k);
        release(d_gfeT_k); release(d_gfeT_ptr); release(d_gfeT_val); release(d_Hfe);
        release(d_units); release(d_owners);
        release(d_gfe_val); release(d_gpd_val); release(d_ov_N); release(d_Hneg_inv);
        release(d_colbuf); release(d_lam0); release(d_lam); release(d_y);
        for (auto &b : d_B)
            release(b);
        release(d_gpd_ptr); release(d_near); release(d_changed);
        release(d_Hinv_df); release(d_ydf); release(d_df_scale); release(d_absmax);
    }
};

template <typename T>
static int h2d(T *dst, const std::vector<T> &src, cudaStream_t s)
{
    if (src.empty())
        return PDMTS_OK;
    PDMTS_CUDA_TRY(cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s));
    return PDMTS_OK;
}

// Row-major ELL (rows x W) to the transposed device layout (W x rows). The
// copy is synchronous: the host vector is a temporary.
template <typename T>
static int h2d_ell_t(T *dst, const std::vector<T> &src, int64_t rows, int W, cudaStream_t s)
{
    std::vector<T> t(src.size());
    for (int64_t i = 0; i < rows; ++i)
        for (int e = 0; e < W; ++e)
            t[(size_t)e * rows + i] = src[(size_t)i * W + e];
    PDMTS_TRY(h2d(dst, t, s));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(s));
    return PDMTS_OK;
}

// ------------------------------------------------------------ FE kernels --
// Per-dof operations, shared by the FE kernels of one subdomain and their
// batched forms (so both give the same bits).
__device__ __forceinline__ void fe_predict_dof(const int64_t i, const double *__restrict__ u,
                                               const double *__restrict__ v, const double *__restrict__ a,
                                               const double dt, const double beta, const double gamma,
                                               double *__restrict__ ut, double *__restrict__ vt)
{
    ut[i] = u[i] + dt * v[i] + (0.5 - beta) * dt * dt * a[i];
    vt[i] = v[i] + (1.0 - gamma) * dt * a[i];
}
// r = b - A x for row i of a transposed-ELL matrix (b may be null: r = -A x)
__device__ __forceinline__ double fe_residual_dof(const int64_t ndof, const int64_t i, const int W,
                                                  const int32_t *__restrict__ col, const double *__restrict__ val,
                                                  const double *__restrict__ x, const double *__restrict__ b)
{
    double ax = 0.0;
    for (int e = 0; e < W; ++e)
        ax += val[e * ndof + i] * x[col[e * ndof + i]];
    return (b ? b[i] : 0.0) - ax;
}
// One Chebyshev iteration for node ix (rows ix and nfe + ix share one column
// list): x += d, r -= A d, dn = c1 d + c2 M^-1 r (dn null on the last).
__device__ __forceinline__ void fe_cheb_node(const int64_t nfe, const int64_t ix, const int W,
                                             const int32_t *__restrict__ col, const double *__restrict__ val,
                                             const double *__restrict__ Minv, double *__restrict__ x,
                                             double *__restrict__ r, const double *__restrict__ d,
                                             double *__restrict__ dn, const double c1, const double c2)
{
    const int64_t ndof = 2 * nfe, iy = nfe + ix;
    double adx = 0.0, ady = 0.0;
    for (int e = 0; e < W; ++e) {
        const double dv = d[col[e * ndof + ix]];
        adx += val[e * ndof + ix] * dv;
        ady += val[e * ndof + iy] * dv;
    }
    x[ix] += d[ix];
    x[iy] += d[iy];
    const double rx = r[ix] - adx, ry = r[iy] - ady;
    r[ix] = rx;
    r[iy] = ry;
    if (dn) {
        dn[ix] = c1 * d[ix] + c2 * Minv[ix] * rx;
        dn[iy] = c1 * d[iy] + c2 * Minv[iy] * ry;
    }
}
__device__ __forceinline__ void fe_correct_dof(const int64_t i, const double *__restrict__ ut,
                                               const double *__restrict__ vt, const double *__restrict__ a,
                                               const double dt, const double beta, const double gamma,
                                               double *__restrict__ u, double *__restrict__ v)
{
    u[i] = ut[i] + beta * dt * dt * a[i];
    v[i] = vt[i] + gamma * dt * a[i];
}
// b = -G_FE^T lambda at dof i (component c of FE node `node`)
__device__ __forceinline__ double fe_gfe_lam_dof(const int c, const int64_t node, const int64_t nl,
                                                 const int64_t *__restrict__ ptr, const int32_t *__restrict__ kk,
                                                 const double *__restrict__ val, const double *__restrict__ lam)
{
    double s = 0.0;
    for (int64_t j = ptr[node]; j < ptr[node + 1]; ++j)
        s += val[j] * lam[(int64_t)c * nl + kk[j]];
    return -s;
}
__device__ __forceinline__ void fe_apply_link_dof(const int64_t i, const double *__restrict__ aw, const double dt,
                                                  const double beta, const double gamma, double *__restrict__ u,
                                                  double *__restrict__ v, double *__restrict__ a)
{
    const double w = aw[i];
    u[i] += beta * dt * dt * w;
    v[i] += gamma * dt * w;
    a[i] += w;
}

// Newmark predictor (Eq. 38 / Eq. 39): u~ = u + dt v + (1/2 - beta) dt^2 a,
// v~ = v + (1 - gamma) dt a, and b = P - K u~ needs the full u~ (second kernel).
__global__ void k_fe_predict(const int64_t ndof, const double *__restrict__ u, const double *__restrict__ v,
                             const double *__restrict__ a, const double dt, const double beta, const double gamma,
                             double *__restrict__ ut, double *__restrict__ vt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ndof)
        return;
    fe_predict_dof(i, u, v, a, dt, beta, gamma, ut, vt);
}

// y = b - A x (ELL rows), optionally d = y / (theta M)
__global__ void k_fe_residual(const int64_t ndof, const int W, const int32_t *__restrict__ col,
                              const double *__restrict__ val, const double *__restrict__ x,
                              const double *__restrict__ b, double *__restrict__ r, const double *__restrict__ Minv,
                              const double inv_theta, double *__restrict__ d)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ndof)
        return;
    const double ri = fe_residual_dof(ndof, i, W, col, val, x, b);
    r[i] = ri;
    if (d)
        d[i] = inv_theta * Minv[i] * ri;
}

// Rows of wide ELL matrices (Hex8: 81 entries) with G threads per row: lane
// `sub` of a row sums entries sub, sub + G, ...; the partial sums meet in a
// butterfly, whose pairwise sums are commutative, so every lane of the group
// holds the same bits. Used when the rows of a node do not share one column
// list (3D), where one thread per row leaves the SMs waiting on a chain of 81
// dependent FP64 products.
constexpr int kRowGroup = 8;
__device__ __forceinline__ double row_dot_group(const int64_t ndof, const int64_t i, const int W, const int sub,
                                                const int32_t *__restrict__ col, const double *__restrict__ val,
                                                const double *__restrict__ x, const bool act)
{
    double s = 0.0;
    if (act)
        for (int e = sub; e < W; e += kRowGroup)
            s += val[e * ndof + i] * x[col[e * ndof + i]];
#pragma unroll
    for (int o = kRowGroup / 2; o > 0; o >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// r = b - A x (and d = M^-1 r / theta) with kRowGroup threads per row.
__global__ void k_fe_residual_group(const int64_t ndof, const int W, const int32_t *__restrict__ col,
                                    const double *__restrict__ val, const double *__restrict__ x,
                                    const double *__restrict__ b, double *__restrict__ r,
                                    const double *__restrict__ Minv, const double inv_theta, double *__restrict__ d)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / kRowGroup;
    const int sub = (int)(t % kRowGroup);
    const bool act = i < ndof;
    const double ax = row_dot_group(ndof, act ? i : 0, W, sub, col, val, x, act);
    if (!act || sub != 0)
        return;
    const double ri = (b ? b[i] : 0.0) - ax;
    r[i] = ri;
    if (d)
        d[i] = inv_theta * Minv[i] * ri;
}

// One Chebyshev iteration for K_eff x = b preconditioned by the lumped mass,
// on nrhs column-major vectors (x += d; r -= K_eff d; d' = c1 d + c2 M^-1 r),
// with kRowGroup threads per row.
__global__ void k_cheb_iter_group(const int64_t ndof, const int nrhs, const int W, const int32_t *__restrict__ col,
                                  const double *__restrict__ val, const double *__restrict__ Minv,
                                  double *__restrict__ x, double *__restrict__ r, const double *__restrict__ d,
                                  double *__restrict__ dn, const double c1, const double c2)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = t / kRowGroup;
    const int sub = (int)(t % kRowGroup);
    const bool act = row < ndof * nrhs;
    const int64_t c = act ? row / ndof : 0, i = act ? row - c * ndof : 0;
    const double ad = row_dot_group(ndof, i, W, sub, col, val, d + c * ndof, act);
    if (!act || sub != 0)
        return;
    x[row] += d[row];
    const double rn = r[row] - ad;
    r[row] = rn;
    if (dn)
        dn[row] = c1 * d[row] + c2 * Minv[i] * rn;
}

// Newmark corrector: u = u~ + beta dt^2 a, v = v~ + gamma dt a.
__global__ void k_fe_correct_state(const int64_t ndof, const double *__restrict__ ut, const double *__restrict__ vt,
                                   const double *__restrict__ a, const double dt, const double beta,
                                   const double gamma, double *__restrict__ u, double *__restrict__ v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ndof)
        return;
    fe_correct_dof(i, ut, vt, a, dt, beta, gamma, u, v);
}

// b = -G_FE^T lambda on the FE dofs (gather over the transpose, so the sum
// order is fixed and the result reproducible).
__global__ void k_gfe_lam(const int64_t nfe, const int dim, const int64_t nl, const int64_t *__restrict__ ptr,
                          const int32_t *__restrict__ kk, const double *__restrict__ val,
                          const double *__restrict__ lam, double *__restrict__ b)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)dim * nfe)
        return;
    const int c = (int)(i / nfe);
    const int64_t node = i - (int64_t)c * nfe;
    b[i] = fe_gfe_lam_dof(c, node, nl, ptr, kk, val, lam);
}

// FE link correction (Eq. 47b with Newmark): u += beta dt^2 a_W,
// v += gamma dt a_W, a += a_W.
__global__ void k_fe_apply_link(const int64_t ndof, const double *__restrict__ aw, const double dt, const double beta,
                                const double gamma, double *__restrict__ u, double *__restrict__ v,
                                double *__restrict__ a)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ndof)
        return;
    fe_apply_link_dof(i, aw, dt, beta, gamma, u, v, a);
}

// Right-hand sides G_FE^T e_q for a batch of multiplier columns q0..q0+nb-1.
__global__ void k_gfe_rhs(const int64_t nfe, const int dim, const int64_t nl, const int gfe_w,
                          const int32_t *__restrict__ gcol, const double *__restrict__ gval, const int64_t q0,
                          const int nb, double *__restrict__ B)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nb)
        return;
    const int64_t q = q0 + t;
    const int c = (int)(q / nl);
    const int64_t k = q - (int64_t)c * nl;
    const int64_t ndof = (int64_t)dim * nfe;
    for (int e = 0; e < gfe_w; ++e) {
        const double g = gval[k * gfe_w + e];
        if (g != 0.0)
            B[t * ndof + (int64_t)c * nfe + gcol[k * gfe_w + e]] += g;
    }
}

// Columns q0..q0+nb-1 of H_FE = -gamma dt G_FE K_eff^-1 G_FE^T from the solved
// batch cols (column-major, ndof rows): H[r, q0 + c] for every row r.
__global__ void k_hfe_cols(const int64_t nfe, const int dim, const int64_t nl, const int gfe_w,
                           const int32_t *__restrict__ gcol, const double *__restrict__ gval, const int64_t q0,
                           const int nb, const double *__restrict__ cols, const double scale, double *__restrict__ H)
{
    const int64_t nlam = (int64_t)dim * nl, ndof = (int64_t)dim * nfe;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nlam * nb)
        return;
    const int64_t r = t / nb;
    const int c = (int)(t - r * nb);
    const int cd = (int)(r / nl);
    const int64_t k = r - (int64_t)cd * nl;
    const double *x = cols + (int64_t)c * ndof + (int64_t)cd * nfe;
    double s = 0.0;
    for (int e = 0; e < gfe_w; ++e)
        s += gval[k * gfe_w + e] * x[gcol[k * gfe_w + e]];
    H[r * nlam + q0 + c] = scale * s;
}

// H[r, owner[r]] += sign * y[r] for the rows a colored link run measures.
__global__ void k_scatter_color(const int64_t nlam, const int32_t *__restrict__ owner, const double *__restrict__ y,
                                const double sign, double *__restrict__ H)
{
    // blockIdx.y: one of several colours (owner rows and y of colour y at y nlam)
    owner += (int64_t)blockIdx.y * nlam;
    y += (int64_t)blockIdx.y * nlam;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nlam)
        return;
    const int32_t q = owner[r];
    if (q >= 0)
        H[r * nlam + q] += sign * y[r];
}

__global__ void k_negate(const int64_t n, double *__restrict__ A)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        A[i] = -A[i];
}

// ---- the multiplier product in FP32 pairs (FP32-bulk precision) ----------
// GB300 runs FP64 fused multiply-adds at 2 per SM per cycle, so the n^2 FP64
// FMAs of lambda = (-H)^-1 y bound the FP64 product rather than its bytes.
// With each entry split into an FP32 pair (hi + lo, the FP64 value to about
// 2^-48 relative) the product takes error-free FP32 products and compensated
// sums (Dekker's and Knuth's constructions): about 12 FP32 operations per
// entry, the same 8 bytes per entry, FP64-level accuracy (about 2^-40 of
// sum |a_j x_j|).

// largest |A_i| as the bit pattern of a non-negative double (ordered like
// the values)
__global__ void k_absmax_bits(const int64_t n, const double *__restrict__ A, unsigned long long *__restrict__ m)
{
    unsigned long long v = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v = max(v, (unsigned long long)__double_as_longlong(fabs(A[i])));
    for (int o = 16; o > 0; o >>= 1)
        v = max(v, (unsigned long long)__shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v)
        atomicMax(m, v);
}

// out_i = A_i 2^-e as an FP32 pair (the scaled value is exact in FP64, so hi
// and lo are its nearest FP32 value and the nearest FP32 value of the rest);
// e is the exponent of the largest |A_i|, and inv_scale = 2^e
__global__ void k_df_split(const int64_t n, const double *__restrict__ A, const unsigned long long *__restrict__ m,
                           float2 *__restrict__ out, double *__restrict__ inv_scale)
{
    const double mx = __longlong_as_double((long long)*m);
    const int e = mx > 0.0 ? ilogb(mx) : 0;
    const double sc = ldexp(1.0, -e);
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0)
        *inv_scale = ldexp(1.0, e);
    for (int64_t i = i0; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = A[i] * sc;
        const float hi = __double2float_rn(v);
        out[i] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

// (sh, sl) += (ah + al)(xh + xl): the product ah xh exactly as p + e (one
// FMA), the cross terms rounded once (al xl is below 2^-48 of the product),
// p added to sh by two-sum, the error terms gathered in sl
__device__ __forceinline__ void df_mac(float &sh, float &sl, const float ah, const float al, const float xh,
                                       const float xl)
{
    const float p = __fmul_rn(ah, xh);
    const float e = __fmaf_rn(ah, xh, -p);
    const float c = __fmaf_rn(ah, xl, __fmaf_rn(al, xh, e));
    const float t = __fadd_rn(sh, p);
    const float bp = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, c));
}

// y = inv_scale (A x) for a row-major n x n matrix of FP32 pairs (n even:
// rows start 16-byte aligned and two entries load as one float4), one warp per
// row, four 16-byte loads of A in flight per lane, two independent pair
// accumulators per lane, the lanes' sums added in FP64.
__global__ void k_gemv_df(const int64_t n, const float2 *__restrict__ A, const float2 *__restrict__ x,
                          const double *__restrict__ inv_scale, double *__restrict__ y)
{
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n)
        return;
    const float4 *a4 = reinterpret_cast<const float4 *>(A + row * n);
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const int64_t n2 = n / 2;
    float sh[2] = {0.f, 0.f}, sl[2] = {0.f, 0.f};
    int64_t j = lane;
    for (; j + 96 < n2; j += 128) {
        float4 a[4], v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            a[u] = __ldcs(a4 + j + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            v[u] = __ldg(x4 + j + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            df_mac(sh[u & 1], sl[u & 1], a[u].x, a[u].y, v[u].x, v[u].y);
            df_mac(sh[u & 1], sl[u & 1], a[u].z, a[u].w, v[u].z, v[u].w);
        }
    }
    for (; j < n2; j += 32) {
        const float4 a = __ldcs(a4 + j), v = __ldg(x4 + j);
        df_mac(sh[0], sl[0], a.x, a.y, v.x, v.y);
        df_mac(sh[0], sl[0], a.z, a.w, v.z, v.w);
    }
    double s = ((double)sh[0] + (double)sl[0]) + ((double)sh[1] + (double)sl[1]);
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0)
        y[row] = s * *inv_scale;
}

// y = scale A x for a row-major n x n matrix, one warp per row. The matrix
// is read once per call from DRAM (it does not fit in L2 beside the PD
// state), so each lane keeps four independent 16-byte loads in flight: a
// warp streams 2 KB at a time and the ~26 warps an SM holds cover the memory
// latency. Even n (rows 16-byte aligned) takes the paired loads; odd n the
// plain loop.
__global__ void k_gemv_rows(const int64_t n, const double *__restrict__ A, const double *__restrict__ x,
                            const double scale, double *__restrict__ y)
{
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n)
        return;
    double s = 0.0;
    if ((n & 1) == 0) {
        const double2 *a2 = reinterpret_cast<const double2 *>(A + row * n);
        const double2 *x2 = reinterpret_cast<const double2 *>(x);
        const int64_t n2 = n / 2;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        int64_t j = lane;
        for (; j + 96 < n2; j += 128) {
            double2 p[4], q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                p[u] = __ldcs(a2 + j + 32 * u);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                q[u] = __ldg(x2 + j + 32 * u);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                acc[u] = fma(p[u].y, q[u].y, fma(p[u].x, q[u].x, acc[u]));
        }
        for (; j < n2; j += 32) {
            const double2 p = __ldcs(a2 + j), q = __ldg(x2 + j);
            acc[0] = fma(p.y, q.y, fma(p.x, q.x, acc[0]));
        }
        s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    } else {
        for (int64_t j = lane; j < n; j += 32)
            s += A[row * n + j] * x[j];
    }
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0)
        y[row] = scale * s;
}

// k_cheb_iter with one thread per FE node and right-hand side: the node's x
// and y rows (dofs i and nfe + i) have the same column list, so every value of
// d a row needs is read once for both rows. Per row the same operations in the
// same order as k_cheb_iter.
__global__ void k_cheb_iter_node(const int64_t nfe, const int nrhs, const int W, const int32_t *__restrict__ col,
                                 const double *__restrict__ val, const double *__restrict__ Minv,
                                 double *__restrict__ x, double *__restrict__ r, const double *__restrict__ d,
                                 double *__restrict__ dn, const double c1, const double c2)
{
    // launched as a programmatic dependent of the previous kernel of the
    // solve: wait for its results, then let the next iteration's CTAs take
    // SM slots as they free up (no-ops when launched plainly)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nfe * nrhs)
        return;
    const int64_t ndof = 2 * nfe;
    const int64_t c = t / nfe, ix = t - c * nfe;
    fe_cheb_node(nfe, ix, W, col, val, Minv, x + c * ndof, r + c * ndof, d + c * ndof,
                 dn ? dn + c * ndof : nullptr, c1, c2);
}

static inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------- batched FE solves --
// The FE free step and FE correction of many subdomains at once: each CTA
// takes 256 nodes of one subdomain (a block table {subdomain, first node}),
// each thread both rows of a node, with the per-dof operations above.
struct FeDev {
    int64_t nfe, nl;
    int W, it;
    const int32_t *col;
    const double *K, *Keff, *Minv, *P, *cheb;
    double *u, *v, *a, *ut, *vt, *b, *r, *d0, *d1, *aw, *bw;
    double inv_theta, dt, beta, gamma;
    const int64_t *gT_ptr;
    const int32_t *gT_k;
    const double *gT_val, *lam;
};

__global__ void k_feb_predict(const FeDev *__restrict__ M, const int2 *__restrict__ blk)
{
    const int2 q = blk[blockIdx.x];
    const FeDev &F = M[q.x];
    const int64_t node = (int64_t)q.y + threadIdx.x;
    if (node >= F.nfe)
        return;
    for (int c = 0; c < 2; ++c)
        fe_predict_dof(c * F.nfe + node, F.u, F.v, F.a, F.dt, F.beta, F.gamma, F.ut, F.vt);
}

// b = P - K u~, then r = b - K_eff a (warm start) and d0 = M^-1 r / theta
__global__ void k_feb_residual(const FeDev *__restrict__ M, const int2 *__restrict__ blk)
{
    const int2 q = blk[blockIdx.x];
    const FeDev &F = M[q.x];
    const int64_t node = (int64_t)q.y + threadIdx.x;
    if (node >= F.nfe)
        return;
    const int64_t ndof = 2 * F.nfe;
    for (int c = 0; c < 2; ++c) {
        const int64_t i = c * F.nfe + node;
        F.b[i] = fe_residual_dof(ndof, i, F.W, F.col, F.K, F.ut, F.P);
        const double ri = fe_residual_dof(ndof, i, F.W, F.col, F.Keff, F.a, F.b);
        F.r[i] = ri;
        F.d0[i] = F.inv_theta * F.Minv[i] * ri;
    }
}

// b = -G_FE^T lambda, x = a_W = 0, r = b (the residual at the zero start), d0
__global__ void k_feb_link_init(const FeDev *__restrict__ M, const int2 *__restrict__ blk)
{
    const int2 q = blk[blockIdx.x];
    const FeDev &F = M[q.x];
    const int64_t node = (int64_t)q.y + threadIdx.x;
    if (node >= F.nfe)
        return;
    for (int c = 0; c < 2; ++c) {
        const int64_t i = c * F.nfe + node;
        const double bi = fe_gfe_lam_dof(c, node, F.nl, F.gT_ptr, F.gT_k, F.gT_val, F.lam);
        F.bw[i] = bi;
        F.aw[i] = 0.0;
        const double ri = bi - 0.0;  // K_eff times the zero start is +0 in every sum
        F.r[i] = ri;
        F.d0[i] = F.inv_theta * F.Minv[i] * ri;
    }
}

__global__ void k_feb_cheb(const FeDev *__restrict__ M, const int2 *__restrict__ blk, const int k, const int link)
{
    // a programmatic dependent of the previous kernel of the solve (see
    // k_cheb_iter_node)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int2 q = blk[blockIdx.x];
    const FeDev &F = M[q.x];
    const int64_t node = (int64_t)q.y + threadIdx.x;
    if (node >= F.nfe || k >= F.it)
        return;
    const double *d = (k & 1) ? F.d1 : F.d0;
    double *dn = (k == F.it - 1) ? nullptr : ((k & 1) ? F.d0 : F.d1);
    fe_cheb_node(F.nfe, node, F.W, F.col, F.Keff, F.Minv, link ? F.aw : F.a, F.r, d, dn, F.cheb[k],
                 F.cheb[F.it + k]);
}

__global__ void k_feb_finish(const FeDev *__restrict__ M, const int2 *__restrict__ blk, const int link)
{
    const int2 q = blk[blockIdx.x];
    const FeDev &F = M[q.x];
    const int64_t node = (int64_t)q.y + threadIdx.x;
    if (node >= F.nfe)
        return;
    for (int c = 0; c < 2; ++c) {
        const int64_t i = c * F.nfe + node;
        if (link)
            fe_apply_link_dof(i, F.aw, F.dt, F.beta, F.gamma, F.u, F.v, F.a);
        else
            fe_correct_dof(i, F.ut, F.vt, F.a, F.dt, F.beta, F.gamma, F.u, F.v);
    }
}

// ------------------------------------------------------- FE assembly ------
// alpha-weighted Q4 plane-stress element stiffness and lumped mass with 2 x 2
// Gauss points (Eq. 24 ff., Eq. 34).
static void q4_element(const pdmts_fem *fe, const std::vector<BandDesc> &bands, int kind, int64_t e, double ke[8][8],
                       double me[4])
{
    const double g = 1.0 / std::sqrt(3.0);
    const double nat[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
    const double c = fe->E / (1.0 - fe->nu * fe->nu);
    const double D[3][3] = {{c, c * fe->nu, 0}, {c * fe->nu, c, 0}, {0, 0, c * (1.0 - fe->nu) / 2.0}};
    double xe[4][2];
    for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 2; ++d)
            xe[a][d] = fe->X[(size_t)d * fe->n + fe->conn[(size_t)e * 4 + a]];
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b)
            ke[a][b] = 0.0;
    for (int a = 0; a < 4; ++a)
        me[a] = 0.0;
    for (int gi = 0; gi < 2; ++gi)
        for (int gj = 0; gj < 2; ++gj) {
            const double xi = gi ? g : -g, et = gj ? g : -g;
            double N[4], dxi[4], det_[4];
            for (int a = 0; a < 4; ++a) {
                N[a] = 0.25 * (1 + nat[a][0] * xi) * (1 + nat[a][1] * et);
                dxi[a] = 0.25 * nat[a][0] * (1 + nat[a][1] * et);
                det_[a] = 0.25 * nat[a][1] * (1 + nat[a][0] * xi);
            }
            double J[2][2] = {{0, 0}, {0, 0}}, xg[2] = {0, 0};
            for (int a = 0; a < 4; ++a) {
                J[0][0] += dxi[a] * xe[a][0];
                J[0][1] += dxi[a] * xe[a][1];
                J[1][0] += det_[a] * xe[a][0];
                J[1][1] += det_[a] * xe[a][1];
                xg[0] += N[a] * xe[a][0];
                xg[1] += N[a] * xe[a][1];
            }
            const double detJ = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            double dNx[4], dNy[4];
            for (int a = 0; a < 4; ++a) {
                dNx[a] = (J[1][1] * dxi[a] - J[0][1] * det_[a]) / detJ;
                dNy[a] = (-J[1][0] * dxi[a] + J[0][0] * det_[a]) / detJ;
            }
            double B[3][8];
            for (int a = 0; a < 4; ++a) {
                B[0][2 * a] = dNx[a]; B[0][2 * a + 1] = 0;
                B[1][2 * a] = 0;      B[1][2 * a + 1] = dNy[a];
                B[2][2 * a] = dNy[a]; B[2][2 * a + 1] = dNx[a];
            }
            const double al = arlequin_alpha(bands, kind, xg, 1.0);
            const double w = al * detJ * fe->thick;
            for (int a = 0; a < 8; ++a)
                for (int b = 0; b < 8; ++b) {
                    double s = 0.0;
                    for (int p = 0; p < 3; ++p)
                        for (int q = 0; q < 3; ++q)
                            s += B[p][a] * D[p][q] * B[q][b];
                    ke[a][b] += w * s;
                }
            for (int a = 0; a < 4; ++a)
                me[a] += al * fe->rho * N[a] * detJ * fe->thick;
        }
}

// Hex8 corners in natural coordinates: the bottom face (zeta = -1)
// counter-clockwise seen from +z, then the top face in the same order.
static const double kHexNat[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                     {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

// Trilinear shape functions and their natural derivatives at (xi, eta, zeta).
static void hex8_shape(const double xi, const double et, const double ze, double N[8], double dN[8][3])
{
    for (int a = 0; a < 8; ++a) {
        const double p = 1 + kHexNat[a][0] * xi, q = 1 + kHexNat[a][1] * et, r = 1 + kHexNat[a][2] * ze;
        N[a] = 0.125 * p * q * r;
        dN[a][0] = 0.125 * kHexNat[a][0] * q * r;
        dN[a][1] = 0.125 * kHexNat[a][1] * p * r;
        dN[a][2] = 0.125 * kHexNat[a][2] * p * q;
    }
}

// Jacobian of the Hex8 map at a point, its determinant, the physical shape
// derivatives and the physical position.
static double hex8_map(const double xe[8][3], const double N[8], const double dN[8][3], double dNx[8][3],
                       double xg[3])
{
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int d = 0; d < 3; ++d)
        xg[d] = 0.0;
    for (int a = 0; a < 8; ++a)
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j)
                J[i][j] += dN[a][i] * xe[a][j];  // J[i][j] = d x_j / d xi_i
            xg[i] += N[a] * xe[a][i];
        }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    double Ji[3][3];  // inverse of J
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    // d N / d x_j = sum_i (J^-1)[j][i] d N / d xi_i
    for (int a = 0; a < 8; ++a)
        for (int j = 0; j < 3; ++j)
            dNx[a][j] = Ji[j][0] * dN[a][0] + Ji[j][1] * dN[a][1] + Ji[j][2] * dN[a][2];
    return det;
}

// alpha-weighted Hex8 isotropic linear-elastic element stiffness and lumped
// mass with 2 x 2 x 2 Gauss points (Eq. 24 ff. in 3D, Eq. 34). Local dof
// order: node-major, a * 3 + component.
static void hex8_element(const pdmts_fem *fe, const std::vector<BandDesc> &bands, int kind, int64_t e,
                         double ke[24][24], double me[8])
{
    const double g = 1.0 / std::sqrt(3.0);
    const double lam = fe->E * fe->nu / ((1.0 + fe->nu) * (1.0 - 2.0 * fe->nu));
    const double mu = fe->E / (2.0 * (1.0 + fe->nu));
    double D[6][6] = {};
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            D[i][j] = lam;
        D[i][i] = lam + 2.0 * mu;
        D[3 + i][3 + i] = mu;
    }
    double xe[8][3];
    for (int a = 0; a < 8; ++a)
        for (int d = 0; d < 3; ++d)
            xe[a][d] = fe->X[(size_t)d * fe->n + fe->conn[(size_t)e * 8 + a]];
    for (int a = 0; a < 24; ++a)
        for (int b = 0; b < 24; ++b)
            ke[a][b] = 0.0;
    for (int a = 0; a < 8; ++a)
        me[a] = 0.0;
    for (int gi = 0; gi < 2; ++gi)
        for (int gj = 0; gj < 2; ++gj)
            for (int gk = 0; gk < 2; ++gk) {
                double N[8], dN[8][3], dNx[8][3], xg[3];
                hex8_shape(gi ? g : -g, gj ? g : -g, gk ? g : -g, N, dN);
                const double detJ = hex8_map(xe, N, dN, dNx, xg);
                // strains (xx, yy, zz, yz, xz, xy), engineering shears
                double B[6][24] = {};
                for (int a = 0; a < 8; ++a) {
                    const double *d = dNx[a];
                    B[0][3 * a] = d[0];
                    B[1][3 * a + 1] = d[1];
                    B[2][3 * a + 2] = d[2];
                    B[3][3 * a + 1] = d[2]; B[3][3 * a + 2] = d[1];
                    B[4][3 * a] = d[2];     B[4][3 * a + 2] = d[0];
                    B[5][3 * a] = d[1];     B[5][3 * a + 1] = d[0];
                }
                const double al = arlequin_alpha(bands, kind, xg, 1.0);
                const double w = al * detJ;
                double DB[6][24];
                for (int p = 0; p < 6; ++p)
                    for (int b = 0; b < 24; ++b) {
                        double t = 0.0;
                        for (int q = 0; q < 6; ++q)
                            t += D[p][q] * B[q][b];
                        DB[p][b] = t;
                    }
                for (int a = 0; a < 24; ++a)
                    for (int b = 0; b < 24; ++b) {
                        double t = 0.0;
                        for (int p = 0; p < 6; ++p)
                            t += B[p][a] * DB[p][b];
                        ke[a][b] += w * t;
                    }
                for (int a = 0; a < 8; ++a)
                    me[a] += al * fe->rho * N[a] * detJ;
            }
}

// Largest eigenvalue of the symmetric n x n matrix a (row-major, cyclic
// Jacobi rotations; a is overwritten).
static double sym_max_eig(std::vector<double> &A, const int n)
{
    auto a = [&](int i, int j) -> double & { return A[(size_t)i * n + j]; };
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < n; ++i) {
            diag += a(i, i) * a(i, i);
            for (int j = i + 1; j < n; ++j)
                off += a(i, j) * a(i, j);
        }
        if (off <= 1e-30 * diag)
            break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (a(p, q) == 0.0)
                    continue;
                const double th = 0.5 * (a(q, q) - a(p, p)) / a(p, q);
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = a(k, p), akq = a(k, q);
                    a(k, p) = c * akp - sn * akq;
                    a(k, q) = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = a(p, k), aqk = a(q, k);
                    a(p, k) = c * apk - sn * aqk;
                    a(q, k) = sn * apk + c * aqk;
                }
            }
    }
    double mx = a(0, 0);
    for (int i = 1; i < n; ++i)
        mx = std::max(mx, a(i, i));
    return mx;
}

static int fe_assemble(pdmts_fem *fe, const std::vector<BandDesc> &bands, int kind)
{
    const int64_t n = fe->n, ndof = fe->ndof();
    std::vector<std::map<int32_t, double>> rows((size_t)ndof);
    fe->mass.assign((size_t)ndof, 0.0);
    // element bound on the spectrum of M^-1 K: with K = sum K_e and the lumped
    // M = sum M_e, x'Kx / x'Mx <= max_e of the largest eigenvalue of
    // M_e^-1/2 K_e M_e^-1/2 (every term is a ratio of non-negative sums)
    double elem_bound = 0.0;
    const int dim = fe->dim, npe = fe->npe, nle = dim * npe;  // local dofs: node-major, a * dim + d
    std::vector<double> K((size_t)nle * nle), sk((size_t)nle * nle);
    double me[8];
    for (int64_t e = 0; e < fe->ne; ++e) {
        if (dim == 2) {
            double ke[8][8];
            q4_element(fe, bands, kind, e, ke, me);
            for (int a = 0; a < 8; ++a)
                for (int b = 0; b < 8; ++b)
                    K[(size_t)a * nle + b] = ke[a][b];
        } else {
            static thread_local double ke[24][24];
            hex8_element(fe, bands, kind, e, ke, me);
            for (int a = 0; a < 24; ++a)
                for (int b = 0; b < 24; ++b)
                    K[(size_t)a * nle + b] = ke[a][b];
        }
        bool massive = true;
        for (int a = 0; a < npe; ++a)
            massive = massive && me[a] > 0;
        if (massive) {
            for (int a = 0; a < nle; ++a)
                for (int b = 0; b < nle; ++b)
                    sk[(size_t)a * nle + b] = K[(size_t)a * nle + b] / std::sqrt(me[a / dim] * me[b / dim]);
            elem_bound = std::max(elem_bound, sym_max_eig(sk, nle));
        }
        int64_t dof[24];
        for (int a = 0; a < npe; ++a) {
            const int64_t node = fe->conn[(size_t)e * npe + a];
            for (int d = 0; d < dim; ++d) {
                dof[dim * a + d] = d * n + node;
                fe->mass[(size_t)(d * n + node)] += me[a];
            }
        }
        for (int a = 0; a < nle; ++a)
            for (int b = 0; b < nle; ++b)
                rows[(size_t)dof[a]][(int32_t)dof[b]] += K[(size_t)a * nle + b];
    }
    // Dirichlet dofs (held at zero): their rows and columns keep only the
    // diagonal, so K u, the residual and every iterate vanish there exactly and
    // the free dofs see the reduced system; the entries stay in place (as
    // zeros) so the x and y rows of a node keep one column list
    if (!fe->fixed.empty())
        for (int64_t i = 0; i < ndof; ++i)
            for (auto &kv : rows[(size_t)i])
                if (kv.first != i && (fe->fixed[(size_t)i] || fe->fixed[(size_t)kv.first]))
                    kv.second = 0.0;
    int W = 0;
    for (auto &r : rows)
        W = std::max<int>(W, (int)r.size());
    fe->W = std::max(W, 1);
    fe->col.assign((size_t)ndof * fe->W, 0);
    fe->kval.assign((size_t)ndof * fe->W, 0.0);
    double gersh = 0.0;
    for (int64_t i = 0; i < ndof; ++i) {
        if (!(fe->mass[(size_t)i] > 0))
            return fail(PDMTS_ERR_MASS, "FE dof %lld has no mass (alpha vanishes on its support)", (long long)i);
        int e = 0;
        double rs = 0.0;
        for (auto &kv : rows[(size_t)i]) {
            fe->col[(size_t)i * fe->W + e] = kv.first;
            fe->kval[(size_t)i * fe->W + e] = kv.second;
            rs += std::fabs(kv.second);
            ++e;
        }
        // padding (zero values) repeats the node's x dof in both of its rows, so
        // the x and y rows of a node keep one column list
        for (; e < fe->W; ++e)
            fe->col[(size_t)i * fe->W + e] = (int32_t)(i % n);
        gersh = std::max(gersh, rs / fe->mass[(size_t)i]);
    }
    fe->paired_rows = dim == 2;
    for (int64_t i = 0; i < n && fe->paired_rows; ++i)
        for (int e = 0; e < fe->W; ++e)
            if (fe->col[(size_t)i * fe->W + e] != fe->col[(size_t)(n + i) * fe->W + e]) {
                fe->paired_rows = false;
                break;
            }
    // both are upper bounds; the element bound is the tighter on Q4 meshes
    // (a relative margin covers the rounding of the rotations)
    fe->gersh = elem_bound > 0 ? std::min(gersh, elem_bound * (1.0 + 1e-9)) : gersh;
    // consistent traction loads, weighted by alpha at the face midpoint (Eq. 34):
    // 2D segments (2 nodes, length x thickness), 3D planar quads (4 nodes,
    // area from the diagonals), the load shared equally by the face's nodes
    fe->load.assign((size_t)ndof, 0.0);
    if (dim == 3) {
        const int64_t nf3 = (int64_t)fe->faces.size() / 4;
        for (int64_t f = 0; f < nf3; ++f) {
            const int32_t *fn = &fe->faces[(size_t)4 * f];
            double d1[3], d2[3], xm[3] = {0, 0, 0};
            for (int d = 0; d < 3; ++d) {
                d1[d] = fe->X[(size_t)d * n + fn[2]] - fe->X[(size_t)d * n + fn[0]];
                d2[d] = fe->X[(size_t)d * n + fn[3]] - fe->X[(size_t)d * n + fn[1]];
                for (int a = 0; a < 4; ++a)
                    xm[d] += 0.25 * fe->X[(size_t)d * n + fn[a]];
            }
            const double cx = d1[1] * d2[2] - d1[2] * d2[1], cy = d1[2] * d2[0] - d1[0] * d2[2],
                         cz = d1[0] * d2[1] - d1[1] * d2[0];
            const double area = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
            const double al = arlequin_alpha(bands, kind, xm, 1.0);
            for (int a = 0; a < 4; ++a)
                for (int d = 0; d < 3; ++d)
                    fe->load[(size_t)(d * n + fn[a])] += al * fe->face_tr[(size_t)f * 3 + d] * area / 4.0;
        }
    }
    const int64_t nf = dim == 2 ? (int64_t)fe->faces.size() / 2 : 0;
    for (int64_t f = 0; f < nf; ++f) {
        const int64_t i = fe->faces[(size_t)2 * f], j = fe->faces[(size_t)2 * f + 1];
        const double dx = fe->X[(size_t)j] - fe->X[(size_t)i], dy = fe->X[(size_t)n + j] - fe->X[(size_t)n + i];
        const double L = std::sqrt(dx * dx + dy * dy);
        const double xm[2] = {0.5 * (fe->X[(size_t)i] + fe->X[(size_t)j]),
                              0.5 * (fe->X[(size_t)n + i] + fe->X[(size_t)n + j])};
        const double al = arlequin_alpha(bands, kind, xm, 1.0);
        for (int64_t node : {i, j})
            for (int d = 0; d < 2; ++d)
                fe->load[(size_t)(d * n + node)] += al * fe->face_tr[(size_t)f * 2 + d] * L * fe->thick / 2.0;
    }
    if (!fe->fixed.empty())
        for (int64_t i = 0; i < ndof; ++i)
            if (fe->fixed[(size_t)i])
                fe->load[(size_t)i] = 0.0;
    cudaStream_t s = fe->ctx->stream;
    PDMTS_TRY(fe->alloc(fe->d_col, ndof * fe->W));
    PDMTS_TRY(fe->alloc(fe->d_K, ndof * fe->W));
    PDMTS_TRY(fe->alloc(fe->d_Keff, ndof * fe->W));
    PDMTS_TRY(fe->alloc(fe->d_Minv, ndof));
    PDMTS_TRY(fe->alloc(fe->d_P, ndof));
    std::vector<double> minv((size_t)ndof);
    for (int64_t i = 0; i < ndof; ++i)
        minv[(size_t)i] = 1.0 / fe->mass[(size_t)i];
    PDMTS_TRY(h2d_ell_t(fe->d_col.p, fe->col, ndof, fe->W, s));
    PDMTS_TRY(h2d_ell_t(fe->d_K.p, fe->kval, ndof, fe->W, s));
    PDMTS_TRY(h2d(fe->d_Minv.p, minv, s));
    PDMTS_TRY(h2d(fe->d_P.p, fe->load, s));
    for (DevArr<double> *a : {&fe->d_u, &fe->d_v, &fe->d_a, &fe->d_ut, &fe->d_vt, &fe->d_b, &fe->d_r, &fe->d_d[0],
                              &fe->d_d[1], &fe->d_aw, &fe->d_bw}) {
        PDMTS_TRY(fe->alloc(*a, ndof));
        PDMTS_CUDA_TRY(cudaMemsetAsync(a->p, 0, sizeof(double) * ndof, s));
    }
    // initial acceleration from the equation of motion with u = 0, lambda_0 = 0
    std::vector<double> a0((size_t)ndof);
    for (int64_t i = 0; i < ndof; ++i)
        a0[(size_t)i] = fe->load[(size_t)i] / fe->mass[(size_t)i];
    PDMTS_TRY(h2d(fe->d_a.p, a0, s));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(s));
    fe->assembled = true;
    fe->keff_dt = -1;
    fe->g_free.reset();
    fe->g_link.reset();
    return PDMTS_OK;
}

// K_eff = M + beta dt^2 K and its Chebyshev schedule. The spectrum of
// M^-1 K_eff lies in [1, 1 + beta dt^2 rho(M^-1 K)] with an upper bound for
// rho; the iteration count bounds the error by 1e-14 of the initial error.
static int fe_prepare_keff(pdmts_fem *fe, double dt, double beta)
{
    if (fe->keff_dt == dt)
        return PDMTS_OK;
    const int64_t ndof = fe->ndof();
    std::vector<double> keff(fe->kval);
    for (int64_t i = 0; i < ndof; ++i) {
        for (int e = 0; e < fe->W; ++e)
            keff[(size_t)i * fe->W + e] *= beta * dt * dt;
        bool found = false;
        for (int e = 0; e < fe->W; ++e)
            if (fe->col[(size_t)i * fe->W + e] == (int32_t)i && !found) {
                keff[(size_t)i * fe->W + e] += fe->mass[(size_t)i];
                found = true;
            }
        if (!found)
            return fail(PDMTS_ERR_STATE, "FE matrix row %lld lacks a diagonal entry", (long long)i);
    }
    PDMTS_TRY(h2d_ell_t(fe->d_Keff.p, keff, ndof, fe->W, fe->ctx->stream));
    const double lmin = 1.0, lmax = 1.0 + beta * dt * dt * fe->gersh;
    fe->cheb_theta = 0.5 * (lmax + lmin);
    fe->cheb_delta = 0.5 * (lmax - lmin);
    const double kappa = lmax / lmin;
    const double q = (std::sqrt(kappa) - 1.0) / (std::sqrt(kappa) + 1.0);
    int it = q > 0 ? (int)std::ceil(std::log(2.0 / 1e-14) / std::log(1.0 / q)) + 2 : 1;
    it = std::max(it, 1);
    fe->cheb_c1.assign((size_t)it, 0.0);
    fe->cheb_c2.assign((size_t)it, 0.0);
    const double sigma = fe->cheb_theta / std::max(fe->cheb_delta, 1e-300);
    double rho = 1.0 / sigma;
    for (int k = 0; k < it; ++k) {
        const double rn = 1.0 / (2.0 * sigma - rho);
        fe->cheb_c1[(size_t)k] = rn * rho;
        fe->cheb_c2[(size_t)k] = 2.0 * rn / std::max(fe->cheb_delta, 1e-300);
        rho = rn;
    }
    std::vector<double> sched(fe->cheb_c1);
    sched.insert(sched.end(), fe->cheb_c2.begin(), fe->cheb_c2.end());
    PDMTS_TRY(fe->alloc(fe->d_cheb, 2 * (int64_t)it));
    PDMTS_TRY(h2d(fe->d_cheb.p, sched, fe->ctx->stream));
    fe->keff_dt = dt;
    fe->keff_version += 1;
    PDMTS_CUDA_TRY(cudaStreamSynchronize(fe->ctx->stream));
    return PDMTS_OK;
}

// x <- K_eff^-1 b on nrhs column-major vectors (x holds the initial guess).
// Work arrays r, d0, d1 have the same shape.
static int fe_cheb_solve(pdmts_fem *fe, int nrhs, double *x, const double *b, double *r, double *d0, double *d1,
                         cudaStream_t s, int64_t *launches)
{
    const int64_t ndof = fe->ndof();
    const int64_t tot = ndof * nrhs;
    for (int c = 0; c < nrhs; ++c) {
        if (fe->paired_rows)
            k_fe_residual<<<blocks(ndof, 512), 512, 0, s>>>(ndof, fe->W, fe->d_col.p, fe->d_Keff.p, x + c * ndof,
                                                      b + c * ndof, r + c * ndof, fe->d_Minv.p, 1.0 / fe->cheb_theta,
                                                      d0 + c * ndof);
        else
            k_fe_residual_group<<<blocks(ndof * kRowGroup), 256, 0, s>>>(
                ndof, fe->W, fe->d_col.p, fe->d_Keff.p, x + c * ndof, b + c * ndof, r + c * ndof, fe->d_Minv.p,
                1.0 / fe->cheb_theta, d0 + c * ndof);
        ++*launches;
    }
    double *d = d0, *dn = d1;
    const int it = (int)fe->cheb_c1.size();
    for (int k = 0; k < it; ++k) {
        const bool last = k == it - 1;
        const double c1 = fe->cheb_c1[(size_t)k], c2 = fe->cheb_c2[(size_t)k];
        if (fe->paired_rows) {
            // each iteration a programmatic dependent of the kernel before it
            // (2D: the small solve no longer trails the PD chain beside it);
            // CTAs of 512 threads (16K registers): a resident FE CTA takes the
            // register share of one PD lattice CTA, like a 256-thread one, for
            // twice the work
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(blocks(fe->n * nrhs, 512));
            cfg.blockDim = dim3(512);
            cfg.stream = s;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            PDMTS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_cheb_iter_node, (int64_t)fe->n, nrhs, fe->W,
                                              (const int32_t *)fe->d_col.p, (const double *)fe->d_Keff.p,
                                              (const double *)fe->d_Minv.p, x, r, (const double *)d,
                                              last ? nullptr : dn, c1, c2));
        } else {
            // plain launches: the 3D solve, placed as eagerly, took SM slots
            // from the PD chain on the step's critical path (1.41 -> 1.57 ms)
            k_cheb_iter_group<<<blocks(tot * kRowGroup), 256, 0, s>>>(
                ndof, nrhs, fe->W, fe->d_col.p, fe->d_Keff.p, fe->d_Minv.p, x, r, d, last ? nullptr : dn, c1, c2);
        }
        ++*launches;
        std::swap(d, dn);
    }
    PDMTS_CUDA_TRY(cudaGetLastError());
    return PDMTS_OK;
}

// Free FE step (Eq. 47a + Eq. 39): predictor, K_eff a = P - K u~, corrector.
static int fe_free_enqueue(pdmts_fem *fe, double dt, double beta, double gamma, cudaStream_t s, int64_t *launches)
{
    const int64_t ndof = fe->ndof();
    k_fe_predict<<<blocks(ndof), 256, 0, s>>>(ndof, fe->d_u.p, fe->d_v.p, fe->d_a.p, dt, beta, gamma, fe->d_ut.p,
                                              fe->d_vt.p);
    if (fe->paired_rows)
        k_fe_residual<<<blocks(ndof, 512), 512, 0, s>>>(ndof, fe->W, fe->d_col.p, fe->d_K.p, fe->d_ut.p, fe->d_P.p,
                                                   fe->d_b.p, nullptr, 0.0, nullptr);
    else
        k_fe_residual_group<<<blocks(ndof * kRowGroup), 256, 0, s>>>(ndof, fe->W, fe->d_col.p, fe->d_K.p, fe->d_ut.p,
                                                                     fe->d_P.p, fe->d_b.p, nullptr, 0.0, nullptr);
    *launches += 2;
    // warm start from the previous acceleration (kept in d_a)
    PDMTS_TRY(fe_cheb_solve(fe, 1, fe->d_a.p, fe->d_b.p, fe->d_r.p, fe->d_d[0].p, fe->d_d[1].p, s, launches));
    k_fe_correct_state<<<blocks(ndof), 256, 0, s>>>(ndof, fe->d_ut.p, fe->d_vt.p, fe->d_a.p, dt, beta, gamma,
                                                    fe->d_u.p, fe->d_v.p);
    ++*launches;
    PDMTS_CUDA_TRY(cudaGetLastError());
    return PDMTS_OK;
}

// Launch arguments an FE graph depends on: step scalars, the K_eff schedule
// version and every FE array pointer.
static std::vector<uint64_t> fe_graph_key(const pdmts_fem *fe, double dt, double beta, double gamma)
{
    std::vector<uint64_t> k{key_bits(dt), key_bits(beta), key_bits(gamma), (uint64_t)fe->keff_version};
    for (const void *p : {(const void *)fe->d_col.p, (const void *)fe->d_K.p, (const void *)fe->d_Keff.p,
                          (const void *)fe->d_Minv.p, (const void *)fe->d_P.p, (const void *)fe->d_u.p,
                          (const void *)fe->d_v.p, (const void *)fe->d_a.p, (const void *)fe->d_ut.p,
                          (const void *)fe->d_vt.p, (const void *)fe->d_b.p, (const void *)fe->d_r.p,
                          (const void *)fe->d_d[0].p, (const void *)fe->d_d[1].p, (const void *)fe->d_aw.p,
                          (const void *)fe->d_bw.p})
        k.push_back(key_bits(p));
    return k;
}

static int fe_free_step(pdmts_fem *fe, double dt, double beta, double gamma, cudaStream_t s, int64_t *launches)
{
    return run_graph(
        fe->ctx, fe->g_free, fe_graph_key(fe, dt, beta, gamma), s,
        [&](int64_t *n) { return fe_free_enqueue(fe, dt, beta, gamma, s, n); }, launches);
}

// ------------------------------------------------------------ FE ABI -----
extern "C" int fem_create(pdmts_ctx *ctx, int dim, int64_t n_nodes, const double *Xn, int64_t n_elems,
                          int nodes_per_elem, const int32_t *conn, double E, double nu, double rho, double thickness,
                          pdmts_fem **out)
{
    clear_error();
    if (!ctx || !Xn || !conn || !out)
        return fail(PDMTS_ERR_ARG, "fem_create: NULL argument");
    *out = nullptr;
    if (ctx->fem)
        return fail(PDMTS_ERR_STATE, "fem_create: context already has a finite-element subdomain");
    if (!((dim == 2 && nodes_per_elem == 4) || (dim == 3 && nodes_per_elem == 8)))
        return fail(PDMTS_ERR_UNSUPPORTED, "fem_create: supported elements are Q4 (dim 2, 4 nodes) and Hex8 (dim 3, 8 nodes)");
    if (n_nodes <= 0 || n_elems <= 0 || n_nodes >= ((int64_t)1 << 30))
        return fail(PDMTS_ERR_ARG, "fem_create: bad sizes");
    if (!(E > 0) || !(rho > 0) || !(thickness > 0) || !(nu > -1.0 && nu < 0.5))
        return fail(PDMTS_ERR_ARG, "fem_create: bad material (E, rho, thickness > 0; -1 < nu < 1/2)");
    auto *fe = new (std::nothrow) pdmts_fem();
    if (!fe)
        return fail(PDMTS_ERR_NOMEM, "fem_create: out of host memory");
    fe->ctx = ctx;
    fe->dim = dim;
    fe->n = n_nodes;
    fe->ne = n_elems;
    fe->npe = nodes_per_elem;
    fe->E = E;
    fe->nu = nu;
    fe->rho = rho;
    fe->thick = thickness;
    fe->X.resize((size_t)dim * n_nodes);
    fe->conn.resize((size_t)n_elems * nodes_per_elem);
    if (cudaMemcpy(fe->X.data(), Xn, sizeof(double) * fe->X.size(), cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(fe->conn.data(), conn, sizeof(int32_t) * fe->conn.size(), cudaMemcpyDefault) != cudaSuccess) {
        delete fe;
        return fail(PDMTS_ERR_CUDA, "fem_create: copying inputs failed");
    }
    for (int32_t c : fe->conn)
        if (c < 0 || c >= n_nodes) {
            delete fe;
            return fail(PDMTS_ERR_ARG, "fem_create: connectivity index out of range");
        }
    for (double x : fe->X)
        if (!std::isfinite(x)) {
            delete fe;
            return fail(PDMTS_ERR_ARG, "fem_create: non-finite node coordinate");
        }
    ctx->fem = fe;
    *out = fe;
    return PDMTS_OK;
}

extern "C" int fem_set_traction(pdmts_fem *fe, int64_t n_faces, const int32_t *face_nodes, const double *traction)
{
    clear_error();
    if (!fe || n_faces < 0 || (n_faces > 0 && (!face_nodes || !traction)))
        return fail(PDMTS_ERR_ARG, "fem_set_traction: bad arguments");
    const int npf = fe->dim == 2 ? 2 : 4;  // nodes per face
    std::vector<int32_t> f((size_t)npf * n_faces);
    std::vector<double> t((size_t)fe->dim * n_faces);
    if (n_faces > 0 &&
        (cudaMemcpy(f.data(), face_nodes, sizeof(int32_t) * f.size(), cudaMemcpyDefault) != cudaSuccess ||
         cudaMemcpy(t.data(), traction, sizeof(double) * t.size(), cudaMemcpyDefault) != cudaSuccess))
        return fail(PDMTS_ERR_CUDA, "fem_set_traction: copying inputs failed");
    for (int32_t c : f)
        if (c < 0 || c >= fe->n)
            return fail(PDMTS_ERR_ARG, "fem_set_traction: face node out of range");
    for (double x : t)
        if (!std::isfinite(x))
            return fail(PDMTS_ERR_ARG, "fem_set_traction: non-finite traction");
    if (fe->assembled)
        return fail(PDMTS_ERR_STATE, "fem_set_traction: set tractions before arlequin_bind");
    fe->faces.swap(f);
    fe->face_tr.swap(t);
    return PDMTS_OK;
}

extern "C" int fem_set_fixed(pdmts_fem *fe, int64_t n_fixed, const int64_t *dofs)
{
    clear_error();
    if (!fe || n_fixed < 0 || (n_fixed > 0 && !dofs))
        return fail(PDMTS_ERR_ARG, "fem_set_fixed: bad arguments");
    if (fe->assembled)
        return fail(PDMTS_ERR_STATE, "fem_set_fixed: fix dofs before arlequin_bind");
    std::vector<int64_t> d((size_t)n_fixed);
    if (n_fixed > 0 && cudaMemcpy(d.data(), dofs, sizeof(int64_t) * d.size(), cudaMemcpyDefault) != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "fem_set_fixed: copying inputs failed");
    std::vector<char> f;
    if (n_fixed > 0)
        f.assign((size_t)fe->ndof(), 0);
    for (int64_t k : d) {
        if (k < 0 || k >= fe->ndof())
            return fail(PDMTS_ERR_ARG, "fem_set_fixed: dof %lld out of range", (long long)k);
        f[(size_t)k] = 1;
    }
    fe->fixed.swap(f);
    return PDMTS_OK;
}

extern "C" int fem_destroy(pdmts_fem *fe)
{
    clear_error();
    if (!fe)
        return PDMTS_OK;
    cudaSetDevice(fe->ctx->device);
    cudaStreamSynchronize(fe->ctx->stream);
    if (fe->ctx->fem == fe)
        fe->ctx->fem = nullptr;
    fe->release_all();
    delete fe;
    return PDMTS_OK;
}

static int fem_read(pdmts_fem *fe, int which, double *out)
{
    if (!fe || !out)
        return fail(PDMTS_ERR_ARG, "fem_read: NULL argument");
    if (!fe->assembled)
        return fail(PDMTS_ERR_STATE, "fem_read: the FE subdomain is not bound to a coupling yet");
    PDMTS_CUDA_TRY(cudaSetDevice(fe->ctx->device));
    PDMTS_TRY(fe->ctx->begin());
    const double *src = which == 0 ? fe->d_u.p : which == 1 ? fe->d_v.p : fe->d_a.p;
    PDMTS_CUDA_TRY(cudaMemcpyAsync(out, src, sizeof(double) * fe->ndof(), cudaMemcpyDefault, fe->ctx->stream));
    PDMTS_TRY(fe->ctx->sync_checked("fem_read"));
    return fe->ctx->end();
}
extern "C" int fem_set_state(pdmts_fem *fe, const double *u, const double *v)
{
    clear_error();
    if (!fe)
        return fail(PDMTS_ERR_ARG, "fem_set_state: fe is NULL");
    if (!fe->assembled)
        return fail(PDMTS_ERR_STATE, "fem_set_state: bind the FE subdomain to a coupling first");
    const int64_t nd = fe->ndof();
    std::vector<double> hu((size_t)nd, 0.0), hv((size_t)nd, 0.0);
    if (u)
        PDMTS_CUDA_TRY(cudaMemcpy(hu.data(), u, sizeof(double) * nd, cudaMemcpyDefault));
    if (v)
        PDMTS_CUDA_TRY(cudaMemcpy(hv.data(), v, sizeof(double) * nd, cudaMemcpyDefault));
    for (int64_t i = 0; i < nd; ++i)
        if (!std::isfinite(hu[(size_t)i]) || !std::isfinite(hv[(size_t)i]))
            return fail(PDMTS_ERR_ARG, "fem_set_state: non-finite value");
    if (!fe->fixed.empty())
        for (int64_t i = 0; i < nd; ++i)
            if (fe->fixed[(size_t)i])
                hu[(size_t)i] = hv[(size_t)i] = 0.0;
    // acceleration from the equation of motion M a = P - K u (lambda = 0)
    std::vector<double> a((size_t)nd);
    for (int64_t i = 0; i < nd; ++i) {
        double ku = 0.0;
        for (int e = 0; e < fe->W; ++e)
            ku += fe->kval[(size_t)i * fe->W + e] * hu[(size_t)fe->col[(size_t)i * fe->W + e]];
        a[(size_t)i] = (fe->load[(size_t)i] - ku) / fe->mass[(size_t)i];
    }
    PDMTS_CUDA_TRY(cudaSetDevice(fe->ctx->device));
    PDMTS_TRY(fe->ctx->begin());
    cudaStream_t s = fe->ctx->stream;
    PDMTS_TRY(h2d(fe->d_u.p, hu, s));
    PDMTS_TRY(h2d(fe->d_v.p, hv, s));
    PDMTS_TRY(h2d(fe->d_a.p, a, s));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(s));
    return fe->ctx->end();
}

extern "C" int fem_read_displacement(pdmts_fem *fe, double *u) { clear_error(); return fem_read(fe, 0, u); }
extern "C" int fem_read_velocity(pdmts_fem *fe, double *v) { clear_error(); return fem_read(fe, 1, v); }
extern "C" int fem_read_acceleration(pdmts_fem *fe, double *a) { clear_error(); return fem_read(fe, 2, a); }

// ------------------------------------------------------- coupling set-up --
// Multiplier nodes, G_FE, G_PD and the PD overlap interpolation (Eq. 33, Eq. 41).
static int build_constraint(pdmts_arl *A)
{
    pdmts_fem *fe = A->fe;
    pdmts_pd *pd = A->pd;
    const int64_t nfe = fe->n, npd = pd->n;
    const int dim = fe->dim, npe = fe->npe;
    // overlap elements: centroid strictly inside a band
    std::vector<int64_t> ov_el;
    std::vector<char> is_lam((size_t)nfe, 0);
    for (int64_t e = 0; e < fe->ne; ++e) {
        double c[3] = {0, 0, 0};
        for (int a = 0; a < npe; ++a)
            for (int d = 0; d < dim; ++d)
                c[d] += fe->X[(size_t)d * nfe + fe->conn[(size_t)e * npe + a]] / npe;
        for (const BandDesc &b : A->bands)
            if (c[b.axis] > b.lo && c[b.axis] < b.hi) {
                ov_el.push_back(e);
                for (int a = 0; a < npe; ++a)
                    is_lam[(size_t)fe->conn[(size_t)e * npe + a]] = 1;
                break;
            }
    }
    if (ov_el.empty())
        return fail(PDMTS_ERR_ARG, "arlequin_bind: no finite element lies inside an overlap band");
    std::vector<int32_t> pos((size_t)nfe, -1);
    A->lam_node.clear();
    for (int64_t i = 0; i < nfe; ++i)
        if (is_lam[(size_t)i]) {
            pos[(size_t)i] = (int32_t)A->lam_node.size();
            A->lam_node.push_back((int32_t)i);
        }
    A->nl = (int64_t)A->lam_node.size();
    A->nlam = dim * A->nl;
    // a Dirichlet dof carries no multiplier force: keep fixed dofs out of the overlap
    if (!fe->fixed.empty())
        for (int32_t k : A->lam_node)
            for (int d = 0; d < dim; ++d)
                if (fe->fixed[(size_t)(d * nfe + k)])
                    return fail(PDMTS_ERR_ARG, "arlequin_bind: FE node %d is fixed and lies in an overlap element", k);
    A->corners = npe;
    // G_FE[k, I] = int_O N_k N_I dV (2 x 2 Gauss in 2D, 2 x 2 x 2 in 3D), rows of width 9 or 27
    std::vector<std::map<int32_t, double>> grow((size_t)A->nl);
    const double g = 1.0 / std::sqrt(3.0);
    const double nat[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
    for (int64_t e : ov_el) {
        const int32_t *cn = &fe->conn[(size_t)e * npe];
        if (dim == 2) {
            double xe[4][2];
            for (int a = 0; a < 4; ++a)
                for (int d = 0; d < 2; ++d)
                    xe[a][d] = fe->X[(size_t)d * nfe + cn[a]];
            for (int gi = 0; gi < 2; ++gi)
                for (int gj = 0; gj < 2; ++gj) {
                    const double xi = gi ? g : -g, et = gj ? g : -g;
                    double N[4], dxi[4], det_[4];
                    for (int a = 0; a < 4; ++a) {
                        N[a] = 0.25 * (1 + nat[a][0] * xi) * (1 + nat[a][1] * et);
                        dxi[a] = 0.25 * nat[a][0] * (1 + nat[a][1] * et);
                        det_[a] = 0.25 * nat[a][1] * (1 + nat[a][0] * xi);
                    }
                    double J00 = 0, J01 = 0, J10 = 0, J11 = 0;
                    for (int a = 0; a < 4; ++a) {
                        J00 += dxi[a] * xe[a][0]; J01 += dxi[a] * xe[a][1];
                        J10 += det_[a] * xe[a][0]; J11 += det_[a] * xe[a][1];
                    }
                    const double w = (J00 * J11 - J01 * J10) * fe->thick;
                    for (int a = 0; a < 4; ++a)
                        for (int b = 0; b < 4; ++b)
                            grow[(size_t)pos[(size_t)cn[a]]][cn[b]] += N[a] * N[b] * w;
                }
        } else {
            double xe[8][3];
            for (int a = 0; a < 8; ++a)
                for (int d = 0; d < 3; ++d)
                    xe[a][d] = fe->X[(size_t)d * nfe + cn[a]];
            for (int gi = 0; gi < 2; ++gi)
                for (int gj = 0; gj < 2; ++gj)
                    for (int gk = 0; gk < 2; ++gk) {
                        double N[8], dN[8][3], dNx[8][3], xg[3];
                        hex8_shape(gi ? g : -g, gj ? g : -g, gk ? g : -g, N, dN);
                        const double w = hex8_map(xe, N, dN, dNx, xg);
                        for (int a = 0; a < 8; ++a)
                            for (int b = 0; b < 8; ++b)
                                grow[(size_t)pos[(size_t)cn[a]]][cn[b]] += N[a] * N[b] * w;
                    }
        }
    }
    A->gfe_w = 0;
    for (auto &r : grow)
        A->gfe_w = std::max<int>(A->gfe_w, (int)r.size());
    A->gfe_col.assign((size_t)A->nl * A->gfe_w, 0);
    A->gfe_val.assign((size_t)A->nl * A->gfe_w, 0.0);
    for (int64_t k = 0; k < A->nl; ++k) {
        int e = 0;
        for (auto &kv : grow[(size_t)k]) {
            A->gfe_col[(size_t)k * A->gfe_w + e] = kv.first;
            A->gfe_val[(size_t)k * A->gfe_w + e] = kv.second;
            ++e;
        }
    }
    // the transpose by FE node, for the FE link correction
    A->gfeT_ptr.assign((size_t)nfe + 1, 0);
    for (int64_t k = 0; k < A->nl; ++k)
        for (auto &kv : grow[(size_t)k])
            A->gfeT_ptr[(size_t)kv.first + 1] += 1;
    for (int64_t i = 0; i < nfe; ++i)
        A->gfeT_ptr[(size_t)i + 1] += A->gfeT_ptr[(size_t)i];
    A->gfeT_k.assign((size_t)A->gfeT_ptr[(size_t)nfe], 0);
    A->gfeT_val.assign((size_t)A->gfeT_ptr[(size_t)nfe], 0.0);
    {
        std::vector<int64_t> fill(A->gfeT_ptr.begin(), A->gfeT_ptr.end() - 1);
        for (int64_t k = 0; k < A->nl; ++k)
            for (auto &kv : grow[(size_t)k]) {
                const int64_t j = fill[(size_t)kv.first]++;
                A->gfeT_k[(size_t)j] = (int32_t)k;
                A->gfeT_val[(size_t)j] = kv.second;
            }
    }
    // PD nodes inside overlap elements: G_PD[k, p] = N_k(x_p) V_p, N the
    // bilinear (2D) or trilinear (3D) shape of the axis-aligned element
    std::vector<std::vector<std::pair<int32_t, double>>> prow((size_t)A->nl);
    A->ov_node.clear(); A->ov_k.clear(); A->ov_N.clear();
    for (int64_t e : ov_el) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        const int32_t *cn = &fe->conn[(size_t)e * npe];
        for (int a = 0; a < npe; ++a)
            for (int d = 0; d < dim; ++d) {
                lo[d] = std::min(lo[d], fe->X[(size_t)d * nfe + cn[a]]);
                hi[d] = std::max(hi[d], fe->X[(size_t)d * nfe + cn[a]]);
            }
        for (int64_t p = 0; p < npd; ++p) {
            bool inside = true;
            double xi[3] = {0, 0, 0};
            for (int d = 0; d < dim && inside; ++d) {
                const double x = pd->X[(size_t)d * npd + p];
                inside = x > lo[d] && x < hi[d];
                xi[d] = 2.0 * (x - lo[d]) / (hi[d] - lo[d]) - 1.0;
            }
            if (!inside)
                continue;
            A->ov_node.push_back((int32_t)p);
            for (int a = 0; a < npe; ++a) {
                // natural coordinates of the corner from its position
                double Na = dim == 2 ? 0.25 : 0.125;
                for (int d = 0; d < dim; ++d) {
                    const double ad = fe->X[(size_t)d * nfe + cn[a]] > 0.5 * (lo[d] + hi[d]) ? 1.0 : -1.0;
                    Na *= 1 + ad * xi[d];
                }
                const int32_t k = pos[(size_t)cn[a]];
                A->ov_k.push_back(k);
                A->ov_N.push_back(Na);
                prow[(size_t)k].push_back({(int32_t)p, Na * pd->V[(size_t)p]});
            }
        }
    }
    A->n_ov = (int64_t)A->ov_node.size();
    A->gpd_ptr.assign((size_t)A->nl + 1, 0);
    A->gpd_col.clear();
    A->gpd_val.clear();
    for (int64_t k = 0; k < A->nl; ++k) {
        auto &r = prow[(size_t)k];
        std::sort(r.begin(), r.end());
        for (auto &pv : r) {
            A->gpd_col.push_back(pv.first);
            A->gpd_val.push_back(pv.second);
        }
        A->gpd_ptr[(size_t)k + 1] = (int64_t)A->gpd_col.size();
    }
    cudaStream_t s = A->ctx->stream;
    PDMTS_TRY(A->alloc(A->d_gfe_col, (int64_t)A->gfe_col.size()));
    PDMTS_TRY(A->alloc(A->d_gfe_val, (int64_t)A->gfe_val.size()));
    PDMTS_TRY(A->alloc(A->d_gpd_ptr, (int64_t)A->gpd_ptr.size()));
    PDMTS_TRY(A->alloc(A->d_gpd_col, std::max<int64_t>((int64_t)A->gpd_col.size(), 1)));
    PDMTS_TRY(A->alloc(A->d_gpd_val, std::max<int64_t>((int64_t)A->gpd_val.size(), 1)));
    PDMTS_TRY(A->alloc(A->d_ov_node, std::max<int64_t>(A->n_ov, 1)));
    PDMTS_TRY(A->alloc(A->d_ov_k, std::max<int64_t>(npe * A->n_ov, 1)));
    PDMTS_TRY(A->alloc(A->d_ov_N, std::max<int64_t>(npe * A->n_ov, 1)));
    PDMTS_TRY(A->alloc(A->d_gfeT_ptr, (int64_t)A->gfeT_ptr.size()));
    PDMTS_TRY(A->alloc(A->d_gfeT_k, std::max<int64_t>((int64_t)A->gfeT_k.size(), 1)));
    PDMTS_TRY(A->alloc(A->d_gfeT_val, std::max<int64_t>((int64_t)A->gfeT_val.size(), 1)));
    PDMTS_TRY(h2d(A->d_gfe_col.p, A->gfe_col, s));
    PDMTS_TRY(h2d(A->d_gfe_val.p, A->gfe_val, s));
    PDMTS_TRY(h2d(A->d_gfeT_ptr.p, A->gfeT_ptr, s));
    PDMTS_TRY(h2d(A->d_gfeT_k.p, A->gfeT_k, s));
    PDMTS_TRY(h2d(A->d_gfeT_val.p, A->gfeT_val, s));
    PDMTS_TRY(h2d(A->d_gpd_ptr.p, A->gpd_ptr, s));
    PDMTS_TRY(h2d(A->d_gpd_col.p, A->gpd_col, s));
    PDMTS_TRY(h2d(A->d_gpd_val.p, A->gpd_val, s));
    PDMTS_TRY(h2d(A->d_ov_node.p, A->ov_node, s));
    PDMTS_TRY(h2d(A->d_ov_k.p, A->ov_k, s));
    PDMTS_TRY(h2d(A->d_ov_N.p, A->ov_N, s));
    for (DevArr<double> *a : {&A->d_lam0, &A->d_lam, &A->d_y, &A->d_colbuf}) {
        PDMTS_TRY(A->alloc(*a, A->nlam));
        PDMTS_CUDA_TRY(cudaMemsetAsync(a->p, 0, sizeof(double) * A->nlam, s));
    }
    PDMTS_TRY(A->alloc(A->d_Hneg_inv, A->nlam * A->nlam));
    PDMTS_TRY(A->alloc(A->d_changed, 1));
    // bond words of PD nodes within (m + 1) delta of a band (rebuild rule)
    PDMTS_CUDA_TRY(cudaStreamSynchronize(s));
    return PDMTS_OK;
}

static int update_near_flags(pdmts_arl *A, int m)
{
    pdmts_pd *pd = A->pd;
    const int64_t npd = pd->n;
    const double reach = (m + 1) * pd->horizon;
    std::vector<uint8_t> near_node((size_t)npd, 0);
    for (int64_t p = 0; p < npd; ++p)
        for (const BandDesc &b : A->bands) {
            const double c = pd->X[(size_t)b.axis * npd + p];
            if (c >= b.lo - reach && c <= b.hi + reach)
                near_node[(size_t)p] = 1;
        }
    std::vector<uint8_t> wflag((size_t)std::max<int64_t>(pd->n_mask_words, 1), 0);
    if (pd->layout == pdmts_pd::LAYOUT_LATTICE2D || pd->layout == pdmts_pd::LAYOUT_LATTICE3D) {
        for (int64_t w = 0; w < pd->n_mask_words / npd; ++w)
            for (int64_t p = 0; p < npd; ++p)
                wflag[(size_t)(w * npd + p)] = near_node[(size_t)p];
    } else {
        for (int64_t p = 0; p < npd; ++p) {
            const int64_t t = p / 32, lane = p % 32;
            const int words = (pd->tile_k[(size_t)t] + 31) / 32;
            for (int w = 0; w < words; ++w)
                wflag[(size_t)(pd->mask_ptr[(size_t)t] + 32 * w + lane)] = near_node[(size_t)p];
        }
    }
    PDMTS_TRY(A->alloc(A->d_near, (int64_t)wflag.size()));
    PDMTS_TRY(h2d(A->d_near.p, wflag, A->ctx->stream));
    // Tile rows of the lattice kernel that the link problem can reach: its
    // response stays within m delta of the loaded overlap nodes, so tile rows
    // holding no node within (m + 1) delta of a band stay exactly zero.
    pd->link_win_n[0] = pd->link_win_n[1] = 0;
    pd->link_bonds = -1;
    if (pd->layout == pdmts_pd::LAYOUT_LATTICE2D && A->bands.size() <= 2) {
        const int ny = pd->lat_dims[1], nx = pd->lat_dims[0];
        const int ntr = (ny + lat2d::TY - 1) / lat2d::TY;
        std::vector<char> need((size_t)ntr, 0);
        for (int y = 0; y < ny; ++y)
            if (near_node[(size_t)y * nx])  // a lattice row is near iff its nodes are (bands span x)
                need[(size_t)(y / lat2d::TY)] = 1;
        bool all_x = true;
        for (const BandDesc &b : A->bands)
            all_x = all_x && b.axis == 1;
        int lo[2] = {0, 0}, cnt[2] = {0, 0}, nw = 0;
        bool ok = all_x;
        for (int t = 0; t < ntr && ok; ++t) {
            if (!need[(size_t)t])
                continue;
            if (nw > 0 && lo[nw - 1] + cnt[nw - 1] == t) {
                cnt[nw - 1]++;
            } else if (nw < 2) {
                lo[nw] = t;
                cnt[nw] = 1;
                ++nw;
            } else {
                ok = false;
            }
        }
        if (ok && nw > 0 && cnt[0] + cnt[1] < ntr) {
            int64_t bonds = 0;
            for (int w = 0; w < 2; ++w) {
                pd->link_win_lo[w] = lo[w];
                pd->link_win_n[w] = cnt[w];
                const int64_t r0 = std::min<int64_t>((int64_t)lo[w] * lat2d::TY, ny);
                const int64_t r1 = std::min<int64_t>((int64_t)(lo[w] + cnt[w]) * lat2d::TY, ny);
                bonds += pd->row_ptr[(size_t)(r1 * nx)] - pd->row_ptr[(size_t)(r0 * nx)];
            }
            pd->link_bonds = bonds;
        }
    }
    // A link run starts from rest and is loaded on the overlap nodes only, so
    // after substep k (0-based) its state is nonzero only within k delta of a
    // band: substep k evaluates the tile rows within (k + 2) delta (the rows
    // left out hold exact zeros and would compute exact zeros). The windows
    // grow to the fixed ones above at k = m - 1.
    pd->link_step_win.clear();
    pd->link_step_bonds.clear();
    if (pd->link_win_n[0] > 0) {
        const int ny = pd->lat_dims[1], nx = pd->lat_dims[0];
        const int ntr = (ny + lat2d::TY - 1) / lat2d::TY;
        for (int k = 0; k < m; ++k) {
            const double reach = (k + 2) * pd->horizon;
            std::vector<char> need((size_t)ntr, 0);
            for (int y = 0; y < ny; ++y) {
                const double c = pd->X[(size_t)npd + (size_t)y * nx];
                for (const BandDesc &b : A->bands)
                    if (c >= b.lo - reach && c <= b.hi + reach)
                        need[(size_t)(y / lat2d::TY)] = 1;
            }
            std::array<int, 4> w = {0, 0, 0, 0};
            int nw = 0;
            bool ok = true;
            for (int t = 0; t < ntr && ok; ++t) {
                if (!need[(size_t)t])
                    continue;
                if (nw > 0 && w[2 * (nw - 1)] + w[2 * (nw - 1) + 1] == t)
                    w[2 * (nw - 1) + 1]++;
                else if (nw < 2)
                    w[2 * nw] = t, w[2 * nw + 1] = 1, ++nw;
                else
                    ok = false;
            }
            if (!ok || nw == 0) {  // keep the fixed windows for every substep
                pd->link_step_win.clear();
                pd->link_step_bonds.clear();
                break;
            }
            int64_t bonds = 0;
            for (int q = 0; q < 2; ++q) {
                const int64_t r0 = std::min<int64_t>((int64_t)w[2 * q] * lat2d::TY, ny);
                const int64_t r1 = std::min<int64_t>((int64_t)(w[2 * q] + w[2 * q + 1]) * lat2d::TY, ny);
                bonds += pd->row_ptr[(size_t)(r1 * nx)] - pd->row_ptr[(size_t)(r0 * nx)];
            }
            pd->link_step_win.push_back(w);
            pd->link_step_bonds.push_back(bonds);
        }
    }
    // node ranges a link run may write: the windows widened to 32 rows
    pd->link_seg_lo[0] = pd->link_seg_lo[1] = 0;
    pd->link_seg_n[0] = pd->n;
    pd->link_seg_n[1] = 0;
    if (pd->link_win_n[0] > 0) {
        const int64_t nx = pd->lat_dims[0], ny = pd->lat_dims[1];
        int64_t lo[2] = {0, 0}, hi[2] = {0, 0};
        int nw = 0;
        for (int w = 0; w < 2; ++w) {
            if (pd->link_win_n[w] <= 0)
                continue;
            const int64_t r0 = (int64_t)pd->link_win_lo[w] * lat2d::TY / 32 * 32;
            const int64_t r1 = std::min<int64_t>(ny, ((int64_t)(pd->link_win_lo[w] + pd->link_win_n[w]) * lat2d::TY + 31) / 32 * 32);
            if (nw > 0 && r0 <= hi[nw - 1]) {
                hi[nw - 1] = std::max(hi[nw - 1], r1);
            } else {
                lo[nw] = r0;
                hi[nw] = r1;
                ++nw;
            }
        }
        for (int w = 0; w < 2; ++w) {
            pd->link_seg_lo[w] = w < nw ? lo[w] * nx : 0;
            pd->link_seg_n[w] = w < nw ? (hi[w] - lo[w]) * nx : 0;
        }
    }
    // the previous windows may have left link state outside the new ones
    PDMTS_TRY(pd->zero_link_state(A->ctx->stream, true));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(A->ctx->stream));
    return PDMTS_OK;
}

// FE part of the interface operator, H_FE = -gamma dt_FE G_FE K_eff^-1 G_FE^T
// (Eq. 49 with the Newmark velocity response of a unit multiplier), by block
// Chebyshev over batches of unit columns. It does not depend on the PD bond
// state, so it is kept until dt_FE changes.
static int build_Hfe(pdmts_arl *A, double dtf, int64_t *launches)
{
    pdmts_fem *fe = A->fe;
    const int64_t ndof = fe->ndof();
    const int64_t nlam = A->nlam;
    cudaStream_t s = A->ctx->stream;
    PDMTS_TRY(A->alloc(A->d_Hfe, nlam * nlam));
    const int batch = (int)std::min<int64_t>(nlam, 512);
    DevArr<double> xb;
    PDMTS_TRY(A->alloc(xb, ndof * batch));
    for (int b = 0; b < 4; ++b)
        PDMTS_TRY(A->alloc(A->d_B[b], ndof * batch));
    for (int64_t q0 = 0; q0 < nlam; q0 += batch) {
        const int nb = (int)std::min<int64_t>(batch, nlam - q0);
        PDMTS_CUDA_TRY(cudaMemsetAsync(A->d_B[0].p, 0, sizeof(double) * ndof * nb, s));
        k_gfe_rhs<<<blocks(nb), 256, 0, s>>>(fe->n, fe->dim, A->nl, A->gfe_w, A->d_gfe_col.p, A->d_gfe_val.p, q0, nb,
                                             A->d_B[0].p);
        PDMTS_CUDA_TRY(cudaMemsetAsync(xb.p, 0, sizeof(double) * ndof * nb, s));
        PDMTS_TRY(fe_cheb_solve(fe, nb, xb.p, A->d_B[0].p, A->d_B[1].p, A->d_B[2].p, A->d_B[3].p, s, launches));
        k_hfe_cols<<<blocks(nlam * nb), 256, 0, s>>>(fe->n, fe->dim, A->nl, A->gfe_w, A->d_gfe_col.p, A->d_gfe_val.p, q0,
                                                     nb, xb.p, -A->ctx->gamma_fe * dtf, A->d_Hfe.p);
        *launches += 2;
    }
    PDMTS_CUDA_TRY(cudaStreamSynchronize(s));
    A->release(xb);
    for (int b = 0; b < 4; ++b)
        A->release(A->d_B[b]);
    A->Hfe_valid = true;
    PDMTS_CUDA_TRY(cudaGetLastError());
    return PDMTS_OK;
}

// FE link correction (Eq. 47b): K_eff a_W = -G_FE^T lambda_m from a zero
// start with the free step's Chebyshev schedule, then the Newmark update.
static int fe_link_enqueue(pdmts_arl *A, double dt, double beta, double gamma, cudaStream_t s, int64_t *launches)
{
    pdmts_fem *fe = A->fe;
    const int64_t ndof = fe->ndof();
    k_gfe_lam<<<blocks(ndof), 256, 0, s>>>(fe->n, fe->dim, A->nl, A->d_gfeT_ptr.p, A->d_gfeT_k.p, A->d_gfeT_val.p,
                                           A->d_lam.p, fe->d_bw.p);
    PDMTS_CUDA_TRY(cudaMemsetAsync(fe->d_aw.p, 0, sizeof(double) * ndof, s));
    ++*launches;
    PDMTS_TRY(fe_cheb_solve(fe, 1, fe->d_aw.p, fe->d_bw.p, fe->d_r.p, fe->d_d[0].p, fe->d_d[1].p, s, launches));
    k_fe_apply_link<<<blocks(ndof), 256, 0, s>>>(ndof, fe->d_aw.p, dt, beta, gamma, fe->d_u.p, fe->d_v.p,
                                                 fe->d_a.p);
    ++*launches;
    PDMTS_CUDA_TRY(cudaGetLastError());
    return PDMTS_OK;
}

static int fe_link_step(pdmts_arl *A, double dt, double beta, double gamma, cudaStream_t s, int64_t *launches)
{
    std::vector<uint64_t> key = fe_graph_key(A->fe, dt, beta, gamma);
    for (const void *p : {(const void *)A->d_gfeT_ptr.p, (const void *)A->d_gfeT_k.p,
                          (const void *)A->d_gfeT_val.p, (const void *)A->d_lam.p})
        key.push_back(key_bits(p));
    key.push_back((uint64_t)A->nl);
    return run_graph(
        A->ctx, A->fe->g_link, key, s, [&](int64_t *n) { return fe_link_enqueue(A, dt, beta, gamma, s, n); },
        launches);
}

int pd_run_chain(pdmts_pd *pd, int len, int sched, const double *theta, cudaStream_t s, bool link);
int pd_invalidate_graphs(pdmts_pd *pd);

// The PD link run (Eq. 48b) for the multiplier in dev_lam: W_0 = 0, m
// substeps with factor j/m, bond words of the step start, no breaking.
static int pd_link_run(pdmts_arl *A, const double *dev_lam, int m, cudaStream_t s)
{
    pdmts_pd *pd = A->pd;
    const bool f64 = pd->precision == PDMTS_FP64;
    cudaError_t e = launch_interface_force(pd->dim, pd->n, A->n_ov, A->d_ov_node.p, A->d_ov_k.p, A->d_ov_N.p, A->corners,
                                           dev_lam, A->nl, f64 ? 0.0 : 1.0 / pd->h, f64 ? pd->lk_g.p : nullptr,
                                           f64 ? nullptr : pd->lk_gf.p, s);
    if (e != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "interface force: %s", cudaGetErrorString(e));
    PDMTS_TRY(pd->zero_link_state(s));
    PDMTS_TRY(pd_run_chain(pd, m, 2, A->theta_link.data(), s, true));
    pd->ctx->stats.kernel_launches += 1;
    return PDMTS_OK;
}

// Colouring of the multiplier columns for the link runs of build_H: columns
// whose supports are more than 2R apart (R = 2 h_FE + m delta) share a colour,
// and each constraint row is attributed to the one column of its colour
// within R. Depends on the geometry and m only: computed once per m, with
// every colour's unit vector and row owners uploaded together.
static int build_colors(pdmts_arl *A, int m, cudaStream_t s)
{
    if (A->colors_m == m && !A->color_cols.empty())
        return PDMTS_OK;
    pdmts_fem *fe = A->fe;
    pdmts_pd *pd = A->pd;
    const int64_t nlam = A->nlam, nl = A->nl;
    double hmax = 0.0;
    for (int64_t e = 0; e < fe->ne; ++e) {
        // opposite corners of the (axis-aligned) element
        const int32_t a = fe->conn[(size_t)e * fe->npe], c = fe->conn[(size_t)e * fe->npe + (fe->dim == 2 ? 2 : 6)];
        for (int d = 0; d < fe->dim; ++d)
            hmax = std::max(hmax, std::fabs(fe->X[(size_t)d * fe->n + c] - fe->X[(size_t)d * fe->n + a]));
    }
    const double R = 2.0 * hmax + m * pd->horizon;
    auto xk = [&](int64_t q, int d) { return fe->X[(size_t)d * fe->n + A->lam_node[(size_t)(q % nl)]]; };
    auto dist_inf = [&](int64_t q, int64_t o) {
        double dd = 0.0;
        for (int d = 0; d < fe->dim; ++d)
            dd = std::max(dd, std::fabs(xk(q, d) - xk(o, d)));
        return dd;
    };
    std::vector<std::vector<int64_t>> colors;
    for (int64_t q = 0; q < nlam; ++q) {
        bool placed = false;
        for (auto &cl : colors) {
            bool ok = true;
            for (int64_t o : cl) {
                if (dist_inf(q, o) <= 2.0 * R) {
                    ok = false;
                    break;
                }
            }
            if (ok) {
                cl.push_back(q);
                placed = true;
                break;
            }
        }
        if (!placed)
            colors.push_back({q});
    }
    const int64_t nc = (int64_t)colors.size();
    std::vector<double> unit((size_t)(nc * nlam), 0.0);
    std::vector<int32_t> owner((size_t)(nc * nlam), -1);
    for (int64_t c = 0; c < nc; ++c) {
        for (int64_t q : colors[(size_t)c])
            unit[(size_t)(c * nlam + q)] = 1.0;
        for (int64_t r = 0; r < nlam; ++r)
            for (int64_t q : colors[(size_t)c]) {
                if (dist_inf(q, r) <= R) {
                    owner[(size_t)(c * nlam + r)] = (int32_t)q;
                    break;
                }
            }
    }
    PDMTS_TRY(A->alloc(A->d_units, nc * nlam));
    PDMTS_TRY(A->alloc(A->d_owners, nc * nlam));
    PDMTS_TRY(h2d(A->d_units.p, unit, s));
    PDMTS_TRY(h2d(A->d_owners.p, owner, s));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(s));
    A->color_cols = std::move(colors);
    A->colors = nc;
    A->colors_m = m;
    return PDMTS_OK;
}

// Row-major symmetric n x n: copy the upper triangle onto the lower.
__global__ void k_mirror_upper(const int64_t n, double *__restrict__ M)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * n)
        return;
    const int64_t i = t / n, j = t - i * n;
    if (i > j)
        M[t] = M[j * n + i];
}

__global__ void k_identity(const int64_t n, double *__restrict__ M)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * n)
        return;
    const int64_t i = t / n, j = t - i * n;
    M[t] = i == j ? 1.0 : 0.0;
}

// In-place inverse of the row-major n x n matrix M = -H (FP64, cuSOLVER).
// -H is symmetric positive definite in exact arithmetic: Cholesky factorisation
// and inversion from the factor (cuSOLVER's column-major lower triangle is
// this row-major upper triangle; the lower one is mirrored afterwards). An
// operator measured by FP32 link runs (FP32-bulk) carries their rounding in
// its weakest directions and need not be numerically definite, and one that
// fails Cholesky is not either: LU with partial pivoting of the full matrix,
// where cuSOLVER solves M^T X = I in its column-major view, and X read
// row-major is M^-1.
static int invert_spd(pdmts_arl *A, double *M, int64_t n, cudaStream_t s, int64_t *launches)
{
    if (n > INT32_MAX)
        return fail(PDMTS_ERR_UNSUPPORTED, "interface operator of %lld rows", (long long)n);
    if (!A->solver && cusolverDnCreate(&A->solver) != CUSOLVER_STATUS_SUCCESS)
        return fail(PDMTS_ERR_CUDA, "cusolverDnCreate failed");
    if (cusolverDnSetStream(A->solver, s) != CUSOLVER_STATUS_SUCCESS)
        return fail(PDMTS_ERR_CUDA, "cusolverDnSetStream failed");
    const int ni = (int)n;
    int l1 = 0, l2 = 0, l3 = 0;
    if (cusolverDnDpotrf_bufferSize(A->solver, CUBLAS_FILL_MODE_LOWER, ni, M, ni, &l1) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnDpotri_bufferSize(A->solver, CUBLAS_FILL_MODE_LOWER, ni, M, ni, &l2) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnDgetrf_bufferSize(A->solver, ni, ni, M, ni, &l3) != CUSOLVER_STATUS_SUCCESS)
        return fail(PDMTS_ERR_CUDA, "cuSOLVER workspace query failed");
    const int lw = std::max({l1, l2, l3, 1});
    DevArr<double> work, keep;
    DevArr<int> info, piv;
    int r = PDMTS_OK;
    auto cleanup = [&]() {
        A->release(work);
        A->release(keep);
        A->release(info);
        A->release(piv);
    };
    if ((r = A->alloc(work, lw)) != PDMTS_OK || (r = A->alloc(keep, n * n)) != PDMTS_OK ||
        (r = A->alloc(info, 2)) != PDMTS_OK || (r = A->alloc(piv, n)) != PDMTS_OK) {
        cleanup();
        return r;
    }
    int hinfo[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(keep.p, M, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(info.p, 0, 2 * sizeof(int), s);
    // an operator measured by FP32 link runs carries their rounding in its
    // weakest directions and need not be numerically definite: LU at once
    if (A->pd->precision != PDMTS_FP64) {
        hinfo[0] = 1;
    } else if (e != cudaSuccess ||
               cusolverDnDpotrf(A->solver, CUBLAS_FILL_MODE_LOWER, ni, M, ni, work.p, lw, info.p) !=
                   CUSOLVER_STATUS_SUCCESS ||
               cusolverDnDpotri(A->solver, CUBLAS_FILL_MODE_LOWER, ni, M, ni, work.p, lw, info.p + 1) !=
                   CUSOLVER_STATUS_SUCCESS ||
               cudaMemcpyAsync(hinfo, info.p, sizeof(hinfo), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
               cudaStreamSynchronize(s) != cudaSuccess) {
        cleanup();
        return fail(PDMTS_ERR_CUDA, "Cholesky inverse failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if (hinfo[0] == 0 && hinfo[1] == 0) {
        k_mirror_upper<<<blocks(n * n), 256, 0, s>>>(n, M);
        *launches += 1;
    } else {
        // LU with partial pivoting of the kept copy; the inverse lands in M
        k_identity<<<blocks(n * n), 256, 0, s>>>(n, M);
        *launches += 1;
        hinfo[0] = hinfo[1] = 0;
        if (cudaMemsetAsync(info.p, 0, 2 * sizeof(int), s) != cudaSuccess ||
            cusolverDnDgetrf(A->solver, ni, ni, keep.p, ni, work.p, piv.p, info.p) != CUSOLVER_STATUS_SUCCESS ||
            cusolverDnDgetrs(A->solver, CUBLAS_OP_N, ni, ni, keep.p, ni, piv.p, M, ni, info.p + 1) !=
                CUSOLVER_STATUS_SUCCESS ||
            cudaMemcpyAsync(hinfo, info.p, sizeof(hinfo), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            r = fail(PDMTS_ERR_CUDA, "LU inverse failed: %s", cudaGetErrorString(cudaGetLastError()));
        else if (hinfo[0] != 0 || hinfo[1] != 0)
            r = fail(PDMTS_ERR_STATE, "interface operator H is singular (cuSOLVER info %d, %d)", hinfo[0], hinfo[1]);
        A->lu_inverses += 1;
    }
    PDMTS_CUDA_TRY(cudaStreamSynchronize(s));
    cleanup();
    return r;
}

// The PD columns of H for an FP32-bulk 2D lattice, up to kLinkGroup colours
// at a time: every colour of a group gets its own link state (a slot of one
// pool), the m substeps of all the group's link runs are one batched launch
// each over the (colour, tile) work items of that substep's window, and each
// colour's constraint rows are then scattered into H. The batched launch runs
// the single-lattice tile code, so every column has the bits of its own link
// run. Returns PDMTS_ERR_UNSUPPORTED (nothing enqueued) for other set-ups.
constexpr int kLinkGroup = 32;
static int build_H_pd_grouped(pdmts_arl *A, int m, double *H, cudaStream_t s, int64_t *launches)
{
    pdmts_pd *pd = A->pd;
    const int64_t n = pd->n, nlam = A->nlam;
    if (pd->precision == PDMTS_FP64 || pd->layout != pdmts_pd::LAYOUT_LATTICE2D || pd->dim != 2 || A->colors < 2)
        return PDMTS_ERR_UNSUPPORTED;
    // slots of 16 n floats (64 B per node): u4 x 2, v4, a (float2), g (2 planes)
    const int64_t slot_floats = 16 * n;
    const int64_t budget = (int64_t)1 << 31;
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)kLinkGroup, A->colors,
                                                                budget / (int64_t)(sizeof(float) * slot_floats)}));
    if (G < 2)
        return PDMTS_ERR_UNSUPPORTED;
    constexpr int tile = 1;  // a batchable tile configuration (all give the same bits)
    DevArr<float> pool;
    DevArr<Lat2DArgs> d_args;
    DevArr<int2> d_work;
    DevArr<double> d_ys;
    int r = A->alloc(pool, (int64_t)G * slot_floats);
    if (r == PDMTS_OK)
        r = A->alloc(d_ys, (int64_t)G * nlam);
    auto cleanup = [&]() {
        A->release(pool);
        A->release(d_args);
        A->release(d_work);
        A->release(d_ys);
    };
    if (r != PDMTS_OK) {
        cleanup();
        return r;
    }
    auto slot = [&](int g) { return pool.p + (int64_t)g * slot_floats; };
    // launch arguments and work items of every substep for G slots; the first
    // q slots' items are a prefix of each substep's list
    std::vector<Lat2DArgs> args((size_t)m * G);
    std::vector<int2> work;
    std::vector<int64_t> work_off((size_t)m * (G + 1));
    for (int j = 0; j < m; ++j) {
        for (int g = 0; g < G; ++g) {
            float *b = slot(g);
            F32NodeArgs N = pd->f32_node_args(false, A->theta_link[(size_t)j], true);
            // substep j of a run started from W_0 = 0 (both buffers zero, a_0 = 0)
            // reads buffer (j + 1) & 1 and writes buffer j & 1
            float4 *u4[2] = {reinterpret_cast<float4 *>(b), reinterpret_cast<float4 *>(b + 4 * n)};
            N.u4_in = u4[(j + 1) & 1];
            N.u4_out = u4[j & 1];
            N.v4 = reinterpret_cast<float4 *>(b + 8 * n);
            N.a = b + 12 * n;
            N.g = b + 14 * n;
            N.u2_in = nullptr;
            N.u2_out = nullptr;
            N.v2 = nullptr;
            pd->chain_k = j;
            Lat2DArgs L = pd->lattice_args(N, pd->d_mask_link.p, true);
            pd->chain_k = 0;
            L.tile = tile;
            const int nt = lattice2d_batch_prepare(L, tile);
            if (nt < 0) {
                cleanup();
                return PDMTS_ERR_UNSUPPORTED;
            }
            work_off[(size_t)j * (G + 1) + g] = (int64_t)work.size();
            for (int t = 0; t < nt; ++t)
                work.push_back(make_int2(g, t));
            args[(size_t)j * G + g] = L;
        }
        work_off[(size_t)j * (G + 1) + G] = (int64_t)work.size();
    }
    if ((r = A->alloc(d_args, (int64_t)args.size())) != PDMTS_OK ||
        (r = A->alloc(d_work, (int64_t)std::max<size_t>(work.size(), 1))) != PDMTS_OK ||
        (r = h2d(d_args.p, args, s)) != PDMTS_OK || (r = h2d(d_work.p, work, s)) != PDMTS_OK) {
        cleanup();
        return r;
    }
    const bool pmb = pd->force_kind == PDMTS_FORCE_PMB;
    cudaError_t e = cudaSuccess;
    int64_t bonds_per_run = 0;
    for (int j = 0; j < m; ++j)
        bonds_per_run += pd->substep_bonds(true, j);
    for (int64_t c0 = 0; c0 < A->colors && e == cudaSuccess; c0 += G) {
        const int q = (int)std::min<int64_t>(G, A->colors - c0);
        e = cudaMemsetAsync(pool.p, 0, sizeof(float) * slot_floats * q, s);
        for (int g = 0; g < q && e == cudaSuccess; ++g)
            e = launch_interface_force(pd->dim, n, A->n_ov, A->d_ov_node.p, A->d_ov_k.p, A->d_ov_N.p, A->corners,
                                       A->d_units.p + (c0 + g) * nlam, A->nl, 1.0 / pd->h, nullptr, slot(g) + 14 * n,
                                       s);
        for (int j = 0; j < m && e == cudaSuccess; ++j) {
            const int64_t w0 = work_off[(size_t)j * (G + 1)], w1 = work_off[(size_t)j * (G + 1) + q];
            e = launch_lattice2d_batch(d_args.p + (int64_t)j * G, d_work.p + w0, (int)(w1 - w0), tile, pmb, s);
        }
        // y = G_PD v_link of every colour of the group, scattered into H
        if (e == cudaSuccess)
            e = launch_constraint_pd_many(A->nl, A->d_gpd_ptr.p, A->d_gpd_col.p, A->d_gpd_val.p, n,
                                          reinterpret_cast<const float4 *>(slot(0) + 8 * n), slot_floats / 4, q,
                                          pd->h, 1.0, d_ys.p, nlam, s);
        if (e == cudaSuccess) {
            k_scatter_color<<<dim3(blocks(nlam), (unsigned)q), 256, 0, s>>>(nlam, A->d_owners.p + c0 * nlam, d_ys.p,
                                                                           -1.0, H);
            e = cudaGetLastError();
        }
        *launches += 3 + (int64_t)q + m;
        pd->ctx->stats.pd_substeps += (int64_t)q * m;
        pd->ctx->stats.bond_updates += (int64_t)q * bonds_per_run;
    }
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);  // the pool and the work lists are released below
    cleanup();
    if (e != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "grouped link runs: %s", cudaGetErrorString(e));
    return PDMTS_OK;
}

// Interface operator H = G_FE Ydot_FE - G_PD Ydot_PD (Eq. 49) and its inverse.
// Columns of H_PD come from link runs of several unit multipliers at once:
// columns whose supports are more than 2R apart (R = 2 h_FE + m delta, the
// reach of a link response over m substeps plus the shape-function supports)
// cannot be seen by the same constraint row, so each row is attributed to the
// one column of the run within R of it.
static int build_H(pdmts_arl *A, int m)
{
    pdmts_fem *fe = A->fe;
    pdmts_pd *pd = A->pd;
    pdmts_ctx *ctx = A->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t nlam = A->nlam, nl = A->nl;
    int64_t launches = 0;
    const double dtf = m * ctx->dt_pd;
    if (!A->Hfe_valid)
        PDMTS_TRY(build_Hfe(A, dtf, &launches));
    double *H = A->d_Hneg_inv.p;  // holds H while building, then (-H)^-1
    PDMTS_CUDA_TRY(cudaMemcpyAsync(H, A->d_Hfe.p, sizeof(double) * nlam * nlam, cudaMemcpyDeviceToDevice, s));
    PDMTS_TRY(build_colors(A, m, s));
    const bool f64 = pd->precision == PDMTS_FP64;
    const int gr = build_H_pd_grouped(A, m, H, s, &launches);
    if (gr != PDMTS_OK && gr != PDMTS_ERR_UNSUPPORTED)
        return gr;
    for (int64_t cidx = 0; gr == PDMTS_ERR_UNSUPPORTED && cidx < A->colors; ++cidx) {
        PDMTS_TRY(pd_link_run(A, A->d_units.p + cidx * nlam, m, s));
        // y = G_PD v_link
        cudaError_t e = launch_constraint(pd->dim, nl, A->d_gpd_ptr.p, A->d_gpd_col.p, A->d_gpd_val.p, pd->n,
                                          f64 ? pd->lk_v.p : nullptr, f64 ? nullptr : pd->lk_v4.p,
                                          f64 ? nullptr : pd->lk_v2.p, pd->h, nullptr, nullptr, 0, 0, nullptr, 1.0,
                                          0.0, A->d_y.p, s);
        if (e != cudaSuccess)
            return fail(PDMTS_ERR_CUDA, "constraint rows: %s", cudaGetErrorString(e));
        k_scatter_color<<<blocks(nlam), 256, 0, s>>>(nlam, A->d_owners.p + cidx * nlam, A->d_y.p, -1.0, H);
        launches += 2;
    }
    // (-H)^-1 (-H is symmetric positive definite)
    const int64_t n2 = nlam * nlam;
    k_negate<<<blocks(n2), 256, 0, s>>>(n2, H);
    ++launches;
    PDMTS_TRY(invert_spd(A, H, nlam, s, &launches));
    if (!f64 && nlam % 2 == 0) {
        // the FP32-pair copy the FP32-bulk steps multiply with
        if (A->d_Hinv_df.count != n2) {
            PDMTS_TRY(A->alloc(A->d_Hinv_df, n2));
            PDMTS_TRY(A->alloc(A->d_ydf, nlam));
            PDMTS_TRY(A->alloc(A->d_df_scale, 1));
            PDMTS_TRY(A->alloc(A->d_absmax, 1));
        }
        PDMTS_CUDA_TRY(cudaMemsetAsync(A->d_absmax.p, 0, sizeof(unsigned long long), s));
        const unsigned g = (unsigned)std::min<int64_t>(blocks(n2), 4096);
        k_absmax_bits<<<g, 256, 0, s>>>(n2, H, A->d_absmax.p);
        k_df_split<<<g, 256, 0, s>>>(n2, H, A->d_absmax.p, A->d_Hinv_df.p, A->d_df_scale.p);
        launches += 2;
    }
    PDMTS_CUDA_TRY(cudaGetLastError());
    PDMTS_CUDA_TRY(cudaStreamSynchronize(s));
    ctx->stats.kernel_launches += launches;
    A->H_valid = true;
    A->built_m = m;
    A->rebuilds++;
    return PDMTS_OK;
}

// ------------------------------------------------------------ ABI ---------
extern "C" int arlequin_bind(pdmts_ctx *ctx, pdmts_pd *pd, pdmts_fem *fe, int weight_kind, int n_bands,
                             const double *bands, pdmts_arl **out)
{
    clear_error();
    if (!ctx || !pd || !fe || !out || n_bands <= 0 || !bands)
        return fail(PDMTS_ERR_ARG, "arlequin_bind: bad arguments");
    *out = nullptr;
    if (ctx->arl)
        return fail(PDMTS_ERR_STATE, "arlequin_bind: context already has a coupling");
    if (pd->ctx != ctx || fe->ctx != ctx)
        return fail(PDMTS_ERR_ARG, "arlequin_bind: subdomains belong to another context");
    if (pd->dim != fe->dim)
        return fail(PDMTS_ERR_ARG, "arlequin_bind: PD subdomain in %dD, FE subdomain in %dD", pd->dim, fe->dim);
    if (weight_kind < PDMTS_WEIGHT_CONSTANT || weight_kind > PDMTS_WEIGHT_CUBIC)
        return fail(PDMTS_ERR_ARG, "arlequin_bind: unknown weight kind %d", weight_kind);
    std::vector<double> bv((size_t)5 * n_bands);
    PDMTS_CUDA_TRY(cudaMemcpy(bv.data(), bands, sizeof(double) * bv.size(), cudaMemcpyDefault));
    std::vector<BandDesc> bl;
    for (int k = 0; k < n_bands; ++k) {
        BandDesc b{(int)bv[(size_t)5 * k], bv[(size_t)5 * k + 1], bv[(size_t)5 * k + 2], (int)bv[(size_t)5 * k + 3]};
        if (b.axis < 0 || b.axis >= fe->dim || !(b.hi > b.lo) || (b.fe_side != -1 && b.fe_side != 1))
            return fail(PDMTS_ERR_ARG, "arlequin_bind: band %d is malformed", k);
        bl.push_back(b);
    }
    PDMTS_CUDA_TRY(cudaSetDevice(ctx->device));
    auto *A = new (std::nothrow) pdmts_arl();
    if (!A)
        return fail(PDMTS_ERR_NOMEM, "arlequin_bind: out of host memory");
    A->ctx = ctx;
    A->pd = pd;
    A->fe = fe;
    A->kind = weight_kind;
    A->bands = bl;
    int r = PDMTS_OK;
    // PD weights alpha_i (0 outside the bands)
    std::vector<double> alpha((size_t)pd->n);
    for (int64_t p = 0; p < pd->n; ++p) {
        double x[3] = {0, 0, 0};
        for (int d = 0; d < pd->dim; ++d)
            x[d] = pd->X[(size_t)d * pd->n + p];
        alpha[(size_t)p] = arlequin_alpha(bl, weight_kind, x, 0.0);
    }
    r = pd_set_weights(pd, alpha.data());
    if (r == PDMTS_OK)
        r = pd->alloc_link_state();
    if (r == PDMTS_OK)
        r = fe_assemble(fe, bl, weight_kind);
    if (r == PDMTS_OK)
        r = build_constraint(A);
    if (r == PDMTS_OK) {
        int lo_prio = 0, hi_prio = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) != cudaSuccess ||
            cudaStreamCreateWithPriority(&A->fe_stream, cudaStreamNonBlocking, hi_prio) != cudaSuccess ||
            cudaEventCreateWithFlags(&A->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&A->ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&A->ev_flag, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&A->h_changed, sizeof(unsigned long long)) != cudaSuccess)
            r = fail(PDMTS_ERR_CUDA, "arlequin_bind: stream/event creation failed");
    }
    if (r != PDMTS_OK) {
        std::string msg = pdmts_last_error();
        A->release_all();
        if (A->fe_stream) cudaStreamDestroy(A->fe_stream);
        if (A->ev_fork) cudaEventDestroy(A->ev_fork);
        if (A->ev_join) cudaEventDestroy(A->ev_join);
        if (A->ev_flag) cudaEventDestroy(A->ev_flag);
        if (A->h_changed) cudaFreeHost(A->h_changed);
        delete A;
        return fail(r, "%s", msg.c_str());
    }
    *A->h_changed = 0;
    ctx->arl = A;
    *out = A;
    return PDMTS_OK;
}

static void batch_drop_member(pdmts_batch *b, pdmts_ctx *c);

extern "C" int arlequin_destroy(pdmts_arl *A)
{
    clear_error();
    if (!A)
        return PDMTS_OK;
    if (A->batch)
        batch_drop_member(A->batch, A->ctx);  // the batch goes on without this member
    cudaSetDevice(A->ctx->device);
    cudaStreamSynchronize(A->ctx->stream);
    if (A->fe_stream) {
        cudaStreamSynchronize(A->fe_stream);
        cudaStreamDestroy(A->fe_stream);
    }
    if (A->ev_fork) cudaEventDestroy(A->ev_fork);
    if (A->ev_join) cudaEventDestroy(A->ev_join);
    if (A->ev_flag) cudaEventDestroy(A->ev_flag);
    if (A->h_changed) cudaFreeHost(A->h_changed);
    if (A->solver) cusolverDnDestroy(A->solver);
    if (A->ctx->arl == A)
        A->ctx->arl = nullptr;
    A->release_all();
    delete A;
    return PDMTS_OK;
}

extern "C" int mts_destroy_coupling(pdmts_ctx *ctx)
{
    if (ctx && ctx->arl)
        arlequin_destroy(ctx->arl);
    if (ctx && ctx->fem)
        fem_destroy(ctx->fem);
    return PDMTS_OK;
}

int mts_time_changed(pdmts_ctx *ctx)
{
    if (ctx->arl) {
        ctx->arl->H_valid = false;
        ctx->arl->Hfe_valid = false;
    }
    return PDMTS_OK;
}

// ------------------------------------------------- coarse step phases -----
// One coarse step of Algorithm 1 is enqueued in phases so that a batch of
// coupled problems can interleave them around batched PD substeps:
//   step_prepare     host: rebuild flag of the previous step, schedules, H;
//   step_free_begin  s: fork mark, interface force of lambda_0 (Eq. 48a);
//   (m free PD substeps with factor 1 - j/m)
//   step_fe_free     fs: FE free step (Eq. 47a);
//   step_lambda      s: join, lambda_m = (-H)^-1 (G_FE v_FE - G_PD v_PD) (Eq. 49);
//   step_fe_link     fs: the FE correction (Eq. 47b);
//   step_link_begin  s: interface force of lambda_m, W_0 = 0 (Eq. 48b);
//   (m link PD substeps with factor j/m)
//   step_finish      s: U += W, rebuild flag, lambda_0 <- lambda_m, join fs.
static int batch_settle(pdmts_batch *b);

static int step_prepare(pdmts_arl *A, cudaStream_t s)
{
    pdmts_ctx *ctx = A->ctx;
    pdmts_pd *pd = A->pd;
    const int m = ctx->m_ratio;
    // a round of a batch this member belongs to may still be in flight
    if (A->batch)
        PDMTS_TRY(batch_settle(A->batch));
    // rebuild flag of the previous step (a bond near an overlap band broke)
    if (A->flag_pending) {
        PDMTS_CUDA_TRY(cudaEventSynchronize(A->ev_flag));
        if (*A->h_changed)
            A->H_valid = false;
        A->flag_pending = false;
    }
    if (A->built_m != m || (int)A->theta_free.size() != m) {
        A->theta_free.resize((size_t)m);
        A->theta_link.resize((size_t)m);
        for (int j = 1; j <= m; ++j) {
            A->theta_free[(size_t)j - 1] = 1.0 - (double)j / m;  // S_j = (1 - j/m) lambda_0
            A->theta_link[(size_t)j - 1] = (double)j / m;        // (j/m) lambda_m
        }
        PDMTS_TRY(update_near_flags(A, m));
        A->H_valid = false;
        pd_invalidate_graphs(pd);
        // the link problem starts from the current bond state
        PDMTS_CUDA_TRY(cudaMemcpyAsync(pd->d_mask_link.p, pd->d_mask.p, sizeof(uint32_t) * pd->n_mask_words,
                                       cudaMemcpyDeviceToDevice, s));
    }
    PDMTS_TRY(fe_prepare_keff(A->fe, m * ctx->dt_pd, ctx->beta_fe));
    PDMTS_TRY(pd->tune_lattice(s));
    PDMTS_TRY(pd->ensure_init(s));
    if (!A->H_valid)
        PDMTS_TRY(build_H(A, m));
    return PDMTS_OK;
}

// may_skip: the free-chain force may be taken from the previous step's
// link-force launch (not in a captured round, whose replays must each
// compute it)
static int step_free_begin(pdmts_arl *A, cudaStream_t s, int64_t *launches, bool may_skip = false)
{
    pdmts_pd *pd = A->pd;
    const bool f64 = pd->precision == PDMTS_FP64;
    // the FE free step may start once the previous step has ended
    PDMTS_CUDA_TRY(cudaEventRecord(A->ev_fork, s));
    if (may_skip && A->g0_ready)  // written by the previous step's link force (same lambda)
        return PDMTS_OK;
    cudaError_t e = launch_interface_force(pd->dim, pd->n, A->n_ov, A->d_ov_node.p, A->d_ov_k.p, A->d_ov_N.p, A->corners,
                                           A->d_lam0.p, A->nl, f64 ? 0.0 : 1.0 / pd->h, f64 ? pd->d_g.p : nullptr,
                                           f64 ? nullptr : pd->f_g.p, s);
    if (e != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "interface force: %s", cudaGetErrorString(e));
    ++*launches;
    return PDMTS_OK;
}

// graphs: replay the FE sequences as captured graphs (not while the caller
// captures the step itself)
static int step_fe_free(pdmts_arl *A, cudaStream_t fs, bool graphs, int64_t *launches)
{
    pdmts_ctx *ctx = A->ctx;
    const double dtf = ctx->m_ratio * ctx->dt_pd;
    PDMTS_CUDA_TRY(cudaStreamWaitEvent(fs, A->ev_fork, 0));
    if (graphs)
        PDMTS_TRY(fe_free_step(A->fe, dtf, ctx->beta_fe, ctx->gamma_fe, fs, launches));
    else
        PDMTS_TRY(fe_free_enqueue(A->fe, dtf, ctx->beta_fe, ctx->gamma_fe, fs, launches));
    PDMTS_CUDA_TRY(cudaEventRecord(A->ev_join, fs));
    return PDMTS_OK;
}

// fe_join: wait for the member's own FE free step (a batch orders its batched
// FE solves itself)
static int step_lambda(pdmts_arl *A, cudaStream_t s, int64_t *launches, bool fe_join = true)
{
    pdmts_pd *pd = A->pd;
    pdmts_fem *fe = A->fe;
    const bool f64 = pd->precision == PDMTS_FP64;
    if (fe_join)
        PDMTS_CUDA_TRY(cudaStreamWaitEvent(s, A->ev_join, 0));
    const float4 *v4 = f64 ? nullptr : pd->f_v4.p;
    const float2 *v2 = f64 ? nullptr : pd->f_v2.p;
    // FP32-bulk: the product in FP32 pairs (FP64-level accuracy at the FP32
    // rate); FP64: the FP64 product
    const bool df = !f64 && A->product_kind == PDMTS_PRODUCT_AUTO && A->d_Hinv_df.p &&
                    A->d_Hinv_df.count == A->nlam * A->nlam;
    cudaError_t e = launch_constraint(pd->dim, A->nl, A->d_gpd_ptr.p, A->d_gpd_col.p, A->d_gpd_val.p, pd->n,
                                      f64 ? pd->d_v.p : nullptr, v4, v2, pd->h, A->d_gfe_col.p, A->d_gfe_val.p,
                                      A->gfe_w, fe->n, fe->d_v.p, -1.0, 1.0, A->d_y.p, s, df ? A->d_ydf.p : nullptr);
    if (e != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "interface residual: %s", cudaGetErrorString(e));
    if (df)
        k_gemv_df<<<blocks(A->nlam * 32), 256, 0, s>>>(A->nlam, A->d_Hinv_df.p, A->d_ydf.p, A->d_df_scale.p,
                                                        A->d_lam.p);
    else
        k_gemv_rows<<<blocks(A->nlam * 32), 256, 0, s>>>(A->nlam, A->d_Hneg_inv.p, A->d_y.p, 1.0, A->d_lam.p);
    *launches += 2;
    return PDMTS_OK;
}

// FE correction U = V + Y lambda_m on the FE stream, after lambda_m on s.
static int step_fe_link(pdmts_arl *A, cudaStream_t s, cudaStream_t fs, bool graphs, int64_t *launches)
{
    pdmts_ctx *ctx = A->ctx;
    const double dtf = ctx->m_ratio * ctx->dt_pd;
    PDMTS_CUDA_TRY(cudaEventRecord(A->ev_fork, s));
    PDMTS_CUDA_TRY(cudaStreamWaitEvent(fs, A->ev_fork, 0));
    if (graphs)
        PDMTS_TRY(fe_link_step(A, dtf, ctx->beta_fe, ctx->gamma_fe, fs, launches));
    else
        PDMTS_TRY(fe_link_enqueue(A, dtf, ctx->beta_fe, ctx->gamma_fe, fs, launches));
    PDMTS_CUDA_TRY(cudaEventRecord(A->ev_join, fs));
    return PDMTS_OK;
}

static int step_link_begin(pdmts_arl *A, const double *dev_lam, cudaStream_t s, int64_t *launches)
{
    pdmts_pd *pd = A->pd;
    const bool f64 = pd->precision == PDMTS_FP64;
    // lambda_m becomes the next step's lambda_0 (step_finish): its force is
    // also the next free chain's, written now into the free-chain field (the
    // free chain of this step has finished)
    const bool next_g0 = dev_lam == A->d_lam.p;
    cudaError_t e = launch_interface_force(pd->dim, pd->n, A->n_ov, A->d_ov_node.p, A->d_ov_k.p, A->d_ov_N.p, A->corners,
                                           dev_lam, A->nl, f64 ? 0.0 : 1.0 / pd->h, f64 ? pd->lk_g.p : nullptr,
                                           f64 ? nullptr : pd->lk_gf.p, s,
                                           next_g0 && f64 ? pd->d_g.p : nullptr,
                                           next_g0 && !f64 ? pd->f_g.p : nullptr);
    if (e != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "interface force: %s", cudaGetErrorString(e));
    A->g0_ready = next_g0;
    ++*launches;
    PDMTS_TRY(pd->zero_link_state(s));
    return PDMTS_OK;
}

static int step_finish(pdmts_arl *A, cudaStream_t s, int64_t *launches, bool fe_join = true)
{
    pdmts_ctx *ctx = A->ctx;
    pdmts_pd *pd = A->pd;
    const bool f64 = pd->precision == PDMTS_FP64;
    PDAddLink L{};
    L.dim = pd->dim;
    L.n = pd->n;
    for (int w = 0; w < 2; ++w) {
        L.seg_lo[w] = pd->link_seg_lo[w];
        L.seg_n[w] = pd->link_seg_n[w];
    }
    L.dt = ctx->dt_pd;
    L.hdt2 = 0.5 * ctx->dt_pd * ctx->dt_pd;
    if (f64) {
        L.u = pd->d_u[pd->cur].p;
        L.u_pred = pd->d_u[1 - pd->cur].p;
        L.v = pd->d_v.p;
        L.a = pd->d_a.p;
        L.wu = pd->lk_u[pd->lk_cur].p;
        L.wv = pd->lk_v.p;
        L.wa = pd->lk_a.p;
    } else {
        L.u4 = pd->f_u4[pd->cur].p;
        L.u2 = pd->f_u2[pd->cur].p;
        L.u4_pred = pd->f_u4[1 - pd->cur].p;
        L.u2_pred = pd->f_u2[1 - pd->cur].p;
        L.v4 = pd->f_v4.p;
        L.v2 = pd->f_v2.p;
        L.af = pd->f_a.p;
        L.wu4 = pd->lk_u4[pd->lk_cur].p;
        L.wu2 = pd->lk_u2[pd->lk_cur].p;
        L.wv4 = pd->lk_v4.p;
        L.wv2 = pd->lk_v2.p;
        L.waf = pd->lk_af.p;
    }
    // one launch: U_PD += W; the rebuild flag (bonds near a band broken this
    // step) counted; the bond words copied into the next step's start words
    // and lambda_m into lambda_0 (the counter is cleared within the step, so
    // a captured round replays correctly)
    unsigned long long *cnt = A->d_changed.p;
    PDMTS_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    cudaError_t e = launch_finish_step(L, pd->n_mask_words, pd->d_mask.p, pd->d_mask_link.p, A->d_near.p, cnt,
                                       A->nlam, A->d_lam.p, A->d_lam0.p, s);
    if (e != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "PD correction and rebuild flag: %s", cudaGetErrorString(e));
    PDMTS_CUDA_TRY(cudaMemcpyAsync(A->h_changed, cnt, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    PDMTS_CUDA_TRY(cudaEventRecord(A->ev_flag, s));
    A->flag_pending = true;
    // the step ends when the FE correction has also finished
    if (fe_join)
        PDMTS_CUDA_TRY(cudaStreamWaitEvent(s, A->ev_join, 0));
    *launches += 1;
    ctx->stats.coarse_steps += 1;
    return PDMTS_OK;
}

// One coarse step of Algorithm 1.
static int coarse_step(pdmts_arl *A)
{
    pdmts_ctx *ctx = A->ctx;
    pdmts_pd *pd = A->pd;
    cudaStream_t s = ctx->stream;
    const int m = ctx->m_ratio;
    int64_t launches = 0;
    PDMTS_TRY(step_prepare(A, s));
    std::array<cudaEvent_t, 5> ph{};
    PDMTS_TRY(ctx->mark(&ph[0]));
    // the PD chain is enqueued before the FE step so that it starts without waiting for the host
    PDMTS_TRY(step_free_begin(A, s, &launches, true));
    PDMTS_TRY(pd_run_chain(pd, m, 1, A->theta_free.data(), s, false));
    PDMTS_TRY(step_fe_free(A, A->fe_stream, true, &launches));
    PDMTS_CUDA_TRY(cudaStreamWaitEvent(s, A->ev_join, 0));
    PDMTS_TRY(ctx->mark(&ph[1]));
    PDMTS_TRY(step_lambda(A, s, &launches));
    PDMTS_TRY(ctx->mark(&ph[2]));
    PDMTS_TRY(step_fe_link(A, s, A->fe_stream, true, &launches));
    PDMTS_TRY(step_link_begin(A, A->d_lam.p, s, &launches));
    PDMTS_TRY(pd_run_chain(pd, m, 2, A->theta_link.data(), s, true));
    PDMTS_TRY(ctx->mark(&ph[3]));
    PDMTS_TRY(step_finish(A, s, &launches));
    PDMTS_TRY(ctx->mark(&ph[4]));
    if (ph[0])
        ctx->phase_marks.push_back(ph);
    ctx->stats.kernel_launches += launches;
    PDMTS_CUDA_TRY(cudaGetLastError());
    return PDMTS_OK;
}

int mts_advance_coupled(pdmts_ctx *ctx, int64_t n_coarse)
{
    PDMTS_CUDA_TRY(cudaSetDevice(ctx->device));
    PDMTS_TRY(ctx->begin());
    for (int64_t k = 0; k < n_coarse; ++k)
        PDMTS_TRY(coarse_step(ctx->arl));
    return ctx->end();
}

// ------------------------------------------------------------- batches ----
// Several independent coupled problems (members, one context each, on one
// device) advanced together: every round takes each member through one of
// its own coarse steps, and the PD substeps of all members that are in the
// same substep slot run as one batched launch over a work list of (member,
// tile). Per member the kernels and their arguments are those of its own
// coarse step, so the batch reproduces each member's solo run bit for bit.
struct pdmts_batch {
    int device = 0;
    std::vector<pdmts_ctx *> members;
    cudaStream_t s = nullptr;               // batched substeps and per-member interface work
    std::vector<cudaStream_t> fe_streams;   // per-member work, members round-robin
    std::vector<cudaEvent_t> ev_lane;       // one per member stream: its part of a phase is done
    cudaEvent_t ev_in = nullptr, ev_end = nullptr, ev_phase = nullptr;
    cudaEvent_t ev_t[6] = {};               // marks of the last round (phase times)
    // batched FE solves: their stream, events, and the device table of the members' FE subdomains
    cudaStream_t fs = nullptr;
    cudaEvent_t ev_fe_free = nullptr, ev_fe_link = nullptr;
    FeDev *d_fe = nullptr;
    int2 *d_feblk = nullptr;
    int nfeblk = 0, itmax = 0;
    std::vector<uint64_t> fe_key;
    int tile = -1;                          // batched lattice tile configuration (-1: tune)
    // argument blocks and work lists of one phase's slots: host staging (pinned) and device copies
    Lat2DArgs *h_args = nullptr;
    int2 *h_work = nullptr;
    Lat2DArgs *d_args = nullptr;
    int2 *d_work = nullptr;
    int64_t cap_args = 0, cap_work = 0;
    int64_t rounds = 0, work_items = 0, batched_launches = 0, kernel_launches = 0;
    bool pending = false;                   // a round is in flight (staging in use)
    // the argument blocks and work lists of a phase depend only on what the key
    // records (buffer parities, schedules, windows, pointers): built once, kept
    struct Plan {
        std::vector<uint64_t> key;
        Lat2DArgs *d_args = nullptr;
        int2 *d_work = nullptr;
        std::vector<int64_t> arg_off, work_off;
    };
    std::vector<Plan> plans;
    struct RoundGraph {
        std::vector<uint64_t> key;
        cudaGraphExec_t exec = nullptr;
        std::vector<struct MemberSnap> after, delta;
        int64_t work_items = 0, batched_launches = 0, kernel_launches = 0;
    };
    std::vector<RoundGraph> graphs;
};

static void batch_free_buffers(pdmts_batch *b)
{
    if (b->h_args) cudaFreeHost(b->h_args);
    if (b->h_work) cudaFreeHost(b->h_work);
    if (b->d_args) cudaFree(b->d_args);
    if (b->d_work) cudaFree(b->d_work);
    b->h_args = nullptr; b->h_work = nullptr; b->d_args = nullptr; b->d_work = nullptr;
    b->cap_args = b->cap_work = 0;
}

static int batch_reserve(pdmts_batch *b, int64_t nargs, int64_t nwork)
{
    if (nargs <= b->cap_args && nwork <= b->cap_work)
        return PDMTS_OK;
    batch_free_buffers(b);
    const int64_t na = std::max<int64_t>(nargs, 1), nw = std::max<int64_t>(nwork, 1);
    if (cudaMallocHost(&b->h_args, sizeof(Lat2DArgs) * na) != cudaSuccess ||
        cudaMallocHost(&b->h_work, sizeof(int2) * nw) != cudaSuccess ||
        cudaMalloc(&b->d_args, sizeof(Lat2DArgs) * na) != cudaSuccess ||
        cudaMalloc(&b->d_work, sizeof(int2) * nw) != cudaSuccess) {
        batch_free_buffers(b);
        return fail(PDMTS_ERR_NOMEM, "batch: staging of %lld argument blocks and %lld work items failed",
                    (long long)na, (long long)nw);
    }
    b->cap_args = na;
    b->cap_work = nw;
    return PDMTS_OK;
}

static std::vector<uint64_t> batch_plan_key(const pdmts_batch *b, bool link)
{
    std::vector<uint64_t> k{(uint64_t)link, (uint64_t)b->tile};
    for (pdmts_ctx *c : b->members) {
        const pdmts_pd *pd = c->arl->pd;
        double dt = c->dt_pd;
        uint64_t dtb;
        std::memcpy(&dtb, &dt, sizeof dtb);
        k.insert(k.end(), {(uint64_t)(link ? pd->lk_cur : pd->cur), (uint64_t)c->m_ratio, dtb,
                           (uint64_t)pd->link_win_lo[0], (uint64_t)pd->link_win_n[0], (uint64_t)pd->link_win_lo[1],
                           (uint64_t)pd->link_win_n[1], (uint64_t)pd->has_g, (uint64_t)pd->breaking,
                           (uint64_t)(uintptr_t)pd->f_u4[0].p, (uint64_t)(uintptr_t)pd->f_u4[1].p,
                           (uint64_t)(uintptr_t)pd->lk_u4[0].p, (uint64_t)(uintptr_t)pd->f_wb.p});
    }
    return k;
}

static void batch_free_plans(pdmts_batch *b)
{
    for (auto &p : b->plans) {
        if (p.d_args) cudaFree(p.d_args);
        if (p.d_work) cudaFree(p.d_work);
    }
    b->plans.clear();
}

// The slots of one phase (free or link) of the current round: one batched
// launch per slot over the members whose chain has that substep, with the
// arguments each member's own substep would take. Each member's buffer parity
// and counters advance as if it had run the substeps itself.
static int batch_plan(pdmts_batch *b, bool link, pdmts_batch::Plan **out)
{
    const int nm = (int)b->members.size();
    int M = 0;
    for (pdmts_ctx *c : b->members)
        M = std::max(M, c->m_ratio);
    const std::vector<uint64_t> key = batch_plan_key(b, link);
    pdmts_batch::Plan *plan = nullptr;
    for (auto &p : b->plans)
        if (p.key == key)
            plan = &p;
    if (!plan) {
        if (b->plans.size() >= 8)
            batch_free_plans(b);
        // simulate the parities on copies of the members' counters, then put them back
        std::vector<int> cur0((size_t)nm);
        for (int i = 0; i < nm; ++i) {
            const pdmts_pd *pd = b->members[(size_t)i]->arl->pd;
            cur0[(size_t)i] = link ? pd->lk_cur : pd->cur;
        }
        pdmts_batch::Plan p;
        p.key = key;
        p.arg_off.assign((size_t)M + 1, 0);
        p.work_off.assign((size_t)M + 1, 0);
        std::vector<Lat2DArgs> args;
        std::vector<int2> work;
        for (int j = 0; j < M; ++j) {
            const int64_t a0 = (int64_t)args.size();
            for (int i = 0; i < nm; ++i) {
                pdmts_ctx *c = b->members[(size_t)i];
                if (j >= c->m_ratio)
                    continue;
                pdmts_arl *A = c->arl;
                pdmts_pd *pd = A->pd;
                int &cur = link ? pd->lk_cur : pd->cur;
                cur = (cur0[(size_t)i] + j) & 1;
                const double theta = link ? A->theta_link[(size_t)j] : A->theta_free[(size_t)j];
                const F32NodeArgs N = pd->f32_node_args(false, theta, link);
                // substep j of a link run evaluates that substep's window, as
                // the member's own link chain does
                pd->chain_k = j;
                Lat2DArgs L = pd->lattice_args(N, link ? pd->d_mask_link.p : pd->d_mask.p, link);
                pd->chain_k = 0;
                L.tile = b->tile;
                const int ntiles = lattice2d_batch_prepare(L, b->tile);
                if (ntiles < 0)
                    return fail(PDMTS_ERR_UNSUPPORTED, "batch: tile configuration %d cannot be batched", b->tile);
                const int slot_index = (int)((int64_t)args.size() - a0);
                for (int t = 0; t < ntiles; ++t)
                    work.push_back(make_int2(slot_index, t));
                args.push_back(L);
            }
            p.arg_off[(size_t)j + 1] = (int64_t)args.size();
            p.work_off[(size_t)j + 1] = (int64_t)work.size();
        }
        for (int i = 0; i < nm; ++i) {
            pdmts_pd *pd = b->members[(size_t)i]->arl->pd;
            (link ? pd->lk_cur : pd->cur) = cur0[(size_t)i];
        }
        if (cudaMalloc(&p.d_args, sizeof(Lat2DArgs) * std::max<size_t>(args.size(), 1)) != cudaSuccess ||
            cudaMalloc(&p.d_work, sizeof(int2) * std::max<size_t>(work.size(), 1)) != cudaSuccess) {
            if (p.d_args) cudaFree(p.d_args);
            if (p.d_work) cudaFree(p.d_work);
            return fail(PDMTS_ERR_NOMEM, "batch: plan of %zu work items", work.size());
        }
        PDMTS_CUDA_TRY(cudaMemcpy(p.d_args, args.data(), sizeof(Lat2DArgs) * args.size(), cudaMemcpyHostToDevice));
        PDMTS_CUDA_TRY(cudaMemcpy(p.d_work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice));
        b->plans.push_back(std::move(p));
        plan = &b->plans.back();
    }
    *out = plan;
    return PDMTS_OK;
}

static int batch_phase(pdmts_batch *b, bool link)
{
    const int nm = (int)b->members.size();
    int M = 0;
    for (pdmts_ctx *c : b->members)
        M = std::max(M, c->m_ratio);
    pdmts_batch::Plan *plan = nullptr;
    PDMTS_TRY(batch_plan(b, link, &plan));
    const bool pmb = b->members[0]->arl->pd->force_kind == PDMTS_FORCE_PMB;
    for (int j = 0; j < M; ++j) {
        const int nwork = (int)(plan->work_off[(size_t)j + 1] - plan->work_off[(size_t)j]);
        cudaError_t e = launch_lattice2d_batch(plan->d_args + plan->arg_off[(size_t)j],
                                               plan->d_work + plan->work_off[(size_t)j], nwork, b->tile, pmb, b->s);
        if (e != cudaSuccess)
            return fail(PDMTS_ERR_CUDA, "batched substep: %s", cudaGetErrorString(e));
        b->batched_launches += 1;
        b->kernel_launches += 1;
        b->work_items += nwork;
        for (int i = 0; i < nm; ++i)
            if (j < b->members[(size_t)i]->m_ratio) {
                pdmts_pd *pd = b->members[(size_t)i]->arl->pd;
                pd->chain_k = j;  // the bonds substep j evaluates
                pd->substep_done(false, link);
                pd->chain_k = 0;
            }
    }
    return PDMTS_OK;
}

// Batch tile autotuner: one batched link-mode substep (no breaking, whole
// lattices) per configuration on the members' link-state buffers, which are
// scratch between link runs (cleared afterwards); keeps the fastest.
static int batch_tune(pdmts_batch *b)
{
    if (b->tile >= 0)
        return PDMTS_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PDMTS_CUDA_TRY(cudaEventCreate(&e0));
    PDMTS_CUDA_TRY(cudaEventCreate(&e1));
    int best = 0;
    float best_ms = 0.f;
    int r = PDMTS_OK;
    for (int t = 0; t < kLatBatchTiles && r == PDMTS_OK; ++t) {
        std::vector<Lat2DArgs> args;
        std::vector<int2> work;
        for (size_t i = 0; i < b->members.size(); ++i) {
            pdmts_pd *pd = b->members[i]->arl->pd;
            F32NodeArgs N = pd->f32_node_args(false, 0.0, true);
            N.broken = nullptr;
            Lat2DArgs L = pd->lattice_args(N, pd->d_mask_link.p, false);  // whole lattice
            const int ntiles = lattice2d_batch_prepare(L, t);
            for (int k = 0; k < ntiles; ++k)
                work.push_back(make_int2((int)args.size(), k));
            args.push_back(L);
        }
        if ((r = batch_reserve(b, (int64_t)args.size(), (int64_t)work.size())) != PDMTS_OK)
            break;
        std::memcpy(b->h_args, args.data(), sizeof(Lat2DArgs) * args.size());
        std::memcpy(b->h_work, work.data(), sizeof(int2) * work.size());
        cudaError_t e = cudaMemcpyAsync(b->d_args, b->h_args, sizeof(Lat2DArgs) * args.size(), cudaMemcpyHostToDevice, b->s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_work, b->h_work, sizeof(int2) * work.size(), cudaMemcpyHostToDevice, b->s);
        const bool pmb = b->members[0]->pd->force_kind == PDMTS_FORCE_PMB;
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
            if (k == 1)
                e = cudaEventRecord(e0, b->s);
            if (e == cudaSuccess)
                e = launch_lattice2d_batch(b->d_args, b->d_work, (int)work.size(), t, pmb, b->s);
        }
        if (e == cudaSuccess)
            e = cudaEventRecord(e1, b->s);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess)
            r = fail(PDMTS_ERR_CUDA, "batch autotune: %s", cudaGetErrorString(e));
        else if (t == 0 || ms < best_ms) {
            best = t;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != PDMTS_OK)
        return r;
    for (pdmts_ctx *c : b->members)
        PDMTS_TRY(c->arl->pd->zero_link_state(b->s, true));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(b->s));
    b->tile = best;
    return PDMTS_OK;
}

// Member streams wait for the batch stream (ev_phase just recorded on b->s),
// or the batch stream for every member stream.
static int batch_fan_out(pdmts_batch *b)
{
    PDMTS_CUDA_TRY(cudaEventRecord(b->ev_phase, b->s));
    for (cudaStream_t f : b->fe_streams)
        PDMTS_CUDA_TRY(cudaStreamWaitEvent(f, b->ev_phase, 0));
    return PDMTS_OK;
}
static int batch_fan_in(pdmts_batch *b)
{
    for (size_t k = 0; k < b->fe_streams.size(); ++k) {
        PDMTS_CUDA_TRY(cudaEventRecord(b->ev_lane[k], b->fe_streams[k]));
        PDMTS_CUDA_TRY(cudaStreamWaitEvent(b->s, b->ev_lane[k], 0));
    }
    return PDMTS_OK;
}

// One round: per member on its stream (members round-robin over the member
// streams) the small coupling kernels, and on the batch stream the batched
// substep slots; the FE solves run beside the PD slots.
// Device table of the members' FE subdomains for the batched FE kernels
// (rebuilt when a member's schedule or arrays change).
static int batch_fe_table(pdmts_batch *b)
{
    std::vector<uint64_t> key;
    for (pdmts_ctx *c : b->members) {
        const pdmts_fem *fe = c->arl->fe;
        key.insert(key.end(), {(uint64_t)fe->keff_version, (uint64_t)(uintptr_t)fe->d_cheb.p,
                               (uint64_t)(uintptr_t)fe->d_u.p, (uint64_t)(uintptr_t)fe->d_Keff.p});
    }
    if (key == b->fe_key && b->d_fe)
        return PDMTS_OK;
    std::vector<FeDev> devs;
    std::vector<int2> blk;
    b->itmax = 0;
    for (size_t i = 0; i < b->members.size(); ++i) {
        pdmts_ctx *c = b->members[i];
        pdmts_arl *A = c->arl;
        pdmts_fem *fe = A->fe;
        if (!fe->paired_rows)
            return fail(PDMTS_ERR_UNSUPPORTED, "batch: member %zu: FE rows of a node do not share columns", i);
        FeDev F{};
        F.nfe = fe->n;
        F.nl = A->nl;
        F.W = fe->W;
        F.it = (int)fe->cheb_c1.size();
        F.col = fe->d_col.p;
        F.K = fe->d_K.p;
        F.Keff = fe->d_Keff.p;
        F.Minv = fe->d_Minv.p;
        F.P = fe->d_P.p;
        F.cheb = fe->d_cheb.p;
        F.u = fe->d_u.p; F.v = fe->d_v.p; F.a = fe->d_a.p; F.ut = fe->d_ut.p; F.vt = fe->d_vt.p;
        F.b = fe->d_b.p; F.r = fe->d_r.p; F.d0 = fe->d_d[0].p; F.d1 = fe->d_d[1].p;
        F.aw = fe->d_aw.p; F.bw = fe->d_bw.p;
        F.inv_theta = 1.0 / fe->cheb_theta;
        F.dt = c->m_ratio * c->dt_pd;
        F.beta = c->beta_fe;
        F.gamma = c->gamma_fe;
        F.gT_ptr = A->d_gfeT_ptr.p;
        F.gT_k = A->d_gfeT_k.p;
        F.gT_val = A->d_gfeT_val.p;
        F.lam = A->d_lam.p;
        b->itmax = std::max(b->itmax, F.it);
        for (int64_t n0 = 0; n0 < fe->n; n0 += 256)
            blk.push_back(make_int2((int)i, (int)n0));
        devs.push_back(F);
    }
    if (b->d_fe) cudaFree(b->d_fe);
    if (b->d_feblk) cudaFree(b->d_feblk);
    b->d_fe = nullptr;
    b->d_feblk = nullptr;
    if (cudaMalloc(&b->d_fe, sizeof(FeDev) * devs.size()) != cudaSuccess ||
        cudaMalloc(&b->d_feblk, sizeof(int2) * std::max<size_t>(blk.size(), 1)) != cudaSuccess)
        return fail(PDMTS_ERR_NOMEM, "batch: FE table");
    PDMTS_CUDA_TRY(cudaMemcpy(b->d_fe, devs.data(), sizeof(FeDev) * devs.size(), cudaMemcpyHostToDevice));
    PDMTS_CUDA_TRY(cudaMemcpy(b->d_feblk, blk.data(), sizeof(int2) * blk.size(), cudaMemcpyHostToDevice));
    b->nfeblk = (int)blk.size();
    b->fe_key = key;
    return PDMTS_OK;
}

// The batched FE free step (link = false) or FE correction on b->fs.
static int batch_fe(pdmts_batch *b, bool link)
{
    if (b->nfeblk == 0)
        return PDMTS_OK;
    if (link)
        k_feb_link_init<<<b->nfeblk, 256, 0, b->fs>>>(b->d_fe, b->d_feblk);
    else {
        k_feb_predict<<<b->nfeblk, 256, 0, b->fs>>>(b->d_fe, b->d_feblk);
        k_feb_residual<<<b->nfeblk, 256, 0, b->fs>>>(b->d_fe, b->d_feblk);
    }
    for (int k = 0; k < b->itmax; ++k) {
        // each iteration a programmatic dependent of the kernel before it
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)b->nfeblk);
        cfg.blockDim = dim3(256);
        cfg.stream = b->fs;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        PDMTS_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_feb_cheb, (const FeDev *)b->d_fe, (const int2 *)b->d_feblk, k,
                                          link ? 1 : 0));
    }
    k_feb_finish<<<b->nfeblk, 256, 0, b->fs>>>(b->d_fe, b->d_feblk, link ? 1 : 0);
    PDMTS_CUDA_TRY(cudaGetLastError());
    return PDMTS_OK;
}

// The round's work; enqueued only while b->s is captured (the phase marks
// are external event nodes, so the events can be read after a replay).
static int batch_enqueue_round(pdmts_batch *b, bool graphs)
{
    (void)graphs;
    const size_t nm = b->members.size();
    const size_t K = b->fe_streams.size();
    std::vector<int64_t> launches(nm, 0);
    auto lane = [&](size_t i) { return b->fe_streams[i % K]; };
    PDMTS_CUDA_TRY(cudaEventRecordWithFlags(b->ev_t[0], b->s, cudaEventRecordExternal));
    // FE free steps of all members (batched) beside the PD free substeps
    PDMTS_CUDA_TRY(cudaEventRecord(b->ev_phase, b->s));
    PDMTS_CUDA_TRY(cudaStreamWaitEvent(b->fs, b->ev_phase, 0));
    PDMTS_TRY(batch_fe(b, false));
    PDMTS_CUDA_TRY(cudaEventRecord(b->ev_fe_free, b->fs));
    // interface forces of lambda_0
    PDMTS_TRY(batch_fan_out(b));
    for (size_t i = 0; i < nm; ++i)
        PDMTS_TRY(step_free_begin(b->members[i]->arl, lane(i), &launches[i]));
    PDMTS_TRY(batch_fan_in(b));
    PDMTS_CUDA_TRY(cudaEventRecordWithFlags(b->ev_t[1], b->s, cudaEventRecordExternal));
    PDMTS_TRY(batch_phase(b, false));
    PDMTS_CUDA_TRY(cudaEventRecordWithFlags(b->ev_t[2], b->s, cudaEventRecordExternal));
    // lambda_m and the link-problem start
    PDMTS_TRY(batch_fan_out(b));
    for (cudaStream_t f : b->fe_streams)
        PDMTS_CUDA_TRY(cudaStreamWaitEvent(f, b->ev_fe_free, 0));
    for (size_t i = 0; i < nm; ++i) {
        pdmts_arl *A = b->members[i]->arl;
        PDMTS_TRY(step_lambda(A, lane(i), &launches[i], false));
        PDMTS_TRY(step_link_begin(A, A->d_lam.p, lane(i), &launches[i]));
    }
    PDMTS_TRY(batch_fan_in(b));
    PDMTS_CUDA_TRY(cudaEventRecordWithFlags(b->ev_t[3], b->s, cudaEventRecordExternal));
    // FE corrections of all members (batched) beside the PD link substeps
    PDMTS_CUDA_TRY(cudaEventRecord(b->ev_phase, b->s));
    PDMTS_CUDA_TRY(cudaStreamWaitEvent(b->fs, b->ev_phase, 0));
    PDMTS_TRY(batch_fe(b, true));
    PDMTS_CUDA_TRY(cudaEventRecord(b->ev_fe_link, b->fs));
    PDMTS_TRY(batch_phase(b, true));
    PDMTS_CUDA_TRY(cudaEventRecordWithFlags(b->ev_t[4], b->s, cudaEventRecordExternal));
    // corrections and rebuild flags; the round ends with the FE corrections
    PDMTS_TRY(batch_fan_out(b));
    for (size_t i = 0; i < nm; ++i) {
        PDMTS_TRY(step_finish(b->members[i]->arl, lane(i), &launches[i], false));
        b->kernel_launches += launches[i];
        const pdmts_fem *fe = b->members[i]->arl->fe;
        // the member's share of the batched FE kernels: as many as its own solves would launch
        launches[i] += 2 * (int64_t)fe->cheb_c1.size() + 7;
        b->members[i]->stats.kernel_launches += launches[i];
    }
    PDMTS_TRY(batch_fan_in(b));
    b->kernel_launches += (b->nfeblk > 0 ? 2 * (int64_t)b->itmax + 5 : 0);
    PDMTS_CUDA_TRY(cudaStreamWaitEvent(b->s, b->ev_fe_link, 0));
    PDMTS_CUDA_TRY(cudaEventRecordWithFlags(b->ev_t[5], b->s, cudaEventRecordExternal));
    return PDMTS_OK;
}

// Host-side state a round changes: buffer parities, counters, flags.
struct MemberSnap {
    int cur = 0, lk_cur = 0;
    int64_t steps_done = 0;
    pdmts_stats stats{};
    bool flag_pending = false;
};
static MemberSnap member_snap(const pdmts_ctx *c)
{
    MemberSnap m;
    m.cur = c->arl->pd->cur;
    m.lk_cur = c->arl->pd->lk_cur;
    m.steps_done = c->arl->pd->steps_done;
    m.stats = c->stats;
    m.flag_pending = c->arl->flag_pending;
    return m;
}

static std::vector<uint64_t> batch_round_key(const pdmts_batch *b)
{
    std::vector<uint64_t> k = batch_plan_key(b, false);
    for (pdmts_ctx *c : b->members)
        k.push_back((uint64_t)c->arl->fe->keff_version);
    return k;
}

// One round: per member on its stream (members round-robin over the member
// streams) the small coupling kernels, and on the batch stream the batched
// substep slots; the FE solves run beside the PD slots. The whole round is
// captured once per key (buffer parities, schedules) as a CUDA graph and
// replayed; the host applies the round's bookkeeping to the members.
// Wait for the last round and take its rebuild flags (the flag copies ran
// inside the round; its end event covers them).
static int batch_settle(pdmts_batch *b)
{
    if (!b->pending)
        return PDMTS_OK;
    PDMTS_CUDA_TRY(cudaEventSynchronize(b->ev_end));
    b->pending = false;
    for (pdmts_ctx *c : b->members) {
        pdmts_arl *A = c->arl;
        if (A->flag_pending && *A->h_changed)
            A->H_valid = false;
        A->flag_pending = false;
    }
    return PDMTS_OK;
}

static int batch_round(pdmts_batch *b)
{
    const size_t nm = b->members.size();
    PDMTS_TRY(batch_settle(b));
    for (size_t i = 0; i < nm; ++i) {
        pdmts_arl *A = b->members[i]->arl;
        if (A->pd->lattice_tile < 0)
            A->pd->lattice_tile = b->tile;  // the members' own substeps use the batch's tile (no solo tuning)
        A->batch = nullptr;                 // settled above
        const int r = step_prepare(A, b->s);
        A->batch = b;
        PDMTS_TRY(r);
    }
    // both phases' plans exist before any capture (the link phase starts at parity 0)
    pdmts_batch::Plan *plan = nullptr;
    PDMTS_TRY(batch_plan(b, false, &plan));
    {
        std::vector<int> lk(nm);
        for (size_t i = 0; i < nm; ++i) {
            lk[i] = b->members[i]->arl->pd->lk_cur;
            b->members[i]->arl->pd->lk_cur = 0;
        }
        const int r = batch_plan(b, true, &plan);
        for (size_t i = 0; i < nm; ++i)
            b->members[i]->arl->pd->lk_cur = lk[i];
        PDMTS_TRY(r);
    }
    PDMTS_TRY(batch_fe_table(b));
    const std::vector<uint64_t> key = batch_round_key(b);
    pdmts_batch::RoundGraph *g = nullptr;
    for (auto &rg : b->graphs)
        if (rg.key == key)
            g = &rg;
    if (!g) {
        if (b->graphs.size() >= 4) {
            for (auto &rg : b->graphs)
                cudaGraphExecDestroy(rg.exec);
            b->graphs.clear();
        }
        std::vector<MemberSnap> s0(nm);
        for (size_t i = 0; i < nm; ++i)
            s0[i] = member_snap(b->members[i]);
        const int64_t wi0 = b->work_items, bl0 = b->batched_launches, kl0 = b->kernel_launches;
        cudaGraph_t graph = nullptr;
        PDMTS_CUDA_TRY(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
        const int r = batch_enqueue_round(b, false);
        const cudaError_t ce = cudaStreamEndCapture(b->s, &graph);
        pdmts_batch::RoundGraph rg;
        rg.key = key;
        rg.work_items = b->work_items - wi0;
        rg.batched_launches = b->batched_launches - bl0;
        rg.kernel_launches = b->kernel_launches - kl0;
        b->work_items = wi0;
        b->batched_launches = bl0;
        b->kernel_launches = kl0;
        for (size_t i = 0; i < nm; ++i) {
            pdmts_ctx *c = b->members[i];
            const MemberSnap s1 = member_snap(c);
            rg.after.push_back(s1);
            MemberSnap d = s1;
            d.steps_done -= s0[i].steps_done;
            d.stats.pd_substeps -= s0[i].stats.pd_substeps;
            d.stats.bond_updates -= s0[i].stats.bond_updates;
            d.stats.coarse_steps -= s0[i].stats.coarse_steps;
            d.stats.bonds_broken -= s0[i].stats.bonds_broken;
            d.stats.kernel_launches -= s0[i].stats.kernel_launches;
            d.stats.graph_launches -= s0[i].stats.graph_launches;
            rg.delta.push_back(d);
            c->arl->pd->cur = s0[i].cur;
            c->arl->pd->lk_cur = s0[i].lk_cur;
            c->arl->pd->steps_done = s0[i].steps_done;
            c->stats = s0[i].stats;
            c->arl->flag_pending = s0[i].flag_pending;
        }
        if (r != PDMTS_OK) {
            if (graph)
                cudaGraphDestroy(graph);
            return r;
        }
        if (ce != cudaSuccess)
            return fail(PDMTS_ERR_CUDA, "batch round capture: %s", cudaGetErrorString(ce));
        const cudaError_t ie = cudaGraphInstantiate(&rg.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess)
            return fail(PDMTS_ERR_CUDA, "batch round graph: %s", cudaGetErrorString(ie));
        b->graphs.push_back(std::move(rg));
        g = &b->graphs.back();
    }
    PDMTS_CUDA_TRY(cudaGraphLaunch(g->exec, b->s));
    for (size_t i = 0; i < nm; ++i) {
        pdmts_ctx *c = b->members[i];
        const MemberSnap &a = g->after[i], &d = g->delta[i];
        c->arl->pd->cur = a.cur;
        c->arl->pd->lk_cur = a.lk_cur;
        c->arl->pd->steps_done += d.steps_done;
        c->stats.pd_substeps += d.stats.pd_substeps;
        c->stats.bond_updates += d.stats.bond_updates;
        c->stats.coarse_steps += d.stats.coarse_steps;
        c->stats.kernel_launches += d.stats.kernel_launches;
        c->stats.graph_launches += d.stats.graph_launches;
        c->arl->flag_pending = a.flag_pending;
    }
    b->work_items += g->work_items;
    b->batched_launches += g->batched_launches;
    b->kernel_launches += g->kernel_launches;
    PDMTS_CUDA_TRY(cudaEventRecord(b->ev_end, b->s));
    b->pending = true;
    b->rounds += 1;
    PDMTS_CUDA_TRY(cudaGetLastError());
    return PDMTS_OK;
}

// A member's coupling is being destroyed: wait for the batch, drop the member
// and every cached plan, graph and table that refers to it.
static void batch_drop_member(pdmts_batch *b, pdmts_ctx *c)
{
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->s);
    batch_settle(b);
    b->members.erase(std::remove(b->members.begin(), b->members.end(), c), b->members.end());
    c->arl->batch = nullptr;
    batch_free_plans(b);
    for (auto &rg : b->graphs)
        if (rg.exec)
            cudaGraphExecDestroy(rg.exec);
    b->graphs.clear();
    b->fe_key.clear();
}

extern "C" int mts_batch_create(int n_members, pdmts_ctx *const *members, pdmts_batch **out)
{
    clear_error();
    if (!members || !out || n_members <= 0)
        return fail(PDMTS_ERR_ARG, "mts_batch_create: NULL argument or no members");
    *out = nullptr;
    for (int i = 0; i < n_members; ++i) {
        pdmts_ctx *c = members[i];
        if (!c || !c->arl)
            return fail(PDMTS_ERR_STATE, "mts_batch_create: member %d has no Arlequin coupling", i);
        if (!c->time_set)
            return fail(PDMTS_ERR_STATE, "mts_batch_create: member %d: call mts_set_time first", i);
        pdmts_pd *pd = c->arl->pd;
        if (pd->precision != PDMTS_FP32_BULK || pd->layout != pdmts_pd::LAYOUT_LATTICE2D)
            return fail(PDMTS_ERR_UNSUPPORTED,
                        "mts_batch_create: member %d: batching needs an FP32-bulk PD subdomain on a 2D lattice", i);
        if (c->device != members[0]->device)
            return fail(PDMTS_ERR_ARG, "mts_batch_create: members on different devices");
        if (pd->force_kind != members[0]->arl->pd->force_kind)
            return fail(PDMTS_ERR_ARG, "mts_batch_create: members with different force laws");
        for (int k = 0; k < i; ++k)
            if (members[k] == c)
                return fail(PDMTS_ERR_ARG, "mts_batch_create: member %d appears twice", i);
        if (c->arl->batch)
            return fail(PDMTS_ERR_STATE, "mts_batch_create: member %d already belongs to a batch", i);
    }
    PDMTS_CUDA_TRY(cudaSetDevice(members[0]->device));
    auto *b = new (std::nothrow) pdmts_batch();
    if (!b)
        return fail(PDMTS_ERR_NOMEM, "mts_batch_create: out of host memory");
    b->device = members[0]->device;
    b->members.assign(members, members + n_members);
    int lo = 0, hi = 0;
    bool ok = cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) == cudaSuccess &&
              cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_end, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_phase, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < 6 && ok; ++k)
        ok = cudaEventCreate(&b->ev_t[k]) == cudaSuccess;
    ok = ok && cudaStreamCreateWithPriority(&b->fs, cudaStreamNonBlocking, hi) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_fe_free, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_fe_link, cudaEventDisableTiming) == cudaSuccess;
    const int K = std::min(n_members, 8);
    for (int k = 0; k < K && ok; ++k) {
        cudaStream_t fs = nullptr;
        cudaEvent_t ev = nullptr;
        ok = cudaStreamCreateWithPriority(&fs, cudaStreamNonBlocking, hi) == cudaSuccess;
        if (ok)
            b->fe_streams.push_back(fs);
        ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
        if (ok)
            b->ev_lane.push_back(ev);
    }
    if (!ok) {
        mts_batch_destroy(b);
        return fail(PDMTS_ERR_CUDA, "mts_batch_create: stream/event creation failed");
    }
    for (pdmts_ctx *c : b->members)
        c->arl->batch = b;
    *out = b;
    return PDMTS_OK;
}

extern "C" int mts_batch_advance(pdmts_batch *b, int64_t n_rounds)
{
    clear_error();
    if (!b)
        return fail(PDMTS_ERR_ARG, "mts_batch_advance: batch is NULL");
    if (n_rounds < 0)
        return fail(PDMTS_ERR_ARG, "mts_batch_advance: n_rounds < 0");
    PDMTS_CUDA_TRY(cudaSetDevice(b->device));
    // order the batch after its members' user streams (a member's own stream
    // is ordered into its user stream at the end of every call), once per
    // distinct user stream
    std::vector<cudaStream_t> users;
    for (pdmts_ctx *c : b->members)
        if (std::find(users.begin(), users.end(), c->user_stream) == users.end())
            users.push_back(c->user_stream);
    for (cudaStream_t u : users) {
        PDMTS_CUDA_TRY(cudaEventRecord(b->ev_in, u));
        PDMTS_CUDA_TRY(cudaStreamWaitEvent(b->s, b->ev_in, 0));
    }
    if (b->members.empty())
        return PDMTS_OK;
    for (pdmts_ctx *c : b->members)
        PDMTS_TRY(c->watch_check("mts_batch_advance"));
    PDMTS_TRY(batch_tune(b));
    for (int64_t k = 0; k < n_rounds; ++k)
        PDMTS_TRY(batch_round(b));
    for (pdmts_ctx *c : b->members)
        PDMTS_TRY(c->watch_enqueue(b->s));
    // the users' streams follow the batch; a member's own stream follows its
    // user stream when the member is next used alone
    PDMTS_CUDA_TRY(cudaEventRecord(b->ev_in, b->s));
    for (cudaStream_t u : users)
        PDMTS_CUDA_TRY(cudaStreamWaitEvent(u, b->ev_in, 0));
    return PDMTS_OK;
}

extern "C" int mts_batch_info(const pdmts_batch *b, pdmts_batch_info *info)
{
    clear_error();
    if (!b || !info)
        return fail(PDMTS_ERR_ARG, "mts_batch_info: NULL argument");
    info->n_members = (int32_t)b->members.size();
    info->lattice_tile = b->tile;
    info->rounds = b->rounds;
    info->work_items = b->work_items;
    info->batched_launches = b->batched_launches;
    info->kernel_launches = b->kernel_launches;
    for (int k = 0; k < 5; ++k)
        info->last_round_ms[k] = 0.0;
    if (b->rounds > 0) {
        PDMTS_CUDA_TRY(cudaSetDevice(b->device));
        PDMTS_CUDA_TRY(cudaEventSynchronize(b->ev_t[5]));
        for (int k = 0; k < 5; ++k) {
            float ms = 0.f;
            PDMTS_CUDA_TRY(cudaEventElapsedTime(&ms, b->ev_t[k], b->ev_t[k + 1]));
            info->last_round_ms[k] = ms;
        }
    }
    return PDMTS_OK;
}

extern "C" int mts_batch_destroy(pdmts_batch *b)
{
    if (!b)
        return PDMTS_OK;
    cudaSetDevice(b->device);
    if (b->s)
        cudaStreamSynchronize(b->s);
    batch_settle(b);
    for (pdmts_ctx *c : b->members)
        if (c && c->arl && c->arl->batch == b)
            c->arl->batch = nullptr;
    for (cudaStream_t fs : b->fe_streams) {
        cudaStreamSynchronize(fs);
        cudaStreamDestroy(fs);
    }
    batch_free_buffers(b);
    batch_free_plans(b);
    for (auto &rg : b->graphs)
        if (rg.exec)
            cudaGraphExecDestroy(rg.exec);
    if (b->s) cudaStreamDestroy(b->s);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_end) cudaEventDestroy(b->ev_end);
    if (b->ev_phase) cudaEventDestroy(b->ev_phase);
    if (b->fs) {
        cudaStreamSynchronize(b->fs);
        cudaStreamDestroy(b->fs);
    }
    if (b->ev_fe_free) cudaEventDestroy(b->ev_fe_free);
    if (b->ev_fe_link) cudaEventDestroy(b->ev_fe_link);
    if (b->d_fe) cudaFree(b->d_fe);
    if (b->d_feblk) cudaFree(b->d_feblk);
    for (cudaEvent_t e : b->ev_t)
        if (e)
            cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_lane)
        cudaEventDestroy(e);
    delete b;
    return PDMTS_OK;
}

extern "C" int arlequin_read_lambda(pdmts_arl *A, double *lam, int64_t *n_lambda)
{
    clear_error();
    if (!A || !lam)
        return fail(PDMTS_ERR_ARG, "arlequin_read_lambda: NULL argument");
    PDMTS_CUDA_TRY(cudaSetDevice(A->ctx->device));
    PDMTS_TRY(A->ctx->begin());
    PDMTS_CUDA_TRY(cudaMemcpyAsync(lam, A->d_lam0.p, sizeof(double) * A->nlam, cudaMemcpyDefault, A->ctx->stream));
    PDMTS_TRY(A->ctx->sync_checked("arlequin_read_lambda"));
    if (n_lambda)
        *n_lambda = A->nlam;
    return A->ctx->end();
}

extern "C" int arlequin_set_multiplier_product(pdmts_arl *A, int kind)
{
    clear_error();
    if (!A)
        return fail(PDMTS_ERR_ARG, "arlequin_set_multiplier_product: arl is NULL");
    if (kind != PDMTS_PRODUCT_AUTO && kind != PDMTS_PRODUCT_FP64)
        return fail(PDMTS_ERR_ARG, "arlequin_set_multiplier_product: unknown kind %d", kind);
    A->product_kind = kind;
    return PDMTS_OK;
}

extern "C" int arlequin_constraint_residual(pdmts_arl *A, double *residual, double *reference)
{
    clear_error();
    if (!A || !residual)
        return fail(PDMTS_ERR_ARG, "arlequin_constraint_residual: NULL argument");
    pdmts_pd *pd = A->pd;
    pdmts_fem *fe = A->fe;
    if (!fe->assembled)
        return fail(PDMTS_ERR_STATE, "arlequin_constraint_residual: not assembled");
    PDMTS_CUDA_TRY(cudaSetDevice(A->ctx->device));
    PDMTS_TRY(A->ctx->begin());
    cudaStream_t s = A->ctx->stream;
    const bool f64 = pd->precision == PDMTS_FP64;
    std::vector<double> y((size_t)A->nlam), yf((size_t)A->nlam);
    for (int pass = 0; pass < 2; ++pass) {
        cudaError_t e = launch_constraint(pd->dim, A->nl, A->d_gpd_ptr.p, A->d_gpd_col.p, A->d_gpd_val.p, pd->n,
                                          f64 ? pd->d_v.p : nullptr, f64 ? nullptr : pd->f_v4.p,
                                          f64 ? nullptr : pd->f_v2.p, pd->h, A->d_gfe_col.p, A->d_gfe_val.p,
                                          A->gfe_w, fe->n, fe->d_v.p, pass == 0 ? -1.0 : 0.0, 1.0, A->d_y.p, s);
        if (e != cudaSuccess)
            return fail(PDMTS_ERR_CUDA, "constraint: %s", cudaGetErrorString(e));
        PDMTS_CUDA_TRY(cudaMemcpyAsync(pass == 0 ? y.data() : yf.data(), A->d_y.p, sizeof(double) * A->nlam,
                                       cudaMemcpyDeviceToHost, s));
    }
    PDMTS_TRY(A->ctx->sync_checked("arlequin_constraint_residual"));
    double r2 = 0, f2 = 0;
    for (int64_t k = 0; k < A->nlam; ++k) {
        r2 += y[(size_t)k] * y[(size_t)k];
        f2 += yf[(size_t)k] * yf[(size_t)k];
    }
    *residual = std::sqrt(r2);
    if (reference)
        *reference = std::sqrt(f2);
    return A->ctx->end();
}

extern "C" int arlequin_info(pdmts_arl *A, pdmts_arl_info *info)
{
    clear_error();
    if (!A || !info)
        return fail(PDMTS_ERR_ARG, "arlequin_info: NULL argument");
    info->n_lambda = A->nlam;
    info->n_overlap_pd = A->n_ov;
    info->fe_dofs = A->fe->ndof();
    info->colors = A->colors;
    info->rebuilds = A->rebuilds;
    info->cheb_iterations = (int64_t)A->fe->cheb_c1.size();
    info->device_bytes = A->device_bytes + A->fe->device_bytes;
    return PDMTS_OK;
}

// ------------------------------------------------- checkpoint / resume --
// The time-stepping state of a context as one opaque image: a header that
// identifies the set-up, then the raw device arrays that carry state from one
// coarse step to the next, in a fixed order. Everything else (operators,
// loads, the interface operator, tuned tiles, captured graphs) follows from
// the set-up calls; the interface operator is rebuilt after a load, from the
// bond words near the overlap bands, which by the rebuild rule are the ones
// it was last built from.
namespace {
struct StateHeader {
    char magic[8];
    int32_t version, precision, layout, dim;
    int64_t n, n_mask_words, fe_ndof, nlam;
    int32_t cur, need_init, lk_cur, has_link;
    int64_t steps_done, n_segments, payload_bytes;
};
constexpr char kStateMagic[8] = {'P', 'D', 'M', 'T', 'S', 'S', 'T', '1'};

template <typename T>
static void add_seg(std::vector<std::pair<void *, size_t>> &segs, DevArr<T> &a)
{
    if (a.p)
        segs.emplace_back((void *)a.p, sizeof(T) * (size_t)std::max<int64_t>(a.count, 1));
}

static int state_layout(pdmts_ctx *ctx, StateHeader &h, std::vector<std::pair<void *, size_t>> &segs)
{
    pdmts_pd *pd = ctx->pd;
    if (!pd)
        return fail(PDMTS_ERR_STATE, "checkpoint: the context has no PD subdomain");
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, kStateMagic, sizeof h.magic);
    h.version = 1;
    h.precision = pd->precision;
    h.layout = pd->layout;
    h.dim = pd->dim;
    h.n = pd->n;
    h.n_mask_words = pd->n_mask_words;
    h.cur = pd->cur;
    h.need_init = pd->need_init ? 1 : 0;
    h.lk_cur = pd->lk_cur;
    h.has_link = pd->has_link && pd->d_mask_link.p ? 1 : 0;
    h.steps_done = pd->steps_done;
    segs.clear();
    if (pd->precision == PDMTS_FP64) {
        add_seg(segs, pd->d_u[0]);
        add_seg(segs, pd->d_u[1]);
        add_seg(segs, pd->d_v);
        add_seg(segs, pd->d_a);
    } else {
        add_seg(segs, pd->f_u4[0]);
        add_seg(segs, pd->f_u4[1]);
        add_seg(segs, pd->f_u2[0]);
        add_seg(segs, pd->f_u2[1]);
        add_seg(segs, pd->f_v4);
        add_seg(segs, pd->f_v2);
        add_seg(segs, pd->f_a);
    }
    add_seg(segs, pd->d_mask);
    if (h.has_link)
        add_seg(segs, pd->d_mask_link);
    if (ctx->fem && ctx->fem->assembled) {
        h.fe_ndof = ctx->fem->ndof();
        add_seg(segs, ctx->fem->d_u);
        add_seg(segs, ctx->fem->d_v);
        add_seg(segs, ctx->fem->d_a);
    }
    if (ctx->arl) {
        h.nlam = ctx->arl->nlam;
        add_seg(segs, ctx->arl->d_lam0);
        add_seg(segs, ctx->arl->d_lam);
    }
    h.n_segments = (int64_t)segs.size();
    for (auto &sg : segs)
        h.payload_bytes += (int64_t)sg.second;
    return PDMTS_OK;
}

// Wait for the context's work, including a batch round it takes part in and
// its FE stream.
static int state_quiesce(pdmts_ctx *ctx)
{
    PDMTS_CUDA_TRY(cudaSetDevice(ctx->device));
    if (ctx->arl && ctx->arl->batch)
        PDMTS_TRY(batch_settle(ctx->arl->batch));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (ctx->arl && ctx->arl->fe_stream)
        PDMTS_CUDA_TRY(cudaStreamSynchronize(ctx->arl->fe_stream));
    return PDMTS_OK;
}
}  // namespace

extern "C" int mts_state_size(pdmts_ctx *ctx, int64_t *bytes)
{
    clear_error();
    if (!ctx || !bytes)
        return fail(PDMTS_ERR_ARG, "mts_state_size: NULL argument");
    StateHeader h;
    std::vector<std::pair<void *, size_t>> segs;
    PDMTS_TRY(state_layout(ctx, h, segs));
    *bytes = (int64_t)sizeof(StateHeader) + h.payload_bytes;
    return PDMTS_OK;
}

extern "C" int mts_state_save(pdmts_ctx *ctx, void *image, int64_t bytes)
{
    clear_error();
    if (!ctx || !image)
        return fail(PDMTS_ERR_ARG, "mts_state_save: NULL argument");
    StateHeader h;
    std::vector<std::pair<void *, size_t>> segs;
    PDMTS_TRY(state_layout(ctx, h, segs));
    if (bytes != (int64_t)sizeof(StateHeader) + h.payload_bytes)
        return fail(PDMTS_ERR_ARG, "mts_state_save: image of %lld bytes, the state needs %lld", (long long)bytes,
                    (long long)(sizeof(StateHeader) + h.payload_bytes));
    PDMTS_TRY(state_quiesce(ctx));
    PDMTS_TRY(ctx->sync_checked("mts_state_save"));
    char *dst = static_cast<char *>(image);
    PDMTS_CUDA_TRY(cudaMemcpy(dst, &h, sizeof h, cudaMemcpyDefault));
    dst += sizeof h;
    for (auto &sg : segs) {
        PDMTS_CUDA_TRY(cudaMemcpy(dst, sg.first, sg.second, cudaMemcpyDefault));
        dst += sg.second;
    }
    return PDMTS_OK;
}

extern "C" int mts_state_load(pdmts_ctx *ctx, const void *image, int64_t bytes)
{
    clear_error();
    if (!ctx || !image)
        return fail(PDMTS_ERR_ARG, "mts_state_load: NULL argument");
    StateHeader mine, h;
    std::vector<std::pair<void *, size_t>> segs;
    PDMTS_TRY(state_layout(ctx, mine, segs));
    if (bytes != (int64_t)sizeof(StateHeader) + mine.payload_bytes)
        return fail(PDMTS_ERR_ARG, "mts_state_load: image of %lld bytes, this context's state has %lld",
                    (long long)bytes, (long long)(sizeof(StateHeader) + mine.payload_bytes));
    PDMTS_TRY(state_quiesce(ctx));
    PDMTS_CUDA_TRY(cudaMemcpy(&h, image, sizeof h, cudaMemcpyDefault));
    if (std::memcmp(h.magic, kStateMagic, sizeof h.magic) != 0 || h.version != mine.version ||
        h.precision != mine.precision || h.layout != mine.layout || h.dim != mine.dim || h.n != mine.n ||
        h.n_mask_words != mine.n_mask_words || h.fe_ndof != mine.fe_ndof || h.nlam != mine.nlam ||
        h.has_link != mine.has_link || h.n_segments != mine.n_segments || h.payload_bytes != mine.payload_bytes)
        return fail(PDMTS_ERR_ARG, "mts_state_load: the image was saved from a different set-up");
    if (h.cur < 0 || h.cur > 1 || h.lk_cur < 0 || h.lk_cur > 1 || h.steps_done < 0)
        return fail(PDMTS_ERR_ARG, "mts_state_load: corrupt image header");
    const char *src = static_cast<const char *>(image) + sizeof h;
    for (auto &sg : segs) {
        PDMTS_CUDA_TRY(cudaMemcpy(sg.first, src, sg.second, cudaMemcpyDefault));
        src += sg.second;
    }
    pdmts_pd *pd = ctx->pd;
    pd->cur = h.cur;
    pd->need_init = h.need_init != 0;
    pd->lk_cur = h.lk_cur;
    pd->steps_done = h.steps_done;
    pd_invalidate_graphs(pd);
    if (ctx->arl) {
        ctx->arl->H_valid = false;  // rebuilt from the loaded bond words at the next step
        ctx->arl->g0_ready = false; // lambda_0 comes from the image
        ctx->arl->flag_pending = false;
    }
    // the loaded image replaces a state a give-up left undefined
    PDMTS_CUDA_TRY(cudaMemsetAsync(ctx->d_counter + 2, 0, sizeof(unsigned long long), ctx->stream));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    __atomic_store_n(ctx->h_watch, 0ull, __ATOMIC_RELEASE);
    ctx->gave_up = false;
    return PDMTS_OK;
}
