// pd.h -- the PD subdomain handle (host mirror + device arrays).
#pragma once

#include <array>
#include <vector>

#include "internal.h"

template <typename T>
struct DevArr {
    T *p = nullptr;
    int64_t count = 0;
};

struct pdmts_pd {
    pdmts_ctx *ctx = nullptr;
    int dim = 2;
    int64_t n = 0;
    int precision = PDMTS_FP64;
    double horizon = 0, c = 0, l = 0, s0 = 0, rho = 0;
    int micro_kind = PDMTS_MICRO_POWER;
    int force_kind = PDMTS_FORCE_LINEAR;
    bool breaking = true;

    // host mirror of the problem statement
    std::vector<double> X;  // dim * n
    std::vector<double> V;  // n
    bool uniform_vol = true;
    std::vector<int64_t> row_ptr;
    std::vector<int32_t> col;

    // lattice description (x = x0 + k h)
    bool on_lattice = false;
    double h = 0.0;
    std::array<double, 3> x0{0, 0, 0};
    std::vector<int32_t> lk;  // dim * n integer lattice coordinates

    // family layout: sliced ELL (general) or the 2D lattice stencil
    enum { LAYOUT_SELL = 0, LAYOUT_LATTICE2D = 1, LAYOUT_LATTICE3D = 2 };
    int layout = LAYOUT_SELL;
    int32_t lat_dims[3] = {0, 0, 0};      // nodes per axis (lattice layout)
    std::vector<int8_t> slot_of_csr;      // lattice layout: stencil slot of each CSR bond
    DevArr<uint32_t> d_exists;            // lattice layout: existing-bond bits per node

    // sliced-ELL layout
    int64_t ntiles = 0, n_slots = 0, n_mask_words = 0;
    int32_t max_deg = 0;
    std::vector<int64_t> tile_ptr, mask_ptr;
    std::vector<int32_t> tile_k, deg;
    std::vector<uint32_t> mask_host;  // initial / staged mask

    // loads and weights
    std::vector<double> alpha;  // n (empty: all zero)
    bool has_b = false;         // body force set (raw field kept on the device in d_b)
    std::vector<double> g;      // dim * n interface force density (empty: none)

    // device arrays common to both precisions
    DevArr<int64_t> d_tile_ptr, d_mask_ptr;
    DevArr<int32_t> d_tile_k, d_col, d_deg;
    DevArr<uint32_t> d_mask;
    DevArr<double> d_V, d_out;  // d_out: dim * n staging for read-back and uploads
    DevArr<double> d_b;         // raw body force b, dim * n
    // FP64
    DevArr<double> d_X, d_cb, d_alpha, d_mass, d_wb, d_g, d_v, d_a;
    DevArr<double> d_u[2];
    // FP32 bulk
    DevArr<pdmts::StencilEntry> d_stencil;
    int n_stencil = 0;
    DevArr<float> f_alpha, f_invm, f_wb, f_g;
    DevArr<pdmts::Row3DEnt> d_rowtab;  // 3D lattice layout: the stencil rows' constants and offsets
    DevArr<int32_t> f_rowalpha;  // lattice layouts: ny + 1 prefix counts of the rows with a weighted node
    // state in lattice units, compensated pairs, per-node packed:
    // 2D: u4 = {hx, hy, lx, ly}; 3D: u4 = {hx, hy, hz, lx}, u2 = {ly, lz}
    DevArr<float4> f_u4[2], f_v4;
    DevArr<float2> f_u2[2], f_v2;
    DevArr<float> f_a;   // 2D: {ax, ay} per node; 3D: {ax, ay, az, 0} per node (lattice units)

    // Link problem of the MTS coupling (Eq. 48b): a second velocity-Verlet
    // state driven only by the interpolated multiplier, with its own bond
    // words (the state at the start of the coarse step) and no breaking.
    bool has_link = false;
    DevArr<double> lk_u[2], lk_v, lk_a, lk_g;       // FP64
    DevArr<float4> lk_u4[2], lk_v4;                 // FP32 bulk
    DevArr<float2> lk_u2[2], lk_v2;
    DevArr<float> lk_af, lk_gf;
    DevArr<uint32_t> d_mask_link;
    int lk_cur = 0;
    int link_win_lo[2] = {0, 0}, link_win_n[2] = {0, 0};  // TY-row units the link problem can reach
    // node ranges holding every node a link run may write (the windows widened
    // to 32 rows, a multiple of every lattice tile height); {0, n} without windows
    int64_t link_seg_lo[2] = {0, 0}, link_seg_n[2] = {0, 0};
    int lattice_tile = -1;                                // lattice tile configuration (-1: tune)
    int link_tile = -1;   // configuration of link chains, tuned on their windows (-1: lattice_tile)
    int64_t link_bonds = -1;  // directed bonds evaluated per link substep (-1: all)
    // growing windows of the link chain: substep k (0-based) of a link run
    // evaluates step_win[k] = {lo0, n0, lo1, n1} (TY-row units), holding every
    // node within (k + 2) delta of a band; empty: link_win for every substep
    std::vector<std::array<int, 4>> link_step_win;
    std::vector<int64_t> link_step_bonds;
    int chain_k = 0;  // index of the substep being launched within its chain
    // directed bonds a substep evaluates (substep k of a link chain: its window)
    int64_t substep_bonds(bool link, int k) const
    {
        if (link && k >= 0 && k < (int)link_step_bonds.size())
            return link_step_bonds[(size_t)k];
        return (link && link_bonds >= 0) ? link_bonds : (int64_t)row_ptr[(size_t)n];
    }
    // interface force density of the free problem (G_PD^T lambda_0 / V): FP64 d_g or FP32 f_g
    bool has_g = false;

    // captured substep chains, keyed by (starting buffer parity, length, theta schedule id)
    struct GraphEntry {
        int parity, len, sched;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
    bool use_graphs = true;
    bool chain_follow = false;  // the substep being launched follows another one in its chain

    int cur = 0;            // buffer holding u at the current time
    bool need_init = true;  // a must be recomputed from u before the next step
    int64_t steps_done = 0;
    int64_t device_bytes = 0;

    template <typename T>
    int alloc(DevArr<T> &a, int64_t count);
    template <typename T>
    void release(DevArr<T> &a);
    void release_all();

    int upload_weights_and_loads();  // (re)build mass, wb, g device arrays
    int step(bool init, double theta, cudaStream_t s, bool link = false);  // one substep
    pdmts::Lat2DArgs lattice_args(const pdmts::F32NodeArgs &N, uint32_t *mask, bool link) const;
    pdmts::Lat3DArgs lattice3d_args(const pdmts::F32NodeArgs &N, uint32_t *mask, bool link) const;
    pdmts::F32NodeArgs f32_node_args(bool init, double theta, bool link) const;
    void substep_done(bool init, bool link);  // parity and counters after an enqueued substep
    int tune_lattice(cudaStream_t s);        // pick the lattice tile configuration (once)
    int tune_lattice3d(cudaStream_t s);      // the same for the 3D lattice layout
    int alloc_link_state();                  // link-problem arrays (MTS coupling)
    int zero_link_state(cudaStream_t s, bool all = false);  // W_0 = 0 before a link run
    int ensure_init(cudaStream_t s);
};
