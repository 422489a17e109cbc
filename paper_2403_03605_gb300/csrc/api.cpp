// api.cpp -- C ABI of the pdmts library: context, PD subdomain set-up and
// read-back, pure-PD time stepping. The hot path itself is in pd_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <map>
#include <new>
#include <tuple>

#include "pd.h"

namespace pdmts {

static thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

void clear_error() { g_err.clear(); }

static bool finite_all(const double *p, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i]))
            return false;
    return true;
}

// Copy `count` elements from a host or device pointer into a host vector.
template <typename T>
static int fetch(std::vector<T> &out, const T *src, int64_t count)
{
    out.resize((size_t)count);
    if (count == 0)
        return PDMTS_OK;
    PDMTS_CUDA_TRY(cudaMemcpy(out.data(), src, sizeof(T) * (size_t)count, cudaMemcpyDefault));
    return PDMTS_OK;
}

}  // namespace pdmts

using namespace pdmts;

// ------------------------------------------------------------- context ------
void *pdmts_ctx::dalloc(size_t bytes)
{
    if (bytes == 0)
        bytes = 256;
    void *p = nullptr;
    if (alloc) {
        p = alloc(bytes, alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p)
        device_bytes += (int64_t)bytes;
    return p;
}

void pdmts_ctx::dfree(void *p)
{
    if (!p)
        return;
    if (free_fn)
        free_fn(p, alloc_user);
    else
        cudaFree(p);
}

int pdmts_ctx::begin()
{
    PDMTS_CUDA_TRY(cudaSetDevice(device));
    PDMTS_CUDA_TRY(cudaEventRecord(ev_in, user_stream));
    PDMTS_CUDA_TRY(cudaStreamWaitEvent(stream, ev_in, 0));
    return PDMTS_OK;
}

int pdmts_ctx::end()
{
    PDMTS_CUDA_TRY(cudaGetLastError());
    PDMTS_CUDA_TRY(cudaEventRecord(ev_out, stream));
    PDMTS_CUDA_TRY(cudaStreamWaitEvent(user_stream, ev_out, 0));
    return PDMTS_OK;
}

int pdmts_ctx::watch_enqueue(cudaStream_t s)
{
    PDMTS_CUDA_TRY(cudaMemcpyAsync(h_watch, d_counter + 2, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    return PDMTS_OK;
}

int pdmts_ctx::watch_check(const char *who)
{
    if (!gave_up && __atomic_load_n(h_watch, __ATOMIC_ACQUIRE) != 0)
        gave_up = true;
    if (gave_up)
        return fail(PDMTS_ERR_TIMEOUT,
                    "%s: a bounded tensor-copy wait of the lattice kernel gave up; the state is undefined "
                    "(load a checkpoint image with mts_state_load to continue)",
                    who);
    return PDMTS_OK;
}

int pdmts_ctx::sync_checked(const char *who)
{
    PDMTS_TRY(watch_enqueue(stream));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(stream));
    return watch_check(who);
}

int pdmts_ctx::pool_event(cudaEvent_t *e)
{
    if (ev_pool.empty()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t ev;
            PDMTS_CUDA_TRY(cudaEventCreate(&ev));
            ev_pool.push_back(ev);
        }
    }
    *e = ev_pool.back();
    ev_pool.pop_back();
    return PDMTS_OK;
}

int pdmts_ctx::mark(cudaEvent_t *e)
{
    *e = nullptr;
    if (!timing)
        return PDMTS_OK;
    PDMTS_TRY(pool_event(e));
    PDMTS_CUDA_TRY(cudaEventRecord(*e, stream));
    return PDMTS_OK;
}

int pdmts_ctx::time_begin(cudaEvent_t *start)
{
    return mark(start);
}

int pdmts_ctx::time_end(cudaEvent_t start, int64_t substeps)
{
    if (!start)
        return PDMTS_OK;
    cudaEvent_t stop = nullptr;
    PDMTS_TRY(pool_event(&stop));
    PDMTS_CUDA_TRY(cudaEventRecord(stop, stream));
    ev_marks.push_back({start, stop});
    ev_counts.push_back(substeps);
    return PDMTS_OK;
}

extern "C" int pdmts_set_timing(pdmts_ctx *ctx, int enabled)
{
    clear_error();
    if (!ctx)
        return fail(PDMTS_ERR_ARG, "pdmts_set_timing: ctx is NULL");
    ctx->timing = enabled != 0;
    return PDMTS_OK;
}

extern int pd_invalidate_graphs(pdmts_pd *pd);  // pd_kernels.cu

extern "C" int pdmts_set_debug_poll_limit(pdmts_ctx *ctx, int64_t polls)
{
    clear_error();
    if (!ctx)
        return fail(PDMTS_ERR_ARG, "pdmts_set_debug_poll_limit: ctx is NULL");
    const unsigned lim = polls < 0 ? kWaitPolls : (unsigned)std::min<int64_t>(polls, kWaitPolls);
    if (lim != ctx->first_wait_polls) {
        ctx->first_wait_polls = lim;
        if (ctx->pd)
            pd_invalidate_graphs(ctx->pd);  // captured chains hold the launch arguments
    }
    return PDMTS_OK;
}

extern "C" int pdmts_get_timing(pdmts_ctx *ctx, double *substep_ms, int64_t *substeps)
{
    clear_error();
    if (!ctx || !substep_ms || !substeps)
        return fail(PDMTS_ERR_ARG, "pdmts_get_timing: NULL argument");
    PDMTS_CUDA_TRY(cudaSetDevice(ctx->device));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    double ms = 0.0;
    int64_t cnt = 0;
    for (size_t k = 0; k < ctx->ev_marks.size(); ++k) {
        float t = 0.f;
        PDMTS_CUDA_TRY(cudaEventElapsedTime(&t, ctx->ev_marks[k].first, ctx->ev_marks[k].second));
        ms += t;
        cnt += ctx->ev_counts[k];
        ctx->ev_pool.push_back(ctx->ev_marks[k].first);
        ctx->ev_pool.push_back(ctx->ev_marks[k].second);
    }
    ctx->ev_marks.clear();
    ctx->ev_counts.clear();
    *substep_ms = ms;
    *substeps = cnt;
    return PDMTS_OK;
}

extern "C" int mts_get_phase_timing(pdmts_ctx *ctx, double *phase_ms, int64_t *n_steps)
{
    clear_error();
    if (!ctx || !phase_ms || !n_steps)
        return fail(PDMTS_ERR_ARG, "mts_get_phase_timing: NULL argument");
    PDMTS_CUDA_TRY(cudaSetDevice(ctx->device));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < 5; ++k)
        phase_ms[k] = 0.0;
    for (auto &m : ctx->phase_marks) {
        float t = 0.f;
        for (int k = 0; k < 4; ++k) {
            PDMTS_CUDA_TRY(cudaEventElapsedTime(&t, m[(size_t)k], m[(size_t)k + 1]));
            phase_ms[k] += t;
        }
        PDMTS_CUDA_TRY(cudaEventElapsedTime(&t, m[0], m[4]));
        phase_ms[4] += t;
        for (cudaEvent_t e : m)
            ctx->ev_pool.push_back(e);
    }
    *n_steps = (int64_t)ctx->phase_marks.size();
    ctx->phase_marks.clear();
    return PDMTS_OK;
}

extern "C" const char *pdmts_last_error(void) { return g_err.c_str(); }

extern "C" int pdmts_ctx_create(pdmts_ctx **ctx, int device, void *cuda_stream)
{
    clear_error();
    if (!ctx)
        return fail(PDMTS_ERR_ARG, "pdmts_ctx_create: ctx is NULL");
    *ctx = nullptr;
    int ndev = 0;
    PDMTS_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev)
        return fail(PDMTS_ERR_ARG, "pdmts_ctx_create: device %d out of range (%d devices)", device, ndev);
    PDMTS_CUDA_TRY(cudaSetDevice(device));
    auto *c = new (std::nothrow) pdmts_ctx();
    if (!c)
        return fail(PDMTS_ERR_NOMEM, "pdmts_ctx_create: out of host memory");
    c->device = device;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || c->num_sms < 1)
        c->num_sms = 1;
    c->user_stream = (cudaStream_t)cuda_stream;
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&c->d_counter, 64) != cudaSuccess ||
        cudaMallocHost(&c->h_watch, 64) != cudaSuccess) {
        cudaGetLastError();
        pdmts_ctx_destroy(c);
        return fail(PDMTS_ERR_CUDA, "pdmts_ctx_create: stream/event/counter creation failed");
    }
    std::memset(c->h_watch, 0, 64);
    if (cudaMemset(c->d_counter, 0, 64) != cudaSuccess) {
        pdmts_ctx_destroy(c);
        return fail(PDMTS_ERR_CUDA, "pdmts_ctx_create: memset failed");
    }
    *ctx = c;
    return PDMTS_OK;
}

extern "C" int mts_destroy_coupling(pdmts_ctx *ctx);  // mts.cu

extern "C" int pdmts_ctx_destroy(pdmts_ctx *ctx)
{
    clear_error();
    if (!ctx)
        return PDMTS_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream)
        cudaStreamSynchronize(ctx->stream);
    mts_destroy_coupling(ctx);
    if (ctx->pd)
        pd_destroy(ctx->pd);
    if (ctx->d_counter)
        cudaFree(ctx->d_counter);
    if (ctx->h_watch)
        cudaFreeHost(ctx->h_watch);
    for (auto &m : ctx->ev_marks) {
        ctx->ev_pool.push_back(m.first);
        ctx->ev_pool.push_back(m.second);
    }
    for (cudaEvent_t e : ctx->ev_pool)
        cudaEventDestroy(e);
    if (ctx->ev_in)
        cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_out)
        cudaEventDestroy(ctx->ev_out);
    if (ctx->stream)
        cudaStreamDestroy(ctx->stream);
    delete ctx;
    return PDMTS_OK;
}

extern "C" int pdmts_set_allocator(pdmts_ctx *ctx, pdmts_alloc_fn alloc, pdmts_free_fn free_fn, void *user)
{
    clear_error();
    if (!ctx)
        return fail(PDMTS_ERR_ARG, "pdmts_set_allocator: ctx is NULL");
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(PDMTS_ERR_ARG, "pdmts_set_allocator: give both alloc and free, or neither");
    if (ctx->pd || ctx->fem)
        return fail(PDMTS_ERR_STATE, "pdmts_set_allocator: subdomains already created");
    ctx->alloc = alloc;
    ctx->free_fn = free_fn;
    ctx->alloc_user = user;
    return PDMTS_OK;
}

extern "C" int pdmts_ctx_synchronize(pdmts_ctx *ctx)
{
    clear_error();
    if (!ctx)
        return fail(PDMTS_ERR_ARG, "pdmts_ctx_synchronize: ctx is NULL");
    PDMTS_CUDA_TRY(cudaSetDevice(ctx->device));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return PDMTS_OK;
}

extern "C" int pdmts_get_stats(pdmts_ctx *ctx, pdmts_stats *stats)
{
    clear_error();
    if (!ctx || !stats)
        return fail(PDMTS_ERR_ARG, "pdmts_get_stats: NULL argument");
    PDMTS_CUDA_TRY(cudaSetDevice(ctx->device));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    unsigned long long word[3] = {0, 0, 0};
    PDMTS_CUDA_TRY(cudaMemcpy(word, ctx->d_counter, sizeof(word), cudaMemcpyDeviceToHost));
    if (word[2])
        ctx->gave_up = true;
    PDMTS_TRY(ctx->watch_check("pdmts_get_stats"));
    ctx->stats.bonds_broken = (int64_t)word[0];
    *stats = ctx->stats;
    return PDMTS_OK;
}

// ------------------------------------------------------- PD handle helpers -
template <typename T>
int pdmts_pd::alloc(DevArr<T> &a, int64_t count)
{
    release(a);
    a.p = (T *)ctx->dalloc(sizeof(T) * (size_t)std::max<int64_t>(count, 1));
    if (!a.p)
        return fail(PDMTS_ERR_NOMEM, "device allocation of %lld bytes failed",
                    (long long)(sizeof(T) * count));
    a.count = count;
    device_bytes += (int64_t)(sizeof(T) * std::max<int64_t>(count, 1));
    return PDMTS_OK;
}

template <typename T>
void pdmts_pd::release(DevArr<T> &a)
{
    if (a.p) {
        ctx->dfree(a.p);
        device_bytes -= (int64_t)(sizeof(T) * std::max<int64_t>(a.count, 1));
    }
    a.p = nullptr;
    a.count = 0;
}

extern int pd_invalidate_graphs(pdmts_pd *pd);  // pd_kernels.cu

void pdmts_pd::release_all()
{
    pd_invalidate_graphs(this);
    release(d_tile_ptr); release(d_mask_ptr); release(d_tile_k); release(d_col); release(d_deg);
    release(d_mask); release(d_V); release(d_out); release(d_b); release(d_exists);
    release(d_X); release(d_cb); release(d_alpha); release(d_mass); release(d_wb); release(d_g);
    release(d_v); release(d_a); release(d_u[0]); release(d_u[1]);
    release(d_stencil); release(f_alpha); release(f_invm); release(f_wb); release(f_g); release(f_rowalpha); release(d_rowtab);
    release(f_v4); release(f_v2); release(f_a);
    release(f_u4[0]); release(f_u4[1]); release(f_u2[0]); release(f_u2[1]);
    release(lk_u[0]); release(lk_u[1]); release(lk_v); release(lk_a); release(lk_g);
    release(lk_u4[0]); release(lk_u4[1]); release(lk_v4); release(lk_u2[0]); release(lk_u2[1]); release(lk_v2);
    release(lk_af); release(lk_gf); release(d_mask_link);
}

int pdmts_pd::alloc_link_state()
{
    if (has_link)
        return PDMTS_OK;
    const int64_t m = (int64_t)dim * n;
    if (precision == PDMTS_FP64) {
        PDMTS_TRY(alloc(lk_u[0], m));
        PDMTS_TRY(alloc(lk_u[1], m));
        PDMTS_TRY(alloc(lk_v, m));
        PDMTS_TRY(alloc(lk_a, m));
        PDMTS_TRY(alloc(lk_g, m));
        if (!d_g.p)
            PDMTS_TRY(alloc(d_g, m));
    } else {
        for (int b = 0; b < 2; ++b) {
            PDMTS_TRY(alloc(lk_u4[b], n));
            if (dim == 3)
                PDMTS_TRY(alloc(lk_u2[b], n));
        }
        PDMTS_TRY(alloc(lk_v4, n));
        if (dim == 3)
            PDMTS_TRY(alloc(lk_v2, n));
        PDMTS_TRY(alloc(lk_af, (int64_t)(dim == 2 ? 2 : 4) * n));
        PDMTS_TRY(alloc(lk_gf, m));
        if (!f_g.p)
            PDMTS_TRY(alloc(f_g, m));
    }
    PDMTS_TRY(alloc(d_mask_link, std::max<int64_t>(n_mask_words, 1)));
    cudaStream_t s = ctx->stream;
    PDMTS_CUDA_TRY(cudaMemcpyAsync(d_mask_link.p, d_mask.p, sizeof(uint32_t) * std::max<int64_t>(n_mask_words, 1),
                                   cudaMemcpyDeviceToDevice, s));
    // interface forces are written only at overlap nodes: every other entry must be zero
    // (device memory may come recycled from the allocator)
    if (precision == PDMTS_FP64) {
        PDMTS_CUDA_TRY(cudaMemsetAsync(d_g.p, 0, sizeof(double) * m, s));
        PDMTS_CUDA_TRY(cudaMemsetAsync(lk_g.p, 0, sizeof(double) * m, s));
    } else {
        PDMTS_CUDA_TRY(cudaMemsetAsync(f_g.p, 0, sizeof(float) * m, s));
        PDMTS_CUDA_TRY(cudaMemsetAsync(lk_gf.p, 0, sizeof(float) * m, s));
    }
    has_link = true;
    has_g = true;
    link_seg_lo[0] = link_seg_lo[1] = 0;
    link_seg_n[0] = n;
    link_seg_n[1] = 0;
    PDMTS_TRY(zero_link_state(s, true));
    pd_invalidate_graphs(this);
    return PDMTS_OK;
}

int pdmts_pd::zero_link_state(cudaStream_t s, bool all)
{
    // only the node ranges a link run writes (the link state is zero
    // elsewhere), or everything
    for (int w = 0; w < 2; ++w) {
        const int64_t lo = all ? 0 : link_seg_lo[w], cnt = all ? (w == 0 ? n : 0) : link_seg_n[w];
        if (cnt <= 0)
            continue;
        if (precision == PDMTS_FP64) {
            for (int d = 0; d < dim; ++d) {
                for (int b = 0; b < 2; ++b)
                    PDMTS_CUDA_TRY(cudaMemsetAsync(lk_u[b].p + (int64_t)d * n + lo, 0, sizeof(double) * cnt, s));
                PDMTS_CUDA_TRY(cudaMemsetAsync(lk_v.p + (int64_t)d * n + lo, 0, sizeof(double) * cnt, s));
                PDMTS_CUDA_TRY(cudaMemsetAsync(lk_a.p + (int64_t)d * n + lo, 0, sizeof(double) * cnt, s));
            }
        } else {
            for (int b = 0; b < 2; ++b) {
                PDMTS_CUDA_TRY(cudaMemsetAsync(lk_u4[b].p + lo, 0, sizeof(float4) * cnt, s));
                if (dim == 3)
                    PDMTS_CUDA_TRY(cudaMemsetAsync(lk_u2[b].p + lo, 0, sizeof(float2) * cnt, s));
            }
            PDMTS_CUDA_TRY(cudaMemsetAsync(lk_v4.p + lo, 0, sizeof(float4) * cnt, s));
            if (dim == 3)
                PDMTS_CUDA_TRY(cudaMemsetAsync(lk_v2.p + lo, 0, sizeof(float2) * cnt, s));
            const int per = dim == 2 ? 2 : 4;
            PDMTS_CUDA_TRY(cudaMemsetAsync(lk_af.p + (int64_t)per * lo, 0, sizeof(float) * per * cnt, s));
        }
    }
    lk_cur = 0;  // W_0 = 0: current and predicted displacement both zero, a_0 = 0
    return PDMTS_OK;
}

template <typename T>
static int upload(DevArr<T> &a, const T *src, int64_t count, cudaStream_t s)
{
    if (count == 0)
        return PDMTS_OK;
    PDMTS_CUDA_TRY(cudaMemcpyAsync(a.p, src, sizeof(T) * (size_t)count, cudaMemcpyHostToDevice, s));
    return PDMTS_OK;
}

// Family H_delta of every node (Sec. 2.1): all j != i with |x_j - x_i|^2 <=
// delta^2 (closed ball), rows ascending. Nodes are bucketed by a counting
// sort over a grid of cell size delta; each node scans the 3^dim cells
// around its own.
static int build_family(pdmts_pd *pd)
{
    const int dim = pd->dim;
    const int64_t n = pd->n;
    const double delta = pd->horizon;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int64_t nc[3] = {1, 1, 1};
    for (int d = 0; d < dim; ++d) {
        const double *x = &pd->X[(size_t)d * n];
        lo[d] = *std::min_element(x, x + n);
        hi[d] = *std::max_element(x, x + n);
        nc[d] = (int64_t)std::floor((hi[d] - lo[d]) / delta) + 1;
    }
    const int64_t ncell = nc[0] * nc[1] * nc[2];
    if (ncell > (int64_t)4 * n + 1024)  // very sparse clouds: coarsen is not needed for lattices
        return fail(PDMTS_ERR_UNSUPPORTED, "pd_create: node cloud too sparse for the cell grid");
    std::vector<int64_t> cell_of((size_t)n), start((size_t)ncell + 1, 0), order((size_t)n);
    std::vector<std::array<int64_t, 3>> cidx((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        int64_t id = 0;
        for (int d = 2; d >= 0; --d) {
            int64_t k = 0;
            if (d < dim) {
                k = (int64_t)std::floor((pd->X[(size_t)d * n + i] - lo[d]) / delta);
                k = std::min(std::max<int64_t>(k, 0), nc[d] - 1);
            }
            cidx[(size_t)i][(size_t)d] = k;
            id = id * nc[d] + k;
        }
        cell_of[(size_t)i] = id;
        start[(size_t)id + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c)
        start[(size_t)c + 1] += start[(size_t)c];
    {
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            order[(size_t)fill[(size_t)cell_of[(size_t)i]]++] = i;
    }
    const double d2max = delta * delta;
    pd->row_ptr.assign((size_t)n + 1, 0);
    pd->col.clear();
    pd->col.reserve((size_t)n * (dim == 2 ? 29 : 123));
    std::vector<int32_t> row;
    for (int64_t i = 0; i < n; ++i) {
        row.clear();
        const auto &ci = cidx[(size_t)i];
        int64_t r0 = dim > 0 ? 1 : 0, r1 = dim > 1 ? 1 : 0, r2 = dim > 2 ? 1 : 0;
        for (int64_t o2 = -r2; o2 <= r2; ++o2)
            for (int64_t o1 = -r1; o1 <= r1; ++o1)
                for (int64_t o0 = -r0; o0 <= r0; ++o0) {
                    int64_t k0 = ci[0] + o0, k1 = ci[1] + o1, k2 = ci[2] + o2;
                    if (k0 < 0 || k0 >= nc[0] || k1 < 0 || k1 >= nc[1] || k2 < 0 || k2 >= nc[2])
                        continue;
                    int64_t id = (k2 * nc[1] + k1) * nc[0] + k0;
                    for (int64_t q = start[(size_t)id]; q < start[(size_t)id + 1]; ++q) {
                        int64_t j = order[(size_t)q];
                        if (j == i)
                            continue;
                        double r2s = 0.0;
                        for (int d = 0; d < dim; ++d) {
                            double e = pd->X[(size_t)d * n + j] - pd->X[(size_t)d * n + i];
                            r2s += e * e;
                        }
                        if (r2s <= d2max)
                            row.push_back((int32_t)j);
                    }
                }
        std::sort(row.begin(), row.end());
        pd->col.insert(pd->col.end(), row.begin(), row.end());
        pd->row_ptr[(size_t)i + 1] = (int64_t)pd->col.size();
    }
    return PDMTS_OK;
}

// Detect x = x0 + k h with integer k (|k| < 32768) for all nodes.
static void detect_lattice(pdmts_pd *pd)
{
    pd->on_lattice = false;
    const int dim = pd->dim;
    const int64_t n = pd->n;
    double hmin2 = INFINITY;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = pd->row_ptr[(size_t)i]; k < pd->row_ptr[(size_t)i + 1]; ++k) {
            int64_t j = pd->col[(size_t)k];
            double r2 = 0;
            for (int d = 0; d < dim; ++d) {
                double e = pd->X[(size_t)d * n + j] - pd->X[(size_t)d * n + i];
                r2 += e * e;
            }
            hmin2 = std::min(hmin2, r2);
        }
    if (!std::isfinite(hmin2) || hmin2 <= 0)
        return;
    const double h = std::sqrt(hmin2);
    std::vector<int32_t> lk((size_t)dim * n);
    for (int d = 0; d < dim; ++d) {
        const double *x = &pd->X[(size_t)d * n];
        double x0 = *std::min_element(x, x + n);
        for (int64_t i = 0; i < n; ++i) {
            double q = (x[i] - x0) / h;
            double k = std::nearbyint(q);
            if (std::fabs(q - k) > 1e-6 || k > 32767.0)
                return;
            lk[(size_t)d * n + i] = (int32_t)k;
        }
        pd->x0[(size_t)d] = x0;
    }
    pd->h = h;
    pd->lk.swap(lk);
    pd->on_lattice = true;
}

static void build_sell(pdmts_pd *pd)
{
    const int64_t n = pd->n;
    pd->ntiles = (n + 31) / 32;
    pd->tile_ptr.assign((size_t)pd->ntiles + 1, 0);
    pd->mask_ptr.assign((size_t)pd->ntiles + 1, 0);
    pd->tile_k.assign((size_t)pd->ntiles, 0);
    pd->deg.assign((size_t)n, 0);
    pd->max_deg = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t dg = (int32_t)(pd->row_ptr[(size_t)i + 1] - pd->row_ptr[(size_t)i]);
        pd->deg[(size_t)i] = dg;
        pd->max_deg = std::max(pd->max_deg, dg);
        int64_t t = i / 32;
        pd->tile_k[(size_t)t] = std::max(pd->tile_k[(size_t)t], dg);
    }
    for (int64_t t = 0; t < pd->ntiles; ++t) {
        int64_t K = pd->tile_k[(size_t)t];
        pd->tile_ptr[(size_t)t + 1] = pd->tile_ptr[(size_t)t] + 32 * K;
        pd->mask_ptr[(size_t)t + 1] = pd->mask_ptr[(size_t)t] + 32 * ((K + 31) / 32);
    }
    pd->n_slots = pd->tile_ptr[(size_t)pd->ntiles];
    pd->n_mask_words = pd->mask_ptr[(size_t)pd->ntiles];
    // all existing bonds intact, padding slots 0
    pd->mask_host.assign((size_t)std::max<int64_t>(pd->n_mask_words, 1), 0u);
    for (int64_t i = 0; i < n; ++i) {
        int64_t t = i / 32, lane = i % 32;
        for (int32_t k = 0; k < pd->deg[(size_t)i]; ++k)
            pd->mask_host[(size_t)(pd->mask_ptr[(size_t)t] + 32 * (k / 32) + lane)] |= 1u << (k % 32);
    }
}

// Word and bit of the k-th CSR bond of node i in the device bond-status array.
static inline void bond_bit(const pdmts_pd *pd, int64_t i, int32_t k, int64_t &word, int &bit)
{
    if (pd->layout == pdmts_pd::LAYOUT_LATTICE2D) {
        word = i;
        bit = pd->slot_of_csr[(size_t)(pd->row_ptr[(size_t)i] + k)];
    } else if (pd->layout == pdmts_pd::LAYOUT_LATTICE3D) {
        const int slot = pd->slot_of_csr[(size_t)(pd->row_ptr[(size_t)i] + k)];
        word = (int64_t)(slot / 32) * pd->n + i;
        bit = slot % 32;
    } else {
        word = pd->mask_ptr[(size_t)(i / 32)] + 32 * (k / 32) + (i % 32);
        bit = k % 32;
    }
}

// The 2D lattice layout applies when the nodes are exactly the nx * ny
// rectangle numbered x + nx y and every family is the 28-offset stencil
// clipped to the rectangle. Builds the per-node bond words on success.
static bool try_lattice2d(pdmts_pd *pd)
{
    if (pd->dim != 2 || !pd->on_lattice)
        return false;
    const int64_t n = pd->n;
    int32_t nx = 0, ny = 0;
    for (int64_t i = 0; i < n; ++i) {
        nx = std::max(nx, pd->lk[(size_t)i] + 1);
        ny = std::max(ny, pd->lk[(size_t)n + i] + 1);
    }
    if ((int64_t)nx * ny != n)
        return false;
    for (int64_t i = 0; i < n; ++i)
        if (pd->lk[(size_t)i] + (int64_t)nx * pd->lk[(size_t)n + i] != i)
            return false;
    // stencil slot of every offset, then every family must be stencil ∩ rectangle
    int slot_of[7][7];
    for (auto &r : slot_of)
        for (int &v : r)
            v = -1;
    for (int k = 0; k < lat2d::NS; ++k)
        slot_of[lat2d::DY(k) + 3][lat2d::DX(k) + 3] = k;
    std::vector<int8_t> slot((size_t)pd->row_ptr[(size_t)n]);
    std::vector<uint32_t> words((size_t)n, 0u);
    for (int64_t i = 0; i < n; ++i) {
        const int xi = pd->lk[(size_t)i], yi = pd->lk[(size_t)n + i];
        for (int64_t k = pd->row_ptr[(size_t)i]; k < pd->row_ptr[(size_t)i + 1]; ++k) {
            const int64_t j = pd->col[(size_t)k];
            const int ox = pd->lk[(size_t)j] - xi, oy = pd->lk[(size_t)n + j] - yi;
            if (ox < -3 || ox > 3 || oy < -3 || oy > 3 || slot_of[oy + 3][ox + 3] < 0)
                return false;
            slot[(size_t)k] = (int8_t)slot_of[oy + 3][ox + 3];
            words[(size_t)i] |= 1u << slot_of[oy + 3][ox + 3];
        }
        int expect = 0;
        for (int k = 0; k < lat2d::NS; ++k) {
            const int x = xi + lat2d::DX(k), y = yi + lat2d::DY(k);
            expect += (x >= 0 && x < nx && y >= 0 && y < ny);
        }
        if (expect != pd->row_ptr[(size_t)i + 1] - pd->row_ptr[(size_t)i])
            return false;
    }
    pd->layout = pdmts_pd::LAYOUT_LATTICE2D;
    pd->lat_dims[0] = nx;
    pd->lat_dims[1] = ny;
    pd->slot_of_csr.swap(slot);
    pd->mask_host.swap(words);
    pd->n_mask_words = n;
    pd->max_deg = 0;
    for (int64_t i = 0; i < n; ++i)
        pd->max_deg = std::max<int32_t>(pd->max_deg, (int32_t)(pd->row_ptr[(size_t)i + 1] - pd->row_ptr[(size_t)i]));
    return true;
}

// The 3D lattice layout: the nodes are exactly the nx * ny * nz box numbered
// x + nx (y + ny z) and every family is the 122-offset stencil |d|^2 <= 9
// clipped to the box. Builds the four bond words of every node on success.
static bool try_lattice3d(pdmts_pd *pd)
{
    if (pd->dim != 3 || !pd->on_lattice)
        return false;
    const int64_t n = pd->n;
    int32_t nx = 0, ny = 0, nz = 0;
    for (int64_t i = 0; i < n; ++i) {
        nx = std::max(nx, pd->lk[(size_t)i] + 1);
        ny = std::max(ny, pd->lk[(size_t)n + i] + 1);
        nz = std::max(nz, pd->lk[(size_t)2 * n + i] + 1);
    }
    if ((int64_t)nx * ny * nz != n || nx < 7 || ny < 7)
        return false;
    for (int64_t i = 0; i < n; ++i)
        if (pd->lk[(size_t)i] + (int64_t)nx * (pd->lk[(size_t)n + i] + (int64_t)ny * pd->lk[(size_t)2 * n + i]) != i)
            return false;
    int slot_of[7][7][7];
    int k = 0;
    for (int dz = -3; dz <= 3; ++dz)
        for (int dy = -3; dy <= 3; ++dy)
            for (int dx = -3; dx <= 3; ++dx) {
                const int r2 = dx * dx + dy * dy + dz * dz;
                slot_of[dz + 3][dy + 3][dx + 3] = (r2 == 0 || r2 > 9) ? -1 : k++;
            }
    if (k != lat3d::NS)
        return false;
    std::vector<int8_t> slot((size_t)pd->row_ptr[(size_t)n]);
    std::vector<uint32_t> words((size_t)lat3d::W * n, 0u);
    for (int64_t i = 0; i < n; ++i) {
        const int xi = pd->lk[(size_t)i], yi = pd->lk[(size_t)n + i], zi = pd->lk[(size_t)2 * n + i];
        for (int64_t q = pd->row_ptr[(size_t)i]; q < pd->row_ptr[(size_t)i + 1]; ++q) {
            const int64_t j = pd->col[(size_t)q];
            const int ox = pd->lk[(size_t)j] - xi, oy = pd->lk[(size_t)n + j] - yi, oz = pd->lk[(size_t)2 * n + j] - zi;
            if (ox < -3 || ox > 3 || oy < -3 || oy > 3 || oz < -3 || oz > 3 || slot_of[oz + 3][oy + 3][ox + 3] < 0)
                return false;
            const int sl = slot_of[oz + 3][oy + 3][ox + 3];
            slot[(size_t)q] = (int8_t)sl;
            words[(size_t)(sl / 32) * n + i] |= 1u << (sl % 32);
        }
        int expect = 0;
        for (int dz = -3; dz <= 3; ++dz)
            for (int dy = -3; dy <= 3; ++dy)
                for (int dx = -3; dx <= 3; ++dx)
                    if (slot_of[dz + 3][dy + 3][dx + 3] >= 0) {
                        const int x = xi + dx, y = yi + dy, z = zi + dz;
                        expect += x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz;
                    }
        if (expect != pd->row_ptr[(size_t)i + 1] - pd->row_ptr[(size_t)i])
            return false;
    }
    pd->layout = pdmts_pd::LAYOUT_LATTICE3D;
    pd->lat_dims[0] = nx;
    pd->lat_dims[1] = ny;
    pd->lat_dims[2] = nz;
    pd->slot_of_csr.swap(slot);
    pd->mask_host.swap(words);
    pd->n_mask_words = (int64_t)lat3d::W * n;
    pd->max_deg = 0;
    for (int64_t i = 0; i < n; ++i)
        pd->max_deg = std::max<int32_t>(pd->max_deg, (int32_t)(pd->row_ptr[(size_t)i + 1] - pd->row_ptr[(size_t)i]));
    return true;
}

static double micromodulus_host(const pdmts_pd *pd, double xi2)
{
    double r = std::sqrt(xi2);
    if (pd->micro_kind == PDMTS_MICRO_EXP)
        return pd->c * std::exp(-r / pd->l);
    return pd->c / (xi2 * r);
}

// Device arrays of the family and the state.
static int alloc_f32_state(pdmts_pd *pd);

// The 3D lattice kernel's row table: per stencil row (dz, dy) the per-|d|^2
// constants of its bonds (the expressions and rounding of the sliced-ELL
// stencil table), its node offset and its reach in dx.
static int upload_row_table(pdmts_pd *pd)
{
    const lat3d::RowTab t = lat3d::make_row_tab();
    const double h = pd->h;
    const int64_t nx = pd->lat_dims[0], ny = pd->lat_dims[1];
    if (3 * nx * ny > (int64_t)INT32_MAX)
        return fail(PDMTS_ERR_UNSUPPORTED, "pd_create: 3D lattice planes of %lld nodes too large",
                    (long long)(nx * ny));
    std::vector<Row3DEnt> rows(lat3d::NR);
    for (int r = 0; r < lat3d::NR; ++r) {
        const int dy = t.dy[r], dz = t.dz[r];
        float c[4] = {0.f, 0.f, 0.f, 0.f}, q[4] = {0.f, 0.f, 0.f, 0.f}, rr[4] = {0.f, 0.f, 0.f, 0.f},
              rd[4] = {0.f, 0.f, 0.f, 0.f};
        for (int a = 0; a < 4; ++a) {
            const int r2 = dy * dy + dz * dz + a * a;
            if (r2 > 9)
                continue;
            c[a] = (float)(micromodulus_host(pd, r2 * h * h) * h * h * pd->V[0]);
            q[a] = (float)(1.0 / r2);
            rr[a] = (float)r2;
            rd[a] = (float)std::sqrt((double)r2);
        }
        Row3DEnt &E = rows[(size_t)r];
        E.coef = make_float4(c[0], c[1], c[2], c[3]);
        E.ir2 = make_float4(q[0], q[1], q[2], q[3]);
        E.rr = make_float4(rr[0], rr[1], rr[2], rr[3]);
        E.rd = make_float4(rd[0], rd[1], rd[2], rd[3]);
        E.off = (int)(dz * nx * ny + dy * nx);
        E.fdy = (float)dy;
        E.fdz = (float)dz;
        E.rx = t.rx[r];
    }
    PDMTS_TRY(pd->alloc(pd->d_rowtab, lat3d::NR));
    return upload(pd->d_rowtab, rows.data(), lat3d::NR, pd->ctx->stream);
}

static int upload_family_and_state(pdmts_pd *pd)
{
    cudaStream_t s = pd->ctx->stream;
    const int dim = pd->dim;
    const int64_t n = pd->n;
    if (pd->layout == pdmts_pd::LAYOUT_LATTICE2D || pd->layout == pdmts_pd::LAYOUT_LATTICE3D) {
        const int64_t nw = pd->n_mask_words;
        PDMTS_TRY(pd->alloc(pd->d_mask, nw));
        PDMTS_TRY(pd->alloc(pd->d_exists, nw));
        PDMTS_TRY(pd->alloc(pd->d_V, n));
        PDMTS_TRY(pd->alloc(pd->d_out, (int64_t)dim * n));
        PDMTS_TRY(upload(pd->d_mask, pd->mask_host.data(), nw, s));
        PDMTS_TRY(upload(pd->d_exists, pd->mask_host.data(), nw, s));
        PDMTS_TRY(upload(pd->d_V, pd->V.data(), n, s));
        if (pd->layout == pdmts_pd::LAYOUT_LATTICE3D)
            PDMTS_TRY(upload_row_table(pd));
        return alloc_f32_state(pd);
    }
    PDMTS_TRY(pd->alloc(pd->d_tile_ptr, pd->ntiles + 1));
    PDMTS_TRY(pd->alloc(pd->d_mask_ptr, pd->ntiles + 1));
    PDMTS_TRY(pd->alloc(pd->d_tile_k, pd->ntiles));
    PDMTS_TRY(pd->alloc(pd->d_col, pd->n_slots));
    PDMTS_TRY(pd->alloc(pd->d_deg, n));
    PDMTS_TRY(pd->alloc(pd->d_mask, std::max<int64_t>(pd->n_mask_words, 1)));
    PDMTS_TRY(pd->alloc(pd->d_V, n));
    PDMTS_TRY(pd->alloc(pd->d_out, (int64_t)dim * n));
    PDMTS_TRY(upload(pd->d_tile_ptr, pd->tile_ptr.data(), pd->ntiles + 1, s));
    PDMTS_TRY(upload(pd->d_mask_ptr, pd->mask_ptr.data(), pd->ntiles + 1, s));
    PDMTS_TRY(upload(pd->d_tile_k, pd->tile_k.data(), pd->ntiles, s));
    PDMTS_TRY(upload(pd->d_deg, pd->deg.data(), n, s));
    PDMTS_TRY(upload(pd->d_mask, pd->mask_host.data(), std::max<int64_t>(pd->n_mask_words, 1), s));
    PDMTS_TRY(upload(pd->d_V, pd->V.data(), n, s));

    std::vector<int32_t> colS((size_t)std::max<int64_t>(pd->n_slots, 1), 0);
    if (pd->precision == PDMTS_FP64) {
        std::vector<double> cb((size_t)std::max<int64_t>(pd->n_slots, 1), 0.0);
        for (int64_t i = 0; i < n; ++i) {
            int64_t t = i / 32, lane = i % 32;
            for (int32_t k = 0; k < pd->tile_k[(size_t)t]; ++k) {
                int64_t slot = pd->tile_ptr[(size_t)t] + 32 * (int64_t)k + lane;
                if (k < pd->deg[(size_t)i]) {
                    int64_t j = pd->col[(size_t)(pd->row_ptr[(size_t)i] + k)];
                    colS[(size_t)slot] = (int32_t)j;
                    double xi2 = 0.0;
                    for (int d = 0; d < dim; ++d) {
                        double e = pd->X[(size_t)d * n + j] - pd->X[(size_t)d * n + i];
                        xi2 += e * e;
                    }
                    cb[(size_t)slot] = micromodulus_host(pd, xi2);
                } else {
                    colS[(size_t)slot] = (int32_t)i;  // padding: self, bit 0
                }
            }
        }
        // padding of the last tile's missing lanes
        for (int64_t i = n; i < pd->ntiles * 32; ++i) {
            int64_t t = i / 32, lane = i % 32;
            for (int32_t k = 0; k < pd->tile_k[(size_t)t]; ++k)
                colS[(size_t)(pd->tile_ptr[(size_t)t] + 32 * (int64_t)k + lane)] = 0;
        }
        PDMTS_TRY(pd->alloc(pd->d_cb, pd->n_slots));
        PDMTS_TRY(upload(pd->d_cb, cb.data(), pd->n_slots, s));
        PDMTS_TRY(upload(pd->d_col, colS.data(), pd->n_slots, s));
        PDMTS_TRY(pd->alloc(pd->d_X, (int64_t)dim * n));
        PDMTS_TRY(upload(pd->d_X, pd->X.data(), (int64_t)dim * n, s));
        for (int b = 0; b < 2; ++b)
            PDMTS_TRY(pd->alloc(pd->d_u[b], (int64_t)dim * n));
        PDMTS_TRY(pd->alloc(pd->d_v, (int64_t)dim * n));
        PDMTS_TRY(pd->alloc(pd->d_a, (int64_t)dim * n));
        PDMTS_CUDA_TRY(cudaMemsetAsync(pd->d_u[0].p, 0, sizeof(double) * dim * n, s));
        PDMTS_CUDA_TRY(cudaMemsetAsync(pd->d_u[1].p, 0, sizeof(double) * dim * n, s));
        PDMTS_CUDA_TRY(cudaMemsetAsync(pd->d_v.p, 0, sizeof(double) * dim * n, s));
        PDMTS_CUDA_TRY(cudaMemsetAsync(pd->d_a.p, 0, sizeof(double) * dim * n, s));
    } else {
        // stencil table over the distinct lattice offsets
        std::map<std::array<int32_t, 3>, int> ids;
        std::vector<StencilEntry> table;
        const double h = pd->h;
        const double V = pd->V[0];
        for (int64_t i = 0; i < n; ++i) {
            int64_t t = i / 32, lane = i % 32;
            for (int32_t k = 0; k < pd->tile_k[(size_t)t]; ++k) {
                int64_t slot = pd->tile_ptr[(size_t)t] + 32 * (int64_t)k + lane;
                if (k >= pd->deg[(size_t)i]) {
                    colS[(size_t)slot] = (int32_t)((uint32_t)i << 8);
                    continue;
                }
                int64_t j = pd->col[(size_t)(pd->row_ptr[(size_t)i] + k)];
                std::array<int32_t, 3> off{0, 0, 0};
                for (int d = 0; d < dim; ++d)
                    off[(size_t)d] = pd->lk[(size_t)d * n + j] - pd->lk[(size_t)d * n + i];
                auto it = ids.find(off);
                int id;
                if (it == ids.end()) {
                    id = (int)table.size();
                    if (id >= kMaxStencil)
                        return fail(PDMTS_ERR_UNSUPPORTED, "pd_create: more than %d lattice offsets", kMaxStencil);
                    ids[off] = id;
                    double r2 = 0.0;
                    for (int d = 0; d < dim; ++d)
                        r2 += (double)off[(size_t)d] * off[(size_t)d];
                    StencilEntry e{};
                    for (int d = 0; d < 3; ++d)
                        e.d[d] = (float)off[(size_t)d];
                    double xi2 = r2 * h * h;
                    e.coef = (float)(micromodulus_host(pd, xi2) * h * h * V);
                    e.thr = (float)(pd->s0 * (2.0 + pd->s0) * r2);
                    e.rd = (float)std::sqrt(r2);
                    e.r2 = (float)r2;
                    table.push_back(e);
                } else {
                    id = it->second;
                }
                colS[(size_t)slot] = (int32_t)(((uint32_t)j << 8) | (uint32_t)id);
            }
        }
        for (int64_t i = n; i < pd->ntiles * 32; ++i) {
            int64_t t = i / 32, lane = i % 32;
            for (int32_t k = 0; k < pd->tile_k[(size_t)t]; ++k)
                colS[(size_t)(pd->tile_ptr[(size_t)t] + 32 * (int64_t)k + lane)] = 0;
        }
        pd->n_stencil = (int)table.size();
        PDMTS_TRY(pd->alloc(pd->d_stencil, std::max<int64_t>(pd->n_stencil, 1)));
        PDMTS_TRY(upload(pd->d_stencil, table.data(), pd->n_stencil, s));
        PDMTS_TRY(upload(pd->d_col, colS.data(), pd->n_slots, s));
        PDMTS_TRY(alloc_f32_state(pd));
    }
    return PDMTS_OK;
}

static int alloc_f32_state(pdmts_pd *pd)
{
    cudaStream_t s = pd->ctx->stream;
    const int dim = pd->dim;
    const int64_t n = pd->n;
    const int adim = dim == 2 ? 2 : 4;
    for (int b = 0; b < 2; ++b) {
        PDMTS_TRY(pd->alloc(pd->f_u4[b], n));
        PDMTS_CUDA_TRY(cudaMemsetAsync(pd->f_u4[b].p, 0, sizeof(float4) * n, s));
        if (dim == 3) {
            PDMTS_TRY(pd->alloc(pd->f_u2[b], n));
            PDMTS_CUDA_TRY(cudaMemsetAsync(pd->f_u2[b].p, 0, sizeof(float2) * n, s));
        }
    }
    PDMTS_TRY(pd->alloc(pd->f_v4, n));
    PDMTS_CUDA_TRY(cudaMemsetAsync(pd->f_v4.p, 0, sizeof(float4) * n, s));
    if (dim == 3) {
        PDMTS_TRY(pd->alloc(pd->f_v2, n));
        PDMTS_CUDA_TRY(cudaMemsetAsync(pd->f_v2.p, 0, sizeof(float2) * n, s));
    }
    PDMTS_TRY(pd->alloc(pd->f_a, (int64_t)adim * n));
    PDMTS_CUDA_TRY(cudaMemsetAsync(pd->f_a.p, 0, sizeof(float) * adim * n, s));
    return PDMTS_OK;
}

// (Re)build the per-node weight and load arrays: mass (1 - alpha) rho,
// (1 - alpha) b, and the interface force density g (Eq. 33-34).
int pdmts_pd::upload_weights_and_loads()
{
    pd_invalidate_graphs(this);
    cudaStream_t s = ctx->stream;
    const bool has_alpha = !alpha.empty();
    for (int64_t i = 0; i < n; ++i) {
        double ai = has_alpha ? alpha[(size_t)i] : 0.0;
        if (!((1.0 - ai) * rho > 0.0))
            return fail(PDMTS_ERR_MASS, "PD node %lld has non-positive weighted mass (alpha = %g)",
                        (long long)i, ai);
    }
    if (precision == PDMTS_FP64) {
        std::vector<double> mass((size_t)n);
        for (int64_t i = 0; i < n; ++i)
            mass[(size_t)i] = (1.0 - (has_alpha ? alpha[(size_t)i] : 0.0)) * rho;
        PDMTS_TRY(alloc(d_mass, n));
        PDMTS_TRY(upload(d_mass, mass.data(), n, s));
        if (has_alpha) {
            PDMTS_TRY(alloc(d_alpha, n));
            PDMTS_TRY(upload(d_alpha, alpha.data(), n, s));
        } else {
            release(d_alpha);
        }
        if (has_b) {
            if (!d_wb.p)
                PDMTS_TRY(alloc(d_wb, (int64_t)dim * n));
            cudaError_t e = launch_weighted_load(dim, n, d_b.p, d_alpha.p, nullptr, 0.0, d_wb.p, nullptr,
                                                 nullptr, s);
            if (e != cudaSuccess)
                return fail(PDMTS_ERR_CUDA, "weighted load kernel: %s", cudaGetErrorString(e));
        } else {
            release(d_wb);
        }
    } else {
        std::vector<float> invm((size_t)n);
        for (int64_t i = 0; i < n; ++i)
            invm[(size_t)i] = (float)(1.0 / ((1.0 - (has_alpha ? alpha[(size_t)i] : 0.0)) * rho));
        PDMTS_TRY(alloc(f_invm, n));
        PDMTS_TRY(upload(f_invm, invm.data(), n, s));
        std::vector<int32_t> rowa;
        if (has_alpha) {
            std::vector<float> af(alpha.begin(), alpha.end());
            PDMTS_TRY(alloc(f_alpha, n));
            PDMTS_TRY(upload(f_alpha, af.data(), n, s));
            if (layout == LAYOUT_LATTICE2D || layout == LAYOUT_LATTICE3D) {
                const int64_t nx = lat_dims[0], ny = lat_dims[1];
                std::vector<uint8_t> flag((size_t)ny, 0);
                for (int64_t i = 0; i < n; ++i)
                    if (af[(size_t)i] != 0.f)
                        flag[(size_t)((i / nx) % ny)] = 1;
                rowa.assign((size_t)ny + 1, 0);
                for (int64_t y = 0; y < ny; ++y)
                    rowa[(size_t)y + 1] = rowa[(size_t)y] + flag[(size_t)y];
                PDMTS_TRY(alloc(f_rowalpha, ny + 1));
                PDMTS_TRY(upload(f_rowalpha, rowa.data(), ny + 1, s));
            }
        } else {
            release(f_alpha);
            release(f_rowalpha);
        }
        if (has_b) {
            if (!f_wb.p)
                PDMTS_TRY(alloc(f_wb, (int64_t)dim * n));
            cudaError_t e = launch_weighted_load(dim, n, d_b.p, nullptr, f_alpha.p, 1.0 / h, nullptr, f_wb.p,
                                                 nullptr, s);
            if (e != cudaSuccess)
                return fail(PDMTS_ERR_CUDA, "weighted load kernel: %s", cudaGetErrorString(e));
        } else {
            release(f_wb);
        }
    }
    PDMTS_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors above are temporaries
    return PDMTS_OK;
}

// One substep. u[cur] holds the displacement at the current time and
// u[1 - cur] its velocity-Verlet prediction for the next time. A substep
// evaluates forces (with breaking) at the prediction u[1 - cur], updates a and
// v, writes the following prediction over the old u[cur], and swaps, so that
// cur again names the current time. With init, a is computed from u[cur] and
// the first prediction u + dt v + dt^2/2 a is written to u[1 - cur]; no swap.
// Arguments of the lattice kernel around the per-node arguments N.
pdmts::Lat2DArgs pdmts_pd::lattice_args(const pdmts::F32NodeArgs &N, uint32_t *mask, bool link) const
{
    Lat2DArgs A{};
    A.nx = lat_dims[0];
    A.ny = lat_dims[1];
    A.mask = mask;
    A.alpha = f_alpha.p;
    A.alpha_rows = f_alpha.p ? f_rowalpha.p : nullptr;
    for (int r2 = 0; r2 < 10; ++r2) {
        const double coef = r2 > 0 ? micromodulus_host(this, r2 * h * h) * h * h * V[0] : 0.0;
        A.clin[r2] = (float)(coef * r2 / 2.0);
        A.cpmb[r2] = (float)(coef * r2 * r2);
    }
    A.qthr = (float)(s0 * (2.0 + s0));
    A.qfast = (float)(s0 * (2.0 + s0) * (1.0 - 1.0 / 4096.0));
    A.tile = link && link_tile >= 0 ? link_tile : lattice_tile >= 0 ? lattice_tile : 0;
    A.num_sms = ctx->num_sms;
    A.first_polls = ctx->first_wait_polls;
    A.nd = N;
    const bool grow = link && chain_k >= 0 && chain_k < (int)link_step_win.size();
    for (int w = 0; w < 2; ++w) {
        A.win_lo[w] = !link ? 0 : grow ? link_step_win[(size_t)chain_k][2 * w] : link_win_lo[w];
        A.win_n[w] = !link ? 0 : grow ? link_step_win[(size_t)chain_k][2 * w + 1] : link_win_n[w];
    }
    return A;
}

// Arguments of one 3D lattice substep: the per-|d|^2 constants are the ones
// the sliced-ELL stencil table holds (same expressions, same rounding).
pdmts::Lat3DArgs pdmts_pd::lattice3d_args(const pdmts::F32NodeArgs &N, uint32_t *mask, bool link) const
{
    Lat3DArgs A{};
    A.nx = lat_dims[0];
    A.ny = lat_dims[1];
    A.nz = lat_dims[2];
    A.mask = mask;
    A.exists = d_exists.p;
    A.alpha = f_alpha.p;
    A.alpha_rows = f_alpha.p ? f_rowalpha.p : nullptr;
    A.rows = d_rowtab.p;
    for (int r2 = 1; r2 < 10; ++r2) {
        const double xi2 = r2 * h * h;
        A.coef[r2] = (float)(micromodulus_host(this, xi2) * h * h * V[0]);
        A.thr[r2] = (float)(s0 * (2.0 + s0) * r2);
        A.rd[r2] = (float)std::sqrt((double)r2);
        A.r2[r2] = (float)r2;
        A.ir2[r2] = (float)(1.0 / r2);
    }
    A.qfast = (float)(s0 * (2.0 + s0) * (1.0 - 1.0 / 65536.0));
    A.tile = link && link_tile >= 0 ? link_tile : lattice_tile >= 0 ? lattice_tile : 0;
    A.nd = N;
    return A;
}

// Lattice tile autotuner: times every tile configuration on scratch copies of
// the FP32 state (the simulation state and counters are not touched) and keeps
// the fastest. Runs once, before the first substep chain is captured.
int pdmts_pd::tune_lattice(cudaStream_t s)
{
    if (layout == LAYOUT_LATTICE3D)
        return tune_lattice3d(s);
    if (lattice_tile >= 0 || layout != LAYOUT_LATTICE2D || precision == PDMTS_FP64)
        return PDMTS_OK;
    DevArr<float4> su[2], sv;
    DevArr<float> sa;
    DevArr<uint32_t> sm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int best = 0;
    float best_ms = 0.f;
    int r = PDMTS_OK;
    auto release_all = [&]() {
        release(su[0]); release(su[1]); release(sv); release(sa); release(sm);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if ((r = alloc(su[0], n)) != PDMTS_OK || (r = alloc(su[1], n)) != PDMTS_OK || (r = alloc(sv, n)) != PDMTS_OK ||
        (r = alloc(sa, 2 * n)) != PDMTS_OK || (r = alloc(sm, n_mask_words)) != PDMTS_OK) {
        release_all();
        return r;
    }
    cudaError_t e = cudaMemcpyAsync(su[0].p, f_u4[cur].p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sv.p, f_v4.p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sa.p, f_a.p, sizeof(float) * 2 * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sm.p, d_mask.p, sizeof(uint32_t) * n_mask_words, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    F32NodeArgs N{};
    N.n = n;
    N.inv_m = f_invm.p;
    N.wb = f_wb.p;
    N.g = has_g ? f_g.p : nullptr;
    N.v4 = sv.p;
    N.a = sa.p;
    N.dt = (float)ctx->dt_pd;
    N.hdt = (float)(0.5 * ctx->dt_pd);
    N.hdt2 = (float)(0.5 * ctx->dt_pd * ctx->dt_pd);
    N.breaking = breaking ? 1 : 0;
    N.pmb = force_kind == PDMTS_FORCE_PMB;
    N.broken = nullptr;
    for (int t = 0; t < kLatTiles && e == cudaSuccess; ++t) {
        Lat2DArgs A = lattice_args(N, sm.p, false);
        A.tile = t;
        int c = 0;
        for (int k = 0; k < 12 && e == cudaSuccess; ++k) {
            if (k == 2)
                e = cudaEventRecord(e0, s);
            A.nd.u4_in = su[c].p;
            A.nd.u4_out = su[1 - c].p;
            if (e == cudaSuccess)
                e = launch_pd_step_lattice2d(A, false, s);
            c = 1 - c;
        }
        if (e == cudaSuccess)
            e = cudaEventRecord(e1, s);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (t == 0 || ms < best_ms)) {
            best = t;
            best_ms = ms;
        }
    }
    // link chains (coupled subdomains): the launches of a link run cover only
    // the growing windows around the overlap bands, a few hundred tiles each,
    // where a CTA's latency rather than the work decides; time every
    // configuration over one chain of those windows (second of two passes)
    int best_link = -1;
    float best_link_ms = 0.f;
    const int nwin = (int)link_step_win.size();
    for (int t = 0; t < kLatTiles && nwin > 0 && e == cudaSuccess; ++t) {
        Lat2DArgs A = lattice_args(N, sm.p, false);
        A.tile = t;
        int c = 0;
        for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
            if (pass == 1)
                e = cudaEventRecord(e0, s);
            for (int k = 0; k < nwin && e == cudaSuccess; ++k) {
                for (int w = 0; w < 2; ++w) {
                    A.win_lo[w] = link_step_win[(size_t)k][2 * w];
                    A.win_n[w] = link_step_win[(size_t)k][2 * w + 1];
                }
                A.nd.u4_in = su[c].p;
                A.nd.u4_out = su[1 - c].p;
                e = launch_pd_step_lattice2d(A, false, s);
                c = 1 - c;
            }
        }
        if (e == cudaSuccess)
            e = cudaEventRecord(e1, s);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best_link < 0 || ms < best_link_ms)) {
            best_link = t;
            best_link_ms = ms;
        }
    }
    release_all();
    if (e != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "lattice autotune: %s", cudaGetErrorString(e));
    lattice_tile = best;
    link_tile = best_link;
    pd_invalidate_graphs(this);
    return PDMTS_OK;
}

// The 3D lattice tile configurations (blocks of 32 x 4 and 32 x 8 nodes) timed
// the same way on scratch copies of the state; all give the same bits. The
// link chains of a coupled subdomain run on the whole box and take the same
// configuration.
int pdmts_pd::tune_lattice3d(cudaStream_t s)
{
    if (lattice_tile >= 0 || precision == PDMTS_FP64)
        return PDMTS_OK;
    DevArr<float4> su4[2], sv4, sa;
    DevArr<float2> su2[2], sv2;
    DevArr<uint32_t> sm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int best = 0;
    float best_ms = 0.f;
    int r = PDMTS_OK;
    auto release_all = [&]() {
        release(su4[0]); release(su4[1]); release(sv4); release(sa); release(su2[0]); release(su2[1]);
        release(sv2); release(sm);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if ((r = alloc(su4[0], n)) != PDMTS_OK || (r = alloc(su4[1], n)) != PDMTS_OK ||
        (r = alloc(su2[0], n)) != PDMTS_OK || (r = alloc(su2[1], n)) != PDMTS_OK || (r = alloc(sv4, n)) != PDMTS_OK ||
        (r = alloc(sv2, n)) != PDMTS_OK || (r = alloc(sa, n)) != PDMTS_OK || (r = alloc(sm, n_mask_words)) != PDMTS_OK) {
        release_all();
        return r;
    }
    cudaError_t e = cudaMemcpyAsync(su4[0].p, f_u4[cur].p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(su2[0].p, f_u2[cur].p, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sv4.p, f_v4.p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sv2.p, f_v2.p, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sa.p, f_a.p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sm.p, d_mask.p, sizeof(uint32_t) * n_mask_words, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    F32NodeArgs N{};
    N.n = n;
    N.inv_m = f_invm.p;
    N.wb = f_wb.p;
    N.g = has_g ? f_g.p : nullptr;
    N.v4 = sv4.p;
    N.v2 = sv2.p;
    N.a = reinterpret_cast<float *>(sa.p);
    N.dt = (float)ctx->dt_pd;
    N.hdt = (float)(0.5 * ctx->dt_pd);
    N.hdt2 = (float)(0.5 * ctx->dt_pd * ctx->dt_pd);
    N.breaking = breaking ? 1 : 0;
    N.pmb = force_kind == PDMTS_FORCE_PMB;
    N.broken = nullptr;
    for (int t = 0; t < kLat3DTiles && e == cudaSuccess; ++t) {
        Lat3DArgs A = lattice3d_args(N, sm.p, false);
        A.tile = t;
        int c = 0;
        for (int k = 0; k < 12 && e == cudaSuccess; ++k) {
            if (k == 2)
                e = cudaEventRecord(e0, s);
            A.nd.u4_in = su4[c].p;
            A.nd.u2_in = su2[c].p;
            A.nd.u4_out = su4[1 - c].p;
            A.nd.u2_out = su2[1 - c].p;
            if (e == cudaSuccess)
                e = launch_pd_step_lattice3d(A, false, s);
            c = 1 - c;
        }
        if (e == cudaSuccess)
            e = cudaEventRecord(e1, s);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (t == 0 || ms < best_ms)) {
            best = t;
            best_ms = ms;
        }
    }
    release_all();
    if (e != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "3D lattice autotune: %s", cudaGetErrorString(e));
    lattice_tile = best;
    link_tile = -1;
    pd_invalidate_graphs(this);
    return PDMTS_OK;
}

// Per-node arguments of one FP32-bulk substep at the current buffer parity.
F32NodeArgs pdmts_pd::f32_node_args(bool init, double theta, bool link) const
{
    const double dt = ctx->dt_pd;
    const int c = link ? lk_cur : cur;
    const int src = init ? c : 1 - c;  // buffer the forces are evaluated at
    const int dst = 1 - src;           // buffer receiving the next prediction
    F32NodeArgs N{};
    N.n = n;
    N.inv_m = f_invm.p;
    N.wb = link ? nullptr : f_wb.p;
    N.g = link ? lk_gf.p : (has_g ? f_g.p : nullptr);
    N.u4_in = link ? lk_u4[src].p : f_u4[src].p;
    N.u2_in = link ? lk_u2[src].p : f_u2[src].p;
    N.u4_out = link ? lk_u4[dst].p : f_u4[dst].p;
    N.u2_out = link ? lk_u2[dst].p : f_u2[dst].p;
    N.v4 = link ? lk_v4.p : f_v4.p;
    N.v2 = link ? lk_v2.p : f_v2.p;
    N.a = link ? lk_af.p : f_a.p;
    N.dt = (float)dt;
    N.hdt = (float)(0.5 * dt);
    N.hdt2 = (float)(0.5 * dt * dt);
    N.theta = (float)theta;
    N.breaking = (breaking && !link) ? 1 : 0;
    N.pmb = force_kind == PDMTS_FORCE_PMB;
    N.broken = ctx->d_counter;
    return N;
}

// Bookkeeping after a substep was enqueued: buffer parity and counters.
void pdmts_pd::substep_done(bool init, bool link)
{
    ctx->stats.kernel_launches++;
    if (init)
        return;
    int &c = link ? lk_cur : cur;
    c = 1 - c;
    if (!link)
        steps_done++;
    ctx->stats.pd_substeps++;
    ctx->stats.bond_updates += substep_bonds(link, chain_k);
}

int pdmts_pd::step(bool init, double theta, cudaStream_t s, bool link)
{
    const double dt = ctx->dt_pd;
    cudaError_t e;
    SellView fam{d_tile_ptr.p, d_tile_k.p, d_mask_ptr.p, d_col.p, d_mask.p, d_deg.p, n, ntiles};
    const int c = link ? lk_cur : cur;
    const int src = init ? c : 1 - c;  // buffer the forces are evaluated at
    const int dst = 1 - src;           // buffer receiving the next prediction
    uint32_t *mask = link ? d_mask_link.p : d_mask.p;
    fam.mask = mask;
    if (precision == PDMTS_FP64) {
        F64StepArgs A{};
        A.fam = fam;
        A.X = d_X.p;
        A.V = d_V.p;
        A.cb = d_cb.p;
        A.alpha = d_alpha.p;
        A.mass = d_mass.p;
        A.wb = link ? nullptr : d_wb.p;
        A.g = link ? lk_g.p : (has_g ? d_g.p : nullptr);
        A.u_in = link ? lk_u[src].p : d_u[src].p;
        A.u_out = link ? lk_u[dst].p : d_u[dst].p;
        A.v = link ? lk_v.p : d_v.p;
        A.a = link ? lk_a.p : d_a.p;
        A.s0p2 = (1.0 + s0) * (1.0 + s0);
        A.dt = dt;
        A.hdt = 0.5 * dt;
        A.hdt2 = 0.5 * dt * dt;
        A.theta = theta;
        A.breaking = (breaking && !link) ? 1 : 0;
        A.pmb = force_kind == PDMTS_FORCE_PMB;
        A.broken = ctx->d_counter;
        e = launch_pd_step_f64(dim, A, init, s);
    } else {
        const F32NodeArgs N = f32_node_args(init, theta, link);
        if (layout == LAYOUT_LATTICE2D) {
            Lat2DArgs A = lattice_args(N, mask, link);
            A.pdl = chain_follow ? 1 : 0;
            e = launch_pd_step_lattice2d(A, init, s);
        } else if (layout == LAYOUT_LATTICE3D) {
            Lat3DArgs A = lattice3d_args(N, mask, link);
            A.pdl = chain_follow ? 1 : 0;
            e = launch_pd_step_lattice3d(A, init, s);
        } else {
            F32StepArgs A{};
            A.fam = fam;
            A.stencil = d_stencil.p;
            A.n_stencil = n_stencil;
            A.alpha = f_alpha.p;
            A.nd = N;
            e = launch_pd_step_f32(dim, A, init, s);
        }
    }
    if (e != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "PD substep launch failed: %s", cudaGetErrorString(e));
    substep_done(init, link);
    return PDMTS_OK;
}

int pdmts_pd::ensure_init(cudaStream_t s)
{
    if (!need_init)
        return PDMTS_OK;
    PDMTS_TRY(step(true, 0.0, s));
    need_init = false;
    return PDMTS_OK;
}

// ------------------------------------------------------------ PD ABI ------
extern "C" int pd_create(pdmts_ctx *ctx, int dim, int64_t n, const double *X, const double *vol,
                         double vol_uniform, double horizon, int micro_kind, double c, double l,
                         double s0, double rho, int precision, pdmts_pd **out)
{
    clear_error();
    if (!ctx || !X || !out)
        return fail(PDMTS_ERR_ARG, "pd_create: NULL argument");
    *out = nullptr;
    if (ctx->pd)
        return fail(PDMTS_ERR_STATE, "pd_create: context already has a PD subdomain");
    if (dim != 2 && dim != 3)
        return fail(PDMTS_ERR_ARG, "pd_create: dim must be 2 or 3 (got %d)", dim);
    if (n <= 0 || n >= ((int64_t)1 << 31))
        return fail(PDMTS_ERR_ARG, "pd_create: n out of range (%lld)", (long long)n);
    if (!(horizon > 0) || !std::isfinite(horizon))
        return fail(PDMTS_ERR_ARG, "pd_create: horizon must be > 0");
    if (!(s0 > 0) || !std::isfinite(s0))
        return fail(PDMTS_ERR_ARG, "pd_create: s0 must be > 0");
    if (!(rho > 0) || !std::isfinite(rho))
        return fail(PDMTS_ERR_ARG, "pd_create: rho must be > 0");
    if (!(c > 0) || !std::isfinite(c))
        return fail(PDMTS_ERR_ARG, "pd_create: micromodulus constant must be > 0");
    if (micro_kind != PDMTS_MICRO_POWER && micro_kind != PDMTS_MICRO_EXP)
        return fail(PDMTS_ERR_ARG, "pd_create: unknown micromodulus kind %d", micro_kind);
    if (micro_kind == PDMTS_MICRO_EXP && !(l > 0))
        return fail(PDMTS_ERR_ARG, "pd_create: exponential micromodulus needs l > 0");
    if (precision != PDMTS_FP64 && precision != PDMTS_FP32_BULK && precision != PDMTS_FP32_BULK_SELL)
        return fail(PDMTS_ERR_ARG, "pd_create: unknown precision %d", precision);
    const bool force_sell = precision == PDMTS_FP32_BULK_SELL;
    if (force_sell)
        precision = PDMTS_FP32_BULK;
    if (!vol && !(vol_uniform > 0))
        return fail(PDMTS_ERR_ARG, "pd_create: vol_uniform must be > 0 when vol is NULL");
    PDMTS_CUDA_TRY(cudaSetDevice(ctx->device));

    auto *pd = new (std::nothrow) pdmts_pd();
    if (!pd)
        return fail(PDMTS_ERR_NOMEM, "pd_create: out of host memory");
    pd->ctx = ctx;
    pd->dim = dim;
    pd->n = n;
    pd->precision = precision;
    pd->horizon = horizon;
    pd->c = c;
    pd->l = l;
    pd->s0 = s0;
    pd->rho = rho;
    pd->micro_kind = micro_kind;
    int r = fetch(pd->X, X, (int64_t)dim * n);
    if (r == PDMTS_OK && !finite_all(pd->X.data(), (int64_t)dim * n))
        r = fail(PDMTS_ERR_ARG, "pd_create: X contains NaN/Inf");
    if (r == PDMTS_OK) {
        if (vol) {
            r = fetch(pd->V, vol, n);
            pd->uniform_vol = false;
            for (int64_t i = 0; r == PDMTS_OK && i < n; ++i)
                if (!(pd->V[(size_t)i] > 0) || !std::isfinite(pd->V[(size_t)i]))
                    r = fail(PDMTS_ERR_ARG, "pd_create: vol[%lld] must be finite and > 0", (long long)i);
        } else {
            pd->V.assign((size_t)n, vol_uniform);
        }
    }
    if (r == PDMTS_OK)
        r = build_family(pd);
    if (r == PDMTS_OK) {
        detect_lattice(pd);
        if (precision == PDMTS_FP32_BULK) {
            if (!pd->on_lattice)
                r = fail(PDMTS_ERR_UNSUPPORTED, "pd_create: FP32_BULK needs nodes on a regular lattice");
            else if (vol)
                r = fail(PDMTS_ERR_UNSUPPORTED, "pd_create: FP32_BULK needs a uniform nodal volume");
            else if (n >= ((int64_t)1 << 24))
                r = fail(PDMTS_ERR_UNSUPPORTED, "pd_create: FP32_BULK supports n < 2^24 nodes");
        }
    }
    if (r == PDMTS_OK) {
        if (precision == PDMTS_FP64 || force_sell || (!try_lattice2d(pd) && !try_lattice3d(pd)))
            build_sell(pd);
        r = upload_family_and_state(pd);
    }
    if (r == PDMTS_OK)
        r = pd->upload_weights_and_loads();
    if (r == PDMTS_OK) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess)
            r = fail(PDMTS_ERR_CUDA, "pd_create: %s", cudaGetErrorString(e));
    }
    if (r != PDMTS_OK) {
        std::string msg = pdmts_last_error();
        pd->release_all();
        delete pd;
        return fail(r, "%s", msg.c_str());
    }
    ctx->pd = pd;
    *out = pd;
    return PDMTS_OK;
}

extern "C" int pd_destroy(pdmts_pd *pd)
{
    clear_error();
    if (!pd)
        return PDMTS_OK;
    cudaSetDevice(pd->ctx->device);
    cudaStreamSynchronize(pd->ctx->stream);
    if (pd->ctx->pd == pd)
        pd->ctx->pd = nullptr;
    pd->release_all();
    delete pd;
    return PDMTS_OK;
}

// Exact pre-crack test in half-spacing units (lattice) or FP64 (otherwise).
extern "C" int pd_set_precrack(pdmts_pd *pd, int n_cuts, const double *cuts)
{
    clear_error();
    if (!pd || (n_cuts > 0 && !cuts) || n_cuts < 0)
        return fail(PDMTS_ERR_ARG, "pd_set_precrack: bad arguments");
    std::vector<double> cv;
    PDMTS_TRY(fetch(cv, cuts, (int64_t)5 * n_cuts));
    const int dim = pd->dim;
    const int64_t n = pd->n;
    struct CutI {
        int na, pa;
        int64_t level, lo, hi;
        double lv, lod, hid;
        bool exact;
    };
    std::vector<CutI> cl;
    for (int c = 0; c < n_cuts; ++c) {
        const double *q = &cv[(size_t)5 * c];
        CutI k{};
        k.na = (int)q[0];
        k.pa = (int)q[2];
        if (k.na < 0 || k.na >= dim || k.pa < 0 || k.pa >= dim || k.na == k.pa || (double)k.na != q[0] ||
            (double)k.pa != q[2] || !std::isfinite(q[1]) || !std::isfinite(q[3]) || !std::isfinite(q[4]))
            return fail(PDMTS_ERR_ARG, "pd_set_precrack: cut %d is malformed", c);
        k.lv = q[1];
        k.lod = q[3];
        k.hid = q[4];
        k.exact = false;
        if (pd->on_lattice) {
            // half-spacing units relative to the lattice box corner x0 - h/2
            auto hu = [&](double v, int ax, int64_t &outv) {
                double t = (v - (pd->x0[(size_t)ax] - 0.5 * pd->h)) / (0.5 * pd->h);
                double r = std::nearbyint(t);
                if (std::fabs(t - r) > 1e-6 || std::fabs(r) > 4e9)
                    return false;
                outv = (int64_t)r;
                return true;
            };
            k.exact = hu(q[1], k.na, k.level) && hu(q[3], k.pa, k.lo) && hu(q[4], k.pa, k.hi);
        }
        cl.push_back(k);
    }
    // current bond status from the device
    PDMTS_CUDA_TRY(cudaSetDevice(pd->ctx->device));
    PDMTS_TRY(pd->ctx->begin());
    PDMTS_CUDA_TRY(cudaMemcpyAsync(pd->mask_host.data(), pd->d_mask.p, sizeof(uint32_t) * pd->n_mask_words,
                                   cudaMemcpyDeviceToHost, pd->ctx->stream));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(pd->ctx->stream));
    for (int64_t i = 0; i < n; ++i) {
        const int32_t deg_i = (int32_t)(pd->row_ptr[(size_t)i + 1] - pd->row_ptr[(size_t)i]);
        for (int32_t k = 0; k < deg_i; ++k) {
            int64_t j = pd->col[(size_t)(pd->row_ptr[(size_t)i] + k)];
            bool cut = false;
            for (const CutI &q : cl) {
                if (q.exact) {
                    int64_t ni = 2 * (int64_t)pd->lk[(size_t)q.na * n + i] + 1;
                    int64_t nj = 2 * (int64_t)pd->lk[(size_t)q.na * n + j] + 1;
                    int64_t ai = 2 * (int64_t)pd->lk[(size_t)q.pa * n + i] + 1;
                    int64_t aj = 2 * (int64_t)pd->lk[(size_t)q.pa * n + j] + 1;
                    if (!((ni < q.level && q.level < nj) || (nj < q.level && q.level < ni)))
                        continue;
                    // crossing point along pa: ai + (level - ni)(aj - ai)/(nj - ni) in [lo, hi)
                    int64_t den = nj - ni;
                    int64_t num = ai * den + (q.level - ni) * (aj - ai);
                    if (den < 0) {
                        den = -den;
                        num = -num;
                    }
                    if (num >= q.lo * den && num < q.hi * den)
                        cut = true;
                } else {
                    double ni = pd->X[(size_t)q.na * n + i], nj = pd->X[(size_t)q.na * n + j];
                    if (!((ni < q.lv && q.lv < nj) || (nj < q.lv && q.lv < ni)))
                        continue;
                    double ai = pd->X[(size_t)q.pa * n + i], aj = pd->X[(size_t)q.pa * n + j];
                    double xc = ai + (q.lv - ni) * (aj - ai) / (nj - ni);
                    if (xc >= q.lod && xc < q.hid)
                        cut = true;
                }
                if (cut)
                    break;
            }
            if (cut) {
                int64_t word;
                int bit;
                bond_bit(pd, i, k, word, bit);
                pd->mask_host[(size_t)word] &= ~(1u << bit);
            }
        }
    }
    PDMTS_CUDA_TRY(cudaMemcpyAsync(pd->d_mask.p, pd->mask_host.data(), sizeof(uint32_t) * pd->n_mask_words,
                                   cudaMemcpyHostToDevice, pd->ctx->stream));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(pd->ctx->stream));
    pd->need_init = true;
    return pd->ctx->end();
}

extern "C" int pd_set_body_force(pdmts_pd *pd, const double *b)
{
    clear_error();
    if (!pd)
        return fail(PDMTS_ERR_ARG, "pd_set_body_force: pd is NULL");
    PDMTS_CUDA_TRY(cudaSetDevice(pd->ctx->device));
    PDMTS_TRY(pd->ctx->begin());
    cudaStream_t s = pd->ctx->stream;
    const int64_t m = (int64_t)pd->dim * pd->n;
    if (!b) {
        pd->has_b = false;
        pd->release(pd->d_b);
        PDMTS_TRY(pd->upload_weights_and_loads());
        pd->need_init = true;
        return pd->ctx->end();
    }
    // stage, validate on the device, then commit (the state is untouched on failure)
    unsigned long long *flag = pd->ctx->d_counter + 1;
    PDMTS_CUDA_TRY(cudaMemcpyAsync(pd->d_out.p, b, sizeof(double) * m, cudaMemcpyDefault, s));
    PDMTS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(unsigned long long), s));
    cudaError_t e = launch_weighted_load(pd->dim, pd->n, pd->d_out.p, nullptr, nullptr, 0.0, nullptr, nullptr,
                                         flag, s);
    if (e != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "body force check: %s", cudaGetErrorString(e));
    unsigned long long bad = 0;
    PDMTS_CUDA_TRY(cudaMemcpyAsync(&bad, flag, sizeof(bad), cudaMemcpyDeviceToHost, s));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad)
        return fail(PDMTS_ERR_ARG, "pd_set_body_force: NaN/Inf in b");
    const bool fresh_arrays = !pd->has_b;
    if (!pd->d_b.p)
        PDMTS_TRY(pd->alloc(pd->d_b, m));
    PDMTS_CUDA_TRY(cudaMemcpyAsync(pd->d_b.p, pd->d_out.p, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    pd->has_b = true;
    if (fresh_arrays) {
        PDMTS_TRY(pd->upload_weights_and_loads());  // allocates the weighted-load arrays once
    } else {
        // same arrays, new values: captured substep graphs stay valid
        e = pd->precision == PDMTS_FP64
                ? launch_weighted_load(pd->dim, pd->n, pd->d_b.p, pd->d_alpha.p, nullptr, 0.0, pd->d_wb.p,
                                       nullptr, nullptr, s)
                : launch_weighted_load(pd->dim, pd->n, pd->d_b.p, nullptr, pd->f_alpha.p, 1.0 / pd->h, nullptr,
                                       pd->f_wb.p, nullptr, s);
        if (e != cudaSuccess)
            return fail(PDMTS_ERR_CUDA, "weighted load kernel: %s", cudaGetErrorString(e));
        pd->ctx->stats.kernel_launches++;
    }
    return pd->ctx->end();
}

extern "C" int pd_set_weights(pdmts_pd *pd, const double *alpha)
{
    clear_error();
    if (!pd)
        return fail(PDMTS_ERR_ARG, "pd_set_weights: pd is NULL");
    std::vector<double> na;
    if (alpha) {
        PDMTS_TRY(fetch(na, alpha, pd->n));
        for (int64_t i = 0; i < pd->n; ++i)
            if (!std::isfinite(na[(size_t)i]) || na[(size_t)i] < 0.0)
                return fail(PDMTS_ERR_ARG, "pd_set_weights: alpha[%lld] must be finite and >= 0", (long long)i);
    }
    PDMTS_CUDA_TRY(cudaSetDevice(pd->ctx->device));
    PDMTS_TRY(pd->ctx->begin());
    std::vector<double> old;
    old.swap(pd->alpha);
    pd->alpha.swap(na);
    int r = pd->upload_weights_and_loads();
    if (r != PDMTS_OK) {
        std::string msg = pdmts_last_error();
        pd->alpha.swap(old);
        pd->upload_weights_and_loads();
        return fail(r, "%s", msg.c_str());
    }
    pd->need_init = true;
    return pd->ctx->end();
}

extern "C" int pd_set_state(pdmts_pd *pd, const double *u, const double *v)
{
    clear_error();
    if (!pd)
        return fail(PDMTS_ERR_ARG, "pd_set_state: pd is NULL");
    const int64_t m = (int64_t)pd->dim * pd->n;
    std::vector<double> hu, hv;
    if (u) {
        PDMTS_TRY(fetch(hu, u, m));
        if (!finite_all(hu.data(), m))
            return fail(PDMTS_ERR_ARG, "pd_set_state: NaN/Inf in u");
    }
    if (v) {
        PDMTS_TRY(fetch(hv, v, m));
        if (!finite_all(hv.data(), m))
            return fail(PDMTS_ERR_ARG, "pd_set_state: NaN/Inf in v");
    }
    PDMTS_CUDA_TRY(cudaSetDevice(pd->ctx->device));
    PDMTS_TRY(pd->ctx->begin());
    cudaStream_t s = pd->ctx->stream;
    if (pd->precision == PDMTS_FP64) {
        if (u)
            PDMTS_CUDA_TRY(cudaMemcpyAsync(pd->d_u[pd->cur].p, hu.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
        else
            PDMTS_CUDA_TRY(cudaMemsetAsync(pd->d_u[pd->cur].p, 0, sizeof(double) * m, s));
        if (v)
            PDMTS_CUDA_TRY(cudaMemcpyAsync(pd->d_v.p, hv.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
        else
            PDMTS_CUDA_TRY(cudaMemsetAsync(pd->d_v.p, 0, sizeof(double) * m, s));
    } else {
        // compensated pairs in lattice units, packed per node
        const int dim = pd->dim;
        const int64_t n = pd->n;
        const double inv_h = 1.0 / pd->h;
        std::vector<float4> p4((size_t)n);
        std::vector<float2> p2((size_t)n);
        auto pack = [&](const std::vector<double> &src, float4 *d4, float2 *d2) -> int {
            float hv[3] = {0, 0, 0}, lv[3] = {0, 0, 0};
            for (int64_t i = 0; i < n; ++i) {
                for (int d = 0; d < dim; ++d) {
                    double x = src.empty() ? 0.0 : src[(size_t)d * n + i] * inv_h;
                    hv[d] = (float)x;
                    lv[d] = (float)(x - (double)hv[d]);
                }
                if (dim == 2) {
                    p4[(size_t)i] = make_float4(hv[0], hv[1], lv[0], lv[1]);
                } else {
                    p4[(size_t)i] = make_float4(hv[0], hv[1], hv[2], lv[0]);
                    p2[(size_t)i] = make_float2(lv[1], lv[2]);
                }
            }
            PDMTS_CUDA_TRY(cudaMemcpyAsync(d4, p4.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, s));
            if (dim == 3)
                PDMTS_CUDA_TRY(cudaMemcpyAsync(d2, p2.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, s));
            PDMTS_CUDA_TRY(cudaStreamSynchronize(s));
            return PDMTS_OK;
        };
        PDMTS_TRY(pack(hu, pd->f_u4[pd->cur].p, pd->f_u2[pd->cur].p));
        PDMTS_TRY(pack(hv, pd->f_v4.p, pd->f_v2.p));
    }
    PDMTS_CUDA_TRY(cudaStreamSynchronize(s));
    pd->need_init = true;
    return pd->ctx->end();
}

extern "C" int pd_set_breaking(pdmts_pd *pd, int enabled)
{
    clear_error();
    if (!pd)
        return fail(PDMTS_ERR_ARG, "pd_set_breaking: pd is NULL");
    pd->breaking = enabled != 0;
    pd_invalidate_graphs(pd);
    return PDMTS_OK;
}

extern "C" int pd_set_force_law(pdmts_pd *pd, int kind)
{
    clear_error();
    if (!pd)
        return fail(PDMTS_ERR_ARG, "pd_set_force_law: pd is NULL");
    if (kind != PDMTS_FORCE_LINEAR && kind != PDMTS_FORCE_PMB)
        return fail(PDMTS_ERR_ARG, "pd_set_force_law: unknown kind %d", kind);
    pd->force_kind = kind;
    pd->need_init = true;
    pd_invalidate_graphs(pd);
    return PDMTS_OK;
}

extern "C" int pd_set_lattice_tile(pdmts_pd *pd, int tile)
{
    clear_error();
    if (!pd)
        return fail(PDMTS_ERR_ARG, "pd_set_lattice_tile: pd is NULL");
    const int ntiles = pd->layout == pdmts_pd::LAYOUT_LATTICE3D ? kLat3DTiles : kLatTiles;
    if (tile != PDMTS_LATTICE_TILE_AUTO && (tile < 0 || tile >= ntiles))
        return fail(PDMTS_ERR_ARG, "pd_set_lattice_tile: tile %d outside [0, %d) and not AUTO", tile, ntiles);
    static_assert(kLatTiles == PDMTS_LATTICE_TILES, "tile table and ABI disagree");
    pd->lattice_tile = tile;
    pd->link_tile = -1;  // a fixed configuration serves the link chains too; AUTO tunes both
    pd_invalidate_graphs(pd);
    return PDMTS_OK;
}

extern "C" int pd_info(const pdmts_pd *pd, pdmts_pd_info *info)
{
    clear_error();
    if (!pd || !info)
        return fail(PDMTS_ERR_ARG, "pd_info: NULL argument");
    info->dim = pd->dim;
    info->precision = pd->precision;
    info->n = pd->n;
    info->n_bonds = pd->row_ptr.empty() ? 0 : pd->row_ptr[(size_t)pd->n];
    info->n_slots = pd->n_slots;
    info->max_degree = pd->max_deg;
    info->on_lattice = pd->on_lattice ? 1 : 0;
    info->layout = pd->layout;
    info->lattice_nx = pd->lat_dims[0];
    info->lattice_ny = pd->lat_dims[1];
    info->lattice_tile = pd->lattice_tile;
    info->lattice_h = pd->on_lattice ? pd->h : 0.0;
    info->steps_done = pd->steps_done;
    info->device_bytes = pd->device_bytes;
    info->lattice_nz = pd->layout == pdmts_pd::LAYOUT_LATTICE3D ? pd->lat_dims[2] : 0;
    info->link_tile = pd->link_tile >= 0 ? pd->link_tile : pd->lattice_tile;
    return PDMTS_OK;
}

// Copy a dim * n field at the current time into `out` (host or device).
static int read_field(pdmts_pd *pd, int which, double *out)
{
    if (!pd || !out)
        return fail(PDMTS_ERR_ARG, "pd_read: NULL argument");
    PDMTS_CUDA_TRY(cudaSetDevice(pd->ctx->device));
    PDMTS_TRY(pd->ctx->begin());
    cudaStream_t s = pd->ctx->stream;
    const int64_t m = (int64_t)pd->dim * pd->n;
    if (which == 2)
        PDMTS_TRY(pd->ensure_init(s));
    const double *src = nullptr;
    if (pd->precision == PDMTS_FP64) {
        src = which == 0 ? pd->d_u[pd->cur].p : which == 1 ? pd->d_v.p : pd->d_a.p;
    } else {
        const float4 *p4 = which == 0 ? pd->f_u4[pd->cur].p : which == 1 ? pd->f_v4.p : (const float4 *)pd->f_a.p;
        const float2 *p2 = which == 0 ? pd->f_u2[pd->cur].p : which == 1 ? pd->f_v2.p : nullptr;
        cudaError_t e = launch_unpack_f32(pd->dim, pd->n, p4, p2, which == 2, pd->h, pd->d_out.p, s);
        if (e != cudaSuccess)
            return fail(PDMTS_ERR_CUDA, "read-back conversion failed: %s", cudaGetErrorString(e));
        src = pd->d_out.p;
    }
    PDMTS_CUDA_TRY(cudaMemcpyAsync(out, src, sizeof(double) * m, cudaMemcpyDefault, s));
    PDMTS_TRY(pd->ctx->sync_checked("pd_read"));
    return pd->ctx->end();
}

extern "C" int pd_read_displacement(pdmts_pd *pd, double *u)
{
    clear_error();
    return read_field(pd, 0, u);
}
extern "C" int pd_read_velocity(pdmts_pd *pd, double *v)
{
    clear_error();
    return read_field(pd, 1, v);
}
extern "C" int pd_read_acceleration(pdmts_pd *pd, double *a)
{
    clear_error();
    return read_field(pd, 2, a);
}

extern "C" int pd_read_damage(pdmts_pd *pd, double *phi)
{
    clear_error();
    if (!pd || !phi)
        return fail(PDMTS_ERR_ARG, "pd_read_damage: NULL argument");
    PDMTS_CUDA_TRY(cudaSetDevice(pd->ctx->device));
    PDMTS_TRY(pd->ctx->begin());
    cudaStream_t s = pd->ctx->stream;
    SellView fam{pd->d_tile_ptr.p, pd->d_tile_k.p, pd->d_mask_ptr.p, pd->d_col.p, pd->d_mask.p, pd->d_deg.p,
                 pd->n, pd->ntiles};
    cudaError_t e = pd->layout != pdmts_pd::LAYOUT_SELL
                        ? launch_damage_lattice(pd->n, pd->d_mask.p, pd->d_exists.p,
                                                pd->layout == pdmts_pd::LAYOUT_LATTICE3D ? lat3d::W : 1, pd->d_out.p, s)
                        : launch_damage(fam, pd->precision == PDMTS_FP32_BULK, pd->d_V.p, pd->d_out.p, s);
    if (e != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "damage kernel failed: %s", cudaGetErrorString(e));
    pd->ctx->stats.kernel_launches++;
    PDMTS_CUDA_TRY(cudaMemcpyAsync(phi, pd->d_out.p, sizeof(double) * pd->n, cudaMemcpyDefault, s));
    PDMTS_TRY(pd->ctx->sync_checked("pd_read_damage"));
    return pd->ctx->end();
}

extern "C" int pd_read_bond_status(pdmts_pd *pd, uint8_t *mu, int64_t *n_intact)
{
    clear_error();
    if (!pd || !mu)
        return fail(PDMTS_ERR_ARG, "pd_read_bond_status: NULL argument");
    PDMTS_CUDA_TRY(cudaSetDevice(pd->ctx->device));
    PDMTS_TRY(pd->ctx->begin());
    cudaStream_t s = pd->ctx->stream;
    PDMTS_CUDA_TRY(cudaMemcpyAsync(pd->mask_host.data(), pd->d_mask.p, sizeof(uint32_t) * pd->n_mask_words,
                                   cudaMemcpyDeviceToHost, s));
    PDMTS_TRY(pd->ctx->sync_checked("pd_read_bond_status"));
    std::vector<uint8_t> st((size_t)pd->row_ptr[(size_t)pd->n]);
    int64_t intact = 0;
    for (int64_t i = 0; i < pd->n; ++i) {
        const int32_t deg_i = (int32_t)(pd->row_ptr[(size_t)i + 1] - pd->row_ptr[(size_t)i]);
        for (int32_t k = 0; k < deg_i; ++k) {
            int64_t word;
            int b;
            bond_bit(pd, i, k, word, b);
            uint8_t bit = (uint8_t)((pd->mask_host[(size_t)word] >> b) & 1u);
            st[(size_t)(pd->row_ptr[(size_t)i] + k)] = bit;
            intact += bit;
        }
    }
    PDMTS_CUDA_TRY(cudaMemcpy(mu, st.data(), st.size(), cudaMemcpyDefault));
    if (n_intact)
        *n_intact = intact;
    return pd->ctx->end();
}

extern "C" int pd_read_family(pdmts_pd *pd, int64_t *row_ptr, int32_t *col)
{
    clear_error();
    if (!pd || !row_ptr || !col)
        return fail(PDMTS_ERR_ARG, "pd_read_family: NULL argument");
    PDMTS_CUDA_TRY(cudaMemcpy(row_ptr, pd->row_ptr.data(), sizeof(int64_t) * (pd->n + 1), cudaMemcpyDefault));
    PDMTS_CUDA_TRY(cudaMemcpy(col, pd->col.data(), sizeof(int32_t) * pd->col.size(), cudaMemcpyDefault));
    return PDMTS_OK;
}

// ------------------------------------------------------ time integration --
// Velocity-Verlet critical time step of the PD model (Silling-Askari bound
// for the linearised bond model): dt <= sqrt(2 rho_i / sum_j V_j C_ij) with
// the bond stiffness C_ij = c(|xi|) |xi|^2 (Eq. 2 projected on the bond).
static double pd_dt_crit(const pdmts_pd *pd)
{
    double worst = INFINITY;
    const int64_t n = pd->n;
    for (int64_t i = 0; i < n; ++i) {
        double sum = 0.0;
        for (int64_t k = pd->row_ptr[(size_t)i]; k < pd->row_ptr[(size_t)i + 1]; ++k) {
            int64_t j = pd->col[(size_t)k];
            double xi2 = 0.0;
            for (int d = 0; d < pd->dim; ++d) {
                double e = pd->X[(size_t)d * n + j] - pd->X[(size_t)d * n + i];
                xi2 += e * e;
            }
            sum += pd->V[(size_t)j] * micromodulus_host(pd, xi2) * xi2;
        }
        if (sum > 0)
            worst = std::min(worst, std::sqrt(2.0 * pd->rho / sum));
    }
    return worst;
}

int mts_time_changed(pdmts_ctx *ctx);                          // mts.cu
int pd_run_steps_graph(pdmts_pd *pd, int64_t nsteps, int chunk, cudaStream_t s);  // pd_kernels.cu

extern "C" int mts_set_time(pdmts_ctx *ctx, double dt_pd, int m_ratio, double gamma_fe, double beta_fe,
                            int check_stability)
{
    clear_error();
    if (!ctx)
        return fail(PDMTS_ERR_ARG, "mts_set_time: ctx is NULL");
    if (!(dt_pd > 0) || !std::isfinite(dt_pd) || m_ratio < 1)
        return fail(PDMTS_ERR_ARG, "mts_set_time: need dt_pd > 0 and m_ratio >= 1");
    if (!(gamma_fe >= 0.5) || !(beta_fe >= 0.0))
        return fail(PDMTS_ERR_ARG, "mts_set_time: Newmark parameters need gamma >= 1/2, beta >= 0");
    if (check_stability && ctx->pd) {
        double dc = pd_dt_crit(ctx->pd);
        if (dt_pd > dc)
            return fail(PDMTS_ERR_STABILITY, "mts_set_time: dt_pd = %g exceeds the PD bound %g", dt_pd, dc);
    }
    if (ctx->pd && ctx->dt_pd != dt_pd) {
        ctx->pd->need_init = true;  // the prediction u + dt v + dt^2/2 a depends on dt
        pd_invalidate_graphs(ctx->pd);
    }
    ctx->dt_pd = dt_pd;
    ctx->m_ratio = m_ratio;
    ctx->gamma_fe = gamma_fe;
    ctx->beta_fe = beta_fe;
    ctx->time_set = true;
    return mts_time_changed(ctx);
}

extern int mts_advance_coupled(pdmts_ctx *ctx, int64_t n_coarse);  // mts.cu

extern "C" int mts_advance(pdmts_ctx *ctx, int64_t n_coarse)
{
    clear_error();
    if (!ctx)
        return fail(PDMTS_ERR_ARG, "mts_advance: ctx is NULL");
    if (n_coarse < 0)
        return fail(PDMTS_ERR_ARG, "mts_advance: n_coarse < 0");
    if (!ctx->pd)
        return fail(PDMTS_ERR_STATE, "mts_advance: no PD subdomain");
    if (!ctx->time_set)
        return fail(PDMTS_ERR_STATE, "mts_advance: call mts_set_time first");
    PDMTS_TRY(ctx->watch_check("mts_advance"));
    if (ctx->arl) {
        PDMTS_TRY(mts_advance_coupled(ctx, n_coarse));
        return ctx->watch_enqueue(ctx->stream);
    }
    PDMTS_CUDA_TRY(cudaSetDevice(ctx->device));
    PDMTS_TRY(ctx->begin());
    pdmts_pd *pd = ctx->pd;
    cudaStream_t s = ctx->stream;
    PDMTS_TRY(pd->tune_lattice(s));
    PDMTS_TRY(pd->ensure_init(s));
    const int64_t nsteps = n_coarse * ctx->m_ratio;
    // one coarse step of m substeps is one captured chain (m = 1: chains of 16)
    const int chunk = ctx->m_ratio >= 2 ? ctx->m_ratio : 16;
    PDMTS_TRY(pd_run_steps_graph(pd, nsteps, chunk, s));
    ctx->stats.coarse_steps += n_coarse;
    PDMTS_TRY(ctx->watch_enqueue(s));
    return ctx->end();
}
