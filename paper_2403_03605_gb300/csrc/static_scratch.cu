// static_scratch.cu -- damage read-back that allocates nothing.
//
// Some callers cannot let a library allocate device memory when they ask for
// results: an application whose device memory is entirely reserved by its own
// pool allocator (a cudaMalloc from the library would fail, or would take
// memory the pool counts on), or a time-critical loop in which an allocation
// is not allowed because cudaMalloc/cudaFree may synchronise the device and
// stall the work on other streams. pd_read_damage_static serves them: it runs
// the same damage kernel as pd_read_damage, but stages the per-node result in
// a file-scope device array instead of library-allocated memory, and calls no
// allocating routine (no cudaMalloc / cudaFree, no host heap).
//
// The array is part of the library's device image: every GPU that loads the
// library holds its kStaticDamageMax doubles until the process exits. All
// calls share it, and it keeps what the last call wrote; the kernel writes
// every entry it reads back, so nothing needs clearing first. Calls whose work
// overlaps on one GPU (other contexts, other host threads) race on it.
#include <atomic>

#include "pd.h"

using namespace pdmts;

namespace {

// Largest PD subdomain pd_read_damage_static serves: 2^20 nodes (8 MiB).
constexpr int64_t kStaticDamageMax = (int64_t)1 << 20;

static __device__ __align__(256) double g_damage_scratch[kStaticDamageMax];

// Device address of g_damage_scratch per device ordinal. In host code the
// array's name is only a host-side stand-in, never a device address, so the
// address is taken once per device with that device current.
constexpr int kMaxDevices = 64;
std::atomic<double *> g_scratch_addr[kMaxDevices];

int scratch_address(int device, double **out)
{
    if (device < 0 || device >= kMaxDevices)
        return fail(PDMTS_ERR_UNSUPPORTED, "pd_read_damage_static: device ordinal %d above %d", device,
                    kMaxDevices - 1);
    double *p = g_scratch_addr[device].load(std::memory_order_acquire);
    if (!p) {
        void *addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_damage_scratch);
        if (e != cudaSuccess || !addr)
            return fail(PDMTS_ERR_CUDA, "pd_read_damage_static: cudaGetSymbolAddress failed: %s",
                        cudaGetErrorString(e));
        p = static_cast<double *>(addr);
        g_scratch_addr[device].store(p, std::memory_order_release);
    }
    *out = p;
    return PDMTS_OK;
}

}  // namespace

extern "C" int pd_read_damage_static(pdmts_pd *pd, double *phi)
{
    clear_error();
    if (!pd || !phi)
        return fail(PDMTS_ERR_ARG, "pd_read_damage_static: NULL argument");
    if (pd->n > kStaticDamageMax)
        return fail(PDMTS_ERR_UNSUPPORTED,
                    "pd_read_damage_static: %lld nodes exceed the static scratch of %lld nodes; use pd_read_damage",
                    (long long)pd->n, (long long)kStaticDamageMax);
    PDMTS_CUDA_TRY(cudaSetDevice(pd->ctx->device));
    double *scratch = nullptr;
    PDMTS_TRY(scratch_address(pd->ctx->device, &scratch));
    PDMTS_TRY(pd->ctx->begin());
    cudaStream_t s = pd->ctx->stream;
    // The kernel writes every entry [0, n) of the scratch, so nothing left by
    // an earlier call needs clearing.
    SellView fam{pd->d_tile_ptr.p, pd->d_tile_k.p, pd->d_mask_ptr.p, pd->d_col.p, pd->d_mask.p, pd->d_deg.p,
                 pd->n, pd->ntiles};
    cudaError_t e = pd->layout != pdmts_pd::LAYOUT_SELL
                        ? launch_damage_lattice(pd->n, pd->d_mask.p, pd->d_exists.p,
                                                pd->layout == pdmts_pd::LAYOUT_LATTICE3D ? lat3d::W : 1, scratch, s)
                        : launch_damage(fam, pd->precision == PDMTS_FP32_BULK, pd->d_V.p, scratch, s);
    if (e != cudaSuccess)
        return fail(PDMTS_ERR_CUDA, "pd_read_damage_static: damage kernel failed: %s", cudaGetErrorString(e));
    pd->ctx->stats.kernel_launches++;
    PDMTS_CUDA_TRY(cudaMemcpyAsync(phi, scratch, sizeof(double) * pd->n, cudaMemcpyDefault, s));
    PDMTS_CUDA_TRY(cudaStreamSynchronize(s));
    return pd->ctx->end();
}
