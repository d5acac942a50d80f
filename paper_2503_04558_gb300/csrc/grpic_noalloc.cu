// grpic_noalloc.cu -- the particle sort by cell without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a CUDA stream
// capture that must not see allocation calls, host frameworks whose memory
// pools own every device allocation (the process may not grow the pool on its
// own), and embedded or plugin hosts that forbid the library from allocating
// on the device at all.  grpic_sort_noalloc serves them: it runs the same
// kernels as grpic_sort but takes its scratch (keys, histogram, offsets,
// cursors, index list) from one file-scope __device__ array of fixed size
// instead of a context.  Every GPU that loads the library holds that array
// (about 20 MB) until the process exits.
#include "grpic_internal.cuh"

#include <cuda.h>  // driver types only (the two driver calls are looked up at run time)

#include <cmath>
#include <cstring>
#include <mutex>
#include <utility>

namespace grpic {
namespace {

constexpr int64_t NA_MAX_P = GRPIC_NOALLOC_MAX_PARTICLES;
constexpr int64_t NA_MAX_C = GRPIC_NOALLOC_MAX_CELLS;

struct NoAllocScratch {
    int32_t keys[NA_MAX_P];
    int32_t perm[NA_MAX_P];
    int32_t count[NA_MAX_C + 2];
    int32_t offset[NA_MAX_C + 3];
    int32_t cursor[NA_MAX_C + 3];
    int32_t blocksum[8192];
    int32_t bigseg[NA_MAX_C + 1];
    int32_t status[16];
};

// The scratch itself.  In host code this name is only a stand-in for the
// device object: its device address is obtained with cudaGetSymbolAddress.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;

// The set-up is per CUDA context: after cudaDeviceReset (or when the caller
// makes another context current) the module is loaded again, the array may
// sit at another address and kernel attributes are unset.  Entries are keyed
// on (device, context id); the id comes from the driver's cuCtxGetId, reached
// through the runtime's entry-point lookup so that the library needs no link
// against the driver library.
struct SetupEntry {
    int dev;
    unsigned long long ctx;
    NoAllocScratch *ptr;
};
constexpr int MAX_ENTRIES = 64;
SetupEntry g_entries[MAX_ENTRIES];
int g_nentries = 0, g_next = 0;

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;
bool g_looked_up = false;

// id of the current context, 0 if none is current yet (caller holds the mutex)
unsigned long long current_context_id()
{
    if (!g_looked_up) {
        g_looked_up = true;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void **)&g_get_current, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess || q != cudaDriverEntryPointSuccess)
            g_get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void **)&g_get_id, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess)
            g_get_id = nullptr;
    }
    CUcontext c = nullptr;
    if (!g_get_current || g_get_current(&c) != CUDA_SUCCESS || !c) return 0;
    unsigned long long id = 0;
    if (!g_get_id || g_get_id(c, &id) != CUDA_SUCCESS) return (unsigned long long)(uintptr_t)c;
    return id;
}

// Once per device and context, with that device current: the device address
// of the scratch array and the kernel attribute the sort's large-segment pass
// needs.
cudaError_t setup_device(int dev, NoAllocScratch **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long ctx = current_context_id();
    if (ctx != 0) {
        for (int k = 0; k < g_nentries; ++k)
            if (g_entries[k].dev == dev && g_entries[k].ctx == ctx) {
                *out = g_entries[k].ptr;
                return cudaSuccess;
            }
    }
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);  // also makes the runtime's context current
    if (e != cudaSuccess) return e;
    e = sort_setup();
    if (e != cudaSuccess) return e;
    if (ctx == 0) ctx = current_context_id();
    SetupEntry ent{dev, ctx, (NoAllocScratch *)ptr};
    if (g_nentries < MAX_ENTRIES) {
        g_entries[g_nentries++] = ent;
    } else {
        g_entries[g_next] = ent;
        g_next = (g_next + 1) % MAX_ENTRIES;
    }
    *out = ent.ptr;
    return cudaSuccess;
}

}  // namespace
}  // namespace grpic

extern "C" grpic_status grpic_sort_noalloc(const grpic_grid *grid, int32_t precision, grpic_particles *p,
                                           grpic_particles *scratch, void *stream)
{
    using namespace grpic;
    if (!grid || !p || !scratch || (precision != 64 && precision != 32)) return GRPIC_EINVAL;
    if (grid->n_r < 4 || grid->n_theta < 4 || !(grid->r_in > 0.0 && grid->r_out > grid->r_in)) return GRPIC_EINVAL;
    if (p->n < 0 || p->capacity < p->n || scratch->capacity < p->n) return GRPIC_EINVAL;
    if (p->n > 0 && (!p->x1 || !p->x2 || !p->u1 || !p->u2 || !p->u3 || !p->tag || !scratch->x1 || !scratch->x2 ||
                     !scratch->u1 || !scratch->u2 || !scratch->u3 || !scratch->tag))
        return GRPIC_EINVAL;
    if (precision == 32 && p->n > 0 && (!p->cell || !scratch->cell)) return GRPIC_EINVAL;
    int64_t ncell = (int64_t)grid->n_r * grid->n_theta;
    // sizes beyond the fixed scratch are refused before anything is launched
    if (p->n > NA_MAX_P || ncell > NA_MAX_C) return GRPIC_EOVERFLOW;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return GRPIC_ECUDA;
    NoAllocScratch *sc = nullptr;
    if (setup_device(dev, &sc) != cudaSuccess) return GRPIC_ECUDA;

    // a context on the stack that points into the fixed scratch (no allocation)
    grpic_ctx ctx;
    memset((void *)&ctx, 0, sizeof ctx);
    ctx.device = dev;
    ctx.grid = *grid;
    ctx.prm.precision = precision;
    GridDev &g = ctx.g;
    g.nr = grid->n_r;
    g.nth = grid->n_theta;
    g.ld_tab = grid->n_r + 2 * NG;
    g.r_in = grid->r_in;
    g.r_out = grid->r_out;
    g.dx1 = std::log(grid->r_out / grid->r_in) / grid->n_r;
    g.dth = M_PI / grid->n_theta;
    g.ln_rin = std::log(grid->r_in);
    ctx.d_keys = sc->keys;
    ctx.d_perm = sc->perm;
    ctx.d_count = sc->count;
    ctx.d_offset = sc->offset;
    ctx.d_cursor = sc->cursor;
    ctx.d_blocksum = sc->blocksum;
    ctx.d_bigseg = sc->bigseg;
    ctx.d_status = sc->status;
    ctx.keys_cap = NA_MAX_P;
    ctx.perm_cap = NA_MAX_P;

    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear the histogram
    if (cudaMemsetAsync(sc->count, 0, sizeof(int32_t) * (ncell + 1), s) != cudaSuccess) return GRPIC_ECUDA;
    if (launch_keys(&ctx, p, s) != cudaSuccess) return GRPIC_ECUDA;
    if (launch_sort(&ctx, p, scratch, s) != cudaSuccess) return GRPIC_ECUDA;
    std::swap(p->x1, scratch->x1);
    std::swap(p->x2, scratch->x2);
    std::swap(p->u1, scratch->u1);
    std::swap(p->u2, scratch->u2);
    std::swap(p->u3, scratch->u3);
    std::swap(p->tag, scratch->tag);
    std::swap(p->cell, scratch->cell);
    return GRPIC_OK;
}
