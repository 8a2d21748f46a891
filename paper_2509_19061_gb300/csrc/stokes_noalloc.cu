// stokes_noalloc.cu -- stokes_energy_norm_noalloc: the energy-norm reduction
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a stream-ordered
// allocator's or a framework's memory budget that forbids side allocations,
// callers that hold every byte of the device for their own pools, or
// callers whose device work must not synchronise the device (which
// cudaMalloc/cudaFree may do).  Such callers cannot create a stokes_ctx, which
// allocates its buffers.  This entry point needs no context: the caller
// passes every input and the output buffer, and the reduction's only scratch
// (one partial sum per block) lives in the file-scope device array below.
#include <mutex>

#include <cudaTypedefs.h>

#include "../../include/stokes.h"
#include "internal.h"

namespace stokes {
namespace {

// One triple of partial sums per reduction block.  Every GPU that loads the
// library holds these bytes until the process exits.
constexpr int NOALLOC_PARTIALS = 152 * 4;
__device__ __align__(256) double g_noalloc_partials[NOALLOC_PARTIALS * 3];

// Largest grid the entry point accepts: element offsets of a field stay
// below 2^31 and each side is at most 46340 cells.
constexpr int NOALLOC_MAX_SIDE = 46340;

constexpr int MAX_DEVICES = 128;
std::mutex g_mu;
double *g_addr[MAX_DEVICES] = {};
unsigned long long g_ctx_id[MAX_DEVICES] = {};

// Unique id of the calling thread's current CUDA context (0 if none is
// current yet), through the driver entry points the runtime hands out.
unsigned long long current_context_id()
{
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            return 0;
        }
        get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
        get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and again only if the device's
// context was replaced since (cudaDeviceReset ends the context the address
// belonged to; the module, and with it the array, is then loaded anew).
int scratch_on_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return STOKES_ERR_CUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return STOKES_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long id = current_context_id();
    if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) return STOKES_ERR_CUDA;
        g_addr[dev] = static_cast<double *>(p);
        g_ctx_id[dev] = current_context_id(); // the lookup makes the primary context current
    }
    *out = g_addr[dev];
    return STOKES_OK;
}

} // namespace
} // namespace stokes

using namespace stokes;

extern "C" int stokes_energy_norm_noalloc(int nx, int ny, double lx, double ly, int dtype, int pitch,
                                          const void *eta_c, const void *eta_n, const void *fx, const void *fy,
                                          const void *p, const void *vx, const void *vy, double *out_dev,
                                          void *cuda_stream)
{
    if (nx < 2 || ny < 2 || nx > NOALLOC_MAX_SIDE || ny > NOALLOC_MAX_SIDE || pitch < nx + 1 ||
        (long long)(ny + 1) * (long long)pitch >= (1LL << 31) || !(lx > 0.0) || !(ly > 0.0))
        return STOKES_ERR_ARG; // grid outside the supported range (see include/stokes.h)
    if (dtype != STOKES_F32 && dtype != STOKES_F64) return STOKES_ERR_ARG;
    if (!eta_c || !eta_n || !fx || !fy || !vx || !vy || !out_dev) return STOKES_ERR_ARG;
    double *scratch = nullptr;
    int st = scratch_on_current_device(&scratch);
    if (st != STOKES_OK) return st;
    if (energy_partials() > NOALLOC_PARTIALS) return STOKES_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const double hx = lx / nx, hy = ly / ny;
    cudaError_t e;
    if (dtype == STOKES_F64)
        e = launch_energy_raw<double>(make_grid<double>(nx, ny, pitch, hx, hy), (const double *)eta_c,
                                      (const double *)eta_n, (const double *)fx, (const double *)fy,
                                      (const double *)p, (const double *)vx, (const double *)vy, scratch, out_dev, s);
    else
        e = launch_energy_raw<float>(make_grid<float>(nx, ny, pitch, hx, hy), (const float *)eta_c,
                                     (const float *)eta_n, (const float *)fx, (const float *)fy, (const float *)p,
                                     (const float *)vx, (const float *)vy, scratch, out_dev, s);
    return e == cudaSuccess ? STOKES_OK : STOKES_ERR_CUDA;
}
