// noalloc.cu -- charge density of caller-provided particles with no device
// allocation at all, for callers that cannot allocate device memory.
//
// The regular path (pic_read_fields with PIC_RHO) accumulates the charge in
// an FP64 scratch grid that the library allocates with the handle.  This
// variant keeps that scratch in a file-scope static device array of fixed
// size instead, so a caller that owns no allocator (a host framework that
// hands the library only its own buffers, code running under a memory
// budget that forbids new allocations, or a loop that must not allocate
// once it is running) can still get the charge density.  Every GPU that
// loads the library holds the array until the process exits.
#include <cstdint>
#include <cstring>
#include <mutex>

#include "pic.h"
#include "common.cuh"
#include "internal.h"

namespace pic {
namespace {

// Largest grid (cells) the static scratch can hold: 2^21 cells = 16 MiB of FP64.
constexpr long long kStaticMaxCells = 1ll << 21;
static_assert(kStaticMaxCells == PIC_STATIC_MAX_CELLS, "header and implementation disagree");

__device__ __align__(256) double g_rho_scratch[kStaticMaxCells];

// Device address of g_rho_scratch per device.  In host code the symbol is
// only a stand-in, so the address is looked up with cudaGetSymbolAddress
// with that device current.  The lookup is cached together with the unique
// id of the context it was made in: after cudaDeviceReset the module is
// loaded again into a new context, the id changes and the address is looked
// up again instead of reusing a stale one.  A mutex guards the cache, so
// host threads may call concurrently (their kernels still share the array).
constexpr int kMaxDevices = 64;
struct ScratchSlot {
    unsigned long long ctx_id;  // 0: not looked up
    double *ptr;
};
ScratchSlot g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Unique id of the calling thread's current context (cuCtxGetId through the
// runtime's driver entry point, so the library does not link libcuda), or 0
// when there is none or the driver lacks the call.
unsigned long long current_context_id()
{
    using GetIdFn = int (*)(void *ctx, unsigned long long *id);
    static GetIdFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<GetIdFn>(f);
    }();
    unsigned long long id = 0;
    if (!fn || fn(nullptr, &id) != 0) return 0;
    return id;
}

// Device address of the scratch array on device `dev` (current), or null.
double *scratch_address(int dev)
{
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchSlot &slot = g_scratch[dev];
    const unsigned long long id = current_context_id();
    if (slot.ptr && id != 0 && slot.ctx_id == id) return slot.ptr;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_rho_scratch) != cudaSuccess || !p) return nullptr;
    // (the lookup creates the context if there was none yet: take its id now)
    slot.ctx_id = current_context_id();
    slot.ptr = static_cast<double *>(p);
    return slot.ptr;
}

struct GridArgs {
    int n[3];
    int ncell;
};

__global__ void zero_kernel(double *s, int ncell)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) s[i] = 0.0;
}

template <int DIM, int P>
__global__ void charge_static_kernel(GridArgs g, double q, double w_const, long long n,
                                     const int32_t *__restrict__ cell, const float *__restrict__ off,
                                     const float *__restrict__ w, double *__restrict__ s)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int base[3] = {0, 0, 0};
    float wt[3][P + 1] = {};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const int c = cell[(long long)a * n + i];
        Shape<P>::node(c, off[(long long)a * n + i], base[a], wt[a]);
    }
    const double qw = q * (w ? (double)w[i] : w_const);
#pragma unroll
    for (int qz = 0; qz < (DIM == 3 ? P + 1 : 1); ++qz)
#pragma unroll
        for (int qy = 0; qy <= P; ++qy)
#pragma unroll
            for (int qx = 0; qx <= P; ++qx) {
                const double v = qw * (double)wt[0][qx] * (double)wt[1][qy] * (DIM == 3 ? (double)wt[2][qz] : 1.0);
                const int x = modi(base[0] + qx, g.n[0]), y = modi(base[1] + qy, g.n[1]);
                const int z = DIM == 3 ? modi(base[2] + qz, g.n[2]) : 0;
                atomicAdd(s + x + g.n[0] * (y + g.n[1] * z), v);
            }
}

__global__ void store_kernel(const double *s, float *rho, int ncell)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x)
        rho[i] = (float)s[i];
}

template <int DIM>
cudaError_t launch_charge_static(int order, GridArgs g, double q, double w_const, long long n, const int32_t *cell,
                                 const float *off, const float *w, double *s, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + kBlock - 1) / kBlock);
    if (order == 1) charge_static_kernel<DIM, 1><<<blocks, kBlock, 0, st>>>(g, q, w_const, n, cell, off, w, s);
    else if (order == 2) charge_static_kernel<DIM, 2><<<blocks, kBlock, 0, st>>>(g, q, w_const, n, cell, off, w, s);
    else if (order == 3) charge_static_kernel<DIM, 3><<<blocks, kBlock, 0, st>>>(g, q, w_const, n, cell, off, w, s);
    else charge_static_kernel<DIM, 4><<<blocks, kBlock, 0, st>>>(g, q, w_const, n, cell, off, w, s);
    return cudaGetLastError();
}

}  // namespace
}  // namespace pic

extern "C" int pic_charge_density_static(const pic_grid *grid, int32_t shape_order, double q, double w_const,
                                         int64_t n, const int32_t *cell, const float *off, const float *w,
                                         float *rho, void *stream)
{
    using namespace pic;
    if (!grid || (grid->dim != 2 && grid->dim != 3) || shape_order < 1 || shape_order > 4 || n < 0 || !rho)
        return PIC_EINVAL;
    if (n > 0 && (!cell || !off)) return PIC_EINVAL;
    long long ncell = 1;
    GridArgs g{{1, 1, 1}, 1};
    for (int a = 0; a < grid->dim; ++a) {
        if (grid->n[a] < 1) return PIC_EINVAL;
        // the static scratch holds PIC_STATIC_MAX_CELLS cells; checked per
        // axis before multiplying, so the product cannot overflow
        if (grid->n[a] > kStaticMaxCells / ncell) return PIC_EINVAL;
        g.n[a] = grid->n[a];
        ncell *= grid->n[a];
    }
    g.ncell = (int)ncell;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIC_ECUDA;
    // first call on a device (or in a new context of it): look up the array's device address
    double *s = scratch_address(dev);
    if (!s) return PIC_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned zb = (unsigned)((ncell + kBlock - 1) / kBlock < 4096 ? (ncell + kBlock - 1) / kBlock : 4096);
    zero_kernel<<<zb, kBlock, 0, st>>>(s, g.ncell);  // the array keeps the previous call's sums
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = grid->dim == 3 ? launch_charge_static<3>(shape_order, g, q, w_const, n, cell, off, w, s, st)
                           : launch_charge_static<2>(shape_order, g, q, w_const, n, cell, off, w, s, st);
    if (e == cudaSuccess) {
        store_kernel<<<zb, kBlock, 0, st>>>(s, rho, g.ncell);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
