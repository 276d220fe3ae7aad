// An allocation-free variant of the one-launch coarse PCG (no counterpart in the paper).
//
// Some callers cannot call cudaMalloc: code that runs where the CUDA allocator must not be
// touched (inside a real-time control loop with a fixed memory budget, a plug-in of a host
// program that owns every device allocation, or a process that hands this library only
// the buffers it will read and write).  cgp_pcg_sell_noalloc solves A x = b with the same
// Jacobi-preconditioned Chronopoulos-Gear PCG as the coarse Poisson solve, but keeps all of
// its scratch (the grid-barrier counter, per-CTA partial sums, the solver state and eight
// work vectors) in one file-scope __device__ array of fixed size, so the call allocates
// nothing: the caller passes only the operator, the right-hand side, the solution buffer
// and a two-int status buffer.
#include <mutex>

#include "coarse_pcg.cuh"

namespace cgp {

// Largest system the scratch array can hold, and its layout (offsets in doubles).
constexpr int kNoAllocMaxRows = 65536;
constexpr int kNoAllocMaxCtas = 2048;
constexpr size_t kNaState = 0;                                            // KrylovState (padded to 32 doubles)
constexpr size_t kNaCount = 32;                                           // barrier counter + error word
constexpr size_t kNaPartials = 64;                                        // 2 x kNoAllocMaxCtas x 4
constexpr size_t kNaWork = kNaPartials + 2 * (size_t)kNoAllocMaxCtas * 4; // 8 x kNoAllocMaxRows
constexpr size_t kNaDoubles = kNaWork + 8 * (size_t)kNoAllocMaxRows;

// Shared by every call on a device, and kept until the process exits (about 4.3 MB).
static __device__ __align__(256) double g_noalloc_scratch[kNaDoubles];

static_assert(sizeof(KrylovState) <= 32 * sizeof(double), "state slot too small");

__global__ void k_noalloc_status(const KrylovState* st, int32_t* info) {
    info[0] = st->iter;
    info[1] = st->status;
}

}  // namespace cgp

using namespace cgp;

namespace {
constexpr int kMaxDevices = 64;
// Per device: the context the address was looked up in, the array's device address there,
// and the launch size.  A symbol's address belongs to a context, so a new primary context
// (after cudaDeviceReset) is looked up again.  The mutex orders first calls from several
// host threads.
struct NoAllocSlot {
    void* ctx;
    double* ptr;
    int grid;
};
NoAllocSlot g_slot[kMaxDevices] = {};
std::mutex g_slot_mu;
typedef int (*CtxGetCurrentFn)(void**);   // the driver's cuCtxGetCurrent, reached through the runtime

// The calling thread's current context on `dev` (made current by cudaSetDevice, which
// initialises the device's primary context), or nullptr where the driver does not give it.
void* current_context(int dev) {
    static CtxGetCurrentFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)f;
        looked = true;
    }
    if (cudaSetDevice(dev) != cudaSuccess || !fn) return nullptr;
    void* ctx = nullptr;
    return fn(&ctx) == 0 ? ctx : nullptr;
}
}  // namespace

extern "C" int cgp_pcg_sell_noalloc(int32_t n, int32_t nslices, const int32_t* sell_ptr, const int32_t* sell_col,
                                    const double* val, const double* dinv, const double* b, double* x, double tol,
                                    int32_t maxit, int32_t* info, cgp_stream_t stream) {
    clear_error();
    if (n < 1 || nslices != (n + 31) / 32 || !sell_ptr || !sell_col || !val || !dinv || !b || !x || !info ||
        !(tol > 0) || maxit < 1) {
        set_error("cgp_pcg_sell_noalloc: bad arguments");
        return CGP_EINVAL;
    }
    if (n > kNoAllocMaxRows) {
        set_error("cgp_pcg_sell_noalloc: %d rows exceed the fixed scratch of %d rows", n, kNoAllocMaxRows);
        return CGP_EINVAL;
    }
    int dev = 0;
    CGP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("cgp_pcg_sell_noalloc: device index %d out of range", dev);
        return CGP_EINVAL;
    }
    double* base = nullptr;
    int max_grid = 0;
    {
        std::lock_guard<std::mutex> lock(g_slot_mu);
        NoAllocSlot& sl = g_slot[dev];
        void* ctx = current_context(dev);
        if (!sl.ptr || ctx != sl.ctx) {
            // first call on this device (or in a new context of it): the device address of
            // the scratch array, and the number of co-resident CTAs of the cooperative launch
            void* p = nullptr;
            CGP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            int sms = 0, per_sm = 0, coop = 0;
            CGP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            CGP_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
            CGP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_grid, kGridThreads, 0));
            if (!coop || per_sm < 1) {
                set_error("cgp_pcg_sell_noalloc: cooperative launch unavailable");
                return CGP_EINVAL;
            }
            const int g = sms * (per_sm < 2 ? per_sm : 2);
            sl.grid = g < kNoAllocMaxCtas ? g : kNoAllocMaxCtas;
            sl.ptr = (double*)p;
            sl.ctx = ctx;
        }
        base = sl.ptr;
        max_grid = sl.grid;
    }
    int grid = (nslices + kGridThreads / 32 - 1) / (kGridThreads / 32);
    if (grid > max_grid) grid = max_grid;
    if (grid < 1) grid = 1;
    cudaStream_t st = (cudaStream_t)stream;
    CoarsePcgArgs a = {};
    a.A = SellView{n, nslices, sell_ptr, sell_col};
    a.val = val;
    a.valf = nullptr;
    a.dinv = dinv;
    a.dinvf = nullptr;
    a.b = const_cast<double*>(b);   // read only: no projection is asked for
    a.x = x;
    a.x_alt = nullptr;
    a.w64 = base + kNaWork;
    a.w32 = nullptr;
    a.mlump = nullptr;
    a.st = reinterpret_cast<KrylovState*>(base + kNaState);
    a.tol2 = tol * tol;
    a.inner_tol = 0.0;
    a.maxit = maxit;
    a.zero_x = 0;
    a.project = 0;
    a.mixed = 0;
    a.max_outer = 50;
    a.bar_count = reinterpret_cast<unsigned int*>(base + kNaCount);
    a.bar_err = reinterpret_cast<int*>(base + kNaCount) + 1;
    a.partials = base + kNaPartials;
    // the barrier counter and its error word must start at zero on every call
    CGP_CUDA(cudaMemsetAsync(base + kNaCount, 0, 2 * sizeof(unsigned int), st));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(kGridThreads, 1, 1);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CGP_CUDA(cudaLaunchKernelEx(&cfg, k_pcg_grid, a));
    k_noalloc_status<<<1, 1, 0, st>>>(a.st, info);
    CGP_LAUNCH_CHECK();
    return CGP_OK;
}
