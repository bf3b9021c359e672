// noalloc.cu -- pic_field_solve_noalloc: the right-hand side of Eq. (7) and its PCG solve
// for callers that must not allocate device memory.
//
// Its working vectors (residual, direction, A-product), reduction partials, solver state
// and status words live in one file-scope device array of fixed size, so a call performs
// no cudaMalloc, cudaFree or other allocating call: only asynchronous copies and sets on
// that array, kernel launches and a synchronisation of the caller's stream. It runs the
// same kernels as the solve inside pic_step.
#include <cuda_runtime.h>

#include <mutex>

#include "engine.h"
#include "pic.h"

namespace pic {
namespace {

constexpr long long kNaMaxCells = PIC_NOALLOC_MAX_CELLS;
constexpr int kNaMaxBlocks = (int)((kNaMaxCells + kFieldThreads - 1) / kFieldThreads);

constexpr size_t up256(size_t b) { return (b + 255) / 256 * 256; }
// layout of the scratch array (byte offsets)
constexpr size_t kOffR = 0;
constexpr size_t kVec = up256(3 * kNaMaxCells * sizeof(double));
constexpr size_t kOffP = kOffR + kVec;
constexpr size_t kOffQ = kOffP + kVec;
constexpr size_t kOffPart = kOffQ + kVec;
constexpr size_t kOffGrid = kOffPart + up256(4 * (size_t)kNaMaxBlocks * sizeof(double));
constexpr size_t kOffCg = kOffGrid + up256(sizeof(GridDev));
constexpr size_t kOffDone = kOffCg + up256(sizeof(CgState));
constexpr size_t kOffSt = kOffDone + up256(sizeof(unsigned int));
constexpr size_t kOffBlk = kOffSt + up256(sizeof(DevStatus));
constexpr size_t kScratchBytes = kOffBlk + up256((size_t)kNaMaxBlocks * sizeof(int));

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_addr[kMaxDevices] = {nullptr};

void set_err(char* buf, size_t len, const char* msg) {
    if (!buf || len == 0) return;
    size_t i = 0;
    for (; msg[i] && i + 1 < len; i++) buf[i] = msg[i];
    buf[i] = '\0';
}

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" PIC_API int pic_field_solve_noalloc(int32_t nx, int32_t ny, double dx, double dy,
                                               double cfl, double theta, double cg_rtol,
                                               int32_t cg_max_iter, const double* F,
                                               const double* J, double* dB, int32_t* iters,
                                               double* rel_resid, void* stream, char* errbuf,
                                               size_t errlen) {
    if (nx < 8 || ny < 8 || (long long)nx * ny > kNaMaxCells) {
        set_err(errbuf, errlen, "nx, ny must be >= 8 with nx*ny <= PIC_NOALLOC_MAX_CELLS");
        return PIC_EINVAL;
    }
    if (!(dx > 0) || !(dy > 0) || !(cfl > 0) || cfl > 1.0 || cfl * dx > dy * (1.0 + 1e-12) ||
        !(theta >= 0.5) || theta > 1.0 || !(cg_rtol > 0) || cg_rtol >= 1 || cg_max_iter < 1) {
        set_err(errbuf, errlen, "invalid dx, dy, cfl, theta, cg_rtol or cg_max_iter");
        return PIC_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_err(errbuf, errlen, "no usable CUDA device");
        return PIC_ECUDA;
    }
    // device memory of the current device, or managed memory; memory of another GPU
    // would be read across the interconnect (or fault without peer access)
    const void* ptrs[3] = {F, J, dB};
    for (const void* q : ptrs) {
        cudaPointerAttributes at{};
        const bool ok = q && cudaPointerGetAttributes(&at, q) == cudaSuccess &&
                        (at.type == cudaMemoryTypeManaged ||
                         (at.type == cudaMemoryTypeDevice && at.device == dev));
        if (!ok) {
            cudaGetLastError();
            set_err(errbuf, errlen, "F, J and dB must be device memory of the current device (or managed)");
            return PIC_EINVAL;
        }
    }
    unsigned char* base = nullptr;
    {
        // one-time set-up on this device: the device address of the scratch array
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                set_err(errbuf, errlen, "cudaGetSymbolAddress of the solver scratch failed");
                return PIC_ECUDA;
            }
            g_addr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long N = (long long)nx * ny;
    GridDev G{};
    G.nx = nx;
    G.ny = ny;
    G.order = 1;
    G.ncell = (int)N;
    G.dx = dx;
    G.dy = dy;
    G.dt = cfl * dx;
    G.theta = theta;
    G.idx = 1.0 / dx;
    G.idy = 1.0 / dy;
    G.a = (theta * G.dt) * (theta * G.dt);
    G.cx = G.a / (dx * dx);
    G.cy = G.a / (dy * dy);
    G.c0 = 1.0 + 2.0 * G.cx + 2.0 * G.cy;
    G.cell_off = 0;
    G.blk_first = 0;
    G.nblk = (int)((N + kFieldThreads - 1) / kFieldThreads);
    G.rtol = cg_rtol;
    G.maxit = cg_max_iter;
    G.warm = 0;
    FieldArgs a{};
    a.grids = reinterpret_cast<const GridDev*>(base + kOffGrid);
    a.blk_grid = reinterpret_cast<const int*>(base + kOffBlk);
    a.ngrids = 1;
    a.nblk = G.nblk;
    a.ntot = N;
    a.F = const_cast<double*>(F);  // read only by the rhs and PCG kernels
    a.J64 = J;
    a.x = dB;
    a.r = reinterpret_cast<double*>(base + kOffR);
    a.p = reinterpret_cast<double*>(base + kOffP);
    a.q = reinterpret_cast<double*>(base + kOffQ);
    a.part = reinterpret_cast<double*>(base + kOffPart);
    a.cg = reinterpret_cast<CgState*>(base + kOffCg);
    a.done = reinterpret_cast<unsigned int*>(base + kOffDone);
    a.st = reinterpret_cast<DevStatus*>(base + kOffSt);
    a.use_cond = 0;
    // the array keeps the previous call's contents: clear what must start at zero
    cudaError_t e = cudaMemcpyAsync(base + kOffGrid, &G, sizeof G, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffBlk, 0, (size_t)G.nblk * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffCg, 0, sizeof(CgState), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffDone, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffSt, 0, sizeof(DevStatus), s);
    if (e != cudaSuccess) {
        set_err(errbuf, errlen, cudaGetErrorString(e));
        return PIC_ECUDA;
    }
    launch_rhs(a, s);
    // PCG iterations in batches; kernels of a converged solve return at once
    unsigned int n_active = 1;
    int launched = 0;
    while (n_active && launched < cg_max_iter) {
        const int batch = (cg_max_iter - launched) < 4 ? (cg_max_iter - launched) : 4;
        for (int k = 0; k < batch; k++) launch_cg_iteration(a, s);
        launched += batch;
        e = cudaMemcpyAsync(&n_active, &a.st->n_active, sizeof n_active, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_err(errbuf, errlen, cudaGetErrorString(e));
            return PIC_ECUDA;
        }
    }
    CgState c{};
    DevStatus st{};
    e = cudaMemcpyAsync(&c, a.cg, sizeof c, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, a.st, sizeof st, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_err(errbuf, errlen, cudaGetErrorString(e));
        return PIC_ECUDA;
    }
    if (iters) *iters = c.iters;
    if (rel_resid) *rel_resid = c.rel;
    if (st.cg_noconv || c.active) {
        set_err(errbuf, errlen, "PCG reached cg_max_iter before cg_rtol");
        return PIC_ECG_NOCONV;
    }
    set_err(errbuf, errlen, "");
    return PIC_OK;
}
