// sht_forward_noalloc: the forward transform with its scratch in a fixed device array.
//
// sht_forward keeps its scratch (the order-major bins W, the solved orders F and the split-K
// partial sums) in workspaces that the plan allocates on first use.  Some callers cannot let a
// call allocate device memory: code that owns a fixed memory budget handed to it by a host
// application, or that runs where cudaMalloc is not allowed (for example while other work is being
// captured into a CUDA graph, or under an allocator that must not be bypassed).  For them this
// entry point takes the same scratch from one file-scope __device__ array instead, so a call
// allocates nothing (the plan itself, created beforehand, still holds its tables).
//
// The array is kNoAllocScratchBytes (64 MiB) on every GPU that loads the library, kept until the
// process exits.  Every call on a device shares it and leaves its contents behind; nothing in it
// needs to start at zero, because each call writes every element it later reads.  Calls whose
// GPU work overlaps in time (different streams, or different plans on one device) race on it.
//
// Host code cannot pass the array's name to a kernel (in host code the name is a host-side
// stand-in, not a device address), so the first call in each CUDA context, with that context
// current, looks up the device address with cudaGetSymbolAddress and caches it together with the
// context's unique id.  A later call in another context of the same device (after
// cudaDeviceReset, or after the primary context was released and created again) sees a different
// id and looks the address up again, so no call uses an address of a destroyed context.  The first
// call in a context should therefore come before any stream capture.
//
// Whatever the plan's arithmetic (SHT_F64, SHT_F64_TENSOR or a refined form), this call runs the
// float64 SIMT order chain on the plan's float64 tables: float64-accurate like sht_forward, but not
// bit-identical to the tensor-core chain or to a refined forward.
#include <cuda.h>

#include <mutex>

#include "sht_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct ScratchSlot {
    unsigned long long ctx_id = 0;   // unique id of the context the address belongs to
    void *ptr = nullptr;
};

std::mutex g_scratch_mutex;
ScratchSlot g_scratch[kMaxDevices];

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the current context (driver entry points reached through the runtime, so the
// library needs no link against the driver library).  A device whose primary context is not yet
// current is made current by cudaSetDevice, which creates that context.
sht_status current_context_id(int dev, unsigned long long *id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return sht::cuda_check(e, "sht_forward_noalloc: driver entry points");
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return sht::set_error(SHT_ERR_CUDA, "sht_forward_noalloc: cuCtxGetCurrent / cuCtxGetId not found");
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS)
        return sht::set_error(SHT_ERR_CUDA, "sht_forward_noalloc: cuCtxGetCurrent failed");
    if (!ctx) {
        cudaError_t e = cudaSetDevice(dev);
        if (e != cudaSuccess) return sht::cuda_check(e, "sht_forward_noalloc: cudaSetDevice");
        if (get_current(&ctx) != CUDA_SUCCESS || !ctx)
            return sht::set_error(SHT_ERR_CUDA, "sht_forward_noalloc: no current context");
    }
    if (get_id(ctx, id) != CUDA_SUCCESS)
        return sht::set_error(SHT_ERR_CUDA, "sht_forward_noalloc: cuCtxGetId failed");
    return SHT_OK;
}

// Device address of the scratch array in the current context (looked up once per context).
sht_status scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices)
        return sht::set_error(SHT_ERR_UNSUPPORTED, "sht_forward_noalloc: device ordinal above 63");
    unsigned long long id = 0;
    sht_status st = current_context_id(dev, &id);
    if (st != SHT_OK) return st;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchSlot &slot = g_scratch[dev];
    if (!slot.ptr || slot.ctx_id != id) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return sht::cuda_check(e, "sht_forward_noalloc: cudaGetSymbolAddress");
        slot.ptr = p;
        slot.ctx_id = id;
    }
    *out = slot.ptr;
    return SHT_OK;
}

}  // namespace

extern "C" sht_status sht_forward_noalloc(sht_plan_t p, const void *d_samples, void *d_coeffs,
                                          int64_t batch, void *stream) {
    using namespace sht;
    sht_status st = check_io(p, d_samples, d_coeffs, batch);
    if (st != SHT_OK) return st;
    if (p->dtype == SHT_F32)
        return set_error(SHT_ERR_UNSUPPORTED, "sht_forward_noalloc: complex128 plans only (not SHT_F32)");
    if (p->spin != 0) return set_error(SHT_ERR_UNSUPPORTED, "sht_forward_noalloc: scalar (spin-0) plans only");
    if (batch == 0) return SHT_OK;
    const int L = p->L;

    // scratch: bins W and solved orders F (rows_total(L) x 4B doubles each), split-K partials
    const int64_t Nc = 4 * batch;
    const size_t wf = round256(sizeof(double) * (size_t)rows_total(L) * (size_t)Nc);
    const size_t part = round256(sizeof(double) * (size_t)kSplitCap * L * (size_t)Nc);
    if (2 * wf + part > kNoAllocScratchBytes)
        return set_error(SHT_ERR_UNSUPPORTED,
                         "sht_forward_noalloc: L and batch need " + std::to_string(2 * wf + part) +
                             " bytes of scratch; the fixed array holds " +
                             std::to_string(kNoAllocScratchBytes) + " (use sht_forward)");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
    void *base = nullptr;
    st = scratch_address(dev, &base);
    if (st != SHT_OK) return st;
    double *W = (double *)base;
    double *F = (double *)((char *)base + wf);
    double *P = (double *)((char *)base + 2 * wf);

    cudaStream_t s = (cudaStream_t)stream;
    e = ring_dft_to_bins(L, p->dft, (const double2 *)d_samples, W, batch, true, s);
    GemmArgs ga{};
    ga.L = L; ga.batch = batch; ga.coeffs = (double2 *)d_coeffs; ga.W = W;
    ga.part = P; ga.part_cap = (int64_t)kSplitCap * L * Nc;
    for (int m = L - 1; m >= 0 && e == cudaSuccess; --m) {
        const int n = L - m;
        ga.m = m;
        e = gemm_f64(false, n, n, (int)Nc, p->pinv + pinv_off(L, m), n, W + rows_off(L, m) * Nc, Nc,
                     F + rows_off(L, m) * Nc, Nc, EPI_SOLVE, ga, s);
        if (m > 0 && e == cudaSuccess)
            e = gemm_f64(false, m, n, (int)Nc, p->pt + pt_off(L, m), n, F + rows_off(L, m) * Nc, Nc,
                         nullptr, Nc, EPI_ALIAS, ga, s);
    }
    return cuda_check(e, "sht_forward_noalloc");
}
