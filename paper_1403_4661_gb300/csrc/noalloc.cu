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
// stand-in, not a device address), so the first call on each device, with that device current,
// looks up the device address with cudaGetSymbolAddress and caches it.  That first call should
// therefore come before any stream capture.
#include <mutex>

#include "sht_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (looked up once per device).
sht_status scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices)
        return sht::set_error(SHT_ERR_UNSUPPORTED, "sht_forward_noalloc: device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return sht::cuda_check(e, "sht_forward_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return SHT_OK;
}

}  // namespace

extern "C" sht_status sht_forward_noalloc(sht_plan_t p, const void *d_samples, void *d_coeffs,
                                          int64_t batch, void *stream) {
    using namespace sht;
    if (!p) return set_error(SHT_ERR_INVALID_ARG, "plan is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
    if (dev != p->device) return set_error(SHT_ERR_INVALID_ARG, "current device is not the plan's device");
    if (p->dtype == SHT_F32)
        return set_error(SHT_ERR_UNSUPPORTED, "sht_forward_noalloc: complex128 plans only (not SHT_F32)");
    if (batch < 0 || batch > 65535) return set_error(SHT_ERR_INVALID_ARG, "batch out of range [0, 65535]");
    if (batch == 0) return SHT_OK;
    if (!d_samples || !d_coeffs) return set_error(SHT_ERR_INVALID_ARG, "NULL buffer");
    if (((uintptr_t)d_samples & 15u) || ((uintptr_t)d_coeffs & 15u))
        return set_error(SHT_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    const int L = p->L;
    const uintptr_t io = (uintptr_t)16 * (uintptr_t)L * (uintptr_t)L * (uintptr_t)batch;
    const uintptr_t a = (uintptr_t)d_samples, b = (uintptr_t)d_coeffs;
    if (a < b + io && b < a + io) return set_error(SHT_ERR_INVALID_ARG, "input and output overlap");

    // scratch: bins W and solved orders F (rows_total(L) x 4B doubles each), split-K partials
    const int64_t Nc = 4 * batch;
    const size_t wf = round256(sizeof(double) * (size_t)rows_total(L) * (size_t)Nc);
    const size_t part = round256(sizeof(double) * (size_t)kSplitCap * L * (size_t)Nc);
    if (2 * wf + part > kNoAllocScratchBytes)
        return set_error(SHT_ERR_UNSUPPORTED,
                         "sht_forward_noalloc: L and batch need " + std::to_string(2 * wf + part) +
                             " bytes of scratch; the fixed array holds " +
                             std::to_string(kNoAllocScratchBytes) + " (use sht_forward)");
    void *base = nullptr;
    sht_status st = scratch_address(dev, &base);
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
