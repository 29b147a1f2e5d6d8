// C ABI of libsht (declared in include/sht.h): plans, argument checking, and the launch
// sequences of the transforms.  All arithmetic runs in the kernels of this directory.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "sht_internal.cuh"

namespace sht {

static thread_local std::string g_error;

sht_status set_error(sht_status st, const std::string &msg) {
    g_error = msg;
    return st;
}

sht_status cuda_check(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SHT_OK;
    g_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return SHT_ERR_OOM;
    return SHT_ERR_CUDA;
}

}  // namespace sht

using namespace sht;

namespace {

constexpr int kMaxL = 2048;           // longest ring 4095 -> Bluestein length 8192 in shared memory
constexpr int64_t kMaxBatch = 65535;  // batch is a grid dimension of the ring kernels

void free_workspaces(sht_plan_t p) {
    cudaFree(p->ws_a); cudaFree(p->ws_b); cudaFree(p->ws_g); cudaFree(p->ws_part);
    p->ws_a = p->ws_b = p->ws_g = p->ws_part = nullptr;
    p->ws_batch = 0;
    p->ws_bytes = 0;
}

void destroy(sht_plan_t p) {
    if (!p) return;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device) cudaSetDevice(p->device);
    cudaFree(p->d_theta); cudaFree(p->pt); cudaFree(p->pinv);
    dft_plan_destroy(p->dft);
    for (int st = 0; st < SHT_NUM_STAGES; ++st)
        for (auto &pr : p->spans[st]) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    free_workspaces(p);
    if (dev >= 0 && dev != p->device) cudaSetDevice(dev);
    delete p;
}

sht_status ensure_workspace(sht_plan_t p, int64_t batch) {
    if (batch <= p->ws_batch) return SHT_OK;
    free_workspaces(p);
    const size_t L = (size_t)p->L;
    const size_t a = sizeof(double) * (size_t)rows_total(p->L) * 4 * (size_t)batch;
    const size_t g = sizeof(double) * L * L * 4 * (size_t)batch;
    const size_t sp = sizeof(double) * (size_t)kSplitCap * L * 4 * (size_t)batch;
    cudaError_t e = cudaMalloc(&p->ws_a, a);
    if (e == cudaSuccess) e = cudaMalloc(&p->ws_b, a);
    if (e == cudaSuccess) e = cudaMalloc(&p->ws_g, g);
    if (e == cudaSuccess) e = cudaMalloc(&p->ws_part, sp);
    if (e != cudaSuccess) {
        free_workspaces(p);
        return cuda_check(e, "workspace allocation");
    }
    p->ws_batch = batch;
    p->ws_bytes = 2 * a + g + sp;
    return SHT_OK;
}

sht_status build_plan(int L, sht_dtype dtype, const std::vector<double> &theta, double order_s,
                      sht_plan_t *out) {
    auto t0 = std::chrono::steady_clock::now();
    sht_plan_t p = new sht_plan_s;
    p->L = L;
    p->dtype = (int)dtype;
    p->theta = theta;
    p->order_seconds = order_s;
    cudaGetDevice(&p->device);
    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete p; return cuda_check(e, "plan stream"); }
    const size_t pt_bytes = sizeof(double) * (size_t)pt_off(L, L);
    const size_t pi_bytes = sizeof(double) * (size_t)pinv_off(L, L);
    uint64_t dft_bytes = 0;
    sht_status st = SHT_OK;
    if ((e = cudaMalloc(&p->d_theta, sizeof(double) * L)) != cudaSuccess ||
        (e = cudaMalloc(&p->pt, pt_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&p->pinv, pi_bytes)) != cudaSuccess) {
        st = cuda_check(e, "plan table allocation");
    }
    if (st == SHT_OK) {
        cudaMemcpyAsync(p->d_theta, theta.data(), sizeof(double) * L, cudaMemcpyHostToDevice, s);
        e = build_ptilde_table(L, p->d_theta, L, p->pt, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_check(e, "Legendre table");
    }
    if (st == SHT_OK) {
        e = build_inverses(L, p->pt, p->pinv, s);
        if (e == cudaErrorInvalidValue)
            st = set_error(SHT_ERR_INVALID_ARG, "a per-order matrix P_m is singular for these co-latitudes");
        else if (e != cudaSuccess)
            st = cuda_check(e, "per-order inverses");
    }
    if (st == SHT_OK) {
        e = dft_plan_create(L, p->dft, dft_bytes, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_check(e, "ring DFT plan");
    }
    cudaStreamDestroy(s);
    if (st != SHT_OK) { destroy(p); *out = nullptr; return st; }
    p->table_bytes = pt_bytes + pi_bytes + dft_bytes + sizeof(double) * L;
    p->plan_seconds = order_s + std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return SHT_OK;
}

// Number of ring-DFT launches per transform: direct rings, then one per chirp-z length class.
int64_t ring_launches(int L) {
    int64_t n = 1;
    for (int j = 5; (1 << j) < L; ++j) ++n;
    return n;
}

cudaEvent_t take_event(sht_plan_t p) {
    if (!p->ev_pool.empty()) {
        cudaEvent_t e = p->ev_pool.back();
        p->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records a CUDA event pair around one stage when the plan's timing is on.
struct Span {
    sht_plan_t p;
    int stage;
    cudaStream_t s;
    cudaEvent_t b = nullptr;
    Span(sht_plan_t p_, int stage_, cudaStream_t s_) : p(p_), stage(stage_), s(s_) {
        if (p->timing) { b = take_event(p); cudaEventRecord(b, s); }
    }
    ~Span() {
        if (p->timing) {
            cudaEvent_t e = take_event(p);
            cudaEventRecord(e, s);
            p->spans[stage].push_back({b, e});
        }
    }
};

sht_status check_plan(sht_plan_t p) {
    if (!p) return set_error(SHT_ERR_INVALID_ARG, "plan is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
    if (dev != p->device) return set_error(SHT_ERR_INVALID_ARG, "current device is not the plan's device");
    return SHT_OK;
}

sht_status check_io(sht_plan_t p, const void *in, const void *out, int64_t batch) {
    sht_status st = check_plan(p);
    if (st != SHT_OK) return st;
    if (batch < 0 || batch > kMaxBatch) return set_error(SHT_ERR_INVALID_ARG, "batch out of range [0, 65535]");
    if (batch == 0) return SHT_OK;
    if (!in || !out) return set_error(SHT_ERR_INVALID_ARG, "NULL buffer");
    if (((uintptr_t)in & 15u) || ((uintptr_t)out & 15u))
        return set_error(SHT_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    const uintptr_t bytes = (uintptr_t)16 * (uintptr_t)p->L * (uintptr_t)p->L * (uintptr_t)batch;
    const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
    if (a < b + bytes && b < a + bytes) return set_error(SHT_ERR_INVALID_ARG, "input and output overlap");
    return SHT_OK;
}

}  // namespace

extern "C" {

const char *sht_status_string(sht_status s) {
    switch (s) {
        case SHT_OK: return "SHT_OK";
        case SHT_ERR_INVALID_ARG: return "SHT_ERR_INVALID_ARG";
        case SHT_ERR_UNSUPPORTED: return "SHT_ERR_UNSUPPORTED";
        case SHT_ERR_OOM: return "SHT_ERR_OOM";
        case SHT_ERR_CUDA: return "SHT_ERR_CUDA";
        case SHT_ERR_NOT_CONVERGED: return "SHT_ERR_NOT_CONVERGED";
        case SHT_ERR_TIMEOUT: return "SHT_ERR_TIMEOUT";
    }
    return "SHT_ERR_UNKNOWN";
}

const char *sht_last_error_message(void) { return g_error.c_str(); }

sht_status sht_plan_with_thetas(int L, sht_dtype dtype, const double *theta_host, uint32_t flags,
                                sht_plan_t *out) {
    (void)flags;
    if (!out) return set_error(SHT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (L < 1 || L > kMaxL) return set_error(SHT_ERR_UNSUPPORTED, "L must be in [1, 2048]");
    if (dtype != SHT_F64) return set_error(SHT_ERR_UNSUPPORTED, "dtype not supported");
    if (!theta_host) return set_error(SHT_ERR_INVALID_ARG, "theta_host is NULL");
    std::vector<double> th(theta_host, theta_host + L);
    for (double t : th)
        if (!(t >= 0.0 && t <= M_PI)) return set_error(SHT_ERR_INVALID_ARG, "theta outside [0, pi]");
    return build_plan(L, dtype, th, 0.0, out);
}

sht_status sht_plan(int L, sht_dtype dtype, uint32_t flags, sht_plan_t *out) {
    if (!out) return set_error(SHT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (L < 1 || L > kMaxL) return set_error(SHT_ERR_UNSUPPORTED, "L must be in [1, 2048]");
    if (dtype != SHT_F64) return set_error(SHT_ERR_UNSUPPORTED, "dtype not supported");
    std::vector<int> order(L);
    auto t0 = std::chrono::steady_clock::now();
    if ((flags & SHT_ORDER_MASK) == SHT_ORDER_SIMPLE) {
        // Eq. (20): Theta_{L-1} (= pi), then Theta_0, Theta_{L-2}, Theta_1, Theta_{L-3}, ...
        order[0] = L - 1;
        int lo = 0, hi = L - 2;
        for (int k = 1; k < L; ++k) order[k] = (k & 1) ? lo++ : hi--;
    } else {
        sht_status st = greedy_order(L, order);
        if (st != SHT_OK) return st;
    }
    double order_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    std::vector<double> th(L);
    for (int k = 0; k < L; ++k) th[k] = M_PI * (2.0 * order[k] + 1.0) / (2.0 * L - 1.0);
    return build_plan(L, dtype, th, order_s, out);
}

sht_status sht_plan_thetas(sht_plan_t p, double *theta_host_out) {
    if (!p || !theta_host_out) return set_error(SHT_ERR_INVALID_ARG, "NULL argument");
    std::memcpy(theta_host_out, p->theta.data(), sizeof(double) * p->L);
    return SHT_OK;
}

int sht_plan_bandlimit(sht_plan_t p) { return p ? p->L : 0; }

sht_status sht_plan_reserve(sht_plan_t p, int64_t batch) {
    sht_status st = check_plan(p);
    if (st != SHT_OK) return st;
    if (batch < 0 || batch > kMaxBatch) return set_error(SHT_ERR_INVALID_ARG, "batch out of range");
    return ensure_workspace(p, batch);
}

sht_status sht_plan_destroy(sht_plan_t p) {
    if (!p) return SHT_OK;
    cudaDeviceSynchronize();
    destroy(p);
    return SHT_OK;
}

sht_status sht_get_info(sht_plan_t p, sht_info *out) {
    if (!p || !out) return set_error(SHT_ERR_INVALID_ARG, "NULL argument");
    out->L = p->L;
    out->dtype = p->dtype;
    out->table_bytes = p->table_bytes;
    out->workspace_bytes = p->ws_bytes;
    out->workspace_batch = p->ws_batch;
    out->plan_seconds = p->plan_seconds;
    out->order_seconds = p->order_seconds;
    out->kernel_launches = p->launches;
    return SHT_OK;
}

sht_status sht_plan_set_timing(sht_plan_t p, int enable) {
    if (!p) return set_error(SHT_ERR_INVALID_ARG, "plan is NULL");
    p->timing = enable != 0;
    return SHT_OK;
}

sht_status sht_plan_stage_times(sht_plan_t p, double *ms, int64_t *spans) {
    if (!p) return set_error(SHT_ERR_INVALID_ARG, "plan is NULL");
    cudaError_t err = cudaSuccess;
    for (int st = 0; st < SHT_NUM_STAGES; ++st) {
        double tot = 0.0;
        for (auto &pr : p->spans[st]) {
            float t = 0.f;
            cudaError_t e = cudaEventSynchronize(pr.second);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pr.first, pr.second);
            if (e != cudaSuccess && err == cudaSuccess) err = e;
            tot += t;
            p->ev_pool.push_back(pr.first);
            p->ev_pool.push_back(pr.second);
        }
        if (ms) ms[st] = tot;
        if (spans) spans[st] = (int64_t)p->spans[st].size();
        p->spans[st].clear();
    }
    return cuda_check(err, "sht_plan_stage_times");
}

sht_status sht_forward(sht_plan_t p, const void *d_samples, void *d_coeffs, int64_t batch,
                       void *stream) {
    sht_status st = check_io(p, d_samples, d_coeffs, batch);
    if (st != SHT_OK || batch == 0) return st;
    if ((st = ensure_workspace(p, batch)) != SHT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = p->L;
    const int64_t Nc = 4 * batch;
    double *W = p->ws_a, *F = p->ws_b;
    cudaError_t e;
    {
        Span sp(p, SHT_STAGE_RING_DFT, s);
        e = ring_dft_to_bins(L, p->dft, (const double2 *)d_samples, W, batch, true, s);
    }
    GemmArgs ga{};
    ga.L = L; ga.batch = batch; ga.coeffs = (double2 *)d_coeffs; ga.W = W;
    ga.part = p->ws_part; ga.part_cap = (int64_t)kSplitCap * L * Nc;
    ga.launches = &p->launches;
    for (int m = L - 1; m >= 0 && e == cudaSuccess; --m) {
        const int n = L - m;
        ga.m = m;
        {   // Eq. (14): F_m = P_m^{-1} g_m, with g_m = bins +-m of rings k >= m (alias-free by now)
            Span sp(p, SHT_STAGE_SOLVE, s);
            e = gemm_f64(false, n, n, (int)Nc, p->pinv + pinv_off(L, m), n, W + rows_off(L, m) * Nc,
                         Nc, F + rows_off(L, m) * Nc, Nc, EPI_SOLVE, ga, s);
        }
        if (m > 0 && e == cudaSuccess) {  // Eqs. (15)-(16): remove orders +-m from rings k < m
            Span sp(p, SHT_STAGE_ALIAS, s);
            e = gemm_f64(false, m, n, (int)Nc, p->pt + pt_off(L, m), n, F + rows_off(L, m) * Nc, Nc,
                         nullptr, Nc, EPI_ALIAS, ga, s);
        }
    }
    p->launches += ring_launches(L);
    return cuda_check(e, "sht_forward");
}

sht_status sht_inverse(sht_plan_t p, const void *d_coeffs, void *d_samples, int64_t batch,
                       void *stream) {
    sht_status st = check_io(p, d_coeffs, d_samples, batch);
    if (st != SHT_OK || batch == 0) return st;
    if ((st = ensure_workspace(p, batch)) != SHT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = p->L;
    cudaError_t e;
    {
        Span sp(p, SHT_STAGE_LAYOUT, s);
        e = coeffs_to_orders(L, batch, (const double2 *)d_coeffs, p->ws_a, s);
    }
    if (e == cudaSuccess) {  // Eq. (11): G_{+-m}(theta_k) for every order and ring
        Span sp(p, SHT_STAGE_SYNTHESIS, s);
        e = synthesis_all_orders(L, batch, p->pt, p->ws_a, p->ws_g, s);
    }
    if (e == cudaSuccess) {  // Eq. (18): fold into ring bins, inverse ring DFTs
        Span sp(p, SHT_STAGE_RING_IDFT, s);
        e = fold_ring_idft(L, p->dft, p->ws_g, (double2 *)d_samples, batch, s);
    }
    p->launches += 2 + ring_launches(L);
    return cuda_check(e, "sht_inverse");
}

sht_status sht_inverse_adjoint(sht_plan_t p, const void *d_samples, void *d_coeffs, int64_t batch,
                               void *stream) {
    sht_status st = check_io(p, d_samples, d_coeffs, batch);
    if (st != SHT_OK || batch == 0) return st;
    if ((st = ensure_workspace(p, batch)) != SHT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = p->L;
    cudaError_t e;
    {
        Span sp(p, SHT_STAGE_RING_DFT, s);
        e = ring_dft_unfold(L, p->dft, (const double2 *)d_samples, p->ws_g, batch, s);
    }
    if (e == cudaSuccess) {
        Span sp(p, SHT_STAGE_SYNTHESIS, s);
        e = analysis_all_orders(L, batch, p->pt, p->ws_g, p->ws_a, s);
    }
    if (e == cudaSuccess) {
        Span sp(p, SHT_STAGE_LAYOUT, s);
        e = orders_to_coeffs(L, batch, p->ws_a, (double2 *)d_coeffs, s);
    }
    p->launches += 2 + ring_launches(L);
    return cuda_check(e, "sht_inverse_adjoint");
}

sht_status sht_forward_adjoint(sht_plan_t p, const void *d_coeffs, void *d_samples, int64_t batch,
                               void *stream) {
    sht_status st = check_io(p, d_coeffs, d_samples, batch);
    if (st != SHT_OK || batch == 0) return st;
    if ((st = ensure_workspace(p, batch)) != SHT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int L = p->L;
    const int64_t Nc = 4 * batch;
    double *X = p->ws_b, *W = p->ws_a, *U = p->ws_g;
    cudaError_t e;
    {
        Span sp(p, SHT_STAGE_LAYOUT, s);
        e = coeffs_to_orders(L, batch, (const double2 *)d_coeffs, X, s);
    }
    GemmArgs ga{};
    ga.L = L; ga.batch = batch;
    ga.part = p->ws_part; ga.part_cap = (int64_t)kSplitCap * L * Nc;
    ga.launches = &p->launches;
    // reverse of the forward chain: m = 0 .. L-1
    for (int m = 0; m < L && e == cudaSuccess; ++m) {
        const int n = L - m;
        double *Xm = X + rows_off(L, m) * Nc;
        if (m > 0) {
            // adjoint of the alias subtraction: X_m -= Q_m^T U, U[k] = bins alias_k(+-m) of rings k < m
            Span sp(p, SHT_STAGE_ALIAS, s);
            e = gather_alias_bins(L, m, batch, W, U, s);
            if (e == cudaSuccess)
                e = gemm_f64(true, n, m, (int)Nc, p->pt + pt_off(L, m), n, U, Nc, Xm, Nc, EPI_SUB,
                             ga, s, Xm);
        }
        if (e == cudaSuccess) {  // adjoint of the solve: bins +-m of rings k >= m = P_m^{-T} X_m
            Span sp(p, SHT_STAGE_SOLVE, s);
            e = gemm_f64(true, n, n, (int)Nc, p->pinv + pinv_off(L, m), n, Xm, Nc,
                         W + rows_off(L, m) * Nc, Nc, EPI_STORE, ga, s);
        }
    }
    if (e == cudaSuccess) {
        Span sp(p, SHT_STAGE_RING_IDFT, s);
        e = bins_to_ring_adjoint(L, p->dft, W, (double2 *)d_samples, batch, s);
    }
    p->launches += 1 + (L - 1) + ring_launches(L);  // layout, alias gathers, ring DFTs
    return cuda_check(e, "sht_forward_adjoint");
}

}  // extern "C"
