// C ABI of libsht (declared in include/sht.h): plans, argument checking, and the launch
// sequences of the transforms.  All arithmetic runs in the kernels of this directory.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
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

// Elements of one complex value of the plan's signals: complex64 for SHT_F32, else complex128.
static int64_t plan_elem_bytes(sht_plan_t p) { return p->dtype == SHT_F32 ? 8 : 16; }

sht_status check_plan(sht_plan_t p) {
    if (!p) return set_error(SHT_ERR_INVALID_ARG, "plan is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
    if (dev != p->device) return set_error(SHT_ERR_INVALID_ARG, "current device is not the plan's device");
    return SHT_OK;
}

sht_status check_io(sht_plan_t p, const void *in, const void *out, int64_t batch, bool need_ptilde) {
    sht_status st = check_plan(p);
    if (st != SHT_OK) return st;
    if (need_ptilde && !p->pt)
        return set_error(SHT_ERR_UNSUPPORTED, "the plan keeps no P~ table (SHT_PLAN_NO_PTILDE): only the "
                                              "uneven-batch launches (sht_uneven_*) take it");
    if (batch < 0 || batch > kMaxBatch) return set_error(SHT_ERR_INVALID_ARG, "batch out of range [0, 65535]");
    if (batch == 0) return SHT_OK;
    if (!in || !out) return set_error(SHT_ERR_INVALID_ARG, "NULL buffer");
    const uintptr_t eb = (uintptr_t)plan_elem_bytes(p);   // alignment: one complex element
    if (((uintptr_t)in & (eb - 1)) || ((uintptr_t)out & (eb - 1)))
        return set_error(SHT_ERR_INVALID_ARG, eb == 16 ? "buffers must be 16-byte aligned"
                                                       : "buffers must be 8-byte aligned");
    const uintptr_t bytes = eb * (uintptr_t)p->L * (uintptr_t)p->L * (uintptr_t)batch;
    const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
    if (a < b + bytes && b < a + bytes) return set_error(SHT_ERR_INVALID_ARG, "input and output overlap");
    return SHT_OK;
}

}  // namespace sht

using namespace sht;

namespace {

constexpr int kMaxL = 2048;           // longest ring 4095 -> Bluestein length 8192 in shared memory
constexpr int kMaxSpinL = 1024;       // spin plans: host least-squares pseudo-inverses for |m| < |s|
constexpr int kMaxSpin = 8;

void free_ws(Workspace &w) {
    cudaFree(w.a); cudaFree(w.b); cudaFree(w.g); cudaFree(w.part);
    cudaFree(w.xS); cudaFree(w.xE); cudaFree(w.tmX);
    cudaFree(w.r); cudaFree(w.dx); cudaFree(w.bar); cudaFree(w.part2);
    w = Workspace{};
}

void destroy(sht_plan_t p) {
    if (!p) return;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device) cudaSetDevice(p->device);
    cudaFree(p->d_theta); cudaFree(p->pt); cudaFree(p->pinv); cudaFree(p->pt2); cudaFree(p->pinv2);
    cudaFree(p->sect_mant); cudaFree(p->sect_expo); cudaFree(p->rec_a); cudaFree(p->rec_b);
    cudaFree(p->ptS); cudaFree(p->piS); cudaFree(p->ptE); cudaFree(p->piE);
    cudaFree(p->d_ptk_off); cudaFree(p->d_pik_off); cudaFree(p->d_status); cudaFree(p->d_refine_max);
    cudaFree(p->d_tmaps);
    cudaFree(p->ptT); cudaFree(p->piT); cudaFree(p->d_tmaps_tf32); cudaFree(p->chainQ);
    cudaFree(p->ptF); cudaFree(p->pinvF);
    dft_plan_destroy(p->dft);
    for (int st = 0; st < SHT_NUM_STAGES; ++st)
        for (auto &pr : p->spans[st]) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    free_ws(p->ws);
    cudaFree(p->stage);
    if (dev >= 0 && dev != p->device) cudaSetDevice(dev);
    delete p;
}

// Plans whose contractions run on the tensor cores (every arithmetic but SHT_F64 and SHT_F32).
bool tensor_plan(sht_plan_t p) { return p->dtype != SHT_F64 && p->dtype != SHT_F32; }
// Bytes of one complex element of the plan's signals (complex64 for SHT_F32, else complex128).
int64_t elem_bytes(sht_plan_t p) { return p->dtype == SHT_F32 ? 8 : 16; }

// Scratch of one workspace for `batch` signals (grows, never shrinks).  SHT_F32 plans use the
// same buffers as float arrays.
sht_status alloc_ws(sht_plan_t p, Workspace &w, int64_t batch) {
    if (batch <= w.batch) return SHT_OK;
    free_ws(w);
    const size_t L = (size_t)p->L;
    const size_t Nc = 4 * (size_t)batch;
    const size_t a = sizeof(double) * (size_t)rows_total(p->L) * Nc;
    const size_t g = sizeof(double) * L * L * Nc;
    const size_t sp = sizeof(double) * (size_t)kSplitCap * L * Nc;
    cudaError_t e = cudaMalloc(&w.a, a);
    if (e == cudaSuccess) e = cudaMalloc(&w.b, a);
    if (e == cudaSuccess) e = cudaMalloc(&w.g, g);
    if (e == cudaSuccess) e = cudaMalloc(&w.part, sp);
    uint64_t bytes = 2 * a + g + sp;
    if (e == cudaSuccess && p->refine_nsl > 0) {
        const size_t io = sizeof(double2) * L * L * (size_t)batch;
        e = cudaMalloc(&w.r, io);
        if (e == cudaSuccess) e = cudaMalloc(&w.dx, io);
        bytes += 2 * io;
    }
    if (e == cudaSuccess && tensor_plan(p)) {
        const size_t xs = sizeof(__nv_bfloat16) * kTcSlices * Nc * (size_t)p->ptk_off[p->L];
        const size_t words = sizeof(unsigned) * (size_t)tc_chain_words(p->L, batch);
        const size_t sp2 = sizeof(double) * (size_t)kChainB * L * Nc;
        e = cudaMalloc(&w.xS, xs);
        if (e == cudaSuccess) e = cudaMalloc(&w.xE, sizeof(int) * Nc * L);
        if (e == cudaSuccess) e = cudaMalloc(&w.bar, words);
        if (e == cudaSuccess) e = cudaMalloc(&w.part2, sp2);
        if (e == cudaSuccess) e = tc_x_tensor_maps(p->L, batch, w.xS, p->ptk_off, &w.tmX);
        bytes += xs + sizeof(int) * Nc * L + words + sp2 + (uint64_t)p->L * kTensorMapBytes;
    }
    if (e != cudaSuccess) {
        free_ws(w);
        return cuda_check(e, "workspace allocation");
    }
    w.batch = batch;
    w.bytes = bytes;
    return SHT_OK;
}

sht_status ensure_workspace(sht_plan_t p, int64_t batch) { return alloc_ws(p, p->ws, batch); }

// Slices of the P~ table and of the per-order inverses for SHT_F64_TENSOR plans.
sht_status build_tensor_tables(sht_plan_t p, cudaStream_t s, uint64_t &bytes) {
    const int L = p->L;
    p->ptk_off.assign(L + 1, 0);
    p->pik_off.assign(L + 1, 0);
    for (int m = 0; m < L; ++m) {
        const int64_t n = L - m, kp = (n + 7) & ~7;
        p->ptk_off[m + 1] = p->ptk_off[m] + kp;
        p->pik_off[m + 1] = p->pik_off[m] + n * kp;
    }
    const size_t pts = sizeof(__nv_bfloat16) * kTcSlices * (size_t)L * (size_t)p->ptk_off[L];
    const size_t pis = sizeof(__nv_bfloat16) * kTcSlices * (size_t)p->pik_off[L];
    cudaError_t e;
    if ((e = cudaMalloc(&p->ptS, pts)) != cudaSuccess ||
        (e = cudaMalloc(&p->piS, pis)) != cudaSuccess ||
        (e = cudaMalloc(&p->ptE, sizeof(int) * (size_t)L * L)) != cudaSuccess ||
        (e = cudaMalloc(&p->piE, sizeof(int) * (size_t)rows_total(L))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_ptk_off, sizeof(int64_t) * (L + 1))) != cudaSuccess ||
        (e = cudaMalloc(&p->d_pik_off, sizeof(int64_t) * (L + 1))) != cudaSuccess)
        return cuda_check(e, "tensor-core table allocation");
    bytes = pts + pis + sizeof(int) * ((size_t)L * L + rows_total(L)) + 2 * sizeof(int64_t) * (L + 1);
    cudaMemcpyAsync(p->d_ptk_off, p->ptk_off.data(), sizeof(int64_t) * (L + 1), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(p->d_pik_off, p->pik_off.data(), sizeof(int64_t) * (L + 1), cudaMemcpyHostToDevice, s);
    if ((e = tc_prepare_kernels()) != cudaSuccess || (e = tc_prepare_chain(&p->chain_grid)) != cudaSuccess)
        return cuda_check(e, "tensor-core kernel attributes");
    if ((e = tc_slice_table(p->pt, L, false, p->d_ptk_off, p->ptS, p->ptE, s)) != cudaSuccess ||
        (e = tc_slice_table(p->pinv, L, true, p->d_pik_off, p->piS, p->piE, s)) != cudaSuccess)
        return cuda_check(e, "tensor-core table slices");
    if ((e = tc_table_tensor_maps(L, p->piS, p->pik_off, p->ptS, p->ptk_off, &p->d_tmaps)) != cudaSuccess)
        return cuda_check(e, "tensor maps of the table slices");
    bytes += (uint64_t)2 * L * kTensorMapBytes;
    // Q_m = P~_m(rings of m's block below m) P_m^{-1}: the chain's tracked entries
    const size_t qb = sizeof(double) * (size_t)kChainB * (size_t)rows_total(L);
    if ((e = cudaMalloc(&p->chainQ, qb)) != cudaSuccess) return cuda_check(e, "chain table allocation");
    if ((e = tc_chain_q_table(L, p->pt, p->pinv, p->chainQ, s)) != cudaSuccess) return cuda_check(e, "chain table");
    bytes += qb;
    if (p->refine_tf32) {
        // TF32 copies of both tables for the low-precision chain, rows scaled like the slices
        const size_t ptt = sizeof(float) * (size_t)L * (size_t)p->ptk_off[L];
        const size_t pit = sizeof(float) * (size_t)p->pik_off[L];
        if ((e = cudaMalloc(&p->ptT, ptt)) != cudaSuccess || (e = cudaMalloc(&p->piT, pit)) != cudaSuccess)
            return cuda_check(e, "TF32 table allocation");
        if ((e = tc_tf32_table(p->pt, L, false, p->d_ptk_off, p->ptE, p->ptT, s)) != cudaSuccess ||
            (e = tc_tf32_table(p->pinv, L, true, p->d_pik_off, p->piE, p->piT, s)) != cudaSuccess)
            return cuda_check(e, "TF32 tables");
        if ((e = tc_table_tensor_maps_tf32(L, p->piT, p->pik_off, p->ptT, p->ptk_off, &p->d_tmaps_tf32)) != cudaSuccess)
            return cuda_check(e, "tensor maps of the TF32 tables");
        bytes += ptt + pit + (uint64_t)2 * L * kTensorMapBytes;
    }
    e = cudaStreamSynchronize(s);
    return cuda_check(e, "tensor-core table slices");
}

sht_status build_plan(int L, sht_dtype dtype, const std::vector<double> &theta, double order_s,
                      sht_plan_t *out, int spin = 0, bool keep_ptilde = true) {
    auto t0 = std::chrono::steady_clock::now();
    sht_plan_t p = new sht_plan_s;
    p->L = L;
    p->dtype = (int)dtype;
    p->spin = spin;
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
    if (st == SHT_OK && spin != 0) {
        // spin-s tables of both signs of m and their (pseudo-)inverses (Sec. III-H)
        bool singular = false;
        if ((e = cudaMalloc(&p->pt2, pt_bytes)) != cudaSuccess || (e = cudaMalloc(&p->pinv2, pi_bytes)) != cudaSuccess) {
            st = cuda_check(e, "spin table allocation");
        } else {
            cudaMemcpyAsync(p->d_theta, theta.data(), sizeof(double) * L, cudaMemcpyHostToDevice, s);
            e = build_spin_tables(L, spin, p->d_theta, p->pt, p->pt2, p->pinv, p->pinv2, singular, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (singular)
                st = set_error(SHT_ERR_INVALID_ARG, "a per-order spin matrix is singular for these co-latitudes");
            else if (e != cudaSuccess)
                st = cuda_check(e, "spin tables");
        }
    }
    if (st == SHT_OK && spin == 0) {
        cudaMemcpyAsync(p->d_theta, theta.data(), sizeof(double) * L, cudaMemcpyHostToDevice, s);
        e = build_ptilde_table(L, p->d_theta, L, p->pt, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_check(e, "Legendre table");
    }
    if (st == SHT_OK && spin == 0) {
        e = build_inverses(L, p->pt, p->pinv, s);
        if (e == cudaErrorInvalidValue)
            st = set_error(SHT_ERR_INVALID_ARG, "a per-order matrix P_m is singular for these co-latitudes");
        else if (e != cudaSuccess)
            st = cuda_check(e, "per-order inverses");
    }
    uint64_t rec_bytes = 0;
    if (st == SHT_OK && spin == 0) {
        // what regenerates P~ on the fly: sectoral start values and recursion coefficients
        const size_t LL = (size_t)L * L, R = (size_t)rows_total(L);
        if ((e = cudaMalloc(&p->sect_mant, sizeof(double) * LL)) != cudaSuccess ||
            (e = cudaMalloc(&p->sect_expo, sizeof(int) * LL)) != cudaSuccess ||
            (e = cudaMalloc(&p->rec_a, sizeof(double) * R)) != cudaSuccess ||
            (e = cudaMalloc(&p->rec_b, sizeof(double) * R)) != cudaSuccess ||
            (e = sectoral_values(L, p->d_theta, L, p->sect_mant, p->sect_expo, s)) != cudaSuccess ||
            (e = recursion_coeffs(L, p->rec_a, p->rec_b, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            st = cuda_check(e, "recursion data");
        rec_bytes = (sizeof(double) + sizeof(int)) * LL + 2 * sizeof(double) * R;
    }
    if (st == SHT_OK && !keep_ptilde) {   // SHT_PLAN_NO_PTILDE: the inverses are built; drop P~
        cudaFree(p->pt);
        p->pt = nullptr;
    }
    if (st == SHT_OK) {
        e = dft_plan_create(L, p->dft, dft_bytes, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_check(e, "ring DFT plan");
    }
    uint64_t tc_bytes = 0;
    if (st == SHT_OK) {
        e = cudaMalloc(&p->d_status, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&p->d_refine_max, sizeof(double));
        if (e != cudaSuccess) st = cuda_check(e, "status word");
    }
    if (dtype == SHT_BF16_REFINED) p->refine_nsl = 1;
    if (dtype == SHT_BF16X2_REFINED) p->refine_nsl = 2;
    if (dtype == SHT_TF32_REFINED) { p->refine_nsl = 1; p->refine_tf32 = true; }
    uint64_t f32_bytes = 0;
    if (st == SHT_OK && dtype == SHT_F32) {
        // float32 copies of the float64 tables (both are computed in float64 first)
        const int64_t npt = pt_off(L, L), npi = pinv_off(L, L);
        uint64_t dft_f = 0;
        if ((e = cudaMalloc(&p->ptF, sizeof(float) * npt)) == cudaSuccess &&
            (e = cudaMalloc(&p->pinvF, sizeof(float) * npi)) == cudaSuccess &&
            (e = table_to_f32(p->pt, p->ptF, npt, s)) == cudaSuccess &&
            (e = table_to_f32(p->pinv, p->pinvF, npi, s)) == cudaSuccess &&
            (e = dft_plan_make_f32(L, p->dft, dft_f, s)) == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_check(e, "float32 tables");
        f32_bytes = sizeof(float) * (uint64_t)(npt + npi) + dft_f;
    }
    if (st == SHT_OK && tensor_plan(p)) st = build_tensor_tables(p, s, tc_bytes);
    cudaStreamDestroy(s);
    if (st != SHT_OK) { destroy(p); *out = nullptr; return st; }
    p->table_bytes = (spin ? 2 : 1) * ((p->pt ? pt_bytes : 0) + pi_bytes) + dft_bytes + tc_bytes + f32_bytes +
                     rec_bytes + sizeof(double) * L;
    p->plan_seconds = order_s + std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = p;
    return SHT_OK;
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
    // "external" records stay real event records when the stream is being captured into a graph
    Span(sht_plan_t p_, int stage_, cudaStream_t s_) : p(p_), stage(stage_), s(s_) {
        if (p->timing) { b = take_event(p); cudaEventRecordWithFlags(b, s, cudaEventRecordExternal); }
    }
    ~Span() {
        if (p->timing) {
            cudaEvent_t e = take_event(p);
            cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
            p->spans[stage].push_back({b, e});
        }
    }
};

// The execution choices recorded for this batch size (sht_plan_set_paths / sht_plan_autotune).
const sht_tuning *tuning_for(sht_plan_t p, int64_t batch) {
    auto it = p->tuned.find(batch);
    return it == p->tuned.end() ? nullptr : &it->second;
}

// SIMT contractions of the float64 (T = double) and float32 (T = float) plans: tables and GEMM.
template <typename T> const T *pt_table(sht_plan_t p);
template <> const double *pt_table<double>(sht_plan_t p) { return p->pt; }
template <> const float *pt_table<float>(sht_plan_t p) { return p->ptF; }
template <typename T> const T *pinv_table(sht_plan_t p);
template <> const double *pinv_table<double>(sht_plan_t p) { return p->pinv; }
template <> const float *pinv_table<float>(sht_plan_t p) { return p->pinvF; }
cudaError_t gemm_simt(bool tA, int M, int K, int N, const double *A, int64_t lda, const double *B, int64_t ldb,
                      double *C, int64_t ldc, int epi, const GemmArgsT<double> &ga, cudaStream_t s,
                      const double *C0 = nullptr) {
    return gemm_f64(tA, M, K, N, A, lda, B, ldb, C, ldc, epi, ga, s, C0);
}
cudaError_t gemm_simt(bool tA, int M, int K, int N, const float *A, int64_t lda, const float *B, int64_t ldb,
                      float *C, int64_t ldc, int epi, const GemmArgsT<float> &ga, cudaStream_t s,
                      const float *C0 = nullptr) {
    return gemm_f32(tA, M, K, N, A, lda, B, ldb, C, ldc, epi, ga, s, C0);
}

// Eqs. (14)-(16) on the SIMT pipes, one solve and one alias product per order, m = L-1..0; W holds
// the ring bins on entry.
template <typename T>
cudaError_t simt_chain(sht_plan_t p, Workspace &w, T *W, cplx_t<T> *d_coeffs, int64_t batch, cudaStream_t s) {
    const int L = p->L;
    const int64_t Nc = 4 * batch;
    T *F = reinterpret_cast<T *>(w.b);
    const T *pt = pt_table<T>(p), *pinv = pinv_table<T>(p);
    cudaError_t e = cudaSuccess;
    GemmArgsT<T> ga{};
    ga.L = L; ga.batch = batch; ga.coeffs = d_coeffs; ga.W = W;
    ga.part = reinterpret_cast<T *>(w.part); ga.part_cap = (int64_t)kSplitCap * L * Nc;
    ga.launches = &p->launches;
    if (const sht_tuning *t = tuning_for(p, batch)) ga.split_cap = t->split_cap;
    for (int m = L - 1; m >= 0 && e == cudaSuccess; --m) {
        const int n = L - m;
        ga.m = m;
        {   // Eq. (14): F_m = P_m^{-1} g_m, with g_m = bins +-m of rings k >= m (alias-free by now)
            Span sp(p, SHT_STAGE_SOLVE, s);
            e = gemm_simt(false, n, n, (int)Nc, pinv + pinv_off(L, m), n, W + rows_off(L, m) * Nc,
                          Nc, F + rows_off(L, m) * Nc, Nc, EPI_SOLVE, ga, s);
        }
        if (m > 0 && e == cudaSuccess) {  // Eqs. (15)-(16): remove orders +-m from rings k < m
            Span sp(p, SHT_STAGE_ALIAS, s);
            e = gemm_simt(false, m, n, (int)Nc, pt + pt_off(L, m), n, F + rows_off(L, m) * Nc, Nc,
                          (T *)nullptr, Nc, EPI_ALIAS, ga, s);
        }
    }
    return e;
}

// Forward transform of a float32 plan: ring DFTs into bins, then the SIMT chain, all in float32.
cudaError_t forward_f32(sht_plan_t p, Workspace &w, const float2 *d_samples, float2 *d_coeffs,
                        int64_t batch, cudaStream_t s) {
    float *W = reinterpret_cast<float *>(w.a);
    cudaError_t e;
    {
        Span sp(p, SHT_STAGE_RING_DFT, s);
        e = ring_dft_to_bins(p->L, p->dft, d_samples, W, batch, true, s);
    }
    p->launches += dft_launches(p->dft);
    if (e == cudaSuccess) e = simt_chain<float>(p, w, W, d_coeffs, batch, s);
    return e;
}

// Inverse transform on the SIMT pipes (float64 and float32 plans): layout, synthesis, fold + DFTs.
template <typename T>
cudaError_t simt_inverse(sht_plan_t p, Workspace &w, const cplx_t<T> *d_coeffs, cplx_t<T> *d_samples,
                         int64_t batch, cudaStream_t s) {
    const int L = p->L;
    T *X = reinterpret_cast<T *>(w.a), *G = reinterpret_cast<T *>(w.g);
    cudaError_t e;
    {
        Span sp(p, SHT_STAGE_LAYOUT, s);
        e = coeffs_to_orders(L, batch, d_coeffs, X, s);
    }
    if (e == cudaSuccess) {  // Eq. (11): G_{+-m}(theta_k) for every order and ring
        Span sp(p, SHT_STAGE_SYNTHESIS, s);
        e = synthesis_all_orders(L, batch, pt_table<T>(p), X, G, s);
    }
    if (e == cudaSuccess) {  // Eq. (18): fold into ring bins, inverse ring DFTs
        Span sp(p, SHT_STAGE_RING_IDFT, s);
        e = fold_ring_idft(L, p->dft, G, d_samples, batch, s);
    }
    p->launches += 2 + dft_launches(p->dft);
    return e;
}

// Adjoint of the inverse (A^H): forward ring DFTs unfolded to every order, the transposed
// synthesis, layout back to coefficients.
template <typename T>
cudaError_t simt_inverse_adjoint(sht_plan_t p, const cplx_t<T> *d_samples, cplx_t<T> *d_coeffs, int64_t batch,
                                 cudaStream_t s) {
    const int L = p->L;
    T *G = reinterpret_cast<T *>(p->ws.g), *X = reinterpret_cast<T *>(p->ws.a);
    cudaError_t e;
    {
        Span sp(p, SHT_STAGE_RING_DFT, s);
        e = ring_dft_unfold(L, p->dft, d_samples, G, batch, s);
    }
    if (e == cudaSuccess) {
        Span sp(p, SHT_STAGE_SYNTHESIS, s);
        e = analysis_all_orders(L, batch, pt_table<T>(p), G, X, s);
    }
    if (e == cudaSuccess) {
        Span sp(p, SHT_STAGE_LAYOUT, s);
        e = orders_to_coeffs(L, batch, X, d_coeffs, s);
    }
    p->launches += 2 + dft_launches(p->dft);
    return e;
}

// Adjoint of the forward ((A^{-1})^H): the order chain in reverse (m = 0..L-1) with transposed
// per-order inverses and alias gathers, then the adjoint ring DFTs.
template <typename T>
cudaError_t simt_forward_adjoint(sht_plan_t p, const cplx_t<T> *d_coeffs, cplx_t<T> *d_samples, int64_t batch,
                                 cudaStream_t s) {
    const int L = p->L;
    const int64_t Nc = 4 * batch;
    T *X = reinterpret_cast<T *>(p->ws.b), *W = reinterpret_cast<T *>(p->ws.a), *U = reinterpret_cast<T *>(p->ws.g);
    const T *pt = pt_table<T>(p), *pinv = pinv_table<T>(p);
    cudaError_t e;
    {
        Span sp(p, SHT_STAGE_LAYOUT, s);
        e = coeffs_to_orders(L, batch, d_coeffs, X, s);
    }
    GemmArgsT<T> ga{};
    ga.L = L; ga.batch = batch;
    ga.part = reinterpret_cast<T *>(p->ws.part); ga.part_cap = (int64_t)kSplitCap * L * Nc;
    ga.launches = &p->launches;
    for (int m = 0; m < L && e == cudaSuccess; ++m) {
        const int n = L - m;
        T *Xm = X + rows_off(L, m) * Nc;
        if (m > 0) {
            // adjoint of the alias subtraction: X_m -= Q_m^T U, U[k] = bins alias_k(+-m) of rings k < m
            Span sp(p, SHT_STAGE_ALIAS, s);
            e = gather_alias_bins(L, m, batch, W, U, s);
            if (e == cudaSuccess)
                e = gemm_simt(true, n, m, (int)Nc, pt + pt_off(L, m), n, U, Nc, Xm, Nc, EPI_SUB, ga, s, Xm);
        }
        if (e == cudaSuccess) {  // adjoint of the solve: bins +-m of rings k >= m = P_m^{-T} X_m
            Span sp(p, SHT_STAGE_SOLVE, s);
            e = gemm_simt(true, n, n, (int)Nc, pinv + pinv_off(L, m), n, Xm, Nc, W + rows_off(L, m) * Nc, Nc,
                          EPI_STORE, ga, s);
        }
    }
    if (e == cudaSuccess) {
        Span sp(p, SHT_STAGE_RING_IDFT, s);
        e = bins_to_ring_adjoint(L, p->dft, W, d_samples, batch, s);
    }
    p->launches += 1 + (L - 1) + dft_launches(p->dft);  // layout, alias gathers, ring DFTs
    return e;
}

// Forward transform (Procedure 1 in bin space).  Float64 plans run the float64 kernels; the
// tensor plans run the contractions on the tensor cores with `nsl` slices per operand (kTcSlices:
// float64-accurate; fewer: the low-precision forward of the refinement).
cudaError_t forward_impl(sht_plan_t p, Workspace &w, const double2 *d_samples, double2 *d_coeffs,
                         int64_t batch, cudaStream_t s, int nsl) {
    const int L = p->L;
    double *W = w.a, *F = w.b;
    cudaError_t e;
    {
        Span sp(p, SHT_STAGE_RING_DFT, s);
        e = ring_dft_to_bins(L, p->dft, d_samples, W, batch, true, s);
    }
    p->launches += dft_launches(p->dft);
    const sht_tuning *tu = tuning_for(p, batch);
    const bool simt = !tensor_plan(p) || (nsl == kTcSlices && tu && tu->forward_path == SHT_PATH_SIMT);
    if (!simt) {
        // Eqs. (14)-(16) for every order in one persistent launch (stage span: solve)
        Span sp(p, SHT_STAGE_SOLVE, s);
        const bool tf32 = p->refine_tf32 && nsl < kTcSlices;   // the TF32 refinement's F_lo
        const ChainTables t{p->piS, p->piE, p->d_pik_off, p->ptS, p->ptE, p->d_ptk_off,
                            tf32 ? p->d_tmaps_tf32 : p->d_tmaps, p->chainQ};
        if (e == cudaSuccess)
            e = tc_forward_chain(t, L, batch, W, F, d_coeffs, w.part2, w.bar, p->d_status, nsl,
                                 tf32, p->chain_grid, p->wait_ns, s);
        p->launches += 1;
        return e;
    }
    if (e == cudaSuccess) e = simt_chain<double>(p, w, W, d_coeffs, batch, s);
    return e;
}

// Inverse transform (Procedure 2), float64-accurate for every plan arithmetic but SHT_F32.
cudaError_t inverse_impl(sht_plan_t p, Workspace &w, const double2 *d_coeffs, double2 *d_samples,
                         int64_t batch, cudaStream_t s) {
    const sht_tuning *tu = tuning_for(p, batch);
    if (!tensor_plan(p) || (tu && tu->inverse_path == SHT_PATH_SIMT))
        return simt_inverse<double>(p, w, d_coeffs, d_samples, batch, s);
    const int L = p->L;
    cudaError_t e;
    {
        Span sp(p, SHT_STAGE_LAYOUT, s);
        e = coeffs_to_orders(L, batch, d_coeffs, w.a, s);
    }
    if (e == cudaSuccess) {  // Eq. (11): G_{+-m}(theta_k) for every order and ring
        Span sp(p, SHT_STAGE_SYNTHESIS, s);
        e = tc_slice_orders(w.a, L, batch, p->d_ptk_off, w.xS, w.xE, s);
        if (e == cudaSuccess)
            e = tc_synthesis_all_orders(L, batch, p->ptE, p->d_tmaps, w.xE, w.tmX, w.g, p->d_status,
                                        p->wait_ns, s);
        p->launches += 1;
    }
    if (e == cudaSuccess) {  // Eq. (18): fold into ring bins, inverse ring DFTs
        Span sp(p, SHT_STAGE_RING_IDFT, s);
        e = fold_ring_idft(L, p->dft, w.g, d_samples, batch, s);
    }
    p->launches += 2 + dft_launches(p->dft);
    return e;
}

// Iterative refinement of the forward transform: x_0 = F_lo(s), then
// x_{i+1} = x_i + F_lo(s - A x_i), A the float64-accurate inverse, F_lo the forward with
// low-precision (refine_nsl slices) contractions.  With a tolerance, each iteration reads
// max |Re, Im (x_{i+1} - x_i)| to the host and stops below it; with tolerance 0 it runs exactly
// refine_max_iters iterations and never synchronises (capturable in a CUDA graph).
sht_status refined_forward(sht_plan_t p, const double2 *d_samples, double2 *d_coeffs, int64_t batch,
                           cudaStream_t s) {
    Workspace &w = p->ws;
    const int64_t n = (int64_t)p->L * p->L * batch;
    cudaError_t e = forward_impl(p, w, d_samples, d_coeffs, batch, s, p->refine_nsl);
    int it = 0;
    double last = INFINITY;
    bool converged = false;
    for (; it < p->refine_max_iters && e == cudaSuccess; ++it) {
        e = inverse_impl(p, w, d_coeffs, w.r, batch, s);
        if (e == cudaSuccess) e = residual(n, d_samples, w.r, s);
        if (e == cudaSuccess) e = forward_impl(p, w, w.r, w.dx, batch, s, p->refine_nsl);
        if (e == cudaSuccess) e = update_with_max(n, d_coeffs, w.dx, p->d_refine_max, s);
        p->launches += 2;
        if (e == cudaSuccess && p->refine_tol > 0.0) {
            e = cudaMemcpyAsync(&last, p->d_refine_max, sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e == cudaSuccess && last <= p->refine_tol) { ++it; converged = true; break; }
        }
    }
    p->refine_iters = it;
    p->refine_last = last;
    if (e != cudaSuccess) return cuda_check(e, "sht_forward (refinement)");
    if (p->refine_tol > 0.0 && !converged)
        return set_error(SHT_ERR_NOT_CONVERGED, "refinement did not reach the tolerance in max_iters iterations");
    return SHT_OK;
}

// One transform direction over signals of different band-limits: group by plan, run each group as
// one batch, directly when its signals are consecutive in both buffers, else through the plan's
// staging buffers (one device copy per signal each way).
sht_status uneven(bool forward, const sht_plan_t *plans, int nplans, int64_t nsig, const int *plan_index,
                  const int64_t *offsets, const void *d_in, void *d_out, void *stream) {
    if (nsig < 0 || nplans < 0) return set_error(SHT_ERR_INVALID_ARG, "negative count");
    if (nsig == 0) return SHT_OK;
    if (!plans || !plan_index || !offsets || nplans == 0)
        return set_error(SHT_ERR_INVALID_ARG, "NULL plan, index or offset array");
    if (!d_in || !d_out) return set_error(SHT_ERR_INVALID_ARG, "NULL buffer");
    if (((uintptr_t)d_in & 15u) || ((uintptr_t)d_out & 15u))
        return set_error(SHT_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    for (int g = 0; g < nplans; ++g) {
        sht_status st = check_plan(plans[g]);
        if (st != SHT_OK) return st;
        if (plans[g]->dtype == SHT_F32)
            return set_error(SHT_ERR_UNSUPPORTED, "uneven batches take complex128 plans (not SHT_F32)");
        if (plans[g]->spin != 0) return set_error(SHT_ERR_UNSUPPORTED, "uneven batches take scalar (spin-0) plans");
    }
    // signals as intervals [offset, offset + L^2) of complex elements: in range, disjoint
    std::vector<std::pair<int64_t, int64_t>> iv((size_t)nsig);
    for (int64_t i = 0; i < nsig; ++i) {
        const int g = plan_index[i];
        if (g < 0 || g >= nplans) return set_error(SHT_ERR_INVALID_ARG, "plan index out of range");
        if (offsets[i] < 0) return set_error(SHT_ERR_INVALID_ARG, "negative offset");
        const int64_t L = plans[g]->L;
        iv[(size_t)i] = {offsets[i], offsets[i] + L * L};
    }
    std::sort(iv.begin(), iv.end());
    for (size_t i = 1; i < iv.size(); ++i)
        if (iv[i].first < iv[i - 1].second) return set_error(SHT_ERR_INVALID_ARG, "signals overlap");
    const uintptr_t bytes = (uintptr_t)16 * (uintptr_t)iv.back().second;
    const uintptr_t a = (uintptr_t)d_in, b = (uintptr_t)d_out;
    if (a < b + bytes && b < a + bytes) return set_error(SHT_ERR_INVALID_ARG, "input and output overlap");
    cudaStream_t s = (cudaStream_t)stream;
    const double2 *in = (const double2 *)d_in;
    double2 *out = (double2 *)d_out;
    std::vector<int64_t> members;
    for (int g = 0; g < nplans; ++g) {
        sht_plan_t p = plans[g];
        members.clear();
        for (int64_t i = 0; i < nsig; ++i)
            if (plan_index[i] == g) members.push_back(i);
        if (members.empty()) continue;
        const int64_t L2 = (int64_t)p->L * p->L, nb = (int64_t)members.size();
        bool run = true;   // consecutive in the order given
        for (size_t j = 1; j < members.size() && run; ++j)
            run = offsets[members[j]] == offsets[members[j - 1]] + L2;
        for (int64_t b0 = 0; b0 < nb; b0 += kMaxBatch) {
            const int64_t bn = std::min<int64_t>(kMaxBatch, nb - b0);
            sht_status st;
            if (run) {
                const int64_t off = offsets[members[(size_t)b0]];
                st = forward ? sht_forward(p, in + off, out + off, bn, stream)
                             : sht_inverse(p, in + off, out + off, bn, stream);
            } else {
                if (bn > p->stage_batch) {
                    cudaFree(p->stage);
                    p->stage = nullptr;
                    p->stage_batch = 0;
                    cudaError_t e = cudaMalloc(&p->stage, sizeof(double2) * 2 * L2 * bn);
                    if (e != cudaSuccess) return cuda_check(e, "staging buffers");
                    p->stage_batch = bn;
                }
                double2 *si = p->stage, *so = p->stage + L2 * p->stage_batch;
                for (int64_t j = 0; j < bn; ++j) {
                    cudaError_t e = cudaMemcpyAsync(si + j * L2, in + offsets[members[(size_t)(b0 + j)]],
                                                    sizeof(double2) * L2, cudaMemcpyDeviceToDevice, s);
                    if (e != cudaSuccess) return cuda_check(e, "gather");
                }
                st = forward ? sht_forward(p, si, so, bn, stream) : sht_inverse(p, si, so, bn, stream);
                for (int64_t j = 0; j < bn && st == SHT_OK; ++j) {
                    cudaError_t e = cudaMemcpyAsync(out + offsets[members[(size_t)(b0 + j)]], so + j * L2,
                                                    sizeof(double2) * L2, cudaMemcpyDeviceToDevice, s);
                    if (e != cudaSuccess) return cuda_check(e, "scatter");
                }
            }
            if (st != SHT_OK) return st;
        }
    }
    return SHT_OK;
}

// Integral of |tan t|^(1/3) over [0, x], x in [0, pi], in closed form: with T = tan(x)^(2/3) the
// integrand becomes (3/2) T / (1 + T^3) dT, whose partial fractions -1/(3(1+T)) + (T+1)/(3(T^2-T+1))
// integrate to h(T) below; |tan| is symmetric about pi/2 and the integral over [0, pi/2] is
// pi / sqrt(3).
static double tan13_half(double y) {
    const double s3 = std::sqrt(3.0);
    if (y >= M_PI / 2) return M_PI / s3;
    const double T = std::pow(std::tan(y), 2.0 / 3.0);
    const double h = -std::log1p(T) / 3.0 + std::log(T * T - T + 1.0) / 6.0 +
                     (std::atan((2.0 * T - 1.0) / s3) + M_PI / 6.0) / s3;
    return 1.5 * h;
}
static double tan13_integral(double x) {
    return x <= M_PI / 2 ? tan13_half(x) : 2.0 * M_PI / std::sqrt(3.0) - tan13_half(M_PI - x);
}

// The ascending ring set of a placement measure.  SHT_MEASURE_UNIFORM: Eq. (19).  The sets of
// Sec. III-F start at Theta_0 = pi and put 1/L of the measure between consecutive elements, so the
// measure of [Theta_t, pi] is t/L of the total: 1 + cos(Theta_t) = 2t/L for sin(theta) dtheta, and
// for |tan(theta)|^(1/3) dtheta Theta_t solves the closed-form integral by bisection.
std::vector<double> ring_set(int L, uint32_t measure) {
    std::vector<double> T((size_t)L);
    if (measure == SHT_MEASURE_UNIFORM) {
        for (int t = 0; t < L; ++t) T[t] = M_PI * (2.0 * t + 1.0) / (2.0 * L - 1.0);
        return T;
    }
    const double total = 2.0 * M_PI / std::sqrt(3.0);
    T[0] = M_PI;
    for (int t = 1; t < L; ++t) {
        if (measure == SHT_MEASURE_SIN) {
            T[t] = std::acos(2.0 * t / L - 1.0);
        } else {
            const double target = total * (1.0 - (double)t / L);   // integral over [0, Theta_t]
            double lo = 0.0, hi = M_PI;
            for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                (tan13_integral(mid) < target ? lo : hi) = mid;
            }
            T[t] = 0.5 * (lo + hi);
        }
    }
    std::sort(T.begin(), T.end());
    return T;
}

// Index of the element nearest pi/2 (mirror pairs, equal within 1e-12, to the lowest index).
int middle_index(const std::vector<double> &T) {
    double dmin = INFINITY;
    for (double v : T) dmin = std::min(dmin, std::fabs(v - M_PI / 2));
    for (size_t i = 0; i < T.size(); ++i)
        if (std::fabs(T[i] - M_PI / 2) <= dmin + 1e-12) return (int)i;
    return 0;
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
    if (!out) return set_error(SHT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (L < 1 || L > kMaxL) return set_error(SHT_ERR_UNSUPPORTED, "L must be in [1, 2048]");
    if ((int)dtype < 0 || (int)dtype > SHT_F32) return set_error(SHT_ERR_UNSUPPORTED, "dtype not supported");
    if (!theta_host) return set_error(SHT_ERR_INVALID_ARG, "theta_host is NULL");
    const bool keep = !(flags & SHT_PLAN_NO_PTILDE);
    if (!keep && dtype != SHT_F64) return set_error(SHT_ERR_UNSUPPORTED, "SHT_PLAN_NO_PTILDE takes SHT_F64 plans");
    std::vector<double> th(theta_host, theta_host + L);
    // the equiangular set's end point pi (2L-1)/(2L-1) may round one ulp past pi: allow 1e-12
    for (double t : th)
        if (!(t >= -1e-12 && t <= M_PI + 1e-12)) return set_error(SHT_ERR_INVALID_ARG, "theta outside [0, pi]");
    return build_plan(L, dtype, th, 0.0, out, 0, keep);
}

}  // extern "C"

// The ordered ring co-latitudes of sht_plan's flags (Sec. III-E, III-F); order_s receives the time
// the ordering took.
static sht_status ordered_rings(int L, uint32_t flags, std::vector<double> &th, double &order_s) {
    const uint32_t measure = flags & SHT_MEASURE_MASK;
    if (measure != SHT_MEASURE_UNIFORM && measure != SHT_MEASURE_SIN && measure != SHT_MEASURE_TAN13)
        return set_error(SHT_ERR_INVALID_ARG, "unknown ring measure in flags");
    const std::vector<double> Theta = ring_set(L, measure);
    std::vector<int> order(L);
    auto t0 = std::chrono::steady_clock::now();
    if ((flags & SHT_ORDER_MASK) == SHT_ORDER_SIMPLE) {
        // Eq. (20): Theta_{L-1} (= pi), then Theta_0, Theta_{L-2}, Theta_1, Theta_{L-3}, ...
        order[0] = L - 1;
        int lo = 0, hi = L - 2;
        for (int k = 1; k < L; ++k) order[k] = (k & 1) ? lo++ : hi--;
    } else {
        const bool uniform = measure == SHT_MEASURE_UNIFORM;
        sht_status st = greedy_order(L, Theta, uniform ? (L - 1) / 2 : middle_index(Theta),
                                     uniform ? 0.0 : 1e-9, order);
        if (st != SHT_OK) return st;
    }
    order_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    th.assign((size_t)L, 0.0);
    for (int k = 0; k < L; ++k) th[k] = Theta[order[k]];
    return SHT_OK;
}

static sht_status check_spin_args(int L, int spin, sht_dtype dtype) {
    if (L < 1 || L > kMaxSpinL) return set_error(SHT_ERR_UNSUPPORTED, "spin plans take L in [1, 1024]");
    if (spin == 0 || spin < -kMaxSpin || spin > kMaxSpin)
        return set_error(SHT_ERR_UNSUPPORTED, "spin must be in [-8, 8] and non-zero (use sht_plan for s = 0)");
    if (std::abs(spin) >= L) return set_error(SHT_ERR_INVALID_ARG, "|spin| must be below L");
    if (dtype != SHT_F64) return set_error(SHT_ERR_UNSUPPORTED, "spin plans run the SHT_F64 arithmetic only");
    return SHT_OK;
}

extern "C" {

sht_status sht_plan(int L, sht_dtype dtype, uint32_t flags, sht_plan_t *out) {
    if (!out) return set_error(SHT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (L < 1 || L > kMaxL) return set_error(SHT_ERR_UNSUPPORTED, "L must be in [1, 2048]");
    if ((int)dtype < 0 || (int)dtype > SHT_F32) return set_error(SHT_ERR_UNSUPPORTED, "dtype not supported");
    const bool keep = !(flags & SHT_PLAN_NO_PTILDE);
    if (!keep && dtype != SHT_F64) return set_error(SHT_ERR_UNSUPPORTED, "SHT_PLAN_NO_PTILDE takes SHT_F64 plans");
    std::vector<double> th;
    double order_s = 0.0;
    sht_status st = ordered_rings(L, flags, th, order_s);
    if (st != SHT_OK) return st;
    return build_plan(L, dtype, th, order_s, out, 0, keep);
}

sht_status sht_plan_spin(int L, int spin, sht_dtype dtype, uint32_t flags, sht_plan_t *out) {
    if (!out) return set_error(SHT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    sht_status st = check_spin_args(L, spin, dtype);
    if (st != SHT_OK) return st;
    std::vector<double> th;
    double order_s = 0.0;
    if ((st = ordered_rings(L, flags, th, order_s)) != SHT_OK) return st;
    return build_plan(L, dtype, th, order_s, out, spin);
}

sht_status sht_plan_spin_with_thetas(int L, int spin, sht_dtype dtype, const double *theta_host, uint32_t flags,
                                     sht_plan_t *out) {
    (void)flags;
    if (!out) return set_error(SHT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    sht_status st = check_spin_args(L, spin, dtype);
    if (st != SHT_OK) return st;
    if (!theta_host) return set_error(SHT_ERR_INVALID_ARG, "theta_host is NULL");
    std::vector<double> th(theta_host, theta_host + L);
    for (double t : th)
        if (!(t >= -1e-12 && t <= M_PI + 1e-12)) return set_error(SHT_ERR_INVALID_ARG, "theta outside [0, pi]");
    return build_plan(L, dtype, th, 0.0, out, spin);
}

// 64-bit FNV-1a over a byte range (the file hash of sht_plan_save / sht_plan_load).
static uint64_t fnv1a64(const unsigned char *b, size_t n, uint64_t h = 0xcbf29ce484222325ull) {
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 0x100000001b3ull; }
    return h;
}
static const char kThetaTag[8] = {'S', 'H', 'T', 'T', 'H', 'E', 'T', 'A'};

sht_status sht_plan_save(sht_plan_t p, const char *path) {
    if (!p || !path) return set_error(SHT_ERR_INVALID_ARG, "NULL argument");
    if (p->spin != 0) return set_error(SHT_ERR_UNSUPPORTED, "sht_plan_save: scalar (spin-0) plans only");
    std::vector<unsigned char> buf(16 + 8 * (size_t)p->L);
    std::memcpy(buf.data(), kThetaTag, 8);
    const int32_t hdr[2] = {p->L, 0};
    std::memcpy(buf.data() + 8, hdr, 8);
    std::memcpy(buf.data() + 16, p->theta.data(), 8 * (size_t)p->L);
    const uint64_t h = fnv1a64(buf.data(), buf.size());
    FILE *f = std::fopen(path, "wb");
    if (!f) return set_error(SHT_ERR_INVALID_ARG, std::string("cannot write ") + path);
    const bool ok = std::fwrite(buf.data(), 1, buf.size(), f) == buf.size() && std::fwrite(&h, 8, 1, f) == 1;
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed) return set_error(SHT_ERR_INVALID_ARG, std::string("cannot write ") + path);
    return SHT_OK;
}

sht_status sht_plan_load(const char *path, sht_dtype dtype, sht_plan_t *out) {
    if (!out || !path) return set_error(SHT_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return set_error(SHT_ERR_INVALID_ARG, std::string("cannot open ") + path);
    std::vector<unsigned char> buf;
    unsigned char chunk[4096];
    size_t n;
    while ((n = std::fread(chunk, 1, sizeof(chunk), f)) > 0 && buf.size() <= 16 + 8 * (size_t)kMaxL + 8)
        buf.insert(buf.end(), chunk, chunk + n);
    std::fclose(f);
    if (buf.size() < 24 || std::memcmp(buf.data(), kThetaTag, 8) != 0)
        return set_error(SHT_ERR_INVALID_ARG, "not a co-latitude file (tag)");
    int32_t hdr[2];
    std::memcpy(hdr, buf.data() + 8, 8);
    const int L = hdr[0];
    if (L < 1 || L > kMaxL || hdr[1] != 0)
        return set_error(SHT_ERR_INVALID_ARG, "co-latitude file: L outside [1, 2048] or bad header");
    if (buf.size() != 16 + 8 * (size_t)L + 8)
        return set_error(SHT_ERR_INVALID_ARG, "co-latitude file: size does not match L");
    uint64_t h;
    std::memcpy(&h, buf.data() + 16 + 8 * (size_t)L, 8);
    if (h != fnv1a64(buf.data(), 16 + 8 * (size_t)L))
        return set_error(SHT_ERR_INVALID_ARG, "co-latitude file: hash mismatch");
    std::vector<double> th((size_t)L);
    std::memcpy(th.data(), buf.data() + 16, 8 * (size_t)L);
    return sht_plan_with_thetas(L, dtype, th.data(), 0u, out);
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
    out->workspace_bytes = p->ws.bytes;
    out->workspace_batch = p->ws.batch;
    out->plan_seconds = p->plan_seconds;
    out->order_seconds = p->order_seconds;
    out->kernel_launches = p->launches;
    out->refine_iterations = p->refine_iters;
    out->refine_last_update = p->refine_last;
    out->spin = p->spin;
    return SHT_OK;
}

sht_status sht_plan_set_wait_limit(sht_plan_t p, double seconds) {
    sht_status st = check_plan(p);
    if (st != SHT_OK) return st;
    if (!(seconds >= 1e-9 && seconds <= 60.0))
        return set_error(SHT_ERR_INVALID_ARG, "wait limit must be in [1e-9, 60] seconds");
    p->wait_ns = (uint64_t)(seconds * 1e9);
    return SHT_OK;
}

sht_status sht_plan_set_refinement(sht_plan_t p, int max_iters, double tol) {
    if (!p) return set_error(SHT_ERR_INVALID_ARG, "plan is NULL");
    if (max_iters < 0 || !(tol >= 0.0)) return set_error(SHT_ERR_INVALID_ARG, "max_iters < 0 or tol < 0");
    p->refine_max_iters = max_iters;
    p->refine_tol = tol;
    return SHT_OK;
}

sht_status sht_plan_set_paths(sht_plan_t p, int64_t batch, int forward_path, int inverse_path, int split_cap) {
    sht_status st = check_plan(p);
    if (st != SHT_OK) return st;
    if (p->spin != 0) return set_error(SHT_ERR_UNSUPPORTED, "spin plans have one execution path");
    if (batch < 1 || batch > kMaxBatch) return set_error(SHT_ERR_INVALID_ARG, "batch out of range [1, 65535]");
    if (split_cap < 0 || split_cap > 16) return set_error(SHT_ERR_INVALID_ARG, "split_cap outside 0..16");
    const bool tensor = tensor_plan(p), refined = p->refine_nsl > 0;
    auto offered = [&](int path, bool fwd) {
        if (path == SHT_PATH_DEFAULT) return true;
        if (path == SHT_PATH_TENSOR) return tensor;
        if (path == SHT_PATH_SIMT) return !(fwd && refined);
        return false;
    };
    if (!offered(forward_path, true) || !offered(inverse_path, false))
        return set_error(SHT_ERR_INVALID_ARG, "execution path not offered by this plan's arithmetic");
    sht_tuning t{};
    t.forward_path = forward_path;
    t.inverse_path = inverse_path;
    t.split_cap = split_cap;
    p->tuned[batch] = t;
    return SHT_OK;
}

sht_status sht_plan_autotune(sht_plan_t p, int64_t batch, sht_tuning *out) {
    sht_status st = check_plan(p);
    if (st != SHT_OK) return st;
    if (p->spin != 0) return set_error(SHT_ERR_UNSUPPORTED, "spin plans have one execution path");
    if (batch < 1 || batch > kMaxBatch) return set_error(SHT_ERR_INVALID_ARG, "batch out of range [1, 65535]");
    if ((st = ensure_workspace(p, batch)) != SHT_OK) return st;
    const bool tensor = tensor_plan(p), refined = p->refine_nsl > 0;
    const size_t bytes = (size_t)elem_bytes(p) * (size_t)p->L * (size_t)p->L * (size_t)batch;
    void *in = nullptr, *outb = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&in, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&outb, bytes);
    if (e == cudaSuccess) e = cudaMemset(in, 0, bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // best of three timed calls after one warm-up, with `cand` recorded for this batch
    auto time_call = [&](bool fwd, const sht_tuning &cand, double &ms) -> sht_status {
        p->tuned[batch] = cand;
        ms = INFINITY;
        for (int r = 0; r < 4; ++r) {
            cudaEventRecord(e0, s);
            sht_status cs = fwd ? sht_forward(p, in, outb, batch, s) : sht_inverse(p, in, outb, batch, s);
            if (cs != SHT_OK) return cs;
            cudaEventRecord(e1, s);
            cudaError_t ce = cudaEventSynchronize(e1);
            float t = 0.f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
            if (ce != cudaSuccess) return cuda_check(ce, "sht_plan_autotune timing");
            if (r > 0) ms = std::min(ms, (double)t);
        }
        return SHT_OK;
    };
    sht_tuning best{};
    if (e != cudaSuccess) {
        st = cuda_check(e, "sht_plan_autotune buffers");
    } else {
        std::vector<sht_tuning> fwd, inv;
        sht_tuning c{};
        if (refined) {
            fwd.push_back(c);   // the refinement keeps its forward
        } else {
            if (tensor) { c.forward_path = SHT_PATH_TENSOR; fwd.push_back(c); }
            for (int cap : {16, 4, 1}) { c.forward_path = SHT_PATH_SIMT; c.split_cap = cap; fwd.push_back(c); }
        }
        c = sht_tuning{};
        if (tensor) { c.inverse_path = SHT_PATH_TENSOR; inv.push_back(c); }
        c.inverse_path = SHT_PATH_SIMT;
        inv.push_back(c);
        double bf = INFINITY, bi = INFINITY;
        for (const sht_tuning &cand : fwd) {
            if (refined) break;
            double ms = 0;
            if ((st = time_call(true, cand, ms)) != SHT_OK) break;
            if (ms < bf) { bf = ms; best.forward_path = cand.forward_path; best.split_cap = cand.split_cap; }
        }
        for (size_t i = 0; i < inv.size() && st == SHT_OK; ++i) {
            sht_tuning cand = inv[i];
            cand.forward_path = best.forward_path;
            cand.split_cap = best.split_cap;
            double ms = 0;
            if ((st = time_call(false, cand, ms)) != SHT_OK) break;
            if (ms < bi) { bi = ms; best.inverse_path = cand.inverse_path; }
        }
        best.forward_ms = refined ? 0.0 : bf;
        best.inverse_ms = bi;
    }
    if (st == SHT_OK) p->tuned[batch] = best;
    else p->tuned.erase(batch);
    if (s) cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(in);
    cudaFree(outb);
    if (st == SHT_OK && out) *out = best;
    return st;
}

sht_status sht_plan_check(sht_plan_t p) {
    if (!p) return set_error(SHT_ERR_INVALID_ARG, "plan is NULL");
    int h = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h) e = cudaMemset(p->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_check(e, "sht_plan_check");
    if (h) return set_error(SHT_ERR_TIMEOUT, "a bounded wait in a tensor-core kernel gave up");
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
    if (p->spin != 0)
        return cuda_check(spin_forward(p, (const double2 *)d_samples, (double2 *)d_coeffs, batch, s), "sht_forward (spin)");
    if (p->dtype == SHT_F32)
        return cuda_check(forward_f32(p, p->ws, (const float2 *)d_samples, (float2 *)d_coeffs, batch, s), "sht_forward");
    if (p->refine_nsl > 0) return refined_forward(p, (const double2 *)d_samples, (double2 *)d_coeffs, batch, s);
    return cuda_check(forward_impl(p, p->ws, (const double2 *)d_samples, (double2 *)d_coeffs, batch, s,
                                   kTcSlices),
                      "sht_forward");
}

sht_status sht_inverse(sht_plan_t p, const void *d_coeffs, void *d_samples, int64_t batch,
                       void *stream) {
    sht_status st = check_io(p, d_coeffs, d_samples, batch);
    if (st != SHT_OK || batch == 0) return st;
    if ((st = ensure_workspace(p, batch)) != SHT_OK) return st;
    if (p->spin != 0)
        return cuda_check(spin_inverse(p, (const double2 *)d_coeffs, (double2 *)d_samples, batch, (cudaStream_t)stream),
                          "sht_inverse (spin)");
    if (p->dtype == SHT_F32)
        return cuda_check(simt_inverse<float>(p, p->ws, (const float2 *)d_coeffs, (float2 *)d_samples, batch,
                                              (cudaStream_t)stream),
                          "sht_inverse");
    return cuda_check(inverse_impl(p, p->ws, (const double2 *)d_coeffs, (double2 *)d_samples, batch,
                                   (cudaStream_t)stream),
                      "sht_inverse");
}

sht_status sht_ring_analysis(sht_plan_t p, const void *d_samples, void *d_bins, int64_t batch, void *stream) {
    sht_status st = check_io(p, d_samples, d_bins, batch, false);   // ring DFTs only: no P~
    if (st != SHT_OK || batch == 0) return st;
    if ((st = ensure_workspace(p, batch)) != SHT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (p->dtype == SHT_F32) {
        float *W = reinterpret_cast<float *>(p->ws.a);
        e = ring_dft_to_bins(p->L, p->dft, (const float2 *)d_samples, W, batch, true, s);
        if (e == cudaSuccess) e = bins_to_rings(p->L, batch, W, (float2 *)d_bins, s);
    } else {
        double *W = p->ws.a;
        e = ring_dft_to_bins(p->L, p->dft, (const double2 *)d_samples, W, batch, true, s);
        if (e == cudaSuccess) e = bins_to_rings(p->L, batch, W, (double2 *)d_bins, s);
    }
    p->launches += 1 + dft_launches(p->dft);
    return cuda_check(e, "sht_ring_analysis");
}

sht_status sht_ring_synthesis(sht_plan_t p, const void *d_bins, void *d_samples, int64_t batch, void *stream) {
    sht_status st = check_io(p, d_bins, d_samples, batch, false);
    if (st != SHT_OK || batch == 0) return st;
    if ((st = ensure_workspace(p, batch)) != SHT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (p->dtype == SHT_F32) {
        float *G = reinterpret_cast<float *>(p->ws.g);
        e = rings_to_table(p->L, batch, (const float2 *)d_bins, G, s);
        if (e == cudaSuccess) e = fold_ring_idft(p->L, p->dft, G, (float2 *)d_samples, batch, s);
    } else {
        double *G = p->ws.g;
        e = rings_to_table(p->L, batch, (const double2 *)d_bins, G, s);
        if (e == cudaSuccess) e = fold_ring_idft(p->L, p->dft, G, (double2 *)d_samples, batch, s);
    }
    p->launches += 1 + dft_launches(p->dft);
    return cuda_check(e, "sht_ring_synthesis");
}

sht_status sht_forward_uneven(const sht_plan_t *plans, int nplans, int64_t nsig, const int *plan_index,
                              const int64_t *offsets, const void *d_samples, void *d_coeffs, void *stream) {
    return uneven(true, plans, nplans, nsig, plan_index, offsets, d_samples, d_coeffs, stream);
}

sht_status sht_inverse_uneven(const sht_plan_t *plans, int nplans, int64_t nsig, const int *plan_index,
                              const int64_t *offsets, const void *d_coeffs, void *d_samples, void *stream) {
    return uneven(false, plans, nplans, nsig, plan_index, offsets, d_coeffs, d_samples, stream);
}

sht_status sht_inverse_adjoint(sht_plan_t p, const void *d_samples, void *d_coeffs, int64_t batch,
                               void *stream) {
    sht_status st = check_io(p, d_samples, d_coeffs, batch);
    if (st != SHT_OK || batch == 0) return st;
    if ((st = ensure_workspace(p, batch)) != SHT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->spin != 0)
        return cuda_check(spin_inverse_adjoint(p, (const double2 *)d_samples, (double2 *)d_coeffs, batch, s),
                          "sht_inverse_adjoint (spin)");
    const cudaError_t e =
        p->dtype == SHT_F32
            ? simt_inverse_adjoint<float>(p, (const float2 *)d_samples, (float2 *)d_coeffs, batch, s)
            : simt_inverse_adjoint<double>(p, (const double2 *)d_samples, (double2 *)d_coeffs, batch, s);
    return cuda_check(e, "sht_inverse_adjoint");
}

sht_status sht_forward_adjoint(sht_plan_t p, const void *d_coeffs, void *d_samples, int64_t batch,
                               void *stream) {
    sht_status st = check_io(p, d_coeffs, d_samples, batch);
    if (st != SHT_OK) return st;
    if (p->spin != 0) return set_error(SHT_ERR_UNSUPPORTED, "sht_forward_adjoint: not offered for spin plans");
    if (batch == 0) return st;
    if ((st = ensure_workspace(p, batch)) != SHT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const cudaError_t e =
        p->dtype == SHT_F32
            ? simt_forward_adjoint<float>(p, (const float2 *)d_coeffs, (float2 *)d_samples, batch, s)
            : simt_forward_adjoint<double>(p, (const double2 *)d_coeffs, (double2 *)d_samples, batch, s);
    return cuda_check(e, "sht_forward_adjoint");
}

}  // extern "C"
