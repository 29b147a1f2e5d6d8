// Ring ordering by condition-number minimisation (Sec. III-E), on the GPU, plan time only.
//
// theta_{L-1} is the ring of the set (Eq. (19), or a set of Sec. III-F) farthest from the poles;
// then for m = L-2, ..., 0, theta_m is the unused ring minimising the 2-norm condition number of
// P_m (Eq. (12)) whose other rows theta_{m+1..L-1} are already fixed.  Exact ties go to the lowest
// index of the set (within a relative tolerance on the mirror-symmetric sets of Sec. III-F).
//
// Scoring every candidate at once: with B the fixed (n-1) x n block and r a candidate row,
// P_m^T P_m = B^T B + r r^T.  From one eigen-decomposition B^T B = V diag(mu) V^T per order
// (cuSOLVER syevd, plan time), z = V^T r gives the eigenvalues of P_m^T P_m as the roots of the
// secular equation 1 + sum_i z_i^2 / (mu_i - x) = 0; by interlacing the smallest lies in
// [mu_0, mu_1] and the largest in [mu_max, mu_max + |r|^2].  Both are bracketed by bisection in a
// warp per candidate, kappa = sqrt(largest / smallest).  Cost O(L^4) instead of O(L^5).
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>

#include "sht_internal.cuh"

namespace sht {
namespace {

// rows of block m of a (L rows) P~ table: fixed rows -> Bf (nf x n), candidates -> Rt (n x nc)
__global__ void k_gather_rows(const double *__restrict__ blk, int n, const int *__restrict__ fixed,
                              int nf, const int *__restrict__ cand, int nc, double *__restrict__ Bf,
                              double *__restrict__ Rt) {
    int r = blockIdx.x;
    if (r < nf) {
        const double *src = blk + (int64_t)fixed[r] * n;
        for (int c = threadIdx.x; c < n; c += blockDim.x) Bf[(int64_t)r * n + c] = src[c];
    } else {
        int cidx = r - nf;
        const double *src = blk + (int64_t)cand[cidx] * n;
        for (int c = threadIdx.x; c < n; c += blockDim.x) Rt[(int64_t)c * nc + cidx] = src[c];
    }
}

__device__ double secular_root(const double *__restrict__ mu, const double *__restrict__ Zt,
                               int n, int nc, int c, double lo, double hi) {
    const int lane = threadIdx.x & 31;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double f = 0.0;
        for (int i = lane; i < n; i += 32) {
            double z = Zt[(int64_t)i * nc + c];
            f += z * z / (mu[i] - mid);
        }
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        f += 1.0;
        // f increases on the bracket: f < 0 (or a pole) means the root is above mid
        if (!(f >= 0.0)) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

__global__ void k_kappa(const double *__restrict__ mu_in, const double *__restrict__ Zt, int n,
                        int nc, double *__restrict__ kappa) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= nc) return;
    const int lane = threadIdx.x & 31;
    double r2 = 0.0;
    for (int i = lane; i < n; i += 32) { double z = Zt[(int64_t)i * nc + c]; r2 += z * z; }
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    const double mu0 = fmax(mu_in[0], 0.0), mu1 = fmax(mu_in[1], 0.0), mun = mu_in[n - 1];
    double lmin = secular_root(mu_in, Zt, n, nc, c, mu0, mu1);
    double lmax = secular_root(mu_in, Zt, n, nc, c, mun, mun + r2);
    if (lane == 0) kappa[c] = (lmin > 0.0) ? sqrt(lmax / lmin) : INFINITY;
}

struct Scratch {
    double *theta = nullptr, *table = nullptr, *Bf = nullptr, *Rt = nullptr, *gram = nullptr,
           *Zt = nullptr, *mu = nullptr, *kap = nullptr, *work = nullptr;
    int *fixed = nullptr, *cand = nullptr, *info = nullptr;
    ~Scratch() {
        cudaFree(theta); cudaFree(table); cudaFree(Bf); cudaFree(Rt); cudaFree(gram);
        cudaFree(Zt); cudaFree(mu); cudaFree(kap); cudaFree(work);
        cudaFree(fixed); cudaFree(cand); cudaFree(info);
    }
};

}  // namespace

sht_status greedy_order(int L, const std::vector<double> &Theta, int middle, double tie_rtol,
                        std::vector<int> &order) {
    order.assign(L, -1);
    order[L - 1] = middle;
    if (L <= 2) {
        if (L == 2) order[0] = 1 - order[1];
        return SHT_OK;
    }

    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        return set_error(SHT_ERR_CUDA, "planner: stream creation failed");
    cusolverDnHandle_t h = nullptr;
    if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) {
        cudaStreamDestroy(s);
        return set_error(SHT_ERR_CUDA, "planner: cusolverDnCreate failed");
    }
    cusolverDnSetStream(h, s);
    sht_status st = SHT_OK;
    {
        Scratch sc;
        const size_t LL = (size_t)L * L;
        cudaError_t e = cudaSuccess;
        auto al = [&](void **p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
        al((void **)&sc.theta, sizeof(double) * L);
        al((void **)&sc.table, sizeof(double) * (size_t)pt_off(L, L));
        al((void **)&sc.Bf, sizeof(double) * LL);
        al((void **)&sc.Rt, sizeof(double) * LL);
        al((void **)&sc.gram, sizeof(double) * LL);
        al((void **)&sc.Zt, sizeof(double) * LL);
        al((void **)&sc.mu, sizeof(double) * L);
        al((void **)&sc.kap, sizeof(double) * L);
        al((void **)&sc.fixed, sizeof(int) * L);
        al((void **)&sc.cand, sizeof(int) * L);
        al((void **)&sc.info, sizeof(int));
        int lwork = 0;
        if (e == cudaSuccess &&
            cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, L,
                                        sc.gram, L, sc.mu, &lwork) != CUSOLVER_STATUS_SUCCESS)
            e = cudaErrorUnknown;
        al((void **)&sc.work, sizeof(double) * (size_t)std::max(lwork, 1));
        if (e != cudaSuccess) { st = cuda_check(e, "planner: allocation"); goto done; }
        cudaMemcpyAsync(sc.theta, Theta.data(), sizeof(double) * L, cudaMemcpyHostToDevice, s);
        e = build_ptilde_table(L, sc.theta, L, sc.table, s);
        if (e != cudaSuccess) { st = cuda_check(e, "planner: table"); goto done; }

        {
            std::vector<char> used(L, 0);
            used[order[L - 1]] = 1;
            std::vector<int> fixed, cand;
            std::vector<double> kap(L);
            for (int m = L - 2; m >= 0; --m) {
                const int n = L - m, nf = n - 1;
                cand.clear();
                for (int t = 0; t < L; ++t) if (!used[t]) cand.push_back(t);
                const int nc = (int)cand.size();
                if (nc == 1) { order[m] = cand[0]; used[cand[0]] = 1; continue; }
                fixed.assign(order.begin() + m + 1, order.end());
                cudaMemcpyAsync(sc.fixed, fixed.data(), sizeof(int) * nf, cudaMemcpyHostToDevice, s);
                cudaMemcpyAsync(sc.cand, cand.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, s);
                const double *blk = sc.table + pt_off(L, m);
                k_gather_rows<<<nf + nc, 128, 0, s>>>(blk, n, sc.fixed, nf, sc.cand, nc, sc.Bf, sc.Rt);
                GemmArgs ga{};
                ga.L = L;
                // Gram = Bf^T Bf  (n x n)
                e = gemm_f64(true, n, nf, n, sc.Bf, n, sc.Bf, n, sc.gram, n, EPI_STORE, ga, s);
                if (e != cudaSuccess) { st = cuda_check(e, "planner: gram"); goto done; }
                if (cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, sc.gram,
                                     n, sc.mu, sc.work, lwork, sc.info) != CUSOLVER_STATUS_SUCCESS) {
                    st = set_error(SHT_ERR_CUDA, "planner: syevd failed");
                    goto done;
                }
                // gram now holds eigenvectors, column-major: row j of the row-major view is v_j.
                // Zt[j][c] = v_j . r_c  =  (gram_rowmajor x Rt)[j][c]
                e = gemm_f64(false, n, n, nc, sc.gram, n, sc.Rt, nc, sc.Zt, nc, EPI_STORE, ga, s);
                if (e != cudaSuccess) { st = cuda_check(e, "planner: projection"); goto done; }
                k_kappa<<<(nc + 3) / 4, 128, 0, s>>>(sc.mu, sc.Zt, n, nc, sc.kap);
                cudaMemcpyAsync(kap.data(), sc.kap, sizeof(double) * nc, cudaMemcpyDeviceToHost, s);
                e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) { st = cuda_check(e, "planner: scoring"); goto done; }
                int best = 0;
                for (int c = 1; c < nc; ++c)
                    if (kap[c] < kap[best]) best = c;
                if (tie_rtol > 0.0)   // the lowest index within the tolerance of the smallest
                    for (int c = 0; c < best; ++c)
                        if (kap[c] <= kap[best] * (1.0 + tie_rtol)) { best = c; break; }
                order[m] = cand[best];
                used[cand[best]] = 1;
            }
        }
    done:;
    }
    cusolverDnDestroy(h);
    cudaStreamDestroy(s);
    return st;
}

}  // namespace sht
