// Plan-time explicit inverses of the per-order matrices P_m (Eq. (12), without its 2 pi factor),
// so that the order-m solve of the forward transform (Eq. (14); Procedure 1, step 5) becomes a
// matrix product.  P_m[k][l] = P~_l^m(theta_k), k, l = m..L-1; it is invertible for the plan's
// ring ordering (Remark 1).  Method: in-place Gauss-Jordan elimination with partial (row)
// pivoting, float64, one thread block per order m, the matrix held in the output buffer.
#include "sht_internal.cuh"

namespace sht {
namespace {

constexpr int kThreads = 512;

__global__ void __launch_bounds__(kThreads) k_gauss_jordan(int L, int m_first, const double *__restrict__ pt,
                                                           double *__restrict__ pinv,
                                                           int *__restrict__ status) {
    extern __shared__ double sm[];
    const int m = m_first + (int)blockIdx.x;
    const int n = L - m;
    double *f = sm;               // column j of the rows, before elimination
    double *rowj = sm + n;        // pivot row after scaling
    int *perm = (int *)(sm + 2 * n);
    __shared__ double red_v[kThreads / 32];
    __shared__ int red_i[kThreads / 32];
    __shared__ int s_piv;

    double *a = pinv + pinv_off(L, m);
    const double *src = pt + pt_off(L, m);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int r = warp; r < n; r += nwarps)
        for (int c = lane; c < n; c += 32) a[(int64_t)r * n + c] = src[(int64_t)(m + r) * n + c];
    __syncthreads();

    for (int j = 0; j < n; ++j) {
        // 1. pivot: largest |a[i][j]|, i >= j (lowest i on ties)
        double bv = -1.0;
        int bi = n;
        for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
            double v = fabs(a[(int64_t)i * n + j]);
            if (v > bv) { bv = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_down_sync(0xffffffffu, bv, o);
            int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if ((threadIdx.x & 31) == 0) { red_v[threadIdx.x >> 5] = bv; red_i[threadIdx.x >> 5] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double v = red_v[0];
            int i0 = red_i[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (red_v[w] > v || (red_v[w] == v && red_i[w] < i0)) { v = red_v[w]; i0 = red_i[w]; }
            if (!(v > 0.0)) { atomicOr(status, 1); i0 = j; }
            s_piv = i0;
            perm[j] = i0;
        }
        __syncthreads();
        const int p = s_piv;
        // 2. swap rows p and j
        if (p != j)
            for (int c = threadIdx.x; c < n; c += blockDim.x) {
                double t0 = a[(int64_t)p * n + c];
                a[(int64_t)p * n + c] = a[(int64_t)j * n + c];
                a[(int64_t)j * n + c] = t0;
            }
        __syncthreads();
        // 3. scale the pivot row; the pivot position receives 1/pivot
        const double piv = a[(int64_t)j * n + j];
        const double rp = (piv != 0.0) ? 1.0 / piv : 0.0;
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            double v = (c == j) ? rp : a[(int64_t)j * n + c] * rp;
            rowj[c] = v;
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) f[i] = a[(int64_t)i * n + j];
        __syncthreads();
        for (int c = threadIdx.x; c < n; c += blockDim.x) a[(int64_t)j * n + c] = rowj[c];
        // 4. eliminate column j from every other row; column j receives -f_i / pivot
        for (int i = warp; i < n; i += nwarps) {
            if (i == j) continue;
            const double fi = f[i];
            double *ai = a + (int64_t)i * n;
            for (int c = lane; c < n; c += 32) {
                double base = (c == j) ? 0.0 : ai[c];
                ai[c] = base - fi * rowj[c];
            }
        }
        __syncthreads();
    }
    // 5. undo the row interchanges as column interchanges, last first
    for (int j = n - 1; j >= 0; --j) {
        int p = perm[j];
        if (p != j)
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                double t0 = a[(int64_t)i * n + p];
                a[(int64_t)i * n + p] = a[(int64_t)i * n + j];
                a[(int64_t)i * n + j] = t0;
            }
        __syncthreads();
    }
}

}  // namespace

cudaError_t build_inverses(int L, const double *d_pt, double *d_pinv, cudaStream_t s, int m_first) {
    if (m_first >= L) return cudaSuccess;
    int *status = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&status, sizeof(int), s);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(status, 0, sizeof(int), s);
    size_t smem = sizeof(double) * 2 * (size_t)L + sizeof(int) * (size_t)L;
    e = cudaFuncSetAttribute(k_gauss_jordan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) { cudaFreeAsync(status, s); return e; }
    k_gauss_jordan<<<L - m_first, kThreads, smem, s>>>(L, m_first, d_pt, d_pinv, status);
    e = cudaGetLastError();
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(status, s);
    if (e == cudaSuccess && h != 0) return cudaErrorInvalidValue;  // a P_m is singular
    return e;
}

}  // namespace sht
