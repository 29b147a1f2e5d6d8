// Coefficient layout <-> order-major layout.
// Coefficients: f_l^m at l^2 + l + m (per signal).  Order-major block m >= 0: row l - m holds
// (f_l^{+m}, (-1)^m f_l^{-m}) for every signal; the (-1)^m is Eq. (23) (P~^{-m} = (-1)^m P~^m)
// moved onto the data so that one real table P~^m serves both signs of m.
#include "sht_internal.cuh"

namespace sht {
namespace {

__device__ __forceinline__ void decode(int64_t idx, int &l, int &m) {
    int ll = (int)sqrt((double)idx);
    while ((int64_t)ll * ll > idx) --ll;
    while ((int64_t)(ll + 1) * (ll + 1) <= idx) ++ll;
    l = ll;
    m = (int)(idx - (int64_t)ll * ll - ll);
}

template <typename T>
__global__ void k_coeffs_to_orders(int L, int64_t batch, const cplx_t<T> *__restrict__ coeffs,
                                   T *__restrict__ X) {
    const int64_t L2 = (int64_t)L * L;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L2 * batch) return;
    const int64_t b = t / L2, idx = t - b * L2;
    int l, m;
    decode(idx, l, m);
    const int o = m < 0 ? -m : m;
    T *x = X + (rows_off(L, o) + (l - o)) * (4 * batch) + 4 * b;
    cplx_t<T> v = coeffs[t];
    if (m >= 0) {
        x[0] = v.x; x[1] = v.y;
        if (m == 0) { x[2] = 0; x[3] = 0; }
    } else {
        const T sg = (o & 1) ? (T)-1 : (T)1;
        x[2] = sg * v.x; x[3] = sg * v.y;
    }
}

template <typename T>
__global__ void k_orders_to_coeffs(int L, int64_t batch, const T *__restrict__ X,
                                   cplx_t<T> *__restrict__ coeffs) {
    const int64_t L2 = (int64_t)L * L;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L2 * batch) return;
    const int64_t b = t / L2, idx = t - b * L2;
    int l, m;
    decode(idx, l, m);
    const int o = m < 0 ? -m : m;
    const T *x = X + (rows_off(L, o) + (l - o)) * (4 * batch) + 4 * b;
    if (m >= 0) {
        coeffs[t] = mk2<T>(x[0], x[1]);
    } else {
        const T sg = (o & 1) ? (T)-1 : (T)1;
        coeffs[t] = mk2<T>(sg * x[2], sg * x[3]);
    }
}

// U[k][4b + 2s + c], k < m: bin alias_k(+m) (s = 0) and alias_k(-m) (s = 1) of ring k, read from
// the order-major bins W (bin q of ring k: block |q|, row k - |q|, slot 0 for q >= 0, 2 for q < 0).
template <typename T>
__global__ void k_gather_alias_bins(int L, int m, int64_t batch, const T *__restrict__ W,
                                    T *__restrict__ U) {
    const int64_t Nc = 4 * batch;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)m * batch) return;
    const int k = (int)(t / batch), b = (int)(t - (int64_t)k * batch);
    const int a = alias_bin(m, k);
    const int o = a < 0 ? -a : a;
    const T *w = W + (rows_off(L, o) + (k - o)) * Nc + 4 * b;
    const int sp = a >= 0 ? 0 : 2, sn = a > 0 ? 2 : 0;  // slots of bins a and -a (bin 0: slot 0)
    T *u = U + (int64_t)k * Nc + 4 * b;
    u[0] = w[sp]; u[1] = w[sp + 1];
    u[2] = w[sn]; u[3] = w[sn + 1];
}

// float64 -> float32 copy of a plan table (SHT_F32 plans)
__global__ void k_to_f32(const double *__restrict__ in, float *__restrict__ out, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = (float)in[t];
}

__global__ void k_residual(int64_t n, const double2 *__restrict__ s_in, double2 *__restrict__ r) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double2 a = s_in[t], b = r[t];
    r[t] = make_double2(a.x - b.x, a.y - b.y);
}

// x += dx; the largest |Re dx|, |Im dx| goes to *mx through an integer atomicMax on the bit
// pattern (non-negative doubles order like their bits).
__global__ void k_update_max(int64_t n, double2 *__restrict__ x, const double2 *__restrict__ dx,
                             unsigned long long *__restrict__ mx) {
    __shared__ unsigned long long red[8];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long m = 0;
    if (t < n) {
        const double2 a = x[t], d = dx[t];
        x[t] = make_double2(a.x + d.x, a.y + d.y);
        const unsigned long long ur = (unsigned long long)__double_as_longlong(d.x) & 0x7FFFFFFFFFFFFFFFull;
        const unsigned long long ui = (unsigned long long)__double_as_longlong(d.y) & 0x7FFFFFFFFFFFFFFFull;
        m = ur > ui ? ur : ui;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long q = __shfl_xor_sync(0xffffffffu, m, o);
        m = q > m ? q : m;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
        atomicMax(mx, m);
    }
}

// Ring-major bins (per signal: bin j of ring k at k^2 + k + j, |j| <= k) from the order-major bins
// W (bin q of ring k: block |q|, row k - |q|, slot 0 for q >= 0, 2 for q < 0).  Thread = one bin.
template <typename T>
__global__ void k_bins_to_rings(int L, int64_t batch, const T *__restrict__ W, cplx_t<T> *__restrict__ bins) {
    const int64_t L2 = (int64_t)L * L;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L2 * batch) return;
    const int64_t b = t / L2, idx = t - b * L2;
    int k, j;
    decode(idx, k, j);
    const int o = j < 0 ? -j : j;
    const T *w = W + (rows_off(L, o) + (k - o)) * (4 * batch) + 4 * b + (j < 0 ? 2 : 0);
    bins[t] = mk2<T>(w[0], w[1]);
}

// Synthesis table Gt (row m L + k, columns 4b + 2s + c) holding ring k's bins as orders:
// G_{+m}(theta_k) = bin +m, G_{-m}(theta_k) = bin -m for m <= k, zero for m > k, so that the fold
// of Eq. (18) gives back the bins.  Thread = (row, signal), signal fastest: the four values of a
// row's signals are written side by side.
template <typename T>
__global__ void k_rings_to_table(int L, int64_t batch, const cplx_t<T> *__restrict__ bins, T *__restrict__ Gt) {
    const int64_t L2 = (int64_t)L * L;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L2 * batch) return;
    const int64_t row = t / batch, b = t - row * batch;
    const int m = (int)(row / L), k = (int)(row - (int64_t)m * L);
    T v[4] = {0, 0, 0, 0};
    if (m <= k) {
        const cplx_t<T> *r = bins + b * L2 + (int64_t)k * k + k;
        v[0] = r[m].x; v[1] = r[m].y;
        if (m > 0) { v[2] = r[-m].x; v[3] = r[-m].y; }
    }
    T *g = Gt + row * (4 * batch) + 4 * b;
#pragma unroll
    for (int q = 0; q < 4; ++q) g[q] = v[q];
}

}  // namespace

cudaError_t residual(int64_t n, const double2 *s_in, double2 *r, cudaStream_t s) {
    k_residual<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, s_in, r);
    return cudaGetLastError();
}

cudaError_t update_with_max(int64_t n, double2 *x, const double2 *dx, double *mx, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(double), s);
    if (e != cudaSuccess) return e;
    k_update_max<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, dx, (unsigned long long *)mx);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gather_alias_bins_t(int L, int m, int64_t batch, const T *W, T *U, cudaStream_t s) {
    int64_t n = (int64_t)m * batch;
    if (n <= 0) return cudaSuccess;
    k_gather_alias_bins<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, m, batch, W, U);
    return cudaGetLastError();
}
cudaError_t gather_alias_bins(int L, int m, int64_t batch, const double *W, double *U, cudaStream_t s) {
    return gather_alias_bins_t<double>(L, m, batch, W, U, s);
}
cudaError_t gather_alias_bins(int L, int m, int64_t batch, const float *W, float *U, cudaStream_t s) {
    return gather_alias_bins_t<float>(L, m, batch, W, U, s);
}

template <typename T>
cudaError_t coeffs_to_orders_t(int L, int64_t batch, const cplx_t<T> *coeffs, T *X, cudaStream_t s) {
    int64_t n = (int64_t)L * L * batch;
    k_coeffs_to_orders<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, batch, coeffs, X);
    return cudaGetLastError();
}
cudaError_t coeffs_to_orders(int L, int64_t batch, const double2 *coeffs, double *X, cudaStream_t s) {
    return coeffs_to_orders_t<double>(L, batch, coeffs, X, s);
}
cudaError_t coeffs_to_orders(int L, int64_t batch, const float2 *coeffs, float *X, cudaStream_t s) {
    return coeffs_to_orders_t<float>(L, batch, coeffs, X, s);
}

template <typename T>
cudaError_t orders_to_coeffs_t(int L, int64_t batch, const T *X, cplx_t<T> *coeffs, cudaStream_t s) {
    int64_t n = (int64_t)L * L * batch;
    k_orders_to_coeffs<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, batch, X, coeffs);
    return cudaGetLastError();
}
cudaError_t orders_to_coeffs(int L, int64_t batch, const double *X, double2 *coeffs, cudaStream_t s) {
    return orders_to_coeffs_t<double>(L, batch, X, coeffs, s);
}
cudaError_t orders_to_coeffs(int L, int64_t batch, const float *X, float2 *coeffs, cudaStream_t s) {
    return orders_to_coeffs_t<float>(L, batch, X, coeffs, s);
}

cudaError_t table_to_f32(const double *in, float *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t bins_to_rings_t(int L, int64_t batch, const T *W, cplx_t<T> *bins, cudaStream_t s) {
    const int64_t n = (int64_t)L * L * batch;
    k_bins_to_rings<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, batch, W, bins);
    return cudaGetLastError();
}
cudaError_t bins_to_rings(int L, int64_t batch, const double *W, double2 *bins, cudaStream_t s) {
    return bins_to_rings_t<double>(L, batch, W, bins, s);
}
cudaError_t bins_to_rings(int L, int64_t batch, const float *W, float2 *bins, cudaStream_t s) {
    return bins_to_rings_t<float>(L, batch, W, bins, s);
}

template <typename T>
cudaError_t rings_to_table_t(int L, int64_t batch, const cplx_t<T> *bins, T *Gt, cudaStream_t s) {
    const int64_t n = (int64_t)L * L * batch;
    k_rings_to_table<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L, batch, bins, Gt);
    return cudaGetLastError();
}
cudaError_t rings_to_table(int L, int64_t batch, const double2 *bins, double *Gt, cudaStream_t s) {
    return rings_to_table_t<double>(L, batch, bins, Gt, s);
}
cudaError_t rings_to_table(int L, int64_t batch, const float2 *bins, float *Gt, cudaStream_t s) {
    return rings_to_table_t<float>(L, batch, bins, Gt, s);
}

}  // namespace sht
