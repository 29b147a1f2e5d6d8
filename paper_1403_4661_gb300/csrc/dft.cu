// K1 / K5 / K7: ring DFTs of odd length N_k = 2k+1 and the order <-> bin fold, in float64 (and
// in float32 for SHT_F32 plans: the same kernels instantiated for float, with float32 copies of
// the twiddle, chirp and filter tables).
//
// Forward (Procedure 1, step 3; Eq. (11)): bin q in [-k, k] of ring k is
//     H_k[q] = (1/N_k) sum_n s_k[n] e^{-2 pi i q n / N_k} = sum_{m = q mod N_k, |m| < L} G_m(theta_k),
// so every ring is transformed once and the orders are separated later in bin space.
// Inverse (Procedure 2; Eq. (18)): s_k[n] = sum_m G_m(theta_k) e^{i m phi_n}; orders congruent mod
// N_k meet at the same sample values, so they are first folded into the N_k bins and one inverse
// DFT of length N_k per ring finishes the sum.
//
// Ring lengths are odd and often prime.  Rings with N <= kDirectMaxN are transformed directly
// (O(N^2), twiddles from a per-ring table of N roots).  Longer rings use Bluestein's chirp-z
// identity  j n = (j^2 + n^2 - (j - n)^2) / 2: with c_n = e^{-i pi n^2 / N},
//     X_j = c_j sum_n (x_n c_n) conj(c_{j-n}),
// a linear convolution computed as a cyclic one of power-of-two length M >= 2N - 1 with a radix-2
// FFT held in shared memory (one thread block per ring and signal).  c_n is evaluated from the
// exactly reduced integer n^2 mod 2N, so no twiddle carries an argument-reduction error.
// Rings are launched in classes k in [2^j, 2^(j+1)), which share M = 2^(j+3).
#include "sht_internal.cuh"

namespace sht {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
template <typename C> __device__ __forceinline__ C conjd(C a) { a.y = -a.y; return a; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
__device__ __forceinline__ void sincospi_t(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ void sincospi_t(float x, float *s, float *c) { sincospif(x, s, c); }

// In-place decimation-in-time FFT of a[0..M) in shared memory, natural-order input and output:
// bit-reversal permutation, then the radix-2 stages taken two at a time as radix-4 butterflies
// (stages s, s+1 with half-width h share the twiddle u = W_{4h}^j: the four outputs need u x2,
// u^2 x1, u^3 x3 and the factor W_{4h}^h = -i, i.e. 3 complex products instead of 4), plus one
// radix-2 stage of twiddle 1 when log2 M is odd.  tw[t] = e^{-2 pi i t / Mmax}, t < Mmax;
// inverse = conjugate twiddles, unnormalised.
template <typename C>
__device__ void block_fft(C *a, int M, int logM, const C *__restrict__ tw, int Mmax, bool inverse) {
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        int j = (int)(__brev((unsigned)i) >> (32 - logM));
        if (i < j) { C t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    __syncthreads();
    int s = 1;
    if (logM & 1) {
        for (int t = threadIdx.x; t < (M >> 1); t += blockDim.x) {
            const C u = a[2 * t], v = a[2 * t + 1];
            a[2 * t] = cadd(u, v);
            a[2 * t + 1] = csub(u, v);
        }
        __syncthreads();
        s = 2;
    }
    for (; s < logM; s += 2) {
        const int h = 1 << (s - 1);
        const int stride = Mmax >> (s + 1);   // u = W_{4h}^j = tw[j * stride]
        for (int t = threadIdx.x; t < (M >> 2); t += blockDim.x) {
            const int j = t & (h - 1);
            const int i0 = ((t >> (s - 1)) << (s + 1)) + j;
            const C x0 = a[i0], x1 = a[i0 + h], x2 = a[i0 + 2 * h], x3 = a[i0 + 3 * h];
            C t1 = x1, t2 = x2, t3 = x3;
            if (h > 1) {   // h == 1: j == 0, every twiddle is 1
                C u = __ldg(&tw[j * stride]), u2 = __ldg(&tw[2 * j * stride]), u3 = __ldg(&tw[3 * j * stride]);
                if (inverse) { u.y = -u.y; u2.y = -u2.y; u3.y = -u3.y; }
                t1 = cmul(x1, u2);
                t2 = cmul(x2, u);
                t3 = cmul(x3, u3);
            }
            const C A = cadd(x0, t1), Bm = csub(x0, t1), Cs = cadd(t2, t3), D = csub(t2, t3);
            a[i0] = cadd(A, Cs);
            a[i0 + 2 * h] = csub(A, Cs);
            C o1 = Bm, o3 = Bm;
            if (!inverse) {   // W_{4h}^h = -i
                o1.x += D.y; o1.y -= D.x;
                o3.x -= D.y; o3.y += D.x;
            } else {          // +i
                o1.x -= D.y; o1.y += D.x;
                o3.x += D.y; o3.y -= D.x;
            }
            a[i0 + h] = o1;
            a[i0 + 3 * h] = o3;
        }
        __syncthreads();
    }
}

__global__ void k_twiddle(double2 *tw, int Mmax) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Mmax) return;
    double s, c;
    sincospi(2.0 * (double)t / (double)Mmax, &s, &c);
    tw[t] = make_double2(c, -s);
}

__global__ void k_chirp(double2 *chirp, int L) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= (int64_t)L * L) return;
    int k = (int)sqrt((double)j);
    while ((int64_t)k * k > j) --k;
    while ((int64_t)(k + 1) * (k + 1) <= j) ++k;
    int64_t n = j - (int64_t)k * k, N = 2 * k + 1;
    int64_t r = (n * n) % (2 * N);
    double s, c;
    sincospi((double)r / (double)N, &s, &c);
    chirp[j] = make_double2(c, -s);  // e^{-i pi r / N}
}

// float64 table -> float32 copy (SHT_F32 plans)
__global__ void k_to_f32c(const double2 *__restrict__ in, float2 *__restrict__ out, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = make_float2((float)in[t].x, (float)in[t].y);
}

// Filter of ring k: FFT_M of b_t = conj(c_t) (t < N), b_{M-t} = conj(c_t) (0 < t < N), scaled 1/M.
__global__ void k_filter(int k0, const double2 *__restrict__ chirp, const int64_t *__restrict__ foff,
                         const int *__restrict__ fM, const double2 *__restrict__ tw, int Mmax,
                         double2 *__restrict__ filt) {
    extern __shared__ double2 sa[];
    const int k = k0 + blockIdx.x;
    const int N = 2 * k + 1, M = fM[k];
    int logM = 31 - __clz(M);
    const double2 *c = chirp + (int64_t)k * k;
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        if (t < N) v = conjd(c[t]);
        else if (t > M - N) v = conjd(c[M - t]);
        sa[t] = v;
    }
    __syncthreads();
    block_fft(sa, M, logM, tw, Mmax, false);
    const double sc = 1.0 / (double)M;
    for (int t = threadIdx.x; t < M; t += blockDim.x)
        filt[foff[k] + t] = make_double2(sa[t].x * sc, sa[t].y * sc);
}

enum OutMode : int { OUT_BINS = 0, OUT_UNFOLD = 1 };
enum InMode : int { IN_FOLD = 0, IN_BINS = 1 };

template <typename T>
struct DftArgs {
    int L, k0;
    int64_t Nc;             // 4 * batch columns of the order-major buffers
    const cplx_t<T> *chirp, *filt, *tw;
    const int64_t *foff;
    int Mmax, M, logM;
};

// Forward DFT of ring k = k0 + blockIdx.x of signal b = blockIdx.y.
//  OUT_BINS:   W rows of bins +-q (scaled 1/N)           - forward transform
//  OUT_UNFOLD: Gt rows (|m|, k) for every |m| < L, value of bin alias_k(m) (unscaled)
//              - adjoint of fold_ring_idft
template <typename T, int OUT>
__global__ void k_ring_dft(DftArgs<T> d, const cplx_t<T> *__restrict__ samples, T *__restrict__ out) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sa = reinterpret_cast<C *>(smem_raw);
    const int k = d.k0 + blockIdx.x, b = blockIdx.y, L = d.L;
    const int N = 2 * k + 1;
    const C *x = samples + (int64_t)b * L * L + (int64_t)k * k;
    C *X;  // natural-order DFT, N values
    if (d.M == 0) {
        C *xs = sa, *roots = sa + N;
        X = sa + 2 * N;
        for (int t = threadIdx.x; t < N; t += blockDim.x) {
            xs[t] = x[t];
            T s, c;
            sincospi_t((T)2 * (T)t / (T)N, &s, &c);
            roots[t] = mk2<T>(c, -s);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            C acc = mk2<T>(0, 0);
            int idx = 0;
            for (int n = 0; n < N; ++n) {
                C p = cmul(xs[n], roots[idx]);
                acc.x += p.x; acc.y += p.y;
                idx += j; if (idx >= N) idx -= N;
            }
            X[j] = acc;
        }
        __syncthreads();
    } else {
        const C *c = d.chirp + (int64_t)k * k;
        const C *f = d.filt + d.foff[k];
        for (int t = threadIdx.x; t < d.M; t += blockDim.x)
            sa[t] = (t < N) ? cmul(x[t], c[t]) : mk2<T>(0, 0);
        __syncthreads();
        block_fft(sa, d.M, d.logM, d.tw, d.Mmax, false);
        for (int t = threadIdx.x; t < d.M; t += blockDim.x) sa[t] = cmul(sa[t], f[t]);
        __syncthreads();
        block_fft(sa, d.M, d.logM, d.tw, d.Mmax, true);
        for (int t = threadIdx.x; t < N; t += blockDim.x) sa[t] = cmul(c[t], sa[t]);
        __syncthreads();
        X = sa;
    }
    if (OUT == OUT_BINS) {
        const T sc = (T)1 / (T)N;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            const int q = (j <= k) ? j : j - N;
            const int o = q < 0 ? -q : q;
            T *w = out + (rows_off(L, o) + (k - o)) * d.Nc + 4 * b;
            C v = X[j];
            if (q >= 0) { w[0] = v.x * sc; w[1] = v.y * sc; }
            else        { w[2] = v.x * sc; w[3] = v.y * sc; }
            if (q == 0) { w[2] = 0; w[3] = 0; }
        }
    } else {
        for (int m = -(L - 1) + (int)threadIdx.x; m <= L - 1; m += blockDim.x) {
            int q = alias_bin(m, k);
            int j = q >= 0 ? q : q + N;
            int o = m < 0 ? -m : m;
            T *g = out + ((int64_t)o * L + k) * d.Nc + 4 * b;
            C v = X[j];
            if (m >= 0) { g[0] = v.x; g[1] = v.y; }
            else        { g[2] = v.x; g[3] = v.y; }
            if (m == 0) { g[2] = 0; g[3] = 0; }
        }
    }
}

// Inverse DFT of ring k of signal b: gathers the ring's N bins, then s_n = sum_j B_j e^{+2 pi i jn/N}.
//  IN_FOLD: B_q = sum_{m = q mod N, |m| < L} Gt[(|m|, k)]             - inverse transform
//  IN_BINS: B_q = W[bin q of ring k] / N                              - adjoint of the forward DFT
template <typename T, int IN>
__global__ void k_ring_idft(DftArgs<T> d, const T *__restrict__ in, cplx_t<T> *__restrict__ samples) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sa = reinterpret_cast<C *>(smem_raw);
    const int k = d.k0 + blockIdx.x, b = blockIdx.y, L = d.L;
    const int N = 2 * k + 1;
    C *B = sa;  // natural-order bins
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const int q = (j <= k) ? j : j - N;
        C acc = mk2<T>(0, 0);
        if (IN == IN_FOLD) {
            int m = q - ((q + L - 1) / N) * N;
            for (; m <= L - 1; m += N) {
                const int o = m < 0 ? -m : m;
                const T *g = in + ((int64_t)o * L + k) * d.Nc + 4 * b + (m < 0 ? 2 : 0);
                acc.x += g[0];
                acc.y += g[1];
            }
        } else {
            const int o = q < 0 ? -q : q;
            const T *w = in + (rows_off(L, o) + (k - o)) * d.Nc + 4 * b + (q < 0 ? 2 : 0);
            const T sc = (T)1 / (T)N;
            acc = mk2<T>(w[0] * sc, w[1] * sc);
        }
        B[j] = acc;
    }
    __syncthreads();
    C *y = samples + (int64_t)b * L * L + (int64_t)k * k;
    if (d.M == 0) {
        C *roots = sa + N;
        for (int t = threadIdx.x; t < N; t += blockDim.x) {
            T s, c;
            sincospi_t((T)2 * (T)t / (T)N, &s, &c);
            roots[t] = mk2<T>(c, s);  // e^{+2 pi i t / N}
        }
        __syncthreads();
        for (int n = threadIdx.x; n < N; n += blockDim.x) {
            C acc = mk2<T>(0, 0);
            int idx = 0;
            for (int j = 0; j < N; ++j) {
                C p = cmul(B[j], roots[idx]);
                acc.x += p.x; acc.y += p.y;
                idx += n; if (idx >= N) idx -= N;
            }
            y[n] = acc;
        }
    } else {
        // y = conj(DFT(conj(B))) with the forward chirp machinery
        const C *c = d.chirp + (int64_t)k * k;
        const C *f = d.filt + d.foff[k];
        for (int t = threadIdx.x; t < d.M; t += blockDim.x)
            sa[t] = (t < N) ? cmul(conjd(sa[t]), c[t]) : mk2<T>(0, 0);
        __syncthreads();
        block_fft(sa, d.M, d.logM, d.tw, d.Mmax, false);
        for (int t = threadIdx.x; t < d.M; t += blockDim.x) sa[t] = cmul(sa[t], f[t]);
        __syncthreads();
        block_fft(sa, d.M, d.logM, d.tw, d.Mmax, true);
        for (int t = threadIdx.x; t < N; t += blockDim.x) y[t] = conjd(cmul(c[t], sa[t]));
    }
}

int ilog2(int x) { int r = 0; while ((1 << r) < x) ++r; return r; }

// Ring classes: direct rings k < 32 (N <= 63), then k in [2^j, 2^(j+1)) with M = 2^(j+3).
template <typename F>
cudaError_t for_each_class(int L, F &&fn) {
    int kd = L < 32 ? L : 32;
    cudaError_t e = fn(0, kd, 0);
    if (e != cudaSuccess) return e;
    for (int j = 5; (1 << j) < L; ++j) {
        int k0 = 1 << j, k1 = (1 << (j + 1)) < L ? (1 << (j + 1)) : L;
        e = fn(k0, k1 - k0, 1 << (j + 3));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
DftArgs<T> make_args(int L, const DftPlan &dp, int64_t batch, int k0, int M) {
    DftArgs<T> d{};
    d.L = L; d.k0 = k0; d.Nc = 4 * batch;
    if constexpr (sizeof(T) == 8) {
        d.chirp = dp.chirp; d.filt = dp.filt; d.tw = dp.twiddle;
    } else {
        d.chirp = dp.chirp_f; d.filt = dp.filt_f; d.tw = dp.twiddle_f;
    }
    d.foff = dp.filt_off;
    d.Mmax = dp.Mmax; d.M = M; d.logM = M ? ilog2(M) : 0;
    return d;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Raise the dynamic shared-memory limit of the ring kernels once, at plan time, so that the
// transform calls themselves make no attribute calls (they may run under stream capture).
template <typename T>
cudaError_t set_ring_kernel_limits_t(int Mmax) {
    const size_t b = sizeof(cplx_t<T>) * (size_t)Mmax;
    cudaError_t e;
    if ((e = set_smem(k_ring_dft<T, OUT_BINS>, b)) != cudaSuccess) return e;
    if ((e = set_smem(k_ring_dft<T, OUT_UNFOLD>, b)) != cudaSuccess) return e;
    if ((e = set_smem(k_ring_idft<T, IN_FOLD>, b)) != cudaSuccess) return e;
    return set_smem(k_ring_idft<T, IN_BINS>, b);
}
cudaError_t set_ring_kernel_limits(int Mmax) { return set_ring_kernel_limits_t<double>(Mmax); }

template <typename T>
size_t smem_bytes(int k0, int cnt, int M) {
    if (M == 0) { int N = 2 * (k0 + cnt - 1) + 1; return sizeof(cplx_t<T>) * 3 * (size_t)N; }
    return sizeof(cplx_t<T>) * (size_t)M;
}

}  // namespace

cudaError_t dft_plan_create(int L, DftPlan &dp, uint64_t &bytes, cudaStream_t s) {
    int Mmax = 2;
    for (int j = 5; (1 << j) < L; ++j) Mmax = 1 << (j + 3);
    dp.Mmax = Mmax;
    dp.h_filt_off.assign(L, -1);
    dp.h_filt_M.assign(L, 0);
    int64_t total = 0;
    for (int k = 32; k < L; ++k) {
        int N = 2 * k + 1, M = 1 << ilog2(2 * N - 1);
        dp.h_filt_off[k] = total;
        dp.h_filt_M[k] = M;
        total += M;
    }
    cudaError_t e;
    size_t b_tw = sizeof(double2) * Mmax, b_ch = sizeof(double2) * (size_t)L * L;
    size_t b_f = sizeof(double2) * (size_t)(total > 0 ? total : 1);
    if ((e = cudaMalloc(&dp.twiddle, b_tw)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&dp.chirp, b_ch)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&dp.filt, b_f)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&dp.filt_off, sizeof(int64_t) * L)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&dp.filt_M, sizeof(int) * L)) != cudaSuccess) return e;
    bytes = b_tw + b_ch + b_f + sizeof(int64_t) * L + sizeof(int) * L;
    dp.filt_total = total;
    cudaMemcpyAsync(dp.filt_off, dp.h_filt_off.data(), sizeof(int64_t) * L, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dp.filt_M, dp.h_filt_M.data(), sizeof(int) * L, cudaMemcpyHostToDevice, s);
    k_twiddle<<<(Mmax + 255) / 256, 256, 0, s>>>(dp.twiddle, Mmax);
    int64_t LL = (int64_t)L * L;
    k_chirp<<<(unsigned)((LL + 255) / 256), 256, 0, s>>>(dp.chirp, L);
    if ((e = set_ring_kernel_limits(Mmax)) != cudaSuccess) return e;
    if (L > 32) {
        if ((e = set_smem(k_filter, sizeof(double2) * Mmax)) != cudaSuccess) return e;
        e = for_each_class(L, [&](int k0, int cnt, int M) -> cudaError_t {
            if (M == 0 || cnt <= 0) return cudaSuccess;
            k_filter<<<cnt, 256, sizeof(double2) * M, s>>>(k0, dp.chirp, dp.filt_off, dp.filt_M,
                                                          dp.twiddle, Mmax, dp.filt);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t dft_plan_make_f32(int L, DftPlan &dp, uint64_t &bytes, cudaStream_t s) {
    const int64_t n_tw = dp.Mmax, n_ch = (int64_t)L * L, n_f = dp.filt_total > 0 ? dp.filt_total : 1;
    cudaError_t e;
    if ((e = cudaMalloc(&dp.twiddle_f, sizeof(float2) * n_tw)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&dp.chirp_f, sizeof(float2) * n_ch)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&dp.filt_f, sizeof(float2) * n_f)) != cudaSuccess) return e;
    bytes = sizeof(float2) * (n_tw + n_ch + n_f);
    k_to_f32c<<<(unsigned)((n_tw + 255) / 256), 256, 0, s>>>(dp.twiddle, dp.twiddle_f, n_tw);
    k_to_f32c<<<(unsigned)((n_ch + 255) / 256), 256, 0, s>>>(dp.chirp, dp.chirp_f, n_ch);
    if (dp.filt_total > 0)
        k_to_f32c<<<(unsigned)((n_f + 255) / 256), 256, 0, s>>>(dp.filt, dp.filt_f, n_f);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return set_ring_kernel_limits_t<float>(dp.Mmax);
}

void dft_plan_destroy(DftPlan &dp) {
    cudaFree(dp.twiddle_f); cudaFree(dp.chirp_f); cudaFree(dp.filt_f);
    cudaFree(dp.twiddle); cudaFree(dp.chirp); cudaFree(dp.filt);
    cudaFree(dp.filt_off); cudaFree(dp.filt_M);
    dp = DftPlan{};
}

template <typename T, int OUT>
static cudaError_t ring_dft_impl(int L, const DftPlan &dp, const cplx_t<T> *samples, T *out,
                                 int64_t batch, cudaStream_t s) {
    return for_each_class(L, [&](int k0, int cnt, int M) -> cudaError_t {
        if (cnt <= 0) return cudaSuccess;
        size_t sm = smem_bytes<T>(k0, cnt, M);
        dim3 grid(cnt, (unsigned)batch);
        k_ring_dft<T, OUT><<<grid, M == 0 ? 64 : 256, sm, s>>>(make_args<T>(L, dp, batch, k0, M), samples, out);
        return cudaGetLastError();
    });
}

template <typename T, int IN>
static cudaError_t ring_idft_impl(int L, const DftPlan &dp, const T *in, cplx_t<T> *samples,
                                  int64_t batch, cudaStream_t s) {
    return for_each_class(L, [&](int k0, int cnt, int M) -> cudaError_t {
        if (cnt <= 0) return cudaSuccess;
        size_t sm = smem_bytes<T>(k0, cnt, M);
        dim3 grid(cnt, (unsigned)batch);
        k_ring_idft<T, IN><<<grid, M == 0 ? 64 : 256, sm, s>>>(make_args<T>(L, dp, batch, k0, M), in, samples);
        return cudaGetLastError();
    });
}

cudaError_t ring_dft_to_bins(int L, const DftPlan &dp, const double2 *samples, double *W,
                             int64_t batch, bool, cudaStream_t s) {
    return ring_dft_impl<double, OUT_BINS>(L, dp, samples, W, batch, s);
}
cudaError_t ring_dft_unfold(int L, const DftPlan &dp, const double2 *samples, double *Gt,
                            int64_t batch, cudaStream_t s) {
    return ring_dft_impl<double, OUT_UNFOLD>(L, dp, samples, Gt, batch, s);
}
cudaError_t fold_ring_idft(int L, const DftPlan &dp, const double *Gt, double2 *samples,
                           int64_t batch, cudaStream_t s) {
    return ring_idft_impl<double, IN_FOLD>(L, dp, Gt, samples, batch, s);
}
cudaError_t bins_to_ring_adjoint(int L, const DftPlan &dp, const double *W, double2 *samples,
                                 int64_t batch, cudaStream_t s) {
    return ring_idft_impl<double, IN_BINS>(L, dp, W, samples, batch, s);
}

cudaError_t ring_dft_to_bins(int L, const DftPlan &dp, const float2 *samples, float *W,
                             int64_t batch, bool, cudaStream_t s) {
    return ring_dft_impl<float, OUT_BINS>(L, dp, samples, W, batch, s);
}
cudaError_t ring_dft_unfold(int L, const DftPlan &dp, const float2 *samples, float *Gt,
                            int64_t batch, cudaStream_t s) {
    return ring_dft_impl<float, OUT_UNFOLD>(L, dp, samples, Gt, batch, s);
}
cudaError_t fold_ring_idft(int L, const DftPlan &dp, const float *Gt, float2 *samples,
                           int64_t batch, cudaStream_t s) {
    return ring_idft_impl<float, IN_FOLD>(L, dp, Gt, samples, batch, s);
}
cudaError_t bins_to_ring_adjoint(int L, const DftPlan &dp, const float *W, float2 *samples,
                                 int64_t batch, cudaStream_t s) {
    return ring_idft_impl<float, IN_BINS>(L, dp, W, samples, batch, s);
}

}  // namespace sht
