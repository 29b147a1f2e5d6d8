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
// (O(N^2)).  Longer rings use Bluestein's chirp-z identity  j n = (j^2 + n^2 - (j - n)^2) / 2:
// with c_n = e^{-i pi n^2 / N},
//     X_j = c_j sum_n (x_n c_n) conj(c_{j-n}),
// a linear convolution computed as a cyclic one of length M >= 2N - 1, the smallest M of the
// form 2^a or 3 * 2^a (c_n is evaluated from the exactly reduced integer n^2 mod 2N).  On GB300
// these kernels are bound by the float64 pipe (one FP64 instruction per 64 cycles per scheduler;
// an add costs as much as an FMA), so the design minimises float64 instructions:
//   * the forward FFT is decimation-in-frequency (natural order in, digit-reversed order out),
//     the filter FFT(conj c) is stored in that digit-reversed order, and the inverse FFT is the
//     matching decimation-in-time network (digit-reversed in, natural out): no permutation pass;
//   * radix-4 stages, then a radix-2 and / or radix-3 stage (3 * 2^a lengths cut M by up to 25 %);
//   * the input holds N <= M/2 values, so the first stage's radix-4 butterflies have two zero
//     inputs; only N <= M/2 outputs are needed, so the last stage computes two of its four;
//   * the chirp premultiply and the fold (or sample load) are fused into the first stage, the
//     filter product into the last forward stage, the chirp postmultiply and the output layout
//     into the last inverse stage; one __syncthreads per stage, data in shared memory.
// Rings are launched in classes of consecutive k sharing M.
#include <algorithm>

#include "fft_device.cuh"

namespace sht {
namespace {

using namespace fft;

__global__ void k_twiddle(double2 *tw, int Mtab) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Mtab) return;
    double s, c;
    sincospi(2.0 * (double)t / (double)Mtab, &s, &c);
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

// Filter of ring k0 + blockIdx.x, stored in the forward FFT's (digit-reversed) output order:
// DIF-FFT_M of b_t = conj(c_t) (t < N), b_{M-t} = conj(c_t) (0 < t < N), scaled 1/M.
__global__ void k_filter(int k0, int M, Stages st, const double2 *__restrict__ chirp, const double2 *__restrict__ tw,
                         int Mtab, double2 *__restrict__ filt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *a = reinterpret_cast<double2 *>(smem_raw);
    const int k = k0 + blockIdx.x;
    const int N = 2 * k + 1;
    const double2 *c = chirp + (int64_t)k * k;
    for (int t = threadIdx.x; t < M; t += blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        if (t < N) v = conjd(c[t]);
        else if (t > M - N) v = conjd(c[M - t]);
        a[t] = v;
    }
    __syncthreads();
    for (int s = 0; s < st.n; ++s) {
        dif_stage(a, M, st.S[s], st.R[s], tw, Mtab, (const double2 *)nullptr);
        __syncthreads();
    }
    const double sc = 1.0 / (double)M;
    double2 *f = filt + (int64_t)blockIdx.x * M;
    for (int t = threadIdx.x; t < M; t += blockDim.x) f[t] = make_double2(a[t].x * sc, a[t].y * sc);
}

enum OutMode : int { OUT_BINS = 0, OUT_UNFOLD = 1 };
enum InMode : int { IN_FOLD = 0, IN_BINS = 1 };

template <typename T>
struct DftArgs {
    int L, k0;
    int64_t Nc;             // 4 * batch columns of the order-major buffers
    const cplx_t<T> *chirp, *filt, *tw;
    int Mtab, M;            // M = 0: direct rings
    Stages st;
};

// Store of one forward-transform value X_t (bin q = t or t - N) of ring k, signal b.
//  OUT_BINS:   W rows of bins +-q (scaled 1/N)           - forward transform
//  OUT_UNFOLD: Gt rows (|m|, k) for every |m| < L with m = q mod N (unscaled)
//              - adjoint of fold_ring_idft
template <typename T, int OUT>
__device__ __forceinline__ void store_bin(const DftArgs<T> &d, T *__restrict__ out, int k, int b, int t, cplx_t<T> v) {
    const int N = 2 * k + 1, L = d.L;
    const int q = (t <= k) ? t : t - N;
    if (OUT == OUT_BINS) {
        const T sc = (T)1 / (T)N;
        const int o = q < 0 ? -q : q;
        T *w = out + (rows_off(L, o) + (k - o)) * d.Nc + 4 * b;
        if (q >= 0) { w[0] = v.x * sc; w[1] = v.y * sc; }
        else        { w[2] = v.x * sc; w[3] = v.y * sc; }
        if (q == 0) { w[2] = 0; w[3] = 0; }
    } else {
        // every order m = q + j N with |m| < L
        int m = q - ((q + L - 1) / N) * N;
        for (; m <= L - 1; m += N) {
            const int o = m < 0 ? -m : m;
            T *g = out + ((int64_t)o * L + k) * d.Nc + 4 * b;
            if (m >= 0) { g[0] = v.x; g[1] = v.y; }
            else        { g[2] = v.x; g[3] = v.y; }
            if (m == 0) { g[2] = 0; g[3] = 0; }
        }
    }
}

// Bin value B_t of ring k, signal b, for the inverse direction.
//  IN_FOLD: B_q = sum_{m = q mod N, |m| < L} Gt[(|m|, k)]             - inverse transform
//  IN_BINS: B_q = W[bin q of ring k] / N                              - adjoint of the forward DFT
template <typename T, int IN>
__device__ __forceinline__ cplx_t<T> load_bin(const DftArgs<T> &d, const T *__restrict__ in, int k, int b, int t) {
    const int N = 2 * k + 1, L = d.L;
    const int q = (t <= k) ? t : t - N;
    if (IN == IN_FOLD) {
        // the orders of bin q, four loads in flight per step
        const int m0 = q - ((q + L - 1) / N) * N;
        T ax = 0, ay = 0;
        int m = m0;
        for (; m + 3 * N <= L - 1; m += 4 * N) {
            T x[4], y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int mm = m + u * N, o = mm < 0 ? -mm : mm;
                const T *g = in + ((int64_t)o * L + k) * d.Nc + 4 * b + (mm < 0 ? 2 : 0);
                x[u] = g[0];
                y[u] = g[1];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) { ax += x[u]; ay += y[u]; }
        }
        for (; m <= L - 1; m += N) {
            const int o = m < 0 ? -m : m;
            const T *g = in + ((int64_t)o * L + k) * d.Nc + 4 * b + (m < 0 ? 2 : 0);
            ax += g[0];
            ay += g[1];
        }
        return mk2<T>(ax, ay);
    } else {
        const int o = q < 0 ? -q : q;
        const T *w = in + (rows_off(L, o) + (k - o)) * d.Nc + 4 * b + (q < 0 ? 2 : 0);
        const T sc = (T)1 / (T)N;
        return mk2<T>(w[0] * sc, w[1] * sc);
    }
}

// Forward DFT of ring k = k0 + blockIdx.x of signal b = blockIdx.y into the order-major layout.
template <typename T, int OUT>
__global__ void __launch_bounds__(kThreads) k_ring_dft(DftArgs<T> d, const cplx_t<T> *__restrict__ samples,
                                                       T *__restrict__ out) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sa = reinterpret_cast<C *>(smem_raw);
    const int k = d.k0 + blockIdx.x, b = blockIdx.y, L = d.L;
    const int N = 2 * k + 1;
    const C *x = samples + (int64_t)b * L * L + (int64_t)k * k;
    if (d.M == 0) {
        C *xs = sa, *roots = sa + N;
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
            store_bin<T, OUT>(d, out, k, b, j, acc);
        }
        return;
    }
    const C *c = d.chirp + (int64_t)k * k;
    const C *f = d.filt + (int64_t)blockIdx.x * d.M;
    bluestein(sa, N, d.M, d.st, d.tw, d.Mtab, c, f,
              [&](int t) { return x[t]; },
              [&](int t, C v) { store_bin<T, OUT>(d, out, k, b, t, v); });
}

// Inverse DFT of ring k of signal b: s_n = sum_j B_j e^{+2 pi i jn/N} with the bins B of load_bin.
template <typename T, int IN>
__global__ void __launch_bounds__(kThreads) k_ring_idft(DftArgs<T> d, const T *__restrict__ in,
                                                        cplx_t<T> *__restrict__ samples) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *sa = reinterpret_cast<C *>(smem_raw);
    const int k = d.k0 + blockIdx.x, b = blockIdx.y, L = d.L;
    const int N = 2 * k + 1;
    C *y = samples + (int64_t)b * L * L + (int64_t)k * k;
    if (d.M == 0) {
        // direct ring: the N bins (each summed by a group of threads), then the direct sum
        C *B = sa, *roots = sa + N, *part = sa + 2 * N;
        if (IN == IN_FOLD) {
            // bin q = t mod N, thread group g = t / N sums the orders of q with index = g mod G
            const int G = max(1, (int)blockDim.x / N);
            for (int t = threadIdx.x; t < N * G; t += blockDim.x) {
                const int j = t % N, g = t / N;
                const int q = (j <= k) ? j : j - N;
                int m = q - ((q + L - 1) / N) * N + g * N;
                T ax = 0, ay = 0;
                for (; m + 3 * G * N <= L - 1; m += 4 * G * N) {
                    T xv[4], yv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int mm = m + u * G * N, o = mm < 0 ? -mm : mm;
                        const T *gp = in + ((int64_t)o * L + k) * d.Nc + 4 * b + (mm < 0 ? 2 : 0);
                        xv[u] = gp[0];
                        yv[u] = gp[1];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) { ax += xv[u]; ay += yv[u]; }
                }
                for (; m <= L - 1; m += G * N) {
                    const int o = m < 0 ? -m : m;
                    const T *gp = in + ((int64_t)o * L + k) * d.Nc + 4 * b + (m < 0 ? 2 : 0);
                    ax += gp[0];
                    ay += gp[1];
                }
                part[t] = mk2<T>(ax, ay);
            }
            __syncthreads();
            for (int j = threadIdx.x; j < N; j += blockDim.x) {
                C acc = part[j];
                for (int g = 1; g < G; ++g) acc = cadd(acc, part[g * N + j]);
                B[j] = acc;
            }
        } else {
            for (int j = threadIdx.x; j < N; j += blockDim.x) B[j] = load_bin<T, IN>(d, in, k, b, j);
        }
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
        return;
    }
    // y = conj(DFT(conj(B))) with the forward chirp machinery
    const C *c = d.chirp + (int64_t)k * k;
    const C *f = d.filt + (int64_t)blockIdx.x * d.M;
    bluestein(sa, N, d.M, d.st, d.tw, d.Mtab, c, f,
              [&](int t) { return conjd(load_bin<T, IN>(d, in, k, b, t)); },
              [&](int t, C v) { y[t] = conjd(v); });
}

template <typename T>
DftArgs<T> make_args(int L, const DftPlan &dp, int64_t batch, const RingClass &rc) {
    DftArgs<T> d{};
    d.L = L; d.k0 = rc.k0; d.Nc = 4 * batch;
    if constexpr (sizeof(T) == 8) {
        d.chirp = dp.chirp; d.filt = dp.filt + rc.filt_off; d.tw = dp.twiddle;
    } else {
        d.chirp = dp.chirp_f; d.filt = dp.filt_f + rc.filt_off; d.tw = dp.twiddle_f;
    }
    d.Mtab = dp.Mtab; d.M = rc.M;
    d.st = rc.M ? stages_of(rc.M) : Stages{};
    return d;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Shared memory of a class's blocks: M complex values (chirp-z), or the direct rings' bins,
// roots and fold partials.
template <typename T>
size_t smem_bytes(const RingClass &rc) {
    if (rc.M == 0) {
        const int N = 2 * (rc.k0 + rc.cnt - 1) + 1;
        return sizeof(cplx_t<T>) * ((size_t)2 * N + (size_t)std::max(N, kThreads));
    }
    return sizeof(cplx_t<T>) * (size_t)rc.M;
}

// Raise the dynamic shared-memory limit of the ring kernels once, at plan time, so that the
// transform calls themselves make no attribute calls (they may run under stream capture).
template <typename T>
cudaError_t set_ring_kernel_limits_t(int Mmax) {
    const size_t b = sizeof(cplx_t<T>) * (size_t)std::max(Mmax, 3 * 64);
    cudaError_t e;
    if ((e = set_smem(k_ring_dft<T, OUT_BINS>, b)) != cudaSuccess) return e;
    if ((e = set_smem(k_ring_dft<T, OUT_UNFOLD>, b)) != cudaSuccess) return e;
    if ((e = set_smem(k_ring_idft<T, IN_FOLD>, b)) != cudaSuccess) return e;
    return set_smem(k_ring_idft<T, IN_BINS>, b);
}

}  // namespace

cudaError_t dft_plan_create(int L, DftPlan &dp, uint64_t &bytes, cudaStream_t s) {
    // ring classes: the direct rings, then runs of consecutive k sharing the chirp-z length
    dp.classes.clear();
    const int kd = std::min(L, (kDirectMaxN + 1) / 2);
    dp.classes.push_back(RingClass{0, kd, 0, 0});
    int Mmax = 0;
    int64_t total = 0;
    for (int k = kd; k < L; ++k) {
        const int M = bluestein_length(2 * k + 1);
        if (dp.classes.back().M != M) dp.classes.push_back(RingClass{k, 0, M, total});
        dp.classes.back().cnt += 1;
        total += M;
        Mmax = std::max(Mmax, M);
    }
    dp.Mmax = Mmax;
    // twiddle table length: a multiple of every 2^a and 3 * 2^a length used
    int p2 = 16;
    while (p2 < Mmax) p2 <<= 1;
    dp.Mtab = 3 * p2;
    dp.filt_total = total;
    cudaError_t e;
    const size_t b_tw = sizeof(double2) * dp.Mtab, b_ch = sizeof(double2) * (size_t)L * L;
    const size_t b_f = sizeof(double2) * (size_t)(total > 0 ? total : 1);
    if ((e = cudaMalloc(&dp.twiddle, b_tw)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&dp.chirp, b_ch)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&dp.filt, b_f)) != cudaSuccess) return e;
    bytes = b_tw + b_ch + b_f;
    {   // per-ring length and filter offset, for kernels that walk rings of several plans
        std::vector<int> rm((size_t)L, 0);
        std::vector<int64_t> rf((size_t)L, -1);
        for (const RingClass &rc : dp.classes)
            for (int i = 0; i < rc.cnt; ++i) {
                rm[(size_t)(rc.k0 + i)] = rc.M;
                if (rc.M) rf[(size_t)(rc.k0 + i)] = rc.filt_off + (int64_t)i * rc.M;
            }
        if ((e = cudaMalloc(&dp.d_ring_M, sizeof(int) * L)) != cudaSuccess) return e;
        if ((e = cudaMalloc(&dp.d_ring_foff, sizeof(int64_t) * L)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(dp.d_ring_M, rm.data(), sizeof(int) * L, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dp.d_ring_foff, rf.data(), sizeof(int64_t) * L, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return e;
        bytes += (sizeof(int) + sizeof(int64_t)) * (uint64_t)L;
    }
    k_twiddle<<<(dp.Mtab + 255) / 256, 256, 0, s>>>(dp.twiddle, dp.Mtab);
    const int64_t LL = (int64_t)L * L;
    k_chirp<<<(unsigned)((LL + 255) / 256), 256, 0, s>>>(dp.chirp, L);
    if ((e = set_ring_kernel_limits_t<double>(Mmax)) != cudaSuccess) return e;
    if ((e = set_smem(k_filter, sizeof(double2) * (size_t)std::max(Mmax, 16))) != cudaSuccess) return e;
    for (const RingClass &rc : dp.classes) {
        if (rc.M == 0 || rc.cnt <= 0) continue;
        k_filter<<<rc.cnt, kThreads, sizeof(double2) * rc.M, s>>>(rc.k0, rc.M, stages_of(rc.M), dp.chirp,
                                                                  dp.twiddle, dp.Mtab, dp.filt + rc.filt_off);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t dft_plan_make_f32(int L, DftPlan &dp, uint64_t &bytes, cudaStream_t s) {
    const int64_t n_tw = dp.Mtab, n_ch = (int64_t)L * L, n_f = dp.filt_total > 0 ? dp.filt_total : 1;
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
    cudaFree(dp.d_ring_M); cudaFree(dp.d_ring_foff);
    dp = DftPlan{};
}

int64_t dft_launches(const DftPlan &dp) { return (int64_t)dp.classes.size(); }

template <typename T, int OUT>
static cudaError_t ring_dft_impl(int L, const DftPlan &dp, const cplx_t<T> *samples, T *out,
                                 int64_t batch, cudaStream_t s) {
    for (const RingClass &rc : dp.classes) {
        if (rc.cnt <= 0) continue;
        const dim3 grid(rc.cnt, (unsigned)batch);
        k_ring_dft<T, OUT><<<grid, rc.M == 0 ? 64 : kThreads, smem_bytes<T>(rc), s>>>(
            make_args<T>(L, dp, batch, rc), samples, out);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T, int IN>
static cudaError_t ring_idft_impl(int L, const DftPlan &dp, const T *in, cplx_t<T> *samples,
                                  int64_t batch, cudaStream_t s) {
    for (const RingClass &rc : dp.classes) {
        if (rc.cnt <= 0) continue;
        const dim3 grid(rc.cnt, (unsigned)batch);
        k_ring_idft<T, IN><<<grid, rc.M == 0 ? 64 : kThreads, smem_bytes<T>(rc), s>>>(
            make_args<T>(L, dp, batch, rc), in, samples);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
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
