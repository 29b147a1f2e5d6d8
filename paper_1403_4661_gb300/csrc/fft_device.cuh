// Device building blocks of the ring DFTs (csrc/dft.cu) shared with the persistent uneven-batch
// kernels (csrc/uneven.cu): complex helpers, the stage plan of a chirp-z length, the in-place
// decimation-in-frequency / decimation-in-time stages and the Bluestein convolution of one ring.
// See csrc/dft.cu for the method.
#pragma once

#include "sht_internal.cuh"

namespace sht {
namespace fft {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
template <typename C> __device__ __forceinline__ C conjd(C a) { a.y = -a.y; return a; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
// -i a and +i a
template <typename C> __device__ __forceinline__ C mul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }
template <typename C> __device__ __forceinline__ C mul_pi(C a) { C r; r.x = -a.y; r.y = a.x; return r; }
__device__ __forceinline__ void sincospi_t(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ void sincospi_t(float x, float *s, float *c) { sincospif(x, s, c); }

constexpr int kMaxStages = 10;
constexpr int kThreads = 256;

// Radices of one convolution length M, in decimation-in-frequency order: 4, .., 4, then 2 when
// log2 of the power-of-two part is odd, then 3 for M = 3 * 2^a.  st.S[s] is the sub-transform
// length entering stage s (S[0] = M).
struct Stages {
    int n;
    int R[kMaxStages];
    int S[kMaxStages];
};

__host__ __device__ inline Stages stages_of(int M) {
    Stages st{};
    int p = M, three = 0;
    if (p % 3 == 0) { three = 1; p /= 3; }
    int a = 0;
    while ((1 << a) < p) ++a;
    for (int i = 0; i < a / 2; ++i) st.R[st.n++] = 4;
    if (a & 1) st.R[st.n++] = 2;
    if (three) st.R[st.n++] = 3;
    int S = M;
    for (int s = 0; s < st.n; ++s) { st.S[s] = S; S /= st.R[s]; }
    return st;
}

// Smallest 2^a or 3 * 2^a >= 2N - 1 (and >= 16).
inline int bluestein_length(int N) {
    int best = 1 << 30;
    for (int a = 4; a < 30; ++a) {
        const int p2 = 1 << a, p3 = 3 << (a - 1);
        if (p3 >= 2 * N - 1 && p3 >= 16) best = p3 < best ? p3 : best;
        if (p2 >= 2 * N - 1) { best = p2 < best ? p2 : best; break; }
    }
    return best;
}

// sin(2 pi / 3)
template <typename T> __device__ __forceinline__ T sin60() { return (T)0.86602540378443864676372317075293618; }

// ---- decimation-in-frequency stage s (forward FFT), in place -------------------------------
// Block of length S = R S': for j < S', inputs a_q = x[o + j + q S'], outputs
// y_p = DFT_R(a)_p * w_S^{p j} at o + j + p S' (w_S = e^{-2 pi i / S}, tw[t] = w_Mtab^t).
template <typename C>
__device__ __forceinline__ void dif_stage(C *a, int M, int S, int R, const C *__restrict__ tw, int Mtab,
                                          const C *__restrict__ filt) {
    const int Sp = S / R, nb = M / R, ts = Mtab / S;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        const int blk = idx / Sp, j = idx - blk * Sp;
        C *p = a + blk * S + j;
        if (R == 4) {
            C a0 = p[0], a1 = p[Sp], a2 = p[2 * Sp], a3 = p[3 * Sp];
            const C A = cadd(a0, a2), Bm = csub(a0, a2), Cc = cadd(a1, a3), D = csub(a1, a3);
            a0 = cadd(A, Cc);
            a2 = csub(A, Cc);
            a1 = cadd(Bm, mul_mi(D));
            a3 = csub(Bm, mul_mi(D));
            if (j) {
                a1 = cmul(a1, __ldg(&tw[j * ts]));
                a2 = cmul(a2, __ldg(&tw[2 * j * ts]));
                a3 = cmul(a3, __ldg(&tw[3 * j * ts]));
            }
            if (filt) {
                const int o = blk * S + j;
                a0 = cmul(a0, __ldg(&filt[o])); a1 = cmul(a1, __ldg(&filt[o + Sp]));
                a2 = cmul(a2, __ldg(&filt[o + 2 * Sp])); a3 = cmul(a3, __ldg(&filt[o + 3 * Sp]));
            }
            p[0] = a0; p[Sp] = a1; p[2 * Sp] = a2; p[3 * Sp] = a3;
        } else if (R == 2) {
            C a0 = p[0], a1 = p[Sp];
            const C s0 = cadd(a0, a1);
            C s1 = csub(a0, a1);
            if (j) s1 = cmul(s1, __ldg(&tw[j * ts]));
            if (filt) {
                const int o = blk * S + j;
                p[0] = cmul(s0, __ldg(&filt[o])); p[Sp] = cmul(s1, __ldg(&filt[o + Sp]));
            } else {
                p[0] = s0; p[Sp] = s1;
            }
        } else {   // R == 3: y0 = a0 + t1, y1,2 = a0 - t1/2 -+ i sin60 (a1 - a2), t1 = a1 + a2
            using T = decltype(a[0].x);
            const C a0 = p[0], a1 = p[Sp], a2 = p[2 * Sp];
            const C t1 = cadd(a1, a2);
            C t2;
            t2.x = fma((T)-0.5, t1.x, a0.x);
            t2.y = fma((T)-0.5, t1.y, a0.y);
            C d = csub(a1, a2);
            d.x *= sin60<T>();
            d.y *= sin60<T>();
            C y0 = cadd(a0, t1), y1 = cadd(t2, mul_mi(d)), y2 = csub(t2, mul_mi(d));
            if (j) {
                y1 = cmul(y1, __ldg(&tw[j * ts]));
                y2 = cmul(y2, __ldg(&tw[2 * j * ts]));
            }
            if (filt) {
                const int o = blk * S + j;
                y0 = cmul(y0, __ldg(&filt[o])); y1 = cmul(y1, __ldg(&filt[o + Sp]));
                y2 = cmul(y2, __ldg(&filt[o + 2 * Sp]));
            }
            p[0] = y0; p[Sp] = y1; p[2 * Sp] = y2;
        }
    }
}

// ---- decimation-in-time stage s (inverse FFT, unnormalised), in place ------------------------
// The inverse of dif_stage: b_p = y[o + j + p S'] * conj(w_S^{p j}), x_q = sum_p b_p e^{+2 pi i pq/R}.
template <typename C>
__device__ __forceinline__ void dit_stage(C *a, int M, int S, int R, const C *__restrict__ tw, int Mtab) {
    const int Sp = S / R, nb = M / R, ts = Mtab / S;
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        const int blk = idx / Sp, j = idx - blk * Sp;
        C *p = a + blk * S + j;
        if (R == 4) {
            C b0 = p[0], b1 = p[Sp], b2 = p[2 * Sp], b3 = p[3 * Sp];
            if (j) {
                b1 = cmulc(b1, __ldg(&tw[j * ts]));
                b2 = cmulc(b2, __ldg(&tw[2 * j * ts]));
                b3 = cmulc(b3, __ldg(&tw[3 * j * ts]));
            }
            const C A = cadd(b0, b2), Bm = csub(b0, b2), Cc = cadd(b1, b3), D = csub(b1, b3);
            p[0] = cadd(A, Cc);
            p[2 * Sp] = csub(A, Cc);
            p[Sp] = cadd(Bm, mul_pi(D));
            p[3 * Sp] = csub(Bm, mul_pi(D));
        } else if (R == 2) {
            C b0 = p[0], b1 = p[Sp];
            if (j) b1 = cmulc(b1, __ldg(&tw[j * ts]));
            p[0] = cadd(b0, b1);
            p[Sp] = csub(b0, b1);
        } else {
            using T = decltype(a[0].x);
            C b0 = p[0], b1 = p[Sp], b2 = p[2 * Sp];
            if (j) {
                b1 = cmulc(b1, __ldg(&tw[j * ts]));
                b2 = cmulc(b2, __ldg(&tw[2 * j * ts]));
            }
            const C t1 = cadd(b1, b2);
            C t2;
            t2.x = fma((T)-0.5, t1.x, b0.x);
            t2.y = fma((T)-0.5, t1.y, b0.y);
            C d = csub(b1, b2);
            d.x *= sin60<T>();
            d.y *= sin60<T>();
            p[0] = cadd(b0, t1);
            p[Sp] = cadd(t2, mul_pi(d));
            p[2 * Sp] = csub(t2, mul_pi(d));
        }
    }
}

// Bluestein convolution of one ring: X_t = c_t sum_n (x_n c_n) conj(c_{t-n}), t < N, with
// x_n = in(n) (n < N) and out(t, X_t) for t < N.  a: M complex values of shared memory.
template <typename C, typename In, typename Out>
__device__ __forceinline__ void bluestein(C *a, int N, int M, const Stages &st, const C *__restrict__ tw, int Mtab,
                                          const C *__restrict__ chirp, const C *__restrict__ filt, In in, Out out) {
    // first forward stage (R = 4, S = M) with the chirp premultiply; inputs j + 2M/4, j + 3M/4 are
    // beyond N <= M/2, input j + M/4 is beyond N for j >= N - M/4
    {
        const int Q = M >> 2, ts = Mtab / M;
        for (int j = threadIdx.x; j < Q; j += blockDim.x) {
            const C a0 = cmul(in(j), __ldg(&chirp[j]));
            C a1;
            if (j + Q < N) a1 = cmul(in(j + Q), __ldg(&chirp[j + Q]));
            else { a1.x = 0; a1.y = 0; }
            C y0 = cadd(a0, a1), y1 = cadd(a0, mul_mi(a1)), y2 = csub(a0, a1), y3 = csub(a0, mul_mi(a1));
            if (j) {
                y1 = cmul(y1, __ldg(&tw[j * ts]));
                y2 = cmul(y2, __ldg(&tw[2 * j * ts]));
                y3 = cmul(y3, __ldg(&tw[3 * j * ts]));
            }
            if (st.n == 1) {
                y0 = cmul(y0, __ldg(&filt[j])); y1 = cmul(y1, __ldg(&filt[j + Q]));
                y2 = cmul(y2, __ldg(&filt[j + 2 * Q])); y3 = cmul(y3, __ldg(&filt[j + 3 * Q]));
            }
            a[j] = y0; a[j + Q] = y1; a[j + 2 * Q] = y2; a[j + 3 * Q] = y3;
        }
        __syncthreads();
    }
    for (int s = 1; s < st.n; ++s) {
        dif_stage(a, M, st.S[s], st.R[s], tw, Mtab, s == st.n - 1 ? filt : (const C *)nullptr);
        __syncthreads();
    }
    for (int s = st.n - 1; s >= 1; --s) {
        dit_stage(a, M, st.S[s], st.R[s], tw, Mtab);
        __syncthreads();
    }
    // last inverse stage (R = 4, S = M): outputs j and j + M/4 only (the others are >= M/2 >= N),
    // with the chirp postmultiply
    {
        const int Q = M >> 2, ts = Mtab / M;
        for (int j = threadIdx.x; j < Q; j += blockDim.x) {
            C b0 = a[j], b1 = a[j + Q], b2 = a[j + 2 * Q], b3 = a[j + 3 * Q];
            if (j) {
                b1 = cmulc(b1, __ldg(&tw[j * ts]));
                b2 = cmulc(b2, __ldg(&tw[2 * j * ts]));
                b3 = cmulc(b3, __ldg(&tw[3 * j * ts]));
            }
            out(j, cmul(cadd(cadd(b0, b2), cadd(b1, b3)), __ldg(&chirp[j])));
            if (j + Q < N) out(j + Q, cmul(cadd(csub(b0, b2), mul_pi(csub(b1, b3))), __ldg(&chirp[j + Q])));
        }
    }
}

}  // namespace fft
}  // namespace sht
