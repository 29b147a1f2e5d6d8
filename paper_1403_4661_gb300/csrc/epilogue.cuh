// Epilogues shared by the float64 (and float32) and the tensor-core contractions: one output row r
// and the four columns c0..c0+3 of one signal, (+m re, +m im, -m re, -m im).  `slots` selects the
// column pairs an epilogue writes (bit 0: +m, bit 1: -m); spin plans run each contraction once per
// sign of m, with that sign's table, and keep only that sign's columns.
#pragma once

#include "sht_internal.cuh"

namespace sht {

template <typename T>
struct EpiArgsT {
    T *C; int64_t ldc;
    const T *C0;        // EPI_SUB
    int m, L, N;
    cplx_t<T> *coeffs;  // EPI_SOLVE
    T *W;               // EPI_ALIAS
    int slots = 3;      // column pairs written: bit 0 the +m pair, bit 1 the -m pair
};
using EpiArgs = EpiArgsT<double>;

template <int EPI, typename T>
__device__ __forceinline__ void epilogue_row4(const EpiArgsT<T> &p, int r, int c0, const T v[4]) {
    const int m = p.m, N = p.N;
    if ((EPI == EPI_STORE || EPI == EPI_SOLVE) && p.slots != 3) {
        T *cr = p.C + (int64_t)r * p.ldc + c0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (c0 + j < N && ((p.slots >> (j >> 1)) & 1)) cr[j] = v[j];
    } else if (EPI == EPI_STORE || EPI == EPI_SOLVE) {
        T *cr = p.C + (int64_t)r * p.ldc + c0;
        if (c0 + 4 <= N && (p.ldc & 1) == 0) {
            *reinterpret_cast<cplx_t<T> *>(cr) = mk2<T>(v[0], v[1]);
            *reinterpret_cast<cplx_t<T> *>(cr + 2) = mk2<T>(v[2], v[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (c0 + j < N) cr[j] = v[j];
        }
    }
    if (EPI == EPI_SUB) {
        const T *c0r = p.C0 + (int64_t)r * p.ldc + c0;
        T *cr = p.C + (int64_t)r * p.ldc + c0;
#pragma unroll
        for (int j = 0; j < 4; ++j) cr[j] = c0r[j] - v[j];
    }
    if (EPI == EPI_SOLVE) {
        // row r is degree l = m + r; columns (b, +m re/im, -m re/im)
        const int64_t L2 = (int64_t)p.L * p.L;
        const int l = m + r, b = c0 >> 2;
        cplx_t<T> *cb = p.coeffs + (int64_t)b * L2 + (int64_t)l * l + l;
        if (p.slots & 1) cb[m] = mk2<T>(v[0], v[1]);
        if (m > 0 && (p.slots & 2)) {
            const T sg = (m & 1) ? (T)-1 : (T)1;   // f_l^{-m} = (-1)^m F_l^{-}
            cb[-m] = mk2<T>(sg * v[2], sg * v[3]);
        }
    }
    if (EPI == EPI_ALIAS) {
        // row r is ring k = r < m; subtract G_{+m}, G_{-m} from bins a, -a of ring k
        const int k = r, b = c0 >> 2;
        const int a = alias_bin(m, k);
        const int o = a < 0 ? -a : a;
        T *w = p.W + (rows_off(p.L, o) + (k - o)) * (int64_t)N + 4 * b;
        // read through L2 (__ldcg): in the persistent chain kernel other SMs updated these bins
        const T up = (p.slots & 1) ? (T)1 : (T)0, um = (p.slots & 2) ? (T)1 : (T)0;
        if (a == 0) {
            w[0] = __ldcg(w) - (up * v[0] + um * v[2]);
            w[1] = __ldcg(w + 1) - (up * v[1] + um * v[3]);
        } else {
            const int sp = a > 0 ? 0 : 2;   // slot of bin a  (+o or -o)
            const int sm = 2 - sp;          // slot of bin -a
            if (p.slots & 1) {
                w[sp] = __ldcg(w + sp) - v[0];
                w[sp + 1] = __ldcg(w + sp + 1) - v[1];
            }
            if (p.slots & 2) {
                w[sm] = __ldcg(w + sm) - v[2];
                w[sm + 1] = __ldcg(w + sm + 1) - v[3];
            }
        }
    }
}

}  // namespace sht
