// Internal declarations of libsht (not part of the C ABI).
//
// Device data layouts (all float64; complex data interleaved re, im):
//
//  P~ table  pt      block m >= 0 at pt_off(L, m): L rows (ring k = 0..L-1, in theta order),
//                    n_m = L - m columns (degree l = m..L-1); row-major.  P~_l^m(theta_k),
//                    the functions of Sec. III-G evaluated at every ring.
//  inverses  pinv    block m at pinv_off(L, m): n_m x n_m row-major, row l - m, column k - m:
//                    (P_m)^{-1} with P_m[k][l] = P~_l^m(theta_k), k, l >= m (Eq. (12) without the
//                    2 pi factor, which the project's scaling of G_m drops).
//  order-major work  W, F, X   block m at rows_off(L, m) rows, n_m rows (k - m or l - m), each row
//                    4B doubles: column 4b + 2s + c for signal b, s = 0 (+m) / 1 (-m), c = re/im.
//                    In W (forward bins): row k holds bin +-m of ring k.  In F / X (coefficients):
//                    row l holds f_l^{+m} and (-1)^m f_l^{-m}  (the sign folds Eq. (23) into the
//                    data so that P~^{-m} never appears).
//  synthesis G      Gt   row m * L + k (m >= 0, every ring k), 4B doubles, same column layout:
//                    slot s = 0 holds G_{+m}(theta_k), slot s = 1 holds G_{-m}(theta_k).
//
// Scaling convention: G_m(theta_k) here is sum_l P~_l^m(theta_k) f_l^m (Eq. (11) without 2 pi),
// ring DFTs carry 1/N_k, so that bin j of ring k equals sum_{m = j mod N_k} G_m(theta_k).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/sht.h"

namespace sht {

__host__ __device__ inline int64_t pt_off(int64_t L, int64_t m) {
    return L * (m * L - m * (m - 1) / 2);
}
__host__ __device__ inline int64_t sq_sum(int64_t n) { return n * (n + 1) * (2 * n + 1) / 6; }
__host__ __device__ inline int64_t pinv_off(int64_t L, int64_t m) {
    return sq_sum(L) - sq_sum(L - m);
}
__host__ __device__ inline int64_t rows_off(int64_t L, int64_t m) {
    return m * L - m * (m - 1) / 2;
}
__host__ __device__ inline int64_t rows_total(int64_t L) { return L * (L + 1) / 2; }

// Bin of ring k (length 2k+1) that order m aliases to, in [-k, k].
__host__ __device__ inline int alias_bin(int m, int k) {
    int N = 2 * k + 1;
    int r = (m + k) % N;
    if (r < 0) r += N;
    return r - k;
}

// Complex type of a real type (the float64 path and the float32 path of SHT_F32).
template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };
template <typename T> using cplx_t = typename Cplx<T>::type;
template <typename T>
__host__ __device__ __forceinline__ cplx_t<T> mk2(T x, T y) {
    cplx_t<T> r;
    r.x = x;
    r.y = y;
    return r;
}

// Split-K partial buffer of the order chain holds this many L x 4B slices.
constexpr int kSplitCap = 16;

// Rings whose DFT is taken directly (O(N^2)); longer rings use Bluestein's chirp-z transform.
constexpr int kDirectMaxN = 63;

// Consecutive rings k0 .. k0 + cnt - 1 sharing one chirp-z convolution length M (M = 0: rings
// short enough for the direct DFT); their filters start at filt_off, M values per ring.
struct RingClass {
    int k0, cnt, M;
    int64_t filt_off;
};

struct DftPlan {
    int Mmax = 0;                  // largest convolution length (2^a or 3 * 2^a)
    int Mtab = 0;                  // twiddle table length: a multiple of every convolution length
    double2 *chirp = nullptr;      // e^{-i pi n^2 / N_k}, n < N_k, ring k at offset k^2
    double2 *filt = nullptr;       // per chirp-z ring: FFT_M of the conjugate chirp, scaled 1/M,
                                   // in the forward FFT's digit-reversed output order
    double2 *twiddle = nullptr;    // e^{-2 pi i t / Mtab}, t < Mtab
    int64_t filt_total = 0;        // complex values in filt
    // SHT_F32 plans: the same tables rounded to float32 (dft_plan_make_f32)
    float2 *chirp_f = nullptr, *filt_f = nullptr, *twiddle_f = nullptr;
    std::vector<RingClass> classes;
    int *d_ring_M = nullptr;           // device, per ring: chirp-z length (0: direct ring)
    int64_t *d_ring_foff = nullptr;    // device, per ring: offset of its filter in filt
};

// Per-call device scratch, sized for `batch` signals.
struct Workspace {
    int64_t batch = 0;
    double *a = nullptr;             // W (forward bins) / X (inverse coefficients): rows_total * 4B
    double *b = nullptr;             // F (forward solved coefficients): rows_total * 4B
    double *g = nullptr;             // Gt (inverse synthesis): L * L * 4B
    double *part = nullptr;          // split-K partials: kSplitCap * L * 4B
    __nv_bfloat16 *xS = nullptr;     // tensor plans: slices of X (all orders)
    int *xE = nullptr;
    unsigned char *tmX = nullptr;    // tensor plans: TMA maps of the X slices
    unsigned *bar = nullptr;         // tensor plans: words of the chain kernel (tc_chain_words)
    double *part2 = nullptr;         // tensor plans: the chain's alias values, kChainB * L * 4B
    double2 *r = nullptr, *dx = nullptr;  // refinement: residual, update
    uint64_t bytes = 0;
};

}  // namespace sht

struct sht_plan_s {
    int L = 0;
    int dtype = 0;
    int device = 0;
    std::vector<double> theta;
    double *d_theta = nullptr;
    double *pt = nullptr;       // P~ table (spin plans: sP~^{+m})
    double *pinv = nullptr;     // per-order inverses (spin plans: of the +m matrices)
    int spin = 0;               // spin weight s of the plan's signals (Sec. III-H); 0: scalar
    // scalar plans: what regenerates P~ on the fly (kernels that walk the recursion instead of
    // reading pt): sectoral start values (L x L, order-major) and recursion coefficients
    double *sect_mant = nullptr;
    int *sect_expo = nullptr;
    double *rec_a = nullptr, *rec_b = nullptr;
    double *pt2 = nullptr;      // spin plans: (-1)^m sP~^{-m}, layout of pt
    double *pinv2 = nullptr;    // spin plans: inverses of the -m matrices, layout of pinv
    float *ptF = nullptr;       // SHT_F32: the P~ table rounded to float32
    float *pinvF = nullptr;     // SHT_F32: the per-order inverses rounded to float32
    sht::DftPlan dft;
    sht::Workspace ws;    // per-call scratch, grown to the largest batch seen
    double2 *stage = nullptr;     // uneven batches: gathered inputs, then outputs (stage_batch each)
    int64_t stage_batch = 0;
    uint64_t table_bytes = 0;
    uint64_t ws_bytes = 0;
    double plan_seconds = 0.0;
    double order_seconds = 0.0;
    int64_t launches = 0;
    // SHT_F64_TENSOR: slices of the tables, their exponents and per-order offsets
    __nv_bfloat16 *ptS = nullptr, *piS = nullptr;
    int *ptE = nullptr, *piE = nullptr;
    int64_t *d_ptk_off = nullptr, *d_pik_off = nullptr;
    unsigned char *d_tmaps = nullptr;   // TMA maps of the sliced tables (chain kernel)
    // SHT_TF32_REFINED: TF32 copies of the tables (rows scaled by the slices' row exponents) and
    // their TMA maps, read by the low-precision chain
    float *ptT = nullptr, *piT = nullptr;
    unsigned char *d_tmaps_tf32 = nullptr;
    double *chainQ = nullptr;           // tensor plans: tc_chain_q_table
    bool refine_tf32 = false;
    std::vector<int64_t> ptk_off, pik_off;
    int *d_status = nullptr;

    int chain_grid = 0;                 // CTAs of the persistent order-chain kernel (tensor plans)
    uint64_t wait_ns = 1000000000ull;   // limit of the tensor kernels' waits (sht_plan_set_wait_limit)
    // refinement (SHT_BF16_REFINED, SHT_BF16X2_REFINED, SHT_TF32_REFINED)
    int refine_nsl = 0;           // slices of the low-precision forward (1 for TF32); 0: no refinement
    int refine_max_iters = 10;
    double refine_tol = 1e-11;
    int refine_iters = 0;
    double refine_last = 0.0;
    double *d_refine_max = nullptr;
    // execution choices per batch size (sht_plan_set_paths, sht_plan_autotune)
    std::map<int64_t, sht_tuning> tuned;
    // stage timing (sht_plan_set_timing)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spans[SHT_NUM_STAGES];
};

namespace sht {

// error reporting (api.cu)
sht_status set_error(sht_status st, const std::string &msg);
sht_status cuda_check(cudaError_t e, const char *what);

// Largest batch of one call: the batch is a grid dimension of the ring kernels.
constexpr int64_t kMaxBatch = 65535;
// Argument checks shared by the entry points (api.cu): plan non-NULL and on the current device;
// batch in [0, kMaxBatch]; for batch > 0, non-NULL buffers aligned to one element and disjoint;
// with need_ptilde, a plan that keeps its P~ table (every transform but the ring stages).
sht_status check_plan(sht_plan_t p);
sht_status check_io(sht_plan_t p, const void *in, const void *out, int64_t batch, bool need_ptilde = true);

// legendre.cu: P~ table for arbitrary co-latitudes (rows), all orders.
cudaError_t build_ptilde_table(int L, const double *d_theta_rows, int nrows, double *d_table,
                               cudaStream_t s);
// Table layout for nrows != L: block m at nrows * rows_off(L, m), nrows x n_m.
// The sectoral values P~_m^m(theta_r) = mant[m * nrows + r] * 2^expo[m * nrows + r], m < L.
cudaError_t sectoral_values(int L, const double *d_theta_rows, int nrows, double *mant, int *expo,
                            cudaStream_t s);
// Recursion coefficients a_lm, b_lm of the table recursion, block m at rows_off(L, m), entry l - m
// (the step producing degree l; a = sqrt(2m+3), b = 0 for l = m + 1).
cudaError_t recursion_coeffs(int L, double *ra, double *rb, cudaStream_t s);

// invert.cu: explicit inverses of P_m for every m >= m_first from the P~ table (blocks of
// orders below m_first are left as they are).
cudaError_t build_inverses(int L, const double *d_pt, double *d_pinv, cudaStream_t s, int m_first = 0);

// spin.cu: spin-s tables (pt: sP~^{+m}, pt2: (-1)^m sP~^{-m}; scalar P~ layout) and per-order
// (pseudo-)inverses; `singular` is set when a square P_m is singular for these co-latitudes.
cudaError_t build_spin_tables(int L, int spin, const double *d_theta, double *pt, double *pt2,
                              double *pinv, double *pinv2, bool &singular, cudaStream_t s);
// spin-s transforms on the float64 SIMT kernels (workspaces of p->ws)
cudaError_t spin_forward(sht_plan_t p, const double2 *d_samples, double2 *d_coeffs, int64_t batch, cudaStream_t s);
cudaError_t spin_inverse(sht_plan_t p, const double2 *d_coeffs, double2 *d_samples, int64_t batch, cudaStream_t s);
cudaError_t spin_inverse_adjoint(sht_plan_t p, const double2 *d_samples, double2 *d_coeffs, int64_t batch,
                                 cudaStream_t s);

// dft.cu
cudaError_t dft_plan_create(int L, DftPlan &dp, uint64_t &bytes, cudaStream_t s);
void dft_plan_destroy(DftPlan &dp);
// kernel launches of one ring-DFT pass (one per ring class)
int64_t dft_launches(const DftPlan &dp);
// forward ring DFTs of every ring of every signal, 1/N scaled, into the order-major bins W
cudaError_t ring_dft_to_bins(int L, const DftPlan &dp, const double2 *samples, double *W,
                             int64_t batch, bool scale, cudaStream_t s);
// fold of the synthesis table into ring bins + inverse ring DFTs
cudaError_t fold_ring_idft(int L, const DftPlan &dp, const double *Gt, double2 *samples,
                           int64_t batch, cudaStream_t s);
// adjoint of ring_dft_to_bins (scale = 1/N): bins -> samples
cudaError_t bins_to_ring_adjoint(int L, const DftPlan &dp, const double *W, double2 *samples,
                                 int64_t batch, cudaStream_t s);
// adjoint of fold_ring_idft: samples -> unfolded synthesis table Gt
cudaError_t ring_dft_unfold(int L, const DftPlan &dp, const double2 *samples, double *Gt,
                            int64_t batch, cudaStream_t s);
// float32 tables of the ring DFTs (SHT_F32 plans), computed from the float64 ones
cudaError_t dft_plan_make_f32(int L, DftPlan &dp, uint64_t &bytes, cudaStream_t s);
// the same four transforms in float32 (complex64 samples, float order-major buffers)
cudaError_t ring_dft_to_bins(int L, const DftPlan &dp, const float2 *samples, float *W,
                             int64_t batch, bool scale, cudaStream_t s);
cudaError_t fold_ring_idft(int L, const DftPlan &dp, const float *Gt, float2 *samples,
                           int64_t batch, cudaStream_t s);
cudaError_t bins_to_ring_adjoint(int L, const DftPlan &dp, const float *W, float2 *samples,
                                 int64_t batch, cudaStream_t s);
cudaError_t ring_dft_unfold(int L, const DftPlan &dp, const float2 *samples, float *Gt,
                            int64_t batch, cudaStream_t s);

// gemm_f64.cu
enum Epilogue : int {
    EPI_STORE = 0,       // C = A B
    EPI_SOLVE = 1,       // C = A B, and coefficients of order m written to the output
    EPI_ALIAS = 2,       // rows k < m: W[alias bins] -= A B
    EPI_ADJ_SOLVE = 3,   // adjoint chain: W bins of order m (rows k >= m) = A^T B
    EPI_SUB = 4,         // C = C0 - A B (C0 given)
};
template <typename T>
struct GemmArgsT {
    int L;
    int64_t batch;
    int m;                 // order of this problem (single-problem launches)
    cplx_t<T> *coeffs;     // EPI_SOLVE output
    T *W;                  // EPI_ALIAS target
    T *part = nullptr;     // split-K partial sums (none: no split)
    int64_t part_cap = 0;  // elements available at part
    int split_cap = 0;     // most K-splits per product (0: the launcher's default, 16)
    int64_t *launches = nullptr;  // incremented by the number of kernels launched
    int slots = 3;         // epilogue column pairs written (bit 0: +m, bit 1: -m; spin plans)
};
using GemmArgs = GemmArgsT<double>;
// Single problem: C[M x N] (+)= op(A)[M x K] * B[K x N], row-major, N = 4 * batch.
cudaError_t gemm_f64(bool transA, int M, int K, int N, const double *A, int64_t lda,
                     const double *B, int64_t ldb, double *C, int64_t ldc, int epi,
                     const GemmArgs &ga, cudaStream_t s, const double *C0 = nullptr);
// The same contraction in float32 (SHT_F32 plans), on the FP32 pipe.
cudaError_t gemm_f32(bool transA, int M, int K, int N, const float *A, int64_t lda,
                     const float *B, int64_t ldb, float *C, int64_t ldc, int epi,
                     const GemmArgsT<float> &ga, cudaStream_t s, const float *C0 = nullptr);
// Grouped over every order m: Gt[m][k][:] = P~[m][k][:] . X[m] (all k), or the transposed
// contraction for the adjoint (out[m][l][:] = sum_k P~[m][k][l] U[m][k][:]).
cudaError_t synthesis_all_orders(int L, int64_t batch, const double *pt, const double *X,
                                 double *Gt, cudaStream_t s);
cudaError_t analysis_all_orders(int L, int64_t batch, const double *pt, const double *U,
                                double *X, cudaStream_t s);
cudaError_t synthesis_all_orders(int L, int64_t batch, const float *pt, const float *X,
                                 float *Gt, cudaStream_t s);
// The float64 grouped contractions writing only the column pairs in `slots` (spin plans).
cudaError_t synthesis_all_orders_slots(int L, int64_t batch, const double *pt, const double *X,
                                       double *Gt, int slots, cudaStream_t s);
cudaError_t analysis_all_orders_slots(int L, int64_t batch, const double *pt, const double *U,
                                      double *X, int slots, cudaStream_t s);
cudaError_t analysis_all_orders(int L, int64_t batch, const float *pt, const float *U,
                                float *X, cudaStream_t s);

// layout.cu: coefficient <-> order-major conversions
cudaError_t coeffs_to_orders(int L, int64_t batch, const double2 *coeffs, double *X,
                             cudaStream_t s);
cudaError_t orders_to_coeffs(int L, int64_t batch, const double *X, double2 *coeffs,
                             cudaStream_t s);
cudaError_t coeffs_to_orders(int L, int64_t batch, const float2 *coeffs, float *X, cudaStream_t s);
cudaError_t orders_to_coeffs(int L, int64_t batch, const float *X, float2 *coeffs, cudaStream_t s);
// ring-major bins (k^2 + k + j) from the order-major bins W; and ring-major bins placed in a
// synthesis table Gt as orders |m| <= k (zero elsewhere), the input of fold_ring_idft
cudaError_t bins_to_rings(int L, int64_t batch, const double *W, double2 *bins, cudaStream_t s);
cudaError_t bins_to_rings(int L, int64_t batch, const float *W, float2 *bins, cudaStream_t s);
cudaError_t rings_to_table(int L, int64_t batch, const double2 *bins, double *Gt, cudaStream_t s);
cudaError_t rings_to_table(int L, int64_t batch, const float2 *bins, float *Gt, cudaStream_t s);
// n float64 values rounded to float32 (tables of SHT_F32 plans)
cudaError_t table_to_f32(const double *in, float *out, int64_t n, cudaStream_t s);
// refinement: r = s - r (n complex values); x += dx and max |Re, Im dx| into *mx
cudaError_t residual(int64_t n, const double2 *s_in, double2 *r, cudaStream_t s);
cudaError_t update_with_max(int64_t n, double2 *x, const double2 *dx, double *mx, cudaStream_t s);
// adjoint chain: U[k] (k < m) = the bins of ring k that orders +m / -m alias to
cudaError_t gather_alias_bins(int L, int m, int64_t batch, const double *W, double *U,
                              cudaStream_t s);
cudaError_t gather_alias_bins(int L, int m, int64_t batch, const float *W, float *U, cudaStream_t s);

// tc_gemm.cu: float64-accurate contractions on the tensor cores from exact BF16 slices
constexpr int kTcSlices = 8;     // slices per operand
constexpr int kTcSliceBits = 7;  // bits per slice
cudaError_t tc_prepare_kernels();
// Plan tables: slices of every order's P~ block (inverses = false; slice block m at
// kTcSlices * L * koff[m] elements, exponents at m * L) or P_m^{-1} block (inverses = true; slices
// at kTcSlices * koff[m], exponents at rows_off(L, m)).
cudaError_t tc_slice_table(const double *tab, int L, bool inverses, const int64_t *koff,
                           __nv_bfloat16 *out, int *expo, cudaStream_t s);
// Order-major coefficients X of a batch: slices of block m at kTcSlices * 4B * koff[m], exponents
// at m * 4B.
cudaError_t tc_slice_orders(const double *X, int L, int64_t batch, const int64_t *koff,
                            __nv_bfloat16 *out, int *expo, cudaStream_t s);
// TF32 copies of a plan table (layouts of tc_slice_table without the slice factor): row r of
// block m = the row times 2^-expo[r] rounded to TF32, zero padded to kp; expo as written by
// tc_slice_table.
cudaError_t tc_tf32_table(const double *tab, int L, bool inverses, const int64_t *koff, const int *expo,
                          float *out, cudaStream_t s);
// The forward's whole order chain (m = L-1 .. 0: solves, alias products) as one persistent
// cooperative launch of `grid` CTAs (tc_prepare_chain); W holds the ring bins on entry.
struct ChainTables {
    const __nv_bfloat16 *piS; const int *piE; const int64_t *pik_off;   // device offsets
    const __nv_bfloat16 *ptS; const int *ptE; const int64_t *ptk_off;
    const unsigned char *tmaps;   // device: 2 L TMA maps (tc_table_tensor_maps)
    const double *Q;              // device: tc_chain_q_table
};
// The chain kernel takes the orders in blocks of kChainB (L-1 down): block b covers orders
// hi = L-1-b kChainB .. lo = max(0, hi-kChainB+1).
constexpr int kChainB = 32;
// Q_m = P~_m(theta_k) P_m^{-1} for the rings lo <= k < m of m's block (float64, from the plan's pt
// and pinv): order m at kChainB * rows_off(L, m), (m - lo) rows of n_m, row k - lo.  The chain's
// tracked entries follow from it (the alias contribution of order m at ring k is Q_m[k] g_m).
cudaError_t tc_chain_q_table(int L, const double *pt, const double *pinv, double *Q, cudaStream_t s);
constexpr int kTensorMapBytes = 128;
// TMA maps of the sliced tables for the chain kernel, order m at 2m (P_m^{-1} block: {kp, n, S})
// and 2m + 1 (P~ block: {kp, L, S}), boxes of 32 x 128 x S, 64-byte swizzle; written to a new
// device array *d_maps of 2 L * kTensorMapBytes bytes (the caller frees it).
cudaError_t tc_table_tensor_maps(int L, const __nv_bfloat16 *piS, const std::vector<int64_t> &pik_off,
                                 const __nv_bfloat16 *ptS, const std::vector<int64_t> &ptk_off,
                                 unsigned char **d_maps);
// The same for the TF32 tables: 2-D float32 maps {kp, rows}, boxes of 16 x 128, 64-byte swizzle.
cudaError_t tc_table_tensor_maps_tf32(int L, const float *piT, const std::vector<int64_t> &pik_off,
                                      const float *ptT, const std::vector<int64_t> &ptk_off,
                                      unsigned char **d_maps);
constexpr int kChainBarWords = 96;   // grid barrier of the chain kernel: three 128-byte lines
cudaError_t tc_prepare_chain(int *grid);
// G: kChainB L Nc doubles of scratch (a block's alias values, and the look-ahead's contributions);
// words: tc_chain_words(L, batch) (barrier, exponent fields).
cudaError_t tc_forward_chain(const ChainTables &t, int L, int64_t batch, double *W, double *F,
                             double2 *coeffs, double *G, unsigned *words, int *status,
                             int nsl, bool tf32, int grid, uint64_t wait_ns, cudaStream_t s);
// Device words the chain kernel needs beside W, F and part (barrier, column scales).
int64_t tc_chain_words(int L, int64_t batch);
// TMA maps of the per-call X slices (order m at m: {kp, 4B, S}, boxes 32 x 64 x S), written to a
// new device array *d_maps of L * kTensorMapBytes bytes (the caller frees it).
cudaError_t tc_x_tensor_maps(int L, int64_t batch, const __nv_bfloat16 *xS,
                             const std::vector<int64_t> &ptk_off, unsigned char **d_maps);
// Eq. (11) for every order in one launch: Gt[m] (L x 4B) = P~_m X_m.
cudaError_t tc_synthesis_all_orders(int L, int64_t batch, const int *ptE, const unsigned char *tmA,
                                    const int *xE, const unsigned char *tmB, double *Gt, int *status,
                                    uint64_t wait_ns, cudaStream_t s);

// planner.cu: greedy condition-number ordering (indices into the ascending ring set Theta);
// candidates within a relative tie_rtol of the smallest condition number go to the lowest index
// (0: exact ties only); `middle` is the index of the ring kept farthest from the poles.
sht_status greedy_order(int L, const std::vector<double> &Theta, int middle, double tie_rtol,
                        std::vector<int> &order);

}  // namespace sht
