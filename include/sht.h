/*
 * sht.h - C ABI of libsht: forward and inverse spherical harmonic transforms on the
 * optimal-dimensionality sampling of Khalid, Kennedy and McEwen (L^2 samples on L rings),
 * computed on one NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Sampling (Sec. III-A, Eqs. (7)-(9)): L rings at co-latitudes theta_0..theta_{L-1}; ring k
 *    carries 2k+1 samples at phi_{k,n} = 2 pi n/(2k+1), n = 0..2k.  A signal is L^2 complex
 *    values, ring-major: sample (k, n) at index k^2 + n.
 *  Coefficients (Eq. (6)): f_l^m for 0 <= l < L, |m| <= l, at index l^2 + l + m.
 *  Basis (Appendix A, Eq. (29)): orthonormal Y_l^m with the Condon-Shortley phase;
 *    P~_l^m(theta) = Y_l^m(theta, 0).
 *  Element type: complex128, interleaved (re, im) doubles - the layout of torch.complex128 and
 *    C99 double _Complex - for every plan arithmetic but SHT_F32, whose signals are complex64
 *    (interleaved floats, torch.complex64).  A batch of B signals is B consecutive blocks of L^2
 *    elements.
 *  Device pointers must be aligned to one element (16 bytes; 8 for SHT_F32); input and output
 *    must not overlap.
 *  Ownership: the caller owns every buffer it passes.  The plan owns its tables (the P~ table and
 *    the per-order inverses, allocated at plan creation) and its workspaces (allocated on the
 *    first call that needs them, or by sht_plan_reserve, and kept until sht_plan_destroy).
 *  Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *    are asynchronous and stream-ordered; after a call returns SHT_OK the result is valid once
 *    the stream has reached that point.  A plan's workspaces are shared by all calls on it, so
 *    calls on one plan must not overlap in time (use one stream per plan, or one plan per stream).
 *    A call that finds its workspaces large enough allocates nothing and does not synchronise.
 *  Errors: no entry point aborts.  Argument errors return SHT_ERR_INVALID_ARG (or
 *    SHT_ERR_UNSUPPORTED) before any work is queued; a failed CUDA call returns SHT_ERR_CUDA
 *    (the CUDA error string is kept for sht_last_error_message); allocation failure returns
 *    SHT_ERR_OOM.  The current CUDA device must be the one the plan was created on.
 */
#ifndef SHT_H
#define SHT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sht_plan_s *sht_plan_t;

typedef enum {
    SHT_OK = 0,
    SHT_ERR_INVALID_ARG = 1,
    SHT_ERR_UNSUPPORTED = 2,
    SHT_ERR_OOM = 3,
    SHT_ERR_CUDA = 4,
    SHT_ERR_NOT_CONVERGED = 5,
    SHT_ERR_TIMEOUT = 6
} sht_status;

/*
 * Arithmetic of the transforms.
 *   SHT_F64         every step in float64 on the FP64 pipe.
 *   SHT_F64_TENSOR  float64-accurate results; the Legendre contractions (synthesis, per-order
 *                   solves, alias products) run on the BF16 tensor cores on exact 7-bit slices of
 *                   the float64 operands (8 slices per operand, 36 slice-pair products, exact FP32
 *                   accumulation of the leading diagonals, int64 folding), the ring DFTs and the
 *                   Legendre recursion stay in float64.  Errors are of the order of a float64
 *                   contraction.  The plan additionally holds the slices of its tables (about
 *                   2x the float64 tables).  The adjoints run the float64 kernels.
 *   SHT_BF16_REFINED, SHT_BF16X2_REFINED
 *                   forward by iterative refinement: x_0 = F_lo(s), x_{i+1} = x_i + F_lo(s - A x_i),
 *                   F_lo being the forward with its contractions on the tensor cores from 1 (BF16)
 *                   or 2 (BF16 x 2, ~15-bit) slices per operand with FP32 accumulation, and A the
 *                   float64-accurate inverse of SHT_F64_TENSOR; the ring DFTs, the Legendre
 *                   recursion and the residual s - A x stay float64-accurate.  The inverse and the
 *                   adjoints are those of SHT_F64_TENSOR.  See sht_plan_set_refinement.
 *   SHT_TF32_REFINED
 *                   the same refinement with F_lo's contractions on the TF32 tensor cores
 *                   (tcgen05 kind::tf32, FP32 accumulation): the table rows scaled by a power of two
 *                   and rounded to TF32 at plan time (10 stored significand bits), the right-hand
 *                   sides scaled per column and rounded to TF32 in the kernel.  The plan holds TF32
 *                   copies of both tables (L^3/2 + L^3/3 floats) besides the SHT_F64_TENSOR slices.
 *   SHT_F32         every step in float32 on the FP32 pipe (the float64 kernels instantiated for
 *                   float), complex64 samples and coefficients.  The Legendre table, the per-order
 *                   inverses and the ring-DFT tables are computed in float64 at plan time and rounded
 *                   to float32.  Errors are those of float32 arithmetic amplified as in float64
 *                   (about 1e-6 relative to the largest coefficient at L = 64, growing with L).
 *                   Refinement does not apply; sht_forward_noalloc and the uneven calls do not take
 *                   SHT_F32 plans (SHT_ERR_UNSUPPORTED).
 */
typedef enum {
    SHT_F64 = 0,
    SHT_F64_TENSOR = 1,
    SHT_BF16_REFINED = 2,
    SHT_BF16X2_REFINED = 3,
    SHT_TF32_REFINED = 4,
    SHT_F32 = 5
} sht_dtype;

/* Plan flags: ring ordering (Sec. III-E). */
#define SHT_ORDER_GREEDY 0u   /* condition-number minimisation: theta_{L-1} nearest the equator,
                                 then for m = L-2..0 the unused ring minimising kappa_2(P_m)   */
#define SHT_ORDER_SIMPLE 1u   /* Eq. (20): pi, then alternately north / south to the equator   */
#define SHT_ORDER_MASK   1u

/* Plan flags: the set the rings are drawn from (Sec. III-E, III-F), ordered by the rule above. */
#define SHT_MEASURE_UNIFORM 0u   /* Eq. (19): Theta_t = pi (2t+1)/(2L-1)                          */
#define SHT_MEASURE_SIN     2u   /* Theta^1: from the south pole, equal steps of sin(theta) dtheta */
#define SHT_MEASURE_TAN13   4u   /* Theta^2: equal steps of |tan(theta)|^(1/3) dtheta              */
#define SHT_MEASURE_MASK    6u

/* Plan flag: keep no P~ table (L^3/2 doubles): it is built to invert the P_m and then freed.
   Such plans (SHT_F64 only) serve the uneven-batch launches (sht_uneven_*), whose kernels
   regenerate P~ by its recursion; every other transform entry point returns SHT_ERR_UNSUPPORTED
   for them.  Cuts a plan's tables from 5/6 L^3 to 1/3 L^3 doubles. */
#define SHT_PLAN_NO_PTILDE 8u

#define SHT_MAX_L 2048   /* longest ring 4095: its chirp-z length 8192 fits one SM */

/*
 * sht_plan - build a plan for band-limit L (1 <= L <= SHT_MAX_L); batch is at most 65535.
 *   Ring co-latitudes come from the equiangular set Theta_t = pi (2t+1)/(2L-1) (Eq. (19)), or
 *   from the sets Theta^1, Theta^2 of the alternative measures (Sec. III-F, SHT_MEASURE_* flags;
 *   the paper shows they make P_m far worse conditioned), ordered by the rule in `flags`
 *   (Sec. III-E).  The ring kept farthest from the poles is the element nearest pi/2; on the
 *   mirror-symmetric sets Theta^1, Theta^2 candidates within a relative 1e-9 of the smallest
 *   condition number count as ties (lowest index wins).  The greedy ordering scores every candidate ring
 *   by the exact 2-norm condition number of P_m (Eq. (12)) through the eigen-decomposition of the
 *   fixed rows' Gram matrix and a rank-one secular equation; it costs O(L^4) and runs on the GPU.
 *   Then builds, on the current device: the P~_l^m(theta_k) table for all m >= 0, k, l >= m
 *   (L^3/2 doubles) and the explicit inverses of P_m for every m (L^3/3 doubles).
 *   Blocking (synchronises the device).  *out receives the plan, or NULL on error.
 */
sht_status sht_plan(int L, sht_dtype dtype, uint32_t flags, sht_plan_t *out);

/*
 * sht_plan_with_thetas - as sht_plan, with the L ring co-latitudes given by the caller (host
 *   array of L doubles, theta_host[k] = theta_k in radians, any values in [0, pi] (to within
 *   1e-12) for which every P_m is invertible; Remark 1).  The ordering and measure bits of `flags`
 *   are ignored; SHT_PLAN_NO_PTILDE applies.
 */
sht_status sht_plan_with_thetas(int L, sht_dtype dtype, const double *theta_host, uint32_t flags,
                                sht_plan_t *out);

/*
 * sht_plan_spin, sht_plan_spin_with_thetas - plans for spin-s functions (Sec. III-H: the transforms
 *   carry over with f -> sf, f_l^m -> sf_l^m, Y_l^m -> sY_l^m; Appendix A defines
 *   sY_l^m(theta, phi) = (-1)^s sqrt((2l+1)/(4 pi)) e^{i m phi} d^l_{m,-s}(theta), the Wigner small-d
 *   function d computed by its three-term recursion in l (Appendix A)).  Same sampling and ring
 *   orderings as sht_plan / sht_plan_with_thetas (flags and theta_host as there).
 *   spin: -8..8, non-zero, |spin| < L; L in 1..1024; dtype SHT_F64 only (SHT_ERR_UNSUPPORTED
 *   otherwise).  Coefficients use the scalar layout (index l^2 + l + m); the entries with l < |s|
 *   are ignored on input and written as 0.  The plan holds the tables of both signs of m (there is
 *   no P_{-m} = (-1)^m P_m relation for s != 0): twice the float64 tables of a scalar plan.  For
 *   |m| >= |s| the order-m systems are square and inverted; for |m| < |s| they have more rings
 *   than degrees and the forward solves them in the least-squares sense (exact for band-limited
 *   spin signals).
 *   Entry points on spin plans: sht_forward, sht_inverse, sht_inverse_adjoint.  The others
 *   (sht_forward_adjoint, sht_forward_noalloc, the uneven calls, sht_plan_set_paths,
 *   sht_plan_autotune, sht_plan_save) return SHT_ERR_UNSUPPORTED.
 *   Accuracy: the inverse and its adjoint are plain sums (float64 rounding).  The forward follows
 *   Procedure 1, whose order-by-order elimination amplifies rounding errors far more for s != 0
 *   than for s = 0 on these rings (measured round-trip errors: about 3e-10 at L = 16, s = 1, and
 *   order 1 at L = 16, s = 2, while the whole L^2-dimensional system stays well conditioned there);
 *   it is meant for small L.
 */
sht_status sht_plan_spin(int L, int spin, sht_dtype dtype, uint32_t flags, sht_plan_t *out);
sht_status sht_plan_spin_with_thetas(int L, int spin, sht_dtype dtype, const double *theta_host,
                                     uint32_t flags, sht_plan_t *out);

/*
 * sht_plan_save, sht_plan_load - keep a plan's ring co-latitudes on disk, so that a later process
 *   skips the greedy ordering (Sec. III-E; O(L^4), 23 s at L = 1024 on GB300) and rebuilds only the
 *   tables.  The paper stores the co-latitudes once per L for the same reason (Sec. III-E).
 *   File (little-endian): the 8 bytes "SHTTHETA", int32 L, int32 0, L float64 co-latitudes in
 *   ring order, then the 64-bit FNV-1a hash of all preceding bytes.
 *   sht_plan_save writes the file at `path` (host data only, no device work); SHT_ERR_INVALID_ARG
 *   if it cannot be written.  sht_plan_load reads and checks it (size, tag, L in 1..SHT_MAX_L,
 *   hash; SHT_ERR_INVALID_ARG on any mismatch, before any device work), then builds a plan of
 *   arithmetic `dtype` exactly as sht_plan_with_thetas does.
 */
sht_status sht_plan_save(sht_plan_t plan, const char *path);
sht_status sht_plan_load(const char *path, sht_dtype dtype, sht_plan_t *out);

/* sht_plan_thetas - copy the plan's L ring co-latitudes to theta_host_out (host, L doubles). */
sht_status sht_plan_thetas(sht_plan_t plan, double *theta_host_out);

/* sht_plan_bandlimit - the plan's L. */
int sht_plan_bandlimit(sht_plan_t plan);

/*
 * sht_plan_reserve - allocate the workspaces for batches of up to `batch` signals now, so that
 *   later calls with batch <= `batch` allocate nothing (required before capturing calls in a CUDA
 *   graph).  Blocking.
 */
sht_status sht_plan_reserve(sht_plan_t plan, int64_t batch);

/* sht_plan_destroy - free the plan and everything it owns (synchronises the device). */
sht_status sht_plan_destroy(sht_plan_t plan);

/*
 * sht_forward - coefficients from samples (the forward SHT, Procedure 1 of Sec. III-C).
 *   d_samples: device, batch * L^2 complex128, ring-major.   d_coeffs: device, batch * L^2.
 *   Computed in bin space: every ring's DFT is taken once, then for m = L-1..0 the order-m system
 *   g_m = P_m f_m (Eq. (14)) is solved with the plan's explicit inverse and the solved orders'
 *   aliased contribution (Eq. (16)) is subtracted from the bins of the rings k < m (Eq. (15)).
 *   batch >= 0 (0 is a no-op).
 */
sht_status sht_forward(sht_plan_t plan, const void *d_samples, void *d_coeffs, int64_t batch,
                       void *stream);

/*
 * sht_inverse - samples from coefficients (the inverse SHT, Procedure 2 of Sec. III-D, Eq. (18)).
 *   d_coeffs: device, batch * L^2 complex128.   d_samples: device, batch * L^2, ring-major.
 *   G_m(theta_k) (Eq. (11)) for every order and ring, then per ring the fold of the 2L-1 orders
 *   into the ring's 2k+1 frequency bins and an inverse DFT of length 2k+1.
 */
sht_status sht_inverse(sht_plan_t plan, const void *d_coeffs, void *d_samples, int64_t batch,
                       void *stream);

/*
 * sht_ring_analysis - the forward ring DFTs alone (the first step of Procedure 1, Sec. III-C: the
 *   DFT along each iso-latitude ring, Eq. (11)'s sum over phi).  d_samples: device, batch * L^2
 *   complex, ring-major (ring k = 0..L-1 at offset k^2, sample n at phi = 2 pi n / (2k+1)).
 *   d_bins: device, batch * L^2 complex, ring-major like the samples: bin j (|j| <= k) of ring k at
 *   k^2 + k + j, holding (1/N_k) sum_n s_k[n] e^{-2 pi i j n / N_k}, N_k = 2k+1.  The 1/N_k makes
 *   bin j the sum of the orders m = j mod N_k of the ring's G_m(theta_k) (Eq. (15)); the paper's
 *   2 pi factor of Eq. (11) is left out, as in every entry point of this library.
 *   The same kernels and launches as the ring-DFT step of sht_forward, followed by one layout
 *   kernel (the forward keeps its bins order-major).  complex128 for every arithmetic but SHT_F32
 *   (complex64, float32 DFTs).  Uses the plan's workspace (grown for batch as sht_forward does);
 *   accepts plans made with SHT_PLAN_NO_PTILDE.  Errors: those of sht_forward's argument checks.
 */
sht_status sht_ring_analysis(sht_plan_t plan, const void *d_samples, void *d_bins, int64_t batch,
                             void *stream);

/*
 * sht_ring_synthesis - the inverse ring DFTs alone (the last step of Procedure 2, Sec. III-D,
 *   Eq. (18)): s_k[n] = sum_{|j| <= k} B_k[j] e^{+2 pi i j n / N_k} from ring-major bins
 *   (layout of sht_ring_analysis), so that sht_ring_synthesis(sht_ring_analysis(s)) = s.
 *   Runs the inverse's fold + inverse-DFT kernels on a synthesis table that holds bin j of ring k
 *   as order j (zero for |m| > k), after one layout kernel that writes that table.  Arithmetic,
 *   workspace and errors as sht_ring_analysis.
 */
sht_status sht_ring_synthesis(sht_plan_t plan, const void *d_bins, void *d_samples, int64_t batch,
                              void *stream);

/*
 * sht_forward_uneven, sht_inverse_uneven - one transform direction over nsig signals of different
 *   band-limits (the per-signal transform is the paper's; batching signals of uneven L is ours).
 *   plans[0..nplans): plans created beforehand on the calling device, one per band-limit (any
 *   arithmetic).  Signal i (0 <= i < nsig) uses plans[plan_index[i]] and occupies the L^2 complex128
 *   values (L of that plan; samples ring-major, coefficients at l^2 + l + m as for the batched calls)
 *   at complex-element offset offsets[i] of both the input and the output array (device, 16-byte
 *   aligned).  plans, plan_index and offsets are host arrays, read during the call only.  Signals of
 *   one plan run as one batch: in place when they are consecutive in the order given, otherwise
 *   gathered into the plan's staging buffers (grown on demand, kept until the plan is destroyed)
 *   and scattered back by one device-to-device copy per signal.  Stream-ordered; once the staging
 *   buffers and workspaces have their size (a first call), a call allocates nothing and can be
 *   captured in a CUDA graph (refined plans with a tolerance synchronise, as in sht_forward).
 *   Errors: SHT_ERR_INVALID_ARG for an index outside [0, nplans), a negative offset, overlapping
 *   signals or overlapping input and output; otherwise those of sht_forward / sht_inverse.
 */
sht_status sht_forward_uneven(const sht_plan_t *plans, int nplans, int64_t nsig, const int *plan_index,
                              const int64_t *offsets, const void *d_samples, void *d_coeffs, void *stream);
sht_status sht_inverse_uneven(const sht_plan_t *plans, int nplans, int64_t nsig, const int *plan_index,
                              const int64_t *offsets, const void *d_coeffs, void *d_samples, void *stream);

/*
 * Uneven batches in one persistent launch per direction (a project addition: the per-signal
 * transforms are the paper's Procedures 1 and 2, batching signals of different band-limits is not
 * in the paper).
 *   sht_uneven_create - describe a batch once: nsig signals, signal i transformed by
 *     plans[plan_index[i]] (complex128 scalar plans of any arithmetic, created beforehand on the
 *     current device and kept alive while the batch object exists) and occupying the L^2 complex128
 *     values (L of its plan) at complex-element offset offsets[i] of the input and output arrays
 *     (samples ring-major, coefficients at l^2 + l + m).  Host arrays, read during the call only.
 *     Copies the descriptors to the device and allocates the scratch of every signal (about
 *     32 L^2 bytes each).  SHT_ERR_INVALID_ARG for an index outside [0, nplans), a negative offset or
 *     overlapping signals; SHT_ERR_UNSUPPORTED for SHT_F32 or spin plans.  Blocking.
 *   sht_uneven_forward / sht_uneven_inverse - the whole batch in ONE cooperative launch whose CTAs
 *     stay resident and walk its work items: inverse = synthesis per (signal, order), one grid
 *     barrier, fold + inverse ring DFT per (signal, ring); forward = ring DFT per (signal, ring),
 *     one grid barrier, then each signal's order chain (solves and alias subtractions, m = L-1..0):
 *     the signals whose chain is a large share of the batch on teams of up to 16 CTAs (bounded
 *     team barriers, two per order), the others on one CTA each, largest L first.  Plans made with
 *     SHT_PLAN_NO_PTILDE have P~ regenerated by its recursion inside the launches.  float64 SIMT
 *     arithmetic on the plans' float64 tables (results
 *     float64-accurate, as the batched calls).  Device buffers 16-byte aligned, input and output
 *     disjoint.  Stream-ordered; allocates nothing and never synchronises (capturable in a CUDA
 *     graph); calls on one batch object must not overlap in time (they share its scratch).
 *   sht_uneven_set_wait_limit - limit (1e-9 .. 60 s; default: that of plans[0]) of each wait on
 *     other CTAs (the grid barrier, the team barriers); a CTA that reaches it abandons the call
 *     (results invalid) and sets the batch's status word.
 *   sht_uneven_check - synchronise the device and report SHT_ERR_TIMEOUT if a barrier gave up
 *     since the last check (clears the flag).
 *   sht_uneven_destroy - free the batch object (synchronises the device; the plans are not freed).
 */
typedef struct sht_uneven_s *sht_uneven_t;
sht_status sht_uneven_create(const sht_plan_t *plans, int nplans, int64_t nsig, const int *plan_index,
                             const int64_t *offsets, sht_uneven_t *out);
sht_status sht_uneven_forward(sht_uneven_t batch, const void *d_samples, void *d_coeffs, void *stream);
sht_status sht_uneven_inverse(sht_uneven_t batch, const void *d_coeffs, void *d_samples, void *stream);
sht_status sht_uneven_set_wait_limit(sht_uneven_t batch, double seconds);
sht_status sht_uneven_check(sht_uneven_t batch);
sht_status sht_uneven_destroy(sht_uneven_t batch);

/*
 * sht_inverse_adjoint - the adjoint A^H of the inverse map A (A[(k,n),(l,m)] = Y_l^m(theta_k,
 *   phi_kn)): coefficients-shaped output from samples-shaped input,
 *   out_l^m = sum_{k,n} P~_l^m(theta_k) e^{-i m phi_kn} y_kn.  Same layouts as sht_forward.
 *   With PyTorch's convention this is the backward of sht_inverse.
 */
sht_status sht_inverse_adjoint(sht_plan_t plan, const void *d_samples, void *d_coeffs,
                               int64_t batch, void *stream);

/*
 * sht_forward_adjoint - the adjoint (A^{-1})^H of the forward map: samples-shaped output from
 *   coefficients-shaped input.  Runs the forward's order chain in reverse (m = 0..L-1) with the
 *   transposed per-order inverses and alias gathers, then the adjoint ring DFTs.  Same layouts as
 *   sht_inverse.  With PyTorch's convention this is the backward of sht_forward.
 */
sht_status sht_forward_adjoint(sht_plan_t plan, const void *d_coeffs, void *d_samples,
                               int64_t batch, void *stream);

/*
 * sht_forward_noalloc - sht_forward for callers that cannot let a call allocate device memory
 *   (a library embedded in a host application that hands it a fixed memory budget, or code that
 *   runs where cudaMalloc is not allowed, e.g. while other work is being captured into a CUDA
 *   graph).  The paper has no counterpart: this is a deployment variant of sht_forward.
 *   Same arguments, layouts and argument checks as sht_forward (a plan created beforehand; device
 *   buffers owned by the caller).  Whatever the plan's arithmetic, it runs the float64 SIMT order
 *   chain on the plan's float64 tables: float64-accurate (within 1e-11 of sht_forward on the
 *   workloads tested), but not bit-identical to the tensor-core chain of SHT_F64_TENSOR or to a
 *   refined forward; SHT_F32 plans are refused (SHT_ERR_UNSUPPORTED).  Its scratch - the bins,
 *   the solved orders and the split-K partial sums - lives in one fixed 64 MiB (67108864-byte)
 *   __device__ array of the library instead of the plan's workspaces, so the call allocates
 *   nothing.  It needs 2 * r256(32 * L(L+1)/2 * batch) + r256(512 * L * batch) bytes, r256
 *   rounding up to a multiple of 256: for example L = 1024 with batch 1 fits and batch 2 does not.
 *   Larger sizes return SHT_ERR_UNSUPPORTED with the required size in sht_last_error_message.
 *   The array exists on every GPU that loads the library until the process exits.  All calls on
 *   a device share it and leave their contents in it (nothing needs to start at zero: every
 *   element read is written earlier in the same call); calls whose GPU work overlaps in time race.
 *   The first call in each CUDA context looks up the array's device address
 *   (cudaGetSymbolAddress) and keeps it with the context's unique id, so make that first call
 *   before any stream capture; after cudaDeviceReset the next call looks it up again.
 */
sht_status sht_forward_noalloc(sht_plan_t plan, const void *d_samples, void *d_coeffs,
                               int64_t batch, void *stream);

/*
 * sht_plan_set_refinement - iteration control of the refined forward (SHT_*_REFINED plans).
 *   tol > 0: iterate until the largest |Re|, |Im| over the last update of the coefficients is
 *   <= tol, at most max_iters iterations; each iteration reads that maximum to the host
 *   (synchronises the call's stream); not reaching tol returns SHT_ERR_NOT_CONVERGED with the last
 *   iterate in the output.  tol == 0: exactly max_iters iterations and no synchronisation (the
 *   call can be captured in a CUDA graph).  Defaults: max_iters = 10, tol = 1e-11.
 *   sht_get_info reports the iterations and the last update of the most recent refined call.
 */
sht_status sht_plan_set_refinement(sht_plan_t plan, int max_iters, double tol);

/*
 * Execution choices of a plan for one batch size (a project addition; the paper has no
 * counterpart: it fixes the method's arithmetic, not how a GPU schedules it).
 *   forward_path, inverse_path: SHT_PATH_DEFAULT (the plan's arithmetic: tensor-core kernels for
 *     SHT_F64_TENSOR and the refined plans, SIMT kernels for SHT_F64 and SHT_F32),
 *     SHT_PATH_TENSOR, or SHT_PATH_SIMT (the float64 SIMT kernels on the plan's float64 tables;
 *     offered to SHT_F64_TENSOR plans for both directions and to refined plans for the inverse;
 *     float64-accurate like the tensor path).
 *   split_cap: most K-splits of one per-order product of the SIMT order chain (0 = default 16,
 *     else 1..16).
 *   forward_ms, inverse_ms: the times sht_plan_autotune measured for the chosen paths (0 when set
 *     by sht_plan_set_paths).
 */
#define SHT_PATH_DEFAULT 0
#define SHT_PATH_TENSOR  1
#define SHT_PATH_SIMT    2
typedef struct {
    int forward_path;
    int inverse_path;
    int split_cap;
    double forward_ms;
    double inverse_ms;
} sht_tuning;

/*
 * sht_plan_set_paths - use these choices for later calls whose batch equals `batch` (other
 *   batches keep the defaults).  SHT_ERR_INVALID_ARG for a path the plan does not offer or a
 *   split_cap outside 0..16.
 */
sht_status sht_plan_set_paths(sht_plan_t plan, int64_t batch, int forward_path, int inverse_path,
                              int split_cap);

/*
 * sht_plan_autotune - time every choice the plan offers for batches of `batch` signals (forward:
 *   the tensor chain where offered, the SIMT chain with split caps 16, 4 and 1; inverse: the
 *   tensor synthesis where offered and the SIMT synthesis), each as the best of three calls after
 *   one warm-up on zero-filled device buffers of its own, keep the fastest for later calls with
 *   that batch, and report it in *out (may be NULL).  Refined plans tune their inverse only.
 *   Blocking; allocates and frees its buffers and the plan's workspaces grow to `batch`; do not
 *   call it while a stream is being captured.
 */
sht_status sht_plan_autotune(sht_plan_t plan, int64_t batch, sht_tuning *out);

/*
 * sht_plan_set_wait_limit - limit, in seconds (1e-9 .. 60), of every wait inside the tensor-core
 *   kernels of the plan on other CTAs or on its own copy and MMA pipeline (grid barriers of the
 *   forward chain, mbarriers).  A wait that reaches the limit abandons the call: its CTA sets the
 *   plan's status word (sht_plan_check then returns SHT_ERR_TIMEOUT), the other CTAs leave at their
 *   next wait, each waits up to one second for its own copies and MMAs in flight and releases its
 *   tensor memory; the results of that call are invalid, later calls are unaffected.  Default 1.
 */
sht_status sht_plan_set_wait_limit(sht_plan_t plan, double seconds);

/*
 * sht_plan_check - wait for the plan's queued work (synchronises the device) and report whether a
 *   bounded wait inside a tensor-core kernel gave up since the last check (SHT_ERR_TIMEOUT; the
 *   results of the affected call are then invalid).  Clears the flag.
 */
sht_status sht_plan_check(sht_plan_t plan);

/* Plan information. */
typedef struct {
    int L;
    int dtype;
    uint64_t table_bytes;      /* device bytes held by the plan's tables */
    uint64_t workspace_bytes;  /* device bytes held by the plan's workspaces */
    int64_t workspace_batch;   /* batch the workspaces are sized for */
    double plan_seconds;       /* wall time of plan creation */
    double order_seconds;      /* part of it spent ordering the rings */
    int64_t kernel_launches;   /* kernels this plan's transform calls have launched so far */
    int refine_iterations;     /* refined forward: iterations of the most recent call */
    double refine_last_update; /* refined forward: largest |Re|, |Im| of its last update (tol > 0) */
    int spin;                  /* spin weight s of the plan (0: scalar functions) */
} sht_info;

/* Stages of the transforms, for sht_plan_stage_times. */
#define SHT_STAGE_RING_DFT   0  /* forward ring DFTs into bins (forward; adjoint of inverse)   */
#define SHT_STAGE_SOLVE      1  /* per-order solves P_m^{-1} g_m (forward chain, all m); for
                                   tensor plans the whole chain, solves and alias products,
                                   which runs as one persistent launch                         */
#define SHT_STAGE_ALIAS      2  /* alias subtractions from lower rings (forward chain, all m;
                                   float64 plans)                                              */
#define SHT_STAGE_LAYOUT     3  /* coefficient <-> order-major conversions                      */
#define SHT_STAGE_SYNTHESIS  4  /* G_m(theta_k) for all m, k (inverse; adjoint: analysis)       */
#define SHT_STAGE_RING_IDFT  5  /* fold + inverse ring DFTs (inverse; adjoint of forward)       */
#define SHT_NUM_STAGES       6

/*
 * sht_plan_set_timing - when enable != 0, later transform calls on this plan record a CUDA event
 *   pair on the call's stream around each stage (no synchronisation, no allocation after the
 *   first few calls).  Off by default.
 */
sht_status sht_plan_set_timing(sht_plan_t plan, int enable);

/*
 * sht_plan_stage_times - wait for the recorded events, write the summed milliseconds of each
 *   stage to ms[SHT_NUM_STAGES] and the number of timed spans to spans[SHT_NUM_STAGES] (either
 *   may be NULL), then clear the record.  Blocking on the recorded events only.
 */
sht_status sht_plan_stage_times(sht_plan_t plan, double *ms, int64_t *spans);

sht_status sht_get_info(sht_plan_t plan, sht_info *out);

/* Human-readable name of a status code (static string). */
const char *sht_status_string(sht_status status);

/* Detail of the last error raised on this thread (static per-thread buffer; "" if none). */
const char *sht_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* SHT_H */
